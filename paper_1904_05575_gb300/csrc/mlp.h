// The learned preconditioner of the Davidson solver (see mlp.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/bse.h"

namespace bse {

struct MlpNet;

bool mlp_features_supported(int n_features);   // 4 or 10
MlpNet* mlp_create(int n_features, uint64_t seed);
void mlp_destroy(MlpNet* net);
int64_t mlp_num_params(const MlpNet* net);
int mlp_num_features(const MlpNet* net);
void mlp_get_params(const MlpNet* net, float* host);   // the FP16 weights, as floats
void mlp_set_params(MlpNet* net, const float* host);

// The neighbouring momentum transfers' exact X+Y used by the 10-feature set:
// count (1 or 2) blocks of [n x nev] column-major, device, caller-owned (kept
// by pointer); NULL / count 0 clears.
void mlp_set_neighbours(MlpNet* net, int n, int nev, const bse_c128* nbr, int count,
                        cudaStream_t s);
// throws BSE_ERR_ARG unless a 10-feature net has neighbours for n and >= nev excitons
void mlp_check_neighbours(const MlpNet* net, int n, int nev);

// Training samples from exact pairs (features [2 nev n][4], target, weight).
void mlp_samples(int n, const bse_c128* A, const bse_c128* B, int64_t ld, int nev,
                 const double* E, const bse_c128* xpy, const bse_c128* noise, double eps,
                 float* feat, float* target, float* weight, cudaStream_t s);
double mlp_loss_grad(MlpNet* net, const float* feat, const float* target, const float* weight,
                     int64_t nsamp, float* grad_host, cudaStream_t s);
double mlp_train(MlpNet* net, const float* feat, const float* target, const float* weight,
                 int64_t nsamp, int steps, double lr, cudaStream_t s);
void mlp_predict(const MlpNet* net, const float* feat, int64_t nsamp, float* out, cudaStream_t s);

// Per-transition inputs of the preconditioners: diagonals of A+B and A-B and
// the off-diagonal row norms of A (device arrays of n).
void mlp_diag_features(int n, const bse_c128* A, const bse_c128* B, int64_t ld, double* dp,
                       double* dm, double* srow, cudaStream_t s);

// Features of ncol residual columns (all arrays device): eq[c] 0 = residual
// of the (A+B) equation, 1 = the (A-B) equation; lam[c] the exciton (column
// of the neighbour blocks); theta[c] its Ritz value; R the residuals and X the
// current vectors they correct (X+Y for eq 0, X-Y for eq 1), n x ncol with
// leading dimensions ldr, ldx.  feat: [ncol n][nf].
void mlp_features(const MlpNet* net, int n, int ncol, const int* eq, const int* lam,
                  const double* theta, const double* dp, const double* dm, const double* srow,
                  const double2* R, int64_t ldr, const double2* X, int64_t ldx, float* feat,
                  cudaStream_t s);

// T[:, c] = (1 + y(f)) R[:, c] / (D_q - theta_c) with the features above
// (feat: scratch of n ncol nf floats).
void mlp_precondition(const MlpNet* net, int n, int ncol, const int* eq, const int* lam,
                      const double* dp, const double* dm, const double* srow, const double* theta,
                      const double2* R, int64_t ldr, const double2* X, int64_t ldx, float* feat,
                      double2* T, int64_t ldt, cudaStream_t s);

// Davidson trajectory recording: with the exact pairs of the problem known,
// each iteration's residuals and current errors (Ritz vector minus the
// phase-aligned exact vector) become training samples (features of the
// sink's network).  Owned by the caller; count advances until capacity.
struct TrajectorySink {
  const MlpNet* net = nullptr;           // feature set (4 or 10; neighbours set for 10)
  const bse_c128* xpy_exact = nullptr;   // n x nev, column-major (device)
  const double* e_exact = nullptr;       // nev (host)
  int64_t capacity = 0;                  // samples
  int64_t count = 0;
  float* feat = nullptr;                 // [capacity][nf] (device)
  float* target = nullptr;               // [capacity]
  float* weight = nullptr;               // [capacity]
};

// Samples of one residual vector r of exciton lam (x the vector it corrects,
// step its error; all length n): c* = Re(conj(r) step)/|r|^2 (D_q - E),
// weight |r|^2/(D_q - E)^2 normalised over the vector.
void mlp_record(const MlpNet* net, int n, const double* dp, const double* dm, const double* srow,
                double E, int lam, bool plus, const double2* r, const double2* x,
                const double2* step, float* feat, float* target, float* weight, cudaStream_t s);

}  // namespace bse
