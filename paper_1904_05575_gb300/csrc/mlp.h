// The learned preconditioner of the Davidson solver (see mlp.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/bse.h"

namespace bse {

struct MlpNet;

MlpNet* mlp_create(uint64_t seed);
void mlp_destroy(MlpNet* net);
int64_t mlp_num_params(const MlpNet* net);
void mlp_get_params(const MlpNet* net, float* host);   // the FP16 weights, as floats
void mlp_set_params(MlpNet* net, const float* host);

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

// T[:, c] = (1 + y(f)) R[:, c] / (D_q - E_c): columns c < k/2 are residuals of
// the (A+B) equation, the others of the (A-B) equation.
void mlp_precondition(const MlpNet* net, int n, int k, const double* dp, const double* dm,
                      const double* srow, const double* E, const double2* R, int64_t ldr,
                      double2* T, int64_t ldt, cudaStream_t s);

// Davidson trajectory recording: with the exact pairs of the problem known,
// each iteration's residuals and current errors (Ritz vector minus the
// phase-aligned exact vector) become training samples of the same kind as
// mlp_samples.  Owned by the caller; count advances until capacity.
struct TrajectorySink {
  const bse_c128* xpy_exact = nullptr;   // n x nev, column-major (device)
  const double* e_exact = nullptr;       // nev (host)
  int64_t capacity = 0;                  // samples
  int64_t count = 0;
  float* feat = nullptr;                 // [capacity][4] (device)
  float* target = nullptr;               // [capacity]
  float* weight = nullptr;               // [capacity]
};

// Samples of one residual vector r against the error step (both length n):
// c* = Re(conj(r) step)/|r|^2 (D_q - E), weight |r|^2/(D_q - E)^2 normalised.
void mlp_record(int n, const double* dp, const double* dm, const double* srow, double E,
                bool plus, const double2* r, const double2* step, float* feat, float* target,
                float* weight, cudaStream_t s);

}  // namespace bse
