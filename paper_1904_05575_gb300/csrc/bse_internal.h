// Internal declarations shared by the translation units of libbse.so.
#pragma once

#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <cstdint>
#include <mutex>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/bse.h"

namespace bse {

constexpr double kHartreeEv = 27.211386245988;   // CODATA 2018

// Error carried from deep inside a launcher to the ABI boundary.
struct Error : std::runtime_error {
  int status;
  Error(int s, const std::string& m) : std::runtime_error(m), status(s) {}
};

void set_last_error(const std::string& msg);

// Count of kernels launched by this library (see bse_kernel_launches).
void note_launches(int64_t n);

// RAII phase timer: when bse_phase_timing(1) is on, records a start event on
// construction and a stop event on destruction, both on the given stream.
class Phase {
 public:
  Phase(const char* name, cudaStream_t s);
  ~Phase();
  Phase(const Phase&) = delete;
  Phase& operator=(const Phase&) = delete;

 private:
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t start_ = nullptr;
};

#define BSE_CUDA(call)                                                           \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      throw ::bse::Error(BSE_ERR_CUDA, std::string(#call) + ": " +               \
                                           cudaGetErrorString(e_) + " at " +     \
                                           __FILE__ + ":" + std::to_string(__LINE__)); \
    }                                                                            \
  } while (0)

#define BSE_CHECK_ARG(cond, msg)                                                 \
  do {                                                                           \
    if (!(cond)) throw ::bse::Error(BSE_ERR_ARG, msg);                           \
  } while (0)

// Stream-ordered scratch buffer (cudaMallocAsync / cudaFreeAsync).
struct DeviceBuffer {
  void* ptr = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  DeviceBuffer() = default;
  DeviceBuffer(size_t n, cudaStream_t s) : bytes(n), stream(s) {
    if (n == 0) return;
    cudaError_t e = cudaMallocAsync(&ptr, n, s);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      throw Error(BSE_ERR_NOMEM, "cudaMallocAsync of " + std::to_string(n) +
                                     " bytes failed: " + cudaGetErrorString(e));
    }
  }
  DeviceBuffer(const DeviceBuffer&) = delete;
  DeviceBuffer& operator=(const DeviceBuffer&) = delete;
  ~DeviceBuffer() {
    if (ptr) cudaFreeAsync(ptr, stream);
  }
  template <class T>
  T* as() const { return static_cast<T*>(ptr); }
};

// One problem after host-side validation, with derived sizes.
struct Problem {
  bse_problem p;
  int64_t n;          // nk * nv * nc
  double kappa;       // Ha / (nk * omega_cell)
  std::vector<int32_t> qm_host, qp_host;   // host copies of q_minus / q_plus (checked, whole)
  int kb = 0, kn = 0; // k-row slab [kb, kb + kn) (kn = nk for the whole problem)
  int64_t rows() const { return (int64_t)kn * p.nv * p.nc; }        // rows of A, B written
  int64_t row0() const { return (int64_t)kb * p.nv * p.nc; }        // first of them
  int64_t slab_pairs() const { return (int64_t)kn * p.nk; }         // (k, k') with k in the slab
};

// FP64 build (CUDA cores).  Writes A (and B when coupling) completely.
void build_fp64(const Problem& pr, cudaStream_t stream);

// True when build_mixed serves the precision.
bool mixed_supported(int precision);

// FP64 build whose stage-1 intermediate lives in a fixed module array of
// kFp64StaticScratchBytes (no device allocation); rejects larger problems.
constexpr size_t kFp64StaticScratchBytes = (size_t)16 << 20;
size_t fp64_static_scratch_need(const Problem& pr);
void build_fp64_static(const Problem& pr, cudaStream_t stream);

// Pair matrix elements from plane-wave coefficients (pair_elements.cu);
// basis_h / gout_h are host integer coordinates; NULL outputs are skipped.  Syncs.
void pair_elements_fp64(int n, int nv, int nc, int npw, int ng, const bse_c128* cv,
                        const bse_c128* cc, const int32_t* basis_h, const int32_t* gout_h,
                        int kb, int kn, bse_c128* m_x, bse_c128* m_vv, bse_c128* m_cc,
                        bse_c128* n_vc, cudaStream_t s);

// Exact FP64 diagonal of A (and B) over the problem's rows (diag_fp64.cu):
// overwrites A_aa, B_aa with the FP64 sums; workspace of diag_fp64_workspace
// bytes (device).
size_t diag_fp64_workspace(const Problem& pr);
void diag_fp64(const Problem& pr, bse_c128* workspace, cudaStream_t stream);

// Split-precision tensor-core build (tcgen05) of several problems through a
// cached batched plan.  Writes every A (and B) completely.  Syncs.
void build_mixed_batch(const std::vector<Problem>& probs, int precision, cudaStream_t stream);

// The per-device cuSOLVER / cuBLAS handles; the lock serialises their use.
struct LibHandles {
  cusolverDnHandle_t solver;
  cublasHandle_t blas;
};
LibHandles acquire_handles(std::unique_lock<std::mutex>& lock);

// Lowest excitons by block Davidson (product form); precond 0 = diagonal, 1 = MLP.
struct MlpNet;
struct TrajectorySink;
void davidson_fp64(int n, const bse_c128* A, const bse_c128* B, int64_t ld, int nev, double tol,
                   int max_iter, int precond, const MlpNet* mlp, double* E_out, bse_c128* XpY_out,
                   int32_t* iters_out, cudaStream_t stream, TrajectorySink* sink = nullptr,
                   int matvec_precision = BSE_PREC_FP64, const bse_c128* V0 = nullptr,
                   int k0 = 0);

// Hermitian matrix-vector blocks on the tensor cores (build_mixed.cu): A and
// B split once; apply writes AV = A V and BV = B V (n x k, column-major, ld n).
struct TcMatvec;
TcMatvec* tc_matvec_create(int n, const bse_c128* A, const bse_c128* B, int64_t ld, int precision,
                           int kmax, cudaStream_t stream);
void tc_matvec_apply(TcMatvec* m, const bse_c128* V, int k, bse_c128* AV, bse_c128* BV,
                     cudaStream_t stream);
void tc_matvec_destroy(TcMatvec* m);

// Batched plans (build_mixed.cu).
struct BatchPlan;
BatchPlan* plan_create(std::vector<Problem> probs, int precision, int flags, cudaStream_t s);
void plan_execute(BatchPlan* plan, cudaStream_t s);
int plan_status(BatchPlan* plan, cudaStream_t s);
int plan_tile_cols(const BatchPlan* plan);
void plan_stage2_shape(const BatchPlan* plan, int* tile_cols, int* stages);
int plan_fused(const BatchPlan* plan);
void plan_set_wait(BatchPlan* plan, double seconds);
void plan_destroy(BatchPlan* plan);

// Reduction and spectrum.
void reduce_fp64(int n, const bse_c128* A, const bse_c128* B, int64_t ld, bse_c128* S,
                 bse_c128* L, int32_t* failed_minor, cudaStream_t stream);
void xpy_fp64(int n, int k, const bse_c128* Z, const bse_c128* L, int64_t ld, const double* E,
              bse_c128* XpY, int64_t ldx, cudaStream_t stream);
void spectrum_tensor_fp64(int n, const bse_c128* Z, const bse_c128* L, int64_t ld,
                          const bse_c128* D, int64_t ldd, double c_q, double vc, int n_omega,
                          const double* omega, double delta, const double* E, bse_c128* eps_out,
                          cudaStream_t s);
void loss_fp64(int n_omega, const bse_c128* eps, double v_inv, double* loss_out, double* sqw_out,
               cudaStream_t s);
void rpa_screening(int nk, int nv, int nc, int ng, double omega_cell, const double* e_v,
                   const double* e_c_kq, const bse_c128* m, const double* v, int precision,
                   bse_c128* w_out, cudaStream_t s);
// X[G][G'] = sum_a conj(m_a(G)) m_a(G') / (e_c - e_v) (row-major, FP64 result) on the
// tensor cores in the split precision `precision` (build_mixed.cu)
void rpa_x_mixed(int nk, int nv, int nc, int ng, const double* e_v, const double* e_c_kq,
                 const bse_c128* m, int precision, double2* x_out, cudaStream_t s);
void spectrum_fp64(int n, bse_c128* S, const bse_c128* L, int64_t ld, const bse_c128* rho,
                   double c_q, double vc, int n_omega, const double* omega, double delta,
                   double* E_out, double* osc_out, bse_c128* eps_out, cudaStream_t stream);

}  // namespace bse
