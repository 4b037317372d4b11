// Lowest excitons of the full BSE by block Davidson on the product form.
//
// The full problem H (X;Y) = E Delta (X;Y) (Eq. gevpbse) with H = [[A,B],[B,A]]
// (Eq. Hetr) is equivalent to (A+B)(X+Y) = E (X-Y), (A-B)(X-Y) = E (X+Y), so
// (A-B)(A+B)(X+Y) = E^2 (X+Y): the half-size form behind Eq. auxevp.  The
// solver keeps one orthonormal basis V for both X+Y and X-Y (the scheme of
// Stratmann, Scuseria and Frisch, J. Chem. Phys. 109, 8218 (1998)):
//   P = (A+B) V, M = (A-B) V                   matvecs: FP64 GEMM kernel, or the
//                                               split-precision tensor-core GEMM
//   a+ = V^H P, a- = V^H M                      projected (m x m) matrices
//   a- = l l^H, s = l^H a+ l, s z = E^2 z       the projected problem, in the
//   u = l z E^-1/2, w = a+ u / E                Cholesky form used by bse_reduce
//   X+Y = V u, X-Y = V w                        Ritz vectors, (X+Y)^H (X-Y) = 1
//   r+ = P u - E V w, r- = M w - E V u          residuals of the two equations
// Unconverged residuals are preconditioned (diagonal: r / (A_aa - E), or the
// trained MLP of mlp.cu), orthogonalised against V as one block (two
// Gram-Schmidt passes by GEMM, then Cholesky QR twice) and appended; the
// basis restarts from the current Ritz vectors when full.
// Small dense steps (projections, m x m factorisations) are cuBLAS / cuSOLVER
// calls; the host drives the iteration and reads residual norms each step.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <memory>
#include <numeric>
#include <vector>

#include "bse_internal.h"
#include "mlp.h"
#include "zgemm.cuh"

namespace bse {
namespace {

#define BSE_CUSOLVER(call)                                                        \
  do {                                                                            \
    cusolverStatus_t st_ = (call);                                                \
    if (st_ != CUSOLVER_STATUS_SUCCESS)                                           \
      throw ::bse::Error(BSE_ERR_CUDA, std::string(#call) + " failed with status " + \
                                           std::to_string((int)st_));             \
  } while (0)
#define BSE_CUBLAS(call)                                                          \
  do {                                                                            \
    cublasStatus_t st_ = (call);                                                  \
    if (st_ != CUBLAS_STATUS_SUCCESS)                                             \
      throw ::bse::Error(BSE_ERR_CUDA, std::string(#call) + " failed with status " + \
                                           std::to_string((int)st_));             \
  } while (0)

// P = AV + BV, M = AV - BV (B absent: both AV)
__global__ void k_plus_minus_cols(int64_t total, const double2* av, const double2* bv,
                                  double2* P, double2* M) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = av[i];
    const double2 b = bv ? bv[i] : make_double2(0.0, 0.0);
    P[i] = make_double2(a.x + b.x, a.y + b.y);
    M[i] = make_double2(a.x - b.x, a.y - b.y);
  }
}

__global__ void k_diag_real(int n, const double2* A, int64_t ld, double* d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = A[i + (int64_t)i * ld].x;
}

// After columns m0..m-1 of s were computed (rows 0..m-1): rows m0..m-1 of
// the old columns become the conjugates of what was computed, and the new
// square block becomes (s + s^H) / 2 with a real diagonal.
__global__ void k_hermitize_new(int m0, int m, double2* s, int lds) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = m0 + blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= m || j >= m) return;
  if (i < m0) {
    const double2 a = s[i + (int64_t)j * lds];
    s[j + (int64_t)i * lds] = make_double2(a.x, -a.y);
  } else if (i < j) {
    double2 a = s[i + (int64_t)j * lds], b = s[j + (int64_t)i * lds];
    double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    s[i + (int64_t)j * lds] = h;
    s[j + (int64_t)i * lds] = make_double2(h.x, -h.y);
  } else if (i == j) {
    s[i + (int64_t)i * lds].y = 0.0;
  }
}

__global__ void k_zero_strict_upper(int m, double2* l, int ldl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i < m && j < m && i < j) l[i + (int64_t)j * ldl] = make_double2(0.0, 0.0);
}

// scale column j of x (rows x k, ld) by f[j]
__global__ void k_scale_cols(int rows, int k, double2* x, int64_t ld, const double* f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i < rows && j < k) {
    double2 v = x[i + (int64_t)j * ld];
    x[i + (int64_t)j * ld] = make_double2(v.x * f[j], v.y * f[j]);
  }
}

// t[:, j] = r[:, j] / (D_q - E_j) with D_q the diagonal of A+B for the first
// k/2 columns (residuals of the (A+B) equation) and of A-B for the rest;
// denominators kept at least 1e-2 eV away from 0
__global__ void k_precond_diag(int n, int k, const double* dp, const double* dm, const double* e,
                               const double2* r, int64_t ldr, double2* t, int64_t ldt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i < n && j < k) {
    double den = (j < k / 2 ? dp[i] : dm[i]) - e[j];
    if (fabs(den) < 1e-2) den = den < 0 ? -1e-2 : 1e-2;
    double2 v = r[i + (int64_t)j * ldr];
    t[i + (int64_t)j * ldt] = make_double2(v.x / den, v.y / den);
  }
}

// out[j] = max(|r1[:, j]|, |r2[:, j]|) (r2 NULL: |r1[:, j]|), one block per
// column, FP64 sums of squares reduced in shared memory
__global__ void __launch_bounds__(256) k_col_norms(int n, const double2* r1, const double2* r2,
                                                   int64_t ld, double* out) {
  __shared__ double sa[256], sb[256];
  const int j = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
    const double2 x = r1[i + (int64_t)j * ld];
    a += x.x * x.x + x.y * x.y;
    if (r2) {
      const double2 y = r2[i + (int64_t)j * ld];
      b += y.x * y.x + y.y * y.y;
    }
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sa[threadIdx.x] += sa[threadIdx.x + w];
      sb[threadIdx.x] += sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = sqrt(fmax(sa[0], sb[0]));
}

// copy the listed columns of x (ld n) into consecutive columns of y (ld n)
__global__ void k_gather_cols(int n, int k, const int* idx, const double2* x, double2* y) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i + (int64_t)j * n] = x[i + (int64_t)idx[j] * n];
}

struct Solver {
  int n, nev, mmax;
  const bse_c128 *A, *B;
  int64_t ld;
  cudaStream_t s;
  LibHandles h;
  DeviceBuffer V, P, M, AV, BV, ap, am, L, S, U, W, R1, R2, T, C, info, dE, dF, dD, dDp, dDm,
      dS;
  std::unique_ptr<DeviceBuffer> work_;
  int lwork = 0;
  int m = 0;          // current basis size
  int m_proj = 0;     // columns of the projected a+ and a- already computed
  std::vector<double> D;
  // block orthogonalisation: Gram matrix and triangular factor (b x b, b <=
  // 4 nev or mmax), column norms and the indices of kept columns
  int bmax;
  DeviceBuffer G, Rt, nrm, idx;

  Solver(int n_, int nev_, int mmax_, const bse_c128* A_, const bse_c128* B_, int64_t ld_,
         cudaStream_t s_, LibHandles h_)
      : n(n_), nev(nev_), mmax(mmax_), A(A_), B(B_), ld(ld_), s(s_), h(h_),
        V((size_t)n_ * mmax_ * 16, s_), P((size_t)n_ * mmax_ * 16, s_),
        M((size_t)n_ * mmax_ * 16, s_), AV((size_t)n_ * std::max(mmax_, 2 * nev_) * 16, s_),
        BV((size_t)n_ * std::max(mmax_, 2 * nev_) * 16, s_), ap((size_t)mmax_ * mmax_ * 16, s_),
        am((size_t)mmax_ * mmax_ * 16, s_), L((size_t)mmax_ * mmax_ * 16, s_),
        S((size_t)mmax_ * mmax_ * 16, s_), U((size_t)mmax_ * mmax_ * 16, s_),
        W((size_t)mmax_ * mmax_ * 16, s_), R1((size_t)n_ * std::max(mmax_, 4 * nev_) * 16, s_),
        R2((size_t)n_ * mmax_ * 16, s_), T((size_t)n_ * 2 * std::max(mmax_, nev_) * 16, s_),
        C((size_t)mmax_ * 16, s_), info(sizeof(int), s_), dE((size_t)mmax_ * 8, s_),
        dF((size_t)std::max(mmax_, 2 * nev_) * 8, s_), dD((size_t)n_ * 8, s_),
        dDp((size_t)n_ * 8, s_), dDm((size_t)n_ * 8, s_), dS((size_t)n_ * 8, s_),
        bmax(std::max(mmax_, 4 * nev_)), G((size_t)bmax * bmax * 16, s_),
        Rt((size_t)bmax * bmax * 16, s_), nrm((size_t)bmax * 8, s_),
        idx((size_t)bmax * 4, s_) {
    int lw1 = 0, lw2 = 0;
    BSE_CUSOLVER(cusolverDnZpotrf_bufferSize(h.solver, CUBLAS_FILL_MODE_LOWER, mmax,
                                             L.as<cuDoubleComplex>(), mmax, &lw1));
    // (the Jacobi solver cusolverDnZheevj measured 12x slower than zheevd on
    // these 64-384 sized projected problems)
    BSE_CUSOLVER(cusolverDnZheevd_bufferSize(h.solver, CUSOLVER_EIG_MODE_VECTOR,
                                             CUBLAS_FILL_MODE_LOWER, mmax,
                                             S.as<cuDoubleComplex>(), mmax, dE.as<double>(),
                                             &lw2));
    lwork = std::max(std::max(lw1, lw2), 1);
    work_.reset(new DeviceBuffer((size_t)lwork * 16, s));
  }

  cuDoubleComplex* col(const DeviceBuffer& b, int j, int64_t ldb) const {
    return b.as<cuDoubleComplex>() + (int64_t)j * ldb;
  }

  // tensor-core matvecs (split-precision A, B), or NULL for the FP64 kernel
  TcMatvec* tcm = nullptr;

  // P, M for basis columns [j0, j1)
  void matvec(int j0, int j1) {
    const int k = j1 - j0;
    if (k <= 0) return;
    if (tcm) {
      tc_matvec_apply(tcm, V.as<bse_c128>() + (int64_t)j0 * n, k, AV.as<bse_c128>(),
                      B ? BV.as<bse_c128>() : nullptr, s);
    } else {
      MatvecProb pa{n, k, n, A, ld, V.as<bse_c128>() + (int64_t)j0 * n, n,
                    AV.as<bse_c128>(), n};
      launch_zgemm(pa, 1, s);
      if (B) {
        MatvecProb pb{n, k, n, B, ld, V.as<bse_c128>() + (int64_t)j0 * n, n,
                      BV.as<bse_c128>(), n};
        launch_zgemm(pb, 1, s);
      }
    }
    const int64_t total = (int64_t)n * k;
    k_plus_minus_cols<<<(int)std::min<int64_t>((total + 255) / 256, 152 * 16), 256, 0, s>>>(
        total, AV.as<double2>(), B ? BV.as<double2>() : nullptr,
        P.as<double2>() + (int64_t)j0 * n, M.as<double2>() + (int64_t)j0 * n);
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
  }

  // Orthonormalise the b columns of X (device, n x b, leading dimension n;
  // overwritten) against V[:, :m] and among themselves, in column order, and
  // append the survivors to V (at most mmax - m): two classical Gram-Schmidt passes against V (GEMMs), then a Cholesky QR
  // of the block whose in-order factorisation drops a column when what
  // remains of it is below 1e-6 of its norm before the projections, then a
  // second projection and Cholesky QR pass (CholQR2) for orthogonality to
  // working precision.  Returns the number appended.
  int append_block(cuDoubleComplex* X, int b) {
    if (b <= 0 || m >= mmax) return 0;
    const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0),
                          mone = make_cuDoubleComplex(-1, 0);
    std::vector<double> n0(b);
    k_col_norms<<<b, 256, 0, s>>>(n, reinterpret_cast<const double2*>(X), nullptr, n,
                                  nrm.as<double>());
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
    BSE_CUDA(cudaMemcpyAsync(n0.data(), nrm.ptr, (size_t)b * 8, cudaMemcpyDeviceToHost, s));
    auto project = [&](cuDoubleComplex* Y, int k) {
      if (m == 0) return;
      BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_C, CUBLAS_OP_N, m, k, n, &one,
                             V.as<cuDoubleComplex>(), n, Y, n, &zero, G.as<cuDoubleComplex>(), m));
      BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, k, m, &mone,
                             V.as<cuDoubleComplex>(), n, G.as<cuDoubleComplex>(), m, &one, Y, n));
    };
    // Gram matrix of k columns to the host (column-major k x k)
    auto gram = [&](const cuDoubleComplex* Y, int k, std::vector<cuDoubleComplex>& g) {
      BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_C, CUBLAS_OP_N, k, k, n, &one, Y, n, Y, n, &zero,
                             G.as<cuDoubleComplex>(), k));
      g.resize((size_t)k * k);
      BSE_CUDA(cudaMemcpyAsync(g.data(), G.ptr, (size_t)k * k * 16, cudaMemcpyDeviceToHost, s));
      BSE_CUDA(cudaStreamSynchronize(s));
    };
    // in-order Cholesky g = r^H r over the columns in `cols`, dropping those
    // whose remaining squared norm is below thr[j]; r is upper triangular over
    // the kept columns (kk x kk, column-major)
    auto chol = [&](const std::vector<cuDoubleComplex>& g, int k, const std::vector<double>& thr,
                    int limit, std::vector<int>& kept, std::vector<cuDoubleComplex>& r) {
      kept.clear();
      std::vector<std::vector<cuDoubleComplex>> rows;   // r rows of kept columns, over all k
      for (int j = 0; j < k && (int)kept.size() < limit; ++j) {
        double v = cuCreal(g[(size_t)j * k + j]);
        for (const auto& ri : rows) v -= cuCreal(cuCmul(cuConj(ri[j]), ri[j]));
        if (!(v > thr[j])) continue;
        const double rjj = std::sqrt(v);
        std::vector<cuDoubleComplex> rj(k, zero);
        rj[j] = make_cuDoubleComplex(rjj, 0.0);
        for (int l = j + 1; l < k; ++l) {
          cuDoubleComplex acc = g[(size_t)l * k + j];   // g[j][l]
          for (const auto& ri : rows) acc = cuCsub(acc, cuCmul(cuConj(ri[j]), ri[l]));
          rj[l] = make_cuDoubleComplex(cuCreal(acc) / rjj, cuCimag(acc) / rjj);
        }
        rows.push_back(std::move(rj));
        kept.push_back(j);
      }
      const int kk = (int)kept.size();
      r.assign((size_t)kk * kk, zero);
      for (int a = 0; a < kk; ++a)
        for (int c = a; c < kk; ++c) r[(size_t)c * kk + a] = rows[a][kept[c]];
    };
    // first pass
    project(X, b);
    project(X, b);
    std::vector<cuDoubleComplex> g, r;
    std::vector<int> kept;
    gram(X, b, g);
    std::vector<double> thr(b);
    for (int j = 0; j < b; ++j) thr[j] = (1e-6 * n0[j]) * (1e-6 * n0[j]);
    chol(g, b, thr, mmax - m, kept, r);
    const int kk = (int)kept.size();
    if (kk == 0) return 0;
    cuDoubleComplex* Y = col(V, m, n);   // survivors go straight to their place in V
    BSE_CUDA(cudaMemcpyAsync(idx.ptr, kept.data(), (size_t)kk * 4, cudaMemcpyHostToDevice, s));
    k_gather_cols<<<dim3((n + 255) / 256, kk), 256, 0, s>>>(
        n, kk, idx.as<int>(), reinterpret_cast<const double2*>(X), reinterpret_cast<double2*>(Y));
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
    BSE_CUDA(cudaMemcpyAsync(Rt.ptr, r.data(), (size_t)kk * kk * 16, cudaMemcpyHostToDevice, s));
    BSE_CUBLAS(cublasZtrsm(h.blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                           CUBLAS_DIAG_NON_UNIT, n, kk, &one, Rt.as<cuDoubleComplex>(), kk, Y, n));
    // second pass: project again, orthonormalise again (nothing expected to drop)
    project(Y, kk);
    gram(Y, kk, g);
    std::vector<double> thr2(kk, 1e-20);
    chol(g, kk, thr2, kk, kept, r);
    if ((int)kept.size() != kk)
      throw Error(BSE_ERR_NO_CONV, "Davidson basis lost orthogonality in the second pass");
    BSE_CUDA(cudaMemcpyAsync(Rt.ptr, r.data(), (size_t)kk * kk * 16, cudaMemcpyHostToDevice, s));
    BSE_CUBLAS(cublasZtrsm(h.blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                           CUBLAS_DIAG_NON_UNIT, n, kk, &one, Rt.as<cuDoubleComplex>(), kk, Y, n));
    m += kk;
    return kk;
  }

  // projected problem on the current basis; fills U (u, m x nev), W (w, m x nev), E (host)
  void rayleigh_ritz(int k, std::vector<double>& E) {
    const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0);
    // a+ = V^H P, a- = V^H M: only the columns of the vectors added since the
    // last step (the basis only grows between restarts); the rows of the new
    // vectors in the old columns follow from Hermiticity
    const int m0 = m_proj < m ? m_proj : 0, nw = m - m0;
    BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_C, CUBLAS_OP_N, m, nw, n, &one,
                           V.as<cuDoubleComplex>(), n, P.as<cuDoubleComplex>() + (int64_t)m0 * n, n,
                           &zero, ap.as<cuDoubleComplex>() + (int64_t)m0 * mmax, mmax));
    BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_C, CUBLAS_OP_N, m, nw, n, &one,
                           V.as<cuDoubleComplex>(), n, M.as<cuDoubleComplex>() + (int64_t)m0 * n, n,
                           &zero, am.as<cuDoubleComplex>() + (int64_t)m0 * mmax, mmax));
    m_proj = m;
    dim3 tb(16, 16), gb((m + 15) / 16, (m + 15) / 16);
    dim3 gn((m + 15) / 16, (nw + 15) / 16);
    k_hermitize_new<<<gn, tb, 0, s>>>(m0, m, ap.as<double2>(), mmax);
    k_hermitize_new<<<gn, tb, 0, s>>>(m0, m, am.as<double2>(), mmax);
    note_launches(2);
    // a- = l l^H
    BSE_CUDA(cudaMemcpy2DAsync(L.ptr, (size_t)mmax * 16, am.ptr, (size_t)mmax * 16, (size_t)m * 16,
                               m, cudaMemcpyDeviceToDevice, s));
    BSE_CUSOLVER(cusolverDnZpotrf(h.solver, CUBLAS_FILL_MODE_LOWER, m, L.as<cuDoubleComplex>(),
                                  mmax, work_->as<cuDoubleComplex>(), lwork, info.as<int>()));
    int hinfo = 0;
    BSE_CUDA(cudaMemcpyAsync(&hinfo, info.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaStreamSynchronize(s));
    if (hinfo != 0)
      throw Error(BSE_ERR_NOT_PD, "projected A-B is not positive definite (A-B or A+B not PD)");
    k_zero_strict_upper<<<gb, tb, 0, s>>>(m, L.as<double2>(), mmax);
    note_launches(1);
    // s = l^H a+ l
    BSE_CUBLAS(cublasZtrmm(h.blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N,
                           CUBLAS_DIAG_NON_UNIT, m, m, &one, L.as<cuDoubleComplex>(), mmax,
                           ap.as<cuDoubleComplex>(), mmax, W.as<cuDoubleComplex>(), mmax));
    BSE_CUBLAS(cublasZtrmm(h.blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_C,
                           CUBLAS_DIAG_NON_UNIT, m, m, &one, L.as<cuDoubleComplex>(), mmax,
                           W.as<cuDoubleComplex>(), mmax, S.as<cuDoubleComplex>(), mmax));
    BSE_CUSOLVER(cusolverDnZheevd(h.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m,
                                  S.as<cuDoubleComplex>(), mmax, dE.as<double>(),
                                  work_->as<cuDoubleComplex>(), lwork, info.as<int>()));
    std::vector<double> e2(m);
    BSE_CUDA(cudaMemcpyAsync(e2.data(), dE.ptr, m * 8, cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaMemcpyAsync(&hinfo, info.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaStreamSynchronize(s));
    if (hinfo != 0) throw Error(BSE_ERR_CUDA, "zheevd on the projected problem failed");
    E.assign(k, 0.0);
    std::vector<double> f(k);
    for (int j = 0; j < k; ++j) {
      if (!(e2[j] > 0.0)) throw Error(BSE_ERR_NOT_PD, "projected E^2 <= 0 (A+B not PD)");
      E[j] = std::sqrt(e2[j]);
      f[j] = 1.0 / std::sqrt(E[j]);
    }
    // u = l z E^-1/2
    BSE_CUBLAS(cublasZtrmm(h.blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N,
                           CUBLAS_DIAG_NON_UNIT, m, k, &one, L.as<cuDoubleComplex>(), mmax,
                           S.as<cuDoubleComplex>(), mmax, U.as<cuDoubleComplex>(), mmax));
    BSE_CUDA(cudaMemcpyAsync(dF.ptr, f.data(), k * 8, cudaMemcpyHostToDevice, s));
    k_scale_cols<<<dim3((m + 127) / 128, k), 128, 0, s>>>(m, k, U.as<double2>(), mmax,
                                                          dF.as<double>());
    // w = a+ u / E
    BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, m, k, m, &one,
                           ap.as<cuDoubleComplex>(), mmax, U.as<cuDoubleComplex>(), mmax, &zero,
                           W.as<cuDoubleComplex>(), mmax));
    for (int j = 0; j < k; ++j) f[j] = 1.0 / E[j];
    BSE_CUDA(cudaMemcpyAsync(dF.ptr, f.data(), k * 8, cudaMemcpyHostToDevice, s));
    k_scale_cols<<<dim3((m + 127) / 128, k), 128, 0, s>>>(m, k, W.as<double2>(), mmax,
                                                          dF.as<double>());
    note_launches(2);
    BSE_CUDA(cudaMemcpyAsync(dE.ptr, E.data(), k * 8, cudaMemcpyHostToDevice, s));
  }

  // r+ = P u - V (w E), r- = M w - V (u E) into R1, R2 (n x k); returns max column norms
  void residuals(int k, const std::vector<double>& E, std::vector<double>& res) {
    const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0),
                          mone = make_cuDoubleComplex(-1, 0);
    // X+Y and X-Y as full vectors, scaled by E: T[:, 0:k] = V (w E), T[:, k:2k] = V (u E)
    BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, k, m, &one,
                           V.as<cuDoubleComplex>(), n, W.as<cuDoubleComplex>(), mmax, &zero,
                           T.as<cuDoubleComplex>(), n));
    BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, k, m, &one,
                           V.as<cuDoubleComplex>(), n, U.as<cuDoubleComplex>(), mmax, &zero,
                           col(T, k, n), n));
    k_scale_cols<<<dim3((n + 127) / 128, k), 128, 0, s>>>(n, k, T.as<double2>(), n, dE.as<double>());
    k_scale_cols<<<dim3((n + 127) / 128, k), 128, 0, s>>>(n, k, T.as<double2>() + (int64_t)k * n, n,
                                                          dE.as<double>());
    note_launches(2);
    BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, k, m, &one,
                           P.as<cuDoubleComplex>(), n, U.as<cuDoubleComplex>(), mmax, &zero,
                           R1.as<cuDoubleComplex>(), n));
    BSE_CUBLAS(cublasZaxpy(h.blas, n * k, &mone, T.as<cuDoubleComplex>(), 1,
                           R1.as<cuDoubleComplex>(), 1));
    BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, k, m, &one,
                           M.as<cuDoubleComplex>(), n, W.as<cuDoubleComplex>(), mmax, &zero,
                           R2.as<cuDoubleComplex>(), n));
    BSE_CUBLAS(cublasZaxpy(h.blas, n * k, &mone, col(T, k, n), 1, R2.as<cuDoubleComplex>(), 1));
    res.assign(k, 0.0);
    k_col_norms<<<k, 256, 0, s>>>(n, R1.as<double2>(), R2.as<double2>(), n, nrm.as<double>());
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
    BSE_CUDA(cudaMemcpyAsync(res.data(), nrm.ptr, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaStreamSynchronize(s));
  }
};

// Training samples from one Davidson iteration (see TrajectorySink): for every
// unconverged pair, the Ritz vectors X+Y = V u, X-Y = V w against the exact
// pair aligned in phase, with the residuals in R1 / R2.
void record_trajectory(Solver& sv, TrajectorySink& sink, std::unique_ptr<DeviceBuffer>& xm_exact,
                       const std::vector<int>& todo, const std::vector<double>& E,
                       cudaStream_t s) {
  const int n = sv.n;
  const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0);
  DeviceBuffer xt((size_t)n * 16, s), st((size_t)n * 16, s);
  for (int lam : todo) {
    if (sink.count + 2 * (int64_t)n > sink.capacity) return;
    for (int eq = 0; eq < 2; ++eq) {
      // current vector of this equation's unknown
      BSE_CUBLAS(cublasZgemv(sv.h.blas, CUBLAS_OP_N, n, sv.m, &one, sv.V.as<cuDoubleComplex>(), n,
                             (eq == 0 ? sv.U : sv.W).as<cuDoubleComplex>() + (int64_t)lam * sv.mmax,
                             1, &zero, xt.as<cuDoubleComplex>(), 1));
      const cuDoubleComplex* xe =
          eq == 0 ? reinterpret_cast<const cuDoubleComplex*>(sink.xpy_exact) + (int64_t)lam * n
                  : xm_exact->as<cuDoubleComplex>() + (int64_t)lam * n;
      cuDoubleComplex ov;
      BSE_CUBLAS(cublasZdotc(sv.h.blas, n, xe, 1, xt.as<cuDoubleComplex>(), 1, &ov));
      const double mag = std::hypot(ov.x, ov.y);
      const cuDoubleComplex ph = mag > 0 ? make_cuDoubleComplex(-ov.x / mag, -ov.y / mag)
                                         : make_cuDoubleComplex(-1, 0);
      // step = x~ - phase * x
      BSE_CUBLAS(cublasZcopy(sv.h.blas, n, xt.as<cuDoubleComplex>(), 1, st.as<cuDoubleComplex>(), 1));
      BSE_CUBLAS(cublasZaxpy(sv.h.blas, n, &ph, xe, 1, st.as<cuDoubleComplex>(), 1));
      const double2* r = (eq == 0 ? sv.R1 : sv.R2).as<double2>() + (int64_t)lam * n;
      mlp_record(sink.net, n, sv.dDp.as<double>(), sv.dDm.as<double>(), sv.dS.as<double>(),
                 E[lam], lam, eq == 0, r, xt.as<double2>(), st.as<double2>(),
                 sink.feat + sink.count * mlp_num_features(sink.net), sink.target + sink.count,
                 sink.weight + sink.count, s);
      sink.count += n;
    }
  }
}

// xm = (AX + BX) / E per column (X-Y from X+Y of exact pairs)
__global__ void k_xmy(int64_t total, int n, const double2* ax, const double2* bx, const double* e,
                      double2* xm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ie = 1.0 / e[i / n];
    const double2 a = ax[i], b = bx ? bx[i] : make_double2(0.0, 0.0);
    xm[i] = make_double2((a.x + b.x) * ie, (a.y + b.y) * ie);
  }
}

}  // namespace

// Largest basis per wanted exciton (vectors of V per nev).  The projected
// m x m eigensolve grows as m^3, so a smaller basis trades more restarts for
// cheaper iterations; which wins depends on the problem.  Lowest 50 core-level
// excitons: at N = 8,640, 24 per exciton took 70 iterations in 8.4 s and 12
// took 97 in 6.3 s; at N = 20,480, 24 took 84 in 16.6 s and 12 took 161 in
// 26.5 s.  The environment variable BSE_DAVIDSON_BASIS_PER_EV (6 to 48)
// overrides the default for tuning.
static int basis_per_ev() {
  const char* e = getenv("BSE_DAVIDSON_BASIS_PER_EV");
  const int v = e ? atoi(e) : 24;
  return v >= 6 && v <= 48 ? v : 24;
}

void davidson_fp64(int n, const bse_c128* A, const bse_c128* B, int64_t ld, int nev, double tol,
                   int max_iter, int precond, const MlpNet* mlp, double* E_out,
                   bse_c128* XpY_out, int32_t* iters_out, cudaStream_t s, TrajectorySink* sink,
                   int matvec_precision, const bse_c128* V0, int k0) {
  std::unique_lock<std::mutex> lock;
  LibHandles h = acquire_handles(lock);
  BSE_CUSOLVER(cusolverDnSetStream(h.solver, s));
  BSE_CUBLAS(cublasSetStream(h.blas, s));
  BSE_CUBLAS(cublasSetPointerMode(h.blas, CUBLAS_POINTER_MODE_HOST));

  // basis of up to basis_per_ev() nev vectors; a restart keeps X+Y and X-Y of
  // the 2 nev lowest Ritz pairs (thick restart)
  const int mmax = std::min(n, std::max(basis_per_ev() * nev, nev + 96));
  Solver sv(n, nev, mmax, A, B, ld, s, h);
  // learned preconditioner: per-column records (eq, exciton) and feature scratch
  std::unique_ptr<DeviceBuffer> pc_cols, pc_feat;
  if (precond == 1) {
    mlp_check_neighbours(mlp, n, nev);
    pc_cols.reset(new DeviceBuffer((size_t)4 * nev * sizeof(int), s));
    pc_feat.reset(new DeviceBuffer((size_t)n * 2 * nev * mlp_num_features(mlp) * sizeof(float), s));
  }
  std::unique_ptr<TcMatvec, void (*)(TcMatvec*)> tcm(nullptr, tc_matvec_destroy);
  if (matvec_precision != BSE_PREC_FP64) {
    tcm.reset(tc_matvec_create(n, A, B, ld, matvec_precision, mmax, s));
    sv.tcm = tcm.get();
  }

  // diagonal of A: initial guess (unit vectors at the smallest A_aa); diagonals
  // of A+B and A-B and off-diagonal row norms for the preconditioners
  k_diag_real<<<(n + 255) / 256, 256, 0, s>>>(n, reinterpret_cast<const double2*>(A), ld,
                                              sv.dD.as<double>());
  note_launches(1);
  mlp_diag_features(n, A, B, ld, sv.dDp.as<double>(), sv.dDm.as<double>(), sv.dS.as<double>(), s);
  sv.D.resize(n);
  BSE_CUDA(cudaMemcpyAsync(sv.D.data(), sv.dD.ptr, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sv.D[a] < sv.D[b]; });
  const int b0 = std::min(n, std::min(mmax, nev + std::max(4, nev / 4)));
  int m_done = 0;   // basis columns whose P and M are computed
  if (V0 && k0 > 0) {
    // warm start: the given vectors (X+Y of nearby excitons) and their images
    // under A+B (proportional to the matching X-Y, which the one basis must
    // also hold), orthonormalised, then unit vectors at the smallest A_aa
    // until the basis holds b0 vectors (dependent ones drop)
    BSE_CUDA(cudaMemcpyAsync(sv.T.ptr, V0, (size_t)n * k0 * 16, cudaMemcpyDeviceToDevice, s));
    sv.m = 0;
    sv.append_block(sv.T.as<cuDoubleComplex>(), k0);
    sv.matvec(0, sv.m);
    m_done = sv.m;
    BSE_CUDA(cudaMemcpyAsync(sv.T.ptr, sv.P.ptr, (size_t)n * m_done * 16, cudaMemcpyDeviceToDevice,
                             s));
    sv.append_block(sv.T.as<cuDoubleComplex>(), m_done);
    sv.matvec(m_done, sv.m);
    m_done = sv.m;
    int next = 0;
    while (sv.m < b0 && next < n) {
      const int b = std::min(b0 - sv.m, n - next);
      BSE_CUDA(cudaMemsetAsync(sv.T.ptr, 0, (size_t)n * b * 16, s));
      for (int j = 0; j < b; ++j) {
        const double2 one = make_double2(1.0, 0.0);
        BSE_CUDA(cudaMemcpyAsync(sv.T.as<double2>() + (int64_t)j * n + order[next + j], &one, 16,
                                 cudaMemcpyHostToDevice, s));
      }
      next += b;
      sv.append_block(sv.T.as<cuDoubleComplex>(), b);
    }
  } else {
    BSE_CUDA(cudaMemsetAsync(sv.V.ptr, 0, (size_t)n * b0 * 16, s));
    for (int j = 0; j < b0; ++j) {
      const double2 one = make_double2(1.0, 0.0);
      BSE_CUDA(cudaMemcpyAsync(sv.V.as<double2>() + (int64_t)j * n + order[j], &one, 16,
                               cudaMemcpyHostToDevice, s));
    }
    sv.m = b0;
  }
  sv.matvec(m_done, sv.m);

  // exact X-Y of the recorded problem (trajectory samples only)
  std::unique_ptr<DeviceBuffer> xm_exact;
  if (sink) {
    xm_exact.reset(new DeviceBuffer((size_t)n * nev * 16, s));
    DeviceBuffer de((size_t)nev * 8, s);
    BSE_CUDA(cudaMemcpyAsync(de.ptr, sink->e_exact, (size_t)nev * 8, cudaMemcpyHostToDevice, s));
    MatvecProb pa{n, nev, n, A, ld, sink->xpy_exact, n, sv.AV.as<bse_c128>(), n};
    launch_zgemm(pa, 1, s);
    if (B) {
      MatvecProb pb{n, nev, n, B, ld, sink->xpy_exact, n, sv.BV.as<bse_c128>(), n};
      launch_zgemm(pb, 1, s);
    }
    const int64_t tot = (int64_t)n * nev;
    k_xmy<<<(int)std::min<int64_t>((tot + 255) / 256, 152 * 8), 256, 0, s>>>(
        tot, n, sv.AV.as<double2>(), B ? sv.BV.as<double2>() : nullptr, de.as<double>(),
        xm_exact->as<double2>());
    note_launches(1);   // AV / BV are scratch: P and M of the start basis are untouched
  }

  std::vector<double> E, res;
  const int k = nev;
  int it = 0;
  bool converged = false;
  for (it = 1; it <= max_iter; ++it) {
    const int kr = std::min(sv.m, 2 * k);   // Ritz pairs kept at a restart
    {
      Phase ph("davidson_rayleigh_ritz", s);
      sv.rayleigh_ritz(kr, E);
    }
    {
      Phase ph("davidson_residuals", s);
      sv.residuals(k, E, res);
    }
    std::vector<int> todo;
    for (int j = 0; j < k; ++j)
      if (!(res[j] < tol)) todo.push_back(j);
    if (sink) record_trajectory(sv, *sink, xm_exact, todo, E, s);
    if (todo.empty()) {
      converged = true;
      break;
    }
    if (it == max_iter) break;
    const int nt = (int)todo.size();
    // preconditioned corrections of both residuals, columns in T
    std::vector<double> et(nt);
    for (int i = 0; i < nt; ++i) et[i] = E[todo[i]];
    BSE_CUDA(cudaMemcpyAsync(sv.dF.ptr, et.data(), nt * 8, cudaMemcpyHostToDevice, s));
    for (int i = 0; i < nt; ++i) {
      BSE_CUDA(cudaMemcpyAsync(sv.AV.as<double2>() + (int64_t)i * n,
                               sv.R1.as<double2>() + (int64_t)todo[i] * n, (size_t)n * 16,
                               cudaMemcpyDeviceToDevice, s));
      BSE_CUDA(cudaMemcpyAsync(sv.AV.as<double2>() + (int64_t)(nt + i) * n,
                               sv.R2.as<double2>() + (int64_t)todo[i] * n, (size_t)n * 16,
                               cudaMemcpyDeviceToDevice, s));
    }
    // both blocks use the same eigenvalue list
    BSE_CUDA(cudaMemcpyAsync(sv.dF.as<double>() + nt, et.data(), nt * 8, cudaMemcpyHostToDevice, s));
    if (precond == 1) {
      // the vectors the residuals correct: X+Y = T[:, k + lam] / E for the (A+B)
      // equation, X-Y = T[:, lam] / E for the other (scale irrelevant), into BV
      std::vector<int> cols(4 * nt);
      for (int i = 0; i < nt; ++i) {
        BSE_CUDA(cudaMemcpyAsync(sv.BV.as<double2>() + (int64_t)i * n,
                                 sv.T.as<double2>() + (int64_t)(k + todo[i]) * n, (size_t)n * 16,
                                 cudaMemcpyDeviceToDevice, s));
        BSE_CUDA(cudaMemcpyAsync(sv.BV.as<double2>() + (int64_t)(nt + i) * n,
                                 sv.T.as<double2>() + (int64_t)todo[i] * n, (size_t)n * 16,
                                 cudaMemcpyDeviceToDevice, s));
        cols[i] = 0;
        cols[nt + i] = 1;
        cols[2 * nt + i] = cols[3 * nt + i] = todo[i];
      }
      BSE_CUDA(cudaMemcpyAsync(pc_cols->ptr, cols.data(), cols.size() * sizeof(int),
                               cudaMemcpyHostToDevice, s));
      const int* ceq = pc_cols->as<int>();
      mlp_precondition(mlp, n, 2 * nt, ceq, ceq + 2 * nt, sv.dDp.as<double>(), sv.dDm.as<double>(),
                       sv.dS.as<double>(), sv.dF.as<double>(), sv.AV.as<double2>(), n,
                       sv.BV.as<double2>(), n, pc_feat->as<float>(), sv.T.as<double2>(), n, s);
      BSE_CUDA(cudaStreamSynchronize(s));   // cols (host) is read by the copy above
    } else {
      k_precond_diag<<<dim3((n + 127) / 128, 2 * nt), 128, 0, s>>>(
          n, 2 * nt, sv.dDp.as<double>(), sv.dDm.as<double>(), sv.dF.as<double>(),
          sv.AV.as<double2>(), n, sv.T.as<double2>(), n);
      BSE_CUDA(cudaGetLastError());
      note_launches(1);
    }
    // restart from the Ritz vectors when the new block would not fit
    Phase ph_o("davidson_basis", s);
    if (sv.m + 2 * nt > mmax) {
      const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0);
      // X+Y and X-Y of the kr lowest pairs into R1 (n x 2 kr), then rebuild V
      BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, kr, sv.m, &one,
                             sv.V.as<cuDoubleComplex>(), n, sv.U.as<cuDoubleComplex>(), mmax,
                             &zero, sv.R1.as<cuDoubleComplex>(), n));
      BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, kr, sv.m, &one,
                             sv.V.as<cuDoubleComplex>(), n, sv.W.as<cuDoubleComplex>(), mmax,
                             &zero, sv.R1.as<cuDoubleComplex>() + (int64_t)kr * n, n));
      sv.m = 0;
      sv.m_proj = 0;
      sv.append_block(sv.R1.as<cuDoubleComplex>(), 2 * kr);
      sv.matvec(0, sv.m);
    }
    const int m0 = sv.m;
    sv.append_block(sv.T.as<cuDoubleComplex>(), 2 * nt);
    if (sv.m == m0) break;   // no new direction: stagnated
    sv.matvec(m0, sv.m);
  }
  if (iters_out) *iters_out = std::min(it, max_iter);

  // outputs: E and X+Y = V u for the nev lowest
  BSE_CUDA(cudaMemcpyAsync(E_out, E.data(), (size_t)k * 8, cudaMemcpyHostToDevice, s));
  if (XpY_out) {
    const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0);
    BSE_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, n, k, sv.m, &one,
                           sv.V.as<cuDoubleComplex>(), n, sv.U.as<cuDoubleComplex>(), mmax, &zero,
                           reinterpret_cast<cuDoubleComplex*>(XpY_out), n));
  }
  BSE_CUDA(cudaStreamSynchronize(s));
  if (!converged)
    throw Error(BSE_ERR_NO_CONV, "Davidson did not reach the residual tolerance in " +
                                     std::to_string(max_iter) + " iterations");
}

}  // namespace bse
