// Half-size reduction (Eq. auxham, Cholesky form), eigensolve (Eq. auxevp)
// and the spectrum (Eqs. osci, chir, epsmtensor), all FP64.
//
// The dense Cholesky factorisation and the Hermitian eigensolver are
// cuSOLVER calls and the two triangular products cuBLAS ZTRMM; the
// element-wise set-up, the oscillator strengths and the eps_M sum are the
// kernels below.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <mutex>
#include <memory>
#include <vector>

#include "bse_internal.h"
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

// One cuSOLVER and one cuBLAS handle per device, created on first use and
// kept until exit; calls on them are serialised by a mutex.
struct Handles {
  cusolverDnHandle_t solver = nullptr;
  cublasHandle_t blas = nullptr;
};
std::mutex g_handle_mutex;
std::vector<Handles> g_handles;

Handles& handles_for_current_device() {
  int dev = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  if ((int)g_handles.size() <= dev) g_handles.resize(dev + 1);
  Handles& h = g_handles[dev];
  if (!h.solver) BSE_CUSOLVER(cusolverDnCreate(&h.solver));
  if (!h.blas) BSE_CUBLAS(cublasCreate(&h.blas));
  return h;
}

__global__ void k_plus_minus(int n, const double2* A, const double2* B, int64_t ld,
                             double2* S, double2* L) {
  int64_t total = (int64_t)n * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i % n, c = i / n;
    int64_t off = r + c * ld;
    double2 a = A[off];
    double2 b = B ? B[off] : make_double2(0.0, 0.0);
    S[off] = make_double2(a.x + b.x, a.y + b.y);
    L[off] = make_double2(a.x - b.x, a.y - b.y);
  }
}

__global__ void k_zero_upper(int n, double2* L, int64_t ld) {
  int64_t total = (int64_t)n * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i % n, c = i / n;
    if (r < c) L[r + c * ld] = make_double2(0.0, 0.0);
  }
}

// E = sqrt(E^2) in place; flag any E^2 <= 0.
__global__ void k_sqrt_energies(int n, double* e, int* bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double v = e[i];
    if (!(v > 0.0)) {
      atomicExch(bad, 1);
      e[i] = 0.0;
    } else {
      e[i] = sqrt(v);
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// r_j = sum_i L_ij rho_i  (r = L^T rho, no conjugate): one warp per column j.
__global__ void k_lt_rho(int n, const double2* L, int64_t ld, const double2* rho, double2* r) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double2* col = L + (int64_t)warp * ld;
  double sx = 0.0, sy = 0.0;
  for (int i = warp + lane; i < n; i += 32) {   // L is lower triangular
    double2 l = col[i], p = rho[i];
    sx = fma(l.x, p.x, fma(-l.y, p.y, sx));
    sy = fma(l.x, p.y, fma(l.y, p.x, sy));
  }
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  if (lane == 0) r[warp] = make_double2(sx, sy);
}

// u_lambda = sum_j Z_{j lambda} r_j, |t_lambda|^2 = |u|^2 / (E_lambda vc): one warp per lambda.
__global__ void k_oscillators(int n, const double2* Z, int64_t ld, const double2* r,
                              const double* e, double vc, double* osc) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double2* col = Z + (int64_t)warp * ld;
  double sx = 0.0, sy = 0.0;
  for (int j = lane; j < n; j += 32) {
    double2 z = col[j], q = r[j];
    sx = fma(z.x, q.x, fma(-z.y, q.y, sx));
    sy = fma(z.x, q.y, fma(z.y, q.x, sy));
  }
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  if (lane == 0) osc[warp] = (sx * sx + sy * sy) / (e[warp] * vc);
}

// eps(w) = 1 - c Ha sum_l osc_l [1/(w - E_l + i d) - 1/(w + E_l + i d)]: one block per w.
__global__ void k_eps(int n, const double* e, const double* osc, int n_omega,
                      const double* omega, double delta, double pref, double2* eps) {
  __shared__ double sx[32], sy[32];
  int iw = blockIdx.x;
  if (iw >= n_omega) return;
  double w = omega[iw];
  double d2 = delta * delta;
  double ax = 0.0, ay = 0.0;
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    double el = e[l], f = osc[l];
    double a = w - el, b = w + el;
    double ia = 1.0 / (a * a + d2), ib = 1.0 / (b * b + d2);
    // 1/(a + i d) = (a - i d)/(a^2 + d^2)
    ax += f * (a * ia - b * ib);
    ay += f * (-delta * ia + delta * ib);
  }
  ax = warp_sum(ax);
  ay = warp_sum(ay);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sx[wid] = ax;
    sy[wid] = ay;
  }
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    ax = lane < nw ? sx[lane] : 0.0;
    ay = lane < nw ? sy[lane] : 0.0;
    ax = warp_sum(ax);
    ay = warp_sum(ay);
    if (lane == 0) eps[iw] = make_double2(1.0 - pref * ax, -pref * ay);
  }
}

int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

}  // namespace

LibHandles acquire_handles(std::unique_lock<std::mutex>& lock) {
  lock = std::unique_lock<std::mutex>(g_handle_mutex);
  Handles& h = handles_for_current_device();
  return LibHandles{h.solver, h.blas};
}

void reduce_fp64(int n, const bse_c128* A, const bse_c128* B, int64_t ld, bse_c128* S,
                 bse_c128* L, int32_t* failed_minor, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_handle_mutex);
  Handles& h = handles_for_current_device();
  BSE_CUSOLVER(cusolverDnSetStream(h.solver, s));
  BSE_CUBLAS(cublasSetStream(h.blas, s));

  // S <- A + B, L <- A - B
  k_plus_minus<<<grid_for((int64_t)n * n, 256), 256, 0, s>>>(
      n, reinterpret_cast<const double2*>(A), reinterpret_cast<const double2*>(B), ld,
      reinterpret_cast<double2*>(S), reinterpret_cast<double2*>(L));
  BSE_CUDA(cudaGetLastError());
  note_launches(1);

  // A - B = L L^H
  int lwork = 0;
  BSE_CUSOLVER(cusolverDnZpotrf_bufferSize(h.solver, CUBLAS_FILL_MODE_LOWER, n,
                                           reinterpret_cast<cuDoubleComplex*>(L), (int)ld,
                                           &lwork));
  DeviceBuffer work((size_t)(lwork > 0 ? lwork : 1) * sizeof(cuDoubleComplex), s);
  DeviceBuffer info(sizeof(int), s);
  {
    Phase ph("reduce_potrf", s);
    BSE_CUSOLVER(cusolverDnZpotrf(h.solver, CUBLAS_FILL_MODE_LOWER, n,
                                  reinterpret_cast<cuDoubleComplex*>(L), (int)ld,
                                  work.as<cuDoubleComplex>(), lwork, info.as<int>()));
  }
  int hinfo = 0;
  BSE_CUDA(cudaMemcpyAsync(&hinfo, info.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  if (failed_minor) *failed_minor = hinfo > 0 ? hinfo : 0;
  if (hinfo > 0)
    throw Error(BSE_ERR_NOT_PD, "A-B is not positive definite: leading minor " +
                                    std::to_string(hinfo) + " failed");
  if (hinfo < 0) throw Error(BSE_ERR_CUDA, "zpotrf: invalid parameter " + std::to_string(-hinfo));
  k_zero_upper<<<grid_for((int64_t)n * n, 256), 256, 0, s>>>(n, reinterpret_cast<double2*>(L),
                                                               ld);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);

  // S = L^H (A+B) L:  C = (A+B) L, then S = L^H C
  DeviceBuffer c((size_t)ld * n * sizeof(bse_c128), s);
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0);
  Phase ph("reduce_trmm", s);
  BSE_CUBLAS(cublasZtrmm(h.blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N,
                         CUBLAS_DIAG_NON_UNIT, n, n, &one,
                         reinterpret_cast<const cuDoubleComplex*>(L), (int)ld,
                         reinterpret_cast<const cuDoubleComplex*>(S), (int)ld,
                         c.as<cuDoubleComplex>(), (int)ld));
  BSE_CUBLAS(cublasZtrmm(h.blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_C,
                         CUBLAS_DIAG_NON_UNIT, n, n, &one,
                         reinterpret_cast<const cuDoubleComplex*>(L), (int)ld,
                         c.as<const cuDoubleComplex>(), (int)ld,
                         reinterpret_cast<cuDoubleComplex*>(S), (int)ld));
  BSE_CUDA(cudaStreamSynchronize(s));
}

__global__ void k_scale_cols_rsqrt(int n, int k, double2* x, int64_t ld, const double* e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i < n && j < k) {
    const double f = 1.0 / sqrt(e[j]);
    double2 v = x[i + (int64_t)j * ld];
    x[i + (int64_t)j * ld] = make_double2(v.x * f, v.y * f);
  }
}

void xpy_fp64(int n, int k, const bse_c128* Z, const bse_c128* L, int64_t ld, const double* E,
              bse_c128* XpY, int64_t ldx, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_handle_mutex);
  Handles& h = handles_for_current_device();
  BSE_CUBLAS(cublasSetStream(h.blas, s));
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0);
  // X+Y = L Z E^{-1/2} for the first k columns of Z
  BSE_CUBLAS(cublasZtrmm(h.blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N,
                         CUBLAS_DIAG_NON_UNIT, n, k, &one,
                         reinterpret_cast<const cuDoubleComplex*>(L), (int)ld,
                         reinterpret_cast<const cuDoubleComplex*>(Z), (int)ld,
                         reinterpret_cast<cuDoubleComplex*>(XpY), (int)ldx));
  k_scale_cols_rsqrt<<<dim3((n + 127) / 128, k), 128, 0, s>>>(
      n, k, reinterpret_cast<double2*>(XpY), ldx, E);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
}

void spectrum_fp64(int n, bse_c128* S, const bse_c128* L, int64_t ld, const bse_c128* rho,
                   double c_q, double vc, int n_omega, const double* omega, double delta,
                   double* E_out, double* osc_out, bse_c128* eps_out, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_handle_mutex);
  Handles& h = handles_for_current_device();
  BSE_CUSOLVER(cusolverDnSetStream(h.solver, s));

  // 64-bit generic interface: the 32-bit zheevd rejects N of tens of thousands
  cusolverDnParams_t params = nullptr;
  BSE_CUSOLVER(cusolverDnCreateParams(&params));
  std::unique_ptr<cusolverDnParams, cusolverStatus_t (*)(cusolverDnParams_t)> params_guard(
      params, cusolverDnDestroyParams);
  size_t dev_bytes = 0, host_bytes = 0;
  BSE_CUSOLVER(cusolverDnXsyevd_bufferSize(h.solver, params, CUSOLVER_EIG_MODE_VECTOR,
                                           CUBLAS_FILL_MODE_LOWER, n, CUDA_C_64F, S, ld,
                                           CUDA_R_64F, E_out, CUDA_C_64F, &dev_bytes,
                                           &host_bytes));
  DeviceBuffer work(dev_bytes > 0 ? dev_bytes : 16, s);
  std::vector<char> host_work(host_bytes > 0 ? host_bytes : 16);
  DeviceBuffer flags(2 * sizeof(int), s);
  BSE_CUDA(cudaMemsetAsync(flags.ptr, 0, 2 * sizeof(int), s));
  {
    Phase ph("eig_heevd", s);
    BSE_CUSOLVER(cusolverDnXsyevd(h.solver, params, CUSOLVER_EIG_MODE_VECTOR,
                                  CUBLAS_FILL_MODE_LOWER, n, CUDA_C_64F, S, ld, CUDA_R_64F, E_out,
                                  CUDA_C_64F, work.ptr, dev_bytes, host_work.data(), host_bytes,
                                  flags.as<int>()));
  }
  Phase ph("spectrum_kernels", s);
  k_sqrt_energies<<<(n + 255) / 256, 256, 0, s>>>(n, E_out, flags.as<int>() + 1);
  BSE_CUDA(cudaGetLastError());

  DeviceBuffer r((size_t)n * sizeof(bse_c128), s);
  const int warps_per_block = 8;
  int blocks = (n + warps_per_block - 1) / warps_per_block;
  k_lt_rho<<<blocks, 32 * warps_per_block, 0, s>>>(
      n, reinterpret_cast<const double2*>(L), ld, reinterpret_cast<const double2*>(rho),
      r.as<double2>());
  k_oscillators<<<blocks, 32 * warps_per_block, 0, s>>>(
      n, reinterpret_cast<const double2*>(S), ld, r.as<const double2>(), E_out, vc, osc_out);
  if (n_omega > 0)
    k_eps<<<n_omega, 256, 0, s>>>(n, E_out, osc_out, n_omega, omega, delta,
                                  c_q * kHartreeEv, reinterpret_cast<double2*>(eps_out));
  BSE_CUDA(cudaGetLastError());
  note_launches(n_omega > 0 ? 4 : 3);

  int hflags[2] = {0, 0};
  BSE_CUDA(cudaMemcpyAsync(hflags, flags.ptr, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  if (hflags[0] != 0)
    throw Error(BSE_ERR_CUDA, "zheevd failed, info = " + std::to_string(hflags[0]));
  if (hflags[1] != 0)
    throw Error(BSE_ERR_NOT_PD, "an eigenvalue E^2 <= 0: A+B is not positive definite");
}


// ---------------------------------------------------------------------------
// Cartesian dielectric tensor (Eq. epsmij) and loss function (Eq. Lofeps)
// ---------------------------------------------------------------------------
namespace {

// u[lambda][i] = sum_j Z_{j lambda} r_i[j] for the three directions (r_i =
// L^T D_i), one warp per lambda; with X+Y = L Z E^{-1/2} this is
// E^{1/2} sum_alpha (X+Y)_{alpha lambda} D_{alpha i}, so that the coefficient
// t*_{lambda i} t_{lambda j} of Eq. tlambdai is u_i conj(u_j) / (E vc)
__global__ void k_tensor_u(int n, const double2* Z, int64_t ld, const double2* r, double2* u) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double2* col = Z + (int64_t)warp * ld;
  double sx[3] = {0, 0, 0}, sy[3] = {0, 0, 0};
  for (int j = lane; j < n; j += 32) {
    const double2 z = col[j];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double2 q = r[(int64_t)i * n + j];
      sx[i] = fma(z.x, q.x, fma(-z.y, q.y, sx[i]));
      sy[i] = fma(z.x, q.y, fma(z.y, q.x, sy[i]));
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    sx[i] = warp_sum(sx[i]);
    sy[i] = warp_sum(sy[i]);
    if (lane == 0) u[(int64_t)warp * 3 + i] = make_double2(sx[i], sy[i]);
  }
}

// eps^{ij}(w) = delta_ij - pref sum_l u_i conj(u_j) / (E_l vc) [1/(w - E_l + i d)
// - 1/(w + E_l + i d)], one block per w; 9 complex sums reduced per block
__global__ void __launch_bounds__(256) k_eps_tensor(int n, const double* e, const double2* u,
                                                    double vc, int n_omega, const double* omega,
                                                    double delta, double pref, double2* eps) {
  __shared__ double red[18][8];
  const int iw = blockIdx.x;
  if (iw >= n_omega) return;
  const double w = omega[iw], d2 = delta * delta;
  double acc[18];
#pragma unroll
  for (int q = 0; q < 18; ++q) acc[q] = 0.0;
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    const double el = e[l];
    const double a = w - el, b = w + el;
    const double ia = 1.0 / (a * a + d2), ib = 1.0 / (b * b + d2);
    const double fx = (a * ia - b * ib) / (el * vc), fy = (-delta * ia + delta * ib) / (el * vc);
    double2 ui[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) ui[i] = u[(int64_t)l * 3 + i];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        // c = u_i conj(u_j); c * f
        const double cx = ui[i].x * ui[j].x + ui[i].y * ui[j].y;
        const double cy = ui[i].y * ui[j].x - ui[i].x * ui[j].y;
        acc[2 * (3 * i + j)] += cx * fx - cy * fy;
        acc[2 * (3 * i + j) + 1] += cx * fy + cy * fx;
      }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 18; ++q) {
    const double v = warp_sum(acc[q]);
    if (lane == 0) red[q][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 18) {
    double v = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += red[threadIdx.x][k];
    red[threadIdx.x][0] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    const int i = threadIdx.x / 3, j = threadIdx.x % 3;
    eps[(int64_t)iw * 9 + threadIdx.x] =
        make_double2((i == j ? 1.0 : 0.0) - pref * red[2 * threadIdx.x][0],
                     -pref * red[2 * threadIdx.x + 1][0]);
  }
}

// L = -Im 1/eps = Im eps / |eps|^2; S = v_inv L / pi
__global__ void k_loss(int n_omega, const double2* eps, double v_inv, double* loss, double* sqw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_omega) return;
  const double2 e = eps[i];
  const double l = e.y / (e.x * e.x + e.y * e.y);
  if (loss) loss[i] = l;
  if (sqw) sqw[i] = v_inv * l / 3.14159265358979323846;
}

}  // namespace

void spectrum_tensor_fp64(int n, const bse_c128* Z, const bse_c128* L, int64_t ld,
                          const bse_c128* D, int64_t ldd, double c_q, double vc, int n_omega,
                          const double* omega, double delta, const double* E, bse_c128* eps_out,
                          cudaStream_t s) {
  DeviceBuffer r((size_t)3 * n * sizeof(bse_c128), s);
  DeviceBuffer u((size_t)3 * n * sizeof(bse_c128), s);
  const int warps_per_block = 8;
  const int blocks = (n + warps_per_block - 1) / warps_per_block;
  for (int i = 0; i < 3; ++i)
    k_lt_rho<<<blocks, 32 * warps_per_block, 0, s>>>(
        n, reinterpret_cast<const double2*>(L), ld,
        reinterpret_cast<const double2*>(D) + (int64_t)i * ldd, r.as<double2>() + (int64_t)i * n);
  k_tensor_u<<<blocks, 32 * warps_per_block, 0, s>>>(n, reinterpret_cast<const double2*>(Z), ld,
                                                     r.as<double2>(), u.as<double2>());
  if (n_omega > 0)
    k_eps_tensor<<<n_omega, 256, 0, s>>>(n, E, u.as<double2>(), vc, n_omega, omega, delta,
                                         c_q * kHartreeEv, reinterpret_cast<double2*>(eps_out));
  BSE_CUDA(cudaGetLastError());
  note_launches(n_omega > 0 ? 5 : 4);
  BSE_CUDA(cudaStreamSynchronize(s));   // r, u are stream-ordered workspace
}

void loss_fp64(int n_omega, const bse_c128* eps, double v_inv, double* loss_out, double* sqw_out,
               cudaStream_t s) {
  if (n_omega <= 0) return;
  k_loss<<<(n_omega + 255) / 256, 256, 0, s>>>(n_omega, reinterpret_cast<const double2*>(eps),
                                               v_inv, loss_out, sqw_out);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
}

// ---------------------------------------------------------------------------
// Static RPA screening (Sec. 2: Eq. wggq with the RPA dielectric matrix), FP64
// ---------------------------------------------------------------------------
namespace {

// Partial polarisability sums of the FP64 path, one K range of kc transitions
// per batch entry b: part[b][G][G'] = sum_{a in range b} conj(mt[a][G]) mt[a][G']
struct RpaXProb {
  int M, N, K;            // ng, ng, kc
  const bse_c128* mt;     // [ntr][ng]
  int64_t ntr;
  double2* part;          // [batches][ng][ng]
  __device__ cplx a(int b, int m, int k) const {
    const int64_t t = (int64_t)b * K + k;
    return t < ntr ? conj(ldc(mt + t * M + m)) : cmake(0.0, 0.0);
  }
  __device__ cplx b(int b, int n, int k) const {
    const int64_t t = (int64_t)b * K + k;
    return t < ntr ? ldc(mt + t * N + n) : cmake(0.0, 0.0);
  }
  __device__ void store(int b, int m, int n, cplx v) const {
    part[((int64_t)b * M + m) * N + n] = make_double2(v.x, v.y);
  }
};

// x[i] = sum over batches of part[b][i], in batch order
__global__ void k_rpa_sum64(const double2* part, int batches, int64_t nn, double2* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
       i += (int64_t)gridDim.x * blockDim.x) {
    double sx = 0.0, sy = 0.0;
    for (int b = 0; b < batches; ++b) {
      const double2 p = part[(int64_t)b * nn + i];
      sx += p.x;
      sy += p.y;
    }
    x[i] = make_double2(sx, sy);
  }
}

// mt[a][G] = m[a][G] / sqrt(e_c_kq[k][c] - e_v[k][v]), a = (k v c)
__global__ void k_rpa_scale(int64_t total, int nv, int nc, int ng, const double* e_v,
                            const double* e_c_kq, const double2* m, double2* mt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = i / ng;
    const int c = (int)(a % nc), v = (int)((a / nc) % nv);
    const int64_t k = a / ((int64_t)nv * nc);
    const double f = 1.0 / sqrt(e_c_kq[k * nc + c] - e_v[k * nv + v]);
    const double2 x = m[i];
    mt[i] = make_double2(x.x * f, x.y * f);
  }
}

// eps[G][G'] = delta + 2 kappa X[G][G'] v[G'] in place (row-major), and the
// identity into rhs (column-major, the right-hand side of the solve)
__global__ void k_rpa_eps(int ng, double two_kappa, const double* v, double2* x, double2* rhs) {
  const int64_t total = (int64_t)ng * ng;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(i / ng), gp = (int)(i % ng);
    double2 e = x[i];
    e.x *= two_kappa * v[gp];
    e.y *= two_kappa * v[gp];
    if (g == gp) e.x += 1.0;
    x[i] = e;
    rhs[i] = make_double2(g == gp ? 1.0 : 0.0, 0.0);
  }
}

// w[G][G'] = v[G] inv[G][G'] (row-major)
__global__ void k_rpa_w(int ng, const double* v, const double2* inv, double2* w) {
  const int64_t total = (int64_t)ng * ng;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double f = v[i / ng];
    const double2 y = inv[i];
    w[i] = make_double2(f * y.x, f * y.y);
  }
}

}  // namespace

void rpa_screening(int nk, int nv, int nc, int ng, double omega_cell, const double* e_v,
                   const double* e_c_kq, const bse_c128* m, const double* v, int precision,
                   bse_c128* w_out, cudaStream_t s) {
  const int64_t ntr = (int64_t)nk * nv * nc;
  // X[G][G'] (row-major) into eps, by the library's own kernels: tensor cores
  // in split precision, or the FP64 GEMM kernel over K ranges of at most
  // 1,024 transitions with the partials added in FP64
  DeviceBuffer eps((size_t)ng * ng * sizeof(bse_c128), s);
  if (precision != BSE_PREC_FP64) {
    rpa_x_mixed(nk, nv, nc, ng, e_v, e_c_kq, m, precision, eps.as<double2>(), s);
  } else {
    Phase ph("rpa_x_fp64", s);
    DeviceBuffer mt((size_t)ntr * ng * sizeof(bse_c128), s);
    k_rpa_scale<<<grid_for(ntr * ng, 256), 256, 0, s>>>(ntr * ng, nv, nc, ng, e_v, e_c_kq,
                                                       reinterpret_cast<const double2*>(m),
                                                       mt.as<double2>());
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
    const int kc = (int)std::min<int64_t>(ntr, 1024);
    const int batches = (int)((ntr + kc - 1) / kc);
    DeviceBuffer part((size_t)batches * ng * ng * sizeof(bse_c128), s);
    RpaXProb P{ng, ng, kc, mt.as<bse_c128>(), ntr, part.as<double2>()};
    launch_zgemm(P, batches, s);
    k_rpa_sum64<<<grid_for((int64_t)ng * ng, 256), 256, 0, s>>>(part.as<double2>(), batches,
                                                                (int64_t)ng * ng, eps.as<double2>());
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
  }
  std::lock_guard<std::mutex> lock(g_handle_mutex);
  Handles& h = handles_for_current_device();
  BSE_CUSOLVER(cusolverDnSetStream(h.solver, s));
  BSE_CUBLAS(cublasSetStream(h.blas, s));
  DeviceBuffer rhs((size_t)ng * ng * sizeof(bse_c128), s);
  const double two_kappa = 2.0 * kHartreeEv / ((double)nk * omega_cell);
  k_rpa_eps<<<grid_for((int64_t)ng * ng, 256), 256, 0, s>>>(ng, two_kappa, v, eps.as<double2>(),
                                                           rhs.as<double2>());
  BSE_CUDA(cudaGetLastError());
  // the row-major eps is, column-major, eps^T; its inverse (eps^T)^-1 =
  // (eps^-1)^T in column-major storage is eps^-1 in row-major storage
  int lwork = 0;
  BSE_CUSOLVER(cusolverDnZgetrf_bufferSize(h.solver, ng, ng, eps.as<cuDoubleComplex>(), ng, &lwork));
  DeviceBuffer work((size_t)(lwork > 0 ? lwork : 1) * sizeof(cuDoubleComplex), s);
  DeviceBuffer ipiv((size_t)ng * sizeof(int), s);
  DeviceBuffer info(sizeof(int), s);
  BSE_CUSOLVER(cusolverDnZgetrf(h.solver, ng, ng, eps.as<cuDoubleComplex>(), ng,
                                work.as<cuDoubleComplex>(), ipiv.as<int>(), info.as<int>()));
  int hinfo = 0;
  BSE_CUDA(cudaMemcpyAsync(&hinfo, info.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  if (hinfo != 0)
    throw Error(BSE_ERR_CUDA, "zgetrf of the dielectric matrix failed (info " +
                                  std::to_string(hinfo) + ")");
  BSE_CUSOLVER(cusolverDnZgetrs(h.solver, CUBLAS_OP_N, ng, ng, eps.as<cuDoubleComplex>(), ng,
                                ipiv.as<int>(), rhs.as<cuDoubleComplex>(), ng, info.as<int>()));
  k_rpa_w<<<grid_for((int64_t)ng * ng, 256), 256, 0, s>>>(ng, v, rhs.as<double2>(),
                                                         reinterpret_cast<double2*>(w_out));
  BSE_CUDA(cudaGetLastError());
  note_launches(2);   // k_rpa_eps and k_rpa_w (the LU solve is cuSOLVER's)
  BSE_CUDA(cudaStreamSynchronize(s));   // the workspace is stream-ordered
}

}  // namespace bse
