// eps_M on a frequency grid without the eigensolve: a Lanczos recursion on
// the product form and a continued fraction.
//
// The spectrum of Eqs. chir / osci / epsmtensor sums over the excitons,
//   eps(w) = 1 - c_Q Ha sum_l |t_l|^2 [1/(w - E_l + i d) - 1/(w + E_l + i d)],
// with |t_l|^2 = |u_l|^2 / (E_l V_c), u = Z^T L^T rho, S Z = Z E^2 and
// S = L^H (A+B) L, A-B = L L^H (Eq. auxham).  Since 1/(z - E) - 1/(z + E) =
// 2E/(z^2 - E^2), the sum is (2 / V_c) w^H (z^2 - S)^-1 w with w = L^H conj(rho),
// and with K = (A-B)(A+B) = L S L^-1 it becomes
//   Q(z^2) = conj(rho)^H (z^2 - K)^-1 (A-B) conj(rho),   z = w + i d.
// K is self-adjoint in the inner product <a, b> = a^H (A-B)^-1 b, and
// Q = <v, (z^2 - K)^-1 v> for v = (A-B) conj(rho), <v, v> = conj(rho)^H (A-B)
// conj(rho).  Lanczos in that inner product keeps, beside each vector v_j,
// y_j = (A-B)^-1 v_j, so that no inverse or factorisation is needed:
//   u = (A+B) v_j,  alpha_j = v_j^H u,
//   y = u - alpha_j y_j - beta_{j-1} y_{j-1},  x = (A-B) y,  beta_j^2 = y^H x,
//   v_{j+1} = x / beta_j,  y_{j+1} = y / beta_j,
// two Hermitian matrix-vector products per step.  Q is then <v, v> over the
// continued fraction z^2 - alpha_0 - beta_0^2 / (z^2 - alpha_1 - ...) of the
// tridiagonal matrix (the recursion-method form of a resolvent element).
// The recursion stops when eps on the grid changes by less than tol (relative
// to its largest value) between checks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "bse_internal.h"
#include "lanczos.h"

namespace bse {
namespace {

constexpr int kGvRows = 256;     // rows per block of the matrix-vector kernel
constexpr int kGvCols = 64;      // columns of x staged in shared memory at a time

// partial[c][i] = sum_{j in chunk c} (A_ij + s B_ij) x_j  (column-major, ld)
__global__ void __launch_bounds__(kGvRows) k_pm_gemv(int n, const double2* __restrict__ A,
                                                     const double2* __restrict__ B, int64_t ld,
                                                     double s, const double2* __restrict__ x,
                                                     int chunk, double2* __restrict__ partial) {
  __shared__ double2 xs[kGvCols];
  const int i = blockIdx.x * kGvRows + threadIdx.x;
  const int j0 = blockIdx.y * chunk, j1 = min(n, j0 + chunk);
  double ax = 0.0, ay = 0.0;
  for (int jb = j0; jb < j1; jb += kGvCols) {
    const int jn = min(kGvCols, j1 - jb);
    __syncthreads();
    if (threadIdx.x < jn) xs[threadIdx.x] = x[jb + threadIdx.x];
    __syncthreads();
    if (i < n) {
      const double2* a = A + (int64_t)jb * ld + i;
      const double2* b = B ? B + (int64_t)jb * ld + i : nullptr;
#pragma unroll 8
      for (int t = 0; t < jn; ++t) {
        double2 m = a[(int64_t)t * ld];
        if (b) {
          const double2 bb = b[(int64_t)t * ld];
          m.x = fma(s, bb.x, m.x);
          m.y = fma(s, bb.y, m.y);
        }
        const double2 xv = xs[t];
        ax = fma(m.x, xv.x, fma(-m.y, xv.y, ax));
        ay = fma(m.x, xv.y, fma(m.y, xv.x, ay));
      }
    }
  }
  if (i < n) partial[(int64_t)blockIdx.y * n + i] = make_double2(ax, ay);
}

// the dot-product target: coef[2 j + off] for the step j held at jdev, or
// base itself (jdev NULL)
__device__ __forceinline__ double* dot_target(double* base, const int* jdev, int off) {
  return jdev ? base + 2 * (*jdev) + off : base;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  v = 0.0;
  if (threadIdx.x < (blockDim.x >> 5)) v = red[threadIdx.x];
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;   // valid in thread 0
}

// out = sum_c partial[c]; dot += Re(sum_i conj(w_i) out_i) (w NULL: no dot)
__global__ void __launch_bounds__(256) k_sum_partials(int n, int chunks, const double2* partial,
                                                      double2* out, const double2* w, double* dot,
                                                      const int* jdev, int off) {
  __shared__ double red[8];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double d = 0.0;
  if (i < n) {
    double2 acc = make_double2(0.0, 0.0);
    for (int c = 0; c < chunks; ++c) {
      const double2 p = partial[(int64_t)c * n + i];
      acc.x += p.x;
      acc.y += p.y;
    }
    out[i] = acc;
    if (w) d = w[i].x * acc.x + w[i].y * acc.y;
  }
  if (w) {
    d = block_sum(d, red);
    if (threadIdx.x == 0) atomicAdd(dot_target(dot, jdev, off), d);
  }
}

// y_new = u - alpha_j y_j - beta_{j-1} y_prev  (coef: alpha at 2j, beta^2 at
// 2j - 1; j the step held at jdev)
__global__ void k_lanczos_y(int n, const double2* u, const double2* yj, const double2* yprev,
                            const double* coef, const int* jdev, double2* ynew) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = *jdev;
  const double a = coef[2 * j];
  const double b = j > 0 ? sqrt(fmax(coef[2 * j - 1], 0.0)) : 0.0;
  const double2 uy = u[i], y1 = yj[i], y0 = yprev[i];
  ynew[i] = make_double2(uy.x - a * y1.x - b * y0.x, uy.y - a * y1.y - b * y0.y);
}

// scale x and y by 1 / sqrt(coef[k]), k = 2 j + 1 for the step held at jdev,
// or k_fixed (jdev NULL)
__global__ void k_lanczos_scale(int n, const double* coef, const int* jdev, int k_fixed, double2* x,
                                double2* y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double b2 = coef[jdev ? 2 * (*jdev) + 1 : k_fixed];
  const double f = b2 > 0.0 ? 1.0 / sqrt(b2) : 0.0;
  const double2 xv = x[i], yv = y[i];
  x[i] = make_double2(xv.x * f, xv.y * f);
  y[i] = make_double2(yv.x * f, yv.y * f);
}

// out = av + s bv (bv NULL: av); dot += Re(sum_i conj(w_i) out_i)
__global__ void __launch_bounds__(256) k_combine_dot(int n, const double2* av, const double2* bv,
                                                     double s, double2* out, const double2* w,
                                                     double* dot, const int* jdev, int off) {
  __shared__ double red[8];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double d = 0.0;
  if (i < n) {
    double2 o = av[i];
    if (bv) {
      o.x = fma(s, bv[i].x, o.x);
      o.y = fma(s, bv[i].y, o.y);
    }
    out[i] = o;
    d = w[i].x * o.x + w[i].y * o.y;
  }
  d = block_sum(d, red);
  if (threadIdx.x == 0) atomicAdd(dot_target(dot, jdev, off), d);
}

// C = A + B, D = A - B (n x n, C and D with leading dimension n)
__global__ void k_form_pm(int n, const double2* A, const double2* B, int64_t ld, double2* C,
                          double2* D) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e - j * n;
    const double2 a = A[i + j * ld], b = B[i + j * ld];
    C[e] = make_double2(a.x + b.x, a.y + b.y);
    D[e] = make_double2(a.x - b.x, a.y - b.y);
  }
}

// the step counter of the recursion: one thread, after a step's last kernel
__global__ void k_step_inc(int* jdev) { ++*jdev; }

// y = conj(rho)
__global__ void k_conj(int n, const double2* rho, double2* y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = make_double2(rho[i].x, -rho[i].y);
}

// eps(w) = 1 - pref <v,v> / (z^2 - alpha_0 - beta_0^2/(z^2 - alpha_1 - ...)),
// m coefficients (alpha_0 .. alpha_{m-1}, beta_0^2 .. beta_{m-2}^2); one thread
// per frequency
__global__ void k_lanczos_eps(int m, const double* coef, double nv2, int n_omega,
                              const double* omega, double delta, double pref, double2* eps) {
  const int iw = blockIdx.x * blockDim.x + threadIdx.x;
  if (iw >= n_omega) return;
  const double w = omega[iw];
  const double zr = w * w - delta * delta, zi = 2.0 * w * delta;   // (w + i d)^2
  double fr = zr - coef[2 * (m - 1)], fi = zi;
  for (int j = m - 2; j >= 0; --j) {
    const double b2 = coef[2 * j + 1];
    const double den = fr * fr + fi * fi;
    // f = z^2 - alpha_j - b2 / f
    const double qr = b2 * fr / den, qi = -b2 * fi / den;
    fr = zr - coef[2 * j] - qr;
    fi = zi - qi;
  }
  const double den = fr * fr + fi * fi;
  eps[iw] = make_double2(1.0 - pref * nv2 * fr / den, pref * nv2 * fi / den);
}

// diff[0] = max |a - b|, diff[1] = max |b| over the grid (one block)
__global__ void __launch_bounds__(256) k_eps_change(int n_omega, const double2* a, const double2* b,
                                                    double* diff) {
  __shared__ double r0[256], r1[256];
  double d = 0.0, m = 0.0;
  for (int i = threadIdx.x; i < n_omega; i += 256) {
    d = fmax(d, hypot(a[i].x - b[i].x, a[i].y - b[i].y));
    m = fmax(m, hypot(b[i].x, b[i].y));
  }
  r0[threadIdx.x] = d;
  r1[threadIdx.x] = m;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      r0[threadIdx.x] = fmax(r0[threadIdx.x], r0[threadIdx.x + h]);
      r1[threadIdx.x] = fmax(r1[threadIdx.x], r1[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    diff[0] = r0[0];
    diff[1] = r1[0];
  }
}

}  // namespace


// eps on the grid from the recursion above; returns the steps taken.
//
// The step index lives on the device (every step kernel reads it, a one-thread
// kernel advances it), so the kernels of a step take the same arguments at
// every step but for the buffer rotation, which repeats every 6 steps (v, x
// swap; y_{j-1}, y_j, y_{j+1} rotate).  With FP64 products, 6 steps are
// captured once as a CUDA graph and replayed: the launches, not the
// arithmetic, bound a step at small N.  The tensor-core products synchronise
// inside each call and run as plain launches.
int spectrum_lanczos(int n, const bse_c128* A, const bse_c128* B, int64_t ld, const bse_c128* rho,
                     double c_q, double vc, int n_omega, const double* omega, double delta,
                     double tol, int max_steps, int matvec_precision, bse_c128* eps_out,
                     cudaStream_t s) {
  const double2* A2 = reinterpret_cast<const double2*>(A);
  const double2* B2 = reinterpret_cast<const double2*>(B);
  int dev = 0, sms = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  BSE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // (row block, column chunk) blocks: about 16 per SM, so that enough loads
  // of A and B are in flight, but chunks of at least 32 columns
  const int row_blocks = (n + kGvRows - 1) / kGvRows;
  const int chunks = std::max(1, std::min(std::max(1, n / 32), (sms * 16 + row_blocks - 1) / row_blocks));
  const int chunk = (n + chunks - 1) / chunks;
  const size_t vb = (size_t)n * sizeof(double2);
  DeviceBuffer part((size_t)chunks * vb, s), bv(vb, s), bx(vb, s), by0(vb, s), by1(vb, s),
      by2(vb, s), bu(vb, s), coef((size_t)(2 * max_steps + 2) * sizeof(double), s),
      ea((size_t)std::max(n_omega, 1) * sizeof(double2), s), diff(2 * sizeof(double), s),
      jbuf(sizeof(int), s);
  double2 *V = bv.as<double2>(), *X = bx.as<double2>(), *Y0 = by0.as<double2>(),
          *Y1 = by1.as<double2>(), *Y2 = by2.as<double2>(), *U = bu.as<double2>();
  double* cf = coef.as<double>();
  int* jdev = jbuf.as<int>();
  const int eb = (n + 255) / 256;
  int launches = 0;
  // A+B and A-B formed once (each product then reads one matrix: 4 instead
  // of 6 FP64 FMAs and 16 instead of 32 bytes per element); B = NULL: both A
  std::unique_ptr<DeviceBuffer> pm;
  const double2 *Cp = A2, *Dp = A2;
  int64_t ldp = ld;
  if (B) {
    pm.reset(new DeviceBuffer(2 * (size_t)n * n * sizeof(double2), s));
    k_form_pm<<<sms * 8, 256, 0, s>>>(n, A2, B2, ld, pm->as<double2>(),
                                      pm->as<double2>() + (size_t)n * n);
    ++launches;
    Cp = pm->as<double2>();
    Dp = Cp + (size_t)n * n;
    ldp = n;
  }
  // split-precision products: A+B and A-B split once into BF16 pieces, the
  // products on the tensor cores (the diagonal in FP64), FP64 results
  std::unique_ptr<TcMatvec, void (*)(TcMatvec*)> tcp(nullptr, tc_matvec_destroy);
  std::unique_ptr<TcMatvec, void (*)(TcMatvec*)> tcd(nullptr, tc_matvec_destroy);
  std::unique_ptr<DeviceBuffer> av;
  if (matvec_precision != BSE_PREC_FP64) {
    tcp.reset(tc_matvec_create(n, reinterpret_cast<const bse_c128*>(Cp), nullptr, ldp,
                               matvec_precision, 1, s));
    if (B)
      tcd.reset(tc_matvec_create(n, reinterpret_cast<const bse_c128*>(Dp), nullptr, ldp,
                                 matvec_precision, 1, s));
    av.reset(new DeviceBuffer(vb, s));
  }
  const bool tc = (bool)tcp;
  // out = (A + sign B) x; dot target as for dot_target(dot, jd, off)
  auto gemv = [&](cudaStream_t st, double sign, const double2* x, double2* out, const double2* w,
                  double* dot, const int* jd, int off) {
    if (tc) {
      TcMatvec* m = sign > 0 || !tcd ? tcp.get() : tcd.get();
      tc_matvec_apply(m, reinterpret_cast<const bse_c128*>(x), 1, av->as<bse_c128>(), nullptr, st);
      k_combine_dot<<<eb, 256, 0, st>>>(n, av->as<double2>(), nullptr, 0.0, out, w, dot, jd, off);
      launches += 1;
      return;
    }
    k_pm_gemv<<<dim3(row_blocks, chunks), kGvRows, 0, st>>>(n, sign > 0 ? Cp : Dp, nullptr, ldp,
                                                            0.0, x, chunk, part.as<double2>());
    k_sum_partials<<<eb, 256, 0, st>>>(n, chunks, part.as<double2>(), out, w, dot, jd, off);
    launches += 2;
  };
  // one step on stream st with the current buffer assignment, then rotate
  auto step = [&](cudaStream_t st) {
    gemv(st, +1.0, V, U, V, cf, jdev, 0);                 // u = (A+B) v_j, alpha_j
    k_lanczos_y<<<eb, 256, 0, st>>>(n, U, Y1, Y0, cf, jdev, Y2);
    gemv(st, -1.0, Y2, X, Y2, cf, jdev, 1);               // x = (A-B) y, beta_j^2
    k_lanczos_scale<<<eb, 256, 0, st>>>(n, cf, jdev, 0, X, Y2);
    k_step_inc<<<1, 1, 0, st>>>(jdev);
    launches += 3;
    std::swap(V, X);                                      // v_{j+1}
    double2* t = Y0;                                      // y_{j-1} <- y_j <- y_{j+1}
    Y0 = Y1;
    Y1 = Y2;
    Y2 = t;
  };
  Phase ph("spectrum_lanczos", s);
  BSE_CUDA(cudaMemsetAsync(cf, 0, (size_t)(2 * max_steps + 2) * sizeof(double), s));
  BSE_CUDA(cudaMemsetAsync(Y0, 0, vb, s));
  BSE_CUDA(cudaMemsetAsync(jdev, 0, sizeof(int), s));
  // start: y_0 = conj(rho), v_0 = (A-B) y_0, <v_0, v_0> = y_0^H v_0; the
  // squared norm is kept in the last coefficient slot
  double* nv2_dev = cf + 2 * max_steps + 1;
  k_conj<<<eb, 256, 0, s>>>(n, reinterpret_cast<const double2*>(rho), Y1);
  ++launches;
  gemv(s, -1.0, Y1, X, Y1, nv2_dev, nullptr, 0);
  double nv2 = 0.0;
  BSE_CUDA(cudaMemcpyAsync(&nv2, nv2_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  if (!(nv2 > 0.0)) {
    note_launches(launches);
    throw Error(nv2 == 0.0 ? BSE_ERR_ARG : BSE_ERR_NOT_PD,
                nv2 == 0.0 ? "rho is zero" : "conj(rho)^H (A-B) conj(rho) <= 0: A-B is not positive definite");
  }
  k_lanczos_scale<<<eb, 256, 0, s>>>(n, cf, nullptr, 2 * max_steps + 1, X, Y1);
  ++launches;
  std::swap(V, X);

  // six steps as one graph (FP64 products)
  constexpr int kGraphSteps = 6;
  cudaGraphExec_t exec = nullptr;
  struct GraphGuard {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    cudaStream_t cs = nullptr;
    ~GraphGuard() {
      if (e) cudaGraphExecDestroy(e);
      if (g) cudaGraphDestroy(g);
      if (cs) cudaStreamDestroy(cs);
    }
  } gg;
  if (!tc && max_steps >= kGraphSteps) {
    BSE_CUDA(cudaStreamCreateWithFlags(&gg.cs, cudaStreamNonBlocking));
    BSE_CUDA(cudaStreamBeginCapture(gg.cs, cudaStreamCaptureModeThreadLocal));
    const int l0 = launches;
    for (int q = 0; q < kGraphSteps; ++q) step(gg.cs);   // the rotation returns to the start
    BSE_CUDA(cudaStreamEndCapture(gg.cs, &gg.g));
    BSE_CUDA(cudaGraphInstantiate(&gg.e, gg.g, 0));
    exec = gg.e;
    launches = l0;   // captured, not launched; counted per replay below
  }
  const int per_graph = tc ? 0 : kGraphSteps * 7;
  const double pref = c_q * kHartreeEv * 2.0 / vc;
  // eps is compared every `check` steps; at least min_steps are taken (past
  // n steps the recursion only repeats what the Krylov space already holds)
  const int check = exec ? std::max(kGraphSteps, std::min(48, (n / kGraphSteps) * kGraphSteps))
                         : std::max(10, std::min(50, n));
  const int min_steps = std::min(100, 2 * n);
  int steps = 0;
  bool have_prev = false, converged = false;
  while (steps < max_steps) {
    if (exec && steps + kGraphSteps <= max_steps) {
      BSE_CUDA(cudaGraphLaunch(exec, s));
      launches += per_graph;
      steps += kGraphSteps;
    } else {
      step(s);
      steps += 1;
    }
    if (steps % check == 0 || steps == max_steps) {
      double2* cur = have_prev ? ea.as<double2>() : reinterpret_cast<double2*>(eps_out);
      k_lanczos_eps<<<(n_omega + 127) / 128, 128, 0, s>>>(steps, cf, nv2, n_omega, omega, delta,
                                                          pref, cur);
      ++launches;
      if (have_prev) {
        k_eps_change<<<1, 256, 0, s>>>(n_omega, reinterpret_cast<double2*>(eps_out), cur,
                                       diff.as<double>());
        BSE_CUDA(cudaMemcpyAsync(eps_out, cur, (size_t)n_omega * sizeof(double2),
                                 cudaMemcpyDeviceToDevice, s));
        ++launches;
        double hd[2];
        BSE_CUDA(cudaMemcpyAsync(hd, diff.ptr, sizeof(hd), cudaMemcpyDeviceToHost, s));
        BSE_CUDA(cudaStreamSynchronize(s));
        if (steps >= min_steps && hd[0] <= tol * hd[1]) {
          converged = true;
          break;
        }
      }
      have_prev = true;
    }
  }
  BSE_CUDA(cudaGetLastError());
  note_launches(launches);
  BSE_CUDA(cudaStreamSynchronize(s));
  if (!converged)
    throw Error(BSE_ERR_NO_CONV, "eps changed by more than tol after " + std::to_string(steps) +
                                     " Lanczos steps");
  return steps;
}

}  // namespace bse
