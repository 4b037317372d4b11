// Learned preconditioner for the lowest-exciton Davidson solve.
//
// A small network (4 features -> 128 -> 128 -> 1, ReLU, FP16 weights, FP32
// arithmetic) predicts, per transition a and target energy E, a factor c that
// rescales the diagonal gain: the preconditioned correction is
//   t_a = c(f_a) r_a / (D_a - E)        c = 1 + y,  y = network output
// with D the diagonal of A+B for the residual of (A+B)(X+Y) = E(X-Y) and of
// A-B for the other.  Features f_a = [D_a - E, D'_a - E, S_a, E / 10] (D' the
// other equation's diagonal, S_a the off-diagonal row norm of A).
//
// Training data come from exact eigenpairs (the dense solve at other momentum
// transfers): perturbing X+Y and X-Y by eps p gives residuals whose best
// per-component gain onto the perturbation is known (bse_mlp_samples); the
// network is fitted to those factors by weighted least squares with Adam,
// all in the kernels below (forward, backward, update).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bse_internal.h"
#include "mlp.h"
#include "zgemm.cuh"

namespace bse {

constexpr int kF = 4;      // features
constexpr int kH = 128;    // hidden width (both layers)
constexpr int kTS = 32;    // samples per tile
constexpr float kClamp = 1e-2f;

struct MlpNet {
  int device = 0;
  int64_t np = 0;
  float* master = nullptr;   // FP32 parameters: W1 [H][F], b1, W2 [H][H], b2, w3, b3
  __half* wh = nullptr;      // FP16 copies used by every forward pass
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  float* grad = nullptr;
  double* acc = nullptr;     // [0] weighted squared error, [1] weight sum
  int64_t step = 0;
};

namespace {

constexpr int64_t oW1 = 0, ob1 = oW1 + kH * kF, oW2 = ob1 + kH, ob2 = oW2 + kH * kH,
                  ow3 = ob2 + kH, ob3 = ow3 + kH, kNP = ob3 + 1;

// splitmix64 (Steele, Lea, Flood 2014), one draw per parameter index
__device__ __forceinline__ uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_init(float* w, __half* wh, int64_t np, uint64_t seed) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float u = (float)((splitmix(seed ^ (uint64_t)i * 0xD1B54A32D192ED03ull) >> 40) *
                          (1.0 / 16777216.0)) * 2.f - 1.f;   // U(-1, 1)
  float val = 0.f;
  if (i < ob1) val = u * sqrtf(6.f / (kF + kH));             // W1: Glorot uniform
  else if (i < oW2) val = 0.01f;                             // b1
  else if (i < ob2) val = u * sqrtf(6.f / (kH + kH));        // W2
  else if (i < ow3) val = 0.01f;                             // b2
  else if (i < ob3) val = u * 1e-3f;                         // w3: start at y ~ 0
  w[i] = val;
  wh[i] = __float2half_rn(val);
}

struct TileSmem {          // dynamic shared memory of the forward / backward kernels
  __half w2t[kH][kH];      // W2 transposed: w2t[i][j] = W2[j][i]
  __half w2n[kH][kH];      // W2 as stored:  w2n[j][i] = W2[j][i]
  float x[kTS][kF];
  float h1[kTS][kH];
  float h2[kTS][kH];
  float dz2[kTS][kH];
  float y[kTS];
  float red[4][kTS];
};

__device__ void load_w2(TileSmem& sm, const __half* wh) {
  for (int idx = threadIdx.x; idx < kH * kH; idx += blockDim.x) {
    const int j = idx / kH, i = idx % kH;
    const __half w = wh[oW2 + idx];
    sm.w2n[j][i] = w;
    sm.w2t[i][j] = w;
  }
}

// Forward pass of one tile: h1, h2 in shared memory, y[s] for s < ns.
// Thread j is hidden unit j of both layers.
__device__ void forward_tile(TileSmem& sm, const __half* wh, int ns) {
  const int j = threadIdx.x;
  float w1[kF];
#pragma unroll
  for (int f = 0; f < kF; ++f) w1[f] = __half2float(wh[oW1 + j * kF + f]);
  const float b1 = __half2float(wh[ob1 + j]), b2 = __half2float(wh[ob2 + j]);
  const float w3 = __half2float(wh[ow3 + j]);
  for (int s = 0; s < kTS; ++s) {
    float z = b1;
#pragma unroll
    for (int f = 0; f < kF; ++f) z = fmaf(w1[f], sm.x[s][f], z);
    sm.h1[s][j] = s < ns ? fmaxf(z, 0.f) : 0.f;
  }
  __syncthreads();
  float acc[kTS];
#pragma unroll
  for (int s = 0; s < kTS; ++s) acc[s] = b2;
  for (int i = 0; i < kH; ++i) {
    const float w = __half2float(sm.w2t[i][j]);
#pragma unroll
    for (int s = 0; s < kTS; ++s) acc[s] = fmaf(w, sm.h1[s][i], acc[s]);
  }
  const int lane = j & 31, warp = j >> 5;
#pragma unroll
  for (int s = 0; s < kTS; ++s) {
    const float h = fmaxf(acc[s], 0.f);
    sm.h2[s][j] = h;
    float c = h * w3;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) sm.red[warp][s] = c;
  }
  __syncthreads();
  if (j < kTS)
    sm.y[j] = sm.red[0][j] + sm.red[1][j] + sm.red[2][j] + sm.red[3][j] +
              __half2float(wh[ob3]);
  __syncthreads();
}

// Loss and gradient over nsamp samples (weights already summing to wsum).
__global__ void __launch_bounds__(kH) k_loss_grad(const __half* wh, const float* feat,
                                                  const float* target, const float* weight,
                                                  int64_t nsamp, float wsum, float* grad,
                                                  double* acc) {
  extern __shared__ __align__(16) unsigned char raw[];
  TileSmem& sm = *reinterpret_cast<TileSmem*>(raw);
  const int j = threadIdx.x;
  load_w2(sm, wh);
  const float w3 = __half2float(wh[ow3 + j]);
  float gw2[kH];
#pragma unroll
  for (int i = 0; i < kH; ++i) gw2[i] = 0.f;
  float gw1[kF] = {0.f, 0.f, 0.f, 0.f};
  float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f;
  double lsum = 0.0;
  const int64_t ntiles = (nsamp + kTS - 1) / kTS;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t s0 = t * kTS;
    const int ns = (int)((nsamp - s0) < kTS ? (nsamp - s0) : kTS);
    __syncthreads();
    for (int idx = j; idx < kTS * kF; idx += kH) {
      const int s = idx / kF, f = idx % kF;
      sm.x[s][f] = s < ns ? feat[(s0 + s) * kF + f] : 0.f;
    }
    __syncthreads();
    forward_tile(sm, wh, ns);
    // dL/dy per sample (thread s < kTS), kept in sm.y
    if (j < kTS) {
      float dy = 0.f;
      if (j < ns) {
        const float r = 1.f + sm.y[j] - target[s0 + j];
        const float w = weight[s0 + j];
        lsum += (double)w * r * r;
        dy = 2.f * w * r / wsum;
      }
      sm.y[j] = dy;
    }
    __syncthreads();
    for (int s = 0; s < kTS; ++s) {
      const float dy = sm.y[s];
      const float h = sm.h2[s][j];
      gw3 = fmaf(dy, h, gw3);
      const float d = h > 0.f ? dy * w3 : 0.f;
      sm.dz2[s][j] = d;
      gb2 += d;
      if (j == 0) gb3 += dy;
    }
    __syncthreads();
    // gW2[j][i] += sum_s dz2[s][j] h1[s][i]
    for (int s = 0; s < kTS; ++s) {
      const float d = sm.dz2[s][j];
#pragma unroll
      for (int i = 0; i < kH; ++i) gw2[i] = fmaf(d, sm.h1[s][i], gw2[i]);
    }
    // dz1[s][i] with i = j: sum_k W2[k][j] dz2[s][k], masked by h1 > 0
    float dz1[kTS];
#pragma unroll
    for (int s = 0; s < kTS; ++s) dz1[s] = 0.f;
    for (int k = 0; k < kH; ++k) {
      const float w = __half2float(sm.w2n[k][j]);
#pragma unroll
      for (int s = 0; s < kTS; ++s) dz1[s] = fmaf(w, sm.dz2[s][k], dz1[s]);
    }
#pragma unroll
    for (int s = 0; s < kTS; ++s) {
      const float d = sm.h1[s][j] > 0.f ? dz1[s] : 0.f;
      gb1 += d;
#pragma unroll
      for (int f = 0; f < kF; ++f) gw1[f] = fmaf(d, sm.x[s][f], gw1[f]);
    }
  }
  // one atomic per gradient entry per block
#pragma unroll
  for (int i = 0; i < kH; ++i) atomicAdd(&grad[oW2 + j * kH + i], gw2[i]);
#pragma unroll
  for (int f = 0; f < kF; ++f) atomicAdd(&grad[oW1 + j * kF + f], gw1[f]);
  atomicAdd(&grad[ob1 + j], gb1);
  atomicAdd(&grad[ob2 + j], gb2);
  atomicAdd(&grad[ow3 + j], gw3);
  if (j == 0) atomicAdd(&grad[ob3], gb3);
  // loss numerator: partial sums per thread (threads < kTS hold them)
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (j == 0) atomicAdd(&acc[0], lsum);
}

__global__ void k_weight_sum(const float* w, int64_t n, double* acc) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += w[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&acc[1], s);
}

__global__ void k_adam(float* w, __half* wh, float* m, float* v, const float* g, int64_t np,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float nw = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = nw;
  wh[i] = __float2half_rn(nw);
}

// factor c = 1 + y for nsamp feature rows
__global__ void __launch_bounds__(kH) k_predict(const __half* wh, const float* feat, int64_t nsamp,
                                                float* out) {
  extern __shared__ __align__(16) unsigned char raw[];
  TileSmem& sm = *reinterpret_cast<TileSmem*>(raw);
  load_w2(sm, wh);
  const int j = threadIdx.x;
  const int64_t ntiles = (nsamp + kTS - 1) / kTS;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t s0 = t * kTS;
    const int ns = (int)((nsamp - s0) < kTS ? (nsamp - s0) : kTS);
    __syncthreads();
    for (int idx = j; idx < kTS * kF; idx += kH) {
      const int s = idx / kF, f = idx % kF;
      sm.x[s][f] = s < ns ? feat[(s0 + s) * kF + f] : 0.f;
    }
    __syncthreads();
    forward_tile(sm, wh, ns);
    if (j < ns) out[s0 + j] = 1.f + sm.y[j];
  }
}

__device__ __forceinline__ float clamp_den(float d) {
  return fabsf(d) < kClamp ? (d < 0.f ? -kClamp : kClamp) : d;
}

// Davidson preconditioner: sample (a, column c) with c < k/2 the (A+B)
// residual and c >= k/2 the (A-B) residual of eigenvalue e[c]
__global__ void __launch_bounds__(kH) k_mlp_precond(const __half* wh, int n, int k,
                                                    const double* dp, const double* dm,
                                                    const double* srow, const double* e,
                                                    const double2* r, int64_t ldr, double2* t,
                                                    int64_t ldt) {
  extern __shared__ __align__(16) unsigned char raw[];
  TileSmem& sm = *reinterpret_cast<TileSmem*>(raw);
  load_w2(sm, wh);
  const int j = threadIdx.x;
  const int64_t nsamp = (int64_t)n * k;
  const int64_t ntiles = (nsamp + kTS - 1) / kTS;
  const int half_k = k / 2;
  for (int64_t tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
    const int64_t s0 = tt * kTS;
    const int ns = (int)((nsamp - s0) < kTS ? (nsamp - s0) : kTS);
    __syncthreads();
    if (j < kTS) {
      float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
      if (j < ns) {
        const int64_t sidx = s0 + j;
        const int c = (int)(sidx / n), a = (int)(sidx % n);
        const double ec = e[c];
        const bool plus = c < half_k;
        f0 = (float)((plus ? dp[a] : dm[a]) - ec);
        f1 = (float)((plus ? dm[a] : dp[a]) - ec);
        f2 = (float)srow[a];
        f3 = (float)(ec / 10.0);
      }
      sm.x[j][0] = f0;
      sm.x[j][1] = f1;
      sm.x[j][2] = f2;
      sm.x[j][3] = f3;
    }
    __syncthreads();
    forward_tile(sm, wh, ns);
    if (j < ns) {
      const int64_t sidx = s0 + j;
      const int c = (int)(sidx / n), a = (int)(sidx % n);
      const float g = (1.f + sm.y[j]) / clamp_den(sm.x[j][0]);
      const double2 rv = r[a + (int64_t)c * ldr];
      t[a + (int64_t)c * ldt] = make_double2(rv.x * g, rv.y * g);
    }
  }
}

// ---- training samples -------------------------------------------------------
__global__ void k_diag_pm(int n, const double2* A, const double2* B, int64_t ld, double* dp,
                          double* dm) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) {
    const double x = A[a + (int64_t)a * ld].x, y = B ? B[a + (int64_t)a * ld].x : 0.0;
    dp[a] = x + y;
    dm[a] = x - y;
  }
}

// off-diagonal row norms of Hermitian A (= column norms): one warp per column
__global__ void k_offdiag_norm(int n, const double2* A, int64_t ld, double* s) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= n) return;
  double acc = 0.0;
  for (int i = lane; i < n; i += 32) {
    if (i == w) continue;
    const double2 v = A[i + (int64_t)w * ld];
    acc += v.x * v.x + v.y * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) s[w] = sqrt(acc);
}

// xm = (AX + BX)/E; t+ = x+ + eps p; t- = xm + eps p (column-major n x nev)
__global__ void k_perturb(int n, int nev, const double2* xp, const double2* ax, const double2* bx,
                          const double* e, const double2* p, double eps, double2* tp,
                          double2* tm) {
  const int64_t total = (int64_t)n * nev;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / n);
    const double2 a = ax[i], b = bx ? bx[i] : make_double2(0.0, 0.0);
    const double ie = 1.0 / e[c];
    const double2 xm = make_double2((a.x + b.x) * ie, (a.y + b.y) * ie);
    tp[i] = make_double2(xp[i].x + eps * p[i].x, xp[i].y + eps * p[i].y);
    tm[i] = make_double2(xm.x + eps * p[i].x, xm.y + eps * p[i].y);
  }
}

// r+ = (At+ + Bt+) - E t-, r- = (At- - Bt-) - E t+; targets and raw weights
__global__ void k_sample_targets(int n, int nev, const double2* atp, const double2* btp,
                                 const double2* atm, const double2* btm, const double2* tp,
                                 const double2* tm, const double* e, const double2* p, double eps,
                                 const double* dp, const double* dm, const double* srow,
                                 float* feat, float* target, float* weight, double* wsum) {
  const int64_t total = (int64_t)n * nev * 2;
  for (int64_t sidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sidx < total;
       sidx += (int64_t)gridDim.x * blockDim.x) {
    const int vec = (int)(sidx / n), a = (int)(sidx % n);
    const int lam = vec / 2;
    const bool plus = (vec % 2) == 0;
    const int64_t i = (int64_t)lam * n + a;
    const double ec = e[lam];
    double2 r;
    if (plus) {
      const double2 x = atp[i], y = btp ? btp[i] : make_double2(0.0, 0.0);
      r = make_double2(x.x + y.x - ec * tm[i].x, x.y + y.y - ec * tm[i].y);
    } else {
      const double2 x = atm[i], y = btm ? btm[i] : make_double2(0.0, 0.0);
      r = make_double2(x.x - y.x - ec * tp[i].x, x.y - y.y - ec * tp[i].y);
    }
    const double2 step = make_double2(eps * p[i].x, eps * p[i].y);
    const double r2 = r.x * r.x + r.y * r.y;
    const double g = r2 > 0.0 ? (r.x * step.x + r.y * step.y) / r2 : 0.0;
    const double dq = plus ? dp[a] : dm[a], dother = plus ? dm[a] : dp[a];
    double den = dq - ec;
    if (fabs(den) < kClamp) den = den < 0 ? -kClamp : kClamp;
    const double w = r2 / (den * den);
    target[sidx] = (float)(g * den);
    weight[sidx] = (float)w;
    atomicAdd(&wsum[vec], w);
    feat[sidx * kF + 0] = (float)(dq - ec);
    feat[sidx * kF + 1] = (float)(dother - ec);
    feat[sidx * kF + 2] = (float)srow[a];
    feat[sidx * kF + 3] = (float)(ec / 10.0);
  }
}

__global__ void k_normalise_weights(int64_t total, int n, float* weight, const double* wsum) {
  for (int64_t sidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sidx < total;
       sidx += (int64_t)gridDim.x * blockDim.x) {
    const double ws = wsum[sidx / n];
    weight[sidx] = ws > 0.0 ? (float)(weight[sidx] / ws) : 0.f;
  }
}

__global__ void k_record(int n, const double* dp, const double* dm, const double* srow, double ec,
                         int plus, const double2* r, const double2* step, float* feat,
                         float* target, float* weight, double* wsum) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  const double2 rv = r[a], st = step[a];
  const double r2 = rv.x * rv.x + rv.y * rv.y;
  const double g = r2 > 0.0 ? (rv.x * st.x + rv.y * st.y) / r2 : 0.0;
  const double dq = plus ? dp[a] : dm[a], dother = plus ? dm[a] : dp[a];
  double den = dq - ec;
  if (fabs(den) < kClamp) den = den < 0 ? -kClamp : kClamp;
  const double w = r2 / (den * den);
  target[a] = (float)(g * den);
  weight[a] = (float)w;
  atomicAdd(wsum, w);
  feat[a * kF + 0] = (float)(dq - ec);
  feat[a * kF + 1] = (float)(dother - ec);
  feat[a * kF + 2] = (float)srow[a];
  feat[a * kF + 3] = (float)(ec / 10.0);
}

size_t tile_smem() { return sizeof(TileSmem); }

int grid_tiles(int64_t nsamp) {
  int64_t t = (nsamp + kTS - 1) / kTS;
  return (int)(t < 152 * 2 ? (t < 1 ? 1 : t) : 152 * 2);
}

void set_smem_attrs() {
  static bool done = false;
  if (done) return;
  BSE_CUDA(cudaFuncSetAttribute(k_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tile_smem()));
  BSE_CUDA(cudaFuncSetAttribute(k_predict, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tile_smem()));
  BSE_CUDA(cudaFuncSetAttribute(k_mlp_precond, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tile_smem()));
  done = true;
}

}  // namespace

// ---------------------------------------------------------------------------
MlpNet* mlp_create(uint64_t seed) {
  MlpNet* net = new MlpNet;
  BSE_CUDA(cudaGetDevice(&net->device));
  net->np = kNP;
  try {
    BSE_CUDA(cudaMalloc(&net->master, kNP * sizeof(float)));
    BSE_CUDA(cudaMalloc(&net->wh, kNP * sizeof(__half)));
    BSE_CUDA(cudaMalloc(&net->m, kNP * sizeof(float)));
    BSE_CUDA(cudaMalloc(&net->v, kNP * sizeof(float)));
    BSE_CUDA(cudaMalloc(&net->grad, kNP * sizeof(float)));
    BSE_CUDA(cudaMalloc(&net->acc, 2 * sizeof(double)));
    BSE_CUDA(cudaMemset(net->m, 0, kNP * sizeof(float)));
    BSE_CUDA(cudaMemset(net->v, 0, kNP * sizeof(float)));
    k_init<<<(int)((kNP + 255) / 256), 256>>>(net->master, net->wh, kNP, seed);
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
    BSE_CUDA(cudaDeviceSynchronize());
  } catch (...) {
    mlp_destroy(net);
    throw;
  }
  return net;
}

void mlp_destroy(MlpNet* net) {
  if (!net) return;
  cudaFree(net->master);
  cudaFree(net->wh);
  cudaFree(net->m);
  cudaFree(net->v);
  cudaFree(net->grad);
  cudaFree(net->acc);
  delete net;
}

int64_t mlp_num_params(const MlpNet*) { return kNP; }

void mlp_get_params(const MlpNet* net, float* host) {
  std::vector<__half> h(kNP);
  BSE_CUDA(cudaMemcpy(h.data(), net->wh, kNP * sizeof(__half), cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < kNP; ++i) host[i] = __half2float(h[i]);
}

void mlp_set_params(MlpNet* net, const float* host) {
  std::vector<__half> h(kNP);
  for (int64_t i = 0; i < kNP; ++i) h[i] = __float2half_rn(host[i]);
  BSE_CUDA(cudaMemcpy(net->master, host, kNP * sizeof(float), cudaMemcpyHostToDevice));
  BSE_CUDA(cudaMemcpy(net->wh, h.data(), kNP * sizeof(__half), cudaMemcpyHostToDevice));
  BSE_CUDA(cudaMemset(net->m, 0, kNP * sizeof(float)));
  BSE_CUDA(cudaMemset(net->v, 0, kNP * sizeof(float)));
  net->step = 0;
}

// loss and gradient (device grad buffer); returns the loss
static double loss_grad(MlpNet* net, const float* feat, const float* target, const float* weight,
                        int64_t nsamp, cudaStream_t s, bool want_loss, double wsum_known) {
  set_smem_attrs();
  BSE_CUDA(cudaMemsetAsync(net->grad, 0, kNP * sizeof(float), s));
  BSE_CUDA(cudaMemsetAsync(net->acc, 0, 2 * sizeof(double), s));
  double wsum = wsum_known;
  if (wsum <= 0.0) {
    k_weight_sum<<<152, 256, 0, s>>>(weight, nsamp, net->acc);
    note_launches(1);
    double hacc[2];
    BSE_CUDA(cudaMemcpyAsync(hacc, net->acc, sizeof(hacc), cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaStreamSynchronize(s));
    wsum = hacc[1];
    if (!(wsum > 0.0)) throw Error(BSE_ERR_ARG, "sample weights sum to zero");
    BSE_CUDA(cudaMemsetAsync(net->acc, 0, 2 * sizeof(double), s));
  }
  k_loss_grad<<<grid_tiles(nsamp), kH, tile_smem(), s>>>(net->wh, feat, target, weight, nsamp,
                                                         (float)wsum, net->grad, net->acc);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
  if (!want_loss) return wsum;
  double hacc[2];
  BSE_CUDA(cudaMemcpyAsync(hacc, net->acc, sizeof(hacc), cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  return hacc[0] / wsum;
}

double mlp_loss_grad(MlpNet* net, const float* feat, const float* target, const float* weight,
                     int64_t nsamp, float* grad_host, cudaStream_t s) {
  const double L = loss_grad(net, feat, target, weight, nsamp, s, true, 0.0);
  if (grad_host)
    BSE_CUDA(cudaMemcpy(grad_host, net->grad, kNP * sizeof(float), cudaMemcpyDeviceToHost));
  return L;
}

double mlp_train(MlpNet* net, const float* feat, const float* target, const float* weight,
                 int64_t nsamp, int steps, double lr, cudaStream_t s) {
  // full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8)
  const double wsum = loss_grad(net, feat, target, weight, nsamp, s, false, 0.0);
  double L = 0.0;
  for (int it = 0; it < steps; ++it) {
    if (it > 0) loss_grad(net, feat, target, weight, nsamp, s, false, wsum);
    net->step += 1;
    const float c1 = 1.f - powf(0.9f, (float)net->step), c2 = 1.f - powf(0.999f, (float)net->step);
    k_adam<<<(int)((kNP + 255) / 256), 256, 0, s>>>(net->master, net->wh, net->m, net->v,
                                                    net->grad, kNP, (float)lr, 0.9f, 0.999f,
                                                    1e-8f, c1, c2);
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
  }
  L = loss_grad(net, feat, target, weight, nsamp, s, true, wsum);
  return L;
}

void mlp_predict(const MlpNet* net, const float* feat, int64_t nsamp, float* out, cudaStream_t s) {
  set_smem_attrs();
  k_predict<<<grid_tiles(nsamp), kH, tile_smem(), s>>>(net->wh, feat, nsamp, out);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
}

void mlp_samples(int n, const bse_c128* A, const bse_c128* B, int64_t ld, int nev,
                 const double* E, const bse_c128* xpy, const bse_c128* noise, double eps,
                 float* feat, float* target, float* weight, cudaStream_t s) {
  const int64_t nn = (int64_t)n * nev;
  DeviceBuffer dp(n * 8, s), dm(n * 8, s), sr(n * 8, s), ax(nn * 16, s), bx(nn * 16, s),
      tp(nn * 16, s), tm(nn * 16, s), atp(nn * 16, s), btp(nn * 16, s), atm(nn * 16, s),
      btm(nn * 16, s), wsum(2 * nev * 8, s);
  const double2* A2 = reinterpret_cast<const double2*>(A);
  const double2* B2 = reinterpret_cast<const double2*>(B);
  k_diag_pm<<<(n + 255) / 256, 256, 0, s>>>(n, A2, B2, ld, dp.as<double>(), dm.as<double>());
  k_offdiag_norm<<<(n + 7) / 8, 256, 0, s>>>(n, A2, ld, sr.as<double>());
  note_launches(2);
  auto matvec = [&](const bse_c128* H, const void* V, void* out) {
    MatvecProb pr{n, nev, n, H, ld, static_cast<const bse_c128*>(V), n,
                  static_cast<bse_c128*>(out), n};
    launch_zgemm(pr, 1, s);
  };
  matvec(A, xpy, ax.ptr);
  if (B) matvec(B, xpy, bx.ptr);
  const int blocks = (int)std::min<int64_t>((nn + 255) / 256, 152 * 8);
  k_perturb<<<blocks, 256, 0, s>>>(n, nev, reinterpret_cast<const double2*>(xpy), ax.as<double2>(),
                                   B ? bx.as<double2>() : nullptr, E,
                                   reinterpret_cast<const double2*>(noise), eps, tp.as<double2>(),
                                   tm.as<double2>());
  note_launches(1);
  matvec(A, tp.ptr, atp.ptr);
  matvec(A, tm.ptr, atm.ptr);
  if (B) {
    matvec(B, tp.ptr, btp.ptr);
    matvec(B, tm.ptr, btm.ptr);
  }
  BSE_CUDA(cudaMemsetAsync(wsum.ptr, 0, 2 * nev * 8, s));
  k_sample_targets<<<(int)std::min<int64_t>((2 * nn + 255) / 256, 152 * 8), 256, 0, s>>>(
      n, nev, atp.as<double2>(), B ? btp.as<double2>() : nullptr, atm.as<double2>(),
      B ? btm.as<double2>() : nullptr, tp.as<double2>(), tm.as<double2>(), E,
      reinterpret_cast<const double2*>(noise), eps, dp.as<double>(), dm.as<double>(),
      sr.as<double>(), feat, target, weight, wsum.as<double>());
  k_normalise_weights<<<(int)std::min<int64_t>((2 * nn + 255) / 256, 152 * 8), 256, 0, s>>>(
      2 * nn, n, weight, wsum.as<double>());
  BSE_CUDA(cudaGetLastError());
  note_launches(2);
}

void mlp_precondition(const MlpNet* net, int n, int k, const double* dp, const double* dm,
                      const double* srow, const double* E, const double2* R, int64_t ldr,
                      double2* T, int64_t ldt, cudaStream_t s) {
  set_smem_attrs();
  const int64_t nsamp = (int64_t)n * k;
  k_mlp_precond<<<grid_tiles(nsamp), kH, tile_smem(), s>>>(net->wh, n, k, dp, dm, srow, E, R, ldr,
                                                           T, ldt);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
}

void mlp_record(int n, const double* dp, const double* dm, const double* srow, double E,
                bool plus, const double2* r, const double2* step, float* feat, float* target,
                float* weight, cudaStream_t s) {
  DeviceBuffer wsum(sizeof(double), s);
  BSE_CUDA(cudaMemsetAsync(wsum.ptr, 0, sizeof(double), s));
  k_record<<<(n + 255) / 256, 256, 0, s>>>(n, dp, dm, srow, E, plus ? 1 : 0, r, step, feat,
                                            target, weight, wsum.as<double>());
  k_normalise_weights<<<(n + 255) / 256, 256, 0, s>>>(n, n, weight, wsum.as<double>());
  BSE_CUDA(cudaGetLastError());
  note_launches(2);
}

void mlp_diag_features(int n, const bse_c128* A, const bse_c128* B, int64_t ld, double* dp,
                       double* dm, double* srow, cudaStream_t s) {
  const double2* A2 = reinterpret_cast<const double2*>(A);
  k_diag_pm<<<(n + 255) / 256, 256, 0, s>>>(n, A2, reinterpret_cast<const double2*>(B), ld, dp, dm);
  k_offdiag_norm<<<(n + 7) / 8, 256, 0, s>>>(n, A2, ld, srow);
  BSE_CUDA(cudaGetLastError());
  note_launches(2);
}

}  // namespace bse
