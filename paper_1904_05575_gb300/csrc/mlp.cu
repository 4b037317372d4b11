// Learned preconditioner for the lowest-exciton Davidson solve.
//
// A small network (F features -> 128 -> 128 -> 1, ReLU, FP16 weights, FP32
// arithmetic) predicts, per transition a and target energy E, a factor c that
// rescales the diagonal gain: the preconditioned correction is
//   t_a = c(f_a) r_a / (D_a - E)        c = 1 + y,  y = network output
// with D the diagonal of A+B for the residual of (A+B)(X+Y) = E(X-Y) and of
// A-B for the other.  Two feature sets:
//   F = 4   [D_a - E, D'_a - E, S_a, E / 10]  (D' the other equation's
//           diagonal, S_a the off-diagonal row norm of A)
//   F = 10  [(D_a - E)/10, (D'_a - E)/10, S_a/10, E/100] and, for each of two
//           neighbouring momentum transfers Q_i whose exact X+Y of the same
//           exciton (v_i, unit norm) the caller supplies: |u_a| sqrt(n) and
//           the real and imaginary parts of conj(b_a)(u_a - x_a) sqrt(n)/|b_a|,
//           u = v_i aligned in phase with the current vector x (unit norm, the
//           Ritz X+Y or X-Y this residual corrects), b = r / (D - E).  They
//           tell the network how far, and in which direction relative to the
//           diagonal correction, the current vector is from the neighbours'.
//
// Training data come from Davidson trajectories whose exact pairs are known
// (the dense solve at other momentum transfers): at every iteration the
// residual and the error of the Ritz vector give, per component, the gain
// that maps one onto the other; the network is fitted to those factors by
// weighted least squares with Adam, all in the kernels below (forward,
// backward, update).  The hidden 128 x 128 layer of the forward pass runs on
// the tensor cores (mma.sync m16n8k16, FP16 operands, FP32 accumulation; the
// FP32 activations enter as two FP16 pieces so that the layer keeps FP32
// accuracy with the FP16 weights exact).
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

constexpr int kH = 128;     // hidden width (both layers)
constexpr int kTS = 32;     // samples per tile
constexpr int kFMax = 16;   // feature slots in shared memory
constexpr int kNb = 2;      // neighbouring momentum transfers in the F = 10 features
constexpr float kClamp = 1e-2f;

// parameter offsets: W1 [H][F], b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1]
struct Lay {
  int64_t W1, b1, W2, b2, w3, b3, np;
  __host__ __device__ explicit Lay(int f)
      : W1(0), b1((int64_t)kH * f), W2(b1 + kH), b2(W2 + (int64_t)kH * kH), w3(b2 + kH),
        b3(w3 + kH), np(b3 + 1) {}
};

struct MlpNet {
  int device = 0;
  int nf = 4;
  int64_t np = 0;
  float* master = nullptr;   // FP32 parameters
  __half* wh = nullptr;      // FP16 copies used by every forward pass
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  float* grad = nullptr;
  double* acc = nullptr;     // [0] weighted squared error, [1] weight sum
  int64_t step = 0;
  // neighbouring-Q exact X+Y (caller-owned, F = 10): nbr_count blocks of
  // [n x nev] column-major, and 1 / their column norms (owned)
  const double2* nbr = nullptr;
  int nbr_n = 0, nbr_nev = 0, nbr_count = 0;
  double* nbr_inv = nullptr;
};

namespace {

// splitmix64 (Steele, Lea, Flood 2014), one draw per parameter index
__device__ __forceinline__ uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_init(float* w, __half* wh, int f, uint64_t seed) {
  const Lay L(f);
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= L.np) return;
  const float u = (float)((splitmix(seed ^ (uint64_t)i * 0xD1B54A32D192ED03ull) >> 40) *
                          (1.0 / 16777216.0)) * 2.f - 1.f;   // U(-1, 1)
  float val = 0.f;
  if (i < L.b1) val = u * sqrtf(6.f / (f + kH));              // W1: Glorot uniform
  else if (i < L.W2) val = 0.01f;                            // b1
  else if (i < L.b2) val = u * sqrtf(6.f / (kH + kH));       // W2
  else if (i < L.w3) val = 0.01f;                            // b2
  else if (i < L.b3) val = u * 1e-3f;                        // w3: start at y ~ 0
  w[i] = val;
  wh[i] = __float2half_rn(val);
}

// Rows padded by 8 halves (4 floats): the fragment loads of the tensor-core
// layer then spread over all 32 shared-memory banks.
struct TileSmem {          // dynamic shared memory of the forward / backward kernels
  __half w2t[kH][kH + 8];  // W2 transposed: w2t[i][j] = W2[j][i]
  __half w2n[kH][kH + 8];  // W2 as stored:  w2n[j][i] = W2[j][i]
  float x[kTS][kFMax];
  float h1[kTS][kH + 4];
  float h2[kTS][kH + 4];
  float dz2[kTS][kH];
  float y[kTS];
  float red[4][kTS];
};

__device__ void load_w2(TileSmem& sm, const __half* wh, const Lay& L) {
  for (int idx = threadIdx.x; idx < kH * kH; idx += blockDim.x) {
    const int j = idx / kH, i = idx % kH;
    const __half w = wh[L.W2 + idx];
    sm.w2n[j][i] = w;
    sm.w2t[i][j] = w;
  }
}

// D += A B for one m16n8k16 tile (A row-major 16 x 16, B column-major 16 x 8,
// FP16 operands, FP32 accumulators; fragment layouts of the PTX ISA)
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// two FP32 values -> (hi, lo) FP16 pairs with x ~ hi + lo (lower column in the low half)
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half h0 = __float2half_rn(x0), h1 = __float2half_rn(x1);
  const __half l0 = __float2half_rn(x0 - __half2float(h0));
  const __half l1 = __float2half_rn(x1 - __half2float(h1));
  const __half2 hh = __halves2half2(h0, h1), ll = __halves2half2(l0, l1);
  hi = *reinterpret_cast<const uint32_t*>(&hh);
  lo = *reinterpret_cast<const uint32_t*>(&ll);
}

// Forward pass of one tile: h1, h2 in shared memory, y[s] for s < ns.
// Layer 1 and the output: thread j is hidden unit j.  Layer 2 on the tensor
// cores: warp w computes the hidden units 32w .. 32w+31 of all 32 samples.
template <int F>
__device__ void forward_tile(TileSmem& sm, const __half* wh, const Lay& L, int ns) {
  const int j = threadIdx.x;
  float w1[F];
#pragma unroll
  for (int f = 0; f < F; ++f) w1[f] = __half2float(wh[L.W1 + j * F + f]);
  const float b1 = __half2float(wh[L.b1 + j]);
  for (int s = 0; s < kTS; ++s) {
    float z = b1;
#pragma unroll
    for (int f = 0; f < F; ++f) z = fmaf(w1[f], sm.x[s][f], z);
    sm.h1[s][j] = s < ns ? fmaxf(z, 0.f) : 0.f;
  }
  __syncthreads();
  {
    const int warp = j >> 5, lane = j & 31, g = lane >> 2, t4 = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[mt][nt][c] = 0.f;
#pragma unroll 2
    for (int k0 = 0; k0 < kH; k0 += 16) {
      uint32_t ahi[2][4], alo[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r0 = 16 * mt + g, c0 = k0 + 2 * t4;
        split2(sm.h1[r0][c0], sm.h1[r0][c0 + 1], ahi[mt][0], alo[mt][0]);
        split2(sm.h1[r0 + 8][c0], sm.h1[r0 + 8][c0 + 1], ahi[mt][1], alo[mt][1]);
        split2(sm.h1[r0][c0 + 8], sm.h1[r0][c0 + 9], ahi[mt][2], alo[mt][2]);
        split2(sm.h1[r0 + 8][c0 + 8], sm.h1[r0 + 8][c0 + 9], ahi[mt][3], alo[mt][3]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int nrow = 32 * warp + 8 * nt + g;
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&sm.w2n[nrow][k0 + 2 * t4]);
        const uint32_t b1v = *reinterpret_cast<const uint32_t*>(&sm.w2n[nrow][k0 + 2 * t4 + 8]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma16816(acc[mt][nt], alo[mt], b0, b1v);
          mma16816(acc[mt][nt], ahi[mt], b0, b1v);
        }
      }
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = 32 * warp + 8 * nt + 2 * t4;
      const float bb0 = __half2float(wh[L.b2 + col]), bb1 = __half2float(wh[L.b2 + col + 1]);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r0 = 16 * mt + g;
        sm.h2[r0][col] = fmaxf(acc[mt][nt][0] + bb0, 0.f);
        sm.h2[r0][col + 1] = fmaxf(acc[mt][nt][1] + bb1, 0.f);
        sm.h2[r0 + 8][col] = fmaxf(acc[mt][nt][2] + bb0, 0.f);
        sm.h2[r0 + 8][col + 1] = fmaxf(acc[mt][nt][3] + bb1, 0.f);
      }
    }
  }
  __syncthreads();
  const float w3 = __half2float(wh[L.w3 + j]);
  const int lane = j & 31, warp = j >> 5;
#pragma unroll 4
  for (int s = 0; s < kTS; ++s) {
    float c = sm.h2[s][j] * w3;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) sm.red[warp][s] = c;
  }
  __syncthreads();
  if (j < kTS)
    sm.y[j] = sm.red[0][j] + sm.red[1][j] + sm.red[2][j] + sm.red[3][j] + __half2float(wh[L.b3]);
  __syncthreads();
}

template <int F>
__device__ void load_features(TileSmem& sm, const float* feat, int64_t s0, int ns) {
  for (int idx = threadIdx.x; idx < kTS * F; idx += blockDim.x) {
    const int s = idx / F, f = idx % F;
    sm.x[s][f] = s < ns ? feat[(s0 + s) * F + f] : 0.f;
  }
}

// Loss and gradient over nsamp samples (weights already summing to wsum).
// The backward products run on the CUDA cores in FP32.
template <int F>
__global__ void __launch_bounds__(kH) k_loss_grad(const __half* wh, const float* feat,
                                                  const float* target, const float* weight,
                                                  int64_t nsamp, float wsum, float* grad,
                                                  double* acc) {
  extern __shared__ __align__(16) unsigned char raw[];
  TileSmem& sm = *reinterpret_cast<TileSmem*>(raw);
  const Lay L(F);
  const int j = threadIdx.x;
  load_w2(sm, wh, L);
  const float w3 = __half2float(wh[L.w3 + j]);
  float gw2[kH];
#pragma unroll
  for (int i = 0; i < kH; ++i) gw2[i] = 0.f;
  float gw1[F];
#pragma unroll
  for (int f = 0; f < F; ++f) gw1[f] = 0.f;
  float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f;
  double lsum = 0.0;
  const int64_t ntiles = (nsamp + kTS - 1) / kTS;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t s0 = t * kTS;
    const int ns = (int)((nsamp - s0) < kTS ? (nsamp - s0) : kTS);
    __syncthreads();
    load_features<F>(sm, feat, s0, ns);
    __syncthreads();
    forward_tile<F>(sm, wh, L, ns);
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
      for (int f = 0; f < F; ++f) gw1[f] = fmaf(d, sm.x[s][f], gw1[f]);
    }
  }
  // one atomic per gradient entry per block
#pragma unroll
  for (int i = 0; i < kH; ++i) atomicAdd(&grad[L.W2 + j * kH + i], gw2[i]);
#pragma unroll
  for (int f = 0; f < F; ++f) atomicAdd(&grad[L.W1 + j * F + f], gw1[f]);
  atomicAdd(&grad[L.b1 + j], gb1);
  atomicAdd(&grad[L.b2 + j], gb2);
  atomicAdd(&grad[L.w3 + j], gw3);
  if (j == 0) atomicAdd(&grad[L.b3], gb3);
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
template <int F>
__global__ void __launch_bounds__(kH) k_predict(const __half* wh, const float* feat, int64_t nsamp,
                                                float* out) {
  extern __shared__ __align__(16) unsigned char raw[];
  TileSmem& sm = *reinterpret_cast<TileSmem*>(raw);
  const Lay L(F);
  load_w2(sm, wh, L);
  const int j = threadIdx.x;
  const int64_t ntiles = (nsamp + kTS - 1) / kTS;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t s0 = t * kTS;
    const int ns = (int)((nsamp - s0) < kTS ? (nsamp - s0) : kTS);
    __syncthreads();
    load_features<F>(sm, feat, s0, ns);
    __syncthreads();
    forward_tile<F>(sm, wh, L, ns);
    if (j < ns) out[s0 + j] = 1.f + sm.y[j];
  }
}

__device__ __forceinline__ double clamp_den(double d) {
  return fabs(d) < kClamp ? (d < 0.0 ? -(double)kClamp : (double)kClamp) : d;
}

// Davidson preconditioner: sample s = c n + a (column c, transition a) takes
// t = (1 + y(feat_s)) r / (D_q - E_c); eq[c] = 0 for a residual of the (A+B)
// equation (D_q = D+), 1 for the (A-B) equation
template <int F>
__global__ void __launch_bounds__(kH) k_mlp_apply(const __half* wh, int n, int ncol,
                                                  const float* feat, const int* eq,
                                                  const double* dp, const double* dm,
                                                  const double* theta, const double2* r,
                                                  int64_t ldr, double2* t, int64_t ldt) {
  extern __shared__ __align__(16) unsigned char raw[];
  TileSmem& sm = *reinterpret_cast<TileSmem*>(raw);
  const Lay L(F);
  load_w2(sm, wh, L);
  const int j = threadIdx.x;
  const int64_t nsamp = (int64_t)n * ncol;
  const int64_t ntiles = (nsamp + kTS - 1) / kTS;
  for (int64_t tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
    const int64_t s0 = tt * kTS;
    const int ns = (int)((nsamp - s0) < kTS ? (nsamp - s0) : kTS);
    __syncthreads();
    load_features<F>(sm, feat, s0, ns);
    __syncthreads();
    forward_tile<F>(sm, wh, L, ns);
    if (j < ns) {
      const int64_t sidx = s0 + j;
      const int c = (int)(sidx / n), a = (int)(sidx % n);
      const double den = clamp_den((eq[c] == 0 ? dp[a] : dm[a]) - theta[c]);
      const double g = (1.0 + (double)sm.y[j]) / den;
      const double2 rv = r[a + (int64_t)c * ldr];
      t[a + (int64_t)c * ldt] = make_double2(rv.x * g, rv.y * g);
    }
  }
}

// ---- features -------------------------------------------------------------
// Per column c: xinv[c] = 1/|x_c| and, per neighbour i, the unit phase
// ph[c][i] = z / |z|, z = sum_a conj(u_i,a) x_c,a (u_i = neighbour X+Y of the
// column's exciton, unit norm).  One block per column.
__global__ void __launch_bounds__(256) k_feature_stats(int n, const double2* x, int64_t ldx,
                                                       const int* lam, const double2* nbr,
                                                       const double* nbr_inv, int nbr_nev,
                                                       int nbr_count, double* xinv,
                                                       double2* ph) {
  __shared__ double red[5][256];
  const int c = blockIdx.x;
  const double2* xc = x + (int64_t)c * ldx;
  double xx = 0.0, zr[kNb] = {0.0, 0.0}, zi[kNb] = {0.0, 0.0};
  const int l = lam ? lam[c] : 0;
  for (int a = threadIdx.x; a < n; a += 256) {
    const double2 v = xc[a];
    xx += v.x * v.x + v.y * v.y;
    for (int i = 0; i < nbr_count; ++i) {
      const double2 u = nbr[a + ((int64_t)i * nbr_nev + l) * n];
      zr[i] += u.x * v.x + u.y * v.y;   // conj(u) x
      zi[i] += u.x * v.y - u.y * v.x;
    }
  }
  red[0][threadIdx.x] = xx;
  red[1][threadIdx.x] = zr[0];
  red[2][threadIdx.x] = zi[0];
  red[3][threadIdx.x] = zr[1];
  red[4][threadIdx.x] = zi[1];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    xinv[c] = red[0][0] > 0.0 ? 1.0 / sqrt(red[0][0]) : 0.0;
    for (int i = 0; i < kNb; ++i) {
      const double a = red[1 + 2 * i][0], b = red[2 + 2 * i][0], m = hypot(a, b);
      ph[c * kNb + i] = m > 0.0 ? make_double2(a / m, b / m) : make_double2(1.0, 0.0);
    }
  }
  (void)nbr_inv;
}

// 1 / column norms of the neighbour blocks (one block per column)
__global__ void __launch_bounds__(256) k_col_inv_norms(int n, const double2* v, double* inv) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int a = threadIdx.x; a < n; a += 256) {
    const double2 x = v[a + (int64_t)c * n];
    s += x.x * x.x + x.y * x.y;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) inv[c] = red[0] > 0.0 ? 1.0 / sqrt(red[0]) : 0.0;
}

// features of sample s = c n + a into feat[s][F]
template <int F>
__global__ void k_features(int n, int ncol, const int* eq, const int* lam, const double* theta,
                           const double* dp, const double* dm, const double* srow,
                           const double2* r, int64_t ldr, const double2* x, int64_t ldx,
                           const double* xinv, const double2* ph, const double2* nbr,
                           const double* nbr_inv, int nbr_nev, int nbr_count, float* feat) {
  const int64_t total = (int64_t)n * ncol;
  const double sn = sqrt((double)n);
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < total;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(s / n), a = (int)(s % n);
    const double e = theta[c];
    const bool plus = eq[c] == 0;
    const double dq = plus ? dp[a] : dm[a], dother = plus ? dm[a] : dp[a];
    float* f = feat + s * F;
    if (F == 4) {
      f[0] = (float)(dq - e);
      f[1] = (float)(dother - e);
      f[2] = (float)srow[a];
      f[3] = (float)(e / 10.0);
      continue;
    }
    f[0] = (float)((dq - e) / 10.0);
    f[1] = (float)((dother - e) / 10.0);
    f[2] = (float)(srow[a] / 10.0);
    f[3] = (float)(e / 100.0);
    const double den = clamp_den(dq - e);
    const double2 rv = r[a + (int64_t)c * ldr];
    const double2 b = make_double2(rv.x / den, rv.y / den);
    const double bm = hypot(b.x, b.y);
    const double2 xv = x[a + (int64_t)c * ldx];
    const double xi = xinv[c];
    const int l = lam[c];
    for (int i = 0; i < kNb; ++i) {
      double g0 = 0.0, g1 = 0.0, g2 = 0.0;
      if (i < nbr_count) {
        const double vi = nbr_inv[i * nbr_nev + l];
        const double2 v = nbr[a + ((int64_t)i * nbr_nev + l) * n];
        const double2 p = ph[c * kNb + i];
        // u = v / |v| * ph, d = u - x / |x|, rel = conj(b) d
        const double2 u = make_double2((v.x * p.x - v.y * p.y) * vi, (v.x * p.y + v.y * p.x) * vi);
        const double2 d = make_double2(u.x - xv.x * xi, u.y - xv.y * xi);
        g0 = hypot(u.x, u.y) * sn;
        if (bm > 0.0) {
          g1 = (b.x * d.x + b.y * d.y) / bm * sn;
          g2 = (b.x * d.y - b.y * d.x) / bm * sn;
        }
      }
      f[4 + 3 * i] = (float)g0;
      f[5 + 3 * i] = (float)g1;
      f[6 + 3 * i] = (float)g2;
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
// (the 4-feature set)
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
    const double den = clamp_den(dq - ec);
    const double w = r2 / (den * den);
    target[sidx] = (float)(g * den);
    weight[sidx] = (float)w;
    atomicAdd(&wsum[vec], w);
    feat[sidx * 4 + 0] = (float)(dq - ec);
    feat[sidx * 4 + 1] = (float)(dother - ec);
    feat[sidx * 4 + 2] = (float)srow[a];
    feat[sidx * 4 + 3] = (float)(ec / 10.0);
  }
}

__global__ void k_normalise_weights(int64_t total, int n, float* weight, const double* wsum) {
  for (int64_t sidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sidx < total;
       sidx += (int64_t)gridDim.x * blockDim.x) {
    const double ws = wsum[sidx / n];
    weight[sidx] = ws > 0.0 ? (float)(weight[sidx] / ws) : 0.f;
  }
}

// target c* = Re(conj(r) step)/|r|^2 (D_q - E) and raw weight |r|^2/(D_q - E)^2
__global__ void k_record_targets(int n, const double* dq, double ec, const double2* r,
                                 const double2* step, float* target, float* weight,
                                 double* wsum) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  const double2 rv = r[a], st = step[a];
  const double r2 = rv.x * rv.x + rv.y * rv.y;
  const double g = r2 > 0.0 ? (rv.x * st.x + rv.y * st.y) / r2 : 0.0;
  const double den = clamp_den(dq[a] - ec);
  const double w = r2 / (den * den);
  target[a] = (float)(g * den);
  weight[a] = (float)w;
  atomicAdd(wsum, w);
}

size_t tile_smem() { return sizeof(TileSmem); }

int grid_tiles(int64_t nsamp) {
  int64_t t = (nsamp + kTS - 1) / kTS;
  return (int)(t < 152 * 2 ? (t < 1 ? 1 : t) : 152 * 2);
}

template <int F>
void set_smem_attrs_f() {
  static bool done = false;
  if (done) return;
  BSE_CUDA(cudaFuncSetAttribute(k_loss_grad<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tile_smem()));
  BSE_CUDA(cudaFuncSetAttribute(k_predict<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tile_smem()));
  BSE_CUDA(cudaFuncSetAttribute(k_mlp_apply<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tile_smem()));
  done = true;
}

void set_smem_attrs(int f) {
  if (f == 4) set_smem_attrs_f<4>();
  else set_smem_attrs_f<10>();
}

}  // namespace

// ---------------------------------------------------------------------------
bool mlp_features_supported(int n_features) { return n_features == 4 || n_features == 10; }

MlpNet* mlp_create(int n_features, uint64_t seed) {
  if (!mlp_features_supported(n_features))
    throw Error(BSE_ERR_UNSUPPORTED, "the network takes 4 or 10 features");
  MlpNet* net = new MlpNet;
  BSE_CUDA(cudaGetDevice(&net->device));
  net->nf = n_features;
  net->np = Lay(n_features).np;
  try {
    BSE_CUDA(cudaMalloc(&net->master, net->np * sizeof(float)));
    BSE_CUDA(cudaMalloc(&net->wh, net->np * sizeof(__half)));
    BSE_CUDA(cudaMalloc(&net->m, net->np * sizeof(float)));
    BSE_CUDA(cudaMalloc(&net->v, net->np * sizeof(float)));
    BSE_CUDA(cudaMalloc(&net->grad, net->np * sizeof(float)));
    BSE_CUDA(cudaMalloc(&net->acc, 2 * sizeof(double)));
    BSE_CUDA(cudaMemset(net->m, 0, net->np * sizeof(float)));
    BSE_CUDA(cudaMemset(net->v, 0, net->np * sizeof(float)));
    k_init<<<(int)((net->np + 255) / 256), 256>>>(net->master, net->wh, n_features, seed);
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
  cudaFree(net->nbr_inv);
  delete net;
}

int64_t mlp_num_params(const MlpNet* net) { return net->np; }
int mlp_num_features(const MlpNet* net) { return net ? net->nf : 4; }

void mlp_get_params(const MlpNet* net, float* host) {
  std::vector<__half> h(net->np);
  BSE_CUDA(cudaMemcpy(h.data(), net->wh, net->np * sizeof(__half), cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < net->np; ++i) host[i] = __half2float(h[i]);
}

void mlp_set_params(MlpNet* net, const float* host) {
  std::vector<__half> h(net->np);
  for (int64_t i = 0; i < net->np; ++i) h[i] = __float2half_rn(host[i]);
  BSE_CUDA(cudaMemcpy(net->master, host, net->np * sizeof(float), cudaMemcpyHostToDevice));
  BSE_CUDA(cudaMemcpy(net->wh, h.data(), net->np * sizeof(__half), cudaMemcpyHostToDevice));
  BSE_CUDA(cudaMemset(net->m, 0, net->np * sizeof(float)));
  BSE_CUDA(cudaMemset(net->v, 0, net->np * sizeof(float)));
  net->step = 0;
}

void mlp_set_neighbours(MlpNet* net, int n, int nev, const bse_c128* nbr, int count,
                        cudaStream_t s) {
  cudaFree(net->nbr_inv);
  net->nbr_inv = nullptr;
  net->nbr = nullptr;
  net->nbr_n = net->nbr_nev = net->nbr_count = 0;
  if (!nbr || count == 0) return;
  if (count < 1 || count > kNb) throw Error(BSE_ERR_ARG, "one or two neighbour blocks");
  BSE_CUDA(cudaMalloc(&net->nbr_inv, (size_t)count * nev * sizeof(double)));
  k_col_inv_norms<<<count * nev, 256, 0, s>>>(n, reinterpret_cast<const double2*>(nbr),
                                              net->nbr_inv);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
  net->nbr = reinterpret_cast<const double2*>(nbr);
  net->nbr_n = n;
  net->nbr_nev = nev;
  net->nbr_count = count;
}

void mlp_check_neighbours(const MlpNet* net, int n, int nev) {
  if (net->nf != 10) return;
  if (!net->nbr || net->nbr_n != n || net->nbr_nev < nev)
    throw Error(BSE_ERR_ARG,
                "the 10-feature network needs the neighbours' X+Y (bse_mlp_set_neighbours) "
                "for this n and at least nev excitons");
}

// loss and gradient (device grad buffer); returns the loss
static double loss_grad(MlpNet* net, const float* feat, const float* target, const float* weight,
                        int64_t nsamp, cudaStream_t s, bool want_loss, double wsum_known) {
  set_smem_attrs(net->nf);
  BSE_CUDA(cudaMemsetAsync(net->grad, 0, net->np * sizeof(float), s));
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
  if (net->nf == 4)
    k_loss_grad<4><<<grid_tiles(nsamp), kH, tile_smem(), s>>>(net->wh, feat, target, weight, nsamp,
                                                              (float)wsum, net->grad, net->acc);
  else
    k_loss_grad<10><<<grid_tiles(nsamp), kH, tile_smem(), s>>>(net->wh, feat, target, weight, nsamp,
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
    BSE_CUDA(cudaMemcpy(grad_host, net->grad, net->np * sizeof(float), cudaMemcpyDeviceToHost));
  return L;
}

double mlp_train(MlpNet* net, const float* feat, const float* target, const float* weight,
                 int64_t nsamp, int steps, double lr, cudaStream_t s) {
  // full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8)
  const double wsum = loss_grad(net, feat, target, weight, nsamp, s, false, 0.0);
  for (int it = 0; it < steps; ++it) {
    if (it > 0) loss_grad(net, feat, target, weight, nsamp, s, false, wsum);
    net->step += 1;
    const float c1 = 1.f - powf(0.9f, (float)net->step), c2 = 1.f - powf(0.999f, (float)net->step);
    k_adam<<<(int)((net->np + 255) / 256), 256, 0, s>>>(net->master, net->wh, net->m, net->v,
                                                        net->grad, net->np, (float)lr, 0.9f,
                                                        0.999f, 1e-8f, c1, c2);
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
  }
  return loss_grad(net, feat, target, weight, nsamp, s, true, wsum);
}

void mlp_predict(const MlpNet* net, const float* feat, int64_t nsamp, float* out, cudaStream_t s) {
  set_smem_attrs(net->nf);
  if (net->nf == 4)
    k_predict<4><<<grid_tiles(nsamp), kH, tile_smem(), s>>>(net->wh, feat, nsamp, out);
  else
    k_predict<10><<<grid_tiles(nsamp), kH, tile_smem(), s>>>(net->wh, feat, nsamp, out);
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

void mlp_features(const MlpNet* net, int n, int ncol, const int* eq, const int* lam,
                  const double* theta, const double* dp, const double* dm, const double* srow,
                  const double2* R, int64_t ldr, const double2* X, int64_t ldx, float* feat,
                  cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(((int64_t)n * ncol + 255) / 256, 152 * 8);
  if (mlp_num_features(net) == 4) {
    k_features<4><<<blocks, 256, 0, s>>>(n, ncol, eq, lam, theta, dp, dm, srow, R, ldr, X, ldx,
                                         nullptr, nullptr, nullptr, nullptr, 0, 0, feat);
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
    return;
  }
  mlp_check_neighbours(net, n, 1);
  DeviceBuffer xinv((size_t)ncol * 8, s), ph((size_t)ncol * kNb * 16, s);
  k_feature_stats<<<ncol, 256, 0, s>>>(n, X, ldx, lam, net->nbr, net->nbr_inv, net->nbr_nev,
                                       net->nbr_count, xinv.as<double>(), ph.as<double2>());
  k_features<10><<<blocks, 256, 0, s>>>(n, ncol, eq, lam, theta, dp, dm, srow, R, ldr, X, ldx,
                                        xinv.as<double>(), ph.as<double2>(), net->nbr,
                                        net->nbr_inv, net->nbr_nev, net->nbr_count, feat);
  BSE_CUDA(cudaGetLastError());
  note_launches(2);
}

void mlp_precondition(const MlpNet* net, int n, int ncol, const int* eq, const int* lam,
                      const double* dp, const double* dm, const double* srow, const double* theta,
                      const double2* R, int64_t ldr, const double2* X, int64_t ldx, float* feat,
                      double2* T, int64_t ldt, cudaStream_t s) {
  set_smem_attrs(net->nf);
  mlp_features(net, n, ncol, eq, lam, theta, dp, dm, srow, R, ldr, X, ldx, feat, s);
  const int64_t nsamp = (int64_t)n * ncol;
  if (net->nf == 4)
    k_mlp_apply<4><<<grid_tiles(nsamp), kH, tile_smem(), s>>>(net->wh, n, ncol, feat, eq, dp, dm,
                                                              theta, R, ldr, T, ldt);
  else
    k_mlp_apply<10><<<grid_tiles(nsamp), kH, tile_smem(), s>>>(net->wh, n, ncol, feat, eq, dp, dm,
                                                               theta, R, ldr, T, ldt);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
}

void mlp_record(const MlpNet* net, int n, const double* dp, const double* dm, const double* srow,
                double E, int lam, bool plus, const double2* r, const double2* x,
                const double2* step, float* feat, float* target, float* weight, cudaStream_t s) {
  DeviceBuffer wsum(sizeof(double), s), cols(2 * sizeof(int) + sizeof(double), s);
  struct {
    int eq, lam;
    double theta;
  } hc{plus ? 0 : 1, lam, E};
  static_assert(sizeof(hc) == 2 * sizeof(int) + sizeof(double), "column record layout");
  BSE_CUDA(cudaMemcpyAsync(cols.ptr, &hc, sizeof(hc), cudaMemcpyHostToDevice, s));
  const int* eq = reinterpret_cast<const int*>(cols.ptr);
  const double* th = reinterpret_cast<const double*>(static_cast<char*>(cols.ptr) + 2 * sizeof(int));
  mlp_features(net, n, 1, eq, eq + 1, th, dp, dm, srow, r, n, x, n, feat, s);
  BSE_CUDA(cudaMemsetAsync(wsum.ptr, 0, sizeof(double), s));
  k_record_targets<<<(n + 255) / 256, 256, 0, s>>>(n, plus ? dp : dm, E, r, step, target, weight,
                                                   wsum.as<double>());
  k_normalise_weights<<<(n + 255) / 256, 256, 0, s>>>(n, n, weight, wsum.as<double>());
  BSE_CUDA(cudaGetLastError());
  note_launches(2);
  BSE_CUDA(cudaStreamSynchronize(s));   // the column record leaves scope
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
