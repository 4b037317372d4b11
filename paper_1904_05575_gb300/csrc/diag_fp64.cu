// Exact FP64 diagonal of A and B, recomputed after a split-precision build.
//
// At alpha = alpha' = (k v c) the terms of Eqs. vrrofM, wrrm and wrabar are
//   V_aa    = kappa sum_G vbar_G |M_x[a][G]|^2
//   W^rr_aa = kappa sum_GG' conj(m_vv[k][k][v][v][G]) W(q-(k,k))[G][G'] m_cc[k][k][c][c][G']
//   W^ra_aa = kappa sum_GG' conj(n_vc[k][k][v][c][G]) W(q+(k,k))[G][G'] n_vc[k][k][v][c][G']
// (the diagonal (k, k) pair block of each direct term).  Per k block one
// FP64 GEMM applies W to the block's vectors (U = W Z, Z the nc vectors
// m_cc[k][k][c][c] and the nv nc vectors n_vc[k][k][v][c]), then one warp
// per transition reduces the plane-wave sums in FP64 and overwrites
//   A_aa = E^ip_a + 2 gamma_x V_aa - gamma_c W^rr_aa   (Eq. diagonalblock)
//   B_aa = 2 gamma_x V_aa - gamma_c W^ra_aa            (Eq. couplingblock)
// as real numbers (the diagonal of a Hermitian matrix).  The W^ra part costs
// 8 NG^2 nv nc FP64 flops per k block: at 20 x 20 bands and 500 plane waves
// about 47 ms on GB300's FP64 units for Nk = 64, which is why it is optional.
#include <cuda_runtime.h>

#include <algorithm>

#include "bse_internal.h"
#include "zgemm.cuh"

namespace bse {
namespace {

// U[b][G][j] = sum_G' W[q(b)][G][G'] z_b,j[G'] for the blocks b of a slab
struct DiagWProb {
  int M, N, K;            // ng, vectors per block, ng
  const bse_c128* w;      // [nq][ng][ng]
  const int32_t* qmap;    // [nk][nk]
  int nk, kb;             // k of block b is kb + b
  const bse_c128* z0;     // vector 0 of block 0
  int64_t zk, zj;         // complex stride between blocks, between vectors
  bse_c128* u;            // [blocks][ng][N]
  __device__ cplx a(int b, int m, int k) const {
    const int kk = kb + b;
    return ldc(w + ((int64_t)qmap[(int64_t)kk * nk + kk] * M + m) * K + k);
  }
  __device__ cplx b(int b, int n, int k) const { return ldc(z0 + b * zk + n * zj + k); }
  __device__ void store(int b, int m, int n, cplx v) const {
    reinterpret_cast<double2*>(u)[((int64_t)b * M + m) * N + n] = make_double2(v.x, v.y);
  }
};

struct DiagArgs {
  int nk, nv, nc, ng, kb, kn;
  const double *e_v, *e_c, *v_bar;
  const double2 *m_x, *m_vv, *n_vc;
  const double2 *u_rr, *u_ra;   // [kn][ng][nc], [kn][ng][nv nc] (u_ra NULL: no coupling)
  double sx, sc;                // 2 gamma_x kappa, gamma_c kappa
  double2 *A, *B;
  int64_t ld;
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// one warp per transition a = (k v c) of the slab
__global__ void __launch_bounds__(256) k_diag_fp64(DiagArgs a) {
  const int64_t nrow = (int64_t)a.kn * a.nv * a.nc;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < nrow; r += nwarps) {
    const int b = (int)(r / (a.nv * a.nc)), v = (int)((r / a.nc) % a.nv), c = (int)(r % a.nc);
    const int k = a.kb + b;
    const int64_t al = (int64_t)k * a.nv * a.nc + (int64_t)v * a.nc + c;
    const double2* mx = a.m_x + al * a.ng;
    // m_vv[b][k][v][v] (slab rows), U_rr[b][G][c]
    const double2* y = a.m_vv + (((int64_t)b * a.nk + k) * a.nv * a.nv + (int64_t)v * (a.nv + 1)) * a.ng;
    const double2* urr = a.u_rr + (int64_t)b * a.ng * a.nc + c;
    double vx = 0.0, wr = 0.0, wi = 0.0, xr = 0.0, xi = 0.0;
    for (int g = lane; g < a.ng; g += 32) {
      const double2 m = mx[g];
      vx += a.v_bar[g] * (m.x * m.x + m.y * m.y);
      const double2 yy = y[g], uu = urr[(int64_t)g * a.nc];
      wr += yy.x * uu.x + yy.y * uu.y;     // conj(y) u
      wi += yy.x * uu.y - yy.y * uu.x;
    }
    if (a.u_ra) {
      const double2* x = a.n_vc + (((int64_t)k * a.nk + k) * a.nv * a.nc + (int64_t)v * a.nc + c) * a.ng;
      const double2* ura = a.u_ra + (int64_t)b * a.ng * a.nv * a.nc + (int64_t)v * a.nc + c;
      for (int g = lane; g < a.ng; g += 32) {
        const double2 xx = x[g], uu = ura[(int64_t)g * a.nv * a.nc];
        xr += xx.x * uu.x + xx.y * uu.y;
        xi += xx.x * uu.y - xx.y * uu.x;
      }
    }
    vx = warp_sum(vx);
    wr = warp_sum(wr);
    xr = warp_sum(xr);
    (void)wi;
    (void)xi;
    if (lane == 0) {
      const int64_t d = al + al * a.ld;
      const double e = a.e_c[(int64_t)k * a.nc + c] - a.e_v[(int64_t)k * a.nv + v];
      a.A[d] = make_double2(e + a.sx * vx - a.sc * wr, 0.0);
      if (a.u_ra) a.B[d] = make_double2(a.sx * vx - a.sc * xr, 0.0);
    }
  }
}

}  // namespace

size_t diag_fp64_workspace(const Problem& pr) {
  const bse_problem& p = pr.p;
  size_t n = (size_t)pr.kn * p.ng * p.nc;
  if (p.coupling) n += (size_t)pr.kn * p.ng * p.nv * p.nc;
  return n * sizeof(bse_c128);
}

void diag_fp64(const Problem& pr, bse_c128* ws, cudaStream_t s) {
  const bse_problem& p = pr.p;
  const int nk = p.nk, nv = p.nv, nc = p.nc, ng = p.ng, kb = pr.kb, kn = pr.kn;
  bse_c128* u_rr = ws;
  bse_c128* u_ra = p.coupling ? ws + (size_t)kn * ng * nc : nullptr;
  if (p.gamma_c != 0.0) {
    // m_cc holds the slab's rows: block b at [b][kb + b][c][c]
    DiagWProb P{ng, nc, ng, p.w, p.q_minus, nk, kb, p.m_cc + (int64_t)kb * nc * nc * ng,
                (int64_t)(nk + 1) * nc * nc * ng, (int64_t)(nc + 1) * ng, u_rr};
    launch_zgemm(P, kn, s);
    if (p.coupling) {
      // n_vc is whole: block k at [k][k][v][c]
      DiagWProb R{ng, nv * nc, ng, p.w, p.q_plus, nk, kb,
                  p.n_vc + ((int64_t)kb * nk + kb) * nv * nc * ng,
                  (int64_t)(nk + 1) * nv * nc * ng, ng, u_ra};
      launch_zgemm(R, kn, s);
    }
  } else {
    BSE_CUDA(cudaMemsetAsync(ws, 0, diag_fp64_workspace(pr), s));
  }
  DiagArgs a{nk, nv, nc, ng, kb, kn, p.e_v, p.e_c, p.v_bar,
             reinterpret_cast<const double2*>(p.m_x), reinterpret_cast<const double2*>(p.m_vv),
             reinterpret_cast<const double2*>(p.n_vc), reinterpret_cast<const double2*>(u_rr),
             reinterpret_cast<const double2*>(u_ra), 2.0 * p.gamma_x * pr.kappa,
             p.gamma_c * pr.kappa, reinterpret_cast<double2*>(p.A),
             p.coupling ? reinterpret_cast<double2*>(p.B) : nullptr, p.ld};
  const int64_t warps = (int64_t)kn * nv * nc;
  const int grid = (int)std::min<int64_t>((warps * 32 + 255) / 256, 152 * 16);
  k_diag_fp64<<<grid, 256, 0, s>>>(a);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
}

}  // namespace bse
