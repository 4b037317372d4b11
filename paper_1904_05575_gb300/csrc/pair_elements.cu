// Plane-wave pair matrix elements from wavefunction coefficients (the matrix
// elements M and N of the LAPW section, interstitial part: the whole element
// for Bloch functions expanded in plane waves only):
//   M(a, b; G, s) = sum_{G1 in S} conj(a(G1)) b(G1 + G + s)
//   N(a, b; G, s) = sum_{G1 in S} conj(a(G1)) conj(b(-G1 - G - s))
// with b(G) = 0 outside the basis S and s the reciprocal vector that brings
// k + q back onto the k grid.  The four inputs of the build, at Q = 0:
//   m_x[k][v][c](G)       = M(C_ck, C_vk; G, 0)
//   m_vv[k][k'][v][v'](G) = M(C_v'k', C_vk; G, s-(k, k')),  q = k - k'
//   m_cc[k][k'][c][c'](G) = M(C_c'k', C_ck; G, s-(k, k'))
//   n_vc[k][k'][v][c'](G) = N(C_vk, C_c'k'; G, s+(k, k')),  q = -k - k'
// One block per (bra vector, group of ket vectors): the bra coefficients,
// the basis coordinates and a lookup table from integer coordinates to basis
// index (over the box the sums can reach) sit in shared memory; each thread
// accumulates outputs (ket, G) over the basis in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "bse_internal.h"

namespace bse {
namespace {

struct PairArgs {
  int n, nk, nv, nc, npw, ng, kb, kn;
  const double2 *cv, *cc;   // [nk][nv][npw], [nk][nc][npw]
  const int* basis;         // [npw][3]
  const int* gout;          // [ng][3]
  const int* table;         // [box^3] basis index or -1
  int half, box;            // coordinate c maps to slot c + half, 0 <= slot < box
  double2 *m_x, *m_vv, *m_cc, *n_vc;
};

enum PairMode { PM_X = 0, PM_VV = 1, PM_CC = 2, PM_N = 3 };

__device__ __forceinline__ void kcoord(int k, int n, int* c) {
  c[0] = k / (n * n);
  c[1] = (k / n) % n;
  c[2] = k % n;
}

template <int MODE>
__global__ void __launch_bounds__(256) k_pair_elements(PairArgs a) {
  extern __shared__ uint8_t smem[];
  double2* bra = reinterpret_cast<double2*>(smem);            // [npw]
  int* bc = reinterpret_cast<int*>(bra + a.npw);              // [npw][3]
  int* tab = bc + 3 * a.npw;                                   // [box^3]
  const int u = blockIdx.x;
  int k, kp, bra_band, nket;
  const double2 *bra_src, *ket0;
  int s[3] = {0, 0, 0};
  int64_t out0, ostride_j;
  double2* out;
  if (MODE == PM_X) {          // u = (k, c): bra C_ck, kets C_vk
    k = u / a.nc;
    bra_band = u % a.nc;
    bra_src = a.cc + ((int64_t)k * a.nc + bra_band) * a.npw;
    ket0 = a.cv + (int64_t)k * a.nv * a.npw;
    nket = a.nv;
    out = a.m_x;
    out0 = ((int64_t)k * a.nv * a.nc + bra_band) * a.ng;   // + j nc ng
    ostride_j = (int64_t)a.nc * a.ng;
  } else if (MODE == PM_VV || MODE == PM_CC) {   // u = (r, k', b'): bra C_b'k', kets C_bk
    const int nb = MODE == PM_VV ? a.nv : a.nc;
    const double2* c = MODE == PM_VV ? a.cv : a.cc;
    const int r = u / (a.nk * nb);
    kp = (u / nb) % a.nk;
    bra_band = u % nb;
    k = a.kb + r;
    bra_src = c + ((int64_t)kp * nb + bra_band) * a.npw;
    ket0 = c + (int64_t)k * nb * a.npw;
    nket = nb;
    int ck[3], ckp[3];
    kcoord(k, a.n, ck);
    kcoord(kp, a.n, ckp);
    for (int d = 0; d < 3; ++d) {   // q = (k - k') mod n; k' + q - k = n s
      const int q = ((ck[d] - ckp[d]) % a.n + a.n) % a.n;
      s[d] = (ckp[d] + q - ck[d]) / a.n;
    }
    out = MODE == PM_VV ? a.m_vv : a.m_cc;
    out0 = (((int64_t)r * a.nk + kp) * nb * nb + bra_band) * a.ng;   // + j nb ng
    ostride_j = (int64_t)nb * a.ng;
  } else {                     // u = (k, k', v): bra C_vk, kets conj(C_c'k')
    k = u / (a.nk * a.nv);
    kp = (u / a.nv) % a.nk;
    bra_band = u % a.nv;
    bra_src = a.cv + ((int64_t)k * a.nv + bra_band) * a.npw;
    ket0 = a.cc + (int64_t)kp * a.nc * a.npw;
    nket = a.nc;
    int ck[3], ckp[3];
    kcoord(k, a.n, ck);
    kcoord(kp, a.n, ckp);
    for (int d = 0; d < 3; ++d) {   // q = (-k - k') mod n; k + k' + q = n s
      const int q = ((-ck[d] - ckp[d]) % a.n + a.n) % a.n;
      s[d] = (ck[d] + ckp[d] + q) / a.n;
    }
    out = a.n_vc;
    out0 = (((int64_t)k * a.nk + kp) * a.nv + bra_band) * a.nc * a.ng;   // + j ng
    ostride_j = a.ng;
  }
  for (int i = threadIdx.x; i < a.npw; i += blockDim.x) {
    bra[i] = bra_src[i];
    bc[3 * i] = a.basis[3 * i];
    bc[3 * i + 1] = a.basis[3 * i + 1];
    bc[3 * i + 2] = a.basis[3 * i + 2];
  }
  const int tsize = a.box * a.box * a.box;
  for (int i = threadIdx.x; i < tsize; i += blockDim.x) tab[i] = a.table[i];
  __syncthreads();
  const int nout = nket * a.ng;
  for (int t = threadIdx.x; t < nout; t += blockDim.x) {
    const int j = t / a.ng, g = t - j * a.ng;
    const double2* ket = ket0 + (int64_t)j * a.npw;
    // G + s (M form) or -G - s (N form), shifted into table slots
    int o[3];
    for (int d = 0; d < 3; ++d)
      o[d] = (MODE == PM_N ? -(a.gout[3 * g + d] + s[d]) : a.gout[3 * g + d] + s[d]) + a.half;
    double sx = 0.0, sy = 0.0;
    for (int i1 = 0; i1 < a.npw; ++i1) {
      int x, y, z;
      if (MODE == PM_N) {
        x = o[0] - bc[3 * i1];
        y = o[1] - bc[3 * i1 + 1];
        z = o[2] - bc[3 * i1 + 2];
      } else {
        x = o[0] + bc[3 * i1];
        y = o[1] + bc[3 * i1 + 1];
        z = o[2] + bc[3 * i1 + 2];
      }
      const int idx = tab[(x * a.box + y) * a.box + z];
      if (idx < 0) continue;
      const double2 p = bra[i1];
      const double2 q = __ldg(ket + idx);
      const double qy = MODE == PM_N ? -q.y : q.y;
      // conj(p) * q (or conj(p) * conj(q))
      sx = fma(p.x, q.x, fma(p.y, qy, sx));
      sy = fma(p.x, qy, fma(-p.y, q.x, sy));
    }
    out[out0 + (int64_t)j * ostride_j + g] = make_double2(sx, sy);
  }
}

template <int MODE>
void launch_pairs(const PairArgs& a, int units, size_t smem, cudaStream_t s) {
  if (units <= 0) return;
  auto kern = k_pair_elements<MODE>;
  BSE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<units, 256, smem, s>>>(a);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
}

}  // namespace

void pair_elements_fp64(int n, int nv, int nc, int npw, int ng, const bse_c128* cv,
                        const bse_c128* cc, const int32_t* basis_h, const int32_t* gout_h,
                        int kb, int kn, bse_c128* m_x, bse_c128* m_vv, bse_c128* m_cc,
                        bse_c128* n_vc, cudaStream_t s) {
  const int nk = n * n * n;
  int rb = 0, rg = 0;
  for (int i = 0; i < 3 * npw; ++i) rb = std::max(rb, std::abs(basis_h[i]));
  for (int i = 0; i < 3 * ng; ++i) rg = std::max(rg, std::abs(gout_h[i]));
  // every index the sums form lies in [-(rb + rg + 2), rb + rg + 2] per direction
  const int half = rb + rg + 2, box = 2 * half + 1;
  if (box > 64) throw Error(BSE_ERR_UNSUPPORTED, "basis or output vectors too far from the origin");
  std::vector<int32_t> table((size_t)box * box * box, -1);
  for (int i = 0; i < npw; ++i) {
    const int x = basis_h[3 * i] + half, y = basis_h[3 * i + 1] + half, z = basis_h[3 * i + 2] + half;
    if (x < 0 || y < 0 || z < 0 || x >= box || y >= box || z >= box)
      throw Error(BSE_ERR_ARG, "basis vector outside the lookup box");
    int32_t& e = table[((size_t)x * box + y) * box + z];
    if (e >= 0) throw Error(BSE_ERR_ARG, "basis vector " + std::to_string(i) + " repeats one before it");
    e = i;
  }
  const size_t smem = (size_t)npw * 16 + (size_t)npw * 12 + table.size() * 4;
  if (smem > 200 * 1024) throw Error(BSE_ERR_UNSUPPORTED, "plane-wave basis too large for the kernel");
  DeviceBuffer dtab(table.size() * sizeof(int32_t), s), dbasis((size_t)npw * 12, s),
      dgout((size_t)ng * 12, s);
  BSE_CUDA(cudaMemcpyAsync(dtab.ptr, table.data(), table.size() * 4, cudaMemcpyHostToDevice, s));
  BSE_CUDA(cudaMemcpyAsync(dbasis.ptr, basis_h, (size_t)npw * 12, cudaMemcpyHostToDevice, s));
  BSE_CUDA(cudaMemcpyAsync(dgout.ptr, gout_h, (size_t)ng * 12, cudaMemcpyHostToDevice, s));
  PairArgs a{n, nk, nv, nc, npw, ng, kb, kn,
             reinterpret_cast<const double2*>(cv), reinterpret_cast<const double2*>(cc),
             dbasis.as<int>(), dgout.as<int>(), dtab.as<int>(), half, box,
             reinterpret_cast<double2*>(m_x), reinterpret_cast<double2*>(m_vv),
             reinterpret_cast<double2*>(m_cc), reinterpret_cast<double2*>(n_vc)};
  Phase ph("pair_elements", s);
  if (m_x) launch_pairs<PM_X>(a, nk * nc, smem, s);
  if (m_vv) launch_pairs<PM_VV>(a, kn * nk * nv, smem, s);
  if (m_cc) launch_pairs<PM_CC>(a, kn * nk * nc, smem, s);
  if (n_vc) launch_pairs<PM_N>(a, nk * nk * nv, smem, s);
  BSE_CUDA(cudaStreamSynchronize(s));   // the stream-ordered lookup arrays stay alive until used
}

}  // namespace bse
