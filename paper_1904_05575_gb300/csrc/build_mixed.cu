// Split-precision build of the BSE Hamiltonian on tcgen05 tensor cores.
//
// Same algebra as the FP64 build (exchange Eq. vrrofM, direct Eqs. wrrm and
// wrabar, assembly Eqs. diagonalblock / couplingblock), with the two large
// contractions on tensor cores:
//   1. split      complex128 rows -> BF16 planes (Re/Im x P pieces), K padded
//                 to 16; stage-1 rows are gathered in pairs-sorted-by-q order
//                 so every 128-row tile shares one W(q)
//   2. exchange   tensor-core GEMM conj(M_x) diag(v_bar) M_x^T; the epilogue
//                 writes A = E + 2 gx k V and B = 2 gx k V (FP64)
//   3. stage 1    tensor-core GEMM T = X_side W(q)^T per q group -> FP32 T[G][row]
//                 (or T split at once into BF16 planes for a tensor-core stage 2)
//   4. stage 2    contraction of T with the other pair side over G, subtracted
//                 from A (W^rr) or B (W^ra) in FP64: a tensor-core GEMM per pair
//                 block where both sides have >= 64 rows, else FP32 on CUDA
//                 cores reading the complex128 input directly (k_stage2_skinny,
//                 k_stage2_multi, k_stage2_pipe, k_stage2<TX, TT, RX, RT>)
// Where every pair block fits the fused epilogue (rows_t a power of two,
// rows_x <= min(16, rows_t)), steps 3 and 4 run as one tcgen05 launch whose
// epilogue performs the contraction on the TMEM tile (tc_direct.cuh).
// A problem given as a k-row slab (bse_problem.k_begin / k_count) builds only
// the rows (k v c) of its slab: exchange tiles over those rows, direct terms
// over the slab's pairs (k, k'), pair decodes offset by k_begin.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <map>
#include <mutex>
#include <tuple>
#include <numeric>
#include <vector>

#include "bits.cuh"
#include "bse_internal.h"
#include "tc_direct.cuh"
#include "tc_gemm.cuh"

namespace bse {
namespace {

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------------------
// split: one thread per (output row, k); P pieces per real number
// ---------------------------------------------------------------------------
enum SplitMode { SPLIT_DENSE = 0, SPLIT_PAIRS = 1, SPLIT_W = 2 };

struct SplitArgs {
  const double2* src;
  int mode;
  // SPLIT_DENSE: row r is src[r * K + k]
  // SPLIT_PAIRS: row r = (slot, j) with rows_per rows per slot is the j-th row of
  //              pair perm[slot]: src[(perm[slot] * rows_per + j) * K + k]
  // SPLIT_W:     row r = (q, g) with rows_per = padded G per q; g >= K is a zero
  //              row; W[q][g][k] (or, transposed, W[q][k][g])
  const int* perm;
  int rows_per;
  int transpose;
  int K;                    // real K
  int Kp;                   // padded K (multiple of 16)
  int rows;                 // output rows
  int pieces;
  int conj;                 // store the conjugate
  const double* kscale;     // per-k real factor or NULL
  __nv_bfloat16* out;       // [2 * pieces][plane_rows][Kp]
  int64_t plane_rows = 0;   // rows of each destination plane (0: rows)
  int64_t row0 = 0;         // first destination row
  int pair_nb = 0;          // SPLIT_PAIRS: rows_per = nb^2 rows (b, b') stored as (b', b)
  int64_t src_ld = 0;       // SPLIT_DENSE: source row stride (0: K)
  int zero_diag = 0;        // SPLIT_DENSE: element k == row stored as zero
  int bneg = 0;             // B-operand layout: 3P planes (-Im, Re, Im) per piece
  int tdense = 0;           // SPLIT_DENSE read transposed: row r, element k at src[k * src_ld + r]
  int c64 = 0;              // src holds complex64 (float re, im) instead of complex128
};

// One thread per (output row, 8 consecutive k): every element is read as two
// 32-bit words, rounded to FP32 with integer instructions and split in FP32
// into P BF16 pieces; each plane gets one 16-byte store of 8 pieces.
template <int P>
__global__ void __launch_bounds__(256) k_split(SplitArgs a) {
  const int kg = a.Kp / 8;
  const int64_t total = (int64_t)a.rows * kg;
  const int64_t plane = (a.plane_rows ? a.plane_rows : (int64_t)a.rows) * a.Kp;
  const uint4* src = reinterpret_cast<const uint4*>(a.src);   // one complex128 per uint4
  const uint2* src64 = reinterpret_cast<const uint2*>(a.src);  // or one complex64 per uint2
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int row = (int)(i / kg), k0 = (int)(i % kg) * 8;
    int64_t off = (int64_t)row * (a.src_ld ? a.src_ld : a.K), kstride = 1;
    if (a.tdense) {   // consecutive threads on consecutive rows: coalesced reads
      row = (int)(i % a.rows);
      k0 = (int)(i / a.rows) * 8;
      off = row;
      kstride = a.src_ld;
    }
    if (a.mode == SPLIT_PAIRS) {
      const int slot = row / a.rows_per;
      int j = row % a.rows_per;
      if (a.pair_nb) j = (j % a.pair_nb) * a.pair_nb + j / a.pair_nb;
      off = ((int64_t)a.perm[slot] * a.rows_per + j) * a.K;
    } else if (a.mode == SPLIT_W) {
      const int q = row / a.rows_per, g = row % a.rows_per;
      off = g >= a.K ? -1 : (int64_t)q * a.K * a.K + (a.transpose ? g : (int64_t)g * a.K);
      kstride = a.transpose ? a.K : 1;
    }
    uint32_t hr[P][8], hi[P][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = k0 + e;
      const bool take = k < a.K && off >= 0 && !(a.zero_diag && k == row);
      uint32_t fr = 0u, fi = 0u;
      if (a.c64) {   // already FP32
        if (take) {
          const uint2 x = __ldg(src64 + off + (int64_t)k * kstride);
          fr = x.x;
          fi = x.y;
        }
      } else {
        uint4 x = make_uint4(0u, 0u, 0u, 0u);
        if (take) x = __ldg(src + off + (int64_t)k * kstride);
        fr = f64w_to_f32_bits(x.x, x.y);
        fi = f64w_to_f32_bits(x.z, x.w);
      }
      if (a.kscale && k < a.K) {   // exchange operand only: scale in FP32
        const float sc = (float)a.kscale[k];
        fr = __float_as_uint(__uint_as_float(fr) * sc);
        fi = __float_as_uint(__uint_as_float(fi) * sc);
      }
      if (a.conj) fi ^= 0x80000000u;
      uint32_t tr[P], ti[P];
      split_f32_bf16<P>(fr, tr);
      split_f32_bf16<P>(fi, ti);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        hr[p][e] = tr[p];
        hi[p][e] = ti[p];
      }
    }
    const int64_t o = (a.row0 + row) * a.Kp + k0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      uint4 vr, vi;
      vr.x = hr[p][0] | (hr[p][1] << 16); vr.y = hr[p][2] | (hr[p][3] << 16);
      vr.z = hr[p][4] | (hr[p][5] << 16); vr.w = hr[p][6] | (hr[p][7] << 16);
      vi.x = hi[p][0] | (hi[p][1] << 16); vi.y = hi[p][2] | (hi[p][3] << 16);
      vi.z = hi[p][4] | (hi[p][5] << 16); vi.w = hi[p][6] | (hi[p][7] << 16);
      if (a.bneg) {   // planes 3p: -Im (both BF16 signs flipped), 3p + 1: Re, 3p + 2: Im
        const uint4 vn = make_uint4(vi.x ^ 0x80008000u, vi.y ^ 0x80008000u, vi.z ^ 0x80008000u,
                                    vi.w ^ 0x80008000u);
        *reinterpret_cast<uint4*>(a.out + (int64_t)(3 * p) * plane + o) = vn;
        *reinterpret_cast<uint4*>(a.out + (int64_t)(3 * p + 1) * plane + o) = vr;
        *reinterpret_cast<uint4*>(a.out + (int64_t)(3 * p + 2) * plane + o) = vi;
      } else {
        *reinterpret_cast<uint4*>(a.out + (int64_t)p * plane + o) = vr;
        *reinterpret_cast<uint4*>(a.out + (int64_t)(P + p) * plane + o) = vi;
      }
    }
  }
}

void launch_split(const SplitArgs& a, cudaStream_t s) {
  const int64_t total = (int64_t)a.rows * (a.Kp / 8);
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (a.pieces == 3)
    k_split<3><<<(int)std::max<int64_t>(blocks, 1), 256, 0, s>>>(a);
  else
    k_split<2><<<(int)std::max<int64_t>(blocks, 1), 256, 0, s>>>(a);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
}

// ---------------------------------------------------------------------------
// epilogues of the tensor-core GEMM
// ---------------------------------------------------------------------------
// V[alpha][alpha'] -> A, B (column-major FP64).  V is Hermitian (Eq. vrrofM)
// and so are A and B (Eq. Hetr): with `upper`, only tiles touching the blocks
// k <= k' are computed and the epilogue writes the elements of those blocks
// (alpha in block k, alpha' in block k', k = alpha / (nv nc)); the blocks
// k > k' are filled afterwards from their mirror by k_hermitian_complete.
// The diagonal of V is stored real.  Lanes are consecutive rows of one
// column: every store is coalesced.
struct ExchangeEpi {
  double2 *A, *B;
  int64_t ld;
  float scale;         // 2 gamma_x kappa (the product is formed in FP32, then widened exactly)
  const double *e_v, *e_c;
  int nv, nc;
  int upper;
  __device__ __forceinline__ void operator()(const tc::Tile& t, int row, int c0, const float* re,
                                             const float* im) const {
    const int al = t.out_row0 + row;              // N < 2^30 (checked at validation)
    const int nb = nv * nc;
    const int kal = al / nb;
    // block k' of column ap is >= k of the row exactly when ap >= k nb
    const int ap_min = upper ? kal * nb : 0;
    double2* a_col = A + al + (int64_t)(t.n0 + c0) * ld;
    double2* b_col = B ? B + al + (int64_t)(t.n0 + c0) * ld : nullptr;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int col = c0 + j;
      const int ap = t.n0 + col;
      if (col < t.n_valid && ap >= ap_min) {
        double2 val = make_double2(f32_to_f64_bits(scale * re[j]), f32_to_f64_bits(scale * im[j]));
        if (al == ap) val.y = 0.0;   // the diagonal of a Hermitian V is real
        if (b_col) b_col[(int64_t)j * ld] = val;
        if (al == ap) {
          const int r = al - kal * nb, v = r / nc, c = r - v * nc;
          val.x += e_c[kal * nc + c] - e_v[kal * nv + v];
        }
        a_col[(int64_t)j * ld] = val;
      }
    }
  }
};

// Hermitian completion (Eq. Hetr: A and B Hermitian): every element of a block
// k > k' is set to the conjugate of its mirror in block (k', k).  Tiles of
// 32 x 32 elements of the lower half, staged through shared memory so that
// the reads (a run of rows of one source column) and the writes (a run of
// rows of one destination column) are both coalesced.  Elements of the
// diagonal blocks are left alone.
struct CompleteArgs {
  double2* M;       // A or B, column-major
  int64_t ld;
  int n, nb;        // N; rows per k block (nv nc)
};

__global__ void __launch_bounds__(256) k_hermitian_complete(CompleteArgs a) {
  __shared__ double2 t[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t nt = (a.n + 31) / 32;
  const int64_t ntiles = nt * (nt + 1) / 2;
  for (int64_t L = blockIdx.x; L < ntiles; L += gridDim.x) {
    // tile (tr, tc), tr >= tc, of the lower triangle of the tile grid (an FP32
    // estimate of the row, corrected with integers: no FP64 arithmetic)
    int64_t tr = (int64_t)((sqrtf(8.f * (float)L + 1.f) - 1.f) * 0.5f);
    while (tr * (tr + 1) / 2 > L) --tr;
    while ((tr + 1) * (tr + 2) / 2 <= L) ++tr;
    const int64_t tcol = L - tr * (tr + 1) / 2;
    const int r0 = (int)(tr * 32), c0 = (int)(tcol * 32);
    const int rlast = min(r0 + 31, a.n - 1);
    if (rlast / a.nb <= c0 / a.nb) continue;   // no element below the diagonal blocks
    // source: (c, r) for c in [c0, c0+32), r in [r0, r0+32): column r, rows c
    for (int j = ty; j < 32; j += 8) {
      const int r = r0 + j, c = c0 + tx;
      if (r < a.n && c < a.n) t[j][tx] = a.M[c + (int64_t)r * a.ld];
    }
    __syncthreads();
    // destination: (r, c) = conj of the source (c, r), column c, rows r
    for (int j = ty; j < 32; j += 8) {
      const int c = c0 + j, r = r0 + tx;
      if (r < a.n && c < a.n && r / a.nb > c / a.nb) {
        const double2 v = t[tx][j];
        a.M[r + (int64_t)c * a.ld] = make_double2(v.x, -v.y);
      }
    }
    __syncthreads();
  }
}

void launch_hermitian_complete(double2* M, int64_t ld, int n, int nb, cudaStream_t s) {
  if (!M || n <= nb) return;
  const int64_t nt = (n + 31) / 32;
  const int64_t ntiles = nt * (nt + 1) / 2;
  const int grid = (int)std::min<int64_t>(ntiles, 152 * 8);
  k_hermitian_complete<<<grid, 256, 0, s>>>(CompleteArgs{M, ld, n, nb});
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
}

// Stage-1 output per direct term (Tile::prob = term): FP32 T[G][row] for the
// CUDA-core stage 2, or, for a term whose stage 2 runs on the tensor cores,
// T split at once into BF16 planes [2P][plane_rows][Kp] (K = G', row-major,
// the operand layout of the GEMM), conjugated when opT conjugates.
struct TOut {
  float2* T;                  // FP32 path (NULL: planes)
  int64_t t_ld;
  __nv_bfloat16* planes;      // split path
  int64_t plane_rows;
  int Kp, pieces, conj;
  int bneg = 0;               // planes in the B-operand layout (3P: -Im, Re, Im per piece)
  int64_t row_off = 0;        // row of the planes = stage-1 row + row_off
};

struct TEpiMulti {
  const TOut* outs;
  __device__ __forceinline__ void operator()(const tc::Tile& t, int row, int c0, const float* re,
                                             const float* im) const {
    const TOut o = outs[t.prob];
    const int64_t r = t.out_row0 + row;
    if (o.T) {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < t.n_valid) o.T[(int64_t)(t.n0 + c0 + j) * o.t_ld + r] = make_float2(re[j], im[j]);
      return;
    }
    // 8 columns per 16-byte store and plane; a group starting at or past the
    // padded K is not written (columns past NG hold zeros from set-up)
    const int64_t plane = o.plane_rows * o.Kp;
    const uint32_t flip = o.conj ? 0x80000000u : 0u;
    const int64_t rp = r + o.row_off;
#pragma unroll
    for (int g8 = 0; g8 < 4; ++g8) {
      const int col = t.n0 + c0 + 8 * g8;
      if (col >= o.Kp) continue;
      uint32_t hr[3][8], hi[3][8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = 8 * g8 + e;
        const bool ok = c0 + j < t.n_valid;
        const uint32_t ur = ok ? __float_as_uint(re[j]) : 0u;
        const uint32_t ui = ok ? (__float_as_uint(im[j]) ^ flip) : 0u;
        uint32_t a3[3], b3[3];
        if (o.pieces == 3) {
          split_f32_bf16<3>(ur, a3);
          split_f32_bf16<3>(ui, b3);
        } else {
          split_f32_bf16<2>(ur, a3);
          split_f32_bf16<2>(ui, b3);
          a3[2] = b3[2] = 0u;
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          hr[q][e] = a3[q];
          hi[q][e] = b3[q];
        }
      }
      const int64_t off = rp * o.Kp + col;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q < o.pieces) {
          uint4 vr, vi;
          vr.x = hr[q][0] | (hr[q][1] << 16); vr.y = hr[q][2] | (hr[q][3] << 16);
          vr.z = hr[q][4] | (hr[q][5] << 16); vr.w = hr[q][6] | (hr[q][7] << 16);
          vi.x = hi[q][0] | (hi[q][1] << 16); vi.y = hi[q][2] | (hi[q][3] << 16);
          vi.z = hi[q][4] | (hi[q][5] << 16); vi.w = hi[q][6] | (hi[q][7] << 16);
          if (o.bneg) {
            const uint4 vn = make_uint4(vi.x ^ 0x80008000u, vi.y ^ 0x80008000u,
                                        vi.z ^ 0x80008000u, vi.w ^ 0x80008000u);
            *reinterpret_cast<uint4*>(o.planes + (int64_t)(3 * q) * plane + off) = vn;
            *reinterpret_cast<uint4*>(o.planes + (int64_t)(3 * q + 1) * plane + off) = vr;
            *reinterpret_cast<uint4*>(o.planes + (int64_t)(3 * q + 2) * plane + off) = vi;
          } else {
            *reinterpret_cast<uint4*>(o.planes + (int64_t)q * plane + off) = vr;
            *reinterpret_cast<uint4*>(o.planes + (int64_t)(o.pieces + q) * plane + off) = vi;
          }
        }
      }
    }
  }
};

// Stage 2 on the tensor cores (large pair blocks): one pair block per tile
// row range (Tile::out_row0 = pair * rows_r + first row); the epilogue
// subtracts gamma_c kappa P (formed in FP32, widened exactly) from A (W^rr)
// or B (W^ra) in FP64, one owner per element.  The operands are oriented so
// that the tile rows (the TMEM lanes, one per thread) run over the
// conduction index c fastest: consecutive lanes then update consecutive rows
// of one column of A or B (runs of Nc) instead of Nc-strided columns.
struct S2TcParams {
  double2* out;
  int64_t ld;
  int nk, nvnc;     // k points; Nv * Nc
  int k_begin;      // first k row of the slab (pair = (k - k_begin) nk + k')
  float scale;
  int rows_r;       // rows per pair of the side that forms the tile rows
  int row_nb;       // tile rows stored (b', b) for a side indexed (b, b') (0: as stored)
  // each side's pair index is (a, b) with b < nb; it moves the element
  // (row al, column ap) of A or B by a * sa + b * sb in al + ap * ld
  int nb_r, nb_c;   // row side, column side
  int64_t ra, rb, ca, cb;
};

struct S2TcEpi {
  const S2TcParams* params;
  __device__ __forceinline__ void operator()(const tc::Tile& t, int row, int c0, const float* re,
                                             const float* im) const {
    const S2TcParams q = params[t.prob];
    const int rg = t.out_row0 + row;
    const int pair = rg / q.rows_r;
    int ir = rg - pair * q.rows_r;
    if (q.row_nb) ir = (ir % q.row_nb) * q.row_nb + ir / q.row_nb;
    const int kl = pair / q.nk, kp = pair - kl * q.nk, k = q.k_begin + kl;
    const int ar = ir / q.nb_r, br = ir - ar * q.nb_r;
    double2* base = q.out + (int64_t)k * q.nvnc + (int64_t)kp * q.nvnc * q.ld + ar * q.ra + br * q.rb;
    const int jc0 = t.n0 + c0;
    int bc = jc0 % q.nb_c;
    double2* dst = base + (int64_t)(jc0 / q.nb_c) * q.ca + bc * q.cb;
    const int64_t wrap = q.ca - (int64_t)q.nb_c * q.cb;
    // groups of 8: the addresses and loads first, then the stores, so the
    // loads of a group are in flight together
#pragma unroll
    for (int j0 = 0; j0 < 32; j0 += 8) {
      double2* p[8];
      double2 o[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        p[u] = dst;
        dst += q.cb;
        if (++bc == q.nb_c) {
          bc = 0;
          dst += wrap;
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (c0 + j0 + u < t.n_valid) o[u] = *p[u];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (c0 + j0 + u < t.n_valid) {
          o[u].x -= f32_to_f64_bits(q.scale * re[j0 + u]);
          o[u].y -= f32_to_f64_bits(q.scale * im[j0 + u]);
          *p[u] = o[u];
        }
      }
    }
  }
};

// ---------------------------------------------------------------------------
// stage 2: P[rx][rt] = sum_G opX(X_p[rx][G]) * opT(T[G][slot * rows_t + rt])
// ---------------------------------------------------------------------------
enum Stage2Mode { S2_RR_CC = 0, S2_RR_VV = 1, S2_RA = 2 };

struct Stage2Args {
  int mode;
  const double2* x;      // complex128 pair array, [slab pairs][rows_x][ng] ([nk][nk].. when transposed)
  int x_transpose_pair;  // read X of pair (k', k) (W^ra) from the whole array
  int conj_x, conj_t;
  const float2* T;
  int64_t t_ld;
  const int* slot_of_pair;
  const int* pair_of = nullptr;   // index -> pair of the pairs built (NULL: every pair)
  int rows_x, rows_t, ng, nk, nv, nc;
  int64_t t_row0 = 0;    // first T row of this term (batched plans)
  int k_begin = 0;       // first k row of the slab: pair p = (k - k_begin) nk + k'
  double scale;          // gamma_c kappa
  double2* out;          // A or B
  int64_t ld;
};

// i-th pair block of a stage-2 launch: every pair of the slab, or the listed
// ones (the blocks k <= k' of a Hermitian build)
__device__ __forceinline__ int s2_pair(const Stage2Args& a, int i) {
  return a.pair_of ? a.pair_of[i] : i;
}

// asynchronous global -> shared copies (zero-filled when pred is false)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(smem)),
               "l"(gmem), "r"(pred ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool pred) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(tc::smem_u32(smem)),
               "l"(gmem), "r"(pred ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// TX x TT output tile per block (X rows x T rows), RX x RT outputs per thread.
// Software-pipelined: the raw complex128 X rows and FP32 T rows of the next 16
// plane waves are copied to shared memory asynchronously (cp.async, double
// buffered) while the current chunk is converted and contracted.
template <int TX, int TT, int RX, int RT>
__global__ void __launch_bounds__((TX / RX) * (TT / RT)) k_stage2(Stage2Args a) {
  constexpr int NTH = (TX / RX) * (TT / RT), CT = TT / RT, CX = TX / RX;
  constexpr int GC = 16;
  __shared__ __align__(16) uint4 Xr[2][TX][GC];      // raw FP64 complex
  __shared__ __align__(16) float2 Tr[2][GC][TT];     // FP32 complex
  __shared__ float2 Xs[TX][GC + 1];                  // converted X of the current chunk
  const int p = s2_pair(a, blockIdx.x);
  const int k = a.k_begin + p / a.nk, kp = p % a.nk;
  const int rx0 = blockIdx.y * TX, rt0 = blockIdx.z * TT;
  const int64_t xp = a.x_transpose_pair ? (int64_t)kp * a.nk + k : (int64_t)p;
  const uint4* X = reinterpret_cast<const uint4*>(a.x) + xp * a.rows_x * a.ng;
  const int64_t trow0 = a.t_row0 + (int64_t)a.slot_of_pair[p] * a.rows_t;
  const int tid = threadIdx.x;
  const int tx = tid % CT, ty = tid / CT;
  const int nchunks = (a.ng + GC - 1) / GC;

  auto prefetch = [&](int c, int buf) {
    const int g0 = c * GC;
    for (int i = tid; i < TX * GC; i += NTH) {
      const int r = i / GC, g = i % GC;
      const bool ok = rx0 + r < a.rows_x && g0 + g < a.ng;
      cp_async16(&Xr[buf][r][g], ok ? (const void*)(X + (int64_t)(rx0 + r) * a.ng + g0 + g)
                                    : (const void*)X, ok);
    }
    for (int i = tid; i < GC * TT; i += NTH) {
      const int g = i / TT, r = i % TT;
      const bool ok = rt0 + r < a.rows_t && g0 + g < a.ng;
      const float2* src = a.T + (ok ? (int64_t)(g0 + g) * a.t_ld + trow0 + rt0 + r : 0);
      cp_async8(&Tr[buf][g][r], src, ok);
    }
    cp_async_commit();
  };

  // compensated FP32: sums over 8 plane waves in FMA, folded into (hi, lo) pairs
  // with TwoSum, so no FP64 instruction runs inside the loop
  float hx[RX][RT], hy[RX][RT], lx[RX][RT], ly[RX][RT];
#pragma unroll
  for (int i = 0; i < RX; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) hx[i][j] = hy[i][j] = lx[i][j] = ly[i][j] = 0.f;
  const uint32_t xflip = a.conj_x ? 0x80000000u : 0u;
  const float tsign = a.conj_t ? -1.f : 1.f;

  prefetch(0, 0);
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    if (c + 1 < nchunks) {
      prefetch(c + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    for (int i = tid; i < TX * GC; i += NTH) {
      const int r = i / GC, g = i % GC;
      const uint4 d = Xr[buf][r][g];
      Xs[r][g] = make_float2(__uint_as_float(f64w_to_f32_bits(d.x, d.y)),
                             __uint_as_float(f64w_to_f32_bits(d.z, d.w) ^ xflip));
    }
    __syncthreads();
#pragma unroll
    for (int g8 = 0; g8 < GC; g8 += 8) {
      float accx[RX][RT], accy[RX][RT];
#pragma unroll
      for (int i = 0; i < RX; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) accx[i][j] = accy[i][j] = 0.f;
#pragma unroll
      for (int g = g8; g < g8 + 8; ++g) {
        float2 xv[RX], tv[RT];
#pragma unroll
        for (int i = 0; i < RX; ++i) xv[i] = Xs[ty + i * CX][g];
#pragma unroll
        for (int j = 0; j < RT; ++j) {
          tv[j] = Tr[buf][g][tx + j * CT];
          tv[j].y *= tsign;
        }
#pragma unroll
        for (int i = 0; i < RX; ++i)
#pragma unroll
          for (int j = 0; j < RT; ++j) {
            accx[i][j] = fmaf(xv[i].x, tv[j].x, accx[i][j]);
            accx[i][j] = fmaf(-xv[i].y, tv[j].y, accx[i][j]);
            accy[i][j] = fmaf(xv[i].x, tv[j].y, accy[i][j]);
            accy[i][j] = fmaf(xv[i].y, tv[j].x, accy[i][j]);
          }
      }
#pragma unroll
      for (int i = 0; i < RX; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) {
          float s, e;
          two_sum(hx[i][j], accx[i][j], s, e);
          hx[i][j] = s;
          lx[i][j] += e;
          two_sum(hy[i][j], accy[i][j], s, e);
          hy[i][j] = s;
          ly[i][j] += e;
        }
    }
    __syncthreads();   // the next prefetch overwrites this buffer
  }

  const int nv = a.nv, nc = a.nc;
#pragma unroll
  for (int i = 0; i < RX; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) {
      const int rx = rx0 + ty + i * CX, rt = rt0 + tx + j * CT;
      if (rx >= a.rows_x || rt >= a.rows_t) continue;
      int vi, ci, vp, cp;
      if (a.mode == S2_RR_CC) {          // rx = (v, v'), rt = (c, c')
        vi = rx / nv; vp = rx % nv; ci = rt / nc; cp = rt % nc;
      } else if (a.mode == S2_RR_VV) {   // rx = (c, c'), rt = (v, v')
        ci = rx / nc; cp = rx % nc; vi = rt / nv; vp = rt % nv;
      } else {                           // rx = (v', c), rt = (v, c')
        vp = rx / nc; ci = rx % nc; vi = rt / nc; cp = rt % nc;
      }
      const int64_t al = ((int64_t)k * nv + vi) * nc + ci;
      const int64_t ap = ((int64_t)kp * nv + vp) * nc + cp;
      double2* dst = a.out + al + ap * a.ld;
      double2 o = *dst;
      // contribution formed in FP32 (hi + lo carries the compensated sum), widened exactly
      const float sc = (float)a.scale;
      o.x -= f32_to_f64_bits(scale_hi_lo(sc, hx[i][j], lx[i][j]));
      o.y -= f32_to_f64_bits(scale_hi_lo(sc, hy[i][j], ly[i][j]));
      *dst = o;
    }
}

// Stage 2 for pair blocks of at most 16 x 16, software-pipelined: the raw
// complex128 X rows and FP32 T rows of the next 32 plane waves are copied to
// shared memory asynchronously (cp.async, double-buffered) while the current
// chunk is converted and contracted.  Same arithmetic as k_stage2<16, 16, 1, 1>.
__global__ void __launch_bounds__(256) k_stage2_pipe(Stage2Args a) {
  constexpr int GC = 32;
  __shared__ __align__(16) uint4 Xr[2][16][GC];      // raw FP64 complex
  __shared__ __align__(16) float2 Tr[2][GC][16];     // FP32 complex
  __shared__ float2 Xs[16][GC + 1];                  // converted X of the current chunk
  const int p = s2_pair(a, blockIdx.x);
  const int k = a.k_begin + p / a.nk, kp = p % a.nk;
  const int64_t xp = a.x_transpose_pair ? (int64_t)kp * a.nk + k : (int64_t)p;
  const uint4* X = reinterpret_cast<const uint4*>(a.x) + xp * a.rows_x * a.ng;
  const int64_t trow0 = a.t_row0 + (int64_t)a.slot_of_pair[p] * a.rows_t;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int nchunks = (a.ng + GC - 1) / GC;

  auto prefetch = [&](int c, int buf) {
    const int g0 = c * GC;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = tid + u * 256;            // 16 x 32 X elements
      const int r = i >> 5, g = i & 31;
      const bool ok = r < a.rows_x && g0 + g < a.ng;
      cp_async16(&Xr[buf][r][g], ok ? (const void*)(X + (int64_t)r * a.ng + g0 + g) : (const void*)X, ok);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = tid + u * 256;            // 32 x 16 T elements
      const int g = i >> 4, r = i & 15;
      const bool ok = r < a.rows_t && g0 + g < a.ng;
      const float2* src = a.T + (ok ? (int64_t)(g0 + g) * a.t_ld + trow0 + r : 0);
      cp_async8(&Tr[buf][g][r], src, ok);
    }
    cp_async_commit();
  };

  float hx = 0.f, hy = 0.f, lx = 0.f, ly = 0.f;
  const float tsign = a.conj_t ? -1.f : 1.f;
  const uint32_t xflip = a.conj_x ? 0x80000000u : 0u;
  prefetch(0, 0);
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    if (c + 1 < nchunks) {
      prefetch(c + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = tid + u * 256;
      const int r = i >> 5, g = i & 31;
      const uint4 d = Xr[buf][r][g];
      Xs[r][g] = make_float2(__uint_as_float(f64w_to_f32_bits(d.x, d.y)),
                             __uint_as_float(f64w_to_f32_bits(d.z, d.w) ^ xflip));
    }
    __syncthreads();
#pragma unroll
    for (int g8 = 0; g8 < GC; g8 += 8) {
      float ax = 0.f, ay = 0.f;
#pragma unroll
      for (int g = g8; g < g8 + 8; ++g) {
        const float2 xv = Xs[ty][g];
        const float2 tv = Tr[buf][g][tx];
        const float ty_ = tv.y * tsign;
        ax = fmaf(xv.x, tv.x, ax);
        ax = fmaf(-xv.y, ty_, ax);
        ay = fmaf(xv.x, ty_, ay);
        ay = fmaf(xv.y, tv.x, ay);
      }
      float sv, e;
      two_sum(hx, ax, sv, e);
      hx = sv;
      lx += e;
      two_sum(hy, ay, sv, e);
      hy = sv;
      ly += e;
    }
    __syncthreads();   // the next prefetch overwrites this buffer
  }
  const int rx = ty, rt = tx;
  if (rx >= a.rows_x || rt >= a.rows_t) return;
  const int nv = a.nv, nc = a.nc;
  int vi, ci, vp, cp;
  if (a.mode == S2_RR_CC) {
    vi = rx / nv; vp = rx % nv; ci = rt / nc; cp = rt % nc;
  } else if (a.mode == S2_RR_VV) {
    ci = rx / nc; cp = rx % nc; vi = rt / nv; vp = rt % nv;
  } else {
    vp = rx / nc; ci = rx % nc; vi = rt / nc; cp = rt % nc;
  }
  const int64_t al = ((int64_t)k * nv + vi) * nc + ci;
  const int64_t ap = ((int64_t)kp * nv + vp) * nc + cp;
  double2* dst = a.out + al + ap * a.ld;
  const float sc = (float)a.scale;
  double2 o = *dst;
  o.x -= f32_to_f64_bits(scale_hi_lo(sc, hx, lx));
  o.y -= f32_to_f64_bits(scale_hi_lo(sc, hy, ly));
  *dst = o;
}

// Stage 2 for skinny pair blocks: at most RT rows of T against X rows of 16
// or more (W^rr with 2 core levels: 4 (v, v') rows of T, 400 (c, c') rows of
// X; or 2 conduction bands against 4 to 6 valence bands).  One
// thread per X row, SK_ROWS consecutive rows of the term (running across pair
// blocks, at most SK_PAIRS of them) per block.  The raw complex128 X rows
// stream through shared memory in chunks of SK_GC plane waves (cp.async,
// double-buffered, 128-byte runs per row), each thread converts its own row
// once and contracts it against the T rows of its pair, which every thread of
// the pair reads at the same address.  The work is bound by reading X once.
// Same compensated FP32 arithmetic, in the same order, as k_stage2.
constexpr int SK_ROWS = 128, SK_GC = 8, SK_PAIRS = 9;

template <int RT>
__global__ void __launch_bounds__(SK_ROWS) k_stage2_skinny(Stage2Args a, int64_t total_rows) {
  __shared__ __align__(16) uint4 Xr[2][SK_ROWS][SK_GC + 1];   // +16 B per row: no bank conflicts
  static_assert(SK_GC == 8, "one compensation group of 8 plane waves per chunk");
  __shared__ __align__(16) float2 Tr[2][SK_GC][SK_PAIRS][RT];
  __shared__ int64_t xoff[SK_ROWS];      // first complex of each row in X (-1: past the end)
  __shared__ int64_t toff[SK_PAIRS];     // first T row of each pair of the block
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * SK_ROWS;
  const int rows_x = a.rows_x, nk = a.nk;
  const int p_first = (int)(row0 / rows_x);
  {
    const int64_t R = row0 + tid;
    int64_t off = -1;
    if (R < total_rows) {
      const int i = (int)(R / rows_x), r = (int)(R - (int64_t)i * rows_x);
      const int p = s2_pair(a, i);
      const int k = a.k_begin + p / nk, kp = p % nk;
      const int64_t xp = a.x_transpose_pair ? (int64_t)kp * nk + k : (int64_t)p;
      off = (xp * rows_x + r) * a.ng;
    }
    xoff[tid] = off;
    if (tid < SK_PAIRS) {
      const int64_t i = p_first + tid;
      toff[tid] = i * rows_x < total_rows
                      ? a.t_row0 + (int64_t)a.slot_of_pair[s2_pair(a, (int)i)] * a.rows_t : -1;
    }
  }
  __syncthreads();
  const uint4* X = reinterpret_cast<const uint4*>(a.x);
  const int nchunks = (a.ng + SK_GC - 1) / SK_GC;
  // pair blocks this block's rows touch (at most SK_PAIRS)
  const int64_t row_last = (row0 + SK_ROWS < total_rows ? row0 + SK_ROWS : total_rows) - 1;
  const int npp = (int)(row_last / rows_x) - p_first + 1;
  auto prefetch = [&](int c, int buf) {
    const int g0 = c * SK_GC;
#pragma unroll
    for (int u = 0; u < SK_GC; ++u) {   // SK_GC threads per row, 16 B each
      const int i = tid + u * SK_ROWS;
      const int r = i / SK_GC, g = i % SK_GC;
      const int64_t off = xoff[r];
      const bool ok = off >= 0 && g0 + g < a.ng;
      cp_async16(&Xr[buf][r][g], ok ? (const void*)(X + off + g0 + g) : (const void*)X, ok);
    }
    for (int i = tid; i < SK_GC * npp * RT; i += SK_ROWS) {
      const int g = i / (npp * RT), q = (i / RT) % npp, rt = i % RT;
      const bool ok = toff[q] >= 0 && rt < a.rows_t && g0 + g < a.ng;
      const float2* src = a.T + (ok ? (int64_t)(g0 + g) * a.t_ld + toff[q] + rt : 0);
      cp_async8(&Tr[buf][g][q][rt], src, ok);
    }
    cp_async_commit();
  };

  const int64_t R = row0 + tid;
  const int q = (int)(R / rows_x) - p_first;   // this thread's pair within the block
  const uint32_t xflip = a.conj_x ? 0x80000000u : 0u;
  const float tsign = a.conj_t ? -1.f : 1.f;
  float hx[RT], hy[RT], lx[RT], ly[RT];
#pragma unroll
  for (int j = 0; j < RT; ++j) hx[j] = hy[j] = lx[j] = ly[j] = 0.f;
  prefetch(0, 0);
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    if (c + 1 < nchunks) {
      prefetch(c + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int g8 = 0; g8 < SK_GC; g8 += 8) {
      float accx[RT], accy[RT];
#pragma unroll
      for (int j = 0; j < RT; ++j) accx[j] = accy[j] = 0.f;
#pragma unroll
      for (int g = g8; g < g8 + 8; ++g) {
        const uint4 d = Xr[buf][tid][g];
        const float2 xv = make_float2(__uint_as_float(f64w_to_f32_bits(d.x, d.y)),
                                      __uint_as_float(f64w_to_f32_bits(d.z, d.w) ^ xflip));
#pragma unroll
        for (int j = 0; j < RT; ++j) {
          const float2 tv = Tr[buf][g][q < 0 ? 0 : q][j];
          const float ty_ = tv.y * tsign;
          accx[j] = fmaf(xv.x, tv.x, accx[j]);
          accx[j] = fmaf(-xv.y, ty_, accx[j]);
          accy[j] = fmaf(xv.x, ty_, accy[j]);
          accy[j] = fmaf(xv.y, tv.x, accy[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < RT; ++j) {
        float sv, e;
        two_sum(hx[j], accx[j], sv, e);
        hx[j] = sv;
        lx[j] += e;
        two_sum(hy[j], accy[j], sv, e);
        hy[j] = sv;
        ly[j] += e;
      }
    }
    __syncthreads();   // the next prefetch overwrites this buffer
  }
  if (R >= total_rows) return;
  const int i = (int)(R / rows_x), rx = (int)(R - (int64_t)i * rows_x);
  const int p = s2_pair(a, i);
  const int k = a.k_begin + p / nk, kp = p % nk;
  const int nv = a.nv, nc = a.nc;
  const float sc = (float)a.scale;
#pragma unroll
  for (int j = 0; j < RT; ++j) {
    const int rt = j;
    if (rt >= a.rows_t) break;
    int vi, ci, vp, cp;
    if (a.mode == S2_RR_CC) {
      vi = rx / nv; vp = rx % nv; ci = rt / nc; cp = rt % nc;
    } else if (a.mode == S2_RR_VV) {
      ci = rx / nc; cp = rx % nc; vi = rt / nv; vp = rt % nv;
    } else {
      vp = rx / nc; ci = rx % nc; vi = rt / nc; cp = rt % nc;
    }
    const int64_t al = ((int64_t)k * nv + vi) * nc + ci;
    const int64_t ap = ((int64_t)kp * nv + vp) * nc + cp;
    double2* dst = a.out + al + ap * a.ld;
    double2 o = *dst;
    o.x -= f32_to_f64_bits(scale_hi_lo(sc, hx[j], lx[j]));
    o.y -= f32_to_f64_bits(scale_hi_lo(sc, hy[j], ly[j]));
    *dst = o;
  }
}

// true when k_stage2_skinny serves the term: T rows fit the register tile and
// a block's SK_ROWS rows touch at most SK_PAIRS pair blocks
// (rows_t is Nv^2 or Nc^2 there, so at most 4 when skinny; X rows >= 16)
bool stage2_skinny(const Stage2Args& a) {
  return a.rows_t <= 4 && (SK_ROWS - 1 + a.rows_x - 1) / a.rows_x + 1 <= SK_PAIRS;
}

// one pair block per grid.x, tiles of TX x TT outputs over grid.y / grid.z
template <int TX, int TT, int RX, int RT>
void launch_stage2_tiles(const Stage2Args& a, int npair, cudaStream_t s) {
  dim3 grid(npair, (a.rows_x + TX - 1) / TX, (a.rows_t + TT - 1) / TT);
  k_stage2<TX, TT, RX, RT><<<grid, (TX / RX) * (TT / RT), 0, s>>>(a);
}

// Stage 2 for several small pair blocks per thread block (e.g. 4 x 4 for
// 2 x 2 band windows, 6 x 6, 9 x 4): PB pair blocks of rows_x x rows_t
// outputs, one output per thread, so that the 256 threads stay busy where the
// one-pair kernel would leave most of them idle.  The raw complex128 X rows
// and FP32 T rows of the next 8 plane waves of all PB pairs are copied by
// cp.async (double buffered) while the current chunk is contracted.  Same
// compensated FP32 arithmetic, in the same order, as k_stage2.
constexpr int MP_ROWS = 64, MP_GC = 8, MP_MAXPB = 16;

// pair blocks per thread block for the multi-pair kernel (1: not worth it)
int stage2_multi_pairs(const Stage2Args& a) {
  const int rx = a.rows_x, rt = a.rows_t;
  if (rx > 16 || rt > 16) return 1;
  int pb = std::min(MP_MAXPB, 256 / (rx * rt));
  pb = std::min(pb, std::min(MP_ROWS / rx, MP_ROWS / rt));
  return std::max(pb, 1);
}

__global__ void __launch_bounds__(256) k_stage2_multi(Stage2Args a, int npair, int pb) {
  __shared__ __align__(16) uint4 Xr[2][MP_ROWS][MP_GC];     // raw FP64 complex
  __shared__ __align__(16) float2 Tr[2][MP_GC][MP_ROWS];    // FP32 complex
  __shared__ float2 Xs[MP_ROWS][MP_GC + 1];                 // converted X of the chunk
  __shared__ int64_t xbase[MP_MAXPB], tbase[MP_MAXPB];      // -1: no such pair
  const int tid = threadIdx.x;
  const int rx_n = a.rows_x, rt_n = a.rows_t, per = rx_n * rt_n;
  const int p0 = blockIdx.x * pb;
  if (tid < pb) {
    int64_t xb = -1, tb = -1;
    if (p0 + tid < npair) {
      const int p = s2_pair(a, p0 + tid);
      const int k = a.k_begin + p / a.nk, kp = p % a.nk;
      const int64_t xp = a.x_transpose_pair ? (int64_t)kp * a.nk + k : (int64_t)p;
      xb = xp * rx_n * a.ng;
      tb = a.t_row0 + (int64_t)a.slot_of_pair[p] * rt_n;
    }
    xbase[tid] = xb;
    tbase[tid] = tb;
  }
  __syncthreads();
  const uint4* X = reinterpret_cast<const uint4*>(a.x);
  const int xrows = pb * rx_n, trows = pb * rt_n;
  const int nchunks = (a.ng + MP_GC - 1) / MP_GC;
  auto prefetch = [&](int c, int buf) {
    const int g0 = c * MP_GC;
    for (int i = tid; i < xrows * MP_GC; i += 256) {
      const int r = i / MP_GC, g = i % MP_GC;
      const int q = r / rx_n;
      const int64_t xb = xbase[q];
      const bool ok = xb >= 0 && g0 + g < a.ng;
      cp_async16(&Xr[buf][r][g],
                 ok ? (const void*)(X + xb + (int64_t)(r - q * rx_n) * a.ng + g0 + g) : (const void*)X,
                 ok);
    }
    for (int i = tid; i < MP_GC * trows; i += 256) {
      const int g = i / trows, r = i % trows;
      const int q = r / rt_n;
      const int64_t tb = tbase[q];
      const bool ok = tb >= 0 && g0 + g < a.ng;
      const float2* src = a.T + (ok ? (int64_t)(g0 + g) * a.t_ld + tb + (r - q * rt_n) : 0);
      cp_async8(&Tr[buf][g][r], src, ok);
    }
    cp_async_commit();
  };

  const int q = tid / per, o = tid - q * per;
  const int ri = o / rt_n, rj = o - ri * rt_n;
  const bool active = q < pb;
  const int xrow = active ? q * rx_n + ri : 0, trow = active ? q * rt_n + rj : 0;
  const uint32_t xflip = a.conj_x ? 0x80000000u : 0u;
  const float tsign = a.conj_t ? -1.f : 1.f;
  float hx = 0.f, hy = 0.f, lx = 0.f, ly = 0.f;
  prefetch(0, 0);
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    if (c + 1 < nchunks) {
      prefetch(c + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    for (int i = tid; i < xrows * MP_GC; i += 256) {
      const int r = i / MP_GC, g = i % MP_GC;
      const uint4 d = Xr[buf][r][g];
      Xs[r][g] = make_float2(__uint_as_float(f64w_to_f32_bits(d.x, d.y)),
                             __uint_as_float(f64w_to_f32_bits(d.z, d.w) ^ xflip));
    }
    __syncthreads();
    float ax = 0.f, ay = 0.f;
#pragma unroll
    for (int g = 0; g < MP_GC; ++g) {
      const float2 xv = Xs[xrow][g];
      const float2 tv = Tr[buf][g][trow];
      const float ty_ = tv.y * tsign;
      ax = fmaf(xv.x, tv.x, ax);
      ax = fmaf(-xv.y, ty_, ax);
      ay = fmaf(xv.x, ty_, ay);
      ay = fmaf(xv.y, tv.x, ay);
    }
    float sv, e;
    two_sum(hx, ax, sv, e);
    hx = sv;
    lx += e;
    two_sum(hy, ay, sv, e);
    hy = sv;
    ly += e;
    __syncthreads();   // the next prefetch overwrites this buffer
  }
  if (!active || xbase[q] < 0) return;
  const int p = s2_pair(a, p0 + q);
  const int k = a.k_begin + p / a.nk, kp = p % a.nk;
  const int nv = a.nv, nc = a.nc, rx = ri, rt = rj;
  int vi, ci, vp, cp;
  if (a.mode == S2_RR_CC) {
    vi = rx / nv; vp = rx % nv; ci = rt / nc; cp = rt % nc;
  } else if (a.mode == S2_RR_VV) {
    ci = rx / nc; cp = rx % nc; vi = rt / nv; vp = rt % nv;
  } else {
    vp = rx / nc; ci = rx % nc; vi = rt / nc; cp = rt % nc;
  }
  const int64_t al = ((int64_t)k * nv + vi) * nc + ci;
  const int64_t ap = ((int64_t)kp * nv + vp) * nc + cp;
  double2* dst = a.out + al + ap * a.ld;
  const float sc = (float)a.scale;
  double2 o2 = *dst;
  o2.x -= f32_to_f64_bits(scale_hi_lo(sc, hx, lx));
  o2.y -= f32_to_f64_bits(scale_hi_lo(sc, hy, ly));
  *dst = o2;
}

// The kernel whose tile fits the pair block best (every variant adds in the
// same order: the results do not depend on the choice).
void launch_stage2(const Stage2Args& a, int npair, cudaStream_t s) {
  if (stage2_skinny(a)) {
    const int64_t total = (int64_t)npair * a.rows_x;
    const int64_t blocks = (total + SK_ROWS - 1) / SK_ROWS;
    k_stage2_skinny<4><<<(unsigned)blocks, SK_ROWS, 0, s>>>(a, total);
  } else if (a.rows_x <= 16 && a.rows_t <= 16) {
    const int pb = stage2_multi_pairs(a);
    if (pb >= 2)
      k_stage2_multi<<<(npair + pb - 1) / pb, 256, 0, s>>>(a, npair, pb);
    else
      k_stage2_pipe<<<npair, 256, 0, s>>>(a);
  } else if (a.rows_x <= 24 && a.rows_t <= 24) {           // e.g. W^ra, 4 x 6 bands
    launch_stage2_tiles<24, 24, 2, 3>(a, npair, s);
  } else if (a.rows_x <= 32 && a.rows_t <= 16) {           // e.g. W^rr, 3 x 5 bands (25 x 9)
    launch_stage2_tiles<32, 16, 2, 2>(a, npair, s);
  } else if (a.rows_x <= 40 && a.rows_t <= 16) {           // e.g. W^rr, 4 x 6 bands (36 x 16)
    launch_stage2_tiles<40, 16, 2, 2>(a, npair, s);
  } else if (a.rows_x <= 40 && a.rows_t <= 40) {           // e.g. W^ra, 2 x 20 bands (40 x 40)
    launch_stage2_tiles<40, 40, 2, 5>(a, npair, s);
  } else {
    launch_stage2_tiles<32, 32, 2, 2>(a, npair, s);
  }
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
}

// ---------------------------------------------------------------------------
// tensor maps and the GEMM launcher
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  if (!fn) throw Error(BSE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  return fn;
}

// 3-D map over planes [planes][rows][Kp] of BF16, box {16, box_rows, planes}, 32-byte swizzle.
CUtensorMap make_plane_map(const __nv_bfloat16* base, int Kp, int rows, int planes, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * rows};
  cuuint32_t box[3] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows, (cuuint32_t)planes};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw Error(BSE_ERR_CUDA, "cuTensorMapEncodeTiled failed with " + std::to_string((int)r));
  return m;
}

int num_sms() {
  int dev = 0, n = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  BSE_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  return n;
}

// d_err: two ints, the error bits and the counter of the dynamic unit hand-out
template <class Epi>
void launch_gemm(const CUtensorMap& ma, const CUtensorMap& mb, const tc::Tile* d_tiles, int ntiles,
                 const tc::GemmShape& sh, const Epi& epi, int* d_err, cudaStream_t s) {
  if (ntiles == 0) return;
  const size_t smem = tc::gemm_smem_bytes(sh);
  const bool seg = sh.ksegs > 1;
  if (seg && (sh.nt > 64 || sh.acc_bufs != 2))
    throw Error(BSE_ERR_UNSUPPORTED, "K-segmented tiles need two accumulator sets of <= 64 columns");
  const int which = (sh.pieces == 3 ? 2 : 0) + (seg ? 1 : 0);
  void (*const kerns[4])(CUtensorMap, CUtensorMap, const tc::Tile*, int, tc::GemmShape, Epi, int*,
                         int*) = {
      tc::gemm_split_bf16<2, Epi, false>, tc::gemm_split_bf16<2, Epi, true>,
      tc::gemm_split_bf16<3, Epi, false>, tc::gemm_split_bf16<3, Epi, true>};
  auto kern = kerns[which];
  // the shared-memory opt-in is set once per kernel (not per launch, so that a
  // launch can be captured in a CUDA graph)
  static std::once_flag once[4];
  static int max_dyn[4] = {0, 0, 0, 0};
  std::call_once(once[which], [&] {
    int dev = 0, optin = 0;
    BSE_CUDA(cudaGetDevice(&dev));
    BSE_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    BSE_CUDA(cudaFuncGetAttributes(&fa, kern));
    max_dyn[which] = optin - (int)fa.sharedSizeBytes;
    BSE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn[which]));
  });
  if ((int)smem > max_dyn[which]) throw Error(BSE_ERR_UNSUPPORTED, "tile shape needs too much shared memory");
  const int units = (ntiles + sh.group - 1) / sh.group;
  const int grid = std::min<int>(units, num_sms());
  int* units_taken = nullptr;
  if (units > grid) {   // more than one round of units: hand them out in order of need
    units_taken = d_err + 1;
    BSE_CUDA(cudaMemsetAsync(units_taken, 0, sizeof(int), s));
  }
  kern<<<grid, tc::NUM_THREADS, smem, s>>>(ma, mb, d_tiles, ntiles, sh, epi, d_err, units_taken);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
}

// stage 1 + stage 2 in one launch; a work unit is one 128-row tile with all
// its output-column tiles (sh.group of them, consecutive in d_tiles)
void launch_direct(const CUtensorMap& ma, const CUtensorMap& mb, const tc::Tile* d_tiles,
                   int ntiles, const tc::GemmShape& sh, const tc::S2Term* d_terms, int* d_err,
                   cudaStream_t s) {
  if (ntiles == 0) return;
  if (sh.acc_bufs != 2 || sh.group < 1)
    throw Error(BSE_ERR_UNSUPPORTED, "fused direct term needs two accumulator sets");
  const size_t smem = tc::s2_smem_bytes(sh);
  auto kern = sh.pieces == 3 ? tc::gemm_split_bf16_direct<3> : tc::gemm_split_bf16_direct<2>;
  static std::once_flag once3, once2;
  static int max_dyn3 = 0, max_dyn2 = 0;
  int& max_dyn = sh.pieces == 3 ? max_dyn3 : max_dyn2;
  std::call_once(sh.pieces == 3 ? once3 : once2, [&] {
    int dev = 0, optin = 0;
    BSE_CUDA(cudaGetDevice(&dev));
    BSE_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    BSE_CUDA(cudaFuncGetAttributes(&fa, kern));
    max_dyn = optin - (int)fa.sharedSizeBytes;
    BSE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn));
  });
  if ((int)smem > max_dyn) throw Error(BSE_ERR_UNSUPPORTED, "tile shape needs too much shared memory");
  const int units = (ntiles + sh.group - 1) / sh.group;
  const int grid = std::min<int>(units, num_sms());
  kern<<<grid, tc::S2_THREADS, smem, s>>>(ma, mb, d_tiles, ntiles, sh, d_terms, d_err);
  BSE_CUDA(cudaGetLastError());
  note_launches(1);
}

// K segments of a tile: one segment up to `whole` K steps, else segments of at
// most `seg` steps, summed in the epilogue (bounds the number of accumulate
// events any TMEM accumulator sees).  Default: whole up to 12 steps (192 plane
// waves), segments of 8.
int ksegs_for(int Kp, int seg = 8, int whole = 12) {
  const int kchunks = Kp / tc::BK;
  return kchunks <= whole ? 1 : (kchunks + seg - 1) / seg;
}

tc::GemmShape make_shape(int nt, int Kp, int pieces, int seg = 8, int whole = 12) {
  tc::GemmShape sh;
  sh.nt = nt;
  sh.kchunks = Kp / tc::BK;
  sh.pieces = pieces;
  sh.ksegs = ksegs_for(Kp, seg, whole);
  if (sh.ksegs > 1 && nt > 64)
    throw Error(BSE_ERR_UNSUPPORTED, "K-segmented tiles need at most 64 output columns");
  sh.acc_bufs = 8 * nt <= 512 ? 2 : 1;
  const int cols = 4 * nt * sh.acc_bufs;
  sh.tmem_cols = cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
  const uint32_t sb = tc::stage_bytes(sh);
  const size_t budget = 220 * 1024;
  int st = (int)((budget - 2048) / sb);
  sh.stages = std::max(1, std::min(st, 6));
  return sh;
}

// Shape of the fused direct-term launch: nt <= 64 so that two accumulator
// sets fit TMEM (the contraction of one column tile overlaps the MMAs of the
// next), and the pipeline depth reduced to leave room for the pair-side ring.
tc::GemmShape make_shape_direct(int nt, int Kp, int pieces, int group) {
  tc::GemmShape sh = make_shape(nt, Kp, pieces);
  if (sh.ksegs != 1) throw Error(BSE_ERR_UNSUPPORTED, "the fused direct term takes whole-K tiles");
  sh.acc_bufs = 2;
  sh.tmem_cols = 8 * nt <= 256 ? 256 : 512;
  sh.group = group;
  const uint32_t sb = tc::stage_bytes(sh);
  const size_t budget = 220 * 1024 - 2048 - tc::s2_extra_bytes(6);
  sh.stages = std::max(1, std::min((int)(budget / sb), 6));
  return sh;
}

// Largest output-column tile (multiple of 32, <= 128).  Tiles of <= 64 columns
// leave room for two accumulator sets in TMEM (epilogue overlapped with the
// next tile's MMAs); wider tiles read shared memory more efficiently.  The
// environment variable BSE_TC_NT_MAX overrides the default for tuning.
int nt_max() {
  const char* e = getenv("BSE_TC_NT_MAX");
  int v = e ? atoi(e) : 128;
  if (v != 32 && v != 64 && v != 96 && v != 128) v = 128;
  return v;
}

// output columns per tile: the padded N split into equal multiples of 32, each
// <= nt_max() (<= 64 when the K range is segmented)
int tile_cols(int n_pad, int Kp, int seg = 8, int whole = 12) {
  const int mx = ksegs_for(Kp, seg, whole) > 1 ? std::min(64, nt_max()) : nt_max();
  int ntiles = (n_pad + mx - 1) / mx;
  return round_up((n_pad + ntiles - 1) / ntiles, 32);
}

// Pairs sorted by q (stable in pair order); returns perm (slot -> pair) and group bounds.
void group_pairs(const std::vector<int32_t>& qmap, int nq, std::vector<int>& perm,
                 std::vector<int>& group_start) {
  const int npair = (int)qmap.size();
  std::vector<int> count(nq + 1, 0);
  for (int p = 0; p < npair; ++p) count[qmap[p] + 1]++;
  for (int q = 0; q < nq; ++q) count[q + 1] += count[q];
  group_start = count;
  perm.assign(npair, 0);
  std::vector<int> fill(count.begin(), count.end() - 1);
  for (int p = 0; p < npair; ++p) perm[fill[qmap[p]]++] = p;
}

uint64_t fnv1a(const std::vector<int32_t>& v, uint64_t h = 1469598103934665603ull) {
  for (int32_t x : v) {
    h ^= (uint32_t)x;
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

// ===========================================================================
// Batched plans: many momentum transfers prepared once, then built with
// launches only (no allocation, no host synchronisation), so that a build can
// be captured in a CUDA graph.  All problems' exchange tiles share one
// persistent tensor-core launch, and all direct terms' stage-1 tiles another.
// ===========================================================================
namespace {

struct DevMem {
  void* ptr = nullptr;
  DevMem() = default;
  explicit DevMem(size_t n) {
    if (n && cudaMalloc(&ptr, n) != cudaSuccess) {
      (void)cudaGetLastError();
      throw Error(BSE_ERR_NOMEM, "cudaMalloc of " + std::to_string(n) + " bytes failed");
    }
  }
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  DevMem(DevMem&& o) noexcept : ptr(o.ptr) { o.ptr = nullptr; }
  DevMem& operator=(DevMem&& o) noexcept {
    std::swap(ptr, o.ptr);
    return *this;
  }
  ~DevMem() {
    if (ptr) cudaFree(ptr);
  }
  template <class T>
  T* as() const { return static_cast<T*>(ptr); }
};

template <class T>
DevMem upload_mem(const std::vector<T>& v) {
  DevMem m(v.size() * sizeof(T));
  if (!v.empty()) BSE_CUDA(cudaMemcpy(m.ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return m;
}

struct ExParams {
  double2 *A, *B;
  int64_t ld;
  float scale;
  const double *e_v, *e_c;
  int nv, nc;
  int upper;      // the blocks k <= k' only (see ExchangeEpi)
};

struct ExchangeBatchEpi {   // ExchangeEpi with per-problem outputs
  const ExParams* params;
  __device__ __forceinline__ void operator()(const tc::Tile& t, int row, int c0, const float* re,
                                             const float* im) const {
    const ExParams q = params[t.prob];
    ExchangeEpi e{q.A, q.B, q.ld, q.scale, q.e_v, q.e_c, q.nv, q.nc, q.upper};
    e(t, row, c0, re, im);
  }
};

// process-wide autotuning results: padded NG -> best output-column tile width
std::mutex g_tune_mutex;
std::map<int, int> g_tuned_nt;
std::map<int64_t, std::pair<int, int>> g_tuned_s2;   // stage-2 (tile width, depth)

}  // namespace

struct BatchPlan {
  int precision = 0, pieces = 3, planes = 6, ng = 0, Kp = 0, ng_pad = 0, nt_x = 0, nt_g = 0;
  int device = 0;
  std::mutex use_mutex;   // held by bse_build_kernel through a cached plan's execute and status
  long long wait = tc::WAIT_CYCLES;   // clock budget of each pipeline wait in its GEMM launches
  std::vector<Problem> probs;
  // Hermitian build (BSE_PLAN_HERMITIAN): direct terms over the blocks k <= k'
  // only, the blocks k > k' of A and B completed from their mirrors
  bool half = false;
  std::vector<int> upper_probs;   // problems whose exchange wrote the blocks k <= k' only
  // BSE_PLAN_FP64_DIAGONAL: the diagonal of A and B recomputed in FP64 after the build
  std::vector<DevMem> diag_ws;
  // exchange
  int64_t x_rows = 0;
  std::vector<int64_t> x_row0;
  DevMem xa, xb, xtiles, exparams;
  int n_xtiles = 0;
  tc::GemmShape sh_x{}, sh_g{};
  CUtensorMap ma_x{}, mb_x{}, ma_s{}, mb_s{};
  // direct terms
  struct Term {
    int prob = 0;
    int64_t a_row0 = 0, w_row0 = 0;
    bool w_owner = true;     // this term splits its W planes (false: shares the other term's)
    int rows_side = 0;
    const bse_c128* side = nullptr;
    bool w_conj_transpose = false;
    DevMem perm, slot;
    Stage2Args s2{};
    std::vector<int32_t> qh;   // q index of each pair built, in pair-list order
    std::vector<int> act_h;    // the pairs built: every pair of the slab, or k <= k'
    std::vector<int> slot_h;   // pair -> stage-1 slot (-1: not built)
    DevMem act;
    int nact = 0;
    // stage 2 on the tensor cores (large pair blocks)
    bool tc2 = false;
    bool rows_t_side = false;   // stage-2 tile rows are the T side (W^rr with T on (c, c'))
    int side_nb = 0, x_nb = 0;  // (b, b') rows stored (b', b) in the stage-1 side / x2 planes
    int64_t x2_row0 = 0;     // first row of this term's pair side in its x2 array
    int64_t t_row0 = 0;      // first row of this term's T in its T array
    DevMem x2perm;           // pair -> pair whose side rows are read (identity, or (k', k))
  };
  std::vector<Term> terms;
  int64_t a_rows = 0, w_rows = 0;
  DevMem wsplit, asplit, tbuf, stiles;
  int n_stiles = 0;
  // stage 2 on the tensor cores for terms with large pair blocks: T and the
  // other pair side in the layout of their operand role (A: 2P planes, B: 3P)
  int64_t ta_rows = 0, tb_rows = 0, x2a_rows = 0, x2b_rows = 0;
  DevMem ta, tb, x2a, x2b, touts, s2tiles, s2tiles_t, s2params;
  int n_s2tiles = 0, n_s2tiles_t = 0, nt2 = 0, s2_stages = 0, s2_max_cols = 0;
  tc::GemmShape sh_2{};
  CUtensorMap ma_2{}, mb_2{}, ma_2t{}, mb_2t{};   // rows = X side / rows = T side
  // fused direct term (stage 1 + stage 2 in one launch)
  bool fused = false;
  std::vector<tc::S2Term> s2host;
  DevMem s2terms, xmaps;
  DevMem err;
};

namespace {

// Stage-1 tiles, 128-row tile by 128-row tile with all its column tiles
// consecutive; Tile::prob is the direct term (whose output the epilogue
// writes: FP32 T, T split planes, or the fused contraction).
std::vector<tc::Tile> stage1_tiles(const BatchPlan& pl, int nt) {
  std::vector<tc::Tile> tiles;
  for (size_t ti = 0; ti < pl.terms.size(); ++ti) {
    const BatchPlan::Term& t = pl.terms[ti];
    const int id = (int)ti;
    const int nq = pl.probs[t.prob].p.nq_w;
    std::vector<int> perm, gstart;
    group_pairs(t.qh, nq, perm, gstart);
    for (int q = 0; q < nq; ++q) {
      const int64_t r0 = t.a_row0 + (int64_t)gstart[q] * t.rows_side;
      const int64_t r1 = t.a_row0 + (int64_t)gstart[q + 1] * t.rows_side;
      for (int64_t m0 = r0; m0 < r1; m0 += tc::BM)
        for (int n0 = 0; n0 < pl.ng; n0 += nt)
          tiles.push_back({(int)m0, (int)std::min<int64_t>(tc::BM, r1 - m0),
                           (int)(t.w_row0 + (int64_t)q * pl.ng_pad + n0), n0,
                           std::min(nt, pl.ng - n0), (int)m0, id});
    }
  }
  return tiles;
}

void plan_splits(BatchPlan& pl, cudaStream_t s) {
  for (size_t i = 0; i < pl.probs.size(); ++i) {
    const bse_problem& p = pl.probs[i].p;
    const int n = (int)pl.probs[i].n;
    SplitArgs sa{reinterpret_cast<const double2*>(p.m_x), SPLIT_DENSE, nullptr, 0, 0, pl.ng,
                 pl.Kp, n, pl.pieces, 1, p.v_bar, pl.xa.as<__nv_bfloat16>(), pl.x_rows,
                 pl.x_row0[i]};
    sa.c64 = p.in_dtype == BSE_C64;
    launch_split(sa, s);
    SplitArgs sb = sa;
    sb.conj = 0;
    sb.kscale = nullptr;
    sb.out = pl.xb.as<__nv_bfloat16>();
    sb.bneg = 1;
    launch_split(sb, s);
  }
  for (BatchPlan::Term& t : pl.terms) {
    const bse_problem& p = pl.probs[t.prob].p;
    const int npair = t.nact;
    SplitArgs sw{reinterpret_cast<const double2*>(p.w), SPLIT_W, nullptr, pl.ng_pad,
                 t.w_conj_transpose ? 1 : 0, pl.ng, pl.Kp, p.nq_w * pl.ng_pad, pl.pieces,
                 t.w_conj_transpose ? 1 : 0, nullptr, pl.wsplit.as<__nv_bfloat16>(), pl.w_rows,
                 t.w_row0};
    sw.bneg = 1;
    sw.c64 = p.in_dtype == BSE_C64;
    if (t.w_owner) launch_split(sw, s);
    SplitArgs sa{reinterpret_cast<const double2*>(t.side), SPLIT_PAIRS, t.perm.as<int>(),
                 t.rows_side, 0, pl.ng, pl.Kp, npair * t.rows_side, pl.pieces, 0, nullptr,
                 pl.asplit.as<__nv_bfloat16>(), pl.a_rows, t.a_row0};
    sa.pair_nb = t.side_nb;
    sa.c64 = p.in_dtype == BSE_C64;
    launch_split(sa, s);
    if (t.tc2) {   // the other pair side, in pair order, conjugated as opX
      SplitArgs sx{t.s2.x, SPLIT_PAIRS, t.x2perm.as<int>(), t.s2.rows_x, 0, pl.ng, pl.Kp,
                   npair * t.s2.rows_x, pl.pieces, t.s2.conj_x, nullptr,
                   (t.rows_t_side ? pl.x2b : pl.x2a).as<__nv_bfloat16>(),
                   t.rows_t_side ? pl.x2b_rows : pl.x2a_rows, t.x2_row0};
      sx.pair_nb = t.x_nb;
      sx.bneg = t.rows_t_side ? 1 : 0;   // the B operand when T forms the tile rows
      sx.c64 = p.in_dtype == BSE_C64;
      launch_split(sx, s);
    }
  }
}

// blocks k > k' of A and B from their mirrors, for the problems whose
// exchange wrote only the blocks k <= k' (or every problem of a Hermitian plan)
void plan_complete(BatchPlan& pl, bool all, cudaStream_t s) {
  Phase ph("hermitian_complete", s);
  for (size_t i = 0; i < pl.probs.size(); ++i) {
    if (!all && std::find(pl.upper_probs.begin(), pl.upper_probs.end(), (int)i) == pl.upper_probs.end())
      continue;
    const bse_problem& p = pl.probs[i].p;
    const int n = (int)pl.probs[i].n, nb = p.nv * p.nc;
    launch_hermitian_complete(reinterpret_cast<double2*>(p.A), p.ld, n, nb, s);
    if (p.coupling) launch_hermitian_complete(reinterpret_cast<double2*>(p.B), p.ld, n, nb, s);
  }
}

void plan_execute_mixed(BatchPlan& pl, cudaStream_t s) {
  // (the status word is cleared at creation and by plan_status, not here: a
  // timeout in any execute since the last status call stays visible)
  pl.sh_x.wait = pl.sh_g.wait = pl.sh_2.wait = pl.wait;
  {
    Phase ph("mixed_split", s);
    plan_splits(pl, s);
  }
  {
    Phase ph("mixed_exchange", s);
    launch_gemm(pl.ma_x, pl.mb_x, pl.xtiles.as<tc::Tile>(), pl.n_xtiles, pl.sh_x,
                ExchangeBatchEpi{pl.exparams.as<ExParams>()}, pl.err.as<int>(), s);
  }
  // every block of A and B holds its exchange part before the direct terms
  // subtract from it, unless those run over the blocks k <= k' alone
  if (!pl.half && !pl.upper_probs.empty()) plan_complete(pl, false, s);
  if (!pl.terms.empty()) {
    if (pl.fused) {
      Phase ph("mixed_direct_fused", s);
      launch_direct(pl.ma_s, pl.mb_s, pl.stiles.as<tc::Tile>(), pl.n_stiles, pl.sh_g,
                    pl.s2terms.as<tc::S2Term>(), pl.err.as<int>(), s);
    } else {
      {
        Phase ph("mixed_stage1_gemm", s);
        launch_gemm(pl.ma_s, pl.mb_s, pl.stiles.as<tc::Tile>(), pl.n_stiles, pl.sh_g,
                    TEpiMulti{pl.touts.as<TOut>()}, pl.err.as<int>(), s);
      }
      bool any_cuda_core = false;
      for (const BatchPlan::Term& t : pl.terms) any_cuda_core = any_cuda_core || !t.tc2;
      if (any_cuda_core) {
        Phase ph("mixed_stage2", s);
        for (BatchPlan::Term& t : pl.terms) {
          if (t.tc2) continue;
          Phase pt(t.s2.mode == S2_RA ? "mixed_stage2_wra" : "mixed_stage2_wrr", s);
          launch_stage2(t.s2, t.nact, s);
        }
      }
      if (pl.n_s2tiles || pl.n_s2tiles_t) {
        Phase ph("mixed_stage2_tc", s);
        if (pl.n_s2tiles)
          launch_gemm(pl.ma_2, pl.mb_2, pl.s2tiles.as<tc::Tile>(), pl.n_s2tiles, pl.sh_2,
                      S2TcEpi{pl.s2params.as<S2TcParams>()}, pl.err.as<int>(), s);
        if (pl.n_s2tiles_t)
          launch_gemm(pl.ma_2t, pl.mb_2t, pl.s2tiles_t.as<tc::Tile>(), pl.n_s2tiles_t, pl.sh_2,
                      S2TcEpi{pl.s2params.as<S2TcParams>()}, pl.err.as<int>(), s);
      }
    }
  }
  if (pl.half) plan_complete(pl, true, s);
  if (!pl.diag_ws.empty()) {
    Phase ph("fp64_diagonal", s);
    for (size_t i = 0; i < pl.probs.size(); ++i)
      diag_fp64(pl.probs[i], pl.diag_ws[i].as<bse_c128>(), s);
  }
}

// Tensor-core stage 2: products feed A and B directly, K segments of at most
// 8 steps (at NG = 500, 4-, 8- and 16-step segments give A and B within
// 3.41e-7, 3.42e-7 and 3.43e-7 of the FP64 build; 8 is 6 % faster than 4).
int s2_default_cols(const BatchPlan& pl) {
  return tile_cols(round_up(pl.s2_max_cols, 32), pl.Kp, 8, 8);
}

// The tensor-core stage-2 tiles at nt2 output columns per tile (the pair
// blocks' tiles in pair order), pipeline depth stages (0: the deepest that
// fits shared memory).
void plan_set_s2_tiles(BatchPlan& pl, int nt2, int stages) {
  std::vector<tc::Tile> tiles, tiles_t;
  for (size_t ti = 0; ti < pl.terms.size(); ++ti) {
    const BatchPlan::Term& t = pl.terms[ti];
    if (!t.tc2) continue;
    const Stage2Args& a = t.s2;
    for (int j = 0; j < t.nact; ++j) {
      const int pr = t.act_h[j];
      const int64_t xr = t.x2_row0 + (int64_t)j * a.rows_x;            // X rows of the pair
      const int64_t tr = t.t_row0 + (int64_t)t.slot_h[pr] * a.rows_t;  // T rows of the pair
      if (t.rows_t_side) {
        for (int m0 = 0; m0 < a.rows_t; m0 += tc::BM)
          for (int n0 = 0; n0 < a.rows_x; n0 += nt2)
            tiles_t.push_back({(int)(tr + m0), std::min(tc::BM, a.rows_t - m0), (int)(xr + n0), n0,
                               std::min(nt2, a.rows_x - n0), pr * a.rows_t + m0, (int)ti});
      } else {
        for (int m0 = 0; m0 < a.rows_x; m0 += tc::BM)
          for (int n0 = 0; n0 < a.rows_t; n0 += nt2)
            tiles.push_back({(int)(xr + m0), std::min(tc::BM, a.rows_x - m0), (int)(tr + n0), n0,
                             std::min(nt2, a.rows_t - n0), pr * a.rows_x + m0, (int)ti});
      }
    }
  }
  const int ap = tc::a_planes(pl.pieces), bp = tc::b_planes(pl.pieces);
  pl.nt2 = nt2;
  pl.n_s2tiles = (int)tiles.size();
  pl.s2tiles = upload_mem(tiles);
  pl.n_s2tiles_t = (int)tiles_t.size();
  pl.s2tiles_t = upload_mem(tiles_t);
  pl.sh_2 = make_shape(nt2, pl.Kp, pl.pieces, 8, 8);
  if (stages > 0) pl.sh_2.stages = std::min(pl.sh_2.stages, stages);
  pl.s2_stages = pl.sh_2.stages;
  if (pl.n_s2tiles) {
    pl.ma_2 = make_plane_map(pl.x2a.as<__nv_bfloat16>(), pl.Kp, (int)pl.x2a_rows, ap, tc::BM);
    pl.mb_2 = make_plane_map(pl.tb.as<__nv_bfloat16>(), pl.Kp, (int)pl.tb_rows, bp, nt2);
  }
  if (pl.n_s2tiles_t) {
    pl.ma_2t = make_plane_map(pl.ta.as<__nv_bfloat16>(), pl.Kp, (int)pl.ta_rows, ap, tc::BM);
    pl.mb_2t = make_plane_map(pl.x2b.as<__nv_bfloat16>(), pl.Kp, (int)pl.x2b_rows, bp, nt2);
  }
}

void plan_set_tiles(BatchPlan& pl, int nt) {
  pl.nt_g = nt;
  pl.sh_g = pl.fused ? make_shape_direct(nt, pl.Kp, pl.pieces, (pl.ng + nt - 1) / nt)
                     : make_shape(nt, pl.Kp, pl.pieces);
  std::vector<tc::Tile> st = stage1_tiles(pl, nt);
  pl.n_stiles = (int)st.size();
  pl.stiles = upload_mem(st);
  pl.mb_s = make_plane_map(pl.wsplit.as<__nv_bfloat16>(), pl.Kp, (int)pl.w_rows,
                           tc::b_planes(pl.pieces), nt);
}

// time the stage-1 GEMM at each candidate tile width and keep the fastest
void tune_stage1(BatchPlan& pl, cudaStream_t s) {
  const int key = 2 * pl.ng_pad + (pl.fused ? 1 : 0);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned_nt.find(key);
    if (it != g_tuned_nt.end()) {
      plan_set_tiles(pl, it->second);
      return;
    }
  }
  std::vector<int> cands;
  if (pl.fused) {
    cands.push_back(32);
    if (pl.ng_pad >= 64) cands.push_back(64);
  } else {
    for (int mx : {64, 128}) {
      if (mx > 64 && ksegs_for(pl.Kp) > 1) continue;
      int nt = round_up((pl.ng_pad + ((pl.ng_pad + mx - 1) / mx) - 1) / ((pl.ng_pad + mx - 1) / mx), 32);
      if (std::find(cands.begin(), cands.end(), nt) == cands.end()) cands.push_back(nt);
    }
  }
  // the fused launch is timed with its outputs switched off (A and B untouched)
  DevMem timing_terms;
  if (pl.fused) {
    std::vector<tc::S2Term> tt = pl.s2host;
    for (tc::S2Term& x : tt) x.out = nullptr;
    timing_terms = upload_mem(tt);
  }
  plan_splits(pl, s);
  cudaEvent_t e0, e1;
  BSE_CUDA(cudaEventCreate(&e0));
  BSE_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_nt = cands.front();
  for (int nt : cands) {
    plan_set_tiles(pl, nt);
    float ms = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      BSE_CUDA(cudaEventRecord(e0, s));
      if (pl.fused)
        launch_direct(pl.ma_s, pl.mb_s, pl.stiles.as<tc::Tile>(), pl.n_stiles, pl.sh_g,
                      timing_terms.as<tc::S2Term>(), pl.err.as<int>(), s);
      else
        launch_gemm(pl.ma_s, pl.mb_s, pl.stiles.as<tc::Tile>(), pl.n_stiles, pl.sh_g,
                    TEpiMulti{pl.touts.as<TOut>()}, pl.err.as<int>(), s);
      BSE_CUDA(cudaEventRecord(e1, s));
      BSE_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      BSE_CUDA(cudaEventElapsedTime(&t, e0, e1));
      if (rep > 0) ms += t;   // first launch warms up
    }
    if (ms < best) {
      best = ms;
      best_nt = nt;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan_set_tiles(pl, best_nt);
  BSE_CUDA(cudaMemsetAsync(pl.err.ptr, 0, sizeof(int), s));
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned_nt[key] = best_nt;
}

// Time the tensor-core stage-2 launches over the tile widths {default, 32}
// and pipeline depths {deepest, one less}; keep the fastest.  The timed
// launches read the stage-1 output of the tuning above and subtract from the
// blocks of A and B that every execute first stores (exchange), so they leave
// nothing behind that an execute would read.
void tune_stage2(BatchPlan& pl, cudaStream_t s) {
  if (pl.fused || (pl.n_s2tiles == 0 && pl.n_s2tiles_t == 0)) return;
  const int64_t key = ((int64_t)pl.Kp * 4096 + pl.s2_max_cols) * 4 + pl.pieces;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned_s2.find(key);
    if (it != g_tuned_s2.end()) {
      plan_set_s2_tiles(pl, it->second.first, it->second.second);
      return;
    }
  }
  std::vector<std::pair<int, int>> cands;
  const int d2 = s2_default_cols(pl);
  for (int nt2 : {d2, 32}) {
    if (nt2 != d2 && nt2 >= d2) continue;
    const int deep = make_shape(nt2, pl.Kp, pl.pieces, 8, 8).stages;
    cands.push_back({nt2, deep});
    if (deep > 2) cands.push_back({nt2, deep - 1});
  }
  cudaEvent_t e0, e1;
  BSE_CUDA(cudaEventCreate(&e0));
  BSE_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  std::pair<int, int> pick = cands.front();
  for (const auto& c : cands) {
    plan_set_s2_tiles(pl, c.first, c.second);
    float ms = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      BSE_CUDA(cudaEventRecord(e0, s));
      if (pl.n_s2tiles)
        launch_gemm(pl.ma_2, pl.mb_2, pl.s2tiles.as<tc::Tile>(), pl.n_s2tiles, pl.sh_2,
                    S2TcEpi{pl.s2params.as<S2TcParams>()}, pl.err.as<int>(), s);
      if (pl.n_s2tiles_t)
        launch_gemm(pl.ma_2t, pl.mb_2t, pl.s2tiles_t.as<tc::Tile>(), pl.n_s2tiles_t, pl.sh_2,
                    S2TcEpi{pl.s2params.as<S2TcParams>()}, pl.err.as<int>(), s);
      BSE_CUDA(cudaEventRecord(e1, s));
      BSE_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      BSE_CUDA(cudaEventElapsedTime(&t, e0, e1));
      if (rep > 0) ms += t;   // first launch warms up
    }
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan_set_s2_tiles(pl, pick.first, pick.second);
  BSE_CUDA(cudaMemsetAsync(pl.err.ptr, 0, sizeof(int), s));
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned_s2[key] = pick;
}

void plan_autotune(BatchPlan& pl, cudaStream_t s) {
  tune_stage1(pl, s);
  tune_stage2(pl, s);
}

}  // namespace

// True when a term's pair blocks fit the fused epilogue: whole pairs per
// 128-row tile (rows_t a power of two), 4 or 16 sums per thread, and at most
// 128 pair-side rows per block of plane waves (rows_x <= rows_t).  With both
// direct terms this is Nv = Nc in {2, 4}.
bool fused_fits(const Stage2Args& a) {
  const int rt = a.rows_t, rx = a.rows_x;
  return rt >= 1 && rt <= tc::BM && (rt & (rt - 1)) == 0 && (rx == 4 || rx == 16) && rx <= rt;
}

BatchPlan* plan_create(std::vector<Problem> probs, int precision, int flags, cudaStream_t s) {
  const bool autotune = (flags & BSE_PLAN_AUTOTUNE) != 0;
  std::unique_ptr<BatchPlan> pl(new BatchPlan);
  BSE_CUDA(cudaGetDevice(&pl->device));
  pl->precision = precision;
  pl->probs = std::move(probs);
  if (precision == BSE_PREC_FP64) return pl.release();
  pl->half = (flags & BSE_PLAN_HERMITIAN) != 0;
  bool any_c64 = false;
  for (const Problem& pr : pl->probs) any_c64 = any_c64 || pr.p.in_dtype == BSE_C64;
  if (any_c64 && (flags & (BSE_PLAN_FP64_DIAGONAL | BSE_PLAN_CUDA_CORE_STAGE2)))
    throw Error(BSE_ERR_UNSUPPORTED,
                "complex64 inputs: no exact FP64 diagonal and no CUDA-core stage 2");
  if (flags & BSE_PLAN_FP64_DIAGONAL)
    for (const Problem& pr : pl->probs) pl->diag_ws.emplace_back(diag_fp64_workspace(pr));
  if (pl->half)
    for (const Problem& pr : pl->probs)
      if (pr.kn != pr.p.nk)
        throw Error(BSE_ERR_UNSUPPORTED, "a Hermitian plan builds whole problems (no k-row slabs)");
  const int ng = pl->probs.front().p.ng;
  for (const Problem& pr : pl->probs)
    if (pr.p.ng != ng)
      throw Error(BSE_ERR_UNSUPPORTED, "a batched tensor-core plan needs the same ng in every problem");
  pl->pieces = precision == BSE_PREC_BF16X6 ? 3 : 2;
  pl->planes = 2 * pl->pieces;
  pl->ng = ng;
  pl->Kp = round_up(ng, tc::BK);
  pl->ng_pad = round_up(ng, 32);
  pl->err = DevMem(2 * sizeof(int));
  BSE_CUDA(cudaMemsetAsync(pl->err.ptr, 0, sizeof(int), s));

  // exchange operands of all problems, stacked
  std::vector<tc::Tile> xt;
  std::vector<ExParams> xp;
  int64_t nmax = 0;
  for (const Problem& pr : pl->probs) nmax = std::max<int64_t>(nmax, pr.n);
  // exchange tiles: the widest column tile that still gives every SM a tile;
  // the lower triangle only (Hermitian V) when the full square has at least
  // two tiles per SM (below that the half-empty GPU would not gain)
  const int sms = num_sms();
  int64_t full = 0;
  for (int cand : {128, 96, 64, 32}) {
    if (cand > tile_cols(round_up((int)nmax, 32), pl->Kp)) continue;
    pl->nt_x = cand;
    full = 0;
    for (const Problem& pr : pl->probs)
      full += (int64_t)((pr.rows() + tc::BM - 1) / tc::BM) * ((pr.n + cand - 1) / cand);
    if (full >= sms) break;
  }
  const int tri_all = full >= 2 * sms ? 1 : 0;
  for (size_t i = 0; i < pl->probs.size(); ++i) {
    const Problem& pr = pl->probs[i];
    const bse_problem& p = pr.p;
    const int n = (int)pr.n, nb = p.nv * p.nc;
    // whole problems with enough tiles: the blocks k <= k' only, the rest
    // completed from the mirrors; a k-row slab computes its own rows of V
    // for every column
    const int upper = tri_all && pr.kn == p.nk;
    if (upper) pl->upper_probs.push_back((int)i);
    const int r0 = (int)pr.row0(), r1 = (int)(pr.row0() + pr.rows());
    pl->x_row0.push_back(pl->x_rows);
    // tiles in groups of kXGroup row tiles, column by column: the CTAs working
    // at the same time share a few row tiles and each column tile, so both
    // stay in L2 (row by row, every row tile swept all of M_x through L2)
    constexpr int kXGroup = 8;
    for (int g0 = r0; g0 < r1; g0 += kXGroup * tc::BM)
      for (int n0 = 0; n0 < n; n0 += pl->nt_x)
        for (int m0 = g0; m0 < std::min(r1, g0 + kXGroup * tc::BM); m0 += tc::BM) {
          if (upper && m0 / nb > (std::min(n0 + pl->nt_x, n) - 1) / nb) continue;
          xt.push_back({(int)(pl->x_rows + m0), std::min(tc::BM, r1 - m0), (int)(pl->x_rows + n0),
                        n0, std::min(pl->nt_x, n - n0), m0, (int)i});
        }
    xp.push_back({reinterpret_cast<double2*>(p.A), p.coupling ? reinterpret_cast<double2*>(p.B) : nullptr,
                  p.ld, (float)(2.0 * p.gamma_x * pr.kappa), p.e_v, p.e_c, p.nv, p.nc, upper});
    pl->x_rows += n;
  }
  pl->xa = DevMem((size_t)pl->planes * pl->x_rows * pl->Kp * 2);
  pl->xb = DevMem((size_t)tc::b_planes(pl->pieces) * pl->x_rows * pl->Kp * 2);
  pl->n_xtiles = (int)xt.size();
  pl->xtiles = upload_mem(xt);
  pl->exparams = upload_mem(xp);
  pl->sh_x = make_shape(pl->nt_x, pl->Kp, pl->pieces);
  pl->ma_x = make_plane_map(pl->xa.as<__nv_bfloat16>(), pl->Kp, (int)pl->x_rows, pl->planes, tc::BM);
  pl->mb_x = make_plane_map(pl->xb.as<__nv_bfloat16>(), pl->Kp, (int)pl->x_rows,
                            tc::b_planes(pl->pieces), pl->nt_x);

  // direct terms of all problems, stacked
  for (size_t i = 0; i < pl->probs.size(); ++i) {
    const Problem& pr = pl->probs[i];
    const bse_problem& p = pr.p;
    if (p.gamma_c == 0.0) continue;
    // pairs (k, k') of the slab's rows, p = (k - kb) nk + k'
    const int nv = p.nv, nc = p.nc, npair = (int)pr.slab_pairs();
    const int64_t pair_off = (int64_t)pr.kb * p.nk;   // first slab pair in the whole arrays
    const bool cc_side = nc * nc <= nv * nv;
    for (int term = 0; term < (p.coupling ? 2 : 1); ++term) {
      BatchPlan::Term t;
      t.prob = (int)i;
      Stage2Args& a = t.s2;
      if (term == 0) {
        t.rows_side = cc_side ? nc * nc : nv * nv;
        t.side = cc_side ? p.m_cc : p.m_vv;
        t.w_conj_transpose = !cc_side;
        t.qh.assign(pr.qm_host.begin() + pair_off, pr.qm_host.begin() + pair_off + npair);
        a.mode = cc_side ? S2_RR_CC : S2_RR_VV;
        a.x = reinterpret_cast<const double2*>(cc_side ? p.m_vv : p.m_cc);
        a.x_transpose_pair = 0;
        a.conj_x = cc_side ? 1 : 0;
        a.conj_t = cc_side ? 0 : 1;
        a.rows_x = cc_side ? nv * nv : nc * nc;
        a.out = reinterpret_cast<double2*>(p.A);
      } else {
        t.rows_side = nv * nc;
        // the slab's rows of the whole n_vc (elements of 16 or 8 bytes)
        t.side = reinterpret_cast<const bse_c128*>(
            reinterpret_cast<const char*>(p.n_vc) +
            pair_off * nv * nc * p.ng * (p.in_dtype == BSE_C64 ? 8 : 16));
        t.w_conj_transpose = false;
        t.qh.assign(pr.qp_host.begin() + pair_off, pr.qp_host.begin() + pair_off + npair);
        a.mode = S2_RA;
        a.x = reinterpret_cast<const double2*>(p.n_vc);
        a.x_transpose_pair = 1;
        a.conj_x = 1;
        a.conj_t = 0;
        a.rows_x = nv * nc;
        a.out = reinterpret_cast<double2*>(p.B);
      }
      a.rows_t = t.rows_side;
      // the pairs built: every (k, k') of the slab, or k <= k' in a Hermitian
      // plan (the blocks k > k' are the conjugate transposes, Eq. Hetr)
      const std::vector<int32_t> q_all(t.qh);
      t.qh.clear();
      for (int pp = 0; pp < npair; ++pp) {
        const int k = pr.kb + pp / p.nk, kp = pp % p.nk;
        if (pl->half && k > kp) continue;
        t.act_h.push_back(pp);
        t.qh.push_back(q_all[pp]);
      }
      t.nact = (int)t.act_h.size();
      std::vector<int> perm, gstart;
      group_pairs(t.qh, p.nq_w, perm, gstart);   // slot -> index into act_h
      for (int& x : perm) x = t.act_h[x];         // slot -> pair
      t.slot_h.assign(npair, -1);
      for (int j = 0; j < t.nact; ++j) t.slot_h[perm[j]] = j;
      t.perm = upload_mem(perm);
      t.slot = upload_mem(t.slot_h);
      t.act = upload_mem(t.act_h);
      t.a_row0 = pl->a_rows;
      pl->a_rows += (int64_t)t.nact * t.rows_side;
      if (term == 1 && !pl->terms.empty() && pl->terms.back().prob == (int)i &&
          !pl->terms.back().w_conj_transpose) {
        // W^ra uses W(q) as stored, like a W^rr term that applies it to the
        // conduction side: one set of split planes serves both
        t.w_row0 = pl->terms.back().w_row0;
        t.w_owner = false;
      } else {
        t.w_row0 = pl->w_rows;
        pl->w_rows += (int64_t)p.nq_w * pl->ng_pad;
      }
      a.slot_of_pair = t.slot.as<int>();
      a.pair_of = pl->half ? t.act.as<int>() : nullptr;
      a.ng = ng;
      a.nk = p.nk;
      a.k_begin = pr.kb;
      a.nv = nv;
      a.nc = nc;
      a.scale = p.gamma_c * pr.kappa;
      a.ld = p.ld;
      a.t_row0 = t.a_row0;
      pl->terms.push_back(std::move(t));
    }
  }
  if (!pl->terms.empty()) {
    if (pl->a_rows > INT32_MAX || pl->w_rows > INT32_MAX)
      throw Error(BSE_ERR_UNSUPPORTED, "batched stage-1 rows exceed 2^31");
    // (the fused epilogue contracts whole-K tiles: no K segments)
    // the fused epilogue reads the raw complex128 pair side
    pl->fused = (flags & BSE_PLAN_UNFUSED) == 0 && ksegs_for(pl->Kp) == 1 && !any_c64;
    for (const BatchPlan::Term& t : pl->terms) pl->fused = pl->fused && fused_fits(t.s2);
    pl->wsplit = DevMem((size_t)tc::b_planes(pl->pieces) * pl->w_rows * pl->Kp * 2);
    pl->asplit = DevMem((size_t)pl->planes * pl->a_rows * pl->Kp * 2);
    if (pl->fused) {
      // the pair side of every term as a 2-D FP64 tensor [pairs * rows_x][2 ng],
      // boxes of 16 FP64 (8 complex) x rows_x rows, zero-filled past NG
      std::vector<CUtensorMap> maps;
      for (const BatchPlan::Term& t : pl->terms) {
        const Stage2Args& a = t.s2;
        const Problem& pr = pl->probs[t.prob];
        const int64_t x_pairs = a.x_transpose_pair ? (int64_t)pr.p.nk * pr.p.nk : pr.slab_pairs();
        CUtensorMap m;
        cuuint64_t dims[2] = {(cuuint64_t)2 * a.ng, (cuuint64_t)(x_pairs * a.rows_x)};
        cuuint64_t strides[1] = {(cuuint64_t)a.ng * 16};
        cuuint32_t box[2] = {(cuuint32_t)(2 * tc::S2_GB), (cuuint32_t)a.rows_x};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void*)a.x, dims, strides,
                                 box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
          throw Error(BSE_ERR_CUDA, "cuTensorMapEncodeTiled (pair side) failed with " + std::to_string((int)r));
        maps.push_back(m);
      }
      pl->xmaps = upload_mem(maps);
      for (size_t ti = 0; ti < pl->terms.size(); ++ti) {
        const BatchPlan::Term& t = pl->terms[ti];
        const Stage2Args& a = t.s2;
        tc::S2Term x;
        x.xmap = pl->xmaps.as<CUtensorMap>() + ti;
        x.perm = t.perm.as<int>();
        x.out = a.out;
        x.ld = a.ld;
        x.a_row0 = t.a_row0;
        x.rows_x = a.rows_x;
        x.rows_t = a.rows_t;
        x.nk = a.nk;
        x.k_begin = a.k_begin;
        x.nv = a.nv;
        x.nc = a.nc;
        x.ng = a.ng;
        x.mode = a.mode;
        x.x_transpose_pair = a.x_transpose_pair;
        x.conj_x = a.conj_x;
        x.conj_t = a.conj_t;
        x.scale = (float)a.scale;
        pl->s2host.push_back(x);
      }
      pl->s2terms = upload_mem(pl->s2host);
    } else {
      // large pair blocks: stage 2 on the tensor cores, T straight into split planes
      bool any_fp32 = false, any_tc2 = false;
      for (BatchPlan::Term& t : pl->terms) {
        t.tc2 = (flags & BSE_PLAN_CUDA_CORE_STAGE2) == 0 && t.s2.rows_x >= 64 && t.s2.rows_t >= 64;
        if (!t.tc2 && pl->probs[t.prob].p.in_dtype == BSE_C64)
          throw Error(BSE_ERR_UNSUPPORTED,
                      "complex64 inputs need pair blocks of >= 64 rows on both sides (the "
                      "tensor-core stage 2); smaller blocks take the CUDA-core stage 2, "
                      "which reads complex128");
        any_tc2 = any_tc2 || t.tc2;
        any_fp32 = any_fp32 || !t.tc2;
      }
      if (any_fp32) pl->tbuf = DevMem((size_t)pl->ng_pad * pl->a_rows * sizeof(float2));
      std::vector<TOut> outs;
      for (BatchPlan::Term& t : pl->terms) {
        t.s2.T = pl->tbuf.as<float2>();
        t.s2.t_ld = pl->a_rows;
        outs.push_back(TOut{t.tc2 ? nullptr : pl->tbuf.as<float2>(), pl->a_rows, nullptr,
                            pl->a_rows, pl->Kp, pl->pieces, t.s2.conj_t});
      }
      if (any_tc2) {
        // Each term's second contraction is one tensor-core GEMM per pair block,
        // oriented so that the tile rows run over c fastest (see S2TcEpi): T
        // rows as the A operand (W^rr with T on (c, c')) or as the B operand.
        // The A operand is stored in 2P planes, the B operand in 3P (see
        // tc_gemm.cuh), so T and the other pair side go to the arrays of
        // their role: tA / x2B for the first orientation, x2A / tB for the other.
        std::vector<S2TcParams> prm;
        int max_cols = 0;
        for (BatchPlan::Term& t : pl->terms) {
          if (!t.tc2) continue;
          const Stage2Args& a = t.s2;
          t.rows_t_side = a.mode == S2_RR_CC;            // T rows (c, c') -> (c', c)
          t.side_nb = a.mode == S2_RR_CC ? a.nc : 0;
          t.x_nb = a.mode == S2_RR_VV ? a.nc : 0;        // X rows (c, c') -> (c', c)
          max_cols = std::max(max_cols, t.rows_t_side ? a.rows_x : a.rows_t);
          int64_t& trows = t.rows_t_side ? pl->ta_rows : pl->tb_rows;
          int64_t& xrows = t.rows_t_side ? pl->x2b_rows : pl->x2a_rows;
          t.t_row0 = trows;
          trows += (int64_t)t.nact * a.rows_t;
          t.x2_row0 = xrows;
          xrows += (int64_t)t.nact * a.rows_x;
        }
        if (std::max({pl->ta_rows, pl->tb_rows, pl->x2a_rows, pl->x2b_rows}) > INT32_MAX)
          throw Error(BSE_ERR_UNSUPPORTED, "tensor-core stage-2 rows exceed 2^31");
        const int ap = tc::a_planes(pl->pieces), bp = tc::b_planes(pl->pieces);
        // columns of T past NG are never written: zero once
        const size_t ta_bytes = (size_t)ap * pl->ta_rows * pl->Kp * 2;
        const size_t tb_bytes = (size_t)bp * pl->tb_rows * pl->Kp * 2;
        pl->ta = DevMem(ta_bytes);
        pl->tb = DevMem(tb_bytes);
        if (ta_bytes) BSE_CUDA(cudaMemsetAsync(pl->ta.ptr, 0, ta_bytes, s));
        if (tb_bytes) BSE_CUDA(cudaMemsetAsync(pl->tb.ptr, 0, tb_bytes, s));
        pl->x2a = DevMem((size_t)ap * pl->x2a_rows * pl->Kp * 2);
        pl->x2b = DevMem((size_t)bp * pl->x2b_rows * pl->Kp * 2);
        for (size_t ti = 0; ti < pl->terms.size(); ++ti) {
          const BatchPlan::Term& t = pl->terms[ti];
          if (!t.tc2) continue;
          TOut& o = outs[ti];
          o.planes = (t.rows_t_side ? pl->ta : pl->tb).as<__nv_bfloat16>();
          o.plane_rows = t.rows_t_side ? pl->ta_rows : pl->tb_rows;
          o.bneg = t.rows_t_side ? 0 : 1;
          o.row_off = t.t_row0 - t.a_row0;
        }
        pl->s2_max_cols = max_cols;
        for (size_t ti = 0; ti < pl->terms.size(); ++ti) {
          BatchPlan::Term& t = pl->terms[ti];
          const Stage2Args& a = t.s2;
          // (a, b) of each side and its strides in al + ap * ld:
          //   W^rr, T on (c, c'):  X (v, v'): (nc, nc ld)   T (c, c'): (1, ld)
          //   W^rr, T on (v, v'):  X (c, c'): (1, ld)       T (v, v'): (nc, nc ld)
          //   W^ra:                X (v', c): (nc ld, 1)    T (v, c'): (nc, ld)
          const int64_t ld = a.ld, nc = a.nc;
          int nb_x, nb_t;
          int64_t xa, xb, ta, tb;
          if (a.mode == S2_RR_CC) {
            nb_x = a.nv; xa = nc; xb = nc * ld; nb_t = a.nc; ta = 1; tb = ld;
          } else if (a.mode == S2_RR_VV) {
            nb_x = a.nc; xa = 1; xb = ld; nb_t = a.nv; ta = nc; tb = nc * ld;
          } else {
            nb_x = a.nc; xa = nc * ld; xb = 1; nb_t = a.nc; ta = nc; tb = ld;
          }
          S2TcParams q{a.out, a.ld, a.nk, a.nv * a.nc, a.k_begin, (float)a.scale, 0, 0, 0, 0, 0, 0, 0, 0};
          if (t.rows_t_side) {
            q.rows_r = a.rows_t; q.row_nb = t.side_nb;
            q.nb_r = nb_t; q.ra = ta; q.rb = tb; q.nb_c = nb_x; q.ca = xa; q.cb = xb;
          } else {
            q.rows_r = a.rows_x; q.row_nb = t.x_nb;
            q.nb_r = nb_x; q.ra = xa; q.rb = xb; q.nb_c = nb_t; q.ca = ta; q.cb = tb;
          }
          prm.push_back(q);
          if (!t.tc2) continue;
          std::vector<int> xp(t.nact);
          for (int j = 0; j < t.nact; ++j) {   // (k', k) of the whole array, k = k_begin + pr / nk
            const int pr = t.act_h[j];
            xp[j] = a.x_transpose_pair ? (pr % a.nk) * a.nk + a.k_begin + pr / a.nk : pr;
          }
          t.x2perm = upload_mem(xp);
        }
        pl->s2params = upload_mem(prm);
        plan_set_s2_tiles(*pl, s2_default_cols(*pl), 0);
      }
      pl->touts = upload_mem(outs);
    }
    pl->ma_s = make_plane_map(pl->asplit.as<__nv_bfloat16>(), pl->Kp, (int)pl->a_rows, pl->planes,
                              tc::BM);
    if (autotune)
      plan_autotune(*pl, s);
    else
      plan_set_tiles(*pl, pl->fused ? (pl->ng_pad % 64 == 0 ? 64 : 32) : tile_cols(pl->ng_pad, pl->Kp));
  }
  BSE_CUDA(cudaStreamSynchronize(s));
  return pl.release();
}

void plan_execute(BatchPlan* pl, cudaStream_t s) {
  int dev = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  if (dev != pl->device) throw Error(BSE_ERR_ARG, "plan executed on another device");
  if (pl->precision == BSE_PREC_FP64) {
    for (const Problem& pr : pl->probs) build_fp64(pr, s);
    return;
  }
  plan_execute_mixed(*pl, s);
}

int plan_status(BatchPlan* pl, cudaStream_t s) {
  if (pl->precision == BSE_PREC_FP64) {
    BSE_CUDA(cudaStreamSynchronize(s));
    return BSE_OK;
  }
  int herr = 0;
  BSE_CUDA(cudaMemcpyAsync(&herr, pl->err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaMemsetAsync(pl->err.ptr, 0, sizeof(int), s));
  BSE_CUDA(cudaStreamSynchronize(s));
  return herr ? BSE_ERR_TIMEOUT : BSE_OK;
}

int plan_tile_cols(const BatchPlan* pl) { return pl->nt_g; }
void plan_stage2_shape(const BatchPlan* pl, int* tile_cols, int* stages) {
  const bool any = pl->n_s2tiles || pl->n_s2tiles_t;
  *tile_cols = any ? pl->nt2 : 0;
  *stages = any ? pl->s2_stages : 0;
}

int plan_fused(const BatchPlan* pl) { return pl->fused ? 1 : 0; }

void plan_set_wait(BatchPlan* pl, double seconds) {
  int khz = 0;
  BSE_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, pl->device));
  const double cycles = seconds * 1e3 * (khz > 0 ? khz : 2000000);
  pl->wait = std::max<long long>(1, (long long)cycles);
}

void plan_destroy(BatchPlan* pl) { delete pl; }


// ---------------------------------------------------------------------------
// bse_build_kernel with a tensor-core precision: a plan per set of problem
// descriptors (pointers, sizes, spin factors and q maps), cached so that
// repeated builds of the same arrays skip validation-time set-up, then one
// execute and a status check.  At most kPlanCache plans stay alive (their
// scratch is device memory held until eviction or exit).
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kPlanCache = 4;

struct CachedPlan {
  std::vector<uint64_t> key;
  std::shared_ptr<BatchPlan> plan;   // shared with the callers using it (eviction-safe)
};
std::mutex g_cache_mutex;
std::vector<CachedPlan> g_cache;   // most recent last

std::vector<uint64_t> plan_key(const std::vector<Problem>& probs, int precision) {
  std::vector<uint64_t> k;
  int dev = 0;
  cudaGetDevice(&dev);
  k.push_back((uint64_t)dev);
  k.push_back((uint64_t)precision);
  for (const Problem& pr : probs) {
    const bse_problem& p = pr.p;
    const void* ptrs[] = {p.e_v, p.e_c, p.m_x, p.m_vv, p.m_cc, p.n_vc, p.w, p.q_minus, p.q_plus,
                          p.v_bar, p.A, p.B};
    for (const void* q : ptrs) k.push_back((uint64_t)(uintptr_t)q);
    k.push_back(((uint64_t)p.nk << 32) | (uint32_t)p.nv);
    k.push_back(((uint64_t)p.nc << 32) | (uint32_t)p.ng);
    k.push_back(((uint64_t)p.nq_w << 32) | (uint32_t)p.coupling);
    uint64_t bits[4];
    memcpy(&bits[0], &p.omega_cell, 8);
    memcpy(&bits[1], &p.gamma_x, 8);
    memcpy(&bits[2], &p.gamma_c, 8);
    k.push_back(bits[0]);
    k.push_back(bits[1]);
    k.push_back(bits[2]);
    k.push_back((uint64_t)p.ld);
    k.push_back(((uint64_t)(uint32_t)p.k_begin << 32) | (uint32_t)p.k_count);
    k.push_back((uint64_t)(uint32_t)p.in_dtype);
    k.push_back(fnv1a(pr.qp_host, fnv1a(pr.qm_host)));
  }
  return k;
}
}  // namespace

bool mixed_supported(int precision) {
  return precision == BSE_PREC_BF16X6 || precision == BSE_PREC_BF16X3;
}

void build_mixed_batch(const std::vector<Problem>& probs, int precision, cudaStream_t s) {
  // one plan per distinct ng (a tensor-core plan needs one ng)
  std::vector<int> ngs;
  for (const Problem& pr : probs)
    if (std::find(ngs.begin(), ngs.end(), pr.p.ng) == ngs.end()) ngs.push_back(pr.p.ng);
  for (int ng : ngs) {
    std::vector<Problem> group;
    for (const Problem& pr : probs)
      if (pr.p.ng == ng) group.push_back(pr);
    const std::vector<uint64_t> key = plan_key(group, precision);
    std::shared_ptr<BatchPlan> plan;
    {
      std::lock_guard<std::mutex> lock(g_cache_mutex);
      for (size_t i = 0; i < g_cache.size(); ++i)
        if (g_cache[i].key == key) {
          CachedPlan c = std::move(g_cache[i]);
          g_cache.erase(g_cache.begin() + i);
          g_cache.push_back(std::move(c));
          plan = g_cache.back().plan;
          break;
        }
    }
    if (!plan) {
      std::shared_ptr<BatchPlan> created(plan_create(group, precision, 0, s));
      std::lock_guard<std::mutex> lock(g_cache_mutex);
      if (g_cache.size() >= kPlanCache) g_cache.erase(g_cache.begin());
      g_cache.push_back(CachedPlan{key, created});
      plan = created;
    }
    // a cached plan's scratch and status word serve one build at a time:
    // callers on other host threads (or streams) wait for the one using it
    std::lock_guard<std::mutex> use(plan->use_mutex);
    plan_execute(plan.get(), s);
    if (plan_status(plan.get(), s) != BSE_OK)
      throw Error(BSE_ERR_TIMEOUT, "tensor-core GEMM: a bounded pipeline wait expired");
  }
}


// ---------------------------------------------------------------------------
// Matrix-vector blocks of a Hermitian N x N matrix on the tensor cores, for the
// Davidson solve: AV = A V and BV = B V with V an N x k block.  Row m of a
// Hermitian matrix is the conjugate of its column m, which is contiguous in
// the column-major input, so A and B are split once (conjugated columns as
// GEMM rows, K = N); each call splits V's columns and runs one GEMM per
// matrix (K segments of 8 steps), writing FP64 results column-major.  A's
// diagonal (the transition energies, hundreds of eV for core levels) is left
// out of the split and applied in FP64 in the epilogue, so the split error
// scales with the interaction, not with the energies.
// ---------------------------------------------------------------------------
namespace {
struct MatvecEpi {
  double2* out;
  int64_t ld;
  const double2* diag = nullptr;   // the matrix (its diagonal is added in FP64), or NULL
  int64_t diag_ld = 0;
  const double2* v = nullptr;      // the FP64 block V, column-major with leading dimension ld
  __device__ __forceinline__ void operator()(const tc::Tile& t, int row, int c0, const float* re,
                                             const float* im) const {
    const int64_t r = t.out_row0 + row;
    double2 d = make_double2(0.0, 0.0);
    if (diag) d = diag[r * (diag_ld + 1)];
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (c0 + j < t.n_valid) {
        const int64_t o = r + (int64_t)(t.n0 + c0 + j) * ld;
        double2 y = make_double2(f32_to_f64_bits(re[j]), f32_to_f64_bits(im[j]));
        if (diag) {
          const double2 x = v[o];
          y.x += d.x * x.x - d.y * x.y;
          y.y += d.x * x.y + d.y * x.x;
        }
        out[o] = y;
      }
  }
};
}  // namespace

struct TcMatvec {
  int n = 0, Kp = 0, pieces = 3, planes = 6, kmax = 0, kmax_rows = 0, nt = 0, max_tiles = 0;
  bool has_b = false;
  const bse_c128* A = nullptr;   // caller's A (its diagonal, in FP64)
  int64_t ld = 0;
  DevMem ap, bp, vp, tiles, err;
  CUtensorMap ma_a{}, ma_b{}, mb_v{};
  tc::GemmShape sh{};
};

TcMatvec* tc_matvec_create(int n, const bse_c128* A, const bse_c128* B, int64_t ld, int precision,
                           int kmax, cudaStream_t s) {
  std::unique_ptr<TcMatvec> m(new TcMatvec);
  m->n = n;
  m->pieces = precision == BSE_PREC_BF16X6 ? 3 : 2;
  m->planes = 2 * m->pieces;
  m->Kp = round_up(n, tc::BK);
  m->kmax = kmax;
  m->kmax_rows = round_up(kmax, 32);
  m->nt = tile_cols(m->kmax_rows, m->Kp);
  m->sh = make_shape(m->nt, m->Kp, m->pieces);
  m->has_b = B != nullptr;
  m->A = A;
  m->ld = ld;
  m->max_tiles = ((n + tc::BM - 1) / tc::BM) * ((kmax + m->nt - 1) / m->nt);
  const size_t mat_bytes = (size_t)m->planes * n * m->Kp * 2;
  m->ap = DevMem(mat_bytes);
  if (B) m->bp = DevMem(mat_bytes);
  const size_t v_bytes = (size_t)tc::b_planes(m->pieces) * m->kmax_rows * m->Kp * 2;
  m->vp = DevMem(v_bytes);
  BSE_CUDA(cudaMemsetAsync(m->vp.ptr, 0, v_bytes, s));
  m->tiles = DevMem((size_t)m->max_tiles * sizeof(tc::Tile));
  m->err = DevMem(2 * sizeof(int));
  BSE_CUDA(cudaMemsetAsync(m->err.ptr, 0, sizeof(int), s));
  for (int which = 0; which < (B ? 2 : 1); ++which) {
    SplitArgs sa{reinterpret_cast<const double2*>(which ? B : A), SPLIT_DENSE, nullptr, 0, 0, n,
                 m->Kp, n, m->pieces, 1, nullptr,
                 (which ? m->bp : m->ap).as<__nv_bfloat16>(), n, 0};
    sa.src_ld = ld;
    sa.zero_diag = which == 0;
    launch_split(sa, s);
  }
  m->ma_a = make_plane_map(m->ap.as<__nv_bfloat16>(), m->Kp, n, m->planes, tc::BM);
  if (B) m->ma_b = make_plane_map(m->bp.as<__nv_bfloat16>(), m->Kp, n, m->planes, tc::BM);
  m->mb_v = make_plane_map(m->vp.as<__nv_bfloat16>(), m->Kp, m->kmax_rows,
                           tc::b_planes(m->pieces), m->nt);
  return m.release();
}

void tc_matvec_apply(TcMatvec* m, const bse_c128* V, int k, bse_c128* AV, bse_c128* BV,
                     cudaStream_t s) {
  if (k <= 0) return;
  if (k > m->kmax) throw Error(BSE_ERR_UNSUPPORTED, "tensor-core matvec block wider than planned");
  SplitArgs sv{reinterpret_cast<const double2*>(V), SPLIT_DENSE, nullptr, 0, 0, m->n, m->Kp, k,
               m->pieces, 0, nullptr, m->vp.as<__nv_bfloat16>(), m->kmax_rows, 0};
  sv.bneg = 1;   // the B operand of the matvec GEMMs
  launch_split(sv, s);
  std::vector<tc::Tile> tl;
  for (int m0 = 0; m0 < m->n; m0 += tc::BM)
    for (int n0 = 0; n0 < k; n0 += m->nt)
      tl.push_back({m0, std::min(tc::BM, m->n - m0), n0, n0, std::min(m->nt, k - n0), m0, 0});
  BSE_CUDA(cudaMemcpyAsync(m->tiles.ptr, tl.data(), tl.size() * sizeof(tc::Tile),
                           cudaMemcpyHostToDevice, s));
  launch_gemm(m->ma_a, m->mb_v, m->tiles.as<tc::Tile>(), (int)tl.size(), m->sh,
              MatvecEpi{reinterpret_cast<double2*>(AV), m->n, reinterpret_cast<const double2*>(m->A),
                        m->ld, reinterpret_cast<const double2*>(V)},
              m->err.as<int>(), s);
  if (m->has_b && BV)
    launch_gemm(m->ma_b, m->mb_v, m->tiles.as<tc::Tile>(), (int)tl.size(), m->sh,
                MatvecEpi{reinterpret_cast<double2*>(BV), m->n}, m->err.as<int>(), s);
  int herr = 0;
  BSE_CUDA(cudaMemcpyAsync(&herr, m->err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));   // also keeps the host tile list alive until used
  if (herr) throw Error(BSE_ERR_TIMEOUT, "tensor-core matvec: a bounded pipeline wait expired");
}

void tc_matvec_destroy(TcMatvec* m) { delete m; }

// ---------------------------------------------------------------------------
// Static RPA screening: the polarisability sum of the RPA dielectric matrix
// (the equation for eps^RPA before Eq. wggq) at omega = 0 for an insulator,
//   X[G][G'] = sum_a conj(mt_a(G)) mt_a(G'),  mt_a = m_a / sqrt(e_c - e_v),
// a = (k v c), on the tensor cores: both operands are the transposed pair
// elements (rows G, K = the transitions, scaled by (e_c - e_v)^-1/2 when
// split), the K range is cut into tiles of 512 transitions (4 segments of
// 8 K steps accumulated afresh, as in the build), each tile writes an FP32
// partial sum and one kernel adds the partials in FP64 in a fixed order.
// ---------------------------------------------------------------------------
namespace {
constexpr int RPA_KSTEPS = 32;   // K steps per tile (512 transitions)

struct RpaPartialEpi {
  float2* part;   // [splits][ng][ng] row-major partial sums
  int ng;
  __device__ __forceinline__ void operator()(const tc::Tile& t, int row, int c0, const float* re,
                                             const float* im) const {
    float2* dst = part + ((int64_t)t.prob * ng + t.out_row0 + row) * ng + t.n0 + c0;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (c0 + j < t.n_valid) dst[j] = make_float2(re[j], im[j]);
  }
};

__global__ void k_rpa_inv_sqrt_gap(int64_t ntr, int nv, int nc, const double* e_v,
                                   const double* e_c_kq, double* f) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < ntr;
       a += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(a % nc), v = (int)((a / nc) % nv);
    const int64_t k = a / ((int64_t)nv * nc);
    f[a] = 1.0 / sqrt(e_c_kq[k * nc + c] - e_v[k * nv + v]);
  }
}

__global__ void k_rpa_reduce(const float2* part, int splits, int64_t nn, double2* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
       i += (int64_t)gridDim.x * blockDim.x) {
    double sx = 0.0, sy = 0.0;
    for (int s = 0; s < splits; ++s) {
      const float2 p = part[(int64_t)s * nn + i];
      sx += (double)p.x;
      sy += (double)p.y;
    }
    x[i] = make_double2(sx, sy);
  }
}
}  // namespace

void rpa_x_mixed(int nk, int nv, int nc, int ng, const double* e_v, const double* e_c_kq,
                 const bse_c128* m, int precision, double2* x_out, cudaStream_t s) {
  const int pieces = precision == BSE_PREC_BF16X6 ? 3 : 2;
  const int64_t ntr = (int64_t)nk * nv * nc;
  const int kspan = RPA_KSTEPS * tc::BK;                  // transitions per tile
  const int64_t kp = (ntr + kspan - 1) / kspan * kspan;   // padded K (zeros past ntr)
  if (kp > INT32_MAX) throw Error(BSE_ERR_UNSUPPORTED, "too many transitions for the RPA GEMM");
  const int splits = (int)(kp / kspan);
  const int nt = tile_cols(round_up(ng, 32), kspan);
  const tc::GemmShape sh = make_shape(nt, kspan, pieces);
  DevMem f((size_t)ntr * sizeof(double));
  DevMem ap((size_t)tc::a_planes(pieces) * ng * kp * 2);
  DevMem bp((size_t)tc::b_planes(pieces) * ng * kp * 2);
  DevMem part((size_t)splits * ng * ng * sizeof(float2));
  DevMem err(2 * sizeof(int));
  BSE_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
  {
    Phase ph("rpa_split", s);
    k_rpa_inv_sqrt_gap<<<(int)std::min<int64_t>((ntr + 255) / 256, 152 * 8), 256, 0, s>>>(
        ntr, nv, nc, e_v, e_c_kq, f.as<double>());
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
    // rows G, K = transitions: element (G, a) is m[a][G] (transposed read)
    SplitArgs sa{reinterpret_cast<const double2*>(m), SPLIT_DENSE, nullptr, 0, 0, (int)ntr,
                 (int)kp, ng, pieces, 1, f.as<double>(), ap.as<__nv_bfloat16>(), ng, 0};
    sa.tdense = 1;
    sa.src_ld = ng;
    launch_split(sa, s);
    SplitArgs sb = sa;
    sb.conj = 0;
    sb.bneg = 1;
    sb.out = bp.as<__nv_bfloat16>();
    launch_split(sb, s);
  }
  std::vector<tc::Tile> tiles;
  for (int sp = 0; sp < splits; ++sp)
    for (int m0 = 0; m0 < ng; m0 += tc::BM)
      for (int n0 = 0; n0 < ng; n0 += nt)
        tiles.push_back({m0, std::min(tc::BM, ng - m0), n0, n0, std::min(nt, ng - n0), m0, sp,
                         sp * RPA_KSTEPS});
  DevMem dtiles = upload_mem(tiles);
  const CUtensorMap ma = make_plane_map(ap.as<__nv_bfloat16>(), (int)kp, ng, tc::a_planes(pieces),
                                        tc::BM);
  const CUtensorMap mb = make_plane_map(bp.as<__nv_bfloat16>(), (int)kp, ng, tc::b_planes(pieces),
                                        nt);
  {
    Phase ph("rpa_x_gemm", s);
    launch_gemm(ma, mb, dtiles.as<tc::Tile>(), (int)tiles.size(), sh, RpaPartialEpi{part.as<float2>(), ng},
                err.as<int>(), s);
  }
  {
    Phase ph("rpa_reduce", s);
    const int64_t nn = (int64_t)ng * ng;
    k_rpa_reduce<<<(int)std::min<int64_t>((nn + 255) / 256, 152 * 8), 256, 0, s>>>(
        part.as<float2>(), splits, nn, x_out);
    BSE_CUDA(cudaGetLastError());
    note_launches(1);
  }
  int herr = 0;
  BSE_CUDA(cudaMemcpyAsync(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));   // also keeps the workspace alive until used
  if (herr) throw Error(BSE_ERR_TIMEOUT, "RPA tensor-core GEMM: a bounded pipeline wait expired");
}

}  // namespace bse
