// Direct term (screened interaction W^rr or W^ra, Eqs. wrrm / wrabar) in one
// persistent tcgen05 launch: the stage-1 GEMM
//   T[row][G'] = sum_G X_side[row][G] W(q)[G][G']       (rows = pair slots x rows_t)
// accumulates in TMEM exactly as gemm_split_bf16 does, and the epilogue
// contracts each TMEM tile of T at once with the other side of the pair,
//   P[rx][rt] = sum_G' opX(X_pair[rx][G']) opT(T[slot * rows_t + rt][G']),
// so that T never leaves the SM.  A CTA takes one 128-row tile of stage-1
// rows with all its output-column tiles as one work unit (GemmShape::group);
// each thread of the epilogue owns one row of T (one (pair, rt)) and keeps
// the rows_x (4 or 16) sums of its pair in registers across the unit.
//
// Roles (7 warps):
//   warp 0     TMA producer of the BF16 operand planes (shared with the GEMM)
//   warp 1     TMEM allocation and MMA issue (shared with the GEMM)
//   warps 2-5  epilogue: convert the pair side of the current block of 8
//              plane waves from complex128 to FP32 complex in shared memory
//              (each element once), read T from TMEM, accumulate
//   warp 6     pair-side loader: one 2-D TMA box per pair and block
//              (rows_x rows x 8 complex128, zero-filled past NG), S2_XSLOTS
//              blocks in flight
// Arithmetic is that of the two-kernel path (stage-1 T in FP32 = main +
// correction accumulators; sums of 8 plane waves in FMA, folded into
// compensated (hi, lo) pairs with TwoSum; the product with gamma_c kappa formed
// in FP32 and widened exactly), in the same order, so both paths give the
// same bits.  Every wait is bounded; the four epilogue warps agree on giving
// up through one AND-reduction barrier per block.
#pragma once

#include "bits.cuh"
#include "tc_gemm.cuh"

namespace bse {
namespace tc {

constexpr int S2_THREADS = 224;
constexpr int S2_GB = 8;                                    // plane waves per block
constexpr int S2_XSLOTS = 3;                                // raw blocks in flight
constexpr uint32_t S2_RAW_BYTES = BM * S2_GB * 16;          // <= 128 (pair, rx) rows x 8 complex128
// FP32 pair side of one block, per pair: for each plane wave a row of Re
// and a row of -Im over rx (rows_x floats each) and a 16-byte pad, then a
// 16-byte pad per pair (bank-conflict-free writes and broadcast reads);
// largest for rows_x = 4 with 32 pairs
__host__ __device__ constexpr uint32_t s2_gstride(int rx) { return 8u * rx + 16u; }
__host__ __device__ constexpr uint32_t s2_pstride(int rx) { return S2_GB * s2_gstride(rx) + 16u; }
constexpr uint32_t S2_XF_BYTES = (BM / 4) * s2_pstride(4);

struct S2Term {
  const CUtensorMap* xmap;   // other pair side, complex128 [pairs][rows_x][ng] seen as FP64
                             // [pairs * rows_x][2 ng], box {16, rows_x} (device memory);
                             // pairs = the slab's (k, k'), or all nk^2 when transposed
  const int* perm;        // slot -> pair (k - k_begin) nk + k' (sorted by q; -1: padding slot)
  double2* out;           // A (W^rr) or B (W^ra), column-major; NULL: contraction only (timing)
  int64_t ld;
  int64_t a_row0;         // first stage-1 row of this term
  int rows_x, rows_t, nk, nv, nc, ng;
  int k_begin;            // first k row of the slab
  int mode;               // 0: rx = (v,v'), rt = (c,c'); 1: rx = (c,c'), rt = (v,v'); 2: W^ra
  int x_transpose_pair;   // read the side of pair (k', k)
  int conj_x, conj_t;
  float scale;            // gamma_c kappa
};

__host__ __device__ inline uint32_t s2_extra_bytes(int stages) {
  return S2_XSLOTS * S2_RAW_BYTES + 2 * S2_XF_BYTES + (2 * stages + 5 + 2 * S2_XSLOTS) * 8 + 16;
}
__host__ inline size_t s2_smem_bytes(const GemmShape& s) {
  return 1024 + (size_t)s.stages * stage_bytes(s) + s2_extra_bytes(s.stages);
}

// 2-D tensor copy through a tensor map held in device memory
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Barrier 1 over the 128 epilogue threads; true iff every thread passed true.
__device__ __forceinline__ bool epi_bar_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(v ? 1u : 0u)
      : "memory");
  return r != 0;
}

// Packed FP32 pairs (Blackwell f32x2): both lanes rounded to nearest like
// the scalar instructions, element 0 in the low word.
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t fadd2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t fsub2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float lo_of(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi_of(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
// TwoSum of two pairs at once: h + a = h' + e exactly in each lane; l += e
__device__ __forceinline__ void two_sum2(uint64_t& h, uint64_t& l, uint64_t a) {
  const uint64_t sm = fadd2(h, a);
  const uint64_t bp = fsub2(sm, h);
  const uint64_t e = fadd2(fsub2(h, fsub2(sm, bp)), fsub2(a, bp));
  h = sm;
  l = fadd2(l, e);
}

// 8 columns of T for this thread's lane: main + correction, real and imaginary
// (four loads and their wait in one statement, so no use can precede the wait).
__device__ __forceinline__ void tmem_ld_t8(uint32_t taddr, uint32_t nt, float* tr, float* ti) {
  uint32_t r[32];
  asm volatile(
      "{\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%33];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%34];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%35];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n\t}"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr), "r"(taddr + nt), "r"(taddr + 2 * nt), "r"(taddr + 3 * nt)
      : "memory");
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    tr[g] = __uint_as_float(r[g]) + __uint_as_float(r[16 + g]);
    ti[g] = __uint_as_float(r[8 + g]) + __uint_as_float(r[24 + g]);
  }
}

// What the epilogue threads share across work units.
struct EpiCtx {
  const Tile* tiles;
  int ntiles;
  GemmShape sh;
  const S2Term* terms;
  int* err;
  volatile int* abort_flag;
  Pipe pp;
  uint8_t* xraw;       // [S2_XSLOTS][S2_RAW_BYTES] pair side as loaded (complex128)
  uint8_t* xf;         // [2][S2_XF_BYTES] pair side in FP32
  uint64_t *xfull, *xempty;
  uint32_t tmem_base;
  int et;              // 0..127
  int quarter;         // TMEM lane quarter of this warp
  int lane;
};
struct EpiState {      // ring positions, carried from unit to unit
  int local;           // tiles done by this CTA (accumulator set = local & 1)
  int xs, xb;          // raw slot, FP32 buffer
  uint32_t xph;        // phase of the raw ring
};

// One work unit (a 128-row tile and all its column tiles) of the epilogue,
// for RX = rows_x in {4, 16}.  Two rx outputs share each packed instruction:
// per plane wave g and output pair,
//   ax += xr t_re ; ax += (-xi) t_im ; ay += xr t_im ; ay += (-xi)(-t_re)
// (the same products and roundings, in the same order, as the scalar
// two-launch contraction).  Returns false once a bounded wait has failed
// (uniformly across the four warps).
template <int RX>
__device__ __forceinline__ bool direct_unit(const EpiCtx& cx, EpiState& st, int u) {
  static_assert(RX == 4 || RX == 16, "rows_x of the fused epilogue");
  constexpr uint32_t GSTRIDE = s2_gstride(RX), PSTRIDE = s2_pstride(RX);
  constexpr int NP = RX / 2;                            // output pairs per component
  const int row = cx.quarter * 32 + cx.lane;
  const uint32_t nt = (uint32_t)cx.sh.nt;
  const int t0 = u * cx.sh.group;
  const Tile tg = cx.tiles[t0];
  const S2Term& tm = cx.terms[tg.prob];
  const int rows_t = tm.rows_t, ng = tm.ng;
  const int j = row / rows_t, rt = row - j * rows_t;   // pair slot in the tile, row in the pair
  const int nrows = ((tg.m_valid + rows_t - 1) / rows_t) * RX;
  const float tsign = tm.conj_t ? -1.f : 1.f;
  const uint32_t xflip = tm.conj_x ? 0x80000000u : 0u;
  const bool mine = row < tg.m_valid;
  // this thread's elements of every raw block (e = et + 128 i: row r = e / 8 =
  // (pair jj, rx), plane wave g = e % 8) and where their Re goes (-Im: + 4 RX)
  const int gq = cx.et & 7;
  int xoff[S2_GB];
#pragma unroll
  for (int i = 0; i < S2_GB; ++i) {
    const int r = (cx.et + 128 * i) >> 3;
    const int jj = r / RX, rx = r % RX;
    xoff[i] = r < nrows ? (int)(jj * PSTRIDE + gq * GSTRIDE + rx * 4) : -1;
  }
  uint64_t HX[NP], HY[NP], LX[NP], LY[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) HX[i] = HY[i] = LX[i] = LY[i] = 0ull;

  for (int t = t0; t < min(cx.ntiles, t0 + cx.sh.group); ++t, ++st.local) {
    const Tile tl = cx.tiles[t];
    const int buf = st.local & 1;
    const int use = st.local >> 1;
    int okt = 0;
    if (cx.lane == 0)
      okt = mbar_wait(&cx.pp.tmem_full[buf], use & 1, cx.abort_flag, cx.err, cx.sh.wait) ? 1 : 0;
    okt = __shfl_sync(0xffffffffu, okt, 0);
    const uint32_t lane_base =
        cx.tmem_base + (uint32_t)buf * 4u * nt + ((uint32_t)(cx.quarter * 32) << 16);
    for (int c = 0; c < tl.n_valid; c += S2_GB) {
      const bool okx = okt && mbar_wait(&cx.xfull[st.xs], st.xph, cx.abort_flag, cx.err, cx.sh.wait);
      const int g0 = tl.n0 + c;
      uint8_t* xfb = cx.xf + (size_t)st.xb * S2_XF_BYTES;
      if (okx) {   // complex128 -> FP32 (Re, -Im), each element once
        const uint4* raw = reinterpret_cast<const uint4*>(cx.xraw + (size_t)st.xs * S2_RAW_BYTES);
        const bool gin = g0 + gq < ng;
#pragma unroll
        for (int i = 0; i < S2_GB; ++i) {
          if (xoff[i] >= 0) {
            uint32_t re = 0u, mi = 0u;
            if (gin) {
              const uint4 d = raw[cx.et + 128 * i];
              re = f64w_to_f32_bits(d.x, d.y);
              mi = f64w_to_f32_bits(d.z, d.w) ^ xflip ^ 0x80000000u;
            }
            *reinterpret_cast<uint32_t*>(xfb + xoff[i]) = re;
            *reinterpret_cast<uint32_t*>(xfb + xoff[i] + 4 * RX) = mi;
          }
        }
      }
      if (!epi_bar_and(okx)) return false;
      if (cx.et == 0) mbar_arrive(&cx.xempty[st.xs]);
      if (++st.xs == S2_XSLOTS) {
        st.xs = 0;
        st.xph ^= 1;
      }
      tc_fence_after();
      float tr[8], ti[8];
      tmem_ld_t8(lane_base + (uint32_t)c, nt, tr, ti);
      if (c + S2_GB > tl.n_valid) {
#pragma unroll
        for (int g = 0; g < S2_GB; ++g)
          if (c + g >= tl.n_valid) tr[g] = ti[g] = 0.f;
      }
      if (mine) {
        uint64_t TR[S2_GB], TY[S2_GB], TN[S2_GB];   // (t_re, t_re), (t_im, t_im), (-t_re, -t_re)
#pragma unroll
        for (int g = 0; g < S2_GB; ++g) {
          const float ty = ti[g] * tsign;
          TR[g] = pack2(tr[g], tr[g]);
          TY[g] = pack2(ty, ty);
          TN[g] = pack2(-tr[g], -tr[g]);
        }
        const uint8_t* xp = xfb + j * PSTRIDE;
#pragma unroll
        for (int q = 0; q < RX / 4; ++q) {
          uint64_t ax0 = 0ull, ax1 = 0ull, ay0 = 0ull, ay1 = 0ull;
#pragma unroll
          for (int g = 0; g < S2_GB; ++g) {
            const ulonglong2 xr = *reinterpret_cast<const ulonglong2*>(xp + g * GSTRIDE + q * 16);
            const ulonglong2 xn =
                *reinterpret_cast<const ulonglong2*>(xp + g * GSTRIDE + 4 * RX + q * 16);
            ax0 = ffma2(xr.x, TR[g], ax0);
            ax0 = ffma2(xn.x, TY[g], ax0);
            ay0 = ffma2(xr.x, TY[g], ay0);
            ay0 = ffma2(xn.x, TN[g], ay0);
            ax1 = ffma2(xr.y, TR[g], ax1);
            ax1 = ffma2(xn.y, TY[g], ax1);
            ay1 = ffma2(xr.y, TY[g], ay1);
            ay1 = ffma2(xn.y, TN[g], ay1);
          }
          two_sum2(HX[2 * q], LX[2 * q], ax0);
          two_sum2(HY[2 * q], LY[2 * q], ay0);
          two_sum2(HX[2 * q + 1], LX[2 * q + 1], ax1);
          two_sum2(HY[2 * q + 1], LY[2 * q + 1], ay1);
        }
      }
      st.xb ^= 1;
    }
    tc_fence_before();
    __syncwarp();
    if (cx.lane == 0) mbar_arrive(&cx.pp.tmem_empty[buf]);
  }
  if (!mine || tm.out == nullptr) return true;
  // subtract gamma_c kappa P from A or B (FP64 read-modify-write, one owner per element)
  const int pair = tm.perm[((int64_t)tg.out_row0 - tm.a_row0) / rows_t + j];
  if (pair < 0) return true;   // padding slot
  const int nk = tm.nk, nv = tm.nv, nc = tm.nc;
  const int kl = pair / nk, kp = pair - kl * nk, k = tm.k_begin + kl;
  const float sc = tm.scale;
  // groups of 4 outputs: all loads first, then the stores (the loads of a
  // group are independent, so their latencies overlap)
#pragma unroll
  for (int r0 = 0; r0 < RX; r0 += 4) {
    double2* dst[4];
    double2 o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int rx = r0 + u;
      int vi, ci, vp, cp;
      if (tm.mode == 0) {
        vi = rx / nv; vp = rx % nv; ci = rt / nc; cp = rt % nc;
      } else if (tm.mode == 1) {
        ci = rx / nc; cp = rx % nc; vi = rt / nv; vp = rt % nv;
      } else {
        vp = rx / nc; ci = rx % nc; vi = rt / nc; cp = rt % nc;
      }
      const int64_t al = ((int64_t)k * nv + vi) * nc + ci;
      const int64_t ap = ((int64_t)kp * nv + vp) * nc + cp;
      dst[u] = tm.out + al + ap * tm.ld;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) o[u] = dst[u][0];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int rx = r0 + u;
      const uint64_t hx = HX[rx / 2], lx = LX[rx / 2], hy = HY[rx / 2], ly = LY[rx / 2];
      const bool odd = rx & 1;
      o[u].x -= f32_to_f64_bits(scale_hi_lo(sc, odd ? hi_of(hx) : lo_of(hx), odd ? hi_of(lx) : lo_of(lx)));
      o[u].y -= f32_to_f64_bits(scale_hi_lo(sc, odd ? hi_of(hy) : lo_of(hy), odd ? hi_of(ly) : lo_of(ly)));
      dst[u][0] = o[u];
    }
  }
  return true;
}

template <int P>
__global__ void __launch_bounds__(S2_THREADS, 1)
gemm_split_bf16_direct(const __grid_constant__ CUtensorMap tmA,
                       const __grid_constant__ CUtensorMap tmB, const Tile* __restrict__ tiles,
                       int ntiles, GemmShape sh, const S2Term* __restrict__ terms, int* err) {
  extern __shared__ uint8_t smem_raw[];
  Pipe pp;
  pp.smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  pp.sbytes = stage_bytes(sh);
  pp.a_bytes = (uint32_t)a_planes(sh.pieces) * a_plane_bytes();
  uint8_t* xraw = pp.smem + (size_t)sh.stages * pp.sbytes;   // [S2_XSLOTS][S2_RAW_BYTES]
  uint8_t* xf = xraw + S2_XSLOTS * S2_RAW_BYTES;              // [2][S2_XF_BYTES]
  pp.full = reinterpret_cast<uint64_t*>(xf + 2 * S2_XF_BYTES);
  pp.empty = pp.full + sh.stages;
  pp.tmem_full = pp.empty + sh.stages;
  pp.tmem_empty = pp.tmem_full + 2;
  uint64_t* xfull = pp.tmem_empty + 2;
  uint64_t* xempty = xfull + S2_XSLOTS;
  pp.drain = xempty + S2_XSLOTS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(pp.drain + 1);
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < sh.stages; ++s) {
      mbar_init(&pp.full[s], 1);
      mbar_init(&pp.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&pp.tmem_full[b], 1);
      mbar_init(&pp.tmem_empty[b], 4);
    }
    for (int b = 0; b < S2_XSLOTS; ++b) {
      mbar_init(&xfull[b], 1);
      mbar_init(&xempty[b], 1);
    }
    mbar_init(pp.drain, 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, sh.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int units = num_units(ntiles, sh.group);
  UnitQueue uq_static{};   // no counter: the static order b, b + gridDim.x, ...

  if (warp == 0) {
    if (lane == 0) producer_role(pp, &tmA, &tmB, tiles, ntiles, sh, &abort_flag, err, uq_static);
  } else if (warp == 1) {
    if (lane == 0) mma_role<P>(pp, tmem_base, ntiles, sh, &abort_flag, err, uq_static);
  } else if (warp == 6) {
    // ---------------- pair-side loader ----------------
    int xs = 0;
    uint32_t xph = 0;
    int pending[S2_XSLOTS];
    for (int b = 0; b < S2_XSLOTS; ++b) pending[b] = -1;
    bool ok = true;
    for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const int t0 = u * sh.group;
      const Tile tg = tiles[t0];
      const S2Term& tm = terms[tg.prob];
      const CUtensorMap* xmap = tm.xmap;
      const int rows_x = tm.rows_x, nk = tm.nk;
      const int npairs = (tg.m_valid + tm.rows_t - 1) / tm.rows_t;   // <= 128
      const int64_t slot0 = ((int64_t)tg.out_row0 - tm.a_row0) / tm.rows_t;
      const uint32_t box_bytes = (uint32_t)rows_x * 16u * 8u;
      // first map row of each of this lane's pairs (j = lane + 32 i)
      int y[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int j = lane + 32 * i;
        y[i] = 0;
        if (j < npairs) {
          const int pair = tm.perm[slot0 + j];
          if (pair >= 0) {   // a padding slot reads pair 0's rows (its T rows are zero)
            const int kl = pair / nk, kp = pair - kl * nk;
            y[i] = (tm.x_transpose_pair ? kp * nk + tm.k_begin + kl : pair) * rows_x;
          }
        }
      }
      for (int t = t0; t < min(ntiles, t0 + sh.group) && ok; ++t) {
        const Tile tl = tiles[t];
        for (int g0 = tl.n0; g0 < tl.n0 + tl.n_valid; g0 += S2_GB) {
          int w = 1;
          if (lane == 0) w = mbar_wait(&xempty[xs], xph ^ 1, &abort_flag, err, sh.wait) ? 1 : 0;
          w = __shfl_sync(0xffffffffu, w, 0);
          if (!w) {
            ok = false;
            break;
          }
          if (lane == 0) {
            mbar_expect_tx(&xfull[xs], (uint32_t)npairs * box_bytes);
            pending[xs] = (int)xph;
          }
          __syncwarp();
          uint8_t* dst0 = xraw + (size_t)xs * S2_RAW_BYTES;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int j = lane + 32 * i;
            if (j < npairs) tma_load_2d(dst0 + (size_t)j * box_bytes, xmap, 2 * g0, y[i], &xfull[xs]);
          }
          if (++xs == S2_XSLOTS) {
            xs = 0;
            xph ^= 1;
          }
        }
      }
    }
    if (lane == 0 && abort_flag) {   // let issued copies land before shared memory goes away
      long long t0 = clock64();
      for (int b = 0; b < S2_XSLOTS; ++b)
        if (pending[b] >= 0)
          while (!mbar_try_wait(&xfull[b], (uint32_t)pending[b]) && clock64() - t0 < WAIT_CYCLES) {
          }
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    EpiCtx cx{tiles, ntiles, sh, terms, err, &abort_flag, pp, xraw, xf, xfull, xempty, tmem_base,
              (int)threadIdx.x - 64, warp & 3, lane};
    EpiState st{};
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
      const int rows_x = terms[tiles[u * sh.group].prob].rows_x;
      const bool ok = rows_x == 16 ? direct_unit<16>(cx, st, u) : direct_unit<4>(cx, st, u);
      if (!ok) break;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, sh.tmem_cols);
  }
}

}  // namespace tc
}  // namespace bse
