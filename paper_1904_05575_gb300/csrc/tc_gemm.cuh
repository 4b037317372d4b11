// Split-precision complex GEMM on the 5th-generation tensor cores (tcgen05).
//
//   C[m][n] = sum_k A[m][k] * B[n][k]      (complex, FP32 accumulation)
//
// Both operands are stored pre-split as BF16 planes, x = x_0 + x_1 + x_2 with
// each x_i a BF16 number.  The A operand (tile rows) has 2P planes: plane
// (comp * P + piece) holds piece `piece` of the real (comp 0) or imaginary
// (comp 1) part.  The B operand (tile columns) has 3P planes, three per
// piece: plane 3 j holds -Im_j, 3 j + 1 Re_j and 3 j + 2 Im_j, so that the
// nt rows of Re_j followed by those of Im_j, and the nt rows of -Im_j
// followed by those of Re_j, are each one operand of 2 nt rows.  For each K
// step of 16 the kernel issues, for every piece pair (i, j) with i + j < P,
// two MMAs of N = 2 nt into the accumulator pair [re | im] (nt columns each):
//   [re | im] += A_re,i [B_re,j ; B_im,j]^T  +  A_im,i [-B_im,j ; B_re,j]^T
// i.e. re += A_re,i B_re,j - A_im,i B_im,j and im += A_re,i B_im,j + A_im,i B_re,j,
// half as many instructions of twice the width as four MMAs of N = nt, and a
// third fewer shared-memory bytes per multiply-add (the A planes are read
// once per pair of products instead of once per product).
// The leading products (i = j = 0) go to a "main" pair of TMEM accumulators
// and all correction products (i + j > 0, 2^-8 smaller) to a separate pair:
// the tensor core's FP32 accumulation loses low bits at every accumulate
// event, and this keeps the large accumulator at 2 events per K step instead
// of 2 * (number of products).  The epilogue adds main + correction.  For
// long K (more than 12 steps) the K range is cut into ksegs segments, each
// accumulated afresh in the next TMEM set, and the epilogue sums the
// segments in FP32 registers, so no accumulator sees more than 16 events.
// Conjugation of an operand is applied when it is split (Im stored negated).
//
// One CTA per SM, persistent over a list of 128-row tiles:
//   warp 0     TMA producer: one 3-D box per operand per stage (all planes)
//   warp 1     TMEM allocation and MMA issue (one elected thread)
//   warps 2-9  epilogue: tcgen05.ld of D_re / D_im, then the store functor;
//              two warps per TMEM lane quarter (a warp reaches the 32 lanes
//              32 (warp % 4) ...), each taking every other 32-column chunk,
//              so that the stores of one tile (FP64 read-modify-writes, split
//              planes) run on twice as many warps and overlap the next tile's
//              MMAs (timing variants showed the 4-warp epilogue bounding the
//              launch: without MMAs or without operand copies the launches
//              were only 6-20 % shorter)
// Shared-memory tiles are K-major with the 32-byte swizzle (one K step of 16
// BF16 = 32 bytes per row), the layout TMA writes and the MMA descriptor
// reads.  Every pipeline wait on an mbarrier is bounded by a clock budget
// (GemmShape::wait, set at run time); on expiry the thread records
// ERR_TIMEOUT in *err and every role winds down: the producer waits for the
// copies it issued to land and the MMA issuer for the MMAs it issued to
// complete (each with the fixed budget WAIT_CYCLES), then TMEM is released
// and the kernel returns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace bse {
namespace tc {

constexpr int BM = 128;             // tile rows (UMMA M)
constexpr int BK = 16;              // K elements per stage (32 bytes of BF16)
constexpr int NUM_THREADS = 320;    // 10 warps: producer, MMA issuer, 8 epilogue
constexpr int EPI_WARPS = 8;        // two per TMEM lane quarter, alternate 32-column chunks
constexpr int ERR_TIMEOUT = 1;
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz: default budget, and the
                                                  // bound of every wind-down wait

struct Tile {
  int a_row0;    // first row in the A planes
  int m_valid;   // real rows of this tile (<= 128)
  int b_row0;    // first row in the B planes
  int n0;        // first output column
  int n_valid;   // real output columns (<= nt)
  int out_row0;  // first output row
  int prob;      // problem of a batched launch (0 otherwise)
  int kc0 = 0;   // first K step of the tile's K range (split K: partial sums per range)
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false (after
// recording the timeout) if `budget` clock cycles pass or another role has
// already failed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, long long budget) {
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > budget) {
      *abort_flag = 1;
      atomicOr(err, ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 32-byte swizzle, 8-row groups
// 256 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw32(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)1 << 16;                            // leading byte offset (unused here)
  d |= (uint64_t)(256 >> 4) << 32;                   // stride byte offset
  d |= (uint64_t)1 << 46;                            // version
  d |= (uint64_t)6 << 61;                            // layout: 32-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> F32, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n, bool neg_a) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((neg_a ? 1u : 0u) << 13) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct GemmShape {    // stages <= 8
  int nt;          // output columns per tile (multiple of 32, <= 128: 4 accumulators in TMEM)
  int kchunks;     // padded K / 16
  int pieces;      // BF16 pieces per real number (2 or 3)
  int stages;      // pipeline depth
  int acc_bufs;    // accumulator sets in TMEM (2: epilogue of one tile overlaps the next)
  uint32_t tmem_cols;
  int group = 1;   // consecutive tiles a CTA takes as one work unit
  int ksegs = 1;   // K segments per tile (> 1 needs nt <= 64 and acc_bufs == 2)
  long long wait = WAIT_CYCLES;   // clock-cycle budget of each pipeline wait
};

__host__ __device__ inline uint32_t a_plane_bytes() { return BM * BK * 2; }
__host__ __device__ inline uint32_t b_plane_bytes(int nt) { return (uint32_t)nt * BK * 2; }
// planes of each operand: A 2P (Re, Im), B 3P (-Im, Re, Im)
__host__ __device__ inline int a_planes(int pieces) { return 2 * pieces; }
__host__ __device__ inline int b_planes(int pieces) { return 3 * pieces; }
__host__ __device__ inline uint32_t stage_bytes(const GemmShape& s) {
  return (uint32_t)a_planes(s.pieces) * a_plane_bytes() +
         (uint32_t)b_planes(s.pieces) * b_plane_bytes(s.nt);
}
__host__ inline size_t gemm_smem_bytes(const GemmShape& s) {
  return 1024 /* alignment slack */ + (size_t)s.stages * stage_bytes(s) + 64 * 8;   // + barriers
}

// ---------------------------------------------------------------------------
// Work distribution: CTA b takes work units b, b + gridDim.x, ...; unit u is
// the tiles [u * group, (u + 1) * group) (the last unit may be shorter).
// Every role walks the same sequence.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int num_units(int ntiles, int group) { return (ntiles + group - 1) / group; }

// Work-unit hand-out.  Static (no counter): CTA b takes the units b,
// b + gridDim.x, ... .  Dynamic (a zeroed device counter): the producer takes
// the next unit with an atomicAdd and passes it to the MMA issuer and the
// epilogue warps through a ring in shared memory (-1: no more units), so the
// units in flight are always about the gridDim.x lowest not yet taken.  With
// the static order a CTA that runs ahead drifts rounds away from the others
// and the tiles that share an operand tile (a pair block's row tiles, the
// column tiles of one row tile) no longer run at the same time: the operand
// is read from DRAM again instead of from L2.
constexpr int UQ = 4;   // ring depth (units the producer may run ahead)
struct UnitQueue {
  int* counter;         // global, zeroed before the launch; NULL = static order
  volatile int* ring;   // [UQ]
  uint64_t* full;       // [UQ] unit written (producer)
  uint64_t* empty;      // [UQ] unit read (the MMA issuer and every epilogue warp)
};
struct UnitCursor {     // one consumer's (or the producer's) position
  int slot = 0;
  uint32_t phase = 0;
  int next_static;      // static order: the next unit of this CTA
};

// The producer's next unit: >= 0 a unit, -1 none left, -2 a wait gave up.
__device__ __forceinline__ int uq_produce(const UnitQueue& q, UnitCursor& c, int units,
                                          volatile int* abort_flag, int* err, long long budget) {
  if (!q.counter) {
    const int u = c.next_static;
    c.next_static += gridDim.x;
    return u < units ? u : -1;
  }
  // claim the unit only once its ring entry is free, as late as possible
  if (!mbar_wait(&q.empty[c.slot], c.phase ^ 1, abort_flag, err, budget)) return -2;
  int u = atomicAdd(q.counter, 1);
  if (u >= units) u = -1;
  q.ring[c.slot] = u;
  mbar_arrive(&q.full[c.slot]);   // release: the ring entry is visible to the waiters
  if (++c.slot == UQ) {
    c.slot = 0;
    c.phase ^= 1;
  }
  return u;
}

// A consumer's next unit (called by one thread of the consumer).
__device__ __forceinline__ int uq_consume(const UnitQueue& q, UnitCursor& c, int units,
                                          volatile int* abort_flag, int* err, long long budget) {
  if (!q.counter) {
    const int u = c.next_static;
    c.next_static += gridDim.x;
    return u < units ? u : -1;
  }
  if (!mbar_wait(&q.full[c.slot], c.phase, abort_flag, err, budget)) return -2;
  const int u = q.ring[c.slot];
  mbar_arrive(&q.empty[c.slot]);
  if (++c.slot == UQ) {
    c.slot = 0;
    c.phase ^= 1;
  }
  return u;
}

// Shared-memory pipeline of the operand stages and the TMEM accumulator sets.
struct Pipe {
  uint8_t* smem;          // stage 0 (1024-byte aligned)
  uint64_t* full;         // [stages] operand bytes landed
  uint64_t* empty;        // [stages] MMAs that read the stage completed
  uint64_t* tmem_full;    // [2] accumulator set ready for the epilogue
  uint64_t* tmem_empty;   // [2] epilogue done with the set (EPI_WARPS warp arrivals)
  uint64_t* drain;        // [1] every MMA of this CTA completed (before TMEM is released)
  uint32_t sbytes, a_bytes;
};

// TMA producer (one thread): for each tile, each K step, one 3-D box of the A
// planes and one of the B planes into the next free stage.
__device__ __forceinline__ void producer_role(const Pipe& pp, const CUtensorMap* tmA,
                                              const CUtensorMap* tmB, const Tile* tiles, int ntiles,
                                              const GemmShape& sh, volatile int* abort_flag,
                                              int* err, const UnitQueue& uq) {
  int stage = 0;
  uint32_t phase = 0;
  int pending[8];   // parity of the latest arming of each stage, -1 = never armed
  for (int s = 0; s < 8; ++s) pending[s] = -1;
  const int units = num_units(ntiles, sh.group);
  bool ok = true;
  UnitCursor cur;
  cur.next_static = blockIdx.x;
  while (ok && !*abort_flag) {
    const int u = uq_produce(uq, cur, units, abort_flag, err, sh.wait);
    if (u < 0) break;
    for (int t = u * sh.group; t < min(ntiles, (u + 1) * sh.group) && ok; ++t) {
      const Tile tl = tiles[t];
      for (int kc = 0; kc < sh.kchunks; ++kc) {
        if (!mbar_wait(&pp.empty[stage], phase ^ 1, abort_flag, err, sh.wait)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&pp.full[stage], pp.sbytes);
        uint8_t* sa = pp.smem + (size_t)stage * pp.sbytes;
        tma_load_3d(sa, tmA, (tl.kc0 + kc) * BK, tl.a_row0, 0, &pp.full[stage]);
        tma_load_3d(sa + pp.a_bytes, tmB, (tl.kc0 + kc) * BK, tl.b_row0, 0, &pp.full[stage]);
        pending[stage] = (int)phase;
        if (++stage == sh.stages) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
  }
  if (*abort_flag) {
    // let the copies this thread issued land before shared memory goes away:
    // the latest arming of each stage completes when its bytes have arrived
    long long t0 = clock64();
    for (int s = 0; s < sh.stages; ++s)
      if (pending[s] >= 0)
        while (!mbar_try_wait(&pp.full[s], (uint32_t)pending[s]) && clock64() - t0 < WAIT_CYCLES) {
        }
  }
}

// MMA issuer (one thread).  Tile number `local` (counted over this CTA's
// tiles) accumulates into set local % acc_bufs.
template <int P>
__device__ __forceinline__ void mma_role(const Pipe& pp, uint32_t tmem_base, int ntiles,
                                         const GemmShape& sh, volatile int* abort_flag, int* err,
                                         const UnitQueue& uq) {
  int stage = 0;
  uint32_t phase = 0;
  int local = 0;
  const int nbuf = sh.acc_bufs;
  const uint32_t nt = (uint32_t)sh.nt;
  const uint32_t id2 = idesc_bf16(2 * sh.nt, false);   // N = 2 nt: [re | im] at once
  // descriptors of stage 0, plane 0; the start-address field (bytes >> 4, 14 bits)
  // is advanced by plain adds for other stages and planes (all below 256 KB)
  const uint32_t sa0 = smem_u32(pp.smem);
  const uint64_t da0 = smem_desc_sw32(sa0), db0 = smem_desc_sw32(sa0 + pp.a_bytes);
  const uint64_t dstage = pp.sbytes >> 4, dpa = a_plane_bytes() >> 4, dpb = b_plane_bytes(sh.nt) >> 4;
  const int units = num_units(ntiles, sh.group);
  const int seg_len = (sh.kchunks + sh.ksegs - 1) / sh.ksegs;
  bool ok = true;
  UnitCursor cur;
  cur.next_static = blockIdx.x;
  while (ok && !*abort_flag) {
    const int u = uq_consume(uq, cur, units, abort_flag, err, sh.wait);
    if (u < 0) break;
    for (int t = u * sh.group; t < min(ntiles, (u + 1) * sh.group) && ok; ++t) {
     for (int k0 = 0; k0 < sh.kchunks; k0 += seg_len, ++local) {
      const int buf = nbuf == 2 ? (local & 1) : 0;
      const int use = nbuf == 2 ? (local >> 1) : local;    // earlier uses of this buffer
      if (use > 0 && !mbar_wait(&pp.tmem_empty[buf], (use - 1) & 1, abort_flag, err, sh.wait)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem_base + (uint32_t)buf * 4u * nt;
      const uint32_t m_ri = base;            // main [re | im], nt columns each
      const uint32_t c_ri = base + 2 * nt;   // corrections [re | im]
      for (int kc = k0; kc < min(sh.kchunks, k0 + seg_len); ++kc) {
        if (!mbar_wait(&pp.full[stage], phase, abort_flag, err, sh.wait)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t da = da0 + (uint64_t)stage * dstage, db = db0 + (uint64_t)stage * dstage;
        const uint32_t first = kc == k0 ? 0u : 1u;
        // leading products: A_re,0 [B_re,0; B_im,0] + A_im,0 [-B_im,0; B_re,0]
        mma_bf16(m_ri, da, db + 1 * dpb, id2, first);
        mma_bf16(m_ri, da + P * dpa, db, id2, 1);
        // correction products i + j in [1, P)
        uint32_t acc_c = first;
#pragma unroll
        for (int i = 0; i < P; ++i) {
#pragma unroll
          for (int j = 0; i + j < P; ++j) {
            if (i + j == 0) continue;
            mma_bf16(c_ri, da + i * dpa, db + (3 * j + 1) * dpb, id2, acc_c);
            mma_bf16(c_ri, da + (P + i) * dpa, db + (3 * j) * dpb, id2, 1);
            acc_c = 1;
          }
        }
        mma_commit(&pp.empty[stage]);   // frees this stage once its MMAs complete
        if (++stage == sh.stages) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      mma_commit(&pp.tmem_full[buf]);
     }
    }
  }
  // every MMA issued above completes before the block releases TMEM (after a
  // normal finish the epilogue has waited for them already; after an abort
  // it has not)
  mma_commit(pp.drain);
  const long long t0 = clock64();
  while (!mbar_try_wait(pp.drain, 0) && clock64() - t0 < WAIT_CYCLES) {
  }
}

// ---------------------------------------------------------------------------
// The kernel.  Epi provides: __device__ void operator()(const Tile&, int row,
// int col0, const float* re, const float* im) const  for 32 columns at col0.
// SEG: tiles accumulate K in sh.ksegs segments (compiled only where used, so
// the register arrays of the segment sums cost nothing elsewhere).
// units_taken: a device counter zeroed before the launch (dynamic hand-out of
// the work units), or NULL (static order).
// ---------------------------------------------------------------------------
template <int P, class Epi, bool SEG>
__global__ void __launch_bounds__(NUM_THREADS, 1)
gemm_split_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const Tile* __restrict__ tiles, int ntiles, GemmShape sh, Epi epi, int* err,
                int* units_taken) {
  extern __shared__ uint8_t smem_raw[];
  Pipe pp;
  pp.smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  pp.sbytes = stage_bytes(sh);
  pp.a_bytes = (uint32_t)a_planes(sh.pieces) * a_plane_bytes();
  pp.full = reinterpret_cast<uint64_t*>(pp.smem + (size_t)sh.stages * pp.sbytes);
  pp.empty = pp.full + sh.stages;
  pp.tmem_full = pp.empty + sh.stages;
  pp.tmem_empty = pp.tmem_full + 2;
  pp.drain = pp.tmem_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(pp.drain + 1);
  __shared__ volatile int abort_flag;
  __shared__ uint64_t uq_full[UQ], uq_empty[UQ];
  __shared__ int uq_ring[UQ];
  UnitQueue uq;
  uq.counter = units_taken;
  uq.ring = uq_ring;
  uq.full = uq_full;
  uq.empty = uq_empty;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int nbuf = sh.acc_bufs;                 // 1 or 2 accumulator sets of 4 * nt columns

  if (threadIdx.x == 0) {
    for (int s = 0; s < sh.stages; ++s) {
      mbar_init(&pp.full[s], 1);
      mbar_init(&pp.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&pp.tmem_full[b], 1);
      mbar_init(&pp.tmem_empty[b], EPI_WARPS);
    }
    mbar_init(pp.drain, 1);
    for (int q = 0; q < UQ; ++q) {
      mbar_init(&uq_full[q], 1);
      mbar_init(&uq_empty[q], 1 + EPI_WARPS);   // the MMA issuer and each epilogue warp
    }
    abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, sh.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) producer_role(pp, &tmA, &tmB, tiles, ntiles, sh, &abort_flag, err, uq);
  } else if (warp == 1) {
    if (lane == 0) mma_role<P>(pp, tmem_base, ntiles, sh, &abort_flag, err, uq);
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    const int quarter = warp & 3;          // TMEM lanes this warp may access
    const int half = (warp - 2) >> 2;      // chunks c0 = 32 (half + 2 i)
    const int row = quarter * 32 + lane;
    int local = 0;
    const int units = num_units(ntiles, sh.group);
    bool alive = true;
    UnitCursor cur;
    cur.next_static = blockIdx.x;
    while (alive) {
      // lane 0 takes the warp's next unit, the warp follows
      int u = 0;
      if (lane == 0) u = uq_consume(uq, cur, units, &abort_flag, err, sh.wait);
      u = __shfl_sync(0xffffffffu, u, 0);
      if (u < 0) break;
      for (int t = u * sh.group; t < min(ntiles, (u + 1) * sh.group); ++t, ++local) {
        // one lane waits, the warp follows (the tcgen05.ld below is warp-collective);
        // a warp without a chunk still waits and arrives, keeping the count per phase
        const int buf = nbuf == 2 ? (local & 1) : 0;
        const int use = nbuf == 2 ? (local >> 1) : local;
        int ok = 0;
        if (lane == 0) ok = mbar_wait(&pp.tmem_full[buf], use & 1, &abort_flag, err, sh.wait) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          alive = false;
          break;
        }
        __syncwarp();
        tc_fence_after();
        const Tile tl = tiles[t];
        if constexpr (SEG) {
          // K segments (nt <= 64: at most one chunk per warp): sum (main +
          // correction) of each segment in FP32 registers, then one store
          const int c0 = 32 * half;
          const bool mine = c0 < sh.nt;
          float run_re[32], run_im[32], a[32], b[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) run_re[j] = run_im[j] = 0.f;
          for (int sgm = 0; sgm < sh.ksegs; ++sgm) {
            if (sgm > 0) {   // the next segment's accumulator set
              ++local;
              const int bs = local & 1, us = local >> 1;
              int oks = 0;
              if (lane == 0)
                oks = mbar_wait(&pp.tmem_full[bs], us & 1, &abort_flag, err, sh.wait) ? 1 : 0;
              oks = __shfl_sync(0xffffffffu, oks, 0);
              if (!oks) {
                alive = false;
                break;
              }
              __syncwarp();
              tc_fence_after();
            }
            const int bs = local & 1;
            const uint32_t lb =
                tmem_base + (uint32_t)bs * 4u * (uint32_t)sh.nt + ((uint32_t)(quarter * 32) << 16);
            if (mine) {
              tmem_ld32(lb + (uint32_t)c0, a);
              tmem_ld32(lb + (uint32_t)(2 * sh.nt + c0), b);
#pragma unroll
              for (int j = 0; j < 32; ++j) run_re[j] += a[j] + b[j];
              tmem_ld32(lb + (uint32_t)(sh.nt + c0), a);
              tmem_ld32(lb + (uint32_t)(3 * sh.nt + c0), b);
#pragma unroll
              for (int j = 0; j < 32; ++j) run_im[j] += a[j] + b[j];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&pp.tmem_empty[bs]);
          }
          if (!alive) break;
          if (mine && row < tl.m_valid && c0 < tl.n_valid) epi(tl, row, c0, run_re, run_im);
          continue;
        }
        float re[32], im[32], cr[32], ci[32];
        const uint32_t lane_base =
            tmem_base + (uint32_t)buf * 4u * (uint32_t)sh.nt + ((uint32_t)(quarter * 32) << 16);
        for (int c0 = 32 * half; c0 < sh.nt; c0 += 64) {
          tmem_ld32(lane_base + (uint32_t)c0, re);
          tmem_ld32(lane_base + (uint32_t)(sh.nt + c0), im);
          tmem_ld32(lane_base + (uint32_t)(2 * sh.nt + c0), cr);
          tmem_ld32(lane_base + (uint32_t)(3 * sh.nt + c0), ci);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            re[j] += cr[j];
            im[j] += ci[j];
          }
          if (row < tl.m_valid && c0 < tl.n_valid) epi(tl, row, c0, re, im);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&pp.tmem_empty[buf]);
      }
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
