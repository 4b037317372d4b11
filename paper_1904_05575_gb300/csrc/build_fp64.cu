// Plain FP64 build of the BSE Hamiltonian on CUDA cores.
//
// Exchange (Eq. vrrofM), direct resonant-resonant (Eq. wrrm) and direct
// resonant-antiresonant (Eq. wrabar) terms are batched complex GEMMs over
// the plane-wave index; the assembly of Eqs. diagonalblock / couplingblock
// happens in their epilogues:
//   1. exchange GEMM       V = M_x^H diag(v_bar) M_x   -> writes A = E + 2 gx k V, B = 2 gx k V
//   2. direct, stage 1     T_p = M_side(p) W(q(p))^T   (one small GEMM per k-pair p)
//   3. direct, stage 2     P_p = M_other(p)^* T_p^T    -> A (or B) -= gc k P_p, scattered
// Stage 1 applies W to whichever pair side is smaller (s_rr = min(nv^2, nc^2)).
#include <cuda_runtime.h>

#include <mutex>
#include <optional>
#include <vector>

#include "bse_internal.h"
#include "zgemm.cuh"

namespace bse {
namespace {

// ---------------------------------------------------------------------------
// problem functors
// ---------------------------------------------------------------------------
struct ExchangeProb {     // Eq. vrrofM; epilogue initialises rows m0 .. m0+M-1 of A and B
  int M, N, K;
  const bse_c128* mx;     // [n][ng]
  const double* vbar;
  const double *e_v, *e_c;
  int nv, nc;
  double scale;           // 2 gamma_x kappa
  bse_c128 *A, *B;
  int64_t ld;
  int64_t m0;             // first row (a k-row slab)
  __device__ cplx a(int, int m, int k) const {
    cplx v = conj(ldc(mx + (m0 + m) * K + k));
    double s = vbar[k];
    return {v.x * s, v.y * s};
  }
  __device__ cplx b(int, int n, int k) const { return ldc(mx + (int64_t)n * K + k); }
  __device__ void store(int, int m, int n, cplx v) const {
    double2 val = make_double2(scale * v.x, scale * v.y);
    const int64_t row = m0 + m;
    int64_t off = row + (int64_t)n * ld;
    if (B) reinterpret_cast<double2*>(B)[off] = val;
    if (row == n) val.x += trans_energy(e_v, e_c, nv, nc, (int)row);
    reinterpret_cast<double2*>(A)[off] = val;
  }
};

// Stage 1, W applied to rows of X (K = G' contiguous): T[p][r][G] = sum_G' W_q[G][G'] X_p[r][G']
struct Stage1WProb {
  int M, N, K;            // M = rows per pair, N = K = ng
  const bse_c128* x;      // [npair][M][ng]
  const bse_c128* w;      // [nq][ng][ng]
  const int32_t* qmap;    // [npair]
  bse_c128* t;            // [npair][M][ng]
  __device__ cplx a(int p, int m, int k) const { return ldc(x + ((int64_t)p * M + m) * K + k); }
  __device__ cplx b(int p, int n, int k) const {
    return ldc(w + ((int64_t)qmap[p] * N + n) * K + k);
  }
  __device__ void store(int p, int m, int n, cplx v) const {
    reinterpret_cast<double2*>(t)[((int64_t)p * M + m) * N + n] = make_double2(v.x, v.y);
  }
};

// Stage 1, W^H applied: U[p][r][G'] = sum_G conj(W_q[G][G']) X_p[r][G]
struct Stage1WHProb {
  int M, N, K;
  const bse_c128* x;
  const bse_c128* w;
  const int32_t* qmap;
  bse_c128* t;
  __device__ cplx a(int p, int m, int k) const { return ldc(x + ((int64_t)p * M + m) * K + k); }
  __device__ cplx b(int p, int n, int k) const {
    return conj(ldc(w + ((int64_t)qmap[p] * K + k) * N + n));
  }
  __device__ void store(int p, int m, int n, cplx v) const {
    reinterpret_cast<double2*>(t)[((int64_t)p * M + m) * N + n] = make_double2(v.x, v.y);
  }
};

// Stage 2 of W^rr: out[(v v')][(c c')] = sum_G conj(L_p[row][G]) R_p[col][G]
//   cc-side T:  L = m_vv (rows v v'), R = T   (cols c c')
//   vv-side U:  L = U    (rows v v'), R = m_cc (cols c c')
// and A[(k v c)][(k' v' c')] -= gamma_c kappa out.  Pair p = (k - k0) nk + k'.
struct Stage2RRProb {
  int M, N, K;            // M = nv^2, N = nc^2, K = ng
  const bse_c128* l;      // [npair][M][ng]
  const bse_c128* r;      // [npair][N][ng]
  int nk, nv, nc, k0;
  double scale;           // gamma_c kappa
  bse_c128* A;
  int64_t ld;
  __device__ cplx a(int p, int m, int k) const {
    return conj(ldc(l + ((int64_t)p * M + m) * K + k));
  }
  __device__ cplx b(int p, int n, int k) const { return ldc(r + ((int64_t)p * N + n) * K + k); }
  __device__ void store(int p, int m, int n, cplx v) const {
    int k = k0 + p / nk, kp = p % nk;
    int vi = m / nv, vp = m % nv, ci = n / nc, cp = n % nc;
    int64_t al = ((int64_t)k * nv + vi) * nc + ci;
    int64_t ap = ((int64_t)kp * nv + vp) * nc + cp;
    double2* dst = reinterpret_cast<double2*>(A) + al + ap * ld;
    double2 o = *dst;
    o.x -= scale * v.x;
    o.y -= scale * v.y;
    *dst = o;
  }
};

// Stage 2 of W^ra: out[(v' c)][(v c')] = sum_G conj(n_vc[k'][k][v'][c][G]) T_p[(v c')][G]
// and B[(k v c)][(k' v' c')] -= gamma_c kappa out.  Pair p = (k - k0) nk + k'.
struct Stage2RAProb {
  int M, N, K;            // M = N = nv * nc
  const bse_c128* nvc;    // [nk][nk][nv*nc][ng], whole
  const bse_c128* t;      // [npair][nv*nc][ng]
  int nk, nv, nc, k0;
  double scale;
  bse_c128* B;
  int64_t ld;
  __device__ cplx a(int p, int m, int k) const {
    int kk = k0 + p / nk, kp = p % nk;
    int64_t pt = (int64_t)kp * nk + kk;
    return conj(ldc(nvc + (pt * M + m) * K + k));
  }
  __device__ cplx b(int p, int n, int k) const { return ldc(t + ((int64_t)p * N + n) * K + k); }
  __device__ void store(int p, int m, int n, cplx v) const {
    int k = k0 + p / nk, kp = p % nk;
    int vp = m / nc, ci = m % nc;     // row (v', c)
    int vi = n / nc, cp = n % nc;     // col (v, c')
    int64_t al = ((int64_t)k * nv + vi) * nc + ci;
    int64_t ap = ((int64_t)kp * nv + vp) * nc + cp;
    double2* dst = reinterpret_cast<double2*>(B) + al + ap * ld;
    double2 o = *dst;
    o.x -= scale * v.x;
    o.y -= scale * v.y;
    *dst = o;
  }
};

// Stage-1 scratch rows per pair: the larger of the two direct terms' sides.
int fp64_rows_max(const bse_problem& p) {
  const int nv = p.nv, nc = p.nc;
  const int s_rr = nv * nv < nc * nc ? nv * nv : nc * nc;
  return s_rr > nv * nc ? s_rr : (p.coupling ? nv * nc : s_rr);
}

// A phase timer only where the caller asks for one (the allocation-free
// entry point records no events).
struct MaybePhase {
  std::optional<Phase> ph;
  MaybePhase(bool on, const char* name, cudaStream_t s) {
    if (on) ph.emplace(name, s);
  }
};

// The three steps of the build for the slab's pairs p = (k - kb) nk + k',
// with the stage-1 intermediate in t ([slab pairs][rows_max][ng]).
void run_fp64(const Problem& pr, bse_c128* t, cudaStream_t s, bool timed) {
  const bse_problem& p = pr.p;
  const int nk = p.nk, nv = p.nv, nc = p.nc, ng = p.ng, kb = pr.kb;
  const int npair = (int)pr.slab_pairs();
  const double kap = pr.kappa;
  const int64_t pair_off = (int64_t)kb * nk;   // first pair of the slab in the whole arrays

  // 1. exchange: initialises the slab's rows of A and B
  {
    ExchangeProb P{(int)pr.rows(), (int)pr.n, ng, p.m_x, p.v_bar, p.e_v, p.e_c, nv, nc,
                   2.0 * p.gamma_x * kap, p.A, p.coupling ? p.B : nullptr, p.ld, pr.row0()};
    MaybePhase ph(timed, "fp64_exchange", s);
    launch_zgemm(P, 1, s);
  }
  if (p.gamma_c == 0.0) return;

  // 2./3. W^rr (Eq. wrrm); m_vv and m_cc hold the slab's rows only
  if (nc * nc <= nv * nv) {
    Stage1WProb P1{nc * nc, ng, ng, p.m_cc, p.w, p.q_minus + pair_off, t};
    {
      MaybePhase ph(timed, "fp64_wrr_stage1", s);
      launch_zgemm(P1, npair, s);
    }
    Stage2RRProb P2{nv * nv, nc * nc, ng, p.m_vv, t, nk, nv, nc, kb, p.gamma_c * kap, p.A, p.ld};
    MaybePhase ph(timed, "fp64_wrr_stage2", s);
    launch_zgemm(P2, npair, s);
  } else {
    Stage1WHProb P1{nv * nv, ng, ng, p.m_vv, p.w, p.q_minus + pair_off, t};
    {
      MaybePhase ph(timed, "fp64_wrr_stage1", s);
      launch_zgemm(P1, npair, s);
    }
    Stage2RRProb P2{nv * nv, nc * nc, ng, t, p.m_cc, nk, nv, nc, kb, p.gamma_c * kap, p.A, p.ld};
    MaybePhase ph(timed, "fp64_wrr_stage2", s);
    launch_zgemm(P2, npair, s);
  }
  if (!p.coupling) return;

  // 2./3. W^ra (Eq. wrabar): stage 1 on the slab's rows of n_vc, stage 2 reads
  // the swapped pairs (k', k) from the whole array
  Stage1WProb P1{nv * nc, ng, ng, p.n_vc + pair_off * nv * nc * ng, p.w, p.q_plus + pair_off, t};
  {
    MaybePhase ph(timed, "fp64_wra_stage1", s);
    launch_zgemm(P1, npair, s);
  }
  Stage2RAProb P2{nv * nc, nv * nc, ng, p.n_vc, t, nk, nv, nc, kb, p.gamma_c * kap, p.B, p.ld};
  MaybePhase ph(timed, "fp64_wra_stage2", s);
  launch_zgemm(P2, npair, s);
}

}  // namespace

void build_fp64(const Problem& pr, cudaStream_t s) {
  const size_t bytes = pr.p.gamma_c == 0.0 ? 0 :
      (size_t)pr.slab_pairs() * fp64_rows_max(pr.p) * pr.p.ng * sizeof(bse_c128);
  DeviceBuffer tbuf(bytes, s);
  run_fp64(pr, tbuf.as<bse_c128>(), s, true);
}

}  // namespace bse

// ---------------------------------------------------------------------------
// FP64 build without any device allocation: the stage-1 intermediate lives in
// a fixed array compiled into this module instead of stream-ordered workspace.
// ---------------------------------------------------------------------------
namespace bse {

// Fixed scratch for build_fp64_static.  Every GPU that loads this module holds
// it until the process exits; calls share it.
static __device__ __align__(256) unsigned char g_fp64_static_scratch[kFp64StaticScratchBytes];

namespace {
std::mutex g_static_mutex;
std::vector<void*> g_static_scratch_ptr;   // device address of the array, per device

// Host code cannot use the array's name as a device address (on the host it is
// only a stand-in); the address is looked up once per device, with that
// device current, and cached.
void* static_scratch_for_current_device() {
  int dev = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if ((int)g_static_scratch_ptr.size() <= dev) g_static_scratch_ptr.resize(dev + 1, nullptr);
  if (!g_static_scratch_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_fp64_static_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      (void)cudaGetLastError();
      throw Error(BSE_ERR_CUDA, std::string("cudaGetSymbolAddress of the fixed scratch failed: ") +
                                    cudaGetErrorString(e));
    }
    g_static_scratch_ptr[dev] = ptr;
  }
  return g_static_scratch_ptr[dev];
}
}  // namespace

size_t fp64_static_scratch_need(const Problem& pr) {
  if (pr.p.gamma_c == 0.0) return 0;
  return (size_t)pr.slab_pairs() * fp64_rows_max(pr.p) * pr.p.ng * sizeof(bse_c128);
}

void build_fp64_static(const Problem& pr, cudaStream_t s) {
  const size_t need = fp64_static_scratch_need(pr);
  if (need > kFp64StaticScratchBytes)
    throw Error(BSE_ERR_ARG, "problem needs " + std::to_string(need) +
                                 " bytes of stage-1 scratch; the fixed scratch holds " +
                                 std::to_string(kFp64StaticScratchBytes) + " bytes");
  // first call on a device: looks up the array's device address (no allocation);
  // the intermediate is fully written by each stage 1 before its stage 2 reads
  // it, so nothing in the shared array has to start at zero
  run_fp64(pr, static_cast<bse_c128*>(static_scratch_for_current_device()), s, false);
}

}  // namespace bse
