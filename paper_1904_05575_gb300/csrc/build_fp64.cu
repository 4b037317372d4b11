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
#include <vector>

#include "bse_internal.h"
#include "zgemm.cuh"

namespace bse {
namespace {

// ---------------------------------------------------------------------------
// problem functors
// ---------------------------------------------------------------------------
struct ExchangeProb {     // Eq. vrrofM; epilogue initialises A and B
  int M, N, K;
  const bse_c128* mx;     // [n][ng]
  const double* vbar;
  const double *e_v, *e_c;
  int nv, nc;
  double scale;           // 2 gamma_x kappa
  bse_c128 *A, *B;
  int64_t ld;
  __device__ cplx a(int, int m, int k) const {
    cplx v = conj(ldc(mx + (int64_t)m * K + k));
    double s = vbar[k];
    return {v.x * s, v.y * s};
  }
  __device__ cplx b(int, int n, int k) const { return ldc(mx + (int64_t)n * K + k); }
  __device__ void store(int, int m, int n, cplx v) const {
    double2 val = make_double2(scale * v.x, scale * v.y);
    int64_t off = (int64_t)m + (int64_t)n * ld;
    if (B) reinterpret_cast<double2*>(B)[off] = val;
    if (m == n) val.x += trans_energy(e_v, e_c, nv, nc, m);
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
// and A[(k v c)][(k' v' c')] -= gamma_c kappa out.
struct Stage2RRProb {
  int M, N, K;            // M = nv^2, N = nc^2, K = ng
  const bse_c128* l;      // [npair][M][ng]
  const bse_c128* r;      // [npair][N][ng]
  int nk, nv, nc;
  double scale;           // gamma_c kappa
  bse_c128* A;
  int64_t ld;
  __device__ cplx a(int p, int m, int k) const {
    return conj(ldc(l + ((int64_t)p * M + m) * K + k));
  }
  __device__ cplx b(int p, int n, int k) const { return ldc(r + ((int64_t)p * N + n) * K + k); }
  __device__ void store(int p, int m, int n, cplx v) const {
    int k = p / nk, kp = p % nk;
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
// and B[(k v c)][(k' v' c')] -= gamma_c kappa out.
struct Stage2RAProb {
  int M, N, K;            // M = N = nv * nc
  const bse_c128* nvc;    // [nk][nk][nv*nc][ng]
  const bse_c128* t;      // [npair][nv*nc][ng]
  int nk, nv, nc;
  double scale;
  bse_c128* B;
  int64_t ld;
  __device__ cplx a(int p, int m, int k) const {
    int kk = p / nk, kp = p % nk;
    int64_t pt = (int64_t)kp * nk + kk;
    return conj(ldc(nvc + (pt * M + m) * K + k));
  }
  __device__ cplx b(int p, int n, int k) const { return ldc(t + ((int64_t)p * N + n) * K + k); }
  __device__ void store(int p, int m, int n, cplx v) const {
    int k = p / nk, kp = p % nk;
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

}  // namespace

void build_fp64(const Problem& pr, cudaStream_t s) {
  const bse_problem& p = pr.p;
  const int nk = p.nk, nv = p.nv, nc = p.nc, ng = p.ng;
  const int npair = nk * nk;
  const double kap = pr.kappa;

  // 1. exchange: initialises A and B
  {
    ExchangeProb P{(int)pr.n, (int)pr.n, ng, p.m_x, p.v_bar, p.e_v, p.e_c, nv, nc,
                   2.0 * p.gamma_x * kap, p.A, p.coupling ? p.B : nullptr, p.ld};
    Phase ph("fp64_exchange", s);
    launch_zgemm(P, 1, s);
  }
  if (p.gamma_c == 0.0) return;

  const int s_rr = nv * nv < nc * nc ? nv * nv : nc * nc;
  const int rows_max = s_rr > nv * nc ? s_rr : (p.coupling ? nv * nc : s_rr);
  DeviceBuffer tbuf((size_t)npair * rows_max * ng * sizeof(bse_c128), s);
  bse_c128* t = tbuf.as<bse_c128>();

  // 2./3. W^rr (Eq. wrrm)
  if (nc * nc <= nv * nv) {
    Stage1WProb P1{nc * nc, ng, ng, p.m_cc, p.w, p.q_minus, t};
    {
      Phase ph("fp64_wrr_stage1", s);
      launch_zgemm(P1, npair, s);
    }
    Stage2RRProb P2{nv * nv, nc * nc, ng, p.m_vv, t, nk, nv, nc, p.gamma_c * kap, p.A, p.ld};
    Phase ph("fp64_wrr_stage2", s);
    launch_zgemm(P2, npair, s);
  } else {
    Stage1WHProb P1{nv * nv, ng, ng, p.m_vv, p.w, p.q_minus, t};
    {
      Phase ph("fp64_wrr_stage1", s);
      launch_zgemm(P1, npair, s);
    }
    Stage2RRProb P2{nv * nv, nc * nc, ng, t, p.m_cc, nk, nv, nc, p.gamma_c * kap, p.A, p.ld};
    Phase ph("fp64_wrr_stage2", s);
    launch_zgemm(P2, npair, s);
  }
  if (!p.coupling) return;

  // 2./3. W^ra (Eq. wrabar)
  Stage1WProb P1{nv * nc, ng, ng, p.n_vc, p.w, p.q_plus, t};
  {
    Phase ph("fp64_wra_stage1", s);
    launch_zgemm(P1, npair, s);
  }
  Stage2RAProb P2{nv * nc, nv * nc, ng, p.n_vc, t, nk, nv, nc, p.gamma_c * kap, p.B, p.ld};
  Phase ph("fp64_wra_stage2", s);
  launch_zgemm(P2, npair, s);
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
  const bse_problem& p = pr.p;
  if (p.gamma_c == 0.0) return 0;
  const int nv = p.nv, nc = p.nc;
  const int s_rr = nv * nv < nc * nc ? nv * nv : nc * nc;
  const int rows_max = s_rr > nv * nc ? s_rr : (p.coupling ? nv * nc : s_rr);
  return (size_t)p.nk * p.nk * rows_max * p.ng * sizeof(bse_c128);
}

void build_fp64_static(const Problem& pr, cudaStream_t s) {
  const bse_problem& p = pr.p;
  const int nk = p.nk, nv = p.nv, nc = p.nc, ng = p.ng;
  const int npair = nk * nk;
  const double kap = pr.kappa;
  const size_t need = fp64_static_scratch_need(pr);
  if (need > kFp64StaticScratchBytes)
    throw Error(BSE_ERR_ARG, "problem needs " + std::to_string(need) +
                                 " bytes of stage-1 scratch; the fixed scratch holds " +
                                 std::to_string(kFp64StaticScratchBytes) + " bytes");
  // first call on a device: looks up the array's device address (no allocation)
  bse_c128* t = static_cast<bse_c128*>(static_scratch_for_current_device());

  ExchangeProb PX{(int)pr.n, (int)pr.n, ng, p.m_x, p.v_bar, p.e_v, p.e_c, nv, nc,
                  2.0 * p.gamma_x * kap, p.A, p.coupling ? p.B : nullptr, p.ld};
  launch_zgemm(PX, 1, s);
  if (p.gamma_c == 0.0) return;
  // the intermediate is fully written by each stage 1 before its stage 2 reads
  // it, so nothing in the shared array has to start at zero
  if (nc * nc <= nv * nv) {
    launch_zgemm(Stage1WProb{nc * nc, ng, ng, p.m_cc, p.w, p.q_minus, t}, npair, s);
    launch_zgemm(Stage2RRProb{nv * nv, nc * nc, ng, p.m_vv, t, nk, nv, nc, p.gamma_c * kap,
                              p.A, p.ld}, npair, s);
  } else {
    launch_zgemm(Stage1WHProb{nv * nv, ng, ng, p.m_vv, p.w, p.q_minus, t}, npair, s);
    launch_zgemm(Stage2RRProb{nv * nv, nc * nc, ng, t, p.m_cc, nk, nv, nc, p.gamma_c * kap,
                              p.A, p.ld}, npair, s);
  }
  if (!p.coupling) return;
  launch_zgemm(Stage1WProb{nv * nc, ng, ng, p.n_vc, p.w, p.q_plus, t}, npair, s);
  launch_zgemm(Stage2RAProb{nv * nc, nv * nc, ng, p.n_vc, t, nk, nv, nc, p.gamma_c * kap, p.B,
                            p.ld}, npair, s);
}

}  // namespace bse
