// The extern "C" entry points of libbse.so: argument checks on the host,
// then dispatch to the build / reduction / spectrum launchers.  No C++
// exception crosses this boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "bse_internal.h"
#include "lanczos.h"
#include "mlp.h"

namespace bse {

namespace {
thread_local std::string g_last_error;
}

void set_last_error(const std::string& msg) { g_last_error = msg; }

namespace {
std::atomic<int64_t> g_launches{0};
}
void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
struct PhaseRecord {
  std::string name;
  cudaEvent_t start, stop;
};
std::atomic<bool> g_timing{false};
std::mutex g_phase_mutex;
std::vector<PhaseRecord> g_phases;
}  // namespace

Phase::Phase(const char* name, cudaStream_t s) : name_(name), s_(s) {
  if (!g_timing.load()) return;
  if (cudaEventCreate(&start_) != cudaSuccess || cudaEventRecord(start_, s_) != cudaSuccess) {
    (void)cudaGetLastError();
    start_ = nullptr;
  }
}

Phase::~Phase() {
  if (!start_) return;
  cudaEvent_t stop = nullptr;
  if (cudaEventCreate(&stop) != cudaSuccess || cudaEventRecord(stop, s_) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaEventDestroy(start_);
    if (stop) cudaEventDestroy(stop);
    return;
  }
  std::lock_guard<std::mutex> lock(g_phase_mutex);
  g_phases.push_back({name_, start_, stop});
}

template <class F>
int guarded(F&& f) {
  try {
    f();
    g_last_error.clear();
    return BSE_OK;
  } catch (const Error& e) {
    g_last_error = e.what();
    return e.status;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return BSE_ERR_NOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return BSE_ERR_CUDA;
  } catch (...) {
    g_last_error = "unknown error";
    return BSE_ERR_CUDA;
  }
}

namespace {

std::vector<int32_t> check_q_map(const int32_t* dmap, int nk, int nq_w, const char* name,
                                 cudaStream_t s) {
  std::vector<int32_t> h((size_t)nk * nk);
  BSE_CUDA(cudaMemcpyAsync(h.data(), dmap, h.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                           s));
  BSE_CUDA(cudaStreamSynchronize(s));
  for (size_t i = 0; i < h.size(); ++i)
    if (h[i] < 0 || h[i] >= nq_w)
      throw Error(BSE_ERR_ARG, std::string(name) + "[" + std::to_string(i / nk) + "][" +
                                   std::to_string(i % nk) + "] = " + std::to_string(h[i]) +
                                   " is outside [0, nq_w = " + std::to_string(nq_w) + ")");
  return h;
}

// Keep stream-ordered workspace in the device's default pool between calls
// instead of returning it to the driver at every synchronization.
void keep_pool_memory() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  static std::mutex m;
  static std::vector<bool> done;
  std::lock_guard<std::mutex> lock(m);
  if ((int)done.size() <= dev) done.resize(dev + 1, false);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  (void)cudaGetLastError();
  done[dev] = true;
}

// Non-finite input scan: bit `bit` of *flag is set if any double of the
// array is a NaN or an infinity (exponent field all ones).  16-byte words,
// grid-stride.
__global__ void __launch_bounds__(256) k_nonfinite16(const uint4* __restrict__ p, int64_t nwords,
                                                     int bit, int* flag) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nwords;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = __ldg(p + i);
    bad = bad || ((w.y >> 20) & 0x7FFu) == 0x7FFu || ((w.w >> 20) & 0x7FFu) == 0x7FFu;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1 << bit);
}

// the same for floats (complex64 inputs)
__global__ void k_nonfinite4(const float* __restrict__ p, int64_t n, int bit, int* flag) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    bad = bad || ((__float_as_uint(p[i]) >> 23) & 0xFFu) == 0xFFu;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1 << bit);
}

__global__ void k_nonfinite8(const double* __restrict__ p, int64_t n, int bit, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t hi = (uint32_t)(__double_as_longlong(p[i]) >> 32);
    if (((hi >> 20) & 0x7FFu) == 0x7FFu) atomicOr(flag, 1 << bit);
  }
}

// Every input array of the problem read once on the device: BSE_ERR_ARG
// naming the arrays that hold a NaN or an infinity.  Syncs.
void check_finite(const bse_problem& p, int64_t kn, const std::string& at, cudaStream_t s) {
  const int64_t n = (int64_t)p.nk * p.nv * p.nc, ng = p.ng, nk = p.nk;
  // doubles: the count of 8-byte reals; f32: the complex array holds floats
  // (complex64), then `doubles` counts its floats
  struct Arr { const void* ptr; int64_t doubles; const char* name; bool f32; };
  const bool c64 = p.in_dtype == BSE_C64;
  std::vector<Arr> arrs = {{p.e_v, nk * p.nv, "e_v", false}, {p.e_c, nk * p.nc, "e_c", false},
                           {p.m_x, 2 * n * ng, "m_x", c64}, {p.v_bar, ng, "v_bar", false}};
  if (p.gamma_c != 0.0) {
    arrs.push_back({p.m_vv, 2 * kn * nk * p.nv * p.nv * ng, "m_vv", c64});
    arrs.push_back({p.m_cc, 2 * kn * nk * p.nc * p.nc * ng, "m_cc", c64});
    arrs.push_back({p.w, 2 * (int64_t)p.nq_w * ng * ng, "w", c64});
    if (p.coupling) arrs.push_back({p.n_vc, 2 * nk * nk * p.nv * p.nc * ng, "n_vc", c64});
  }
  int* flag = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&flag), sizeof(int), s) != cudaSuccess) {
    (void)cudaGetLastError();
    throw Error(BSE_ERR_NOMEM, "workspace allocation failed (input scan)");
  }
  int h = 0;
  try {
    BSE_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    for (size_t i = 0; i < arrs.size(); ++i) {
      const Arr& a = arrs[i];
      if (a.f32) {
        const int grid = (int)std::min<int64_t>((a.doubles + 255) / 256, 152 * 8);
        k_nonfinite4<<<std::max(grid, 1), 256, 0, s>>>(static_cast<const float*>(a.ptr), a.doubles,
                                                       (int)i, flag);
      } else if (a.doubles % 2 == 0 && (reinterpret_cast<uintptr_t>(a.ptr) & 15) == 0) {
        const int64_t words = a.doubles / 2;
        const int grid = (int)std::min<int64_t>((words + 255) / 256, 152 * 8);
        k_nonfinite16<<<std::max(grid, 1), 256, 0, s>>>(static_cast<const uint4*>(a.ptr), words,
                                                        (int)i, flag);
      } else {
        const int grid = (int)std::min<int64_t>((a.doubles + 255) / 256, 152 * 8);
        k_nonfinite8<<<std::max(grid, 1), 256, 0, s>>>(static_cast<const double*>(a.ptr),
                                                       a.doubles, (int)i, flag);
      }
      BSE_CUDA(cudaGetLastError());
      note_launches(1);
    }
    BSE_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaFreeAsync(flag, s));
    flag = nullptr;
    BSE_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    if (flag) cudaFreeAsync(flag, s);
    throw;
  }
  if (h) {
    std::string names;
    for (size_t i = 0; i < arrs.size(); ++i)
      if (h & (1 << i)) names += std::string(names.empty() ? "" : ", ") + arrs[i].name;
    throw Error(BSE_ERR_ARG, at + "non-finite value (NaN or infinity) in " + names);
  }
}

Problem validate(const bse_problem& p, int index, cudaStream_t s, bool scan = true) {
  const std::string at = "probs[" + std::to_string(index) + "]: ";
  BSE_CHECK_ARG(p.nk >= 1 && p.nv >= 1 && p.nc >= 1 && p.ng >= 1 && p.nq_w >= 1,
                at + "nk, nv, nc, ng and nq_w must all be >= 1");
  const int64_t n = (int64_t)p.nk * p.nv * p.nc;
  BSE_CHECK_ARG(n <= 2147483647LL / 2, at + "N = nk*nv*nc is too large");
  BSE_CHECK_ARG(p.ld >= n, at + "ld (" + std::to_string(p.ld) + ") < N (" + std::to_string(n) + ")");
  BSE_CHECK_ARG(std::isfinite(p.omega_cell) && p.omega_cell > 0.0, at + "omega_cell must be > 0");
  BSE_CHECK_ARG(std::isfinite(p.gamma_x) && std::isfinite(p.gamma_c),
                at + "gamma_x and gamma_c must be finite");
  BSE_CHECK_ARG(p.coupling == 0 || p.coupling == 1, at + "coupling must be 0 or 1");
  BSE_CHECK_ARG(p.k_begin >= 0 && p.k_count >= 0 && (int64_t)p.k_begin + p.k_count <= p.nk &&
                    (p.k_count > 0 || p.k_begin == 0),
                at + "k-row slab [k_begin, k_begin + k_count) must lie in [0, nk) "
                     "(k_begin = k_count = 0: the whole problem)");
  BSE_CHECK_ARG(p.e_v && p.e_c && p.m_x && p.v_bar && p.A, at + "NULL e_v, e_c, m_x, v_bar or A");
  if (p.gamma_c != 0.0) {
    BSE_CHECK_ARG(p.m_vv && p.m_cc && p.w && p.q_minus, at + "NULL m_vv, m_cc, w or q_minus");
    if (p.coupling) BSE_CHECK_ARG(p.n_vc && p.q_plus, at + "NULL n_vc or q_plus");
  }
  if (p.coupling) BSE_CHECK_ARG(p.B, at + "coupling = 1 needs B");
  BSE_CHECK_ARG(p.in_dtype == BSE_C128 || p.in_dtype == BSE_C64,
                at + "in_dtype must be BSE_C128 (0) or BSE_C64 (1)");
  // complex128 arrays are read and written 16 bytes at a time (vector loads,
  // bulk copies), complex64 inputs 8, real arrays 8, q maps 4
  auto aligned = [](const void* q, uintptr_t a) { return (reinterpret_cast<uintptr_t>(q) & (a - 1)) == 0; };
  const uintptr_t ca = p.in_dtype == BSE_C64 ? 8 : 16;
  BSE_CHECK_ARG(aligned(p.m_x, ca) && aligned(p.m_vv, ca) && aligned(p.m_cc, ca) &&
                    aligned(p.n_vc, ca) && aligned(p.w, ca),
                at + (ca == 16 ? "complex128 inputs must be 16-byte aligned"
                               : "complex64 inputs must be 8-byte aligned"));
  BSE_CHECK_ARG(aligned(p.A, 16) && aligned(p.B, 16), at + "A and B must be 16-byte aligned");
  BSE_CHECK_ARG(aligned(p.e_v, 8) && aligned(p.e_c, 8) && aligned(p.v_bar, 8) &&
                    aligned(p.q_minus, 4) && aligned(p.q_plus, 4),
                at + "real arrays must be 8-byte and q maps 4-byte aligned");
  Problem pr;
  if (scan) check_finite(p, p.k_count > 0 ? p.k_count : p.nk, at, s);
  if (p.gamma_c != 0.0) {
    pr.qm_host = check_q_map(p.q_minus, p.nk, p.nq_w, "q_minus", s);
    if (p.coupling) pr.qp_host = check_q_map(p.q_plus, p.nk, p.nq_w, "q_plus", s);
  }
  pr.p = p;
  pr.n = n;
  pr.kappa = kHartreeEv / ((double)p.nk * p.omega_cell);
  pr.kb = p.k_begin;
  pr.kn = p.k_count > 0 ? p.k_count : p.nk;
  return pr;
}

}  // namespace
}  // namespace bse

using namespace bse;

extern "C" int bse_build_kernel(const bse_problem* probs, int32_t nprob, int32_t precision,
                                void* cuda_stream) {
  return guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    BSE_CHECK_ARG(nprob >= 0, "nprob must be >= 0");
    if (nprob == 0) return;
    BSE_CHECK_ARG(probs != nullptr, "probs is NULL");
    BSE_CHECK_ARG(precision == BSE_PREC_FP64 || precision == BSE_PREC_BF16X6 ||
                      precision == BSE_PREC_BF16X3,
                  "unknown precision " + std::to_string(precision));
    keep_pool_memory();
    std::vector<Problem> prs;
    prs.reserve(nprob);
    for (int i = 0; i < nprob; ++i) prs.push_back(validate(probs[i], i, s));
    if (precision == BSE_PREC_FP64) {
      for (const Problem& pr : prs)
        if (pr.p.in_dtype != BSE_C128)
          throw Error(BSE_ERR_UNSUPPORTED, "the FP64 build reads complex128 inputs only");
      for (const Problem& pr : prs) build_fp64(pr, s);
    } else {
      build_mixed_batch(prs, precision, s);
    }
  });
}

extern "C" int bse_build_kernel_fp64_static(const bse_problem* prob, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(prob != nullptr, "prob is NULL");
    const Problem pr = validate(*prob, 0, static_cast<cudaStream_t>(cuda_stream), false);
    if (pr.p.in_dtype != BSE_C128)
      throw Error(BSE_ERR_UNSUPPORTED, "the FP64 build reads complex128 inputs only");
    build_fp64_static(pr, static_cast<cudaStream_t>(cuda_stream));
  });
}

extern "C" int bse_plan_create(const bse_problem* probs, int32_t nprob, int32_t precision,
                               int32_t flags, void** plan, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(plan != nullptr, "plan is NULL");
    *plan = nullptr;
    BSE_CHECK_ARG(nprob >= 1 && probs != nullptr, "need at least one problem");
    BSE_CHECK_ARG(precision == BSE_PREC_FP64 || precision == BSE_PREC_BF16X6 ||
                      precision == BSE_PREC_BF16X3,
                  "unknown precision " + std::to_string(precision));
    BSE_CHECK_ARG((flags & ~(BSE_PLAN_AUTOTUNE | BSE_PLAN_UNFUSED | BSE_PLAN_CUDA_CORE_STAGE2 |
                             BSE_PLAN_HERMITIAN | BSE_PLAN_FP64_DIAGONAL)) == 0,
                  "unknown plan flags");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    keep_pool_memory();
    std::vector<Problem> prs;
    for (int i = 0; i < nprob; ++i) prs.push_back(validate(probs[i], i, s));
    *plan = plan_create(std::move(prs), precision, flags, s);
  });
}

extern "C" int bse_plan_execute(void* plan, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(plan != nullptr, "plan is NULL");
    plan_execute(static_cast<BatchPlan*>(plan), static_cast<cudaStream_t>(cuda_stream));
  });
}

extern "C" int bse_plan_status(void* plan, void* cuda_stream) {
  int st = BSE_OK;
  int rc = guarded([&] {
    BSE_CHECK_ARG(plan != nullptr, "plan is NULL");
    st = plan_status(static_cast<BatchPlan*>(plan), static_cast<cudaStream_t>(cuda_stream));
    if (st != BSE_OK) throw Error(st, "a bounded device wait expired in a plan execute");
  });
  return rc;
}

extern "C" int bse_plan_tile_cols(const void* plan) {
  return plan ? plan_tile_cols(static_cast<const BatchPlan*>(plan)) : 0;
}

extern "C" int bse_plan_stage2_shape(const void* plan, int32_t* tile_cols, int32_t* stages) {
  return guarded([&] {
    BSE_CHECK_ARG(plan && tile_cols && stages, "NULL argument");
    int t = 0, st = 0;
    plan_stage2_shape(static_cast<const BatchPlan*>(plan), &t, &st);
    *tile_cols = t;
    *stages = st;
  });
}

extern "C" int bse_plan_fused(const void* plan) {
  return plan ? plan_fused(static_cast<const BatchPlan*>(plan)) : 0;
}

extern "C" int bse_plan_set_wait_limit(void* plan, double seconds) {
  return guarded([&] {
    BSE_CHECK_ARG(plan != nullptr, "plan is NULL");
    BSE_CHECK_ARG(seconds > 0.0 && seconds <= 60.0, "wait limit must be in (0, 60] seconds");
    plan_set_wait(static_cast<BatchPlan*>(plan), seconds);
  });
}

extern "C" void bse_plan_destroy(void* plan) { plan_destroy(static_cast<BatchPlan*>(plan)); }

extern "C" int bse_reduce(int32_t n, const bse_c128* A, const bse_c128* B, int64_t ld,
                          bse_c128* S, bse_c128* L, int32_t* failed_minor, void* cuda_stream) {
  return guarded([&] {
    if (failed_minor) *failed_minor = 0;
    BSE_CHECK_ARG(n >= 1, "n must be >= 1");
    BSE_CHECK_ARG(ld >= n, "ld < n");
    BSE_CHECK_ARG(A && S && L, "NULL A, S or L");
    BSE_CHECK_ARG(S != L && S != A && L != A && (B == nullptr || (S != B && L != B)),
                  "S and L must not alias A, B or each other");
    keep_pool_memory();
    reduce_fp64(n, A, B, ld, S, L, failed_minor, static_cast<cudaStream_t>(cuda_stream));
  });
}

extern "C" int bse_spectrum_tensor(int32_t n, const bse_c128* Z, const bse_c128* L, int64_t ld,
                                   const bse_c128* D, int64_t ldd, double c_q, double vc,
                                   int32_t n_omega, const double* omega, double delta,
                                   const double* E, bse_c128* eps_out, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(n >= 1 && ld >= n && ldd >= n, "need n >= 1, ld >= n and ldd >= n");
    BSE_CHECK_ARG(Z && L && D && E, "NULL Z, L, D or E");
    BSE_CHECK_ARG(n_omega >= 0 && (n_omega == 0 || (omega && eps_out)), "need omega and eps_out");
    BSE_CHECK_ARG(std::isfinite(delta) && delta > 0.0, "delta must be > 0");
    BSE_CHECK_ARG(std::isfinite(vc) && vc > 0.0, "vc must be > 0");
    keep_pool_memory();
    spectrum_tensor_fp64(n, Z, L, ld, D, ldd, c_q, vc, n_omega, omega, delta, E, eps_out,
                         static_cast<cudaStream_t>(cuda_stream));
  });
}

extern "C" int bse_loss_function(int32_t n_omega, const bse_c128* eps, double v_inv,
                                 double* loss_out, double* sqw_out, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(n_omega >= 0, "n_omega must be >= 0");
    BSE_CHECK_ARG(n_omega == 0 || eps, "NULL eps");
    BSE_CHECK_ARG(loss_out || sqw_out, "need loss_out or sqw_out");
    BSE_CHECK_ARG(std::isfinite(v_inv), "v_inv must be finite");
    loss_fp64(n_omega, eps, v_inv, loss_out, sqw_out, static_cast<cudaStream_t>(cuda_stream));
  });
}

extern "C" int bse_rpa_screening(int32_t nk, int32_t nv, int32_t nc, int32_t ng,
                                 double omega_cell, const double* e_v, const double* e_c_kq,
                                 const bse_c128* m, const double* v, int32_t precision,
                                 bse_c128* w_out, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(precision == BSE_PREC_FP64 || precision == BSE_PREC_BF16X6 ||
                      precision == BSE_PREC_BF16X3,
                  "unknown precision " + std::to_string(precision));
    BSE_CHECK_ARG(nk >= 1 && nv >= 1 && nc >= 1 && ng >= 1, "nk, nv, nc and ng must be >= 1");
    BSE_CHECK_ARG((int64_t)nk * nv * nc <= 2147483647LL, "nk*nv*nc is too large");
    BSE_CHECK_ARG(std::isfinite(omega_cell) && omega_cell > 0.0, "omega_cell must be > 0");
    BSE_CHECK_ARG(e_v && e_c_kq && m && v && w_out, "NULL e_v, e_c_kq, m, v or w_out");
    BSE_CHECK_ARG(((uintptr_t)m & 15) == 0 && ((uintptr_t)w_out & 15) == 0,
                  "m and w_out must be 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // every transition energy must be positive (an insulator's gaps)
    std::vector<double> ev((size_t)nk * nv), ec((size_t)nk * nc);
    BSE_CUDA(cudaMemcpyAsync(ev.data(), e_v, ev.size() * 8, cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaMemcpyAsync(ec.data(), e_c_kq, ec.size() * 8, cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < nk; ++k)
      for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nc; ++b)
          BSE_CHECK_ARG(ec[(size_t)k * nc + b] - ev[(size_t)k * nv + a] > 0.0,
                        "e_c_kq - e_v must be > 0 for every transition (k " + std::to_string(k) +
                            ", v " + std::to_string(a) + ", c " + std::to_string(b) + ")");
    keep_pool_memory();
    Phase ph("rpa_screening", s);
    rpa_screening(nk, nv, nc, ng, omega_cell, e_v, e_c_kq, m, v, precision, w_out, s);
  });
}

extern "C" int bse_pair_elements(int32_t grid, int32_t nv, int32_t nc, int32_t npw, int32_t ng,
                                 const bse_c128* cv, const bse_c128* cc, const int32_t* basis,
                                 const int32_t* gout, int32_t k_begin, int32_t k_count,
                                 bse_c128* m_x, bse_c128* m_vv, bse_c128* m_cc, bse_c128* n_vc,
                                 void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(grid >= 1 && grid <= 64, "grid must be in [1, 64]");
    BSE_CHECK_ARG(nv >= 1 && nc >= 1 && npw >= 1 && ng >= 1, "nv, nc, npw and ng must be >= 1");
    const int64_t nk = (int64_t)grid * grid * grid;
    BSE_CHECK_ARG(nk * nk * std::max(nv, nc) * std::max(nv, nc) <= 2147483647LL,
                  "too many pair blocks");
    BSE_CHECK_ARG(cv && cc && basis && gout, "NULL cv, cc, basis or gout");
    BSE_CHECK_ARG(m_x || m_vv || m_cc || n_vc, "no output requested");
    BSE_CHECK_ARG(k_begin >= 0 && k_count >= 0 && (int64_t)k_begin + k_count <= nk &&
                      (k_count > 0 || k_begin == 0),
                  "k-row slab [k_begin, k_begin + k_count) must lie in [0, nk)");
    auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    BSE_CHECK_ARG(al16(cv) && al16(cc) && al16(m_x) && al16(m_vv) && al16(m_cc) && al16(n_vc),
                  "complex128 arrays must be 16-byte aligned");
    keep_pool_memory();
    pair_elements_fp64(grid, nv, nc, npw, ng, cv, cc, basis, gout, k_begin,
                       k_count > 0 ? k_count : (int)nk, m_x, m_vv, m_cc, n_vc,
                       static_cast<cudaStream_t>(cuda_stream));
  });
}

extern "C" int bse_spectrum(int32_t n, bse_c128* S_inout, const bse_c128* L, int64_t ld,
                            const bse_c128* rho, double c_q, double vc, int32_t n_omega,
                            const double* omega, double delta, double* E_out, double* osc_out,
                            bse_c128* eps_out, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(n >= 1, "n must be >= 1");
    BSE_CHECK_ARG(ld >= n, "ld < n");
    BSE_CHECK_ARG(n_omega >= 0, "n_omega must be >= 0");
    BSE_CHECK_ARG(S_inout && L && rho && E_out && osc_out, "NULL S, L, rho, E_out or osc_out");
    BSE_CHECK_ARG(n_omega == 0 || (omega && eps_out), "NULL omega or eps_out");
    BSE_CHECK_ARG(std::isfinite(vc) && vc > 0.0, "vc must be > 0");
    BSE_CHECK_ARG(std::isfinite(c_q) && std::isfinite(delta) && delta >= 0.0,
                  "c_q must be finite and delta >= 0");
    keep_pool_memory();
    spectrum_fp64(n, S_inout, L, ld, rho, c_q, vc, n_omega, omega, delta, E_out, osc_out,
                  eps_out, static_cast<cudaStream_t>(cuda_stream));
  });
}

extern "C" int bse_spectrum_lanczos(int32_t n, const bse_c128* A, const bse_c128* B, int64_t ld,
                                    const bse_c128* rho, double c_q, double vc, int32_t n_omega,
                                    const double* omega, double delta, double tol,
                                    int32_t max_steps, int32_t matvec_precision,
                                    bse_c128* eps_out, int32_t* steps_out, void* cuda_stream) {
  return guarded([&] {
    if (steps_out) *steps_out = 0;
    BSE_CHECK_ARG(n >= 1, "n must be >= 1");
    BSE_CHECK_ARG(ld >= n, "ld < n");
    BSE_CHECK_ARG(n_omega >= 1, "n_omega must be >= 1");
    BSE_CHECK_ARG(A && rho && omega && eps_out, "NULL A, rho, omega or eps_out");
    BSE_CHECK_ARG(std::isfinite(vc) && vc > 0.0, "vc must be > 0");
    BSE_CHECK_ARG(std::isfinite(c_q) && std::isfinite(delta) && delta > 0.0,
                  "c_q must be finite and delta > 0");
    BSE_CHECK_ARG(std::isfinite(tol) && tol > 0.0, "tol must be > 0");
    BSE_CHECK_ARG(max_steps >= 1, "max_steps must be >= 1");
    BSE_CHECK_ARG(matvec_precision == BSE_PREC_FP64 || matvec_precision == BSE_PREC_BF16X6 ||
                      matvec_precision == BSE_PREC_BF16X3,
                  "unknown matvec precision " + std::to_string(matvec_precision));
    BSE_CHECK_ARG(matvec_precision == BSE_PREC_FP64 || mixed_supported(matvec_precision),
                  "this library has no tensor-core path");
    BSE_CHECK_ARG(((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0 && ((uintptr_t)rho & 15) == 0,
                  "A, B and rho must be 16-byte aligned");
    keep_pool_memory();
    try {
      const int st = spectrum_lanczos(n, A, B, ld, rho, c_q, vc, n_omega, omega, delta, tol,
                                      max_steps, matvec_precision, eps_out,
                                      static_cast<cudaStream_t>(cuda_stream));
      if (steps_out) *steps_out = st;
    } catch (const Error& e) {
      if (e.status == BSE_ERR_NO_CONV && steps_out) *steps_out = max_steps;
      throw;
    }
  });
}

extern "C" int bse_phase_timing(int32_t enable) {
  g_timing.store(enable != 0);
  return BSE_OK;
}

extern "C" int bse_phase_report(char* buf, int64_t buflen) {
  int written = 0;
  int st = guarded([&] {
    BSE_CHECK_ARG(buf && buflen > 0, "NULL buf or buflen <= 0");
    std::vector<PhaseRecord> recs;
    {
      std::lock_guard<std::mutex> lock(g_phase_mutex);
      recs.swap(g_phases);
    }
    std::map<std::string, std::pair<int64_t, double>> acc;
    std::vector<std::string> order;
    std::string err;
    for (auto& r : recs) {
      float ms = 0.f;
      cudaError_t e = cudaEventSynchronize(r.stop);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.start, r.stop);
      if (e != cudaSuccess && err.empty()) err = cudaGetErrorString(e);
      cudaEventDestroy(r.start);
      cudaEventDestroy(r.stop);
      if (!acc.count(r.name)) order.push_back(r.name);
      auto& a = acc[r.name];
      a.first += 1;
      a.second += ms;
    }
    if (!err.empty()) throw Error(BSE_ERR_CUDA, "phase events: " + err);
    std::string out;
    for (auto& n : order) {
      char line[256];
      snprintf(line, sizeof(line), "%s %lld %.6f\n", n.c_str(), (long long)acc[n].first,
               acc[n].second);
      out += line;
    }
    size_t nb = out.size() < (size_t)(buflen - 1) ? out.size() : (size_t)(buflen - 1);
    memcpy(buf, out.data(), nb);
    buf[nb] = 0;
    written = (int)nb;
  });
  return st == BSE_OK ? written : st;
}

extern "C" int bse_precision_supported(int32_t precision) {
  if (precision == BSE_PREC_FP64) return 1;
  if (precision == BSE_PREC_BF16X6 || precision == BSE_PREC_BF16X3)
    return mixed_supported(precision) ? 1 : 0;
  return 0;
}

extern "C" int bse_xpy(int32_t n, int32_t k, const bse_c128* Z, const bse_c128* L, int64_t ld,
                       const double* E, bse_c128* XpY_out, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(n >= 1 && k >= 1 && k <= n && ld >= n, "bad n, k or ld");
    BSE_CHECK_ARG(Z && L && E && XpY_out, "NULL argument");
    xpy_fp64(n, k, Z, L, ld, E, XpY_out, n, static_cast<cudaStream_t>(cuda_stream));
  });
}

namespace {
int lowest_excitons(int32_t n, const bse_c128* A, const bse_c128* B, int64_t ld, int32_t nev,
                    double tol_ev, int32_t max_iter, int32_t precond, const void* mlp,
                    int32_t matvec_precision, const bse_c128* V0, int32_t k0, double* E_out,
                    bse_c128* XpY_out, int32_t* iters_out, void* cuda_stream) {
  return guarded([&] {
    if (iters_out) *iters_out = 0;
    BSE_CHECK_ARG(n >= 1, "n must be >= 1");
    BSE_CHECK_ARG(ld >= n, "ld < n");
    BSE_CHECK_ARG(nev >= 1 && nev <= n, "nev must be in [1, n]");
    BSE_CHECK_ARG(std::isfinite(tol_ev) && tol_ev > 0.0, "tol_ev must be > 0");
    BSE_CHECK_ARG(max_iter >= 1, "max_iter must be >= 1");
    BSE_CHECK_ARG(A && E_out, "NULL A or E_out");
    BSE_CHECK_ARG(precond == 0 || precond == 1, "precond must be 0 (diagonal) or 1 (MLP)");
    BSE_CHECK_ARG(precond == 0 || mlp != nullptr, "precond = 1 needs an MLP handle");
    BSE_CHECK_ARG(matvec_precision == BSE_PREC_FP64 || matvec_precision == BSE_PREC_BF16X6 ||
                      matvec_precision == BSE_PREC_BF16X3,
                  "unknown matvec precision " + std::to_string(matvec_precision));
    BSE_CHECK_ARG(matvec_precision == BSE_PREC_FP64 || mixed_supported(matvec_precision),
                  "this library has no tensor-core path");
    BSE_CHECK_ARG(((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0,
                  "A and B must be 16-byte aligned");
    if (V0 || k0) {
      BSE_CHECK_ARG(V0 && k0 >= 1 && k0 <= 4 * nev && k0 <= n,
                    "a starting block needs V0 and 1 <= k0 <= min(4 nev, n)");
      BSE_CHECK_ARG(((uintptr_t)V0 & 15) == 0, "V0 must be 16-byte aligned");
    }
    keep_pool_memory();
    davidson_fp64(n, A, B, ld, nev, tol_ev, max_iter, precond,
                  static_cast<const MlpNet*>(mlp), E_out, XpY_out, iters_out,
                  static_cast<cudaStream_t>(cuda_stream), nullptr, matvec_precision, V0, k0);
  });
}
}  // namespace

extern "C" int bse_lowest_excitons(int32_t n, const bse_c128* A, const bse_c128* B, int64_t ld,
                                   int32_t nev, double tol_ev, int32_t max_iter, int32_t precond,
                                   const void* mlp, int32_t matvec_precision, double* E_out,
                                   bse_c128* XpY_out, int32_t* iters_out, void* cuda_stream) {
  return lowest_excitons(n, A, B, ld, nev, tol_ev, max_iter, precond, mlp, matvec_precision,
                         nullptr, 0, E_out, XpY_out, iters_out, cuda_stream);
}

extern "C" int bse_lowest_excitons_from(int32_t n, const bse_c128* A, const bse_c128* B,
                                        int64_t ld, int32_t nev, double tol_ev, int32_t max_iter,
                                        int32_t precond, const void* mlp, int32_t matvec_precision,
                                        const bse_c128* V0, int32_t k0, double* E_out,
                                        bse_c128* XpY_out, int32_t* iters_out, void* cuda_stream) {
  return lowest_excitons(n, A, B, ld, nev, tol_ev, max_iter, precond, mlp, matvec_precision, V0,
                         k0, E_out, XpY_out, iters_out, cuda_stream);
}

extern "C" int bse_mlp_create(void** mlp, int32_t n_features, int32_t hidden, uint64_t seed) {
  return guarded([&] {
    BSE_CHECK_ARG(mlp != nullptr, "mlp is NULL");
    *mlp = nullptr;
    if (!mlp_features_supported(n_features) || hidden != 128)
      throw Error(BSE_ERR_UNSUPPORTED,
                  "this library provides n_features = 4 or 10 and hidden = 128");
    *mlp = mlp_create(n_features, seed);
  });
}

extern "C" int bse_mlp_set_neighbours(void* mlp, int32_t n, int32_t nev, const bse_c128* nbr,
                                      int32_t count, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(mlp != nullptr, "mlp is NULL");
    BSE_CHECK_ARG(nbr == nullptr ? count == 0 : (count == 1 || count == 2),
                  "neighbour blocks: NULL with count 0, or 1 or 2 blocks");
    if (nbr) {
      BSE_CHECK_ARG(n >= 1 && nev >= 1 && nev <= n, "bad n or nev");
      BSE_CHECK_ARG(((uintptr_t)nbr & 15) == 0, "nbr must be 16-byte aligned");
    }
    mlp_set_neighbours(static_cast<MlpNet*>(mlp), n, nev, nbr, count,
                       static_cast<cudaStream_t>(cuda_stream));
    BSE_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)));
  });
}

extern "C" int bse_mlp_features(const void* mlp, int32_t n, int32_t ncol, const int32_t* eq,
                                const int32_t* lam, const double* theta, const bse_c128* A,
                                const bse_c128* B, int64_t ld, const bse_c128* R,
                                const bse_c128* X, float* feat_out, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(mlp != nullptr, "mlp is NULL");
    BSE_CHECK_ARG(n >= 1 && ld >= n && ncol >= 1, "bad n, ld or ncol");
    BSE_CHECK_ARG(eq && lam && theta && A && R && X && feat_out, "NULL argument");
    const MlpNet* net = static_cast<const MlpNet*>(mlp);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (mlp_num_features(net) == 10) {
      std::vector<int32_t> lh(ncol);
      BSE_CUDA(cudaMemcpyAsync(lh.data(), lam, ncol * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      BSE_CUDA(cudaStreamSynchronize(s));
      int lmax = 0;
      for (int32_t l : lh) {
        BSE_CHECK_ARG(l >= 0, "lam must be >= 0");
        lmax = std::max(lmax, (int)l);
      }
      mlp_check_neighbours(net, n, lmax + 1);
    }
    keep_pool_memory();
    DeviceBuffer dp((size_t)n * 8, s), dm((size_t)n * 8, s), sr((size_t)n * 8, s);
    mlp_diag_features(n, A, B, ld, dp.as<double>(), dm.as<double>(), sr.as<double>(), s);
    mlp_features(net, n, ncol, eq, lam, theta, dp.as<double>(), dm.as<double>(), sr.as<double>(),
                 reinterpret_cast<const double2*>(R), n, reinterpret_cast<const double2*>(X), n,
                 feat_out, s);
    BSE_CUDA(cudaStreamSynchronize(s));
  });
}

extern "C" void bse_mlp_destroy(void* mlp) { mlp_destroy(static_cast<MlpNet*>(mlp)); }

extern "C" int64_t bse_mlp_num_params(const void* mlp) {
  return mlp ? mlp_num_params(static_cast<const MlpNet*>(mlp)) : 0;
}

extern "C" int bse_mlp_get_params(const void* mlp, float* host, int64_t count) {
  return guarded([&] {
    BSE_CHECK_ARG(mlp && host, "NULL mlp or host buffer");
    BSE_CHECK_ARG(count == mlp_num_params(static_cast<const MlpNet*>(mlp)), "wrong count");
    mlp_get_params(static_cast<const MlpNet*>(mlp), host);
  });
}

extern "C" int bse_mlp_set_params(void* mlp, const float* host, int64_t count) {
  return guarded([&] {
    BSE_CHECK_ARG(mlp && host, "NULL mlp or host buffer");
    BSE_CHECK_ARG(count == mlp_num_params(static_cast<MlpNet*>(mlp)), "wrong count");
    mlp_set_params(static_cast<MlpNet*>(mlp), host);
  });
}

extern "C" int bse_mlp_samples(int32_t n, const bse_c128* A, const bse_c128* B, int64_t ld,
                               int32_t nev, const double* E, const bse_c128* XpY,
                               const bse_c128* noise, double eps, float* feat_out,
                               float* target_out, float* weight_out, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(n >= 1 && ld >= n && nev >= 1 && nev <= n, "bad n, ld or nev");
    BSE_CHECK_ARG(A && E && XpY && noise && feat_out && target_out && weight_out,
                  "NULL argument");
    BSE_CHECK_ARG(std::isfinite(eps) && eps > 0.0, "eps must be > 0");
    keep_pool_memory();
    mlp_samples(n, A, B, ld, nev, E, XpY, noise, eps, feat_out, target_out, weight_out,
                static_cast<cudaStream_t>(cuda_stream));
  });
}

extern "C" int bse_mlp_trajectory_samples(int32_t n, const bse_c128* A, const bse_c128* B,
                                          int64_t ld, int32_t nev, const double* E_exact,
                                          const bse_c128* XpY_exact, double tol_ev,
                                          int32_t max_iter, const void* mlp, const bse_c128* V0,
                                          int32_t k0, int64_t capacity, float* feat_out,
                                          float* target_out, float* weight_out,
                                          int64_t* count_out, void* cuda_stream) {
  return guarded([&] {
    if (count_out) *count_out = 0;
    BSE_CHECK_ARG(n >= 1 && ld >= n && nev >= 1 && nev <= n, "bad n, ld or nev");
    BSE_CHECK_ARG(A && E_exact && XpY_exact && feat_out && target_out && weight_out,
                  "NULL argument");
    BSE_CHECK_ARG(capacity >= 0 && max_iter >= 1 && tol_ev > 0.0, "bad capacity, max_iter or tol");
    if (V0 || k0) {
      BSE_CHECK_ARG(V0 && k0 >= 1 && k0 <= 4 * nev && k0 <= n,
                    "a starting block needs V0 and 1 <= k0 <= min(4 nev, n)");
      BSE_CHECK_ARG(((uintptr_t)V0 & 15) == 0, "V0 must be 16-byte aligned");
    }
    if (mlp) mlp_check_neighbours(static_cast<const MlpNet*>(mlp), n, nev);
    keep_pool_memory();
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    std::vector<double> eh(nev);
    BSE_CUDA(cudaMemcpyAsync(eh.data(), E_exact, nev * sizeof(double), cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaStreamSynchronize(s));
    TrajectorySink sink;
    sink.net = static_cast<const MlpNet*>(mlp);
    sink.xpy_exact = XpY_exact;
    sink.e_exact = eh.data();
    sink.capacity = capacity;
    sink.feat = feat_out;
    sink.target = target_out;
    sink.weight = weight_out;
    DeviceBuffer e_out((size_t)nev * 8, s);
    try {
      davidson_fp64(n, A, B, ld, nev, tol_ev, max_iter, 0, nullptr, e_out.as<double>(), nullptr,
                    nullptr, s, &sink, BSE_PREC_FP64, V0, k0);
    } catch (const Error& e) {
      if (e.status != BSE_ERR_NO_CONV) throw;   // recording ends with the iteration limit
    }
    if (count_out) *count_out = sink.count;
  });
}

extern "C" int bse_mlp_loss_grad(void* mlp, const float* feat, const float* target,
                                 const float* weight, int64_t nsamp, double* loss_out,
                                 float* grad_out, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(mlp && feat && target && weight && nsamp >= 1, "bad MLP arguments");
    const double L = mlp_loss_grad(static_cast<MlpNet*>(mlp), feat, target, weight, nsamp,
                                   grad_out, static_cast<cudaStream_t>(cuda_stream));
    if (loss_out) *loss_out = L;
  });
}

extern "C" int bse_mlp_train(void* mlp, const float* feat, const float* target,
                             const float* weight, int64_t nsamp, int32_t steps, double lr,
                             double* loss_out, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(mlp && feat && target && weight && nsamp >= 1, "bad MLP arguments");
    BSE_CHECK_ARG(steps >= 0 && std::isfinite(lr) && lr > 0.0, "bad steps or lr");
    const double L = mlp_train(static_cast<MlpNet*>(mlp), feat, target, weight, nsamp, steps, lr,
                               static_cast<cudaStream_t>(cuda_stream));
    if (loss_out) *loss_out = L;
  });
}

extern "C" int bse_mlp_predict(const void* mlp, const float* feat, int64_t nsamp,
                               float* factor_out, void* cuda_stream) {
  return guarded([&] {
    BSE_CHECK_ARG(mlp && feat && factor_out && nsamp >= 1, "bad MLP arguments");
    mlp_predict(static_cast<const MlpNet*>(mlp), feat, nsamp, factor_out,
                static_cast<cudaStream_t>(cuda_stream));
  });
}

extern "C" const char* bse_last_error(void) { return g_last_error.c_str(); }

extern "C" int bse_version(void) { return 100; }

extern "C" int64_t bse_kernel_launches(void) { return g_launches.load(); }
