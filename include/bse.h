/*
 * bse.h - C ABI of the GB300 Bethe-Salpeter Hamiltonian library (libbse.so).
 *
 * The library builds the two-particle BSE Hamiltonian of Vorwerk, Aurich,
 * Cocchi, Draxl, "Bethe-Salpeter equation for absorption and scattering
 * spectroscopy: Implementation in the exciting code" (arXiv:1904.05575),
 * forms its half-size Hermitian reduction, solves it, and sums oscillator
 * strengths into the macroscopic dielectric function.  Equation names below
 * are the paper's labels.
 *
 * Conventions shared by every entry point
 *   - All array pointers are DEVICE pointers (cudaMalloc / torch CUDA
 *     memory) owned by the caller, unless a comment says "host".  The
 *     library never frees caller memory and keeps no pointer after return.
 *   - Complex numbers are bse_c128 = interleaved {double re, im}.
 *   - N x N matrices are column-major with leading dimension ld >= N;
 *     element (i, j) is at M[i + j * ld].  The full matrix is written.
 *   - Transition index alpha = (k * nv + v) * nc + c, N = nk * nv * nc.
 *   - Energies are in eV; v and W are in Hartree atomic units
 *     (Ha * bohr^3); kappa = Ha / (nk * omega_cell) with Ha = 27.211386245988
 *     eV multiplies the exchange and both direct terms.
 *   - Device arrays are aligned to their element size: 16 bytes for
 *     complex128, 8 for double, 4 for int32 (BSE_ERR_ARG otherwise).
 *   - Functions return a bse_status and never throw across the ABI.
 *     Argument errors are detected on the host before any launch and leave
 *     outputs untouched.  bse_last_error() returns a thread-local message
 *     describing the last non-OK status.
 *   - cuda_stream is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it; functions documented as "syncs" wait for it.
 *   - Workspace is allocated with cudaMallocAsync on cuda_stream and freed
 *     before return (stream-ordered).  On first use of a device the library
 *     raises the release threshold of that device's default memory pool so
 *     that freed workspace stays in the pool for the next call.  Small
 *     grouping plans of bse_build_kernel (k pairs sorted by q, tile lists)
 *     are cached in device memory per shape and q map until process exit.
 */
#ifndef BSE_H
#define BSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } bse_c128;

typedef enum {
  BSE_OK = 0,
  BSE_ERR_ARG = -1,          /* invalid argument (message says which) */
  BSE_ERR_CUDA = -2,         /* a CUDA runtime / library call failed */
  BSE_ERR_NOMEM = -3,        /* workspace allocation failed */
  BSE_ERR_NOT_PD = -4,       /* A-B or A+B not positive definite */
  BSE_ERR_NO_CONV = -5,      /* iterative solver did not converge */
  BSE_ERR_TIMEOUT = -6,      /* a bounded device-side wait gave up */
  BSE_ERR_UNSUPPORTED = -7   /* valid request this library cannot serve */
} bse_status;

/* Arithmetic of the M / W / v contractions of bse_build_kernel.  The
 * diagonal energies, the reduction, the eigensolve and the spectrum are
 * always FP64. */
typedef enum {
  BSE_PREC_FP64 = 0,     /* plain FP64 on CUDA cores */
  BSE_PREC_BF16X6 = 2,   /* each real operand split into 3 BF16 pieces, the 6
                            leading piece products on tcgen05 tensor cores,
                            FP32 accumulation */
  BSE_PREC_BF16X3 = 3    /* 2 BF16 pieces, 3 products: lower precision */
} bse_precision;

/* Storage of the complex input arrays m_x, m_vv, m_cc, n_vc and w of a
 * bse_problem (e_v, e_c, v_bar stay double; A and B complex128). */
typedef enum {
  BSE_C128 = 0,   /* interleaved {double re, im}, 16-byte aligned */
  BSE_C64 = 1     /* interleaved {float re, im}, 8-byte aligned: half the bytes,
                     the values already FP32 (every split-precision path
                     rounds its inputs to FP32 before splitting them) */
} bse_dtype;

/* One momentum transfer Q.  All pointers are device pointers.
 *   e_v   [nk][nv]             valence energies eps_{v,k} (eV)
 *   e_c   [nk][nc]             conduction energies eps_{c,k} (eV), scissor applied
 *   m_x   [nk][nv][nc][ng]     M_{cv,k}(G, Q) of Eq. vrrofM
 *   m_vv  [nk][nk][nv][nv][ng] m_vv[k][k'][v][v'] = M_{v'v,k'}(G, k-k') of Eq. wrrm
 *   m_cc  [nk][nk][nc][nc][ng] m_cc[k][k'][c][c'] = M_{c'c,k'}(G', k-k') of Eq. wrrm
 *   n_vc  [nk][nk][nv][nc][ng] n_vc[k][k'][v][c'] = N_{v c',k}(G', -k'-k) of Eq.
 *                              wrabar, the modified element with the ket
 *                              time-reversed: int phi*_{vk}(r) e^{-i(G'+q)r}
 *                              phi*_{c'k'}(r) dr, q = -k-k'; the first factor
 *                              N_{c v'} of that equation is read as
 *                              n_vc[k'][k][v'][c].  Unused (may be NULL) when
 *                              coupling == 0.
 *   w     [nq_w][ng][ng]       W_GG'(q), Hermitian, row-major (G' contiguous)
 *   q_minus, q_plus [nk][nk]   index of k-k' and of -k-k' into w, in [0, nq_w)
 *   v_bar [ng]                 4 pi / |G+Q|^2 with the G = 0 term set to 0
 *                              (Eq. vbar_def), non-negative
 * Output (device, column-major, ld >= N):
 *   A = E^ip + 2 gamma_x V^rr - gamma_c W^rr     (Eq. diagonalblock)
 *   B = 2 gamma_x V^rr - gamma_c W^ra            (Eq. couplingblock)
 * with V^rr_{aa'} = kappa sum_G v_bar_G conj(m_x[a][G]) m_x[a'][G]   (Eq. vrrofM)
 *      W^rr_{(kvc)(k'v'c')} = kappa sum_GG' conj(m_vv[k][k'][v][v'][G])
 *                             w[q_minus[k][k']][G][G'] m_cc[k][k'][c][c'][G']   (Eq. wrrm)
 *      W^ra_{(kvc)(k'v'c')} = kappa sum_GG' conj(n_vc[k'][k][v'][c][G])
 *                             w[q_plus[k][k']][G][G'] n_vc[k][k'][v][c'][G']    (Eq. wrabar)
 * B is not touched when coupling == 0 (Tamm-Dancoff, Eq. tdaevp) and may be NULL.
 *
 * k-row slabs (k_begin, k_count; both 0 = the whole problem).  With k_count > 0
 * only the rows (k v c) of A and B with k_begin <= k < k_begin + k_count are
 * written (every column); all other rows are left as they are.  m_vv and m_cc
 * then hold only those k rows, [k_count][nk][..][..][ng] with row 0 = k_begin,
 * so a problem whose pair arrays exceed the device memory is built slab by slab
 * (the terms of Eqs. vrrofM, wrrm, wrabar are sums over independent (k, k')
 * blocks).  n_vc stays whole: W^ra of row k reads n_vc[k'][k] for every k'.
 * e_v, e_c, m_x, w, q_minus, q_plus, v_bar, A and B keep their full shapes.
 * Requires 0 <= k_begin, k_begin + k_count <= nk; else BSE_ERR_ARG.
 *
 * in_dtype (BSE_C128 = 0, the default of a zeroed struct, or BSE_C64): the
 * element type of m_x, m_vv, m_cc, n_vc and w.  BSE_C64 is served by the
 * split-precision builds (BSE_PREC_BF16X6 / BF16X3, bse_build_kernel and
 * plans) whose direct terms run on the tensor cores: every pair block with
 * both sides >= 64 rows, or gamma_c = 0.  It is refused with
 * BSE_ERR_UNSUPPORTED for BSE_PREC_FP64, bse_build_kernel_fp64_static,
 * BSE_PLAN_FP64_DIAGONAL, BSE_PLAN_CUDA_CORE_STAGE2 and pair blocks that
 * would need the CUDA-core stage 2; plans over it never take the fused
 * direct term. */
typedef struct {
  int32_t nk, nv, nc, ng, nq_w;
  double omega_cell;                  /* Omega in bohr^3; V_c = nk * Omega */
  double gamma_x, gamma_c;            /* spin factors, Table tab:approx */
  int32_t coupling;                   /* 1 = full BSE (fill B), 0 = TDA */
  const double *e_v, *e_c;
  const bse_c128 *m_x, *m_vv, *m_cc, *n_vc, *w;
  const int32_t *q_minus, *q_plus;
  const double *v_bar;
  bse_c128 *A, *B;
  int64_t ld;
  int32_t k_begin, k_count;           /* k-row slab; 0, 0 = all rows */
  int32_t in_dtype;                   /* bse_dtype of the complex inputs */
} bse_problem;

/* Build A and B for nprob independent momentum transfers (each Q is its own
 * BSE, Sec. "BSE in matrix form", Eq. chimatrixq).  probs is a HOST array of
 * nprob descriptors (device pointers inside).  precision selects the
 * contraction arithmetic.  Reads q_minus / q_plus back to the host to check
 * their range, and reads every input array once on the device to check that
 * it holds no NaN or infinity (a sync on cuda_stream); the rest is
 * asynchronous.
 * Errors: BSE_ERR_ARG (sizes, NULL pointers, ld < N, q index out of range,
 * a non-finite input value (the message names the arrays), unknown
 * precision), BSE_ERR_NOMEM, BSE_ERR_CUDA, BSE_ERR_UNSUPPORTED. */
int bse_build_kernel(const bse_problem* probs, int32_t nprob, int32_t precision,
                     void* cuda_stream);

/* ---- batched plans ---------------------------------------------------------
 * Many momentum transfers (each its own BSE, Eq. chimatrixq) prepared once and
 * then built repeatedly.  bse_plan_create validates every problem (reading
 * q_minus / q_plus back to the host: their contents are fixed for the plan's
 * lifetime; the input arrays are scanned for NaN and infinity once, at
 * creation), groups the k pairs of every problem by q, allocates all scratch
 * (cudaMalloc, owned by the plan) and, with BSE_PLAN_AUTOTUNE, times the
 * candidate tile widths of the stage-1 tensor-core GEMM and keeps the fastest
 * (remembered per padded NG for the process).  bse_plan_execute enqueues the
 * build of every problem: kernel launches and memsets only, no allocation and
 * no host synchronisation, so it may be captured into a CUDA graph.  With a
 * tensor-core precision all problems must share ng; their exchange tiles run
 * in one persistent GEMM launch and all their direct-term stage-1 tiles in
 * another.  Inputs are read and A, B written at execute time through the
 * pointers given at creation.  bse_plan_status syncs the stream and returns
 * BSE_ERR_TIMEOUT if a bounded device wait expired in an execute since the
 * previous status call, else BSE_OK.  Errors of create: those of
 * bse_build_kernel, BSE_ERR_UNSUPPORTED (ng differs), BSE_ERR_NOMEM.
 *
 * Direct terms (Eqs. wrrm, wrabar) run fused by default when every problem's
 * pair blocks allow it (rows of the stage-1 side a power of two, rows of the
 * other side at most min(16, that)): the stage-1 GEMM and the contraction
 * over G' share one launch and the intermediate T never reaches device
 * memory.  BSE_PLAN_UNFUSED keeps the two-launch form (T written to plan
 * scratch, then contracted); both give the same bits.  Autotuning the fused
 * form times it with its outputs switched off: A and B are not written at
 * create time.
 *
 * Where both pair sides of a direct term have at least 64 rows (e.g. 20
 * valence x 20 conduction bands), its second contraction (over G') also runs
 * on the tensor cores: stage 1 writes T as split BF16 planes and one
 * persistent launch multiplies each pair block; BSE_PLAN_CUDA_CORE_STAGE2
 * keeps the FP32 CUDA-core contraction instead.
 *
 * BSE_PLAN_HERMITIAN: A and B are Hermitian (Eq. Hetr), so the plan computes
 * the direct terms (Eqs. wrrm, wrabar) only for the blocks (k, k') with
 * k <= k' (every block of rows k v c and columns k' v' c') and sets each
 * element of a block k > k' to the conjugate of its mirror, which halves the
 * direct-term work.  The caller asserts the input symmetries under which the
 * full definitions give Hermitian A and B: W(q) Hermitian and W(-q) =
 * conj(W(q)) (q_minus[k'][k] the index of -q_minus[k][k']), and
 * m_vv[k'][k][v'][v] = conj(m_vv[k][k'][v][v']), likewise m_cc (B needs only
 * W(q) Hermitian).  m_vv and m_cc blocks with k > k' are then not read.
 * Whole problems only (k_count 0 or nk; BSE_ERR_UNSUPPORTED for a slab);
 * ignored by BSE_PREC_FP64 plans.  Without the flag every block is computed
 * from its own inputs.
 *
 * The exchange term V (Eq. vrrofM) is Hermitian for any M_x: where a problem
 * has at least two exchange tiles per SM, only its blocks k <= k' are
 * computed and the rest completed from the mirrors (with or without the
 * flag). */
/*
 * BSE_PLAN_FP64_DIAGONAL: after the split-precision build the diagonal of A
 * (and B) is recomputed in FP64 and overwritten (Eqs. emat, vrrofM, wrrm,
 * wrabar at alpha = alpha', the diagonal (k, k) pair blocks: W applied to the
 * block's vectors by the FP64 GEMM kernel, the plane-wave sums reduced in
 * FP64 by one warp per transition), stored real.  Costs 8 NG^2 (Nc + Nv Nc)
 * FP64 flops per k row (the W^ra part dominates); scratch allocated at
 * creation.  Ignored by BSE_PREC_FP64 plans. */
enum { BSE_PLAN_AUTOTUNE = 1, BSE_PLAN_UNFUSED = 2, BSE_PLAN_CUDA_CORE_STAGE2 = 4,
       BSE_PLAN_HERMITIAN = 8, BSE_PLAN_FP64_DIAGONAL = 16 };
int bse_plan_create(const bse_problem* probs, int32_t nprob, int32_t precision, int32_t flags,
                    void** plan, void* cuda_stream);
int bse_plan_execute(void* plan, void* cuda_stream);
int bse_plan_status(void* plan, void* cuda_stream);
/* Clock budget of every bounded wait inside the plan's tensor-core launches
 * (default about 2 s): a wait that runs longer records a timeout, the launch
 * winds down (copies and MMAs already issued complete first) and returns,
 * and bse_plan_status reports BSE_ERR_TIMEOUT; A and B are then incomplete.
 * seconds in (0, 60], converted with the device's peak SM clock; applies to
 * the following executes.  FP64 plans have no bounded waits.  Errors:
 * BSE_ERR_ARG. */
int bse_plan_set_wait_limit(void* plan, double seconds);
/* output-column tile width the plan's stage-1 GEMM uses (0 for FP64 plans) */
int bse_plan_tile_cols(const void* plan);
/* The tensor-core stage-2 launches' output-column tile width and pipeline
 * depth (both 0 when the plan has none), host outputs.  With
 * BSE_PLAN_AUTOTUNE both are timed at creation over the widths {the default,
 * 32} and the depths {the deepest that fits shared memory, one less}; the
 * timed launches subtract from blocks of A and B that every execute stores
 * first.  Errors: BSE_ERR_ARG (NULL). */
int bse_plan_stage2_shape(const void* plan, int32_t* tile_cols, int32_t* stages);
/* 1 if the plan's direct terms run as the fused launch, else 0 */
int bse_plan_fused(const void* plan);
void bse_plan_destroy(void* plan);

/* FP64 build of one problem that allocates no device memory.
 *
 * There is no counterpart in the paper: this entry point exists for callers
 * that cannot allocate device memory when they call the library, for example
 * a host that has handed all of the GPU's memory to an allocator of its own,
 * or a loop that must not pay for the allocator's implicit synchronisation.
 * It computes exactly what bse_build_kernel(prob, 1, BSE_PREC_FP64, stream)
 * computes, with the same kernels; the stage-1 intermediate of the direct
 * terms lives in a fixed 16 MiB array compiled into the library instead of
 * stream-ordered workspace.  Every GPU on which the library's FP64 kernels are
 * loaded holds that array until the process exits.
 *
 * Limits and behaviour:
 *   - a problem whose intermediate needs more than 16 MiB, that is
 *     nk^2 * max(min(nv^2, nc^2), nv*nc if coupling) * ng * 16 bytes, is
 *     rejected with BSE_ERR_ARG before any launch;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, no allocation) and keeps it for the process;
 *     make that first call before any stream capture on that device, and do
 *     not use this entry point after a device reset (cudaDeviceReset) without
 *     restarting the process: the kept address belongs to the old context;
 *   - all calls share the one array and it keeps the previous call's
 *     contents (nothing in it needs to start at zero); calls whose work
 *     overlaps on the GPU (other streams, other host threads) race on it and
 *     must be serialised by the caller;
 *   - like bse_build_kernel it reads q_minus / q_plus back to the host to
 *     check their range (a sync on cuda_stream); it does not scan the inputs
 *     for NaN or infinity (that scan needs a workspace word).
 * Errors: BSE_ERR_ARG, BSE_ERR_CUDA. */
int bse_build_kernel_fp64_static(const bse_problem* prob, void* cuda_stream);

/* Half-size reduction of Eq. auxham in its Cholesky form.  A-B = L L^H (L
 * lower triangular, written to L with the strict upper triangle zeroed) and
 * S = L^H (A+B) L, which is unitarily similar to (A-B)^{1/2}(A+B)(A-B)^{1/2}
 * and has the eigenvalues E^2 of Eq. auxevp.  A, B are read only; S and L
 * are N x N with the same ld.  For the TDA pass B = NULL (then S = L^H A L
 * with A = L L^H, eigenvalues E^2 of the TDA problem Eq. tdaevp).
 * failed_minor: HOST pointer (may be NULL) receiving the order of the
 * leading minor of A-B that is not positive definite (0 on success).
 * Syncs.  Errors: BSE_ERR_ARG, BSE_ERR_NOT_PD, BSE_ERR_NOMEM, BSE_ERR_CUDA. */
int bse_reduce(int32_t n, const bse_c128* A, const bse_c128* B, int64_t ld,
               bse_c128* S, bse_c128* L, int32_t* failed_minor, void* cuda_stream);

/* Eigensolve S Z = E^2 Z (Eq. auxevp, FP64 Hermitian solver; S is
 * overwritten by Z) and the spectrum:
 *   E_lambda = sqrt(E^2_lambda), ascending                       -> E_out [n]
 *   X+Y = E^{-1/2} L Z (from A-B = L L^H)
 *   |t_lambda|^2 = |sum_alpha (X+Y)_{alpha lambda} rho_alpha|^2 / vc  (Eq. osci) -> osc_out [n]
 *   eps(w) = 1 - c_q Ha sum_lambda |t_lambda|^2
 *              [1/(w - E_lambda + i delta) - 1/(w + E_lambda + i delta)]
 *            (Eq. chir and Eq. epsmtensor for one direction)   -> eps_out [n_omega]
 * rho [n] = M_alpha(G=0, Q) (q.D in the optical limit, Eq. mofd); c_q = 4 pi
 * at Q = 0 and 4 pi / |Q|^2 otherwise; vc = nk * Omega (bohr^3); omega
 * [n_omega] and delta (half width) in eV.  All arrays are device pointers.
 * Syncs (reads the eigensolver status).  Errors: BSE_ERR_ARG,
 * BSE_ERR_NOT_PD (an eigenvalue E^2 <= 0), BSE_ERR_NOMEM, BSE_ERR_CUDA. */
int bse_spectrum(int32_t n, bse_c128* S_inout, const bse_c128* L, int64_t ld,
                 const bse_c128* rho, double c_q, double vc, int32_t n_omega,
                 const double* omega, double delta, double* E_out, double* osc_out,
                 bse_c128* eps_out, void* cuda_stream);

/* eps on the grid of bse_spectrum without the reduction or the eigensolve.
 * The exciton sum of bse_spectrum equals (2/vc) Q((w + i delta)^2) with
 *   Q(z2) = conj(rho)^H (z2 - K)^-1 (A-B) conj(rho),  K = (A-B)(A+B),
 * (the sum over lambda of |u_lambda|^2 / (z2 - E_lambda^2), S = L^H (A+B) L
 * being similar to K through L).  K is self-adjoint in the inner product
 * a^H (A-B)^-1 b, so a Lanczos recursion in that inner product, with two
 * products by A+B and A-B per step and no factorisation, gives Q as a
 * continued fraction of its coefficients.  The steps stop when eps changes
 * by at most tol times max |eps| between checks (every 48 steps with FP64
 * products, which run as a CUDA graph of 6 steps, every 50 with tensor-core
 * products; fewer for n < 50; at least min(100, 2n) steps); steps_out
 * (host, may be NULL) receives the number.
 * A, B as for bse_reduce (B = NULL: zero), rho, omega, delta, c_q, vc as for
 * bse_spectrum (delta > 0); eps_out [n_omega] device.  A+B and A-B are
 * formed once (workspace 2 x 16 N^2 bytes when B is given).  matvec_precision:
 * BSE_PREC_FP64 (products in FP64 on CUDA cores) or BSE_PREC_BF16X6 /
 * BF16X3 (A+B and A-B split once into BF16 pieces, products on the tensor
 * cores with the diagonal in FP64, as for bse_lowest_excitons; a further
 * 2 x 12 N^2 bytes for BF16X6); the recursion itself is FP64.
 * Syncs at each check.  Errors: BSE_ERR_ARG, BSE_ERR_NOT_PD
 * (conj(rho)^H (A-B) conj(rho) <= 0), BSE_ERR_NO_CONV (max_steps reached;
 * eps_out holds the last estimate), BSE_ERR_NOMEM, BSE_ERR_CUDA. */
int bse_spectrum_lanczos(int32_t n, const bse_c128* A, const bse_c128* B, int64_t ld,
                         const bse_c128* rho, double c_q, double vc, int32_t n_omega,
                         const double* omega, double delta, double tol, int32_t max_steps,
                         int32_t matvec_precision, bse_c128* eps_out, int32_t* steps_out,
                         void* cuda_stream);

/* Cartesian dielectric tensor (Eq. epsmij) from the eigenpairs that
 * bse_spectrum leaves: Z (its S_inout on return, N x N, ld), L from
 * bse_reduce, E [n] its energies.  D: N x 3 column-major (leading dimension
 * ldd >= n), the momentum matrix elements D_{alpha,i} of Eq. tlambdai for the
 * three Cartesian directions (the scalar spectrum uses rho = q.D).
 *   t*_{lambda i} t_{lambda j} from Eq. tlambdai (with the 1/vc of Eq. osci)
 *   eps_out[w][i][j] = delta_ij - c_q Ha sum_lambda t*_{lambda i} t_{lambda j}
 *                      [1/(w - E + i delta) - 1/(w + E + i delta)]
 * eps_out: [n_omega][3][3] complex, row-major in (i, j).  Contracting it with a
 * real unit vector q gives the scalar eps_M of bse_spectrum for rho = D q.
 * All arrays device pointers.  Syncs.  Errors: BSE_ERR_ARG, BSE_ERR_NOMEM,
 * BSE_ERR_CUDA. */
int bse_spectrum_tensor(int32_t n, const bse_c128* Z, const bse_c128* L, int64_t ld,
                        const bse_c128* D, int64_t ldd, double c_q, double vc, int32_t n_omega,
                        const double* omega, double delta, const double* E, bse_c128* eps_out,
                        void* cuda_stream);

/* Static screened interaction of an insulator in the random-phase
 * approximation (Sec. 2: Eq. wggq, w = v eps^-1, with the RPA dielectric
 * matrix at omega = 0), FP64, for one momentum q:
 *   X_GG'   = sum_{k v c} conj(m[k][v][c][G]) m[k][v][c][G'] / (e_c_kq[k][c] - e_v[k][v])
 *   eps_GG' = delta_GG' + 2 kappa v_G' X_GG'     (kappa = Ha / (nk omega_cell);
 *             the factor 2: the reversed (c, v) pairs, equal at omega = 0)
 *   w_out[G][G'] = v_G (eps^-1)_GG'
 * e_v [nk][nv] valence energies at k, e_c_kq [nk][nc] conduction energies at
 * k + q (eV; every e_c_kq - e_v > 0), m [nk][nv][nc][ng] the pair elements
 * M_vc(k, q)(G), v [ng] = 4 pi / |G+q|^2 (>= 0, Hartree atomic units), w_out
 * [ng][ng] row-major, the layout of one q of bse_problem.w.  Device pointers;
 * m and w_out 16-byte aligned.  precision (bse_precision) selects the
 * arithmetic of the X contraction, on the library's own kernels:
 * BSE_PREC_FP64 the FP64 GEMM kernel over ranges of at most 1,024
 * transitions, BSE_PREC_BF16X6 / BF16X3 the tensor cores (the transitions
 * split into BF16 pieces, FP32 accumulation over ranges of 512 transitions);
 * the partial sums are added in FP64.  eps and w are formed in FP64, eps^-1
 * by cuSOLVER LU.  Syncs.  Errors: BSE_ERR_ARG (sizes, NULL, a non-positive
 * gap, unknown precision), BSE_ERR_NOMEM, BSE_ERR_CUDA (also a singular eps),
 * BSE_ERR_TIMEOUT (a bounded wait of the tensor-core GEMM expired). */
int bse_rpa_screening(int32_t nk, int32_t nv, int32_t nc, int32_t ng, double omega_cell,
                      const double* e_v, const double* e_c_kq, const bse_c128* m, const double* v,
                      int32_t precision, bse_c128* w_out, void* cuda_stream);

/* Plane-wave pair matrix elements from wavefunction coefficients (the
 * elements M and N of the LAPW section, interstitial part: the whole element
 * for Bloch functions expanded in plane waves, phi_{nk}(r) =
 * sum_{G in S} C_{nk}(G) e^{i(k+G)r} with unit-norm plane waves), in FP64:
 *   M(a, b; G, s) = sum_{G1 in S} conj(a(G1)) b(G1 + G + s)
 *   N(a, b; G, s) = sum_{G1 in S} conj(a(G1)) conj(b(-G1 - G - s))
 * (b = 0 outside S; s the reciprocal vector that brings k + q back onto the
 * grid), producing the build's inputs at Q = 0 in the layouts of bse_problem:
 *   m_x[k][v][c](G)       = <c k| e^{-iGr} |v k>                    = M(C_ck, C_vk; G, 0)
 *   m_vv[k][k'][v][v'](G) = <v' k'| e^{-i(G+q)r} |v k>, q = k - k'  = M(C_v'k', C_vk; G, s)
 *   m_cc[k][k'][c][c'](G) likewise with conduction bands
 *   n_vc[k][k'][v][c'](G) = <v k| e^{-i(G+q)r} |(c' k')^*>, q = -k - k'
 * grid: the k grid is grid^3 points, k = (i grid + j) grid + l at integer
 * coordinates (i, j, l) / grid of the reciprocal basis (the order of
 * bse_problem's q maps); cv [nk][nv][npw], cc [nk][nc][npw] device
 * coefficients; basis [npw][3] and gout [ng][3] HOST int32 coordinates of the
 * plane-wave basis S (distinct) and of the output vectors G in the reciprocal
 * basis.  k_begin / k_count select the k rows of m_vv and m_cc as in
 * bse_problem (0, 0: all); m_x and n_vc are whole.  Any output may be NULL
 * (not computed), not all.  Syncs.  Errors: BSE_ERR_ARG, BSE_ERR_UNSUPPORTED
 * (coordinates beyond 30 from the origin, a basis too large for the kernel's
 * shared memory), BSE_ERR_NOMEM, BSE_ERR_CUDA. */
int bse_pair_elements(int32_t grid, int32_t nv, int32_t nc, int32_t npw, int32_t ng,
                      const bse_c128* cv, const bse_c128* cc, const int32_t* basis,
                      const int32_t* gout, int32_t k_begin, int32_t k_count, bse_c128* m_x,
                      bse_c128* m_vv, bse_c128* m_cc, bse_c128* n_vc, void* cuda_stream);

/* Electron energy-loss function L(w) = -Im 1/eps_M(w) (Eq. Lofeps) and the
 * dynamical structure factor S(Q, w) = -(1/pi) v_G(q)^{-1} Im 1/eps_M(q, w)
 * from eps [n_omega] (complex, e.g. bse_spectrum's eps_out).  v_inv =
 * |G+q|^2 / (4 pi), the inverse Coulomb potential of the momentum loss.
 * loss_out, sqw_out: [n_omega] doubles, either may be NULL (not both).
 * Device pointers; asynchronous.  Errors: BSE_ERR_ARG, BSE_ERR_CUDA. */
int bse_loss_function(int32_t n_omega, const bse_c128* eps, double v_inv, double* loss_out,
                      double* sqw_out, void* cuda_stream);

/* Per-phase timing for measurement.  bse_phase_timing(1) makes the library
 * record a CUDA event pair on the launching stream around each of its
 * phases (one or more kernels, or one cuSOLVER / cuBLAS call);
 * bse_phase_timing(0) stops recording.  bse_phase_report synchronizes the
 * recorded events, writes one line "name launches total_ms\n" per phase into
 * buf (host, buflen bytes, NUL-terminated, truncated if short), clears the
 * record and returns the number of bytes written (or a negative status). */
int bse_phase_timing(int32_t enable);
int bse_phase_report(char* buf, int64_t buflen);

/* Eigenvectors of the full problem from the reduction: X+Y = L Z E^{-1/2}
 * (the reconstruction after Eq. auxevp in the Cholesky form, A-B = L L^H), for
 * the first k columns of Z (S_inout of bse_spectrum after it returns), L from
 * bse_reduce, E [k] from bse_spectrum.  XpY_out: n x k column-major (ld n),
 * normalised so that (X+Y)^H (X-Y) = 1.  All device pointers; asynchronous. */
int bse_xpy(int32_t n, int32_t k, const bse_c128* Z, const bse_c128* L, int64_t ld,
            const double* E, bse_c128* XpY_out, void* cuda_stream);

/* Lowest nev excitons of the full BSE without the dense O(N^3) solve: block
 * Davidson on the half-size product form (A-B)(A+B)(X+Y) = E^2 (X+Y), which
 * follows from Eq. gevpbse with H = [[A,B],[B,A]] (Eq. Hetr) and underlies
 * Eqs. auxham / auxevp; projected problems use the Cholesky form of
 * bse_reduce.  A and B: N x N Hermitian, column-major, full storage, ld >= n
 * (device); B = NULL solves the TDA problem A X = E X (Eq. tdaevp); A-B and
 * A+B must be positive definite.
 *   nev        number of lowest excitons (1 <= nev <= n)
 *   tol_ev     convergence: every residual norm of the nev pairs below tol_ev
 *              (eV; 1e-4 gives energies far inside 1 meV)
 *   max_iter   iteration limit
 *   precond    0 = diagonal (r_a / (A_aa - E)), 1 = the trained MLP given in mlp
 *   matvec_precision  BSE_PREC_FP64: matvecs (A+B)V, (A-B)V by the FP64 GEMM;
 *              BSE_PREC_BF16X6 / BF16X3: A and B split once into BF16 pieces
 *              and the matvecs run on the tensor cores (FP32 accumulation in
 *              K segments, FP64 results); workspace 2 x 12 N^2 bytes (BF16X6).
 *              The residual floor then scales with ~1e-7 of the off-diagonal
 *              part of A (A's diagonal is applied in FP64): keep tol_ev above it.
 *   E_out      [nev] device, ascending exciton energies (eV)
 *   XpY_out    [n x nev] device column-major, X+Y with (X+Y)^H (X-Y) = 1, or NULL
 *   iters_out  host, iterations used (may be NULL)
 * Syncs every iteration.  Errors: BSE_ERR_ARG, BSE_ERR_NOT_PD, BSE_ERR_NO_CONV
 * (E_out then holds the last estimates), BSE_ERR_UNSUPPORTED, BSE_ERR_CUDA. */
int bse_lowest_excitons(int32_t n, const bse_c128* A, const bse_c128* B, int64_t ld, int32_t nev,
                        double tol_ev, int32_t max_iter, int32_t precond, const void* mlp,
                        int32_t matvec_precision, double* E_out, bse_c128* XpY_out,
                        int32_t* iters_out, void* cuda_stream);

/* bse_lowest_excitons started from a given subspace instead of unit vectors:
 * the k0 columns of V0 ([n x k0] device column-major, read only), typically
 * the X+Y of the same excitons at a neighbouring momentum transfer when the
 * exciton dispersion E_lambda(Q) is traced over a line of Q (the warm start
 * of an exciton band structure; the problems must share n and the transition
 * order).  The columns and their images under A+B (which carry the matching
 * X-Y) are orthonormalised (dependent ones dropped) and unit vectors at the
 * smallest A_aa are added until the basis holds nev + max(4, nev/4) vectors.  1 <= k0 <= min(4 nev, n); V0 16-byte aligned.
 * Other arguments, outputs and errors as for bse_lowest_excitons. */
int bse_lowest_excitons_from(int32_t n, const bse_c128* A, const bse_c128* B, int64_t ld,
                             int32_t nev, double tol_ev, int32_t max_iter, int32_t precond,
                             const void* mlp, int32_t matvec_precision, const bse_c128* V0,
                             int32_t k0, double* E_out, bse_c128* XpY_out, int32_t* iters_out,
                             void* cuda_stream);

/* ---- learned preconditioner for bse_lowest_excitons -------------------------
 * Not in the paper: a per-transition network (F features -> 128 -> 128 -> 1,
 * ReLU, FP16 weights, FP32 accumulation; the 128 x 128 layer of the forward
 * pass on the tensor cores) predicting a factor c that rescales the diagonal
 * gain of the Davidson correction, t_a = c r_a / (D_a - E), D the diagonal of
 * A+B (residual r of (A+B)(X+Y) = E(X-Y), correcting x = X+Y) or of A-B (the
 * other equation, correcting x = X-Y).  Feature sets, with D' the other
 * equation's diagonal and S_a the off-diagonal row norm of A:
 *   F = 4   [D_a - E, D'_a - E, S_a, E / 10]
 *   F = 10  [(D_a - E)/10, (D'_a - E)/10, S_a/10, E/100] then, for each of
 *           the (up to) two neighbour blocks of bse_mlp_set_neighbours, with
 *           v the neighbour's X+Y of the same exciton, u = v/|v| times the
 *           unit phase of v^H x, b = r/(D - E) (|D - E| clamped to >= 0.01 eV)
 *           and d = u - x/|x|: |u_a| sqrt(n), Re(conj(b_a) d_a) sqrt(n)/|b_a|,
 *           Im(conj(b_a) d_a) sqrt(n)/|b_a| (0 where b_a = 0; 0 for a missing
 *           second neighbour).
 * An untrained network gives c ~ 1, the diagonal preconditioner.
 * The handle owns device memory on the device current at creation. */

/* Create with deterministic initial weights from seed; n_features 4 or 10,
 * hidden 128 (BSE_ERR_UNSUPPORTED otherwise). */
int bse_mlp_create(void** mlp, int32_t n_features, int32_t hidden, uint64_t seed);
void bse_mlp_destroy(void* mlp);
int64_t bse_mlp_num_params(const void* mlp);
/* Parameters in the order W1 [128][F], b1 [128], W2 [128][128], b2, w3 [128],
 * b3 [1] (row-major), as the FP16 values the network uses, to / from host. */
int bse_mlp_get_params(const void* mlp, float* host, int64_t count);
int bse_mlp_set_params(void* mlp, const float* host, int64_t count);

/* The neighbouring momentum transfers of the 10-feature set: count (1 or 2)
 * blocks of [n x nev] column-major complex128 (device, 16-byte aligned), block
 * i the X+Y of the nev lowest excitons at neighbour Q_i in ascending order,
 * with the transition order of the problems solved.  The handle keeps the
 * pointer: the caller keeps the blocks alive and unchanged while solves,
 * samples or features use the network; nbr = NULL with count = 0 clears.
 * A 10-feature network without neighbours for the problem's n and at least
 * its nev excitons is refused (BSE_ERR_ARG) by every call that needs them.
 * Syncs. */
int bse_mlp_set_neighbours(void* mlp, int32_t n, int32_t nev, const bse_c128* nbr, int32_t count,
                           void* cuda_stream);

/* The network's input features for ncol residual columns (all device):
 * eq [ncol] int32, 0 = residual of the (A+B) equation, 1 = of the (A-B)
 * equation; lam [ncol] int32, the exciton (column of the neighbour blocks);
 * theta [ncol] its energy (eV); A, B as for bse_lowest_excitons (B may be
 * NULL); R and X [n x ncol] column-major (ld n): the residuals and the
 * vectors they correct (X+Y for eq 0, X-Y for eq 1).  feat_out
 * [ncol n][F] float32, sample s = c n + a.  Syncs. */
int bse_mlp_features(const void* mlp, int32_t n, int32_t ncol, const int32_t* eq,
                     const int32_t* lam, const double* theta, const bse_c128* A,
                     const bse_c128* B, int64_t ld, const bse_c128* R, const bse_c128* X,
                     float* feat_out, void* cuda_stream);

/* Training samples from exact pairs (E [nev], X+Y [n x nev] column-major, both
 * device) of the full problem: X-Y = (A+B)(X+Y)/E, both perturbed by eps p
 * (noise [n x nev] device, column lambda the direction p of pair lambda); the
 * residuals r of the two half-size equations give, per transition a, the gain
 * g* = Re(conj(r_a) eps p_a)/|r_a|^2 that maps r_a onto the perturbation, the
 * target factor c* = g* (D_a - E) and weight |r_a|^2/(D_a - E)^2 normalised
 * over each vector.  Outputs (device, sample s = (2 lambda + eq) n + a,
 * eq 0 = the (A+B) equation): feat_out [2 nev n][4], target_out and
 * weight_out [2 nev n] (FP32).  B = NULL for the TDA problem. */
int bse_mlp_samples(int32_t n, const bse_c128* A, const bse_c128* B, int64_t ld, int32_t nev,
                    const double* E, const bse_c128* XpY, const bse_c128* noise, double eps,
                    float* feat_out, float* target_out, float* weight_out, void* cuda_stream);

/* Training samples from a Davidson trajectory: runs bse_lowest_excitons with
 * the diagonal preconditioner on (A, B) whose exact lowest pairs (E_exact
 * [nev], XpY_exact [n x nev], device) are known, started from V0 [n x k0]
 * as bse_lowest_excitons_from does (V0 = NULL, k0 = 0: unit vectors); at
 * every iteration each unconverged pair contributes, for both half-size
 * equations, the samples of its residual against the current error (Ritz
 * vector minus the exact vector aligned in phase): target and weight as in
 * bse_mlp_samples with that error as the step, features of mlp's set (mlp =
 * NULL: the 4-feature set; a 10-feature network needs its neighbours).
 * Stops at convergence (tol_ev), max_iter or when the next vector's samples
 * would exceed capacity; count_out (host) receives the number written.
 * feat_out [capacity][F], target_out, weight_out [capacity] (device).  Syncs. */
int bse_mlp_trajectory_samples(int32_t n, const bse_c128* A, const bse_c128* B, int64_t ld,
                               int32_t nev, const double* E_exact, const bse_c128* XpY_exact,
                               double tol_ev, int32_t max_iter, const void* mlp,
                               const bse_c128* V0, int32_t k0, int64_t capacity, float* feat_out,
                               float* target_out, float* weight_out, int64_t* count_out,
                               void* cuda_stream);

/* Loss sum_s w_s (c_s - c*_s)^2 / sum_s w_s over nsamp device samples and its
 * gradient with respect to the FP16 parameters (grad_out: host, count
 * bse_mlp_num_params, or NULL).  Syncs. */
int bse_mlp_loss_grad(void* mlp, const float* feat, const float* target, const float* weight,
                      int64_t nsamp, double* loss_out, float* grad_out, void* cuda_stream);

/* steps of full-batch Adam (beta1 0.9, beta2 0.999) with learning rate lr on
 * the same loss; loss_out (host) receives the final loss.  Syncs. */
int bse_mlp_train(void* mlp, const float* feat, const float* target, const float* weight,
                  int64_t nsamp, int32_t steps, double lr, double* loss_out, void* cuda_stream);

/* factor_out[s] = c(feat[s]) for nsamp device feature rows. */
int bse_mlp_predict(const void* mlp, const float* feat, int64_t nsamp, float* factor_out,
                    void* cuda_stream);

/* 1 if this library serves the given bse_precision in bse_build_kernel, else 0.
 * Host only; no CUDA call. */
int bse_precision_supported(int32_t precision);

/* Thread-local description of the last non-OK status ("" if none). */
const char* bse_last_error(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int bse_version(void);

/* Number of CUDA kernels this library has launched in the calling process
 * (its own kernels only; kernels inside cuSOLVER / cuBLAS calls are not
 * counted).  Monotonic; for measurement. */
int64_t bse_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* BSE_H */
