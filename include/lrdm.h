/*
 * lrdm.h -- C ABI of the GB300 (sm_103a) LRDM Gateaux-derivative library.
 *
 * The library evaluates, for a Kohn-Sham system restricted to its
 * Chebyshev-filtered subspace (Psi, D = diag(eps)), the Gateaux derivatives
 *     t_k = d/dlambda R[rho + lambda v_k] |_{lambda = 0}      (Eq. jlowrank)
 * of the SCF residual R = F[rho] - rho along K direction functions v_k,
 * with the first-order density response computed in the subspace
 * (§II.C, Eqs. densityResponse, densityMatResponseApprox,
 * subspaceDensityMatResponse), and then the low-rank least-squares step
 * (Eqs. plowrank, relativeError, quasinewton).  Per direction:
 *     dV_k  = V_H[v_k] + f_xc(rho) v_k               (K = K_xc + K_c, Eq. jacobian)
 *     X_k   = Psi^T diag(w dV_k) Psi                   (H-breve')
 *     X'_k  = L o (X_k - mu'_k I), Tr X'_k = 0         (canonical DMPT, exact f)
 *     drho_k(r) = g sum_ij Psi(r,i) X'_k,ij Psi(r,j)
 *     f_k   = drho_k - v_k
 * where L is the divided-difference (Loewner) matrix of the Fermi function
 * at eps and g the occupancy factor (2 spin-restricted, 1 per spin channel).
 *
 * Discretisation: periodic grid n0 x n1 x n2 (flat C order, index
 * r = (i0 n1 + i1) n2 + i2), spacing h, quadrature weight w = h0 h1 h2,
 * inner product <a, b> = w sum_r a(r) b(r) (spin pairs: sum of the two
 * channels, Eq. innerproductDirectsumHilbertspace).  Psi holds grid values of
 * w-orthonormal functions: Psi^T diag(w) Psi = I.
 *
 * Conventions
 *  - All array pointers are DEVICE pointers unless stated otherwise.  The
 *    caller owns every input and output buffer; the library only borrows
 *    them for the duration of the stream work it enqueues.
 *  - lrdm_create / lrdm_kp_create allocate everything a context needs
 *    (workspaces sized for k_max, the operand copies of Psi, cuFFT plans) and
 *    lrdm_lrdma_create the history buffers; no other call allocates device
 *    memory (lrdm_apply_static uses a fixed device array).  Calls that take
 *    decisions on the host synchronise their stream: lrdm_krylov_step,
 *    lrdm_lrdma_step, lrdm_lrdma_export / _import, lrdm_status_query with
 *    synchronize = 1 and the create calls; the others only enqueue work.
 *  - Argument errors are returned synchronously, before anything is
 *    enqueued.  Errors found on the device (non-finite values, an expired
 *    bounded wait, a singular least-squares matrix) set a sticky status word
 *    that lrdm_status_query() reads.
 *  - stream arguments are cudaStream_t values passed as void* (NULL = the
 *    legacy default stream).  One context must not be used from two streams
 *    at the same time: its workspaces are shared by its calls.
 */
#ifndef LRDM_H
#define LRDM_H

#ifdef __cplusplus
extern "C" {
#endif

/* The library is built with hidden visibility; what this header declares is
 * its whole exported interface. */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef enum lrdm_status {
  LRDM_OK = 0,
  LRDM_ERR_INVALID_ARG = 1,      /* null pointer, bad enum, K > k_max, ...   */
  LRDM_ERR_SHAPE = 2,            /* inconsistent sizes or leading dimensions */
  LRDM_ERR_OOM = 3,              /* device allocation failed in lrdm_create  */
  LRDM_ERR_CUDA = 4,             /* a CUDA / cuFFT call failed               */
  LRDM_ERR_MU_NOT_CONVERGED = 5, /* no chemical potential for this N_e       */
  LRDM_ERR_SINGULAR = 6,         /* S rank-deficient: a = S^+ c was used     */
  LRDM_ERR_TIMEOUT = 7,          /* a bounded device wait expired            */
  LRDM_ERR_NONFINITE = 8,        /* NaN / Inf met on the device              */
  LRDM_ERR_UNSUPPORTED = 9,      /* precision / feature not available        */
  LRDM_ERR_COLLECTIVE = 10       /* the caller's allreduce (lrdm_rows) failed */
} lrdm_status;

/* Arithmetic of the two dense contractions (X_k and drho_k).  The Loewner
 * entries, mu, mu'_k, the occupations and the K x K least-squares solve are
 * always FP64. */
typedef enum lrdm_precision {
  LRDM_FP64 = 0,    /* FP64 CUDA-core GEMMs                                   */
  LRDM_FP32 = 1,    /* FP32 CUDA-core GEMMs                                   */
  LRDM_TF32 = 2,    /* tcgen05 kind::tf32, FP32 accumulation in tensor memory */
  LRDM_BF16X3 = 3   /* tcgen05 kind::f16 with operands split a = a_hi + a_lo
                       (bf16 each); a_hi b_hi + a_hi b_lo + a_lo b_hi,
                       FP32 accumulation in tensor memory                   */
} lrdm_precision;

/* Element type of Psi, rho and of every direction / residual array. */
typedef enum lrdm_dtype { LRDM_DTYPE_F64 = 0, LRDM_DTYPE_F32 = 1 } lrdm_dtype;

/* One system (device pointers are BORROWED by lrdm_create only: the context
 * keeps its own copies of everything it needs afterwards). */
typedef struct lrdm_system {
  int n[3];              /* periodic grid; N_g = n0 n1 n2                        */
  double h[3];           /* grid spacing (bohr); w = h0 h1 h2                    */
  int nspin;             /* 1: spin-restricted; 2: collinear spin pair (§II.D)  */
  int ns[2];             /* subspace size N_s per channel                        */
  int ld_psi[2];         /* leading dimension (elements) of psi[s], >= ns[s]     */
  const void* psi[2];    /* [N_g][ld] row-major, io dtype; Psi^T diag(w) Psi = I */
  const double* eps[2];  /* [ns] projected eigenvalues (Ha), FP64                */
  const double* occ[2];  /* optional [ns] occupations in [0,1]; NULL ->
                            Fermi-Dirac f(eps, mu) with mu from the electron
                            count (Eq. kseqcont)                                */
  const void* rho[2];    /* optional [N_g] density for the xc kernel (total if
                            nspin = 1, per channel if 2); NULL -> rho =
                            g sum_i f_i psi_i^2 + rho_floor (Eq. densityChFSI)   */
  double n_electrons;    /* N_e (both channels together)                         */
  double kT;             /* Fermi smearing (Ha), > 0                             */
  double occ_factor;     /* g; 0 -> 2 if nspin = 1 else 1                        */
  double rho_floor;      /* added to the computed density when rho[] is NULL     */
  int k_max;             /* directions per call for this system; 0 -> options    */
} lrdm_system;

typedef struct lrdm_options {
  int prec;              /* lrdm_precision                                       */
  int io_dtype;          /* lrdm_dtype of psi, rho and all direction arrays      */
  int k_max;             /* default maximum K per system per call (<= 64)        */
  double pinv_rcond;     /* least-squares cutoff, relative to max eig(S); 1e-12  */
  double degen_tol;      /* |eps_i - eps_j| <= degen_tol * kT counts as
                            degenerate in occupation mode; 1e-5                 */
  int poisson_symbol;    /* 0: 4 pi/|G|^2 (spectral); 1: second-order FD symbol  */
  int use_graph;         /* replay lrdm_gateaux_batch from a captured CUDA graph  */
  int autotune;          /* tensor-core precisions: 0 -> default launch shape
                            (256 x 256 projection tiles on CTA pairs, response
                            256-wide j-tiles over 256-row blocks on CTA pairs,
                            direction group 4); 1 -> lrdm_create
                            times the candidates (projection: pair tiles,
                            128 x 256 tiles, or 128 x 128 tiles with 1 or 2
                            directions; response: j-tile 128, 256
                            or 256 on CTA pairs x group 1, 2, 4) on the context's
                            own problems and keeps the fastest; with the
                            environment variable LRDM_TUNE_CACHE naming a file,
                            results are read from / appended to it (one JSON
                            object per line, keyed by device and problem sizes) */
  int debug_flags;       /* test-only fault injection, 0 in production:
                            LRDM_DEBUG_STALL_PROJECTION makes the next
                            tensor-core projection launch (once) leave one
                            weighted stage of CTA 0 unpublished, so that its
                            MMA thread's bounded wait (4 s) expires: the kernel
                            sets LRDM_ERR_TIMEOUT in the status word, waits for
                            its own copies and MMAs, frees its tensor memory
                            and returns (no trap, no hang); that call's results
                            are undefined, later calls are unaffected.  Not for
                            use with use_graph. */
  int fermi_T;           /* 0: the response uses the Loewner (divided-difference)
                            matrix of Fermi-Dirac; T >= 1: the first-order
                            response of the depth-T recursive Fermi-operator
                            expansion (Eq. recursiveFermiOperator), i.e. the
                            Loewner matrix of f_T(e) = 1/(1 + exp(2^(T+1)
                            artanh(2^-(T+1) (e - mu)/kT))); mu and the
                            occupations stay Fermi-Dirac.  Requires every
                            |eps - mu| < kT 2^(T+1) (else LRDM_ERR_INVALID_ARG at
                            create), no occupations given, and T <= 30;
                            lrdm_backward then returns v_bar only
                            (eps_bar / occ_bar -> LRDM_ERR_UNSUPPORTED)         */
} lrdm_options;

typedef struct lrdm_ctx lrdm_ctx;

/* lrdm_options.debug_flags bits (tests only) */
#define LRDM_DEBUG_STALL_PROJECTION 1

/* Fills *opt with the defaults above (BF16X3, F32 io, k_max 16). */
void lrdm_default_options(lrdm_options* opt);

/* Builds a context for nsys systems: validates shapes, solves mu
 * (g sum f(eps, mu) = N_e by FP64 bisection, Eq. kseqcont; spin channels share
 * mu, §II.D), computes the occupations, the Loewner matrices, f_xc, the
 * density if it is not given, the operand copies of Psi for the chosen
 * precision, cuFFT plans and all workspaces.  Synchronises the stream before
 * returning.  On error *out is NULL and nothing is leaked. */
lrdm_status lrdm_create(lrdm_ctx** out, const lrdm_system* sys, int nsys,
                        const lrdm_options* opt, void* stream);

/* Gateaux derivatives of all systems in one call.
 *   v[s]     : [K[s]][nspin][N_g] directions of system s (io dtype)
 *   K[s]     : HOST array, 0 <= K[s] <= k_max of system s
 *   f_out[s] : [K[s]][nspin][N_g] results f_k = drho_k - v_k (io dtype)
 *   dmu_out  : optional device [sum_s K[s]] FP64, the shifts mu'_k
 * Keeps X_k and mu'_k in the context for a following lrdm_backward.
 * Asynchronous; no allocation. */
lrdm_status lrdm_gateaux_batch(lrdm_ctx* ctx, const void* const* v, const int* K,
                               void* const* f_out, double* dmu_out, void* stream);

/* Low-rank least-squares step for system `sys` (Eqs. plowrank, relativeError,
 * quasinewton), for K directions v and their derivatives f (as written by
 * lrdm_gateaux_batch) and the current residual R ([nspin][N_g]):
 *   S = <f_k, f_l>, c = <f_k, R>, a = S^+ c (FP64; eigenvalues below
 *   pinv_rcond * max dropped, which sets LRDM_ERR_SINGULAR in the status word),
 *   Delta = sum_k a_k v_k,
 *   rho_inout <- rho_inout - alpha Delta   (alpha != 0), or <- Delta (alpha == 0),
 *   coeff_out[K] = a (device, FP64), s_rel_out = ||F a - R|| / ||R|| (device).
 * coeff_out and s_rel_out may be NULL.  Asynchronous; no allocation. */
lrdm_status lrdm_apply(lrdm_ctx* ctx, int sys, const void* R, const void* v, const void* f,
                       int K, double alpha, void* rho_inout, double* coeff_out,
                       double* s_rel_out, void* stream);

/* The least-squares step of lrdm_apply without a context and without any
 * device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc -- code whose device memory is all
 * owned by another allocator (a framework's caching pool or a fixed arena),
 * or code on a latency-critical path where cudaMalloc's implicit device
 * synchronisation is not acceptable.  The caller still passes every input
 * and output:
 *   R [n], v [K][n], f [K][n] (io_dtype; n = nspin * N_g, the two channels of
 *   a spin pair side by side), w the quadrature weight, alpha, pinv_rcond and
 *   rho_inout / coeff_out / s_rel_out exactly as for lrdm_apply; status_out
 *   (optional, device int) receives the call's status bits (4 = singular S,
 *   2 = non-finite input), cleared at the start of every call.
 * Scratch lives in one file-scope device array of the library (about 370 KB,
 * held by every GPU that loads the library until the process exits), so
 * K is limited to 16: larger K returns LRDM_ERR_INVALID_ARG before anything is
 * enqueued.  The first call on each device looks the array's device address
 * up (cudaGetSymbolAddress) with that device current.  The address belongs
 * to the device's primary context: after cudaDeviceReset the library must be
 * loaded again before this entry point is used.  Every call shares the
 * array: calls that overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  Asynchronous. */
lrdm_status lrdm_apply_static(const void* R, const void* v, const void* f, int io_dtype, int K,
                              long long n, double w, double alpha, double pinv_rcond,
                              void* rho_inout, double* coeff_out, double* s_rel_out,
                              int* status_out, void* stream);

/* ---------------------------------------------------------------------------
 * Grid-row sharding (domain decomposition of one system over ranks).  Both
 * contractions are sums over grid rows (X_k = sum_r Psi_r^T w dV_k(r) Psi_r)
 * or row-local (drho_k(r) needs row r of Psi only, Eq. densityResponse), so
 * each rank can hold a slab of Psi's rows; what couples the slabs is the
 * Poisson solve of the directions, the sum of the slabs' X_k, and the
 * least-squares sums over the grid (Eqs. plowrank, relativeError).
 * ------------------------------------------------------------------------- */

/* In-place sum over the ranks of `count` elements of `dtype` (lrdm_dtype) at
 * the device address `buf`, ordered on `stream` (a cudaStream_t) after the
 * work the library has enqueued there and before what it enqueues next;
 * returns 0 on success.  Every rank calls it with the same count and dtype,
 * in the same order.  A caller typically wraps an NCCL all-reduce. */
typedef int (*lrdm_allreduce_fn)(void* user, void* buf, long long count, int dtype, void* stream);

typedef struct lrdm_rows {
  long long row_begin;          /* first grid row (flat index r) held, >= 0          */
  long long n_rows;             /* rows held, >= 1, row_begin + n_rows <= N_g       */
  lrdm_allreduce_fn allreduce;  /* the sum over the ranks (required)                */
  void* user;                   /* passed to allreduce                              */
} lrdm_rows;

/* A context for one system (nsys = 1) of which this rank holds grid rows
 * [row_begin, row_begin + n_rows): psi[c] is [n_rows][ld_psi] (those rows of
 * Psi) and rho[c], if given, [n_rows]; every direction, derivative,
 * residual, cotangent and density array of the calls on this context is
 * [K][nspin][n_rows] (resp. [nspin][n_rows]) over the same rows.  All ranks
 * create their contexts with the same system data (n, h, eps, occ, N_e, kT,
 * g) and options, and then make the same calls in the same order: the calls
 * are collective through `allreduce`, which each of them invokes on its
 * stream between kernels:
 *   lrdm_gateaux_batch -- the spin-summed directions, written into a zeroed
 *     full-grid buffer at this rank's rows (K N_g values, so the sum is the
 *     all-gather the replicated Poisson solve needs), and X_k per channel
 *     (K N_s^2 values after the slab's grid reduction; tensor-core modes: the
 *     padded K N_s,pad^2);
 *   lrdm_apply -- the Gram, right-hand-side and ||R||^2 partial sums and the
 *     residual partial sums behind s_rel (FP64), so every rank obtains the
 *     same coefficients and s_rel and updates its rows of rho;
 *   lrdm_backward -- the adjoint's projection (as X_k) and its spin-summed
 *     Poisson input (as the directions); eps_bar and occ_bar come out equal
 *     on every rank;
 *   lrdm_krylov_step, lrdm_lrdma_step -- besides their forward and
 *     least-squares calls, the per-block sums of every norm and Gram-Schmidt
 *     inner product (FP64), so every rank takes the same decisions; their
 *     directions and the LRDMA history hold this rank's rows (an lrdm_lrdma
 *     created with n = nspin n_rows).
 * The grid reduction is not split into row ranges and use_graph is ignored.
 * A failed allreduce returns LRDM_ERR_COLLECTIVE (the stream holds the work
 * enqueued before it). */
lrdm_status lrdm_create_rows(lrdm_ctx** out, const lrdm_system* sys, const lrdm_rows* rows,
                             const lrdm_options* opt, void* stream);

/* Adjoint of the most recent lrdm_gateaux_batch on this context.
 *   f_bar[s]  : [K[s]][nspin][N_g] cotangents of f_out[s] (io dtype)
 *   v_bar[s]  : [K[s]][nspin][N_g] gradients w.r.t. v[s] (io dtype)
 *   eps_bar[2 s + c], occ_bar[2 s + c] : optional [ns] FP64 gradients w.r.t.
 *     the eigenvalues (at fixed occupations) and the occupations of channel
 *     c of system s; the arrays of pointers may be NULL, as may any entry.
 * Gradients are Euclidean (w.r.t. array entries).  Psi X' products are
 * recomputed, never stored.  Asynchronous; no allocation. */
lrdm_status lrdm_backward(lrdm_ctx* ctx, const void* const* f_bar, void* const* v_bar,
                          double* const* eps_bar, double* const* occ_bar, void* stream);

/* Reads and clears the device status word.  synchronize != 0 first waits
 * for all work of the context.  Returns the most severe pending error. */
lrdm_status lrdm_status_query(lrdm_ctx* ctx, int synchronize);

/* Chemical potential mu of system `sys` (host scalar, set by lrdm_create). */
lrdm_status lrdm_get_mu(lrdm_ctx* ctx, int sys, double* mu_host);

/* Copies the density used for the xc kernel of system `sys`, channel `spin`,
 * into out ([N_g], io dtype, device).  Asynchronous. */
lrdm_status lrdm_get_density(lrdm_ctx* ctx, int sys, int spin, void* out, void* stream);

/* Benchmark instrumentation.  While enabled, each contraction launch and each
 * Poisson solve (cuFFT forward, symbol kernel, cuFFT inverse) is bracketed by
 * CUDA events recorded on its launching stream (at most 4096 records are
 * kept), the library counts the kernels it launches itself (cuFFT's own
 * kernels are not counted), and lrdm_gateaux_batch does not use its CUDA
 * graph.  lrdm_profile_read synchronises those events and returns the summed
 * device times (ms) and counts of the projection GEMM (X_k, forward and
 * backward) launches, the response GEMM (drho_k, forward and backward)
 * launches and the Poisson solves, and the total number of library kernel
 * launches; any output pointer may be NULL; reset != 0 clears the record. */
lrdm_status lrdm_profile_enable(lrdm_ctx* ctx, int on);
lrdm_status lrdm_profile_read(lrdm_ctx* ctx, double* gemm1_ms, long long* gemm1_launches,
                              double* gemm2_ms, long long* gemm2_launches, double* poisson_ms,
                              long long* poisson_calls, long long* kernel_launches, int reset);

/* Launch shape of the tensor-core contractions chosen at create (defaults
 * or the autotuner's choice): projection MMA width (128: square tiles; 256:
 * 128 x 256 tiles, one direction; 512: 256 x 256 tiles, one direction, each
 * computed by a pair of CTAs on neighbouring SMs with M = 256 pair MMAs),
 * directions per projection square tile, response j-tile width (128, 256;
 * 512: 256-wide j-tiles over 256-row blocks on a CTA pair), response
 * direction group.  Any pointer may be NULL. */
lrdm_status lrdm_get_tuning(lrdm_ctx* ctx, int* g1_nb, int* g1_dpt, int* g2_bn, int* g2_kgroup);

/* Sets the launch shape used by the following calls on ctx (values as
 * returned by lrdm_get_tuning: g1_nb 128, 256 or 512; g1_dpt 1, or 2 with
 * g1_nb = 128; g2_bn 128, 256 or 512; g2_kgroup 1, 2 or 4).  Results depend on the
 * shape only through the blocking of the reductions.  A captured forward
 * graph is dropped and captured again by the next call.  Must not be called
 * while another host thread uses ctx.  Errors: INVALID_ARG (null ctx or a
 * value outside the sets above), UNSUPPORTED (a CUDA-core precision, which
 * has no such shape).  No device work. */
lrdm_status lrdm_set_tuning(lrdm_ctx* ctx, int g1_nb, int g1_dpt, int g2_bn, int g2_kgroup);

/* One LRDM preconditioning step of system `sys` with adaptively chosen rank
 * (§II.B, Eqs. jlowrank, krylovOrtho, plowrank, relativeError, quasinewton):
 * u_1 = R/||R||; for i = 1..r_max: t_i = Gateaux derivative along u_i (one
 * direction through the forward path), a = S^+ c over u_1..u_i, s_rel; stop
 * when s_rel < s_tol; else u_{i+1} = t_i Gram-Schmidt-orthonormalised against
 * u_1..u_i.  Then rho_inout <- rho_inout - alpha sum_k a_k u_k when rho_inout
 * is not NULL; alpha < 0 selects the paper's schedule (0.1 while ||R|| >= 2,
 * else 0.5).
 *   R          [nspin][N_g] io dtype, device; ||R|| > 0 (else INVALID_ARG)
 *   U, T       [r_max][nspin][N_g] io dtype, device, caller-owned: the
 *              directions and their Gateaux derivatives (outputs; rows
 *              beyond the final rank are unspecified)
 *   coeff_out  device [r_max] or NULL: a (first `rank` entries)
 *   s_rel_out  HOST double [r_max] or NULL: s_rel after each rank
 *   rank_out   HOST int or NULL;  r_norm_out  HOST double or NULL: ||R||
 * 1 <= r_max <= 64.  Synchronises the stream once per rank (to read s_rel);
 * the forward state of every system of the context is replaced (a following
 * lrdm_backward differentiates the last direction of `sys` only). */
lrdm_status lrdm_krylov_step(lrdm_ctx* ctx, int sys, const void* R, double s_tol, int r_max,
                             double alpha, void* rho_inout, void* U, void* T, double* coeff_out,
                             double* s_rel_out, int* rank_out, double* r_norm_out, void* stream);

/* ---------------------------------------------------------------------------
 * Accumulated LRDM (LRDMA, §II.B.1): a low-rank approximation of the Jacobian
 * kept across SCF steps.  The object holds the history (direction functions
 * u_k and their Gateaux derivatives t_k, grid functions of n = nspin * N_g
 * values in the io dtype) independently of any context, since every SCF step
 * brings a new subspace (a new lrdm_ctx); each step computes new derivatives
 * with the context it is given.
 * ------------------------------------------------------------------------- */
typedef struct lrdm_lrdma lrdm_lrdma;

typedef struct lrdm_lrdma_params {
  double s_tol;          /* rank tolerance on s_rel (0.3)                         */
  double beta_tol;       /* linearity-indicator threshold for clearing (0.1)      */
  double r_norm_clear;   /* clear instead of accumulating when ||R|| > this (1.0) */
  double alpha;          /* damping; < 0 -> 0.1 while ||R|| >= 2, else 0.5 (-1)   */
  int r_max_iter;        /* new directions per accumulating step (5)             */
  int r_max;             /* maximum kept rank, <= the capacity (capacity)         */
} lrdm_lrdma_params;

typedef enum {
  LRDMA_FRESH = 0,            /* no history: rank built afresh                    */
  LRDMA_REUSE = 1,            /* history s_rel < s_tol: used without new ranks     */
  LRDMA_ACCUMULATE = 2,       /* history extended by new directions                */
  LRDMA_CLEAR_LINEARITY = 3,  /* beta > beta_tol: cleared, rebuilt (CL)           */
  LRDMA_CLEAR_RESIDUAL = 4,   /* ||R|| > r_norm_clear: cleared, rebuilt (CR)      */
  LRDMA_CLEAR_TRUNCATED = 5   /* previous accumulation missed s_tol: cleared (CT) */
} lrdm_lrdma_event;

typedef struct lrdm_lrdma_report {
  int event;             /* lrdm_lrdma_event                                     */
  int rank;              /* directions kept after the step                       */
  int rank_new;          /* Gateaux derivatives computed in the step             */
  double s_rel;          /* s_rel of the final low-rank model on R               */
  double beta;           /* linearity indicator (-1 when not evaluated)          */
  double r_norm;         /* ||R||                                                */
  double alpha;          /* damping used                                         */
} lrdm_lrdma_report;

/* Fills the paper's settings (capacity is set by lrdm_lrdma_create). */
void lrdm_lrdma_default_params(lrdm_lrdma_params* p);
/* n = nspin * N_g values per grid function, io dtype, quadrature weight w,
 * history capacity 1..64 directions (2 * capacity * n values of device memory). */
lrdm_status lrdm_lrdma_create(lrdm_lrdma** out, long long n, int io_dtype, double w, int capacity);
/* One step: the decisions of §II.B.1 in the paper's order (CT pending ->
 * clear; with a history: beta > beta_tol -> clear (CL); history s_rel < s_tol
 * -> reuse; ||R|| > r_norm_clear -> clear (CR); else accumulate up to
 * r_max_iter new directions orthogonal to the history, scheduling CT when
 * s_tol is not reached), then rho_inout <- rho_inout - alpha sum a_k u_k
 * (rho_inout may be NULL) and the prediction R_lin = R - alpha sum a_k t_k for
 * the next step's beta.  ctx's io dtype and system `sys` (nspin * N_g = n,
 * quadrature weight w) must match the object.  R: [nspin][N_g] device.
 * Synchronises the stream (decisions are taken on the host).  The forward
 * state of the context is replaced. */
lrdm_status lrdm_lrdma_step(lrdm_lrdma* a, lrdm_ctx* ctx, int sys, const void* R, void* rho_inout,
                            const lrdm_lrdma_params* p, lrdm_lrdma_report* report, void* stream);
/* Drops the history (e.g. at a restart). */
lrdm_status lrdm_lrdma_clear(lrdm_lrdma* a);

/* Checkpoint / resume of the history (no counterpart in the paper, which
 * keeps no state across runs).  get_state returns the kept rank m and the
 * flags (LRDM_LRDMA_CLEAR_NEXT: a CT clearing is pending; LRDM_LRDMA_HAVE_LIN:
 * R_lin holds the previous step's linear prediction).  export copies the m
 * kept directions U ([m][n]), their derivatives T ([m][n]) and R_lin ([n]),
 * io dtype, into the caller's buffers (host or device); import restores them
 * (m <= capacity) together with the flags.  Both synchronise the stream. */
#define LRDM_LRDMA_CLEAR_NEXT 1
#define LRDM_LRDMA_HAVE_LIN 2
lrdm_status lrdm_lrdma_get_state(const lrdm_lrdma* a, int* m, int* flags);
lrdm_status lrdm_lrdma_export(const lrdm_lrdma* a, void* U, void* T, void* R_lin, void* stream);
lrdm_status lrdm_lrdma_import(lrdm_lrdma* a, int m, int flags, const void* U, const void* T,
                              const void* R_lin, void* stream);
void lrdm_lrdma_destroy(lrdm_lrdma* a);

/* ---------------------------------------------------------------------------
 * Periodic systems sampled at several points of the first Brillouin zone
 * (§II.C, closing paragraphs, Eq. tracelessCondition).  Each k-point kappa
 * has its own complex subspace Psi_kappa (the lattice-periodic parts of the
 * Bloch functions, Psi^H diag(w) Psi = I, given as real and imaginary planes)
 * and eigenvalues; the density and the response are BZ averages with weights
 * w_kappa; one chemical potential is shared; mu' comes from the BZ-averaged
 * traceless condition:
 *   X_kappa = Psi_kappa^H diag(w dV_k) Psi_kappa,
 *   sum_kappa w_kappa sum_i L_kappa,ii (X_kappa,ii - mu') = 0,
 *   drho_k = g sum_kappa w_kappa diag(Psi_kappa L_kappa o (X_kappa - mu' I) Psi_kappa^H).
 * Spin-restricted.  FP64 / FP32 run complex contractions on the CUDA cores;
 * TF32 / BF16X3 run the real tensor-core contractions on the stacked operand
 * C = [Re Psi, Im Psi] (N_g x 2 N_s): C^T diag(a) C holds Re X and Im X, and
 * the density is diag(C M C^T) with M = [[Re G, Im G], [-Im G, Re G]],
 * G = L o (X - mu' I).  A k-point context serves lrdm_kp_gateaux,
 * lrdm_apply, lrdm_krylov_step and lrdm_lrdma_step (sys 0, grid functions of
 * n = N_g values), lrdm_backward (v_bar of the last lrdm_kp_gateaux call,
 * f_bar / v_bar [K][N_g]; eps_bar / occ_bar must be NULL, else
 * LRDM_ERR_UNSUPPORTED), lrdm_get_mu, lrdm_get_density, lrdm_get_tuning,
 * lrdm_status_query, lrdm_profile_* and lrdm_destroy; lrdm_gateaux_batch and
 * lrdm_get_projection return LRDM_ERR_UNSUPPORTED for it.
 * ------------------------------------------------------------------------- */
typedef struct lrdm_kpoint_system {
  int n[3];                       /* periodic grid                                 */
  double h[3];                    /* spacing (bohr)                                */
  int nk;                         /* k-points, 1..32                               */
  int ns;                         /* states per k-point                            */
  int ld_psi;                     /* leading dimension of every Psi plane, >= ns    */
  const void* const* psi_re;      /* [nk] device [N_g][ld_psi] io dtype: Re Psi     */
  const void* const* psi_im;      /* [nk] device [N_g][ld_psi] io dtype: Im Psi     */
  const double* const* eps;       /* [nk] device [ns] FP64                         */
  const double* k_weights;        /* HOST [nk], positive, summing to 1 (1e-12)     */
  const void* rho;                /* device [N_g] io dtype, or NULL: g sum_kappa
                                     w_kappa sum_i f_i |psi_i|^2 + rho_floor       */
  double n_electrons;             /* N_e = g sum_kappa w_kappa sum_i f_i            */
  double kT;                      /* Fermi smearing (Ha), > 0                       */
  double occ_factor;              /* g; <= 0 -> 2                                  */
  double rho_floor;
  int k_max;                      /* directions per call; 0 -> options.k_max       */
} lrdm_kpoint_system;

/* Creates a context for one Brillouin-zone-sampled system: copies each Psi
 * plane into the compute type (the caller's buffers are not kept), solves mu
 * over all k-points on the host, builds the Loewner matrices, the density if
 * not given, f_x and the Poisson plans.  Synchronises the stream.
 * Errors: INVALID_ARG (null pointers, nk outside 1..32, weights not positive
 * or not summing to 1, kT <= 0, bad options), MU_NOT_CONVERGED (N_e outside
 * what the states can hold), UNSUPPORTED (tensor-core precision on a device
 * without sm_103a tensor cores), OOM, CUDA. */
lrdm_status lrdm_kp_create(lrdm_ctx** out, const lrdm_kpoint_system* sys, const lrdm_options* opt,
                           void* stream);
/* f_k = drho_k - v_k for K real directions v ([K][N_g] io dtype, device);
 * f_out has the same layout; dmu_out device [K] FP64 or NULL.  0 <= K <= k_max
 * (else INVALID_ARG).  Asynchronous on `stream`; with options.use_graph the
 * call is captured into a CUDA graph on its first use with a given set of
 * buffers, K and stream and replayed afterwards (as lrdm_gateaux_batch). */
lrdm_status lrdm_kp_gateaux(lrdm_ctx* ctx, const void* v, int K, void* f_out, double* dmu_out,
                            void* stream);
/* The number of grid-row ranges the projection of a K-direction call is
 * split into (tensor cores: chosen per call to fill the persistent grid's
 * waves, at most 4; CUDA cores: fixed at create).  For measurement. */
lrdm_status lrdm_kp_get_split(lrdm_ctx* ctx, int K, int* split);

/* Copies the projected perturbation X_k = Psi^T diag(w dV_k) Psi of direction
 * k, channel `spin`, of system `sys` from the most recent lrdm_gateaux_batch
 * into out ([N_s][N_s] FP64, device), for inspection and testing.
 * Asynchronous. */
lrdm_status lrdm_get_projection(lrdm_ctx* ctx, int sys, int spin, int k, double* out,
                                void* stream);

/* Frees the context (synchronises its device work first). NULL is ignored. */
void lrdm_destroy(lrdm_ctx* ctx);

const char* lrdm_status_string(lrdm_status s);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif
#endif /* LRDM_H */
