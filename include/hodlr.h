/*
 * hodlr.h -- C ABI of the GB300 HODLR Gaussian-process likelihood library.
 *
 * The library evaluates, for the physics-based covariance of arXiv 2303.10102
 * (Sec. 2.1, eq. cov model)
 *     K(theta) = L K_u(theta) L^T + tau2 I,   theta = (sigma2, ell, kappa, tau2),
 * the negative log-likelihood, its gradient and the expected Fisher information of the
 * hierarchical (HODLR) approximation K~(theta) (Sec. 4, eq. log-like approximated,
 * eq. score approximated, eq. fisher info approximated).  K~ is built matrix-free from
 * products of K with patterned Gaussian probes (Alg. 1, Sec. 3.2.2); the derivative
 * matrices dK~/dtheta_j are built in the same structure (Alg. 2, Sec. 3.3); K~ is
 * factorized hierarchically (eq. one way factor, App. C); the traces are exact
 * (App. B).  Every arithmetic step runs in the library's own CUDA kernels.
 *
 * Conventions common to all calls
 *   - Return value: HODLR_OK (0) or a negative HODLR_E* code.  A failed call leaves its
 *     outputs untouched; hodlr_last_error() describes the failure; the context stays
 *     usable.
 *   - Device memory: the library allocates nothing.  The caller queries the size with
 *     hodlr_workspace_size() and passes one device buffer to hodlr_create(); the
 *     buffer stays owned by the caller and must outlive the context.
 *   - Stream: all device work is ordered on the CUDA stream given to hodlr_create()
 *     (NULL = legacy default stream).  Calls that return host values synchronise it.
 *   - theta: host array of 4 doubles (sigma2, ell, kappa, tau2), all > 0.
 *     hodlr_nll/grad/fisher rebuild K~ when theta differs bitwise from the last build.
 *   - y: device array of N doubles in natural order (1-D: grid index; 2-D: iy*G + ix;
 *     bivariate: [y1 (all points); y2 (all points)]).
 *   - Sign: outputs are the NLL and its gradient g = -S (S = score of eq. score).
 */
#ifndef HODLR_H
#define HODLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HODLR_OK 0
#define HODLR_EINVAL (-1)    /* bad argument or unsupported combination          */
#define HODLR_ENOMEM (-2)    /* workspace too small                               */
#define HODLR_ENOTPD (-3)    /* a leaf or SMW core Cholesky failed (K~ not SPD)   */
#define HODLR_ENUMERIC (-4)  /* NaN / Inf met in an input or a result             */
#define HODLR_ETIMEOUT (-5)  /* a bounded device wait gave up                     */
#define HODLR_ENOTIMPL (-6)  /* feature not built                                 */
#define HODLR_ECUDA (-7)     /* a CUDA runtime call failed                        */

#define HODLR_FP64 0         /* everything in FP64                                */
#define HODLR_MIXED_FP32 1   /* FP32 sketch and products (3xTF32 on the tcgen05
                                tensor cores where the layout allows, FP32 FFMA
                                otherwise); FP64-class leaf sketch of K~, leaf
                                Cholesky, SMW cores, factorization sweeps and
                                log-det (FP64 or double-float accumulation)      */
#define HODLR_MIXED_BF16 2   /* FP64 storage and FP64 physics recurrences, with the
                                dense products (DST of the operator solve, peeling,
                                projection, leaf, factorization and trace products)
                                carried out on the BF16 tcgen05 tensor cores as
                                exact products of 7-bit digit slices with FP32
                                accumulation (error ~2^-46 of the row/column-scaled
                                bound, FP64-class); small products stay FP64      */

typedef struct hodlr_ctx hodlr_ctx;

/* Model descriptor (copied by hodlr_create).
 *   dim      1 or 2 (regular grid of G points per axis on (0,1)^dim, h = 1/(G+1))
 *   grid     {G, G} for dim 2, {G, 1} for dim 1
 *   nvar     1: y = A^{-1} u   (K = A^{-1} K_u A^{-1} + tau2 I)
 *            2: y = (u, A^{-1} u)  (K = L K_u L^T + tau2 I, L = [I; A^{-1}])
 *   nu       Matern smoothness 0.5 or 1.5 (eq. whittle covariance, no sqrt(2 nu))
 *   precision HODLR_FP64, HODLR_MIXED_FP32 or HODLR_MIXED_BF16                    */
typedef struct {
  int dim;
  int grid[2];
  int nvar;
  double nu;
  int precision;
} hodlr_model;

/* Construction options (Alg. 1 / Sec. 3.2.2 and the readings of the rank rule).
 *   leaf        leaf block size in matrix rows (multiple of nvar)
 *   rank_or_cap kept-rank cap per off-diagonal block (stored factor width)
 *   oversample  probe columns c = rank_or_cap + oversample
 *   tol         relative truncation tolerance of the pivoted QR (0 = fixed rank);
 *               a block keeps the leading |R_ii| > max(tol, guard) |R_11|.
 *   seed        Philox key of the probes (fixed across theta, Sec. 3.3)
 *   guard       rank guard (0 = 1e-5).  It bounds cond(R) and with it the rounding
 *               amplification of the differentiated QR (Alg. 2): derivative matrices
 *               carry errors of order u * cond(R).  It also bounds the truncation
 *               residual that the leaf extraction sums over all leaves, which must stay
 *               below the nugget tau2 for K~ to be positive definite.                */
typedef struct {
  int leaf;
  int rank_or_cap;
  int oversample;
  double tol;
  uint64_t seed;
  double guard;
} hodlr_opts;

/* Bytes of device workspace needed by a context for (m, o).  0 on bad arguments. */
size_t hodlr_workspace_size(const hodlr_model* m, const hodlr_opts* o);

/* Host-only plan of a context for (m, o): no device work, usable without a GPU.
 *   dims_out: host, 6 values {N, tau, leaf rows, probe columns c, rank cap, leaves}
 *             (tau = number of levels, Sec. 3.2.2; leaves = 2^tau; leaf rows = the largest
 *             leaf: median splits of any N give leaves whose sizes differ by at most one);
 *   perm_out: host, N values or NULL: tree position -> natural index (the KD / Morton
 *             order of Sec. 5.2, bivariate rows interleaved per leaf), as hodlr_perm.
 * HODLR_EINVAL for bad arguments.  */
int hodlr_plan(const hodlr_model* m, const hodlr_opts* o, int64_t* dims_out, int64_t* perm_out);

/* Create a context.  workspace: caller-owned device buffer of >= workspace_bytes
 * bytes, 256-byte aligned.  cuda_stream: a cudaStream_t (may be NULL).  */
int hodlr_create(hodlr_ctx** out, const hodlr_model* m, const hodlr_opts* o, void* cuda_stream,
                 void* workspace, size_t workspace_bytes);

/* Build K~(theta) and dK~/d theta_j (Alg. 1, Sec. 3.2.2, Alg. 2, Sec. 3.3) and
 * factorize K~ (eq. one way factor, App. C).  points must be NULL (regular grid).
 * HODLR_ENOTPD: a leaf or SMW-core Cholesky failed; HODLR_ETIMEOUT: a tensor-core product
 * gave up waiting for its operands (bounded mbarrier wait); the context stays usable.  */
int hodlr_build(hodlr_ctx* h, const double* theta, const double* points);

/* NLL of eq. log-like approximated (negated): N/2 log 2pi + 1/2 log|K~| + 1/2 y^T K~^{-1} y.
 * nll_out: host double.  */
int hodlr_nll(hodlr_ctx* h, const double* theta, const double* y, double* nll_out);

/* Gradient of the NLL (eq. score approximated, negated): g_j = 1/2 tr(K~^{-1} K~_j)
 * - 1/2 a^T K~_j a, a = K~^{-1} y, with the exact trace of App. B.  grad_out: host, 4. */
int hodlr_grad(hodlr_ctx* h, const double* theta, const double* y, double* grad_out);

/* Expected Fisher information (eq. fisher info approximated):
 * I_ij = 1/2 tr(K~^{-1} K~_i K~^{-1} K~_j), exact (App. B.2/B.3).  fisher_out: host, 16,
 * row-major.  */
int hodlr_fisher(hodlr_ctx* h, const double* theta, double* fisher_out);

/* NLL, gradient and Fisher of one theta in one call (one "evaluation").  Any output
 * pointer may be NULL.
 * Gradient and Fisher (here and in hodlr_grad / hodlr_fisher / hodlr_traces /
 * hodlr_batch_nll_grad) return HODLR_ENOTIMPL for bivariate models on the mixed FP32 path:
 * its FP32 sketch rounding, multiplied by cond(R) <= 1/guard in Alg. 2, leaves those
 * derivatives inaccurate.  Use HODLR_FP64 for them; the NLL is available on both paths.  */
int hodlr_eval(hodlr_ctx* h, const double* theta, const double* y, double* nll_out,
               double* grad_out, double* fisher_out);

/* NLL and gradient of nb independent contexts (batched 1-D workload), each with its own
 * theta (thetas: nb*4 host doubles) and y (ys: nb device pointers).  Outputs: nll_out
 * [nb], grad_out [nb*4] host.  */
int hodlr_batch_nll_grad(hodlr_ctx* const* hs, int nb, const double* thetas,
                         const double* const* ys, double* nll_out, double* grad_out);

/* Tree order: perm_out[position] = natural index (host, N int64).  The ordering is the
 * KD / Morton order of Sec. 5.2 with the cluster tree of Sec. 3.2.2.  */
int hodlr_perm(const hodlr_ctx* h, int64_t* perm_out);

/* Sizes: out[0]=N, out[1]=tau (levels), out[2]=leaf size, out[3]=probe columns c,
 * out[4]=rank cap, out[5]=number of leaves.  */
int hodlr_dims(const hodlr_ctx* h, int64_t* out);

/* Kept ranks of the last build: ranks_out[(2^(l-1) - 1) + p] for level l, pair p
 * (host int32, 2^tau - 1 entries).  */
int hodlr_ranks(const hodlr_ctx* h, int32_t* ranks_out);

/* Pivot sets J of the last build, and freezing.  Layout: per pair (same order as
 * hodlr_ranks) c int32 entries, the first rank entries are J, the rest -1.
 * hodlr_set_pivots(h, J) makes subsequent builds use the given sets instead of taking
 * pivoted QRs (Sec. 3.3: the sampling pattern is held fixed); J = NULL unfreezes.  */
int hodlr_get_pivots(const hodlr_ctx* h, int32_t* piv_out);
int hodlr_set_pivots(hodlr_ctx* h, const int32_t* piv_in);

/* Physics product (eq. cov model): Y = K X (which=0) or dK/dtheta_which X (which=1..4
 * for sigma2, ell, kappa, tau2) at theta, for X (device, N x ncols column-major, FP64,
 * natural order).  Y: device, same layout.  */
int hodlr_apply(hodlr_ctx* h, const double* theta, int which, const double* X, double* Y,
                int ncols);

/* Probe panel R^(level) of the level sketch (Alg. 1 step 1, patterned as in Sec. 3.2.2)
 * in tree order: out device N x ncols FP64 column-major, ncols <= c.  */
int hodlr_probe(hodlr_ctx* h, int level, int ncols, double* out);

/* Dense form of K~ (which=0) or K~_j (which=1..4) in tree order, N x N column-major
 * FP64 device buffer (small N only; for tests).  Needs a prior build.  */
int hodlr_densify(hodlr_ctx* h, int which, double* out);

/* HODLR product (Table "HODLR operations", Sec. 3.1: the matrix-vector product of the
 * hierarchical form): Y = K~ X (which = 0) or K~_j X (which = 1..4 for sigma2, ell, kappa,
 * tau2; K~_sigma2 = (K~ - tau2 I) / sigma2 and K~_tau2 = I, Sec. 3.3) with the matrices of the
 * last build.  X, Y: device FP64, N x ncols column-major, natural order; Y may not overlap X.
 * HODLR_EINVAL without a build.  Synchronises the context's stream.  */
int hodlr_matvec(hodlr_ctx* h, int which, const double* X, double* Y, int ncols);

/* K~^{-1} b in natural order (device FP64 vectors of length N) and log|K~| (host).  */
int hodlr_solve(hodlr_ctx* h, const double* b, double* x);
int hodlr_logdet(hodlr_ctx* h, double* logdet_out);

/* Gradient of the NLL by reverse mode through the factorization (the adjoint route of the
 * differentiability statement of Sec. 3.3): with Kbar = (K~^{-1} - alpha alpha^T) / 2 the adjoint
 * of the NLL with respect to K~, grad_j = <Kbar, K~_j> is assembled from the adjoints of the
 * HODLR factors -- Kbar's leaf blocks (from solves with the leaves' identity columns) and, per
 * level, the adjoint panel K~^{-1} P - alpha (alpha^T P) of the level's factor panel P restricted
 * to one side of each sibling pair -- contracted with the tangent factors of Alg. 2 (dA_j, dQ_j,
 * dB~_j); sigma2 and tau2 through K~_sigma2 = (K~ - tau2 I) / sigma2, K~_tau2 = I.  Equal to
 * hodlr_grad (the exact traces of App. B) up to rounding.  Builds and factors at theta when the
 * context holds another build.  y: device FP64, natural order; grad_out: host, 4 doubles.
 * HODLR_ENOTIMPL on a HODLR_MIXED_FP32 context (its factors are FP32).  */
int hodlr_grad_adjoint(hodlr_ctx* h, const double* theta, const double* y, double* grad_out);

/* Exact traces (App. B.3): t[i] = tr(K~^{-1} M_i), f[3*i+j] = tr(K~^{-1} M_i K~^{-1} M_j)
 * for M = (I, K~_ell, K~_kappa).  t: host 3, f: host 9.  */
int hodlr_traces(hodlr_ctx* h, double* t_out, double* f_out);

/* Log-determinant split of the last factorization (App. C / Sylvester's identity):
 * out[0] = sum over leaves of log|A_b|, out[l] = sum over the level-l nodes of
 * log|I - Lw^T Sx Lw| (l = 1..tau); host array of tau + 1 doubles.  */
int hodlr_logdet_levels(hodlr_ctx* h, double* out);

/* Inspection of the factorization (tests): copies into `out` (host, FP64) the level-l panel
 * F (what=0, N x w_l: Q in left-child rows, B~ in right-child rows), U = K~_child^{-1} F
 * (what=1, N x w_l), or the per-node Gram matrices Sw (what=2) / Sx (what=3)
 * (2^(l-1) blocks of w_l x w_l).  w_out receives w_l.  `count` is the capacity of `out`.  */
int hodlr_debug_level(hodlr_ctx* h, int what, int level, double* out, int64_t count, int32_t* w_out);

/* Number of K or K_j vector products (columns) of the last build (Sec. 3.2.2 count).  */
int hodlr_napply(const hodlr_ctx* h, int64_t* out);

/* Kernel-time profile of the dense contraction kernel (the batched GEMM that carries the
 * peeling, projection, factorization and trace products).  hodlr_profile(h, 1) records a
 * pair of CUDA events on the context's stream around every GEMM launch from then on;
 * hodlr_profile_read(h, out) synchronises and returns out[0] = total kernel milliseconds,
 * out[1] = launches, out[2] = algorithmic flops (2 M N K per matrix product),
 * out[3] = algorithmic operand bytes (each of A, B read once and C written once), and per
 * kernel family v (0 SIMT tiles, 1 FP32 large tiles, 2 double-float, 3 narrow products,
 * 4 tcgen05 3xTF32, 5 tcgen05 BF16 digit slices from sliced planes, 6 fused long-K digit
 * slices, 7 fused short-K digit slices): out[4 + 4v] = milliseconds, out[5 + 4v] =
 * algorithmic flops (useful 2 M N K), out[6 + 4v] = launches, out[7 + 4v] = algorithmic
 * operand bytes; `out` holds 36 doubles.
 * hodlr_profile(h, 0) stops and clears.  Event pool: 65536 launches.
 * Diagnostics (environment): HODLR_PROFILE_DUMP=<file> makes hodlr_profile_read write one
 * CSV row per GEMM launch (shape, kernel variant, ms); HODLR_TRACE=<file> makes
 * hodlr_profile(h, 1) also record an event after every kernel launch of the library on the
 * context's stream (up to 200000), and hodlr_profile_read write per-launcher totals
 * (name, launches, ms; the time between consecutive launches' completion, idle gaps
 * included).  The trace adds host overhead per launch: not for timed runs.  */
int hodlr_profile(hodlr_ctx* h, int enable);
int hodlr_profile_read(hodlr_ctx* h, double* out);

/* Launch statistics: number of kernels launched since the last reset (host int64).  */
int hodlr_kernel_count(const hodlr_ctx* h, int64_t* out);
int hodlr_reset_kernel_count(hodlr_ctx* h);

/* Measured arithmetic peak of one pipe of the current device (the paper has no counterpart;
 * roofline denominators of the kernels that are not HBM-bound).  which: 0 FP32 FFMA, 1 FP64
 * DFMA (fused multiply-adds of 16 independent chains per thread on every SM), 2 tcgen05
 * kind::tf32, 3 tcgen05 kind::f16 with BF16 operands (one CTA per SM issuing 128 x 256
 * MMAs back to back on shared-memory operands, FP32 accumulation in TMEM).  tflops_out:
 * host, best of three timed launches after a warm-up, in 10^12 flop/s (a multiply-add
 * counts 2).  Runs on the legacy default stream and synchronises it; allocates nothing.
 * HODLR_ETIMEOUT if an MMA completion wait gave up.  */
int hodlr_peak(int which, double* tflops_out);

/* FP64-class batched product on the BF16 tensor cores (the building block of HODLR_MIXED_BF16;
 * a dense contraction in the paper's HODLR arithmetic, Table "HODLR operations", Sec. 3.1):
 *   C_b = alpha op(A_b) op(B_map(b)) + beta C_b,  b = 0 .. batch-1,
 * column-major FP64 device matrices: op(A_b) is M x K (A_b = A + b sA, ld lda, transposed when
 * tA), op(B) is K x N (B_i = B + i sB, ld ldb, transposed when tB), map(b) = b, b^1, b>>1 for
 * bmap = 0, 1, 2, C_b = C + b sC (ld ldc); sA = 0 (sB = 0) shares one A (B) among the batch.
 * Each operand row (A) or column (B) is scaled by a power of two and cut into seven balanced
 * 7-bit digits held exactly in BF16; the 28 digit products with p + q <= 6 run on tcgen05 with
 * FP32 accumulation in tensor memory, exact for the four leading digit groups over 512-long
 * chunks of K; the result is assembled in 64-bit integers and rounded once.  Error below
 * ~2^-46 of sum_k max_k'|A_ik'| max_k'|B_k'j| (finite inputs).
 * work: caller-owned device scratch of work_bytes >= 64 MiB, 256-byte aligned (slice planes and
 * split-K partials; larger problems are processed in batch and column chunks).  cuda_stream may
 * be NULL.  Allocates nothing.  HODLR_ENOMEM if even one product does not fit work_bytes;
 * HODLR_ETIMEOUT if a bounded wait gave up.  Synchronises the stream.  */
int hodlr_dgemm_slices(int M, int N, int K, int batch, const double* A, long long lda, long long sA, int tA,
                       const double* B, long long ldb, long long sB, int tB, int bmap, double alpha, double beta,
                       double* C, long long ldc, long long sC, void* work, size_t work_bytes, void* cuda_stream);

/* Tile autotuner (the project's own, for the batched workloads' kernel choices).  With
 * enable != 0 the context's later builds and evaluations (HODLR_MIXED_BF16 contexts; not
 * inside a captured graph) time, at the first occurrence of each digit-slice product shape,
 * every candidate plan: the product from slice planes in the workspace (128 x 96 tiles, or for
 * K > 128 also 128 x 48 tiles with two CTAs per SM or in a persistent warp-specialised kernel),
 * and where the shape allows, the fused kernels
 * with either tile (64 x 80 or 128 x 48 for long-K A^T B) and one or four times the default
 * chunks of K per CTA.  Each candidate runs once to warm up and twice
 * timed (CUDA events on the context's stream) into a scratch C carved from the slice
 * workspace; the fastest plan is remembered for the process (all contexts and threads) and
 * the product then runs with it, so results are those of the chosen kernels.  Shapes whose
 * scratch C would exceed half the slice workspace keep the default plan.  enable = 0 stops
 * tuning; remembered plans stay in use.  */
int hodlr_autotune(hodlr_ctx* h, int enable);
/* The remembered plans: up to cap rows of 13 int64 each into out (M, N, K, batch, tA, tB, A
 * shared, B shared, bmap, beta mode 0/1/2 for 0/1/other; path 0 planes / 1 fused, tile,
 * chunk multiplier); *n_out = the number of rows in the table (may exceed cap).  */
int hodlr_autotune_table(int64_t* out, int cap, int* n_out);
/* Forgets every remembered plan (products fall back to the default plans).  */
int hodlr_autotune_clear(void);

/* Kernel plan of the following hodlr_dgemm_slices calls on the calling thread (tests and shape
 * studies): path 0 slice planes (tile 0: 128 x 96, tile 1: 128 x 48 with two CTAs per SM, tile 2:
 * persistent warp-specialised 128 x 48, the last two for K > 128), path 1 the fused kernels where the shape allows them (tile 0 default, tile 1 the
 * 128 x 48 long-K tile; cprx: chunks of K per CTA times the default), path -1 automatic (the
 * default plan, or the autotuner's).  A plan a shape does not allow falls back to slice planes
 * with the default tile.  HODLR_EINVAL for other values.  */
int hodlr_dgemm_slices_plan(int path, int tile, int cprx);

/* Failure-detection hook (the paper has no counterpart; for tests of the bounded waits).
 * Sets, on the current device, how many times each tensor-core CTA polls its FIRST operand
 * barrier before giving up (polls < 0 restores the default of 2^22 polls).  A CTA whose
 * wait gives up records HODLR_ETIMEOUT, waits with the full limit for the copies it has
 * already issued, frees its tensor memory and returns, so the next library call that
 * checks the status (hodlr_build, hodlr_apply) returns HODLR_ETIMEOUT and clears it; the
 * context stays usable.  Every other wait keeps the full limit.  Not for production use:
 * a low limit makes correct products fail.  HODLR_ECUDA if the symbol cannot be written. */
int hodlr_debug_wait_limit(int polls);

/* Allocation-free physics product (the paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory -- code running inside another
 * framework's memory pool or under a hard memory budget, or at a point where the
 * allocator must not be called).  Computes Y = K X for the 1-D univariate model
 * (K = A^{-1} K_u A^{-1} + tau2 I on G interior points, Matern nu = 0.5 or 1.5) without a
 * context and without any workspace: X and Y are device arrays of G x ncols doubles,
 * column-major, natural order; theta is a host array of 4 doubles; cuda_stream may be
 * NULL.  Y may not overlap X: overlapping byte ranges return HODLR_EINVAL.
 *   Limit: G <= 2048; larger grids return HODLR_EINVAL.
 *   Scratch: a fixed 160.5 KiB array in device global memory, held by every GPU that loads
 *   the library until the process exits.  The first call on a device looks its address up
 *   (with that device current); make that first call before any stream capture.  All calls
 *   share the one array, so calls that overlap on the GPU (other streams or host threads)
 *   race and must be serialised by the caller.
 *   Allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.  */
int hodlr_apply_static(int G, double nu, const double* theta, const double* X, double* Y, int ncols,
                       void* cuda_stream);

const char* hodlr_last_error(const hodlr_ctx* h);
void hodlr_destroy(hodlr_ctx* h);

#ifdef __cplusplus
}
#endif
#endif /* HODLR_H */
