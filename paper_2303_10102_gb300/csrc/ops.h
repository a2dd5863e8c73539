// Host launchers of the library's CUDA kernels (shared by the translation units).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "tree.cuh"

namespace hodlr {

struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// ------------------------------------------------------------------------------ GEMM
// Batched column-major GEMM  C_b = alpha * op(A_b) op(B_{map(b)}) + beta * C_b  (M x N, inner K).
//   A_b = A + b*sA, B_i = B + i*sB, C_b = C + b*sC (element offsets); map(b) = b, b^1, b>>1
//   for bmap = 0, 1, 2.  Long inner dimensions are split across CTAs and reduced in a
//   fixed order (deterministic) through `scratch`.
enum BMap { BMAP_ID = 0, BMAP_XOR1 = 1, BMAP_SHR1 = 2 };
struct GemmArgs {
  int M = 0, N = 0, K = 0;
  const void* A = nullptr; long long lda = 0, sA = 0; int tA = 0;
  const void* B = nullptr; long long ldb = 0, sB = 0; int tB = 0; int bmap = BMAP_ID;
  void* C = nullptr; long long ldc = 0, sC = 0;
  double alpha = 1.0, beta = 0.0;
  int batch = 1;
  // Variable-size blocks (uneven trees): offmode 1 -> rows of A and C start at off[b] and
  // M_b = off[b+1]-off[b]; offmode 2 -> rows of A and B start at off[b] and K_b likewise
  // (M resp. K above are then the maxima).
  const int* off = nullptr;
  int offmode = 0;
};
template <class TA, class TB, class TC, class Acc>
void gemm(const GemmArgs& g, Scratch s, cudaStream_t st);
// Same contraction with double-float (hi+lo FP32) accumulation on the FP32 pipes (~48 bits).
// Operand types: double (split on load), float, or float2 (already split by df_split).
template <class TA, class TB, class TC>
void gemm_df(const GemmArgs& g, Scratch s, cudaStream_t st);
// y[i] = (hi, lo) FP32 pair of x[i] (hi = x rounded to FP32, lo = x - hi rounded).
void df_split(const double* x, float2* y, long long n, cudaStream_t st);

// FP32-accurate product C (M x N, ld ldc) = A B on the tcgen05 tensor cores (3xTF32).  A is
// given K-major: element (m, k) at A[k + m*lda] (for a symmetric matrix, its plain storage),
// as a TF32 head Ahi and an FP32 remainder Alo (see tf32_split); B is K x N column-major
// (ldb).  Returns false (nothing launched) when the shape or alignment is not supported.
bool tf32x3_gemm(const float* Ahi, const float* Alo, long long lda, const float* B, long long ldb, float* C,
                 long long ldc, int M, int N, int K, cudaStream_t st);
bool tf32x3_supported(int M, int K, long long lda, long long ldb, long long ldc);
// Batched C_b = alpha A_b^T B_b + beta C_b (tA = 1, tB = 0: K contiguous in both operands) on the
// tensor cores (3xTF32, both operands split in the kernel), split across K when the batch has
// few tiles.  The products of a batch must be row ranges of one panel and K a multiple of 32;
// returns false (nothing launched) otherwise.
bool tf32x3_gemm_tn(const GemmArgs& g, Scratch s, cudaStream_t st);
// Batched C_b = alpha A_b B_{map(b)} + beta C_b (tA = tB = 0: A M-contiguous, B K-contiguous) on
// the tensor cores (3xTF32), without a split of K: A_b row ranges of one panel or stacked
// matrices, B_b likewise (a stacked or single B when K is not a multiple of 32).  M >= 128,
// leading dimensions multiples of 4.  Returns false (nothing launched) when not supported.
bool tf32x3_gemm_nn(const GemmArgs& g, cudaStream_t st);
// FP64-class product C_b = alpha op(A_b) op(B_map(b)) + beta C_b of FP64 operands on the BF16
// tensor cores by exact digit slices (six 7-bit digits per operand; error about 2^-41 of
// sum_k max|A_i.| max|B_.j|).  Used in place of the FP64 FMA product while g_oz_cfg.on is set
// (this thread); its slicing planes live in g_oz_cfg.work, split-K partials in `split`.
// Returns false (nothing launched) for shapes it does not take.
struct OzConfig {
  bool on = false;
  bool tune = false;   // time the candidate plans of products not yet tuned (tile autotuner)
  Scratch work;    // slice planes and exponents
  Scratch split;   // split-K partials (used when larger than the caller's scratch)
};
extern thread_local OzConfig g_oz_cfg;
bool oz_eligible(const GemmArgs& g);
bool oz_gemm(const GemmArgs& g, Scratch split, cudaStream_t st);
bool oz_gemm_any(const GemmArgs& g, Scratch split, cudaStream_t st);   // without the size thresholds
int oz_status_take(cudaStream_t st);
// the autotuner's remembered plans: up to cap rows of 13 (shape key of 10, path, tile, chunk
// multiplier) into out; returns the number of rows in the table
int oz_tuned_table(int64_t* out, int cap);
void oz_tuned_clear();
void oz_force_plan(int path, int tile, int cprx);   // this thread's products (path < 0: automatic)   // HODLR_ETIMEOUT recorded by a product (and cleared), or 0
// Ordered reduction of FP32 split-K partials into C (alpha, beta, offsets as in g).
void splitk_reduce_f32(const GemmArgs& g, int nsplit, const float* part, cudaStream_t st);
// hi = x with the low 13 mantissa bits cleared, lo = x - hi (exact); hi may alias x.
void tf32_split(const float* x, float* hi, float* lo, long long n, cudaStream_t st);
// Device status word of the tensor-core kernels (HODLR_ETIMEOUT after a wait gave up);
// returns it (synchronising the stream) and clears it.
int tc_status_take(cudaStream_t st);
int tc_set_first_wait_limit(int polls);   // < 0: restore the default

// ------------------------------------------------------------------------------ elementwise / data movement
template <class TS, class TD> void convert(const TS* src, TD* dst, long long n, cudaStream_t st);
template <class T> void fill(T* p, T v, long long n, cudaStream_t st);
// dst[i + j*ldd] = src[perm[i] + j*lds] (gather rows), or scatter when `scatter`:
// dst[perm[i] + j*ldd] = src[i + j*lds]; optional alpha*src + beta*dst2 for scatter_axpy.
// cluster-tree order on the device (tree.cu): permpad[N] tree-layout row -> natural index (-1 on
// padding rows), rowid[N] (may be null) tree-layout row -> real tree position (-1 on padding),
// real2pad[Nr] real tree position -> tree-layout row
void tree_order(const TreeDesc& t, int N, int* permpad, int* rowid, int* real2pad, cudaStream_t st);
// tree-layout row -> row of a physics panel with variable blocks of Ns x qc (-1 on padding)
void tree_phys_perm(const int* permpad, int N, int Ns, int nvar, int qc, int* out, cudaStream_t st);
// rows of the right children of the level whose nodes are msize rows (real rows only)
void tree_level_mask(int N, int msize, const int* rowid, unsigned char* mask, cudaStream_t st);

template <class TS, class TD>
void permute_rows(const TS* src, long long lds, TD* dst, long long ldd, const int* perm, int n,
                  int ncols, int scatter, cudaStream_t st);
// y = a*x + b*y over n x ncols (ld each)
template <class T>
void axpby(int n, int ncols, double a, const T* x, long long ldx, double b, T* y, long long ldy,
           cudaStream_t st);

// ------------------------------------------------------------------------------ small dense (batched, one CTA per matrix)
// Pivoted Cholesky of Gram matrices G_b (c x c FP64, stride c*c): rank r_b = number of
// leading pivots with sqrt(Schur diagonal) > thr_rel * (first pivot), <= cap; pivots J_b
// (c ints, -1 padded); Rinv_b = inverse of the r_b x r_b upper factor of G[J,J], zero-padded
// to w x w (TR).  frozen != 0: J is an input and only G[J,J] is factored.  work: 2*c*c FP64
// per matrix.  status: set to -3 (not SPD) on failure of a frozen factorization.
template <class TR>
void pivoted_cholesky(int nb, int c, int cap, int w, const double* G, double thr_rel, int* rank, int* J,
                      TR* Rinv, int frozen, double* work, int* status, cudaStream_t st);
// In-place lower Cholesky of nb matrices (n x n, ld, stride); if rank != nullptr the rows and
// columns >= rank[b] are replaced by the identity.  logdet[b] = 2 sum log diag (optional).
void potrf_lower(int nb, int n, double* A, long long ld, long long stride, const int* rank,
                 double* logdet, int* status, cudaStream_t st);
// Inverse of lower-triangular L_b into Linv_b (FP64).
void trtri_lower(int nb, int n, const double* L, long long ld, long long stride, double* Linv,
                 cudaStream_t st);
// Inverses of the 32 x 32 diagonal blocks of L_b written into the same blocks of X_b (n a
// multiple of 32); the off-diagonal blocks of X_b are not touched.
void trtri_diag32(int nb, int n, const double* L, long long ld, long long stride, double* X, cudaStream_t st);
// Set D_b = diag + alpha * D_b for square n x n blocks (alpha*D + I when add_identity).
void shift_identity(int nb, int n, double* D, long long ld, long long stride, double alpha,
                    double diag, cudaStream_t st);
// Copy a square block: dst_b[i,j] = scale * src_b[i,j] (types may differ).
template <class TS, class TD>
void copy_blocks(int nb, int m, int n, const TS* src, long long lds, long long ss, TD* dst, long long ldd,
                 long long sd, double scale, cudaStream_t st);
// gather columns J of Y (rows [b*row_stride, b*row_stride+m)) into dst (zero beyond rank).
template <class T>
void gather_columns(int nb, int m, long long row_stride, const T* Y, long long ldy, const int* J, int c,
                    const int* rank, int w, T* dst, long long ldd, cudaStream_t st);
// Alg. 2 core: M2 = skew(Yp) - Yp with skew(Y) = tril(Y,-1) - tril(Y,-1)^T (w x w per pair).
template <class T> void alg2_core(int nb, int w, const T* Yp, T* M2, cudaStream_t st);
// Leaf solves with the FP64 Cholesky factors: out_b = (L_b L_b^T)^{-1} in_b for every leaf b
// (rows [b*nl, (b+1)*nl) of the panels, q columns).  Forward substitution by column sweeps,
// backward substitution by warp dot products; backward stable, unlike an explicit inverse.
template <class TI, class TO>
void leaf_trsm(int nleaves, int nl, const double* L, const TI* in, long long ldi, TO* out, long long ldo, int q,
               cudaStream_t st);
// symmetrise and gather leaf blocks: A_b = (E_b + E_b^T)/2, E_b = E[b nl + (0:n_b), 0:n_b] with
// n_b = counts[b] real rows in leaf slot b; the padding part of the nl x nl block is pad * I
// (1 for leaves of K~, 0 for leaves of a derivative matrix)
template <class TS, class TD>
void extract_leaves(int nleaves, int nl, const int* counts, const TS* E, long long lde, TD* A, double pad,
                    cudaStream_t st);

// ------------------------------------------------------------------------------ reductions
// out[b] = tr(X_b Y_b) (mode 0) or tr(X_b Y_b^T) (mode 1) over the leading n_b x n_b block
// (n_b = sizes[b] or n), or tr(X_b) when Y == nullptr; X_b = X + b*sX (ld ldx), Y_b likewise.
template <class T>
void trace_products(int nb, int n, const int* sizes, const T* X, long long ldx, long long sX,
                    const T* Y, long long ldy, long long sY, int mode, double* out, cudaStream_t st);
// sum of n doubles -> out (single value, fixed order)
void sum_doubles(const double* x, int n, double* out, int accumulate, cudaStream_t st);
// dot products of columns: out[j] = sum_i x[i,j]*y[i,j] in FP64
template <class TX, class TY>
void dot_columns(int n, int ncols, const TX* x, long long ldx, const TY* y, long long ldy, double* out,
                 cudaStream_t st);
// finite check: sets *flag = 1 when x has NaN/Inf
template <class T> void check_finite(const T* x, long long n, int* flag, cudaStream_t st);
// log of the product of positive diag entries etc. live in the kernels above.

// ------------------------------------------------------------------------------ physics
struct PhysicsDesc {
  int dim, G, nvar;
  double nu, h;
  int L;          // FFT embedding length per axis (power of two >= 2G-1)
  int L1, L2;     // four-step split of a 1-D embedding longer than 4096 (L = L1*L2)
  int df_fft = 0; // FP64 fields: FFT butterflies in double-float arithmetic (FP32 pipes)
};
// Philox probe panel R^(level): N x ncols in tree order; row i non-zero iff it lies in the
// right child of its level pair (right_child[i] = level mask bit).  The counter of row i is
// rowid[i] (its position in the cluster tree without padding rows), or i when rowid is null.
template <class T>
void probe_panel(int N, int ncols, int level, int stream_id, uint64_t seed, const unsigned char* mask,
                 const int* rowid, T* out, long long ld, cudaStream_t st);
// Matern embedding spectra (real parts, in the FFT's internal order):
//   lam[0] for K_u, lam[1] for dK_u/dell.  Computes kernel values, then forward FFT.
template <class T>
void matern_spectra(const PhysicsDesc& p, double sigma2, double ell, T* lam0, T* lam1, void* work,
                    const T* tw, cudaStream_t st);
// twiddle table for length L: tw[k] = (cos, -sin)(2 pi k / L), k < L/2 (interleaved)
template <class T> void twiddles(int L, T* tw, cudaStream_t st);
// FFT convolution of ncols real columns (Ns x ncols, ld) with one or two real spectra:
// out0 = K_u-conv(in), out1 = second-spectrum conv (if lam1 != nullptr).
template <class T>
void fft_convolve(const PhysicsDesc& p, int ncols, const T* in, long long ldi, const T* lam0,
                  const T* lam1, T* out0, T* out1, long long ldo, void* work, const T* tw,
                  cudaStream_t st);
size_t fft_work_bytes(const PhysicsDesc& p, int ncols, int real_bytes);
// A^{-1} on ncols columns (Ns x ncols, ld): 1-D tridiagonal scan, 2-D DST + Thomas.
// coef: per-theta tables (1-D: a[i], b[i] (2*G); 2-D: a,b per x-mode (2*G*G)); S: DST
// matrix (2-D, G x G); work: Ns*ncols T (2-D).  df: DST products with double-float
// accumulation (FP64 fields).  coef32: FP32 copy of the 2-D tables; when given, FP32 fields
// run the Thomas recurrences in FP32 arithmetic.
// tc: TF32 head and remainder of the FP32 DST matrix; when given (FP32 fields), the DST
// products run on the tensor cores (tf32x3_gemm).  df_S / df_X: the DST matrix split into
// double-float pairs and a scratch panel (G x G*ncols pairs) for the split field; when
// given with df (FP64 fields), the double-float products read pre-split operands.
struct DstSplit {
  const float* hi = nullptr;
  const float* lo = nullptr;
  const float2* df_S = nullptr;
  float2* df_X = nullptr;
};
template <class T>
void solve_A(const PhysicsDesc& p, int ncols, const T* in, long long ldi, T* out, long long ldo,
             const double* coef, const T* S, T* work, Scratch s, cudaStream_t st, int df = 0,
             const float* coef32 = nullptr, DstSplit tc = DstSplit());
// per-theta coefficient tables of the Thomas recurrences (see physics.cu)
void tridiag_tables(const PhysicsDesc& p, double kappa, double* coef, cudaStream_t st);
template <class T> void dst_matrix(int G, T* S, cudaStream_t st);

}  // namespace hodlr
