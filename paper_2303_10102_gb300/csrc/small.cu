// Batched small dense kernels (one CTA per matrix) and data-movement / reduction kernels.
//
//   pivoted_cholesky  -- column pivoting of the QR of Alg. 1 step 3, taken on the FP64 Gram
//                        matrix Y^T Y (same pivots and |R_ii| as Householder QR with column
//                        pivoting in exact arithmetic), with the rank rule of the readings;
//   potrf / trtri     -- leaf Cholesky factors and the SMW cores of App. C (FP64);
//   extract_leaves    -- symmetrised leaf blocks of eq. leaf sample;
//   trace_products    -- block traces tr(X_b Y_b) of App. B.3;
//   alg2_core         -- the skew / upper-triangular split of Alg. 2 step 2.
#include <math.h>

#include "common.cuh"
#include "ops.h"

namespace hodlr {
namespace {

constexpr int NTS = 256;

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
  __syncthreads();
  return r;  // valid in thread 0
}

// ---------------------------------------------------------------- pivoted Cholesky (Gram of Y)
template <class TR>
__global__ void pivoted_cholesky_kernel(int c, int cap, int w, const double* Gall, double thr_rel,
                                        int* rank, int* Jall, TR* Rinvall, int frozen, double* work,
                                        int* status, int schur_in_smem) {
  extern __shared__ unsigned char sm_raw[];
  // the c x c Schur complement lives in shared memory when it fits (it is updated at every
  // pivot step), else in the global work area
  double* As = (double*)sm_raw;
  int* piv = (int*)(sm_raw + (schur_in_smem ? (size_t)c * c * sizeof(double) : 0));   // c
  int* done = piv + c;                           // c flags
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_r, s_stop, s_fail;
  __shared__ double s_d0;
  const int b = blockIdx.x;
  const double* G = Gall + (size_t)b * c * c;
  double* Ag = work + (size_t)b * 2 * c * c;
  double* A = schur_in_smem ? As : Ag;           // Schur complement (original indexing)
  double* Rr = Ag + (size_t)c * c;               // factor rows: Rr[k*c + i] = R[k, i]
  int* J = Jall + (size_t)b * c;
  TR* Rinv = Rinvall + (size_t)b * w * w;
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) A[e] = G[e];
  for (int i = threadIdx.x; i < c; i += blockDim.x) { piv[i] = -1; done[i] = 0; }
  if (threadIdx.x == 0) { s_r = 0; s_stop = 0; s_d0 = 0.0; s_fail = 0; }
  __syncthreads();
  int nfix = 0;
  if (frozen) {
    if (threadIdx.x == 0) {
      int r = 0;
      while (r < c && J[r] >= 0) { piv[r] = J[r]; ++r; }
      s_r = r;
    }
    __syncthreads();
    nfix = s_r;
  }
  const int kmax = frozen ? nfix : min(c, cap);
  for (int k = 0; k < kmax; ++k) {
    // choose pivot: largest remaining Schur diagonal (lowest index on ties) or frozen
    int p;
    if (frozen) {
      p = piv[k];
    } else {
      double best = -1.0;
      int bi = 0x7fffffff;
      for (int i = threadIdx.x; i < c; i += blockDim.x) {
        if (done[i]) continue;
        double d = A[i + (size_t)i * c];
        if (d > best || (d == best && i < bi)) { best = d; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_down_sync(0xffffffffu, best, o);
        int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      if (lane == 0) { sv[wid] = best; si[wid] = bi; }
      __syncthreads();
      if (threadIdx.x == 0) {
        double bb = sv[0];
        int ii = si[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
          if (sv[q] > bb || (sv[q] == bb && si[q] < ii)) { bb = sv[q]; ii = si[q]; }
        double rk = bb > 0.0 ? sqrt(bb) : 0.0;
        if (k == 0) s_d0 = rk;
        if (!(bb > 0.0) || rk <= thr_rel * s_d0 || ii >= c) s_stop = 1;
        else piv[k] = ii;
      }
      __syncthreads();
      if (s_stop) break;
      p = piv[k];
    }
    double dpp = A[p + (size_t)p * c];
    if (frozen && !(dpp > 0.0)) {
      if (threadIdx.x == 0) { *status = -3; s_fail = 1; }
      break;
    }
    double rkk = sqrt(dpp);
    // row k of R in original indexing; only not-yet-pivoted columns
    for (int i = threadIdx.x; i < c; i += blockDim.x) {
      double v = 0.0;
      if (i == p) v = rkk;
      else if (!done[i]) v = A[p + (size_t)i * c] / rkk;
      Rr[(size_t)k * c + i] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) { done[p] = 1; s_r = k + 1; }
    __syncthreads();
    // Schur update of the remaining block
    for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
      int i = e % c, j = e / c;
      if (done[i] || done[j]) continue;
      A[e] -= Rr[(size_t)k * c + i] * Rr[(size_t)k * c + j];
    }
    __syncthreads();
  }
  __syncthreads();
  const int r = frozen ? (s_fail ? 0 : nfix) : s_r;
  // outputs: rank, pivots
  if (threadIdx.x == 0) rank[b] = r;
  if (!frozen)
    for (int i = threadIdx.x; i < c; i += blockDim.x) J[i] = i < r ? piv[i] : -1;
  // Rinv: inverse of upper-triangular R_J (r x r), R_J[a][bb] = Rr[a*c + piv[bb]] (a <= bb)
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) Rinv[e] = TR(0);
  __syncthreads();
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    // column j of X = R^{-1}: X[j][j] = 1/R[j][j]; X[i][j] = -sum_{k=i+1..j} R[i][k] X[k][j] / R[i][i]
    double* x = A + (size_t)j * c;  // reuse A as column scratch (c >= r)
    x[j] = 1.0 / Rr[(size_t)j * c + piv[j]];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1; k <= j; ++k) s += Rr[(size_t)i * c + piv[k]] * x[k];
      x[i] = -s / Rr[(size_t)i * c + piv[i]];
    }
    for (int i = 0; i <= j; ++i) Rinv[i + (size_t)j * w] = (TR)x[i];
  }
}

// ---------------------------------------------------------------- lower Cholesky / inverse
__global__ void potrf_lower_kernel(int n, double* Aall, long long ld, long long stride, const int* rank,
                                   double* logdet, int* status) {
  __shared__ int s_fail;
  const int b = blockIdx.x;
  double* A = Aall + (size_t)b * stride;
  const int r = rank ? rank[b] : n;
  if (threadIdx.x == 0) s_fail = 0;
  // padded part -> identity
  if (r < n)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int i = e % n, j = e / n;
      if (i >= r || j >= r) A[i + (size_t)j * ld] = (i == j) ? 1.0 : 0.0;
    }
  __syncthreads();
  double ld_acc = 0.0;
  for (int k = 0; k < r; ++k) {
    double akk = A[k + (size_t)k * ld];
    if (!(akk > 0.0)) {
      if (threadIdx.x == 0) s_fail = 1;
      break;
    }
    double lkk = sqrt(akk);
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) A[i + (size_t)k * ld] /= lkk;
    if (threadIdx.x == 0) { A[k + (size_t)k * ld] = lkk; ld_acc += 2.0 * log(lkk); }
    __syncthreads();
    int m = r - k - 1;
    for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
      int i = k + 1 + (int)(e % m), j = k + 1 + (int)(e / m);
      if (i >= j) A[i + (size_t)j * ld] -= A[i + (size_t)k * ld] * A[j + (size_t)k * ld];
    }
    __syncthreads();
  }
  __syncthreads();
  // zero the strict upper triangle
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e % n, j = e / n;
    if (i < j) A[i + (size_t)j * ld] = 0.0;
  }
  if (threadIdx.x == 0) {
    if (s_fail) *status = -3;
    if (logdet) logdet[b] = s_fail ? NAN : ld_acc;
  }
}

// Blocked right-looking Cholesky of one matrix per CTA (no rank padding), 32-column panels:
// the diagonal block is factored by one warp in shared memory, the rows below it are solved
// against it (one row per thread), and the trailing matrix receives one rank-32 update from
// the panel held in shared memory.  The global matrix is read and written once per panel
// instead of once per column.
constexpr int PB = 32;
__global__ void potrf_blocked_kernel(int n, double* Aall, long long ld, long long stride, double* logdet,
                                     int* status) {
  extern __shared__ double pan[];        // n x (PB + 1): the panel rows below the diagonal block
  __shared__ double D[PB][PB + 1];
  __shared__ int s_fail;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* A = Aall + (size_t)b * stride;
  double ld_acc = 0.0;
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int kb = 0; kb < n; kb += PB) {
    const int nbk = min(PB, n - kb);
    for (int e = tid; e < nbk * nbk; e += blockDim.x) {
      const int i = e % nbk, j = e / nbk;
      D[i][j] = A[kb + i + (size_t)(kb + j) * ld];
    }
    __syncthreads();
    if (warp == 0) {
      for (int k = 0; k < nbk; ++k) {
        const double dkk = D[k][k];
        if (!(dkk > 0.0)) {
          if (lane == 0) s_fail = 1;
          break;
        }
        const double lkk = sqrt(dkk);
        if (lane == 0) ld_acc += 2.0 * log(lkk);
        __syncwarp();
        if (lane > k && lane < nbk) D[lane][k] /= lkk;
        if (lane == k) D[k][k] = lkk;
        __syncwarp();
        if (lane > k && lane < nbk)
          for (int j = k + 1; j <= lane; ++j) D[lane][j] -= D[lane][k] * D[j][k];
        __syncwarp();
      }
    }
    __syncthreads();
    if (s_fail) break;
    for (int e = tid; e < nbk * nbk; e += blockDim.x) {
      const int i = e % nbk, j = e / nbk;
      if (i >= j) A[kb + i + (size_t)(kb + j) * ld] = D[i][j];
    }
    const int r0 = kb + nbk, m = n - r0;
    // panel rows: x D^T = a, forward substitution per row
    for (int r = tid; r < m; r += blockDim.x) {
      double x[PB];
#pragma unroll
      for (int t = 0; t < PB; ++t) x[t] = t < nbk ? A[r0 + r + (size_t)(kb + t) * ld] : 0.0;
#pragma unroll
      for (int t = 0; t < PB; ++t) {
        if (t < nbk) {
          double v = x[t];
          for (int q = 0; q < t; ++q) v -= x[q] * D[t][q];
          x[t] = v / D[t][t];
        }
      }
#pragma unroll
      for (int t = 0; t < PB; ++t) {
        if (t < nbk) {
          pan[(size_t)r * (PB + 1) + t] = x[t];
          A[r0 + r + (size_t)(kb + t) * ld] = x[t];
        }
      }
    }
    __syncthreads();
    // trailing update of the lower triangle: A22 -= P P^T
    for (long long e = tid; e < (long long)m * m; e += blockDim.x) {
      const int i = (int)(e % m), j = (int)(e / m);
      if (i < j) continue;
      const double* pi = pan + (size_t)i * (PB + 1);
      const double* pj = pan + (size_t)j * (PB + 1);
      double acc = 0.0;
#pragma unroll 8
      for (int t = 0; t < nbk; ++t) acc += pi[t] * pj[t];
      A[r0 + i + (size_t)(r0 + j) * ld] -= acc;
    }
    __syncthreads();
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    if (i < j) A[i + (size_t)j * ld] = 0.0;
  }
  if (tid == 0) {
    if (s_fail) *status = -3;
    if (logdet) logdet[b] = s_fail ? NAN : ld_acc;
  }
}

// Inverses of the 32 x 32 diagonal blocks of lower-triangular matrices (one warp per block,
// lane c computes column c by forward substitution in shared memory); the rest of X is left
// to the caller.
__global__ void trtri_diag32_kernel(int nb, int n, const double* Lall, long long ld, long long stride,
                                    double* Xall) {
  __shared__ double Ls[4][32][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = n / 32;
  const long long gw = (long long)blockIdx.x * 4 + warp;   // (matrix, diagonal block)
  const int b = (int)(gw / nblk), d = (int)(gw % nblk);
  if (b >= nb) return;
  const double* L = Lall + (size_t)b * stride + (size_t)d * 32 * (ld + 1);
  double* X = Xall + (size_t)b * stride + (size_t)d * 32 * (ld + 1);
  for (int j = 0; j < 32; ++j) Ls[warp][lane][j] = L[lane + (size_t)j * ld];
  __syncwarp();
  double x[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    double v = k == lane ? 1.0 : 0.0;
#pragma unroll
    for (int q = 0; q < k; ++q) v -= Ls[warp][k][q] * x[q];
    x[k] = v / Ls[warp][k][k];
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) X[k + (size_t)lane * ld] = x[k];
}

__global__ void trtri_lower_kernel(int n, const double* Lall, long long ld, long long stride, double* Xall) {
  const int b = blockIdx.x;
  const double* L = Lall + (size_t)b * stride;
  double* X = Xall + (size_t)b * stride;
  // column j of X = L^{-1}: X[j][j] = 1/L[j][j]; X[i][j] = -sum_{k=j..i-1} L[i][k] X[k][j] / L[i][i]
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    for (int i = 0; i < j; ++i) X[i + (size_t)j * ld] = 0.0;
    X[j + (size_t)j * ld] = 1.0 / L[j + (size_t)j * ld];
    for (int i = j + 1; i < n; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s += L[i + (size_t)k * ld] * X[k + (size_t)j * ld];
      X[i + (size_t)j * ld] = -s / L[i + (size_t)i * ld];
    }
  }
}

__global__ void shift_identity_kernel(int n, double* Dall, long long ld, long long stride, double alpha,
                                      double diag) {
  double* D = Dall + (size_t)blockIdx.y * stride;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  int i = (int)(e % n), j = (int)(e / n);
  double v = alpha * D[i + (size_t)j * ld];
  if (i == j) v += diag;
  D[i + (size_t)j * ld] = v;
}

template <class TS, class TD>
__global__ void copy_blocks_kernel(int m, int n, const TS* src, long long lds, long long ss, TD* dst,
                                   long long ldd, long long sd, double scale) {
  const TS* S = src + (size_t)blockIdx.y * ss;
  TD* D = dst + (size_t)blockIdx.y * sd;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)m * n) return;
  int i = (int)(e % m), j = (int)(e / m);
  D[i + (size_t)j * ldd] = (TD)(scale * (double)S[i + (size_t)j * lds]);
}

template <class T>
__global__ void gather_columns_kernel(int m, long long row_stride, const T* Y, long long ldy, const int* Jall,
                                      int c, const int* rank, int w, T* dst, long long ldd) {
  const int b = blockIdx.z, k = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const long long row = b * row_stride + i;
  const int r = rank[b];
  T v = T(0);
  if (k < r) {
    int col = Jall[(size_t)b * c + k];
    v = Y[row + (size_t)col * ldy];
  }
  dst[row + (size_t)k * ldd] = v;
}

template <class T>
__global__ void alg2_core_kernel(int w, const T* Ypall, T* M2all) {
  const T* Y = Ypall + (size_t)blockIdx.y * w * w;
  T* M = M2all + (size_t)blockIdx.y * w * w;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= w * w) return;
  int i = e % w, j = e / w;
  T sk = T(0);
  if (i > j) sk = Y[i + (size_t)j * w];
  else if (i < j) sk = -Y[j + (size_t)i * w];
  M[e] = sk - Y[e];
}

template <class TS, class TD>
__global__ void extract_leaves_kernel(int nl, const int* counts, const TS* E, long long lde, TD* A, double pad) {
  const int b = blockIdx.y;
  const int lo = b * nl, n = counts[b];   // leaf slot b: its real rows first, then padding rows
  TD* Ab = A + (size_t)b * nl * nl;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)nl * nl) return;
  int i = (int)(e % nl), j = (int)(e / nl);
  double v = 0.0;
  if (i < n && j < n) v = 0.5 * ((double)E[lo + i + (size_t)j * lde] + (double)E[lo + j + (size_t)i * lde]);
  else if (i == j) v = pad;   // padding rows: unit diagonal in K~ (decoupled), zero in dK~
  Ab[i + (size_t)j * nl] = (TD)v;
}

// ---------------------------------------------------------------- reductions
template <class T>
__global__ void trace_products_kernel(int n, const int* sizes, const T* X, long long ldx, long long sX,
                                      const T* Y, long long ldy, long long sY, int swapJ, double* out) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  const int nb = sizes ? sizes[b] : n;
  const T* Xb = X + (size_t)b * sX;
  const T* Yb = Y ? Y + (size_t)b * sY : nullptr;
  double s = 0.0;
  if (!Yb) {
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += (double)Xb[i + (size_t)i * ldx];
  } else {
    // mode 0: tr(X Y) = sum_{i,j} X[i,j] Y[j,i];  mode 1: tr(X Y^T) = sum_{i,j} X[i,j] Y[i,j]
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, nty = blockDim.x >> 5;
    for (int j = ty; j < nb; j += nty)
      for (int i = tx; i < nb; i += 32) {
        const double yv = swapJ ? (double)Yb[i + (size_t)j * ldy] : (double)Yb[j + (size_t)i * ldy];
        s += (double)Xb[i + (size_t)j * ldx] * yv;
      }
  }
  double t = block_sum(s, red);
  if (threadIdx.x == 0) out[b] = t;
}

__global__ void sum_doubles_kernel(const double* x, int n, double* out, int accumulate) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  double t = block_sum(s, red);
  if (threadIdx.x == 0) *out = accumulate ? *out + t : t;
}

template <class TX, class TY>
__global__ void dot_columns_kernel(int n, const TX* x, long long ldx, const TY* y, long long ldy, double* out) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    s += (double)x[i + (size_t)j * ldx] * (double)y[i + (size_t)j * ldy];
  double t = block_sum(s, red);
  if (threadIdx.x == 0) out[j] = t;
}

template <class T>
__global__ void check_finite_kernel(const T* x, long long n, int* flag) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  int bad = 0;
  for (; i < n; i += stride)
    if (!isfinite((double)x[i])) bad = 1;
  if (bad) *flag = 1;
}

template <class TS, class TD>
__global__ void convert_kernel(const TS* s, TD* d, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += stride) d[i] = (TD)s[i];
}

template <class T>
__global__ void fill_kernel(T* p, T v, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += stride) p[i] = v;
}

template <class TS, class TD>
__global__ void permute_rows_kernel(const TS* src, long long lds, TD* dst, long long ldd, const int* perm, int n,
                                    int scatter) {
  const int j = blockIdx.y;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = perm[i];   // -1: a padding row of the tree layout (no natural row)
  if (scatter) {
    if (p >= 0) dst[p + (size_t)j * ldd] = (TD)src[i + (size_t)j * lds];
  } else {
    dst[i + (size_t)j * ldd] = p >= 0 ? (TD)src[p + (size_t)j * lds] : TD(0);
  }
}

template <class T>
__global__ void axpby_kernel(int n, double a, const T* x, long long ldx, double b, T* y, long long ldy) {
  const int j = blockIdx.y;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T* yy = y + (size_t)j * ldy;
  T v = (T)a * x[i + (size_t)j * ldx];   // arithmetic in the field's own type
  if (b != 0.0) v += (T)b * yy[i];
  yy[i] = v;
}

int grid1d(long long n) { return (int)std::min<long long>(std::max<long long>(1, (n + 255) / 256), 152 * 16); }

}  // namespace

template <class TR>
void pivoted_cholesky(int nb, int c, int cap, int w, const double* G, double thr_rel, int* rank, int* J,
                      TR* Rinv, int frozen, double* work, int* status, cudaStream_t st) {
  if (nb <= 0) return;
  // shared memory for the Schur complement when the batch is at most one CTA per SM (the
  // coarse levels, latency-bound); the deep levels keep many small CTAs per SM with it in L2
  const size_t schur = (size_t)c * c * sizeof(double);
  const int in_smem = schur + 2 * c * sizeof(int) <= 200 * 1024 && nb <= 152;
  size_t sm = 2 * c * sizeof(int) + (in_smem ? schur : 0);
  if (sm > 48 * 1024)
    HODLR_CUDA(cudaFuncSetAttribute(pivoted_cholesky_kernel<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  pivoted_cholesky_kernel<TR><<<nb, NTS, sm, st>>>(c, cap, w, G, thr_rel, rank, J, Rinv, frozen, work, status,
                                                   in_smem);
  check_launch("pivoted_cholesky");
}
template void pivoted_cholesky<double>(int, int, int, int, const double*, double, int*, int*, double*, int,
                                       double*, int*, cudaStream_t);
template void pivoted_cholesky<float>(int, int, int, int, const double*, double, int*, int*, float*, int,
                                      double*, int*, cudaStream_t);

void potrf_lower(int nb, int n, double* A, long long ld, long long stride, const int* rank, double* logdet,
                 int* status, cudaStream_t st) {
  if (nb <= 0 || n <= 0) return;
  const size_t pan = (size_t)n * (PB + 1) * sizeof(double);
  if (!rank && n >= 4 * PB && pan <= 200 * 1024) {
    if (pan > 48 * 1024)
      HODLR_CUDA(cudaFuncSetAttribute(potrf_blocked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pan));
    potrf_blocked_kernel<<<nb, 256, pan, st>>>(n, A, ld, stride, logdet, status);
    check_launch("potrf_blocked");
    return;
  }
  potrf_lower_kernel<<<nb, 512, 0, st>>>(n, A, ld, stride, rank, logdet, status);
  check_launch("potrf_lower");
}

void trtri_diag32(int nb, int n, const double* L, long long ld, long long stride, double* X, cudaStream_t st) {
  if (nb <= 0 || n <= 0) return;
  const long long warps = (long long)(n / 32) * nb;
  trtri_diag32_kernel<<<cdiv(warps, 4), 128, 0, st>>>(nb, n, L, ld, stride, X);
  check_launch("trtri_diag32");
}

void trtri_lower(int nb, int n, const double* L, long long ld, long long stride, double* Linv, cudaStream_t st) {
  if (nb <= 0 || n <= 0) return;
  trtri_lower_kernel<<<nb, std::min(512, ((n + 31) / 32) * 32), 0, st>>>(n, L, ld, stride, Linv);
  check_launch("trtri_lower");
}

void shift_identity(int nb, int n, double* D, long long ld, long long stride, double alpha, double diag,
                    cudaStream_t st) {
  if (nb <= 0 || n <= 0) return;
  dim3 g(cdiv((long long)n * n, 256), nb);
  shift_identity_kernel<<<g, 256, 0, st>>>(n, D, ld, stride, alpha, diag);
  check_launch("shift_identity");
}

template <class TS, class TD>
void copy_blocks(int nb, int m, int n, const TS* src, long long lds, long long ss, TD* dst, long long ldd,
                 long long sd, double scale, cudaStream_t st) {
  if (nb <= 0 || m <= 0 || n <= 0) return;
  dim3 g(cdiv((long long)m * n, 256), nb);
  copy_blocks_kernel<TS, TD><<<g, 256, 0, st>>>(m, n, src, lds, ss, dst, ldd, sd, scale);
  check_launch("copy_blocks");
}
#define CB(TS, TD) \
  template void copy_blocks<TS, TD>(int, int, int, const TS*, long long, long long, TD*, long long, long long, \
                                    double, cudaStream_t);
CB(double, double) CB(float, float) CB(double, float) CB(float, double)
#undef CB

template <class T>
void gather_columns(int nb, int m, long long row_stride, const T* Y, long long ldy, const int* J, int c,
                    const int* rank, int w, T* dst, long long ldd, cudaStream_t st) {
  if (nb <= 0 || w <= 0 || m <= 0) return;
  dim3 g(cdiv(m, 256), w, nb);
  gather_columns_kernel<T><<<g, 256, 0, st>>>(m, row_stride, Y, ldy, J, c, rank, w, dst, ldd);
  check_launch("gather_columns");
}
template void gather_columns<double>(int, int, long long, const double*, long long, const int*, int, const int*,
                                     int, double*, long long, cudaStream_t);
template void gather_columns<float>(int, int, long long, const float*, long long, const int*, int, const int*,
                                    int, float*, long long, cudaStream_t);

template <class T>
void alg2_core(int nb, int w, const T* Yp, T* M2, cudaStream_t st) {
  if (nb <= 0 || w <= 0) return;
  dim3 g(cdiv(w * w, 256), nb);
  alg2_core_kernel<T><<<g, 256, 0, st>>>(w, Yp, M2);
  check_launch("alg2_core");
}
template void alg2_core<double>(int, int, const double*, double*, cudaStream_t);
template void alg2_core<float>(int, int, const float*, float*, cudaStream_t);

template <class TS, class TD>
void extract_leaves(int nleaves, int nl, const int* counts, const TS* E, long long lde, TD* A, double pad,
                    cudaStream_t st) {
  dim3 g(cdiv((long long)nl * nl, 256), nleaves);
  extract_leaves_kernel<TS, TD><<<g, 256, 0, st>>>(nl, counts, E, lde, A, pad);
  check_launch("extract_leaves");
}
template void extract_leaves<double, double>(int, int, const int*, const double*, long long, double*, double,
                                             cudaStream_t);
template void extract_leaves<float, double>(int, int, const int*, const float*, long long, double*, double,
                                            cudaStream_t);
template void extract_leaves<float, float>(int, int, const int*, const float*, long long, float*, double,
                                           cudaStream_t);

template <class T>
void trace_products(int nb, int n, const int* sizes, const T* X, long long ldx, long long sX, const T* Y,
                    long long ldy, long long sY, int swapJ, double* out, cudaStream_t st) {
  if (nb <= 0) return;
  trace_products_kernel<T><<<nb, NTS, 0, st>>>(n, sizes, X, ldx, sX, Y, ldy, sY, swapJ, out);
  check_launch("trace_products");
}
template void trace_products<double>(int, int, const int*, const double*, long long, long long, const double*,
                                     long long, long long, int, double*, cudaStream_t);
template void trace_products<float>(int, int, const int*, const float*, long long, long long, const float*,
                                    long long, long long, int, double*, cudaStream_t);

void sum_doubles(const double* x, int n, double* out, int accumulate, cudaStream_t st) {
  sum_doubles_kernel<<<1, 1024, 0, st>>>(x, n, out, accumulate);
  check_launch("sum_doubles");
}

template <class TX, class TY>
void dot_columns(int n, int ncols, const TX* x, long long ldx, const TY* y, long long ldy, double* out,
                 cudaStream_t st) {
  if (ncols <= 0) return;
  dot_columns_kernel<TX, TY><<<ncols, 1024, 0, st>>>(n, x, ldx, y, ldy, out);
  check_launch("dot_columns");
}
template void dot_columns<double, double>(int, int, const double*, long long, const double*, long long, double*,
                                          cudaStream_t);
template void dot_columns<float, double>(int, int, const float*, long long, const double*, long long, double*,
                                         cudaStream_t);
template void dot_columns<float, float>(int, int, const float*, long long, const float*, long long, double*,
                                        cudaStream_t);

template <class T>
void check_finite(const T* x, long long n, int* flag, cudaStream_t st) {
  if (n <= 0) return;
  check_finite_kernel<T><<<grid1d(n), 256, 0, st>>>(x, n, flag);
  check_launch("check_finite");
}
template void check_finite<double>(const double*, long long, int*, cudaStream_t);
template void check_finite<float>(const float*, long long, int*, cudaStream_t);

template <class TS, class TD>
void convert(const TS* src, TD* dst, long long n, cudaStream_t st) {
  if (n <= 0) return;
  convert_kernel<TS, TD><<<grid1d(n), 256, 0, st>>>(src, dst, n);
  check_launch("convert");
}
template void convert<double, float>(const double*, float*, long long, cudaStream_t);
template void convert<float, double>(const float*, double*, long long, cudaStream_t);
template void convert<double, double>(const double*, double*, long long, cudaStream_t);
template void convert<float, float>(const float*, float*, long long, cudaStream_t);

template <class T>
void fill(T* p, T v, long long n, cudaStream_t st) {
  if (n <= 0) return;
  fill_kernel<T><<<grid1d(n), 256, 0, st>>>(p, v, n);
  check_launch("fill");
}
template void fill<double>(double*, double, long long, cudaStream_t);
template void fill<float>(float*, float, long long, cudaStream_t);
template void fill<int>(int*, int, long long, cudaStream_t);

template <class TS, class TD>
void permute_rows(const TS* src, long long lds, TD* dst, long long ldd, const int* perm, int n, int ncols,
                  int scatter, cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return;
  dim3 g(cdiv(n, 256), ncols);
  permute_rows_kernel<TS, TD><<<g, 256, 0, st>>>(src, lds, dst, ldd, perm, n, scatter);
  check_launch("permute_rows");
}
#define PR(TS, TD) \
  template void permute_rows<TS, TD>(const TS*, long long, TD*, long long, const int*, int, int, int, cudaStream_t);
PR(double, double) PR(float, float) PR(double, float) PR(float, double)
#undef PR

template <class T>
void axpby(int n, int ncols, double a, const T* x, long long ldx, double b, T* y, long long ldy, cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return;
  dim3 g(cdiv(n, 256), ncols);
  axpby_kernel<T><<<g, 256, 0, st>>>(n, a, x, ldx, b, y, ldy);
  check_launch("axpby");
}
template void axpby<double>(int, int, double, const double*, long long, double, double*, long long, cudaStream_t);
template void axpby<float>(int, int, double, const float*, long long, double, float*, long long, cudaStream_t);

}  // namespace hodlr

// ---------------------------------------------------------------- leaf triangular solves
namespace hodlr {
namespace {
constexpr int TRSM_WARPS = 8;
template <class TI, class TO>
__global__ void __launch_bounds__(TRSM_WARPS * 32) leaf_trsm_kernel(int nl, const double* Lall, const TI* in,
                                                                     long long ldi, TO* out, long long ldo, int q) {
  extern __shared__ double xs[];   // TRSM_WARPS * nl
  const int b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.y * TRSM_WARPS + warp;
  const double* L = Lall + (size_t)b * nl * nl;
  double* x = xs + (size_t)warp * nl;
  const bool active = j < q;
  if (active)
    for (int i = lane; i < nl; i += 32) x[i] = (double)in[(size_t)b * nl + i + (size_t)j * ldi];
  __syncwarp();
  if (active) {
    // forward: L y = b, column sweeps (L column-major, lower)
    for (int i = 0; i < nl; ++i) {
      double xi = x[i] / L[i + (size_t)i * nl];
      __syncwarp();
      if (lane == 0) x[i] = xi;
      for (int k = i + 1 + lane; k < nl; k += 32) x[k] -= L[k + (size_t)i * nl] * xi;
      __syncwarp();
    }
    // backward: L^T x = y, x_i = (y_i - sum_{k>i} L[k,i] x_k) / L[i,i]
    for (int i = nl - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1 + lane; k < nl; k += 32) s += L[k + (size_t)i * nl] * x[k];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      s = __shfl_sync(0xffffffffu, s, 0);
      double xi = (x[i] - s) / L[i + (size_t)i * nl];
      __syncwarp();
      if (lane == 0) x[i] = xi;
      __syncwarp();
    }
    for (int i = lane; i < nl; i += 32) out[(size_t)b * nl + i + (size_t)j * ldo] = (TO)x[i];
  }
}
}  // namespace

template <class TI, class TO>
void leaf_trsm(int nleaves, int nl, const double* L, const TI* in, long long ldi, TO* out, long long ldo, int q,
               cudaStream_t st) {
  if (nleaves <= 0 || q <= 0) return;
  dim3 g(nleaves, cdiv(q, TRSM_WARPS));
  size_t sm = (size_t)TRSM_WARPS * nl * sizeof(double);
  if (sm > 48 * 1024)
    HODLR_CUDA(cudaFuncSetAttribute(leaf_trsm_kernel<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  leaf_trsm_kernel<TI, TO><<<g, TRSM_WARPS * 32, sm, st>>>(nl, L, in, ldi, out, ldo, q);
  check_launch("leaf_trsm");
}
template void leaf_trsm<double, double>(int, int, const double*, const double*, long long, double*, long long, int,
                                        cudaStream_t);
template void leaf_trsm<float, float>(int, int, const double*, const float*, long long, float*, long long, int,
                                      cudaStream_t);
template void leaf_trsm<float, double>(int, int, const double*, const float*, long long, double*, long long, int,
                                       cudaStream_t);
template void leaf_trsm<double, float>(int, int, const double*, const double*, long long, float*, long long, int,
                                       cudaStream_t);
}  // namespace hodlr
