// Physics products of the covariance model (Sec. 2.1, eq. cov model): probes, the Matern
// latent covariance by FFT circulant embedding, and the Helmholtz solves A^{-1}.
//
//   probe_panel     Philox4x32-10 Gaussian probes, patterned per level (Alg. 1 step 1,
//                   Sec. 3.2.2), drawn directly in tree order.
//   fft_convolve    exact Toeplitz / block-Toeplitz products K_u X: zero-padded radix-2
//                   FFTs in shared memory (decimation in frequency forward, in time inverse,
//                   so the spectrum stays in bit-reversed order and no permutation pass is
//                   needed); two real columns ride in one complex line because the
//                   embedding spectrum is real; 1-D lengths above 4096 use the four-step
//                   split L = L1 * L2; 2-D uses row / column passes.
//   solve_A         A = -Laplacian_h + kappa^2 (Dirichlet): 1-D by the Thomas recurrences
//                   evaluated as parallel affine scans; 2-D by an orthonormal DST-I along x
//                   (a dense G x G product) and Thomas recurrences along y per x-mode.
#include <math.h>

#include "common.cuh"
#include "ops.h"

namespace hodlr {
namespace {

template <class T> struct CT;
template <> struct CT<float> { using C = float2; };
template <> struct CT<double> { using C = double2; };

// Double-float arithmetic for the FFT passes of FP64 fields on the mixed BF16 path: a value is an
// unevaluated sum hi + lo of two FP32 numbers (about 48 significant bits).  Sums use the
// two-sum error-free transformation, products the FMA-based two-product; both renormalise.
// GB300 runs FP32 operations at about seventy times its FP64 rate, so the butterflies are cheaper
// this way although each takes several FP32 operations.  Values enter from and leave to FP64
// storage (the passes exchange FP64 data through global memory).
struct dfl {
  float hi, lo;
  __device__ __forceinline__ dfl() {}
  __device__ __forceinline__ dfl(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ dfl(double d) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
  }
  __device__ __forceinline__ operator double() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ dfl df_renorm(float s, float e) {
  const float h = s + e;
  return dfl(h, e - (h - s));
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const float s = a.hi + b.hi, bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb) + (a.lo + b.lo);
  return df_renorm(s, e);
}
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + dfl(-b.hi, -b.lo); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return df_renorm(p, e);
}
__device__ __forceinline__ dfl operator*(dfl a, double b) { return a * dfl(b); }
struct dcx {
  dfl x, y;
  __device__ __forceinline__ dcx() {}
  __device__ __forceinline__ dcx(dfl a, dfl b) : x(a), y(b) {}
  __device__ __forceinline__ dcx(double2 v) : x(v.x), y(v.y) {}
  __device__ __forceinline__ operator double2() const { return make_double2((double)x, (double)y); }
};
struct DFA {};   // arithmetic tag: FP64 storage, double-float arithmetic
template <> struct CT<DFA> { using C = dcx; };

template <class C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class C> __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

// ------------------------------------------------------------------ Philox probes
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

template <class T>
__global__ void probe_kernel(int N, int level, int stream_id, uint32_t k0, uint32_t k1,
                             const unsigned char* mask, const int* rowid, T* out, long long ld) {
  const int j = blockIdx.y;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  T z = T(0);
  if (mask[i]) {
    // the counter is the row's position in the cluster tree (without padding rows)
    const uint32_t row = rowid ? (uint32_t)rowid[i] : (uint32_t)i;
    uint32_t c[4] = {row, (uint32_t)j, (uint32_t)level, (uint32_t)stream_id};
    philox4x32_10(c, k0, k1);
    if constexpr (sizeof(T) == 8) {
      double u1 = ((double)(c[0] >> 5) * 67108864.0 + (double)(c[1] >> 6) + 1.0) * 0x1p-53;
      double u2 = ((double)(c[2] >> 5) * 67108864.0 + (double)(c[3] >> 6)) * 0x1p-53;
      z = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    } else {
      // the same 53-bit uniforms rounded to FP32 (relative 2^-24, also in the tail), FP32 math
      float u1 = fmaf((float)(c[0] >> 5), 0x1p-27f, (float)((c[1] >> 6) + 1u) * 0x1p-53f);
      float u2 = fmaf((float)(c[2] >> 5), 0x1p-27f, (float)(c[3] >> 6) * 0x1p-53f);
      z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    }
  }
  out[i + (size_t)j * ld] = z;
}

// ------------------------------------------------------------------ FFT building blocks
// x[k * nl + v], k < L: nl interleaved lines of length L in shared memory.
// Radix-2 stages (DIF: halves L/2 .. 1, output in bit-reversed order; DIT: halves 1 .. L/2,
// input in bit-reversed order), executed three at a time: a thread holds the 8 elements
// that three consecutive stages combine and applies their butterflies in registers, so the
// shared-memory passes drop from log2 L to about log2 L / 3.  The butterflies and twiddles
// are those of the radix-2 stages, so the results do not depend on the grouping.
template <class C>
__device__ __forceinline__ void dif_bfly(C& a, C& b, C w) {
  C d = csub(a, b);
  a = cadd(a, b);
  b = cmul(d, w);
}
template <class C>
__device__ __forceinline__ void dit_bfly(C& u, C& v, C w) {
  C t = cmulc(v, w);
  v = csub(u, t);
  u = cadd(u, t);
}
// L and nl are powers of two: index arithmetic by shifts and masks.
__device__ __forceinline__ int log2_pow2(int n) { return __ffs(n) - 1; }

template <class C>
__device__ void dif(C* x, int L, int nl, const C* tw) {
  const int lnl = log2_pow2(nl), lL = log2_pow2(L);
  int half = L >> 1;
  for (; half >= 4; half >>= 3) {                    // stages half, half/2, half/4
    const int q4 = half >> 2, lq4 = log2_pow2(q4);
    const int s1 = L / (2 * half), s2 = 2 * s1, s3 = 4 * s1;
    for (int q = threadIdx.x; q < (nl << (lL - 3)); q += blockDim.x) {
      const int v = q & (nl - 1), g = q >> lnl;
      const int t = g & (q4 - 1), blk = g >> lq4;
      const int i = blk * 2 * half + t;
      C e[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) e[j] = x[((i + j * q4) << lnl) + v];
#pragma unroll
      for (int j = 0; j < 4; ++j) dif_bfly(e[j], e[j + 4], tw[(t + j * q4) * s1]);
#pragma unroll
      for (int j = 0; j < 8; j += 4) {
        dif_bfly(e[j], e[j + 2], tw[t * s2]);
        dif_bfly(e[j + 1], e[j + 3], tw[(t + q4) * s2]);
      }
#pragma unroll
      for (int j = 0; j < 8; j += 2) dif_bfly(e[j], e[j + 1], tw[t * s3]);
#pragma unroll
      for (int j = 0; j < 8; ++j) x[((i + j * q4) << lnl) + v] = e[j];
    }
    __syncthreads();
  }
  for (; half >= 1; half >>= 1) {
    const int step = L / (2 * half), lh = log2_pow2(half);
    for (int q = threadIdx.x; q < (nl << (lL - 1)); q += blockDim.x) {
      const int v = q & (nl - 1), bq = q >> lnl;
      const int t = bq & (half - 1), blk = bq >> lh;
      const int i0 = blk * 2 * half + t, i1 = i0 + half;
      C a = x[(i0 << lnl) + v], b = x[(i1 << lnl) + v];
      dif_bfly(a, b, tw[t * step]);
      x[(i0 << lnl) + v] = a;
      x[(i1 << lnl) + v] = b;
    }
    __syncthreads();
  }
}
template <class C>
__device__ void dit(C* x, int L, int nl, const C* tw) {
  const int lnl = log2_pow2(nl), lL = log2_pow2(L);
  int half = 1;
  for (; 8 * half <= L; half <<= 3) {                // stages half, 2 half, 4 half
    const int lh = log2_pow2(half);
    const int s1 = L / (2 * half), s2 = s1 / 2, s3 = s1 / 4;
    for (int q = threadIdx.x; q < (nl << (lL - 3)); q += blockDim.x) {
      const int v = q & (nl - 1), g = q >> lnl;
      const int t = g & (half - 1), blk = g >> lh;
      const int i = blk * 8 * half + t;
      C e[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) e[j] = x[((i + j * half) << lnl) + v];
#pragma unroll
      for (int j = 0; j < 8; j += 2) dit_bfly(e[j], e[j + 1], tw[t * s1]);
#pragma unroll
      for (int j = 0; j < 8; j += 4) {
        dit_bfly(e[j], e[j + 2], tw[t * s2]);
        dit_bfly(e[j + 1], e[j + 3], tw[(t + half) * s2]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) dit_bfly(e[j], e[j + 4], tw[(t + j * half) * s3]);
#pragma unroll
      for (int j = 0; j < 8; ++j) x[((i + j * half) << lnl) + v] = e[j];
    }
    __syncthreads();
  }
  for (; half < L; half <<= 1) {
    const int step = L / (2 * half), lh = log2_pow2(half);
    for (int q = threadIdx.x; q < (nl << (lL - 1)); q += blockDim.x) {
      const int v = q & (nl - 1), bq = q >> lnl;
      const int t = bq & (half - 1), blk = bq >> lh;
      const int i0 = blk * 2 * half + t, i1 = i0 + half;
      C u = x[(i0 << lnl) + v], w = x[(i1 << lnl) + v];
      dit_bfly(u, w, tw[t * step]);
      x[(i0 << lnl) + v] = u;
      x[(i1 << lnl) + v] = w;
    }
    __syncthreads();
  }
}
template <class C, class G>
__device__ void load_tw(C* s, const G* g, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) s[i] = C(g[i]);
  __syncthreads();
}

__device__ __forceinline__ int bitrev(int k, int logn) { return __brev((unsigned)k) >> (32 - logn); }

template <class T>
__device__ __forceinline__ typename CT<T>::C twiddle_L(long long e, int L) {  // exp(-2 pi i e / L)
  T s, c;
  long long m = e % L;
  if constexpr (sizeof(T) == 8) sincospi(-2.0 * (double)m / (double)L, &s, &c);
  else sincospif(-2.0f * (float)m / (float)L, &s, &c);
  return {c, s};
}

// ---------------------------------------------------------------- 1-D, L <= 4096, one line per CTA
// MODE 0: convolution (forward, multiply by lam0 [and lam1], inverse) of a pair of real columns.
// MODE 1: forward transform of a real sequence `in` (length L), lam0 = Re(X) * scale.
template <class T, int MODE, class A = T>
__global__ void fft1_small_kernel(int L, int Ns, int ncols, const T* in, long long ldi, T* lam0,
                                  const T* lam1, T* out0, T* out1, long long ldo, const typename CT<T>::C* twg,
                                  double scale) {
  using C = typename CT<A>::C;
  extern __shared__ unsigned char sm[];
  C* tw = (C*)sm;
  C* x = tw + L / 2;
  C* y = x + L;
  load_tw(tw, twg, L / 2);
  const int f = blockIdx.x;
  const int c0 = 2 * f, c1 = 2 * f + 1;
  if (MODE == 1) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) x[i] = {in[i], T(0)};
  } else {
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
      C v = {T(0), T(0)};
      if (i < Ns) {
        v.x = in[i + (size_t)c0 * ldi];
        if (c1 < ncols) v.y = in[i + (size_t)c1 * ldi];
      }
      x[i] = v;
    }
  }
  __syncthreads();
  dif(x, L, 1, tw);
  if (MODE == 1) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) lam0[i] = (T)(x[i].x * scale);
    return;
  }
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    C v = x[i];
    if (lam1) y[i] = {v.x * lam1[i], v.y * lam1[i]};
    x[i] = {v.x * lam0[i], v.y * lam0[i]};
  }
  __syncthreads();
  dit(x, L, 1, tw);
  for (int i = threadIdx.x; i < Ns; i += blockDim.x) {
    out0[i + (size_t)c0 * ldo] = x[i].x;
    if (c1 < ncols) out0[i + (size_t)c1 * ldo] = x[i].y;
  }
  if (lam1) {
    dit(y, L, 1, tw);
    for (int i = threadIdx.x; i < Ns; i += blockDim.x) {
      out1[i + (size_t)c0 * ldo] = y[i].x;
      if (c1 < ncols) out1[i + (size_t)c1 * ldo] = y[i].y;
    }
  }
}

// ---------------------------------------------------------------- 1-D four-step (L = L1 * L2 > 4096)
// Pass A: for NV consecutive i2 (lines), DIF over i1 (stride L2), then multiply by W_L^{i2*k1}.
//   src: real pair columns (ncols, ld) [MODE 0] or real sequence of length L [MODE 1];
//   dst: complex W[f][k*L2 + i2].
template <class T, int MODE, class A = T>
__global__ void fft1_passA_kernel(int L1, int L2, int logL1, int Ns, int ncols, const T* in, long long ldi,
                                  typename CT<T>::C* W, const typename CT<T>::C* twg, int nv) {
  using C = typename CT<A>::C;
  extern __shared__ unsigned char sm[];
  C* tw = (C*)sm;
  C* x = tw + L1 / 2;
  const int L = L1 * L2;
  load_tw(tw, twg, L1 / 2);
  const int f = blockIdx.y;
  const int i2b = blockIdx.x * nv;
  const int c0 = 2 * f, c1 = 2 * f + 1;
  for (int e = threadIdx.x; e < L1 * nv; e += blockDim.x) {
    int v = e % nv, k = e / nv;
    long long i = (long long)k * L2 + i2b + v;
    C val = {T(0), T(0)};
    if (MODE == 1) val.x = in[i];
    else if (i < Ns) {
      val.x = in[i + (size_t)c0 * ldi];
      if (c1 < ncols) val.y = in[i + (size_t)c1 * ldi];
    }
    x[k * nv + v] = val;
  }
  __syncthreads();
  dif(x, L1, nv, tw);
  typename CT<T>::C* Wf = W + (size_t)f * L;
  for (int e = threadIdx.x; e < L1 * nv; e += blockDim.x) {
    int v = e % nv, k = e / nv;
    int i2 = i2b + v;
    long long k1 = bitrev(k, logL1);
    Wf[(size_t)k * L2 + i2] = cmul(x[k * nv + v], C(twiddle_L<T>(k1 * i2, L)));
  }
}
// Pass B: per line k (contiguous L2): MODE 0: DIF, multiply lam0 [lam1], DIT (in place to W / W2);
// MODE 1: DIF only, lam0 = Re * scale.
template <class T, int MODE, class A = T>
__global__ void fft1_passB_kernel(int L1, int L2, typename CT<T>::C* W, typename CT<T>::C* W2, T* lam0,
                                  const T* lam1, const typename CT<T>::C* twg, double scale) {
  using C = typename CT<A>::C;
  extern __shared__ unsigned char sm[];
  C* tw = (C*)sm;
  C* x = tw + L2 / 2;
  C* y = x + L2;
  load_tw(tw, twg, L2 / 2);
  const int k = blockIdx.x, f = blockIdx.y;
  const int L = L1 * L2;
  typename CT<T>::C* line = W + (size_t)f * L + (size_t)k * L2;
  for (int i = threadIdx.x; i < L2; i += blockDim.x) x[i] = line[i];
  __syncthreads();
  dif(x, L2, 1, tw);
  const size_t base = (size_t)k * L2;
  if (MODE == 1) {
    for (int i = threadIdx.x; i < L2; i += blockDim.x) lam0[base + i] = (T)(x[i].x * scale);
    return;
  }
  for (int i = threadIdx.x; i < L2; i += blockDim.x) {
    C v = x[i];
    if (lam1) y[i] = {v.x * lam1[base + i], v.y * lam1[base + i]};
    x[i] = {v.x * lam0[base + i], v.y * lam0[base + i]};
  }
  __syncthreads();
  dit(x, L2, 1, tw);
  for (int i = threadIdx.x; i < L2; i += blockDim.x) line[i] = x[i];
  if (lam1) {
    dit(y, L2, 1, tw);
    typename CT<T>::C* line2 = W2 + (size_t)f * L + (size_t)k * L2;
    for (int i = threadIdx.x; i < L2; i += blockDim.x) line2[i] = y[i];
  }
}
// Pass C: multiply by conj W_L^{i2*k1}, DIT over i1, write real pair columns (i < Ns).
template <class T, class A = T>
__global__ void fft1_passC_kernel(int L1, int L2, int logL1, int Ns, int ncols, const typename CT<T>::C* W,
                                  T* out, long long ldo, const typename CT<T>::C* twg, int nv) {
  using C = typename CT<A>::C;
  extern __shared__ unsigned char sm[];
  C* tw = (C*)sm;
  C* x = tw + L1 / 2;
  const int L = L1 * L2;
  load_tw(tw, twg, L1 / 2);
  const int f = blockIdx.y;
  const int i2b = blockIdx.x * nv;
  const int c0 = 2 * f, c1 = 2 * f + 1;
  const typename CT<T>::C* Wf = W + (size_t)f * L;
  for (int e = threadIdx.x; e < L1 * nv; e += blockDim.x) {
    int v = e % nv, k = e / nv;
    int i2 = i2b + v;
    long long k1 = bitrev(k, logL1);
    x[k * nv + v] = cmulc(Wf[(size_t)k * L2 + i2], twiddle_L<T>(k1 * i2, L));
  }
  __syncthreads();
  dit(x, L1, nv, tw);
  for (int e = threadIdx.x; e < L1 * nv; e += blockDim.x) {
    int v = e % nv, k = e / nv;
    long long i = (long long)k * L2 + i2b + v;
    if (i < Ns) {
      out[i + (size_t)c0 * ldo] = x[k * nv + v].x;
      if (c1 < ncols) out[i + (size_t)c1 * ldo] = x[k * nv + v].y;
    }
  }
}

// ---------------------------------------------------------------- 2-D (L x L embedding of a G x G grid)
// Row pass forward: line = row y of field f; input real pair columns (natural p = y*G + x), or the
// L x L real embedding (MODE 1, all L rows).  Output W[f][y][k] (rows y < nrows).
template <class T, int MODE, class A = T>
__global__ void fft2_rows_fwd_kernel(int L, int G, int ncols, const T* in, long long ldi, typename CT<T>::C* W,
                                     const typename CT<T>::C* twg) {
  using C = typename CT<A>::C;
  extern __shared__ unsigned char sm[];
  C* tw = (C*)sm;
  C* x = tw + L / 2;
  load_tw(tw, twg, L / 2);
  const int y = blockIdx.x, f = blockIdx.y;
  const int c0 = 2 * f, c1 = 2 * f + 1;
  const int nrows = (MODE == 1) ? L : G;
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    C v = {T(0), T(0)};
    if (MODE == 1) v.x = in[(size_t)y * L + i];
    else if (i < G) {
      size_t p = (size_t)y * G + i;
      v.x = in[p + (size_t)c0 * ldi];
      if (c1 < ncols) v.y = in[p + (size_t)c1 * ldi];
    }
    x[i] = v;
  }
  __syncthreads();
  dif(x, L, 1, tw);
  typename CT<T>::C* row = W + ((size_t)f * nrows + y) * L;
  for (int i = threadIdx.x; i < L; i += blockDim.x) row[i] = x[i];
}
// Column pass: NV adjacent columns k of field f; rows y < nin loaded (rest zero).
// MODE 0: DIF, multiply by lam0 [lam1], DIT, store rows y < G into W [W2].
// MODE 1: DIF only, lam0[ky*L + k] = Re * scale (spectrum).
template <class T, int MODE, class A = T>
__global__ void fft2_cols_kernel(int L, int nin, typename CT<T>::C* W, typename CT<T>::C* W2, T* lam0,
                                 const T* lam1, const typename CT<T>::C* twg, int nv, double scale, int nout) {
  using C = typename CT<A>::C;
  extern __shared__ unsigned char sm[];
  C* tw = (C*)sm;
  C* x = tw + L / 2;
  C* y = x + (size_t)L * nv;
  load_tw(tw, twg, L / 2);
  const int kb = blockIdx.x * nv, f = blockIdx.y;
  typename CT<T>::C* Wf = W + (size_t)f * nin * L;
  for (int e = threadIdx.x; e < L * nv; e += blockDim.x) {
    int v = e % nv, r = e / nv;
    C val = {T(0), T(0)};
    if (r < nin) val = Wf[(size_t)r * L + kb + v];
    x[r * nv + v] = val;
  }
  __syncthreads();
  dif(x, L, nv, tw);
  if (MODE == 1) {
    for (int e = threadIdx.x; e < L * nv; e += blockDim.x) {
      int v = e % nv, r = e / nv;
      lam0[(size_t)r * L + kb + v] = (T)(x[r * nv + v].x * scale);
    }
    return;
  }
  for (int e = threadIdx.x; e < L * nv; e += blockDim.x) {
    int v = e % nv, r = e / nv;
    size_t li = (size_t)r * L + kb + v;
    C val = x[e];
    if (lam1) y[e] = {val.x * lam1[li], val.y * lam1[li]};
    x[e] = {val.x * lam0[li], val.y * lam0[li]};
  }
  __syncthreads();
  dit(x, L, nv, tw);
  for (int e = threadIdx.x; e < nout * nv; e += blockDim.x) {
    int v = e % nv, r = e / nv;
    Wf[(size_t)r * L + kb + v] = x[r * nv + v];
  }
  if (lam1) {
    dit(y, L, nv, tw);
    typename CT<T>::C* W2f = W2 + (size_t)f * nin * L;
    for (int e = threadIdx.x; e < nout * nv; e += blockDim.x) {
      int v = e % nv, r = e / nv;
      W2f[(size_t)r * L + kb + v] = y[r * nv + v];
    }
  }
}
// Row pass inverse: DIT along x for rows y < G, write x < G into real pair columns.
template <class T, class A = T>
__global__ void fft2_rows_inv_kernel(int L, int G, int ncols, const typename CT<T>::C* W, T* out, long long ldo,
                                     const typename CT<T>::C* twg) {
  using C = typename CT<A>::C;
  extern __shared__ unsigned char sm[];
  C* tw = (C*)sm;
  C* x = tw + L / 2;
  load_tw(tw, twg, L / 2);
  const int y = blockIdx.x, f = blockIdx.y;
  const int c0 = 2 * f, c1 = 2 * f + 1;
  const typename CT<T>::C* row = W + ((size_t)f * G + y) * L;
  for (int i = threadIdx.x; i < L; i += blockDim.x) x[i] = row[i];
  __syncthreads();
  dit(x, L, 1, tw);
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    size_t p = (size_t)y * G + i;
    out[p + (size_t)c0 * ldo] = x[i].x;
    if (c1 < ncols) out[p + (size_t)c1 * ldo] = x[i].y;
  }
}

// ---------------------------------------------------------------- Matern embedding values
__device__ double matern_val(double r, double ell, double nu, int deriv) {
  double z = r / ell;
  double e = exp(-z);
  if (nu < 1.0) return deriv ? (z / ell) * e : e;
  return deriv ? (z * z / ell) * e : (1.0 + z) * e;
}
template <class T>
__global__ void embedding_kernel(int dim, int G, int L, double h, double nu, double sigma2, double ell,
                                 int deriv, T* e) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long n = dim == 1 ? L : (long long)L * L;
  if (idx >= n) return;
  int kx = (int)(idx % L), ky = dim == 1 ? 0 : (int)(idx / L);
  int dx = min(kx, L - kx), dy = min(ky, L - ky);
  double v = 0.0;
  if (dx <= G - 1 && dy <= G - 1) {
    double r = h * sqrt((double)dx * dx + (double)dy * dy);
    v = sigma2 * matern_val(r, ell, nu, deriv);
  }
  e[idx] = (T)v;
}

template <class T>
__global__ void twiddle_kernel(int L, typename CT<T>::C* tw) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L / 2) return;
  double s, c;
  sincospi(-2.0 * (double)k / (double)L, &s, &c);
  tw[k] = {(T)c, (T)s};
}

// ---------------------------------------------------------------- A^{-1}
// Thomas recurrences of T' = tridiag(-1, 2 + m, -1) with constant shift m:
//   u_i = sinh((i+1) mu) / sinh(i mu), cosh mu = 1 + m/2  (i = 1..G)
//   forward  y_p = x_p + a_p y_{p-1},  a_p = 1/u_p (a_0 = 0)      [p = i-1, 0-based]
//   backward z_p = b_p (y_p + z_{p+1}), b_p = 1/u_{p+1}
// Evaluated stably as u_i = e^mu * expm1(-2 (i+1) mu) / expm1(-2 i mu), mu = 2 asinh(sqrt(m)/2).
__device__ void thomas_coef(int G, double m, int p, double* a, double* b) {
  double mu = 2.0 * asinh(0.5 * sqrt(m));
  auto u = [&](int i) { return exp(mu) * expm1(-2.0 * (i + 1) * mu) / expm1(-2.0 * i * mu); };
  *a = p == 0 ? 0.0 : 1.0 / u(p);
  *b = 1.0 / u(p + 1);
}
__global__ void tables_1d_kernel(int G, double m, double* coef) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G) return;
  double a, b;
  thomas_coef(G, m, p, &a, &b);
  coef[p] = a;
  coef[G + p] = b;
}
__global__ void tables_2d_kernel(int G, double kh2, double* coef) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)G * G) return;
  int k = (int)(idx % G), p = (int)(idx / G);          // x-mode k (fast), position p along y
  double s = sinpi((double)(k + 1) / (2.0 * (G + 1)));
  double m = 4.0 * s * s + kh2;                          // lambda_k + kappa^2 h^2
  double a, b;
  thomas_coef(G, m, p, &a, &b);
  coef[idx] = a;                                         // [p][k]
  coef[(size_t)G * G + idx] = b;
}

// 1-D: one CTA per column, tiles of NT*EPT elements, affine scans across the CTA.
struct Aff { double a, b; };  // t -> a t + b
__device__ __forceinline__ Aff compose(Aff f, Aff g) { return {g.a * f.a, g.a * f.b + g.b}; }  // g after f

constexpr int TS_NT = 512, TS_EPT = 4;

__device__ Aff cta_exclusive_scan(Aff v, Aff* sh, Aff* total) {
  // inclusive warp scan (in thread order)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Aff inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    Aff prev;
    prev.a = __shfl_up_sync(0xffffffffu, inc.a, o);
    prev.b = __shfl_up_sync(0xffffffffu, inc.b, o);
    if (lane >= o) inc = compose(prev, inc);
  }
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    Aff run = {1.0, 0.0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      Aff t = sh[w];
      sh[w] = run;
      run = compose(run, t);
    }
    *total = run;
  }
  __syncthreads();
  Aff wpre = sh[wid];
  Aff ex;
  ex.a = __shfl_up_sync(0xffffffffu, inc.a, 1);
  ex.b = __shfl_up_sync(0xffffffffu, inc.b, 1);
  if (lane == 0) ex = {1.0, 0.0};
  Aff res = compose(wpre, ex);
  __syncthreads();
  return res;
}

template <class T>
__global__ void __launch_bounds__(TS_NT) tridiag_1d_kernel(int G, const T* in, long long ldi, T* out,
                                                           long long ldo, const double* coef, double scale) {
  __shared__ Aff sh[32];
  __shared__ Aff tot;
  __shared__ double carry;
  const int j = blockIdx.x;
  const T* x = in + (size_t)j * ldi;
  T* y = out + (size_t)j * ldo;
  const double* ca = coef;
  const double* cb = coef + G;
  const int tile = TS_NT * TS_EPT;
  if (threadIdx.x == 0) carry = 0.0;
  __syncthreads();
  // forward sweep: y_p = a_p y_{p-1} + x_p
  for (int t0 = 0; t0 < G; t0 += tile) {
    int p0 = t0 + threadIdx.x * TS_EPT;
    double xv[TS_EPT];
    Aff f = {1.0, 0.0};
#pragma unroll
    for (int e = 0; e < TS_EPT; ++e) {
      int p = p0 + e;
      xv[e] = p < G ? (double)x[p] : 0.0;
      Aff g = p < G ? Aff{ca[p], xv[e]} : Aff{1.0, 0.0};
      f = compose(f, g);
    }
    Aff pre = cta_exclusive_scan(f, sh, &tot);
    double yin = pre.a * carry + pre.b;
#pragma unroll
    for (int e = 0; e < TS_EPT; ++e) {
      int p = p0 + e;
      if (p < G) {
        yin = ca[p] * yin + xv[e];
        y[p] = (T)yin;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry = tot.a * carry + tot.b;
    __syncthreads();
  }
  // backward sweep: z_p = b_p z_{p+1} + b_p y_p, threads in reverse order
  if (threadIdx.x == 0) carry = 0.0;
  __syncthreads();
  for (int t0 = 0; t0 < G; t0 += tile) {
    // reverse index r = G-1-q
    int q0 = t0 + threadIdx.x * TS_EPT;
    double yv[TS_EPT];
    Aff f = {1.0, 0.0};
#pragma unroll
    for (int e = 0; e < TS_EPT; ++e) {
      int q = q0 + e, p = G - 1 - q;
      yv[e] = q < G ? (double)y[p] : 0.0;
      Aff g = q < G ? Aff{cb[p], cb[p] * yv[e]} : Aff{1.0, 0.0};
      f = compose(f, g);
    }
    Aff pre = cta_exclusive_scan(f, sh, &tot);
    double zin = pre.a * carry + pre.b;
    __syncthreads();   // all reads of y for this tile done before any write
#pragma unroll
    for (int e = 0; e < TS_EPT; ++e) {
      int q = q0 + e, p = G - 1 - q;
      if (q < G) {
        zin = cb[p] * zin + cb[p] * yv[e];
        y[p] = (T)(zin);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry = tot.a * carry + tot.b;
    __syncthreads();
  }
  // scale (h^2) in place
  for (int p = threadIdx.x; p < G; p += blockDim.x) y[p] = (T)((double)y[p] * scale);
}

// 2-D: Thomas along y for each (column, x-mode k); data [p=y][k] with k fastest.
template <class T>
__global__ void thomas_y_kernel(int G, int ncols, T* X, long long ld, const double* coef, double scale) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)G * ncols) return;
  int k = (int)(idx % G), j = (int)(idx / G);
  T* x = X + (size_t)j * ld;
  const double* ca = coef;
  const double* cb = coef + (size_t)G * G;
  double yv = 0.0;
  for (int p = 0; p < G; ++p) {
    size_t o = (size_t)p * G + k;
    yv = ca[o] * yv + (double)x[o];
    x[o] = (T)yv;
  }
  double z = 0.0;
  for (int p = G - 1; p >= 0; --p) {
    size_t o = (size_t)p * G + k;
    z = cb[o] * (z + (double)x[o]);
    x[o] = (T)(z * scale);
  }
}

// Tiled form of the same recurrences: a CTA holds KL x-modes of one column; its NT/KL
// thread groups each take a chunk of consecutive y positions.  Every chunk is first
// solved from a zero start while the chunk's affine map (product of the coefficients,
// end value) is recorded; the maps of the preceding chunks then give the carry-in, and a
// fix-up pass adds (running product) x carry.  The intermediate field stays in shared
// memory, so each element is read and written once in HBM.  R is the arithmetic type: FP64
// for FP64 fields, FP32 (with FP32 coefficient tables) for FP32 fields, whose FP64
// arithmetic would run at a small fraction of the FP32 rate.
constexpr int TY_NT = 256;
template <class T, class R>
__global__ void __launch_bounds__(TY_NT) thomas_y_tiled_kernel(int G, int KL, T* X, long long ld, const R* coef,
                                                              double scale_d) {
  extern __shared__ __align__(16) unsigned char ty_smem[];
  const int NW = TY_NT / KL;
  const int kl = threadIdx.x % KL, w = threadIdx.x / KL;
  const int k = blockIdx.x * KL + kl;
  const bool act = k < G;
  const int Lc = (G + NW - 1) / NW;
  const int p0 = min(G, w * Lc), p1 = min(G, p0 + Lc);
  R* sA = (R*)ty_smem;                       // [NW][KL] chunk coefficient products
  R* sY = sA + TY_NT;                        // [NW][KL] chunk end values
  T* tile = (T*)(sY + TY_NT);                // [G][KL]
  T* x = X + (size_t)blockIdx.y * ld;
  const R* ca = coef;
  const R* cb = coef + (size_t)G * G;
  const R scale = (R)scale_d;
  // forward: y_p = a_p y_{p-1} + x_p
  R y = R(0), A = R(1);
  if (act) {
#pragma unroll 4
    for (int p = p0; p < p1; ++p) {
      const size_t o = (size_t)p * G + k;
      const R a = ca[o];
      y = a * y + (R)x[o];
      A *= a;
      tile[p * KL + kl] = (T)y;
    }
  }
  sA[threadIdx.x] = A;
  sY[threadIdx.x] = y;
  __syncthreads();
  R yin = R(0);
  for (int u = 0; u < w; ++u) yin = sA[u * KL + kl] * yin + sY[u * KL + kl];
  if (act && yin != R(0)) {
    R P = R(1);
    for (int p = p0; p < p1; ++p) {
      P *= ca[(size_t)p * G + k];
      tile[p * KL + kl] = (T)((R)tile[p * KL + kl] + P * yin);
    }
  }
  __syncthreads();
  // backward: z_p = b_p (z_{p+1} + y_p)
  R z = R(0), B = R(1);
  if (act) {
#pragma unroll 4
    for (int p = p1 - 1; p >= p0; --p) {
      const R b = cb[(size_t)p * G + k];
      z = b * (z + (R)tile[p * KL + kl]);
      B *= b;
      tile[p * KL + kl] = (T)z;
    }
  }
  sA[threadIdx.x] = B;
  sY[threadIdx.x] = z;
  __syncthreads();
  R zin = R(0);
  for (int u = NW - 1; u > w; --u) zin = sA[u * KL + kl] * zin + sY[u * KL + kl];
  if (act) {
    R Q = R(1);
    for (int p = p1 - 1; p >= p0; --p) {
      const size_t o = (size_t)p * G + k;
      Q *= cb[o];
      x[o] = (T)(((R)tile[p * KL + kl] + Q * zin) * scale);
    }
  }
}

template <class T>
__global__ void dst_matrix_kernel(int G, T* S) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)G * G) return;
  int i = (int)(idx % G), j = (int)(idx / G);
  long long m = ((long long)(i + 1) * (j + 1)) % (2LL * (G + 1));
  S[idx] = (T)(sqrt(2.0 / (G + 1)) * sinpi((double)m / (double)(G + 1)));
}

template <class T> size_t csize() { return sizeof(typename CT<T>::C); }

template <class K>
void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) HODLR_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

}  // namespace

// ================================================================== launchers
template <class T>
void probe_panel(int N, int ncols, int level, int stream_id, uint64_t seed, const unsigned char* mask,
                 const int* rowid, T* out, long long ld, cudaStream_t st) {
  if (N <= 0 || ncols <= 0) return;
  dim3 g(cdiv(N, 256), ncols);
  probe_kernel<T><<<g, 256, 0, st>>>(N, level, stream_id, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                     mask, rowid, out, ld);
  check_launch("probe_panel");
}
template void probe_panel<double>(int, int, int, int, uint64_t, const unsigned char*, const int*, double*, long long,
                                  cudaStream_t);
template void probe_panel<float>(int, int, int, int, uint64_t, const unsigned char*, const int*, float*, long long,
                                 cudaStream_t);

template <class T> void twiddles(int L, T* tw, cudaStream_t st) {
  twiddle_kernel<T><<<cdiv(std::max(L / 2, 1), 256), 256, 0, st>>>(L, (typename CT<T>::C*)tw);
  check_launch("twiddles");
}
template void twiddles<double>(int, double*, cudaStream_t);
template void twiddles<float>(int, float*, cudaStream_t);

size_t fft_work_bytes(const PhysicsDesc& p, int ncols, int real_bytes) {
  size_t nf = (size_t)(ncols + 1) / 2;
  size_t per = p.dim == 1 ? (size_t)p.L : (size_t)p.L * p.L;   // also covers the spectrum pass (L x L)
  return 2 * nf * per * 2 * real_bytes;                           // W and W2
}

// twiddle tables: tw (length L/2) for the transform length of each pass; for the four-step
// case tw holds L1/2 entries followed by L2/2 entries.
template <class T>
void matern_spectra(const PhysicsDesc& p, double sigma2, double ell, T* lam0, T* lam1, void* work, const T* tw,
                    cudaStream_t st) {
  using C = typename CT<T>::C;
  const C* twc = (const C*)tw;
  T* emb = (T*)work;
  C* W = (C*)((char*)work + (size_t)(p.dim == 1 ? p.L : (size_t)p.L * p.L) * sizeof(T) + 256);
  for (int d = 0; d < 2; ++d) {
    T* lam = d == 0 ? lam0 : lam1;
    long long n = p.dim == 1 ? p.L : (long long)p.L * p.L;
    embedding_kernel<T><<<cdiv(n, 256), 256, 0, st>>>(p.dim, p.G, p.L, p.h, p.nu, sigma2, ell, d, emb);
    check_launch("embedding");
    if (p.dim == 1 && p.L1 == 0) {
      size_t sm = (p.L / 2 + 2 * p.L) * sizeof(C);
      set_smem(fft1_small_kernel<T, 1>, sm);
      fft1_small_kernel<T, 1><<<1, 256, sm, st>>>(p.L, p.L, 1, emb, p.L, lam, nullptr, nullptr, nullptr, 0, twc,
                                                   1.0 / p.L);
      check_launch("fft1_small spectrum");
    } else if (p.dim == 1) {
      int nv = 16;
      size_t smA = (p.L1 / 2 + (size_t)p.L1 * nv) * sizeof(C);
      set_smem(fft1_passA_kernel<T, 1>, smA);
      fft1_passA_kernel<T, 1><<<dim3(p.L2 / nv, 1), 256, smA, st>>>(p.L1, p.L2, ilog2(p.L1), p.L, 1, emb, p.L, W,
                                                                       twc, nv);
      check_launch("fft1_passA spectrum");
      size_t smB = (p.L2 / 2 + 2 * (size_t)p.L2) * sizeof(C);
      set_smem(fft1_passB_kernel<T, 1>, smB);
      fft1_passB_kernel<T, 1><<<dim3(p.L1, 1), 256, smB, st>>>(p.L1, p.L2, W, nullptr, lam, nullptr,
                                                                 twc + p.L1 / 2, 1.0 / p.L);
      check_launch("fft1_passB spectrum");
    } else {
      size_t smR = (p.L / 2 + (size_t)p.L) * sizeof(C);
      set_smem(fft2_rows_fwd_kernel<T, 1>, smR);
      fft2_rows_fwd_kernel<T, 1><<<dim3(p.L, 1), 256, smR, st>>>(p.L, p.G, 1, emb, 0, W, twc);
      check_launch("fft2_rows spectrum");
      int nv = sizeof(T) == 8 ? 2 : 4;
      size_t smC = (p.L / 2 + 2 * (size_t)p.L * nv) * sizeof(C);
      set_smem(fft2_cols_kernel<T, 1>, smC);
      fft2_cols_kernel<T, 1><<<dim3(p.L / nv, 1), 256, smC, st>>>(p.L, p.L, W, nullptr, lam, nullptr, twc, nv,
                                                                  1.0 / ((double)p.L * p.L), 0);
      check_launch("fft2_cols spectrum");
    }
  }
}
template void matern_spectra<double>(const PhysicsDesc&, double, double, double*, double*, void*, const double*,
                                     cudaStream_t);
template void matern_spectra<float>(const PhysicsDesc&, double, double, float*, float*, void*, const float*,
                                    cudaStream_t);

template <class T, class A>
void fft_convolve_impl(const PhysicsDesc& p, int ncols, const T* in, long long ldi, const T* lam0, const T* lam1, T* out0,
                  T* out1, long long ldo, void* work, const T* tw, cudaStream_t st) {
  using C = typename CT<T>::C;
  if (ncols <= 0) return;
  const C* twc = (const C*)tw;
  const int nf = (ncols + 1) / 2;
  const int Ns = p.dim == 1 ? p.G : p.G * p.G;
  if (p.dim == 1 && p.L1 == 0) {
    size_t sm = (p.L / 2 + 2 * (size_t)p.L) * sizeof(C);
    set_smem(fft1_small_kernel<T, 0, A>, sm);
    fft1_small_kernel<T, 0, A><<<nf, 256, sm, st>>>(p.L, Ns, ncols, in, ldi, (T*)lam0, lam1, out0, out1, ldo, twc, 1.0);
    check_launch("fft1_small");
    return;
  }
  C* W = (C*)work;
  size_t per = p.dim == 1 ? (size_t)p.L : (size_t)p.G * p.L;
  C* W2 = W + (size_t)nf * per;
  if (p.dim == 1) {
    int nv = 16;
    size_t smA = (p.L1 / 2 + (size_t)p.L1 * nv) * sizeof(C);
    set_smem(fft1_passA_kernel<T, 0, A>, smA);
    fft1_passA_kernel<T, 0, A><<<dim3(p.L2 / nv, nf), 256, smA, st>>>(p.L1, p.L2, ilog2(p.L1), Ns, ncols, in, ldi, W,
                                                                    twc, nv);
    check_launch("fft1_passA");
    size_t smB = (p.L2 / 2 + 2 * (size_t)p.L2) * sizeof(C);
    set_smem(fft1_passB_kernel<T, 0, A>, smB);
    fft1_passB_kernel<T, 0, A><<<dim3(p.L1, nf), 256, smB, st>>>(p.L1, p.L2, W, W2, (T*)lam0, lam1, twc + p.L1 / 2, 1.0);
    check_launch("fft1_passB");
    size_t smC = smA;
    set_smem(fft1_passC_kernel<T, A>, smC);
    fft1_passC_kernel<T, A><<<dim3(p.L2 / nv, nf), 256, smC, st>>>(p.L1, p.L2, ilog2(p.L1), Ns, ncols, W, out0, ldo,
                                                                  twc, nv);
    check_launch("fft1_passC");
    if (lam1) {
      fft1_passC_kernel<T, A><<<dim3(p.L2 / nv, nf), 256, smC, st>>>(p.L1, p.L2, ilog2(p.L1), Ns, ncols, W2, out1,
                                                                    ldo, twc, nv);
      check_launch("fft1_passC");
    }
    return;
  }
  size_t smR = (p.L / 2 + (size_t)p.L) * sizeof(C);
  set_smem(fft2_rows_fwd_kernel<T, 0, A>, smR);
  fft2_rows_fwd_kernel<T, 0, A><<<dim3(p.G, nf), 256, smR, st>>>(p.L, p.G, ncols, in, ldi, W, twc);
  check_launch("fft2_rows_fwd");
  int nv = sizeof(T) == 8 ? 2 : 4;
  size_t smC = (p.L / 2 + 2 * (size_t)p.L * nv) * sizeof(C);
  set_smem(fft2_cols_kernel<T, 0, A>, smC);
  fft2_cols_kernel<T, 0, A><<<dim3(p.L / nv, nf), 256, smC, st>>>(p.L, p.G, W, W2, (T*)lam0, lam1, twc, nv, 1.0, p.G);
  check_launch("fft2_cols");
  set_smem(fft2_rows_inv_kernel<T, A>, smR);
  fft2_rows_inv_kernel<T, A><<<dim3(p.G, nf), 256, smR, st>>>(p.L, p.G, ncols, W, out0, ldo, twc);
  check_launch("fft2_rows_inv");
  if (lam1) {
    fft2_rows_inv_kernel<T, A><<<dim3(p.G, nf), 256, smR, st>>>(p.L, p.G, ncols, W2, out1, ldo, twc);
    check_launch("fft2_rows_inv");
  }
}
template <class T>
void fft_convolve(const PhysicsDesc& p, int ncols, const T* in, long long ldi, const T* lam0, const T* lam1, T* out0,
                  T* out1, long long ldo, void* work, const T* tw, cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    if (p.df_fft) {
      fft_convolve_impl<T, DFA>(p, ncols, in, ldi, lam0, lam1, out0, out1, ldo, work, tw, st);
      return;
    }
  }
  fft_convolve_impl<T, T>(p, ncols, in, ldi, lam0, lam1, out0, out1, ldo, work, tw, st);
}
template void fft_convolve<double>(const PhysicsDesc&, int, const double*, long long, const double*, const double*,
                                   double*, double*, long long, void*, const double*, cudaStream_t);
template void fft_convolve<float>(const PhysicsDesc&, int, const float*, long long, const float*, const float*,
                                  float*, float*, long long, void*, const float*, cudaStream_t);

void tridiag_tables(const PhysicsDesc& p, double kappa, double* coef, cudaStream_t st) {
  double kh2 = kappa * kappa * p.h * p.h;
  if (p.dim == 1) {
    tables_1d_kernel<<<cdiv(p.G, 256), 256, 0, st>>>(p.G, kh2, coef);
    check_launch("tables_1d");
  } else {
    tables_2d_kernel<<<cdiv((long long)p.G * p.G, 256), 256, 0, st>>>(p.G, kh2, coef);
    check_launch("tables_2d");
  }
}

template <class T> void dst_matrix(int G, T* S, cudaStream_t st) {
  dst_matrix_kernel<T><<<cdiv((long long)G * G, 256), 256, 0, st>>>(G, S);
  check_launch("dst_matrix");
}
template void dst_matrix<double>(int, double*, cudaStream_t);
template void dst_matrix<float>(int, float*, cudaStream_t);

template <class T>
void solve_A(const PhysicsDesc& p, int ncols, const T* in, long long ldi, T* out, long long ldo, const double* coef,
             const T* S, T* work, Scratch s, cudaStream_t st, int df, const float* coef32, DstSplit tc) {
  if (ncols <= 0) return;
  const double scale = p.h * p.h;
  if (p.dim == 1) {
    tridiag_1d_kernel<T><<<ncols, TS_NT, 0, st>>>(p.G, in, ldi, out, ldo, coef, scale);
    check_launch("tridiag_1d");
    return;
  }
  // 2-D: out = S_x * Thomas_y(S_x * in) with S_x the DST-I along x.  Column-major view of a
  // field: G (x) rows by G (y) columns, so S_x acts from the left on G x (G*ncols).
  const int G = p.G;
  const long long Ns = (long long)G * G;
  if (ldi != Ns || ldo != Ns) throw Error(-1, "solve_A: 2-D panels must have ld = G*G");
  GemmArgs g;
  g.M = G; g.N = G * ncols; g.K = G;
  g.A = S; g.lda = G;
  g.B = in; g.ldb = G;
  g.C = work; g.ldc = G;
  auto dst = [&](const GemmArgs& a) {
    if constexpr (sizeof(T) == 8) {
      if (df && tc.df_S && tc.df_X) {
        df_split((const double*)a.B, tc.df_X, (long long)a.K * a.N, st);   // B is K x N with ld K
        GemmArgs b = a;
        b.A = tc.df_S;
        b.B = tc.df_X;
        gemm_df<float2, float2, double>(b, s, st);
        return;
      }
      if (df) { gemm_df<T, T, T>(a, s, st); return; }
    } else {
      // S is symmetric, so its column-major storage is also its K-major form
      if (tc.hi && tf32x3_gemm(tc.hi, tc.lo, G, (const float*)a.B, a.ldb, (float*)a.C, a.ldc, a.M, a.N, a.K, st))
        return;
    }
    gemm<T, T, T, T>(a, s, st);
  };
  dst(g);
  // x-modes per CTA: the widest group whose tile fits in 96 KB of shared memory
  int KL = 32;
  while (KL > 1 && (size_t)G * KL * sizeof(T) > 96 * 1024) KL >>= 1;
  const size_t tbytes = 2 * TY_NT * sizeof(double) + (size_t)G * KL * sizeof(T);
  if (tbytes <= 200 * 1024 && ncols <= 65535) {
    if (sizeof(T) == 4 && coef32) {
      set_smem(thomas_y_tiled_kernel<T, float>, tbytes);
      thomas_y_tiled_kernel<T, float><<<dim3(cdiv(G, KL), ncols), TY_NT, tbytes, st>>>(G, KL, work, Ns, coef32, scale);
    } else {
      set_smem(thomas_y_tiled_kernel<T, double>, tbytes);
      thomas_y_tiled_kernel<T, double><<<dim3(cdiv(G, KL), ncols), TY_NT, tbytes, st>>>(G, KL, work, Ns, coef, scale);
    }
  } else {
    thomas_y_kernel<T><<<cdiv((long long)G * ncols, 128), 128, 0, st>>>(G, ncols, work, Ns, coef, scale);
  }
  check_launch("thomas_y");
  g.B = work; g.C = out;
  dst(g);
}
template void solve_A<double>(const PhysicsDesc&, int, const double*, long long, double*, long long, const double*,
                              const double*, double*, Scratch, cudaStream_t, int, const float*, DstSplit);
template void solve_A<float>(const PhysicsDesc&, int, const float*, long long, float*, long long, const double*,
                             const float*, float*, Scratch, cudaStream_t, int, const float*, DstSplit);

}  // namespace hodlr
