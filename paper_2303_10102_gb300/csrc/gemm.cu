// Batched column-major GEMM on the SIMT pipes (FP64 DFMA or FP32 FFMA), with
// deterministic split-K for the tall-skinny Gram products of the HODLR level sweeps.
//
// Used for: the peeling products (K - sum_l' H^(l')) R (Sec. 3.2.2), the projections
// B~ = B^T Q, the Gram matrices of the QR step (Alg. 1 step 3), Alg. 2's products, the
// Woodbury sweeps of the factorization (App. C) and the trace products (App. B).
#include "common.cuh"
#include "ops.h"

#include <algorithm>
#include <type_traits>

namespace hodlr {

long long g_kernel_launches = 0;
GemmProfile g_prof;
LaunchTrace g_trace;

namespace {

constexpr int BK = 16, NT = 256;
// Output tile configurations (16 x 16 threads each): square, and two shapes for products with
// a narrow side, so that a block with 16..32 rows (or columns) does not fill a 64-wide tile.
template <int BM_, int BN_, int TM_, int TN_>
struct Tile {
  static constexpr int BM = BM_, BN = BN_, TM = TM_, TN = TN_;
  static_assert((BM / TM) * (BN / TN) == NT, "tile threads");
};
using TileSq = Tile<64, 64, 4, 4>;
using TileNarrowN = Tile<128, 32, 8, 2>;
using TileNarrowM = Tile<32, 128, 2, 8>;

template <class TA, class TB, class TC, class Acc, class TL>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs g, int nsplit, int kchunk, Acc* part) {
  constexpr int BM = TL::BM, BN = TL::BN, TM = TL::TM, TN = TL::TN;
  __shared__ Acc As[BK][BM + 1];
  __shared__ Acc Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % (BM / TM);  // row group
  const int ty = tid / (BM / TM);  // col group
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int b = blockIdx.z / nsplit, s = blockIdx.z % nsplit;
  int bi = b;
  if (g.bmap == BMAP_XOR1) bi = b ^ 1;
  else if (g.bmap == BMAP_SHR1) bi = b >> 1;
  long long aoff = (long long)b * g.sA, boff = (long long)bi * g.sB, coff = (long long)b * g.sC;
  int M = g.M, K = g.K;
  if (g.offmode == 1) {
    int r0 = g.off[b];
    M = g.off[b + 1] - r0; aoff = r0; coff = r0;
  } else if (g.offmode == 2) {
    int r0 = g.off[b];
    K = g.off[b + 1] - r0; aoff = r0; boff = r0;
  }
  const int kb = s * kchunk, ke = min(K, kb + kchunk);
  if (m0 >= M) return;
  const TA* A = (const TA*)g.A + aoff;
  const TB* B = (const TB*)g.B + boff;
  Acc acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = Acc(0);

  // the next tile is fetched into registers while the current one is multiplied
  constexpr int LA = BM * BK / NT, LB = BK * BN / NT;
  Acc ra[LA], rb[LB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + r * NT;
      int i, k;
      if (!g.tA) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      const int gi = m0 + i, gk = k0 + k;
      ra[r] = (gi < M && gk < ke) ? (Acc)(g.tA ? A[gk + (long long)gi * g.lda] : A[gi + (long long)gk * g.lda])
                                  : Acc(0);
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + r * NT;
      int k, j;
      if (!g.tB) { k = e % BK; j = e / BK; } else { j = e % BN; k = e / BN; }
      const int gj = n0 + j, gk = k0 + k;
      rb[r] = (gj < g.N && gk < ke) ? (Acc)(g.tB ? B[gj + (long long)gk * g.ldb] : B[gk + (long long)gj * g.ldb])
                                    : Acc(0);
    }
  };
  if (kb < ke) fetch(kb);
  for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + r * NT;
      int i, k;
      if (!g.tA) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      As[k][i] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + r * NT;
      int k, j;
      if (!g.tB) { k = e % BK; j = e / BK; } else { j = e % BN; k = e / BN; }
      Bs[k][j] = rb[r];
    }
    __syncthreads();
    if (k0 + BK < ke) fetch(k0 + BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      Acc a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[k][tx + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[k][ty + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (nsplit == 1) {
    TC* C = (TC*)g.C + coff;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int gj = n0 + ty + j * (BN / TN);
      if (gj >= g.N) continue;
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        int gi = m0 + tx + i * (BM / TM);
        if (gi >= M) continue;
        long long o = gi + (long long)gj * g.ldc;
        Acc v = (Acc)g.alpha * acc[i][j];
        if (g.beta != 0.0) v += (Acc)g.beta * (Acc)C[o];
        C[o] = (TC)v;
      }
    }
  } else {
    Acc* P = part + ((long long)b * nsplit + s) * (long long)g.M * g.N;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int gj = n0 + ty + j * (BN / TN);
      if (gj >= g.N) continue;
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        int gi = m0 + tx + i * (BM / TM);
        if (gi >= g.M) continue;
        P[gi + (long long)gj * g.M] = acc[i][j];
      }
    }
  }
}

template <class TC, class Acc>
__global__ void splitk_reduce(GemmArgs g, int nsplit, const Acc* part) {
  long long mn = (long long)g.M * g.N;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  if (idx >= mn) return;
  const Acc* P = part + (long long)b * nsplit * mn + idx;
  Acc v = Acc(0);
  for (int s = 0; s < nsplit; ++s) v += P[s * mn];
  int i = (int)(idx % g.M), j = (int)(idx / g.M);
  long long coff = (long long)b * g.sC;
  if (g.offmode == 1) {
    coff = g.off[b];
    if (i >= g.off[b + 1] - g.off[b]) return;
  }
  TC* C = (TC*)g.C + coff;
  long long o = i + (long long)j * g.ldc;
  Acc r = (Acc)g.alpha * v;
  if (g.beta != 0.0) r += (Acc)g.beta * (Acc)C[o];
  C[o] = (TC)r;
}

// Narrow products (N <= 4 right-hand sides, e.g. the HODLR matrix-vector products of the
// score): a full output tile would waste (64 - N)/64 of its arithmetic, which on the FP64
// path is the dominant cost.  tA == 0: one thread per output row, the B columns staged in
// shared memory per K chunk.  tA == 1: each output row is a dot product of a stored column
// with the B columns; `wpc` warps share one row (fixed-order reduction, deterministic).
constexpr int GV_NT = 256, GV_MAXN = 4, GV_KC = 256;

template <class TB, class Acc>
__device__ __forceinline__ Acc gv_b(const GemmArgs& g, const TB* B, int k, int j) {
  return (Acc)(g.tB ? B[j + (long long)k * g.ldb] : B[k + (long long)j * g.ldb]);
}

template <class TA, class TB, class TC, class Acc>
__global__ void __launch_bounds__(GV_NT) gemv_n_kernel(GemmArgs g) {
  __shared__ Acc Bs[GV_KC][GV_MAXN];
  const int b = blockIdx.y;
  int bi = b;
  if (g.bmap == BMAP_XOR1) bi = b ^ 1;
  else if (g.bmap == BMAP_SHR1) bi = b >> 1;
  const TA* A = (const TA*)g.A + (long long)b * g.sA;
  const TB* B = (const TB*)g.B + (long long)bi * g.sB;
  TC* C = (TC*)g.C + (long long)b * g.sC;
  const int i = blockIdx.x * GV_NT + threadIdx.x;
  const int N = g.N;
  Acc acc[GV_MAXN];
#pragma unroll
  for (int j = 0; j < GV_MAXN; ++j) acc[j] = Acc(0);
  for (int k0 = 0; k0 < g.K; k0 += GV_KC) {
    const int kn = min(GV_KC, g.K - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < kn * N; e += GV_NT) {
      int k = e % kn, j = e / kn;
      Bs[k][j] = gv_b<TB, Acc>(g, B, k0 + k, j);
    }
    __syncthreads();
    if (i < g.M) {
      const TA* Ai = A + i + (long long)k0 * g.lda;
#pragma unroll 4
      for (int k = 0; k < kn; ++k) {
        Acc a = (Acc)Ai[(long long)k * g.lda];
#pragma unroll
        for (int j = 0; j < GV_MAXN; ++j)
          if (j < N) acc[j] = fma(a, Bs[k][j], acc[j]);
      }
    }
  }
  if (i >= g.M) return;
#pragma unroll
  for (int j = 0; j < GV_MAXN; ++j) {
    if (j >= N) break;
    long long o = i + (long long)j * g.ldc;
    Acc v = (Acc)g.alpha * acc[j];
    if (g.beta != 0.0) v += (Acc)g.beta * (Acc)C[o];
    C[o] = (TC)v;
  }
}

template <class TA, class TB, class TC, class Acc>
__global__ void __launch_bounds__(GV_NT) gemv_t_kernel(GemmArgs g, int wpc) {
  __shared__ Acc red[GV_NT / 32][GV_MAXN];
  const int b = blockIdx.y;
  int bi = b;
  if (g.bmap == BMAP_XOR1) bi = b ^ 1;
  else if (g.bmap == BMAP_SHR1) bi = b >> 1;
  const TA* A = (const TA*)g.A + (long long)b * g.sA;
  const TB* B = (const TB*)g.B + (long long)bi * g.sB;
  TC* C = (TC*)g.C + (long long)b * g.sC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows_per_cta = (GV_NT / 32) / wpc;
  const int i = blockIdx.x * rows_per_cta + warp / wpc;
  const int part = warp % wpc, nthr = 32 * wpc;
  const int N = g.N;
  Acc acc[GV_MAXN];
#pragma unroll
  for (int j = 0; j < GV_MAXN; ++j) acc[j] = Acc(0);
  if (i < g.M) {
    const TA* Ai = A + (long long)i * g.lda;
#pragma unroll 4
    for (int k = part * 32 + lane; k < g.K; k += nthr) {
      Acc a = (Acc)Ai[k];
#pragma unroll
      for (int j = 0; j < GV_MAXN; ++j)
        if (j < N) acc[j] = fma(a, gv_b<TB, Acc>(g, B, k, j), acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < GV_MAXN; ++j) {
    Acc v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (lane != 0 || part != 0 || i >= g.M) return;
  for (int j = 0; j < N; ++j) {
    Acc v = Acc(0);
    for (int p = 0; p < wpc; ++p) v += red[warp + p][j];
    long long o = i + (long long)j * g.ldc;
    Acc r = (Acc)g.alpha * v;
    if (g.beta != 0.0) r += (Acc)g.beta * (Acc)C[o];
    C[o] = (TC)r;
  }
}

template <class TA, class TB, class TC, class Acc>
bool gemv_narrow(const GemmArgs& g, cudaStream_t st) {
  if (g.N > GV_MAXN || g.offmode != 0 || g.batch > 65535) return false;
  const bool prof = g_prof.on && g_prof.n < g_prof.cap;
  if (prof) cudaEventRecord(g_prof.ev[2 * g_prof.n], st);
  if (!g.tA) {
    dim3 grid(cdiv(g.M, GV_NT), g.batch);
    gemv_n_kernel<TA, TB, TC, Acc><<<grid, GV_NT, 0, st>>>(g);
    check_launch("gemv_n_kernel");
  } else {
    int wpc = 1;
    while (wpc < GV_NT / 32 && (long long)wpc * 32 * 64 < g.K) wpc *= 2;
    const int rows_per_cta = (GV_NT / 32) / wpc;
    dim3 grid(cdiv(g.M, rows_per_cta), g.batch);
    gemv_t_kernel<TA, TB, TC, Acc><<<grid, GV_NT, 0, st>>>(g, wpc);
    check_launch("gemv_t_kernel");
  }
  if (prof) {
    cudaEventRecord(g_prof.ev[2 * g_prof.n + 1], st);
    if (g_prof.shape) {
      int* sh = g_prof.shape + 7 * g_prof.n;
      sh[0] = g.M; sh[1] = g.N; sh[2] = g.K; sh[3] = g.batch; sh[4] = g.tA; sh[5] = g.tB; sh[6] = 3;
    }
    ++g_prof.n;
    g_prof.flops += 2.0 * (double)g.M * g.N * g.K * g.batch;
    prof_add_bytes(3, ((double)g.M * g.K * sizeof(TA) + (double)g.K * g.N * sizeof(TB) +
                     (double)g.M * g.N * sizeof(TC) * (g.beta != 0.0 ? 2 : 1)) * g.batch);
  }
  return true;
}

}  // namespace

bool sgemm_large(const GemmArgs& g, cudaStream_t st);

template <class TA, class TB, class TC, class Acc, class TL>
void gemm_tiles(const GemmArgs& g, Scratch s, cudaStream_t st) {
  constexpr int BM = TL::BM, BN = TL::BN;
  int tiles = cdiv(g.M, BM) * cdiv(g.N, BN) * g.batch;
  int nsplit = 1;
  if (g.K >= 512 && tiles < 4 * 152) {
    nsplit = (8 * 152 + tiles - 1) / tiles;
    nsplit = std::min(nsplit, cdiv(g.K, 128));
    size_t per = (size_t)g.batch * g.M * g.N * sizeof(Acc);
    if (per > 0) nsplit = (int)std::min<size_t>(nsplit, s.bytes / per);
    if (nsplit < 2) nsplit = 1;
  }
  int kchunk = g.K;
  if (nsplit > 1) {
    kchunk = ((cdiv(g.K, nsplit) + BK - 1) / BK) * BK;
    nsplit = cdiv(g.K, kchunk);
  }
  if (g.K <= 0) kchunk = 0;
  dim3 grid(cdiv(g.M, BM), cdiv(g.N, BN), g.batch * nsplit);
  if (grid.z > 65535) throw Error(-1, "gemm: batch too large");
  const bool prof = g_prof.on && g_prof.n < g_prof.cap;
  if (prof) cudaEventRecord(g_prof.ev[2 * g_prof.n], st);
  gemm_kernel<TA, TB, TC, Acc, TL><<<grid, NT, 0, st>>>(g, nsplit, kchunk, (Acc*)s.ptr);
  check_launch("gemm_kernel");
  if (prof) {
    cudaEventRecord(g_prof.ev[2 * g_prof.n + 1], st);
    if (g_prof.shape) {
      int* sh = g_prof.shape + 7 * g_prof.n;
      sh[0] = g.M; sh[1] = g.N; sh[2] = g.K; sh[3] = g.batch; sh[4] = g.tA; sh[5] = g.tB; sh[6] = 10 * nsplit;
    }
    ++g_prof.n;
    double mnk = (double)g.M * g.N * g.K * g.batch;
    g_prof.flops += 2.0 * mnk;
    prof_add_bytes(10 * nsplit, ((double)g.M * g.K * sizeof(TA) + (double)g.K * g.N * sizeof(TB) +
                     (double)g.M * g.N * sizeof(TC) * (g.beta != 0.0 ? 2 : 1)) * g.batch);
  }
  if (nsplit > 1) {
    long long mn = (long long)g.M * g.N;
    dim3 rg(cdiv(mn, 256), g.batch);
    splitk_reduce<TC, Acc><<<rg, 256, 0, st>>>(g, nsplit, (const Acc*)s.ptr);
    check_launch("splitk_reduce");
  }
}

// tile choice: a side of at most 32 gets the matching narrow tile
template <class F>
void with_tile(const GemmArgs& g, F&& f) {
  if (g.M <= 32 && g.N > 32) f(TileNarrowM());
  else if (g.N <= 32 && g.M > 32) f(TileNarrowN());
  else f(TileSq());
}

void splitk_reduce_f32(const GemmArgs& g, int nsplit, const float* part, cudaStream_t st) {
  long long mn = (long long)g.M * g.N;
  dim3 rg(cdiv(mn, 256), g.batch);
  splitk_reduce<float, float><<<rg, 256, 0, st>>>(g, nsplit, part);
  check_launch("splitk_reduce");
}

template <class TA, class TB, class TC, class Acc>
void gemm(const GemmArgs& g, Scratch s, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  if (g.K > 0 && gemv_narrow<TA, TB, TC, Acc>(g, st)) return;
  if constexpr (std::is_same<TA, double>::value && std::is_same<TB, double>::value &&
                std::is_same<TC, double>::value && std::is_same<Acc, double>::value) {
    // FP64-class products on the BF16 tensor cores (digit slices) when the context asks for them
    if (g_oz_cfg.on && oz_gemm(g, g_oz_cfg.split.bytes > s.bytes ? g_oz_cfg.split : s, st)) return;
  }
  if constexpr (std::is_same<TA, float>::value && std::is_same<TB, float>::value && std::is_same<TC, float>::value &&
                std::is_same<Acc, float>::value) {
    if (tf32x3_gemm_tn(g, s, st)) return;      // tensor cores, TMA-staged panels with K contiguous
    if (tf32x3_gemm_nn(g, st)) return;         // tensor cores, M-major A and K-major B
    // sketch-width products (N = cap + oversampling, a few columns past a multiple of 128): the
    // large tiles take the multiple of 128 and a narrow tile the remaining columns, instead of a
    // second column of nearly empty 128-wide tiles
    const int rem = g.N % 128;
    if (g.N > 128 && rem > 0 && rem <= 32 && g.offmode == 0) {
      GemmArgs h = g;
      h.N = g.N - rem;
      if (sgemm_large(h, st)) {
        GemmArgs t = g;
        t.N = rem;
        t.B = g.tB ? (const void*)((const float*)g.B + h.N) : (const void*)((const float*)g.B + (size_t)h.N * g.ldb);
        t.C = (void*)((float*)g.C + (size_t)h.N * g.ldc);
        if (!gemv_narrow<TA, TB, TC, Acc>(t, st)) gemm_tiles<TA, TB, TC, Acc, TileNarrowN>(t, s, st);
        return;
      }
    }
    if (sgemm_large(g, st)) return;
  }
  with_tile(g, [&](auto tl) { gemm_tiles<TA, TB, TC, Acc, decltype(tl)>(g, s, st); });
}

template void gemm<double, double, double, double>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm<float, float, float, float>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm<float, float, double, double>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm<float, double, double, double>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm<double, float, float, double>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm<double, double, float, double>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm<float, float, float, double>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm<double, float, float, float>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm<double, float, double, double>(const GemmArgs&, Scratch, cudaStream_t);

}  // namespace hodlr

// =============================================================================================
// Double-float GEMM: operands split into (hi, lo) FP32 pairs and products accumulated in
// double-float (about 48 significant bits) on the FP32 pipes.  GB300's FP64 rate is far below
// its FP32 rate, so sums that need more than FP32 accuracy (leaf sketches whose row sums are
// thousands of times the nugget; the Woodbury factorization sweeps) use this path.
namespace hodlr {
namespace {

struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_from(double x) {
  float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ DF df_from(float x) { return {x, 0.0f}; }
__device__ __forceinline__ DF df_from(float2 x) { return {x.x, x.y}; }   // operand already split
// acc += a * b (double-float): the high parts' product is split exactly (FMA) and added to
// acc.hi exactly (TwoSum); its rounding errors and the cross terms collect in acc.lo, which is
// folded in once at the end (12 FP32 instructions; the collected terms are ~2^-24 |hi| each, so
// K of them add ~K 2^-48 relative, as a per-step renormalisation would).
__device__ __forceinline__ DF df_fma(DF acc, DF a, DF b) {
  const float p = a.hi * b.hi;
  float pe = fmaf(a.hi, b.hi, -p);
  pe = fmaf(a.hi, b.lo, pe);
  pe = fmaf(a.lo, b.hi, pe);
  const float s = acc.hi + p;
  const float bb = s - acc.hi;
  const float e = (acc.hi - (s - bb)) + (p - bb);
  return {s, acc.lo + (e + pe)};
}

template <class TA, class TB, class TC, class TL>
__global__ void __launch_bounds__(NT) gemm_df_kernel(GemmArgs g, int nsplit, int kchunk, double* part) {
  constexpr int BM = TL::BM, BN = TL::BN, TM = TL::TM, TN = TL::TN;
  __shared__ DF As[BK][BM + 1];
  __shared__ DF Bs[BK][BN + 1];
  constexpr int LA = BM * BK / NT, LB = BK * BN / NT;   // tile elements per thread
  const int tid = threadIdx.x;
  const int tx = tid % (BM / TM);
  const int ty = tid / (BM / TM);
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int b = blockIdx.z / nsplit, s = blockIdx.z % nsplit;
  int bi = b;
  if (g.bmap == BMAP_XOR1) bi = b ^ 1;
  else if (g.bmap == BMAP_SHR1) bi = b >> 1;
  long long aoff = (long long)b * g.sA, boff = (long long)bi * g.sB, coff = (long long)b * g.sC;
  int M = g.M, K = g.K;
  if (g.offmode == 1) {
    int r0 = g.off[b];
    M = g.off[b + 1] - r0; aoff = r0; coff = r0;
  } else if (g.offmode == 2) {
    int r0 = g.off[b];
    K = g.off[b + 1] - r0; aoff = r0; boff = r0;
  }
  const int kb = s * kchunk, ke = min(K, kb + kchunk);
  if (m0 >= M) return;
  const TA* A = (const TA*)g.A + aoff;
  const TB* B = (const TB*)g.B + boff;
  DF acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = {0.0f, 0.0f};
  // the next tile is fetched into registers while the current one is multiplied
  DF ra[LA], rb[LB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + r * NT;
      int i, k;
      if (!g.tA) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      const int gi = m0 + i, gk = k0 + k;
      ra[r] = (gi < M && gk < ke) ? df_from(g.tA ? A[gk + (long long)gi * g.lda] : A[gi + (long long)gk * g.lda])
                                  : DF{0.0f, 0.0f};
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + r * NT;
      int k, j;
      if (!g.tB) { k = e % BK; j = e / BK; } else { j = e % BN; k = e / BN; }
      const int gj = n0 + j, gk = k0 + k;
      rb[r] = (gj < g.N && gk < ke) ? df_from(g.tB ? B[gj + (long long)gk * g.ldb] : B[gk + (long long)gj * g.ldb])
                                    : DF{0.0f, 0.0f};
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + r * NT;
      int i, k;
      if (!g.tA) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      As[k][i] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + r * NT;
      int k, j;
      if (!g.tB) { k = e % BK; j = e / BK; } else { j = e % BN; k = e / BN; }
      Bs[k][j] = rb[r];
    }
  };
  if (kb < ke) fetch(kb);
  for (int k0 = kb; k0 < ke; k0 += BK) {
    stash();
    __syncthreads();
    if (k0 + BK < ke) fetch(k0 + BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      DF a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[k][tx + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[k][ty + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = df_fma(acc[i][j], a[i], bb[j]);
    }
    __syncthreads();
  }
  for (int j = 0; j < TN; ++j) {
    int gj = n0 + ty + j * (BN / TN);
    if (gj >= g.N) continue;
    for (int i = 0; i < TM; ++i) {
      int gi = m0 + tx + i * (BM / TM);
      if (gi >= M) continue;
      double v = (double)acc[i][j].hi + (double)acc[i][j].lo;
      if (nsplit == 1) {
        TC* C = (TC*)g.C + coff;
        long long o = gi + (long long)gj * g.ldc;
        double r = g.alpha * v;
        if (g.beta != 0.0) r += g.beta * (double)C[o];
        C[o] = (TC)r;
      } else {
        part[((long long)b * nsplit + s) * (long long)g.M * g.N + gi + (long long)gj * g.M] = v;
      }
    }
  }
}

__global__ void df_split_kernel(const double* x, float2* y, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  const float h = (float)v;
  y[i] = make_float2(h, (float)(v - (double)h));
}

}  // namespace

template <class TA, class TB, class TC, class TL>
void gemm_df_tiles(const GemmArgs& g, Scratch s, cudaStream_t st) {
  constexpr int BM = TL::BM, BN = TL::BN;
  int tiles = cdiv(g.M, BM) * cdiv(g.N, BN) * g.batch;
  int nsplit = 1;
  if (g.K >= 512 && tiles < 2 * 152) {
    nsplit = (4 * 152 + tiles - 1) / tiles;
    nsplit = std::min(nsplit, cdiv(g.K, 256));
    size_t per = (size_t)g.batch * g.M * g.N * sizeof(double);
    if (per > 0) nsplit = (int)std::min<size_t>(nsplit, s.bytes / per);
    if (nsplit < 2) nsplit = 1;
  }
  int kchunk = g.K;
  if (nsplit > 1) {
    kchunk = ((cdiv(g.K, nsplit) + BK - 1) / BK) * BK;
    nsplit = cdiv(g.K, kchunk);
  }
  if (g.K <= 0) kchunk = 0;
  dim3 grid(cdiv(g.M, BM), cdiv(g.N, BN), g.batch * nsplit);
  if (grid.z > 65535) throw Error(-1, "gemm_df: batch too large");
  const bool prof = g_prof.on && g_prof.n < g_prof.cap;
  if (prof) cudaEventRecord(g_prof.ev[2 * g_prof.n], st);
  gemm_df_kernel<TA, TB, TC, TL><<<grid, NT, 0, st>>>(g, nsplit, kchunk, (double*)s.ptr);
  check_launch("gemm_df_kernel");
  if (prof) {
    cudaEventRecord(g_prof.ev[2 * g_prof.n + 1], st);
    if (g_prof.shape) {
      int* sh = g_prof.shape + 7 * g_prof.n;
      sh[0] = g.M; sh[1] = g.N; sh[2] = g.K; sh[3] = g.batch; sh[4] = g.tA; sh[5] = g.tB; sh[6] = 2;
    }
    ++g_prof.n;
    g_prof.flops += 2.0 * (double)g.M * g.N * g.K * g.batch;
    prof_add_bytes(2, ((double)g.M * g.K * sizeof(TA) + (double)g.K * g.N * sizeof(TB) +
                       (double)g.M * g.N * sizeof(TC) * (g.beta != 0.0 ? 2 : 1)) * g.batch);
  }
  if (nsplit > 1) {
    long long mn = (long long)g.M * g.N;
    dim3 rg(cdiv(mn, 256), g.batch);
    splitk_reduce<TC, double><<<rg, 256, 0, st>>>(g, nsplit, (const double*)s.ptr);
    check_launch("splitk_reduce");
  }
}

template <class TA, class TB, class TC>
void gemm_df(const GemmArgs& g, Scratch s, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  with_tile(g, [&](auto tl) { gemm_df_tiles<TA, TB, TC, decltype(tl)>(g, s, st); });
}
template void gemm_df<double, double, double>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm_df<float, double, double>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm_df<double, float, double>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm_df<float, float, double>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm_df<double, double, float>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm_df<float2, float2, double>(const GemmArgs&, Scratch, cudaStream_t);
template void gemm_df<float2, double, double>(const GemmArgs&, Scratch, cudaStream_t);

void df_split(const double* x, float2* y, long long n, cudaStream_t st) {
  if (n <= 0) return;
  df_split_kernel<<<cdiv(n, 256), 256, 0, st>>>(x, y, n);
  check_launch("df_split");
}

}  // namespace hodlr

// =============================================================================================
// Large-tile FP32 GEMM (128 x 128 tile, 8 x 8 outputs per thread, register-prefetched double
// buffering in shared memory).  Used for the wide FP32 contractions of the trace sweeps and the
// Woodbury solves when both M and N are large; everything else goes to the generic kernel.
namespace hodlr {
namespace {

constexpr int LBM = 128, LBN = 128, LBK = 8, LNT = 256;

__global__ void __launch_bounds__(LNT, 2) sgemm_large_kernel(GemmArgs g) {
  __shared__ float As[2][LBK][LBM + 4];
  __shared__ float Bs[2][LBK][LBN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;          // 16 x 16 threads, 8 x 8 outputs each
  const int m0 = blockIdx.x * LBM, n0 = blockIdx.y * LBN;
  const int b = blockIdx.z;
  int bi = b;
  if (g.bmap == BMAP_XOR1) bi = b ^ 1;
  else if (g.bmap == BMAP_SHR1) bi = b >> 1;
  const float* A = (const float*)g.A + (long long)b * g.sA;
  const float* B = (const float*)g.B + (long long)bi * g.sB;
  float* C = (float*)g.C + (long long)b * g.sC;
  const int M = g.M, N = g.N, K = g.K;
  // each thread loads 4 elements of the A tile and 4 of the B tile per stage
  float ra[4], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * LNT;
      int i, k;
      if (!g.tA) { i = e % LBM; k = e / LBM; } else { k = e % LBK; i = e / LBK; }
      int gi = m0 + i, gk = k0 + k;
      ra[r] = (gi < M && gk < K) ? (g.tA ? A[gk + (long long)gi * g.lda] : A[gi + (long long)gk * g.lda]) : 0.f;
      int j;
      if (!g.tB) { k = e % LBK; j = e / LBK; } else { j = e % LBN; k = e / LBN; }
      int gj = n0 + j;
      gk = k0 + k;
      rb[r] = (gj < N && gk < K) ? (g.tB ? B[gj + (long long)gk * g.ldb] : B[gk + (long long)gj * g.ldb]) : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * LNT;
      int i, k;
      if (!g.tA) { i = e % LBM; k = e / LBM; } else { k = e % LBK; i = e / LBK; }
      As[buf][k][i] = ra[r];
      int j;
      if (!g.tB) { k = e % LBK; j = e / LBK; } else { j = e % LBN; k = e / LBN; }
      Bs[buf][k][j] = rb[r];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += LBK) {
    const bool more = k0 + LBK < K;
    if (more) load(k0 + LBK);
#pragma unroll
    for (int k = 0; k < LBK; ++k) {
      float a[8], bb[8];
      // rows tx*4 .. +3 and 64 + tx*4 .. +3; cols ty*4 .. +3 and 64 + ty*4 .. +3
      float4 a0 = *(const float4*)&As[buf][k][tx * 4];
      float4 a1 = *(const float4*)&As[buf][k][64 + tx * 4];
      float4 b0 = *(const float4*)&Bs[buf][k][ty * 4];
      float4 b1 = *(const float4*)&Bs[buf][k][64 + ty * 4];
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w; a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      bb[0] = b0.x; bb[1] = b0.y; bb[2] = b0.z; bb[3] = b0.w; bb[4] = b1.x; bb[5] = b1.y; bb[6] = b1.z; bb[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
  const float alpha = (float)g.alpha, beta = (float)g.beta;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    int gj = n0 + (j < 4 ? ty * 4 + j : 64 + ty * 4 + j - 4);
    if (gj >= N) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int gi = m0 + (i < 4 ? tx * 4 + i : 64 + tx * 4 + i - 4);
      if (gi >= M) continue;
      long long o = gi + (long long)gj * g.ldc;
      float v = alpha * acc[i][j];
      if (beta != 0.f) v += beta * C[o];
      C[o] = v;
    }
  }
}

}  // namespace

bool sgemm_large(const GemmArgs& g, cudaStream_t st) {
  if (g.offmode != 0 || g.M < 256 || g.N < 96 || g.K < 8) return false;
  dim3 grid(cdiv(g.M, LBM), cdiv(g.N, LBN), g.batch);
  if (grid.z > 65535) return false;
  const bool prof = g_prof.on && g_prof.n < g_prof.cap;
  if (prof) cudaEventRecord(g_prof.ev[2 * g_prof.n], st);
  sgemm_large_kernel<<<grid, LNT, 0, st>>>(g);
  check_launch("sgemm_large_kernel");
  if (prof) {
    cudaEventRecord(g_prof.ev[2 * g_prof.n + 1], st);
    if (g_prof.shape) {
      int* sh = g_prof.shape + 7 * g_prof.n;
      sh[0] = g.M; sh[1] = g.N; sh[2] = g.K; sh[3] = g.batch; sh[4] = g.tA; sh[5] = g.tB; sh[6] = 1;
    }
    ++g_prof.n;
    g_prof.flops += 2.0 * (double)g.M * g.N * g.K * g.batch;
    prof_add_bytes(1, ((double)g.M * g.K + (double)g.K * g.N + (double)g.M * g.N * (g.beta != 0.0 ? 2 : 1)) * 4.0 *
                    g.batch);
  }
  return true;
}

}  // namespace hodlr
