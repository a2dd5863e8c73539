// Batched column-major GEMM on the SIMT pipes (FP64 DFMA or FP32 FFMA), with
// deterministic split-K for the tall-skinny Gram products of the HODLR level sweeps.
//
// Used for: the peeling products (K - sum_l' H^(l')) R (Sec. 3.2.2), the projections
// B~ = B^T Q, the Gram matrices of the QR step (Alg. 1 step 3), Alg. 2's products, the
// Woodbury sweeps of the factorization (App. C) and the trace products (App. B).
#include "common.cuh"
#include "ops.h"

#include <algorithm>

namespace hodlr {

long long g_kernel_launches = 0;
GemmProfile g_prof;

namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
constexpr int NT = (BM / TM) * (BN / TN);  // 256 threads

template <class TA, class TB, class TC, class Acc>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs g, int nsplit, int kchunk, Acc* part) {
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

  for (int k0 = kb; k0 < ke; k0 += BK) {
    // A tile: op(A)(i, k), i in [m0, m0+BM), k in [k0, k0+BK)
#pragma unroll
    for (int e = tid; e < BM * BK; e += NT) {
      int i, k;
      if (!g.tA) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      int gi = m0 + i, gk = k0 + k;
      Acc v = Acc(0);
      if (gi < M && gk < ke)
        v = (Acc)(g.tA ? A[gk + (long long)gi * g.lda] : A[gi + (long long)gk * g.lda]);
      As[k][i] = v;
    }
#pragma unroll
    for (int e = tid; e < BK * BN; e += NT) {
      int k, j;
      if (!g.tB) { k = e % BK; j = e / BK; } else { j = e % BN; k = e / BN; }
      int gj = n0 + j, gk = k0 + k;
      Acc v = Acc(0);
      if (gj < g.N && gk < ke)
        v = (Acc)(g.tB ? B[gj + (long long)gk * g.ldb] : B[gk + (long long)gj * g.ldb]);
      Bs[k][j] = v;
    }
    __syncthreads();
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

}  // namespace

template <class TA, class TB, class TC, class Acc>
void gemm(const GemmArgs& g, Scratch s, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  int tiles = cdiv(g.M, BM) * cdiv(g.N, BN) * g.batch;
  int nsplit = 1;
  if (g.K >= 512 && tiles < 2 * 152) {
    nsplit = (4 * 152 + tiles - 1) / tiles;
    nsplit = std::min(nsplit, cdiv(g.K, 256));
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
  gemm_kernel<TA, TB, TC, Acc><<<grid, NT, 0, st>>>(g, nsplit, kchunk, (Acc*)s.ptr);
  check_launch("gemm_kernel");
  if (prof) {
    cudaEventRecord(g_prof.ev[2 * g_prof.n + 1], st);
    ++g_prof.n;
    double mnk = (double)g.M * g.N * g.K * g.batch;
    g_prof.flops += 2.0 * mnk;
    g_prof.bytes += ((double)g.M * g.K * sizeof(TA) + (double)g.K * g.N * sizeof(TB) +
                     (double)g.M * g.N * sizeof(TC) * (g.beta != 0.0 ? 2 : 1)) * g.batch;
  }
  if (nsplit > 1) {
    long long mn = (long long)g.M * g.N;
    dim3 rg(cdiv(mn, 256), g.batch);
    splitk_reduce<TC, Acc><<<rg, 256, 0, st>>>(g, nsplit, (const Acc*)s.ptr);
    check_launch("splitk_reduce");
  }
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
