// FP32-accurate dense products on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
// Used for the DST-I products of the 2-D operator solve (A^{-1} = S T_y S with S the G x G
// sine transform, Sec. 5.1 SPDE representation): C = S X with X a G x (G q) panel, and for the
// batched FP32 products of the HODLR construction and solves (Sec. 3, Alg. 1): F_l^T X with
// K = the block height (both operands K-contiguous) and F_l T or L X with K = a rank width or
// a leaf size (A M-contiguous).  Each operand is split into a TF32 head and an FP32 remainder
// (hi = x with the low 13 mantissa bits cleared, lo = x - hi, exact), and
//   C = A_hi B_hi + A_hi B_lo + A_lo B_hi
// is accumulated in FP32 in tensor memory (3xTF32: the dropped A_lo B_lo term and the TF32
// truncation of the remainders are ~2^-21 relative, the size of FP32 accumulation error).
//
// One CTA (8 warps) computes a 128 x bn tile of C (bn <= 256, a multiple of 16):
//   * TMA (cp.async.bulk.tensor) stages 32-wide K slices of A (128 rows) and B (bn columns)
//     into shared memory with the 128-byte swizzle, double-buffered, completion tracked by
//     mbarrier transaction counts;
//   * the CTA's threads split the B slice in place (hi) and into a second buffer (lo), and A
//     likewise; an M-contiguous A slice arrives as four 32-row boxes and is transposed into the
//     K-major layout by the same pass, so the products always read K-major operands;
//   * one thread issues 12 tcgen05.mma (4 K-steps x 3 products, M=128, N=bn, K=8) into a
//     128 x bn FP32 accumulator in TMEM and commits them to the stage's mbarrier;
//   * the epilogue reads TMEM with tcgen05.ld (each warp its 32-lane slice, alternate column
//     chunks) and stores C column-major (coalesced along the rows), or split-K partial sums.
// Every mbarrier wait is bounded; a wait that gives up records HODLR_ETIMEOUT in a device
// status word, waits (bounded) for the copies and products already issued, frees its TMEM
// and returns.
#include <cuda.h>

#include <mutex>

#include "../../include/hodlr.h"
#include "common.cuh"
#include "ops.h"

namespace hodlr {
namespace {

constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 32, TC_THREADS = 256, TC_STAGES = 2;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 4;                        // 16 KB
constexpr int TC_B_BYTES = TC_BN * TC_BK * 4;                        // 32 KB
constexpr int TC_STAGE_BYTES = 2 * TC_A_BYTES + 2 * TC_B_BYTES;      // 96 KB
constexpr int TC_SMEM_BYTES = TC_STAGES * TC_STAGE_BYTES + 1024 + 128;
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr int TC_WAIT_LIMIT = 1 << 22;

__device__ int g_tc_status;
// Poll limit of each CTA's first operand wait (a test hook: set lower from the host to make
// that wait give up; every other wait, and the drain of issued copies, keeps TC_WAIT_LIMIT).
__device__ int g_tc_first_wait = TC_WAIT_LIMIT;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Wait for the completion of the barrier phase with parity `ph`; false if the wait gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t ph, int limit = TC_WAIT_LIMIT) {
  const uint32_t addr = smem_u32(bar);
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(ph)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of 128 bytes,
// 8-row groups 1024 bytes apart (tcgen05 descriptor format, version 1).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
  d |= (uint64_t)(16u >> 4) << 16;                  // leading byte offset (not used with this swizzle)
  d |= (uint64_t)(1024u >> 4) << 32;                // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)2 << 61;                           // 128-byte swizzle
  return d;
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Problem description of one launch (every product of the batch has the same shape).
struct TcParams {
  int M, N, K;            // per product: C (M x N) = A (M x K) B (K x N), B K-major
  int bn;                 // N tile: multiple of 16, at most 256
  int nsplit, kchunk;     // split of K across CTAs (kchunk a multiple of 32)
  // per-product offsets of the operand maps: along the inner (contiguous) coordinate for
  // products that are row ranges of one panel, along the outer coordinate for stacked matrices
  long long sA_in, sA_out, sB_in, sB_out;
  int bmap;               // B product of product b: b, b^1 or b>>1
  int a_split;            // 1: A is split into head and remainder here; 0: the remainder has its own map
  int a_mn;               // 1: A is M-major (M contiguous): four 32-row boxes per slice, transposed in shared memory
  float alpha, beta;
  float* C;               // nsplit == 1: C_b = C + b*sC, leading dimension ldc
  long long ldc, sC;
  float* part;            // nsplit > 1: partial sums, ((b*nsplit + s) * M * N) + i + j*M
};

__device__ __forceinline__ void split_tile(float* hi_io, float* lo, int n4, int tid) {
  float4* h4 = (float4*)hi_io;
  float4* l4 = (float4*)lo;
  for (int e = tid; e < n4; e += TC_THREADS) {
    float4 v = h4[e], h, l;
    h.x = tf32_head(v.x); l.x = v.x - h.x;
    h.y = tf32_head(v.y); l.y = v.y - h.y;
    h.z = tf32_head(v.z); l.z = v.z - h.z;
    h.w = tf32_head(v.w); l.w = v.w - h.w;
    h4[e] = h;
    l4[e] = l;
  }
}

// M-major A slice: TMA leaves four boxes of 32 rows (128 B of M) x 32 K values, 4 KB apart,
// each with the 128-byte swizzle (16-byte chunk index XOR K row mod 8).  Each thread gathers
// four (m, 4 consecutive k) quads into registers ...
__device__ __forceinline__ void gather_mn(const float* box, float4 (&q)[4], int tid) {
  const unsigned char* bs = (const unsigned char*)box;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int e = tid + TC_THREADS * j, m = e & (TC_BM - 1), kq = e >> 7;
    const int i = m >> 5, mc = (m & 31) >> 2, mo = (m & 3) * 4;
    float v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int k = 4 * kq + t;
      v[t] = *(const float*)(bs + i * 4096 + k * 128 + ((mc ^ (k & 7)) << 4) + mo);
    }
    q[j] = make_float4(v[0], v[1], v[2], v[3]);
  }
}
// ... and, once every thread has read, stores their TF32 heads and remainders K-major (row m of
// 128 B, chunk kq XOR m mod 8: the layout TMA gives a K-major slice).
__device__ __forceinline__ void scatter_km(float* hi, float* lo, const float4 (&q)[4], int tid) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int e = tid + TC_THREADS * j, m = e & (TC_BM - 1), kq = e >> 7;
    const int off = m * 128 + ((kq ^ (m & 7)) << 4);
    float4 h, l;
    h.x = tf32_head(q[j].x); l.x = q[j].x - h.x;
    h.y = tf32_head(q[j].y); l.y = q[j].y - h.y;
    h.z = tf32_head(q[j].z); l.z = q[j].z - h.z;
    h.w = tf32_head(q[j].w); l.w = q[j].w - h.w;
    *(float4*)((unsigned char*)hi + off) = h;
    *(float4*)((unsigned char*)lo + off) = l;
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    tf32x3_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapAlo,
                       const __grid_constant__ CUtensorMap mapB, const TcParams p) {
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + TC_STAGES * TC_STAGE_BYTES);
  uint64_t* done = full + TC_STAGES;
  uint32_t* tslot = (uint32_t*)(done + TC_STAGES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // M tiles vary fastest, so the CTAs that share a B tile run together and reuse it from L2
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * p.bn;
  const int b = blockIdx.z / p.nsplit, sp = blockIdx.z % p.nsplit;
  const int bb = p.bmap == BMAP_XOR1 ? (b ^ 1) : (p.bmap == BMAP_SHR1 ? (b >> 1) : b);
  const int kbeg = sp * p.kchunk, kend = min(p.K, kbeg + p.kchunk);
  const int nk = (kend - kbeg + TC_BK - 1) / TC_BK;
  const long long ax0 = (long long)b * p.sA_in, ay0 = (long long)b * p.sA_out;
  const long long bx0 = (long long)bb * p.sB_in + kbeg, by0 = (long long)bb * p.sB_out + n0;
  const int b_bytes = p.bn * TC_BK * 4;

  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&done[s], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // instruction descriptor: D FP32, A and B TF32, both K-major, N = bn, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(p.bn >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
  auto stage_ptr = [&](int s, int which) -> float* {   // 0 A_hi, 1 A_lo, 2 B_hi, 3 B_lo
    unsigned char* base = sm + s * TC_STAGE_BYTES;
    const int offs[4] = {0, TC_A_BYTES, 2 * TC_A_BYTES, 2 * TC_A_BYTES + TC_B_BYTES};
    return (float*)(base + offs[which]);
  };
  auto issue_loads = [&](int kt) {
    const int s = kt & 1;
    mbar_expect_tx(&full[s], TC_A_BYTES * (p.a_split ? 1 : 2) + b_bytes);
    const int k0 = kbeg + kt * TC_BK;
    if (!p.a_mn) {
      tma_load_2d(stage_ptr(s, 0), &mapA, (int)(ax0 + k0), (int)(ay0 + m0), &full[s]);
      if (!p.a_split) tma_load_2d(stage_ptr(s, 1), &mapAlo, (int)(ax0 + k0), (int)(ay0 + m0), &full[s]);
    } else {
      // M-major A: four boxes of 32 rows (128 B) x 32 K values, 4 KB apart
#pragma unroll
      for (int i = 0; i < TC_BM / 32; ++i)
        tma_load_2d((unsigned char*)stage_ptr(s, 0) + i * 4096, &mapA, (int)(ax0 + m0 + 32 * i), (int)(ay0 + k0),
                    &full[s]);
    }
    tma_load_2d(stage_ptr(s, 2), &mapB, (int)bx0 + kt * TC_BK, (int)by0, &full[s]);
  };

  bool ok = true;
  int issued = 0, committed = 0;   // k-slices whose loads / products were issued (thread 0)
  if (tid == 0 && nk > 0) {
    issue_loads(0);
    issued = 1;
  }
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt & 1;
    if (tid == 0 && kt + 1 < nk) {
      // the other stage was last read by the products of slice kt-1
      if (kt >= 1 && !mbar_wait(&done[s ^ 1], ((kt - 1) >> 1) & 1)) ok = false;
      if (ok) {
        issue_loads(kt + 1);
        issued = kt + 2;
      }
    }
    if (ok && !mbar_wait(&full[s], (kt >> 1) & 1, kt == 0 ? g_tc_first_wait : TC_WAIT_LIMIT)) ok = false;
    if (p.a_mn) {   // uniform over the CTA: every thread reaches the barrier
      float4 q[4];
      if (ok) gather_mn(stage_ptr(s, 0), q, tid);
      __syncthreads();
      if (ok) scatter_km(stage_ptr(s, 0), stage_ptr(s, 1), q, tid);
    }
    if (ok) {
      split_tile(stage_ptr(s, 2), stage_ptr(s, 3), p.bn * TC_BK / 4, tid);
      if (p.a_split && !p.a_mn) split_tile(stage_ptr(s, 0), stage_ptr(s, 1), TC_BM * TC_BK / 4, tid);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    tc_fence_after();
    if (tid == 0) {
      const uint32_t ah = smem_u32(stage_ptr(s, 0)), al = smem_u32(stage_ptr(s, 1));
      const uint32_t bh = smem_u32(stage_ptr(s, 2)), bl = smem_u32(stage_ptr(s, 3));
#pragma unroll
      for (int kk = 0; kk < TC_BK / 8; ++kk) {
        const uint32_t o = kk * 32;   // 8 FP32 values along K: 32 bytes in a K-major row
        mma_tf32(tmem, smem_desc(ah + o), smem_desc(bh + o), idesc, (kt > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(tmem, smem_desc(ah + o), smem_desc(bl + o), idesc, 1u);
        mma_tf32(tmem, smem_desc(al + o), smem_desc(bh + o), idesc, 1u);
      }
      mma_commit(&done[s]);
      committed = kt + 1;
    }
  }
  if (ok && nk > 0) {
    const int last = nk - 1;
    ok = mbar_wait(&done[last & 1], (last >> 1) & 1);
  }
  ok = __syncthreads_and(ok) != 0;
  if (ok) {
    tc_fence_after();
    // warp w reads TMEM lanes 32 (w % 4) .. + 31; the two warp quartets take alternate column chunks
    const int wq = warp & 3, wh = warp >> 2;
    const int row = m0 + 32 * wq + lane;
    const int ncols = min(p.bn, p.N - n0);
    for (int c0 = 32 * wh; c0 < ncols; c0 += 64) {
      uint32_t r[32];
      if (nk > 0) {
        tmem_ld32(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)c0, r);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) r[j] = 0u;
      }
      if (row < p.M) {
        const int nj = min(32, ncols - c0);
        if (p.nsplit == 1) {
          float* c = p.C + (size_t)b * p.sC + (size_t)(n0 + c0) * p.ldc + row;
          // all loads of C before the first store: a store may alias a later load as far as the
          // compiler knows, which would serialise 32 load latencies
          float cv[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) cv[j] = (p.beta != 0.0f && j < nj) ? c[(size_t)j * p.ldc] : 0.0f;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < nj) c[(size_t)j * p.ldc] = p.alpha * __uint_as_float(r[j]) + p.beta * cv[j];
        } else {
          float* part = p.part + ((size_t)b * p.nsplit + sp) * ((size_t)p.M * p.N) + (size_t)(n0 + c0) * p.M + row;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < nj) part[(size_t)j * p.M] = __uint_as_float(r[j]);
        }
      }
    }
  } else if (tid == 0) {
    // give the copies and products already issued a bounded chance to land, then report
    atomicExch(&g_tc_status, HODLR_ETIMEOUT);
    for (int kt = committed - 1; kt >= 0 && kt >= committed - 2; --kt) mbar_wait(&done[kt & 1], (kt >> 1) & 1);
    for (int kt = issued - 1; kt >= committed && kt >= 0; --kt) mbar_wait(&full[kt & 1], (kt >> 1) & 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

__global__ void tf32_split_kernel(const float* x, float* hi, float* lo, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v = x[i], h = tf32_head(v);
  hi[i] = h;
  lo[i] = v - h;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// 2-D FP32 tensor map over a column-major matrix: inner dimension (contiguous) `inner`,
// outer `outer`, leading dimension `ld` elements; box `box_inner` x `box_outer`.
bool make_map(CUtensorMap* m, const float* ptr, long long inner, long long outer, long long ld, int box_inner,
              int box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace

bool tf32x3_supported(int M, int K, long long lda, long long ldb, long long ldc) {
  return M >= TC_BM && K >= TC_BK && lda % 4 == 0 && ldb % 4 == 0 && ldc >= M;
}

void tf32_split(const float* x, float* hi, float* lo, long long n, cudaStream_t st) {
  if (n <= 0) return;
  tf32_split_kernel<<<cdiv(n, 256), 256, 0, st>>>(x, hi, lo, n);
  check_launch("tf32_split");
}

namespace {
void tc_launch(const CUtensorMap& ma, const CUtensorMap& ml, const CUtensorMap& mb, const TcParams& p, int batch,
               cudaStream_t st) {
  // per device and cheap: set on every launch rather than cached in a process-wide flag
  HODLR_CUDA(cudaFuncSetAttribute(tf32x3_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BYTES));
  dim3 grid(cdiv(p.M, TC_BM), cdiv(p.N, p.bn), batch * p.nsplit);
  const bool prof = g_prof.on && g_prof.n < g_prof.cap;
  if (prof) cudaEventRecord(g_prof.ev[2 * g_prof.n], st);
  tf32x3_gemm_kernel<<<grid, TC_THREADS, TC_SMEM_BYTES, st>>>(ma, ml, mb, p);
  check_launch("tf32x3_gemm_kernel");
  if (prof) {
    cudaEventRecord(g_prof.ev[2 * g_prof.n + 1], st);
    if (g_prof.shape) {
      int* sh = g_prof.shape + 7 * g_prof.n;
      sh[0] = p.M; sh[1] = p.N; sh[2] = p.K; sh[3] = batch; sh[4] = p.a_mn ? 0 : 1; sh[5] = 0; sh[6] = 4;
    }
    ++g_prof.n;
    g_prof.flops += 2.0 * (double)p.M * p.N * p.K * batch;
    prof_add_bytes(4, ((double)p.M * p.K + (double)p.K * p.N + (double)p.M * p.N) * 4.0 * batch);
  }
}
}  // namespace

bool tf32x3_gemm(const float* Ahi, const float* Alo, long long lda, const float* B, long long ldb, float* C,
                 long long ldc, int M, int N, int K, cudaStream_t st) {
  if (N <= 0) return true;
  if (!tf32x3_supported(M, K, lda, ldb, ldc)) return false;
  if (((uintptr_t)Ahi | (uintptr_t)Alo | (uintptr_t)B) & 15) return false;
  CUtensorMap ma, ml, mb;
  if (!make_map(&ma, Ahi, K, M, lda, TC_BK, TC_BM) || !make_map(&ml, Alo, K, M, lda, TC_BK, TC_BM) ||
      !make_map(&mb, B, K, N, ldb, TC_BK, TC_BN))
    return false;
  if (cdiv(N, TC_BN) > 65535) return false;
  TcParams p{};
  p.M = M; p.N = N; p.K = K; p.bn = TC_BN; p.nsplit = 1; p.kchunk = ((K + TC_BK - 1) / TC_BK) * TC_BK;
  p.sA_in = 0; p.sA_out = 0; p.sB_in = 0; p.sB_out = 0; p.bmap = BMAP_ID; p.a_split = 0; p.a_mn = 0;
  p.alpha = 1.0f; p.beta = 0.0f;
  p.C = C; p.ldc = ldc; p.sC = 0; p.part = nullptr;
  tc_launch(ma, ml, mb, p, 1, st);
  return true;
}

namespace {
int pick_bn(int N) { return N >= TC_BN ? TC_BN : ((N + 15) / 16) * 16; }
}  // namespace

bool tf32x3_gemm_tn(const GemmArgs& g, Scratch s, cudaStream_t st) {
  // C_b = alpha A_b^T B_{map(b)} + beta C_b with A_b = A + b*sA (K x M, ld lda) and B likewise:
  // both operands have K contiguous.  The products of a batch must be row ranges of one panel
  // (offsets along K inside the leading dimension), K a multiple of the 32-wide slice.
  if (!g.tA || g.tB || g.offmode != 0 || g.M <= 0 || g.N <= 0 || g.batch <= 0) return false;
  if (g.K < 4 * TC_BK || g.K % TC_BK || g.M > 4 * TC_BM) return false;
  if (g.lda % 4 || g.ldb % 4 || g.sA % 4 || g.sB % 4) return false;
  if (((uintptr_t)g.A | (uintptr_t)g.B) & 15) return false;
  const int nbB = g.bmap == BMAP_SHR1 ? (g.batch + 1) / 2 : g.batch;
  if ((long long)(g.batch - 1) * g.sA + g.K > g.lda || (long long)(nbB - 1) * g.sB + g.K > g.ldb) return false;
  if (g.bmap == BMAP_XOR1 && (g.batch & 1)) return false;
  const int bn = pick_bn(g.N);
  const long long tiles = (long long)cdiv(g.M, TC_BM) * cdiv(g.N, bn) * g.batch;
  int nsplit = 1;
  if (tiles < 152) {
    nsplit = (int)std::min<long long>(cdiv(2 * 152, tiles), g.K / (4 * TC_BK));
    const size_t per = (size_t)g.batch * g.M * g.N * sizeof(float);
    nsplit = (int)std::min<size_t>(nsplit, s.bytes / per);
    nsplit = std::max(nsplit, 1);
  }
  int kchunk = ((cdiv(g.K, nsplit) + TC_BK - 1) / TC_BK) * TC_BK;
  nsplit = cdiv(g.K, kchunk);
  if ((long long)g.batch * nsplit > 65535 || cdiv(g.N, bn) > 65535) return false;
  CUtensorMap ma, mb;
  if (!make_map(&ma, (const float*)g.A, g.lda, g.M, g.lda, TC_BK, TC_BM) ||
      !make_map(&mb, (const float*)g.B, g.ldb, g.N, g.ldb, TC_BK, bn))
    return false;
  TcParams p{};
  p.M = g.M; p.N = g.N; p.K = g.K; p.bn = bn; p.nsplit = nsplit; p.kchunk = kchunk;
  p.sA_in = g.sA; p.sA_out = 0; p.sB_in = g.sB; p.sB_out = 0;
  p.bmap = g.bmap; p.a_split = 1; p.a_mn = 0;
  p.alpha = (float)g.alpha; p.beta = (float)g.beta;
  p.C = (float*)g.C; p.ldc = g.ldc; p.sC = g.sC; p.part = (float*)s.ptr;
  tc_launch(ma, ma, mb, p, g.batch, st);
  if (nsplit > 1) splitk_reduce_f32(g, nsplit, (const float*)s.ptr, st);
  return true;
}

bool tf32x3_gemm_nn(const GemmArgs& g, cudaStream_t st) {
  // C_b = alpha A_b B_{map(b)} + beta C_b with A_b (M x K, M contiguous) and B_b (K x N, K
  // contiguous), no split of K (the inner dimension here is a rank width or a leaf size).
  //   A_b: row ranges of one panel (A + b*sA, b*sA + M <= lda; the map's K extent is exact)
  //        or stacked M x K matrices (sA a multiple of lda: the K tail reads the next matrix);
  //   B_b: row ranges of one panel (the K tail would read the next rows: K a multiple of 32)
  //        or stacked K x N matrices / a single matrix (the map's K extent is exact: the tail
  //        reads zeros, which also cancels a stacked A's tail).
  if (g.tA || g.tB || g.offmode != 0 || g.M < TC_BM || g.N <= 0 || g.K <= 0 || g.batch <= 0) return false;
  if (g.lda % 4 || g.ldb % 4 || g.lda < g.M || g.ldb < g.K || g.batch > 65535) return false;
  if (((uintptr_t)g.A | (uintptr_t)g.B) & 15) return false;
  if (g.bmap == BMAP_XOR1 && (g.batch & 1)) return false;
  const int nbB = g.bmap == BMAP_SHR1 ? (g.batch + 1) / 2 : g.batch;
  const int bn = pick_bn(g.N);
  if (cdiv(g.N, bn) > 65535) return false;
  long long a_in = 0, a_out = 0, a_inner = g.M, a_outer = g.K;
  if (g.batch > 1 && g.sA != 0) {
    if (g.sA % 4 == 0 && (long long)(g.batch - 1) * g.sA + g.M <= g.lda) {
      a_in = g.sA;
      a_inner = g.lda;
    } else if (g.sA % g.lda == 0 && g.sA / g.lda >= g.K) {
      a_out = g.sA / g.lda;
      a_outer = (long long)(g.batch - 1) * a_out + g.K;
    } else {
      return false;
    }
  }
  long long b_in = 0, b_out = 0, b_inner = g.K, b_outer = g.N;
  bool b_exact = true;   // the map ends at K: the K tail reads zeros
  if (nbB > 1 && g.sB != 0) {
    if (g.sB % 4 == 0 && (long long)(nbB - 1) * g.sB + g.K <= g.ldb) {
      b_in = g.sB;
      b_inner = g.ldb;
      b_exact = false;
    } else if (g.sB % g.ldb == 0 && g.sB / g.ldb >= g.N) {
      b_out = g.sB / g.ldb;
      b_outer = (long long)(nbB - 1) * b_out + g.N;
    } else {
      return false;
    }
  }
  // a K tail multiplies B's zeros: A's tail must be the next matrix of the batch or the map's
  // zero fill, never gap columns between stacked matrices (possibly uninitialised, NaN x 0 = NaN)
  if (g.K % TC_BK && (!b_exact || (a_out != 0 && a_out != g.K))) return false;
  CUtensorMap ma, mb;
  if (!make_map(&ma, (const float*)g.A, a_inner, a_outer, g.lda, 32, TC_BK) ||
      !make_map(&mb, (const float*)g.B, b_inner, b_outer, g.ldb, TC_BK, bn))
    return false;
  TcParams p{};
  p.M = g.M; p.N = g.N; p.K = g.K; p.bn = bn; p.nsplit = 1; p.kchunk = ((g.K + TC_BK - 1) / TC_BK) * TC_BK;
  p.sA_in = a_in; p.sA_out = a_out; p.sB_in = b_in; p.sB_out = b_out;
  p.bmap = g.bmap; p.a_split = 1; p.a_mn = 1;
  p.alpha = (float)g.alpha; p.beta = (float)g.beta;
  p.C = (float*)g.C; p.ldc = g.ldc; p.sC = g.sC; p.part = nullptr;
  tc_launch(ma, ma, mb, p, g.batch, st);
  return true;
}

int tc_set_first_wait_limit(int polls) {
  const int v = polls < 0 ? TC_WAIT_LIMIT : std::min(polls, TC_WAIT_LIMIT);
  return cudaMemcpyToSymbol(g_tc_first_wait, &v, sizeof(int)) == cudaSuccess ? HODLR_OK : HODLR_ECUDA;
}

int tc_status_take(cudaStream_t st) {
  int v = 0, zero = 0;
  HODLR_CUDA(cudaMemcpyFromSymbolAsync(&v, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  HODLR_CUDA(cudaStreamSynchronize(st));
  if (v) HODLR_CUDA(cudaMemcpyToSymbolAsync(g_tc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
  return v;
}

}  // namespace hodlr
