// Measured arithmetic peaks of this GPU: the roofline denominators of the kernels that run on
// the FP32 and FP64 pipes and on the tcgen05 tensor cores (TF32 and BF16 operands).
//
// Each probe is a kernel that keeps one pipe busy with independent work and does nothing else:
//   FFMA / DFMA: 16 independent fused multiply-add chains per thread, 8 warps per scheduler;
//   tcgen05:     one CTA per SM, one thread issues back-to-back 128 x 256 MMAs (K = 8 TF32 or
//                K = 16 BF16 values each) on zero-filled shared-memory operands into a TMEM
//                accumulator, then commits to an mbarrier (bounded wait) and frees the TMEM.
// The host times a few launches with CUDA events after a warm-up launch and reports the best.
// Nothing is allocated: results go to a static device word; TMEM is allocated and freed on chip.
#include "../../include/hodlr.h"
#include "common.cuh"

namespace hodlr {
namespace {

__device__ double g_peak_sink;
__device__ int g_peak_status;

constexpr int kChains = 16;

template <class V>
__global__ void __launch_bounds__(1024) fma_peak_kernel(int iters, V seed) {
  V a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (V)(threadIdx.x + c);
  const V m = (V)0.999999, k = (V)1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
    }
  }
  V s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == (V)-1.2345) g_peak_sink = (double)s;   // never true: keeps the chains alive
}

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t peak_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

constexpr int kMmaWaitLimit = 1 << 26;

// KIND 0: kind::tf32 (K = 8 per MMA, 32-byte steps in a 128-byte row);
// KIND 1: kind::f16 with BF16 operands (K = 16 per MMA, 32-byte steps).
template <int KIND>
__global__ void __launch_bounds__(128, 1) mma_peak_kernel(int iters) {
  extern __shared__ unsigned char raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  unsigned char* A = sm;              // 128 rows x 128 B
  unsigned char* B = sm + 16384;      // 256 rows x 128 B
  uint64_t* bar = (uint64_t*)(sm + 16384 + 32768);
  uint32_t* slot = (uint32_t*)(bar + 1);
  for (int i = threadIdx.x; i < (16384 + 32768) / 16; i += blockDim.x) ((uint4*)sm)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(su32(slot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *slot;
  // D FP32; A, B TF32 (2) or BF16 (1), K-major; N = 256; M = 128
  const uint32_t ab = KIND == 0 ? 2u : 1u;
  const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
  bool ok = true;
  if (threadIdx.x == 0) {
    const uint32_t a0 = su32(A), b0 = su32(B);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ad = peak_desc(a0 + 32 * kk), bd = peak_desc(b0 + 32 * kk);
        const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
        if (KIND == 0)
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        else
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
    ok = false;
    for (int i = 0; i < kMmaWaitLimit && !ok; ++i) {
      uint32_t done;
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(su32(bar))
          : "memory");
      ok = done != 0;
    }
    if (!ok) atomicExch(&g_peak_status, HODLR_ETIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // a CTA whose MMAs did not complete in time keeps its TMEM (freeing it under running MMAs
  // is undefined); the host reports the timeout
  if (threadIdx.x < 32 && __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
  }
}

}  // namespace
}  // namespace hodlr

using namespace hodlr;

extern "C" int hodlr_peak(int which, double* tflops_out) {
  if (!tflops_out || which < 0 || which > 3) return HODLR_EINVAL;
  try {
    int dev = 0, sms = 0;
    HODLR_CUDA(cudaGetDevice(&dev));
    HODLR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int zero = 0;
    HODLR_CUDA(cudaMemcpyToSymbol(g_peak_status, &zero, sizeof(int)));
    cudaEvent_t e0, e1;
    HODLR_CUDA(cudaEventCreate(&e0));
    HODLR_CUDA(cudaEventCreate(&e1));
    double best = 0.0;
    const size_t smem = 16384 + 32768 + 1024 + 64;
    if (which >= 2) {
      auto k = which == 2 ? mma_peak_kernel<0> : mma_peak_kernel<1>;
      // large enough that one CTA fits per SM
      HODLR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 120 * 1024));
    }
    for (int rep = 0; rep < 4; ++rep) {
      double flops = 0.0;
      HODLR_CUDA(cudaEventRecord(e0, 0));
      if (which == 0) {
        const int iters = 4096;
        fma_peak_kernel<float><<<2 * sms, 1024>>>(iters, 1.0f);
        flops = 2.0 * kChains * 8 * (double)iters * 1024 * 2 * sms;
      } else if (which == 1) {
        const int iters = 256;
        fma_peak_kernel<double><<<2 * sms, 1024>>>(iters, 1.0);
        flops = 2.0 * kChains * 8 * (double)iters * 1024 * 2 * sms;
      } else {
        const int iters = 2048;
        if (which == 2) mma_peak_kernel<0><<<sms, 128, 120 * 1024>>>(iters);
        else mma_peak_kernel<1><<<sms, 128, 120 * 1024>>>(iters);
        flops = 2.0 * 128 * 256 * (which == 2 ? 8 : 16) * 4.0 * iters * sms;
      }
      HODLR_CUDA(cudaGetLastError());
      count_launch();
      HODLR_CUDA(cudaEventRecord(e1, 0));
      HODLR_CUDA(cudaEventSynchronize(e1));
      float ms = 0.0f;
      HODLR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0 && ms > 0.0f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    (void)smem;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int st = 0;
    HODLR_CUDA(cudaMemcpyFromSymbol(&st, g_peak_status, sizeof(int)));
    if (st) return HODLR_ETIMEOUT;
    *tflops_out = best;
  } catch (const Error& x) {
    return x.code;
  }
  return HODLR_OK;
}
