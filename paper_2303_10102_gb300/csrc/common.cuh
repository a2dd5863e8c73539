// Shared definitions of the HODLR CUDA library (device helpers, launch bookkeeping).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <stdexcept>
#include <string>

namespace hodlr {

// Error raised inside the library; converted to a return code at the C ABI.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define HODLR_CUDA(call)                                                                  \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::hodlr::Error(-7, std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

// Kernel-launch counter (per process); every launcher bumps it.
extern long long g_kernel_launches;

// Optional event profile of the GEMM launches (see hodlr_profile in hodlr.h).
struct GemmProfile {
  bool on = false;
  cudaEvent_t* ev = nullptr;   // 2 per launch
  int cap = 0, n = 0;
  double flops = 0.0, bytes = 0.0;
  double fbytes[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // algorithmic operand bytes per kernel family
  int* shape = nullptr;        // per launch: M, N, K, batch, tA, tB, kernel variant
};
extern GemmProfile g_prof;
// kernel family of a recorded variant (0 SIMT tiles incl. split-K variants 10 * nsplit, 1 FP32
// large tiles, 2 double-float, 3 narrow, 4 tcgen05 3xTF32, 5..7 tcgen05 BF16 digit slices)
inline int prof_family(int variant) { return variant >= 10 ? 0 : (variant >= 1 && variant <= 7 ? variant : 0); }
inline void prof_add_bytes(int variant, double b) {
  g_prof.bytes += b;
  g_prof.fbytes[prof_family(variant)] += b;
}

// Optional launch timeline (HODLR_TRACE): an event after every launch on the traced stream;
// the interval between consecutive events is charged to the launch that ends it (idle gaps
// such as host synchronisations included).
struct LaunchTrace {
  bool on = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t* ev = nullptr;   // ev[0] = start, ev[i + 1] after launch i
  const char** name = nullptr;
  int cap = 0, n = 0;
};
extern LaunchTrace g_trace;
inline void count_launch(int n = 1) { g_kernel_launches += n; }

inline void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error(-7, std::string(what) + ": " + cudaGetErrorString(e));
  count_launch();
  if (g_trace.on && g_trace.n < g_trace.cap) {
    cudaEventRecord(g_trace.ev[g_trace.n + 1], g_trace.stream);
    g_trace.name[g_trace.n++] = what;
  }
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

template <class T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

}  // namespace hodlr
