// Allocation-free physics product for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another framework's
// memory pool or under a strict budget, code executing while the allocator must not be
// touched, or host environments that only hand out pre-registered buffers.  For them
// hodlr_apply_static() computes Y = K X for the 1-D univariate model without any
// workspace: its scratch (Thomas-recurrence tables, Matern embedding spectrum, FFT
// twiddles and the embedding itself) lives in the file-scope device array below, which
// every GPU that loads this library keeps for the lifetime of the process.
//
// Set-up: the first call on a device (with that device current) resolves the array's
// device address with cudaGetSymbolAddress and caches it; that first call should be made
// before any stream capture begins.  Every call reuses the same array, whose contents from
// the previous call are left in place: every scratch entry a call reads is written by that
// same call first, so nothing has to start at zero.  Calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array and must be
// serialised by the caller.
#include <mutex>

#include "../../include/hodlr.h"
#include "common.cuh"
#include "ops.h"

namespace hodlr {
namespace {

// Capacity: grids of up to 2048 points (FFT embedding length <= 4096).
constexpr int kStaticMaxG = 2048;
constexpr int kStaticMaxL = 4096;
constexpr size_t kCoef = 2 * (size_t)kStaticMaxG;   // Thomas tables a_i, b_i
constexpr size_t kLam = kStaticMaxL;                 // K_u spectrum
constexpr size_t kLam1 = kStaticMaxL;                // dK_u/dell spectrum (computed alongside)
constexpr size_t kTw = kStaticMaxL;                  // L/2 complex twiddles
constexpr size_t kEmb = kStaticMaxL + 64;            // embedding sequence (+ alignment slack)
constexpr size_t kStaticDoubles = kCoef + kLam + kLam1 + kTw + kEmb;   // 20544 doubles = 160.5 KiB

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

constexpr int kMaxDevices = 64;
double* g_static_ptr[kMaxDevices] = {nullptr};
std::mutex g_static_mu;

double* static_scratch(int dev) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) throw Error(HODLR_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_static_ptr[dev] = (double*)p;
  }
  return g_static_ptr[dev];
}

}  // namespace
}  // namespace hodlr

using namespace hodlr;

extern "C" int hodlr_apply_static(int G, double nu, const double* theta, const double* X, double* Y, int ncols,
                                  void* cuda_stream) {
  if (G < 2 || G > kStaticMaxG || (nu != 0.5 && nu != 1.5) || !theta || !X || !Y || ncols < 0) return HODLR_EINVAL;
  for (int k = 0; k < 4; ++k)
    if (!(theta[k] > 0.0)) return HODLR_EINVAL;
  if (ncols == 0) return HODLR_OK;
  {
    // Y is written while X is still read (the nugget term tau2 X comes last): reject any
    // overlap of the two byte ranges instead of returning a silently wrong product
    const uintptr_t nb = (uintptr_t)G * (uintptr_t)ncols * sizeof(double);
    const uintptr_t x0 = (uintptr_t)X, y0 = (uintptr_t)Y;
    if (x0 < y0 + nb && y0 < x0 + nb) return HODLR_EINVAL;
  }
  try {
    int dev = 0;
    HODLR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return HODLR_EINVAL;
    double* base = static_scratch(dev);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    PhysicsDesc p;
    p.dim = 1; p.G = G; p.nvar = 1; p.nu = nu; p.h = 1.0 / (G + 1);
    int L = 1;
    while (L < 2 * G - 1) L <<= 1;
    p.L = L; p.L1 = 0; p.L2 = 0;
    double* coef = base;
    double* lam0 = coef + kCoef;
    double* lam1 = lam0 + kLam;
    double* tw = lam1 + kLam1;
    double* emb = tw + kTw;
    twiddles<double>(L, tw, st);
    tridiag_tables(p, theta[2], coef, st);
    matern_spectra<double>(p, theta[0], theta[1], lam0, lam1, emb, tw, st);
    // Y = A^{-1} K_u A^{-1} X + tau2 X, computed in place in Y
    Scratch none;
    solve_A<double>(p, ncols, X, G, Y, G, coef, nullptr, nullptr, none, st);
    fft_convolve<double>(p, ncols, Y, G, lam0, nullptr, Y, nullptr, G, nullptr, tw, st);
    solve_A<double>(p, ncols, Y, G, Y, G, coef, nullptr, nullptr, none, st);
    axpby<double>(G, ncols, theta[3], X, G, 1.0, Y, G, st);
    HODLR_CUDA(cudaGetLastError());
  } catch (const Error& x) {
    return x.code;
  }
  return HODLR_OK;
}
