// FP64-class products on the BF16 tensor cores (tcgen05 kind::f16) by exact digit slices.
//
// GB300 executes FP64 fused multiply-adds at about 1 TFLOP/s but BF16 tensor-core products at
// about 2.4 PFLOP/s.  A product C = A B of FP64 matrices is carried out as follows (a slicing
// scheme in the manner of Ozaki, Ogita, Oishi and Rump, with integer digit extraction):
//   * every row i of A gets an exponent ea_i with max_k |A_ik| < 2^ea_i, every column j of B an
//     exponent eb_j likewise;
//   * the scaled row A_ik 2^(6 - ea_i), a number in (-64, 64), is rounded to a fixed-point
//     integer with 42 fractional bits and cut into S = 7 balanced base-2^7 digits a_p in
//     [-64, 64]:  A_ik ~ 2^(ea_i - 6) sum_p a_p 2^(-7p); B likewise (digits b_q);
//   * plane p of A stores a_p 2^(-7p) as BF16 (exact: a digit has at most 7 significant bits),
//     so that the tensor-core product of planes p and q is sum_k a_p b_q 2^(-7(p+q)), and all
//     products of one "group" t = p + q are integer multiples of 2^(-7t);
//   * the products with p + q <= S - 1 are accumulated in FP32 in tensor memory: groups t = 0..3
//     in accumulators of their own, whose sums over a 512-long chunk of K stay within 2^23 units
//     and are therefore exact; groups t = 4..6 share one accumulator (scale 2^-28 of the leading
//     group, so that its FP32 rounding stays near 2^-50 of the result);
//   * each CTA takes one 512-long chunk of K (longer K is split across CTAs and the FP64
//     partials are summed in a fixed order); its exact group sums become one 64-bit integer per
//     element (units 2^-21), which joins the tail group and the scales in integer arithmetic
//     with one rounding to FP64.
// The dropped groups t >= 7 and the fixed-point rounding bound the error by about 2^-47 of
// sum_k max_k'|A_ik'| max_k'|B_k'j| (normwise about 4e-14 on random operands); the FP32
// accumulation of the tail groups in the tensor cores adds about 2e-13 normwise (measured), at a
// cost of 28 BF16 products.
//
// One CTA (8 warps) computes a 128 x 96 tile of C over one chunk of K: TMA
// (cp.async.bulk.tensor, 64-byte swizzle) stages 32-wide K slices of all seven planes of A and
// B (98 KB per stage, two stages) behind mbarrier transaction counts; one thread issues the 56
// tcgen05.mma (M = 128, N = 96, K = 16) of a slice; the five accumulators take 480 of the 512
// TMEM columns; every wait is bounded (a wait that gives up records HODLR_ETIMEOUT, drains what
// was issued and frees the TMEM).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/hodlr.h"
#include "common.cuh"
#include "ops.h"

namespace hodlr {
namespace {

constexpr int OZ_S = 7;                      // digit planes per operand
constexpr int OZ_NPAIR = OZ_S * (OZ_S + 1) / 2;
constexpr int OZ_BM = 128, OZ_BN = 96, OZ_BK = 32;
constexpr int OZ_NACC = 5;                   // accumulators: groups 0..3 exact, groups 4..6 shared
constexpr int OZ_KC = 512;                   // exactness chunk of K
constexpr int OZ_THREADS = 256;
constexpr int OZ_PLANE_A = OZ_BM * OZ_BK * 2;            // 8 KB per plane and slice
// Two tile shapes: 128 x 96 with two 98 KB stages (one CTA per SM, 480 TMEM columns), and for
// short K (at most four slices) 128 x 32 with one 70 KB stage, so that two CTAs share an SM and
// one's loads and epilogue overlap the other's products (160 of 256 TMEM columns each); every
// accumulator starts at a multiple of 32 TMEM columns
template <int BN, int ST> struct OzTile {
  static constexpr int PLANE_B = BN * OZ_BK * 2;
  static constexpr int STAGE = OZ_S * (OZ_PLANE_A + PLANE_B);
  static constexpr int SMEM = ST * STAGE + 1024 + 256;
  static constexpr uint32_t TCOLS = OZ_NACC * BN <= 256 ? 256u : 512u;
};
constexpr int OZ_WAIT_LIMIT = 1 << 22;

__device__ int g_oz_status;

__device__ __forceinline__ uint32_t oz_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void oz_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(oz_smem(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void oz_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(oz_smem(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool oz_wait(uint64_t* bar, uint32_t ph) {
  const uint32_t addr = oz_smem(bar);
  for (int it = 0; it < OZ_WAIT_LIMIT; ++it) {
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
__device__ __forceinline__ void oz_tma3(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(oz_smem(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(oz_smem(bar))
      : "memory");
}
// K-major operand in shared memory with the 64-byte swizzle: rows of 64 bytes (32 BF16 values),
// 8-row groups 512 bytes apart (tcgen05 shared-memory descriptor, version 1, swizzle mode 4).
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}
__device__ __forceinline__ void oz_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void oz_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(oz_smem(bar))
               : "memory");
}
__device__ __forceinline__ void oz_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void oz_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 16 consecutive TMEM columns of this thread's lane (no wait: see oz_ld_wait)
__device__ __forceinline__ void oz_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void oz_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void oz_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

// ---------------------------------------------------------------- slicing
// Operand view: element (b, r, k) at base[b * sb + r * sr + k * sk] (doubles).  The slice planes
// are laid out [p][b][r][Kp] (BF16, K contiguous, Kp a multiple of 32, zero past K) and the
// exponents [b][r].
struct OzView {
  const double* base;
  long long sb, sr, sk;
  int nb, R, K;
};

__device__ __forceinline__ int oz_biased_exp(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7ff);
}

// exponent of every row: e = (largest biased exponent of the row) - 1023 + 1, so that all
// |x| < 2^e; rows of zeros (or subnormals only) get the sentinel -2000
__global__ void oz_rowexp_kernel(OzView v, int* ex) {
  const int b = blockIdx.y;
  const double* base = v.base + (size_t)b * v.sb;
  if (v.sk == 1) {
    // one warp per row, reading along k
    const int warps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * warps + wid;
    if (r >= v.R) return;
    int m = 0;
    for (int k = lane; k < v.K; k += 32) m = max(m, oz_biased_exp(base[(size_t)r * v.sr + k]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) ex[(size_t)b * v.R + r] = m == 0 ? -2000 : m - 1023 + 1;
  } else {
    // one thread per row, threads of a warp on consecutive rows
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= v.R) return;
    int m = 0;
    for (int k = 0; k < v.K; ++k) m = max(m, oz_biased_exp(base[(size_t)r * v.sr + (size_t)k * v.sk]));
    ex[(size_t)b * v.R + r] = m == 0 ? -2000 : m - 1023 + 1;
  }
}

// fixed-point value F = round(x 2^(FB - e)) of |x| < 2^e (|F| <= 2^FB), FB = 6 + 7 (S - 1), by
// integer operations
constexpr int OZ_FB = 6 + 7 * (OZ_S - 1);
__device__ __forceinline__ long long oz_fixed(double x, int e) {
  const long long bits = __double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7ff);
  if (be == 0 || e <= -1000) return 0;                       // zero or subnormal
  const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);   // x = mant 2^(be - 1075)
  // F = mant 2^(be - 1075 + FB - e); the shift is right by sh = e + 1075 - FB - be >= 5
  const int sh = e + 1075 - OZ_FB - be;
  long long f = sh >= 63 ? 0 : ((mant + (1LL << (sh - 1))) >> sh);
  return bits < 0 ? -f : f;
}

// digits of F: d_0 = round(F 2^-(FB - 6)), then the remainder in base 2^7, balanced (|d| <= 64)
__device__ __forceinline__ void oz_digits(long long F, int (&d)[OZ_S]) {
#pragma unroll
  for (int p = 0; p < OZ_S - 1; ++p) {
    const int sh = 7 * (OZ_S - 1 - p);
    const long long q = (F + (1LL << (sh - 1))) >> sh;
    d[p] = (int)q;
    F -= q << sh;
  }
  d[OZ_S - 1] = (int)F;
}

// d 2^(-7p) as BF16 (exact: |d| <= 64 and 2^(-42) is a normal float)
__device__ __forceinline__ __nv_bfloat16 oz_digit_bf16(int d, int p) {
  return __float2bfloat16_rn((float)d * __uint_as_float((uint32_t)(127 - 7 * p) << 23));
}
// the row exponents of an operand whose rows are contiguous (sr == 1) and long along k: the
// biased maxima of (row, 64-long piece of k) go into ex by atomicMax (ex zeroed before), then
// oz_rowexp_fix turns them into exponents; threads of a warp on consecutive rows
__global__ void oz_rowexp_split_kernel(OzView v, int kc, int* ex) {
  const int b = blockIdx.z;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= v.R) return;
  const double* base = v.base + (size_t)b * v.sb + (size_t)r * v.sr;
  const int k0 = blockIdx.y * kc, k1 = min(v.K, k0 + kc);
  int m = 0;
  for (int k = k0; k < k1; ++k) m = max(m, oz_biased_exp(__ldg(base + (size_t)k * v.sk)));
  if (m) atomicMax(ex + (size_t)b * v.R + r, m);
}
__global__ void oz_rowexp_fix_kernel(long long n, int* ex) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) ex[i] = ex[i] == 0 ? -2000 : ex[i] - 1023 + 1;
}
// 32 (r) x 32 (k) tiles through shared memory: loads are coalesced along the operand's
// contiguous direction, plane stores along k
__global__ void oz_slice_kernel(OzView v, const int* ex, __nv_bfloat16* planes, int Kp) {
  __shared__ double tile[32][33];
  const int b = blockIdx.z;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  const double* base = v.base + (size_t)b * v.sb;
  for (int j = ty; j < 32; j += 8) {
    if (v.sk == 1) {   // k contiguous: threads along k
      const int r = r0 + j, k = k0 + tx;
      tile[j][tx] = (r < v.R && k < v.K) ? base[(size_t)r * v.sr + k] : 0.0;
    } else {           // threads along r
      const int r = r0 + tx, k = k0 + j;
      tile[tx][j] = (r < v.R && k < v.K) ? base[(size_t)r * v.sr + (size_t)k * v.sk] : 0.0;
    }
  }
  __syncthreads();
  const size_t plane = (size_t)v.nb * v.R * Kp;
  for (int j = ty; j < 32; j += 8) {
    const int r = r0 + j, k = k0 + tx;
    if (r >= v.R || k >= Kp) continue;
    const int e = ex[(size_t)b * v.R + r];
    int d[OZ_S];
    oz_digits(oz_fixed(tile[j][tx], e), d);
    const size_t o = ((size_t)b * v.R + r) * Kp + k;
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) planes[p * plane + o] = oz_digit_bf16(d[p], p);
  }
}

// Fused exponent and digit passes.  Rows along k (sk == 1): one warp per row reads it twice (the
// second read from L1/L2) and writes the planes along k.  Rows along r (sr == 1) with K <= 128: a
// CTA stages 32 rows x K in shared memory, takes the row maxima there and writes the planes.
__global__ void oz_slice_rows_kernel(OzView v, int* ex, __nv_bfloat16* planes, int Kp) {
  const int warps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.y;
  const int r = blockIdx.x * warps + wid;
  if (r >= v.R) return;
  const double* row = v.base + (size_t)b * v.sb + (size_t)r * v.sr;
  int m = 0;
  for (int k = lane; k < v.K; k += 32) m = max(m, oz_biased_exp(row[k]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int e = m == 0 ? -2000 : m - 1023 + 1;
  if (lane == 0) ex[(size_t)b * v.R + r] = e;
  const size_t plane = (size_t)v.nb * v.R * Kp;
  const size_t o0 = ((size_t)b * v.R + r) * Kp;
  for (int k = lane; k < Kp; k += 32) {
    int d[OZ_S];
    oz_digits(oz_fixed(k < v.K ? row[k] : 0.0, e), d);
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) planes[p * plane + o0 + k] = oz_digit_bf16(d[p], p);
  }
}

__global__ void oz_slice_cols_kernel(OzView v, int* ex, __nv_bfloat16* planes, int Kp) {
  __shared__ double tile[128][33];   // [k][r]
  __shared__ int se[32];
  const int b = blockIdx.y, r0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const double* base = v.base + (size_t)b * v.sb;
  for (int k = ty; k < Kp; k += 8) {
    const int r = r0 + tx;
    tile[k][tx] = (r < v.R && k < v.K) ? base[(size_t)r * v.sr + (size_t)k * v.sk] : 0.0;
  }
  __syncthreads();
  if (ty == 0) {
    int m = 0;
    for (int k = 0; k < v.K; ++k) m = max(m, oz_biased_exp(tile[k][tx]));
    const int e = m == 0 ? -2000 : m - 1023 + 1;
    se[tx] = e;
    if (r0 + tx < v.R) ex[(size_t)b * v.R + r0 + tx] = e;
  }
  __syncthreads();
  const size_t plane = (size_t)v.nb * v.R * Kp;
  for (int j = ty; j < 32; j += 8) {
    const int r = r0 + j;
    if (r >= v.R) continue;
    const size_t o0 = ((size_t)b * v.R + r) * Kp;
    for (int k = tx; k < Kp; k += 32) {
      int d[OZ_S];
      oz_digits(oz_fixed(tile[k][j], se[j]), d);
#pragma unroll
      for (int p = 0; p < OZ_S; ++p) planes[p * plane + o0 + k] = oz_digit_bf16(d[p], p);
    }
  }
}

// ---------------------------------------------------------------- the product kernel
struct OzParams {
  int M, N, K, Kp;          // per product; Kp: padded K of the planes (multiple of 32)
  int nbA, nbB;             // distinct A / B operands (planes per operand: OZ_S)
  int bmap;                 // B operand of product b: b, b^1, b>>1 (or 0 when nbB == 1)
  int nsplit;               // split of K across CTAs: one OZ_KC chunk each
  int nfast;                // 1: blockIdx.x runs over N tiles (the CTAs that share an A tile run
                            //    together and read its planes from L2), 0: over M tiles
  const int *exA, *exB;     // exponents [nbA][M], [nbB][N]
  double alpha, beta;
  int amode, bmode;         // alpha 1 / -1 / other, beta 0 / 1 / other (see oz_out)
  double* C;                // nsplit == 1: C_b = C + b*sC, leading dimension ldc
  long long ldc, sC;
  double* part;             // nsplit > 1: partials ((b*nsplit + s) * M * N) + i + j*M
};

// x 2^e2 for an integer x, rounded to nearest (even) into a double, by integer operations (the
// FP64 pipes of this GPU are slow); results below the normal range flush to zero
__device__ __forceinline__ double oz_i64_to_f64(long long x, int e2) {
  if (x == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)x & 0x8000000000000000ULL;
  const unsigned long long a = x < 0 ? 0ULL - (unsigned long long)x : (unsigned long long)x;
  const int lz = __clzll((long long)a);
  const unsigned long long m = a << lz;                       // leading one at bit 63
  // keep bits 63..11, rounded to nearest even: add 2^10 - 1 and the bit that becomes the last one
  const unsigned long long r = m + (0x3FFULL + ((m >> 11) & 1ULL));
  const int carry = r < m ? 1 : 0;                            // the rounding carried past bit 63
  const unsigned long long mant = carry ? (1ULL << 52) : (r >> 11);   // 53 bits, leading one at 52
  const int ex = 63 - lz + e2 + carry;                        // value = mant 2^(ex - 52)
  if (ex + 1023 <= 0) return 0.0;
  if (ex + 1023 >= 2047) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ULL));
  // the leading one of mant adds the last unit of the biased exponent
  return __longlong_as_double((long long)(sgn | (mant + ((unsigned long long)(ex + 1022) << 52))));
}

// round(f 2^sc) for the FP32 value with bits fb (|f 2^sc| < 2^62), by integer operations (a
// conversion of 64-bit width would run on the FP64 pipes); ties round away from zero
__device__ __forceinline__ long long oz_f32_scaled_ll(uint32_t fb, int sc) {
  const int e = (int)((fb >> 23) & 0xffu);
  if (e == 0) return 0;                                        // zero (or below 2^-126)
  const long long m = (long long)((fb & 0x7fffffu) | 0x800000u);   // f = m 2^(e - 150)
  const int sh = e - 150 + sc;
  long long r;
  if (sh >= 0) r = m << sh;
  else if (sh < -25) r = 0;
  else r = (m + (1LL << (-sh - 1))) >> (-sh);
  return (fb >> 31) ? -r : r;
}
// alpha v + beta c with the modes of alpha (0: 1, 1: -1, 2: other) and beta (0: 0, 1: 1, 2:
// other) decided on the host: at most one FP64 operation per element (the FP64 pipes of this
// GPU are slow)
__device__ __forceinline__ double oz_out(double v, double c, int amode, int bmode, double alpha, double beta) {
  if (amode == 1) v = __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ULL);
  else if (amode == 2) v *= alpha;
  if (bmode == 1) return c + v;
  if (bmode == 2) return fma(beta, c, v);
  return v;
}

// One output element from its five accumulators: groups 0..3 hold exact multiples of 2^(-7g)
// below 2^(24 - 7g), so their values times 2^(7g) are integers that fit 32 bits; they join in
// V = sum_g acc_g 2^21 (units 2^-21, |V| < 2^43) and, with the tail groups (FP32, below 2^-28 of
// the leading scale) in units of 2^-40, in one 64-bit integer W = V 2^19 + round(tail 2^40)
// (|W| < 2^62), rounded once to FP64 with the scales 2^(ea + eb - 12).
__device__ __forceinline__ double oz_combine(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t at, int ea,
                                             int eb) {
  if (ea < -1000 || eb < -1000) return 0.0;
  const long long g0 = __float2int_rz(__uint_as_float(a0));
  const long long g1 = __float2int_rz(__uint_as_float(a1) * 128.0f);
  const long long g2 = __float2int_rz(__uint_as_float(a2) * 16384.0f);
  const long long g3 = __float2int_rz(__uint_as_float(a3) * 2097152.0f);
  const long long V = (g0 << 21) + (g1 << 14) + (g2 << 7) + g3;
  const long long W = (V << 19) + oz_f32_scaled_ll(at, 40);
  return oz_i64_to_f64(W, ea + eb - 12 - 40);
}

template <int BN, int ST>
__global__ void __launch_bounds__(OZ_THREADS, 3 - ST)
    oz_mma_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const OzParams p) {
  using TL = OzTile<BN, ST>;
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + ST * TL::STAGE);
  uint64_t* done = full + ST;
  uint32_t* tslot = (uint32_t*)(done + ST);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = (p.nfast ? blockIdx.y : blockIdx.x) * OZ_BM, n0 = (p.nfast ? blockIdx.x : blockIdx.y) * BN;
  const int b = blockIdx.z / p.nsplit, sp = blockIdx.z % p.nsplit;
  const int bA = p.nbA == 1 ? 0 : b;
  const int bB = p.nbB == 1 ? 0 : (p.bmap == BMAP_XOR1 ? (b ^ 1) : (p.bmap == BMAP_SHR1 ? (b >> 1) : b));
  // one exactness chunk of K per CTA (longer K is split across CTAs)
  const int kbeg = sp * OZ_KC, kend = min(p.Kp, kbeg + OZ_KC);
  const int nk = (kend - kbeg) / OZ_BK;           // slices (kbeg, kend multiples of 32)

  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      oz_mbar_init(&full[s], 1);
      oz_mbar_init(&done[s], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(oz_smem(tslot)),
                 "r"(TL::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  oz_fence_before();
  __syncthreads();
  oz_fence_after();
  const uint32_t tmem = *tslot;
  // D FP32; A, B BF16, K-major; N = BN; M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(OZ_BM >> 4) << 24);
  auto planeA = [&](int s, int q) { return sm + s * TL::STAGE + q * OZ_PLANE_A; };
  auto planeB = [&](int s, int q) { return sm + s * TL::STAGE + OZ_S * OZ_PLANE_A + q * TL::PLANE_B; };
  auto issue_loads = [&](int kt) {
    const int s = kt % ST;
    oz_expect_tx(&full[s], TL::STAGE);
    const int kx = kbeg + kt * OZ_BK;
#pragma unroll
    for (int q = 0; q < OZ_S; ++q) {
      oz_tma3(planeA(s, q), &mapA, kx, m0, q * p.nbA + bA, &full[s]);
      oz_tma3(planeB(s, q), &mapB, kx, n0, q * p.nbB + bB, &full[s]);
    }
  };

  const int wq = warp & 3, wh = warp >> 2;   // TMEM lane quarter and column half of this warp
  bool ok = true;
  int issued = 0, committed = 0;
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt % ST;
    if (tid == 0) {
      // keep ST - 1 slices in flight ahead of this one; a stage is reloaded once the products
      // of its previous slice have completed
      for (; ok && issued < nk && issued <= kt + ST - 1; ++issued) {
        if (issued >= ST && !oz_wait(&done[issued % ST], ((issued - ST) / ST) & 1)) {
          ok = false;
          break;
        }
        issue_loads(issued);
      }
      if (ok && !oz_wait(&full[s], (kt / ST) & 1)) ok = false;
      if (ok) {
        oz_fence_after();
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {   // two K = 16 steps per 32-wide slice: 32 bytes apart
#pragma unroll
          for (int pa = 0; pa < OZ_S; ++pa) {
#pragma unroll
            for (int pb = 0; pb < OZ_S - pa; ++pb) {
              const int t = pa + pb, g = t < OZ_NACC - 1 ? t : OZ_NACC - 1;
              // the first product into each accumulator overwrites it
              const bool first = kt == 0 && kk == 0 && pa == 0 && (g < OZ_NACC - 1 || t == OZ_NACC - 1);
              oz_mma(tmem + (uint32_t)(g * BN), oz_desc(oz_smem(planeA(s, pa)) + 32 * kk),
                     oz_desc(oz_smem(planeB(s, pb)) + 32 * kk), idesc, first ? 0u : 1u);
            }
          }
        }
        oz_commit(&done[s]);
        committed = kt + 1;
      }
    }
  }
  if (nk > 0 && ok && tid == 0) ok = oz_wait(&done[(nk - 1) % ST], ((nk - 1) / ST) & 1);
  ok = __syncthreads_and(ok) != 0;
  if (ok) {
    oz_fence_after();
    const int row = m0 + 32 * wq + lane;
    const int ea = row < p.M ? p.exA[(size_t)bA * p.M + row] : 0;
    const uint32_t lanes = (uint32_t)(32 * wq) << 16;
#pragma unroll 1
    for (int h = 0; h < BN / 16; ++h) {
      // warps w and w + 4 take BN / 2 columns each, in pieces of 8
      const uint32_t col0 = (uint32_t)((BN / 2) * wh + 8 * h);
      uint32_t ra[8], rb[8], rc[8], rd[8], rt[8];
      if (nk > 0) {
        oz_ld8(tmem + lanes + col0, ra);
        oz_ld8(tmem + lanes + (uint32_t)BN + col0, rb);
        oz_ld8(tmem + lanes + (uint32_t)(2 * BN) + col0, rc);
        oz_ld8(tmem + lanes + (uint32_t)(3 * BN) + col0, rd);
        oz_ld8(tmem + lanes + (uint32_t)(4 * BN) + col0, rt);
        oz_ld_wait();
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) ra[j] = rb[j] = rc[j] = rd[j] = rt[j] = 0u;
      }
      if (row >= p.M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = n0 + (int)col0 + j;
        if (col < p.N) {
          const double v = oz_combine(ra[j], rb[j], rc[j], rd[j], rt[j], ea, p.exB[(size_t)bB * p.N + col]);
          if (p.nsplit == 1) {
            double* c = p.C + (size_t)b * p.sC + (size_t)col * p.ldc + row;
            *c = oz_out(v, p.bmode ? *c : 0.0, p.amode, p.bmode, p.alpha, p.beta);
          } else {
            p.part[((size_t)b * p.nsplit + sp) * ((size_t)p.M * p.N) + (size_t)col * p.M + row] = v;
          }
        }
      }
    }
  } else if (tid == 0) {
    // give the products and copies already issued a bounded chance to land, then report
    atomicExch(&g_oz_status, HODLR_ETIMEOUT);
    for (int kt = committed - 1; kt >= 0 && kt >= committed - ST; --kt) oz_wait(&done[kt % ST], (kt / ST) & 1);
    for (int kt = issued - 1; kt >= committed && kt >= 0; --kt) oz_wait(&full[kt % ST], (kt / ST) & 1);
  }
  oz_fence_before();
  __syncthreads();
  if (warp == 0) {
    oz_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TL::TCOLS) : "memory");
  }
}

// ---------------------------------------------------------------- persistent short-K kernel
// For K <= 128 (at most four 32-wide slices) the product is bound by its FP64 C traffic and by
// the integer epilogue, and a CTA per tile serialises loads, products and epilogue.  Here one CTA
// per SM loops over tiles (N tile fastest, so that the CTAs sharing an A tile run together) with
// three roles:
//   warp 8 (one thread): TMA loads of the slices into a ring of three 70 KB stages;
//   warp 9 (one thread): the 56 MMAs of each slice into one of two TMEM accumulator sets;
//   warps 0..7: the epilogue of the previous tile (warp w reads TMEM lanes 32 (w % 4) .. + 31 and
//               columns 16 (w / 4) .. + 15, releases the accumulator set, then updates C in FP64).
// Every wait is bounded; a role whose wait gives up raises an abort flag that stops the others,
// records HODLR_ETIMEOUT, waits (bounded) for what it issued and lets the CTA free its TMEM.
constexpr int WS_BN = 32, WS_NST = 3, WS_THREADS = 320;
template <int BN, int NST> struct WsTile {
  static constexpr int PLANE_B = BN * OZ_BK * 2;
  static constexpr int STAGE = OZ_S * (OZ_PLANE_A + PLANE_B);   // 70 KB (BN 32), 77 KB (BN 48)
  static constexpr int SMEM = NST * STAGE + 1024 + 256;
  static constexpr int EPC = BN / 2;                             // epilogue columns per warp
};
constexpr int WS_SMEM = WsTile<WS_BN, WS_NST>::SMEM;

__device__ __forceinline__ void oz_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(oz_smem(bar)) : "memory");
}

// Work items (product b, K chunk sp, row tile, column tile), the tiles of the smaller operand
// fastest; an item covers
// one 512-long chunk of K (at most 16 slices) and writes C (one chunk) or its split-K partial.
// Tiles 128 x 32 with three stages serve K <= 128; tiles 128 x 48 with two stages serve longer K
// (the accumulator set of the next item is filled while the epilogue drains this one).
template <int BN, int NST>
__global__ void __launch_bounds__(WS_THREADS, 1)
    oz_mma_ws_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                     const OzParams p, int ntm, int ntn, int ntiles) {
  using TL = WsTile<BN, NST>;
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + NST * TL::STAGE);
  uint64_t* empty = full + NST;
  uint64_t* accf = empty + NST;
  uint64_t* acce = accf + 2;
  volatile int* abort_flag = (volatile int*)(acce + 2);
  uint32_t* tslot = (uint32_t*)(acce + 2) + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      oz_mbar_init(&full[s], 1);
      oz_mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      oz_mbar_init(&accf[a], 1);
      oz_mbar_init(&acce[a], 8);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(oz_smem(tslot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  oz_fence_before();
  __syncthreads();
  oz_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(OZ_BM >> 4) << 24);
  auto planeA = [&](int s, int q) { return sm + s * TL::STAGE + q * OZ_PLANE_A; };
  auto planeB = [&](int s, int q) { return sm + s * TL::STAGE + OZ_S * OZ_PLANE_A + q * TL::PLANE_B; };
  // the larger operand's tile is shared by the items that run together (p.nfast: column tiles
  // fastest, A shared; else row tiles fastest, B shared)
  auto decode = [&](int t, int& b, int& m0, int& n0, int& sp) {
    int tm, tn, r2;
    if (p.nfast) {
      tn = t % ntn;
      tm = (t / ntn) % ntm;
      r2 = t / ntn / ntm;
    } else {
      tm = t % ntm;
      tn = (t / ntm) % ntn;
      r2 = t / ntm / ntn;
    }
    m0 = tm * OZ_BM;
    n0 = tn * BN;
    sp = r2 % p.nsplit;
    b = r2 / p.nsplit;
  };
  auto slices = [&](int sp) { return min(OZ_KC / OZ_BK, (p.Kp - sp * OZ_KC) / OZ_BK); };
  int issued = 0, committed = 0;   // producer / MMA progress (slices), for the drain after an abort
  if (warp == 8) {
    if (lane == 0) {
      // ---------------- producer
      int it = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        int b, m0, n0, sp;
        decode(t, b, m0, n0, sp);
        const int bA = p.nbA == 1 ? 0 : b;
        const int bB = p.nbB == 1 ? 0 : (p.bmap == BMAP_XOR1 ? (b ^ 1) : (p.bmap == BMAP_SHR1 ? (b >> 1) : b));
        const int nk = slices(sp);
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int s = it % NST, u = it / NST;
          if (u > 0 && !oz_wait(&empty[s], (u - 1) & 1)) { *abort_flag = 1; break; }
          oz_expect_tx(&full[s], TL::STAGE);
          const int kx = (sp * (OZ_KC / OZ_BK) + kt) * OZ_BK;
#pragma unroll
          for (int q = 0; q < OZ_S; ++q) {
            oz_tma3(planeA(s, q), &mapA, kx, m0, q * p.nbA + bA, &full[s]);
            oz_tma3(planeB(s, q), &mapB, kx, n0, q * p.nbB + bB, &full[s]);
          }
          issued = it + 1;
        }
      }
    }
  } else if (warp == 9) {
    if (lane == 0) {
      // ---------------- products
      int it = 0, j = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++j) {
        const int a = j & 1;
        if (j >= 2 && !oz_wait(&acce[a], ((j >> 1) - 1) & 1)) { *abort_flag = 1; break; }
        oz_fence_after();
        int b, m0, n0, sp;
        decode(t, b, m0, n0, sp);
        const int nk = slices(sp);
        bool ok = true;
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int s = it % NST;
          if (!oz_wait(&full[s], (it / NST) & 1)) { ok = false; break; }
          oz_fence_after();
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
            for (int pa = 0; pa < OZ_S; ++pa) {
#pragma unroll
              for (int pb = 0; pb < OZ_S - pa; ++pb) {
                const int tt = pa + pb, g = tt < OZ_NACC - 1 ? tt : OZ_NACC - 1;
                const bool first = kt == 0 && kk == 0 && pa == 0 && (g < OZ_NACC - 1 || tt == OZ_NACC - 1);
                oz_mma(tmem + (uint32_t)(256 * a + g * BN), oz_desc(oz_smem(planeA(s, pa)) + 32 * kk),
                       oz_desc(oz_smem(planeB(s, pb)) + 32 * kk), idesc, first ? 0u : 1u);
              }
            }
          }
          oz_commit(&empty[s]);
          committed = it + 1;
        }
        if (!ok) { *abort_flag = 1; break; }
        oz_commit(&accf[a]);
      }
    }
  } else {
    // ---------------- epilogue: warp w reads TMEM lanes 32 (w % 4) .., columns EPC (w / 4) ..
    constexpr int EPC = TL::EPC;
    const int wq = warp & 3, wh = warp >> 2;
    const uint32_t lanes = (uint32_t)(32 * wq) << 16;
    int j = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
      if (__any_sync(0xffffffffu, *abort_flag)) break;
      const int a = j & 1;
      bool ok = oz_wait(&accf[a], (j >> 1) & 1);
      if (!__all_sync(0xffffffffu, ok)) { *abort_flag = 1; break; }
      oz_fence_after();
      int b, m0, n0, sp;
      decode(t, b, m0, n0, sp);
      const int bA = p.nbA == 1 ? 0 : b;
      const int bB = p.nbB == 1 ? 0 : (p.bmap == BMAP_XOR1 ? (b ^ 1) : (p.bmap == BMAP_SHR1 ? (b >> 1) : b));
      const int row = m0 + 32 * wq + lane;
      const int c0 = n0 + EPC * wh;
      const int ea = row < p.M ? p.exA[(size_t)bA * p.M + row] : -2000;
      double v[EPC];
#pragma unroll
      for (int h = 0; h < EPC / 8; ++h) {
        uint32_t ra[8], rb[8], rc[8], rd[8], rt[8];
        const uint32_t base = tmem + lanes + (uint32_t)(256 * a + EPC * wh + 8 * h);
        oz_ld8(base, ra);
        oz_ld8(base + (uint32_t)BN, rb);
        oz_ld8(base + (uint32_t)(2 * BN), rc);
        oz_ld8(base + (uint32_t)(3 * BN), rd);
        oz_ld8(base + (uint32_t)(4 * BN), rt);
        oz_ld_wait();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int col = c0 + 8 * h + q;
          const int eb = col < p.N ? p.exB[(size_t)bB * p.N + col] : -2000;
          v[8 * h + q] = oz_combine(ra[q], rb[q], rc[q], rd[q], rt[q], ea, eb);
        }
      }
      // the accumulator set is free for the item after next
      oz_fence_before();
      __syncwarp();
      if (lane == 0) oz_arrive(&acce[a]);
      if (row < p.M) {
        if (p.nsplit > 1) {
          double* pp = p.part + ((size_t)b * p.nsplit + sp) * ((size_t)p.M * p.N) + row;
#pragma unroll
          for (int q = 0; q < EPC; ++q)
            if (c0 + q < p.N) pp[(size_t)(c0 + q) * p.M] = v[q];
        } else {
          double* c = p.C + (size_t)b * p.sC + row;
          double cv[EPC];
          if (p.bmode != 0) {
#pragma unroll
            for (int q = 0; q < EPC; ++q) cv[q] = c0 + q < p.N ? c[(size_t)(c0 + q) * p.ldc] : 0.0;
          }
#pragma unroll
          for (int q = 0; q < EPC; ++q) {
            if (c0 + q >= p.N) continue;
            c[(size_t)(c0 + q) * p.ldc] = oz_out(v[q], cv[q], p.amode, p.bmode, p.alpha, p.beta);
          }
        }
      }
    }
  }
  __syncthreads();
  if (*abort_flag) {
    // wait (bounded) for the copies and products already issued before the TMEM is freed
    if (tid == 0) atomicExch(&g_oz_status, HODLR_ETIMEOUT);
    if (warp == 8 && lane == 0)
      for (int it = issued - 1; it >= 0 && it >= issued - NST; --it) oz_wait(&full[it % NST], (it / NST) & 1);
    if (warp == 9 && lane == 0 && committed > 0)
      oz_wait(&empty[(committed - 1) % NST], ((committed - 1) / NST) & 1);
  }
  oz_fence_before();
  __syncthreads();
  if (warp == 0) {
    oz_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ---------------------------------------------------------------- fused digit production
// The two kernels below read the FP64 operands themselves and store the digit planes straight
// into shared memory, in the layout the TMA loads give (K-major rows of 64 bytes; the 16-byte
// chunk c of row r sits at chunk c ^ ((r >> 1) & 3), the 64-byte swizzle), so that the planes
// never pass through HBM.  The exponents come from a pass of their own (oz_exp_chunks_kernel):
// one per row over the whole K of a short product, one per row and 512-long chunk of K for a
// long one (each chunk's exact group sums are scaled by its own exponents).

// Balanced digits by one biased addition: with C' = 64 sum_{p=1..6} 2^(7(6-p)),
// F + C' = d_0 2^42 + sum_{p=1..6} u_p 2^(7(6-p)), u_p in [0, 127], so that d_0 in [-64, 64] and
// d_p = u_p - 64 in [-64, 63] (|F| <= 2^48).  A digit becomes the FP32 value d 2^(-7p) through a
// float whose exponent field carries the scale: (2^(23-7p) + u 2^(-7p)) - (2^(23-7p) + 64 2^(-7p)),
// exact, and exact again as BF16 (at most seven significant bits).
constexpr long long OZ_CLOW =
    64LL * ((1LL << 35) + (1LL << 28) + (1LL << 21) + (1LL << 14) + (1LL << 7) + 1LL);

__device__ __forceinline__ float oz_dig_f(uint32_t u, int p) {
  const uint32_t ef = (uint32_t)(150 - 7 * p) << 23;
  return __uint_as_float(ef | u) - __uint_as_float(ef | 64u);
}
__device__ __forceinline__ void oz_digits_f(double x, int e, float (&f)[OZ_S]) {
  const long long G = oz_fixed(x, e) + OZ_CLOW;
  const uint32_t hi = (uint32_t)((unsigned long long)G >> 32), lo = (uint32_t)G;
  f[0] = oz_dig_f((uint32_t)((int)(G >> 42) + 64), 0);
  f[1] = oz_dig_f((hi >> 3) & 127u, 1);
  f[2] = oz_dig_f(__funnelshift_r(lo, hi, 28) & 127u, 2);
  f[3] = oz_dig_f((lo >> 21) & 127u, 3);
  f[4] = oz_dig_f((lo >> 14) & 127u, 4);
  f[5] = oz_dig_f((lo >> 7) & 127u, 5);
  f[6] = oz_dig_f(lo & 127u, 6);
}
// digits of 8 consecutive values of row r (k = 8q .. 8q + 7 of a 32-wide slice) into the 16-byte
// chunk q of that row in each of the seven planes (plane p at slice0 + p * pstride)
__device__ __forceinline__ void oz_put8(const double (&x)[8], int e, unsigned char* slice0, int r, int q,
                                        int pstride) {
  uint32_t w[OZ_S][4];
#pragma unroll
  for (int i = 0; i < 8; i += 2) {
    float fa[OZ_S], fb[OZ_S];
    oz_digits_f(x[i], e, fa);
    oz_digits_f(x[i + 1], e, fb);
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) {
      __nv_bfloat162 h = __floats2bfloat162_rn(fa[p], fb[p]);
      w[p][i >> 1] = *reinterpret_cast<uint32_t*>(&h);
    }
  }
  const int off = r * 64 + ((q ^ ((r >> 1) & 3)) << 4);
#pragma unroll
  for (int p = 0; p < OZ_S; ++p)
    *reinterpret_cast<uint4*>(slice0 + p * pstride + off) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}
__device__ __forceinline__ void oz_fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// exponent of every row over chunks of `chunk` values of k: ex[(b * nch + c) * R + r]
__global__ void oz_exp_chunks_kernel(OzView v, int chunk, int nch, int* ex) {
  const int b = blockIdx.z, c = blockIdx.y;
  const double* base = v.base + (size_t)b * v.sb;
  const int k0 = c * chunk, k1 = min(v.K, k0 + chunk);
  int m = 0, r;
  if (v.sk == 1) {   // a warp per row, along k
    const int lane = threadIdx.x & 31;
    r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= v.R) return;
    const double* row = base + (size_t)r * v.sr;
    for (int k = k0 + lane; k < k1; k += 32) m = max(m, oz_biased_exp(__ldg(row + k)));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane) return;
  } else {           // a thread per row, threads on consecutive rows
    r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= v.R) return;
    for (int k = k0; k < k1; ++k) m = max(m, oz_biased_exp(__ldg(base + (size_t)r * v.sr + (size_t)k * v.sk)));
  }
  ex[((size_t)b * nch + c) * v.R + r] = m == 0 ? -2000 : m - 1023 + 1;
}

// ---------------------------------------------------------------- fused long-K products
// C_b = alpha op(A_b) op(B_b) + beta C_b where the rows of op(A) and the columns of op(B) are
// contiguous along K (A^T B of column-major operands: the Gram and projection products of the
// sketch), M <= 128, K long.  A CTA takes BN columns of one product over a range of 512-long
// chunks of K:
//   warps 5..15 (producers): read 32-wide slices of the M rows of op(A) and the BN columns of
//       op(B) in FP64, cut them into digits with the chunk's exponents and store the 14 planes
//       of the slice into one of two shared-memory stages;
//   warp 4 (one thread): the 56 MMAs of each slice into a TMEM accumulator set (two sets used
//       alternately per chunk when they fit in the 512 columns, else one);
//   warps 0..3: after each chunk, the integer epilogue of its accumulators (TMEM lane quarter
//       w) added in FP64 to the CTA's running sums in shared memory; at the end the sums go to
//       C (a single K range) or to the split-K partials.
// Two tiles: AR = 128 rows of A planes with BN = 48 (two accumulator sets), and for M <= 64,
// AR = 64 with BN = 80 (one set): the MMA still reads 128 rows, the upper 64 from whatever
// follows the plane in shared memory, which reaches only rows of D that are never read.  So do
// the unwritten rows beyond M and columns beyond N.  Every wait is bounded (abort flag, status
// HODLR_ETIMEOUT, drain of the issued MMAs before the TMEM is freed).
constexpr int AT_NPROD = 11;
constexpr int AT_THREADS = 32 * (5 + AT_NPROD);
template <int AR, int BN> struct AtTile {
  static constexpr int PLANE_A = AR * 64;                      // bytes per plane and slice
  static constexpr int PLANE_B = BN * 64;
  static constexpr int STAGE = OZ_S * (PLANE_A + PLANE_B);
  static constexpr int SUMS = AR * BN * 8;
  static constexpr int SMEM = 2 * STAGE + SUMS + 1024 + 256;
  static constexpr int NSETS = 2 * OZ_NACC * BN <= 512 ? 2 : 1;
  static constexpr int SETW = NSETS == 2 ? 256 : 0;            // TMEM columns between sets
  // every (row, 8 values) task of a slice has a producer thread, two tasks each
  static_assert(4 * (AR + BN) <= 2 * 32 * AT_NPROD, "producer threads");
};

struct AtParams {
  const double *A, *B;     // row i of op(A_b): A + bA sA + i lda; column j of op(B_b): B + bB sB + j ldb
  long long lda, sA, ldb, sB;
  int M, N, K, nbA, nbB, bmap;
  int nch, cpr, nrange;    // 512-long chunks of K; chunks per range; ranges (split of K across CTAs)
  const int *exA, *exB;    // [nbA][nch][M], [nbB][nch][N]
  double alpha, beta;
  int amode, bmode;        // see oz_out
  double* C;
  long long ldc, sC;
  double* part;            // nrange > 1: partials ((b * nrange + range) * M * N) + i + j * M
};

template <int AR, int BN>
__global__ void __launch_bounds__(AT_THREADS, 1) oz_atb_kernel(const AtParams p) {
  using TL = AtTile<AR, BN>;
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  double* sums = (double*)(sm + 2 * TL::STAGE);   // [column][AR rows]
  uint64_t* full = (uint64_t*)(sm + 2 * TL::STAGE + TL::SUMS);
  uint64_t* empty = full + 2;
  uint64_t* accf = empty + 2;
  uint64_t* acce = accf + 2;
  volatile int* abort_flag = (volatile int*)(acce + 2);
  uint32_t* tslot = (uint32_t*)(acce + 2) + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int part = blockIdx.x, range = blockIdx.y, b = blockIdx.z;
  const int bA = p.nbA == 1 ? 0 : b;
  const int bB = p.nbB == 1 ? 0 : (p.bmap == BMAP_XOR1 ? (b ^ 1) : (p.bmap == BMAP_SHR1 ? (b >> 1) : b));
  const int n0 = part * BN, nv = min(BN, p.N - n0);
  const int c0 = range * p.cpr, c1 = min(p.nch, c0 + p.cpr);
  const int Kp = ((p.K + OZ_BK - 1) / OZ_BK) * OZ_BK;
  const int nsl = (min(c1 * OZ_KC, Kp) - c0 * OZ_KC) / OZ_BK;   // 32-wide slices of this range
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      oz_mbar_init(&full[s], AT_NPROD);
      oz_mbar_init(&empty[s], 1);
      oz_mbar_init(&accf[s], 1);
      oz_mbar_init(&acce[s], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(oz_smem(tslot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int i = tid; i < AR * BN; i += AT_THREADS) sums[i] = 0.0;
  oz_fence_before();
  __syncthreads();
  oz_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(OZ_BM >> 4) << 24);
  int committed = 0;   // MMA progress (slices), for the drain after an abort
  if (warp >= 5) {
    // ---------------- producers: each thread takes at most two of the slice's (row, 8 values)
    // tasks; the loads of slice s + 1 are issued before the digits of slice s are made
    const int ptid = tid - 5 * 32, stride = 32 * AT_NPROD;
    const double* Ab = p.A + (size_t)bA * p.sA;
    const double* Bb = p.B + (size_t)bB * p.sB + (size_t)n0 * p.ldb;
    const int tasks = (p.M + nv) * 4;
    auto load = [&](int s, int t, double (&x)[8]) {
      if (t >= tasks) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = 0.0;
        return -2000;
      }
      const int ks = c0 * (OZ_KC / OZ_BK) + s, ch = ks / (OZ_KC / OZ_BK);
      const int rho = t >> 2, k = ks * OZ_BK + 8 * (t & 3);   // four threads per row: 256 contiguous bytes
      const double* src;
      int e;
      if (rho < p.M) {
        src = Ab + (size_t)rho * p.lda;
        e = __ldg(p.exA + ((size_t)bA * p.nch + ch) * p.M + rho);
      } else {
        src = Bb + (size_t)(rho - p.M) * p.ldb;
        e = __ldg(p.exB + ((size_t)bB * p.nch + ch) * p.N + n0 + rho - p.M);
      }
      if (k + 8 <= p.K && (((uintptr_t)(src + k)) & 15) == 0) {
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
          const double2 v = __ldg(reinterpret_cast<const double2*>(src + k + i));
          x[i] = v.x; x[i + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = k + i < p.K ? __ldg(src + k + i) : 0.0;
      }
      return e;
    };
    auto store = [&](unsigned char* stg, int t, const double (&x)[8], int e) {
      const int rho = t >> 2, q = t & 3;
      if (rho < p.M) oz_put8(x, e, stg, rho, q, TL::PLANE_A);
      else oz_put8(x, e, stg + OZ_S * TL::PLANE_A, rho - p.M, q, TL::PLANE_B);
    };
    double xa[8], xb[8];
    int ea = load(0, ptid, xa), eb = load(0, ptid + stride, xb);
    for (int s = 0; s < nsl; ++s) {
      if (__any_sync(0xffffffffu, *abort_flag)) break;
      double ya[8], yb[8];
      int fa = -2000, fb = -2000;
      if (s + 1 < nsl) {
        fa = load(s + 1, ptid, ya);
        fb = load(s + 1, ptid + stride, yb);
      }
      const int st = s & 1, u = s >> 1;
      if (u > 0) {
        const bool ok = oz_wait(&empty[st], (u - 1) & 1);
        if (!__all_sync(0xffffffffu, ok)) { *abort_flag = 1; break; }
      }
      unsigned char* stg = sm + st * TL::STAGE;
      if (ptid < tasks) store(stg, ptid, xa, ea);
      if (ptid + stride < tasks) store(stg, ptid + stride, xb, eb);
      oz_fence_async_smem();
      __syncwarp();
      if (lane == 0) oz_arrive(&full[st]);
      if (s + 1 < nsl) {
#pragma unroll
        for (int i = 0; i < 8; ++i) { xa[i] = ya[i]; xb[i] = yb[i]; }
        ea = fa; eb = fb;
      }
    }
  } else if (warp == 4) {
    if (lane == 0) {
      // ---------------- products
      for (int s = 0; s < nsl && !*abort_flag; ++s) {
        const int st = s & 1;
        const int ks = c0 * (OZ_KC / OZ_BK) + s;
        const int chl = ks / (OZ_KC / OZ_BK) - c0, a = chl % TL::NSETS;
        const bool first_sl = s == 0 || (ks % (OZ_KC / OZ_BK)) == 0;
        const bool last_sl = s == nsl - 1 || ((ks + 1) % (OZ_KC / OZ_BK)) == 0;
        if (first_sl && chl >= TL::NSETS && !oz_wait(&acce[a], (chl / TL::NSETS - 1) & 1)) {
          *abort_flag = 1;
          break;
        }
        if (!oz_wait(&full[st], (s >> 1) & 1)) { *abort_flag = 1; break; }
        oz_fence_after();
        const unsigned char* stg = sm + st * TL::STAGE;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
          for (int pa = 0; pa < OZ_S; ++pa) {
#pragma unroll
            for (int pb = 0; pb < OZ_S - pa; ++pb) {
              const int t = pa + pb, g = t < OZ_NACC - 1 ? t : OZ_NACC - 1;
              const bool first = first_sl && kk == 0 && pa == 0 && (g < OZ_NACC - 1 || t == OZ_NACC - 1);
              oz_mma(tmem + (uint32_t)(TL::SETW * a + g * BN), oz_desc(oz_smem(stg + pa * TL::PLANE_A) + 32 * kk),
                     oz_desc(oz_smem(stg + OZ_S * TL::PLANE_A + pb * TL::PLANE_B) + 32 * kk), idesc,
                     first ? 0u : 1u);
            }
          }
        }
        oz_commit(&empty[st]);
        if (last_sl) oz_commit(&accf[a]);
        committed = s + 1;
      }
    }
  } else {
    // ---------------- epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31 (rows of this CTA)
    const int row = 32 * warp + lane;
    const uint32_t lanes = (uint32_t)(32 * warp) << 16;
    for (int j = 0; j < c1 - c0; ++j) {
      if (__any_sync(0xffffffffu, *abort_flag)) break;
      const int a = j % TL::NSETS;
      const bool ok = oz_wait(&accf[a], (j / TL::NSETS) & 1);
      if (!__all_sync(0xffffffffu, ok)) { *abort_flag = 1; break; }
      oz_fence_after();
      const int ch = c0 + j;
      const int ea = row < p.M ? __ldg(p.exA + ((size_t)bA * p.nch + ch) * p.M + row) : -2000;
      const int* eB = p.exB + ((size_t)bB * p.nch + ch) * p.N + n0;
#pragma unroll 1
      for (int h = 0; h < BN / 8; ++h) {
        uint32_t ra[8], rb[8], rc[8], rd[8], rt[8];
        const uint32_t base = tmem + lanes + (uint32_t)(TL::SETW * a + 8 * h);
        oz_ld8(base, ra);
        oz_ld8(base + (uint32_t)BN, rb);
        oz_ld8(base + (uint32_t)(2 * BN), rc);
        oz_ld8(base + (uint32_t)(3 * BN), rd);
        oz_ld8(base + (uint32_t)(4 * BN), rt);
        oz_ld_wait();
        if (row < p.M) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int col = 8 * h + q;
            if (col < nv) sums[col * AR + row] += oz_combine(ra[q], rb[q], rc[q], rd[q], rt[q], ea, __ldg(eB + col));
          }
        }
      }
      oz_fence_before();
      __syncwarp();
      if (lane == 0) oz_arrive(&acce[a]);
    }
  }
  __syncthreads();
  if (*abort_flag) {
    if (tid == 0) atomicExch(&g_oz_status, HODLR_ETIMEOUT);
    // the MMAs already issued complete before the TMEM is freed (the producers issue no
    // asynchronous copies)
    if (warp == 4 && lane == 0 && committed > 0) oz_wait(&empty[(committed - 1) & 1], ((committed - 1) >> 1) & 1);
  } else {
    for (int i = tid; i < AR * BN; i += AT_THREADS) {
      const int col = i / AR, row = i % AR;
      if (row >= p.M || col >= nv) continue;
      const double v = sums[i];
      if (p.nrange == 1) {
        double* c = p.C + (size_t)b * p.sC + (size_t)(n0 + col) * p.ldc + row;
        *c = oz_out(v, p.bmode ? *c : 0.0, p.amode, p.bmode, p.alpha, p.beta);
      } else {
        p.part[((size_t)b * p.nrange + range) * ((size_t)p.M * p.N) + (size_t)(n0 + col) * p.M + row] = v;
      }
    }
  }
  oz_fence_before();
  __syncthreads();
  if (warp == 0) {
    oz_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ---------------------------------------------------------------- fused short-K products
// C_b = alpha A_b op(B_b) + beta C_b with A column-major (M x K, consecutive rows adjacent), K at
// most 64 and M large: the peeling updates of Alg. 1 (M block rows, K the rank, N the probe
// columns), bound by the FP64 traffic of C.  One CTA per SM loops over 128-row tiles of A:
//   warps 10..15 (producers): read the tile's rows in FP64 (lanes on consecutive rows), cut
//       them into digits with the row exponents and store all K slices of the seven planes into
//       the A buffer (112 KB), once the MMAs of the previous tile are done with it;
//   warp 8 (one thread): TMA loads of the B planes (sliced beforehand; small and L2-resident)
//       for each 48-column subtile and slice into a ring of three 21 KB stages;
//   warp 9 (one thread): the 56 MMAs of each (subtile, slice) into one of two TMEM sets;
//   warps 0..7: the epilogue of each subtile (warps w and w + 4 share TMEM lane quarter w,
//       24 columns each), with the C loads of the next eight columns issued ahead of their use.
constexpr int AB_BN = 48, AB_NST = 3, AB_KMAX = 64, AB_NPROD = 6;
constexpr int AB_THREADS = 32 * (10 + AB_NPROD);
constexpr int AB_PLANE_B = AB_BN * 64;                                   // 3 KB
constexpr int AB_APLANE = (AB_KMAX / OZ_BK) * OZ_PLANE_A;                // 16 KB: one plane, all slices
constexpr int AB_ABUF = OZ_S * AB_APLANE;                                // 112 KB
constexpr int AB_STAGE = OZ_S * AB_PLANE_B;                              // 21 KB
constexpr int AB_SMEM = AB_ABUF + AB_NST * AB_STAGE + 1024 + 256;

struct AbParams {
  const double* A;        // A_b = A + bA sA, element (i, k) at A_b[i + k lda]
  long long lda, sA;
  int M, N, K, Kp, nbA, nbB, bmap;
  int ntm, ntn, ntiles;   // 128-row tiles per product, 48-column subtiles, tiles in all
  const int *exA, *exB;   // [nbA][M], [nbB][N]
  double alpha, beta;
  int amode, bmode;       // see oz_out
  double* C;
  long long ldc, sC;
};

__global__ void __launch_bounds__(AB_THREADS, 1)
    oz_ab_kernel(const __grid_constant__ CUtensorMap mapB, const AbParams p) {
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* abuf = sm;
  unsigned char* bst = sm + AB_ABUF;
  uint64_t* full = (uint64_t*)(bst + AB_NST * AB_STAGE);
  uint64_t* empty = full + AB_NST;
  uint64_t* accf = empty + AB_NST;
  uint64_t* acce = accf + 2;
  uint64_t* afull = acce + 2;
  uint64_t* afree = afull + 1;
  volatile int* abort_flag = (volatile int*)(afree + 1);
  uint32_t* tslot = (uint32_t*)(afree + 1) + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nk = p.Kp / OZ_BK;   // 1 or 2 slices
  if (tid == 0) {
    for (int s = 0; s < AB_NST; ++s) {
      oz_mbar_init(&full[s], 1);
      oz_mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      oz_mbar_init(&accf[a], 1);
      oz_mbar_init(&acce[a], 8);
    }
    oz_mbar_init(afull, AB_NPROD);
    oz_mbar_init(afree, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(oz_smem(tslot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  oz_fence_before();
  __syncthreads();
  oz_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(AB_BN >> 3) << 17) |
                         ((uint32_t)(OZ_BM >> 4) << 24);
  auto bidx = [&](int b) {
    return p.nbB == 1 ? 0 : (p.bmap == BMAP_XOR1 ? (b ^ 1) : (p.bmap == BMAP_SHR1 ? (b >> 1) : b));
  };
  int issued = 0, committed = 0;   // TMA / MMA progress (slices), for the drain after an abort
  if (warp >= 10) {
    // ---------------- A producers
    const int ptid = tid - 10 * 32;
    int j = 0;
    for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x, ++j) {
      if (__any_sync(0xffffffffu, *abort_flag)) break;
      if (j > 0) {
        const bool ok = oz_wait(afree, (j - 1) & 1);
        if (!__all_sync(0xffffffffu, ok)) { *abort_flag = 1; break; }
      }
      const int b = t / p.ntm, m0 = (t % p.ntm) * OZ_BM;
      const int bA = p.nbA == 1 ? 0 : b;
      const double* Ab = p.A + (size_t)bA * p.sA;
      // two tasks per round: their 16 loads are in flight together
      const int tasks = OZ_BM * (p.Kp / 8), stride = 32 * AB_NPROD;
      auto load = [&](int u, double (&x)[8]) {
        const int r = u % OZ_BM, qq = u / OZ_BM;   // lanes on consecutive rows
        const int row = m0 + r, k0 = 8 * qq;
        const bool live = u < tasks && row < p.M;
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = live && k0 + i < p.K ? __ldg(Ab + row + (size_t)(k0 + i) * p.lda) : 0.0;
        return live ? __ldg(p.exA + (size_t)bA * p.M + row) : -2000;
      };
      for (int u = ptid; u < tasks; u += 2 * stride) {
        double x[8], y[8];
        const int ex = load(u, x), ey = load(u + stride, y);
        oz_put8(x, ex, abuf + ((u / OZ_BM) >> 2) * OZ_PLANE_A, u % OZ_BM, (u / OZ_BM) & 3, AB_APLANE);
        const int u2 = u + stride;
        if (u2 < tasks) oz_put8(y, ey, abuf + ((u2 / OZ_BM) >> 2) * OZ_PLANE_A, u2 % OZ_BM, (u2 / OZ_BM) & 3, AB_APLANE);
      }
      oz_fence_async_smem();
      __syncwarp();
      if (lane == 0) oz_arrive(afull);
    }
  } else if (warp == 8) {
    if (lane == 0) {
      // ---------------- B loads
      int it = 0;
      for (int t = blockIdx.x; t < p.ntiles && !*abort_flag; t += gridDim.x) {
        const int bB = bidx(t / p.ntm);
        for (int n = 0; n < p.ntn && !*abort_flag; ++n)
          for (int s = 0; s < nk; ++s, ++it) {
            const int st = it % AB_NST, u = it / AB_NST;
            if (u > 0 && !oz_wait(&empty[st], (u - 1) & 1)) { *abort_flag = 1; break; }
            oz_expect_tx(&full[st], AB_STAGE);
#pragma unroll
            for (int q = 0; q < OZ_S; ++q)
              oz_tma3(bst + st * AB_STAGE + q * AB_PLANE_B, &mapB, s * OZ_BK, n * AB_BN, q * p.nbB + bB, &full[st]);
            issued = it + 1;
          }
      }
    }
  } else if (warp == 9) {
    if (lane == 0) {
      // ---------------- products
      int it = 0, jt = 0, j = 0;
      for (int t = blockIdx.x; t < p.ntiles && !*abort_flag; t += gridDim.x, ++j) {
        if (!oz_wait(afull, j & 1)) { *abort_flag = 1; break; }
        oz_fence_after();
        bool ok = true;
        for (int n = 0; n < p.ntn && ok; ++n, ++jt) {
          const int a = jt & 1;
          if (jt >= 2 && !oz_wait(&acce[a], ((jt >> 1) - 1) & 1)) { ok = false; break; }
          oz_fence_after();
          for (int s = 0; s < nk; ++s, ++it) {
            const int st = it % AB_NST;
            if (!oz_wait(&full[st], (it / AB_NST) & 1)) { ok = false; break; }
            oz_fence_after();
            const unsigned char* bs = bst + st * AB_STAGE;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
              for (int pa = 0; pa < OZ_S; ++pa) {
#pragma unroll
                for (int pb = 0; pb < OZ_S - pa; ++pb) {
                  const int tt = pa + pb, g = tt < OZ_NACC - 1 ? tt : OZ_NACC - 1;
                  const bool first = s == 0 && kk == 0 && pa == 0 && (g < OZ_NACC - 1 || tt == OZ_NACC - 1);
                  oz_mma(tmem + (uint32_t)(256 * a + g * AB_BN),
                         oz_desc(oz_smem(abuf + pa * AB_APLANE + s * OZ_PLANE_A) + 32 * kk),
                         oz_desc(oz_smem(bs + pb * AB_PLANE_B) + 32 * kk), idesc, first ? 0u : 1u);
                }
              }
            }
            oz_commit(&empty[st]);
            committed = it + 1;
          }
          if (ok) oz_commit(&accf[a]);
        }
        if (!ok) { *abort_flag = 1; break; }
        oz_commit(afree);   // the A buffer is free once this tile's products have completed
      }
    }
  } else {
    // ---------------- epilogue
    const int wq = warp & 3, wh = warp >> 2;
    const uint32_t lanes = (uint32_t)(32 * wq) << 16;
    int jt = 0;
    for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
      if (__any_sync(0xffffffffu, *abort_flag)) break;
      const int b = t / p.ntm, m0 = (t % p.ntm) * OZ_BM;
      const int bA = p.nbA == 1 ? 0 : b, bB = bidx(b);
      const int row = m0 + 32 * wq + lane;
      const bool live = row < p.M;
      const int ea = live ? __ldg(p.exA + (size_t)bA * p.M + row) : -2000;
      double* crow = p.C + (size_t)b * p.sC + row;
      bool stop = false;
      for (int n = 0; n < p.ntn; ++n, ++jt) {
        const int a = jt & 1;
        const int c0 = n * AB_BN + (AB_BN / 2) * wh;
        // the C values of this warp's 24 columns, loaded before the accumulators are waited for
        double cv[AB_BN / 2];
#pragma unroll
        for (int q = 0; q < AB_BN / 2; ++q)
          cv[q] = p.bmode && live && c0 + q < p.N ? crow[(size_t)(c0 + q) * p.ldc] : 0.0;
        const bool ok = oz_wait(&accf[a], (jt >> 1) & 1);
        if (!__all_sync(0xffffffffu, ok)) { *abort_flag = 1; stop = true; break; }
        oz_fence_after();
#pragma unroll
        for (int h = 0; h < AB_BN / 16; ++h) {
          const int cc = c0 + 8 * h;
          uint32_t ra[8], rb[8], rc[8], rd[8], rt[8];
          const uint32_t base = tmem + lanes + (uint32_t)(256 * a + (AB_BN / 2) * wh + 8 * h);
          oz_ld8(base, ra);
          oz_ld8(base + (uint32_t)AB_BN, rb);
          oz_ld8(base + (uint32_t)(2 * AB_BN), rc);
          oz_ld8(base + (uint32_t)(3 * AB_BN), rd);
          oz_ld8(base + (uint32_t)(4 * AB_BN), rt);
          oz_ld_wait();
          if (h + 1 == AB_BN / 16) {
            // the accumulator set is free for the subtile after next
            oz_fence_before();
            __syncwarp();
            if (lane == 0) oz_arrive(&acce[a]);
          }
          if (live) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int col = cc + q;
              if (col >= p.N) continue;
              const double v = oz_combine(ra[q], rb[q], rc[q], rd[q], rt[q], ea, __ldg(p.exB + (size_t)bB * p.N + col));
              crow[(size_t)col * p.ldc] = oz_out(v, cv[8 * h + q], p.amode, p.bmode, p.alpha, p.beta);
            }
          }
        }
      }
      if (stop) break;
    }
  }
  __syncthreads();
  if (*abort_flag) {
    if (tid == 0) atomicExch(&g_oz_status, HODLR_ETIMEOUT);
    if (warp == 8 && lane == 0)
      for (int it = issued - 1; it >= 0 && it >= issued - AB_NST; --it) oz_wait(&full[it % AB_NST], (it / AB_NST) & 1);
    if (warp == 9 && lane == 0 && committed > 0)
      oz_wait(&empty[(committed - 1) % AB_NST], ((committed - 1) / AB_NST) & 1);
  }
  oz_fence_before();
  __syncthreads();
  if (warp == 0) {
    oz_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ordered reduction of the split-K partials (FP64), then alpha / beta
__global__ void oz_reduce_kernel(int M, int N, int nsplit, const double* part, double alpha, double beta, double* C,
                                 long long ldc, long long sC) {
  const int b = blockIdx.y;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)M * N) return;
  const int i = (int)(e % M), j = (int)(e / M);
  const double* pp = part + (size_t)b * nsplit * ((size_t)M * N) + e;
  double v = 0.0;
  for (int s = 0; s < nsplit; ++s) v += pp[(size_t)s * M * N];
  double* c = C + (size_t)b * sC + (size_t)j * ldc + i;
  double out = alpha * v;
  if (beta != 0.0) out = fma(beta, *c, out);
  *c = out;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn oz_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* q = nullptr;
    cudaDriverEntryPointQueryResult r;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault, &r) == cudaSuccess &&
        r == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)q;
  });
  return fn;
}
// planes [S * nb][R][Kp] BF16: a 3-D map with boxes of 32 (K) x rows x 1, 64-byte swizzle; rows
// beyond R read as zeros
bool oz_map(CUtensorMap* m, const __nv_bfloat16* planes, int Kp, int R, int nplanes, int box_rows) {
  EncodeTiledFn fn = oz_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)R, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * (cuuint64_t)R};
  cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)planes, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void oz_slice(const OzView& v, int Kp, int* ex, __nv_bfloat16* planes, cudaStream_t st) {
  if (v.sk == 1 && Kp <= 8192) {
    dim3 g(cdiv(v.R, 8), v.nb);
    oz_slice_rows_kernel<<<g, 256, 0, st>>>(v, ex, planes, Kp);
    check_launch("oz_slice_rows");
    return;
  }
  if (v.sr == 1 && Kp <= 128) {
    dim3 g(cdiv(v.R, 32), v.nb);
    oz_slice_cols_kernel<<<g, 256, 0, st>>>(v, ex, planes, Kp);
    check_launch("oz_slice_cols");
    return;
  }
  if (v.sk == 1) {
    dim3 g(cdiv(v.R, 8), v.nb);
    oz_rowexp_kernel<<<g, 256, 0, st>>>(v, ex);
  } else if (v.K > 128) {
    // many rows of long k: split k across CTAs (one thread per row would leave the GPU idle)
    HODLR_CUDA(cudaMemsetAsync(ex, 0, sizeof(int) * (size_t)v.nb * v.R, st));
    const int kc = 64 * (int)cdiv(cdiv(v.K, 64), 65535);   // pieces of k: at most 65535 across the grid
    dim3 g(cdiv(v.R, 128), cdiv(v.K, kc), v.nb);
    oz_rowexp_split_kernel<<<g, 128, 0, st>>>(v, kc, ex);
    check_launch("oz_rowexp");
    const long long n = (long long)v.nb * v.R;
    oz_rowexp_fix_kernel<<<cdiv(n, 256), 256, 0, st>>>(n, ex);
  } else {
    dim3 g(cdiv(v.R, 128), v.nb);
    oz_rowexp_kernel<<<g, 128, 0, st>>>(v, ex);
  }
  check_launch("oz_rowexp");
  dim3 g(Kp / 32, cdiv(v.R, 32), v.nb);
  oz_slice_kernel<<<g, dim3(32, 8), 0, st>>>(v, ex, planes, Kp);
  check_launch("oz_slice");
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// ---------------------------------------------------------------- host entry points
thread_local OzConfig g_oz_cfg;

bool oz_eligible(const GemmArgs& g) {
  if (!g_oz_cfg.on || !g_oz_cfg.work.ptr) return false;
  if (g.offmode != 0 || g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0) return false;
  if (g.batch > 65535) return false;
  // products this small are cheaper on the FP64 pipes than the slicing passes; narrow sides
  // (a rank width below the tile) waste tensor-core work but these products are bound by the
  // FP64 operand traffic, not by the MMAs
  const double mnk = (double)g.M * g.N * g.K * g.batch;
  return mnk >= (double)(1 << 22);
}

// bytes of slicing workspace for a batch of nb products (A and B planes, exponents)
static size_t oz_bytes(int nbA, int M, int nbB, int N, int Kp) {
  return align256((size_t)OZ_S * nbA * M * Kp * 2) + align256((size_t)OZ_S * nbB * N * Kp * 2) +
         align256((size_t)nbA * M * 4) + align256((size_t)nbB * N * 4);
}

static int oz_amode(double a) { return a == 1.0 ? 0 : (a == -1.0 ? 1 : 2); }
static int oz_bmode(double b) { return b == 0.0 ? 0 : (b == 1.0 ? 1 : 2); }

static int oz_num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    HODLR_CUDA(cudaGetDevice(&dev));
    HODLR_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  }
  return n;
}

struct OzProf {   // CUDA events around a product launch (the context's profile)
  bool on;
  explicit OzProf(cudaStream_t st) : on(g_prof.on && g_prof.n < g_prof.cap) {
    if (on) cudaEventRecord(g_prof.ev[2 * g_prof.n], st);
  }
  void done(const GemmArgs& g, int nc, int nb, int variant, cudaStream_t st) {
    if (!on) return;
    cudaEventRecord(g_prof.ev[2 * g_prof.n + 1], st);
    if (g_prof.shape) {
      int* sh = g_prof.shape + 7 * g_prof.n;
      sh[0] = g.M; sh[1] = nc; sh[2] = g.K; sh[3] = nb; sh[4] = g.tA; sh[5] = g.tB; sh[6] = variant;
    }
    ++g_prof.n;
    g_prof.flops += 2.0 * (double)g.M * nc * g.K * nb;
    prof_add_bytes(variant, ((double)g.M * g.K + (double)g.K * nc + (double)g.M * nc * (g.beta != 0.0 ? 2 : 1)) * 8.0 * nb);
  }
};

// The fused products (digits made in shared memory by the product kernel): long-K A^T B with
// M <= 128, and short-K A B with column-major A and K <= 64.  False when the shape is not one of
// them or its exponents (and the B planes of a short-K product) do not fit the workspace.
static bool oz_fused(const GemmArgs& g, Scratch split, cudaStream_t st, int tile, int cprx) {
  const Scratch w = g_oz_cfg.work;
  const int Kp = ((g.K + OZ_BK - 1) / OZ_BK) * OZ_BK;
  const int nb = g.batch;
  const bool sharedA = g.sA == 0, sharedB = g.sB == 0;
  const int nbA = sharedA ? 1 : nb;
  const int nbB = sharedB ? 1 : (g.bmap == BMAP_SHR1 ? (nb + 1) / 2 : nb);
  const int bmap = sharedB ? BMAP_ID : g.bmap;
  if (g.tA && !g.tB && g.M <= OZ_BM && Kp >= 2 * OZ_KC && nb <= 65535) {
    const int nch = cdiv(Kp, OZ_KC);
    const bool small = g.M <= 64 && tile == 0;
    const int bn = small ? 80 : 48;
    const int nparts = cdiv(g.N, bn);
    const size_t ea_bytes = align256((size_t)nbA * nch * g.M * 4);
    if (ea_bytes + align256((size_t)nbB * nch * g.N * 4) > w.bytes) return false;
    int* eA = (int*)w.ptr;
    int* eB = (int*)((char*)w.ptr + ea_bytes);
    // ranges of chunks per CTA: about one CTA per SM over all products and column parts
    const long long tasks = (long long)nb * nparts * nch;
    int cpr = (int)std::max<long long>(1, (tasks + oz_num_sms() - 1) / oz_num_sms()) * std::max(1, cprx);
    int nrange = cdiv(nch, cpr);
    while (nrange > 1 && (size_t)nb * nrange * g.M * g.N * 8 > split.bytes) {
      cpr *= 2;
      nrange = cdiv(nch, cpr);
    }
    if (nrange > 65535 || nparts > 65535) return false;
    OzView va{(const double*)g.A, g.sA, g.lda, 1, nbA, g.M, g.K};
    OzView vb{(const double*)g.B, g.sB, g.ldb, 1, nbB, g.N, g.K};
    oz_exp_chunks_kernel<<<dim3(cdiv(g.M, 8), nch, nbA), 256, 0, st>>>(va, OZ_KC, nch, eA);
    check_launch("oz_exp_chunks");
    oz_exp_chunks_kernel<<<dim3(cdiv(g.N, 8), nch, nbB), 256, 0, st>>>(vb, OZ_KC, nch, eB);
    check_launch("oz_exp_chunks");
    AtParams p{};
    p.A = (const double*)g.A; p.B = (const double*)g.B;
    p.lda = g.lda; p.sA = g.sA; p.ldb = g.ldb; p.sB = g.sB;
    p.M = g.M; p.N = g.N; p.K = g.K; p.nbA = nbA; p.nbB = nbB; p.bmap = bmap;
    p.nch = nch; p.cpr = cpr; p.nrange = nrange;
    p.exA = eA; p.exB = eB; p.alpha = g.alpha; p.beta = g.beta;
    p.amode = oz_amode(g.alpha); p.bmode = oz_bmode(g.beta);
    p.C = (double*)g.C; p.ldc = g.ldc; p.sC = g.sC; p.part = (double*)split.ptr;
    const dim3 grid(nparts, nrange, nb);
    OzProf prof(st);
    if (small) {
      using TL = AtTile<64, 80>;
      HODLR_CUDA(cudaFuncSetAttribute(oz_atb_kernel<64, 80>, cudaFuncAttributeMaxDynamicSharedMemorySize, TL::SMEM));
      oz_atb_kernel<64, 80><<<grid, AT_THREADS, TL::SMEM, st>>>(p);
    } else {
      using TL = AtTile<128, 48>;
      HODLR_CUDA(cudaFuncSetAttribute(oz_atb_kernel<128, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize, TL::SMEM));
      oz_atb_kernel<128, 48><<<grid, AT_THREADS, TL::SMEM, st>>>(p);
    }
    check_launch("oz_atb_kernel");
    prof.done(g, g.N, nb, 6, st);
    if (nrange > 1) {
      oz_reduce_kernel<<<dim3(cdiv((long long)g.M * g.N, 256), nb), 256, 0, st>>>(g.M, g.N, nrange, p.part, g.alpha,
                                                                                g.beta, p.C, g.ldc, g.sC);
      check_launch("oz_reduce");
    }
    return true;
  }
  if (!g.tA && Kp <= AB_KMAX && g.M >= OZ_BM && (long long)g.M * nb >= 4096) {
    const size_t pb_bytes = align256((size_t)OZ_S * nbB * g.N * Kp * 2);
    const size_t eb_bytes = align256((size_t)nbB * g.N * 4);
    if (pb_bytes + eb_bytes + align256((size_t)nbA * g.M * 4) > w.bytes) return false;
    __nv_bfloat16* pB = (__nv_bfloat16*)w.ptr;
    int* eB = (int*)((char*)w.ptr + pb_bytes);
    int* eA = (int*)((char*)w.ptr + pb_bytes + eb_bytes);
    OzView vb;
    vb.base = (const double*)g.B; vb.sb = g.sB; vb.nb = nbB; vb.R = g.N; vb.K = g.K;
    if (g.tB) { vb.sr = 1; vb.sk = g.ldb; } else { vb.sr = g.ldb; vb.sk = 1; }
    oz_slice(vb, Kp, eB, pB, st);
    CUtensorMap mb;
    if (!oz_map(&mb, pB, Kp, g.N, OZ_S * nbB, AB_BN)) throw Error(HODLR_ECUDA, "oz_gemm: tensor map");
    OzView va{(const double*)g.A, g.sA, 1, g.lda, nbA, g.M, g.K};
    oz_exp_chunks_kernel<<<dim3(cdiv(g.M, 256), 1, nbA), 256, 0, st>>>(va, Kp, 1, eA);
    check_launch("oz_exp_chunks");
    AbParams p{};
    p.A = (const double*)g.A; p.lda = g.lda; p.sA = g.sA;
    p.M = g.M; p.N = g.N; p.K = g.K; p.Kp = Kp; p.nbA = nbA; p.nbB = nbB; p.bmap = bmap;
    p.ntm = cdiv(g.M, OZ_BM); p.ntn = cdiv(g.N, AB_BN);
    const long long ntiles = (long long)nb * p.ntm;
    if (ntiles > 0x7fffffffLL) return false;
    p.ntiles = (int)ntiles;
    p.exA = eA; p.exB = eB; p.alpha = g.alpha; p.beta = g.beta;
    p.amode = oz_amode(g.alpha); p.bmode = oz_bmode(g.beta);
    p.C = (double*)g.C; p.ldc = g.ldc; p.sC = g.sC;
    const int ctas = (int)std::min<long long>(ntiles, oz_num_sms());
    OzProf prof(st);
    HODLR_CUDA(cudaFuncSetAttribute(oz_ab_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, AB_SMEM));
    oz_ab_kernel<<<ctas, AB_THREADS, AB_SMEM, st>>>(mb, p);
    check_launch("oz_ab_kernel");
    prof.done(g, g.N, nb, 7, st);
    return true;
  }
  return false;
}

bool oz_gemm(const GemmArgs& g, Scratch split, cudaStream_t st) {
  if (!oz_eligible(g)) return false;
  return oz_gemm_any(g, split, st);
}

// the products from slice planes in the workspace (oz_mma_kernel / oz_mma_ws_kernel)
// tile 0: 128 x 96 tiles, two stages, one CTA per SM; tile 1: 128 x 48 tiles, one stage, two CTAs
// per SM (one CTA's epilogue overlaps the other's loads and products); tile 2: the persistent
// warp-specialised kernel over 128 x 48 tiles and K chunks; K <= 128 always takes the persistent
// 128 x 32 kernel
static bool oz_sliced(const GemmArgs& g, Scratch split, cudaStream_t st, int tile = 0) {
  const Scratch w = g_oz_cfg.work;
  const int Kp = ((g.K + OZ_BK - 1) / OZ_BK) * OZ_BK;
  const size_t nsp = (size_t)cdiv(Kp, OZ_KC);   // one 512-long chunk of K per CTA
  const bool sharedA = g.sA == 0, sharedB = g.sB == 0;
  const bool paired = g.bmap != BMAP_ID && !sharedB;
  auto nbB_of = [&](int nb) { return sharedB ? 1 : (g.bmap == BMAP_SHR1 ? (nb + 1) / 2 : nb); };
  auto need = [&](int nb, int nc) {   // workspace and partials of a (batch chunk, column chunk)
    const size_t planes = oz_bytes(sharedA ? 1 : nb, g.M, nbB_of(nb), nc, Kp);
    const size_t part = nsp > 1 ? (size_t)nb * g.M * nc * nsp * sizeof(double) : 0;
    return planes <= w.bytes && part <= split.bytes;
  };
  // batch chunk (even when products are paired), then column chunk (multiple of the tile)
  int bchunk = g.batch;
  while (bchunk > (paired ? 2 : 1) && !need(bchunk, g.N)) {
    bchunk = (bchunk + 1) / 2;
    if (paired) bchunk += bchunk & 1;
  }
  int nchunk = g.N;
  while (nchunk > OZ_BN && !need(bchunk, nchunk)) nchunk = ((nchunk / 2 + OZ_BN - 1) / OZ_BN) * OZ_BN;
  if (!need(bchunk, nchunk)) {
    // even one product with a 96-column chunk does not fit: split K into ranges (multiples of
    // the 512-long chunk) whose planes fit, summed into C in FP64 (beta applies to the first)
    if (Kp <= OZ_KC) return false;
    const int bmin = paired ? 2 : 1;
    auto need_k = [&](int kp) {
      const size_t planes = oz_bytes(sharedA ? 1 : bmin, g.M, nbB_of(bmin), std::min(g.N, OZ_BN), kp);
      const size_t part = kp > OZ_KC ? (size_t)bmin * g.M * std::min(g.N, OZ_BN) * cdiv(kp, OZ_KC) * 8 : 0;
      return planes <= w.bytes && part <= split.bytes;
    };
    int kr = Kp;
    while (kr > OZ_KC && !need_k(kr)) kr = cdiv(kr / 2, OZ_KC) * OZ_KC;
    if (!need_k(kr)) return false;
    for (int k0 = 0; k0 < g.K; k0 += kr) {
      GemmArgs h = g;
      h.K = std::min(kr, g.K - k0);
      h.A = (const double*)g.A + (g.tA ? (size_t)k0 : (size_t)k0 * g.lda);
      h.B = (const double*)g.B + (g.tB ? (size_t)k0 * g.ldb : (size_t)k0);
      if (k0 > 0) h.beta = 1.0;
      if (!oz_sliced(h, split, st, tile)) throw Error(HODLR_ECUDA, "oz_gemm: K range did not fit");
    }
    return true;
  }
  // short K (one to four 32-wide slices): the persistent warp-specialised kernel over 128 x 32 tiles
  const bool narrow = Kp <= 4 * OZ_BK;
  const bool half = !narrow && tile == 1;
  const bool ws48 = !narrow && tile == 2;   // persistent warp-specialised 128 x 48 tiles
  using Wide = OzTile<OZ_BN, 2>;
  using Half = OzTile<OZ_BN / 2, 1>;
  using Ws48 = WsTile<48, 2>;
  const int bn = narrow ? WS_BN : (half || ws48 ? OZ_BN / 2 : OZ_BN);
  static int num_sms = 0;
  if (!num_sms) {
    int dev = 0;
    HODLR_CUDA(cudaGetDevice(&dev));
    HODLR_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  if (narrow)
    HODLR_CUDA(cudaFuncSetAttribute(oz_mma_ws_kernel<WS_BN, WS_NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, WS_SMEM));
  else if (ws48)
    HODLR_CUDA(cudaFuncSetAttribute(oz_mma_ws_kernel<48, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Ws48::SMEM));
  else if (half)
    HODLR_CUDA(cudaFuncSetAttribute(oz_mma_kernel<OZ_BN / 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, Half::SMEM));
  else HODLR_CUDA(cudaFuncSetAttribute(oz_mma_kernel<OZ_BN, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Wide::SMEM));
  for (int b0 = 0; b0 < g.batch; b0 += bchunk) {
    const int nb = std::min(bchunk, g.batch - b0);
    const int nbA = sharedA ? 1 : nb, nbB = nbB_of(nb);
    char* base = (char*)w.ptr;
    __nv_bfloat16* pA = (__nv_bfloat16*)base;
    base += align256((size_t)OZ_S * nbA * g.M * Kp * 2);
    int* eA = (int*)base;
    base += align256((size_t)nbA * g.M * 4);
    __nv_bfloat16* pB = (__nv_bfloat16*)base;
    base += align256((size_t)OZ_S * nbB * nchunk * Kp * 2);
    int* eB = (int*)base;
    // A: rows i of op(A), along k
    OzView va;
    va.base = (const double*)g.A + (size_t)b0 * g.sA;
    va.sb = g.sA; va.nb = nbA; va.R = g.M; va.K = g.K;
    if (g.tA) { va.sr = g.lda; va.sk = 1; } else { va.sr = 1; va.sk = g.lda; }
    oz_slice(va, Kp, eA, pA, st);
    CUtensorMap ma;
    if (!oz_map(&ma, pA, Kp, g.M, OZ_S * nbA, OZ_BM)) throw Error(HODLR_ECUDA, "oz_gemm: tensor map");
    const int bB0 = sharedB ? 0 : (g.bmap == BMAP_SHR1 ? b0 / 2 : b0);
    for (int j0 = 0; j0 < g.N; j0 += nchunk) {
      const int nc = std::min(nchunk, g.N - j0);
      // B: rows j of op(B)^T (columns j0 .. j0 + nc of op(B)), along k
      OzView vb;
      const long long coff = g.tB ? (long long)j0 : (long long)j0 * g.ldb;
      vb.base = (const double*)g.B + (size_t)bB0 * g.sB + coff;
      vb.sb = g.sB; vb.nb = nbB; vb.R = nc; vb.K = g.K;
      if (g.tB) { vb.sr = 1; vb.sk = g.ldb; } else { vb.sr = g.ldb; vb.sk = 1; }
      oz_slice(vb, Kp, eB, pB, st);
      CUtensorMap mb;
      if (!oz_map(&mb, pB, Kp, nc, OZ_S * nbB, bn)) throw Error(HODLR_ECUDA, "oz_gemm: tensor map");
      const int nsplit = (int)nsp;
      OzParams p{};
      p.M = g.M; p.N = nc; p.K = g.K; p.Kp = Kp; p.nbA = nbA; p.nbB = nbB;
      p.bmap = sharedB ? BMAP_ID : g.bmap; p.nsplit = nsplit;
      p.exA = eA; p.exB = eB; p.alpha = g.alpha; p.beta = g.beta;
      p.amode = oz_amode(g.alpha); p.bmode = oz_bmode(g.beta);
      p.C = (double*)g.C + (size_t)b0 * g.sC + (size_t)j0 * g.ldc; p.ldc = g.ldc; p.sC = g.sC;
      p.part = (double*)split.ptr;
      if ((long long)nb * nsplit > 65535) throw Error(HODLR_EINVAL, "oz_gemm: batch too large");
      // rasterisation: the larger operand's tiles are shared by the CTAs launched together
      p.nfast = (long long)nbA * g.M > (long long)nbB * nc ? 1 : 0;
      dim3 grid(p.nfast ? cdiv(nc, bn) : cdiv(g.M, OZ_BM), p.nfast ? cdiv(g.M, OZ_BM) : cdiv(nc, bn), nb * nsplit);
      const bool prof = g_prof.on && g_prof.n < g_prof.cap;
      if (prof) cudaEventRecord(g_prof.ev[2 * g_prof.n], st);
      if (narrow || ws48) {
        const int ntm = cdiv(g.M, OZ_BM), ntn = cdiv(nc, bn);
        const long long ntiles = (long long)ntm * ntn * nb * nsplit;
        if (ntiles > 0x7fffffffLL) throw Error(HODLR_EINVAL, "oz_gemm: too many tiles");
        const int ctas = (int)std::min<long long>(ntiles, num_sms);
        if (narrow) oz_mma_ws_kernel<WS_BN, WS_NST><<<ctas, WS_THREADS, WS_SMEM, st>>>(ma, mb, p, ntm, ntn, (int)ntiles);
        else oz_mma_ws_kernel<48, 2><<<ctas, WS_THREADS, Ws48::SMEM, st>>>(ma, mb, p, ntm, ntn, (int)ntiles);
        check_launch("oz_mma_ws_kernel");
      } else {
        if (half) oz_mma_kernel<OZ_BN / 2, 1><<<grid, OZ_THREADS, Half::SMEM, st>>>(ma, mb, p);
        else oz_mma_kernel<OZ_BN, 2><<<grid, OZ_THREADS, Wide::SMEM, st>>>(ma, mb, p);
        check_launch("oz_mma_kernel");
      }
      if (prof) {
        cudaEventRecord(g_prof.ev[2 * g_prof.n + 1], st);
        if (g_prof.shape) {
          int* sh = g_prof.shape + 7 * g_prof.n;
          sh[0] = g.M; sh[1] = nc; sh[2] = g.K; sh[3] = nb; sh[4] = g.tA; sh[5] = g.tB; sh[6] = 5;
        }
        ++g_prof.n;
        g_prof.flops += 2.0 * (double)g.M * nc * g.K * nb;
        prof_add_bytes(5, ((double)g.M * g.K + (double)g.K * nc + (double)g.M * nc * (g.beta != 0.0 ? 2 : 1)) * 8.0 * nb);
      }
      if (nsplit > 1) {
        dim3 rg(cdiv((long long)g.M * nc, 256), nb);
        oz_reduce_kernel<<<rg, 256, 0, st>>>(g.M, nc, nsplit, p.part, g.alpha, g.beta, p.C, g.ldc, g.sC);
        check_launch("oz_reduce");
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------- tile autotuner
// A product runs either from slice planes (path 0; tile 0: 128 x 96, tile 1: 128 x 48 with two
// CTAs per SM, tile 2: persistent warp-specialised 128 x 48) or fused (path 1; tile 0: 64 x 80 for M <= 64 else 128 x 48, tile 1: 128 x 48;
// cprx: chunks of K per CTA times the default).  The default
// plan is the fused path where the shape allows it.  A context with tuning on times, on the
// first occurrence of a shape, every candidate plan once (after a warm-up run, CUDA events on
// the context's stream, into a scratch C carved from the slice workspace so that the real C is
// untouched) and remembers the fastest for the process; the product itself then runs with it.
struct OzPlan {
  int path, tile, cprx;
};
using OzKey = std::array<long long, 10>;
static std::mutex g_tune_mu;
static std::map<OzKey, OzPlan> g_tuned;

static OzKey oz_key(const GemmArgs& g) {
  return {g.M, g.N, g.K, g.batch, g.tA, g.tB, g.sA == 0, g.sB == 0, g.bmap, oz_bmode(g.beta)};
}
// 1: long-K fused shape, 2: short-K fused shape, 0: neither (the conditions of oz_fused)
static int oz_fused_kind(const GemmArgs& g) {
  const int Kp = ((g.K + OZ_BK - 1) / OZ_BK) * OZ_BK;
  if (g.tA && !g.tB && g.M <= OZ_BM && Kp >= 2 * OZ_KC && g.batch <= 65535) return 1;
  if (!g.tA && Kp <= AB_KMAX && g.M >= OZ_BM && (long long)g.M * g.batch >= 4096) return 2;
  return 0;
}
static bool oz_run(const GemmArgs& g, Scratch split, cudaStream_t st, OzPlan pl) {
  if (pl.path == 1 && oz_fused(g, split, st, pl.tile, pl.cprx)) return true;
  return oz_sliced(g, split, st, pl.path == 0 ? pl.tile : 0);
}
static OzPlan oz_tune(const GemmArgs& g, Scratch split, cudaStream_t st, OzPlan def) {
  std::vector<OzPlan> cand{{0, 0, 1}};
  if (((g.K + OZ_BK - 1) / OZ_BK) * OZ_BK > 4 * OZ_BK) {   // 128 x 48 tiles: two CTAs per SM, or persistent
    cand.push_back({0, 1, 1});
    cand.push_back({0, 2, 1});
  }
  const int kind = oz_fused_kind(g);
  if (kind == 1) {
    cand.push_back({1, 0, 1});
    cand.push_back({1, 0, 4});
    if (g.M <= 64) cand.push_back({1, 1, 1});
  } else if (kind == 2) {
    cand.push_back({1, 0, 1});
  }
  if (cand.size() == 1) return cand[0];
  const Scratch w = g_oz_cfg.work;
  const size_t cbytes = align256((size_t)g.batch * g.M * g.N * sizeof(double));
  if (cbytes > w.bytes / 2) return def;
  GemmArgs h = g;
  const size_t keep = (w.bytes - cbytes) & ~(size_t)255;   // the scratch C starts 256-byte aligned
  h.C = (char*)w.ptr + keep;
  h.ldc = g.M;
  h.sC = (long long)g.M * g.N;
  const OzConfig saved = g_oz_cfg;
  const bool prof_on = g_prof.on;
  g_oz_cfg.work.bytes = keep;
  g_oz_cfg.tune = false;
  g_prof.on = false;   // the trial runs stay out of the kernel profile
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  OzPlan best = def;
  try {
    HODLR_CUDA(cudaMemsetAsync(h.C, 0, cbytes, st));
    HODLR_CUDA(cudaEventCreate(&e0));
    HODLR_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    for (const OzPlan& c : cand) {
      if (!oz_run(h, split, st, c)) continue;   // warm-up
      HODLR_CUDA(cudaEventRecord(e0, st));
      oz_run(h, split, st, c);
      oz_run(h, split, st, c);
      HODLR_CUDA(cudaEventRecord(e1, st));
      HODLR_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      HODLR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
  } catch (...) {
    g_oz_cfg = saved;
    g_prof.on = prof_on;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    throw;
  }
  g_oz_cfg = saved;
  g_prof.on = prof_on;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// a plan forced on this thread (hodlr_dgemm_slices_plan; path < 0: automatic)
static thread_local OzPlan g_forced{-1, 0, 1};

bool oz_gemm_any(const GemmArgs& g, Scratch split, cudaStream_t st) {
  if (!g_oz_cfg.work.ptr || g.offmode != 0 || g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0) return false;
  if (g_forced.path >= 0) return oz_run(g, split, st, g_forced);
  OzPlan plan{oz_fused_kind(g) ? 1 : 0, 0, 1};
  const OzKey key = oz_key(g);
  bool known = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) { plan = it->second; known = true; }
  }
  if (!known && g_oz_cfg.tune) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HODLR_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      plan = oz_tune(g, split, st, plan);
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned[key] = plan;
    }
  }
  return oz_run(g, split, st, plan);
}

void oz_force_plan(int path, int tile, int cprx) { g_forced = OzPlan{path, tile, cprx}; }

void oz_tuned_clear() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned.clear();
}

int oz_tuned_table(int64_t* out, int cap) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int n = 0;
  for (const auto& kv : g_tuned) {
    if (out && n < cap) {
      int64_t* r = out + 13 * (size_t)n;
      for (int i = 0; i < 10; ++i) r[i] = kv.first[i];
      r[10] = kv.second.path; r[11] = kv.second.tile; r[12] = kv.second.cprx;
    }
    ++n;
  }
  return n;
}

int oz_status_take(cudaStream_t st) {
  int v = 0, zero = 0;
  HODLR_CUDA(cudaMemcpyFromSymbolAsync(&v, g_oz_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  HODLR_CUDA(cudaStreamSynchronize(st));
  if (v) HODLR_CUDA(cudaMemcpyToSymbolAsync(g_oz_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
  return v;
}

}  // namespace hodlr

using namespace hodlr;

extern "C" int hodlr_dgemm_slices_plan(int path, int tile, int cprx) {
  if (path < -1 || path > 1 || tile < 0 || tile > (path == 0 ? 2 : 1) || cprx < 1) return HODLR_EINVAL;
  oz_force_plan(path, tile, cprx);
  return HODLR_OK;
}

extern "C" int hodlr_dgemm_slices(int M, int N, int K, int batch, const double* A, long long lda, long long sA,
                                  int tA, const double* B, long long ldb, long long sB, int tB, int bmap,
                                  double alpha, double beta, double* C, long long ldc, long long sC, void* work,
                                  size_t work_bytes, void* cuda_stream) {
  if (M < 0 || N < 0 || K < 0 || batch < 1 || !A || !B || !C || !work || bmap < 0 || bmap > 2) return HODLR_EINVAL;
  if (((uintptr_t)work & 255) || work_bytes < (64u << 20)) return HODLR_EINVAL;
  if (M == 0 || N == 0) return HODLR_OK;
  try {
    GemmArgs g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.sA = sA; g.tA = tA ? 1 : 0;
    g.B = B; g.ldb = ldb; g.sB = sB; g.tB = tB ? 1 : 0; g.bmap = bmap;
    g.C = C; g.ldc = ldc; g.sC = sC;
    g.alpha = alpha; g.beta = beta; g.batch = batch;
    // the first quarter of the workspace holds split-K partials, the rest the slice planes
    Scratch split{work, work_bytes / 4};
    OzConfig saved = g_oz_cfg;
    g_oz_cfg.on = true;
    g_oz_cfg.work = Scratch{(char*)work + work_bytes / 4, work_bytes - work_bytes / 4};
    bool done = false;
    try {
      // any shape: the eligibility thresholds of the engine do not apply to this call
      done = K > 0 ? oz_gemm_any(g, split, (cudaStream_t)cuda_stream) : false;
    } catch (...) {
      g_oz_cfg = saved;
      throw;
    }
    g_oz_cfg = saved;
    if (!done && K > 0) return HODLR_ENOMEM;
    if (K == 0) {
      // C = beta C through the plain kernel path
      gemm<double, double, double, double>(g, split, (cudaStream_t)cuda_stream);
    }
    HODLR_CUDA(cudaGetLastError());
    if (oz_status_take((cudaStream_t)cuda_stream)) return HODLR_ETIMEOUT;
  } catch (const Error& x) {
    return x.code;
  }
  return HODLR_OK;
}
