// FP64-accurate GEMM on the BF16 tensor cores (tcgen05 kind::f16) by operand
// slicing, after Ozaki's error-free splitting of floating-point matrix
// products (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012).
//
// Every engine GEMM is first embedded as one real GEMM D = A' B'^T exactly as
// in the split-TF32 kernel (complex operands stacked along rows, columns or
// K).  Each row r of A' (and of B') gets a power-of-two scale 2^E_r with
// |x| < 2^E_r over the row, and each element becomes the 56-bit integer
// X = round(x 2^(55 - E_r)) written in S = 7 balanced base-256 digits
//   x = 2^E_r sum_{s=1..7} d_s 2^(1 - 8 s),   d_s in [-128, 128],
// each digit exact in BF16.  The product keeps the digit pairs (s, t) with
// s + t <= 8 (28 of 49; the rest lie below 2^-53 of the row scales):
//   (A'B'^T)_ij = 2^(E_i + E_j) sum_{d=2..8} 2^(2 - 8 d) sum_{s+t=d} sum_k d_s d_t.
// Products of digits are exact in FP32 (|d_s d_t| <= 2^14), and a diagonal
// accumulates at most 7 pairs over a chunk of 128 of K, at most 7 * 2^21 <
// 2^24 in magnitude: every chunk sum in tensor memory is an exact integer.
// The epilogue scales each chunk sum by 2^(2 - 8 d) (exact) and adds it to a
// compensated FP32 pair (TwoSum, about 48 bits); the pair becomes one FP64
// value at the end, times 2^(E_i + E_j).  The result carries about 2^-48 of
// the row-scale product per term, against 2^-53 for FP64 FMA accumulation,
// and runs on the tensor pipe instead of the FP64 pipe (about two operations
// per clock per SM on this part).
//
// The split-FP16 form (S = 2) uses the same machinery with two FP16 planes
// instead of integer digits: under the row scale, y = x 2^(15 - E) (|y| <
// 2^15, rounded to FP32), hi = fp16(y) and lo = fp16(y - hi), so x = 2^(E -
// 15) (hi + lo) to about 2^-22 of |x| (11 significant bits per plane, as in
// split TF32; below FP16's normal range about 2^-40 of the row scale).  The
// three products hi hi, hi lo and lo hi accumulate in one FP32 accumulator,
// not exactly, and run at the 16-bit tensor rate, twice the TF32 rate.
//
// Operand layout: digit planes [S][batch][row tile][k tile][rows x 32] of
// BF16 (FP16 for S = 2) in 8 x 8 core matrices (K-major, no swizzle; 128 B
// between core matrices along K, 512 B between 8-row groups).  A stage holds all planes of
// one k tile of A (128 rows) and B (64 rows for seven planes, 84 KB, two
// stages; 128 rows for three, 48 KB, four stages).  Tensor memory holds the
// accumulators of one chunk (seven planes: 7 diagonals x 64 columns; three
// planes: 2 x 128 columns, see Cfg), twice over where both sets fit, so a
// chunk drains while the next one accumulates.
//
// Warp roles: warp 0 lane 0 issues the bulk copies, warp 1 owns the tensor
// memory and lane 0 issues the MMAs, the other 8 (16 for 128-column tiles)
// warps drain the accumulators (warp w reads lanes 32*(w%4)..+31 and column
// group (w-2)/4).
// Every wait is bounded; on expiry the CTA records an error code, lets its
// copies land, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace rteom {

namespace oz {

using namespace tc5;

constexpr int BM = 128;                    // rows of A' per tile (TMEM lanes)
constexpr int BK = 32;                     // K per k tile (BF16, 64 bytes per row)
constexpr uint32_t A_TILE = BM * BK * 2;   // 8 KB
constexpr int kZeroExp = INT_MIN / 4;      // scale exponent of an all-zero row
constexpr int kNanExp = INT_MAX / 4;       // ... of a row holding an infinity or NaN

// S digit planes per operand (7: FP64-accurate; 3: the split-BF16 form) and
// output-tile width BN (rows of B' per tile).  A diagonal sums at most S
// digit pairs, so a chunk of K stays exact in FP32 while S * K * 2^14 <
// 2^24: 128 of K for S = 7, 256 for S = 3.
//
// Three planes (the split-BF16 form) use two accumulators instead of one per
// diagonal: the leading pair (0,0), exact over chunks of 512 of K, and the
// five others together, their planes packed pre-scaled by the digit weights
// 2^-8 and 2^-16 (exact in BF16) so that one FP32 accumulator carries them
// at their relative weights (rounding about 2^-24 of a term 2^-8 below the
// leading one).  That leaves room for 128-column tiles, two accumulator sets
// and chunks twice as long.
//
// Two planes (the split-FP16 form) keep one accumulator for all three
// products; its chunk sums are rounded FP32 sums over 512 of K.
template <int S, int BN>
struct Cfg {
  static constexpr bool FUSED = S == 3;
  static constexpr bool F16 = S == 2;              // FP16 hi/lo planes
  static constexpr int NACC = F16 ? 1 : (FUSED ? 2 : S);  // accumulators per set
  static constexpr int CHUNK_KT = (FUSED || F16) ? 16 : (S > 4 ? 4 : 8);  // k tiles per chunk
  static constexpr uint32_t B_TILE = BN * BK * 2;
  static constexpr uint32_t STAGE_BYTES = S * (A_TILE + B_TILE);
  // ring depth: at least about 2500 clocks of MMA work in flight (six 32 KB
  // stages of the two-plane form, four of the others)
  static constexpr int MAX_STAGES = F16 ? 6 : 4;
  static constexpr int STAGES = (200u * 1024u / STAGE_BYTES) < MAX_STAGES
                                    ? (200u * 1024u / STAGE_BYTES) : MAX_STAGES;
  // two accumulator sets (the next chunk accumulates while the last one
  // drains) when both fit the 512 tensor-memory columns
  static constexpr int NBUF = 2 * NACC * BN <= 512 ? 2 : 1;
  static constexpr int ACC_COLS = NBUF * NACC * BN;
  static constexpr uint32_t TMEM_COLS = ACC_COLS <= 128 ? 128 : (ACC_COLS <= 256 ? 256 : 512);
  static constexpr size_t SMEM = STAGES * (size_t)STAGE_BYTES + 256;
  // accumulator drain: 16 warps for 128-column tiles (32 columns each keep
  // their compensated pairs in registers), else 8; four warps per group of
  // 32 tensor-memory lanes
  static constexpr int EPI = BN >= 128 ? 16 : 8;
  static constexpr int THREADS = 64 + 32 * EPI;
  static constexpr int COLS = BN / (EPI / 4);  // columns drained by one warp
  // chunk sums added as compensated pairs, except in 256-column tiles, whose
  // 64 columns per warp leave room for plain FP32 sums only
  static constexpr bool COMP = COLS <= 32;
  static_assert(ACC_COLS <= (int)TMEM_COLS, "diagonal accumulators exceed tensor memory");
  // exactness of the chunk sums: S pairs per diagonal (one pair for the
  // leading accumulator of the fused form), |d_s d_t| <= 2^14
  static_assert(F16 || (FUSED ? 1 : S) * CHUNK_KT * BK * 16384 < (1 << 24),
                "chunk sums must stay exact in FP32");
  static_assert(STAGES >= 2, "at least two pipeline stages");
};

// Instruction descriptor of kind::f16: F32 accumulator, A and B both BF16
// (or both FP16), both K-major, N = bn, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int bn, bool fp16 = false) {
  return (1u << 4) | (fp16 ? 0u : (1u << 7) | (1u << 10)) | ((uint32_t)(bn >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

// v * 2^k on the exponent bits (v finite); results below the normal range
// become signed zeros, above it infinities.
__device__ __forceinline__ double scale2(double v, int k) {
  const long long u = __double_as_longlong(v);
  const long long sign = u & (long long)0x8000000000000000ull;
  const int e = (int)((u >> 52) & 0x7FF);
  if (e == 0) return __longlong_as_double(sign);
  const int ne = e + k;
  if (ne <= 0) return __longlong_as_double(sign);
  if (ne >= 2047) return __longlong_as_double(sign | (0x7FFll << 52));
  return __longlong_as_double((u & ~(0x7FFll << 52)) | ((long long)ne << 52));
}

// ---------------------------------------------------------------- packing
struct PackArgs {
  const double* src;
  bool cplx;
  int64_t s_r, s_c, s_b;  // element strides of logical rows, columns, batch
  int R, C;               // logical extents of the source operand (rows x K)
  int mode;               // 0 plain, 1 complex rows [Re; Im], 2 complex K [Re | Im], 3 complex B
  int part;               // complex source read as one real part (0 re, 1 im, 2 re+im), or -1
  int Rp, Kp, rowtile;    // packed extents (rows multiple of rowtile, K of 32)
  __nv_bfloat16* planes;  // S planes of plane_elems
  int64_t plane_elems;
  int64_t s_out;          // elements per batch entry within a plane
  int* expo;              // [batch][Rp] largest biased exponent of each row
  bool rows_fast;         // consecutive threads walk packed rows (source rows contiguous)
  View2 view;             // strided source view (view.rdims > 0) instead of s_r / s_c
};

// Value of the embedded real operand at packed (row rp, column kp).
__device__ __forceinline__ double embedded(const PackArgs& p, int b, int rp, int kp) {
  int r = rp, c = kp, part = 0;
  bool neg = false, valid;
  switch (p.mode) {
    case 0:
      valid = rp < p.R && kp < p.C;
      break;
    case 1:
      part = rp >= p.R;
      r = rp - part * p.R;
      valid = rp < 2 * p.R && kp < p.C;
      break;
    case 2:
      part = kp >= p.C;
      c = kp - part * p.C;
      valid = rp < p.R && kp < 2 * p.C;
      break;
    default: {  // rows n' = [n; n], K' = [k | k]: [[Re, Im], [-Im, Re]]
      const int ro = rp >= p.R, ko = kp >= p.C;
      r = rp - ro * p.R;
      c = kp - ko * p.C;
      valid = rp < 2 * p.R && kp < 2 * p.C;
      part = ro != ko;
      neg = ko && !ro;
    }
  }
  if (!valid) return 0.0;
  const int64_t off = b * p.s_b + (p.view.rdims ? view_row(p.view, r) + view_col(p.view, c)
                                                 : r * p.s_r + c * p.s_c);
  if (p.part >= 0) {
    const double* q = p.src + 2 * off;
    return p.part == 2 ? q[0] + q[1] : q[p.part];
  }
  const double x = p.cplx ? p.src[2 * off + part] : p.src[off];
  return neg ? neg_f64(x) : x;
}

// Row scale exponents, stored as the row's largest biased exponent emax
// (0 for an all-zero row); the scale is 2^E with E = emax - 1022, so |x| <
// 2^E over the row.  With contiguous source rows a thread walks one row over
// a segment of K (loads coalesced across threads); otherwise a warp walks
// one row over a segment of K.  Segments meet in an atomic max on the
// zeroed array.
constexpr int kExpoSeg = 64;

__device__ __forceinline__ int row_exp(int raw) {
  return raw == 0 ? kZeroExp : (raw == 0x7FF ? kNanExp : raw - 1022);
}

// FP64 value of a compensated pair under the row scales 2^(er + ec); a row
// holding an infinity or NaN makes the product NaN (the propagation reports
// non-finite amplitudes), an all-zero row makes it zero.
__device__ __forceinline__ double scaled_value(float su, float cm, int er, int ec) {
  if (er == kNanExp || ec == kNanExp) return __longlong_as_double(0x7FF8000000000000ll);
  if (er == kZeroExp || ec == kZeroExp) return 0.0;
  return scale2(f32_to_f64(su) + f32_to_f64(cm), er + ec);
}

// FP64 value of a plain FP32 sum under the row scales 2^(er + ec), on the
// integer ALUs (no FP64 operation).
__device__ __forceinline__ double scaled_value1(float su, int er, int ec) {
  if (er == kNanExp || ec == kNanExp) return __longlong_as_double(0x7FF8000000000000ll);
  if (er == kZeroExp || ec == kZeroExp) return 0.0;
  return scale2(f32_to_f64(su), er + ec);
}

__global__ void oz_expo_rows_kernel(PackArgs p, int batch) {
  const int64_t rows = (int64_t)batch * p.Rp;
  const int64_t segs = (p.Kp + kExpoSeg - 1) / kExpoSeg;
  const int64_t units = rows * segs;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sg = u / rows, w = u % rows;  // consecutive threads: consecutive rows
    const int b = (int)(w / p.Rp), rp = (int)(w % p.Rp);
    const int k0 = (int)(sg * kExpoSeg), k1 = min(p.Kp, k0 + kExpoSeg);
    unsigned emax = 0;
    for (int kp = k0; kp < k1; ++kp)
      emax = max(emax, (unsigned)((__double_as_longlong(embedded(p, b, rp, kp)) >> 52) & 0x7FF));
    if (emax) atomicMax(p.expo + w, (int)emax);
  }
}

constexpr int kExpoWarpSeg = 2048;

__global__ void oz_expo_kernel(PackArgs p, int batch) {
  const int64_t rows = (int64_t)batch * p.Rp;
  const int64_t segs = (p.Kp + kExpoWarpSeg - 1) / kExpoWarpSeg;
  const int64_t units = rows * segs;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < units; u += nwarps) {
    const int64_t w = u / segs, sg = u % segs;
    const int b = (int)(w / p.Rp), rp = (int)(w % p.Rp);
    const int k1 = min(p.Kp, (int)((sg + 1) * kExpoWarpSeg));
    unsigned emax = 0;
    for (int kp = (int)(sg * kExpoWarpSeg) + lane; kp < k1; kp += 32) {
      const double x = embedded(p, b, rp, kp);
      emax = max(emax, (unsigned)((__double_as_longlong(x) >> 52) & 0x7FF));
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    if (lane == 0 && emax) atomicMax(p.expo + w, (int)emax);
  }
}

// Digit planes: X = round(x 2^(8S - 1 - E)) on the integer ALUs, then
// balanced base-256 digits from the least significant one.  A warp packs one
// 8-row x 32-column block (four core matrices per plane, 512 contiguous
// bytes): lane t takes row t/4 and the eight columns 8*(t%4).., and writes
// 16 bytes to each plane.
template <int S>
__device__ __forceinline__ void digits_of(double x, int E, int (&d)[S]) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((u >> 52) & 0x7FF);
  long long X = 0;
  if (ex != 0 && E != kZeroExp && E != kNanExp) {
    const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = ex - 1076 + 8 * S - E;  // |x| < 2^E keeps |X| <= 2^(8S-1)
    unsigned long long a = 0;
    if (sh >= 0)
      a = m << sh;
    else if (sh > -64)
      a = (m + (1ull << (-sh - 1))) >> (-sh);
    X = (u >> 63) ? -(long long)a : (long long)a;
  }
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const int r = (int)(X & 255);
    d[s] = r >= 128 ? r - 256 : r;
    X = (X - d[s]) >> 8;
  }
  d[0] = (int)X;
}

// FP16 planes of x under the row scale 2^E (the split-FP16 form): y = x
// 2^(15 - E) rounded to FP32 on the integer ALUs, hi = fp16(y), lo = fp16(y
// - hi), all rounded to nearest; y - hi is exact in FP32 (Sterbenz), so hi +
// lo carries y to about 1.5 * 2^-23 of |y| without an FP64 operation (the
// FP64 pipe, about two operations per clock per SM, would bound the pack).
// Zero and non-finite rows give zero planes (the epilogue reads a
// non-finite row from its exponent).
__device__ __forceinline__ void f16_split(double x, int E, uint32_t& hi, uint32_t& lo) {
  hi = lo = 0u;
  if (E == kZeroExp || E == kNanExp) return;
  const float y = f64_to_f32(scale2(x, 15 - E));
  const __half h = __float2half_rn(y);
  hi = (uint32_t)__half_as_ushort(h);
  lo = (uint32_t)__half_as_ushort(__float2half_rn(y - __half2float(h)));
}

// The 16-bit words of planes s of two consecutive elements x0, x1 (x0 in the
// low half): FP16 hi/lo for S = 2, else BF16 digits (the fused three-plane
// form stores plane s pre-scaled by 2^(-8 s)).
template <int S>
__device__ __forceinline__ void plane_words(double x0, double x1, int E, uint32_t (&w)[S]) {
  if constexpr (S == 2) {
    uint32_t h0, l0, h1, l1;
    f16_split(x0, E, h0, l0);
    f16_split(x1, E, h1, l1);
    w[0] = h0 | (h1 << 16);
    w[1] = l0 | (l1 << 16);
  } else {
    int d0[S], d1[S];
    digits_of<S>(x0, E, d0);
    digits_of<S>(x1, E, d1);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const float ws = S == 3 ? __int_as_float((127 - 8 * s) << 23) : 1.0f;
      const __nv_bfloat162 h = __halves2bfloat162(__float2bfloat16_rn((float)d0[s] * ws),
                                                  __float2bfloat16_rn((float)d1[s] * ws));
      w[s] = *reinterpret_cast<const uint32_t*>(&h);
    }
  }
}

template <int S>
__global__ void oz_digits_kernel(PackArgs p, int batch) {
  const int KT = p.Kp / BK;
  const int64_t groups = (int64_t)(p.Rp / 8) * KT;  // 8-row x 32-column blocks per batch entry
  const int64_t units = groups * batch;
  const int lane = threadIdx.x & 31;
  const int rr8 = lane >> 2, kg = lane & 3;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < units; w += nwarps) {
    const int b = (int)(w / groups);
    const int64_t gq = w - (int64_t)b * groups;
    const int rg = (int)(gq / KT), kt = (int)(gq % KT);
    const int rp = rg * 8 + rr8;
    const int E = row_exp(p.expo[(int64_t)b * p.Rp + rp]);
    uint32_t packed[S][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      uint32_t w[S];
      plane_words<S>(embedded(p, b, rp, kt * BK + kg * 8 + j),
                     embedded(p, b, rp, kt * BK + kg * 8 + j + 1), E, w);
#pragma unroll
      for (int s = 0; s < S; ++s) packed[s][j / 2] = w[s];
    }
    // core matrix (rg, kg) of the tile: 8 rows x 8 columns, row rr8 at 16 bytes
    const int rt = rp / p.rowtile, rr = rp % p.rowtile;
    const int64_t off = (int64_t)b * p.s_out + ((int64_t)rt * KT + kt) * ((int64_t)p.rowtile * BK) +
                        ((rr / 8) * (BK / 8) + kg) * 64 + (rr % 8) * 8;
#pragma unroll
    for (int s = 0; s < S; ++s)
      *reinterpret_cast<uint4*>(p.planes + s * p.plane_elems + off) =
          make_uint4(packed[s][0], packed[s][1], packed[s][2], packed[s][3]);
  }
}

// Digit planes of a source whose rows are contiguous (rows_fast): a warp
// packs 32 rows x 32 columns, lane = row, so each of its loads is one
// coalesced run across the warp; each lane writes one 16-byte core-matrix
// row per plane and column group of 8.
template <int S>
__global__ void oz_digits_rows_kernel(PackArgs p, int batch) {
  const int KT = p.Kp / BK;
  const int64_t groups = (int64_t)(p.Rp / 32) * KT;  // 32-row x 32-column blocks per batch entry
  const int64_t units = groups * batch;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < units; w += nwarps) {
    const int b = (int)(w / groups);
    const int64_t gq = w - (int64_t)b * groups;
    const int rg = (int)(gq / KT), kt = (int)(gq % KT);
    const int rp = rg * 32 + lane;
    const int E = row_exp(p.expo[(int64_t)b * p.Rp + rp]);
    const int rt = rp / p.rowtile, rr = rp % p.rowtile;
#pragma unroll 1
    for (int kg = 0; kg < BK / 8; ++kg) {
      uint32_t packed[S][4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        uint32_t w[S];
        plane_words<S>(embedded(p, b, rp, kt * BK + kg * 8 + j),
                       embedded(p, b, rp, kt * BK + kg * 8 + j + 1), E, w);
#pragma unroll
        for (int s = 0; s < S; ++s) packed[s][j / 2] = w[s];
      }
      const int64_t off = (int64_t)b * p.s_out + ((int64_t)rt * KT + kt) * ((int64_t)p.rowtile * BK) +
                          ((rr / 8) * (BK / 8) + kg) * 64 + (rr % 8) * 8;
#pragma unroll
      for (int s = 0; s < S; ++s)
        *reinterpret_cast<uint4*>(p.planes + s * p.plane_elems + off) =
            make_uint4(packed[s][0], packed[s][1], packed[s][2], packed[s][3]);
    }
  }
}

// ---------------------------------------------------------------- MMA kernel
struct KArgs {
  const __nv_bfloat16 *A, *B;  // digit planes
  int64_t a_plane, b_plane;    // elements per plane
  int64_t sA, sB;              // per-batch element strides within a plane
  const int *ea, *eb;          // row scale exponents of A' [batch][Mp] and B' [batch][Np]
  int KT, kpr, ranges;
  int zs;                      // batch * ranges (work items per output tile)
  float2* P;                   // unscaled (sum, compensation) [batch*ranges][Mp][Np] when ranges > 1
  bool force_p;                // partials even with one range (3M products)
  int Mp, Np;
  int* err;
  long long wait;              // budget (clock cycles) of the MMA and epilogue waits
  double* C;
  bool cplx;
  int M, N, mode;              // logical output extents; mode 0 real, 1 stacked rows, 2 stacked cols
  int64_t ldm, ldn, sC;  // output strides of GEMM rows and columns, batch
  OutModes out;          // C = alpha D + beta C
};

// Work list of one persistent launch.  OneGemm: the items of one GEMM (its
// output tiles times its K ranges).  GemmGroup: several GEMMs of one tile
// configuration in one launch (the grouped ladder of several propagations):
// GEMM p owns the items [first[p], first[p+1]) and reads and writes only its
// own operands, so each tile is computed exactly as in a launch of its GEMM
// alone.  A pipeline timeout marks every GEMM of the launch failed, since the
// CTA that gave up leaves the rest of its items undone.
constexpr int kMaxGroup = 16;
struct KGroup {
  int n = 0;
  int first[kMaxGroup + 1] = {};
  KArgs g[kMaxGroup];
};
static_assert(sizeof(KGroup) <= 4096, "the grouped kernel's table must fit 4 KB of parameters");

template <int BN>
struct OneGemm {
  const KArgs& g;
  __device__ int items() const { return (g.Mp / BM) * (g.Np / BN) * g.zs; }
  __device__ const KArgs& at(int w, int& local) const {
    local = w;
    return g;
  }
  __device__ void fail(int code) const { atomicExch(g.err, code); }
};

struct GemmGroup {
  const KGroup& G;
  __device__ int items() const { return G.first[G.n]; }
  __device__ const KArgs& at(int w, int& local) const {
    int p = 0;
    while (p + 1 < G.n && w >= G.first[p + 1]) ++p;
    local = w - G.first[p];
    return G.g[p];
  }
  __device__ void fail(int code) const {
    for (int p = 0; p < G.n; ++p) atomicExch(G.g[p].err, code);
  }
};

template <int S, int BN, class Work>
__device__ __forceinline__ void oz_gemm_body(const Work& work) {
  using CF = Cfg<S, BN>;
  constexpr int CHUNK_KT = CF::CHUNK_KT;
  constexpr int STAGES = CF::STAGES;
  constexpr uint32_t B_TILE = CF::B_TILE;
  constexpr uint32_t STAGE_BYTES = CF::STAGE_BYTES;
  constexpr uint32_t TMEM_COLS = CF::TMEM_COLS;
  constexpr int HALF = CF::COLS;  // columns drained by one epilogue warp
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  constexpr int NBUF = CF::NBUF;
  uint64_t* acc_full = empty + STAGES;  // [NBUF]: chunk accumulated in set i
  uint64_t* acc_empty = acc_full + 2;   // [NBUF]: set i drained
  uint64_t* mma_done = acc_empty + 2;   // teardown: every issued MMA finished
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int* issued = abort_flag + 1;
  int* mmas = issued + 1;              // stages whose MMAs the issuer launched

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // output tiles on one grid axis (row tiles exceed 65535 for long M)
  // Persistent CTAs: work item w = z * tiles + t (t the output tile in
  // rasterization order: groups of 8 row tiles when a 128-row A' tile
  // carries twice the bytes of a 64-row B' tile, else 12), CTA c takes items
  // c, c + gridDim.x, ...; the stage and chunk counters run on across items,
  // so a tile's drain overlaps the next tile's MMAs.
  // Item w of the work list belongs to GEMM g (work.at) as its local item lw.
  const int items = work.items();
  struct Item {
    int m_tile, n_tile, z, b, kt0, nk, nchunks;
  };
  auto item_of = [&](const KArgs& g, int lw) {
    Item it;
    const int m_tiles = g.Mp / BM, n_tiles = g.Np / BN;
    const int tiles = m_tiles * n_tiles;
    it.z = lw / tiles;
    grouped_tile(lw - it.z * tiles, m_tiles, n_tiles, BN == 64 ? 8 : 12, &it.m_tile, &it.n_tile);
    it.b = it.z / g.ranges;
    const int rg = it.z % g.ranges;
    it.kt0 = rg * g.kpr;
    it.nk = max(min(g.KT, it.kt0 + g.kpr) - it.kt0, 0);
    it.nchunks = (it.nk + CHUNK_KT - 1) / CHUNK_KT;
    return it;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], CF::EPI);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    *issued = 0;
    *mmas = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    int kg = 0;  // k tiles issued so far (all items)
    for (int w = blockIdx.x; w < items && !*(volatile int*)abort_flag; w += gridDim.x) {
      int lw;
      const KArgs& g = work.at(w, lw);
      const Item it = item_of(g, lw);
      const __nv_bfloat16* A = g.A + it.b * g.sA + (int64_t)it.m_tile * g.KT * (BM * BK);
      const __nv_bfloat16* B = g.B + it.b * g.sB + (int64_t)it.n_tile * g.KT * (BN * BK);
      for (int k = 0; k < it.nk; ++k, ++kg) {
        const int s = kg % STAGES;
        if (kg >= STAGES &&
            !mbar_wait_or_abort(&empty[s], ((kg / STAGES) - 1) & 1, abort_flag)) {
          if (!*(volatile int*)abort_flag) work.fail(11);
          *abort_flag = 1;
          break;
        }
        uint8_t* st = smem + s * STAGE_BYTES;
        const int64_t kt = it.kt0 + k;
        mbar_expect_tx(&full[s], STAGE_BYTES);
#pragma unroll
        for (int pl = 0; pl < S; ++pl)
          bulk_load(st + pl * A_TILE, A + pl * g.a_plane + kt * (BM * BK), A_TILE, &full[s]);
#pragma unroll
        for (int pl = 0; pl < S; ++pl)
          bulk_load(st + S * A_TILE + pl * B_TILE, B + pl * g.b_plane + kt * (BN * BK), B_TILE,
                    &full[s]);
        *issued = kg + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // diagonal d = s + t (planes s, t counted from 0) accumulates in columns
    // [d*BN, (d+1)*BN); a chunk's first MMA into d (s = 0) starts it afresh;
    // chunk jg (counted over all items) uses accumulator set jg % NBUF
    const uint32_t idesc = idesc_bf16(BN, CF::F16);
    int kg = 0, jg = 0;
    bool stop = false;
    for (int w = blockIdx.x; w < items && !stop; w += gridDim.x) {
      int lw;
      const KArgs& g = work.at(w, lw);
      const Item it = item_of(g, lw);
      for (int k = 0; k < it.nk; ++k, ++kg) {
        const int kin = k % CHUNK_KT;
        const int j = jg + k / CHUNK_KT;
        if (kin == 0) {
          // chunk j reuses accumulator set j % NBUF once chunk j - NBUF drained
          const int jj = j - NBUF;
          if (jj >= 0 && !mbar_wait(&acc_empty[jj % NBUF], (jj / NBUF) & 1, g.wait)) {
            *abort_flag = 1;
            work.fail(14);
            stop = true;
            break;
          }
        }
        const int s = kg % STAGES;
        if (!mbar_wait(&full[s], (kg / STAGES) & 1, g.wait)) {
          *abort_flag = 1;
          work.fail(12);
          stop = true;
          break;
        }
        tc_fence_after();
        *mmas = kg + 1;
        const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
        for (int sa = 0; sa < S; ++sa) {
#pragma unroll
          for (int sb = 0; sb < S - sa; ++sb) {
            // accumulator of the pair: its diagonal, (fused) leading / rest, or
            // (FP16 planes) the only one; the first pair into an accumulator in
            // a chunk starts it afresh
            const int acc = CF::F16 ? 0 : (CF::FUSED ? (sa + sb > 0 ? 1 : 0) : sa + sb);
            const bool first_pair = sa == 0 && (CF::F16 ? sb == 0 : (!CF::FUSED || sb <= 1));
            const uint32_t dt = tmem + (uint32_t)(((j % NBUF) * CF::NACC + acc) * BN);
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
              const uint64_t ad = smem_desc(base + sa * A_TILE + ks * 256, 128, 512);
              const uint64_t bd =
                  smem_desc(base + S * A_TILE + sb * B_TILE + ks * 256, 128, 512);
              mma_bf16(dt, ad, bd, idesc, (kin > 0 || ks > 0 || !first_pair) ? 1u : 0u);
            }
          }
        }
        mma_commit(&empty[s]);
        if (kin == CHUNK_KT - 1 || k == it.nk - 1) mma_commit(&acc_full[j % NBUF]);
      }
      jg += it.nchunks;
    }
  } else if (warp >= 2) {
    const int q = warp % 4;
    const int h = (warp - 2) / 4;
    const int row = 32 * q + lane;
    int jg = 0;
    for (int w = blockIdx.x; w < items; w += gridDim.x) {
      int lw;
      const KArgs& g = work.at(w, lw);
      const Item it = item_of(g, lw);
      // running chunk sums (and their compensations when CF::COMP)
      float sum[HALF], cmp[CF::COMP ? HALF : 1];
#pragma unroll
      for (int v = 0; v < HALF; ++v) sum[v] = 0.0f;
#pragma unroll
      for (int v = 0; v < (CF::COMP ? HALF : 1); ++v) cmp[v] = 0.0f;
      auto cmpv = [&](int v) -> float {
        if constexpr (CF::COMP)
          return cmp[v];
        else
          return 0.0f;
      };
      bool ok = it.nk > 0 && !*(volatile int*)abort_flag;
#pragma unroll 1
      for (int jl = 0; ok && jl < it.nchunks; ++jl) {
        const int j = jg + jl, set = j % NBUF;
        if (!mbar_wait(&acc_full[set], (j / NBUF) & 1, g.wait)) {
          ok = false;
          *abort_flag = 1;
          work.fail(13);
          break;
        }
        tc_fence_after();
#pragma unroll 1
        for (int d = 0; d < CF::NACC; ++d) {
          // 2^(2 - 8 (d + 2)) for diagonal d; the fused accumulators both carry
          // the weight of the leading diagonal (the rest is pre-scaled); FP16
          // planes carry 2^-15 each
          const float wd = CF::F16 ? __int_as_float((127 - 30) << 23)
                                   : __int_as_float((127 - 14 - 8 * (CF::FUSED ? 0 : d)) << 23);
#pragma unroll
          for (int c = 0; c < HALF; c += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) +
                          (uint32_t)((set * CF::NACC + d) * BN + h * HALF + c),
                      r);
#pragma unroll
            for (int v = 0; v < 16; ++v) {
              if constexpr (CF::COMP)
                two_sum_acc(sum[c + v], cmp[c + v], __uint_as_float(r[v]) * wd);
              else
                sum[c + v] += __uint_as_float(r[v]) * wd;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[set]);
      }
      jg += it.nchunks;
      if (!ok) break;
      const int mr = it.m_tile * BM + row;
      const int er = row_exp(g.ea[(int64_t)it.b * g.Mp + mr]);
      if (g.ranges == 1 && !g.force_p) {
        int m = mr, part = 0;
        if (g.mode == 1 && mr >= g.M) {
          m = mr - g.M;
          part = 1;
        }
        const bool row_ok = g.mode == 1 ? mr < 2 * g.M : mr < g.M;
        if (row_ok) {
          const int64_t rbase = (int64_t)it.b * g.sC + (int64_t)m * g.ldm;
          with_out_modes(g.out, [&](auto ga, auto bm) {
            constexpr int GA = decltype(ga)::value, BMODE = decltype(bm)::value;
#pragma unroll
            for (int v = 0; v < HALF; ++v) {
              const int nr = it.n_tile * BN + h * HALF + v;
              int n = nr, pt = part;
              if (g.mode == 2 && nr >= g.N) {
                n = nr - g.N;
                pt = 1;
              }
              if (n >= g.N || (g.mode == 2 ? nr >= 2 * g.N : nr >= g.N)) continue;
              const int ec = row_exp(g.eb[(int64_t)it.b * g.Np + nr]);
              const double val = CF::COMP ? scaled_value(sum[v], cmpv(v), er, ec)
                                          : scaled_value1(sum[v], er, ec);
              out_update<GA, BMODE>(g.C + (g.cplx ? 2 : 1) * (rbase + (int64_t)n * g.ldn) + pt,
                                    val, g.out);
            }
          });
        }
      } else {
        float4* dst = reinterpret_cast<float4*>(g.P + ((int64_t)it.z * g.Mp + mr) * g.Np +
                                                (int64_t)it.n_tile * BN + h * HALF);
#pragma unroll
        for (int v = 0; v < HALF / 2; ++v)
          dst[v] = make_float4(sum[2 * v], cmpv(2 * v), sum[2 * v + 1], cmpv(2 * v + 1));
      }
    }
  }
  // teardown after an abandoned pipeline: let the issued copies land and the
  // issued MMAs finish (bounded) before the tensor memory is freed
  tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) {
      const int n = *issued;
      for (int k = n > STAGES ? n - STAGES : 0; k < n; ++k)
        mbar_wait(&full[k % STAGES], (k / STAGES) & 1);
    }
    if (warp == 1 && lane == 0 && *mmas > 0) {
      mma_commit(mma_done);
      mbar_wait(mma_done, 0);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

template <int S, int BN>
__global__ void __launch_bounds__(Cfg<S, BN>::THREADS, 1) oz_gemm_kernel(KArgs g) {
  oz_gemm_body<S, BN>(OneGemm<BN>{g});
}

template <int S, int BN>
__global__ void __launch_bounds__(Cfg<S, BN>::THREADS, 1)
    oz_gemm_group_kernel(const __grid_constant__ KGroup G) {
  oz_gemm_body<S, BN>(GemmGroup{G});
}

// ---------------------------------------------------------------- finalize
struct FinArgs {
  const float2* P;  // unscaled (sum, compensation) [batch*ranges][Mp][Np]
  const int *ea, *eb;
  int Mp, Np, ranges;
  int M, N, mode;
  double* C;
  bool cplx;
  int64_t ldm, ldn, sC;  // output strides of GEMM rows and columns, batch
  OutModes out;          // C = alpha D + beta C
};

// Whether the MMA kernel of S planes and BN-column tiles writes compensated
// partial pairs (else plain FP32 sums with zero compensations).
inline bool oz_comp(int S, int bn) {
  static_assert(Cfg<2, 32>::COMP && Cfg<2, 128>::COMP && Cfg<3, 32>::COMP &&
                    Cfg<3, 128>::COMP && Cfg<7, 32>::COMP && Cfg<7, 64>::COMP,
                "only the 256-column tiles drain plain sums");
  return !(S == 2 && bn == 256) || Cfg<2, 256>::COMP;
}

__global__ void oz_finalize_kernel(FinArgs f, int batch) {
  const int64_t per = (int64_t)f.M * f.N;
  with_out_modes(f.out, [&](auto ga, auto bm) {
    constexpr int GA = decltype(ga)::value, BMODE = decltype(bm)::value;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * batch;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int b = (int)(e / per);
      const int64_t q = e - (int64_t)b * per;
      const int m = (int)(q / f.N), n = (int)(q % f.N);
      double* c = f.C + (f.cplx ? 2 : 1) * ((int64_t)b * f.sC + (int64_t)m * f.ldm + (int64_t)n * f.ldn);
      const int parts = f.cplx ? 2 : 1;
      for (int part = 0; part < parts; ++part) {
        const int mr = f.mode == 1 ? m + part * f.M : m;
        const int nr = f.mode == 2 ? n + part * f.N : n;
        float su = 0.0f, cm = 0.0f;
        // ranges in order, four loads in flight at a time
        const float2* pp = f.P + ((int64_t)b * f.ranges * f.Mp + mr) * f.Np + nr;
        const int64_t zs = (int64_t)f.Mp * f.Np;
        int z = 0;
        for (; z + 4 <= f.ranges; z += 4) {
          float2 q[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) q[u] = pp[(z + u) * zs];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            two_sum_acc(su, cm, q[u].x);
            cm += q[u].y;
          }
        }
        for (; z < f.ranges; ++z) {
          const float2 pz = pp[z * zs];
          two_sum_acc(su, cm, pz.x);
          cm += pz.y;
        }
        const int er = row_exp(f.ea[(int64_t)b * f.Mp + mr]);
        const int ec = row_exp(f.eb[(int64_t)b * f.Np + nr]);
        out_update<GA, BMODE>(c + part, scaled_value(su, cm, er, ec), f.out);
      }
    }
  });
}

inline int roundup(int x, int m) { return (x + m - 1) / m * m; }

struct Plan {
  int mode;  // 0 RR, 1 CR, 2 RC, 3 CC
  int bn;    // output tile width (rows of B' per tile)
  int Mp, Np, Kp, KT, ranges, kpr;
  int64_t a_elems, b_elems;  // BF16 per digit plane
  int64_t p_elems;           // float2 partials (0 with one range)
};

}  // namespace oz

// Output-tile width (rows of B' per tile) of the digit-plane kernels.
int oz_tile_n(int64_t rows_b, int S) {
  if (rows_b <= 32) return 32;
  if (S == 2 && rows_b > 128) return 256;
  return S <= 3 ? 128 : 64;
}

namespace oz {

Plan plan(const GemmDesc& d, int S) {
  Plan p;
  p.mode = (d.Acplx && d.part_a < 0 ? 1 : 0) + (d.Bcplx && d.part_b < 0 ? 2 : 0);
  const int Ar = p.mode == 1 ? 2 * d.M : d.M;
  const int Ak = p.mode == 3 ? 2 * d.K : d.K;
  const int Br = (p.mode & 2) ? 2 * d.N : d.N;
  // 32 columns for a narrow B', else 64 with seven planes (one accumulator
  // set of 7 x 64 columns), 128 with three (two sets of two 128-column
  // accumulators: the next chunk accumulates while the last drains) and 256
  // with two (two sets of one): a 128 x 256 MMA reads a quarter fewer
  // shared-memory bytes per product than two 128 x 128 ones
  p.bn = oz_tile_n(Br, S);
  p.Mp = roundup(std::max(Ar, 1), BM);
  p.Np = roundup(std::max(Br, 1), p.bn);
  p.Kp = roundup(std::max(Ak, 1), BK);
  p.KT = p.Kp / BK;
  // K ranges: fewest waves x k tiles per CTA, a range costing about four k
  // tiles for writing and re-reading its partial tile
  const int64_t tiles = (int64_t)(p.Mp / BM) * (p.Np / p.bn) * d.batch;
  double best = 0.0;
  p.ranges = 1;
  p.kpr = p.KT;
  for (int r = 1; r <= p.KT; ++r) {
    const int kpr = (p.KT + r - 1) / r;
    if ((p.KT + kpr - 1) / kpr != r) continue;
    if ((int64_t)d.batch * r > 65535) break;
    const double waves = (double)((tiles * r + 147) / 148);
    const double cost = waves * (kpr + (r > 1 ? 4 : 0));
    if (r == 1 || cost < best) {
      best = cost;
      p.ranges = r;
      p.kpr = kpr;
    }
  }
  if (d.one_range) {  // tiles independent of the rest of the launch
    p.ranges = 1;
    p.kpr = p.KT;
  }
  p.a_elems = (int64_t)p.Mp * p.Kp * d.batch;
  p.b_elems = (int64_t)p.Np * p.Kp * d.batch;
  p.p_elems = (p.ranges == 1 && !d.force_partials) ? 0 : (int64_t)p.ranges * p.Mp * p.Np * d.batch;
  return p;
}

// 3M combine of the digit-plane products: P holds [3][ranges][Mp][Np]
// unscaled pairs, product b scaled by the row exponents ea[b][m], eb[b][n]
// of its packed operands; C = alpha (P1 - P2 + i (P3 - P1 - P2)) + beta C.
// PLAIN: one range of plain FP32 sums (zero compensations), converted
// without an FP64 add.
template <bool PLAIN>
__global__ void oz_combine_3m_kernel(FinArgs f) {
  const int64_t per = (int64_t)f.M * f.N;
  const int64_t zs = (int64_t)f.Mp * f.Np;
  // the partials and the output never overlap
  const float2* __restrict__ Pr = f.P;
  double* __restrict__ Cr = f.C;
  with_out_modes(f.out, [&](auto ga, auto bm) {
    constexpr int GA = decltype(ga)::value, BMODE = decltype(bm)::value;
#pragma unroll 2
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int m = (int)(e / f.N), n = (int)(e % f.N);
      double v[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float2* pp = Pr + ((int64_t)b * f.ranges * f.Mp + m) * f.Np + n;
        const int er = row_exp(f.ea[(int64_t)b * f.Mp + m]);
        const int ec = row_exp(f.eb[(int64_t)b * f.Np + n]);
        if constexpr (PLAIN) {
          v[b] = scaled_value1(pp[0].x, er, ec);
        } else {
          float su = 0.0f, cm = 0.0f;
          for (int z = 0; z < f.ranges; ++z) {
            const float2 q = pp[z * zs];
            two_sum_acc(su, cm, q.x);
            cm += q.y;
          }
          v[b] = scaled_value(su, cm, er, ec);
        }
      }
      const double re = v[0] - v[1], im = v[2] - v[0] - v[1];
      double* c = Cr + 2 * ((int64_t)m * f.ldm + (int64_t)n * f.ldn);
      out_update<GA, BMODE>(c, re, f.out);
      out_update<GA, BMODE>(c + 1, im, f.out);
    }
  });
}

int grid_of(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 148 * 16); }

void pack(PackArgs pa, int64_t elems, int batch, int S, cudaStream_t st) {
  const int64_t rows = (int64_t)batch * pa.Rp;
  RT_CUDA(cudaMemsetAsync(pa.expo, 0, sizeof(int) * rows, st));
  if (pa.rows_fast) {
    oz_expo_rows_kernel<<<grid_of(rows * ((pa.Kp + kExpoSeg - 1) / kExpoSeg)), 256, 0, st>>>(
        pa, batch);
  } else {
    const int64_t units = rows * ((pa.Kp + kExpoWarpSeg - 1) / kExpoWarpSeg);
    oz_expo_kernel<<<(int)std::min<int64_t>((units * 32 + 255) / 256, 148 * 16), 256, 0, st>>>(
        pa, batch);
  }
  RT_CHECK_LAUNCH();
  // 32 x 32 blocks (rows-fast sources) or 8 x 32 blocks, one warp each
  const int64_t units = elems / (pa.rows_fast ? 1024 : 256);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((units * 32 + 255) / 256, 148 * 16));
  if (pa.rows_fast) {
    if (S == 2)
      oz_digits_rows_kernel<2><<<grid, 256, 0, st>>>(pa, batch);
    else if (S == 3)
      oz_digits_rows_kernel<3><<<grid, 256, 0, st>>>(pa, batch);
    else
      oz_digits_rows_kernel<7><<<grid, 256, 0, st>>>(pa, batch);
  } else if (S == 2) {
    oz_digits_kernel<2><<<grid, 256, 0, st>>>(pa, batch);
  } else if (S == 3) {
    oz_digits_kernel<3><<<grid, 256, 0, st>>>(pa, batch);
  } else {
    oz_digits_kernel<7><<<grid, 256, 0, st>>>(pa, batch);
  }
  RT_CHECK_LAUNCH();
}

}  // namespace oz

OzLayout gemm_oz_layout(const GemmDesc& d, int S) {
  const oz::Plan p = oz::plan(d, S);
  OzLayout l;
  l.planes = S;
  l.a_elems = p.a_elems;
  l.b_elems = p.b_elems;
  l.a_rows = (int64_t)p.Mp * d.batch;
  l.b_rows = (int64_t)p.Np * d.batch;
  l.p_elems = p.p_elems;
  l.ranges = p.ranges;
  l.padded_flops = 2.0 * S * (S + 1) / 2 * (double)p.Mp * p.Np * p.Kp * d.batch;
  return l;
}

void gemm_oz_init() {
  auto set = [](auto kernel, size_t smem) {
    RT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  };
  set(oz::oz_gemm_kernel<7, 64>, oz::Cfg<7, 64>::SMEM);
  set(oz::oz_gemm_kernel<7, 32>, oz::Cfg<7, 32>::SMEM);
  set(oz::oz_gemm_kernel<3, 128>, oz::Cfg<3, 128>::SMEM);
  set(oz::oz_gemm_kernel<3, 32>, oz::Cfg<3, 32>::SMEM);
  set(oz::oz_gemm_kernel<2, 256>, oz::Cfg<2, 256>::SMEM);
  set(oz::oz_gemm_kernel<2, 128>, oz::Cfg<2, 128>::SMEM);
  set(oz::oz_gemm_kernel<2, 32>, oz::Cfg<2, 32>::SMEM);
  set(oz::oz_gemm_group_kernel<7, 64>, oz::Cfg<7, 64>::SMEM);
  set(oz::oz_gemm_group_kernel<7, 32>, oz::Cfg<7, 32>::SMEM);
  set(oz::oz_gemm_group_kernel<3, 128>, oz::Cfg<3, 128>::SMEM);
  set(oz::oz_gemm_group_kernel<3, 32>, oz::Cfg<3, 32>::SMEM);
  set(oz::oz_gemm_group_kernel<2, 256>, oz::Cfg<2, 256>::SMEM);
  set(oz::oz_gemm_group_kernel<2, 128>, oz::Cfg<2, 128>::SMEM);
  set(oz::oz_gemm_group_kernel<2, 32>, oz::Cfg<2, 32>::SMEM);
}

void gemm_oz_pack_a(const GemmDesc& d, int S, uint16_t* planes, int* expo, cudaStream_t st,
                    int slot, int nslots) {
  if (d.M <= 0 || d.N <= 0 || d.batch <= 0) return;
  const oz::Plan p = oz::plan(d, S);
  oz::PackArgs pa{};
  pa.src = d.A;
  pa.cplx = d.Acplx;
  pa.s_r = d.transA ? 1 : d.lda;
  pa.s_c = d.transA ? d.lda : 1;
  pa.s_b = d.strideA;
  pa.R = d.M;
  pa.C = d.K;
  pa.mode = p.mode == 1 ? 1 : (p.mode == 3 ? 2 : 0);
  pa.part = d.Acplx ? d.part_a : -1;
  pa.Rp = p.Mp;
  pa.Kp = p.Kp;
  pa.rowtile = oz::BM;
  pa.s_out = (int64_t)p.Mp * p.Kp;
  pa.planes = reinterpret_cast<__nv_bfloat16*>(planes) + (int64_t)slot * pa.s_out * d.batch;
  pa.plane_elems = p.a_elems * nslots;
  pa.expo = expo + (int64_t)slot * p.Mp * d.batch;
  pa.view = d.va;
  pa.rows_fast = d.va.rdims ? (d.va.rstr[d.va.rdims - 1] == 1 && d.va.kstr[d.va.kdims - 1] != 1)
                            : (pa.s_r == 1 && pa.s_c != 1);
  oz::pack(pa, p.a_elems, d.batch, S, st);
}

void gemm_oz_pack_b(const GemmDesc& d, int S, uint16_t* planes, int* expo, cudaStream_t st,
                    int slot, int nslots) {
  if (d.M <= 0 || d.N <= 0 || d.batch <= 0) return;
  const oz::Plan p = oz::plan(d, S);
  oz::PackArgs pb{};
  pb.src = d.B;
  pb.cplx = d.Bcplx;
  pb.s_r = d.transB ? d.ldb : 1;  // rows of B' are the output columns n
  pb.s_c = d.transB ? 1 : d.ldb;
  pb.s_b = d.strideB;
  pb.R = d.N;
  pb.C = d.K;
  pb.mode = p.mode == 2 ? 1 : (p.mode == 3 ? 3 : 0);
  pb.part = d.Bcplx ? d.part_b : -1;
  pb.Rp = p.Np;
  pb.Kp = p.Kp;
  pb.rowtile = p.bn;
  pb.s_out = (int64_t)p.Np * p.Kp;
  pb.planes = reinterpret_cast<__nv_bfloat16*>(planes) + (int64_t)slot * pb.s_out * d.batch;
  pb.plane_elems = p.b_elems * nslots;
  pb.expo = expo + (int64_t)slot * p.Np * d.batch;
  pb.view = d.vb;
  pb.rows_fast = d.vb.rdims ? (d.vb.rstr[d.vb.rdims - 1] == 1 && d.vb.kstr[d.vb.kdims - 1] != 1)
                            : (pb.s_r == 1 && pb.s_c != 1);
  oz::pack(pb, p.b_elems, d.batch, S, st);
}

namespace oz {

// Kernel arguments of one GEMM whose operands are packed for plan p.
KArgs kargs_of(const GemmDesc& d, const Plan& p, const uint16_t* A, const int* ea,
               const uint16_t* B, const int* eb, float2* P, int* err) {
  if ((int64_t)(p.Np / p.bn) * (p.Mp / BM) > 0x7fffffff || (int64_t)d.batch * p.ranges > 65535)
    throw Error(-1, "gemm_oz: grid too large");
  KArgs g{};
  g.A = reinterpret_cast<const __nv_bfloat16*>(A);
  g.B = reinterpret_cast<const __nv_bfloat16*>(B);
  g.a_plane = p.a_elems;
  g.b_plane = p.b_elems;
  g.sA = (int64_t)p.Mp * p.Kp;
  g.sB = (int64_t)p.Np * p.Kp;
  g.ea = ea;
  g.eb = eb;
  g.KT = p.KT;
  g.kpr = p.kpr;
  g.ranges = p.ranges;
  g.P = P;
  g.force_p = d.force_partials;
  g.Mp = p.Mp;
  g.Np = p.Np;
  g.err = err;
  g.wait = d.wait_cycles > 0 ? d.wait_cycles : tc5::kWaitCycles;
  g.C = d.C;
  g.cplx = d.Acplx || d.Bcplx;
  g.M = d.M;
  g.N = d.N;
  g.mode = p.mode == 1 ? 1 : (p.mode >= 2 ? 2 : 0);
  g.ldm = d.transC ? 1 : d.ldc;
  g.ldn = d.transC ? d.ldc : 1;
  g.sC = d.strideC;
  g.out = out_modes(d.alpha, d.beta);
  g.zs = d.batch * p.ranges;
  if ((int64_t)(p.Np / p.bn) * (p.Mp / BM) * g.zs > 0x7fffffff)
    throw Error(-1, "gemm_oz: too many tiles");
  return g;
}

// Work items (output tiles times K ranges) of a GEMM.
int64_t items_of(const KArgs& g, int bn) { return (int64_t)(g.Np / bn) * (g.Mp / BM) * g.zs; }

// One grouped launch: persistent CTAs over the combined items of G.
void launch_group(const KGroup& G, int S, int bn, cudaStream_t st) {
  const int grid = (int)std::min<int64_t>(G.first[G.n], 148);
  if (grid <= 0) return;
  if (S == 2 && bn == 256)
    oz_gemm_group_kernel<2, 256><<<grid, Cfg<2, 256>::THREADS, Cfg<2, 256>::SMEM, st>>>(G);
  else if (S == 2 && bn == 128)
    oz_gemm_group_kernel<2, 128><<<grid, Cfg<2, 128>::THREADS, Cfg<2, 128>::SMEM, st>>>(G);
  else if (S == 2)
    oz_gemm_group_kernel<2, 32><<<grid, Cfg<2, 32>::THREADS, Cfg<2, 32>::SMEM, st>>>(G);
  else if (S == 3 && bn == 128)
    oz_gemm_group_kernel<3, 128><<<grid, Cfg<3, 128>::THREADS, Cfg<3, 128>::SMEM, st>>>(G);
  else if (S == 3)
    oz_gemm_group_kernel<3, 32><<<grid, Cfg<3, 32>::THREADS, Cfg<3, 32>::SMEM, st>>>(G);
  else if (bn == 32)
    oz_gemm_group_kernel<7, 32><<<grid, Cfg<7, 32>::THREADS, Cfg<7, 32>::SMEM, st>>>(G);
  else
    oz_gemm_group_kernel<7, 64><<<grid, Cfg<7, 64>::THREADS, Cfg<7, 64>::SMEM, st>>>(G);
  RT_CHECK_LAUNCH();
}

}  // namespace oz

void gemm_oz_mma(const GemmDesc& d, int S, const uint16_t* A, const int* ea, const uint16_t* B,
                 const int* eb, float2* P, int* err, cudaStream_t st) {
  if (d.M <= 0 || d.N <= 0 || d.batch <= 0) return;
  const oz::Plan p = oz::plan(d, S);
  const oz::KArgs g = oz::kargs_of(d, p, A, ea, B, eb, P, err);
  // persistent CTAs: one per SM (the kernel takes most of the shared memory)
  const int grid = (int)std::min<int64_t>(oz::items_of(g, p.bn), 148);
  using namespace oz;
  if (S == 2 && p.bn == 256)
    oz_gemm_kernel<2, 256><<<grid, Cfg<2, 256>::THREADS, Cfg<2, 256>::SMEM, st>>>(g);
  else if (S == 2 && p.bn == 128)
    oz_gemm_kernel<2, 128><<<grid, Cfg<2, 128>::THREADS, Cfg<2, 128>::SMEM, st>>>(g);
  else if (S == 2)
    oz_gemm_kernel<2, 32><<<grid, Cfg<2, 32>::THREADS, Cfg<2, 32>::SMEM, st>>>(g);
  else if (S == 3 && p.bn == 128)
    oz_gemm_kernel<3, 128><<<grid, Cfg<3, 128>::THREADS, Cfg<3, 128>::SMEM, st>>>(g);
  else if (S == 3)
    oz_gemm_kernel<3, 32><<<grid, Cfg<3, 32>::THREADS, Cfg<3, 32>::SMEM, st>>>(g);
  else if (p.bn == 32)
    oz_gemm_kernel<7, 32><<<grid, Cfg<7, 32>::THREADS, Cfg<7, 32>::SMEM, st>>>(g);
  else
    oz_gemm_kernel<7, 64><<<grid, Cfg<7, 64>::THREADS, Cfg<7, 64>::SMEM, st>>>(g);
  RT_CHECK_LAUNCH();
}

int gemm_oz_mma_group(const OzGroupGemm* gs, int n, int S, cudaStream_t st) {
  // GEMMs by output-tile width (one kernel configuration each), in order
  std::vector<std::pair<int, oz::KArgs>> ks;
  for (int i = 0; i < n; ++i) {
    const GemmDesc& d = gs[i].d;
    if (d.M <= 0 || d.N <= 0 || d.batch <= 0) continue;
    const oz::Plan p = oz::plan(d, S);
    if (p.ranges != 1 || d.force_partials)
      throw Error(-1, "gemm_oz_mma_group: a grouped GEMM takes one K range per tile");
    ks.push_back({p.bn, oz::kargs_of(d, p, gs[i].A, gs[i].ea, gs[i].B, gs[i].eb, nullptr,
                                     gs[i].err)});
  }
  int launches = 0;
  std::vector<bool> done(ks.size(), false);
  for (size_t i = 0; i < ks.size(); ++i) {
    if (done[i]) continue;
    const int bn = ks[i].first;
    oz::KGroup G;
    for (size_t j = i; j < ks.size(); ++j) {
      if (done[j] || ks[j].first != bn) continue;
      const int64_t it = oz::items_of(ks[j].second, bn);
      if (G.n == oz::kMaxGroup || (int64_t)G.first[G.n] + it > 0x7fffffff) {
        oz::launch_group(G, S, bn, st);
        ++launches;
        G = oz::KGroup();
      }
      G.g[G.n] = ks[j].second;
      G.first[G.n + 1] = G.first[G.n] + (int)it;
      ++G.n;
      done[j] = true;
    }
    oz::launch_group(G, S, bn, st);
    ++launches;
  }
  return launches;
}

void gemm_oz_finalize(const GemmDesc& d, int S, const int* ea, const int* eb, const float2* P,
                      cudaStream_t st) {
  if (d.M <= 0 || d.N <= 0 || d.batch <= 0) return;
  const oz::Plan p = oz::plan(d, S);
  if (p.ranges == 1 && !d.force_partials) return;
  oz::FinArgs fa{};
  fa.P = P;
  fa.ea = ea;
  fa.eb = eb;
  fa.Mp = p.Mp;
  fa.Np = p.Np;
  fa.ranges = p.ranges;
  fa.M = d.M;
  fa.N = d.N;
  fa.mode = p.mode == 1 ? 1 : (p.mode >= 2 ? 2 : 0);
  fa.C = d.C;
  fa.cplx = d.Acplx || d.Bcplx;
  fa.ldm = d.transC ? 1 : d.ldc;
  fa.ldn = d.transC ? d.ldc : 1;
  fa.sC = d.strideC;
  fa.out = out_modes(d.alpha, d.beta);
  oz::oz_finalize_kernel<<<oz::grid_of((int64_t)d.M * d.N * d.batch), 256, 0, st>>>(fa, d.batch);
  RT_CHECK_LAUNCH();
}

void gemm_oz_combine_3m(const GemmDesc& d, int S, const int* ea, const int* eb, const float2* P,
                        cudaStream_t st) {
  if (d.M <= 0 || d.N <= 0) return;
  const oz::Plan p = oz::plan(gemm_3m_desc(d), S);
  oz::FinArgs fa{};
  fa.P = P;
  fa.ea = ea;
  fa.eb = eb;
  fa.Mp = p.Mp;
  fa.Np = p.Np;
  fa.ranges = p.ranges;
  fa.M = d.M;
  fa.N = d.N;
  fa.C = d.C;
  fa.cplx = true;
  fa.ldm = d.transC ? 1 : d.ldc;
  fa.ldn = d.transC ? d.ldc : 1;
  fa.out = out_modes(d.alpha, d.beta);
  if (p.ranges == 1 && !oz::oz_comp(S, p.bn))
    oz::oz_combine_3m_kernel<true><<<oz::grid_of((int64_t)d.M * d.N), 256, 0, st>>>(fa);
  else
    oz::oz_combine_3m_kernel<false><<<oz::grid_of((int64_t)d.M * d.N), 256, 0, st>>>(fa);
  RT_CHECK_LAUNCH();
}

}  // namespace rteom
