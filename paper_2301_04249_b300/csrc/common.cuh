// Shared definitions of the RT-EOM-CCSD CUDA library: error handling, the
// device tensor descriptor and the stream-ordered scratch arena.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/rteom.h"

namespace rteom {

// Precision forms of rteom_create: which run their contractions as 16-bit
// planes on the tensor cores, and how many planes per operand.
inline bool valid_precision(int p) {
  return p == RTEOM_FP64 || p == RTEOM_SPLIT_BF16 || p == RTEOM_SPLIT_TF32 ||
         p == RTEOM_FP64_OZAKI || p == RTEOM_SPLIT_FP16;
}
inline bool sliced_form(int p) {
  return p == RTEOM_FP64_OZAKI || p == RTEOM_SPLIT_BF16 || p == RTEOM_SPLIT_FP16;
}
inline int planes_of(int p) {
  return p == RTEOM_SPLIT_BF16 ? 3 : (p == RTEOM_SPLIT_FP16 ? 2 : 7);
}
// The grouped ladder (RTEOM_FLAG_GROUPED) runs on the digit-plane forms with
// the resident ladder blocks and the plain micro-iteration.
inline bool grouped_flags_ok(int precision, int flags) {
  return !(flags & RTEOM_FLAG_GROUPED) ||
         (sliced_form(precision) &&
          !(flags & (RTEOM_FLAG_LADDER_CHOLESKY | RTEOM_FLAG_ANDERSON)));
}

// Error carried from deep inside the library to the C ABI boundary.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define RT_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      throw ::rteom::Error(e_ == cudaErrorMemoryAllocation ? -2 : -3,          \
                           std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                          \
  } while (0)

#define RT_CHECK_LAUNCH() RT_CUDA(cudaGetLastError())

constexpr int kMaxDims = 6;

// IEEE-754 binary32 <-> binary64 conversions on the integer ALUs.  The FP64
// pipe of this part issues about two operations per clock per SM, so the
// elementwise kernels keep FP64 arithmetic to what the result needs and
// convert with bit operations instead.  Both are exact for normal numbers
// and zeros (f64_to_f32 rounds to nearest, ties to even); magnitudes below
// the normal binary32 range become signed zeros, larger ones infinities,
// NaN stays NaN.
#ifdef __CUDACC__
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint64_t man = (uint64_t)(u & 0x7FFFFFu) << 29;
  const uint64_t ex = e == 0xFFu ? 0x7FFull : (uint64_t)(e + 896u);
  return __longlong_as_double(e == 0u ? (long long)sign : (long long)(sign | (ex << 52) | man));
}

__device__ __forceinline__ float f64_to_f32(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7FF);
  const uint64_t m = u & 0xFFFFFFFFFFFFFull;
  if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
  int E = e - 896;
  if (E <= 0) return __uint_as_float(sign);
  uint32_t m23 = (uint32_t)(m >> 29);
  const uint32_t rem = (uint32_t)(m & 0x1FFFFFFFu);
  if (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) ++m23;
  if (m23 == 0x800000u) {
    m23 = 0;
    ++E;
  }
  if (E >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((uint32_t)E << 23) | m23);
}

__device__ __forceinline__ double neg_f64(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

#endif

// Output update c = alpha v + beta c of the GEMM epilogues, finalize and
// combine kernels, with alpha and beta classified once on the host: a
// compare of doubles runs on the FP64 pipe (about two operations per clock
// per SM on this part), and a per-element beta test let the compiler read c
// before knowing it was needed.  alpha = +-1 becomes a sign-bit mask.
struct OutModes {
  long long sign = 0;     // sign-bit mask applied when alpha = +-1
  int general_alpha = 0;  // 1: multiply by alpha
  int bmode = 0;          // 0: beta = 0, 1: beta = 1, 2: general
  double alpha = 1.0, beta = 0.0;
};

inline OutModes out_modes(double alpha, double beta) {
  OutModes o;
  o.alpha = alpha;
  o.beta = beta;
  o.general_alpha = !(alpha == 1.0 || alpha == -1.0);
  o.sign = alpha == -1.0 ? (long long)0x8000000000000000ull : 0ll;
  o.bmode = beta == 0.0 ? 0 : (beta == 1.0 ? 1 : 2);
  return o;
}

#ifdef __CUDACC__
template <int GA, int BMODE>
__device__ __forceinline__ void out_update(double* c, double v, const OutModes& o) {
  if constexpr (GA)
    v *= o.alpha;
  else
    v = __longlong_as_double(__double_as_longlong(v) ^ o.sign);
  if constexpr (BMODE == 0)
    *c = v;
  else if constexpr (BMODE == 1)
    *c = *c + v;
  else
    *c = fma(o.beta, *c, v);
}

template <int V>
struct OutMode {
  static constexpr int value = V;
};

// Calls f(OutMode<GA>, OutMode<BMODE>) for the modes of o, so that the
// caller's loop is compiled once per mode with no test inside.
template <class F>
__device__ __forceinline__ void with_out_modes(const OutModes& o, F&& f) {
  if (o.general_alpha) {
    if (o.bmode == 0)
      f(OutMode<1>{}, OutMode<0>{});
    else if (o.bmode == 1)
      f(OutMode<1>{}, OutMode<1>{});
    else
      f(OutMode<1>{}, OutMode<2>{});
  } else {
    if (o.bmode == 0)
      f(OutMode<0>{}, OutMode<0>{});
    else if (o.bmode == 1)
      f(OutMode<0>{}, OutMode<1>{});
    else
      f(OutMode<0>{}, OutMode<2>{});
  }
}

// Compensated FP32 accumulation (Knuth's TwoSum): s + c carries the running
// sum to about twice the FP32 precision.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}
#endif

// Row-major device tensor, FP64 real or complex128 (interleaved re, im).
struct Tensor {
  double* p = nullptr;
  int nd = 0;
  int64_t dim[kMaxDims] = {0, 0, 0, 0, 0, 0};
  bool cplx = false;
  bool constant = false;  // contents fixed for the context's lifetime (integrals)
  bool released = false;  // device copy freed: usable only through cached tensor-core packs

  int64_t numel() const {
    int64_t n = 1;
    for (int k = 0; k < nd; ++k) n *= dim[k];
    return n;
  }
  int64_t doubles() const { return numel() * (cplx ? 2 : 1); }
};

inline Tensor make_tensor(double* p, bool cplx, std::initializer_list<int64_t> dims) {
  Tensor t;
  t.p = p;
  t.cplx = cplx;
  for (int64_t d : dims) t.dim[t.nd++] = d;
  return t;
}

// Bump allocator over one device buffer.  Allocation order follows stream
// order, so a region released by mark/release can be reused by later
// kernels on the same stream.
class Arena {
 public:
  Arena() = default;
  void init(double* base, int64_t doubles) {
    base_ = base;
    cap_ = doubles;
    top_ = 0;
    peak_ = 0;
  }
  double* alloc(int64_t doubles) {
    int64_t n = (doubles + 31) & ~int64_t(31);  // 256-byte alignment
    if (top_ + n > cap_)
      throw Error(-2, "scratch arena exhausted: need " + std::to_string((top_ + n) * 8) +
                          " bytes of " + std::to_string(cap_ * 8));
    double* p = base_ + top_;
    top_ += n;
    if (top_ > peak_) peak_ = top_;
    return p;
  }
  Tensor tensor(bool cplx, std::initializer_list<int64_t> dims) {
    Tensor t = make_tensor(nullptr, cplx, dims);
    t.p = alloc(t.doubles());
    return t;
  }
  int64_t mark() const { return top_; }
  void release(int64_t m) { top_ = m; }
  int64_t peak_bytes() const { return peak_ * 8; }
  bool measuring() const { return base_ == nullptr; }

 private:
  double* base_ = nullptr;
  int64_t cap_ = 0, top_ = 0, peak_ = 0;
};

}  // namespace rteom
