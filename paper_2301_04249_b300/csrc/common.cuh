// Shared definitions of the RT-EOM-CCSD CUDA library: error handling, the
// device tensor descriptor and the stream-ordered scratch arena.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

namespace rteom {

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

// Row-major device tensor, FP64 real or complex128 (interleaved re, im).
struct Tensor {
  double* p = nullptr;
  int nd = 0;
  int64_t dim[kMaxDims] = {0, 0, 0, 0, 0, 0};
  bool cplx = false;
  bool constant = false;  // contents fixed for the context's lifetime (integrals)

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
