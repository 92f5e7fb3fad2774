// Contraction engine: einsum-style tensor contractions on device tensors,
// executed as (optional) permutes into GEMM layout, one batched GEMM, and an
// (optional) permute-add into the output.  Also owns the stream, the scratch
// arena, launch counting and per-class CUDA-event timing.
#pragma once

#include <functional>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rteom {

enum KernelClass { kLadder = 0, kContract = 1, kPermute = 2, kElementwise = 3, kNumClasses = 4 };

class Engine {
 public:
  cudaStream_t stream = nullptr;
  Arena arena;
  bool dry = false;  // plan only: allocate scratch, launch nothing
  long long launches = 0;
  // split precision: contractions of at least tc_min_flops run on the tensor
  // cores (split TF32, FP32 accumulation); tc_err collects pipeline timeouts
  bool tensor_cores = false;
  double tc_min_flops = 5e7;
  int* tc_err = nullptr;
  // Packed tensor-core operands of constant tensors, keyed by tensor, spec
  // and role.  Entries are created only while tc_cache_fill is set (an eager
  // pass at set-up); later evaluations, captured graphs included, read them.
  bool tc_cache_fill = false;
  std::function<float*(int64_t)> persistent_alloc;  // floats, owned by the context

  // timing (eager execution only)
  bool timing = false;
  double ms[kNumClasses] = {0, 0, 0, 0};
  long long tlaunch[kNumClasses] = {0, 0, 0, 0};
  double tflops[kNumClasses] = {0, 0, 0, 0};

  ~Engine();

  // C = beta*C + alpha * sum over the contracted labels of A*B.
  // spec: "labelsA,labelsB->labelsC", one character per axis.
  void contract(const char* spec, double alpha, const Tensor& A, const Tensor& B, double beta,
                const Tensor& C, KernelClass cls = kContract);
  // Y = beta*Y + alpha * X with axes relabelled: spec "labelsX->labelsY".
  void axpy(const char* spec, double alpha, const Tensor& X, double beta, const Tensor& Y);

  // Wrap a launch: counts it and, when timing, brackets it with events.
  // `what` labels the launch in the optional trace file.
  template <class F>
  void launch(KernelClass cls, double flops, F&& f, const std::string& what = std::string()) {
    if (dry) return;
    ++launches;
    if (!timing) {
      f();
      return;
    }
    cudaEvent_t a = get_event(), b = get_event();
    RT_CUDA(cudaEventRecord(a, stream));
    f();
    RT_CUDA(cudaEventRecord(b, stream));
    pending_.push_back({a, b, cls, flops, trace_on() ? what : std::string()});
    tlaunch[cls] += 1;
    tflops[cls] += flops;
  }
  // Synchronises and folds pending event pairs into ms[]; when the
  // environment variable RTEOM_TRACE names a file, appends one JSON line per
  // timed launch (class, label, flops, ms) to it.
  void collect_timing();

 private:
  struct Pending {
    cudaEvent_t a, b;
    KernelClass cls;
    double flops;
    std::string what;
  };
  bool trace_on() const;
  struct Packed {
    float *hi, *lo;
  };
  std::map<std::string, Packed> tc_cache_;
  std::vector<Pending> pending_;
  std::vector<cudaEvent_t> free_events_;
  cudaEvent_t get_event();
};

}  // namespace rteom
