// Contraction engine: einsum-style tensor contractions on device tensors,
// executed as (optional) permutes into GEMM layout, one batched GEMM, and an
// (optional) permute-add into the output.  Also owns the stream, the scratch
// arena, launch counting and per-class CUDA-event timing.
#pragma once

#include <functional>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rteom {

enum KernelClass { kLadder = 0, kContract = 1, kPermute = 2, kElementwise = 3, kNumClasses = 4 };

// Launch configuration of one GEMM shape picked by the autotuner.
struct GemmChoice {
  bool tc = false;            // tensor-core (split-TF32) path
  bool oz = false;            // tensor-core FP64 emulation (digit slicing)
  int tile = -1, splits = 0;  // FP64 kernel tile index and K slices
};

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
  int* tc_err = nullptr;  // also collects timeouts of the emulated-FP64 kernel
  // budget (clock cycles) of the MMA and epilogue waits of the tensor-core
  // kernels; 0 = their default (about 2 s).  Tests shorten it to make the
  // waits run out on purpose (failure detection without a GPU fault).
  long long tc_wait_cycles = 0;
  // Digit slicing: contractions of at least oz_min_flops run as products of
  // oz_planes 16-bit planes on the tensor cores (7 BF16 digit planes:
  // FP64-level accuracy; 3: the split-BF16 form; 2 FP16 hi/lo planes: the
  // split-FP16 form)
  bool fp64_emulation = false;
  int oz_planes = 7;
  // complex x complex products on the tensor cores as three real GEMMs (3M)
  bool allow_3m = true;
  double oz_min_flops = 5e7;
  // Packed tensor-core operands of constant tensors, keyed by tensor, spec
  // and role.  Entries are created only while tc_cache_fill is set (an eager
  // pass at set-up); later evaluations, captured graphs included, read them.
  bool tc_cache_fill = false;
  std::function<void*(int64_t)> persistent_alloc;  // bytes, owned by the context
  // Cache planning.  Dry runs with tensor_cores record every constant
  // operand a pack would be cached for (key, bytes, tensor).  With
  // tc_cache_select the cache holds only the keys in tc_cache_allowed (and
  // small packs the plan did not see); with plan_cached, dry runs reserve no
  // arena scratch for the packs the cache will hold.
  struct CacheCand {
    int64_t bytes = 0;
    const double* tensor = nullptr;
  };
  std::map<std::string, CacheCand> tc_cache_cands;
  std::set<std::string> tc_cache_allowed;
  bool tc_cache_select = false;
  bool plan_cached = false;
  // pack_only: a tensor-core contraction only packs its constant operands
  // (into the cache) and its held operands (see hold()) and launches
  // nothing else
  bool pack_only = false;
  // Grouped ladder.  With defer_ladder set, every ladder contraction (class
  // kLadder) takes the digit-plane tensor-core path with one K range per
  // output tile (GemmDesc::one_range), and outside pack_only it packs its
  // operands and records its GEMM in `deferred` instead of launching it.  Its
  // packs stay allocated in the arena: the caller launches the recorded GEMMs
  // (possibly with other engines' ones, gemm_oz_mma_group) and releases the
  // arena below them afterwards.
  bool defer_ladder = false;
  struct Deferred {
    OzGroupGemm gemm;
    double flops;
  };
  std::vector<Deferred> deferred;

  // Autotuner.  A GEMM of at most tune_max_flops that is not a matrix-vector
  // product takes its launch configuration (FP64 tile shape and K slices, or
  // the tensor-core path when tensor_cores is set and it has at least
  // tc_tune_min_flops) from timed trials run during eager evaluations with
  // `tuning` set.  Choices are kept process-wide, keyed by the GEMM's shape
  // and form, so every context of the process launches the same kernels and
  // gets the same bits; without a choice the shape heuristics apply.
  bool autotune = true;
  bool tuning = false;
  double tune_max_flops = 2e9;
  double tc_tune_min_flops = 1e6;  // also the floor of the emulated-FP64 candidate
  long long tuned = 0;  // GEMM shapes this engine has tuned

  // Timing.  Eager launches are each bracketed by events.  While a residual
  // graph is being captured (capturing == true) only launches of the classes
  // in graph_timed_mask (bit 1 << class) get event-record nodes; their event
  // pairs are kept in graph_pairs and read back after each replay with
  // collect_graph_timing().  FLOP counters hold the FP64-equivalent
  // algorithmic FLOPs of each contraction as posed (2, 4 or 8 per real,
  // mixed or complex multiply-add), whatever the form executes.
  bool timing = false;
  bool capturing = false;
  unsigned graph_timed_mask = 1u << kLadder;
  struct GraphPair {
    cudaEvent_t a, b;
    KernelClass cls;
    double flops, bytes;
  };
  std::vector<GraphPair>* graph_pairs = nullptr;  // list of the graph being captured
  // per-class launches and FLOPs of the untimed launches of that graph
  struct GraphTally {
    long long launches[kNumClasses] = {0, 0, 0, 0};
    double flops[kNumClasses] = {0, 0, 0, 0};
    double bytes[kNumClasses] = {0, 0, 0, 0};
  };
  GraphTally* graph_tally = nullptr;
  double ms[kNumClasses] = {0, 0, 0, 0};
  long long tlaunch[kNumClasses] = {0, 0, 0, 0};
  double tflops[kNumClasses] = {0, 0, 0, 0};
  double tbytes[kNumClasses] = {0, 0, 0, 0};  // algorithmic DRAM bytes of the launches

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
  void launch(KernelClass cls, double flops, F&& f, const std::string& what = std::string(),
              double bytes = 0.0) {
    if (dry) return;
    ++launches;
    if (!timing) {
      f();
      return;
    }
    if (capturing) {  // event-record nodes only around the timed class
      if (!((graph_timed_mask >> cls) & 1u) || !graph_pairs) {
        if (graph_tally) {
          graph_tally->launches[cls] += 1;
          graph_tally->flops[cls] += flops;
          graph_tally->bytes[cls] += bytes;
        }
        f();
        return;
      }
      cudaEvent_t a, b;
      RT_CUDA(cudaEventCreate(&a));
      RT_CUDA(cudaEventCreate(&b));
      // external records become event-record nodes of the captured graph
      RT_CUDA(cudaEventRecordWithFlags(a, stream, cudaEventRecordExternal));
      f();
      RT_CUDA(cudaEventRecordWithFlags(b, stream, cudaEventRecordExternal));
      graph_pairs->push_back({a, b, cls, flops, bytes});
      return;
    }
    cudaEvent_t a = get_event(), b = get_event();
    RT_CUDA(cudaEventRecord(a, stream));
    f();
    RT_CUDA(cudaEventRecord(b, stream));
    pending_.push_back({a, b, cls, flops, trace_on() ? what : std::string()});
    tlaunch[cls] += 1;
    tflops[cls] += flops;
    tbytes[cls] += bytes;
  }
  // Synchronises and folds pending event pairs into ms[]; when the
  // environment variable RTEOM_TRACE names a file, appends one JSON line per
  // timed launch (class, label, flops, ms) to it.
  void collect_timing();
  // After a replay of a graph captured with timing: fold its pairs in.
  // Returns false (and clears the error) when the driver cannot time
  // event-record nodes; the caller then times residuals eagerly instead.
  bool collect_graph_timing(const std::vector<GraphPair>& pairs);
  // Whether some tensor-core pack of the tensor at p is cached.
  bool tc_cached(const double* p) const { return tc_cached_.count(p) != 0; }
  bool graph_timing_ok = true;

  // Held operands (chunk loops that read one tensor in every chunk).  While
  // the tensor at p is held, a pack_only contraction packs it into the arena
  // below its own scratch, and the later contractions with the same spec,
  // role, own extent and K reuse that pack.  The caller makes the packs
  // ahead of the loop, keeps the tensor unchanged while it is held and calls
  // drop_holds() before it releases the arena below those packs.
  void hold(const double* p) { held_.insert(p); }
  void drop_holds() {
    held_.clear();
    held_packs_.clear();
  }

 private:
  struct Pending {
    cudaEvent_t a, b;
    KernelClass cls;
    double flops;
    std::string what;
  };
  bool trace_on() const;
  void tuning_scratch(const GemmDesc& g, bool tc_ok, bool oz_ok, bool a_const, bool b_const,
                      GemmChoice* out);
  // A packed tensor-core operand: TF32 hi / lo parts, or the digit planes
  // and row exponents of the FP64 emulation.
  struct Packed {
    void *p0 = nullptr, *p1 = nullptr;
  };
  std::map<std::string, Packed> tc_cache_;
  std::set<const double*> tc_cached_;  // tensors with at least one cached pack
  std::set<const double*> held_;
  std::map<std::string, Packed> held_packs_;
  std::vector<Pending> pending_;
  std::vector<cudaEvent_t> free_events_;
  cudaEvent_t get_event();
};

}  // namespace rteom
