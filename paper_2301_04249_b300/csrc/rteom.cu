// C ABI of the RT-EOM-CCSD core-hole propagation (include/rteom.h).
//
// A context owns the device copies of the problem, the integral blocks built
// from the Cholesky vectors, the amplitude buffers of the Adams-Moulton
// micro-iteration (Eq. 9) and the cumulant history (Eqs. 5-6).  Each residual
// evaluation is one CUDA graph (captured on first use); the host reads one
// 8-byte convergence word per micro-iteration.
#include <algorithm>
#include <cerrno>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/rteom.h"
#include "common.cuh"
#include "engine.h"
#include "kernels.h"
#include "residual.h"

using namespace rteom;

namespace {
thread_local std::string g_create_error;
constexpr int kMaxGroupMembers = 1024;  // contexts per rteom_propagate_group call
}

struct rteom_ctx {
  int O = 0, V = 0, nchol = 0, core = 0, precision = 0, flags = 0;
  int nO = 0, nV = 0;
  AmpGeom g{0, 0, 0};
  Engine E;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;

  ResidualOperands op;
  double *foo[2], *fov[2], *fvv[2], *fo[2], *fv[2];
  double* ovov = nullptr;
  double *T_N = nullptr, *R_N = nullptr, *T_K = nullptr, *R_K = nullptr;
  double *histC = nullptr, *histE = nullptr;
  long long hist_cap = 0;
  double* partial = nullptr;
  double* scalars = nullptr;  // [0] E_corr, [1..4] debug energy slots
  unsigned long long* maxdiff = nullptr;
  unsigned long long* h_maxdiff = nullptr;  // pinned
  double* arena_base = nullptr;
  int64_t arena_doubles = 0;

  double eps_core = 0.0, e_corr = 0.0, dt = 0.0;
  long long steps = 0, micro_total = 0;
  long long graph_kernels = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // residual(T_N -> R_N), residual(T_K -> R_K)
  // Grouped ladder (RTEOM_FLAG_GROUPED): a residual runs as graph A (tau and
  // the packed operands of the three ladder GEMMs), the ladder GEMMs in one
  // grouped launch with those of the other contexts of a round, then graph B
  // (the rest of the residual, the ladder results added), per residual kind
  // as graph[]; lad_gemms holds the GEMMs graph A's packs feed.
  bool grouped = false;
  cudaGraphExec_t graph_a[2] = {nullptr, nullptr}, graph_b[2] = {nullptr, nullptr};
  long long graph_ab_kernels[2] = {0, 0};
  std::vector<Engine::Deferred> lad_gemms[2];
  cudaEvent_t ev_group = nullptr;  // orders a round across the members' streams
  bool tune_first = false;  // run the next residual eagerly for the autotuner
  bool eager_timing = false;  // rteom_set_timing(ctx, 2): residuals outside graphs
  // Anderson acceleration of the micro-iteration (RTEOM_FLAG_ANDERSON):
  // g_k = G(x_k), f_{k-1}, g_{k-1}, the dF/dG histories (kAndersonDepth
  // slots each), the partials and result of the normal-equation dots, and
  // their pinned host copy; and_count = history slots in use
  double *and_g = nullptr, *and_fp = nullptr, *and_gp = nullptr, *and_df = nullptr,
         *and_dg = nullptr, *and_partial = nullptr, *and_dots = nullptr;
  double* h_dots = nullptr;
  int and_count = 0;
  long long cache_plan_bytes = 0;  // tensor-core pack cache planned at set-up
  // 0: captured without event nodes, else 1 + the engine's graph_timed_mask
  unsigned graph_timed[2] = {0u, 0u};
  std::vector<Engine::GraphPair> graph_pairs[2];
  Engine::GraphTally graph_tally[2];
  int graph_pending[2] = {0, 0};                   // replays whose timing is not yet read
  std::string err;

  // Non-blocking stepping (the blocking rteom_propagate and the server both
  // drive it): phase 0 = next step not started, 1 = waiting for the status
  // word of micro-iteration k, 2 = all requested steps done.
  struct Run {
    int phase = 2;
    int target = 0, done = 0, k = 0, max_micro = 1;
    double tol = 0.0;
    cudaEvent_t ev = nullptr;
  } run;

  size_t bytes_allocated = 0;
  std::vector<size_t> alloc_sizes;
  // host-side fault injection for tests: device allocations past this many
  // bytes fail as out of memory (RTEOM_INJECT_DEVICE_LIMIT; -1 = off)
  long long inject_limit = -1;
  double* dmalloc(size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    if (inject_limit >= 0 && (long long)(bytes_allocated + bytes) > inject_limit)
      throw Error(RTEOM_ERR_OOM, "cudaMalloc(" + std::to_string(bytes) +
                                     "): injected device limit of " +
                                     std::to_string(inject_limit) + " bytes");
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error(e == cudaErrorMemoryAllocation ? RTEOM_ERR_OOM : RTEOM_ERR_CUDA,
                  "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    allocs.push_back(p);
    alloc_sizes.push_back(bytes);
    bytes_allocated += bytes;
    return static_cast<double*>(p);
  }
  void dfree(void* p) {
    for (size_t k = 0; k < allocs.size(); ++k)
      if (allocs[k] == p) {
        cudaFree(allocs[k]);
        allocs[k] = nullptr;
        bytes_allocated -= alloc_sizes[k];
      }
  }
  ~rteom_ctx() {
    if (stream) cudaStreamSynchronize(stream);
    if (run.ev) cudaEventDestroy(run.ev);
    for (auto& gx : graph)
      if (gx) cudaGraphExecDestroy(gx);
    for (int w = 0; w < 2; ++w) {
      if (graph_a[w]) cudaGraphExecDestroy(graph_a[w]);
      if (graph_b[w]) cudaGraphExecDestroy(graph_b[w]);
    }
    if (ev_group) cudaEventDestroy(ev_group);
    for (auto& v : graph_pairs)
      for (auto& pr : v) {
        cudaEventDestroy(pr.a);
        cudaEventDestroy(pr.b);
      }
    for (void* p : allocs)
      if (p) cudaFree(p);
    if (h_maxdiff) cudaFreeHost(h_maxdiff);
    if (h_dots) cudaFreeHost(h_dots);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

namespace {

int fail(rteom_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

template <class F>
int guarded(rteom_ctx* c, F&& f) {
  try {
    return f();
  } catch (const Error& e) {
    if (c) c->err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    if (c) c->err = "host allocation failed";
    return RTEOM_ERR_OOM;
  } catch (const std::exception& e) {
    if (c) c->err = e.what();
    return RTEOM_ERR_CUDA;
  }
}

bool all_finite(const double* p, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(p[k])) return false;
  return true;
}

double bits_to_double(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
}

void drop_graph(rteom_ctx* c, int which) {
  if (c->graph[which]) cudaGraphExecDestroy(c->graph[which]);
  c->graph[which] = nullptr;
  for (auto& pr : c->graph_pairs[which]) {
    cudaEventDestroy(pr.a);
    cudaEventDestroy(pr.b);
  }
  c->graph_pairs[which].clear();
  c->graph_tally[which] = Engine::GraphTally();
  c->graph_pending[which] = 0;
}

// Fold the timing of finished graph replays into the engine's counters
// (the caller has observed that the stream passed them).
void collect_graph_timing(rteom_ctx* c) {
  for (int w = 0; w < 2; ++w) {
    if (c->graph_pending[w] && c->graph_timed[w]) {
      const auto& ty = c->graph_tally[w];
      for (int k = 0; k < kNumClasses; ++k) {
        c->E.tlaunch[k] += ty.launches[k];
        c->E.tflops[k] += ty.flops[k];
        c->E.tbytes[k] += ty.bytes[k];
      }
      if (!c->E.collect_graph_timing(c->graph_pairs[w])) {
        // the driver cannot time graph event nodes: drop the timed graphs,
        // later timed residuals run eagerly with an event pair per launch
        c->graph_pending[w] = 0;
        drop_graph(c, 0);
        drop_graph(c, 1);
        return;
      }
    }
    c->graph_pending[w] = 0;
  }
}

// The recorded ladder GEMMs of a round, as one grouped launch per tile width
// on stream st; the launch counts are charged to engine E.
void launch_ladders(Engine& E, const std::vector<OzGroupGemm>& gemms, double flops,
                    cudaStream_t st) {
  if (gemms.empty()) return;
  int n = 0;
  E.launch(kLadder, flops,
           [&] { n = gemm_oz_mma_group(gemms.data(), (int)gemms.size(), E.oz_planes, st); },
           "grouped ladder");
  if (n > 1) E.launches += n - 1;
}

// One residual outside graphs: compute_residual, or with the grouped ladder
// its two parts around a launch of this context's own ladder GEMMs.
void residual_eager(rteom_ctx* c, const double* t, double* R) {
  Engine& E = c->E;
  if (!c->grouped) {
    compute_residual(E, c->op, t, R);
    return;
  }
  const int64_t m0 = E.arena.mark();
  LadderOut lo;
  E.deferred.clear();
  ladder_part(E, c->op, t, &lo);
  std::vector<OzGroupGemm> gemms;
  double flops = 0.0;
  for (const auto& d : E.deferred) {
    gemms.push_back(d.gemm);
    flops += d.flops;
  }
  E.deferred.clear();
  launch_ladders(E, gemms, flops, c->stream);
  compute_residual(E, c->op, t, R, &lo);
  E.arena.release(m0);
}

// Capture f's launches on the context's stream as a graph.
template <class F>
cudaGraphExec_t capture_graph(rteom_ctx* c, F&& f, long long* kernels) {
  const long long before = c->E.launches;
  cudaGraph_t gr = nullptr;
  RT_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  try {
    f();
  } catch (...) {
    cudaStreamEndCapture(c->stream, &gr);
    if (gr) cudaGraphDestroy(gr);
    c->E.launches = before;
    throw;
  }
  RT_CUDA(cudaStreamEndCapture(c->stream, &gr));
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ex, gr, 0);
  cudaGraphDestroy(gr);
  RT_CUDA(e);
  *kernels = c->E.launches - before;
  c->E.launches = before;
  return ex;
}

// Graphs A and B of residual kind `which` of a grouped context.  Graph A's
// packs and ladder results sit in the arena above its level between
// residuals, where graph B's own scratch starts above them.
void ensure_group_graphs(rteom_ctx* c, int which) {
  if (c->graph_a[which]) return;
  Engine& E = c->E;
  const double* t = which == 0 ? c->T_N : c->T_K;
  double* R = which == 0 ? c->R_N : c->R_K;
  const int64_t m0 = E.arena.mark();
  LadderOut lo;
  long long ka = 0, kb = 0;
  try {
    E.deferred.clear();
    c->graph_a[which] = capture_graph(c, [&] { ladder_part(E, c->op, t, &lo); }, &ka);
    c->lad_gemms[which] = E.deferred;
    E.deferred.clear();
    c->graph_b[which] =
        capture_graph(c, [&] { compute_residual(E, c->op, t, R, &lo); }, &kb);
  } catch (...) {
    E.arena.release(m0);
    E.deferred.clear();
    if (c->graph_a[which]) cudaGraphExecDestroy(c->graph_a[which]);
    c->graph_a[which] = nullptr;
    c->lad_gemms[which].clear();
    throw;
  }
  E.arena.release(m0);
  c->graph_ab_kernels[which] = ka + kb;
}

// One residual of each member (kinds which[i]) with every member's ladder
// GEMMs in grouped launches: the members' graphs A on their own streams, the
// grouped GEMMs on the first member's stream after all of them, then the
// members' graphs B after the GEMMs.  Each GEMM computes its tiles as it
// would alone (one K range per tile), so results do not depend on the group.
void group_residuals(rteom_ctx* const* cs, const int* which, int n) {
  for (int i = 0; i < n; ++i) ensure_group_graphs(cs[i], which[i]);
  rteom_ctx* lead = cs[0];
  cudaStream_t gs = lead->stream;
  std::vector<OzGroupGemm> gemms;
  double flops = 0.0;
  for (int i = 0; i < n; ++i) {
    rteom_ctx* c = cs[i];
    RT_CUDA(cudaGraphLaunch(c->graph_a[which[i]], c->stream));
    c->E.launches += c->graph_ab_kernels[which[i]];
    for (const auto& d : c->lad_gemms[which[i]]) {
      gemms.push_back(d.gemm);
      flops += d.flops;
    }
    if (c->stream != gs) {
      if (!c->ev_group) RT_CUDA(cudaEventCreateWithFlags(&c->ev_group, cudaEventDisableTiming));
      RT_CUDA(cudaEventRecord(c->ev_group, c->stream));
      RT_CUDA(cudaStreamWaitEvent(gs, c->ev_group, 0));
    }
  }
  launch_ladders(lead->E, gemms, flops, gs);
  if (n > 1) {
    if (!lead->ev_group) RT_CUDA(cudaEventCreateWithFlags(&lead->ev_group, cudaEventDisableTiming));
    RT_CUDA(cudaEventRecord(lead->ev_group, gs));
  }
  for (int i = 0; i < n; ++i) {
    rteom_ctx* c = cs[i];
    if (c->stream != gs) RT_CUDA(cudaStreamWaitEvent(c->stream, lead->ev_group, 0));
    RT_CUDA(cudaGraphLaunch(c->graph_b[which[i]], c->stream));
  }
}

void run_residual(rteom_ctx* c, int which) {
  const double* t = which == 0 ? c->T_N : c->T_K;
  double* R = which == 0 ? c->R_N : c->R_K;
  if (c->grouped) {  // a group of one
    group_residuals(&c, &which, 1);
    return;
  }
  if (c->E.timing && (!c->E.graph_timing_ok || c->eager_timing)) {  // eager, every kernel timed
    compute_residual(c->E, c->op, t, R);
    return;
  }
  if (c->tune_first) {  // eager, the autotuner timing shapes it has not seen
    c->tune_first = false;
    c->E.tuning = true;
    try {
      compute_residual(c->E, c->op, t, R);
    } catch (...) {
      c->E.tuning = false;
      throw;
    }
    c->E.tuning = false;
    return;
  }
  const unsigned timed_key = c->E.timing ? 1u + c->E.graph_timed_mask : 0u;
  if (c->graph[which] && c->graph_timed[which] != timed_key) drop_graph(c, which);
  if (!c->graph[which]) {
    long long before = c->E.launches;
    cudaGraph_t gr;
    RT_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->E.capturing = true;
    c->E.graph_pairs = &c->graph_pairs[which];
    c->graph_tally[which] = Engine::GraphTally();
    c->E.graph_tally = &c->graph_tally[which];
    try {
      compute_residual(c->E, c->op, t, R);
    } catch (...) {
      c->E.capturing = false;
      c->E.graph_pairs = nullptr;
      c->E.graph_tally = nullptr;
      cudaStreamEndCapture(c->stream, &gr);
      if (gr) cudaGraphDestroy(gr);
      throw;
    }
    c->E.capturing = false;
    c->E.graph_pairs = nullptr;
    c->E.graph_tally = nullptr;
    RT_CUDA(cudaStreamEndCapture(c->stream, &gr));
    cudaError_t e = cudaGraphInstantiate(&c->graph[which], gr, 0);
    cudaGraphDestroy(gr);
    RT_CUDA(e);
    c->graph_timed[which] = timed_key;
    c->graph_kernels = c->E.launches - before;
    c->E.launches = before;
  }
  // a replay overwrites the graph's events: read the previous replay first
  if (c->graph_pending[which] && c->graph_timed[which]) {
    RT_CUDA(cudaStreamSynchronize(c->stream));
    collect_graph_timing(c);
  }
  RT_CUDA(cudaGraphLaunch(c->graph[which], c->stream));
  c->E.launches += c->graph_kernels;
  c->graph_pending[which] = 1;
}

void ensure_hist(rteom_ctx* c, long long need) {
  if (need <= c->hist_cap) return;
  long long cap = c->hist_cap ? c->hist_cap : 1024;
  while (cap < need) cap *= 2;
  double* nC = c->dmalloc(16 * cap);
  double* nE = c->dmalloc(16 * cap);
  RT_CUDA(cudaMemsetAsync(nC, 0, 16 * cap, c->stream));
  RT_CUDA(cudaMemsetAsync(nE, 0, 16 * cap, c->stream));
  if (c->hist_cap) {
    RT_CUDA(cudaMemcpyAsync(nC, c->histC, 16 * c->hist_cap, cudaMemcpyDeviceToDevice, c->stream));
    RT_CUDA(cudaMemcpyAsync(nE, c->histE, 16 * c->hist_cap, cudaMemcpyDeviceToDevice, c->stream));
    RT_CUDA(cudaStreamSynchronize(c->stream));
    c->dfree(c->histC);
    c->dfree(c->histE);
  }
  c->histC = nC;
  c->histE = nE;
  c->hist_cap = cap;
}

long long unpadded_size(const rteom_ctx* c) {  // complex elements
  long long oA = c->O, vA = c->V, oB = c->O - 1, vB = c->V + 1;
  return oA * vA + oB * vB + oA * oA * vA * vA + oA * oB * vA * vB + oB * oB * vB * vB;
}

void energy_into(rteom_ctx* c, const double* t, double* Ehist, double* Chist, long long n,
                 int update_c) {
  c->E.launch(kElementwise, 0.0, [&] {
    energy(c->g, t, c->ovov, c->fov[0], c->fov[1], !(c->flags & RTEOM_FLAG_CUMULANT_NO_FOV),
           c->partial, Ehist, Chist, n, c->dt, update_c, c->stream);
  });
}

void plan_context_bytes(int O, int V, int nchol, int precision, bool chol, bool anderson,
                        bool grouped, double out[3]);

// Chunk sizes of the Cholesky-mode residual: values of a per ladder chunk
// (a W chunk of chunk_a*nV^3 doubles) and of m per (mf|ae) chunk, each chunk
// at most 2^29 doubles (4 GB); RTEOM_CHOLESKY_CHUNK=<n> caps both.
void cholesky_chunks(int nO, int nV, int* chunk_a, int* chunk_m) {
  const int64_t nv3 = (int64_t)nV * nV * nV;
  int64_t cap = std::max<int64_t>(1, (int64_t(1) << 29) / nv3);
  if (const char* v = std::getenv("RTEOM_CHOLESKY_CHUNK"))
    cap = std::max<int64_t>(1, std::min<int64_t>(cap, std::atoll(v)));
  *chunk_a = (int)std::min<int64_t>(nV, cap);
  *chunk_m = (int)std::min<int64_t>(nO, cap);
}

void setup(rteom_ctx* c, const double* eps, const double* L, const double* t1_gs,
           const double* t2_gs) {
  const int O = c->O, V = c->V, nb = O + V, nchol = c->nchol;
  const int nO = c->nO, nV = c->nV;
  cudaStream_t st = c->stream;
  Engine& E = c->E;
  E.stream = st;

  // Cholesky mode (no (ov|vv) or (vv|vv) block on the device): asked for by
  // flag, or taken when the plan with resident blocks does not fit the free
  // device memory
  bool chol = false;
  if (nchol > 0) {
    if (c->flags & RTEOM_FLAG_LADDER_CHOLESKY) {
      chol = true;
    } else {
      double pb[3];
      plan_context_bytes(O, V, nchol, c->precision, false, c->flags & RTEOM_FLAG_ANDERSON,
                         c->grouped, pb);
      size_t fr = 0, tot = 0;
      RT_CUDA(cudaMemGetInfo(&fr, &tot));
      chol = pb[1] > 0.97 * (double)fr;
      if (chol && c->grouped)
        throw Error(RTEOM_ERR_OOM, "the grouped ladder needs the resident ladder blocks, which "
                                   "do not fit the free device memory");
    }
  }
  E.defer_ladder = c->grouped;

  // inputs
  double* d_eps = c->dmalloc(8 * nb);
  RT_CUDA(cudaMemcpyAsync(d_eps, eps, 8 * nb, cudaMemcpyHostToDevice, st));
  const size_t Lbytes = 8ull * nchol * nb * nb;
  double* d_L = c->dmalloc(Lbytes);
  if (nchol) RT_CUDA(cudaMemcpyAsync(d_L, L, Lbytes, cudaMemcpyHostToDevice, st));

  // slot-space Cholesky blocks and Fock matrices
  double* Loo = c->dmalloc(8ull * nchol * nO * nO);
  double* Lov = c->dmalloc(8ull * nchol * nO * nV);
  double* Lvv = c->dmalloc(8ull * nchol * nV * nV);
  E.launch(kElementwise, 0.0,
           [&] { gather_cholesky(d_L, nchol, nO, nV, c->core, Loo, Lov, Lvv, st); });
  double *LvvT = nullptr, *LovT = nullptr;
  if (chol) {  // [a][e][Q] and [m][e][Q] copies for the chunked builds
    LvvT = c->dmalloc(8ull * nchol * nV * nV);
    LovT = c->dmalloc(8ull * nchol * nO * nV);
    E.axpy("Qea->eaQ", 1.0, make_tensor(Lvv, false, {nchol, nV, nV}), 0.0,
           make_tensor(LvvT, false, {nV, nV, nchol}));
    E.axpy("Qme->meQ", 1.0, make_tensor(Lov, false, {nchol, nO, nV}), 0.0,
           make_tensor(LovT, false, {nO, nV, nchol}));
  }
  for (int s = 0; s < 2; ++s) {
    c->foo[s] = c->dmalloc(8ull * nO * nO);
    c->fov[s] = c->dmalloc(8ull * nO * nV);
    c->fvv[s] = c->dmalloc(8ull * nV * nV);
    c->fo[s] = c->dmalloc(8ull * nO);
    c->fv[s] = c->dmalloc(8ull * nV);
  }
  E.launch(kElementwise, 0.0, [&] {
    build_fock(d_eps, d_L, nchol, nO, nV, c->core, c->foo[0], c->fov[0], c->fvv[0], c->foo[1],
               c->fov[1], c->fvv[1], c->fo[0], c->fv[0], c->fo[1], c->fv[1], st);
  });
  ResidualOperands& op = c->op;
  op.nO = nO;
  op.nV = nV;
  op.core = c->core;
  for (int s = 0; s < 2; ++s) {
    op.foo[s] = c->foo[s];
    op.fov[s] = c->fov[s];
    op.fvv[s] = c->fvv[s];
    double* fc_oo = c->dmalloc(16ull * nO * nO);
    double* fc_ov = c->dmalloc(16ull * nO * nV);
    double* fc_vv = c->dmalloc(16ull * nV * nV);
    E.axpy("pq->pq", 1.0, make_tensor(c->foo[s], false, {nO, nO}), 0.0,
           make_tensor(fc_oo, true, {nO, nO}));
    E.axpy("pq->pq", 1.0, make_tensor(c->fov[s], false, {nO, nV}), 0.0,
           make_tensor(fc_ov, true, {nO, nV}));
    E.axpy("pq->pq", 1.0, make_tensor(c->fvv[s], false, {nV, nV}), 0.0,
           make_tensor(fc_vv, true, {nV, nV}));
    op.foo_c[s] = fc_oo;
    op.fov_c[s] = fc_ov;
    op.fvv_c[s] = fc_vv;
  }

  // chemists' integral blocks (pq|rs) = sum_Q L_pq L_rs (Section 3.1.1)
  auto Lt = [&](double* p, int a, int b) { return make_tensor(p, false, {nchol, a, b}); };
  double* oooo = c->dmalloc(8ull * nO * nO * nO * nO);
  double* ooov = c->dmalloc(8ull * nO * nO * nO * nV);
  double* oovv = c->dmalloc(8ull * nO * nO * nV * nV);
  double* ovov = c->dmalloc(8ull * nO * nV * nO * nV);
  double* ovvv = chol ? nullptr : c->dmalloc(8ull * nO * nV * nV * nV);
  double* vvvv = chol ? nullptr : c->dmalloc(8ull * nV * nV * nV * nV);
  // antisymmetrised (me|nf) - (mf|ne) and the packed same-spin ladder block
  const int64_t npv = (int64_t)nV * (nV - 1) / 2;
  double* ovov_as = c->dmalloc(8ull * nO * nV * nO * nV);
  double* vvvv_as = chol ? nullptr : c->dmalloc(8ull * (npv > 0 ? npv * npv : 1));
  op.oooo = oooo;
  op.ooov = ooov;
  op.oovv = oovv;
  op.ovov = ovov;
  op.ovvv = ovvv;
  op.vvvv = vvvv;
  op.ovov_as = ovov_as;
  op.vvvv_as = vvvv_as;
  c->ovov = ovov;
  op.chol = chol;
  op.nchol = nchol;
  if (chol) {
    op.Lov = Lov;
    op.Lvv = Lvv;
    op.LvvT = LvvT;
    op.LovT = LovT;
    cholesky_chunks(nO, nV, &op.chunk_a, &op.chunk_m);
  }

  // scratch arena for set-up contractions and, later, the residual, sized
  // by dry runs of the residual as it will run
  // forms with packed tensor-core operands (and a cache of the constant ones)
  const bool split = c->precision != RTEOM_FP64;
  const bool sliced = sliced_form(c->precision);
  if (const char* v = std::getenv("RTEOM_AUTOTUNE")) E.autotune = std::atoi(v) != 0;
  E.tensor_cores = c->precision == RTEOM_SPLIT_TF32;
  E.fp64_emulation = sliced;
  E.oz_planes = planes_of(c->precision);
  if (const char* v = std::getenv("RTEOM_TC_MIN_FLOPS")) E.tc_min_flops = std::atof(v);
  if (const char* v = std::getenv("RTEOM_NO_3M")) E.allow_3m = std::atoi(v) == 0;
  if (const char* v = std::getenv("RTEOM_TEST_CONSUMER_WAIT_CYCLES")) {
    // test hook: shortened MMA/epilogue waits of the tensor-core kernels
    char* end = nullptr;
    const long long w = std::strtoll(v, &end, 10);
    if (end == v || *end != '\0' || w <= 0)
      throw Error(RTEOM_ERR_ARG, std::string("RTEOM_TEST_CONSUMER_WAIT_CYCLES must be a positive "
                                             "cycle count, got '") + v + "'");
    E.tc_wait_cycles = w;
  }
  if (const char* v = std::getenv("RTEOM_OZ_MIN_FLOPS")) E.oz_min_flops = std::atof(v);
  auto dry_peak = [&]() {
    E.dry = true;
    E.arena.init(reinterpret_cast<double*>(uintptr_t(4096)), int64_t(1) << 50);
    if (c->grouped) {  // graph A's packs and results stay below graph B's scratch
      LadderOut lo;
      ladder_part(E, op, reinterpret_cast<double*>(uintptr_t(4096)), &lo);
      compute_residual(E, op, reinterpret_cast<double*>(uintptr_t(4096)),
                       reinterpret_cast<double*>(uintptr_t(4096)), &lo);
    } else {
      compute_residual(E, op, reinterpret_cast<double*>(uintptr_t(4096)),
                       reinterpret_cast<double*>(uintptr_t(4096)));
    }
    E.dry = false;
    return E.arena.peak_bytes() / 8;
  };
  E.plan_cached = split;
  int64_t need = dry_peak();
  // the ladder block is built in chunks of ce values of e, each through a
  // GEMM output of ce*nV^3 doubles that is then permuted into place
  const int64_t nv3 = (int64_t)nV * nV * nV;
  const int ce = (int)std::max<int64_t>(1, std::min<int64_t>(nV, (int64_t(1) << 28) / nv3));
  const int64_t setup_need = chol ? 0 : ce * nv3 + 64;
  if (split) {
    // Memory plan of the tensor-core pack cache: it holds the packs of the
    // FP64 ladder blocks (freed once packed) first, then the other constant
    // operands from small to large, as many as fit beside the arena and the
    // allocations still to come (amplitude sets, set-up temporaries, 1 GB
    // margin).  A constant left out is packed into the arena at every use.
    const int64_t later = 4 * 16 * (int64_t)c->g.total() + 8ll * nchol * nV * nV +
                          8ll * O * O * V * V + (int64_t(1) << 30);
    size_t fr = 0, tot = 0;
    RT_CUDA(cudaMemGetInfo(&fr, &tot));
    std::vector<std::pair<std::string, Engine::CacheCand>> order(E.tc_cache_cands.begin(),
                                                                 E.tc_cache_cands.end());
    auto ladder = [&](const Engine::CacheCand& x) {
      return x.tensor == vvvv || x.tensor == vvvv_as;
    };
    std::stable_sort(order.begin(), order.end(), [&](const auto& a, const auto& b) {
      if (ladder(a.second) != ladder(b.second)) return ladder(a.second);
      return a.second.bytes < b.second.bytes;
    });
    // The ladder packs are made first, each FP64 block freed right after its
    // pack: alpha-beta, then same-spin, then the rest of the cache.
    E.tc_cache_select = true;
    const int64_t f_ab = chol ? 0 : 8 * (int64_t)nV * nV * nV * nV,
                  f_ss = chol ? 0 : 8 * npv * npv;
    for (size_t keep = order.size();; --keep) {
      E.tc_cache_allowed.clear();
      int64_t p_ab = 0, p_ss = 0, p_other = 0;
      for (size_t k = 0; k < keep; ++k) {
        E.tc_cache_allowed.insert(order[k].first);
        const auto& cc = order[k].second;
        (cc.tensor == vvvv ? p_ab : cc.tensor == vvvv_as ? p_ss : p_other) += cc.bytes;
      }
      need = dry_peak();
      const int64_t freed_ab = p_ab ? f_ab : 0, freed_ss = p_ss ? f_ss : 0;
      const int64_t peak = std::max({p_ab, p_ab - freed_ab + p_ss,
                                     p_ab + p_ss + p_other - freed_ab - freed_ss});
      c->cache_plan_bytes = p_ab + p_ss + p_other;
      if (8 * std::max(need, setup_need) + peak + later <= (int64_t)fr || keep == 0) break;
    }
  }
  if (setup_need > need) need = setup_need;
  E.tensor_cores = false;  // set-up contractions in FP64
  E.fp64_emulation = false;
  c->arena_doubles = need + 1024;
  c->arena_base = c->dmalloc(8ull * c->arena_doubles);
  E.arena.init(c->arena_base, c->arena_doubles);

  E.contract("Qpq,Qrs->pqrs", 1.0, Lt(Loo, nO, nO), Lt(Loo, nO, nO), 0.0,
             make_tensor(oooo, false, {nO, nO, nO, nO}));
  E.contract("Qpq,Qrs->pqrs", 1.0, Lt(Loo, nO, nO), Lt(Lov, nO, nV), 0.0,
             make_tensor(ooov, false, {nO, nO, nO, nV}));
  E.contract("Qpq,Qrs->pqrs", 1.0, Lt(Loo, nO, nO), Lt(Lvv, nV, nV), 0.0,
             make_tensor(oovv, false, {nO, nO, nV, nV}));
  E.contract("Qpq,Qrs->pqrs", 1.0, Lt(Lov, nO, nV), Lt(Lov, nO, nV), 0.0,
             make_tensor(ovov, false, {nO, nV, nO, nV}));
  if (!chol)
    E.contract("Qpq,Qrs->pqrs", 1.0, Lt(Lov, nO, nV), Lt(Lvv, nV, nV), 0.0,
               make_tensor(ovvv, false, {nO, nV, nV, nV}));
  // ladder layout [e][f][a][b] = (ae|bf) = sum_Q L_ea L_fb, built for ce
  // values of e at a time from LvvT[e][a][Q] = L_ea
  if (!chol) {
    double* LvvT = c->dmalloc(8ull * nchol * nV * nV);
    E.axpy("Qea->eaQ", 1.0, Lt(Lvv, nV, nV), 0.0, make_tensor(LvvT, false, {nV, nV, nchol}));
    for (int e0 = 0; e0 < nV; e0 += ce) {
      const int n = std::min(ce, nV - e0);
      E.contract("eaQ,Qfb->efab", 1.0,
                 make_tensor(LvvT + (int64_t)e0 * nV * nchol, false, {n, nV, nchol}),
                 Lt(Lvv, nV, nV), 0.0, make_tensor(vvvv + e0 * nv3, false, {n, nV, nV, nV}));
    }
    RT_CUDA(cudaStreamSynchronize(st));
    c->dfree(LvvT);
  }
  // antisymmetrised (me|nf) - (mf|ne), shared by the W_mbej builds
  {
    const Tensor src = make_tensor(ovov, false, {nO, nV, nO, nV});
    const Tensor dst = make_tensor(ovov_as, false, {nO, nV, nO, nV});
    E.axpy("menf->menf", 1.0, src, 0.0, dst);
    E.axpy("mfne->menf", -1.0, src, 1.0, dst);
  }
  // packed antisymmetric ladder block for the same-spin T2 blocks
  if (!chol) E.launch(kElementwise, 0.0, [&] { pack_ladder_antisym(vvvv, vvvv_as, nV, st); });

  // E_N^corr (Eq. 3) from the closed-shell ground-state amplitudes
  c->partial = c->dmalloc(16ull * 2048);
  c->scalars = c->dmalloc(8ull * 16);
  RT_CUDA(cudaMemsetAsync(c->scalars, 0, 8 * 16, st));
  double *d_t1 = nullptr, *d_t2 = nullptr;
  if (t1_gs) {
    d_t1 = c->dmalloc(8ull * O * V);
    RT_CUDA(cudaMemcpyAsync(d_t1, t1_gs, 8ull * O * V, cudaMemcpyHostToDevice, st));
  }
  if (t2_gs) {
    d_t2 = c->dmalloc(8ull * O * O * V * V);
    RT_CUDA(cudaMemcpyAsync(d_t2, t2_gs, 8ull * O * O * V * V, cudaMemcpyHostToDevice, st));
  }
  if (t1_gs || t2_gs)
    E.launch(kElementwise, 0.0,
             [&] { closed_shell_ecorr(ovov, d_t1, d_t2, O, V, c->partial, c->scalars, st); });
  RT_CUDA(cudaMemcpyAsync(&c->e_corr, c->scalars, 8, cudaMemcpyDeviceToHost, st));
  RT_CUDA(cudaMemcpyAsync(&c->eps_core, d_eps + c->core, 8, cudaMemcpyDeviceToHost, st));
  RT_CUDA(cudaStreamSynchronize(st));
  // inputs no longer needed on the device
  for (void* p : {(void*)d_L, (void*)Loo, (void*)d_t1, (void*)d_t2})
    if (p) c->dfree(p);
  if (!chol) {  // the Cholesky mode keeps its slot-space blocks
    c->dfree(Lov);
    c->dfree(Lvv);
  }

  // amplitudes T(0) = 0 and the history C_0 = E_0 = 0
  const size_t ab = 16ull * c->g.total();
  c->T_N = c->dmalloc(ab);
  c->R_N = c->dmalloc(ab);
  c->T_K = c->dmalloc(ab);
  c->R_K = c->dmalloc(ab);
  for (double* p : {c->T_N, c->R_N, c->T_K, c->R_K}) RT_CUDA(cudaMemsetAsync(p, 0, ab, st));
  ensure_hist(c, 1);
  c->maxdiff = reinterpret_cast<unsigned long long*>(c->dmalloc(64));
  RT_CUDA(cudaMemsetAsync(c->maxdiff, 0, 64, st));
  void* hp = nullptr;
  RT_CUDA(cudaMallocHost(&hp, 64));
  c->h_maxdiff = static_cast<unsigned long long*>(hp);
  if (c->flags & RTEOM_FLAG_ANDERSON) {
    const size_t v = 16ull * c->g.total();
    c->and_g = c->dmalloc(v);
    c->and_fp = c->dmalloc(v);
    c->and_gp = c->dmalloc(v);
    c->and_df = c->dmalloc(kAndersonDepth * v);
    c->and_dg = c->dmalloc(kAndersonDepth * v);
    c->and_partial = c->dmalloc(16ull * kAndersonDots * anderson_partials());
    c->and_dots = c->dmalloc(16ull * kAndersonDots);
    void* hd = nullptr;
    RT_CUDA(cudaMallocHost(&hd, 16ull * kAndersonDots));
    c->h_dots = static_cast<double*>(hd);
  }
  RT_CUDA(cudaStreamSynchronize(st));
  // split precision and FP64 emulation: tensor-core contractions inside the
  // residual only (the set-up integrals above are FP64); pipeline timeouts
  // land in maxdiff[1].
  if (split) {
    if (c->precision == RTEOM_SPLIT_TF32) {
      gemm_tc_init();
      E.tensor_cores = true;
    } else {
      gemm_oz_init();
      E.fp64_emulation = true;  // digit slicing, oz_planes as planned above
    }
    E.tc_err = reinterpret_cast<int*>(c->maxdiff + 1);
    E.persistent_alloc = [c](int64_t bytes) {
      return static_cast<void*>(c->dmalloc(bytes > 0 ? bytes : 16));
    };
  }
  // With packed operands one eager residual on T(0) (into the scratch
  // amplitude set) packs every constant operand the cache plan keeps, and
  // the autotuner times the GEMM shapes the process has not seen.  In FP64
  // the first residual of the propagation runs eagerly for the autotuner.
  if (split) {
    E.tc_cache_fill = true;
    // the ladder contractions read only their packed operands once cached:
    // pack them first and free the FP64 ladder blocks (the largest arrays of
    // the context) before the rest of the cache is filled
    if (!chol) {
      prepack_ladder(E, op, false);
      RT_CUDA(cudaStreamSynchronize(st));
      if (E.tc_cached(vvvv)) {
        c->dfree(vvvv);
        op.vvvv_released = true;
      }
      prepack_ladder(E, op, true);
      RT_CUDA(cudaStreamSynchronize(st));
      if (E.tc_cached(vvvv_as)) {
        c->dfree(vvvv_as);
        op.vvvv_as_released = true;
      }
    }
    E.tuning = E.autotune;
    residual_eager(c, c->T_N, c->R_K);
    E.tc_cache_fill = false;
    E.tuning = false;
    RT_CUDA(cudaStreamSynchronize(st));
  } else {
    c->tune_first = E.autotune;
  }
}

// Device bytes of a context of this shape and form, planned on the host with
// the dry runs that size rteom_create's arena (no device calls).  out[0]:
// peak with every constant tensor-core pack cached; out[1]: peak with none
// cached; out[2]: after set-up with every pack cached.  The phases follow
// setup(): integrals built while the Cholesky inputs live, then the pack
// cache filled ladder blocks first, each FP64 ladder block freed after its
// pack.  chol: the Cholesky mode (no (ov|vv)/(vv|vv) blocks; the slot-space
// Cholesky blocks stay); anderson: the buffers of the accelerated
// micro-iteration; grouped: the grouped ladder (its packs and results held
// through the residual).
void plan_context_bytes(int O, int V, int nchol, int precision, bool chol, bool anderson,
                        bool grouped, double out[3]) {
  const double nO = O, nVd = V + 1.0, nb = O + V;
  const int nV = V + 1;
  const double npv = nVd * (nVd - 1.0) / 2.0;
  const AmpGeom g{O, nV, 0};
  Engine E;
  E.tensor_cores = precision == RTEOM_SPLIT_TF32;
  E.fp64_emulation = sliced_form(precision);
  E.oz_planes = planes_of(precision);
  ResidualOperands op;
  op.nO = O;
  op.nV = nV;
  auto fake = [](int k) { return reinterpret_cast<double*>(uintptr_t(4096) * (k + 1)); };
  op.oooo = fake(1);
  op.ooov = fake(2);
  op.oovv = fake(3);
  op.ovov = fake(4);
  op.ovvv = fake(5);
  op.ovov_as = fake(6);
  op.vvvv = chol ? nullptr : fake(7);
  op.vvvv_as = chol ? nullptr : fake(8);
  if (chol) {
    op.ovvv = nullptr;
    op.chol = true;
    op.nchol = nchol;
    op.Lov = fake(22);
    op.Lvv = fake(23);
    op.LvvT = fake(24);
    op.LovT = fake(25);
    cholesky_chunks(O, nV, &op.chunk_a, &op.chunk_m);
  }
  for (int s = 0; s < 2; ++s) {
    op.foo[s] = fake(10 + s);
    op.fov[s] = fake(12 + s);
    op.fvv[s] = fake(14 + s);
    op.foo_c[s] = fake(16 + s);
    op.fov_c[s] = fake(18 + s);
    op.fvv_c[s] = fake(20 + s);
  }
  const bool packed = precision != RTEOM_FP64;
  auto dry = [&](bool cached) {
    E.dry = true;
    E.plan_cached = cached && packed;
    E.arena.init(fake(30), int64_t(1) << 50);
    if (grouped) {
      E.defer_ladder = true;
      LadderOut lo;
      ladder_part(E, op, fake(31), &lo);
      compute_residual(E, op, fake(31), fake(32), &lo);
    } else {
      compute_residual(E, op, fake(31), fake(32));
    }
    return (double)E.arena.peak_bytes();
  };
  const double setup_need =
      chol ? 0.0
           : 8.0 *
                 std::max<int64_t>(1, std::min<int64_t>(nV, (int64_t(1) << 28) /
                                                                ((int64_t)nV * nV * nV))) *
                 nVd * nVd * nVd;
  const double arena_all = std::max(dry(true), setup_need) + 8192.0;
  double p_ab = 0.0, p_ss = 0.0, p_all = 0.0;
  for (const auto& kv : E.tc_cache_cands) {
    p_all += (double)kv.second.bytes;
    if (!chol && kv.second.tensor == op.vvvv) p_ab += (double)kv.second.bytes;
    if (!chol && kv.second.tensor == op.vvvv_as) p_ss += (double)kv.second.bytes;
  }
  const double arena_none = std::max(dry(false), setup_need) + 8192.0;
  const double f_ab = chol ? 0.0 : 8.0 * nVd * nVd * nVd * nVd,
               f_ss = chol ? 0.0 : 8.0 * npv * npv;
  // integral blocks (the Cholesky mode keeps L_ov, L_vv and their transposes
  // instead of (ov|vv), (vv|vv) and the pair block)
  const double ints =
      8.0 * (nO * nO * nO * nO + nO * nO * nO * nVd + 3.0 * nO * nO * nVd * nVd) +
      (chol ? 8.0 * nchol * (2.0 * nO * nVd + 2.0 * nVd * nVd)
            : 8.0 * nO * nVd * nVd * nVd + f_ab + f_ss);
  // inputs on the device during set-up: eps, L, L_oo (and, with resident
  // blocks, L_ov, L_vv and the transposed L_vv of the chunked ladder build)
  const double inputs =
      8.0 * (nb + nchol * nb * nb + nchol * nO * nO) +
      (chol ? 0.0 : 8.0 * nchol * (nO * nVd + 2.0 * nVd * nVd));
  const double fock = 2.0 * (24.0 * (nO * nO + nO * nVd + nVd * nVd) + 8.0 * (nO + nVd));
  const double amps = 4.0 * 16.0 * (double)g.total() + 2.0 * 16.0 * 1024 + 16.0 * 2048 + 256.0 +
                      (anderson ? (3.0 + 2.0 * kAndersonDepth) * 16.0 * (double)g.total() +
                                      16.0 * kAndersonDots * (anderson_partials() + 1.0)
                                : 0.0);
  const double phase_a_all = inputs + fock + ints + arena_all;
  const double phase_a_none = inputs + fock + ints + arena_none;
  const double base_all = ints + fock + arena_all + amps;
  const double cache_peak =
      std::max({p_ab, p_ab - (p_ab > 0 ? f_ab : 0.0) + p_ss,
                p_all - (p_ab > 0 ? f_ab : 0.0) - (p_ss > 0 ? f_ss : 0.0)});
  out[0] = std::max(phase_a_all, base_all + cache_peak);
  out[1] = std::max(phase_a_none, ints + fock + arena_none + amps);
  out[2] = base_all - (p_ab > 0 ? f_ab : 0.0) - (p_ss > 0 ? f_ss : 0.0) + p_all;
}

}  // namespace

// ---- non-blocking stepping (shared by rteom_propagate and the server) ------
int rteom_internal_begin(rteom_ctx* c, int nsteps, double dt, double tol, int max_micro) {
  if (nsteps < 0 || !(dt > 0) || !std::isfinite(dt) || !(tol > 0) || max_micro < 1)
    return fail(c, RTEOM_ERR_ARG, "need nsteps >= 0, dt > 0, tol > 0, max_micro >= 1");
  if (c->dt > 0 && std::fabs(dt - c->dt) > 1e-15 * std::fabs(c->dt))
    return fail(c, RTEOM_ERR_ARG, "dt must stay the same across calls of one context");
  return guarded(c, [&] {
    c->dt = dt;
    ensure_hist(c, c->steps + nsteps + 1);
    if (!c->run.ev) RT_CUDA(cudaEventCreateWithFlags(&c->run.ev, cudaEventDisableTiming));
    c->run.phase = nsteps > 0 ? 0 : 2;
    c->run.target = nsteps;
    c->run.done = 0;
    c->run.k = 0;
    c->run.tol = tol;
    c->run.max_micro = max_micro;
    return RTEOM_OK;
  });
}

// Anderson coefficients: gamma minimising |f - dF gamma| from the normal
// equations H gamma = b (H_ij = <dF_i, dF_j>, b_i = <dF_i, f>, the layout of
// anderson_dots), H regularised by 1e-10 of its largest diagonal entry (the
// normal equations square the condition of dF) and solved by Gaussian
// elimination with partial pivoting.  False when no usable solution exists
// or a coefficient exceeds 1e4 (nearly dependent history); the caller then
// takes the plain step.
static bool anderson_gamma(int m, const double* dots, double* gamma) {
  using cd = std::complex<double>;
  static const int I[6] = {0, 0, 0, 1, 1, 2}, J[6] = {0, 1, 2, 1, 2, 2};
  cd H[kAndersonDepth][kAndersonDepth + 1];
  for (int d = 0; d < 6; ++d) {
    const cd v(dots[2 * d], dots[2 * d + 1]);
    H[I[d]][J[d]] = v;
    H[J[d]][I[d]] = std::conj(v);
  }
  double hmax = 0.0;
  for (int i = 0; i < m; ++i) {
    H[i][i] = cd(H[i][i].real(), 0.0);
    H[i][m] = cd(dots[12 + 2 * i], dots[13 + 2 * i]);
    hmax = std::max(hmax, H[i][i].real());
  }
  if (!(hmax > 0.0) || !std::isfinite(hmax)) return false;
  for (int i = 0; i < m; ++i) H[i][i] += 1e-10 * hmax;
  for (int col = 0; col < m; ++col) {
    int piv = col;
    for (int r = col + 1; r < m; ++r)
      if (std::abs(H[r][col]) > std::abs(H[piv][col])) piv = r;
    if (!(std::abs(H[piv][col]) > 0.0)) return false;
    for (int q = 0; q <= m; ++q) std::swap(H[col][q], H[piv][q]);
    for (int r = col + 1; r < m; ++r) {
      const cd f = H[r][col] / H[col][col];
      for (int q = col; q <= m; ++q) H[r][q] -= f * H[col][q];
    }
  }
  cd x[kAndersonDepth];
  for (int i = m - 1; i >= 0; --i) {
    cd v = H[i][m];
    for (int q = i + 1; q < m; ++q) v -= H[i][q] * x[q];
    x[i] = v / H[i][i];
    if (!std::isfinite(x[i].real()) || !std::isfinite(x[i].imag()) || std::abs(x[i]) > 1e4)
      return false;
  }
  for (int i = 0; i < kAndersonDepth; ++i) {
    gamma[2 * i] = i < m ? x[i].real() : 0.0;
    gamma[2 * i + 1] = i < m ? x[i].imag() : 0.0;
  }
  return true;
}

// Next iterate of the accelerated micro-iteration into T_K: the plain step
// x = g_k while there is no history, else x = g_k - sum_j gamma_j dG_j.
static void anderson_next(rteom_ctx* c) {
  cudaStream_t st = c->stream;
  const int64_t n = c->g.total();
  double gamma[2 * kAndersonDepth];
  if (c->and_count > 0 && anderson_gamma(c->and_count, c->h_dots, gamma)) {
    c->E.launch(kElementwise, 0.0, [&] {
      anderson_mix(n, c->and_g, c->and_dg, c->and_count, gamma, c->T_K, st);
    });
  } else {
    RT_CUDA(cudaMemcpyAsync(c->T_K, c->and_g, 16ull * n, cudaMemcpyDeviceToDevice, st));
  }
}

// Launch the rest of micro-iteration k of the current step after its
// residual (the Adams-Moulton update, the status-word copy) and record the
// run event.
static void launch_update(rteom_ctx* c, int k) {
  cudaStream_t st = c->stream;
  RT_CUDA(cudaMemsetAsync(c->maxdiff, 0, 8, st));
  const double* tk_in = k == 0 ? c->T_N : c->T_K;
  const double* Rk = k == 0 ? c->R_N : c->R_K;
  double* out = c->and_g ? c->and_g : c->T_K;  // Anderson: g_k apart from x_k
  c->E.launch(kElementwise, 0.0, [&] {
    am_update(c->g, c->fo[0], c->fv[0], c->fo[1], c->fv[1], c->dt, c->T_N, c->R_N, tk_in, out, Rk,
              c->maxdiff, st);
  });
  if (c->and_g) {
    const int64_t n = c->g.total();
    const int64_t slot = k == 0 ? 0 : (k - 1) % kAndersonDepth;
    c->E.launch(kElementwise, 0.0, [&] {
      anderson_push(n, c->and_g, tk_in, c->and_fp, c->and_gp, c->and_df + 2 * n * slot,
                    c->and_dg + 2 * n * slot, k == 0, st);
    });
    c->and_count = k == 0 ? 0 : std::min(k, kAndersonDepth);
    if (c->and_count > 0) {
      c->E.launch(kElementwise, 0.0, [&] {
        anderson_dots(n, c->and_df, c->and_fp, c->and_count, c->and_partial, c->and_dots, st);
      });
      RT_CUDA(cudaMemcpyAsync(c->h_dots, c->and_dots, 16ull * kAndersonDots,
                              cudaMemcpyDeviceToHost, st));
    }
  }
  RT_CUDA(cudaMemcpyAsync(c->h_maxdiff, c->maxdiff, 16, cudaMemcpyDeviceToHost, st));
  RT_CUDA(cudaEventRecord(c->run.ev, st));
}

// Launch micro-iteration k of the current step (residual when k > 0, then
// the update).
static void launch_micro(rteom_ctx* c, int k) {
  if (k > 0) run_residual(c, 1);
  launch_update(c, k);
}

// The status word of micro-iteration r.k has arrived.  A pipeline timeout or
// non-finite amplitudes fail the run; on convergence t^(k+1) is accepted and
// the cumulant step taken (*next = 0 while steps remain: R(t_n) of the next
// step; -1 when all are done); otherwise *next = 1 for micro-iteration k+1
// (r.k advanced), unless the cap is reached.
static int after_status(rteom_ctx* c, int* next) {
  auto& r = c->run;
  *next = -1;
  if (c->h_maxdiff[1] != 0) {
    r.phase = 2;
    return fail(c, RTEOM_ERR_CUDA,
                "tensor-core pipeline wait timed out (code " +
                    std::to_string((long long)c->h_maxdiff[1]) + ")");
  }
  const double d = std::sqrt(bits_to_double(c->h_maxdiff[0]));  // the kernel keeps |.|^2
  if (!std::isfinite(d)) {
    r.phase = 2;
    return fail(c, RTEOM_ERR_NONFINITE,
                "amplitudes became non-finite at step " + std::to_string(c->steps));
  }
  if (d < r.tol) {  // converged: accept t^(k+1), cumulant step
    cudaStream_t st = c->stream;
    RT_CUDA(cudaMemcpyAsync(c->T_N, c->and_g ? c->and_g : c->T_K, 16ull * c->g.total(),
                            cudaMemcpyDeviceToDevice, st));
    energy_into(c, c->T_N, c->histE, c->histC, c->steps, 1);
    c->steps += 1;
    c->micro_total += r.k + 1;
    r.done += 1;
    if (r.done >= r.target) {
      r.phase = 2;
    } else {
      r.phase = 0;
      *next = 0;
    }
    return RTEOM_OK;
  }
  if (r.k + 1 >= r.max_micro) {
    r.phase = 2;
    return fail(c, RTEOM_ERR_NOT_CONVERGED,
                "micro-iterations did not reach tol at step " + std::to_string(c->steps));
  }
  r.k += 1;
  *next = 1;
  return RTEOM_OK;
}

// Advance without blocking.  *finished: all requested steps done; *waiting:
// the device still owes the status word of the pending micro-iteration.
int rteom_internal_poll(rteom_ctx* c, bool* finished, int* waiting) {
  *finished = false;
  *waiting = 0;
  return guarded(c, [&]() -> int {
    auto& r = c->run;
    if (r.phase == 2) {
      *finished = true;
      return RTEOM_OK;
    }
    if (r.phase == 0) {  // R(t_n); the first micro-iteration starts from t^(0) = t_n
      run_residual(c, 0);
      r.k = 0;
      launch_micro(c, 0);
      r.phase = 1;
      *waiting = 1;
      return RTEOM_OK;
    }
    cudaError_t q = cudaEventQuery(r.ev);
    if (q == cudaErrorNotReady) {
      *waiting = 1;
      return RTEOM_OK;
    }
    RT_CUDA(q);
    if (c->E.timing) collect_graph_timing(c);  // the stream passed every pending replay
    int next = -1;
    const int rc = after_status(c, &next);
    if (rc != RTEOM_OK) return rc;
    if (next < 0) {
      *finished = true;
      return RTEOM_OK;
    }
    if (next == 0) return RTEOM_OK;  // the next poll starts the next step
    if (c->and_g) anderson_next(c);  // x_{k+1} into T_K
    launch_micro(c, r.k);
    *waiting = 1;
    return RTEOM_OK;
  });
}

// Advance grouped contexts without blocking (the server's stepping of
// requests with RTEOM_FLAG_GROUPED): the contexts of cs that are ready (a
// new step to start, or the status word of their micro-iteration arrived)
// evaluate one residual each, with the ladder GEMMs of all of them in
// grouped launches, then their updates; the others are left running and
// join a later round.  rc[i]: the context's status (an error ends its run);
// done[i]: all its steps are done; *progressed: anything was launched or
// settled.
void rteom_internal_group_poll(rteom_ctx* const* cs, int n, int* rc, bool* done,
                               bool* progressed) {
  std::vector<rteom_ctx*> mem;
  std::vector<int> which, idx;
  for (int i = 0; i < n; ++i) {
    rteom_ctx* c = cs[i];
    int w = -1;
    done[i] = false;
    rc[i] = guarded(c, [&]() -> int {
      auto& r = c->run;
      if (r.phase == 2) {
        done[i] = true;
        return RTEOM_OK;
      }
      if (r.phase == 0) {
        w = 0;
        return RTEOM_OK;
      }
      cudaError_t q = cudaEventQuery(r.ev);
      if (q == cudaErrorNotReady) return RTEOM_OK;  // still running
      RT_CUDA(q);
      *progressed = true;
      const int st = after_status(c, &w);
      if (st == RTEOM_OK && w < 0) done[i] = true;
      return st;
    });
    if (rc[i] == RTEOM_OK && w >= 0) {
      mem.push_back(c);
      which.push_back(w);
      idx.push_back(i);
    }
  }
  if (mem.empty()) return;
  *progressed = true;
  const int st = guarded(mem[0], [&] {
    group_residuals(mem.data(), which.data(), (int)mem.size());
    for (size_t k = 0; k < mem.size(); ++k) {
      auto& r = mem[k]->run;
      if (which[k] == 0) {  // the first micro-iteration starts from t^(0) = t_n
        r.k = 0;
        r.phase = 1;
      }
      launch_update(mem[k], r.k);
    }
    return RTEOM_OK;
  });
  if (st != RTEOM_OK)  // a launch failed: every member of the round fails with it
    for (size_t k = 0; k < mem.size(); ++k) {
      mem[k]->err = mem[0]->err;
      mem[k]->run.phase = 2;
      rc[idx[k]] = st;
    }
}

cudaStream_t rteom_internal_stream(rteom_ctx* c) { return c->stream; }
double rteom_internal_device_bytes(const rteom_ctx* c) {
  return (double)c->bytes_allocated;
}

extern "C" {

int rteom_create(rteom_ctx** out, int nocc, int nvir, int nchol, const double* eps,
                 const double* L, const double* t1_gs, const double* t2_gs, int core_index,
                 int precision, int flags, void* cuda_stream) {
  g_create_error.clear();
  if (!out) {
    g_create_error = "out is NULL";
    return RTEOM_ERR_ARG;
  }
  *out = nullptr;
  auto bad = [&](int code, const std::string& m) {
    g_create_error = m;
    return code;
  };
  if (nocc < 1 || nvir < 1 || nchol < 0) return bad(RTEOM_ERR_ARG, "need nocc >= 1, nvir >= 1, nchol >= 0");
  if (core_index < 0 || core_index >= nocc) return bad(RTEOM_ERR_ARG, "core_index outside the occupied orbitals");
  if (!eps || (nchol > 0 && !L)) return bad(RTEOM_ERR_ARG, "eps (and L when nchol > 0) must be given");
  if (!valid_precision(precision))
    return bad(RTEOM_ERR_ARG, "precision must be RTEOM_FP64, RTEOM_SPLIT_BF16, RTEOM_SPLIT_TF32, "
                              "RTEOM_FP64_OZAKI or RTEOM_SPLIT_FP16");
  if (flags & ~(RTEOM_FLAG_CUMULANT_NO_FOV | RTEOM_FLAG_LADDER_CHOLESKY | RTEOM_FLAG_ANDERSON |
                RTEOM_FLAG_GROUPED))
    return bad(RTEOM_ERR_ARG, "unknown flag bits");
  if (!grouped_flags_ok(precision, flags))
    return bad(RTEOM_ERR_ARG, "RTEOM_FLAG_GROUPED needs RTEOM_FP64_OZAKI, RTEOM_SPLIT_BF16 or "
                              "RTEOM_SPLIT_FP16, without RTEOM_FLAG_LADDER_CHOLESKY or "
                              "RTEOM_FLAG_ANDERSON");
  const size_t nb = size_t(nocc) + nvir;
  if ((double)(nvir + 1) * (nvir + 1) > 2.0e9)
    return bad(RTEOM_ERR_ARG, "nvir too large: (nvir+1)^2 pair indices must fit 32 bits");
  if (!all_finite(eps, nb) || (nchol && !all_finite(L, size_t(nchol) * nb * nb)) ||
      (t1_gs && !all_finite(t1_gs, size_t(nocc) * nvir)) ||
      (t2_gs && !all_finite(t2_gs, size_t(nocc) * nocc * nvir * nvir)))
    return bad(RTEOM_ERR_NONFINITE, "non-finite value in an input array");
  if (nchol) {
    double mx = 0.0;
    for (size_t k = 0; k < size_t(nchol) * nb * nb; ++k) mx = std::fmax(mx, std::fabs(L[k]));
    for (int q = 0; q < nchol; ++q)
      for (size_t p = 0; p < nb; ++p)
        for (size_t r = p + 1; r < nb; ++r)
          if (std::fabs(L[(q * nb + p) * nb + r] - L[(q * nb + r) * nb + p]) > 1e-12 * mx)
            return bad(RTEOM_ERR_ARG, "Cholesky vectors must be symmetric: L[q][p][r] == L[q][r][p]");
  }
  std::unique_ptr<rteom_ctx> c(new rteom_ctx());
  c->O = nocc;
  c->V = nvir;
  c->nchol = nchol;
  c->core = core_index;
  c->precision = precision;
  c->flags = flags;
  c->grouped = (flags & RTEOM_FLAG_GROUPED) != 0;
  c->nO = nocc;
  c->nV = nvir + 1;
  c->g = AmpGeom{c->nO, c->nV, core_index};
  if (const char* v = std::getenv("RTEOM_INJECT_DEVICE_LIMIT")) {
    // test-only fault injection: a plain byte count; anything else is
    // rejected so that a mistyped value cannot pass for a real OOM
    char* end = nullptr;
    errno = 0;
    const long long lim = std::strtoll(v, &end, 10);
    if (end == v || *end != '\0' || errno != 0 || lim < 0)
      return bad(RTEOM_ERR_ARG, std::string("RTEOM_INJECT_DEVICE_LIMIT must be a byte count, got '") +
                                    v + "'");
    c->inject_limit = lim;
    static bool announced = false;
    if (!announced) {
      announced = true;
      std::fprintf(stderr, "rteom: RTEOM_INJECT_DEVICE_LIMIT=%lld: device allocations past this "
                           "total fail as out of memory (fault injection)\n", lim);
    }
  }
  int rc = guarded(c.get(), [&] {
    if (cuda_stream) {
      c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      RT_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    setup(c.get(), eps, L, t1_gs, t2_gs);
    return RTEOM_OK;
  });
  if (rc != RTEOM_OK) {
    g_create_error = c->err;
    return rc;
  }
  *out = c.release();
  return RTEOM_OK;
}

int rteom_propagate(rteom_ctx* c, int nsteps, double dt, double tol, int max_micro,
                    double* C_out) {
  if (!c) return RTEOM_ERR_ARG;
  const long long start = c->steps;
  int rc = rteom_internal_begin(c, nsteps, dt, tol, max_micro);
  if (rc != RTEOM_OK) return rc;
  bool finished = false;
  while (!finished) {
    int waiting = 0;
    rc = rteom_internal_poll(c, &finished, &waiting);
    if (rc != RTEOM_OK) return rc;
    if (waiting) {
      rc = guarded(c, [&] {
        RT_CUDA(cudaEventSynchronize(c->run.ev));
        return RTEOM_OK;
      });
      if (rc != RTEOM_OK) return rc;
    }
  }
  return guarded(c, [&] {
    if (C_out)
      RT_CUDA(cudaMemcpyAsync(C_out, c->histC + 2 * start, 16ull * (nsteps + 1),
                              cudaMemcpyDeviceToHost, c->stream));
    RT_CUDA(cudaStreamSynchronize(c->stream));
    if (c->E.timing) c->E.collect_timing();
    return RTEOM_OK;
  });
}

int rteom_propagate_group(rteom_ctx* const* ctxs, int n, int nsteps, double dt, double tol,
                          int max_micro, double* const* C_out) {
  if (!ctxs || n < 1 || n > kMaxGroupMembers) return RTEOM_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    rteom_ctx* c = ctxs[i];
    if (!c) return RTEOM_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return fail(c, RTEOM_ERR_ARG, "a context appears twice in the group");
    if (!c->grouped)
      return fail(c, RTEOM_ERR_ARG, "a group member was created without RTEOM_FLAG_GROUPED");
    if (c->E.oz_planes != ctxs[0]->E.oz_planes)
      return fail(c, RTEOM_ERR_ARG, "group members must share one precision form");
  }
  std::vector<long long> start(n);
  for (int i = 0; i < n; ++i) {
    start[i] = ctxs[i]->steps;
    const int rc = rteom_internal_begin(ctxs[i], nsteps, dt, tol, max_micro);
    if (rc != RTEOM_OK) return rc;
  }
  // rounds: every member with work left evaluates one residual (R(t_n) of a
  // new step, or R(t^(k)) of its next micro-iteration) and its update
  std::vector<rteom_ctx*> mem;
  std::vector<int> which;
  while (true) {
    mem.clear();
    which.clear();
    for (int i = 0; i < n; ++i) {
      rteom_ctx* c = ctxs[i];
      int w = -1;
      const int rc = guarded(c, [&]() -> int {
        auto& r = c->run;
        if (r.phase == 2) return RTEOM_OK;
        if (r.phase == 0) {
          w = 0;
          return RTEOM_OK;
        }
        RT_CUDA(cudaEventSynchronize(r.ev));
        return after_status(c, &w);
      });
      if (rc != RTEOM_OK) return rc;
      if (w >= 0) {
        mem.push_back(c);
        which.push_back(w);
      }
    }
    if (mem.empty()) break;
    const int rc = guarded(mem[0], [&] {
      group_residuals(mem.data(), which.data(), (int)mem.size());
      for (size_t i = 0; i < mem.size(); ++i) {
        auto& r = mem[i]->run;
        if (which[i] == 0) {  // the first micro-iteration starts from t^(0) = t_n
          r.k = 0;
          r.phase = 1;
        }
        launch_update(mem[i], r.k);
      }
      return RTEOM_OK;
    });
    if (rc != RTEOM_OK) return rc;
  }
  for (int i = 0; i < n; ++i) {
    rteom_ctx* c = ctxs[i];
    const int rc = guarded(c, [&] {
      if (C_out && C_out[i])
        RT_CUDA(cudaMemcpyAsync(C_out[i], c->histC + 2 * start[i], 16ull * (nsteps + 1),
                                cudaMemcpyDeviceToHost, c->stream));
      RT_CUDA(cudaStreamSynchronize(c->stream));
      return RTEOM_OK;
    });
    if (rc != RTEOM_OK) return rc;
  }
  return RTEOM_OK;
}

int rteom_spectrum(rteom_ctx* c, const double* omega, int nomega, double eta, double* A_out) {
  if (!c) return RTEOM_ERR_ARG;
  if (nomega < 0 || (nomega > 0 && (!omega || !A_out)) || !(eta >= 0))
    return fail(c, RTEOM_ERR_ARG, "need nomega >= 0, omega/A_out, eta >= 0");
  if (c->steps < 1) return fail(c, RTEOM_ERR_STATE, "no step propagated yet");
  if (nomega == 0) return RTEOM_OK;
  if (!all_finite(omega, nomega)) return fail(c, RTEOM_ERR_NONFINITE, "non-finite omega");
  return guarded(c, [&] {
    double* d_w = c->dmalloc(8ull * nomega);
    double* d_A = c->dmalloc(8ull * nomega);
    RT_CUDA(cudaMemcpyAsync(d_w, omega, 8ull * nomega, cudaMemcpyHostToDevice, c->stream));
    c->E.launch(kElementwise, 0.0, [&] {
      spectrum(c->histC, c->steps, c->dt, c->eps_core + c->e_corr, d_w, nomega, eta, d_A,
               c->stream);
    });
    RT_CUDA(cudaMemcpyAsync(A_out, d_A, 8ull * nomega, cudaMemcpyDeviceToHost, c->stream));
    RT_CUDA(cudaStreamSynchronize(c->stream));
    c->dfree(d_w);
    c->dfree(d_A);
    return RTEOM_OK;
  });
}

int rteom_get_info(const rteom_ctx* c, double* eps_core, double* e_corr, long long* steps_done,
                   long long* micro_total) {
  if (!c) return RTEOM_ERR_ARG;
  if (eps_core) *eps_core = c->eps_core;
  if (e_corr) *e_corr = c->e_corr;
  if (steps_done) *steps_done = c->steps;
  if (micro_total) *micro_total = c->micro_total;
  return RTEOM_OK;
}

long long rteom_state_size(const rteom_ctx* c) { return c ? 2 * unpadded_size(c) : -1; }

int rteom_get_cumulant(const rteom_ctx* c0, long long count, double* C_out, double* E_out) {
  rteom_ctx* c = const_cast<rteom_ctx*>(c0);
  if (!c) return RTEOM_ERR_ARG;
  if (count < 0 || count > c->steps + 1) return fail(c, RTEOM_ERR_ARG, "count > steps_done + 1");
  return guarded(c, [&] {
    if (C_out && count)
      RT_CUDA(cudaMemcpyAsync(C_out, c->histC, 16ull * count, cudaMemcpyDeviceToHost, c->stream));
    if (E_out && count)
      RT_CUDA(cudaMemcpyAsync(E_out, c->histE, 16ull * count, cudaMemcpyDeviceToHost, c->stream));
    RT_CUDA(cudaStreamSynchronize(c->stream));
    return RTEOM_OK;
  });
}

int rteom_get_state(const rteom_ctx* c0, double* t_out, long long* steps, double* hist) {
  rteom_ctx* c = const_cast<rteom_ctx*>(c0);
  if (!c) return RTEOM_ERR_ARG;
  return guarded(c, [&] {
    if (steps) *steps = c->steps;
    if (t_out) {
      double* tmp = c->dmalloc(16ull * unpadded_size(c));
      c->E.launch(kElementwise, 0.0, [&] { unpack_amplitudes(c->g, c->T_N, tmp, c->stream); });
      RT_CUDA(cudaMemcpyAsync(t_out, tmp, 16ull * unpadded_size(c), cudaMemcpyDeviceToHost,
                              c->stream));
      RT_CUDA(cudaStreamSynchronize(c->stream));
      c->dfree(tmp);
    }
    if (hist) {
      const long long n = c->steps + 1;
      RT_CUDA(cudaMemcpyAsync(hist, c->histC, 16ull * n, cudaMemcpyDeviceToHost, c->stream));
      RT_CUDA(cudaMemcpyAsync(hist + 2 * n, c->histE, 16ull * n, cudaMemcpyDeviceToHost, c->stream));
      RT_CUDA(cudaStreamSynchronize(c->stream));
    }
    return RTEOM_OK;
  });
}

int rteom_set_state(rteom_ctx* c, const double* t_in, long long steps, const double* hist) {
  if (!c) return RTEOM_ERR_ARG;
  if (!t_in || steps < 0) return fail(c, RTEOM_ERR_ARG, "need t_in and steps >= 0");
  if (!all_finite(t_in, 2 * unpadded_size(c)))
    return fail(c, RTEOM_ERR_NONFINITE, "non-finite amplitude");
  if (hist && !all_finite(hist, 4 * (steps + 1)))
    return fail(c, RTEOM_ERR_NONFINITE, "non-finite history");
  return guarded(c, [&] {
    double* tmp = c->dmalloc(16ull * unpadded_size(c));
    RT_CUDA(cudaMemcpyAsync(tmp, t_in, 16ull * unpadded_size(c), cudaMemcpyHostToDevice,
                            c->stream));
    c->E.launch(kElementwise, 0.0, [&] { pack_amplitudes(c->g, tmp, c->T_N, c->stream); });
    ensure_hist(c, steps + 1);
    if (hist) {
      const long long n = steps + 1;
      RT_CUDA(cudaMemcpyAsync(c->histC, hist, 16ull * n, cudaMemcpyHostToDevice, c->stream));
      RT_CUDA(cudaMemcpyAsync(c->histE, hist + 2 * n, 16ull * n, cudaMemcpyHostToDevice, c->stream));
    } else {
      // a restart without history: C = 0 and E = E(t) at this step
      RT_CUDA(cudaMemsetAsync(c->histC, 0, 16ull * (steps + 1), c->stream));
      RT_CUDA(cudaMemsetAsync(c->histE, 0, 16ull * (steps + 1), c->stream));
      energy_into(c, c->T_N, c->histE, c->histC, steps - 1, 0);
    }
    RT_CUDA(cudaStreamSynchronize(c->stream));
    c->dfree(tmp);
    c->steps = steps;
    return RTEOM_OK;
  });
}

int rteom_plan_bytes(int nocc, int nvir, int nchol, int precision, int flags, double* bytes) {
  if (!bytes || nocc < 1 || nvir < 1 || nchol < 0 ||
      (flags & ~(RTEOM_FLAG_CUMULANT_NO_FOV | RTEOM_FLAG_LADDER_CHOLESKY |
                 RTEOM_FLAG_ANDERSON | RTEOM_FLAG_GROUPED)) ||
      !valid_precision(precision) || (double)(nvir + 1) * (nvir + 1) > 2.0e9 ||
      !grouped_flags_ok(precision, flags))
    return RTEOM_ERR_ARG;
  try {
    plan_context_bytes(nocc, nvir, nchol, precision,
                       (flags & RTEOM_FLAG_LADDER_CHOLESKY) && nchol > 0,
                       (flags & RTEOM_FLAG_ANDERSON) != 0, (flags & RTEOM_FLAG_GROUPED) != 0,
                       bytes);
  } catch (const std::exception&) {
    return RTEOM_ERR_ARG;
  }
  return RTEOM_OK;
}

int rteom_debug_residual(rteom_ctx* c, const double* t_in, double* R_out, double* E_out) {
  if (!c) return RTEOM_ERR_ARG;
  if (!t_in || !R_out) return fail(c, RTEOM_ERR_ARG, "need t_in and R_out");
  if (!all_finite(t_in, 2 * unpadded_size(c)))
    return fail(c, RTEOM_ERR_NONFINITE, "non-finite amplitude");
  return guarded(c, [&] {
    const size_t ub = 16ull * unpadded_size(c);
    double* tmp = c->dmalloc(ub);
    RT_CUDA(cudaMemcpyAsync(tmp, t_in, ub, cudaMemcpyHostToDevice, c->stream));
    c->E.launch(kElementwise, 0.0, [&] { pack_amplitudes(c->g, tmp, c->T_K, c->stream); });
    residual_eager(c, c->T_K, c->R_K);
    c->E.launch(kElementwise, 0.0, [&] { unpack_amplitudes(c->g, c->R_K, tmp, c->stream); });
    RT_CUDA(cudaMemcpyAsync(R_out, tmp, ub, cudaMemcpyDeviceToHost, c->stream));
    RT_CUDA(cudaMemcpyAsync(c->h_maxdiff, c->maxdiff, 16, cudaMemcpyDeviceToHost, c->stream));
    if (E_out) {
      // scalars[2..3] receive E (index n+1 = 1 of a two-entry history at scalars+0)
      energy_into(c, c->T_K, c->scalars, c->scalars, 0, 0);
      RT_CUDA(cudaMemcpyAsync(E_out, c->scalars + 2, 16, cudaMemcpyDeviceToHost, c->stream));
    }
    RT_CUDA(cudaStreamSynchronize(c->stream));
    c->dfree(tmp);
    if (c->E.timing) c->E.collect_timing();
    if (c->h_maxdiff[1] != 0)
      return fail(c, RTEOM_ERR_CUDA, "tensor-core pipeline wait timed out");
    return RTEOM_OK;
  });
}

int rteom_debug_residual_sparse(rteom_ctx* c, const long long* t_index, const double* t_val,
                                long long nt, const long long* r_index, long long nr,
                                double* R_out) {
  if (!c) return RTEOM_ERR_ARG;
  if (nt < 0 || nr < 0 || (nt > 0 && (!t_index || !t_val)) || (nr > 0 && (!r_index || !R_out)))
    return fail(c, RTEOM_ERR_ARG, "need nt, nr >= 0 and the index/value arrays they count");
  const long long n = unpadded_size(c);
  for (long long k = 0; k < nt; ++k)
    if (t_index[k] < 0 || t_index[k] >= n)
      return fail(c, RTEOM_ERR_ARG, "t_index[" + std::to_string(k) + "] outside the amplitude vector");
  for (long long k = 0; k < nr; ++k)
    if (r_index[k] < 0 || r_index[k] >= n)
      return fail(c, RTEOM_ERR_ARG, "r_index[" + std::to_string(k) + "] outside the amplitude vector");
  if (nt > 0 && !all_finite(t_val, 2 * (size_t)nt))
    return fail(c, RTEOM_ERR_NONFINITE, "non-finite amplitude");
  return guarded(c, [&] {
    cudaStream_t st = c->stream;
    long long* d_ti = nt ? reinterpret_cast<long long*>(c->dmalloc(8ull * nt)) : nullptr;
    double* d_tv = nt ? c->dmalloc(16ull * nt) : nullptr;
    long long* d_ri = nr ? reinterpret_cast<long long*>(c->dmalloc(8ull * nr)) : nullptr;
    double* d_R = nr ? c->dmalloc(16ull * nr) : nullptr;
    if (nt) {
      RT_CUDA(cudaMemcpyAsync(d_ti, t_index, 8ull * nt, cudaMemcpyHostToDevice, st));
      RT_CUDA(cudaMemcpyAsync(d_tv, t_val, 16ull * nt, cudaMemcpyHostToDevice, st));
    }
    if (nr) RT_CUDA(cudaMemcpyAsync(d_ri, r_index, 8ull * nr, cudaMemcpyHostToDevice, st));
    RT_CUDA(cudaMemsetAsync(c->T_K, 0, 16ull * c->g.total(), st));
    c->E.launch(kElementwise, 0.0, [&] { scatter_unpadded(c->g, d_ti, d_tv, nt, c->T_K, st); });
    residual_eager(c, c->T_K, c->R_K);
    c->E.launch(kElementwise, 0.0, [&] { gather_unpadded(c->g, c->R_K, d_ri, nr, d_R, st); });
    if (nr) RT_CUDA(cudaMemcpyAsync(R_out, d_R, 16ull * nr, cudaMemcpyDeviceToHost, st));
    RT_CUDA(cudaMemcpyAsync(c->h_maxdiff, c->maxdiff, 16, cudaMemcpyDeviceToHost, st));
    RT_CUDA(cudaStreamSynchronize(st));
    for (void* p : {(void*)d_ti, (void*)d_tv, (void*)d_ri, (void*)d_R})
      if (p) c->dfree(p);
    if (c->E.timing) c->E.collect_timing();
    if (c->h_maxdiff[1] != 0)
      return fail(c, RTEOM_ERR_CUDA, "tensor-core pipeline wait timed out");
    return RTEOM_OK;
  });
}

int rteom_set_timing(rteom_ctx* c, int on) {
  if (!c) return RTEOM_ERR_ARG;
  if (on < 0 || on > 3) return fail(c, RTEOM_ERR_ARG, "timing mode must be 0, 1, 2 or 3");
  if (c->grouped && on != 0)
    return fail(c, RTEOM_ERR_ARG, "timing modes are not available with the grouped ladder");
  c->E.timing = on != 0;
  c->eager_timing = on == 2;
  c->E.graph_timed_mask = on == 3 ? (1u << kLadder) | (1u << kContract) : (1u << kLadder);
  return RTEOM_OK;
}

int rteom_get_timing(rteom_ctx* c, double* ms, long long* launches, double* flops, double* bytes,
                     int reset) {
  if (!c) return RTEOM_ERR_ARG;
  return guarded(c, [&] {
    c->E.collect_timing();
    for (int k = 0; k < kNumClasses; ++k) {
      if (ms) ms[k] = c->E.ms[k];
      if (launches) launches[k] = c->E.tlaunch[k];
      if (flops) flops[k] = c->E.tflops[k];
      if (bytes) bytes[k] = c->E.tbytes[k];
      if (reset) {
        c->E.ms[k] = 0;
        c->E.tlaunch[k] = 0;
        c->E.tflops[k] = 0;
        c->E.tbytes[k] = 0;
      }
    }
    return RTEOM_OK;
  });
}

long long rteom_kernel_launches(const rteom_ctx* c) { return c ? c->E.launches : -1; }

void rteom_destroy(rteom_ctx* c) { delete c; }

const char* rteom_last_error(const rteom_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
