// Contraction engine implementation (see engine.h).
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <mutex>

#include "engine.h"

namespace rteom {

namespace {

constexpr int64_t kMin3mK = 2048;  // shortest K of a 3M complex product

struct Parsed {
  std::string a, b, c;
};

Parsed parse(const char* spec) {
  Parsed p;
  const char* arrow = std::strstr(spec, "->");
  if (!arrow) throw Error(-1, std::string("contract: no '->' in spec ") + spec);
  std::string lhs(spec, arrow - spec);
  p.c = std::string(arrow + 2);
  auto comma = lhs.find(',');
  if (comma == std::string::npos) {
    p.a = lhs;
  } else {
    p.a = lhs.substr(0, comma);
    p.b = lhs.substr(comma + 1);
  }
  return p;
}

int64_t prod(const std::string& labels, const int64_t* dimof) {
  int64_t n = 1;
  for (char ch : labels) n *= dimof[(unsigned char)ch];
  return n;
}

// Strides (in elements) of every label of a row-major tensor.
void strides_of(const std::string& labels, const Tensor& t, int64_t* strideof) {
  int64_t s = 1;
  for (int k = (int)labels.size() - 1; k >= 0; --k) {
    strideof[(unsigned char)labels[k]] = s;
    s *= t.dim[k];
  }
}

std::string ordered(const std::string& from, const std::string& keep) {
  std::string r;
  for (char ch : from)
    if (keep.find(ch) != std::string::npos) r += ch;
  return r;
}

}  // namespace

Engine::~Engine() {
  for (auto& p : pending_) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : free_events_) cudaEventDestroy(e);
}

cudaEvent_t Engine::get_event() {
  if (!free_events_.empty()) {
    cudaEvent_t e = free_events_.back();
    free_events_.pop_back();
    return e;
  }
  cudaEvent_t e;
  RT_CUDA(cudaEventCreate(&e));
  return e;
}

bool Engine::trace_on() const {
  const char* t = std::getenv("RTEOM_TRACE");
  return t && *t;
}

void Engine::collect_timing() {
  if (pending_.empty()) return;
  RT_CUDA(cudaStreamSynchronize(stream));
  FILE* tf = trace_on() ? std::fopen(std::getenv("RTEOM_TRACE"), "a") : nullptr;
  static const char* names[kNumClasses] = {"ladder", "contract", "permute", "elementwise"};
  for (auto& p : pending_) {
    float t = 0.f;
    RT_CUDA(cudaEventElapsedTime(&t, p.a, p.b));
    ms[p.cls] += t;
    if (tf)
      std::fprintf(tf, "{\"class\": \"%s\", \"what\": \"%s\", \"flops\": %.6g, \"ms\": %.6g}\n",
                   names[p.cls], p.what.c_str(), p.flops, t);
    free_events_.push_back(p.a);
    free_events_.push_back(p.b);
  }
  if (tf) std::fclose(tf);
  pending_.clear();
}

bool Engine::collect_graph_timing(const std::vector<GraphPair>& pairs) {
  for (const auto& p : pairs) {
    float t = 0.f;
    cudaError_t e = cudaEventElapsedTime(&t, p.a, p.b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      graph_timing_ok = false;
      return false;
    }
    ms[p.cls] += t;
    tlaunch[p.cls] += 1;
    tflops[p.cls] += p.flops;
    tbytes[p.cls] += p.bytes;
  }
  return true;
}

namespace {

std::mutex g_tune_mu;
std::map<std::string, GemmChoice> g_tune;  // process-wide autotuner choices

std::string tune_key(const GemmDesc& g, int form) {
  char buf[320];
  std::snprintf(buf, sizeof buf, "%d,%d,%d,%d|%d%d%d%d|%lld,%lld,%lld,%lld,%lld,%lld|%d|%d", g.M,
                g.N, g.K, g.batch, (int)g.Acplx, (int)g.Bcplx, (int)g.transA, (int)g.transB,
                (long long)g.lda, (long long)g.ldb, (long long)g.ldc, (long long)g.strideA,
                (long long)g.strideB, (long long)g.strideC, (int)(g.beta != 0.0), form);
  return buf;
}

bool tune_lookup(const std::string& k, GemmChoice* c) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *c = it->second;
  return true;
}

// First choice stored for a key wins; returns the stored one.
GemmChoice tune_store(const std::string& k, const GemmChoice& c) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune.emplace(k, c).first->second;
}

// FP64 candidates: every tile shape with 1, 2, 4, ... K slices while a slice
// keeps at least 16 of K, the grid stays within 8 waves and the partial
// sums within 16 outputs' worth (and 256 MB).
std::vector<GemmChoice> f64_candidates(const GemmDesc& g) {
  std::vector<GemmChoice> out;
  const int64_t outd = (int64_t)g.M * g.N * g.batch * ((g.Acplx || g.Bcplx) ? 2 : 1);
  for (int t = 0; t < gemm_f64_tiles(); ++t) {
    int tbm = 0, tbn = 0;
    gemm_f64_tile_shape(t, &tbm, &tbn);
    if ((g.M + tbm - 1) / tbm > 65535) continue;  // grid y limit
    for (int s = 1; s <= 64; s *= 2) {
      if (s > 1 && g.K / s < 16) break;
      GemmDesc d = g;
      d.tile = t;
      d.splits = s;
      if (gemm_f64_splits(d) != s) break;
      const int64_t ws = gemm_f64_workspace(d);
      if (ws > 16 * outd || ws * 8 > (int64_t(256) << 20)) break;
      int bm = 0, bn = 0;
      gemm_f64_tile_shape(t, &bm, &bn);
      const int64_t blocks = (int64_t)((g.M + bm - 1) / bm) * ((g.N + bn - 1) / bn) * g.batch * s;
      if (s > 1 && blocks > 8 * 148) break;
      out.push_back({false, false, t, s});
    }
  }
  return out;
}

// The digit-plane kernels tile A' in 128 rows and B' in 32 to 256 rows: a
// GEMM runs as C^T = B^T A^T (output written transposed) when that pads much
// less, or, with K up to kOzShortK, when its output is row-major and the
// transposed problem pads about as much.  The kernel's drain gives each lane
// one GEMM row, so only the transposed problem stores a row-major output
// coalesced (adjacent lanes, adjacent addresses), and with short K those
// stores, not the MMAs, set the time (a 2255 x 203401 x 1800 product ran at
// a third of the tensor peak with lane-per-row stores).
constexpr int64_t kOzShortK = 4096;

int64_t oz_padded(int64_t ra, int64_t rb, int S) {
  const int64_t bn = oz_tile_n(rb, S);
  return (ra + 127) / 128 * 128 * ((rb + bn - 1) / bn * bn);
}

bool oz_swap(const GemmDesc& g, int S) {
  const int64_t ra = (g.Acplx && !g.Bcplx) ? 2 * g.M : g.M, rb = g.Bcplx ? 2 * g.N : g.N;
  const int64_t sa = (g.Bcplx && !g.Acplx) ? 2 * g.N : g.N, sb = g.Acplx ? 2 * g.M : g.M;
  const int64_t straight = oz_padded(ra, rb, S), transposed = oz_padded(sa, sb, S);
  if (4 * transposed < 3 * straight) return true;
  return !g.transC && g.M > 1 && g.K <= kOzShortK && 10 * transposed <= 11 * straight;
}

GemmDesc swapped(const GemmDesc& g) {
  GemmDesc s = g;
  s.M = g.N;
  s.N = g.M;
  s.A = g.B;
  s.Acplx = g.Bcplx;
  s.transA = !g.transB;
  s.lda = g.ldb;
  s.strideA = g.strideB;
  s.B = g.A;
  s.Bcplx = g.Acplx;
  s.transB = !g.transA;
  s.ldb = g.lda;
  s.strideB = g.strideA;
  s.va = g.vb;
  s.vb = g.va;
  s.transC = !g.transC;
  return s;
}

// View with rows over the labels `rows` and columns over `cols` (each at
// most three labels; an empty group is one index of extent 1).
View2 make_view(const std::string& rows, const std::string& cols, const int64_t* strideof,
                const int64_t* dimof) {
  View2 v;
  auto fill = [&](const std::string& l, int& n, int* ext, int64_t* str) {
    n = 0;
    for (char ch : l) {
      ext[n] = (int)dimof[(unsigned char)ch];
      str[n] = strideof[(unsigned char)ch];
      ++n;
    }
    if (n == 0) {
      ext[0] = 1;
      str[0] = 0;
      n = 1;
    }
  };
  fill(rows, v.rdims, v.rext, v.rstr);
  fill(cols, v.kdims, v.kext, v.kstr);
  // merge neighbouring indices that are contiguous in memory (fewer splits)
  auto merge = [](int& n, int* ext, int64_t* str) {
    for (int d = n - 1; d > 0; --d)
      if (str[d - 1] == (int64_t)ext[d] * str[d]) {
        ext[d - 1] *= ext[d];
        str[d - 1] = str[d];
        for (int e = d; e < n - 1; ++e) {
          ext[e] = ext[e + 1];
          str[e] = str[e + 1];
        }
        --n;
      }
  };
  merge(v.rdims, v.rext, v.rstr);
  merge(v.kdims, v.kext, v.kstr);
  view_prepare(v);
  return v;
}

bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  RT_CUDA(cudaStreamIsCapturing(st, &cs));
  return cs != cudaStreamCaptureStatusNone;
}

}  // namespace

// Scratch of one tuning session: an output of C's size (the trials write it
// with beta = 0), the largest split-K workspace among the FP64 candidates
// and, for the tensor-core candidate, packed operands and partials.  With
// out == nullptr (planning) the scratch is only reserved in the arena;
// otherwise every candidate runs once (screened out when over twice the
// best so far) and then twice more timed, and the fastest is returned.  Operands the tensor-core cache would hold are packed
// outside the timing.
void Engine::tuning_scratch(const GemmDesc& g, bool tc_ok, bool oz_ok, bool a_const,
                            bool b_const, GemmChoice* out) {
  std::vector<GemmChoice> cands = f64_candidates(g);
  if (tc_ok) cands.push_back({true, false, -1, 0});
  if (oz_ok) cands.push_back({false, true, -1, 0});
  const int64_t mark = arena.mark();
  GemmDesc base = g;
  base.beta = 0.0;
  base.tile = -1;
  base.splits = 0;
  base.C = arena.alloc((int64_t)g.M * g.N * g.batch * ((g.Acplx || g.Bcplx) ? 2 : 1));
  int64_t wsmax = 0;
  for (const auto& c : cands) {
    if (c.tc || c.oz) continue;
    GemmDesc d = base;
    d.tile = c.tile;
    d.splits = c.splits;
    wsmax = std::max(wsmax, gemm_f64_workspace(d));
  }
  double* ws = wsmax ? arena.alloc(wsmax) : nullptr;
  auto bytes_alloc = [&](int64_t bytes) { return static_cast<void*>(arena.alloc((bytes + 7) / 8)); };
  void *a0 = nullptr, *a1 = nullptr, *b0 = nullptr, *b1 = nullptr, *P = nullptr;
  if (tc_ok) {
    const TcLayout L = gemm_tc_layout(base);
    a0 = bytes_alloc(4 * L.a_elems);
    a1 = bytes_alloc(4 * L.a_elems);
    b0 = bytes_alloc(4 * L.b_elems);
    b1 = bytes_alloc(4 * L.b_elems);
    if (L.p_elems) P = bytes_alloc(8 * L.p_elems);
  }
  const bool oz_sw = oz_ok && oz_swap(base, oz_planes);
  const GemmDesc ozd = oz_sw ? swapped(base) : base;
  if (oz_ok) {
    const OzLayout L = gemm_oz_layout(ozd, oz_planes);
    a0 = bytes_alloc(2 * L.planes * L.a_elems);
    a1 = bytes_alloc(4 * L.a_rows);
    b0 = bytes_alloc(2 * L.planes * L.b_elems);
    b1 = bytes_alloc(4 * L.b_rows);
    if (L.p_elems) P = bytes_alloc(8 * L.p_elems);
  }
  if (out == nullptr || dry) {
    arena.release(mark);
    return;
  }
  auto pack_a = [&] {
    if (tc_ok)
      gemm_tc_pack_a(base, static_cast<float*>(a0), static_cast<float*>(a1), stream);
    else
      gemm_oz_pack_a(ozd, oz_planes, static_cast<uint16_t*>(a0), static_cast<int*>(a1), stream);
  };
  auto pack_b = [&] {
    if (tc_ok)
      gemm_tc_pack_b(base, static_cast<float*>(b0), static_cast<float*>(b1), stream);
    else
      gemm_oz_pack_b(ozd, oz_planes, static_cast<uint16_t*>(b0), static_cast<int*>(b1), stream);
  };
  // operands the cache would hold are packed outside the timing (with the
  // orientation swapped, the packed A' comes from B and B' from A)
  const bool pa_const = oz_sw ? b_const : a_const, pb_const = oz_sw ? a_const : b_const;
  if (tc_ok || oz_ok) {
    if (pa_const) pack_a();
    if (pb_const) pack_b();
  }
  cudaEvent_t e0 = get_event(), e1 = get_event();
  float best_ms = std::numeric_limits<float>::infinity();
  GemmChoice best;
  for (const auto& c : cands) {
    auto run = [&] {
      if (c.tc || c.oz) {
        if (!pa_const) pack_a();
        if (!pb_const) pack_b();
        if (c.tc) {
          gemm_tc_mma(base, static_cast<float*>(a0), static_cast<float*>(a1),
                      static_cast<float*>(b0), static_cast<float*>(b1), static_cast<float2*>(P),
                      tc_err, stream);
          gemm_tc_finalize(base, static_cast<float2*>(P), stream);
        } else {
          gemm_oz_mma(ozd, oz_planes, static_cast<uint16_t*>(a0), static_cast<int*>(a1),
                      static_cast<uint16_t*>(b0), static_cast<int*>(b1), static_cast<float2*>(P),
                      tc_err, stream);
          gemm_oz_finalize(ozd, oz_planes, static_cast<int*>(a1), static_cast<int*>(b1),
                           static_cast<float2*>(P), stream);
        }
      } else {
        GemmDesc d = base;
        d.tile = c.tile;
        d.splits = c.splits;
        d.work = ws;
        gemm_f64(d, stream);
      }
    };
    auto timed = [&](int reps) {
      RT_CUDA(cudaEventRecord(e0, stream));
      for (int r = 0; r < reps; ++r) run();
      RT_CUDA(cudaEventRecord(e1, stream));
      RT_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      RT_CUDA(cudaEventElapsedTime(&t, e0, e1));
      return t / reps;
    };
    // first run (cold) screens out clearly slower candidates
    if (timed(1) > 2.0f * best_ms) continue;
    const float ms = timed(2);
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  free_events_.push_back(e0);
  free_events_.push_back(e1);
  arena.release(mark);
  *out = best;
}

void Engine::axpy(const char* spec, double alpha, const Tensor& X, double beta, const Tensor& Y) {
  Parsed p = parse(spec);
  if ((int)p.a.size() != X.nd || (int)p.c.size() != Y.nd || p.a.size() != p.c.size())
    throw Error(-1, std::string("axpy: rank mismatch in ") + spec);
  if (X.cplx && !Y.cplx) throw Error(-1, std::string("axpy: complex into real in ") + spec);
  int64_t sx[256];
  strides_of(p.a, X, sx);
  PermDesc d;
  d.nd = Y.nd;
  for (int k = 0; k < Y.nd; ++k) {
    auto pos = p.a.find(p.c[k]);
    if (pos == std::string::npos) throw Error(-1, std::string("axpy: label missing in ") + spec);
    if (X.dim[pos] != Y.dim[k]) throw Error(-1, std::string("axpy: dim mismatch in ") + spec);
    d.out_dim[k] = Y.dim[k];
    d.in_stride[k] = sx[(unsigned char)p.c[k]];
  }
  launch(kPermute, 0.0, [&] { permute_add(X.p, Y.p, d, X.cplx, Y.cplx, alpha, beta, stream); },
         spec);
}

void Engine::contract(const char* spec, double alpha, const Tensor& A, const Tensor& B,
                      double beta, const Tensor& C, KernelClass cls) {
  Parsed p = parse(spec);
  if ((int)p.a.size() != A.nd || (int)p.b.size() != B.nd || (int)p.c.size() != C.nd)
    throw Error(-1, std::string("contract: rank mismatch in ") + spec);
  if (C.cplx != (A.cplx || B.cplx))
    throw Error(-1, std::string("contract: output type mismatch in ") + spec);
  int64_t dimof[256];
  std::fill(dimof, dimof + 256, -1);
  auto setdim = [&](const std::string& l, const Tensor& t) {
    for (size_t k = 0; k < l.size(); ++k) {
      unsigned char ch = l[k];
      if (dimof[ch] >= 0 && dimof[ch] != t.dim[k])
        throw Error(-1, std::string("contract: inconsistent dim for label in ") + spec);
      dimof[ch] = t.dim[k];
    }
  };
  setdim(p.a, A);
  setdim(p.b, B);
  setdim(p.c, C);

  std::string batch, Ml, Nl, Kl;
  for (char ch : p.c) {
    bool inA = p.a.find(ch) != std::string::npos, inB = p.b.find(ch) != std::string::npos;
    if (inA && inB)
      batch += ch;
    else if (inA)
      Ml += ch;
    else if (inB)
      Nl += ch;
    else
      throw Error(-1, std::string("contract: output label in neither input: ") + spec);
  }
  for (char ch : p.a) {
    if (p.c.find(ch) != std::string::npos) continue;
    if (p.b.find(ch) == std::string::npos)
      throw Error(-1, std::string("contract: label summed over one input only: ") + spec);
    Kl += ch;
  }
  for (char ch : p.b)
    if (p.c.find(ch) == std::string::npos && p.a.find(ch) == std::string::npos)
      throw Error(-1, std::string("contract: label summed over one input only: ") + spec);

  // choose label orders of the M, N and K groups that avoid the most copying
  std::string Mc[2] = {Ml, ordered(p.a, Ml)};
  std::string Nc[2] = {Nl, ordered(p.b, Nl)};
  std::string Kc[2] = {ordered(p.a, Kl), ordered(p.b, Kl)};
  int64_t best = -1;
  std::string bM, bN, bK;
  bool bTA = false, bTB = false, bPA = false, bPB = false, bPC = false;
  for (int im = 0; im < 2; ++im)
    for (int in = 0; in < 2; ++in)
      for (int ik = 0; ik < 2; ++ik) {
        const std::string &M = Mc[im], &N = Nc[in], &K = Kc[ik];
        int64_t cost = 0;
        bool ta = false, tb = false, pa = false, pb = false, pc = false;
        if (p.a == batch + M + K) {
        } else if (p.a == batch + K + M) {
          ta = true;
        } else {
          pa = true;
          cost += A.numel();
        }
        if (p.b == batch + K + N) {
        } else if (p.b == batch + N + K) {
          tb = true;
        } else {
          pb = true;
          cost += B.numel();
        }
        if (p.c != batch + M + N) {
          pc = true;
          cost += 2 * C.numel();
        }
        if (best < 0 || cost < best) {
          best = cost;
          bM = M;
          bN = N;
          bK = K;
          bTA = ta;
          bTB = tb;
          bPA = pa;
          bPB = pb;
          bPC = pc;
        }
      }

  const int64_t Mt = prod(bM, dimof), Nt = prod(bN, dimof), Kt = prod(bK, dimof),
                Bt = prod(batch, dimof);
  if (Mt > 0x7fffffff || Nt > 0x7fffffff || Kt > 0x7fffffff || Bt > 65535)
    throw Error(-1, std::string("contract: problem too large: ") + spec);
  int64_t mark = arena.mark();

  auto permuted = [&](const Tensor& T, const std::string& from, const std::string& to) {
    Tensor out;
    out.cplx = T.cplx;
    out.nd = (int)to.size();
    for (int k = 0; k < out.nd; ++k) out.dim[k] = dimof[(unsigned char)to[k]];
    out.p = arena.alloc(out.doubles());
    axpy((from + "->" + to).c_str(), 1.0, T, 0.0, out);
    return out;
  };

  const double mult0 = (A.cplx && B.cplx) ? 8.0 : (A.cplx || B.cplx) ? 4.0 : 2.0;
  const double flops0 = mult0 * (double)Mt * (double)Nt * (double)Kt * (double)Bt;
  bool use_tc = tensor_cores && flops0 >= tc_min_flops;
  bool use_oz = fp64_emulation && flops0 >= oz_min_flops;
  const bool grouped = defer_ladder && cls == kLadder;
  if (grouped) {
    if (!fp64_emulation)
      throw Error(-1, std::string("contract: the grouped ladder needs a digit-plane form: ") + spec);
    use_tc = false;
    use_oz = true;
  }

  GemmDesc g;
  g.M = (int)Mt;
  g.N = (int)Nt;
  g.K = (int)Kt;
  g.batch = (int)Bt;
  g.Acplx = A.cplx;
  g.transA = bTA;
  g.lda = bTA ? Mt : Kt;
  g.strideA = Mt * Kt;
  g.Bcplx = B.cplx;
  g.transB = bTB;
  g.ldb = bTB ? Kt : Nt;
  g.strideB = Kt * Nt;
  g.ldc = Nt;
  g.strideC = Mt * Nt;
  g.alpha = alpha;
  g.beta = bPC ? 0.0 : beta;
  g.wait_cycles = tc_wait_cycles;
  g.one_range = grouped;

  // launch configuration from the autotuner, when it has one for this shape
  const bool tunable =
      autotune && !use_tc && !use_oz && !gemm_f64_is_gemv(g) && flops0 <= tune_max_flops;
  const bool tc_ok = tensor_cores && flops0 >= tc_tune_min_flops;
  const bool oz_ok = fp64_emulation && flops0 >= tc_tune_min_flops;
  // form of the key: FP64 only, or with the split-TF32, 7-plane, 3-plane or
  // FP16 two-plane tensor-core candidate
  const int form = tc_ok ? 1 : (oz_ok ? (oz_planes == 3 ? 3 : (oz_planes == 2 ? 4 : 2)) : 0);
  const std::string tkey = tunable ? tune_key(g, form) : std::string();
  GemmChoice choice;
  bool chosen = tunable && tune_lookup(tkey, &choice);
  if (chosen && choice.tc) use_tc = true;
  if (chosen && choice.oz) use_oz = true;
  const bool packed_path = use_tc || use_oz;

  // tensor-core operands of constant tensors may already be packed
  auto key = [&](const char* role, const Tensor& T) {
    return std::string(role) + "|" + spec + "|" + std::to_string((uintptr_t)T.p) + "|" +
           std::to_string(Mt) + "," + std::to_string(Nt) + "," + std::to_string(Kt) + "," +
           std::to_string(Bt);
  };
  const Packed* cA = nullptr;
  const Packed* cB = nullptr;
  // emulated FP64 may run the GEMM transposed; the packs then change roles
  const bool swap = use_oz && oz_swap(g, oz_planes);
  const char* roleA = swap ? "sB" : "A";
  const char* roleB = swap ? "sA" : "B";
  if (packed_path && A.constant) {
    auto it = tc_cache_.find(key(roleA, A));
    if (it != tc_cache_.end()) cA = &it->second;
  }
  if (packed_path && B.constant) {
    auto it = tc_cache_.find(key(roleB, B));
    if (it != tc_cache_.end()) cB = &it->second;
  }
  // held operands: a pack made by the pack-only pass ahead of the chunk
  // loop (room for it is taken below this call's scratch, so it stays at the
  // loop's level).  A pack depends on its own tensor's extent and K only, so
  // the key leaves out the other operand's extent and narrower chunks share
  // it; a chunk whose GEMM takes another orientation (another role) packs
  // into its own scratch.
  auto hkey = [&](const char* role, const Tensor& T, bool is_a) {
    return std::string(role) + "|" + spec + "|" + std::to_string((uintptr_t)T.p) + "|" +
           std::to_string(is_a ? Mt : Nt) + "," + std::to_string(Kt) + "," + std::to_string(Bt);
  };
  bool holdA = false, holdB = false;
  if (packed_path) {
    if (!cA && !A.constant && held_.count(A.p)) {
      auto it = held_packs_.find(hkey(roleA, A, true));
      if (it != held_packs_.end())
        cA = &it->second;
      else
        holdA = pack_only;  // made only by the pass ahead of the loop
    }
    if (!cB && !B.constant && held_.count(B.p)) {
      auto it = held_packs_.find(hkey(roleB, B, false));
      if (it != held_packs_.end())
        cB = &it->second;
      else
        holdB = pack_only;
    }
  }
  Packed heldA, heldB;
  if (holdA || holdB) {  // nothing of this call is in the arena yet
    int64_t a0 = 0, a1 = 0, b0 = 0, b1 = 0;  // bytes of the A-role and B-role packs
    if (use_tc) {
      const TcLayout L = gemm_tc_layout(g);
      a0 = a1 = 4 * L.a_elems;
      b0 = b1 = 4 * L.b_elems;
    } else {
      const OzLayout L = gemm_oz_layout(swap ? swapped(g) : g, oz_planes);
      a0 = 2 * L.planes * L.a_elems;
      a1 = 4 * L.a_rows;
      b0 = 2 * L.planes * L.b_elems;
      b1 = 4 * L.b_rows;
      if (swap) {  // the tensor A is packed in the B role of the transposed GEMM
        std::swap(a0, b0);
        std::swap(a1, b1);
      }
    }
    if (holdA) {
      heldA.p0 = arena.alloc((a0 + 7) / 8);
      heldA.p1 = arena.alloc((a1 + 7) / 8);
    }
    if (holdB) {
      heldB.p0 = arena.alloc((b0 + 7) / 8);
      heldB.p1 = arena.alloc((b1 + 7) / 8);
    }
    mark = arena.mark();  // the held packs outlive this call
  }

  if (!dry && ((A.released && !cA) || (B.released && !cB)))
    throw Error(-3, std::string("contract: freed operand without a cached pack in ") + spec);
  // The tensor-core packers read strided views of the operands in place of
  // permuted copies (unbatched, at most three labels per index group), where
  // the view keeps their loads coalesced: after merging contiguous indices,
  // either the columns (K) or the rows form one unit-stride run.  Other
  // operands are permuted first, which measured faster.  The output keeps its
  // row-major copy and permute-add when its layout differs: an epilogue
  // writing a permuted, accumulated output directly scatters its stores
  // across rows and waits on every old value, which measured two to three
  // times slower.
  bool fusedA = false, fusedB = false;
  if (packed_path && batch.empty() && bM.size() <= 3 && bN.size() <= 3 && bK.size() <= 3) {
    auto coalesced = [](const View2& v) {
      return (v.kdims == 1 && v.kstr[0] == 1) || (v.rdims == 1 && v.rstr[0] == 1);
    };
    int64_t sa[256], sb[256];
    strides_of(p.a, A, sa);
    strides_of(p.b, B, sb);
    const View2 va = make_view(bM, bK, sa, dimof), vb = make_view(bN, bK, sb, dimof);
    fusedA = bPA && coalesced(va);
    fusedB = bPB && coalesced(vb);
    if (fusedA) g.va = va;
    if (fusedB) g.vb = vb;
  }
  const bool fused = fusedA || fusedB;
  if (pack_only && !packed_path) {  // only tensor-core packs are made ahead
    arena.release(mark);
    return;
  }
  const Tensor Ause = (bPA && !cA && !fusedA && !(pack_only && !A.constant && !holdA))
                          ? permuted(A, p.a, batch + bM + bK)
                          : A;
  const Tensor Buse = (bPB && !cB && !fusedB && !(pack_only && !B.constant && !holdB))
                          ? permuted(B, p.b, batch + bK + bN)
                          : B;
  Tensor Cuse = C;
  const bool outcopy = bPC;
  if (outcopy) {
    Cuse.nd = (int)(batch + bM + bN).size();
    std::string lab = batch + bM + bN;
    for (int k = 0; k < Cuse.nd; ++k) Cuse.dim[k] = dimof[(unsigned char)lab[k]];
    Cuse.p = arena.alloc(Cuse.doubles());
  }
  g.A = Ause.p;
  g.B = Buse.p;
  g.C = Cuse.p;

  if (tunable && dry) tuning_scratch(g, tc_ok, oz_ok, A.constant, B.constant, nullptr);
  if (tunable && !chosen && tuning && !dry && !stream_capturing(stream)) {
    GemmChoice c;
    tuning_scratch(g, tc_ok, oz_ok, A.constant, B.constant, &c);
    choice = tune_store(tkey, c);
    chosen = true;
    ++tuned;
    if (choice.tc) use_tc = true;
    if (choice.oz) use_oz = true;
  }
  if (chosen && !choice.tc && !choice.oz) {
    g.tile = choice.tile;
    g.splits = choice.splits;
  }
  const double flops = flops0;
  const std::string label =
      trace_on() ? std::string(spec) + " M=" + std::to_string(Mt) + " N=" + std::to_string(Nt) +
                       " K=" + std::to_string(Kt) + " b=" + std::to_string(Bt) +
                       (use_tc || use_oz
                            ? std::string(use_tc ? " tc" : (swap ? " oz^T" : " oz")) +
                                  (cA ? " cA" : "") +
                                  (cB ? " cB" : "")
                            : " s=" + std::to_string(gemm_f64_splits(g))) +
                       (fused ? std::string(" views") : std::string()) +
                       (bPA && !fusedA ? " pA" : "") + (bPB && !fusedB ? " pB" : "") +
                       (outcopy ? " pC" : "")
                 : std::string();
  if (cls == kLadder && !dry && !pack_only) nvtxRangePushA("rteom_ladder");
  // RTEOM_NVTX_CONTRACT set: one NVTX range per contraction named after its
  // spec ("c_imae_mbej2ijab" for "imae,mbej->ijab"), so that a profiler can
  // select the launches of one contraction
  static const bool nvtx_each = std::getenv("RTEOM_NVTX_CONTRACT") != nullptr;
  const bool nvtx_here = nvtx_each && !dry && !pack_only;
  if (nvtx_here) {
    std::string nm = "c_";
    for (const char* q = spec; *q; ++q) {
      if (*q == ',') {
        nm += '_';
      } else if (q[0] == '-' && q[1] == '>') {
        nm += '2';
        ++q;
      } else {
        nm += *q;
      }
    }
    nvtxRangePushA(nm.c_str());
  }
  // packed operand of the tensor-core paths: from the cache, stored in it
  // (constant tensors during the cache fill), or packed into the arena
  auto operand = [&](const char* role, const Tensor& T, const Packed* cached, int64_t bytes0,
                     int64_t bytes1, bool is_a, const GemmDesc& gd) -> Packed {
    if (cached) return *cached;
    Packed pk;
    const bool held = (&T == &A && holdA) || (&T == &B && holdB);
    const std::string ck =
        held ? hkey(role, T, &T == &A) : (T.constant ? key(role, T) : std::string());
    const int64_t bytes = bytes0 + bytes1;
    const bool keep = T.constant && (!tc_cache_select || tc_cache_allowed.count(ck) ||
                                      (!tc_cache_cands.count(ck) && bytes <= (int64_t(1) << 28)));
    if (dry && T.constant) {
      CacheCand& cc = tc_cache_cands[ck];
      cc.bytes = bytes;
      cc.tensor = T.p;
      if (plan_cached && keep) return Packed{};  // held by the cache
    }
    const bool store = keep && tc_cache_fill && !dry && persistent_alloc;
    if (pack_only && !store && !held) return pk;  // a pack made ahead is only worth keeping
    if (held) {
      pk = &T == &A ? heldA : heldB;
    } else if (store) {
      pk.p0 = persistent_alloc(bytes0);
      pk.p1 = persistent_alloc(bytes1);
    } else {
      pk.p0 = arena.alloc((bytes0 + 7) / 8);
      pk.p1 = arena.alloc((bytes1 + 7) / 8);
    }
    launch(kPermute, 0.0,
           [&] {
             if (use_tc) {
               float* hi = static_cast<float*>(pk.p0);
               float* lo = static_cast<float*>(pk.p1);
               if (is_a)
                 gemm_tc_pack_a(gd, hi, lo, stream);
               else
                 gemm_tc_pack_b(gd, hi, lo, stream);
             } else {
               uint16_t* planes = static_cast<uint16_t*>(pk.p0);
               int* expo = static_cast<int*>(pk.p1);
               if (is_a)
                 gemm_oz_pack_a(gd, oz_planes, planes, expo, stream);
               else
                 gemm_oz_pack_b(gd, oz_planes, planes, expo, stream);
             }
           },
           trace_on() ? std::string(use_tc ? "tc pack " : "oz pack ") + role + " " + spec
                      : std::string());
    if (store) {
      tc_cache_[ck] = pk;
      tc_cached_.insert(T.p);
    }
    if (held) held_packs_[ck] = pk;
    return pk;
  };
  // Complex x complex on the tensor cores as three real products (3M)
  // instead of the four of the real embedding, for operands packed per call.
  // It writes three partial products and combines them, so it pays only when
  // the saved quarter of the MMA work outweighs that pass over the output:
  // from about 2000 of K on (per output element, 0.25 * 8 K products against
  // about 40 bytes of partials and output).
  const bool use3m = packed_path && allow_3m && A.cplx && B.cplx && Bt == 1 && !pack_only &&
                     Kt >= kMin3mK &&
                     !cA && !cB && !A.constant && !B.constant && !holdA && !holdB &&
                     !held_.count(A.p) && !held_.count(B.p);
  if (use3m) {
    const GemmDesc d3 = use_oz && swap ? swapped(g) : g;
    const GemmDesc r = gemm_3m_desc(d3);
    const double flops3 = 0.75 * flops;  // three real products instead of four
    if (use_tc) {
      const TcLayout L = gemm_tc_layout(r);
      const int64_t sa = L.a_elems / 3, sb = L.b_elems / 3;
      float* ahi = reinterpret_cast<float*>(arena.alloc((4 * L.a_elems + 7) / 8));
      float* alo = reinterpret_cast<float*>(arena.alloc((4 * L.a_elems + 7) / 8));
      float* bhi = reinterpret_cast<float*>(arena.alloc((4 * L.b_elems + 7) / 8));
      float* blo = reinterpret_cast<float*>(arena.alloc((4 * L.b_elems + 7) / 8));
      float2* P = reinterpret_cast<float2*>(arena.alloc(L.p_elems));
      for (int k = 0; k < 3; ++k) {
        GemmDesc pk = d3;
        pk.part_a = pk.part_b = k;
        launch(kPermute, 0.0,
               [&] {
                 gemm_tc_pack_a(pk, ahi + k * sa, alo + k * sa, stream);
                 gemm_tc_pack_b(pk, bhi + k * sb, blo + k * sb, stream);
               },
               trace_on() ? std::string("tc pack 3M ") + spec : std::string());
      }
      launch(cls, flops3,
             [&] { gemm_tc_mma(r, ahi, alo, bhi, blo, P, tc_err, stream); }, label + " 3M",
             8.0 * (double)(L.a_elems + L.b_elems) + 8.0 * (double)L.p_elems);
      launch(kElementwise, 0.0, [&] { gemm_tc_combine_3m(d3, P, stream); }, "tc combine 3M");
    } else {
      const OzLayout L = gemm_oz_layout(r, oz_planes);
      uint16_t* ap = reinterpret_cast<uint16_t*>(arena.alloc((2 * L.planes * L.a_elems + 7) / 8));
      int* ae = reinterpret_cast<int*>(arena.alloc((4 * L.a_rows + 7) / 8));
      uint16_t* bp = reinterpret_cast<uint16_t*>(arena.alloc((2 * L.planes * L.b_elems + 7) / 8));
      int* be = reinterpret_cast<int*>(arena.alloc((4 * L.b_rows + 7) / 8));
      float2* P = reinterpret_cast<float2*>(arena.alloc(L.p_elems));
      for (int k = 0; k < 3; ++k) {
        GemmDesc pk = d3;
        pk.part_a = pk.part_b = k;
        launch(kPermute, 0.0,
               [&] {
                 gemm_oz_pack_a(pk, oz_planes, ap, ae, stream, k, 3);
                 gemm_oz_pack_b(pk, oz_planes, bp, be, stream, k, 3);
               },
               trace_on() ? std::string("oz pack 3M ") + spec : std::string());
      }
      launch(cls, flops3,
             [&] { gemm_oz_mma(r, oz_planes, ap, ae, bp, be, P, tc_err, stream); }, label + " 3M",
             2.0 * L.planes * (double)(L.a_elems + L.b_elems) + 8.0 * (double)L.p_elems);
      launch(kElementwise, 0.0, [&] { gemm_oz_combine_3m(d3, oz_planes, ae, be, P, stream); },
             "oz combine 3M");
    }
  } else if (!packed_path) {
    const int64_t w = gemm_f64_workspace(g);
    if (w) g.work = arena.alloc(w);
    // operands read once, output written (or slabs written and read back)
    const double bytes = 8.0 * ((A.cplx ? 2 : 1) * (double)Mt * Kt * Bt +
                                (B.cplx ? 2 : 1) * (double)Kt * Nt * Bt +
                                (C.cplx ? 2 : 1) * (double)Mt * Nt * Bt * (beta != 0.0 ? 2 : 1)) +
                         16.0 * (double)w;
    launch(cls, flops, [&] { gemm_f64(g, stream); }, label, bytes);
  } else if (use_tc) {
    const TcLayout L = gemm_tc_layout(g);
    if (pack_only) {
      if ((A.constant || holdA) && !cA)
        operand("A", A, cA, 4 * L.a_elems, 4 * L.a_elems, true, g);
      if ((B.constant || holdB) && !cB)
        operand("B", B, cB, 4 * L.b_elems, 4 * L.b_elems, false, g);
      arena.release(mark);
      return;
    }
    const Packed pa = operand("A", A, cA, 4 * L.a_elems, 4 * L.a_elems, true, g);
    const Packed pb = operand("B", B, cB, 4 * L.b_elems, 4 * L.b_elems, false, g);
    float2* P = L.p_elems ? reinterpret_cast<float2*>(arena.alloc(L.p_elems)) : nullptr;
    // packed hi/lo operands read once; partial pairs written (and read back
    // by the finalize) or the output written directly
    const double bytes = 8.0 * (double)(L.a_elems + L.b_elems) + 8.0 * (double)L.p_elems +
                         (L.ranges == 1 ? (C.cplx ? 16.0 : 8.0) * (double)Mt * Nt * Bt : 0.0);
    launch(cls, flops,
           [&] {
             gemm_tc_mma(g, static_cast<float*>(pa.p0), static_cast<float*>(pa.p1),
                         static_cast<float*>(pb.p0), static_cast<float*>(pb.p1), P, tc_err, stream);
           },
           label, bytes);
    if (L.ranges > 1)
      launch(kElementwise, 0.0, [&] { gemm_tc_finalize(g, P, stream); }, "tc finalize");
  } else {
    const GemmDesc go = swap ? swapped(g) : g;
    const OzLayout L = gemm_oz_layout(go, oz_planes);
    if (pack_only) {
      const int64_t abytes = 2 * L.planes * L.a_elems, arow = 4 * L.a_rows;
      const int64_t bbytes = 2 * L.planes * L.b_elems, brow = 4 * L.b_rows;
      if ((A.constant || holdA) && !cA)
        operand(roleA, A, cA, swap ? bbytes : abytes, swap ? brow : arow, !swap, go);
      if ((B.constant || holdB) && !cB)
        operand(roleB, B, cB, swap ? abytes : bbytes, swap ? arow : brow, swap, go);
      arena.release(mark);
      return;
    }
    const Packed pa = swap ? operand(roleB, B, cB, 2 * L.planes * L.a_elems, 4 * L.a_rows, true, go)
                           : operand(roleA, A, cA, 2 * L.planes * L.a_elems, 4 * L.a_rows, true, go);
    const Packed pb = swap ? operand(roleA, A, cA, 2 * L.planes * L.b_elems, 4 * L.b_rows, false, go)
                           : operand(roleB, B, cB, 2 * L.planes * L.b_elems, 4 * L.b_rows, false, go);
    if (grouped) {  // recorded for the caller's grouped launch; the packs stay
      if (L.p_elems || outcopy)
        throw Error(-1, std::string("contract: a grouped ladder needs one K range and its "
                                    "output in GEMM layout: ") + spec);
      if (!dry) {
        OzGroupGemm gg;
        gg.d = go;
        gg.A = static_cast<const uint16_t*>(pa.p0);
        gg.ea = static_cast<const int*>(pa.p1);
        gg.B = static_cast<const uint16_t*>(pb.p0);
        gg.eb = static_cast<const int*>(pb.p1);
        gg.err = tc_err;
        deferred.push_back({gg, flops});
      }
      if (nvtx_here) nvtxRangePop();
      if (!dry) nvtxRangePop();  // rteom_ladder
      return;
    }
    float2* P = L.p_elems ? reinterpret_cast<float2*>(arena.alloc(L.p_elems)) : nullptr;
    // digit planes read once; partial pairs written or the output written
    const double bytes = 2.0 * L.planes * (double)(L.a_elems + L.b_elems) +
                         8.0 * (double)L.p_elems +
                         (L.ranges == 1 ? (C.cplx ? 16.0 : 8.0) * (double)Mt * Nt * Bt : 0.0);
    // counted as the FP64 GEMM it replaces (the tensor cores execute 28 times
    // as many BF16 FLOPs, one product per digit pair)
    launch(cls, flops,
           [&] {
             gemm_oz_mma(go, oz_planes, static_cast<uint16_t*>(pa.p0), static_cast<int*>(pa.p1),
                         static_cast<uint16_t*>(pb.p0), static_cast<int*>(pb.p1), P, tc_err,
                         stream);
           },
           label, bytes);
    if (L.ranges > 1)
      launch(kElementwise, 0.0,
             [&] {
               gemm_oz_finalize(go, oz_planes, static_cast<int*>(pa.p1), static_cast<int*>(pb.p1), P,
                                stream);
             },
             "oz finalize");
  }
  if (outcopy) axpy((batch + bM + bN + "->" + p.c).c_str(), 1.0, Cuse, beta, C);
  if (nvtx_here) nvtxRangePop();
  if (cls == kLadder && !dry) nvtxRangePop();
  if (dry && std::getenv("RTEOM_PLAN_TRACE"))  // scratch planning: arena top inside this call
    std::fprintf(stderr,
                 "plan %-22s M=%lld N=%lld K=%lld %s perm %c%c%c in %.3f GB arena %.3f GB (peak "
                 "%.3f GB)\n",
                 spec, (long long)Mt, (long long)Nt, (long long)Kt, use_tc ? "tc" : "f64",
                 bPA ? 'A' : '-', bPB ? 'B' : '-', bPC ? 'C' : '-', mark * 8e-9,
                 arena.mark() * 8e-9, arena.peak_bytes() * 1e-9);
  arena.release(mark);
}

}  // namespace rteom
