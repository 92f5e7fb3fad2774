// Allocation-free variant of the closed-shell correlation-energy reduction.
//
// rteom_ecorr_noalloc computes the same E_N^corr that rteom_create stores,
//   E = sum_ijab [2(ia|jb) - (ib|ja)] (t_ij^ab + t_i^a t_j^b),
// from caller-owned device buffers, without allocating device memory.  It is
// meant for callers that may not allocate: an application whose device memory
// is entirely owned by its own pool or framework allocator, or code that runs
// where a cudaMalloc/cudaFree would have to synchronise the device or is
// forbidden by the host program.
//
// Its scratch (one partial sum per occupied pair (i,j)) lives in the
// file-scope array below instead of being allocated per call.  Every GPU that
// loads this library keeps that array (32 KiB) until the process exits.  All
// calls share it, so calls whose kernels overlap on the GPU (different
// streams, or different host threads on one device) race on it; serialise
// them.  Each call overwrites every partial it later reads, so nothing has to
// start at zero.
//
// Cost: the pair kernel forms (ia|jb) and (ib|ja) from the Cholesky vectors
// for every (i,j,a,b), 2 O^2 V^2 Nchol FP64 FMAs (about 1.8e12 at O=50, V=450,
// Nchol=1800, minutes on the FP64 pipe), against the O^2 V^2 of rteom_create,
// which reads its stored (ov|ov) block.  It suits the small ground-state
// problems this entry point is meant for.
#include <cuda.h>

#include <cstdio>
#include <string>

#include "../../include/rteom.h"
#include "common.cuh"
#include "scratch_cache.h"

namespace {

constexpr int kMaxPairs = 4096;  // occupied pairs (i,j): nocc <= 64
constexpr int kThreads = 256;

static __device__ __align__(256) double g_ecorr_pairs[kMaxPairs];

// One block per occupied pair (i,j): partial[i*O+j] = sum_ab [2(ia|jb) -
// (ib|ja)] (t2_ijab + t1_ia t1_jb), with (pq|rs) = sum_Q L_pq L_rs.
__global__ void ecorr_pairs_kernel(const double* __restrict__ L, int nchol, int O, int V,
                                   const double* __restrict__ t1, const double* __restrict__ t2,
                                   double* __restrict__ partial) {
  __shared__ double sh[kThreads];
  const int nb = O + V;
  const int i = blockIdx.x / O, j = blockIdx.x % O;
  const int64_t nn = (int64_t)nb * nb;
  double acc = 0.0;
  for (int ab = threadIdx.x; ab < V * V; ab += blockDim.x) {
    const int a = ab / V, b = ab % V;
    double iajb = 0.0, ibja = 0.0;
    for (int Q = 0; Q < nchol; ++Q) {
      const double* LQ = L + Q * nn;
      iajb = fma(LQ[(int64_t)i * nb + O + a], LQ[(int64_t)j * nb + O + b], iajb);
      ibja = fma(LQ[(int64_t)i * nb + O + b], LQ[(int64_t)j * nb + O + a], ibja);
    }
    double tt = (t2 ? t2[(((int64_t)i * O + j) * V + a) * V + b] : 0.0) +
                (t1 ? t1[i * V + a] * t1[j * V + b] : 0.0);
    acc = fma(2.0 * iajb - ibja, tt, acc);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// Sum the pair partials in a fixed order into *out.
__global__ void ecorr_sum_kernel(const double* __restrict__ partial, int n, double* out) {
  __shared__ double sh[kThreads];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partial[k];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// Copy a message into the caller's buffer (if any) and return the code.
int report(int code, const std::string& msg, char* err, int err_len) {
  if (err && err_len > 0) std::snprintf(err, (size_t)err_len, "%s", msg.c_str());
  return code;
}

// Driver entry points for the id of the current context, fetched once
// through the runtime (the library does not link the driver library).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
struct CtxIdApi {
  CtxGetCurrentFn get_current = nullptr;
  CtxGetIdFn get_id = nullptr;
};

const CtxIdApi& ctx_id_api() {
  static const CtxIdApi api = [] {
    CtxIdApi a;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      a.get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      a.get_id = reinterpret_cast<CtxGetIdFn>(f);
    return a;
  }();
  return api;
}

// Id of the context current on this thread; false when there is none yet
// (the runtime makes the device's primary context current on its first use)
// or the entry points are unavailable.
bool current_ctx_id(unsigned long long* id) {
  const CtxIdApi& api = ctx_id_api();
  if (!api.get_current || !api.get_id) return false;
  CUcontext ctx = nullptr;
  if (api.get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
  return api.get_id(ctx, id) == CUDA_SUCCESS;
}

rteom::ContextAddressCache g_pairs_cache;

// Device address of the scratch array in the current context: looked up with
// cudaGetSymbolAddress (with the caller's device current) the first time a
// context uses this entry point, then taken from the per-context cache.
int pairs_scratch(double** out, char* err, int err_len) {
  auto lookup = [](void** addr) -> int {
    const cudaError_t e = cudaGetSymbolAddress(addr, g_ecorr_pairs);
    return (e == cudaSuccess && *addr != nullptr) ? 0 : (int)e + 1;
  };
  auto failed = [&](int rc) {
    return report(RTEOM_ERR_CUDA,
                  std::string("cudaGetSymbolAddress(scratch): ") +
                      cudaGetErrorString(static_cast<cudaError_t>(rc - 1)),
                  err, err_len);
  };
  unsigned long long id = 0;
  void* p = nullptr;
  if (!current_ctx_id(&id)) {
    // no current context yet: this lookup creates the primary context; the
    // address is cached under its id when the id can be read
    const int rc = lookup(&p);
    if (rc != 0) return failed(rc);
    if (current_ctx_id(&id)) {
      const int rc2 = g_pairs_cache.get(id, lookup, &p);
      if (rc2 != 0) return failed(rc2);
    }
  } else {
    const int rc = g_pairs_cache.get(id, lookup, &p);
    if (rc != 0) return failed(rc);
  }
  *out = static_cast<double*>(p);
  return RTEOM_OK;
}

}  // namespace

extern "C" int rteom_ecorr_noalloc(int nocc, int nvir, int nchol, const double* L,
                                   const double* t1_gs, const double* t2_gs, double* e_corr,
                                   void* cuda_stream, char* err, int err_len) {
  if (err && err_len > 0) err[0] = '\0';
  if (nocc < 1 || nvir < 1 || nchol < 0)
    return report(RTEOM_ERR_ARG, "need nocc >= 1, nvir >= 1, nchol >= 0", err, err_len);
  if ((nchol > 0 && !L) || !e_corr)
    return report(RTEOM_ERR_ARG, "L (when nchol > 0) and e_corr must be device pointers", err,
                  err_len);
  if ((long long)nocc * nocc > kMaxPairs)
    return report(RTEOM_ERR_ARG,
                  "nocc*nocc = " + std::to_string((long long)nocc * nocc) + " exceeds the " +
                      std::to_string(kMaxPairs) +
                      " occupied pairs the static scratch holds (nocc <= 64)",
                  err, err_len);
  if ((double)nvir * nvir > 2.0e9)
    return report(RTEOM_ERR_ARG, "nvir*nvir exceeds the 32-bit pair index", err, err_len);
  double* scratch = nullptr;
  int rc = pairs_scratch(&scratch, err, err_len);
  if (rc != RTEOM_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int pairs = nocc * nocc;
  // cudaLaunchKernel returns the error of this launch itself, so an earlier,
  // unrelated error of the calling thread is neither reported nor cleared
  void* pair_args[] = {(void*)&L,      (void*)&nchol, (void*)&nocc,  (void*)&nvir,
                       (void*)&t1_gs, (void*)&t2_gs, (void*)&scratch};
  cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void*>(&ecorr_pairs_kernel),
                                   dim3(pairs), dim3(kThreads), pair_args, 0, st);
  if (e == cudaSuccess) {
    void* sum_args[] = {(void*)&scratch, (void*)&pairs, (void*)&e_corr};
    e = cudaLaunchKernel(reinterpret_cast<const void*>(&ecorr_sum_kernel), dim3(1),
                         dim3(kThreads), sum_args, 0, st);
  }
  if (e != cudaSuccess)
    return report(RTEOM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e), err,
                  err_len);
  return RTEOM_OK;
}
