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
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/rteom.h"
#include "common.cuh"

namespace {

constexpr int kMaxPairs = 4096;  // occupied pairs (i,j): nocc <= 64
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_ecorr_pairs[kMaxPairs];

std::mutex g_setup_mutex;
double* g_pairs_ptr[kMaxDevices] = {nullptr};

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

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
int pairs_scratch(double** out, char* err, int err_len) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return report(RTEOM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e), err,
                  err_len);
  if (dev < 0 || dev >= kMaxDevices)
    return report(RTEOM_ERR_ARG, "device ordinal beyond the supported 64 devices", err, err_len);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_pairs_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_ecorr_pairs);
    if (e != cudaSuccess || p == nullptr)
      return report(RTEOM_ERR_CUDA,
                    std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e), err,
                    err_len);
    g_pairs_ptr[dev] = p;
  }
  *out = g_pairs_ptr[dev];
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
  const int pairs = nocc * nocc;
  ecorr_pairs_kernel<<<pairs, kThreads, 0, st>>>(L, nchol, nocc, nvir, t1_gs, t2_gs, scratch);
  ecorr_sum_kernel<<<1, kThreads, 0, st>>>(scratch, pairs, e_corr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return report(RTEOM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e), err,
                  err_len);
  return RTEOM_OK;
}
