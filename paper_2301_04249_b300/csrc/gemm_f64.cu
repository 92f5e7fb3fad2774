// FP64 batched GEMM for the contraction engine.
//
//   C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b]
//
// A and B are each real (FP64) or complex (complex128, interleaved); C is
// complex when either operand is.  op(A) is [M][K] read from A stored
// [M][K] (lda) or, transposed, [K][M]; likewise op(B) is [K][N] from [K][N]
// or [N][K].  alpha and beta are real.  On B300 the FP64 pipe issues about
// two DFMA per clock per SM, so the kernel only has to keep that pipe busy
// and waste no lanes: an output tile of BM x BN per 256-thread block (64x64,
// 32x64, 16x64, 8x128, 64x16 or 16x16, picked so that thin outputs do not
// compute padding), 8-deep K slices staged in shared memory, each thread
// accumulating a TM x TN sub-tile in registers; long K with few output tiles
// is split into slices whose partial products are summed in slice order.
// Bounds are checked on every load and store.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rteom {

namespace {

struct GemmArgs {
  int M, N, K;
  int kslice;  // K range per split (split-K), or K
  int splits;  // K slices per batch entry (1 = no split)
  const double* A;
  int64_t lda, sA;
  int transA;
  const double* B;
  int64_t ldb, sB;
  int transB;
  double* C;
  int64_t ldc, sC;
  double alpha, beta;
};

template <bool CP>
struct Val;
template <>
struct Val<false> {
  double x;
};
template <>
struct Val<true> {
  double x, y;
};

template <bool CP>
__device__ __forceinline__ Val<CP> load_val(const double* base, int64_t idx, bool ok) {
  Val<CP> v;
  if constexpr (CP) {
    if (ok) {
      double2 d = *reinterpret_cast<const double2*>(base + 2 * idx);
      v.x = d.x;
      v.y = d.y;
    } else {
      v.x = 0.0;
      v.y = 0.0;
    }
  } else {
    v.x = ok ? base[idx] : 0.0;
  }
  return v;
}

constexpr int BK = 8;

template <bool AC, bool BC, int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(256) gemm_kernel(GemmArgs g) {
  constexpr bool CC = AC || BC;
  constexpr int RM = BM / TM;  // thread rows; thread (tx, ty) owns rows ty + RM*i
  constexpr int RN = BN / TN;  // thread cols; and cols tx + RN*j
  static_assert(RM * RN == 256, "tile must map onto 256 threads");
  __shared__ Val<AC> As[BK][BM];
  __shared__ Val<BC> Bs[BK][BN];

  // blockIdx.z = batch * splits + split; a split covers K range
  // [split*kslice, min(K, (split+1)*kslice)) and, when splits > 1, writes its
  // partial product to its own slab of the output (the workspace).
  const int b = blockIdx.z / g.splits;
  const int sp = blockIdx.z % g.splits;
  const double* A = g.A + (AC ? 2 : 1) * g.sA * b;
  const double* B = g.B + (BC ? 2 : 1) * g.sB * b;
  double* C = g.C + (CC ? 2 : 1) * g.sC * blockIdx.z;
  const int kbeg = sp * g.kslice;
  const int kend = min(g.K, kbeg + g.kslice);
  const int m0 = blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  const int tx = threadIdx.x % RN, ty = threadIdx.x / RN;

  double acc_r[TM][TN], acc_i[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc_r[i][j] = acc_i[i][j] = 0.0;

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    // stage A slice: BM x BK elements
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int mm, kk;
      if (g.transA) {  // stored [K][M]: consecutive threads walk m
        mm = e % BM;
        kk = e / BM;
      } else {  // stored [M][K]: consecutive threads walk k
        kk = e % BK;
        mm = e / BK;
      }
      int m = m0 + mm, k = k0 + kk;
      bool ok = (m < g.M) && (k < kend);
      int64_t idx = g.transA ? (int64_t)k * g.lda + m : (int64_t)m * g.lda + k;
      As[kk][mm] = load_val<AC>(A, ok ? idx : 0, ok);
    }
    for (int e = threadIdx.x; e < BN * BK; e += 256) {
      int nn, kk;
      if (g.transB) {  // stored [N][K]
        kk = e % BK;
        nn = e / BK;
      } else {  // stored [K][N]
        nn = e % BN;
        kk = e / BN;
      }
      int n = n0 + nn, k = k0 + kk;
      bool ok = (n < g.N) && (k < kend);
      int64_t idx = g.transB ? (int64_t)n * g.ldb + k : (int64_t)k * g.ldb + n;
      Bs[kk][nn] = load_val<BC>(B, ok ? idx : 0, ok);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Val<AC> a[TM];
      Val<BC> bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + RM * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + RN * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          if constexpr (AC && BC) {
            acc_r[i][j] = fma(a[i].x, bv[j].x, acc_r[i][j]);
            acc_r[i][j] = fma(-a[i].y, bv[j].y, acc_r[i][j]);
            acc_i[i][j] = fma(a[i].x, bv[j].y, acc_i[i][j]);
            acc_i[i][j] = fma(a[i].y, bv[j].x, acc_i[i][j]);
          } else if constexpr (AC) {
            acc_r[i][j] = fma(a[i].x, bv[j].x, acc_r[i][j]);
            acc_i[i][j] = fma(a[i].y, bv[j].x, acc_i[i][j]);
          } else if constexpr (BC) {
            acc_r[i][j] = fma(a[i].x, bv[j].x, acc_r[i][j]);
            acc_i[i][j] = fma(a[i].x, bv[j].y, acc_i[i][j]);
          } else {
            acc_r[i][j] = fma(a[i].x, bv[j].x, acc_r[i][j]);
          }
        }
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int m = m0 + ty + RM * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int n = n0 + tx + RN * j;
      if (n >= g.N) continue;
      int64_t o = (int64_t)m * g.ldc + n;
      if constexpr (CC) {
        double2* cp = reinterpret_cast<double2*>(C + 2 * o);
        double2 r;
        if (g.beta == 0.0) {
          r.x = g.alpha * acc_r[i][j];
          r.y = g.alpha * acc_i[i][j];
        } else {
          double2 c0 = *cp;
          r.x = fma(g.beta, c0.x, g.alpha * acc_r[i][j]);
          r.y = fma(g.beta, c0.y, g.alpha * acc_i[i][j]);
        }
        *cp = r;
      } else {
        double r = g.alpha * acc_r[i][j];
        if (g.beta != 0.0) r = fma(g.beta, C[o], r);
        C[o] = r;
      }
    }
  }
}

// C[b] = beta * C[b] + sum_{s < splits} P[b * splits + s], summed in slice
// order (deterministic).  P slabs are [M][N] with row stride N.
template <bool CC>
__global__ void splitk_reduce(const double* __restrict__ P, double* C, int M, int N, int64_t ldc,
                              int64_t sC, int splits, int batch, double beta) {
  const int64_t per = (int64_t)M * N;
  const int w = CC ? 2 : 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * batch;
       e += (int64_t)gridDim.x * blockDim.x) {
    int b = (int)(e / per);
    int64_t r = e - (int64_t)b * per;
    int m = (int)(r / N), n = (int)(r % N);
    double sx = 0.0, sy = 0.0;
    for (int s = 0; s < splits; ++s) {
      const double* q = P + w * (((int64_t)b * splits + s) * per + r);
      sx += q[0];
      if (CC) sy += q[1];
    }
    double* c = C + w * ((int64_t)b * sC + (int64_t)m * ldc + n);
    if (beta == 0.0) {
      c[0] = sx;
      if (CC) c[1] = sy;
    } else {
      c[0] = fma(beta, c[0], sx);
      if (CC) c[1] = fma(beta, c[1], sy);
    }
  }
}

// Output tile shapes, chosen from the output's extents.
struct Tile {
  int bm, bn;
};

Tile pick_tile(int M, int N) {
  if (M <= 8 && N > 16) return {8, 128};
  if (M <= 16 && N <= 16) return {16, 16};
  if (M <= 16) return {16, 64};
  if (N <= 16) return {64, 16};
  if (M <= 32) return {32, 64};
  return {64, 64};
}

template <bool AC, bool BC>
void launch_typed(const GemmArgs& g, int batch, int splits, cudaStream_t st) {
  const Tile t = pick_tile(g.M, g.N);
  dim3 grid((g.N + t.bn - 1) / t.bn, (g.M + t.bm - 1) / t.bm, batch * splits);
  if (t.bm == 64 && t.bn == 64)
    gemm_kernel<AC, BC, 64, 64, 4, 4><<<grid, 256, 0, st>>>(g);
  else if (t.bm == 32)
    gemm_kernel<AC, BC, 32, 64, 2, 4><<<grid, 256, 0, st>>>(g);
  else if (t.bm == 16 && t.bn == 64)
    gemm_kernel<AC, BC, 16, 64, 1, 4><<<grid, 256, 0, st>>>(g);
  else if (t.bm == 8)
    gemm_kernel<AC, BC, 8, 128, 1, 4><<<grid, 256, 0, st>>>(g);
  else if (t.bn == 16 && t.bm == 64)
    gemm_kernel<AC, BC, 64, 16, 4, 1><<<grid, 256, 0, st>>>(g);
  else
    gemm_kernel<AC, BC, 16, 16, 1, 1><<<grid, 256, 0, st>>>(g);
}

}  // namespace

int gemm_f64_splits(const GemmDesc& d) {
  // Split K when the output alone gives too few blocks to balance 148 SMs
  // (the FP64 pipe is the bottleneck, so only the block count matters); each
  // slice keeps at least 128 of K.
  if (d.M <= 0 || d.N <= 0 || d.K < 256) return 1;
  const Tile t = pick_tile(d.M, d.N);
  int64_t tiles = (int64_t)((d.N + t.bn - 1) / t.bn) * ((d.M + t.bm - 1) / t.bm) * d.batch;
  const int64_t target = 8 * 148;
  if (tiles >= target) return 1;
  int64_t s = (target + tiles - 1) / tiles;
  s = std::min<int64_t>(s, d.K / 128);
  s = std::min<int64_t>(s, 1024);
  if ((int64_t)d.batch * s > 65535) s = 65535 / d.batch;
  return (int)std::max<int64_t>(s, 1);
}

int64_t gemm_f64_workspace(const GemmDesc& d) {
  int s = gemm_f64_splits(d);
  if (s <= 1) return 0;
  return (int64_t)s * d.batch * d.M * d.N * ((d.Acplx || d.Bcplx) ? 2 : 1);
}

void gemm_f64(const GemmDesc& d, cudaStream_t st) {
  if (d.M <= 0 || d.N <= 0 || d.batch <= 0) return;
  if ((d.M + 7) / 8 > 65535 || d.batch > 65535)
    throw Error(-1, "gemm_f64: grid too large");
  const int splits = gemm_f64_splits(d);
  if (splits > 1 && d.work == nullptr) throw Error(-1, "gemm_f64: split-K needs a workspace");
  GemmArgs g;
  g.M = d.M;
  g.N = d.N;
  g.K = d.K;
  g.kslice = splits > 1 ? (d.K + splits - 1) / splits : std::max(d.K, 1);
  g.splits = splits;
  g.A = d.A;
  g.lda = d.lda;
  g.sA = d.strideA;
  g.transA = d.transA;
  g.B = d.B;
  g.ldb = d.ldb;
  g.sB = d.strideB;
  g.transB = d.transB;
  g.alpha = d.alpha;
  if (splits > 1) {  // slices write their own [M][N] slabs; reduce afterwards
    g.C = d.work;
    g.ldc = d.N;
    g.sC = (int64_t)d.M * d.N;
    g.beta = 0.0;
  } else {
    g.C = d.C;
    g.ldc = d.ldc;
    g.sC = d.strideC;
    g.beta = d.beta;
  }
  if (d.Acplx && d.Bcplx)
    launch_typed<true, true>(g, d.batch, splits, st);
  else if (d.Acplx)
    launch_typed<true, false>(g, d.batch, splits, st);
  else if (d.Bcplx)
    launch_typed<false, true>(g, d.batch, splits, st);
  else
    launch_typed<false, false>(g, d.batch, splits, st);
  RT_CHECK_LAUNCH();
  if (splits > 1) {
    const bool cc = d.Acplx || d.Bcplx;
    int64_t n = (int64_t)d.M * d.N * d.batch;
    int grid = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    if (cc)
      splitk_reduce<true><<<grid, 256, 0, st>>>(d.work, d.C, d.M, d.N, d.ldc, d.strideC, splits,
                                                d.batch, d.beta);
    else
      splitk_reduce<false><<<grid, 256, 0, st>>>(d.work, d.C, d.M, d.N, d.ldc, d.strideC, splits,
                                                 d.batch, d.beta);
    RT_CHECK_LAUNCH();
  }
}

}  // namespace rteom
