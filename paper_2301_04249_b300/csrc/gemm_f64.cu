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

#include <type_traits>

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
  int ntn;  // column tiles: blockIdx.x = row tile * ntn + column tile
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

// Complex operand staged for the three-multiplication complex product
// (Gauss's trick, error analysis in Higham, SIAM J. Matrix Anal. Appl. 13,
// 1992): re, im and re + im.
struct Val3 {
  double x, y, s;
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
  // complex x complex: three real products per complex multiply-add,
  // p1 = Re a Re b, p2 = Im a Im b, p3 = (Re a + Im a)(Re b + Im b);
  // Re = p1 - p2, Im = p3 - p1 - p2
  constexpr bool M3 = AC && BC;
  using SA = typename std::conditional<M3, Val3, Val<AC>>::type;
  using SB = typename std::conditional<M3, Val3, Val<BC>>::type;
  constexpr int RM = BM / TM;  // thread rows; thread (tx, ty) owns rows ty + RM*i
  constexpr int RN = BN / TN;  // thread cols; and cols tx + RN*j
  static_assert(RM * RN == 256, "tile must map onto 256 threads");
  __shared__ SA As[BK][BM];
  __shared__ SB Bs[BK][BN];

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
  const int m0 = (int)(blockIdx.x / g.ntn) * BM;
  const int n0 = (int)(blockIdx.x % g.ntn) * BN;
  const int tx = threadIdx.x % RN, ty = threadIdx.x / RN;

  double acc_r[TM][TN], acc_i[TM][TN], acc_s[M3 ? TM : 1][M3 ? TN : 1];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc_r[i][j] = acc_i[i][j] = 0.0;
  if constexpr (M3) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc_s[i][j] = 0.0;
  }

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
      const Val<AC> v = load_val<AC>(A, ok ? idx : 0, ok);
      if constexpr (M3)
        As[kk][mm] = Val3{v.x, v.y, v.x + v.y};
      else
        As[kk][mm] = v;
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
      const Val<BC> v = load_val<BC>(B, ok ? idx : 0, ok);
      if constexpr (M3)
        Bs[kk][nn] = Val3{v.x, v.y, v.x + v.y};
      else
        Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      SA a[TM];
      SB bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + RM * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + RN * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          if constexpr (M3) {
            acc_r[i][j] = fma(a[i].x, bv[j].x, acc_r[i][j]);
            acc_i[i][j] = fma(a[i].y, bv[j].y, acc_i[i][j]);
            acc_s[i][j] = fma(a[i].s, bv[j].s, acc_s[i][j]);
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

  if constexpr (M3) {  // p1, p2, p3 -> Re, Im
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const double p1 = acc_r[i][j], p2 = acc_i[i][j];
        acc_r[i][j] = p1 - p2;
        acc_i[i][j] = acc_s[i][j] - p1 - p2;
      }
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

// Output tile shapes: the table the autotuner walks, and the heuristic pick.
struct Tile {
  int bm, bn;
};

constexpr Tile kTiles[] = {{64, 64}, {32, 64}, {16, 64}, {8, 128},
                           {64, 16}, {16, 16}, {8, 32},  {32, 32}};
constexpr int kNumTiles = sizeof(kTiles) / sizeof(kTiles[0]);

Tile pick_tile(int M, int N) {
  if (M <= 8 && N > 16) return {8, 128};
  if (M <= 16 && N <= 16) return {16, 16};
  if (M <= 16) return {16, 64};
  if (N <= 16) return {64, 16};
  if (M <= 32) return {32, 64};
  return {64, 64};
}

Tile tile_of(const GemmDesc& d) {
  return d.tile >= 0 && d.tile < kNumTiles ? kTiles[d.tile] : pick_tile(d.M, d.N);
}

template <bool AC, bool BC>
void launch_typed(const GemmArgs& g, Tile t, int batch, int splits, cudaStream_t st) {
  dim3 grid(g.ntn * ((g.M + t.bm - 1) / t.bm), 1, batch * splits);
  if (t.bm == 64 && t.bn == 64)
    gemm_kernel<AC, BC, 64, 64, 4, 4><<<grid, 256, 0, st>>>(g);
  else if (t.bm == 32 && t.bn == 64)
    gemm_kernel<AC, BC, 32, 64, 2, 4><<<grid, 256, 0, st>>>(g);
  else if (t.bm == 16 && t.bn == 64)
    gemm_kernel<AC, BC, 16, 64, 1, 4><<<grid, 256, 0, st>>>(g);
  else if (t.bm == 8 && t.bn == 128)
    gemm_kernel<AC, BC, 8, 128, 1, 4><<<grid, 256, 0, st>>>(g);
  else if (t.bm == 64 && t.bn == 16)
    gemm_kernel<AC, BC, 64, 16, 4, 1><<<grid, 256, 0, st>>>(g);
  else if (t.bm == 8 && t.bn == 32)
    gemm_kernel<AC, BC, 8, 32, 1, 1><<<grid, 256, 0, st>>>(g);
  else if (t.bm == 32 && t.bn == 32)
    gemm_kernel<AC, BC, 32, 32, 2, 2><<<grid, 256, 0, st>>>(g);
  else
    gemm_kernel<AC, BC, 16, 16, 1, 1><<<grid, 256, 0, st>>>(g);
}

// ---- matrix-vector shapes (M == 1 or N == 1), deterministic
// Output j of the vector product y_j = sum_k x(k) * Mat(k, j).  When the
// output index is contiguous in Mat, one thread per output walks k (loads
// coalesced across threads); when k is contiguous, one warp per output
// strides k and reduces with a fixed shuffle tree.
template <bool XC, bool MC>
__device__ __forceinline__ void cmad(double& re, double& im, const double* x, int64_t xi,
                                     const double* m, int64_t mi) {
  const double xr = XC ? x[2 * xi] : x[xi], xim = XC ? x[2 * xi + 1] : 0.0;
  const double mr = MC ? m[2 * mi] : m[mi], mim = MC ? m[2 * mi + 1] : 0.0;
  re = fma(xr, mr, re);
  if (XC && MC) re = fma(-xim, mim, re);
  if (XC) im = fma(xim, mr, im);
  if (MC) im = fma(xr, mim, im);
}

struct GemvArgs {
  const double* x;  // vector, element k at x[k * sx]
  int64_t sx;
  const double* m;  // matrix, element (k, j) at m[k * sk + j * sj]
  int64_t sk, sj;
  double* y;        // output j at y[j * sy]
  int64_t sy;
  int n, K;         // outputs, reduction length
  double alpha, beta;
};

// Contiguous outputs: a block covers 32 outputs x 8 K-groups; group g sums
// k = g, g+8, ... and the 8 partials are added in group order.
template <bool XC, bool MC>
__global__ void __launch_bounds__(256) gemv_thread_kernel(GemvArgs a) {
  constexpr bool YC = XC || MC;
  __shared__ double sre[8][32], sim[8][32];
  const int lane = threadIdx.x % 32, grp = threadIdx.x / 32;
  const int j = blockIdx.x * 32 + lane;
  double re = 0.0, im = 0.0;
  if (j < a.n)
    for (int k = grp; k < a.K; k += 8)
      cmad<XC, MC>(re, im, a.x, k * a.sx, a.m, k * a.sk + j * a.sj);
  sre[grp][lane] = re;
  sim[grp][lane] = im;
  __syncthreads();
  if (grp == 0 && j < a.n) {
    re = 0.0;
    im = 0.0;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      re += sre[g][lane];
      im += sim[g][lane];
    }
    double* y = a.y + (YC ? 2 : 1) * (int64_t)j * a.sy;
    y[0] = a.beta == 0.0 ? a.alpha * re : fma(a.beta, y[0], a.alpha * re);
    if (YC) y[1] = a.beta == 0.0 ? a.alpha * im : fma(a.beta, y[1], a.alpha * im);
  }
}

template <bool XC, bool MC>
__global__ void gemv_warp_kernel(GemvArgs a) {
  constexpr bool YC = XC || MC;
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (j >= a.n) return;
  double re = 0.0, im = 0.0;
  for (int k = lane; k < a.K; k += 32)
    cmad<XC, MC>(re, im, a.x, k * a.sx, a.m, k * a.sk + j * a.sj);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    double* y = a.y + (YC ? 2 : 1) * (int64_t)j * a.sy;
    y[0] = a.beta == 0.0 ? a.alpha * re : fma(a.beta, y[0], a.alpha * re);
    if (YC) y[1] = a.beta == 0.0 ? a.alpha * im : fma(a.beta, y[1], a.alpha * im);
  }
}

template <bool XC, bool MC>
void launch_gemv(const GemvArgs& a, cudaStream_t st) {
  if (a.sj == 1) {
    gemv_thread_kernel<XC, MC><<<(a.n + 31) / 32, 256, 0, st>>>(a);
  } else {
    gemv_warp_kernel<XC, MC><<<(a.n + 7) / 8, 256, 0, st>>>(a);
  }
}

void gemv_f64(const GemmDesc& d, cudaStream_t st) {
  GemvArgs a;
  bool xc, mc;
  if (d.M == 1) {  // y[n] = sum_k A[0,k] B[k,n]
    a.x = d.A;
    a.sx = d.transA ? d.lda : 1;
    xc = d.Acplx;
    a.m = d.B;
    mc = d.Bcplx;
    a.sk = d.transB ? 1 : d.ldb;
    a.sj = d.transB ? d.ldb : 1;
    a.y = d.C;
    a.sy = 1;
    a.n = d.N;
  } else {  // N == 1: y[m] = sum_k A[m,k] B[k,0]
    a.x = d.B;
    a.sx = d.transB ? 1 : d.ldb;
    xc = d.Bcplx;
    a.m = d.A;
    mc = d.Acplx;
    a.sk = d.transA ? d.lda : 1;
    a.sj = d.transA ? 1 : d.lda;
    a.y = d.C;
    a.sy = d.ldc;
    a.n = d.M;
  }
  a.K = d.K;
  a.alpha = d.alpha;
  a.beta = d.beta;
  if (xc && mc)
    launch_gemv<true, true>(a, st);
  else if (xc)
    launch_gemv<true, false>(a, st);
  else if (mc)
    launch_gemv<false, true>(a, st);
  else
    launch_gemv<false, false>(a, st);
}

}  // namespace

int gemm_f64_tiles() { return kNumTiles; }

void gemm_f64_tile_shape(int t, int* bm, int* bn) {
  *bm = kTiles[t].bm;
  *bn = kTiles[t].bn;
}

bool gemm_f64_is_gemv(const GemmDesc& d) { return d.batch == 1 && (d.M == 1 || d.N == 1); }

int gemm_f64_splits(const GemmDesc& d) {
  if (gemm_f64_is_gemv(d)) return 1;  // matrix-vector path
  if (d.M <= 0 || d.N <= 0) return 1;
  if (d.splits > 0) {  // autotuner's choice, kept within K and the grid limit
    int64_t s = std::min<int64_t>(d.splits, std::max(d.K, 1));
    if ((int64_t)d.batch * s > 65535) s = 65535 / d.batch;
    return (int)std::max<int64_t>(s, 1);
  }
  // Split K when the output alone gives too few blocks to balance 148 SMs
  // (the FP64 pipe is the bottleneck, so only the block count matters); each
  // slice keeps at least 128 of K.
  if (d.K < 256) return 1;
  const Tile t = tile_of(d);
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
  if (d.batch > 65535) throw Error(-1, "gemm_f64: batch too large");
  if (d.transC) throw Error(-1, "gemm_f64: transposed output not supported");
  if (gemm_f64_is_gemv(d)) {
    gemv_f64(d, st);
    RT_CHECK_LAUNCH();
    return;
  }
  const int splits = gemm_f64_splits(d);
  if (splits > 1 && d.work == nullptr) throw Error(-1, "gemm_f64: split-K needs a workspace");
  if ((int64_t)((d.N + tile_of(d).bn - 1) / tile_of(d).bn) *
          ((d.M + tile_of(d).bm - 1) / tile_of(d).bm) > 0x7fffffff)
    throw Error(-1, "gemm_f64: too many tiles for the grid");
  GemmArgs g;
  g.M = d.M;
  g.N = d.N;
  g.K = d.K;
  g.ntn = (d.N + tile_of(d).bn - 1) / tile_of(d).bn;
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
    launch_typed<true, true>(g, tile_of(d), d.batch, splits, st);
  else if (d.Acplx)
    launch_typed<true, false>(g, tile_of(d), d.batch, splits, st);
  else if (d.Bcplx)
    launch_typed<false, true>(g, tile_of(d), d.batch, splits, st);
  else
    launch_typed<false, false>(g, tile_of(d), d.batch, splits, st);
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
