// HBM-bound kernels of the propagation: tensor permutes, amplitude algebra,
// the Adams-Moulton update (Eq. 9), the cumulant integrand (Eqs. 5-6), the
// spectral transform, set-up gathers, and padded/unpadded conversions.
//
// Every reduction is deterministic: fixed grids, fixed per-thread order,
// shared-memory trees, and bitwise max for the convergence measure, so the
// same inputs give the same bits whatever else runs on the GPU.
#include <type_traits>
#include "common.cuh"
#include "kernels.h"

namespace rteom {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n, int per_sm = 8) {
  int64_t b = (n + kThreads - 1) / kThreads;
  int64_t cap = 148LL * per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---------------------------------------------------------------- permute
// out = alpha * v + beta * out in the forms that need no FP64 multiply (the
// FP64 pipe is the scarce unit for these HBM-bound kernels).
enum AxOp { kCopy = 0, kNeg = 1, kAdd = 2, kSub = 3, kGeneral = 4 };

__device__ __forceinline__ double axop(int op, double v, double c, double alpha, double beta) {
  switch (op) {
    case kCopy:
      return v;
    case kNeg:
      return neg_f64(v);
    case kAdd:
      return c + v;
    case kSub:
      return c - v;
    default:
      return beta == 0.0 ? alpha * v : fma(beta, c, alpha * v);
  }
}

inline int axop_of(double alpha, double beta) {
  if (beta == 0.0 && alpha == 1.0) return kCopy;
  if (beta == 0.0 && alpha == -1.0) return kNeg;
  if (beta == 1.0 && alpha == 1.0) return kAdd;
  if (beta == 1.0 && alpha == -1.0) return kSub;
  return kGeneral;
}

// CPI / CPO: input / output complex.  A real input into a complex output
// scales the real part and leaves beta * imaginary part.  IDX: the integer
// type of the output-index decomposition (32-bit whenever it fits).
template <bool CPI, bool CPO, typename IDX>
__global__ void permute_kernel(const double* __restrict__ in, double* __restrict__ out,
                               PermDesc d, double alpha, double beta, int op, int64_t total) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total;
       o += (int64_t)gridDim.x * blockDim.x) {
    IDX rem = (IDX)o;
    int64_t off = 0;
#pragma unroll
    for (int k = 5; k >= 0; --k) {
      if (k < d.nd) {
        const IDX dim = (IDX)d.out_dim[k];
        const IDX q = rem / dim;
        off += (int64_t)(rem - q * dim) * d.in_stride[k];
        rem = q;
      }
    }
    const bool rd = op == kAdd || op == kSub || (op == kGeneral && beta != 0.0);  // reads out
    if constexpr (CPO) {
      double2 v = CPI ? reinterpret_cast<const double2*>(in)[off] : make_double2(in[off], 0.0);
      double2* po = reinterpret_cast<double2*>(out) + o;
      const double2 c = rd ? *po : make_double2(0.0, 0.0);
      double2 r;
      r.x = axop(op, v.x, c.x, alpha, beta);
      r.y = CPI ? axop(op, v.y, c.y, alpha, beta)
                : (rd ? (op == kGeneral ? beta * c.y : c.y) : 0.0);
      *po = r;
    } else {
      const double c = rd ? out[o] : 0.0;
      out[o] = axop(op, in[off], c, alpha, beta);
    }
  }
}

// Permutes whose output's innermost index is strided in the input while
// another output index is the input's unit-stride one: a 32 x 32 tile of
// (x = output innermost, y = that index) goes through shared memory, read
// along y and written along x, so both sides stay coalesced.  The remaining
// indices ("rest") are walked by blockIdx.y.
struct TileDesc {
  int64_t X, Y;             // extents of the x and y indices
  int64_t in_sx;            // input stride of x (that of y is 1)
  int64_t out_sy;           // output stride of y (that of x is 1)
  int nrest;                // other indices, innermost first
  int64_t rest_dim[4], rest_in[4], rest_out[4];
  int64_t nrest_total;
};

template <bool CPI, bool CPO>
__global__ void permute_tiled_kernel(const double* __restrict__ in, double* __restrict__ out,
                                     TileDesc t, double alpha, double beta, int op) {
  using TI = typename std::conditional<CPI, double2, double>::type;
  __shared__ TI tile[32][33];
  const int64_t tx_tiles = (t.X + 31) / 32;
  const int64_t x0 = (int64_t)(blockIdx.x % tx_tiles) * 32, y0 = (int64_t)(blockIdx.x / tx_tiles) * 32;
  const TI* tin = reinterpret_cast<const TI*>(in);
  const bool rd = op == kAdd || op == kSub || (op == kGeneral && beta != 0.0);
  auto bases = [&](int64_t r, int64_t& ib, int64_t& ob) {
    int64_t rem = r;
    ib = 0;
    ob = 0;
    for (int k = 0; k < t.nrest; ++k) {
      const int64_t q = rem / t.rest_dim[k];
      const int64_t i = rem - q * t.rest_dim[k];
      ib += i * t.rest_in[k];
      ob += i * t.rest_out[k];
      rem = q;
    }
  };
  constexpr int R = 32 / 8;  // tile rows per thread (blockDim.y = 8)
  // software pipeline: the loads of the next rest index are issued before
  // the stores of the current one
  TI v[R];
  int64_t r = blockIdx.y, ib = 0, ob = 0;
  auto load = [&](int64_t ibase) {
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int64_t x = x0 + threadIdx.y + 8 * u, y = y0 + threadIdx.x;
      if (x < t.X && y < t.Y) v[u] = tin[ibase + x * t.in_sx + y];
    }
  };
  if (r < t.nrest_total) {
    bases(r, ib, ob);
    load(ib);
  }
  for (; r < t.nrest_total; r += gridDim.y) {
    __syncthreads();  // the previous rest index finished reading the tile
#pragma unroll
    for (int u = 0; u < R; ++u) tile[threadIdx.y + 8 * u][threadIdx.x] = v[u];
    __syncthreads();
    const int64_t ob_cur = ob;
    const int64_t rn = r + gridDim.y;
    if (rn < t.nrest_total) {
      bases(rn, ib, ob);
      load(ib);
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int yi = threadIdx.y + 8 * u;
      const int64_t x = x0 + threadIdx.x, y = y0 + yi;
      if (x >= t.X || y >= t.Y) continue;
      const int64_t o = ob_cur + y * t.out_sy + x;
      if constexpr (CPO) {
        double2* po = reinterpret_cast<double2*>(out) + o;
        const double2 c = rd ? *po : make_double2(0.0, 0.0);
        double2 w;
        if constexpr (CPI) {
          w = tile[threadIdx.x][yi];
        } else {
          w = make_double2(tile[threadIdx.x][yi], 0.0);
        }
        double2 res;
        res.x = axop(op, w.x, c.x, alpha, beta);
        res.y = CPI ? axop(op, w.y, c.y, alpha, beta)
                    : (rd ? (op == kGeneral ? beta * c.y : c.y) : 0.0);
        *po = res;
      } else {
        const double c = rd ? out[o] : 0.0;
        out[o] = axop(op, (double)tile[threadIdx.x][yi], c, alpha, beta);
      }
    }
  }
}

// ---------------------------------------------------------------- t2 + t1 t1
__global__ void t2_t1t1_kernel(double2* __restrict__ out, const double2* __restrict__ t2,
                               double c1, const double2* __restrict__ x,
                               const double2* __restrict__ y, double c2, double c3, int nO,
                               int nV) {
  int64_t n = (int64_t)nO * nO * nV * nV;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int b = e % nV;
    int a = (e / nV) % nV;
    int j = (e / ((int64_t)nV * nV)) % nO;
    int i = e / ((int64_t)nV * nV * nO);
    double2 r = make_double2(0.0, 0.0);
    if (t2 != nullptr) {
      double2 t = t2[e];
      r = make_double2(c1 * t.x, c1 * t.y);
    }
    if (c2 != 0.0) {
      double2 p = cmul(x[i * nV + a], y[j * nV + b]);
      r.x = fma(c2, p.x, r.x);
      r.y = fma(c2, p.y, r.y);
    }
    if (c3 != 0.0) {
      double2 p = cmul(x[i * nV + b], y[j * nV + a]);
      r.x = fma(c3, p.x, r.x);
      r.y = fma(c3, p.y, r.y);
    }
    out[e] = r;
  }
}

// ---------------------------------------------------------------- P(ij), P(ab)
// R[i][j][a][b] += s0 X[i][j][a][b] + s1 X[j][i][a][b] + s2 X[i][j][b][a] +
// s3 X[j][i][b][a] with every s in {-1, 0, +1}: the terms present are the
// bits of NZ, the signs sign-bit masks, so no FP64 multiply or compare runs
// per element (only the adds).  A block takes one 32 x 32 (a, b) tile of one
// (i, j): the direct terms are read coalesced along b, the transposed ones
// as the (b, a) tile, staged through shared memory.
template <int NZ>
__global__ void antisym_add_kernel(double2* __restrict__ R, const double2* __restrict__ X,
                                   long long m0, long long m1, long long m2, long long m3, int nO,
                                   int nV) {
  __shared__ double2 tt[2][32][33];
  const int tv = (nV + 31) / 32;
  const int64_t units = (int64_t)nO * nO * tv * tv;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  const int64_t vv = (int64_t)nV * nV;
  auto sgn = [](double v, long long m) { return __longlong_as_double(__double_as_longlong(v) ^ m); };
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int tb = (int)(u % tv);
    const int64_t r = u / tv;
    const int ta = (int)(r % tv);
    const int ij = (int)(r / tv);
    const int i = ij / nO, j = ij - (ij / nO) * nO;
    const double2* Xij = X + (int64_t)ij * vv;
    const double2* Xji = X + ((int64_t)j * nO + i) * vv;
    const int a0 = 32 * ta, b0 = 32 * tb;
    if (NZ & 12) {
      __syncthreads();  // the previous unit's reads of the tiles are done
      // tt[0][bb][aa] = Xij[b0 + bb][a0 + aa], tt[1] likewise from Xji
      for (int k = ty; k < 32; k += 8) {
        const int b = b0 + k, a = a0 + tx;
        if (b < nV && a < nV) {
          if (NZ & 4) tt[0][k][tx] = Xij[(int64_t)b * nV + a];
          if (NZ & 8) tt[1][k][tx] = Xji[(int64_t)b * nV + a];
        }
      }
      __syncthreads();
    }
    for (int k = ty; k < 32; k += 8) {
      const int a = a0 + k, b = b0 + tx;
      if (a >= nV || b >= nV) continue;
      const int64_t o = (int64_t)a * nV + b;
      double2 acc = R[(int64_t)ij * vv + o];
      if (NZ & 1) {
        const double2 v = Xij[o];
        acc.x += sgn(v.x, m0);
        acc.y += sgn(v.y, m0);
      }
      if (NZ & 2) {
        const double2 v = Xji[o];
        acc.x += sgn(v.x, m1);
        acc.y += sgn(v.y, m1);
      }
      if (NZ & 4) {
        const double2 v = tt[0][tx][k];
        acc.x += sgn(v.x, m2);
        acc.y += sgn(v.y, m2);
      }
      if (NZ & 8) {
        const double2 v = tt[1][tx][k];
        acc.x += sgn(v.x, m3);
        acc.y += sgn(v.y, m3);
      }
      R[(int64_t)ij * vv + o] = acc;
    }
  }
}

// ---------------------------------------------------------------- antisymmetric pairs

__global__ void pack_pairs_kernel(const double2* __restrict__ t2, double2* __restrict__ out,
                                  int nO, int nV) {
  const int64_t npo = (int64_t)nO * (nO - 1) / 2, npv = (int64_t)nV * (nV - 1) / 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npo * npv;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i, j, a, b;
    pair_of(e / npv, nO, i, j);
    pair_of(e % npv, nV, a, b);
    out[e] = t2[(((int64_t)i * nO + j) * nV + a) * nV + b];
  }
}

__global__ void unpack_pairs_kernel(const double2* __restrict__ Rp, double2* R, int nO, int nV,
                                    double alpha) {
  const int64_t npo = (int64_t)nO * (nO - 1) / 2, npv = (int64_t)nV * (nV - 1) / 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npo * npv;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i, j, a, b;
    pair_of(e / npv, nO, i, j);
    pair_of(e % npv, nV, a, b);
    double2 v = Rp[e];
    v.x *= alpha;
    v.y *= alpha;
    auto at = [&](int p, int q, int r, int s) -> double2& {
      return R[(((int64_t)p * nO + q) * nV + r) * nV + s];
    };
    double2& r0 = at(i, j, a, b);
    r0.x += v.x;
    r0.y += v.y;
    double2& r1 = at(j, i, a, b);
    r1.x -= v.x;
    r1.y -= v.y;
    double2& r2 = at(i, j, b, a);
    r2.x -= v.x;
    r2.y -= v.y;
    double2& r3 = at(j, i, b, a);
    r3.x += v.x;
    r3.y += v.y;
  }
}

__global__ void pack_ladder_kernel(const double* __restrict__ W, double* __restrict__ Wm, int nV) {
  const int64_t npv = (int64_t)nV * (nV - 1) / 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npv * npv;
       e += (int64_t)gridDim.x * blockDim.x) {
    int ef, fe, a, b;
    pair_of(e / npv, nV, ef, fe);
    pair_of(e % npv, nV, a, b);
    const int64_t v2 = (int64_t)nV * nV;
    Wm[e] = W[((int64_t)ef * nV + fe) * v2 + (int64_t)a * nV + b] -
            W[((int64_t)fe * nV + ef) * v2 + (int64_t)a * nV + b];
  }
}

// Column chunks of the pair ladder: the pairs (a<b) with a in [a0, a0+n) are
// the contiguous pair indices [pair_start(a0), pair_start(a0+n)).  The largest
// a of the chunk whose first pair index is <= k, by bisection.
__device__ __forceinline__ void pair_in_chunk(int64_t k, int nV, int a0, int n, int& a, int& b) {
  int lo = a0, hi = a0 + n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pair_start(nV, mid) <= k)
      lo = mid;
    else
      hi = mid - 1;
  }
  a = lo;
  b = a + 1 + (int)(k - pair_start(nV, a));
}

// Wm[(e<f)][c] = Wc[e][f][a-a0][b] - Wc[f][e][a-a0][b] for the pair columns c
// of the chunk; Wc holds (ae|bf) for a in the chunk: [e][f][n][b] (real).
__global__ void pack_ladder_cols_kernel(const double* __restrict__ Wc, double* __restrict__ Wm,
                                        int nV, int a0, int n, int64_t p0, int64_t ncols) {
  const int64_t npv = (int64_t)nV * (nV - 1) / 2;
  for (int64_t r = blockIdx.x; r < npv; r += gridDim.x) {
    int e, f;
    pair_of(r, nV, e, f);
    const double* we = Wc + ((int64_t)e * nV + f) * n * nV;
    const double* wf = Wc + ((int64_t)f * nV + e) * n * nV;
    for (int64_t c = threadIdx.x; c < ncols; c += blockDim.x) {
      int a, b;
      pair_in_chunk(p0 + c, nV, a0, n, a, b);
      const int64_t o = (int64_t)(a - a0) * nV + b;
      Wm[r * ncols + c] = we[o] - wf[o];
    }
  }
}

// R[i,j,a,b] += alpha*Rq[P][c], with the three antisymmetric images, for the
// pair columns c of the chunk (complex).
__global__ void unpack_pairs_cols_kernel(const double2* __restrict__ Rq, double2* R, int nO,
                                         int nV, int a0, int n, int64_t p0, int64_t ncols,
                                         double alpha) {
  const int64_t npo = (int64_t)nO * (nO - 1) / 2;
  for (int64_t r = blockIdx.x; r < npo; r += gridDim.x) {
    int i, j;
    pair_of(r, nO, i, j);
    for (int64_t c = threadIdx.x; c < ncols; c += blockDim.x) {
      int a, b;
      pair_in_chunk(p0 + c, nV, a0, n, a, b);
      double2 v = Rq[r * ncols + c];
      v.x *= alpha;
      v.y *= alpha;
      auto at = [&](int p, int q, int u, int w) -> double2& {
        return R[(((int64_t)p * nO + q) * nV + u) * nV + w];
      };
      double2& r0 = at(i, j, a, b);
      r0.x += v.x;
      r0.y += v.y;
      double2& r1 = at(j, i, a, b);
      r1.x -= v.x;
      r1.y -= v.y;
      double2& r2 = at(i, j, b, a);
      r2.x -= v.x;
      r2.y -= v.y;
      double2& r3 = at(j, i, b, a);
      r3.x += v.x;
      r3.y += v.y;
    }
  }
}

// dst[r*ldd + c] += src[r*lds + c]
__global__ void add_block_kernel(double* __restrict__ dst, int64_t ldd,
                                 const double* __restrict__ src, int64_t lds, int64_t rows,
                                 int64_t cols) {
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
    for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) dst[r * ldd + c] += src[r * lds + c];
}

// ---------------------------------------------------------------- Anderson mixing
// Type-II Anderson acceleration of the fixed-point micro-iteration (Walker and
// Ni, SIAM J. Numer. Anal. 49, 1715 (2011)): with g_k = G(x_k), f_k = g_k - x_k
// and the last differences dF_j = f_{j+1} - f_j, dG_j = g_{j+1} - g_j,
// x_{k+1} = g_k - sum_j gamma_j dG_j where gamma minimises |f_k - sum_j gamma_j dF_j|.

// f = g - x.  first: Fp = f, Gp = g.  Otherwise dF[slot] = f - Fp,
// dG[slot] = g - Gp, then Fp = f, Gp = g.
__global__ void anderson_push_kernel(int64_t n, const double2* __restrict__ g,
                                     const double2* __restrict__ x, double2* Fp, double2* Gp,
                                     double2* __restrict__ dF, double2* __restrict__ dG,
                                     int first) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 gv = g[e], xv = x[e];
    const double2 f = make_double2(gv.x - xv.x, gv.y - xv.y);
    if (!first) {
      const double2 fp = Fp[e], gp = Gp[e];
      dF[e] = make_double2(f.x - fp.x, f.y - fp.y);
      dG[e] = make_double2(gv.x - gp.x, gv.y - gp.y);
    }
    Fp[e] = f;
    Gp[e] = gv;
  }
}

// Inner products <u, v> = sum conj(u) v of the normal equations: positions
// 0..5 hold <dF_i, dF_j> for (i, j) = (0,0),(0,1),(0,2),(1,1),(1,2),(2,2) and
// 6..8 hold <dF_i, f>; entries with an index >= count are zero.  Pass 1: one
// partial per block (fixed grid), pass 2: fixed-order sums (deterministic).
__device__ __forceinline__ void and_pair(int d, int& i, int& j) {
  const int I[6] = {0, 0, 0, 1, 1, 2}, J[6] = {0, 1, 2, 1, 2, 2};
  i = I[d];
  j = J[d];
}

__global__ void anderson_dots_pass1(int64_t n, const double2* __restrict__ dF, int64_t slot,
                                    const double2* __restrict__ f, int count,
                                    double2* __restrict__ partial) {
  double2 acc[kAndersonDots];
#pragma unroll
  for (int d = 0; d < kAndersonDots; ++d) acc[d] = make_double2(0.0, 0.0);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double2 u[kAndersonDepth];
#pragma unroll
    for (int q = 0; q < kAndersonDepth; ++q)
      u[q] = q < count ? dF[q * slot + e] : make_double2(0.0, 0.0);
    const double2 fv = f[e];
#pragma unroll
    for (int d = 0; d < kAndersonDots; ++d) {
      double2 a, b;
      if (d < 6) {
        int i, j;
        and_pair(d, i, j);
        a = u[i];
        b = u[j];
      } else {
        a = u[d - 6];
        b = fv;
      }
      acc[d].x += a.x * b.x + a.y * b.y;
      acc[d].y += a.x * b.y - a.y * b.x;
    }
  }
  __shared__ double2 red[kThreads];
  for (int d = 0; d < kAndersonDots; ++d) {
    red[threadIdx.x] = acc[d];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) {
        red[threadIdx.x].x += red[threadIdx.x + w].x;
        red[threadIdx.x].y += red[threadIdx.x + w].y;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * kAndersonDots + d] = red[0];
    __syncthreads();
  }
}

__global__ void anderson_dots_pass2(const double2* __restrict__ partial, int np,
                                    double2* __restrict__ out) {
  const int d = threadIdx.x;
  if (d >= kAndersonDots) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < np; ++b) {
    const double2 v = partial[(int64_t)b * kAndersonDots + d];
    s.x += v.x;
    s.y += v.y;
  }
  out[d] = s;
}

// x = g - sum_{j < count} gamma_j dG_j
__global__ void anderson_mix_kernel(int64_t n, const double2* __restrict__ g,
                                    const double2* __restrict__ dG, int64_t slot, int count,
                                    double2 g0, double2 g1, double2 g2,
                                    double2* __restrict__ x) {
  const double2 gam[3] = {g0, g1, g2};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double2 v = g[e];
    for (int q = 0; q < count; ++q) {
      const double2 w = dG[q * slot + e];
      v.x -= gam[q].x * w.x - gam[q].y * w.y;
      v.y -= gam[q].x * w.y + gam[q].y * w.x;
    }
    x[e] = v;
  }
}

// ---------------------------------------------------------------- amplitude geometry
struct Elem {
  int blk, i, j, a, b;
};

__device__ __forceinline__ Elem decode(const AmpGeom& g, int64_t e) {
  Elem r;
  int64_t n1 = g.n1(), n2 = g.n2();
  if (e < 2 * n1) {
    r.blk = (int)(e / n1);
    int64_t q = e - r.blk * n1;
    r.i = (int)(q / g.nV);
    r.a = (int)(q % g.nV);
    r.j = r.b = 0;
  } else {
    int64_t q = e - 2 * n1;
    r.blk = 2 + (int)(q / n2);
    q -= (int64_t)(r.blk - 2) * n2;
    r.b = (int)(q % g.nV);
    r.a = (int)((q / g.nV) % g.nV);
    r.j = (int)((q / ((int64_t)g.nV * g.nV)) % g.nO);
    r.i = (int)(q / ((int64_t)g.nV * g.nV * g.nO));
  }
  return r;
}

// Spins of (i,a) and (j,b) for each block: t1a, t1b, t2aa, t2ab, t2bb.
__device__ __forceinline__ int spin_ia(int blk) { return (blk == 1 || blk == 4) ? 1 : 0; }
__device__ __forceinline__ int spin_jb(int blk) { return (blk == 3 || blk == 4) ? 1 : 0; }

__device__ __forceinline__ bool is_pad(const AmpGeom& g, const Elem& x) {
  // alpha virtual slot 0 (the core is occupied in alpha) and beta occupied
  // slot `core` (the ionised electron) do not exist.
  int s1 = spin_ia(x.blk);
  if (s1 == 0 && x.a == 0) return true;
  if (s1 == 1 && x.i == g.core) return true;
  if (x.blk >= 2) {
    int s2 = spin_jb(x.blk);
    if (s2 == 0 && x.b == 0) return true;
    if (s2 == 1 && x.j == g.core) return true;
  }
  return false;
}

__device__ __forceinline__ unsigned long long umax_warp(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// 1/x for x >= 1 (here x = 1 + (h D)^2): an FP32 reciprocal refined by two
// Newton-Raphson steps r <- r (2 - x r) in FP64, each squaring the relative
// error (2^-22 -> 2^-44 -> below 2^-53 before rounding).
__device__ __forceinline__ double recip_newton(double x) {
  double r = (double)__frcp_rn((float)x);
  r = r * fma(-x, r, 2.0);
  r = r * fma(-x, r, 2.0);
  return r;
}

// One block per row of an amplitude block, or per segment of kUpdateSeg
// entries of a long row: a T1 row (i) holds nV entries, a T2 row (i, j)
// nV*nV entries (a, b).  The row's occupied part of the
// denominator, its spins and its pad status are fixed per block; the
// virtual part comes from two table reads.  With R' = R - D t the update of
// Eq. 9 reduces to
//   t_new = [t_n + i h (R_n + R_k - D t_k)] (1 + i h D) / (1 + (h D)^2),
// h = dt/2, and the convergence measure is max |t_new - t_k|^2.
constexpr int kUpdateSeg = 2048;  // entries per block of a T2 row

__global__ void am_update_kernel(AmpGeom g, const double* __restrict__ fo_a,
                                 const double* __restrict__ fv_a, const double* __restrict__ fo_b,
                                 const double* __restrict__ fv_b, double dt,
                                 const double2* __restrict__ tn, const double2* __restrict__ Rn,
                                 const double2* tk_in, double2* tk_out,
                                 const double2* __restrict__ Rk, unsigned long long* maxdiff) {
  __shared__ unsigned long long red[kThreads / 32];
  const int nO = g.nO, nV = g.nV;
  const int rows1 = 2 * nO, rows = rows1 + 3 * nO * nO;
  const int segs = (nV * nV + kUpdateSeg - 1) / kUpdateSeg;  // segments of a T2 row
  const int units = rows1 + 3 * nO * nO * segs;
  const double h = 0.5 * dt;
  unsigned long long m = 0ull;
  for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
    // unit -> (row, segment): a T1 row is one unit, a T2 row `segs` units
    const int row = unit < rows1 ? unit : rows1 + (unit - rows1) / segs;
    const int seg = unit < rows1 ? 0 : (unit - rows1) % segs;
    int blk, i, j;
    int64_t base;
    int len;
    if (row < rows1) {
      blk = row / nO;
      i = row - blk * nO;
      j = 0;
      base = g.off(blk) + (int64_t)i * nV;
      len = nV;
    } else {
      const int q = row - rows1;
      const int t = q / (nO * nO);
      blk = 2 + t;
      const int ij = q - t * nO * nO;
      i = ij / nO;
      j = ij - i * nO;
      base = g.off(blk) + (int64_t)ij * nV * nV;
      len = nV * nV;
    }
    const int s1 = spin_ia(blk), s2 = spin_jb(blk);
    const double* fv1 = s1 ? fv_b : fv_a;
    const double* fv2 = s2 ? fv_b : fv_a;
    bool row_pad = (s1 == 1 && i == g.core);
    double Drow = -(s1 ? fo_b : fo_a)[i];
    if (blk >= 2) {
      row_pad = row_pad || (s2 == 1 && j == g.core);
      Drow -= (s2 ? fo_b : fo_a)[j];
    }
    // a T1 row is taken whole; a T2 row in segments of kUpdateSeg entries
    const int q0 = seg * kUpdateSeg, q1 = blk < 2 ? len : min(len, q0 + kUpdateSeg);
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
      int a, b;
      if (blk >= 2) {
        a = q / nV;
        b = q - a * nV;
      } else {
        a = q;
        b = -1;
      }
      const int64_t e = base + q;
      const double2 old = tk_in[e];
      double2 nw = make_double2(0.0, 0.0);
      const bool pad = row_pad || (s1 == 0 && a == 0) || (b >= 0 && s2 == 0 && b == 0);
      if (!pad) {
        double D = Drow + fv1[a];
        if (b >= 0) D += fv2[b];
        const double2 t0 = tn[e], rn = Rn[e], rk = Rk[e];
        const double sx = fma(-D, old.x, rn.x + rk.x);
        const double sy = fma(-D, old.y, rn.y + rk.y);
        const double nx = fma(-h, sy, t0.x);
        const double ny = fma(h, sx, t0.y);
        const double hd = h * D;
        const double inv = recip_newton(fma(hd, hd, 1.0));
        nw.x = fma(-hd, ny, nx) * inv;
        nw.y = fma(hd, nx, ny) * inv;
      }
      tk_out[e] = nw;
      const double dx = nw.x - old.x, dy = nw.y - old.y;
      const double d2 = fma(dx, dx, dy * dy);
      unsigned long long bits = (unsigned long long)__double_as_longlong(d2);
      if (d2 != d2) bits = 0x7ff8000000000000ull;
      m = bits > m ? bits : m;
    }
  }
  m = umax_warp(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long v = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0ull;
    v = umax_warp(v);
    if (threadIdx.x == 0) atomicMax(maxdiff, v);
  }
}

__global__ void mask_kernel(AmpGeom g, double2* t) {
  int64_t total = g.total();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (is_pad(g, decode(g, e))) t[e] = make_double2(0.0, 0.0);
  }
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double2 block_sum2(double2 v, double2* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sh[threadIdx.x].x += sh[threadIdx.x + s].x;
      sh[threadIdx.x].y += sh[threadIdx.x + s].y;
    }
    __syncthreads();
  }
  double2 r = sh[0];
  __syncthreads();
  return r;
}

__global__ void energy_pass1(AmpGeom g, const double2* __restrict__ t,
                             const double* __restrict__ ovov, const double* __restrict__ fov_a,
                             const double* __restrict__ fov_b, int include_fov,
                             double2* __restrict__ partial) {
  __shared__ double2 sh[kThreads];
  const int nO = g.nO, nV = g.nV;
  const double2* t1a = t;
  const double2* t1b = t + g.n1();
  const double2* t2aa = t + 2 * g.n1();
  const double2* t2ab = t2aa + g.n2();
  const double2* t2bb = t2ab + g.n2();
  double2 acc = make_double2(0.0, 0.0);
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (include_fov) {
    for (int64_t e = tid; e < g.n1(); e += stride) {
      double fa = fov_a[e], fb = fov_b[e];
      acc.x += fa * t1a[e].x + fb * t1b[e].x;
      acc.y += fa * t1a[e].y + fb * t1b[e].y;
    }
  }
  for (int64_t e = tid; e < g.n2(); e += stride) {
    int b = e % nV;
    int a = (e / nV) % nV;
    int j = (e / ((int64_t)nV * nV)) % nO;
    int i = e / ((int64_t)nV * nV * nO);
    // (ia|jb) and (ib|ja) from ovov[p][q][r][s] = (pq|rs)
    double I1 = ovov[(((int64_t)i * nV + a) * nO + j) * nV + b];
    double I2 = ovov[(((int64_t)i * nV + b) * nO + j) * nV + a];
    double2 saa = t2aa[e], sab = t2ab[e], sbb = t2bb[e];
    double2 ta_ia = t1a[i * nV + a], ta_jb = t1a[j * nV + b];
    double2 tb_ia = t1b[i * nV + a], tb_jb = t1b[j * nV + b];
    double2 paa = cmul(ta_ia, ta_jb), pbb = cmul(tb_ia, tb_jb), pab = cmul(ta_ia, tb_jb);
    // 1/2 I (t2aa + t2bb) + I t2ab + 1/2 (I1 - I2)(t1a t1a + t1b t1b) + I t1a t1b
    acc.x += 0.5 * I1 * (saa.x + sbb.x) + I1 * sab.x + 0.5 * (I1 - I2) * (paa.x + pbb.x) +
             I1 * pab.x;
    acc.y += 0.5 * I1 * (saa.y + sbb.y) + I1 * sab.y + 0.5 * (I1 - I2) * (paa.y + pbb.y) +
             I1 * pab.y;
  }
  double2 s = block_sum2(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void energy_pass2(const double2* __restrict__ partial, int np, double2* E_hist,
                             double2* C_hist, long long n, double dt, int update_c) {
  __shared__ double2 sh[kThreads];
  double2 acc = make_double2(0.0, 0.0);
  for (int k = threadIdx.x; k < np; k += blockDim.x) {
    acc.x += partial[k].x;
    acc.y += partial[k].y;
  }
  double2 E = block_sum2(acc, sh);
  if (threadIdx.x == 0) {
    E_hist[n + 1] = E;
    if (update_c) {
      double2 Ep = E_hist[n];
      double2 Cp = C_hist[n];
      // C_{n+1} = C_n + (i dt / 2)(E_n + E_{n+1})
      double sx = Ep.x + E.x, sy = Ep.y + E.y;
      C_hist[n + 1] = make_double2(Cp.x - 0.5 * dt * sy, Cp.y + 0.5 * dt * sx);
    }
  }
}

// ---------------------------------------------------------------- pack / unpack
// Unpadded spin-block index of a padded element, or -1 for a pad.
__device__ __forceinline__ int64_t unpadded_index(const AmpGeom& g, const Elem& x) {
  if (is_pad(g, x)) return -1;
  const int64_t oA = g.nO, vA = g.nV - 1, oB = g.nO - 1, vB = g.nV;
  auto occ_u = [&](int s, int i) -> int64_t { return s ? (i < g.core ? i : i - 1) : i; };
  auto vir_u = [&](int s, int a) -> int64_t { return s ? a : a - 1; };
  int64_t o1a = 0, o1b = oA * vA, o2aa = o1b + oB * vB, o2ab = o2aa + oA * oA * vA * vA,
          o2bb = o2ab + oA * oB * vA * vB;
  switch (x.blk) {
    case 0: return o1a + occ_u(0, x.i) * vA + vir_u(0, x.a);
    case 1: return o1b + occ_u(1, x.i) * vB + vir_u(1, x.a);
    case 2: return o2aa + ((occ_u(0, x.i) * oA + occ_u(0, x.j)) * vA + vir_u(0, x.a)) * vA + vir_u(0, x.b);
    case 3: return o2ab + ((occ_u(0, x.i) * oB + occ_u(1, x.j)) * vA + vir_u(0, x.a)) * vB + vir_u(1, x.b);
    default: return o2bb + ((occ_u(1, x.i) * oB + occ_u(1, x.j)) * vB + vir_u(1, x.a)) * vB + vir_u(1, x.b);
  }
}

__global__ void pack_kernel(AmpGeom g, const double2* __restrict__ u, double2* __restrict__ p) {
  int64_t total = g.total();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t k = unpadded_index(g, decode(g, e));
    p[e] = k < 0 ? make_double2(0.0, 0.0) : u[k];
  }
}

__global__ void unpack_kernel(AmpGeom g, const double2* __restrict__ p, double2* __restrict__ u) {
  int64_t total = g.total();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t k = unpadded_index(g, decode(g, e));
    if (k >= 0) u[k] = p[e];
  }
}

// Padded index of the entry with flat index k of the unpadded spin-block
// vector (the inverse of unpadded_index on real entries).
__device__ __forceinline__ int64_t padded_of_unpadded(const AmpGeom& g, int64_t k) {
  const int64_t oA = g.nO, vA = g.nV - 1, oB = g.nO - 1, vB = g.nV;
  const int64_t n1a = oA * vA, n1b = oB * vB, n2aa = oA * oA * vA * vA, n2ab = oA * oB * vA * vB;
  int blk = 0;
  int64_t q = k;
  if (q >= n1a) {
    q -= n1a;
    blk = 1;
    if (q >= n1b) {
      q -= n1b;
      blk = 2;
      if (q >= n2aa) {
        q -= n2aa;
        blk = 3;
        if (q >= n2ab) {
          q -= n2ab;
          blk = 4;
        }
      }
    }
  }
  const int si = spin_ia(blk), sj = spin_jb(blk);
  auto occ_slot = [&](int s, int64_t i) -> int64_t { return (s && i >= g.core) ? i + 1 : i; };
  auto vir_slot = [&](int s, int64_t a) -> int64_t { return s ? a : a + 1; };
  const int64_t nva = si ? vB : vA, nvb = sj ? vB : vA, noj = sj ? oB : oA;
  if (blk < 2) {
    const int64_t i = q / nva, a = q % nva;
    return g.off(blk) + occ_slot(si, i) * g.nV + vir_slot(si, a);
  }
  const int64_t b = q % nvb;
  q /= nvb;
  const int64_t a = q % nva;
  q /= nva;
  const int64_t j = q % noj, i = q / noj;
  return g.off(blk) + ((occ_slot(si, i) * g.nO + occ_slot(sj, j)) * g.nV + vir_slot(si, a)) * g.nV +
         vir_slot(sj, b);
}

__global__ void scatter_unpadded_kernel(AmpGeom g, const long long* __restrict__ idx,
                                        const double2* __restrict__ val, int64_t n,
                                        double2* __restrict__ padded) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    padded[padded_of_unpadded(g, idx[e])] = val[e];
}

__global__ void gather_unpadded_kernel(AmpGeom g, const double2* __restrict__ padded,
                                       const long long* __restrict__ idx, int64_t n,
                                       double2* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = padded[padded_of_unpadded(g, idx[e])];
}

// ---------------------------------------------------------------- set-up
__device__ __forceinline__ int vmap(int a, int nO, int core) { return a == 0 ? core : nO + a - 1; }

__global__ void gather_L_kernel(const double* __restrict__ L, int nchol, int nO, int nV, int core,
                                double* Loo, double* Lov, double* Lvv) {
  const int nb = nO + nV - 1;
  int64_t per = (int64_t)nO * nO + (int64_t)nO * nV + (int64_t)nV * nV;
  int64_t total = per * nchol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int Q = (int)(e / per);
    int64_t r = e - (int64_t)Q * per;
    const double* LQ = L + (int64_t)Q * nb * nb;
    if (r < (int64_t)nO * nO) {
      int i = r / nO, j = r % nO;
      Loo[(int64_t)Q * nO * nO + r] = LQ[(int64_t)i * nb + j];
    } else if (r < (int64_t)nO * nO + (int64_t)nO * nV) {
      r -= (int64_t)nO * nO;
      int i = r / nV, a = r % nV;
      Lov[(int64_t)Q * nO * nV + r] = LQ[(int64_t)i * nb + vmap(a, nO, core)];
    } else {
      r -= (int64_t)nO * nO + (int64_t)nO * nV;
      int a = r / nV, b = r % nV;
      Lvv[(int64_t)Q * nV * nV + r] = LQ[(int64_t)vmap(a, nO, core) * nb + vmap(b, nO, core)];
    }
  }
}

// f^a_pq = eps_p d_pq - (pq|cc);  f^b_pq = f^a_pq + (pc|cq)
__device__ double fock_elem(const double* eps, const double* L, int nchol, int nb, int core,
                            int p, int q, int spin) {
  double J = 0.0, K = 0.0;
  const int64_t nn = (int64_t)nb * nb;
  for (int Q = 0; Q < nchol; ++Q) {
    const double* LQ = L + Q * nn;
    J = fma(LQ[(int64_t)p * nb + q], LQ[(int64_t)core * nb + core], J);
    K = fma(LQ[(int64_t)p * nb + core], LQ[(int64_t)core * nb + q], K);
  }
  double f = (p == q ? eps[p] : 0.0) - J;
  if (spin) f += K;
  return f;
}

__global__ void fock_kernel(const double* __restrict__ eps, const double* __restrict__ L,
                            int nchol, int nO, int nV, int core, double* foo_a, double* fov_a,
                            double* fvv_a, double* foo_b, double* fov_b, double* fvv_b) {
  const int nb = nO + nV - 1;
  int64_t per = (int64_t)nO * nO + (int64_t)nO * nV + (int64_t)nV * nV;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 2 * per;
       e += (int64_t)gridDim.x * blockDim.x) {
    int spin = e >= per;
    int64_t r = e - spin * per;
    double *foo = spin ? foo_b : foo_a, *fov = spin ? fov_b : fov_a, *fvv = spin ? fvv_b : fvv_a;
    if (r < (int64_t)nO * nO) {
      int i = r / nO, j = r % nO;
      foo[r] = fock_elem(eps, L, nchol, nb, core, i, j, spin);
    } else if (r < (int64_t)nO * nO + (int64_t)nO * nV) {
      r -= (int64_t)nO * nO;
      int i = r / nV, a = r % nV;
      fov[r] = fock_elem(eps, L, nchol, nb, core, i, vmap(a, nO, core), spin);
    } else {
      r -= (int64_t)nO * nO + (int64_t)nO * nV;
      int a = r / nV, b = r % nV;
      fvv[r] = fock_elem(eps, L, nchol, nb, core, vmap(a, nO, core), vmap(b, nO, core), spin);
    }
  }
}

__global__ void diag_kernel(const double* foo_a, const double* fvv_a, const double* foo_b,
                            const double* fvv_b, int nO, int nV, double* fo_a, double* fv_a,
                            double* fo_b, double* fv_b) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nO) {
    fo_a[k] = foo_a[k * nO + k];
    fo_b[k] = foo_b[k * nO + k];
  }
  if (k < nV) {
    fv_a[k] = fvv_a[k * nV + k];
    fv_b[k] = fvv_b[k * nV + k];
  }
}

__global__ void ecorr_pass1(const double* __restrict__ ovov, const double* __restrict__ t1,
                            const double* __restrict__ t2, int O, int V,
                            double2* __restrict__ partial) {
  __shared__ double2 sh[kThreads];
  const int nO = O, nV = V + 1;
  double acc = 0.0;
  int64_t n = (int64_t)O * O * V * V;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int b = e % V;
    int a = (e / V) % V;
    int j = (e / ((int64_t)V * V)) % O;
    int i = e / ((int64_t)V * V * O);
    double iajb = ovov[(((int64_t)i * nV + a + 1) * nO + j) * nV + b + 1];
    double ibja = ovov[(((int64_t)i * nV + b + 1) * nO + j) * nV + a + 1];
    double tt = (t2 ? t2[e] : 0.0) + (t1 ? t1[i * V + a] * t1[j * V + b] : 0.0);
    acc += (2.0 * iajb - ibja) * tt;
  }
  double2 s = block_sum2(make_double2(acc, 0.0), sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void ecorr_pass2(const double2* partial, int np, double* out) {
  __shared__ double2 sh[kThreads];
  double2 acc = make_double2(0.0, 0.0);
  for (int k = threadIdx.x; k < np; k += blockDim.x) acc.x += partial[k].x;
  double2 s = block_sum2(acc, sh);
  if (threadIdx.x == 0) *out = s.x;
}

// ---------------------------------------------------------------- spectrum
// A(w) = -(1/pi) Im sum_n w_n dt G_n exp(i w tau_n - eta tau_n),
// G_n = -i exp(-i shift tau_n) exp(C_n), shift = eps_c + E_corr.
__global__ void spectrum_kernel(const double2* __restrict__ C, long long M, double dt,
                                double shift, const double* __restrict__ omega, double eta,
                                double* __restrict__ A) {
  __shared__ double2 sh[kThreads];
  const double w = omega[blockIdx.x];
  double2 acc = make_double2(0.0, 0.0);
  for (long long n = threadIdx.x; n <= M; n += blockDim.x) {
    double tau = dt * (double)n;
    double2 c = C[n];
    double mag = exp(c.x - eta * tau);
    double s, co;
    sincos(c.y + (w - shift) * tau, &s, &co);
    double wt = (n == 0 || n == M) ? 0.5 : 1.0;
    // -i * (co + i s) = s - i co
    acc.x += wt * mag * s;
    acc.y -= wt * mag * co;
  }
  double2 S = block_sum2(acc, sh);
  if (threadIdx.x == 0) A[blockIdx.x] = -(dt / 3.14159265358979323846) * S.y;
}

__global__ void maxabs_kernel(const double* __restrict__ x, int64_t n, unsigned long long* out) {
  __shared__ unsigned long long red[kThreads / 32];
  unsigned long long m = 0ull;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v = x[e];
    unsigned long long bits = (unsigned long long)__double_as_longlong(fabs(v));
    if (v != v) bits = 0x7ff8000000000000ull;
    m = bits > m ? bits : m;
  }
  m = umax_warp(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long v = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0ull;
    v = umax_warp(v);
    if (threadIdx.x == 0) atomicMax(out, v);
  }
}

}  // namespace

// ============================================================== launchers
void permute_add(const double* in, double* out, const PermDesc& d, bool in_cplx, bool out_cplx,
                 double alpha, double beta, cudaStream_t st) {
  int64_t total = 1;
  for (int k = 0; k < d.nd; ++k) total *= d.out_dim[k];
  if (total == 0) return;
  if (in_cplx && !out_cplx) throw Error(-1, "permute_add: complex input into real output");
  const int op = axop_of(alpha, beta);
  // tiled transpose when the output's innermost index is strided in the
  // input and another output index is the input's unit-stride one
  const int xo = d.nd - 1;
  int yo = -1;
  for (int k = 0; k < xo; ++k)
    if (d.in_stride[k] == 1 && d.out_dim[k] > 1) yo = k;
  if (d.nd >= 2 && d.nd <= 6 && d.in_stride[xo] != 1 && yo >= 0 && d.out_dim[xo] >= 16 &&
      d.out_dim[yo] >= 16) {
    TileDesc t{};
    t.X = d.out_dim[xo];
    t.Y = d.out_dim[yo];
    t.in_sx = d.in_stride[xo];
    int64_t os = 1;
    int64_t out_stride[6];
    for (int k = d.nd - 1; k >= 0; --k) {
      out_stride[k] = os;
      os *= d.out_dim[k];
    }
    t.out_sy = out_stride[yo];
    t.nrest = 0;
    t.nrest_total = 1;
    for (int k = d.nd - 1; k >= 0; --k) {
      if (k == xo || k == yo) continue;
      t.rest_dim[t.nrest] = d.out_dim[k];
      t.rest_in[t.nrest] = d.in_stride[k];
      t.rest_out[t.nrest] = out_stride[k];
      t.nrest_total *= d.out_dim[k];
      ++t.nrest;
    }
    const int64_t tiles = ((t.X + 31) / 32) * ((t.Y + 31) / 32);
    if (tiles <= 0x7fffffffll) {
      // about eight blocks per SM in all; each walks several rest indices
      int64_t gy = (148 * 8 + tiles - 1) / tiles;
      if (gy > t.nrest_total) gy = t.nrest_total;
      if (gy > 65535) gy = 65535;
      if (gy < 1) gy = 1;
      dim3 grid((unsigned)tiles, (unsigned)gy);
      dim3 block(32, 8);
      if (in_cplx)
        permute_tiled_kernel<true, true><<<grid, block, 0, st>>>(in, out, t, alpha, beta, op);
      else if (out_cplx)
        permute_tiled_kernel<false, true><<<grid, block, 0, st>>>(in, out, t, alpha, beta, op);
      else
        permute_tiled_kernel<false, false><<<grid, block, 0, st>>>(in, out, t, alpha, beta, op);
      RT_CHECK_LAUNCH();
      return;
    }
  }
  int grid = grid_for(total, 16);
  auto go = [&](auto idx_tag) {
    using I = decltype(idx_tag);
    if (in_cplx)
      permute_kernel<true, true, I><<<grid, kThreads, 0, st>>>(in, out, d, alpha, beta, op, total);
    else if (out_cplx)
      permute_kernel<false, true, I><<<grid, kThreads, 0, st>>>(in, out, d, alpha, beta, op, total);
    else
      permute_kernel<false, false, I><<<grid, kThreads, 0, st>>>(in, out, d, alpha, beta, op,
                                                                  total);
  };
  if (total <= 0xFFFFFFFFll)
    go(0u);
  else
    go((uint64_t)0);
  RT_CHECK_LAUNCH();
}

void t2_plus_t1t1(double* out, const double* t2, double c1, const double* x, const double* y,
                  double c2, double c3, int nO, int nV, cudaStream_t st) {
  int64_t n = (int64_t)nO * nO * nV * nV;
  if (n == 0) return;
  t2_t1t1_kernel<<<grid_for(n, 16), kThreads, 0, st>>>(
      reinterpret_cast<double2*>(out), reinterpret_cast<const double2*>(t2), c1,
      reinterpret_cast<const double2*>(x), reinterpret_cast<const double2*>(y), c2, c3, nO, nV);
  RT_CHECK_LAUNCH();
}

void antisym_add(double* R, const double* X, double c0, double c1, double c2, double c3, int nO,
                 int nV, cudaStream_t st) {
  const int64_t tv = (nV + 31) / 32;
  const int64_t units = (int64_t)nO * nO * tv * tv;
  if (units == 0) return;
  const double c[4] = {c0, c1, c2, c3};
  int nz = 0;
  long long m[4];
  for (int k = 0; k < 4; ++k) {
    if (c[k] != 0.0 && c[k] != 1.0 && c[k] != -1.0)
      throw Error(-1, "antisym_add: coefficients must be 0 or +-1");
    if (c[k] != 0.0) nz |= 1 << k;
    m[k] = c[k] == -1.0 ? (long long)0x8000000000000000ull : 0ll;
  }
  const int grid = (int)std::min<int64_t>(units, 148 * 8);
  auto R2 = reinterpret_cast<double2*>(R);
  auto X2 = reinterpret_cast<const double2*>(X);
#define RT_ANTISYM(NZ)                                                                         \
  case NZ:                                                                                     \
    antisym_add_kernel<NZ><<<grid, kThreads, 0, st>>>(R2, X2, m[0], m[1], m[2], m[3], nO, nV); \
    break;
  switch (nz) {
    RT_ANTISYM(1) RT_ANTISYM(2) RT_ANTISYM(3) RT_ANTISYM(4) RT_ANTISYM(5) RT_ANTISYM(6)
    RT_ANTISYM(7) RT_ANTISYM(8) RT_ANTISYM(9) RT_ANTISYM(10) RT_ANTISYM(11) RT_ANTISYM(12)
    RT_ANTISYM(13) RT_ANTISYM(14) RT_ANTISYM(15)
    default:
      return;  // all coefficients zero
  }
#undef RT_ANTISYM
  RT_CHECK_LAUNCH();
}

void pack_pairs(const double* t2, double* out, int nO, int nV, cudaStream_t st) {
  int64_t n = (int64_t)nO * (nO - 1) / 2 * ((int64_t)nV * (nV - 1) / 2);
  if (n == 0) return;
  pack_pairs_kernel<<<grid_for(n, 16), kThreads, 0, st>>>(
      reinterpret_cast<const double2*>(t2), reinterpret_cast<double2*>(out), nO, nV);
  RT_CHECK_LAUNCH();
}

void unpack_pairs_antisym(const double* Rp, double* R, int nO, int nV, double alpha,
                          cudaStream_t st) {
  int64_t n = (int64_t)nO * (nO - 1) / 2 * ((int64_t)nV * (nV - 1) / 2);
  if (n == 0) return;
  unpack_pairs_kernel<<<grid_for(n, 16), kThreads, 0, st>>>(
      reinterpret_cast<const double2*>(Rp), reinterpret_cast<double2*>(R), nO, nV, alpha);
  RT_CHECK_LAUNCH();
}

void pack_ladder_antisym(const double* W, double* Wm, int nV, cudaStream_t st) {
  int64_t npv = (int64_t)nV * (nV - 1) / 2;
  if (npv == 0) return;
  pack_ladder_kernel<<<grid_for(npv * npv, 16), kThreads, 0, st>>>(W, Wm, nV);
  RT_CHECK_LAUNCH();
}

void pack_ladder_cols(const double* Wc, double* Wm, int nV, int a0, int n, cudaStream_t st) {
  const int64_t npv = (int64_t)nV * (nV - 1) / 2;
  const int64_t p0 = pair_start(nV, a0), ncols = pair_start(nV, a0 + n) - p0;
  if (npv == 0 || ncols == 0) return;
  pack_ladder_cols_kernel<<<(int)std::min<int64_t>(npv, 148 * 16), kThreads, 0, st>>>(
      Wc, Wm, nV, a0, n, p0, ncols);
  RT_CHECK_LAUNCH();
}

void unpack_pairs_cols(const double* Rq, double* R, int nO, int nV, int a0, int n, double alpha,
                       cudaStream_t st) {
  const int64_t npo = (int64_t)nO * (nO - 1) / 2;
  const int64_t p0 = pair_start(nV, a0), ncols = pair_start(nV, a0 + n) - p0;
  if (npo == 0 || ncols == 0) return;
  unpack_pairs_cols_kernel<<<(int)std::min<int64_t>(npo, 148 * 16), kThreads, 0, st>>>(
      reinterpret_cast<const double2*>(Rq), reinterpret_cast<double2*>(R), nO, nV, a0, n, p0,
      ncols, alpha);
  RT_CHECK_LAUNCH();
}

void add_block(double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows,
               int64_t cols, cudaStream_t st) {
  if (rows == 0 || cols == 0) return;
  add_block_kernel<<<(int)std::min<int64_t>(rows, 148 * 16), kThreads, 0, st>>>(dst, ldd, src,
                                                                                 lds, rows, cols);
  RT_CHECK_LAUNCH();
}

void am_update(const AmpGeom& g, const double* fo_a, const double* fv_a, const double* fo_b,
               const double* fv_b, double dt, const double* tn, const double* Rn,
               const double* tk_in, double* tk_out, const double* Rk,
               unsigned long long* maxdiff_bits, cudaStream_t st) {
  const int segs = (g.nV * g.nV + kUpdateSeg - 1) / kUpdateSeg;
  const int units = 2 * g.nO + 3 * g.nO * g.nO * segs;
  am_update_kernel<<<std::min(units, 148 * 16), kThreads, 0, st>>>(
      g, fo_a, fv_a, fo_b, fv_b, dt, reinterpret_cast<const double2*>(tn),
      reinterpret_cast<const double2*>(Rn), reinterpret_cast<const double2*>(tk_in),
      reinterpret_cast<double2*>(tk_out), reinterpret_cast<const double2*>(Rk), maxdiff_bits);
  RT_CHECK_LAUNCH();
}

void anderson_push(int64_t n, const double* g, const double* x, double* Fp, double* Gp,
                   double* dF, double* dG, int first, cudaStream_t st) {
  if (n == 0) return;
  anderson_push_kernel<<<grid_for(n, 16), kThreads, 0, st>>>(
      n, reinterpret_cast<const double2*>(g), reinterpret_cast<const double2*>(x),
      reinterpret_cast<double2*>(Fp), reinterpret_cast<double2*>(Gp),
      reinterpret_cast<double2*>(dF), reinterpret_cast<double2*>(dG), first);
  RT_CHECK_LAUNCH();
}

int anderson_partials() { return 148 * 4; }

void anderson_dots(int64_t n, const double* dF, const double* f, int count, double* partial,
                   double* out, cudaStream_t st) {
  const int np = anderson_partials();
  anderson_dots_pass1<<<np, kThreads, 0, st>>>(n, reinterpret_cast<const double2*>(dF), n,
                                               reinterpret_cast<const double2*>(f), count,
                                               reinterpret_cast<double2*>(partial));
  RT_CHECK_LAUNCH();
  anderson_dots_pass2<<<1, 32, 0, st>>>(reinterpret_cast<const double2*>(partial), np,
                                        reinterpret_cast<double2*>(out));
  RT_CHECK_LAUNCH();
}

void anderson_mix(int64_t n, const double* g, const double* dG, int count, const double* gamma,
                  double* x, cudaStream_t st) {
  if (n == 0) return;
  const double2 g0 = make_double2(gamma[0], gamma[1]), g1 = make_double2(gamma[2], gamma[3]),
                g2 = make_double2(gamma[4], gamma[5]);
  anderson_mix_kernel<<<grid_for(n, 16), kThreads, 0, st>>>(
      n, reinterpret_cast<const double2*>(g), reinterpret_cast<const double2*>(dG), n, count, g0,
      g1, g2, reinterpret_cast<double2*>(x));
  RT_CHECK_LAUNCH();
}

void mask_pads(const AmpGeom& g, double* t, cudaStream_t st) {
  mask_kernel<<<grid_for(g.total(), 16), kThreads, 0, st>>>(g, reinterpret_cast<double2*>(t));
  RT_CHECK_LAUNCH();
}

int energy_partials(const AmpGeom& g) { return grid_for(g.n2() > g.n1() ? g.n2() : g.n1(), 4); }

void energy(const AmpGeom& g, const double* t, const double* ovov, const double* fov_a,
            const double* fov_b, int include_fov, double* partial, double* E_hist, double* C_hist,
            long long n, double dt, int update_c, cudaStream_t st) {
  int np = energy_partials(g);
  energy_pass1<<<np, kThreads, 0, st>>>(g, reinterpret_cast<const double2*>(t), ovov, fov_a,
                                        fov_b, include_fov, reinterpret_cast<double2*>(partial));
  RT_CHECK_LAUNCH();
  energy_pass2<<<1, kThreads, 0, st>>>(reinterpret_cast<const double2*>(partial), np,
                                       reinterpret_cast<double2*>(E_hist),
                                       reinterpret_cast<double2*>(C_hist), n, dt, update_c);
  RT_CHECK_LAUNCH();
}

void scatter_unpadded(const AmpGeom& g, const long long* idx, const double* val, int64_t n,
                      double* padded, cudaStream_t st) {
  if (n <= 0) return;
  scatter_unpadded_kernel<<<grid_for(n, 1), kThreads, 0, st>>>(
      g, idx, reinterpret_cast<const double2*>(val), n, reinterpret_cast<double2*>(padded));
  RT_CHECK_LAUNCH();
}

void gather_unpadded(const AmpGeom& g, const double* padded, const long long* idx, int64_t n,
                     double* out, cudaStream_t st) {
  if (n <= 0) return;
  gather_unpadded_kernel<<<grid_for(n, 1), kThreads, 0, st>>>(
      g, reinterpret_cast<const double2*>(padded), idx, n, reinterpret_cast<double2*>(out));
  RT_CHECK_LAUNCH();
}

void pack_amplitudes(const AmpGeom& g, const double* unpadded, double* padded, cudaStream_t st) {
  pack_kernel<<<grid_for(g.total(), 16), kThreads, 0, st>>>(
      g, reinterpret_cast<const double2*>(unpadded), reinterpret_cast<double2*>(padded));
  RT_CHECK_LAUNCH();
}

void unpack_amplitudes(const AmpGeom& g, const double* padded, double* unpadded, cudaStream_t st) {
  unpack_kernel<<<grid_for(g.total(), 16), kThreads, 0, st>>>(
      g, reinterpret_cast<const double2*>(padded), reinterpret_cast<double2*>(unpadded));
  RT_CHECK_LAUNCH();
}

void gather_cholesky(const double* L, int nchol, int nO, int nV, int core, double* Loo,
                     double* Lov, double* Lvv, cudaStream_t st) {
  int64_t total = ((int64_t)nO * nO + (int64_t)nO * nV + (int64_t)nV * nV) * nchol;
  if (total == 0) return;
  gather_L_kernel<<<grid_for(total, 16), kThreads, 0, st>>>(L, nchol, nO, nV, core, Loo, Lov, Lvv);
  RT_CHECK_LAUNCH();
}

void build_fock(const double* eps, const double* L, int nchol, int nO, int nV, int core,
                double* foo_a, double* fov_a, double* fvv_a, double* foo_b, double* fov_b,
                double* fvv_b, double* fo_a, double* fv_a, double* fo_b, double* fv_b,
                cudaStream_t st) {
  int64_t per = (int64_t)nO * nO + (int64_t)nO * nV + (int64_t)nV * nV;
  fock_kernel<<<grid_for(2 * per, 16), kThreads, 0, st>>>(eps, L, nchol, nO, nV, core, foo_a,
                                                          fov_a, fvv_a, foo_b, fov_b, fvv_b);
  RT_CHECK_LAUNCH();
  int n = nO > nV ? nO : nV;
  diag_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(foo_a, fvv_a, foo_b, fvv_b, nO,
                                                                  nV, fo_a, fv_a, fo_b, fv_b);
  RT_CHECK_LAUNCH();
}

void closed_shell_ecorr(const double* ovov, const double* t1, const double* t2, int O, int V,
                        double* partial, double* out, cudaStream_t st) {
  int64_t n = (int64_t)O * O * V * V;
  int np = grid_for(n, 4);
  ecorr_pass1<<<np, kThreads, 0, st>>>(ovov, t1, t2, O, V, reinterpret_cast<double2*>(partial));
  RT_CHECK_LAUNCH();
  ecorr_pass2<<<1, kThreads, 0, st>>>(reinterpret_cast<const double2*>(partial), np, out);
  RT_CHECK_LAUNCH();
}

void spectrum(const double* C, long long M, double dt, double shift, const double* omega,
              int nomega, double eta, double* A, cudaStream_t st) {
  if (nomega <= 0) return;
  spectrum_kernel<<<nomega, kThreads, 0, st>>>(reinterpret_cast<const double2*>(C), M, dt, shift,
                                               omega, eta, A);
  RT_CHECK_LAUNCH();
}

void maxabs_bits(const double* x, int64_t n, unsigned long long* out, cudaStream_t st) {
  if (n == 0) return;
  maxabs_kernel<<<grid_for(n, 8), kThreads, 0, st>>>(x, n, out);
  RT_CHECK_LAUNCH();
}

}  // namespace rteom
