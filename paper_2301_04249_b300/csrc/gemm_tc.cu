// Split-TF32 tensor-core GEMM on tcgen05 (sm_103a) for the contraction engine.
//
// Every engine GEMM C = alpha op(A) op(B) + beta C (A, B real or complex
// FP64) becomes one real GEMM D = A' B'^T:
//   real x real        A' = A,                 B'^T = B
//   complex x real     A' = [Re A ; Im A] (rows), B'^T = B
//   real x complex     A' = A,                 B'^T = [Re B | Im B] (columns)
//   complex x complex  A' = [Re A | Im A] (K),  B'^T = [[Re B, Im B], [-Im B, Re B]]
// Each operand is packed once per call by `tc_pack` into TF32 hi/lo parts
// (x = hi + lo, hi = tf32(x), lo = tf32(x - hi)), laid out as 128-row x 32-col
// tiles of 8x4 core matrices (K-major, no swizzle), each tile contiguous so a
// stage is four 16 KB bulk copies.  The product hi*hi + hi*lo + lo*hi is
// accumulated in FP32 in tensor memory over slices of at most 512 of K; the
// epilogue warps add every slice into compensated FP32 pairs (TwoSum, about
// 48 bits) while the next slice accumulates in the other half of the tensor
// memory.  A CTA owns one output tile and a contiguous range of K; with one
// range it writes alpha*acc + beta*C straight into the FP64 (complex)
// output, otherwise it writes its (sum, compensation) pair and `tc_finalize`
// combines the ranges in order (deterministic).  The FP64 pipe of this part
// is slow, so conversions use integer bit operations and FP64 arithmetic is
// spent only on a general alpha and a non-zero beta.
//
// Warp roles (320 threads): warp 0 lane 0 issues the bulk copies, warp 1 owns
// the tensor-memory allocation and lane 0 issues the MMAs, warps 2-9 drain
// the accumulator (warp w reads lanes 32*(w%4)..+31, half (w-2)/4 of the
// columns).  Every mbarrier wait is bounded by a clock budget; on expiry the
// CTA records an error code, lets its copies land, frees its tensor memory
// and returns.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace rteom {

namespace tc {

using namespace tc5;

constexpr int BM = 128;   // rows of A' per tile (TMEM lanes)
constexpr int BK = 32;    // K per stage (tf32 elements, 128 bytes)
constexpr int TILE_ELEMS = BM * BK;            // 4096 floats
constexpr uint32_t TILE_BYTES = TILE_ELEMS * 4;  // 16 KB
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int kSliceKt = 16;  // k-tiles per FP32 accumulation slice (512 of K)
// row tiles per rasterization group: 148 CTAs in flight cover about 12 x 12
// square 128 x 128 output tiles
constexpr int kGroupM = 12;

// Instruction descriptor of kind::tf32: F32 accumulator, TF32 A and B, both
// K-major, N = bn, M = 128.
__host__ __device__ constexpr uint32_t idesc_tf32(int bn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(bn >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

struct KArgs {
  const float *Ahi, *Alo, *Bhi, *Blo;  // packed tiles: [batch][rowtile][ktile][4096]
  int64_t sA, sB;                      // per-batch element strides of the packed operands
  int KT;                              // k-tiles per row tile
  int kpr;                             // k-tiles per K range
  int ranges;                          // K ranges (CTAs along K per tile)
  int zs;                              // batch * ranges (work items per output tile)
  float2* P;         // (sum, compensation) partials [batch*ranges][Mp][Np] when ranges > 1
  bool force_p;      // partials even with one range (3M products)
  int Mp, Np;        // padded extents of the partials
  uint32_t lbo, sbo;
  int* err;          // set to a non-zero code when a wait runs out
  long long wait;    // budget (clock cycles) of the MMA and epilogue waits
  // output (single range): alpha*acc + beta*C into the FP64 output
  double* C;
  bool cplx;
  int M, N, mode;    // logical output extents; mode 0 real, 1 stacked rows, 2 stacked cols
  int64_t ldm, ldn, sC;  // output strides of GEMM rows and columns, batch
  OutModes out;  // C = alpha D + beta C
};

template <int BN, int STAGES>
__global__ void __launch_bounds__(THREADS, 1) tc_gemm_kernel(KArgs g) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr uint32_t A_BYTES = TILE_BYTES;
  constexpr uint32_t B_BYTES = (uint32_t)BN * BK * 4;
  constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  constexpr int HALF = BN / 2;  // columns drained by one epilogue warp
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;  // [2]: slice accumulated in buffer i
  uint64_t* acc_empty = acc_full + 2;   // [2]: buffer i drained by the epilogue
  uint64_t* mma_done = acc_empty + 2;   // teardown: every issued MMA finished
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int* issued = abort_flag + 1;  // bulk-load stages issued by the producer
  int* mmas = issued + 1;        // stages whose MMAs the issuer launched

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // Persistent CTAs: work item w = z * tiles + t (t the output tile in
  // rasterization order, z = batch * ranges + K range), CTA c takes items
  // c, c + gridDim.x, ...  The pipeline counters (k tiles for the stage
  // ring, slices for the two accumulator buffers) run on across items, so a
  // tile's drain overlaps the next tile's MMAs.
  const int m_tiles = g.Mp / BM, n_tiles = g.Np / BN;
  const int tiles = m_tiles * n_tiles;
  const int items = tiles * g.zs;
  struct Item {
    int m_tile, n_tile, z, b, kt0, nk, nslices;
  };
  auto item_of = [&](int w) {
    Item it;
    it.z = w / tiles;
    grouped_tile(w - it.z * tiles, m_tiles, n_tiles, kGroupM, &it.m_tile, &it.n_tile);
    it.b = it.z / g.ranges;
    const int rg = it.z % g.ranges;
    it.kt0 = rg * g.kpr;
    it.nk = max(min(g.KT, it.kt0 + g.kpr) - it.kt0, 0);
    it.nslices = (it.nk + kSliceKt - 1) / kSliceKt;
    return it;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], EPI_WARPS);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    *issued = 0;
    *mmas = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, 2 * BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: stage s holds Ahi, Alo, Bhi, Blo of one k-tile
    int kg = 0;  // k tiles issued so far (all items)
    for (int w = blockIdx.x; w < items && !*(volatile int*)abort_flag; w += gridDim.x) {
      const Item it = item_of(w);
      const float* Ahi = g.Ahi + it.b * g.sA + (int64_t)it.m_tile * g.KT * TILE_ELEMS;
      const float* Alo = g.Alo + it.b * g.sA + (int64_t)it.m_tile * g.KT * TILE_ELEMS;
      const float* Bhi = g.Bhi + it.b * g.sB + (int64_t)it.n_tile * g.KT * (BN * BK);
      const float* Blo = g.Blo + it.b * g.sB + (int64_t)it.n_tile * g.KT * (BN * BK);
      for (int k = 0; k < it.nk; ++k, ++kg) {
        const int s = kg % STAGES;
        if (kg >= STAGES &&
            !mbar_wait_or_abort(&empty[s], ((kg / STAGES) - 1) & 1, abort_flag)) {
          if (!*(volatile int*)abort_flag) atomicExch(g.err, 1);
          *abort_flag = 1;
          break;
        }
        uint8_t* st = smem + s * STAGE_BYTES;
        const int kt = it.kt0 + k;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        bulk_load(st, Ahi + (int64_t)kt * TILE_ELEMS, A_BYTES, &full[s]);
        bulk_load(st + A_BYTES, Alo + (int64_t)kt * TILE_ELEMS, A_BYTES, &full[s]);
        bulk_load(st + 2 * A_BYTES, Bhi + (int64_t)kt * (BN * BK), B_BYTES, &full[s]);
        bulk_load(st + 2 * A_BYTES + B_BYTES, Blo + (int64_t)kt * (BN * BK), B_BYTES, &full[s]);
        *issued = kg + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 K-steps of 8 per stage, three hi/lo products each; slice
    // jg (counted over all items) accumulates in tensor-memory buffer jg % 2
    const uint32_t idesc = idesc_tf32(BN);
    int kg = 0, jg = 0;
    bool stop = false;
    for (int w = blockIdx.x; w < items && !stop; w += gridDim.x) {
      const Item it = item_of(w);
      for (int k = 0; k < it.nk; ++k, ++kg) {
        const int kin = k % kSliceKt;
        const int j = jg + k / kSliceKt, buf = j & 1;
        if (kin == 0 && j >= 2) {
          if (!mbar_wait(&acc_empty[buf], ((j >> 1) - 1) & 1, g.wait)) {
            *abort_flag = 1;
            atomicExch(g.err, 4);
            stop = true;
            break;
          }
        }
        const int s = kg % STAGES;
        if (!mbar_wait(&full[s], (kg / STAGES) & 1, g.wait)) {
          *abort_flag = 1;
          atomicExch(g.err, 2);
          stop = true;
          break;
        }
        tc_fence_after();
        *mmas = kg + 1;
        const uint32_t dt = tmem + (uint32_t)(buf * BN);
        const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
        const uint32_t a_hi = base, a_lo = base + A_BYTES;
        const uint32_t b_hi = base + 2 * A_BYTES, b_lo = b_hi + B_BYTES;
#pragma unroll
        for (int q = 0; q < BK / 8; ++q) {
          const uint32_t off = q * 256;  // two 16-byte core matrices along K
          const uint64_t ah = smem_desc(a_hi + off, g.lbo, g.sbo);
          const uint64_t al = smem_desc(a_lo + off, g.lbo, g.sbo);
          const uint64_t bh = smem_desc(b_hi + off, g.lbo, g.sbo);
          const uint64_t bl = smem_desc(b_lo + off, g.lbo, g.sbo);
          mma_tf32(dt, ah, bh, idesc, (kin > 0 || q > 0) ? 1u : 0u);
          mma_tf32(dt, ah, bl, idesc, 1u);
          mma_tf32(dt, al, bh, idesc, 1u);
        }
        mma_commit(&empty[s]);
        if (kin == kSliceKt - 1 || k == it.nk - 1) mma_commit(&acc_full[buf]);
      }
      jg += it.nslices;
    }
  } else if (warp >= 2) {
    // epilogue: row r of the tile lives in TMEM lane r; this warp adds the
    // columns [h*HALF, (h+1)*HALF) of every slice into compensated pairs
    const int q = warp % 4;
    const int h = (warp - 2) / 4;
    const int row = 32 * q + lane;
    int jg = 0;
    for (int w = blockIdx.x; w < items; w += gridDim.x) {
      const Item it = item_of(w);
      float sum[HALF], cmp[HALF];
#pragma unroll
      for (int v = 0; v < HALF; ++v) sum[v] = cmp[v] = 0.0f;
      bool ok = it.nk > 0 && !*(volatile int*)abort_flag;
#pragma unroll 1
      for (int jl = 0; ok && jl < it.nslices; ++jl) {
        const int j = jg + jl, buf = j & 1;
        if (!mbar_wait(&acc_full[buf], (j >> 1) & 1, g.wait)) {
          ok = false;
          *abort_flag = 1;
          atomicExch(g.err, 3);
          break;
        }
        tc_fence_after();
        const uint32_t taddr =
            tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN + h * HALF);
#pragma unroll
        for (int c = 0; c < HALF / 32; ++c) {
          uint32_t r[32];
          tmem_ld32(taddr + (uint32_t)(c * 32), r);
#pragma unroll
          for (int v = 0; v < 32; ++v)
            two_sum_acc(sum[c * 32 + v], cmp[c * 32 + v], __uint_as_float(r[v]));
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
      }
      jg += it.nslices;
      if (!ok) break;
      if (g.ranges == 1 && !g.force_p) {
        // map (row', col') of D = A'B'^T onto one real or imaginary part of C
        const int mr = it.m_tile * BM + row;
        int m = mr, part = 0;
        if (g.mode == 1 && mr >= g.M) {
          m = mr - g.M;
          part = 1;
        }
        const bool row_ok = g.mode == 1 ? mr < 2 * g.M : mr < g.M;
        if (row_ok) {
          const int64_t rbase = (int64_t)it.b * g.sC + (int64_t)m * g.ldm;
          with_out_modes(g.out, [&](auto ga, auto bm) {
            constexpr int GA = decltype(ga)::value, BMODE = decltype(bm)::value;
#pragma unroll
            for (int v = 0; v < HALF; ++v) {
              const int nr = it.n_tile * BN + h * HALF + v;
              int n = nr, pt = part;
              if (g.mode == 2 && nr >= g.N) {
                n = nr - g.N;
                pt = 1;
              }
              if (n >= g.N || (g.mode == 2 ? nr >= 2 * g.N : nr >= g.N)) continue;
              out_update<GA, BMODE>(g.C + (g.cplx ? 2 : 1) * (rbase + (int64_t)n * g.ldn) + pt,
                                    f32_to_f64(sum[v] + cmp[v]), g.out);
            }
          });
        }
      } else {
        float4* dst = reinterpret_cast<float4*>(
            g.P + ((int64_t)it.z * g.Mp + (int64_t)it.m_tile * BM + row) * g.Np +
            (int64_t)it.n_tile * BN + h * HALF);
#pragma unroll
        for (int v = 0; v < HALF / 2; ++v)
          dst[v] = make_float4(sum[2 * v], cmp[2 * v], sum[2 * v + 1], cmp[2 * v + 1]);
      }
    }
  }
  // teardown after an abandoned pipeline: let the issued copies land and the
  // issued MMAs finish (bounded) before the tensor memory is freed
  tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) {
      const int n = *issued;
      for (int k = n > STAGES ? n - STAGES : 0; k < n; ++k)
        mbar_wait(&full[k % STAGES], (k / STAGES) & 1);
    }
    if (warp == 1 && lane == 0 && *mmas > 0) {
      mma_commit(mma_done);
      mbar_wait(mma_done, 0);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * BN);
  }
}

// ---------------------------------------------------------------- packing
// Source element (r, c) of a logical operand matrix, read with strides.
struct PackArgs {
  const double* src;
  bool cplx;
  int64_t s_r, s_c, s_b;  // element strides of logical rows, columns, batch
  int R, C;               // logical extents of the source operand (rows x K)
  int mode;               // see PackMode
  int part;               // complex source read as one real part (0 re, 1 im, 2 re+im), or -1
  int Rp, Kp;             // packed (padded) extents: rows multiple of rowtile, K of 32
  int rowtile;            // 128 for A', BN for B'
  float *hi, *lo;
  int64_t s_out;          // elements per batch entry of the packed output
  bool rows_fast;         // consecutive threads walk packed rows (source rows contiguous)
  View2 view;             // strided source view (view.rdims > 0) instead of s_r / s_c
};

// Packed row r' / column k' -> (source row, source column, part, sign).
enum PackMode {
  kPlain = 0,       // real source
  kStackRows = 1,   // complex: rows [Re; Im]
  kStackK = 2,      // complex: K [Re | Im]
  kBcc = 3,         // complex B of a complex x complex product
};

// Value of the embedded real operand at packed (row rp, column kp), FP32.
__device__ __forceinline__ float packed_value(const PackArgs& p, int b, int rp, int kp) {
  int r = rp, c = kp, part = 0;
  bool neg = false;
  bool valid = true;
  switch (p.mode) {
    case kPlain:
      valid = rp < p.R && kp < p.C;
      break;
    case kStackRows:
      part = rp >= p.R;
      r = rp - part * p.R;
      valid = rp < 2 * p.R && kp < p.C;
      break;
    case kStackK:
      part = kp >= p.C;
      c = kp - part * p.C;
      valid = rp < p.R && kp < 2 * p.C;
      break;
    default: {  // kBcc: rows n' (output columns), K' = [K | K]
      const int ro = rp >= p.R, ko = kp >= p.C;
      r = rp - ro * p.R;
      c = kp - ko * p.C;
      valid = rp < 2 * p.R && kp < 2 * p.C;
      // [[Re, Im], [-Im, Re]] indexed by (k-half, n-half): part = Im when halves differ
      part = ro != ko;
      neg = ko && !ro;
    }
  }
  if (!valid) return 0.0f;
  const int64_t off = b * p.s_b + (p.view.rdims ? view_row(p.view, r) + view_col(p.view, c)
                                                 : r * p.s_r + c * p.s_c);
  float xf;
  if (p.part >= 0) {
    const double* q = p.src + 2 * off;
    xf = f64_to_f32(p.part == 2 ? q[0] + q[1] : q[p.part]);
  } else {
    xf = f64_to_f32(p.cplx ? p.src[2 * off + part] : p.src[off]);
  }
  return neg ? -xf : xf;
}

// x ~ hi + lo: hi = tf32(x), lo = tf32(x - hi) (the difference is exact in FP32)
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  uint32_t hb, lb;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(x));
  hi = __uint_as_float(hb);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"(x - hi));
  lo = __uint_as_float(lb);
}

// Packed layout: tile (row tile rt, k tile kt) of rowtile x 32 is contiguous;
// inside it the core matrix (8 rows x 4 k) of row group rr/8 and k quad kq
// sits at ((rr/8)*8 + kq)*32 floats, row rr%8 at 4 floats: one thread writes
// one 16-byte row of a core matrix.  A warp packs one block of 32 rows x 32 k
// when the source rows are contiguous (lane = row: each load coalesced across
// the warp), else one block of 8 rows x 32 k (lane = row r/8-th quarter and k
// quad: each lane loads 4 consecutive k).
__global__ void tc_pack_kernel(PackArgs p, int batch) {
  const int KT = p.Kp / BK;
  const int rows_per = p.rows_fast ? 32 : 8;
  const int64_t groups = (int64_t)(p.Rp / rows_per) * KT;  // blocks per batch entry
  const int64_t units = groups * batch;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < units; w += nwarps) {
    const int b = (int)(w / groups);
    const int64_t gq = w - (int64_t)b * groups;
    const int rg = (int)(gq / KT), kt = (int)(gq % KT);
    float* hi_t = p.hi + (int64_t)b * p.s_out;
    float* lo_t = p.lo + (int64_t)b * p.s_out;
    if (p.rows_fast) {
      const int rp = rg * 32 + lane;
      const int rt = rp / p.rowtile, rr = rp % p.rowtile;
      const int64_t tile = ((int64_t)rt * KT + kt) * ((int64_t)p.rowtile * BK);
#pragma unroll 2
      for (int kq = 0; kq < BK / 4; ++kq) {
        float4 h, l;
        tf32_split(packed_value(p, b, rp, kt * BK + kq * 4 + 0), h.x, l.x);
        tf32_split(packed_value(p, b, rp, kt * BK + kq * 4 + 1), h.y, l.y);
        tf32_split(packed_value(p, b, rp, kt * BK + kq * 4 + 2), h.z, l.z);
        tf32_split(packed_value(p, b, rp, kt * BK + kq * 4 + 3), h.w, l.w);
        const int64_t dst = tile + ((rr / 8) * 8 + kq) * 32 + (rr % 8) * 4;
        *reinterpret_cast<float4*>(hi_t + dst) = h;
        *reinterpret_cast<float4*>(lo_t + dst) = l;
      }
    } else {
      const int kq = lane & 7;
#pragma unroll
      for (int pass = 0; pass < 2; ++pass) {
        const int rp = rg * 8 + pass * 4 + (lane >> 3);
        const int rt = rp / p.rowtile, rr = rp % p.rowtile;
        const int k0 = kt * BK + kq * 4;
        float4 h, l;
        tf32_split(packed_value(p, b, rp, k0 + 0), h.x, l.x);
        tf32_split(packed_value(p, b, rp, k0 + 1), h.y, l.y);
        tf32_split(packed_value(p, b, rp, k0 + 2), h.z, l.z);
        tf32_split(packed_value(p, b, rp, k0 + 3), h.w, l.w);
        const int64_t dst = ((int64_t)rt * KT + kt) * ((int64_t)p.rowtile * BK) +
                            ((rr / 8) * 8 + kq) * 32 + (rr % 8) * 4;
        *reinterpret_cast<float4*>(hi_t + dst) = h;
        *reinterpret_cast<float4*>(lo_t + dst) = l;
      }
    }
  }
}

// ---------------------------------------------------------------- finalize
struct FinArgs {
  const float2* P;  // (sum, compensation) [batch*ranges][Mp][Np]
  int Mp, Np, ranges;
  int M, N;        // logical output extents
  int mode;        // 0 real, 1 stacked rows (C re/im = row halves), 2 stacked columns
  double* C;
  bool cplx;
  int64_t ldm, ldn, sC;  // output strides of GEMM rows and columns, batch
  OutModes out;          // C = alpha D + beta C
};

__global__ void tc_finalize_kernel(FinArgs f, int batch) {
  const int64_t per = (int64_t)f.M * f.N;
  with_out_modes(f.out, [&](auto ga, auto bm) {
    constexpr int GA = decltype(ga)::value, BMODE = decltype(bm)::value;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * batch;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int b = (int)(e / per);
      const int64_t q = e - (int64_t)b * per;
      const int m = (int)(q / f.N), n = (int)(q % f.N);
      double* c = f.C + (f.cplx ? 2 : 1) * ((int64_t)b * f.sC + (int64_t)m * f.ldm + (int64_t)n * f.ldn);
      const int parts = f.cplx ? 2 : 1;
      for (int part = 0; part < parts; ++part) {
        int mr = m, nr = n;
        if (f.mode == 1) mr = m + part * f.M;
        if (f.mode == 2) nr = n + part * f.N;
        float s = 0.0f, cm = 0.0f;
        // ranges in order, four loads in flight at a time
        const float2* pp = f.P + ((int64_t)b * f.ranges * f.Mp + mr) * f.Np + nr;
        const int64_t zs = (int64_t)f.Mp * f.Np;
        int z = 0;
        for (; z + 4 <= f.ranges; z += 4) {
          float2 q[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) q[u] = pp[(z + u) * zs];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            two_sum_acc(s, cm, q[u].x);
            cm += q[u].y;
          }
        }
        for (; z < f.ranges; ++z) {
          const float2 pz = pp[z * zs];
          two_sum_acc(s, cm, pz.x);
          cm += pz.y;
        }
        out_update<GA, BMODE>(c + part, f32_to_f64(s + cm), f.out);
      }
    }
  });
}

constexpr int kBN = 128;
constexpr int kStages = 3;
constexpr size_t kSmemBytes = kStages * (2 * TILE_BYTES + 2 * (size_t)kBN * BK * 4) + 256;

inline int roundup(int x, int m) { return (x + m - 1) / m * m; }

struct Plan {
  int mode;  // 0 RR, 1 CR, 2 RC, 3 CC
  int Mp, Np, Kp, KT, ranges, kpr;
  int64_t a_elems, b_elems;  // per operand part (hi or lo)
  int64_t p_elems;           // (sum, compensation) partials (0 with one range)
};

Plan plan(const GemmDesc& d) {
  Plan p;
  p.mode = (d.Acplx && d.part_a < 0 ? 1 : 0) + (d.Bcplx && d.part_b < 0 ? 2 : 0);
  const int Ar = p.mode == 1 ? 2 * d.M : d.M;
  const int Ak = p.mode == 3 ? 2 * d.K : d.K;
  const int Br = (p.mode & 2) ? 2 * d.N : d.N;
  p.Mp = roundup(std::max(Ar, 1), BM);
  p.Np = roundup(std::max(Br, 1), kBN);
  p.Kp = roundup(std::max(Ak, 1), BK);
  p.KT = p.Kp / BK;
  // K ranges: fewest waves x k-tiles per CTA, a range costing about four
  // k-tiles for writing and re-reading its partial tile
  const int64_t tiles = (int64_t)(p.Mp / BM) * (p.Np / kBN) * d.batch;
  double best = 0.0;
  p.ranges = 1;
  p.kpr = p.KT;
  for (int r = 1; r <= p.KT; ++r) {
    const int kpr = (p.KT + r - 1) / r;
    if ((p.KT + kpr - 1) / kpr != r) continue;  // same split as a smaller r
    if ((int64_t)d.batch * r > 65535) break;
    const double waves = (double)((tiles * r + 147) / 148);
    const double cost = waves * (kpr + (r > 1 ? 4 : 0));
    if (r == 1 || cost < best) {
      best = cost;
      p.ranges = r;
      p.kpr = kpr;
    }
  }
  p.a_elems = (int64_t)p.Mp * p.Kp * d.batch;
  p.b_elems = (int64_t)p.Np * p.Kp * d.batch;
  p.p_elems = (p.ranges == 1 && !d.force_partials) ? 0 : (int64_t)p.ranges * p.Mp * p.Np * d.batch;
  return p;
}

// 3M combine: P holds [3][ranges][Mp][Np] (sum, compensation) pairs of the
// products P1 = Re A Re B, P2 = Im A Im B, P3 = (Re A + Im A)(Re B + Im B);
// C = alpha (P1 - P2 + i (P3 - P1 - P2)) + beta C, the ranges summed in order.
__global__ void tc_combine_3m_kernel(FinArgs f) {
  const int64_t per = (int64_t)f.M * f.N;
  const int64_t zs = (int64_t)f.Mp * f.Np;
  // the partials and the output never overlap
  const float2* __restrict__ Pr = f.P;
  double* __restrict__ Cr = f.C;
  with_out_modes(f.out, [&](auto ga, auto bm) {
    constexpr int GA = decltype(ga)::value, BMODE = decltype(bm)::value;
#pragma unroll 2
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int m = (int)(e / f.N), n = (int)(e % f.N);
      // products as compensated FP32 pairs (s, c); the differences are formed
      // with TwoSum on the leading parts, so only the final value takes an
      // FP64 add (the FP64 pipe is the scarce unit)
      float s[3], cm[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float2* pp = Pr + ((int64_t)b * f.ranges * f.Mp + m) * f.Np + n;
        s[b] = 0.0f;
        cm[b] = 0.0f;
        for (int z = 0; z < f.ranges; ++z) {
          const float2 q = pp[z * zs];
          two_sum_acc(s[b], cm[b], q.x);
          cm[b] += q.y;
        }
      }
      float re_h = s[0], re_l = cm[0] - cm[1];
      two_sum_acc(re_h, re_l, -s[1]);                 // P1 - P2
      float im_h = s[2], im_l = cm[2] - cm[0] - cm[1];
      two_sum_acc(im_h, im_l, -s[0]);
      two_sum_acc(im_h, im_l, -s[1]);                 // P3 - P1 - P2
      const double re = f32_to_f64(re_h) + f32_to_f64(re_l);
      const double im = f32_to_f64(im_h) + f32_to_f64(im_l);
      double* c = Cr + 2 * ((int64_t)m * f.ldm + (int64_t)n * f.ldn);
      out_update<GA, BMODE>(c, re, f.out);
      out_update<GA, BMODE>(c + 1, im, f.out);
    }
  });
}

}  // namespace tc

TcLayout gemm_tc_layout(const GemmDesc& d) {
  tc::Plan p = tc::plan(d);
  TcLayout l;
  l.a_elems = p.a_elems;
  l.b_elems = p.b_elems;
  l.p_elems = p.p_elems;
  l.ranges = p.ranges;
  l.padded_flops = 3LL * 2 * (int64_t)p.Mp * p.Np * p.Kp * d.batch;
  return l;
}

void gemm_tc_init() {
  RT_CUDA(cudaFuncSetAttribute(tc::tc_gemm_kernel<tc::kBN, tc::kStages>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tc::kSmemBytes));
}

namespace {
int grid_of(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 148 * 16); }

void launch_pack(const tc::PackArgs& pa, int64_t elems, int batch, cudaStream_t st) {
  // one warp per block of 32 x 32 (rows-fast) or 8 x 32 packed elements
  const int64_t units = elems / (pa.rows_fast ? 1024 : 256);
  const int grid = (int)std::min<int64_t>((units * 32 + 255) / 256, 148 * 16);
  tc::tc_pack_kernel<<<std::max(grid, 1), 256, 0, st>>>(pa, batch);
  RT_CHECK_LAUNCH();
}
}  // namespace

void gemm_tc_pack_a(const GemmDesc& d, float* hi, float* lo, cudaStream_t st) {
  using namespace tc;
  if (d.M <= 0 || d.N <= 0 || d.batch <= 0) return;
  const Plan p = plan(d);
  PackArgs pa{};
  pa.src = d.A;
  pa.cplx = d.Acplx;
  pa.s_r = d.transA ? 1 : d.lda;
  pa.s_c = d.transA ? d.lda : 1;
  pa.s_b = d.strideA;
  pa.R = d.M;
  pa.C = d.K;
  pa.mode = p.mode == 1 ? kStackRows : (p.mode == 3 ? kStackK : kPlain);
  pa.part = d.Acplx ? d.part_a : -1;
  pa.Rp = p.Mp;
  pa.Kp = p.Kp;
  pa.rowtile = BM;
  pa.hi = hi;
  pa.lo = lo;
  pa.s_out = (int64_t)p.Mp * p.Kp;
  pa.view = d.va;
  pa.rows_fast = d.va.rdims ? (d.va.rstr[d.va.rdims - 1] == 1 && d.va.kstr[d.va.kdims - 1] != 1)
                            : (pa.s_r == 1 && pa.s_c != 1);
  launch_pack(pa, p.a_elems, d.batch, st);
}

void gemm_tc_pack_b(const GemmDesc& d, float* hi, float* lo, cudaStream_t st) {
  using namespace tc;
  if (d.M <= 0 || d.N <= 0 || d.batch <= 0) return;
  const Plan p = plan(d);
  PackArgs pb{};
  pb.src = d.B;
  pb.cplx = d.Bcplx;
  pb.s_r = d.transB ? d.ldb : 1;  // rows of B' are the output columns n
  pb.s_c = d.transB ? 1 : d.ldb;
  pb.s_b = d.strideB;
  pb.R = d.N;
  pb.C = d.K;
  pb.mode = p.mode == 2 ? kStackRows : (p.mode == 3 ? kBcc : kPlain);
  pb.part = d.Bcplx ? d.part_b : -1;
  pb.Rp = p.Np;
  pb.Kp = p.Kp;
  pb.rowtile = kBN;
  pb.hi = hi;
  pb.lo = lo;
  pb.s_out = (int64_t)p.Np * p.Kp;
  pb.view = d.vb;
  pb.rows_fast = d.vb.rdims ? (d.vb.rstr[d.vb.rdims - 1] == 1 && d.vb.kstr[d.vb.kdims - 1] != 1)
                            : (pb.s_r == 1 && pb.s_c != 1);
  launch_pack(pb, p.b_elems, d.batch, st);
}

void gemm_tc_mma(const GemmDesc& d, const float* Ahi, const float* Alo, const float* Bhi,
                 const float* Blo, float2* P, int* err, cudaStream_t st) {
  using namespace tc;
  if (d.M <= 0 || d.N <= 0 || d.batch <= 0) return;
  const Plan p = plan(d);
  if ((int64_t)(p.Np / kBN) * (p.Mp / BM) > 0x7fffffff || (int64_t)d.batch * p.ranges > 65535)
    throw Error(-1, "gemm_tc: grid too large");
  KArgs g{};
  g.Ahi = Ahi;
  g.Alo = Alo;
  g.Bhi = Bhi;
  g.Blo = Blo;
  g.sA = (int64_t)p.Mp * p.Kp;
  g.sB = (int64_t)p.Np * p.Kp;
  g.KT = p.KT;
  g.kpr = p.kpr;
  g.ranges = p.ranges;
  g.P = P;
  g.force_p = d.force_partials;
  g.Mp = p.Mp;
  g.Np = p.Np;
  g.lbo = 128;   // core matrices adjacent along K
  g.sbo = 1024;  // 8-row groups
  g.err = err;
  g.wait = d.wait_cycles > 0 ? d.wait_cycles : tc5::kWaitCycles;
  g.C = d.C;
  g.cplx = d.Acplx || d.Bcplx;
  g.M = d.M;
  g.N = d.N;
  g.mode = p.mode == 1 ? 1 : (p.mode >= 2 ? 2 : 0);
  g.ldm = d.transC ? 1 : d.ldc;
  g.ldn = d.transC ? d.ldc : 1;
  g.sC = d.strideC;
  g.out = out_modes(d.alpha, d.beta);
  g.zs = d.batch * p.ranges;
  // persistent CTAs: one per SM (the kernel takes most of the shared memory)
  const int64_t items = (int64_t)(p.Np / kBN) * (p.Mp / BM) * g.zs;
  if (items > 0x7fffffff) throw Error(-1, "gemm_tc: too many tiles");
  const int grid = (int)std::min<int64_t>(items, 148);
  tc_gemm_kernel<kBN, kStages><<<grid, THREADS, kSmemBytes, st>>>(g);
  RT_CHECK_LAUNCH();
}

void gemm_tc_finalize(const GemmDesc& d, const float2* P, cudaStream_t st) {
  using namespace tc;
  if (d.M <= 0 || d.N <= 0 || d.batch <= 0) return;
  const Plan p = plan(d);
  if (p.ranges == 1 && !d.force_partials) return;  // the MMA kernel wrote C directly
  FinArgs fa{};
  fa.P = P;
  fa.Mp = p.Mp;
  fa.Np = p.Np;
  fa.ranges = p.ranges;
  fa.M = d.M;
  fa.N = d.N;
  fa.mode = p.mode == 1 ? 1 : (p.mode >= 2 ? 2 : 0);
  fa.C = d.C;
  fa.cplx = d.Acplx || d.Bcplx;
  fa.ldm = d.transC ? 1 : d.ldc;
  fa.ldn = d.transC ? d.ldc : 1;
  fa.sC = d.strideC;
  fa.out = out_modes(d.alpha, d.beta);
  tc_finalize_kernel<<<grid_of((int64_t)d.M * d.N * d.batch), 256, 0, st>>>(fa, d.batch);
  RT_CHECK_LAUNCH();
}

GemmDesc gemm_3m_desc(const GemmDesc& d) {
  GemmDesc r = d;
  r.part_a = 0;
  r.part_b = 0;
  r.batch = 3;
  r.force_partials = true;
  return r;
}

void gemm_tc_combine_3m(const GemmDesc& d, const float2* P, cudaStream_t st) {
  using namespace tc;
  if (d.M <= 0 || d.N <= 0) return;
  const Plan p = plan(gemm_3m_desc(d));
  FinArgs fa{};
  fa.P = P;
  fa.Mp = p.Mp;
  fa.Np = p.Np;
  fa.ranges = p.ranges;
  fa.M = d.M;
  fa.N = d.N;
  fa.C = d.C;
  fa.cplx = true;
  fa.ldm = d.transC ? 1 : d.ldc;
  fa.ldn = d.transC ? d.ldc : 1;
  fa.out = out_modes(d.alpha, d.beta);
  tc_combine_3m_kernel<<<grid_of((int64_t)d.M * d.N), 256, 0, st>>>(fa);
  RT_CHECK_LAUNCH();
}

}  // namespace rteom
