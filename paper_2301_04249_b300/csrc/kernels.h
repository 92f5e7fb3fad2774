// Launchers of the library's CUDA kernels (host-callable, stream-ordered).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

namespace rteom {

// ---- contractions ---------------------------------------------------------
// A strided 2-D view of an operand, read by the tensor-core packers in place
// of a permuted copy: row r and column k each
// split row-major into up to three indices with element strides.  rdims == 0
// means no view (the GemmDesc leading dimensions apply).  The index splits
// divide by invariant extents with precomputed multipliers (Granlund and
// Montgomery, PLDI 1994): q = (n * mag) >> sh, exact for 0 <= n < 2^31.
struct View2 {
  int rdims = 0, kdims = 0;
  int rext[3] = {1, 1, 1}, kext[3] = {1, 1, 1};
  int64_t rstr[3] = {0, 0, 0}, kstr[3] = {0, 0, 0};
  uint64_t rmag[3] = {0, 0, 0}, kmag[3] = {0, 0, 0};
  int rsh[3] = {0, 0, 0}, ksh[3] = {0, 0, 0};
};

// Fills the division multipliers of a view from its extents.
inline void view_prepare(View2& v) {
  auto mk = [](int d, uint64_t& mag, int& sh) {
    int l = 0;
    while ((1ull << l) < (uint64_t)d) ++l;  // ceil(log2 d)
    sh = 32 + l;
    mag = (uint64_t)((((unsigned __int128)1) << sh) / (unsigned)d) + 1;
  };
  for (int d = 0; d < 3; ++d) {
    mk(v.rext[d], v.rmag[d], v.rsh[d]);
    mk(v.kext[d], v.kmag[d], v.ksh[d]);
  }
}

#ifdef __CUDACC__
__host__ __device__ inline int64_t view_row(const View2& v, int r) {
  int64_t o = 0;
#pragma unroll
  for (int d = 2; d >= 1; --d)
    if (d < v.rdims) {
      const int q = (int)(((uint64_t)(unsigned)r * v.rmag[d]) >> v.rsh[d]);
      o += (int64_t)(r - q * v.rext[d]) * v.rstr[d];
      r = q;
    }
  return o + (int64_t)r * v.rstr[0];  // the outermost index needs no split
}
__host__ __device__ inline int64_t view_col(const View2& v, int k) {
  int64_t o = 0;
#pragma unroll
  for (int d = 2; d >= 1; --d)
    if (d < v.kdims) {
      const int q = (int)(((uint64_t)(unsigned)k * v.kmag[d]) >> v.ksh[d]);
      o += (int64_t)(k - q * v.kext[d]) * v.kstr[d];
      k = q;
    }
  return o + (int64_t)k * v.kstr[0];  // the outermost index needs no split
}
#endif

struct GemmDesc {
  int M = 0, N = 0, K = 0, batch = 1;
  const double* A = nullptr;
  int64_t lda = 0, strideA = 0;  // strides in elements (complex counts 1)
  bool transA = false, Acplx = false;
  const double* B = nullptr;
  int64_t ldb = 0, strideB = 0;
  bool transB = false, Bcplx = false;
  double* C = nullptr;
  int64_t ldc = 0, strideC = 0;
  bool transC = false;  // element (m, n) at C[n * ldc + m] (tensor-core paths only)
  // tensor-core paths only: views of A (rows m, columns k) and B (rows n,
  // columns k) replacing lda/ldb and transA/B
  View2 va, vb;
  double alpha = 1.0, beta = 0.0;
  double* work = nullptr;  // split-K partial sums, gemm_f64_workspace() doubles
  // launch configuration chosen by the autotuner: tile index < gemm_f64_tiles()
  // and K slices; -1 / 0 = the shape heuristic
  int tile = -1, splits = 0;
  // tensor-core paths only: clock-cycle budget of the waits of the MMA and
  // epilogue warps on their pipeline barriers (0 = the default, about 2 s);
  // a wait that runs out sets the error word and the CTA winds down
  long long wait_cycles = 0;
  // tensor-core paths only: a complex operand enters as the real matrix of
  // one of its parts (0 real, 1 imaginary, 2 real + imaginary) instead of its
  // real embedding (-1).  The three products of the 3M complex GEMM use them.
  int part_a = -1, part_b = -1;
  // tensor-core paths only: write (sum, compensation) partials even with one
  // K range per tile (the 3M combine reads them)
  bool force_partials = false;
  // digit-plane path only: one K range per output tile (no split-K partial
  // sums), so that a tile's result does not depend on the other tiles of its
  // launch (the grouped ladder)
  bool one_range = false;
};
// Number of K slices the kernel will use for this shape (1 = no split).
int gemm_f64_splits(const GemmDesc& d);
// Number of output tile shapes of the FP64 kernel (autotuner candidates).
int gemm_f64_tiles();
void gemm_f64_tile_shape(int t, int* bm, int* bn);
// True when the shape takes the matrix-vector path (no tile or split choice).
bool gemm_f64_is_gemv(const GemmDesc& d);
// Scratch (doubles) a split-K launch needs; 0 when no split is used.
int64_t gemm_f64_workspace(const GemmDesc& d);
void gemm_f64(const GemmDesc& d, cudaStream_t st);

// Split-TF32 tensor-core GEMM (tcgen05) with the same contract as gemm_f64:
// pack A and pack B into TF32 hi/lo tiles (a_elems / b_elems floats each
// part), then the tcgen05 MMA kernel (FP32 accumulation over slices of at
// most 512 of K, slices summed as compensated FP32 pairs; err set non-zero
// if a pipeline wait ran out).  With one K range per tile it writes C with
// alpha/beta itself; otherwise it writes p_elems (sum, compensation) pairs
// and the finalize combines them in range order into C.  gemm_tc_init()
// once per process first.
struct TcLayout {
  int64_t a_elems, b_elems;  // floats per packed hi (or lo) operand
  int64_t p_elems;           // float2 partials; 0 = the MMA kernel writes C directly
  int64_t padded_flops;
  int ranges;                // K ranges per output tile (1 = finalize is a no-op)
};
TcLayout gemm_tc_layout(const GemmDesc& d);
void gemm_tc_init();
void gemm_tc_pack_a(const GemmDesc& d, float* hi, float* lo, cudaStream_t st);
void gemm_tc_pack_b(const GemmDesc& d, float* hi, float* lo, cudaStream_t st);
void gemm_tc_mma(const GemmDesc& d, const float* Ahi, const float* Alo, const float* Bhi,
                 const float* Blo, float2* P, int* err, cudaStream_t st);
void gemm_tc_finalize(const GemmDesc& d, const float2* P, cudaStream_t st);
// Complex x complex GEMM of d (batch 1) as three real products (Gauss; error
// analysis in Higham, SIAM J. Matrix Anal. Appl. 13, 1992): P1 = Re A Re B,
// P2 = Im A Im B, P3 = (Re A + Im A)(Re B + Im B) run as one batch-3 real
// GEMM (operands packed with part_a = part_b = 0, 1, 2 into consecutive batch
// slots, partials forced), then C = alpha (P1 - P2 + i (P3 - P1 - P2)) +
// beta C.  gemm_tc_3m_desc gives the batch-3 real GEMM whose layout sizes
// the buffers.
GemmDesc gemm_3m_desc(const GemmDesc& d);
void gemm_tc_combine_3m(const GemmDesc& d, const float2* P, cudaStream_t st);

// FP64-accurate GEMM on the BF16 tensor cores (operand slicing into seven
// 8-bit digit planes with per-row power-of-two scales; exact chunk sums,
// compensated accumulation, about 2^-48 relative to the row scales), with
// the same contract as gemm_f64: pack A and pack B (digit planes of
// a_elems / b_elems BF16 each, and a_rows / b_rows row exponents), then the
// MMA kernel, which writes C itself with one K range per tile or p_elems
// unscaled (sum, compensation) pairs that the finalize combines in range
// order.  gemm_oz_init() once per process first.
struct OzLayout {
  int planes;
  int64_t a_elems, b_elems;  // BF16 per digit plane
  int64_t a_rows, b_rows;    // int row exponents
  int64_t p_elems;           // float2 partials; 0 = the MMA kernel writes C directly
  int ranges;
  double padded_flops;       // executed tensor-core FLOPs (28 digit-pair products)
};
// S = 7 digit planes (FP64-accurate), 3 (the split-BF16 form, about 2^-24
// of the row scales) or 2 (the split-FP16 form: FP16 hi/lo planes).
OzLayout gemm_oz_layout(const GemmDesc& d, int S);
// Output-tile width (rows of B' per tile) for a B' of rows_b rows.
int oz_tile_n(int64_t rows_b, int S);
void gemm_oz_init();
// slot / nslots: pack into batch slot `slot` of a buffer laid out for
// nslots batch entries of this (batch-1) operand (the 3M products).
void gemm_oz_pack_a(const GemmDesc& d, int S, uint16_t* planes, int* expo, cudaStream_t st,
                    int slot = 0, int nslots = 1);
void gemm_oz_pack_b(const GemmDesc& d, int S, uint16_t* planes, int* expo, cudaStream_t st,
                    int slot = 0, int nslots = 1);
void gemm_oz_mma(const GemmDesc& d, int S, const uint16_t* A, const int* ea, const uint16_t* B,
                 const int* eb, float2* P, int* err, cudaStream_t st);
void gemm_oz_finalize(const GemmDesc& d, int S, const int* ea, const int* eb, const float2* P,
                      cudaStream_t st);
// One GEMM of a grouped digit-plane launch: its description (one_range set)
// and its packed operands; err is the pipeline-timeout word of its owner.
struct OzGroupGemm {
  GemmDesc d;
  const uint16_t* A = nullptr;
  const int* ea = nullptr;
  const uint16_t* B = nullptr;
  const int* eb = nullptr;
  int* err = nullptr;
};
// The GEMMs of gs (S planes each) as persistent launches over their combined
// output tiles: one launch per output-tile width and up to 16 GEMMs.  Every
// tile is computed exactly as gemm_oz_mma computes it for its GEMM alone, so
// results do not depend on the grouping; a pipeline timeout sets every err
// of its launch.  Returns the number of kernel launches.
int gemm_oz_mma_group(const OzGroupGemm* gs, int n, int S, cudaStream_t st);
// The 3M combine of the digit-plane form (row scales of each product applied).
void gemm_oz_combine_3m(const GemmDesc& d, int S, const int* ea, const int* eb, const float2* P,
                        cudaStream_t st);

// out[o] = alpha * in[sum_k idx_k(o) * in_stride[k]] + beta * out[o]; out is
// contiguous with dims out_dim[0..nd-1]; strides count elements.  A real
// input may feed a complex output (imaginary part only scaled by beta).
struct PermDesc {
  int nd = 0;
  int64_t out_dim[6] = {1, 1, 1, 1, 1, 1};
  int64_t in_stride[6] = {0, 0, 0, 0, 0, 0};
};
void permute_add(const double* in, double* out, const PermDesc& d, bool in_cplx, bool out_cplx,
                 double alpha, double beta, cudaStream_t st);

// ---- amplitude algebra (padded [nO][nO][nV][nV] blocks) -------------------
// out[i,j,a,b] = c1*t2[i,j,a,b] + c2*x[i,a]*y[j,b] + c3*x[i,b]*y[j,a]
// (t2 may be null when c1 == 0); all complex.
void t2_plus_t1t1(double* out, const double* t2, double c1, const double* x, const double* y,
                  double c2, double c3, int nO, int nV, cudaStream_t st);

// R[i,j,a,b] += c0*X[i,j,a,b] + c1*X[j,i,a,b] + c2*X[i,j,b,a] + c3*X[j,i,b,a],
// every c in {-1, 0, +1} (anything else throws)
// (complex [nO][nO][nV][nV]; the permutation operators P(ij), P(ab)).
void antisym_add(double* R, const double* X, double c0, double c1, double c2, double c3, int nO,
                 int nV, cudaStream_t st);

// Antisymmetric pair packing of same-spin blocks.  Pairs are listed as
// (p < q) in row-major order: pair index k <-> (p, q), npair = n(n-1)/2.
// pack: out[P][Q] = t2[i,j,a,b] for P = (i<j), Q = (a<b)  (complex).
void pack_pairs(const double* t2, double* out, int nO, int nV, cudaStream_t st);
// R[i,j,a,b] += alpha*Rp[P][Q]; R[j,i,a,b] -= ...; R[i,j,b,a] -= ...;
// R[j,i,b,a] += ...  (complex; the four targets of one (P,Q) are distinct).
void unpack_pairs_antisym(const double* Rp, double* R, int nO, int nV, double alpha,
                          cudaStream_t st);
// Wm[(e<f)][(a<b)] = W[e][f][a][b] - W[f][e][a][b] from the ladder block
// W[e][f][a][b] = (ae|bf) (real).
void pack_ladder_antisym(const double* W, double* Wm, int nV, cudaStream_t st);

// First pair index of row p among the pairs (p < q) of n items.
__host__ __device__ inline int64_t pair_start(int n, int p) {
  return (int64_t)p * (2 * (int64_t)n - p - 1) / 2;
}
// Pair k (0 <= k < n(n-1)/2) of n items in the order (0,1),(0,2),...,
// (0,n-1),(1,2),...: the row p with pair_start(p) <= k < pair_start(p+1)
// is the root of a quadratic, estimated in FP32 and corrected by integer
// steps (at most a few for n below 2^16).
__host__ __device__ inline void pair_of(int64_t k, int n, int& p, int& q) {
  const int64_t m = 2 * (int64_t)n - 1;
  const int64_t disc = m * m - 8 * k;  // >= 1 for valid k
  int r = (int)(((float)m - sqrtf((float)(disc > 0 ? disc : 0))) * 0.5f);
  r = r < 0 ? 0 : (r > n - 2 ? n - 2 : r);
  while (r > 0 && pair_start(n, r) > k) --r;
  while (r < n - 2 && pair_start(n, r + 1) <= k) ++r;
  p = r;
  q = r + 1 + (int)(k - pair_start(n, r));
}
// Column chunk a in [a0, a0+n) of the same-spin pair ladder (the pair
// columns (a<b) of those a, contiguous).  Wc: [e][f][n][b] = (ae|bf) for the
// chunk (real); Wm: [(e<f)][chunk columns] = (ae|bf) - (af|be).
void pack_ladder_cols(const double* Wc, double* Wm, int nV, int a0, int n, cudaStream_t st);
// R[i,j,a,b] += alpha*Rq[(i<j)][c] (and the three antisymmetric images) for
// the chunk's pair columns c (complex).
void unpack_pairs_cols(const double* Rq, double* R, int nO, int nV, int a0, int n, double alpha,
                       cudaStream_t st);
// dst[r*ldd + c] += src[r*lds + c] over rows x cols doubles.
void add_block(double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows,
               int64_t cols, cudaStream_t st);

// Anderson acceleration of the micro-iteration (depth 3); vectors are n
// complex elements, the dF and dG histories kAndersonDepth slots of n each.
constexpr int kAndersonDepth = 3;
constexpr int kAndersonDots = kAndersonDepth * (kAndersonDepth + 1) / 2 + kAndersonDepth;
// f = g - x; first: Fp = f, Gp = g; otherwise dF = f - Fp, dG = g - Gp (one
// slot), then Fp = f, Gp = g.
void anderson_push(int64_t n, const double* g, const double* x, double* Fp, double* Gp,
                   double* dF, double* dG, int first, cudaStream_t st);
// out (complex [kAndersonDots]): <dF_i, dF_j> for (i,j) = (0,0),(0,1),(0,2),
// (1,1),(1,2),(2,2), then <dF_i, f>, with <u,v> = sum conj(u) v; entries with
// an index >= count are zero.  partial: complex [anderson_partials()][9].
int anderson_partials();
void anderson_dots(int64_t n, const double* dF, const double* f, int count, double* partial,
                   double* out, cudaStream_t st);
// x = g - sum_{j < count} gamma_j dG_j; gamma: host, 3 complex (interleaved).
void anderson_mix(int64_t n, const double* g, const double* dG, int count, const double* gamma,
                  double* x, cudaStream_t st);

// Geometry of the padded amplitude vector: blocks t1a, t1b (nO*nV) then
// t2aa, t2ab, t2bb (nO*nO*nV*nV), complex.  Pads: alpha virtual slot 0 and
// beta occupied slot `core`.
struct AmpGeom {
  int nO, nV, core;
  __host__ __device__ int64_t n1() const { return (int64_t)nO * nV; }
  __host__ __device__ int64_t n2() const { return (int64_t)nO * nO * nV * nV; }
  __host__ __device__ int64_t total() const { return 2 * n1() + 3 * n2(); }
  __host__ __device__ int64_t off(int blk) const {
    return blk < 2 ? blk * n1() : 2 * n1() + (blk - 2) * n2();
  }
};

// One Adams-Moulton micro-iteration (Eq. 9) over every element:
// tk <- [(1 + i dt D/2) tn + (i dt/2)(Rn - D tn + Rk - D tk)] / (1 - i dt D/2),
// pads forced to zero; *maxdiff_bits = max over elements of |new - old|^2
// (as IEEE bits of a non-negative double; NaN compares largest).
// tk_in and tk_out may alias (in-place update).
void am_update(const AmpGeom& g, const double* fo_a, const double* fv_a, const double* fo_b,
               const double* fv_b, double dt, const double* tn, const double* Rn,
               const double* tk_in, double* tk_out, const double* Rk,
               unsigned long long* maxdiff_bits, cudaStream_t st);

// Zero the pad entries of an amplitude vector.
void mask_pads(const AmpGeom& g, double* t, cudaStream_t st);

// Cumulant integrand E(t) (Eq. 5) with a deterministic two-pass reduction.
// partial: scratch of energy_partials() complex entries.  The second pass
// writes E into E_hist[n+1] and C_hist[n+1] = C_hist[n] + (i dt/2)(E_hist[n] + E)
// when update_c != 0 (else only writes E to *E_hist at index n+1).
int energy_partials(const AmpGeom& g);
void energy(const AmpGeom& g, const double* t, const double* ovov, const double* fov_a,
            const double* fov_b, int include_fov, double* partial, double* E_hist, double* C_hist,
            long long n, double dt, int update_c, cudaStream_t st);

// Pack an unpadded host-layout amplitude vector (device copy) into padded
// blocks (pads zeroed), and the reverse.  O, V are the spatial counts.
void pack_amplitudes(const AmpGeom& g, const double* unpadded, double* padded, cudaStream_t st);
void unpack_amplitudes(const AmpGeom& g, const double* padded, double* unpadded, cudaStream_t st);
// Sparse access by flat index k of the unpadded vector (0 <= k < unpadded
// length, complex entries): padded[slot(k)] = val for each k, and
// out[e] = padded[slot(idx[e])].  Indices are checked by the caller.
void scatter_unpadded(const AmpGeom& g, const long long* idx, const double* val, int64_t n,
                      double* padded, cudaStream_t st);
void gather_unpadded(const AmpGeom& g, const double* padded, const long long* idx, int64_t n,
                     double* out, cudaStream_t st);

// ---- set-up (once per context) ----------------------------------------------
// Slot-space Cholesky blocks from L [nchol][nb][nb]:
// Loo[Q][i][j], Lov[Q][i][a], Lvv[Q][a][b] with virtual slot 0 = core.
void gather_cholesky(const double* L, int nchol, int nO, int nV, int core, double* Loo,
                     double* Lov, double* Lvv, cudaStream_t st);
// (N-1) Fock matrices per spin (Section 2.1), as slot blocks and diagonals.
void build_fock(const double* eps, const double* L, int nchol, int nO, int nV, int core,
                double* foo_a, double* fov_a, double* fvv_a, double* foo_b, double* fov_b,
                double* fvv_b, double* fo_a, double* fv_a, double* fo_b, double* fv_b,
                cudaStream_t st);
// Closed-shell E_N^corr (Eq. 3) into *out (device), deterministic.
void closed_shell_ecorr(const double* ovov, const double* t1, const double* t2, int O, int V,
                        double* partial, double* out, cudaStream_t st);

// ---- spectrum ----------------------------------------------------------------
void spectrum(const double* C, long long M, double dt, double shift, const double* omega,
              int nomega, double eta, double* A, cudaStream_t st);

// Largest |x| over n doubles as IEEE bits (non-negative), for finiteness checks.
void maxabs_bits(const double* x, int64_t n, unsigned long long* out, cudaStream_t st);

}  // namespace rteom
