// Spin-explicit CCSD projections R_mu = <Phi_mu|(H_N e^{T1+T2})_C|Phi>
// (Eqs. 7-8) of the core-ionised reference, on padded slot-space blocks.
#pragma once

#include "engine.h"

namespace rteom {

// Device operands shared by every residual evaluation (owned elsewhere).
// Slot spaces: occupied slots 0..nO-1 = spatial 0..O-1; virtual slot 0 =
// the core orbital, slot a >= 1 = spatial O + a - 1.  The same integral
// arrays serve both spins; only the Fock matrix is spin dependent.
struct ResidualOperands {
  int nO = 0, nV = 0, core = 0;
  // chemists' integrals (pq|rs) stored [p][q][r][s] over the named slot classes
  const double *oooo = nullptr, *ooov = nullptr, *oovv = nullptr, *ovov = nullptr,
               *ovvv = nullptr;
  const double* ovov_as = nullptr;  // [m][e][n][f] = (me|nf) - (mf|ne)
  const double* vvvv = nullptr;  // ladder layout [e][f][a][b] = (ae|bf)
  // same-spin ladder block [(e<f)][(a<b)] = (ae|bf) - (af|be)
  const double* vvvv_as = nullptr;
  // the FP64 ladder blocks were freed after their tensor-core packs were
  // cached (split precision); the pointers remain the cache keys
  bool vvvv_released = false, vvvv_as_released = false;
  // Cholesky mode (no (ov|vv) or (vv|vv) block on the device): the terms
  // with three or four virtual indices are formed from the slot-space
  // Cholesky vectors at every residual, the ladder in chunks of chunk_a
  // values of a and the tau*(mf|ae) terms in chunks of chunk_m values of m.
  bool chol = false;
  int nchol = 0, chunk_a = 1, chunk_m = 1;
  const double* Lov = nullptr;   // [Q][m][e] = L^Q_me
  const double* Lvv = nullptr;   // [Q][a][e] = L^Q_ae
  const double* LvvT = nullptr;  // [a][e][Q]
  const double* LovT = nullptr;  // [m][e][Q]
  // (N-1) Fock slot blocks per spin (0 = alpha, 1 = beta), real and complex
  const double *foo[2] = {nullptr, nullptr}, *fov[2] = {nullptr, nullptr},
               *fvv[2] = {nullptr, nullptr};
  const double *foo_c[2] = {nullptr, nullptr}, *fov_c[2] = {nullptr, nullptr},
               *fvv_c[2] = {nullptr, nullptr};
};

// Results of the particle-particle ladder computed ahead of the rest of a
// residual (the grouped ladder): ab[i][j][a][b] = sum_ef tau_ij^ef (ae|bf)
// for the alpha-beta block and ss[s][(i<j)][(a<b)] = sum_(e<f) tau_ij^ef
// [(ae|bf) - (af|be)] for the same-spin blocks (complex; ss[s] null when the
// spin has no pair).
struct LadderOut {
  double* ab = nullptr;
  double* ss[2] = {nullptr, nullptr};
};

// R = full projections for amplitudes t (both padded amplitude vectors,
// layout of AmpGeom).  Scratch comes from E.arena; pad entries of R are
// unspecified.  Issues only stream-ordered work (capturable).  With `lad`
// (resident ladder blocks only) the ladder terms are added from it instead
// of being contracted here.
void compute_residual(Engine& E, const ResidualOperands& op, const double* t, double* R,
                      const LadderOut* lad = nullptr);

// First part of a residual with the grouped ladder (Section 3.1: the
// dominant contraction sum_cd v_abcd tau_ij^cd, resident ladder blocks): tau
// of the three T2 blocks and the three ladder GEMMs posed into `out`, which
// E (defer_ladder set) records in E.deferred with their operands packed
// instead of launching them.  Everything allocated here stays in the arena
// (the caller releases it after compute_residual(..., out) has run).
void ladder_part(Engine& E, const ResidualOperands& op, const double* t, LadderOut* out);

// Packs the constant operand of the alpha-beta ladder (same_spin false) or of
// the same-spin pair ladder into the engine's cache, through the same
// contraction calls as compute_residual but without running them (the
// engine's pack_only mode; needs tc_cache_fill).
void prepack_ladder(Engine& E, const ResidualOperands& op, bool same_spin);

}  // namespace rteom
