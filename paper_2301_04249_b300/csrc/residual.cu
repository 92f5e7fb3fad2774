// Spin-explicit CCSD projections on the GPU (Eqs. 7-8).
//
// The terms are those of the non-canonical spin-orbital CCSD equations in
// the intermediate form of Stanton, Gauss, Watts and Bartlett (J. Chem.
// Phys. 94, 4334 (1991)), integrated over spin for the three unique T2
// blocks (alpha-alpha, alpha-beta, beta-beta) and two T1 blocks that
// Section 3.1.1 keeps.  The tau*tau*<mn||ef> term is carried entirely by
// W_mnij.  The (N-1) reference has non-zero occupied-virtual Fock elements,
// which appear in F_me, F_ae, F_mi and the T1 projection.
//
// Layout: every block is padded to the same slot shapes (occupied nO, virtual
// nV = V+1) so that both spins share one set of integral arrays; the pad
// slots (alpha virtual 0, beta occupied `core`) hold zero amplitudes, and
// every summed index touches an amplitude, so pads never leak into real
// entries.  Two-electron integrals are chemists' (pq|rs) built from the
// Cholesky vectors once per context; the particle-particle ladder
// sum_ef tau_ij^ef (ae|bf) is one GEMM per spin block against (ae|bf).
#include "residual.h"

namespace rteom {

void compute_residual(Engine& E, const ResidualOperands& op, const double* tp, double* Rp) {
  const int nO = op.nO, nV = op.nV;
  const AmpGeom g{nO, nV, op.core};
  const int64_t mark = E.arena.mark();
  Arena& A = E.arena;
  auto blk = [&](const double* base, int b) { return const_cast<double*>(base) + 2 * g.off(b); };
  auto T2 = [&](double* p) { return make_tensor(p, true, {nO, nO, nV, nV}); };
  auto T1 = [&](double* p) { return make_tensor(p, true, {nO, nV}); };
  auto new2 = [&]() { return A.tensor(true, {nO, nO, nV, nV}); };
  auto newc = [&](std::initializer_list<int64_t> d) { return A.tensor(true, d); };
  auto R_ = [&](const double* p, std::initializer_list<int64_t> d) {  // integrals, Fock
    Tensor t = make_tensor(const_cast<double*>(p), false, d);
    t.constant = true;
    return t;
  };
  auto C_ = [&](const double* p, std::initializer_list<int64_t> d) {
    return make_tensor(const_cast<double*>(p), true, d);
  };
  auto ein = [&](const char* s, double a, const Tensor& X, const Tensor& Y, double b,
                 const Tensor& Z) { E.contract(s, a, X, Y, b, Z); };
  auto axpy = [&](const char* s, double a, const Tensor& X, double b, const Tensor& Y) {
    E.axpy(s, a, X, b, Y);
  };
  // R += c0 X + c1 P_ij X + c2 P_ab X + c3 P_ij P_ab X (one pass)
  auto asym = [&](const Tensor& R, const Tensor& X, double c0, double c1, double c2, double c3) {
    E.launch(kPermute, 0.0,
             [&] { antisym_add(R.p, X.p, c0, c1, c2, c3, nO, nV, E.stream); }, "antisym");
  };
  auto t2t1 = [&](const Tensor& out, const Tensor* t2, double c1, const Tensor& x,
                  const Tensor& y, double c2, double c3) {
    E.launch(kElementwise, 0.0, [&] {
      t2_plus_t1t1(out.p, t2 ? t2->p : nullptr, c1, x.p, y.p, c2, c3, nO, nV, E.stream);
    });
  };

  // integrals
  const Tensor oooo = R_(op.oooo, {nO, nO, nO, nO});
  const Tensor ooov = R_(op.ooov, {nO, nO, nO, nV});
  const Tensor oovv = R_(op.oovv, {nO, nO, nV, nV});
  const Tensor ovov = R_(op.ovov, {nO, nV, nO, nV});
  const Tensor ovov_as = R_(op.ovov_as, {nO, nV, nO, nV});
  const Tensor ovvv = R_(op.ovvv, {nO, nV, nV, nV});
  Tensor vvvv = R_(op.vvvv, {nV, nV, nV, nV});
  vvvv.released = op.vvvv_released;
  Tensor fov[2], foo_c[2], fov_c[2], fvv_c[2];
  for (int s = 0; s < 2; ++s) {
    fov[s] = R_(op.fov[s], {nO, nV});
    foo_c[s] = C_(op.foo_c[s], {nO, nO});
    fov_c[s] = C_(op.fov_c[s], {nO, nV});
    fvv_c[s] = C_(op.fvv_c[s], {nV, nV});
  }

  // amplitudes and outputs
  Tensor t1[2] = {T1(blk(tp, 0)), T1(blk(tp, 1))};
  Tensor t2ss[2] = {T2(blk(tp, 2)), T2(blk(tp, 4))};
  Tensor t2ab = T2(blk(tp, 3));
  Tensor R1[2] = {T1(blk(Rp, 0)), T1(blk(Rp, 1))};
  Tensor R2ss[2] = {T2(blk(Rp, 2)), T2(blk(Rp, 4))};
  Tensor R2ab = T2(blk(Rp, 3));

  // t2su[s]: [i in occ_s][j in occ_u][a in vir_s][b in vir_u]
  Tensor t2su[2] = {t2ab, new2()};
  axpy("jiba->ijab", 1.0, t2ab, 0.0, t2su[1]);
  Tensor t1sum = newc({nO, nV});
  axpy("ia->ia", 1.0, t1[0], 0.0, t1sum);
  axpy("ia->ia", 1.0, t1[1], 1.0, t1sum);

  Tensor tau_ss[2], tau_su[2], taut_sum[2], t2sum[2];
  for (int s = 0; s < 2; ++s) {
    const int u = 1 - s;
    tau_ss[s] = new2();
    t2t1(tau_ss[s], &t2ss[s], 1.0, t1[s], t1[s], 1.0, -1.0);
    tau_su[s] = new2();
    t2t1(tau_su[s], &t2su[s], 1.0, t1[s], t1[u], 1.0, 0.0);
    // tau~_ss + tau~_su (they always meet the same integral)
    taut_sum[s] = new2();
    t2t1(taut_sum[s], &t2ss[s], 1.0, t1[s], t1[s], 0.5, -0.5);
    Tensor tmp = new2();
    t2t1(tmp, &t2su[s], 1.0, t1[s], t1[u], 0.5, 0.0);
    axpy("ijab->ijab", 1.0, tmp, 1.0, taut_sum[s]);
    t2sum[s] = new2();
    axpy("ijab->ijab", 1.0, t2ss[s], 0.0, t2sum[s]);
    axpy("ijab->ijab", 1.0, t2su[s], 1.0, t2sum[s]);
  }

  // ---- one-particle intermediates F_me, F_ae, F_mi
  Tensor Fme[2], Fae[2], Fmi[2];
  for (int s = 0; s < 2; ++s) {
    Fme[s] = newc({nO, nV});
    axpy("me->me", 1.0, fov_c[s], 0.0, Fme[s]);
    ein("nf,menf->me", 1.0, t1sum, ovov, 1.0, Fme[s]);
    ein("nf,mfne->me", -1.0, t1[s], ovov, 1.0, Fme[s]);

    Fae[s] = newc({nV, nV});
    axpy("ae->ae", 1.0, fvv_c[s], 0.0, Fae[s]);
    ein("me,ma->ae", -0.5, fov[s], t1[s], 1.0, Fae[s]);
    ein("mf,mfae->ae", 1.0, t1sum, ovvv, 1.0, Fae[s]);
    ein("mf,meaf->ae", -1.0, t1[s], ovvv, 1.0, Fae[s]);
    ein("mnaf,menf->ae", -1.0, taut_sum[s], ovov, 1.0, Fae[s]);

    Fmi[s] = newc({nO, nO});
    axpy("mi->mi", 1.0, foo_c[s], 0.0, Fmi[s]);
    ein("ie,me->mi", 0.5, t1[s], fov[s], 1.0, Fmi[s]);
    ein("ne,mine->mi", 1.0, t1sum, ooov, 1.0, Fmi[s]);
    ein("ne,nime->mi", -1.0, t1[s], ooov, 1.0, Fmi[s]);
    ein("inef,menf->mi", 1.0, taut_sum[s], ovov, 1.0, Fmi[s]);
  }

  // ---- T1 projections (Eq. 7)
  for (int s = 0; s < 2; ++s) {
    const int u = 1 - s;
    axpy("ia->ia", 1.0, fov_c[s], 0.0, R1[s]);
    ein("ie,ae->ia", 1.0, t1[s], Fae[s], 1.0, R1[s]);
    ein("ma,mi->ia", -1.0, t1[s], Fmi[s], 1.0, R1[s]);
    ein("imae,me->ia", 1.0, t2ss[s], Fme[s], 1.0, R1[s]);
    ein("imae,me->ia", 1.0, t2su[s], Fme[u], 1.0, R1[s]);
    ein("nf,niaf->ia", -1.0, t1[s], oovv, 1.0, R1[s]);
    ein("nf,nfia->ia", 1.0, t1sum, ovov, 1.0, R1[s]);
    ein("imef,mfae->ia", 1.0, t2sum[s], ovvv, 1.0, R1[s]);
    ein("mnae,mine->ia", -1.0, t2sum[s], ooov, 1.0, R1[s]);
  }

  // F'_be = F_be - 1/2 t_m^b F_me,  F'_mj = F_mj + 1/2 t_j^e F_me
  Tensor Fvv[2], Foo[2];
  for (int s = 0; s < 2; ++s) {
    Fvv[s] = newc({nV, nV});
    axpy("be->be", 1.0, Fae[s], 0.0, Fvv[s]);
    ein("mb,me->be", -0.5, t1[s], Fme[s], 1.0, Fvv[s]);
    Foo[s] = newc({nO, nO});
    axpy("mj->mj", 1.0, Fmi[s], 0.0, Foo[s]);
    ein("je,me->mj", 0.5, t1[s], Fme[s], 1.0, Foo[s]);
  }

  // ---- W_mnij (same spin; alpha-beta)
  Tensor Wss[2];
  for (int s = 0; s < 2; ++s) {
    Wss[s] = newc({nO, nO, nO, nO});
    axpy("minj->mnij", 1.0, oooo, 0.0, Wss[s]);
    axpy("mjni->mnij", -1.0, oooo, 1.0, Wss[s]);
    Tensor x = newc({nO, nO, nO, nO});
    ein("je,mine->mnij", 1.0, t1[s], ooov, 0.0, x);
    ein("je,nime->mnij", -1.0, t1[s], ooov, 1.0, x);
    axpy("mnij->mnij", 1.0, x, 1.0, Wss[s]);
    axpy("mnji->mnij", -1.0, x, 1.0, Wss[s]);
    ein("ijef,menf->mnij", 1.0, tau_ss[s], ovov, 1.0, Wss[s]);
  }
  Tensor Wab = newc({nO, nO, nO, nO});
  axpy("minj->mnij", 1.0, oooo, 0.0, Wab);
  ein("je,mine->mnij", 1.0, t1[1], ooov, 1.0, Wab);
  ein("ie,njme->mnij", 1.0, t1[0], ooov, 1.0, Wab);
  ein("ijef,menf->mnij", 1.0, tau_su[0], ovov, 1.0, Wab);

  // ---- W_mbej spin blocks [m][b][e][j]; superscripts name the spins of (m,b,e,j)
  auto newW = [&]() { return newc({nO, nV, nV, nO}); };
  auto W_same = [&](int s) {  // ssss
    const int u = 1 - s;
    Tensor X = new2();
    t2t1(X, &t2ss[s], 0.5, t1[s], t1[s], 1.0, 0.0);
    Tensor W = newW();
    axpy("mejb->mbej", 1.0, ovov, 0.0, W);
    axpy("mjbe->mbej", -1.0, oovv, 1.0, W);
    ein("jf,mebf->mbej", 1.0, t1[s], ovvv, 1.0, W);
    ein("jf,mfbe->mbej", -1.0, t1[s], ovvv, 1.0, W);
    ein("nb,njme->mbej", -1.0, t1[s], ooov, 1.0, W);
    ein("nb,mjne->mbej", 1.0, t1[s], ooov, 1.0, W);
    ein("jnfb,menf->mbej", -1.0, X, ovov_as, 1.0, W);
    ein("jnbf,menf->mbej", 0.5, t2su[s], ovov, 1.0, W);
    (void)u;
    return W;
  };
  auto W_usus = [&](int s) {  // m u, b s, e u, j s
    Tensor X = new2();
    t2t1(X, &t2ss[s], 0.5, t1[s], t1[s], 1.0, 0.0);
    Tensor W = newW();
    axpy("mejb->mbej", 1.0, ovov, 0.0, W);
    ein("jf,mebf->mbej", 1.0, t1[s], ovvv, 1.0, W);
    ein("nb,njme->mbej", -1.0, t1[s], ooov, 1.0, W);
    ein("jnbf,menf->mbej", 0.5, t2su[s], ovov_as, 1.0, W);
    ein("jnfb,menf->mbej", -1.0, X, ovov, 1.0, W);
    return W;
  };
  auto W_suus = [&](int s) {  // m s, b u, e u, j s
    const int u = 1 - s;
    Tensor Y = new2();
    t2t1(Y, &t2su[s], 0.5, t1[s], t1[u], 1.0, 0.0);
    Tensor W = newW();
    axpy("mjbe->mbej", -1.0, oovv, 0.0, W);
    ein("jf,mfbe->mbej", -1.0, t1[s], ovvv, 1.0, W);
    ein("nb,mjne->mbej", 1.0, t1[u], ooov, 1.0, W);
    ein("jnfb,mfne->mbej", 1.0, Y, ovov, 1.0, W);
    return W;
  };
  Tensor Waaaa = W_same(0), Wbbbb = W_same(1);
  Tensor Wbaba = W_usus(0), Wabab = W_usus(1);
  Tensor Wabba = W_suus(0), Wbaab = W_suus(1);
  Tensor Wsame[2] = {Waaaa, Wbbbb};
  Tensor Wx[2] = {Wbaba, Wabab};

  // ---- T2 projections, same spin (Eq. 8)
  for (int s = 0; s < 2; ++s) {
    Tensor& R = R2ss[s];
    axpy("iajb->ijab", 1.0, ovov, 0.0, R);
    axpy("ibja->ijab", -1.0, ovov, 1.0, R);
    Tensor x = new2();
    ein("ijae,be->ijab", 1.0, t2ss[s], Fvv[s], 0.0, x);
    asym(R, x, 1.0, 0.0, -1.0, 0.0);
    ein("imab,mj->ijab", 1.0, t2ss[s], Foo[s], 0.0, x);
    asym(R, x, -1.0, 1.0, 0.0, 0.0);
    ein("mnab,mnij->ijab", 0.5, tau_ss[s], Wss[s], 1.0, R);
    // ladder over antisymmetric pairs: sum_{e<f} tau_ij^ef [(ae|bf) - (af|be)]
    // for i<j, a<b, scattered to the four (i,j,a,b) sign patterns
    {
      const int64_t npo = (int64_t)nO * (nO - 1) / 2, npv = (int64_t)nV * (nV - 1) / 2;
      if (npo > 0 && npv > 0) {
        Tensor tp = newc({npo, npv});
        Tensor Rp = newc({npo, npv});
        E.launch(kElementwise, 0.0, [&] { pack_pairs(tau_ss[s].p, tp.p, nO, nV, E.stream); });
        Tensor Wm = R_(op.vvvv_as, {npv, npv});
        Wm.released = op.vvvv_as_released;
        E.contract("pq,qr->pr", 1.0, tp, Wm, 0.0, Rp, kLadder);
        E.launch(kElementwise, 0.0,
                 [&] { unpack_pairs_antisym(Rp.p, R.p, nO, nV, 1.0, E.stream); });
      }
    }
    Tensor Z = newc({nO, nO, nV, nO});
    ein("ijef,mfae->ijam", 1.0, tau_ss[s], ovvv, 0.0, Z);
    ein("mb,ijam->ijab", 1.0, t1[s], Z, 0.0, x);
    asym(R, x, -1.0, 0.0, 1.0, 0.0);
    // ring: P(ij)P(ab) [t_im^ae W_mbej - t_i^e t_m^a <mb||ej>]
    ein("imae,mbej->ijab", 1.0, t2ss[s], Wsame[s], 0.0, x);
    ein("imae,mbej->ijab", 1.0, t2su[s], Wx[s], 1.0, x);
    Tensor Q = newc({nO, nO, nV, nO});
    ein("ie,mejb->imbj", 1.0, t1[s], ovov, 0.0, Q);
    ein("ie,mjbe->imbj", -1.0, t1[s], oovv, 1.0, Q);
    ein("ma,imbj->ijab", -1.0, t1[s], Q, 1.0, x);
    asym(R, x, 1.0, -1.0, -1.0, 1.0);
    // P(ij) t_i^e <ab||ej>
    ein("ie,jbae->ijab", 1.0, t1[s], ovvv, 0.0, x);
    ein("ie,jabe->ijab", -1.0, t1[s], ovvv, 1.0, x);
    asym(R, x, 1.0, -1.0, 0.0, 0.0);
    // -P(ab) t_m^a <mb||ij>
    ein("ma,mijb->ijab", 1.0, t1[s], ooov, 0.0, x);
    ein("ma,mjib->ijab", -1.0, t1[s], ooov, 1.0, x);
    asym(R, x, -1.0, 0.0, 1.0, 0.0);
  }

  // ---- T2 projection, alpha-beta (Eq. 8)
  {
    Tensor& R = R2ab;
    const Tensor& t1a = t1[0];
    const Tensor& t1b = t1[1];
    const Tensor& tau_ab = tau_su[0];
    axpy("iajb->ijab", 1.0, ovov, 0.0, R);
    ein("ijae,be->ijab", 1.0, t2ab, Fvv[1], 1.0, R);
    ein("ijeb,ae->ijab", 1.0, t2ab, Fvv[0], 1.0, R);
    ein("imab,mj->ijab", -1.0, t2ab, Foo[1], 1.0, R);
    ein("mjab,mi->ijab", -1.0, t2ab, Foo[0], 1.0, R);
    ein("mnab,mnij->ijab", 1.0, tau_ab, Wab, 1.0, R);
    E.contract("ijef,efab->ijab", 1.0, tau_ab, vvvv, 1.0, R, kLadder);
    Tensor Z1 = newc({nO, nO, nV, nO});
    ein("ijef,mfae->ijam", 1.0, tau_ab, ovvv, 0.0, Z1);
    ein("mb,ijam->ijab", -1.0, t1b, Z1, 1.0, R);
    Tensor Z2 = newc({nO, nO, nO, nV});
    ein("ijef,mebf->ijmb", 1.0, tau_ab, ovvv, 0.0, Z2);
    ein("ma,ijmb->ijab", -1.0, t1a, Z2, 1.0, R);
    // ring terms, one per spin case of the contracted (m, e) pair
    ein("imae,mbej->ijab", 1.0, t2ss[0], Wabab, 1.0, R);
    ein("imae,mbej->ijab", 1.0, t2ab, Wbbbb, 1.0, R);
    Tensor Q = newc({nO, nO, nO, nV});
    ein("ie,mejb->imjb", 1.0, t1a, ovov, 0.0, Q);
    ein("ma,imjb->ijab", -1.0, t1a, Q, 1.0, R);
    ein("mjae,mbei->ijab", 1.0, t2ab, Wabba, 1.0, R);
    ein("je,mibe->jmib", 1.0, t1b, oovv, 0.0, Q);
    ein("ma,jmib->ijab", -1.0, t1a, Q, 1.0, R);
    ein("imeb,maej->ijab", 1.0, t2ab, Wbaab, 1.0, R);
    ein("ie,mjae->imja", 1.0, t1a, oovv, 0.0, Q);
    ein("mb,imja->ijab", -1.0, t1b, Q, 1.0, R);
    ein("mjeb,maei->ijab", 1.0, t2ab, Waaaa, 1.0, R);
    ein("jmbe,maei->ijab", 1.0, t2ss[1], Wbaba, 1.0, R);
    ein("je,meia->jmia", 1.0, t1b, ovov, 0.0, Q);
    ein("mb,jmia->ijab", -1.0, t1b, Q, 1.0, R);
    // t_i^e <a b||e j>-type and t_m^a <m b||i j>-type terms
    ein("ie,jbae->ijab", 1.0, t1a, ovvv, 1.0, R);
    ein("je,iabe->ijab", 1.0, t1b, ovvv, 1.0, R);
    ein("ma,mijb->ijab", -1.0, t1a, ooov, 1.0, R);
    ein("mb,mjia->ijab", -1.0, t1b, ooov, 1.0, R);
  }
  E.arena.release(mark);
}

void prepack_ladder(Engine& E, const ResidualOperands& op, bool same_spin) {
  const int nO = op.nO, nV = op.nV;
  const int64_t mark = E.arena.mark();
  E.pack_only = true;
  // stand-ins for the amplitude side: same shapes as in compute_residual,
  // never read (only the constant operand is packed)
  if (!same_spin) {
    Tensor vvvv = make_tensor(const_cast<double*>(op.vvvv), false, {nV, nV, nV, nV});
    vvvv.constant = true;
    const Tensor tau = E.arena.tensor(true, {nO, nO, nV, nV});
    const Tensor R = E.arena.tensor(true, {nO, nO, nV, nV});
    E.contract("ijef,efab->ijab", 1.0, tau, vvvv, 1.0, R, kLadder);
  } else {
    const int64_t npo = (int64_t)nO * (nO - 1) / 2, npv = (int64_t)nV * (nV - 1) / 2;
    if (npo > 0 && npv > 0) {
      Tensor Wm = make_tensor(const_cast<double*>(op.vvvv_as), false, {npv, npv});
      Wm.constant = true;
      const Tensor tp = E.arena.tensor(true, {npo, npv});
      const Tensor Rp = E.arena.tensor(true, {npo, npv});
      E.contract("pq,qr->pr", 1.0, tp, Wm, 0.0, Rp, kLadder);
    }
  }
  E.pack_only = false;
  E.arena.release(mark);
}

}  // namespace rteom
