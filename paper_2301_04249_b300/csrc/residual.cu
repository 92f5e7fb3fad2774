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

void compute_residual(Engine& E, const ResidualOperands& op, const double* tp, double* Rp,
                      const LadderOut* lad) {
  const int nO = op.nO, nV = op.nV, nQ = op.nchol;
  const bool chol = op.chol;
  const AmpGeom g{nO, nV, op.core};
  E.drop_holds();  // none from an evaluation that did not finish
  const int64_t mark = E.arena.mark();
  Arena& A = E.arena;
  auto blk = [&](const double* base, int b) { return const_cast<double*>(base) + 2 * g.off(b); };
  auto T2 = [&](double* p) { return make_tensor(p, true, {nO, nO, nV, nV}); };
  auto T1 = [&](double* p) { return make_tensor(p, true, {nO, nV}); };
  auto new2 = [&]() { return A.tensor(true, {nO, nO, nV, nV}); };
  auto newc = [&](std::initializer_list<int64_t> d) { return A.tensor(true, d); };
  auto newr = [&](std::initializer_list<int64_t> d) { return A.tensor(false, d); };
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
  Tensor ovvv, vvvv, Lov, Lvv;
  if (chol) {
    Lov = R_(op.Lov, {nQ, nO, nV});
    Lvv = R_(op.Lvv, {nQ, nV, nV});
  } else {
    ovvv = R_(op.ovvv, {nO, nV, nV, nV});
    vvvv = R_(op.vvvv, {nV, nV, nV, nV});
    vvvv.released = op.vvvv_released;
  }
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

  // ---- amplitude combinations that live through the whole evaluation
  // t2su[s]: [i in occ_s][j in occ_u][a in vir_s][b in vir_u]
  Tensor t2su[2] = {t2ab, new2()};
  axpy("jiba->ijab", 1.0, t2ab, 0.0, t2su[1]);
  Tensor t1sum = newc({nO, nV});
  axpy("ia->ia", 1.0, t1[0], 0.0, t1sum);
  axpy("ia->ia", 1.0, t1[1], 1.0, t1sum);
  Tensor tau_ss[2];
  for (int s = 0; s < 2; ++s) {
    tau_ss[s] = new2();
    t2t1(tau_ss[s], &t2ss[s], 1.0, t1[s], t1[s], 1.0, -1.0);
  }
  Tensor tau_ab = new2();
  t2t1(tau_ab, &t2su[0], 1.0, t1[0], t1[1], 1.0, 0.0);
  // Cholesky mode: U[s][Q][i][a] = sum_e t_i^e L^Q_ae carries every t1 x
  // (ov|vv) product: sum_e t_i^e (jb|ae) = sum_Q L^Q_jb U[s][Q][i][a]
  Tensor U[2];
  if (chol)
    for (int s = 0; s < 2; ++s) {
      U[s] = newc({nQ, nO, nV});
      ein("ie,Qae->Qia", 1.0, t1[s], Lvv, 0.0, U[s]);
    }

  // small intermediates kept to the end
  Tensor Fme[2], Fae[2], Fmi[2], Fvv[2], Foo[2], Wss[2];
  for (int s = 0; s < 2; ++s) {
    Fme[s] = newc({nO, nV});
    Fae[s] = newc({nV, nV});
    Fmi[s] = newc({nO, nO});
    Fvv[s] = newc({nV, nV});
    Foo[s] = newc({nO, nO});
    Wss[s] = newc({nO, nO, nO, nO});
  }
  Tensor Wab = newc({nO, nO, nO, nO});

  {
    const int64_t mk = A.mark();
    // tau~_ss + tau~_su (they always meet the same integral) and t2_ss + t2_su
    Tensor taut_sum[2], t2sum[2];
    for (int s = 0; s < 2; ++s) {
      taut_sum[s] = new2();
      t2sum[s] = new2();
    }
    {
      const int64_t mt = A.mark();
      Tensor tmp = new2();
      for (int s = 0; s < 2; ++s) {
        const int u = 1 - s;
        t2t1(taut_sum[s], &t2ss[s], 1.0, t1[s], t1[s], 0.5, -0.5);
        t2t1(tmp, &t2su[s], 1.0, t1[s], t1[u], 0.5, 0.0);
        axpy("ijab->ijab", 1.0, tmp, 1.0, taut_sum[s]);
        axpy("ijab->ijab", 1.0, t2ss[s], 0.0, t2sum[s]);
        axpy("ijab->ijab", 1.0, t2su[s], 1.0, t2sum[s]);
      }
      A.release(mt);
    }
    // Cholesky mode: y[Q] = sum_mf (t_a + t_b)_m^f L^Q_mf
    Tensor y;
    if (chol) {
      y = newc({nQ});
      ein("mf,Qmf->Q", 1.0, t1sum, Lov, 0.0, y);
    }

    // ---- one-particle intermediates F_me, F_ae, F_mi
    for (int s = 0; s < 2; ++s) {
      axpy("me->me", 1.0, fov_c[s], 0.0, Fme[s]);
      ein("nf,menf->me", 1.0, t1sum, ovov, 1.0, Fme[s]);
      ein("nf,mfne->me", -1.0, t1[s], ovov, 1.0, Fme[s]);

      axpy("ae->ae", 1.0, fvv_c[s], 0.0, Fae[s]);
      ein("me,ma->ae", -0.5, fov[s], t1[s], 1.0, Fae[s]);
      if (chol) {
        ein("Q,Qae->ae", 1.0, y, Lvv, 1.0, Fae[s]);         // sum_mf t_m^f (mf|ae)
        ein("Qme,Qma->ae", -1.0, Lov, U[s], 1.0, Fae[s]);   // sum_mf t_m^f (me|af)
      } else {
        ein("mf,mfae->ae", 1.0, t1sum, ovvv, 1.0, Fae[s]);
        ein("mf,meaf->ae", -1.0, t1[s], ovvv, 1.0, Fae[s]);
      }
      ein("mnaf,menf->ae", -1.0, taut_sum[s], ovov, 1.0, Fae[s]);

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
      if (chol) {  // sum_mef t_im^ef (mf|ae) = sum_Qe [sum_mf t_im^ef L^Q_mf] L^Q_ae
        const int64_t mv = A.mark();
        Tensor v = newc({nQ, nO, nV});
        ein("imef,Qmf->Qie", 1.0, t2sum[s], Lov, 0.0, v);
        ein("Qie,aeQ->ia", 1.0, v, R_(op.LvvT, {nV, nV, nQ}), 1.0, R1[s]);
        A.release(mv);
      } else {
        ein("imef,mfae->ia", 1.0, t2sum[s], ovvv, 1.0, R1[s]);
      }
      ein("mnae,mine->ia", -1.0, t2sum[s], ooov, 1.0, R1[s]);
    }

    // F'_be = F_be - 1/2 t_m^b F_me,  F'_mj = F_mj + 1/2 t_j^e F_me
    for (int s = 0; s < 2; ++s) {
      axpy("be->be", 1.0, Fae[s], 0.0, Fvv[s]);
      ein("mb,me->be", -0.5, t1[s], Fme[s], 1.0, Fvv[s]);
      axpy("mj->mj", 1.0, Fmi[s], 0.0, Foo[s]);
      ein("je,me->mj", 0.5, t1[s], Fme[s], 1.0, Foo[s]);
    }

    // ---- W_mnij (same spin; alpha-beta)
    for (int s = 0; s < 2; ++s) {
      axpy("minj->mnij", 1.0, oooo, 0.0, Wss[s]);
      axpy("mjni->mnij", -1.0, oooo, 1.0, Wss[s]);
      const int64_t mx = A.mark();
      Tensor x = newc({nO, nO, nO, nO});
      ein("je,mine->mnij", 1.0, t1[s], ooov, 0.0, x);
      ein("je,nime->mnij", -1.0, t1[s], ooov, 1.0, x);
      axpy("mnij->mnij", 1.0, x, 1.0, Wss[s]);
      axpy("mnji->mnij", -1.0, x, 1.0, Wss[s]);
      A.release(mx);
      ein("ijef,menf->mnij", 1.0, tau_ss[s], ovov, 1.0, Wss[s]);
    }
    axpy("minj->mnij", 1.0, oooo, 0.0, Wab);
    ein("je,mine->mnij", 1.0, t1[1], ooov, 1.0, Wab);
    ein("ie,njme->mnij", 1.0, t1[0], ooov, 1.0, Wab);
    ein("ijef,menf->mnij", 1.0, tau_ab, ovov, 1.0, Wab);
    A.release(mk);
  }

  // one scratch block for the terms that go through P(ij)/P(ab)
  Tensor x = new2();

  // ---- T2 projections, same spin (Eq. 8), all but the W_mbej ring terms
  for (int s = 0; s < 2; ++s) {
    Tensor& R = R2ss[s];
    axpy("iajb->ijab", 1.0, ovov, 0.0, R);
    axpy("ibja->ijab", -1.0, ovov, 1.0, R);
    ein("ijae,be->ijab", 1.0, t2ss[s], Fvv[s], 0.0, x);
    asym(R, x, 1.0, 0.0, -1.0, 0.0);
    ein("imab,mj->ijab", 1.0, t2ss[s], Foo[s], 0.0, x);
    asym(R, x, -1.0, 1.0, 0.0, 0.0);
    ein("mnab,mnij->ijab", 0.5, tau_ss[s], Wss[s], 1.0, R);
    if (!chol) {
      // ladder over antisymmetric pairs: sum_{e<f} tau_ij^ef [(ae|bf) - (af|be)]
      // for i<j, a<b, scattered to the four (i,j,a,b) sign patterns
      const int64_t npo = (int64_t)nO * (nO - 1) / 2, npv = (int64_t)nV * (nV - 1) / 2;
      if (lad && lad->ss[s]) {  // computed ahead (grouped ladder)
        const double* Rq = lad->ss[s];
        E.launch(kElementwise, 0.0,
                 [&] { unpack_pairs_antisym(Rq, R.p, nO, nV, 1.0, E.stream); });
      } else if (npo > 0 && npv > 0) {
        const int64_t mp = A.mark();
        Tensor tpk = newc({npo, npv});
        Tensor Rq = newc({npo, npv});
        E.launch(kElementwise, 0.0, [&] { pack_pairs(tau_ss[s].p, tpk.p, nO, nV, E.stream); });
        Tensor Wm = R_(op.vvvv_as, {npv, npv});
        Wm.released = op.vvvv_as_released;
        E.contract("pq,qr->pr", 1.0, tpk, Wm, 0.0, Rq, kLadder);
        E.launch(kElementwise, 0.0,
                 [&] { unpack_pairs_antisym(Rq.p, R.p, nO, nV, 1.0, E.stream); });
        A.release(mp);
      }
      const int64_t mz = A.mark();
      Tensor Z = newc({nO, nO, nV, nO});
      ein("ijef,mfae->ijam", 1.0, tau_ss[s], ovvv, 0.0, Z);
      ein("mb,ijam->ijab", 1.0, t1[s], Z, 0.0, x);
      asym(R, x, -1.0, 0.0, 1.0, 0.0);
      A.release(mz);
    }
    // ring, t1 t1 part: -P(ij)P(ab) t_i^e t_m^a <mb||ej>
    {
      const int64_t mq = A.mark();
      Tensor Q = newc({nO, nO, nV, nO});
      ein("ie,mejb->imbj", 1.0, t1[s], ovov, 0.0, Q);
      ein("ie,mjbe->imbj", -1.0, t1[s], oovv, 1.0, Q);
      ein("ma,imbj->ijab", -1.0, t1[s], Q, 0.0, x);
      asym(R, x, 1.0, -1.0, -1.0, 1.0);
      A.release(mq);
    }
    // P(ij) t_i^e <ab||ej>
    if (chol) {
      ein("Qjb,Qia->ijab", 1.0, Lov, U[s], 0.0, x);
      ein("Qja,Qib->ijab", -1.0, Lov, U[s], 1.0, x);
    } else {
      ein("ie,jbae->ijab", 1.0, t1[s], ovvv, 0.0, x);
      ein("ie,jabe->ijab", -1.0, t1[s], ovvv, 1.0, x);
    }
    asym(R, x, 1.0, -1.0, 0.0, 0.0);
    // -P(ab) t_m^a <mb||ij>
    ein("ma,mijb->ijab", 1.0, t1[s], ooov, 0.0, x);
    ein("ma,mjib->ijab", -1.0, t1[s], ooov, 1.0, x);
    asym(R, x, -1.0, 0.0, 1.0, 0.0);
  }

  // ---- T2 projection, alpha-beta (Eq. 8), all but the W_mbej ring terms
  const Tensor& t1a = t1[0];
  const Tensor& t1b = t1[1];
  {
    Tensor& R = R2ab;
    axpy("iajb->ijab", 1.0, ovov, 0.0, R);
    ein("ijae,be->ijab", 1.0, t2ab, Fvv[1], 1.0, R);
    ein("ijeb,ae->ijab", 1.0, t2ab, Fvv[0], 1.0, R);
    ein("imab,mj->ijab", -1.0, t2ab, Foo[1], 1.0, R);
    ein("mjab,mi->ijab", -1.0, t2ab, Foo[0], 1.0, R);
    ein("mnab,mnij->ijab", 1.0, tau_ab, Wab, 1.0, R);
    if (!chol) {
      if (lad)  // computed ahead (grouped ladder)
        axpy("ijab->ijab", 1.0, C_(lad->ab, {nO, nO, nV, nV}), 1.0, R);
      else
        E.contract("ijef,efab->ijab", 1.0, tau_ab, vvvv, 1.0, R, kLadder);
      const int64_t mz = A.mark();
      Tensor Z1 = newc({nO, nO, nV, nO});
      ein("ijef,mfae->ijam", 1.0, tau_ab, ovvv, 0.0, Z1);
      ein("mb,ijam->ijab", -1.0, t1b, Z1, 1.0, R);
      Tensor Z2 = newc({nO, nO, nO, nV});
      ein("ijef,mebf->ijmb", 1.0, tau_ab, ovvv, 0.0, Z2);
      ein("ma,ijmb->ijab", -1.0, t1a, Z2, 1.0, R);
      A.release(mz);
    }
    // t1 t1 parts of the ring terms, one per spin case of (m, e)
    const int64_t mq = A.mark();
    Tensor Q = newc({nO, nO, nO, nV});
    ein("ie,mejb->imjb", 1.0, t1a, ovov, 0.0, Q);
    ein("ma,imjb->ijab", -1.0, t1a, Q, 1.0, R);
    ein("je,mibe->jmib", 1.0, t1b, oovv, 0.0, Q);
    ein("ma,jmib->ijab", -1.0, t1a, Q, 1.0, R);
    ein("ie,mjae->imja", 1.0, t1a, oovv, 0.0, Q);
    ein("mb,imja->ijab", -1.0, t1b, Q, 1.0, R);
    ein("je,meia->jmia", 1.0, t1b, ovov, 0.0, Q);
    ein("mb,jmia->ijab", -1.0, t1b, Q, 1.0, R);
    A.release(mq);
    // t_i^e <a b||e j>-type and t_m^a <m b||i j>-type terms
    if (chol) {
      ein("Qjb,Qia->ijab", 1.0, Lov, U[0], 1.0, R);
      ein("Qia,Qjb->ijab", 1.0, Lov, U[1], 1.0, R);
    } else {
      ein("ie,jbae->ijab", 1.0, t1a, ovvv, 1.0, R);
      ein("je,iabe->ijab", 1.0, t1b, ovvv, 1.0, R);
    }
    ein("ma,mijb->ijab", -1.0, t1a, ooov, 1.0, R);
    ein("mb,mjia->ijab", -1.0, t1b, ooov, 1.0, R);
  }

  // ---- Cholesky mode: the tau*(mf|ae) terms through X[e][f][m][a] = (mf|ae),
  // formed for chunk_m values of m at a time (Z laid out [m][i][j][a])
  if (chol) {
    const int64_t mz = A.mark();
    Tensor Zs[2] = {newc({nO, nO, nO, nV}), newc({nO, nO, nO, nV})};
    Tensor Z1 = newc({nO, nO, nO, nV}), Z2 = newc({nO, nO, nO, nV});
    {
      const int64_t mt = A.mark();
      Tensor tauT = new2();  // tau_ab with e and f swapped: [i][j][f][e]
      axpy("ijef->ijfe", 1.0, tau_ab, 0.0, tauT);
      const int64_t zs = (int64_t)nO * nO * nV;
      // the four tau operands enter every chunk: packed once, with the
      // shapes of a full chunk
      {
        const int n = std::min(op.chunk_m, nO);
        const Tensor X = make_tensor(nullptr, false, {nV, nV, n, nV});
        const Tensor Zc = make_tensor(nullptr, true, {n, nO, nO, nV});
        for (const Tensor* T : {&tau_ss[0], &tau_ss[1], &tau_ab}) E.hold(T->p);
        E.hold(tauT.p);
        E.pack_only = true;
        for (int s = 0; s < 2; ++s) ein("ijef,efma->mija", 1.0, tau_ss[s], X, 0.0, Zc);
        ein("ijef,efma->mija", 1.0, tau_ab, X, 0.0, Zc);
        ein("ijfe,femb->mijb", 1.0, tauT, X, 0.0, Zc);
        E.pack_only = false;
      }
      for (int m0 = 0; m0 < nO; m0 += op.chunk_m) {
        const int n = std::min(op.chunk_m, nO - m0);
        const int64_t mc = A.mark();
        Tensor X = newr({nV, nV, n, nV});
        ein("mfQ,Qae->efma", 1.0, R_(op.LovT + (int64_t)m0 * nV * nQ, {n, nV, nQ}), Lvv, 0.0, X);
        auto slice = [&](const Tensor& Z) {
          return make_tensor(Z.p + 2 * zs * m0, true, {n, nO, nO, nV});
        };
        for (int s = 0; s < 2; ++s) ein("ijef,efma->mija", 1.0, tau_ss[s], X, 0.0, slice(Zs[s]));
        ein("ijef,efma->mija", 1.0, tau_ab, X, 0.0, slice(Z1));
        ein("ijfe,femb->mijb", 1.0, tauT, X, 0.0, slice(Z2));  // (me|bf) = X[f][e][m][b]
        A.release(mc);
      }
      E.drop_holds();
      A.release(mt);
    }
    for (int s = 0; s < 2; ++s) {
      ein("mb,mija->ijab", 1.0, t1[s], Zs[s], 0.0, x);
      asym(R2ss[s], x, -1.0, 0.0, 1.0, 0.0);
    }
    ein("mb,mija->ijab", -1.0, t1b, Z1, 1.0, R2ab);
    ein("ma,mijb->ijab", -1.0, t1a, Z2, 1.0, R2ab);
    A.release(mz);
  }

  // ---- W_mbej spin blocks [m][b][e][j] (superscripts name the spins of
  // (m,b,e,j)), each built, applied to the ring terms and dropped:
  // same spin  P(ij)P(ab) t_im^ae W_mbej,  alpha-beta one term per spin case
  auto newW = [&]() { return newc({nO, nV, nV, nO}); };
  // + sum_f t_j^f <mb||ef>-type pieces through the Cholesky vectors or (ov|vv)
  auto w_mebf = [&](int s, double c, const Tensor& W) {  // c sum_f t_j^f (me|bf)
    if (chol)
      ein("Qme,Qjb->mbej", c, Lov, U[s], 1.0, W);
    else
      ein("jf,mebf->mbej", c, t1[s], ovvv, 1.0, W);
  };
  auto w_mfbe = [&](int s, double c, const Tensor& W) {  // c sum_f t_j^f (mf|be)
    if (chol) {
      const int64_t mw = A.mark();
      Tensor w = newc({nQ, nO, nO});
      ein("jf,Qmf->Qjm", 1.0, t1[s], Lov, 0.0, w);
      ein("Qjm,Qbe->mbej", c, w, Lvv, 1.0, W);
      A.release(mw);
    } else {
      ein("jf,mfbe->mbej", c, t1[s], ovvv, 1.0, W);
    }
  };
  // c sum_nf Y_jn^{x} (me|nf) with the Coulomb integral: O^3 V^3 through the
  // assembled (ov|ov), or, in the Cholesky mode, sum_Q L^Q_me [sum_nf Y L^Q_nf]
  // (2 O^2 V^2 Nchol, several times less when Nchol < O (V+1) / 2)
  auto w_coulomb = [&](const char* spec, const char* yspec, double c, const Tensor& Y,
                       const Tensor& W) {
    if (chol) {
      const int64_t mq = A.mark();
      Tensor q = newc({nQ, nO, nV});
      ein(yspec, 1.0, Y, Lov, 0.0, q);  // q[Q][j][b] = sum_nf Y L^Q_nf
      ein("Qme,Qjb->mbej", c, Lov, q, 1.0, W);
      A.release(mq);
    } else {
      ein(spec, c, Y, ovov, 1.0, W);
    }
  };
  auto W_same = [&](int s, const Tensor& W) {  // ssss
    axpy("mejb->mbej", 1.0, ovov, 0.0, W);
    axpy("mjbe->mbej", -1.0, oovv, 1.0, W);
    w_mebf(s, 1.0, W);
    w_mfbe(s, -1.0, W);
    ein("nb,njme->mbej", -1.0, t1[s], ooov, 1.0, W);
    ein("nb,mjne->mbej", 1.0, t1[s], ooov, 1.0, W);
    const int64_t m2 = A.mark();
    Tensor X = new2();
    t2t1(X, &t2ss[s], 0.5, t1[s], t1[s], 1.0, 0.0);
    ein("jnfb,menf->mbej", -1.0, X, ovov_as, 1.0, W);
    A.release(m2);
    w_coulomb("jnbf,menf->mbej", "jnbf,Qnf->Qjb", 0.5, t2su[s], W);
  };
  auto W_usus = [&](int s, const Tensor& W) {  // m u, b s, e u, j s
    axpy("mejb->mbej", 1.0, ovov, 0.0, W);
    w_mebf(s, 1.0, W);
    ein("nb,njme->mbej", -1.0, t1[s], ooov, 1.0, W);
    ein("jnbf,menf->mbej", 0.5, t2su[s], ovov_as, 1.0, W);
    const int64_t m2 = A.mark();
    Tensor X = new2();
    t2t1(X, &t2ss[s], 0.5, t1[s], t1[s], 1.0, 0.0);
    w_coulomb("jnfb,menf->mbej", "jnfb,Qnf->Qjb", -1.0, X, W);
    A.release(m2);
  };
  auto W_suus = [&](int s, const Tensor& W) {  // m s, b u, e u, j s
    const int u = 1 - s;
    axpy("mjbe->mbej", -1.0, oovv, 0.0, W);
    w_mfbe(s, -1.0, W);
    ein("nb,mjne->mbej", 1.0, t1[u], ooov, 1.0, W);
    const int64_t m2 = A.mark();
    Tensor Y = new2();
    t2t1(Y, &t2su[s], 0.5, t1[s], t1[u], 1.0, 0.0);
    ein("jnfb,mfne->mbej", 1.0, Y, ovov, 1.0, W);
    A.release(m2);
  };
  {
    const int64_t mw = A.mark();
    Tensor W = newW();
    // W^aaaa, W^bbbb
    for (int s = 0; s < 2; ++s) {
      W_same(s, W);
      ein("imae,mbej->ijab", 1.0, t2ss[s], W, 0.0, x);
      asym(R2ss[s], x, 1.0, -1.0, -1.0, 1.0);
      if (s == 0)
        ein("mjeb,maei->ijab", 1.0, t2ab, W, 1.0, R2ab);
      else
        ein("imae,mbej->ijab", 1.0, t2ab, W, 1.0, R2ab);
    }
    // W^baba (s = 0), W^abab (s = 1)
    for (int s = 0; s < 2; ++s) {
      W_usus(s, W);
      ein("imae,mbej->ijab", 1.0, t2su[s], W, 0.0, x);
      asym(R2ss[s], x, 1.0, -1.0, -1.0, 1.0);
      if (s == 0)
        ein("jmbe,maei->ijab", 1.0, t2ss[1], W, 1.0, R2ab);
      else
        ein("imae,mbej->ijab", 1.0, t2ss[0], W, 1.0, R2ab);
    }
    // W^abba (s = 0), W^baab (s = 1)
    W_suus(0, W);
    ein("mjae,mbei->ijab", 1.0, t2ab, W, 1.0, R2ab);
    W_suus(1, W);
    ein("imeb,maej->ijab", 1.0, t2ab, W, 1.0, R2ab);
    A.release(mw);
  }

  // ---- Cholesky mode: the particle-particle ladder (Section 3.1.1),
  // (ae|bf) formed for chunk_a values of a at a time as W[e][f][a][b] and
  // applied to all three T2 blocks (same spin over antisymmetric pairs)
  if (chol) {
    const int64_t ml = A.mark();
    const int64_t npo = (int64_t)nO * (nO - 1) / 2, npv = (int64_t)nV * (nV - 1) / 2;
    Tensor tpk[2];
    if (npo > 0 && npv > 0)
      for (int s = 0; s < 2; ++s) {
        tpk[s] = newc({npo, npv});
        E.launch(kElementwise, 0.0,
                 [&] { pack_pairs(tau_ss[s].p, tpk[s].p, nO, nV, E.stream); });
      }
    // tau_ab and the pair-packed tau enter every chunk: their tensor-core
    // packs are made once, here, with the shapes of a full chunk
    {
      const int n = std::min(op.chunk_a, nV);
      const int64_t ncols = pair_start(nV, n) - pair_start(nV, 0);
      const Tensor Wc = make_tensor(nullptr, false, {nV, nV, n, nV});
      const Tensor Rc = make_tensor(nullptr, true, {nO, nO, n, nV});
      E.hold(tau_ab.p);
      E.pack_only = true;
      E.contract("ijef,efab->ijab", 1.0, tau_ab, Wc, 0.0, Rc, kLadder);
      if (tpk[0].p && ncols > 0) {
        const Tensor Wm = make_tensor(nullptr, false, {npv, ncols});
        const Tensor Rq = make_tensor(nullptr, true, {npo, ncols});
        for (int s = 0; s < 2; ++s) {
          E.hold(tpk[s].p);
          E.contract("pq,qr->pr", 1.0, tpk[s], Wm, 0.0, Rq, kLadder);
        }
      }
      E.pack_only = false;
    }
    for (int a0 = 0; a0 < nV; a0 += op.chunk_a) {
      const int n = std::min(op.chunk_a, nV - a0);
      const int64_t mc = A.mark();
      Tensor Wc = newr({nV, nV, n, nV});
      E.contract("aeQ,Qbf->efab", 1.0, R_(op.LvvT + (int64_t)a0 * nV * nQ, {n, nV, nQ}), Lvv,
                 0.0, Wc, kLadder);
      {
        const int64_t mr = A.mark();
        Tensor Rc = newc({nO, nO, n, nV});
        E.contract("ijef,efab->ijab", 1.0, tau_ab, Wc, 0.0, Rc, kLadder);
        E.launch(kElementwise, 0.0, [&] {
          add_block(R2ab.p + 2 * (int64_t)a0 * nV, 2 * (int64_t)nV * nV, Rc.p,
                    2 * (int64_t)n * nV, (int64_t)nO * nO, 2 * (int64_t)n * nV, E.stream);
        });
        A.release(mr);
      }
      const int64_t ncols = pair_start(nV, a0 + n) - pair_start(nV, a0);
      if (npo > 0 && ncols > 0) {
        Tensor Wm = newr({npv, ncols});
        E.launch(kElementwise, 0.0, [&] { pack_ladder_cols(Wc.p, Wm.p, nV, a0, n, E.stream); });
        for (int s = 0; s < 2; ++s) {
          const int64_t mr = A.mark();
          Tensor Rq = newc({npo, ncols});
          E.contract("pq,qr->pr", 1.0, tpk[s], Wm, 0.0, Rq, kLadder);
          E.launch(kElementwise, 0.0, [&] {
            unpack_pairs_cols(Rq.p, R2ss[s].p, nO, nV, a0, n, 1.0, E.stream);
          });
          A.release(mr);
        }
      }
      A.release(mc);
    }
    E.drop_holds();
    A.release(ml);
  }
  E.arena.release(mark);
}

void ladder_part(Engine& E, const ResidualOperands& op, const double* tp, LadderOut* out) {
  const int nO = op.nO, nV = op.nV;
  if (op.chol) throw Error(-1, "ladder_part: the grouped ladder needs the resident ladder blocks");
  const AmpGeom g{nO, nV, op.core};
  Arena& A = E.arena;
  auto blk = [&](int b) { return const_cast<double*>(tp) + 2 * g.off(b); };
  auto t2t1 = [&](const Tensor& o, const Tensor& t2, const Tensor& x, const Tensor& y, double c3) {
    E.launch(kElementwise, 0.0,
             [&] { t2_plus_t1t1(o.p, t2.p, 1.0, x.p, y.p, 1.0, c3, nO, nV, E.stream); });
  };
  const Tensor t1[2] = {make_tensor(blk(0), true, {nO, nV}), make_tensor(blk(1), true, {nO, nV})};
  // tau as compute_residual forms it: t2 + t1 t1 (antisymmetrised same-spin)
  const Tensor tau_ab = A.tensor(true, {nO, nO, nV, nV});
  t2t1(tau_ab, make_tensor(blk(3), true, {nO, nO, nV, nV}), t1[0], t1[1], 0.0);
  Tensor vvvv = make_tensor(const_cast<double*>(op.vvvv), false, {nV, nV, nV, nV});
  vvvv.constant = true;
  vvvv.released = op.vvvv_released;
  const Tensor lab = A.tensor(true, {nO, nO, nV, nV});
  out->ab = lab.p;
  E.contract("ijef,efab->ijab", 1.0, tau_ab, vvvv, 0.0, lab, kLadder);
  const int64_t npo = (int64_t)nO * (nO - 1) / 2, npv = (int64_t)nV * (nV - 1) / 2;
  for (int s = 0; s < 2; ++s) {
    out->ss[s] = nullptr;
    if (npo == 0 || npv == 0) continue;
    const Tensor tau = A.tensor(true, {nO, nO, nV, nV});
    t2t1(tau, make_tensor(blk(s == 0 ? 2 : 4), true, {nO, nO, nV, nV}), t1[s], t1[s], -1.0);
    const Tensor tpk = A.tensor(true, {npo, npv});
    E.launch(kElementwise, 0.0, [&] { pack_pairs(tau.p, tpk.p, nO, nV, E.stream); });
    Tensor Wm = make_tensor(const_cast<double*>(op.vvvv_as), false, {npv, npv});
    Wm.constant = true;
    Wm.released = op.vvvv_as_released;
    const Tensor Rq = A.tensor(true, {npo, npv});
    out->ss[s] = Rq.p;
    E.contract("pq,qr->pr", 1.0, tpk, Wm, 0.0, Rq, kLadder);
  }
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
