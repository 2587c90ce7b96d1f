// Set-up of Adaptive-Multilevel BDDC (Algorithm 3) and one application of
// the Multilevel BDDC preconditioner (Algorithm 1), batched over all
// substructures of a level.
//
// Per level (Sec. 2, Sec. 5):
//   * assemble the dense local matrices in the order [interior | delta | corner];
//   * factor them through the interior columns: A_II = L L^T; the panel
//     below becomes X^T = (L^{-1} K_IG)^T and the trailing block becomes
//     S = K_GG - X^T X (the Schur complement, eq. Schur-definition);
//   * continue the factorization through the non-corner interface columns:
//     S_DD = L_D L_D^T, the Neumann matrix with the corner dofs fixed (the
//     corner part of the constrained saddle problem);
//   * explicit inverses L^{-1}, L_D^{-1} so that every later solve is a
//     streaming triangular product;
//   * coarse basis from eq. local_saddle_point_problem with corners primal:
//     Y = L_D^{-1} C_D^T, G = Y^T Y, Psi, and the coarse matrix Psi^T S Psi
//     (= -mu, the level-(i+1) element matrix).
// Algorithm 1 on all levels is captured once per context as a CUDA graph and
// replayed for every PCG iteration (precond).
#include <cmath>
#include <map>

#include "engine_impl.h"
#include "tc_gemm.h"

namespace amb {

template <typename T>
void Engine<T>::check_status(const char* what, int code) {
  int h[4] = {0, 0, 0, 0};
  AMB_CUDA(cudaMemcpyAsync(h, status.p, sizeof(h), cudaMemcpyDeviceToHost, st));
  AMB_CUDA(cudaStreamSynchronize(st));
  if (h[0] != 0) {
    AMB_CUDA(cudaMemsetAsync(status.p, 0, 4 * sizeof(int), st));
    if (h[0] == AMB_ETIMEOUT)
      throw Error(AMB_ETIMEOUT, std::string(what) + ": a bounded wait inside a kernel ran out");
    if (h[0] == AMB_ENOCONV)
      throw Error(AMB_ENOCONV, std::string(what) + ": a dense symmetric eigensolver exceeded its sweep limit");
    throw Error(code ? code : h[0], std::string(what) + ": non-positive pivot in substructure " +
                                        std::to_string(h[1]) + " at column " + std::to_string(h[2]));
  }
}

template <typename T>
void Engine<T>::upload_par(LevelData<T>& L) {
  const int ns = L.ns;
  L.par_h.assign((size_t)ns * NPAR, 0);
  for (int s = 0; s < ns; ++s) {
    int64_t* p = &L.par_h[(size_t)s * NPAR];
    p[P_NI] = L.ni[s];
    p[P_NG] = L.ng[s];
    p[P_NCRN] = L.ncrn[s];
    p[P_ND] = L.nd[s];
    p[P_NC] = L.nc.empty() ? 0 : L.nc[s];
    p[P_NCP] = L.ncp.empty() ? 0 : L.ncp[s];
    p[P_NN] = L.nn[s];
    p[P_OM] = L.pM.off[s];
    p[P_OS] = L.pS.off[s];
    p[P_OLI] = L.pLI.off[s];
    p[P_OLD] = L.pLD.off[s];
    p[P_OCD] = L.pCd.off.empty() ? 0 : L.pCd.off[s];
    p[P_OY] = L.pY.off.empty() ? 0 : L.pY.off[s];
    p[P_OG] = L.pG.off.empty() ? 0 : L.pG.off[s];
    p[P_OPSI] = L.pPsi.off.empty() ? 0 : L.pPsi.off[s];
    p[P_OAC] = L.pAc.off.empty() ? 0 : L.pAc.off[s];
    p[P_VI] = L.vI.off[s];
    p[P_VG] = L.vG.off[s];
    p[P_VD] = L.vD.off[s];
    p[P_VC] = L.vC.off.empty() ? 0 : L.vC.off[s];
    p[P_VCP] = L.vCP.off.empty() ? 0 : L.vCP.off[s];
  }
  upload(L.par, L.par_h, st);
}

template <typename T>
void Engine<T>::alloc_level(LevelData<T>& L) {
  const LevelTopo& tp = L.topo;
  const int ns = tp.n_subs;
  L.ns = ns;
  L.ni.resize(ns);
  L.ng.resize(ns);
  L.ncrn.resize(ns);
  L.nd.resize(ns);
  L.nn.resize(ns);
  std::vector<int64_t> sM(ns), sS(ns), sLI(ns), sLD(ns), si(ns), sg(ns), sd(ns);
  for (int s = 0; s < ns; ++s) {
    const SubTopo& sb = tp.subs[s];
    L.ni[s] = sb.n_i;
    L.ng[s] = sb.n_g;
    L.ncrn[s] = sb.n_crn;
    L.nd[s] = sb.n_d();
    L.nn[s] = sb.n_i + sb.n_g;
    sM[s] = (int64_t)L.nn[s] * L.nn[s];
    sS[s] = (int64_t)sb.n_g * sb.n_g;
    sLI[s] = (int64_t)sb.n_i * sb.n_i;
    sLD[s] = (int64_t)sb.n_d() * sb.n_d();
    si[s] = sb.n_i;
    sg[s] = sb.n_g;
    sd[s] = sb.n_d();
  }
  L.pM.build(sM);
  L.pS.build(sS);
  L.pLI.build(sLI);
  L.pLD.build(sLD);
  L.vI.build(si);
  L.vG.build(sg);
  L.vD.build(sd);
  L.M.alloc(L.pM.total * sizeof(T));
  L.S.alloc(L.pS.total * sizeof(T));
  L.LinvI.alloc(L.pLI.total * sizeof(T));
  L.LinvD.alloc(L.pLD.total * sizeof(T));
  L.diagG.alloc(L.vG.total * sizeof(double));
  L.w.alloc(L.vG.total * sizeof(T));
  // index maps
  std::vector<int64_t> idof;
  idof.reserve(L.vI.total);
  for (int s = 0; s < ns; ++s) idof.insert(idof.end(), tp.subs[s].dofs.begin(), tp.subs[s].dofs.begin() + tp.subs[s].n_i);
  upload(L.idof, idof, st);
  upload(L.iface_dof, tp.iface_dofs, st);
  L.n_iface = (int64_t)tp.iface_dofs.size();
  upload(L.own_off, tp.own_off, st);
  std::vector<int32_t> own_flat(tp.own_sub.size()), gidx(L.vG.total);
  for (size_t q = 0; q < tp.own_sub.size(); ++q) own_flat[q] = (int32_t)(L.vG.off[tp.own_sub[q]] + tp.own_pos[q]);
  upload(L.own_flat, own_flat, st);
  for (int s = 0; s < ns; ++s)
    for (int l = 0; l < L.ng[s]; ++l) gidx[L.vG.off[s] + l] = tp.gidx[s][l];
  upload(L.gidx, gidx, st);
  // work vectors
  L.xI.alloc(L.vI.total * sizeof(T));
  L.tI.alloc(L.vI.total * sizeof(T));
  L.gG.alloc(L.vG.total * sizeof(T));
  L.vGw.alloc(L.vG.total * sizeof(T));
  L.zD.alloc(L.vD.total * sizeof(T));
  L.rB.alloc(L.n_iface * sizeof(double));
  L.uGd.alloc(L.n_iface * sizeof(double));
  upload_par(L);
}

template <typename T>
void Engine<T>::assemble(LevelData<T>& L, const LevelData<T>* prev, const std::vector<int32_t>& loc) {
  AMB_CUDA(cudaMemsetAsync(L.M.p, 0, L.pM.total * sizeof(T), st));
  DevBuf off, n;
  std::vector<int32_t> nn32(L.nn.begin(), L.nn.end());
  upload(off, L.pM.off, st);
  upload(n, nn32, st);
  if (!prev) {
    assemble_level1<T>(st, dptr<T>(L.M), dptr<int64_t>(off), dptr<int32_t>(n), dptr<int32_t>(mesh.elem_sub),
                       dptr<int32_t>(mesh.elem_local), dptr<double>(mesh.coeff), dptr<double>(mesh.khat), 8 * mesh.dpn,
                       mesh.nx, mesh.ny, mesh.nz);
  } else {
    const int nch = prev->ns;
    std::vector<int32_t> parent(cfg.parents[L.level - 2].begin(), cfg.parents[L.level - 2].end());
    std::vector<int64_t> loc_off(nch);
    std::vector<int32_t> nc32(nch);
    int64_t lo = 0;
    for (int s = 0; s < nch; ++s) {
      loc_off[s] = lo;
      lo += prev->nc[s];
      nc32[s] = prev->nc[s];
    }
    // children ordered by (rank among their siblings, index): pass r adds
    // the r-th child of every parent
    std::vector<int> rank(nch), seen(L.ns, 0);
    int nrank = 0;
    for (int s = 0; s < nch; ++s) {
      rank[s] = seen[parent[s]]++;
      nrank = std::max(nrank, rank[s] + 1);
    }
    std::vector<int> pass_beg(nrank + 1, 0);
    for (int s = 0; s < nch; ++s) ++pass_beg[rank[s] + 1];
    for (int r = 0; r < nrank; ++r) pass_beg[r + 1] += pass_beg[r];
    std::vector<int32_t> child(nch);
    {
      std::vector<int> cur(pass_beg.begin(), pass_beg.end() - 1);
      for (int s = 0; s < nch; ++s) child[cur[rank[s]]++] = s;
    }
    std::vector<int64_t> ent_off(nch + 1, 0);
    for (int q = 0; q < nch; ++q) ent_off[q + 1] = ent_off[q] + (int64_t)nc32[child[q]] * nc32[child[q]];
    DevBuf dpar, dacoff, dnc, dlocoff, dloc, dent, dchild;
    upload(dpar, parent, st);
    upload(dacoff, prev->pAc.off, st);
    upload(dnc, nc32, st);
    upload(dlocoff, loc_off, st);
    upload(dloc, loc, st);
    upload(dent, ent_off, st);
    upload(dchild, child, st);
    assemble_next<T>(st, dptr<T>(L.M), dptr<int64_t>(off), dptr<int32_t>(n), dptr<int32_t>(dpar), dptr<int64_t>(dacoff),
                     dptr<int32_t>(dnc), dptr<int64_t>(dlocoff), dptr<int32_t>(dloc), dptr<double>(prev->Ac),
                     dptr<int32_t>(dchild), dptr<int64_t>(dent), pass_beg, ent_off);
    AMB_CUDA(cudaStreamSynchronize(st));   // keep the temporaries alive until the kernels ran
  }
  AMB_CUDA(cudaStreamSynchronize(st));
}

template <typename T>
void Engine<T>::factor_level(LevelData<T>& L) {
  const int ns = L.ns;
  const int64_t* par = dptr<int64_t>(L.par);
  extract_iface_diag<T>(st, dptr<double>(L.diagG), dptr<T>(L.M), par, ns, imax(L.ng));
  scaling_weights<T>(st, dptr<T>(L.w), dptr<double>(L.diagG), dptr<int32_t>(L.own_off), dptr<int32_t>(L.own_flat),
                     L.n_iface);
  double fl = 0;
  {
    FamTimer ft(st, &tm, AMB_FAM_FACTOR, timing());
    std::vector<CholDesc> d1;
    for (int s = 0; s < ns; ++s)
      d1.push_back(CholDesc{L.pM.off[s], L.nn[s], L.nn[s], 0, L.ni[s], L.pLI.off[s], std::max(L.ni[s], 1), s});
    partial_cholesky<T>(st, ring, d1, dptr<T>(L.M), dptr<T>(L.LinvI), dptr<int>(status), &fl, &tm, timing());
    check_status("interior factorization A_II = L L^T", AMB_ENOTSPD);
    copy_schur<T>(st, dptr<T>(L.S), dptr<T>(L.M), par, ns, imax(L.ng));
    std::vector<CholDesc> d2;
    for (int s = 0; s < ns; ++s)
      d2.push_back(CholDesc{L.pM.off[s], L.nn[s], L.nn[s], L.ni[s], L.ni[s] + L.nd[s], L.pLD.off[s],
                            std::max(L.nd[s], 1), s});
    partial_cholesky<T>(st, ring, d2, dptr<T>(L.M), dptr<T>(L.LinvD), dptr<int>(status), &fl, &tm, timing());
    check_status("corner-constrained Neumann factorization S_DD = L_D L_D^T (Assumption 1: corners must fix the "
                 "substructure's zero-energy modes)",
                 AMB_EASSUMPTION);
  }
  tm.fam_flops[AMB_FAM_FACTOR] += fl;
  L.factor_flops += fl;
  double ft_ = 0;
  {
    FamTimer ft(st, &tm, AMB_FAM_TRTRI, timing());
    std::vector<TrtriDesc> t;
    for (int s = 0; s < ns; ++s) {
      if (L.ni[s] > 0) t.push_back(TrtriDesc{L.pM.off[s], L.pLI.off[s], L.nn[s], L.ni[s], L.ni[s], 0});
    }
    trtri_from_blocks<T>(st, ring, t, dptr<T>(L.M), dptr<T>(L.LinvI), &ft_, dptr<int>(status));
    t.clear();
    for (int s = 0; s < ns; ++s) {
      if (L.nd[s] > 0)
        t.push_back(TrtriDesc{L.pM.off[s] + L.ni[s] + (int64_t)L.ni[s] * L.nn[s], L.pLD.off[s], L.nn[s], L.nd[s],
                              L.nd[s], 0});
    }
    trtri_from_blocks<T>(st, ring, t, dptr<T>(L.M), dptr<T>(L.LinvD), &ft_, dptr<int>(status));
  }
  check_status("explicit triangular inverses", AMB_ETIMEOUT);
  tm.fam_flops[AMB_FAM_TRTRI] += ft_;
  L.trtri_flops += ft_;
  AMB_CUDA(cudaStreamSynchronize(st));
}

template <typename T>
void Engine<T>::coarse_basis(LevelData<T>& L) {
  FamTimer ft(st, &tm, AMB_FAM_COARSE, timing());
  const LevelTopo& tp = L.topo;
  const int ns = L.ns;
  L.nc.resize(ns);
  L.ncp.resize(ns);
  std::vector<int64_t> sCd(ns), sPsi(ns), sAc(ns), sG(ns), sc(ns), scp(ns), sZ(ns), sW(ns), sT2(ns), sT1(ns);
  for (int s = 0; s < ns; ++s) {
    L.nc[s] = tp.subs[s].n_c();
    L.ncp[s] = tp.subs[s].n_cp();
    sCd[s] = (int64_t)L.ncp[s] * L.nd[s];
    sPsi[s] = (int64_t)L.ng[s] * L.nc[s];
    sAc[s] = (int64_t)L.nc[s] * L.nc[s];
    sG[s] = (int64_t)L.ncp[s] * L.ncp[s];
    sc[s] = L.nc[s];
    scp[s] = L.ncp[s];
    sZ[s] = (int64_t)L.nd[s] * L.nc[s];
    sW[s] = (int64_t)L.ncp[s] * L.nc[s];
    sT1[s] = (int64_t)L.ng[s] * L.nc[s];
    sT2[s] = (int64_t)L.nc[s] * L.nc[s];
  }
  L.pCd.build(sCd);
  L.pY.build(sCd);
  L.pG.build(sG);
  L.pPsi.build(sPsi);
  L.pAc.build(sAc);
  L.vC.build(sc);
  L.vCP.build(scp);
  L.Cd.alloc(L.pCd.total * sizeof(T));
  L.Y.alloc(L.pY.total * sizeof(T));
  L.Ginv.alloc(L.pG.total * sizeof(T));
  L.Yd.alloc(L.pY.total * sizeof(double));
  L.Ginvd.alloc(L.pG.total * sizeof(double));
  L.zDd.alloc(L.vD.total * sizeof(double));
  L.qCPd.alloc(L.vCP.total * sizeof(double));
  L.lCPd.alloc(L.vCP.total * sizeof(double));
  L.Psi.alloc(L.pPsi.total * sizeof(T));
  L.Ac.alloc(L.pAc.total * sizeof(double));
  L.cC.alloc(L.vC.total * sizeof(T));
  L.ucC.alloc(L.vC.total * sizeof(T));
  L.rcg.alloc(tp.n_coarse * sizeof(double));
  L.ucg.alloc(tp.n_coarse * sizeof(double));
  upload_par(L);
  // coarse index maps
  std::vector<int64_t> rc(L.vC.total);
  std::vector<std::vector<int32_t>> owners(tp.n_coarse);
  for (int s = 0; s < ns; ++s)
    for (int q = 0; q < L.nc[s]; ++q) {
      rc[L.vC.off[s] + q] = tp.subs[s].rc[q];
      owners[tp.subs[s].rc[q]].push_back((int32_t)(L.vC.off[s] + q));
    }
  upload(L.rc, rc, st);
  std::vector<int32_t> coff(1, 0), cflat;
  for (auto& o : owners) {
    cflat.insert(cflat.end(), o.begin(), o.end());
    coff.push_back((int32_t)cflat.size());
  }
  upload(L.cown_off, coff, st);
  upload(L.cown_flat, cflat, st);
  // constraint rows Cd (ncp x nd, column-major)
  std::vector<int64_t> coff_v;
  std::vector<double> cval;
  for (int s = 0; s < ns; ++s) {
    const SubTopo& sb = tp.subs[s];
    for (int q = 0; q < (int)sb.crows.size(); ++q)
      for (auto& e : sb.crows[q]) {
        coff_v.push_back(L.pCd.off[s] + q + (int64_t)e.first * L.ncp[s]);
        cval.push_back(e.second);
      }
  }
  AMB_CUDA(cudaMemsetAsync(L.Cd.p, 0, L.pCd.total * sizeof(T), st));
  DevBuf doff, dval;
  upload(doff, coff_v, st);
  upload(dval, cval, st);
  scatter_values<T>(st, dptr<T>(L.Cd), dptr<int64_t>(doff), dptr<double>(dval), (int64_t)cval.size());

  Pools pZ, pW, pT1, pT2;
  pZ.build(sZ);
  pW.build(sW);
  pT1.build(sT1);
  pT2.build(sT2);
  // The constraint space is carried in FP64 in both forms: with strong
  // coefficient contrast G = C_D S_DD^{-1} C_D^T is very ill-conditioned, and
  // FP32 rounding of G (or of its inverse) makes the constrained Neumann
  // solve non-SPD.  Products over the factor-precision L_D use the extended
  // FP32-pair accumulation in the FP32 form (gemm_batched<double, T>).
  DevBuf Gd, CdD, Z2, Z2d, Z3d, W1d, Lamd, PsiD, T1d, T2d, dz, dw, dt2;
  Gd.alloc(L.pG.total * sizeof(double));
  Z2.alloc(pZ.total * sizeof(T));
  Z3d.alloc(pZ.total * sizeof(double));
  W1d.alloc(pW.total * sizeof(double));
  Lamd.alloc(pW.total * sizeof(double));
  PsiD.alloc(L.pPsi.total * sizeof(double));
  T1d.alloc(pT1.total * sizeof(double));
  T2d.alloc(pT2.total * sizeof(double));
  upload(dz, pZ.off, st);
  upload(dw, pW.off, st);
  upload(dt2, pT2.off, st);
  // B operands of the mixed products must be FP64
  const double* cdd = nullptr;
  const double* z2d = nullptr;
  if constexpr (std::is_same<T, double>::value) {
    cdd = dptr<double>(L.Cd);
    z2d = dptr<double>(Z2);
  } else {
    CdD.alloc(L.pCd.total * sizeof(double));
    Z2d.alloc(pZ.total * sizeof(double));
    convert<double, T>(st, dptr<double>(CdD), dptr<T>(L.Cd), L.pCd.total);
    cdd = dptr<double>(CdD);
    z2d = dptr<double>(Z2d);
  }
  std::vector<GemmDesc> d;
  // Yd = L_D^{-1} C_D^T
  d.clear();
  for (int s = 0; s < ns; ++s)
    d.push_back(GemmDesc{L.nd[s], L.ncp[s], L.nd[s], std::max(L.nd[s], 1), std::max(L.ncp[s], 1),
                         std::max(L.nd[s], 1), L.pLD.off[s], L.pCd.off[s], L.pY.off[s]});
  gemm_batched<double, T>(st, ring, d, G_TRI_A_LOWER | G_TRANS_B | G_TUNE, 1.0, 0.0, dptr<T>(L.LinvD), cdd, dptr<double>(L.Yd));
  // G = Yd^T Yd (FP64, positive semi-definite by construction), Ginvd = G^{-1}
  d.clear();
  for (int s = 0; s < ns; ++s)
    d.push_back(GemmDesc{L.ncp[s], L.ncp[s], L.nd[s], std::max(L.nd[s], 1), std::max(L.nd[s], 1),
                         std::max(L.ncp[s], 1), L.pY.off[s], L.pY.off[s], L.pG.off[s]});
  gemm_batched<double>(st, ring, d, G_TRANS_A | G_TUNE, 1.0, 0.0, dptr<double>(L.Yd), dptr<double>(L.Yd), dptr<double>(Gd));
  DevBuf dgo;
  upload(dgo, L.pG.off, st);
  small_spd_inverse<double>(st, dptr<double>(L.Ginvd), dptr<double>(Gd), dptr<int64_t>(dgo), dptr<int64_t>(L.par), ns,
                            imax(L.ncp), dptr<int>(status));
  check_status("constraint Schur complement C_D S_DD^{-1} C_D^T (dependent constraint rows)", AMB_EASSUMPTION);
  // factor-precision copies for the pair preconditioner of LOBPCG
  convert<T, double>(st, dptr<T>(L.Y), dptr<double>(L.Yd), L.pY.total);
  convert<T, double>(st, dptr<T>(L.Ginv), dptr<double>(L.Ginvd), L.pG.total);
  // R = [-S_Dc | 0]; Z3 = L_D^{-1} R
  psi_rhs<T>(st, dptr<T>(Z2), dptr<int64_t>(dz), dptr<T>(L.S), dptr<int64_t>(L.par), ns, imax(L.nd), imax(L.nc));
  if constexpr (!std::is_same<T, double>::value)
    convert<double, T>(st, dptr<double>(Z2d), dptr<T>(Z2), pZ.total);
  // only the corner columns of R are nonzero: Z3 = [L_D^{-1} R_c | 0]
  AMB_CUDA(cudaMemsetAsync(Z3d.p, 0, pZ.total * sizeof(double), st));
  d.clear();
  for (int s = 0; s < ns; ++s)
    d.push_back(GemmDesc{L.nd[s], L.ncrn[s], L.nd[s], std::max(L.nd[s], 1), std::max(L.nd[s], 1),
                         std::max(L.nd[s], 1), L.pLD.off[s], pZ.off[s], pZ.off[s]});
  gemm_batched<double, T>(st, ring, d, G_TRI_A_LOWER | G_TUNE, 1.0, 0.0, dptr<T>(L.LinvD), z2d, dptr<double>(Z3d));
  // W1 = Yd^T Z3 - [0 | I]
  d.clear();
  for (int s = 0; s < ns; ++s)
    d.push_back(GemmDesc{L.ncp[s], L.nc[s], L.nd[s], std::max(L.nd[s], 1), std::max(L.nd[s], 1),
                         std::max(L.ncp[s], 1), L.pY.off[s], pZ.off[s], pW.off[s]});
  gemm_batched<double>(st, ring, d, G_TRANS_A | G_TUNE, 1.0, 0.0, dptr<double>(L.Yd), dptr<double>(Z3d), dptr<double>(W1d));
  sub_identity<double>(st, dptr<double>(W1d), dptr<int64_t>(dw), dptr<int64_t>(L.par), ns, imax(L.ncp));
  // Lam = G^{-1} W1
  d.clear();
  for (int s = 0; s < ns; ++s)
    d.push_back(GemmDesc{L.ncp[s], L.nc[s], L.ncp[s], std::max(L.ncp[s], 1), std::max(L.ncp[s], 1),
                         std::max(L.ncp[s], 1), L.pG.off[s], pW.off[s], pW.off[s]});
  gemm_batched<double>(st, ring, d, G_TUNE, 1.0, 0.0, dptr<double>(L.Ginvd), dptr<double>(W1d), dptr<double>(Lamd));
  // Z3 -= Yd Lam
  d.clear();
  for (int s = 0; s < ns; ++s)
    d.push_back(GemmDesc{L.nd[s], L.nc[s], L.ncp[s], std::max(L.nd[s], 1), std::max(L.ncp[s], 1),
                         std::max(L.nd[s], 1), L.pY.off[s], pW.off[s], pZ.off[s]});
  gemm_batched<double>(st, ring, d, 0, -1.0, 1.0, dptr<double>(L.Yd), dptr<double>(Lamd), dptr<double>(Z3d));
  // Psi_D = L_D^{-T} Z3 ; Psi_c = [I 0]  (FP64; the factor-precision copy feeds Algorithm 1)
  AMB_CUDA(cudaMemsetAsync(PsiD.p, 0, L.pPsi.total * sizeof(double), st));
  d.clear();
  for (int s = 0; s < ns; ++s)
    d.push_back(GemmDesc{L.nd[s], L.nc[s], L.nd[s], std::max(L.nd[s], 1), std::max(L.nd[s], 1),
                         std::max(L.ng[s], 1), L.pLD.off[s], pZ.off[s], L.pPsi.off[s]});
  gemm_batched<double, T>(st, ring, d, G_TRANS_A | G_TRI_A_UPPER | G_TUNE, 1.0, 0.0, dptr<T>(L.LinvD), dptr<double>(Z3d),
                          dptr<double>(PsiD));
  psi_corner_rows<double>(st, dptr<double>(PsiD), dptr<int64_t>(L.par), ns, imax(L.nc));
  convert<T, double>(st, dptr<T>(L.Psi), dptr<double>(PsiD), L.pPsi.total);
  // Ac = Psi^T S Psi: S Psi = C^T(-mu) is small where S and Psi are not (it
  // cancels on every unconstrained dof): S Psi with the FP64 Psi and extended
  // accumulation over S, then Psi^T (S Psi) in FP64
  std::vector<GemmDesc> d1, d2;
  for (int s = 0; s < ns; ++s) {
    d1.push_back(GemmDesc{L.ng[s], L.nc[s], L.ng[s], std::max(L.ng[s], 1), std::max(L.ng[s], 1),
                          std::max(L.ng[s], 1), L.pS.off[s], L.pPsi.off[s], pT1.off[s]});
    d2.push_back(GemmDesc{L.nc[s], L.nc[s], L.ng[s], std::max(L.ng[s], 1), std::max(L.ng[s], 1),
                          std::max(L.nc[s], 1), L.pPsi.off[s], pT1.off[s], pT2.off[s]});
  }
  gemm_batched<double, T>(st, ring, d1, G_TUNE, 1.0, 0.0, dptr<T>(L.S), dptr<double>(PsiD), dptr<double>(T1d));
  gemm_batched<double>(st, ring, d2, G_TRANS_A | G_TUNE, 1.0, 0.0, dptr<double>(PsiD), dptr<double>(T1d), dptr<double>(T2d));
  coarse_to_double<double>(st, dptr<double>(L.Ac), dptr<double>(T2d), dptr<int64_t>(dt2), dptr<int64_t>(L.par), ns,
                           imax(L.nc));
  AMB_CUDA(cudaStreamSynchronize(st));
}

template <typename T>
void Engine<T>::setup_top() {
  FamTimer ft(st, &tm, AMB_FAM_COARSE, timing());
  LevelData<T>& L = *lv.back();
  nC = L.topo.n_coarse;
  if (nC == 0) return;
  AC.alloc((size_t)nC * nC * sizeof(double));
  LinvC.alloc((size_t)nC * nC * sizeof(double));
  topT.alloc((size_t)nC * sizeof(double));
  AMB_CUDA(cudaMemsetAsync(AC.p, 0, (size_t)nC * nC * sizeof(double), st));
  top_assemble(st, dptr<double>(AC), nC, dptr<double>(L.Ac), dptr<int64_t>(L.rc), dptr<int64_t>(L.par), L.nc);
  std::vector<CholDesc> d{CholDesc{0, (int32_t)nC, (int32_t)nC, 0, (int32_t)nC, 0, (int32_t)nC, -1}};
  double fl = 0;
  partial_cholesky<double>(st, ring, d, dptr<double>(AC), dptr<double>(LinvC), dptr<int>(status), &fl);
  check_status("top-level coarse factorization", AMB_EASSUMPTION);
  std::vector<TrtriDesc> t{TrtriDesc{0, 0, (int32_t)nC, (int32_t)nC, (int32_t)nC, 0}};
  trtri_from_blocks<double>(st, ring, t, dptr<double>(AC), dptr<double>(LinvC), &fl);
  AMB_CUDA(cudaStreamSynchronize(st));
}

template <typename T>
void Engine<T>::setup() {
  const int initial = cfg.opt.initial_constraints;
  const LevelData<T>* prev = nullptr;
  for (int i = 0; i < cfg.levels - 1; ++i) {
    auto L = std::make_unique<LevelData<T>>();
    L->level = i + 1;
    std::vector<int32_t> loc;
    EventPair ev;
    ev.start(st);
    if (i == 0) {
      std::vector<int32_t> elem_local;
      L->topo = build_level_one(mesh.nx, mesh.ny, mesh.nz, mesh.dpn, mesh.dir_h.data(), mesh.elem_sub_h.data(),
                                cfg.nsubs[0], initial, elem_local);
      upload(mesh.elem_local, elem_local, st);
    } else {
      L->topo = build_level_next(prev->topo, cfg.parents[i - 1].data(), cfg.nsubs[i], initial, loc);
    }
    alloc_level(*L);
    assemble(*L, prev, loc);
    tm.phase_ms[0] += ev.lap(st);
    ev.start(st);
    factor_level(*L);
    tm.phase_ms[1] += ev.lap(st);
    ev.start(st);
    coarse_basis(*L);
    tm.phase_ms[4] += ev.lap(st);
    if (cfg.opt.adaptive) {
      ev.start(st);
      adapt_level(*L);
      tm.phase_ms[2] += ev.lap(st);
      ev.start(st);
      coarse_basis(*L);
      tm.phase_ms[4] += ev.lap(st);
    } else {
      omega.push_back(0.0);
      nadapt.push_back(0);
    }
    lv.push_back(std::move(L));
    prev = lv.back().get();
  }
  setup_top();
}

// ------------------------------------------------------------------ Algorithm 1

template <typename T>
void Engine<T>::drop_graph() {
  if (pgraph) {
    cudaStreamSynchronize(st);   // a replay may still be running
    cudaGraphExecDestroy(pgraph);
  }
  pgraph = nullptr;
  pg_r = nullptr;
  pg_z = nullptr;
}

template <typename T>
void Engine<T>::precond(const double* r, double* z) {
  if (!pgraph || r != pg_r || z != pg_z) {
    drop_graph();
    // the graph's descriptor uploads copy from gring's pinned host buffer at
    // every replay, so gring is written only here and never wraps
    gring.reset(kGraphRingBytes);
    // capture on a private stream (the context's stream may be the legacy
    // NULL stream, which cannot be captured); the graph is launched on the
    // context's stream, so ordering with the caller's work is unchanged
    if (!cstream) AMB_CUDA(cudaStreamCreateWithFlags(&cstream, cudaStreamNonBlocking));
    const cudaStream_t st0 = st;
    st = cstream;
    aring = &gring;
    cudaGraph_t g = nullptr;
    const int64_t l0 = g_launches;
    AMB_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
      apply_level(0, r, z);
    } catch (...) {
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      aring = &ring;
      st = st0;
      throw;
    }
    const cudaError_t ec = cudaStreamEndCapture(st, &g);
    aring = &ring;
    st = st0;
    AMB_CUDA(ec);
    // captured kernels did not run: count them at every replay instead
    pg_kernels = g_launches - l0;
    g_launches = l0;
    const cudaError_t e = cudaGraphInstantiate(&pgraph, g, 0);
    cudaGraphDestroy(g);
    AMB_CUDA(e);
    pg_r = r;
    pg_z = z;
  }
  AMB_CUDA(cudaGraphLaunch(pgraph, st));
  g_launches += pg_kernels;
  ++pg_replays;
}

template <typename T>
void Engine<T>::apply_level(int i, const double* r, double* u) {
  DescRing& ring = aring ? *aring : this->ring;
  LevelData<T>& L = *lv[i];
  const int ns = L.ns;
  const T one = T(1), zero = T(0);
  AMB_CUDA(cudaMemsetAsync(u, 0, L.topo.n_dofs * sizeof(double), st));
  std::vector<GemvDesc> d;
  auto mk = [](int m, int n, int lda, int64_t a, int64_t x, int64_t y) {
    return GemvDesc{m, n, std::max(lda, 1), 0, a, x, y};
  };
  // eq. ML-uIi: u_I = A_II^{-1} r_I, kept as t = L^{-1} r_I
  gather<T, double>(st, dptr<T>(L.xI), r, dptr<int64_t>(L.idof), L.vI.total);
  d.clear();
  for (int s = 0; s < ns; ++s) d.push_back(mk(L.ni[s], L.ni[s], L.ni[s], L.pLI.off[s], L.vI.off[s], L.vI.off[s]));
  gemv_batched<T>(st, ring, d, G_TRI_A_LOWER, one, zero, dptr<T>(L.LinvI), dptr<T>(L.xI), dptr<T>(L.tI));
  // eq. ML-rBi: r_B = r - A u_I on the interface: K_GI A_II^{-1} r_I = X^T t
  d.clear();
  for (int s = 0; s < ns; ++s) d.push_back(mk(L.ng[s], L.ni[s], L.nn[s], L.pM.off[s] + L.ni[s], L.vI.off[s], L.vG.off[s]));
  gemv_batched<T>(st, ring, d, 0, one, zero, dptr<T>(L.M), dptr<T>(L.tI), dptr<T>(L.gG));
  iface_residual<T>(st, dptr<double>(L.rB), r, dptr<int64_t>(L.iface_dof), dptr<int32_t>(L.own_off),
                    dptr<int32_t>(L.own_flat), dptr<T>(L.gG), L.n_iface);
  // E^T: g^s = D^s R^s r_B
  gather32<T, double>(st, dptr<T>(L.gG), dptr<double>(L.rB), dptr<int32_t>(L.gidx), dptr<T>(L.w), L.vG.total);
  // eq. ML-wDi: Neumann problem with the coarse dofs fixed: corners zero, the
  // rest through S_DD^{-1} and the constraint Schur complement G
  d.clear();
  for (int s = 0; s < ns; ++s) d.push_back(mk(L.nd[s], L.nd[s], L.nd[s], L.pLD.off[s], L.vG.off[s], L.vD.off[s]));
  gemv_batched<T>(st, ring, d, G_TRI_A_LOWER, one, zero, dptr<T>(L.LinvD), dptr<T>(L.gG), dptr<T>(L.zD));
  // G correction in FP64 (constraint space): q = Yd^T z; l = Ginvd q; z -= Yd l
  double* zd = nullptr;
  if constexpr (std::is_same<T, double>::value) {
    zd = dptr<double>(L.zD);
  } else {
    zd = dptr<double>(L.zDd);
    convert<double, T>(st, zd, dptr<T>(L.zD), L.vD.total);
  }
  d.clear();
  for (int s = 0; s < ns; ++s) d.push_back(mk(L.nd[s], L.ncp[s], L.nd[s], L.pY.off[s], L.vD.off[s], L.vCP.off[s]));
  gemv_batched<double>(st, ring, d, G_TRANS_A, 1.0, 0.0, dptr<double>(L.Yd), zd, dptr<double>(L.qCPd));
  d.clear();
  for (int s = 0; s < ns; ++s) d.push_back(mk(L.ncp[s], L.ncp[s], L.ncp[s], L.pG.off[s], L.vCP.off[s], L.vCP.off[s]));
  gemv_batched<double>(st, ring, d, 0, 1.0, 0.0, dptr<double>(L.Ginvd), dptr<double>(L.qCPd), dptr<double>(L.lCPd));
  d.clear();
  for (int s = 0; s < ns; ++s) d.push_back(mk(L.nd[s], L.ncp[s], L.nd[s], L.pY.off[s], L.vCP.off[s], L.vD.off[s]));
  gemv_batched<double>(st, ring, d, 0, -1.0, 1.0, dptr<double>(L.Yd), dptr<double>(L.lCPd), zd);
  if constexpr (!std::is_same<T, double>::value) convert<T, double>(st, dptr<T>(L.zD), zd, L.vD.total);
  AMB_CUDA(cudaMemsetAsync(L.vGw.p, 0, L.vG.total * sizeof(T), st));
  d.clear();
  for (int s = 0; s < ns; ++s) d.push_back(mk(L.nd[s], L.nd[s], L.nd[s], L.pLD.off[s], L.vD.off[s], L.vG.off[s]));
  gemv_batched<T>(st, ring, d, G_TRANS_A | G_TRI_A_UPPER, one, zero, dptr<T>(L.LinvD), dptr<T>(L.zD), dptr<T>(L.vGw));
  // eq. ML-coarse / ML-ri+1: r_{i+1} = sum R_c^T Psi^T g
  d.clear();
  for (int s = 0; s < ns; ++s) d.push_back(mk(L.ng[s], L.nc[s], L.ng[s], L.pPsi.off[s], L.vG.off[s], L.vC.off[s]));
  gemv_batched<T>(st, ring, d, G_TRANS_A, one, zero, dptr<T>(L.Psi), dptr<T>(L.gG), dptr<T>(L.cC));
  owner_sum<T>(st, dptr<double>(L.rcg), dptr<int32_t>(L.cown_off), dptr<int32_t>(L.cown_flat), dptr<T>(L.cC), nullptr,
               nullptr, nullptr, L.topo.n_coarse);
  if (i == (int)lv.size() - 1) {
    if (nC > 0) {
      std::vector<GemvDesc> t{GemvDesc{(int)nC, (int)nC, (int)nC, 0, 0, 0, 0}};
      gemv_batched<double>(st, ring, t, G_TRI_A_LOWER, 1.0, 0.0, dptr<double>(LinvC), dptr<double>(L.rcg),
                           dptr<double>(topT));
      gemv_batched<double>(st, ring, t, G_TRANS_A | G_TRI_A_UPPER, 1.0, 0.0, dptr<double>(LinvC), dptr<double>(topT),
                           dptr<double>(L.ucg));
    }
  } else {
    apply_level(i + 1, dptr<double>(L.rcg), dptr<double>(L.ucg));
  }
  // eq. ML-uBi-1: u_B = E (w + Psi u_c)
  gather<T, double>(st, dptr<T>(L.ucC), dptr<double>(L.ucg), dptr<int64_t>(L.rc), L.vC.total);
  d.clear();
  for (int s = 0; s < ns; ++s) d.push_back(mk(L.ng[s], L.nc[s], L.ng[s], L.pPsi.off[s], L.vC.off[s], L.vG.off[s]));
  gemv_batched<T>(st, ring, d, 0, one, one, dptr<T>(L.Psi), dptr<T>(L.ucC), dptr<T>(L.vGw));
  owner_sum<T>(st, dptr<double>(L.uGd), dptr<int32_t>(L.own_off), dptr<int32_t>(L.own_flat), dptr<T>(L.vGw), dptr<T>(L.w),
               u, dptr<int64_t>(L.iface_dof), L.n_iface);
  // eq. ML-vIi, ML-ui: u_I = L^{-T} (t - X u_G)
  gather32<T, double>(st, dptr<T>(L.gG), dptr<double>(L.uGd), dptr<int32_t>(L.gidx), nullptr, L.vG.total);
  d.clear();
  for (int s = 0; s < ns; ++s) d.push_back(mk(L.ng[s], L.ni[s], L.nn[s], L.pM.off[s] + L.ni[s], L.vG.off[s], L.vI.off[s]));
  gemv_batched<T>(st, ring, d, G_TRANS_A, T(-1), one, dptr<T>(L.M), dptr<T>(L.gG), dptr<T>(L.tI));
  d.clear();
  for (int s = 0; s < ns; ++s) d.push_back(mk(L.ni[s], L.ni[s], L.ni[s], L.pLI.off[s], L.vI.off[s], L.vI.off[s]));
  gemv_batched<T>(st, ring, d, G_TRANS_A | G_TRI_A_UPPER, one, zero, dptr<T>(L.LinvI), dptr<T>(L.tI), dptr<T>(L.xI));
  scatter<double, T>(st, u, dptr<T>(L.xI), dptr<int64_t>(L.idof), L.vI.total);
}

template <typename T>
void Engine<T>::schur_apply(int level, int width, const void* x, void* y) {
  AMB_CHECK(level >= 1 && level <= (int)lv.size(), AMB_EINVAL, "level out of range");
  AMB_CHECK(width >= 1, AMB_EINVAL, "width must be >= 1");
  LevelData<T>& L = *lv[level - 1];
  FamTimer ft(st, &tm, AMB_FAM_SCHUR, timing());
  std::vector<GemmDesc> d;
  int64_t off = 0;
  double fl = 0, by = 0;
  for (int s = 0; s < L.ns; ++s) {
    const int ng = L.ng[s];
    d.push_back(GemmDesc{ng, width, ng, std::max(ng, 1), std::max(ng, 1), std::max(ng, 1), L.pS.off[s], off, off});
    off += (int64_t)ng * width;
    fl += 2.0 * ng * ng * width;
    by += (double)ng * ng * sizeof(T) + 2.0 * ng * width * sizeof(T);
  }
  bool tc = false;
  if (width == 1) {
    std::vector<GemvDesc> g;
    for (auto& q : d) g.push_back(GemvDesc{q.m, q.k, q.lda, 0, q.a, q.b, q.c});
    gemv_batched<T>(st, ring, g, 0, T(1), T(0), dptr<T>(L.S), static_cast<const T*>(x), static_cast<T*>(y));
  } else if constexpr (std::is_same<T, float>::value) {
    if (width >= kTcSchurWidth) {
      // FP32 form, wide blocks: tensor cores (3xTF32); Y(i, j) = sum_k S(i, k) X(k, j), X read K-major
      std::vector<TcGemm> t;
      for (auto& q : d) t.push_back(TcGemm{q.a, q.b, q.c, q.lda, q.ldb, q.ldc, q.m, q.n, q.k, 0, 1, 0});
      tc_gemm(st, ring, t, 1.f, 0.f, dptr<float>(L.S), static_cast<const float*>(x), static_cast<float*>(y),
              dptr<int>(status));
      tc = true;
    } else {
      gemm_batched<T>(st, ring, d, 0, T(1), T(0), dptr<T>(L.S), static_cast<const T*>(x), static_cast<T*>(y));
    }
  } else {
    gemm_batched<T>(st, ring, d, 0, T(1), T(0), dptr<T>(L.S), static_cast<const T*>(x), static_cast<T*>(y));
  }
  tm.fam_flops[AMB_FAM_SCHUR] += fl;
  tm.fam_bytes[AMB_FAM_SCHUR] += by;
  if (tc) check_status("Schur apply on the tensor cores", AMB_ETIMEOUT);
}

template <typename T>
void Engine<T>::schur_apply_staged(int level, int width, const void* x, void* y, void* scratch, size_t bytes) {
  AMB_CHECK(level >= 1 && level <= (int)lv.size(), AMB_EINVAL, "level out of range");
  AMB_CHECK(width >= 1, AMB_EINVAL, "width must be >= 1");
  const LevelData<T>& L = *lv[level - 1];
  AMB_CHECK(L.ns <= kStagedMaxDesc, AMB_EINVAL,
            "more than " + std::to_string(kStagedMaxDesc) + " substructures on the level");
  // descriptors are built in per-thread host buffers of static storage
  // (allocated on a thread's first call, never on the device); they are
  // large (about 90 KB together), so they stay off the stack, whose size a
  // caller's thread may limit
  static thread_local std::vector<GemmDesc> gd_buf(kStagedMaxDesc);
  static thread_local std::vector<GemvDesc> vd_buf(kStagedMaxDesc);
  static thread_local std::vector<int> pre_buf(kStagedMaxDesc + 1);
  GemmDesc* gd = gd_buf.data();
  GemvDesc* vd = vd_buf.data();
  int* prefix = pre_buf.data();
  int nd = 0, total = 0;
  int64_t off = 0;
  for (int s = 0; s < L.ns; ++s) {
    const int ng = L.ng[s];
    if (ng == 0) continue;
    prefix[nd] = total;
    if (width == 1) {
      vd[nd] = GemvDesc{ng, ng, ng, 0, L.pS.off[s], off, off};
      total += gemv_ctas(vd[nd], false);
    } else {
      gd[nd] = GemmDesc{ng, width, ng, ng, ng, ng, L.pS.off[s], off, off};
      total += gemm_ctas<T>(gd[nd]);
    }
    off += (int64_t)ng * width;
    ++nd;
  }
  prefix[nd] = total;
  if (nd == 0) return;
  const size_t dbytes = (size_t)nd * (width == 1 ? sizeof(GemvDesc) : sizeof(GemmDesc));
  const size_t poff = (dbytes + 255) & ~size_t(255);
  AMB_CHECK(poff + (size_t)(nd + 1) * sizeof(int) <= bytes, AMB_EINVAL, "launch descriptors exceed the scratch size");
  char* sc = static_cast<char*>(scratch);
  AMB_CUDA(cudaMemcpyAsync(sc, width == 1 ? (const void*)vd : (const void*)gd, dbytes, cudaMemcpyHostToDevice, st));
  AMB_CUDA(cudaMemcpyAsync(sc + poff, prefix, (size_t)(nd + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  const int* dpre = reinterpret_cast<const int*>(sc + poff);
  if (width == 1)
    gemv_launch_prepared<T>(st, reinterpret_cast<const GemvDesc*>(sc), dpre, nd, total, 0, T(1), T(0),
                            dptr<T>(L.S), static_cast<const T*>(x), static_cast<T*>(y));
  else
    gemm_launch_prepared<T>(st, reinterpret_cast<const GemmDesc*>(sc), dpre, nd, total, 0, T(1), T(0),
                            dptr<T>(L.S), static_cast<const T*>(x), static_cast<T*>(y));
}

// ------------------------------------------------------------------ exports

template <typename T>
void Engine<T>::export_sub(int what, int level, int idx, std::vector<char>& out) {
  AMB_CHECK(level >= 1 && level <= (int)lv.size(), AMB_EINVAL, "level out of range");
  LevelData<T>& L = *lv[level - 1];
  const LevelTopo& tp = L.topo;
  auto put = [&](const void* p, size_t n) {
    size_t o = out.size();
    out.resize(o + n);
    if (n) memcpy(out.data() + o, p, n);
  };
  if (what == AMB_X_CORNERS) {
    put(tp.corner_dofs.data(), tp.corner_dofs.size() * sizeof(int64_t));
    return;
  }
  if (what == AMB_X_PAIR_ROWS) {
    AMB_CHECK(idx >= 0 && idx < (int)tp.pairs.size(), AMB_EINVAL, "pair index out of range");
    const auto& rows = L.pair_rows.empty() ? std::vector<std::vector<double>>() : L.pair_rows[idx];
    for (auto& r : rows) put(r.data(), r.size() * sizeof(double));
    put(tp.pairs[idx].face_dofs.data(), tp.pairs[idx].face_dofs.size() * sizeof(int64_t));
    return;
  }
  AMB_CHECK(idx >= 0 && idx < L.ns, AMB_EINVAL, "substructure index out of range");
  const SubTopo& sb = tp.subs[idx];
  if (what == AMB_X_SUB_DOFS) {
    put(sb.dofs.data(), sb.dofs.size() * sizeof(int64_t));
  } else if (what == AMB_X_SUB_SIZES) {
    int32_t v[4] = {sb.n_i, sb.n_g, sb.n_crn, sb.n_c()};
    put(v, sizeof(v));
  } else if (what == AMB_X_SCHUR) {
    std::vector<T> h((size_t)sb.n_g * sb.n_g);
    AMB_CUDA(cudaMemcpyAsync(h.data(), dptr<T>(L.S) + L.pS.off[idx], h.size() * sizeof(T), cudaMemcpyDeviceToHost, st));
    AMB_CUDA(cudaStreamSynchronize(st));
    std::vector<double> dd(h.begin(), h.end());
    put(dd.data(), dd.size() * sizeof(double));
  } else if (what == AMB_X_COARSE_EL) {
    std::vector<double> h((size_t)L.nc[idx] * L.nc[idx]);
    AMB_CUDA(cudaMemcpyAsync(h.data(), dptr<double>(L.Ac) + L.pAc.off[idx], h.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    AMB_CUDA(cudaStreamSynchronize(st));
    put(h.data(), h.size() * sizeof(double));
  } else if (what == AMB_X_CONSTR) {
    const int nc = sb.n_c(), ng = sb.n_g;
    std::vector<double> c((size_t)nc * ng, 0.0);
    for (int q = 0; q < sb.n_crn; ++q) c[(size_t)q * ng + sb.n_d() + q] = 1.0;
    for (int q = 0; q < (int)sb.crows.size(); ++q)
      for (auto& e : sb.crows[q]) c[(size_t)(sb.n_crn + q) * ng + e.first] = e.second;
    put(c.data(), c.size() * sizeof(double));
  } else {
    throw Error(AMB_EINVAL, "unknown export kind");
  }
}

template class Engine<float>;
template class Engine<double>;

std::unique_ptr<EngineBase> make_engine(int precision, Mesh& mesh, const EngineConfig& cfg, cudaStream_t st,
                                        DescRing& ring, Timers& tm, std::vector<PairReportH>& reports,
                                        std::vector<double>& omega, std::vector<int>& nadapt, DevBuf& status) {
  if (precision == AMB_FP32)
    return std::make_unique<Engine<float>>(mesh, cfg, st, ring, tm, reports, omega, nadapt, status);
  return std::make_unique<Engine<double>>(mesh, cfg, st, ring, tm, reports, omega, nadapt, status);
}

}  // namespace amb
