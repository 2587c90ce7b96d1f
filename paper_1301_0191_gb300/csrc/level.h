// Device-resident data of one decomposition level (HBM layout).
//
// Per substructure s (all column-major, pooled in one allocation per kind):
//   M     (n_i+n_g)^2   assembled local matrix, ordered [interior | delta |
//                        corner]; after set-up: L_II (top-left), X^T =
//                        (L_II^{-1} K_IG)^T (bottom-left), L_D (delta block)
//   S     n_g^2         Schur complement K_GG - X^T X (full symmetric)
//   LinvI n_i^2         explicit L_II^{-1} (lower)
//   LinvD n_d^2         explicit L_D^{-1}  (lower), S_DD = L_D L_D^T
//   Cd    n_cp x n_d    non-corner constraint rows (edge averages, adaptive)
//   Y     n_d x n_cp    L_D^{-1} Cd^T
//   Ginv  n_cp^2        (Y^T Y)^{-1}
//   Psi   n_g x n_c     coarse basis (eq. local_saddle_point_problem)
//   Ac    n_c^2 (FP64)  Psi^T S Psi, the level-(i+1) element matrix
#pragma once

#include <memory>
#include <vector>

#include "common.h"
#include "topology.h"

namespace amb {

struct Pools {
  std::vector<int64_t> off;   // per substructure element offset
  int64_t total = 0;
  void build(const std::vector<int64_t>& sizes) {
    off.resize(sizes.size());
    total = 0;
    for (size_t i = 0; i < sizes.size(); ++i) {
      off[i] = total;
      total += sizes[i];
    }
  }
};

template <typename T>
struct LevelData {
  int level = 1;               // 1-based
  LevelTopo topo;
  int ns = 0;
  std::vector<int> ni, ng, ncrn, nd, nc, ncp, nn;
  Pools pM, pS, pLI, pLD, pCd, pY, pG, pPsi, pAc;
  Pools vI, vG, vD, vC, vCP;   // flattened per-sub vector offsets
  DevBuf M, S, LinvI, LinvD, Cd, Y, Ginv, Psi, Ac;
  // FP64 constraint space in both forms: Yd = L_D^{-1} C_D^T and Ginvd =
  // (Yd^T Yd)^{-1}; Y and Ginv above are factor-precision copies used only
  // by the pair preconditioner of LOBPCG
  DevBuf Yd, Ginvd;
  DevBuf zDd, qCPd, lCPd;      // double work vectors of the G correction
  DevBuf diagG;                // double, diag(K_GG) before elimination (sum n_g)
  DevBuf w;                    // T, stiffness-scaling weights (sum n_g)
  // index maps
  DevBuf idof;                 // int64 level dof of each interior entry (sum n_i)
  DevBuf iface_dof;            // int64 level dof of each global interface index
  DevBuf own_off, own_flat;    // int32 CSR: global interface -> flat interface entry
  DevBuf gidx;                 // int32 flat interface entry -> global interface index
  DevBuf rc;                   // int64 flat coarse entry -> global coarse id (sum n_c)
  DevBuf cown_off, cown_flat;  // int32 CSR: global coarse -> flat coarse entry
  int64_t n_iface = 0;
  // work vectors (T): interior x2, interface x2, delta, coarse-nc x2
  DevBuf xI, tI, gG, vGw, zD, cC, ucC;
  DevBuf rB, rcg, ucg, uGd;    // double global vectors
  DevBuf par;                  // int64 ns x NPAR parameter table (kernels.h)
  std::vector<int64_t> par_h;
  std::vector<std::vector<std::vector<double>>> pair_rows;   // adaptive rows per pair (host copy)
  double factor_flops = 0, trtri_flops = 0;
};

}  // namespace amb
