// Per-level helper kernels (kernels.cu): interface gathers/scatters
// (E, E^T, residual assembly, Sec. 3 Algorithm 1 and Sec. 7 stiffness
// scaling), per-substructure copies, small dense inverses, reductions.
#pragma once

#include <vector>

#include "common.h"

namespace amb {

// Fields of the per-substructure parameter table (int64, ns x NPAR).
enum ParField {
  P_NI, P_NG, P_NCRN, P_ND, P_NC, P_NCP, P_NN,
  P_OM, P_OS, P_OLI, P_OLD, P_OCD, P_OY, P_OG, P_OPSI, P_OAC,
  P_VI, P_VG, P_VD, P_VC, P_VCP,
  NPAR
};

// out[i] = (To) in[idx[i]]  (idx == nullptr: identity)
template <typename To, typename Ti>
void gather(cudaStream_t st, To* out, const Ti* in, const int64_t* idx, int64_t n);
// out[idx[i]] = (To) in[i]
template <typename To, typename Ti>
void scatter(cudaStream_t st, To* out, const Ti* in, const int64_t* idx, int64_t n);
// out[i] = (To) in[gidx[i]] with int32 indices, optionally scaled by w[i]
template <typename To, typename Ti>
void gather32(cudaStream_t st, To* out, const Ti* in, const int32_t* gidx, const To* w, int64_t n);

// rB[j] = r[dof[j]] - sum_{owners} y[flat]  (global interface residual, eq. ML-rBi)
template <typename T>
void iface_residual(cudaStream_t st, double* rB, const double* r, const int64_t* dof, const int32_t* off,
                    const int32_t* flat, const T* y, int64_t n);
// out[j] = sum_{owners} (w ? w[flat] : 1) * v[flat]; if u: u[dof[j]] = out[j]  (E, eq. ML-uBi-1)
template <typename T>
void owner_sum(cudaStream_t st, double* out, const int32_t* off, const int32_t* flat, const T* v, const T* w,
               double* u, const int64_t* dof, int64_t n);
// stiffness-scaling weights from diag(K_GG): w[flat] = d[flat] / sum_{owners} d
template <typename T>
void scaling_weights(cudaStream_t st, T* w, const double* d, const int32_t* off, const int32_t* flat, int64_t n);

// diagG[vG + l] = M[oM + (ni + l)(nn + 1)]
template <typename T>
void extract_iface_diag(cudaStream_t st, double* diagG, const T* M, const int64_t* par, int ns, int max_ng);
// S (full) from the lower trailing block of M
template <typename T>
void copy_schur(cudaStream_t st, T* S, const T* M, const int64_t* par, int ns, int max_ng);
// scatter (offset, value) pairs
template <typename T>
void scatter_values(cudaStream_t st, T* base, const int64_t* off, const double* val, int64_t n);
// R := [-S_Dc | 0] into Z (nd x nc per sub, ld nd, offset vD*... given by zoff)
template <typename T>
void psi_rhs(cudaStream_t st, T* Z, const int64_t* zoff, const T* S, const int64_t* par, int ns, int max_nd, int max_nc);
// W1(:, ncrn + q) -= e_q  (W1 ncp x nc, ld ncp)
template <typename T>
void sub_identity(cudaStream_t st, T* W1, const int64_t* woff, const int64_t* par, int ns, int max_ncp);
// Psi corner rows: [I 0]
template <typename T>
void psi_corner_rows(cudaStream_t st, T* Psi, const int64_t* par, int ns, int max_nc);
// Ac (double, symmetrized) from T1 = Psi^T S Psi (T, nc x nc, ld nc at toff)
// elementwise type conversion
template <typename To, typename Ti>
void convert(cudaStream_t st, To* out, const Ti* in, int64_t n);

template <typename T>
void coarse_to_double(cudaStream_t st, double* Ac, const T* T1, const int64_t* toff, const int64_t* par, int ns,
                      int max_nc);
// Ginv = G^{-1} for small SPD G (order ncp <= 256), FP64 Gauss-Jordan in shared memory
template <typename T>
void small_spd_inverse(cudaStream_t st, T* Ginv, const T* G, const int64_t* goff, const int64_t* par, int ns,
                       int max_ncp, int* status);

// deterministic dot product (two-stage), result in dst (device double)
void dot(cudaStream_t st, double* dst, const double* a, const double* b, int64_t n, double* partial);
// PCG updates
void axpy2(cudaStream_t st, double* x, double* r, const double* p, const double* q, double alpha, int64_t n);
void xpby(cudaStream_t st, double* p, const double* z, double beta, int64_t n);
void sub_vec(cudaStream_t st, double* out, const double* a, const double* b, int64_t n);
// extreme eigenvalues of the CG Lanczos tridiagonal (bisection), out[0]=min, out[1]=max
void tridiag_extremes(cudaStream_t st, double* out, const double* alphas, const double* betas, int k);

// dense top-level coarse matrix: atomic scatter of every substructure's Ac
void top_assemble(cudaStream_t st, double* AC, int64_t nC, const double* Ac, const int64_t* rc, const int64_t* par,
                  const std::vector<int>& nc);

}  // namespace amb
