// Per-level helper kernels; see kernels.h.
#include "kernels.h"

namespace amb {

namespace {
inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }
}

// ------------------------------------------------------------------ gathers

template <typename To, typename Ti>
__global__ void k_gather(To* out, const Ti* in, const int64_t* idx, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (To)in[idx ? idx[i] : i];
}
template <typename To, typename Ti>
void gather(cudaStream_t st, To* out, const Ti* in, const int64_t* idx, int64_t n) {
  if (n <= 0) return;
  k_gather<To, Ti><<<blocks(n), 256, 0, st>>>(out, in, idx, n);
  AMB_LAUNCHED();
}

template <typename To, typename Ti>
__global__ void k_scatter(To* out, const Ti* in, const int64_t* idx, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[idx[i]] = (To)in[i];
}
template <typename To, typename Ti>
void scatter(cudaStream_t st, To* out, const Ti* in, const int64_t* idx, int64_t n) {
  if (n <= 0) return;
  k_scatter<To, Ti><<<blocks(n), 256, 0, st>>>(out, in, idx, n);
  AMB_LAUNCHED();
}

template <typename To, typename Ti>
__global__ void k_gather32(To* out, const Ti* in, const int32_t* gidx, const To* w, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  To v = (To)in[gidx[i]];
  out[i] = w ? w[i] * v : v;
}
template <typename To, typename Ti>
void gather32(cudaStream_t st, To* out, const Ti* in, const int32_t* gidx, const To* w, int64_t n) {
  if (n <= 0) return;
  k_gather32<To, Ti><<<blocks(n), 256, 0, st>>>(out, in, gidx, w, n);
  AMB_LAUNCHED();
}

#define INST_G(To, Ti)                                                                          \
  template void gather<To, Ti>(cudaStream_t, To*, const Ti*, const int64_t*, int64_t);          \
  template void scatter<To, Ti>(cudaStream_t, To*, const Ti*, const int64_t*, int64_t);         \
  template void gather32<To, Ti>(cudaStream_t, To*, const Ti*, const int32_t*, const To*, int64_t);
INST_G(float, double)
INST_G(double, double)
INST_G(double, float)
INST_G(float, float)

// ------------------------------------------------------------------ owner sums

template <typename T>
__global__ void k_iface_residual(double* rB, const double* r, const int64_t* dof, const int32_t* off,
                                 const int32_t* flat, const T* y, int64_t n) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = r[dof[j]];
  for (int q = off[j]; q < off[j + 1]; ++q) s -= (double)y[flat[q]];
  rB[j] = s;
}
template <typename T>
void iface_residual(cudaStream_t st, double* rB, const double* r, const int64_t* dof, const int32_t* off,
                    const int32_t* flat, const T* y, int64_t n) {
  if (n <= 0) return;
  k_iface_residual<T><<<blocks(n), 256, 0, st>>>(rB, r, dof, off, flat, y, n);
  AMB_LAUNCHED();
}

template <typename T>
__global__ void k_owner_sum(double* out, const int32_t* off, const int32_t* flat, const T* v, const T* w, double* u,
                            const int64_t* dof, int64_t n) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int q = off[j]; q < off[j + 1]; ++q) {
    const int f = flat[q];
    s += w ? (double)w[f] * (double)v[f] : (double)v[f];
  }
  out[j] = s;
  if (u) u[dof[j]] = s;
}
template <typename T>
void owner_sum(cudaStream_t st, double* out, const int32_t* off, const int32_t* flat, const T* v, const T* w,
               double* u, const int64_t* dof, int64_t n) {
  if (n <= 0) return;
  k_owner_sum<T><<<blocks(n), 256, 0, st>>>(out, off, flat, v, w, u, dof, n);
  AMB_LAUNCHED();
}

template <typename T>
__global__ void k_weights(T* w, const double* d, const int32_t* off, const int32_t* flat, int64_t n) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int q = off[j]; q < off[j + 1]; ++q) s += d[flat[q]];
  for (int q = off[j]; q < off[j + 1]; ++q) w[flat[q]] = (T)(d[flat[q]] / s);
}
template <typename T>
void scaling_weights(cudaStream_t st, T* w, const double* d, const int32_t* off, const int32_t* flat, int64_t n) {
  if (n <= 0) return;
  k_weights<T><<<blocks(n), 256, 0, st>>>(w, d, off, flat, n);
  AMB_LAUNCHED();
}

#define INST_O(T)                                                                                              \
  template void iface_residual<T>(cudaStream_t, double*, const double*, const int64_t*, const int32_t*,        \
                                  const int32_t*, const T*, int64_t);                                          \
  template void owner_sum<T>(cudaStream_t, double*, const int32_t*, const int32_t*, const T*, const T*, double*, \
                             const int64_t*, int64_t);                                                         \
  template void scaling_weights<T>(cudaStream_t, T*, const double*, const int32_t*, const int32_t*, int64_t);
INST_O(float)
INST_O(double)

// ------------------------------------------------------------------ per-substructure copies
#define PAR(s, f) par[(int64_t)(s) * NPAR + (f)]

template <typename T>
__global__ void k_extract_diag(double* diagG, const T* M, const int64_t* par) {
  const int s = blockIdx.y;
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= PAR(s, P_NG)) return;
  const int64_t ni = PAR(s, P_NI), nn = PAR(s, P_NN);
  diagG[PAR(s, P_VG) + l] = (double)M[PAR(s, P_OM) + (ni + l) * (nn + 1)];
}
template <typename T>
void extract_iface_diag(cudaStream_t st, double* diagG, const T* M, const int64_t* par, int ns, int max_ng) {
  if (max_ng <= 0 || ns <= 0) return;
  k_extract_diag<T><<<dim3(blocks(max_ng), ns), 256, 0, st>>>(diagG, M, par);
  AMB_LAUNCHED();
}

template <typename T>
__global__ void k_copy_schur(T* S, const T* M, const int64_t* par) {
  const int s = blockIdx.y;
  const int64_t ng = PAR(s, P_NG);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ng * ng) return;
  const int64_t l = idx % ng, m = idx / ng;
  const int64_t hi = l > m ? l : m, lo = l > m ? m : l;
  const int64_t ni = PAR(s, P_NI), nn = PAR(s, P_NN);
  S[PAR(s, P_OS) + idx] = M[PAR(s, P_OM) + (ni + hi) + (ni + lo) * nn];
}
template <typename T>
void copy_schur(cudaStream_t st, T* S, const T* M, const int64_t* par, int ns, int max_ng) {
  if (max_ng <= 0 || ns <= 0) return;
  k_copy_schur<T><<<dim3(blocks((int64_t)max_ng * max_ng), ns), 256, 0, st>>>(S, M, par);
  AMB_LAUNCHED();
}

template <typename T>
__global__ void k_scatter_values(T* base, const int64_t* off, const double* val, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) base[off[i]] = (T)val[i];
}
template <typename T>
void scatter_values(cudaStream_t st, T* base, const int64_t* off, const double* val, int64_t n) {
  if (n <= 0) return;
  k_scatter_values<T><<<blocks(n), 256, 0, st>>>(base, off, val, n);
  AMB_LAUNCHED();
}

template <typename T>
__global__ void k_psi_rhs(T* Z, const int64_t* zoff, const T* S, const int64_t* par) {
  const int s = blockIdx.y;
  const int64_t nd = PAR(s, P_ND), nc = PAR(s, P_NC), ncrn = PAR(s, P_NCRN), ng = PAR(s, P_NG);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nd * nc) return;
  const int64_t r = idx % nd, c = idx / nd;
  T v = T(0);
  if (c < ncrn) v = -S[PAR(s, P_OS) + r + (nd + c) * ng];
  Z[zoff[s] + idx] = v;
}
template <typename T>
void psi_rhs(cudaStream_t st, T* Z, const int64_t* zoff, const T* S, const int64_t* par, int ns, int max_nd, int max_nc) {
  if (ns <= 0 || (int64_t)max_nd * max_nc == 0) return;
  k_psi_rhs<T><<<dim3(blocks((int64_t)max_nd * max_nc), ns), 256, 0, st>>>(Z, zoff, S, par);
  AMB_LAUNCHED();
}

template <typename T>
__global__ void k_sub_identity(T* W1, const int64_t* woff, const int64_t* par) {
  const int s = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ncp = PAR(s, P_NCP), ncrn = PAR(s, P_NCRN);
  if (q >= ncp) return;
  W1[woff[s] + q + (ncrn + q) * ncp] -= T(1);
}
template <typename T>
void sub_identity(cudaStream_t st, T* W1, const int64_t* woff, const int64_t* par, int ns, int max_ncp) {
  if (ns <= 0 || max_ncp <= 0) return;
  k_sub_identity<T><<<dim3(blocks(max_ncp), ns), 256, 0, st>>>(W1, woff, par);
  AMB_LAUNCHED();
}

template <typename T>
__global__ void k_psi_corner_rows(T* Psi, const int64_t* par) {
  const int s = blockIdx.y;
  const int64_t ncrn = PAR(s, P_NCRN), nc = PAR(s, P_NC), nd = PAR(s, P_ND), ng = PAR(s, P_NG);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ncrn * nc) return;
  const int64_t r = idx % ncrn, c = idx / ncrn;
  Psi[PAR(s, P_OPSI) + (nd + r) + c * ng] = (c == r) ? T(1) : T(0);
}
template <typename T>
void psi_corner_rows(cudaStream_t st, T* Psi, const int64_t* par, int ns, int max_nc) {
  if (ns <= 0 || max_nc <= 0) return;
  k_psi_corner_rows<T><<<dim3(blocks((int64_t)max_nc * max_nc), ns), 256, 0, st>>>(Psi, par);
  AMB_LAUNCHED();
}

template <typename To, typename Ti>
__global__ void k_convert(To* out, const Ti* in, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (To)in[i];
}
template <typename To, typename Ti>
void convert(cudaStream_t st, To* out, const Ti* in, int64_t n) {
  if (n <= 0) return;
  k_convert<To, Ti><<<blocks(n), 256, 0, st>>>(out, in, n);
  AMB_LAUNCHED();
}
template void convert<double, float>(cudaStream_t, double*, const float*, int64_t);
template void convert<float, double>(cudaStream_t, float*, const double*, int64_t);
template void convert<double, double>(cudaStream_t, double*, const double*, int64_t);

template <typename T>
__global__ void k_coarse_to_double(double* Ac, const T* T1, const int64_t* toff, const int64_t* par) {
  const int s = blockIdx.y;
  const int64_t nc = PAR(s, P_NC);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nc * nc) return;
  const int64_t r = idx % nc, c = idx / nc;
  const T* t = T1 + toff[s];
  Ac[PAR(s, P_OAC) + idx] = 0.5 * ((double)t[r + c * nc] + (double)t[c + r * nc]);
}
template <typename T>
void coarse_to_double(cudaStream_t st, double* Ac, const T* T1, const int64_t* toff, const int64_t* par, int ns,
                      int max_nc) {
  if (ns <= 0 || max_nc <= 0) return;
  k_coarse_to_double<T><<<dim3(blocks((int64_t)max_nc * max_nc), ns), 256, 0, st>>>(Ac, T1, toff, par);
  AMB_LAUNCHED();
}

// Gauss-Jordan inverse of an SPD matrix (no pivoting needed), FP64 in
// dynamic shared memory, one CTA per substructure.
template <typename T>
__global__ void k_spd_inverse(T* Ginv, const T* G, const int64_t* goff, const int64_t* par, int* status) {
  extern __shared__ double a[];
  const int s = blockIdx.x;
  const int n = (int)PAR(s, P_NCP);
  if (n == 0) return;
  const T* g = G + goff[s];
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx % n, c = idx / n;
    a[idx] = 0.5 * ((double)g[r + c * n] + (double)g[c + r * n]);
  }
  __syncthreads();
  __shared__ double piv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      double p = a[k + k * n];
      if (!(p > 0.0)) {
        if (atomicCAS(status, 0, AMB_EASSUMPTION) == 0) {
          status[1] = s;
          status[2] = k;
        }
        p = 1.0;
      }
      piv = p;
    }
    __syncthreads();
    const double p = piv;
    // in-place Gauss-Jordan step k: a_ij -= a_ik a_kj / p, then row k /= p,
    // column k /= -p and a_kk = 1/p; after n steps a holds G^{-1}
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int r = idx % n, c = idx / n;
      if (r != k && c != k) a[idx] -= a[r + k * n] * a[k + c * n] / p;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      if (q != k) {
        a[q + k * n] = -a[q + k * n] / p;   // pivot column
        a[k + q * n] = a[k + q * n] / p;    // pivot row
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) a[k + k * n] = 1.0 / p;
    __syncthreads();
  }
  T* out = Ginv + goff[s];
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) out[idx] = (T)(a[idx]);
}
template <typename T>
void small_spd_inverse(cudaStream_t st, T* Ginv, const T* G, const int64_t* goff, const int64_t* par, int ns,
                       int max_ncp, int* status) {
  if (ns <= 0 || max_ncp <= 0) return;
  AMB_CHECK(max_ncp <= 160, AMB_EINVAL, "more than 160 non-corner constraints on one substructure");
  const size_t smem = (size_t)max_ncp * max_ncp * sizeof(double);
  AMB_CUDA(cudaFuncSetAttribute(k_spd_inverse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_spd_inverse<T><<<ns, 256, smem, st>>>(Ginv, G, goff, par, status);
  AMB_LAUNCHED();
}

#define INST_P(T)                                                                                              \
  template void extract_iface_diag<T>(cudaStream_t, double*, const T*, const int64_t*, int, int);              \
  template void copy_schur<T>(cudaStream_t, T*, const T*, const int64_t*, int, int);                          \
  template void scatter_values<T>(cudaStream_t, T*, const int64_t*, const double*, int64_t);                  \
  template void psi_rhs<T>(cudaStream_t, T*, const int64_t*, const T*, const int64_t*, int, int, int);        \
  template void sub_identity<T>(cudaStream_t, T*, const int64_t*, const int64_t*, int, int);                  \
  template void psi_corner_rows<T>(cudaStream_t, T*, const int64_t*, int, int);                               \
  template void coarse_to_double<T>(cudaStream_t, double*, const T*, const int64_t*, const int64_t*, int, int); \
  template void small_spd_inverse<T>(cudaStream_t, T*, const T*, const int64_t*, const int64_t*, int, int, int*);
INST_P(float)
INST_P(double)

// ------------------------------------------------------------------ reductions and PCG updates

__global__ void k_dot_partial(double* partial, const double* a, const double* b, int64_t n) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}
__global__ void k_dot_final(double* dst, const double* partial, int nb) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *dst = sh[0];
}
void dot(cudaStream_t st, double* dst, const double* a, const double* b, int64_t n, double* partial) {
  const int nb = 608;   // 4 x 152 SMs
  k_dot_partial<<<nb, 256, 0, st>>>(partial, a, b, n);
  AMB_LAUNCHED();
  k_dot_final<<<1, 256, 0, st>>>(dst, partial, nb);
  AMB_LAUNCHED();
}

__global__ void k_axpy2(double* x, double* r, const double* p, const double* q, double a, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = fma(a, p[i], x[i]);
  r[i] = fma(-a, q[i], r[i]);
}
void axpy2(cudaStream_t st, double* x, double* r, const double* p, const double* q, double alpha, int64_t n) {
  k_axpy2<<<blocks(n), 256, 0, st>>>(x, r, p, q, alpha, n);
  AMB_LAUNCHED();
}
__global__ void k_xpby(double* p, const double* z, double beta, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = fma(beta, p[i], z[i]);
}
void xpby(cudaStream_t st, double* p, const double* z, double beta, int64_t n) {
  k_xpby<<<blocks(n), 256, 0, st>>>(p, z, beta, n);
  AMB_LAUNCHED();
}
__global__ void k_sub_vec(double* out, const double* a, const double* b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] - b[i];
}
void sub_vec(cudaStream_t st, double* out, const double* a, const double* b, int64_t n) {
  k_sub_vec<<<blocks(n), 256, 0, st>>>(out, a, b, n);
  AMB_LAUNCHED();
}

// Extreme eigenvalues of the Lanczos tridiagonal T of CG,
// T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j,
// by Sturm-sequence multisection: the diagonal and the squared off-diagonal
// are formed once in shared memory; each half-warp narrows one extreme by
// counting at 16 interior points per round (17-fold per round).
__device__ int sturm_count(const double* dg, const double* e2, int k, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int j = 0; j < k; ++j) {
    q = dg[j] - x - (j > 0 ? e2[j] / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}
__global__ void k_tridiag_extremes(double* out, const double* alphas, const double* betas, int k) {
  extern __shared__ double tsh[];
  double* dg = tsh;
  double* e2 = tsh + k;
  __shared__ double bnd[2];
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    dg[j] = 1.0 / alphas[j] + (j > 0 ? betas[j - 1] / alphas[j - 1] : 0.0);
    e2[j] = j > 0 ? betas[j - 1] / (alphas[j - 1] * alphas[j - 1]) : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {   // Gershgorin bounds
    double lo = 1e300, hi = -1e300;
    for (int j = 0; j < k; ++j) {
      double r = 0.0;
      if (j > 0) r += sqrt(e2[j]);
      if (j < k - 1) r += sqrt(e2[j + 1]);
      lo = fmin(lo, dg[j] - r);
      hi = fmax(hi, dg[j] + r);
    }
    bnd[0] = lo;
    bnd[1] = hi;
  }
  __syncthreads();
  const int half = threadIdx.x >> 4, l = threadIdx.x & 15;   // half-warp 0: smallest, 1: largest
  const int target = half == 0 ? 1 : k;   // count of eigenvalues below x reaching target
  const unsigned mask = half == 0 ? 0x0000ffffu : 0xffff0000u;
  double a = bnd[0], b = bnd[1];
  for (int round = 0; round < 40 && b - a > 1e-15 * fmax(fabs(a), fabs(b)); ++round) {
    const double x = a + (b - a) * (l + 1) / 17.0;
    const int hit = sturm_count(dg, e2, k, x) >= target;
    // the first point reaching the target brackets the eigenvalue
    const unsigned bal = __ballot_sync(mask, hit) >> (half * 16);
    const int f = bal ? __ffs(bal) - 1 : 16;   // index of that point (16: none)
    const double na = f == 0 ? a : a + (b - a) * f / 17.0;
    const double nb = f == 16 ? b : a + (b - a) * (f + 1) / 17.0;
    a = na;
    b = nb;
  }
  if (l == 0) out[half] = 0.5 * (a + b);
}
void tridiag_extremes(cudaStream_t st, double* out, const double* alphas, const double* betas, int k) {
  if (k <= 0) return;
  const size_t smem = (size_t)2 * k * sizeof(double);
  AMB_CHECK(smem <= 200 * 1024, AMB_EINVAL, "Lanczos tridiagonal too long for the condition estimate");
  AMB_CUDA(cudaFuncSetAttribute(k_tridiag_extremes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_tridiag_extremes<<<1, 32, smem, st>>>(out, alphas, betas, k);
  AMB_LAUNCHED();
}

// Top coarse matrix: one launch per substructure, in order.  The coarse ids
// of one substructure are distinct, so a launch writes each entry at most
// once and the sums are formed in the same order on every run.
__global__ void k_top_assemble(double* AC, int64_t nC, const double* Ac, const int64_t* rc, const int64_t* par, int s) {
  const int64_t nc = PAR(s, P_NC);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nc * nc) return;
  const int64_t r = idx % nc, c = idx / nc;
  const int64_t base = PAR(s, P_VC);
  AC[rc[base + r] + rc[base + c] * nC] += Ac[PAR(s, P_OAC) + idx];
}
void top_assemble(cudaStream_t st, double* AC, int64_t nC, const double* Ac, const int64_t* rc, const int64_t* par,
                  const std::vector<int>& nc) {
  for (int s = 0; s < (int)nc.size(); ++s) {
    if (nc[s] <= 0) continue;
    k_top_assemble<<<blocks((int64_t)nc[s] * nc[s]), 256, 0, st>>>(AC, nC, Ac, rc, par, s);
    AMB_LAUNCHED();
  }
}

}  // namespace amb
