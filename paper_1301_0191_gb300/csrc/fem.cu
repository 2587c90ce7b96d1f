// Finite-element kernels (Sec. 2; Sec. 8.1 uses tri-linear hexahedra):
// the Q1 reference element, dense substructure assembly (level 1 from the
// elements, level >= 2 from the children's coarse matrices, Sec. 3), the
// matrix-free FP64 operator A p used by PCG, consistent loads and the
// element-wise adjoint gradient.
#include "fem.h"

namespace amb {

// Reference element for unit coefficient on a cube of side h: 2x2x2 Gauss
// (exact for Q1 on a box).  Node a = ax + 2 ay + 4 az; dof a*dpn + c.
__global__ void k_khat(double* khat, int dpn, double h, double nu) {
  const int nd = 8 * dpn;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nd * nd) return;
  const int r = idx % nd, c = idx / nd;
  const int a = r / dpn, ca = r % dpn, b = c / dpn, cb = c % dpn;
  const double g0 = 0.5 - 0.5 / sqrt(3.0), g1 = 0.5 + 0.5 / sqrt(3.0);
  double lam = 0.0, mu = 0.0;
  if (dpn == 3) {
    lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    mu = 1.0 / (2.0 * (1.0 + nu));
  }
  double sum = 0.0;
  for (int q = 0; q < 8; ++q) {
    const double x[3] = {(q & 1) ? g1 : g0, (q & 2) ? g1 : g0, (q & 4) ? g1 : g0};
    double ga[3], gb[3];
    for (int pass = 0; pass < 2; ++pass) {
      const int n = pass ? b : a;
      double* g = pass ? gb : ga;
      double f[3], df[3];
      for (int ax = 0; ax < 3; ++ax) {
        const int bit = (n >> ax) & 1;
        f[ax] = bit ? x[ax] : 1.0 - x[ax];
        df[ax] = bit ? 1.0 : -1.0;
      }
      g[0] = df[0] * f[1] * f[2] / h;
      g[1] = f[0] * df[1] * f[2] / h;
      g[2] = f[0] * f[1] * df[2] / h;
    }
    double v;
    if (dpn == 1) {
      v = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
    } else {
      // lam div(N_a e_ca) div(N_b e_cb) + mu (grad_cb N_a grad_ca N_b + delta grad N_a . grad N_b)
      v = lam * ga[ca] * gb[cb] + mu * (ga[cb] * gb[ca] + (ca == cb ? ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2] : 0.0));
    }
    sum += v;
  }
  khat[idx] = sum * 0.125 * h * h * h;
}

void compute_khat(cudaStream_t st, double* khat, int dpn, double h, double nu) {
  const int n = 64 * dpn * dpn;
  k_khat<<<(n + 255) / 256, 256, 0, st>>>(khat, dpn, h, nu);
  AMB_LAUNCHED();
}

// Level-1 assembly without atomics.  The elements are split into 8 colours
// by the parities of their grid coordinates; two elements of one colour share
// no node, so one colour pass adds to every entry of a substructure matrix
// (column-major, order n_s) at most once, and the passes run in a fixed
// order: the sums are the same on every run.
template <typename T>
__global__ void k_assemble1(T* M, const int64_t* sub_off, const int32_t* sub_n, const int32_t* elem_sub,
                            const int32_t* elem_local, const double* coeff, const double* khat, int nd, int nx,
                            int ny, int cx, int cy, int cz, int64_t hx, int64_t hy, int64_t ncol) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)nd * nd;
  if (idx >= ncol * per) return;
  const int64_t q = idx / per;
  const int rc = (int)(idx % per);
  const int64_t i = 2 * (q % hx) + cx, j = 2 * ((q / hx) % hy) + cy, k = 2 * (q / (hx * hy)) + cz;
  const int64_t e = i + nx * (j + (int64_t)ny * k);
  const int a = rc % nd, b = rc / nd;
  const int la = elem_local[e * nd + a], lb = elem_local[e * nd + b];
  if (la < 0 || lb < 0) return;
  const int s = elem_sub[e];
  const int64_t n = sub_n[s];
  T* dst = &M[sub_off[s] + la + lb * n];
  *dst += (T)(coeff[e] * khat[a + b * nd]);
}

template <typename T>
void assemble_level1(cudaStream_t st, T* M, const int64_t* sub_off, const int32_t* sub_n, const int32_t* elem_sub,
                     const int32_t* elem_local, const double* coeff, const double* khat, int nd, int nx, int ny,
                     int nz) {
  for (int c = 0; c < 8; ++c) {
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    const int64_t hx = (nx - cx + 1) / 2, hy = (ny - cy + 1) / 2, hz = (nz - cz + 1) / 2;
    const int64_t ncol = hx * hy * hz;
    if (ncol <= 0) continue;
    const int64_t total = ncol * nd * nd;
    k_assemble1<T><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(M, sub_off, sub_n, elem_sub, elem_local, coeff,
                                                                     khat, nd, nx, ny, cx, cy, cz, hx, hy, ncol);
    AMB_LAUNCHED();
  }
}

// Level >= 2: child s contributes its coarse matrix (FP64, order nc_s).  One
// pass per sibling rank: the children of one pass have distinct parents, so
// no entry is written twice within a pass, and the passes run in rank order.
// child[0..nlist) lists the pass's children, ent_off[0..nlist] the running
// entry offsets of their coarse matrices.
template <typename T>
__global__ void k_assemble_next(T* M, const int64_t* par_off, const int32_t* par_n, const int32_t* parent,
                                const int64_t* ac_off, const int32_t* nc, const int64_t* loc_off,
                                const int32_t* loc, const double* ac, const int32_t* child, const int64_t* ent_off,
                                int nlist) {
  const int64_t idx = ent_off[0] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ent_off[nlist]) return;
  int lo = 0, hi = nlist - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (ent_off[mid] <= idx) lo = mid; else hi = mid - 1;
  }
  const int s = child[lo];
  const int64_t r = idx - ent_off[lo];
  const int n = nc[s];
  const int a = (int)(r % n), b = (int)(r / n);
  const int la = loc[loc_off[s] + a], lb = loc[loc_off[s] + b];
  const int P = parent[s];
  M[par_off[P] + la + (int64_t)lb * par_n[P]] += (T)ac[ac_off[s] + a + (int64_t)b * n];
}

template <typename T>
void assemble_next(cudaStream_t st, T* M, const int64_t* par_off, const int32_t* par_n, const int32_t* parent,
                   const int64_t* ac_off, const int32_t* nc, const int64_t* loc_off, const int32_t* loc,
                   const double* ac, const int32_t* child, const int64_t* ent_off, const std::vector<int>& pass_beg,
                   const std::vector<int64_t>& ent_h) {
  for (size_t r = 0; r + 1 < pass_beg.size(); ++r) {
    const int b = pass_beg[r], e = pass_beg[r + 1];
    const int64_t total = ent_h[e] - ent_h[b];
    if (total <= 0) continue;
    k_assemble_next<T><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(M, par_off, par_n, parent, ac_off, nc, loc_off,
                                                                       loc, ac, child + b, ent_off + b, e - b);
    AMB_LAUNCHED();
  }
}

template void assemble_level1<float>(cudaStream_t, float*, const int64_t*, const int32_t*, const int32_t*,
                                     const int32_t*, const double*, const double*, int, int, int, int);
template void assemble_level1<double>(cudaStream_t, double*, const int64_t*, const int32_t*, const int32_t*,
                                      const int32_t*, const double*, const double*, int, int, int, int);
template void assemble_next<float>(cudaStream_t, float*, const int64_t*, const int32_t*, const int32_t*,
                                   const int64_t*, const int32_t*, const int64_t*, const int32_t*, const double*,
                                   const int32_t*, const int64_t*, const std::vector<int>&,
                                   const std::vector<int64_t>&);
template void assemble_next<double>(cudaStream_t, double*, const int64_t*, const int32_t*, const int32_t*,
                                    const int64_t*, const int32_t*, const int64_t*, const int32_t*, const double*,
                                    const int32_t*, const int64_t*, const std::vector<int>&,
                                    const std::vector<int64_t>&);

// y = A x on full-grid nodal vectors, one thread per node: the node's rows
// of the (up to 8) element matrices around it.  Dirichlet rows are zero
// and Dirichlet entries of x are treated as zero.
__global__ void k_matvec(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ coeff,
                         const double* __restrict__ khat, const uint8_t* __restrict__ dir, int nx, int ny, int nz,
                         int dpn) {
  const int64_t nnx = nx + 1, nny = ny + 1;
  const int64_t nn = nnx * nny * (nz + 1);
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int nd = 8 * dpn;
  double acc[3] = {0.0, 0.0, 0.0};
  if (!dir[n]) {
    const int i = (int)(n % nnx), j = (int)((n / nnx) % nny), k = (int)(n / (nnx * nny));
    for (int a = 0; a < 8; ++a) {
      // element whose local node a is n
      const int ei = i - (a & 1), ej = j - ((a >> 1) & 1), ek = k - ((a >> 2) & 1);
      if (ei < 0 || ej < 0 || ek < 0 || ei >= nx || ej >= ny || ek >= nz) continue;
      const int64_t e = ei + (int64_t)nx * (ej + (int64_t)ny * ek);
      const double ce = coeff[e];
      for (int b = 0; b < 8; ++b) {
        const int64_t m = (ei + (b & 1)) + nnx * ((ej + ((b >> 1) & 1)) + nny * (ek + ((b >> 2) & 1)));
        if (dir[m]) continue;
        for (int cb = 0; cb < dpn; ++cb) {
          const double xv = ce * x[m * dpn + cb];
          for (int ca = 0; ca < dpn; ++ca) acc[ca] += khat[(a * dpn + ca) + (b * dpn + cb) * nd] * xv;
        }
      }
    }
  }
  for (int c = 0; c < dpn; ++c) y[n * dpn + c] = acc[c];
}

void matvec(cudaStream_t st, double* y, const double* x, const double* coeff, const double* khat, const uint8_t* dir,
            int nx, int ny, int nz, int dpn) {
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  k_matvec<<<(unsigned)((nn + 127) / 128), 128, 0, st>>>(y, x, coeff, khat, dir, nx, ny, nz, dpn);
  AMB_LAUNCHED();
}

// Consistent load of a per-element constant density b_e: int N_a = V/8.
__global__ void k_load(double* f, const double* body, const uint8_t* dir, int nx, int ny, int nz, int dpn, double h) {
  const int64_t nnx = nx + 1, nny = ny + 1;
  const int64_t nn = nnx * nny * (nz + 1);
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int i = (int)(n % nnx), j = (int)((n / nnx) % nny), k = (int)(n / (nnx * nny));
  double acc[3] = {0.0, 0.0, 0.0};
  if (!dir[n]) {
    for (int a = 0; a < 8; ++a) {
      const int ei = i - (a & 1), ej = j - ((a >> 1) & 1), ek = k - ((a >> 2) & 1);
      if (ei < 0 || ej < 0 || ek < 0 || ei >= nx || ej >= ny || ek >= nz) continue;
      const int64_t e = ei + (int64_t)nx * (ej + (int64_t)ny * ek);
      for (int c = 0; c < dpn; ++c) acc[c] += body[e * dpn + c];
    }
  }
  const double w = h * h * h / 8.0;
  for (int c = 0; c < dpn; ++c) f[n * dpn + c] = acc[c] * w;
}

void load_vector(cudaStream_t st, double* f, const double* body, const uint8_t* dir, int nx, int ny, int nz, int dpn,
                 double h) {
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  k_load<<<(unsigned)((nn + 127) / 128), 128, 0, st>>>(f, body, dir, nx, ny, nz, dpn, h);
  AMB_LAUNCHED();
}

// Zero the entries of Dirichlet nodes (they are not unknowns of A u = f).
__global__ void k_mask(double* v, const uint8_t* dir, int64_t nn, int dpn) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nn * dpn && dir[i / dpn]) v[i] = 0.0;
}

void mask_dirichlet(cudaStream_t st, double* v, const uint8_t* dir, int64_t nnodes, int dpn) {
  const int64_t n = nnodes * dpn;
  k_mask<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, dir, nnodes, dpn);
  AMB_LAUNCHED();
}

// g_e = -coeff_e lambda_e^T Khat u_e  (d q / d log coeff_e).
__global__ void k_grad(double* g, const double* u, const double* lam, const double* coeff, const double* khat,
                       const uint8_t* dir, int nx, int ny, int nz, int dpn) {
  const int64_t nel = (int64_t)nx * ny * nz;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  const int64_t nnx = nx + 1, nny = ny + 1;
  const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
  const int nd = 8 * dpn;
  double ue[24], le[24];
  for (int a = 0; a < 8; ++a) {
    const int64_t m = (i + (a & 1)) + nnx * ((j + ((a >> 1) & 1)) + nny * (k + ((a >> 2) & 1)));
    for (int c = 0; c < dpn; ++c) {
      ue[a * dpn + c] = dir[m] ? 0.0 : u[m * dpn + c];
      le[a * dpn + c] = dir[m] ? 0.0 : lam[m * dpn + c];
    }
  }
  double s = 0.0;
  for (int q = 0; q < nd; ++q) {
    double t = 0.0;
    for (int r = 0; r < nd; ++r) t += khat[r + q * nd] * le[r];
    s += t * ue[q];
  }
  g[e] = -coeff[e] * s;
}

void element_gradient(cudaStream_t st, double* g, const double* u, const double* lam, const double* coeff,
                      const double* khat, const uint8_t* dir, int nx, int ny, int nz, int dpn) {
  const int64_t nel = (int64_t)nx * ny * nz;
  k_grad<<<(unsigned)((nel + 127) / 128), 128, 0, st>>>(g, u, lam, coeff, khat, dir, nx, ny, nz, dpn);
  AMB_LAUNCHED();
}

}  // namespace amb
