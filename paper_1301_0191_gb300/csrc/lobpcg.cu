// Adaptive selection of face constraints on one level (Sec. 4, 5, 7.2):
// all pair eigenproblems of the level run in lockstep as one batch.
//
// For a pair (s, t) the vectors live on Gamma^s + Gamma^t (two interface
// copies, length N = n_g^s + n_g^t).  With shared dofs f, pair weights
// d_s = K^s_jj/(K^s_jj + K^t_jj), d_t = 1 - d_s (Sec. 7.2) and the jump
// j = w^s_f - w^t_f:
//   (I - E) w          = [ d_t j on f (s copy) ; -d_s j on f (t copy) ], 0 elsewhere
//   (I - E)^T v        = [ x ; -x ] on f,  x = d_t v^s_f - d_s v^t_f
//   Pi                 = I - D^T (D D^T)^{-1} D, D = jump rows of the initial
//                        coarse dofs shared by s and t; their supports are
//                        disjoint, so Pi acts group by group
//   A  = Pi (I-E)^T S (I-E) Pi   (only S_ff of each side is touched)
//   B  = Pi S Pi
//   M  = Pi ( Neumann^s + Neumann^t + Psi (Psi^T S Psi)^+ Psi^T ) Pi   (eq. bddc_pair)
// LOBPCG (block size m) finds the m largest eigenpairs of A w = lambda B w
// in the factor space modulo null(B) (eq. eig-nullspace): Rayleigh-Ritz on
// [X W P] with FP64 Gram matrices and an SVQB B-orthonormalization that
// drops directions of negligible B-norm.  Rows c_l = A w_l (eq. d-def) for
// lambda_l > tau, restricted to the face dofs, orthonormalized (Sec. 7.2).
#include <cmath>

#include "engine_impl.h"
#include "tc_gemm.h"

namespace amb {

namespace {

enum PairField {
  Q_S, Q_T, Q_NS, Q_NT, Q_N, Q_NF, Q_OQ, Q_OT, Q_OJ, Q_OF, Q_FOFF, Q_GBEG, Q_GEND, Q_FACEOFF, Q_FACEN,
  Q_CMS, Q_CMT, Q_NCP, Q_NCS, Q_NCT, Q_OC, Q_OPI, Q_OGR, Q_OCC, Q_OR, Q_OO, Q_NPAIRF
};
#define QP(p, f) qp[(int64_t)(p) * Q_NPAIRF + (f)]

constexpr int kJacobiMax = 112;
// Threads of the Jacobi kernels: the rotation rounds are FP64-bound on one
// SM, and 32 warps keep its FP64 pipes busier than 8 (latency hiding).
constexpr int kJacobiThreads = 1024;
constexpr int kJacobiMaxBlocks = (kJacobiMax / 2 + 1) * (kJacobiMax / 2 + 2) / 2;   // 2 x 2 blocks of a triangle

// ---------------------------------------------------------------- block helpers

__device__ double block_sum(double v, double* red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

// Cyclic Jacobi sweeps on a symmetric n x n matrix in shared memory
// (column-major, leading dimension ld >= n + (n & 1)), accumulating the
// rotations into V (V *= R).  Each round rotates the disjoint index pairs of
// a round-robin ordering at once, and the two-sided update is applied
// block-wise: B <- R_k^T B R_l on the 2 x 2 block of index pairs (k, l),
// k <= l, mirrored to (l, k), with V <- V R in the same pass (one barrier per
// round; only the upper blocks are computed).  For odd n the extra index n is
// a zero row and column that is never rotated.  Stops when the off-diagonal
// Frobenius norm squared is at most tol times the total, or after maxs sweeps.
template <typename F>
__device__ void jacobi_sweeps(F* A, F* V, int n, int ld, double* red, double* cs, double* sn, int* P, int* Q,
                              double tol, int maxs) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ne = n + (n & 1), half = ne / 2;
  const int nblk = half * (half + 1) / 2;
  // rotations below this relative size are skipped (FP64: far below rounding)
  const double skip = sizeof(F) == 8 ? 1e-18 : 1e-9;
  // block (k, l), k <= l, of each triangular index, decoded once
  __shared__ uint16_t bk[kJacobiMaxBlocks], bl[kJacobiMaxBlocks];
  for (int idx = tid; idx < nblk; idx += nt) {
    int l = (int)((sqrtf(8.f * idx + 1.f) - 1.f) * 0.5f);
    while (l * (l + 1) / 2 > idx) --l;
    while ((l + 1) * (l + 2) / 2 <= idx) ++l;
    bl[idx] = (uint16_t)l;
    bk[idx] = (uint16_t)(idx - l * (l + 1) / 2);
  }
  __syncthreads();
  for (int sweep = 0; sweep < maxs; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int idx = tid; idx < n * n; idx += nt) {
      int r = idx % n, c = idx / n;
      double a = (double)A[r + c * ld];
      tot += a * a;
      if (r != c) off += a * a;
    }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    if (off <= tol * tot || tot == 0.0) break;
    for (int round = 0; round < ne - 1; ++round) {
      for (int k = tid; k < half; k += nt) {
        int a = (k == 0) ? 0 : 1 + ((k - 1 + round) % (ne - 1));
        int b = 1 + ((ne - 2 - k + round) % (ne - 1));
        int p = a < b ? a : b, q = a < b ? b : a;
        F c = F(1), s = F(0);
        if (q < n) {
          const F apq = A[p + q * ld];
          const F app = A[p + p * ld], aqq = A[q + q * ld];
          if constexpr (sizeof(F) == 8) {
            if (fabs(apq) > 1e-300 && fabs(apq) > skip * sqrt(fabs(app * aqq))) {
              const F th = (aqq - app) / (F(2) * apq);
              const F t = (th >= F(0) ? F(1) : F(-1)) / (fabs(th) + sqrt(th * th + F(1)));
              c = F(1) / sqrt(t * t + F(1));
              s = t * c;
            }
          } else {
            // FP32 sweeps: the angle in FP64 arithmetic.  (Single-precision
            // angles are faster, but the FP32 form's pair eigenproblems are
            // sensitive to which of the equally accurate FP64 end states the
            // refinement reaches: on the 1e4-contrast channels workload that
            // variant lost an eigenvalue of one pair.)
            if (fabs((double)apq) > 1e-300 && fabs((double)apq) > skip * sqrt(fabs((double)app * (double)aqq))) {
              const F th = (aqq - app) / (F(2) * apq);
              const F t = (th >= F(0) ? F(1) : F(-1)) / (F(fabs((double)th)) + F(sqrt((double)th * (double)th + 1.0)));
              c = F(1) / F(sqrt((double)t * (double)t + 1.0));
              s = t * c;
            }
          }
        }
        P[k] = p;
        Q[k] = q;
        cs[k] = (double)c;
        sn[k] = (double)s;
      }
      __syncthreads();
      for (int idx = tid; idx < nblk + n * half; idx += nt) {
        if (idx < nblk) {
          const int k = bk[idx], l = bl[idx];
          const F sk = (F)sn[k], sl = (F)sn[l];
          if (sk == F(0) && sl == F(0)) continue;
          const F ck = (F)cs[k], cl = (F)cs[l];
          const int pk = P[k], qk = Q[k], pl = P[l], ql = Q[l];
          const F b00 = A[pk + pl * ld], b01 = A[pk + ql * ld], b10 = A[qk + pl * ld], b11 = A[qk + ql * ld];
          const F t00 = cl * b00 - sl * b01, t01 = sl * b00 + cl * b01;
          const F t10 = cl * b10 - sl * b11, t11 = sl * b10 + cl * b11;
          const F n00 = ck * t00 - sk * t10, n01 = ck * t01 - sk * t11;
          const F n10 = sk * t00 + ck * t10, n11 = sk * t01 + ck * t11;
          if (k == l) {
            A[pk + pk * ld] = n00;
            A[qk + qk * ld] = n11;
            A[pk + qk * ld] = n01;
            A[qk + pk * ld] = n01;
          } else {
            A[pk + pl * ld] = n00;
            A[pk + ql * ld] = n01;
            A[qk + pl * ld] = n10;
            A[qk + ql * ld] = n11;
            A[pl + pk * ld] = n00;
            A[ql + pk * ld] = n01;
            A[pl + qk * ld] = n10;
            A[ql + qk * ld] = n11;
          }
        } else {
          const int v = idx - nblk, l = v / n, i = v % n;
          const F sl = (F)sn[l];
          if (sl == F(0)) continue;
          const F cl = (F)cs[l];
          const int pl = P[l], ql = Q[l];
          const F vp = V[i + pl * ld], vq = V[i + ql * ld];
          V[i + pl * ld] = cl * vp - sl * vq;
          V[i + ql * ld] = sl * vp + cl * vq;
        }
      }
      __syncthreads();
    }
  }
}

// D = X^T Y (transx) or X Y, n x n, all in shared memory with leading dimension ld
__device__ void small_gemm(double* D, const double* X, const double* Y, int n, int ld, bool transx) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx % n, c = idx / n;
    double s = 0.0;
    if (transx)
      for (int k = 0; k < n; ++k) s = fma(X[k + r * ld], Y[k + c * ld], s);
    else
      for (int k = 0; k < n; ++k) s = fma(X[r + k * ld], Y[k + c * ld], s);
    D[r + c * ld] = s;
  }
  __syncthreads();
}

// Eigen-decomposition of a symmetric n x n matrix in shared memory: on exit A
// holds the eigenvalues on its diagonal, V the eigenvectors (FP64 accuracy).
// FP64 runs at 1/64 of the FP32 rate on this GPU, so with scratch space
// (T, W: ld x ld doubles each; may be null) the sweeps start in FP32 on a
// copy of A (to a relative off-diagonal norm of 1e-5); the FP32 rotations are
// then made orthonormal in FP64 (two Newton-Schulz steps V <- V (3I - V^T V)/2),
// A is transformed to V^T A V in FP64, and FP64 sweeps finish from there
// (quadratic convergence: two or three sweeps instead of about ten).  If the
// FP32 rotations are not orthonormal to 1e-3 the FP32 part is discarded.
__device__ void jacobi_eig(double* A, double* V, int n, int ld, double* red, double* cs, double* sn, int* P, int* Q,
                           double* T = nullptr, double* W = nullptr) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ne = n + (n & 1);
  for (int idx = tid; idx < ne * ne; idx += nt) {
    int r = idx % ne, c = idx / ne;
    V[r + c * ld] = (r == c) ? 1.0 : 0.0;
    if (r == n || c == n) A[r + c * ld] = 0.0;
  }
  __syncthreads();
  if (n <= 1) return;
  if (T && W && n >= 8) {
    float* A32 = reinterpret_cast<float*>(W);
    float* V32 = A32 + ld * ld;
    for (int idx = tid; idx < ne * ne; idx += nt) {
      int r = idx % ne, c = idx / ne;
      A32[r + c * ld] = (float)A[r + c * ld];
      V32[r + c * ld] = (r == c) ? 1.f : 0.f;
    }
    __syncthreads();
    jacobi_sweeps<float>(A32, V32, n, ld, red, cs, sn, P, Q, 1e-10, 20);
    for (int idx = tid; idx < n * n; idx += nt) {
      int r = idx % n, c = idx / n;
      V[r + c * ld] = (double)V32[r + c * ld];
    }
    __syncthreads();
    // Newton-Schulz: T = V^T V, T <- (3I - T)/2, V <- V T (through W)
    double dev = 0.0;
    for (int step = 0; step < 2; ++step) {
      small_gemm(T, V, V, n, ld, true);
      double e = 0.0;
      for (int idx = tid; idx < n * n; idx += nt) {
        int r = idx % n, c = idx / n;
        const double t = T[r + c * ld] - (r == c ? 1.0 : 0.0);
        e = fmax(e, fabs(t));
        T[r + c * ld] = (r == c ? 1.0 : 0.0) - 0.5 * t;
      }
      red[tid] = e;
      __syncthreads();
      for (int o = nt >> 1; o > 0; o >>= 1) {
        if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
        __syncthreads();
      }
      if (step == 0) dev = red[0];
      __syncthreads();
      if (!(dev <= 1e-3)) break;   // also catches NaN
      small_gemm(W, V, T, n, ld, false);
      for (int idx = tid; idx < n * n; idx += nt) V[(idx % n) + (idx / n) * ld] = W[(idx % n) + (idx / n) * ld];
      __syncthreads();
    }
    if (dev <= 1e-3) {
      // A <- V^T (A V), symmetrized
      small_gemm(W, A, V, n, ld, false);
      small_gemm(T, V, W, n, ld, true);
      for (int idx = tid; idx < n * n; idx += nt) {
        int r = idx % n, c = idx / n;
        A[r + c * ld] = 0.5 * (T[r + c * ld] + T[c + r * ld]);
      }
      __syncthreads();
    } else {
      for (int idx = tid; idx < ne * ne; idx += nt) {
        int r = idx % ne, c = idx / ne;
        V[r + c * ld] = (r == c) ? 1.0 : 0.0;
      }
      __syncthreads();
    }
  }
  // off-diagonal Frobenius norm below 1e-13 of the total: converged (the
  // FP64 rounding floor is near 1e-16, so a tighter test may never pass)
  jacobi_sweeps<double>(A, V, n, ld, red, cs, sn, P, Q, 1e-26, 40);
}

// descending order of the diagonal of A (n <= kJacobiMax), by one thread
__device__ void sort_desc(const double* A, int n, int ld, int* ord) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) ord[i] = i;
    for (int i = 0; i < n; ++i) {
      int b = i;
      for (int j = i + 1; j < n; ++j)
        if (A[ord[j] + ord[j] * ld] > A[ord[b] + ord[b] * ld]) b = j;
      int t = ord[i];
      ord[i] = ord[b];
      ord[b] = t;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- null modes of floating substructures
//
// A level-1 substructure without Dirichlet dofs floats: its Schur complement
// annihilates the rigid modes restricted to its interface (constants for the
// scalar problem; three translations and three rotations for elasticity),
// exactly (Sec. 2: S is the energy of the discrete harmonic extension).  The
// rounded S gives these modes an energy of the order of the factorization's
// rounding (about 1e-7 of its norm in the FP32 form), and the pair
// denominator B = Pi S Pi (eq. eig-matrix) is nearly singular exactly there:
// the pencils' large eigenvalues then move by per cents and LOBPCG stalls on
// the pairs of two floating substructures.  In the FP64 form the same
// happens on stiff inclusions, where the pencils' eigenvalues reach 1e6 and
// the spurious directions win by chance of rounding.  Both forms therefore
// apply B with P S P, P = I - Q Q^T the orthogonal projector off the modes
// (Q orthonormal): P S P x = S x - T a - Q b with a = Q^T x, T = S Q,
// b = Q^T (S x - T a), in FP64 after the product.  For the exact S,
// P S P = S.

// Q (n_g x r per floating substructure, column-major) <- orthonormal basis of
// its columns, two passes of classical Gram-Schmidt in FP64; one CTA each.
__global__ void k_orth_modes(double* Qn, const int64_t* off, const int32_t* ng, int r) {
  __shared__ double red[256];
  const int64_t o = off[blockIdx.x];
  const int n = ng[blockIdx.x];
  double* Qs = Qn + o;
  for (int k = 0; k < r; ++k) {
    double* qk = Qs + (int64_t)k * n;
    for (int pass = 0; pass < 2; ++pass) {
      for (int l = 0; l < k; ++l) {
        const double* ql = Qs + (int64_t)l * n;
        double d = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) d += ql[i] * qk[i];
        d = block_sum(d, red);
        for (int i = threadIdx.x; i < n; i += blockDim.x) qk[i] -= d * ql[i];
        __syncthreads();
      }
    }
    double nn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) nn += qk[i] * qk[i];
    nn = block_sum(nn, red);
    const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) qk[i] *= inv;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- pair kernels

// pseudo-random start block (counter-based hash, SplitMix64 finalizer)
__device__ inline double hash_uniform(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

template <typename T>
__global__ void k_lob_random(T* Qb, const int64_t* qp, int m, uint64_t seed) {
  const int p = blockIdx.y;
  const int64_t N = QP(p, Q_N);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * 9 * m) return;
  const int64_t col = idx / N;
  T v = T(0);
  if (col < m) v = (T)hash_uniform(seed * 0x100000001B3ull ^ ((uint64_t)p << 40) ^ (uint64_t)idx);
  Qb[QP(p, Q_OQ) + idx] = v;
}

// B-product correction on floating pair sides: y <- y - T a - Q b with
// a = Q^T x, b = Q^T (y - T a), for the columns of the input slot cin (x)
// and output slot cout (y) of the FP64 panel.  One CTA per (pair, side), one
// warp per column (fixed-order lane sums and shuffles: deterministic, no
// block barriers).  ncol: per pair, the number of leading columns that can
// be nonzero (nullptr: all m).
__global__ void k_lob_nullproj(double* base, const int64_t* qp, int cin, int cout, int m, const int* act,
                               const int64_t* qoff, const double* Qn, const double* Tn, int r, const int* ncol) {
  const int p = blockIdx.x >> 1, side = blockIdx.x & 1;
  if (!act[p]) return;
  const int sub = (int)QP(p, side ? Q_T : Q_S);
  const int64_t o = qoff[sub];
  if (o < 0) return;
  const int64_t N = QP(p, Q_N);
  const int n = (int)QP(p, side ? Q_NT : Q_NS);
  const int64_t r0 = side ? QP(p, Q_NS) : 0;
  const double* Qs = Qn + o;
  const double* Ts = Tn + o;
  const double* x = base + QP(p, Q_OQ) + (int64_t)cin * m * N + r0;
  double* y = base + QP(p, Q_OQ) + (int64_t)cout * m * N + r0;
  const int nc = ncol ? min(ncol[p], m) : m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int c = warp; c < nc; c += nwarp) {
    const double* xc = x + (int64_t)c * N;
    double* yc = y + (int64_t)c * N;
    double a[6] = {0, 0, 0, 0, 0, 0}, b[6] = {0, 0, 0, 0, 0, 0};
    for (int i = lane; i < n; i += 32) {
      const double xv = xc[i];
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (k < r) a[k] = fma(Qs[(int64_t)k * n + i], xv, a[k]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
      for (int off = 16; off > 0; off >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], off);
    for (int i = lane; i < n; i += 32) {
      double v = yc[i];
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (k < r) v = fma(-Ts[(int64_t)k * n + i], a[k], v);
      yc[i] = v;
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (k < r) b[k] = fma(Qs[(int64_t)k * n + i], v, b[k]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
      for (int off = 16; off > 0; off >>= 1) b[k] += __shfl_xor_sync(0xffffffffu, b[k], off);
    for (int i = lane; i < n; i += 32) {
      double v = yc[i];
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (k < r) v = fma(-Qs[(int64_t)k * n + i], b[k], v);
      yc[i] = v;
    }
  }
}

// x <- x - Q (Q^T x) on the leading columns of one slot of the FP64 panel,
// for the pairs with a deflation basis Q (N x r, orthonormal, at Qp +
// qoff[p]; qoff[p] < 0: none).  One CTA per pair, one warp per column
// (fixed-order lane sums and shuffles: deterministic).  ncol: per pair, the
// number of leading columns that can be nonzero (nullptr: all m).
__global__ void k_lob_deflate(double* base, const int64_t* qp, int slot, int m, const int* act, const int64_t* qoff,
                              const double* Qp, int r, const int* ncol) {
  const int p = blockIdx.x;
  if (!act[p]) return;
  const int64_t o = qoff[p];
  if (o < 0) return;
  const int64_t N = QP(p, Q_N);
  const double* Qs = Qp + o;
  double* x = base + QP(p, Q_OQ) + (int64_t)slot * m * N;
  const int nc = ncol ? min(ncol[p], m) : m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int c = warp; c < nc; c += nwarp) {
    double* xc = x + (int64_t)c * N;
    double a[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = lane; i < N; i += 32) {
      const double xv = xc[i];
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (k < r) a[k] = fma(Qs[(int64_t)k * N + i], xv, a[k]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
      for (int off = 16; off > 0; off >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], off);
    for (int64_t i = lane; i < N; i += 32) {
      double v = xc[i];
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (k < r) v = fma(-Qs[(int64_t)k * N + i], a[k], v);
      xc[i] = v;
    }
  }
}

// Pi on columns [c0, c0+w) of a block with leading dimension N at base
// offset QP(p, which) (+ c0*N).  One warp per (group, column).
template <typename T>
__global__ void k_lob_project(T* base, const int64_t* qp, int which, int c0, int w, const int32_t* goff,
                              const int32_t* gent, const double* gw, const int32_t* ps, const int32_t* pt,
                              const int* act) {
  const int p = blockIdx.x;
  if (!act[p]) return;
  const int64_t N = QP(p, Q_N), ns = QP(p, Q_NS);
  const int64_t g0 = QP(p, Q_GBEG), g1 = QP(p, Q_GEND), foff = QP(p, Q_FOFF);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t ngr = g1 - g0;
  for (int64_t job = warp; job < ngr * w; job += nw) {
    const int64_t g = g0 + job % ngr;
    const int col = c0 + (int)(job / ngr);
    T* v = base + QP(p, which) + (int64_t)col * N;
    double num = 0.0, den = 0.0;
    for (int e = goff[g] + lane; e < goff[g + 1]; e += 32) {
      const int f = gent[e];
      const double c = (double)gw[e];
      num += c * ((double)v[ps[foff + f]] - (double)v[ns + pt[foff + f]]);
      den += c * c;
    }
    for (int o = 16; o > 0; o >>= 1) {
      num += __shfl_xor_sync(0xffffffffu, num, o);
      den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    const double a = den > 0 ? num / (2.0 * den) : 0.0;
    for (int e = goff[g] + lane; e < goff[g + 1]; e += 32) {
      const int f = gent[e];
      const double c = (double)gw[e];
      v[ps[foff + f]] = (T)((double)v[ps[foff + f]] - c * a);
      v[ns + pt[foff + f]] = (T)((double)v[ns + pt[foff + f]] + c * a);
    }
  }
}

// J_s = d_t * j, J_t = -d_s * j with j = v^s_f - v^t_f (nf x w each).  The
// block vectors (V) are FP64; J is in the operator precision T.
template <typename T, typename V>
__global__ void k_lob_jump(T* J, const V* base, const int64_t* qp, int which, int c0, int w, const int32_t* ps,
                           const int32_t* pt, const double* ws, const double* wt) {
  const int p = blockIdx.y;
  const int64_t N = QP(p, Q_N), ns = QP(p, Q_NS), nf = QP(p, Q_NF), foff = QP(p, Q_FOFF);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nf * w) return;
  const int64_t f = idx % nf, col = idx / nf;
  const V* v = base + QP(p, which) + (c0 + col) * N;
  const double j = (double)v[ps[foff + f]] - (double)v[ns + pt[foff + f]];
  T* Jb = J + QP(p, Q_OJ);
  Jb[f + col * nf] = (T)(wt[foff + f] * j);
  Jb[nf * w + f + col * nf] = (T)(-ws[foff + f] * j);
}

// out = (I - E)^T [Y_s ; Y_t] scattered on f (s copy x, t copy -x), zero elsewhere
template <typename T, typename V>
__global__ void k_lob_iet(V* base, const int64_t* qp, int which, int c0, const T* J, int w, const int32_t* ps,
                          const int32_t* pt, const double* ws, const double* wt) {
  const int p = blockIdx.x, col = blockIdx.y;
  const int64_t N = QP(p, Q_N), ns = QP(p, Q_NS), nf = QP(p, Q_NF), foff = QP(p, Q_FOFF);
  V* v = base + QP(p, which) + (int64_t)(c0 + col) * N;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) v[i] = V(0);
  __syncthreads();
  const T* Y = J + QP(p, Q_OJ) + 2 * nf * w;
  for (int64_t f = threadIdx.x; f < nf; f += blockDim.x) {
    const double x = wt[foff + f] * (double)Y[f + col * nf] - ws[foff + f] * (double)Y[nf * w + f + col * nf];
    v[ps[foff + f]] = (V)x;
    v[ns + pt[foff + f]] = (V)(-x);
  }
}

// copy an N x w column block between the FP64 block vectors and the
// operator-precision staging blocks (per pair offsets QP(p, wd), QP(p, ws))
template <typename To, typename Ti>
__global__ void k_lob_convert(To* dst, const Ti* src, const int64_t* qp, int wd, int cd, int wsrc, int cs, int w) {
  const int p = blockIdx.y;
  const int64_t N = QP(p, Q_N);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * w) return;
  dst[QP(p, wd) + cd * N + idx] = (To)src[QP(p, wsrc) + cs * N + idx];
}

template <typename T>
__global__ void k_lob_zero(T* base, const int64_t* qp, int which, int c0, int w) {
  const int p = blockIdx.y;
  const int64_t N = QP(p, Q_N);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * w) return;
  base[QP(p, which) + c0 * N + idx] = T(0);
}

// S_ff of both sides of each pair: the rows and columns of S^(s) (S^(t)) at
// the shared positions ps (pt), column-major nf x nf.  One CTA per (column,
// pair side); grid.x = 2 x pairs, grid.y covers the largest nf.
template <typename T>
__global__ void k_lob_sff(T* Sff, const T* S, const int64_t* qp, const int64_t* soff, const int32_t* ps,
                          const int32_t* pt) {
  const int p = blockIdx.x >> 1, side = blockIdx.x & 1;
  const int64_t nf = QP(p, Q_NF);
  const int64_t b = blockIdx.y;
  if (b >= nf) return;
  const int sub = (int)(side ? QP(p, Q_T) : QP(p, Q_S));
  const int64_t ng = side ? QP(p, Q_NT) : QP(p, Q_NS);
  const int32_t* pos = (side ? pt : ps) + QP(p, Q_FOFF);
  const T* src = S + soff[sub] + (int64_t)pos[b] * ng;
  T* dst = Sff + QP(p, Q_OF) + side * nf * nf + b * nf;
  for (int64_t a = threadIdx.x; a < nf; a += blockDim.x) dst[a] = src[pos[a]];
}

// Neumann solves of the pair preconditioner are batched per substructure:
// the Delta rows of every active pair-side block of one substructure sit
// side by side in a substructure-major buffer.  One map entry per pair-side:
// its rows in the pair block (offset, leading dimension N) and its column
// block in the substructure buffer (offset, leading dimension n_Delta).
struct NeuMap {
  int64_t pair_off, sub_off;
  int32_t ldp, nd;
};
template <typename T>
__global__ void k_lob_neu_move(T* dst, const T* src, const NeuMap* mp, int m, int to_sub) {
  const NeuMap x = mp[blockIdx.y];
  const int64_t n = (int64_t)x.nd * m;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % x.nd, c = idx / x.nd;
    const int64_t po = x.pair_off + i + c * x.ldp, so = x.sub_off + i + c * x.nd;
    if (to_sub) dst[so] = src[po]; else dst[po] = src[so];
  }
}

// coarse gather/scatter of the pair coarse space
template <typename T>
__global__ void k_lob_cgather(T* C, const int64_t* qp, int m, const int32_t* cms, const int32_t* cmt) {
  const int p = blockIdx.x;
  const int64_t ncp = QP(p, Q_NCP), ncs = QP(p, Q_NCS), nct = QP(p, Q_NCT), oc = QP(p, Q_OC);
  T* cs = C + oc;
  T* ct = cs + ncs * m;
  T* cp = ct + nct * m;
  for (int64_t i = threadIdx.x; i < ncp * m; i += blockDim.x) cp[i] = T(0);
  __syncthreads();
  for (int64_t i = threadIdx.x; i < ncs * m; i += blockDim.x) {
    int64_t q = i % ncs, col = i / ncs;
    cp[cms[QP(p, Q_CMS) + q] + col * ncp] += cs[i];
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < nct * m; i += blockDim.x) {
    int64_t q = i % nct, col = i / nct;
    cp[cmt[QP(p, Q_CMT) + q] + col * ncp] += ct[i];
  }
}
template <typename T>
__global__ void k_lob_cscatter(T* C, const int64_t* qp, int m, const int32_t* cms, const int32_t* cmt) {
  const int p = blockIdx.x;
  const int64_t ncp = QP(p, Q_NCP), ncs = QP(p, Q_NCS), nct = QP(p, Q_NCT), oc = QP(p, Q_OC);
  T* cs = C + oc;
  T* ct = cs + ncs * m;
  const T* up = ct + nct * m + ncp * m;
  T* us = (T*)up + ncp * m;
  T* ut = us + ncs * m;
  for (int64_t i = threadIdx.x; i < ncs * m; i += blockDim.x) {
    int64_t q = i % ncs, col = i / ncs;
    us[i] = up[cms[QP(p, Q_CMS) + q] + col * ncp];
  }
  for (int64_t i = threadIdx.x; i < nct * m; i += blockDim.x) {
    int64_t q = i % nct, col = i / nct;
    ut[i] = up[cmt[QP(p, Q_CMT) + q] + col * ncp];
  }
}

// pseudo-inverse of the pair coarse matrix Psi^T S^{st} Psi (Sec. 5: dense
// eigen-decomposition, eigenvalues below a tolerance dropped)
template <typename T>
__global__ void __launch_bounds__(kJacobiThreads) k_pair_pinv(T* pinv, const int64_t* qp, const double* Ac, const int64_t* acs, const int64_t* act,
                            const int32_t* cms, const int32_t* cmt, const int* nnull, int* status) {
  extern __shared__ double sh[];
  const int p = blockIdx.x;
  const int n = (int)QP(p, Q_NCP), ncs = (int)QP(p, Q_NCS), nct = (int)QP(p, Q_NCT);
  const int ld = n + (n & 1);
  double* A = sh;
  double* V = A + ld * ld;
  __shared__ double red[kJacobiThreads], cs_[kJacobiMax / 2 + 1], sn_[kJacobiMax / 2 + 1];
  __shared__ int P_[kJacobiMax / 2 + 1], Q_[kJacobiMax / 2 + 1];
  for (int i = threadIdx.x; i < ld * ld; i += blockDim.x) A[i] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double* as = Ac + acs[p];
    const double* at = Ac + act[p];
    const int32_t* ms = cms + QP(p, Q_CMS);
    const int32_t* mt = cmt + QP(p, Q_CMT);
    for (int b = 0; b < ncs; ++b)
      for (int a = 0; a < ncs; ++a) A[ms[a] + ms[b] * ld] += as[a + b * ncs];
    for (int b = 0; b < nct; ++b)
      for (int a = 0; a < nct; ++a) A[mt[a] + mt[b] * ld] += at[a + b * nct];
  }
  __syncthreads();
  jacobi_eig(A, V, n, ld, red, cs_, sn_, P_, Q_);
  double mx = 0.0;
  for (int i = 0; i < n; ++i) mx = fmax(mx, A[i + i * ld]);
  // a floating pair's coarse matrix annihilates the coarse values of the
  // pair's rigid modes exactly; its computed eigenvalues there are rounding
  // (which the relative cut below can keep), and their inverses would blow
  // the rigid directions up by the inverse of that rounding: the nnull[p]
  // smallest eigenvalues are left out, as the pseudo-inverse of the exact
  // matrix leaves out its null space
  __shared__ double cut_sh;
  if (threadIdx.x == 0) {
    double cut = 1e-12 * mx;
    const int k = min(nnull ? nnull[p] : 0, n);
    if (k > 0) {
      // the k-th smallest eigenvalue, by repeated minimum
      double last = -1e300;
      int taken = 0;
      while (taken < k) {
        double mn = 1e300;
        int cnt = 0;
        for (int i = 0; i < n; ++i) {
          const double l = A[i + i * ld];
          if (l > last && l < mn) mn = l, cnt = 0;
          if (l == mn) ++cnt;
        }
        last = mn;
        taken += max(cnt, 1);
      }
      cut = fmax(cut, last);
    }
    cut_sh = cut;
  }
  __syncthreads();
  const double tol = cut_sh;
  T* out = pinv + QP(p, Q_OPI);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    int r = idx % n, c = idx / n;
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
      double l = A[k + k * ld];
      if (l > tol) s += V[r + k * ld] * V[c + k * ld] / l;
    }
    out[idx] = (T)s;
  }
}

// Gram matrices G = U^T V over the first w columns of the panel (kind 0:
// V = A-block, kind 1: V = B-block), upper triangle computed and mirrored.
// The FP64 entries are split into FP32 pairs (x = x_h + x_l) and the dot
// products carried in FP32 pairs (exact x_h*y_h by FMA, TwoSum, cross terms
// into the low word): about 46 significant bits, at FP32 throughput.
// Pass 1 (k_lob_gram_part): one CTA per (pair, kind, chunk of kGramRows
// rows); a thread owns a 2 x 2 block of the upper triangle, so each staged
// row costs two operand loads per two multiply-adds.  Pass 2
// (k_lob_gram_sum) adds the chunks in order (the sums are deterministic).
constexpr int kGramRows = 512;

__device__ __forceinline__ void df_mac(float& h, float& l, float2 x, float2 y) {
  const float pr = __fmul_rn(x.x, y.x);
  const float e = fmaf(x.x, y.x, -pr);
  const float s = __fadd_rn(h, pr);
  const float bb = __fsub_rn(s, h);
  const float er = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(pr, bb));
  h = s;
  l = fmaf(x.x, y.y, fmaf(x.y, y.x, __fadd_rn(l, __fadd_rn(er, e))));
}

template <typename T>
__global__ void k_lob_gram_part(double* part, const T* Qb, const int64_t* qp, int m, int wfull, const int* act,
                                int nchunk, const int* nwa) {
  const int p = blockIdx.x, kind = blockIdx.y, ch = blockIdx.z;
  double* out = part + (((int64_t)p * 2 + kind) * nchunk + ch) * (int64_t)wfull * wfull;
  // compact active columns (soft locking): X, then the first nw of W and of P
  const int nwp = wfull > m ? min(nwa[p], m) : 0;
  const int w = m + nwp * (wfull / m - 1);
  const int nb = (w + 1) / 2, nblk = nb * (nb + 1) / 2;
  const int64_t N = QP(p, Q_N);
  const int64_t rb = (int64_t)ch * kGramRows, re = min(N, rb + kGramRows);
  if (!act[p] || rb >= re) {
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) out[idx] = 0.0;
    return;
  }
  const T* U = Qb + QP(p, Q_OQ);
  const T* Vb = U + (int64_t)(kind ? 6 * m : 3 * m) * N;
  __shared__ float2 us[32][3 * AMB_MAX_EIG + 2], vs[32][3 * AMB_MAX_EIG + 2];
  // 2 x 2 block (bi, bj), bi <= bj, from the triangular thread index
  const int t = threadIdx.x;
  int bj = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
  while (bj * (bj + 1) / 2 > t) --bj;
  while ((bj + 1) * (bj + 2) / 2 <= t) ++bj;
  const int bi = t - bj * (bj + 1) / 2;
  const bool mine = t < nblk;
  const int a0 = 2 * bi, b0 = 2 * bj;
  float h[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, l[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  const int wp = 2 * nb;   // staged columns (w rounded up to even; the extra one is zero)
  for (int64_t r0 = rb; r0 < re; r0 += 32) {
    const int rn = (re - r0) < 32 ? (int)(re - r0) : 32;
    for (int idx = threadIdx.x; idx < 32 * wp; idx += blockDim.x) {
      const int r = idx % 32, c = idx / 32;
      const bool in = r < rn && c < w;
      const int cc = c < m + nwp ? c : 2 * m + (c - m - nwp);
      const double u = in ? (double)U[r0 + r + (int64_t)cc * N] : 0.0;
      const double v = in ? (double)Vb[r0 + r + (int64_t)cc * N] : 0.0;
      const float uh = (float)u, vh = (float)v;
      us[r][c] = make_float2(uh, (float)(u - (double)uh));
      vs[r][c] = make_float2(vh, (float)(v - (double)vh));
    }
    __syncthreads();
    if (mine) {
      for (int r = 0; r < rn; ++r) {
        const float2 x0 = us[r][a0], x1 = us[r][a0 + 1], y0 = vs[r][b0], y1 = vs[r][b0 + 1];
        df_mac(h[0][0], l[0][0], x0, y0);
        df_mac(h[0][1], l[0][1], x0, y1);
        df_mac(h[1][0], l[1][0], x1, y0);
        df_mac(h[1][1], l[1][1], x1, y1);
      }
    }
    __syncthreads();
  }
  if (mine) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int a = a0 + i, b = b0 + j;
        if (a < w && b < w && a <= b) out[a + b * w] = (double)h[i][j] + (double)l[i][j];
      }
  }
}

__global__ void k_lob_gram_sum(double* G, const double* part, const int64_t* qp, int m, int wfull, const int* act,
                               int nchunk, const int* nwa) {
  const int p = blockIdx.x, kind = blockIdx.y;
  if (!act[p]) return;
  const int m3 = 3 * m;
  const int nwp = wfull > m ? min(nwa[p], m) : 0;
  const int w = m + nwp * (wfull / m - 1);
  const double* in = part + ((int64_t)p * 2 + kind) * nchunk * (int64_t)wfull * wfull;
  double* g = G + QP(p, Q_OGR) + (int64_t)kind * m3 * m3;
  for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
    const int a = idx % w, b = idx / w;
    if (a > b) continue;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += in[(int64_t)c * wfull * wfull + idx];
    g[a + b * m3] = s;
    g[b + a * m3] = s;
  }
}

// Rayleigh-Ritz on the width-w basis: SVQB with column scaling, then the
// reduced standard eigenproblem; coefficients Cc = [Cx | Cp] (3m x 2m, T)
// and the m largest Ritz values.  Frozen pairs keep X (Cx = I, Cp = 0).
template <typename T, int NT>
__global__ void __launch_bounds__(NT, kJacobiThreads / NT) k_lob_rr(T* Cc, double* lam, const double* G, const int64_t* qp, const int* active, int m, int wfull,
                         double drop, const int* nwa) {
  extern __shared__ double sh[];
  const int p = blockIdx.x;
  const int m3 = 3 * m;
  // active basis columns: X (m), then the first nw columns of W and of P
  // (soft locking: the other columns of W and P are zero or unused)
  const int nwp = wfull > m ? min(nwa[p], m) : 0;
  const int w = m + nwp * (wfull / m - 1);
  __shared__ int cmap[3 * AMB_MAX_EIG];
  for (int i = threadIdx.x; i < w; i += blockDim.x)
    cmap[i] = i < m ? i : (i < m + nwp ? i : 2 * m + (i - m - nwp));
  const int ld = w + (w & 1);   // padded for the Jacobi rounds
  double* GA = sh;
  double* GB = GA + ld * ld;
  double* V = GB + ld * ld;
  double* Mr = V + ld * ld;
  double* Yr = Mr + ld * ld;
  double* dsc = Yr + ld * ld;   // w
  __shared__ double red[NT], cs_[kJacobiMax / 2 + 1], sn_[kJacobiMax / 2 + 1];
  __shared__ int P_[kJacobiMax / 2 + 1], Q_[kJacobiMax / 2 + 1], ord[kJacobiMax], ord2[kJacobiMax];
  __shared__ int rank_sh;
  T* C = Cc + QP(p, Q_OCC);
  double* L = lam + (int64_t)p * m;
  if (!active[p]) {
    for (int idx = threadIdx.x; idx < m3 * 2 * m; idx += blockDim.x) {
      int r = idx % m3, c = idx / m3;
      C[idx] = (c < m && r == c) ? T(1) : T(0);
    }
    return;
  }
  const double* ga = G + QP(p, Q_OGR);
  const double* gb = ga + m3 * m3;
  __syncthreads();
  // the Gram matrices are stored in the compact column order
  for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
    int r = idx % w, c = idx / w;
    GA[r + c * ld] = 0.5 * (ga[r + c * m3] + ga[c + r * m3]);
    GB[r + c * ld] = 0.5 * (gb[r + c * m3] + gb[c + r * m3]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double dmax = 0.0;
    for (int i = 0; i < w; ++i) dmax = fmax(dmax, GB[i + i * ld]);
    for (int i = 0; i < w; ++i) {
      double d = GB[i + i * ld];
      dsc[i] = (d > 1e-14 * dmax && d > 0.0) ? 1.0 / sqrt(d) : 0.0;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
    int r = idx % w, c = idx / w;
    GA[r + c * ld] *= dsc[r] * dsc[c];
    GB[r + c * ld] *= dsc[r] * dsc[c];
  }
  __syncthreads();
  jacobi_eig(GB, V, w, ld, red, cs_, sn_, P_, Q_, Mr, Yr);   // Mr, Yr: scratch until Tm is formed
  sort_desc(GB, w, ld, ord);
  if (threadIdx.x == 0) {
    double smax = GB[ord[0] + ord[0] * ld];
    int r = 0;
    while (r < w && GB[ord[r] + ord[r] * ld] > drop * smax && smax > 0.0) ++r;
    rank_sh = r;
  }
  __syncthreads();
  const int r = rank_sh;
  // Tm = V[:, ord[:r]] diag(sigma^{-1/2}) stored in Yr (w x r)
  for (int idx = threadIdx.x; idx < w * r; idx += blockDim.x) {
    int i = idx % w, k = idx / w;
    int c = ord[k];
    Yr[i + k * ld] = V[i + c * ld] / sqrt(GB[c + c * ld]);
  }
  __syncthreads();
  // V := GA Tm (w x r), then Mr := Tm^T V (r x r)
  for (int idx = threadIdx.x; idx < w * r; idx += blockDim.x) {
    int i = idx % w, k = idx / w;
    double s = 0.0;
    for (int j = 0; j < w; ++j) s += GA[i + j * ld] * Yr[j + k * ld];
    V[i + k * ld] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    int a = idx % r, b = idx / r;
    double s = 0.0;
    for (int j = 0; j < w; ++j) s += Yr[j + a * ld] * V[j + b * ld];
    Mr[a + b * ld] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    int a = idx % r, b = idx / r;
    if (a > b) {
      double s = 0.5 * (Mr[a + b * ld] + Mr[b + a * ld]);
      Mr[a + b * ld] = s;
      Mr[b + a * ld] = s;
    }
  }
  __syncthreads();
  jacobi_eig(Mr, GB, r, ld, red, cs_, sn_, P_, Q_, GA, V);   // eigenvectors into GB (r x r, ld); GA, V: scratch
  sort_desc(Mr, r, ld, ord2);
  const int mm = min(m, r);
  // Cx(:, k) = D Tm y_k ; Cp = Cx with the X rows zeroed; rows of the
  // inactive columns are zero
  for (int idx = threadIdx.x; idx < m3 * 2 * m; idx += blockDim.x) C[idx] = T(0);
  __syncthreads();
  for (int idx = threadIdx.x; idx < w * m; idx += blockDim.x) {
    int i = idx % w, k = idx / w;
    double s = 0.0;
    if (k < mm) {
      int c = ord2[k];
      for (int j = 0; j < r; ++j) s += Yr[i + j * ld] * GB[j + c * ld];
      s *= dsc[i];
    }
    const int ri = cmap[i];
    C[ri + (int64_t)k * m3] = (T)s;
    C[ri + (int64_t)(m + k) * m3] = (ri < m) ? T(0) : (T)s;
  }
  if (threadIdx.x < m) {
    int k = threadIdx.x;
    L[k] = k < mm ? Mr[ord2[k] + ord2[k] * ld] : 0.0;
  }
}

// R = A X - B X diag(lambda) into the W slot; residual and B-norms per column
template <typename T>
__global__ void k_lob_resid(T* Qb, double* rn, double* bn, const double* lam, const int64_t* qp, int m,
                            const int* act) {
  const int p = blockIdx.x, col = blockIdx.y;
  if (!act[p]) return;
  const int64_t N = QP(p, Q_N);
  T* base = Qb + QP(p, Q_OQ);
  const T* AX = base + (int64_t)(3 * m + col) * N;
  const T* BX = base + (int64_t)(6 * m + col) * N;
  T* R = base + (int64_t)(m + col) * N;
  const T l = (T)lam[(int64_t)p * m + col];
  __shared__ double red[256];
  double s = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    T v = AX[i] - l * BX[i];
    R[i] = v;
    s += (double)v * (double)v;
    b += (double)BX[i] * (double)BX[i];
  }
  s = block_sum(s, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    rn[(int64_t)p * m + col] = sqrt(s);
    bn[(int64_t)p * m + col] = sqrt(b);
  }
}

// copy the updated blocks back: Tp = [Xn' Pn | AXn' APn | BXn' BPn] -> panel,
// where the X-type blocks hold only the X-row part (X Cx_X) and receive the
// P-type block here: Xn = X Cx_X + Pn (and likewise for AX, BX)
template <typename T>
__global__ void k_lob_copyback(T* Qb, const T* Tp, const int64_t* qp, int m, const int* act) {
  const int p = blockIdx.y;
  if (!act[p]) return;
  const int64_t N = QP(p, Q_N);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * 6 * m) return;
  const int64_t col = idx / N, row = idx % N;
  const int grp = (int)(col / (2 * m)), within = (int)(col % (2 * m));
  // within < m: X-type block (slot 0 of the group), else P-type (slot 2)
  const int slot = grp * 3 + (within < m ? 0 : 2);
  const int c = within % m;
  const T* t = Tp + QP(p, Q_OT) + idx;
  const T v = within < m ? t[0] + t[(int64_t)m * N] : t[0];
  Qb[QP(p, Q_OQ) + (int64_t)(slot * m + c) * N + row] = v;
}

// adaptive rows: columns 0..k-1 of A X restricted to the face dofs (s copy),
// orthonormalized by two passes of classical Gram-Schmidt; rows with a
// negligible diagonal of R are dropped.
template <typename T>
__global__ void k_lob_rows(double* rows, int* kept, const T* Qb, const int64_t* qp, const int* nsel,
                           const int32_t* ps, const int32_t* face, int m) {
  const int p = blockIdx.x;
  const int64_t N = QP(p, Q_N), foff = QP(p, Q_FOFF), nfc = QP(p, Q_FACEN), fco = QP(p, Q_FACEOFF);
  const int k = nsel[p];
  double* Rw = rows + QP(p, Q_OR);
  const T* AX = Qb + QP(p, Q_OQ) + (int64_t)3 * m * N;
  __shared__ double red[256], rkk[AMB_MAX_EIG];
  for (int64_t idx = threadIdx.x; idx < nfc * k; idx += blockDim.x) {
    int64_t e = idx % nfc, l = idx / nfc;
    Rw[e + l * nfc] = (double)AX[ps[foff + face[fco + e]] + l * N];
  }
  __syncthreads();
  for (int l = 0; l < k; ++l) {
    double* v = Rw + (int64_t)l * nfc;
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = 0; j < l; ++j) {
        const double* q = Rw + (int64_t)j * nfc;
        double d = 0.0;
        for (int64_t e = threadIdx.x; e < nfc; e += blockDim.x) d += q[e] * v[e];
        d = block_sum(d, red);
        if (rkk[j] == 0.0) d = 0.0;
        for (int64_t e = threadIdx.x; e < nfc; e += blockDim.x) v[e] -= d * q[e];
        __syncthreads();
      }
    }
    double nrm = 0.0;
    for (int64_t e = threadIdx.x; e < nfc; e += blockDim.x) nrm += v[e] * v[e];
    nrm = sqrt(block_sum(nrm, red));
    if (threadIdx.x == 0) rkk[l] = nrm;
    __syncthreads();
    const double sc = nrm > 0 ? 1.0 / nrm : 0.0;
    for (int64_t e = threadIdx.x; e < nfc; e += blockDim.x) v[e] *= sc;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int l = 0; l < k; ++l) mx = fmax(mx, rkk[l]);
    int c = 0;
    for (int l = 0; l < k; ++l) {
      bool keep = rkk[l] >= 1e-10 * mx && mx > 0.0;
      if (keep) {
        if (c != l)
          for (int64_t e = 0; e < nfc; ++e) Rw[e + c * nfc] = Rw[e + l * nfc];
        ++c;
      }
    }
    kept[p] = c;
  }
}

// R (W slot) -> temp panel columns 0..m; columns >= nw[p] (soft-locked: no
// new search direction) are zero, so that M R, A W and B W vanish there
template <typename T>
__global__ void k_lob_copy_w(T* Tp, const T* Qb, const int64_t* qp, int m, const int* act, const int* nw) {
  const int p = blockIdx.y;
  if (!act[p]) return;
  const int64_t N = QP(p, Q_N);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * m) return;
  Tp[QP(p, Q_OT) + idx] = (idx / N < nw[p]) ? Qb[QP(p, Q_OQ) + (int64_t)m * N + idx] : T(0);
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// ---------------------------------------------------------------- driver

template <typename T>
void Engine<T>::adapt_level(LevelData<T>& L) {
  FamTimer ftm(st, &tm, AMB_FAM_LOBPCG, timing());
  LevelTopo& tp = L.topo;
  const int np = (int)tp.pairs.size();
  const int lvl = L.level;
  if (np == 0) {
    omega.push_back(0.0);
    nadapt.push_back(0);
    return;
  }
  const int maxad = std::max(0, cfg.opt.max_adaptive_per_face);
  int n_sms = 0, dev = 0;
  AMB_CUDA(cudaGetDevice(&dev));
  AMB_CUDA(cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev));
  // block size: the rows the method may add, the indicator column and 4
  // guard columns that keep the last used column from converging slowly
  const int m = std::min(AMB_MAX_EIG, maxad + 1 + 4);
  const int m3 = 3 * m;
  // SVQB: directions whose scaled B-Gram eigenvalue is below drop * max are
  // numerically dependent and are discarded.  The Gram matrices come from
  // FP64 vectors and extended-precision operator products in both forms.
  const double svqb_drop = 1e-10;
  // ------------------------------------------------ pair tables
  std::vector<int64_t> qp((size_t)np * Q_NPAIRF, 0);
  std::vector<int32_t> hps, hpt, hgoff(1, 0), hgent, hface, hcms, hcmt;
  std::vector<double> hws, hwt, hgw;
  std::vector<int64_t> acs(np), act(np);
  std::vector<double> dg_h(L.vG.total);
  AMB_CUDA(cudaMemcpyAsync(dg_h.data(), L.diagG.p, dg_h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  AMB_CUDA(cudaStreamSynchronize(st));
  int64_t oQ = 0, oT = 0, oJ = 0, oF = 0, oC = 0, oPi = 0, oGr = 0, oCc = 0, oR = 0, oZ = 0, oQc = 0;
  std::vector<int64_t> zoff(np), qcoff(np);
  int max_ncp = 0;
  for (int p = 0; p < np; ++p) {
    const PairTopo& P = tp.pairs[p];
    int64_t* q = &qp[(size_t)p * Q_NPAIRF];
    const int s = P.s, t = P.t;
    const int64_t N = L.ng[s] + L.ng[t], nf = (int64_t)P.ps.size();
    q[Q_S] = s;
    q[Q_T] = t;
    q[Q_NS] = L.ng[s];
    q[Q_NT] = L.ng[t];
    q[Q_N] = N;
    q[Q_NF] = nf;
    q[Q_OQ] = oQ;
    oQ += N * 9 * m;
    q[Q_OT] = oT;
    oT += N * 6 * m;
    q[Q_OJ] = oJ;
    oJ += 4 * nf * m;
    q[Q_OF] = oF;
    oF += 2 * nf * nf;
    q[Q_FOFF] = (int64_t)hps.size();
    for (size_t e = 0; e < P.ps.size(); ++e) {
      hps.push_back(P.ps[e]);
      hpt.push_back(P.pt[e]);
      const double ks = dg_h[L.vG.off[s] + P.ps[e]], kt = dg_h[L.vG.off[t] + P.pt[e]];
      hws.push_back(ks / (ks + kt));
      hwt.push_back(kt / (ks + kt));
    }
    q[Q_GBEG] = (int64_t)hgoff.size() - 1;
    for (size_t g = 0; g + 1 < P.goff.size(); ++g) {
      for (int e = P.goff[g]; e < P.goff[g + 1]; ++e) {
        hgent.push_back(P.gent[e]);
        hgw.push_back(P.gw[e]);
      }
      hgoff.push_back((int32_t)hgent.size());
    }
    q[Q_GEND] = (int64_t)hgoff.size() - 1;
    q[Q_FACEOFF] = (int64_t)hface.size();
    q[Q_FACEN] = (int64_t)P.face.size();
    hface.insert(hface.end(), P.face.begin(), P.face.end());
    q[Q_CMS] = (int64_t)hcms.size();
    hcms.insert(hcms.end(), P.cmap_s.begin(), P.cmap_s.end());
    q[Q_CMT] = (int64_t)hcmt.size();
    hcmt.insert(hcmt.end(), P.cmap_t.begin(), P.cmap_t.end());
    q[Q_NCP] = P.n_cpair;
    q[Q_NCS] = L.nc[s];
    q[Q_NCT] = L.nc[t];
    max_ncp = std::max(max_ncp, P.n_cpair);
    q[Q_OC] = oC;
    oC += (int64_t)(2 * L.nc[s] + 2 * L.nc[t] + 2 * P.n_cpair) * m;
    q[Q_OPI] = oPi;
    oPi += (int64_t)P.n_cpair * P.n_cpair;
    q[Q_OGR] = oGr;
    oGr += 2LL * m3 * m3;
    q[Q_OCC] = oCc;
    oCc += (int64_t)m3 * 2 * m;
    q[Q_OR] = oR;
    oR += (int64_t)P.face.size() * m;
    zoff[p] = oZ;
    oZ += (int64_t)(L.nd[s] + L.nd[t]) * m;
    qcoff[p] = oQc;
    oQc += (int64_t)2 * (L.ncp[s] + L.ncp[t]) * m;
    acs[p] = L.pAc.off[s];
    act[p] = L.pAc.off[t];
  }
  AMB_CHECK(max_ncp <= kJacobiMax, AMB_EINVAL,
            "pair coarse space larger than " + std::to_string(kJacobiMax) + " dofs");
  // operator staging blocks (N x m in the factor precision)
  int64_t oO = 0;
  for (int p = 0; p < np; ++p) {
    qp[(size_t)p * Q_NPAIRF + Q_OO] = oO;
    oO += qp[(size_t)p * Q_NPAIRF + Q_N] * m;
  }
  DevBuf dqp, dps, dpt, dws, dwt, dgoff, dgent, dgw, dface, dcms, dcmt, dacs, dact;
  upload(dqp, qp, st);
  upload(dps, hps, st);
  upload(dpt, hpt, st);
  upload(dws, hws, st);
  upload(dwt, hwt, st);
  upload(dgoff, hgoff, st);
  upload(dgent, hgent, st);
  upload(dgw, hgw, st);
  upload(dface, hface, st);
  upload(dcms, hcms, st);
  upload(dcmt, hcmt, st);
  upload(dacs, acs, st);
  upload(dact, act, st);
  // Block vectors, their operator images and the Rayleigh-Ritz coefficients
  // are FP64 (V); only the operator products run in the factor precision T.
  using V = double;
  DevBuf Qb, Tp, Jb, Sff, Zb, Qc, Cb, Pinv, Gr, Cc, lam, rn, bn, act_d, rows, kept, nsel_d, Oin, Oout;
  Qb.alloc(oQ * sizeof(V));
  Tp.alloc(oT * sizeof(V));
  Oin.alloc(oO * sizeof(T));
  Oout.alloc(oO * sizeof(T));
  Jb.alloc(oJ * sizeof(V));
  Sff.alloc(oF * sizeof(T));
  Zb.alloc(oZ * sizeof(T));
  DevBuf Xs;   // substructure-major Neumann right-hand sides and solutions
  Xs.alloc(oZ * sizeof(T));
  Qc.alloc(oQc * sizeof(T));
  Cb.alloc(oC * sizeof(T));
  Pinv.alloc(oPi * sizeof(T));
  Gr.alloc(oGr * sizeof(double));
  int64_t maxN0 = 0;
  for (int p = 0; p < np; ++p) maxN0 = std::max(maxN0, qp[(size_t)p * Q_NPAIRF + Q_N]);
  const int ngchunk = (int)std::max<int64_t>(1, (maxN0 + kGramRows - 1) / kGramRows);
  AMB_CHECK(ngchunk < 65536, AMB_EINVAL, "pair space too large for the Gram kernels");
  DevBuf Gpart;
  Gpart.alloc((size_t)np * 2 * ngchunk * m3 * m3 * sizeof(double));
  Cc.alloc(oCc * sizeof(V));
  lam.alloc((size_t)np * m * sizeof(double));
  rn.alloc((size_t)np * m * sizeof(double));
  bn.alloc((size_t)np * m * sizeof(double));
  act_d.alloc(np * sizeof(int));
  // soft locking (FP32 form): per pair, the number of leading columns that
  // get a new search direction (W) and keep a previous one (P) in the
  // Rayleigh-Ritz basis: the used columns (the selected ones and the
  // indicator) and kGuard more, which keep the last used column converging
  // at the rate of a wider block; the other columns of X stay in the basis
  // without them.  The FP64 form keeps the full block: the pairs of stiff
  // slabs crossing a face (lambda_1 ~ 1e5 tau, whose eigenvector has a
  // B-energy near 1e-13 of the operator's scale) converge there only with
  // every column's search direction, and which rounding path reaches them is
  // fragile.
  const int kGuard = sizeof(T) == sizeof(float) ? 4 : m;
  DevBuf nw_d;
  nw_d.alloc(np * sizeof(int));
  std::vector<int> nwh(np, m);
  rows.alloc(std::max<int64_t>(oR, 1) * sizeof(double));
  kept.alloc(np * sizeof(int));
  nsel_d.alloc(np * sizeof(int));
  AMB_CUDA(cudaMemsetAsync(Gr.p, 0, oGr * sizeof(double), st));
  const int64_t* QPd = dptr<int64_t>(dqp);
  V* Q = dptr<V>(Qb);
  const T one = T(1), zero = T(0);
  std::vector<int> active(np, 1), iters(np, 0), conv(np, 0);

  // S_ff of each side (gathered once, on the device)
  {
    int64_t maxnf0 = 0;
    for (int p = 0; p < np; ++p) maxnf0 = std::max(maxnf0, qp[(size_t)p * Q_NPAIRF + Q_NF]);
    DevBuf dsoff;
    upload(dsoff, L.pS.off, st);
    if (maxnf0 > 0) {
      AMB_CHECK(maxnf0 < 65536, AMB_EINVAL, "pair face larger than 65535 dofs");
      k_lob_sff<T><<<dim3(2 * np, (unsigned)maxnf0), 128, 0, st>>>(dptr<T>(Sff), dptr<T>(L.S), QPd, dptr<int64_t>(dsoff),
                                                                 dptr<int32_t>(dps), dptr<int32_t>(dpt));
      AMB_LAUNCHED();
    }
    AMB_CUDA(cudaStreamSynchronize(st));   // keep the offset table alive until the kernel ran
  }
  // level 1: rigid modes of the floating substructures (those whose elements
  // touch no Dirichlet node), orthonormalized, and T = S Q with the same
  // product as the B applies.  A pair of two floating substructures also
  // keeps the rigid modes of the pair as a whole: they are continuous, so
  // they lie in the range of Pi, and S annihilates them on both sides, so B
  // does (and so does A: the averaging E leaves a continuous function as it
  // is).  The eigenproblem lives on the complement of null(B) (the factor
  // space); the iteration removes these directions from X and W.
  DevBuf nQ, nT, nqoff, pQ, pqoff, pnull_d;
  int nr = 0;
  bool nullproj = false, pairdefl = false;
  std::vector<int> pnull(np, 0);   // rigid modes of the pair as a whole (both sides floating)
  if (lvl == 1) {
    const int dpn = mesh.dpn;
    nr = dpn == 1 ? 1 : 6;
    std::vector<uint8_t> touched(L.ns, 0);
    const int nx = mesh.nx, ny = mesh.ny;
    for (int64_t e = 0; e < mesh.nel; ++e) {
      const int64_t ei = e % nx, ej = (e / nx) % ny, ek = e / ((int64_t)nx * ny);
      bool dir = false;
      for (int c = 0; c < 8 && !dir; ++c) {
        const int64_t node = (ei + (c & 1)) + (int64_t)(nx + 1) * ((ej + ((c >> 1) & 1)) + (int64_t)(ny + 1) * (ek + (c >> 2)));
        dir = mesh.dir_h[node] != 0;
      }
      if (dir) touched[mesh.elem_sub_h[e]] = 1;
    }
    auto node_xyz = [&](int64_t dof, double* c3) {
      const int64_t node = dof / dpn;
      c3[0] = (double)(node % (nx + 1));
      c3[1] = (double)((node / (nx + 1)) % (ny + 1));
      c3[2] = (double)(node / ((int64_t)(nx + 1) * (ny + 1)));
    };
    // the interface centroid of substructure s (accumulated into cen with
    // weight 1 / total)
    auto add_centroid = [&](int s2, double total, double* cen) {
      const SubTopo& sb = tp.subs[s2];
      for (int l = 0; l < L.ng[s2]; ++l) {
        double c3[3];
        node_xyz(sb.dofs[sb.n_i + l], c3);
        for (int a2 = 0; a2 < 3; ++a2) cen[a2] += c3[a2] / total;
      }
    };
    // rigid modes on substructure s2's interface about cen: column k at
    // out + k * ld, rows row0 .. row0 + n_g
    auto fill_modes = [&](int s2, const double* cen, double* out, int64_t ld, int64_t row0) {
      const SubTopo& sb = tp.subs[s2];
      for (int l = 0; l < L.ng[s2]; ++l) {
        double* q = out + row0 + l;
        if (dpn == 1) {
          q[0] = 1.0;
          continue;
        }
        const int64_t dof = sb.dofs[sb.n_i + l];
        const int comp = (int)(dof % dpn);
        double c3[3];
        node_xyz(dof, c3);
        const double px = c3[0] - cen[0], py = c3[1] - cen[1], pz = c3[2] - cen[2];
        q[(int64_t)comp * ld] = 1.0;   // translations
        // rotations w x p about the three axes, component `comp`
        const double rx[3] = {0.0, -pz, py}, ry[3] = {pz, 0.0, -px}, rz[3] = {-py, px, 0.0};
        q[3 * ld] = rx[comp];
        q[4 * ld] = ry[comp];
        q[5 * ld] = rz[comp];
      }
    };
    std::vector<int64_t> qoff(L.ns, -1), foff;
    std::vector<int32_t> fng;
    std::vector<double> hq;
    for (int s2 = 0; s2 < L.ns; ++s2) {
      if (touched[s2] || L.ng[s2] < nr) continue;
      const int n = L.ng[s2];
      qoff[s2] = (int64_t)hq.size();
      foff.push_back(qoff[s2]);
      fng.push_back(n);
      double cen[3] = {0.0, 0.0, 0.0};
      add_centroid(s2, n, cen);
      hq.resize(hq.size() + (size_t)n * nr, 0.0);
      fill_modes(s2, cen, hq.data() + qoff[s2], n, 0);
    }
    if (!foff.empty()) {
      nullproj = true;
      DevBuf dfoff, dfng;
      upload(nQ, hq, st);
      upload(nqoff, qoff, st);
      upload(dfoff, foff, st);
      upload(dfng, fng, st);
      nT.alloc(hq.size() * sizeof(double));
      k_orth_modes<<<(unsigned)foff.size(), 256, 0, st>>>(dptr<double>(nQ), dptr<int64_t>(dfoff), dptr<int32_t>(dfng), nr);
      AMB_LAUNCHED();
      std::vector<GemmDesc> d;
      for (int s2 = 0; s2 < L.ns; ++s2)
        if (qoff[s2] >= 0) d.push_back(GemmDesc{L.ng[s2], nr, L.ng[s2], L.ng[s2], L.ng[s2], L.ng[s2], L.pS.off[s2], qoff[s2], qoff[s2]});
      gemm_batched<double, T>(st, ring, d, 0, 1.0, 0.0, dptr<T>(L.S), dptr<double>(nQ), dptr<double>(nT));
      AMB_CUDA(cudaStreamSynchronize(st));   // keep the host tables alive until the kernels ran
    }
    // pairs of two floating substructures: the pair's rigid modes on
    // [Gamma^s; Gamma^t] about the pair's interface centroid
    std::vector<int64_t> poff(np, -1), pfoff;
    std::vector<int32_t> pfn;
    std::vector<double> hp;
    for (int p = 0; p < np; ++p) {
      const int64_t* q = &qp[(size_t)p * Q_NPAIRF];
      const int s2 = (int)q[Q_S], t2 = (int)q[Q_T];
      if (qoff[s2] < 0 || qoff[t2] < 0) continue;
      const int64_t N = q[Q_N];
      pnull[p] = nr;
      poff[p] = (int64_t)hp.size();
      pfoff.push_back(poff[p]);
      pfn.push_back((int32_t)N);
      double cen[3] = {0.0, 0.0, 0.0};
      add_centroid(s2, (double)N, cen);
      add_centroid(t2, (double)N, cen);
      hp.resize(hp.size() + (size_t)N * nr, 0.0);
      fill_modes(s2, cen, hp.data() + poff[p], N, 0);
      fill_modes(t2, cen, hp.data() + poff[p], N, q[Q_NS]);
    }
    if (!pfoff.empty()) {
      pairdefl = true;
      DevBuf dpfoff, dpfn;
      upload(pQ, hp, st);
      upload(pqoff, poff, st);
      upload(dpfoff, pfoff, st);
      upload(dpfn, pfn, st);
      k_orth_modes<<<(unsigned)pfoff.size(), 256, 0, st>>>(dptr<double>(pQ), dptr<int64_t>(dpfoff), dptr<int32_t>(dpfn), nr);
      AMB_LAUNCHED();
      AMB_CUDA(cudaStreamSynchronize(st));
    }
  }
  // pseudo-inverse of the pair coarse matrices (initial constraints)
  {
    const int nl = max_ncp + (max_ncp & 1);
    const size_t smem = (size_t)2 * nl * nl * sizeof(double);
    AMB_CUDA(cudaFuncSetAttribute(k_pair_pinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 1)));
    upload(pnull_d, pnull, st);
    k_pair_pinv<T><<<np, kJacobiThreads, smem, st>>>(dptr<T>(Pinv), QPd, dptr<double>(L.Ac), dptr<int64_t>(dacs),
                                          dptr<int64_t>(dact), dptr<int32_t>(dcms), dptr<int32_t>(dcmt),
                                          dptr<int>(pnull_d), dptr<int>(status));
    AMB_LAUNCHED();
  }

  // ------------------------------------------------ operators on panel column blocks
  // slot indices (column offsets in units of m): X 0, W 1, P 2, AX 3, AW 4, AP 5, BX 6, BW 7, BP 8
  auto project = [&](V* base, int which, int c0, int w) {
    k_lob_project<V><<<np, 256, 0, st>>>(base, QPd, which, c0, w, dptr<int32_t>(dgoff), dptr<int32_t>(dgent),
                                         dptr<double>(dgw), dptr<int32_t>(dps), dptr<int32_t>(dpt),
                                         dptr<int>(act_d));
    AMB_LAUNCHED();
  };
  int64_t maxN = 0, maxnf = 0;
  for (int p = 0; p < np; ++p) {
    maxN = std::max(maxN, qp[(size_t)p * Q_NPAIRF + Q_N]);
    maxnf = std::max(maxnf, qp[(size_t)p * Q_NPAIRF + Q_NF]);
  }
  auto zero_block = [&](T* base, int which, int c0, int w) {
    k_lob_zero<T><<<dim3(nblk(maxN * w), np), 256, 0, st>>>(base, QPd, which, c0, w);
    AMB_LAUNCHED();
  };
  // FP64 block -> operator staging block, and back
  auto to_op = [&](const V* src, int which, int c0) {
    k_lob_convert<T, V><<<dim3(nblk(maxN * m), np), 256, 0, st>>>(dptr<T>(Oin), src, QPd, Q_OO, 0, which, c0, m);
    AMB_LAUNCHED();
  };
  auto from_op = [&](int cout) {
    k_lob_convert<V, T><<<dim3(nblk(maxN * m), np), 256, 0, st>>>(Q, dptr<T>(Oout), QPd, Q_OQ, cout * m, Q_OO, 0, m);
    AMB_LAUNCHED();
  };
  // out slot = A * (in slot); in and out are column blocks of the panel
  // for the W slot (cin == 1) only the first nwh[p] columns are nonzero:
  // the products run on those, and the outputs start from zero
  auto applyA = [&](int cin, int cout) {
    if (cin == 1) AMB_CUDA(cudaMemsetAsync(Jb.p, 0, oJ * sizeof(V), st));
    k_lob_jump<V, V><<<dim3(nblk(maxnf * m), np), 256, 0, st>>>(dptr<V>(Jb), Q, QPd, Q_OQ, cin * m, m,
                                                                dptr<int32_t>(dps), dptr<int32_t>(dpt),
                                                                dptr<double>(dws), dptr<double>(dwt));
    AMB_LAUNCHED();
    std::vector<GemmDesc> d;
    for (int p = 0; p < np; ++p) {
      const int64_t* q = &qp[(size_t)p * Q_NPAIRF];
      if (!active[p]) continue;
      const int nf = (int)q[Q_NF];
      const int wcol = cin == 1 ? nwh[p] : m;
      for (int side = 0; side < 2; ++side)
        d.push_back(GemmDesc{nf, wcol, nf, std::max(nf, 1), std::max(nf, 1), std::max(nf, 1),
                             q[Q_OF] + side * (int64_t)nf * nf, q[Q_OJ] + side * (int64_t)nf * m,
                             q[Q_OJ] + (2 + side) * (int64_t)nf * m});
    }
    {
      FamTimer fo(st, &tm, AMB_FAM_LOBOP, timing());
      gemm_batched<V, T>(st, ring, d, G_TUNE, 1.0, 0.0, dptr<T>(Sff), dptr<V>(Jb), dptr<V>(Jb));
      for (const GemmDesc& g : d) {
        tm.fam_flops[AMB_FAM_LOBOP] += 2.0 * g.m * g.k * g.n;
        tm.fam_bytes[AMB_FAM_LOBOP] += (double)sizeof(T) * g.m * g.k;
      }
    }
    k_lob_iet<V, V><<<dim3(np, m), 256, 0, st>>>(Q, QPd, Q_OQ, cout * m, dptr<V>(Jb), m, dptr<int32_t>(dps),
                                                dptr<int32_t>(dpt), dptr<double>(dws), dptr<double>(dwt));
    AMB_LAUNCHED();
    project(Q, Q_OQ, cout * m, m);
  };
  auto applyB = [&](int cin, int cout) {
    // FP32 operator entries, FP64 block vectors and accumulation
    if (cin == 1) {
      k_lob_zero<V><<<dim3(nblk(maxN * m), np), 256, 0, st>>>(Q, QPd, Q_OQ, cout * m, m);
      AMB_LAUNCHED();
    }
    std::vector<GemmDesc> d;
    for (int p = 0; p < np; ++p) {
      const int64_t* q = &qp[(size_t)p * Q_NPAIRF];
      if (!active[p]) continue;
      const int64_t N = q[Q_N];
      for (int side = 0; side < 2; ++side) {
        const int sub = (int)(side ? q[Q_T] : q[Q_S]);
        const int ng = L.ng[sub];
        const int64_t r0 = side ? q[Q_NS] : 0;
        d.push_back(GemmDesc{ng, cin == 1 ? nwh[p] : m, ng, std::max(ng, 1), (int)N, (int)N, L.pS.off[sub],
                             q[Q_OQ] + cin * m * N + r0, q[Q_OQ] + cout * m * N + r0});
      }
    }
    {
      FamTimer fo(st, &tm, AMB_FAM_LOBOP, timing());
      if constexpr (std::is_same<T, double>::value) {
        // FP64 form: S X from exact slice products on the tensor cores; the
        // pair sides of one substructure share its S, split once per chunk
        std::vector<TcGemm> tg;
        std::vector<int> key;
        tg.reserve(d.size());
        key.reserve(d.size());
        size_t i = 0;
        for (int p = 0; p < np; ++p) {
          if (!active[p]) continue;
          for (int side = 0; side < 2; ++side, ++i) {
            const GemmDesc& g = d[i];
            tg.push_back(TcGemm{g.a, g.b, g.c, g.lda, g.ldb, g.ldc, g.m, g.n, g.k, 0, 1, 0});
            key.push_back((int)qp[(size_t)p * Q_NPAIRF + (side ? Q_T : Q_S)]);
          }
        }
        tc_gemm_f64(st, ring, tg, 1.0, 0.0, dptr<double>(L.S), Q, Q, dptr<int>(status), &key);
      } else {
        gemm_batched<V, T>(st, ring, d, G_TUNE, 1.0, 0.0, dptr<T>(L.S), Q, Q);
      }
      std::vector<char> seen(L.ns, 0);
      for (size_t i = 0; i < d.size(); ++i) {
        const GemmDesc& g = d[i];
        tm.fam_flops[AMB_FAM_LOBOP] += 2.0 * g.m * g.k * g.n;
      }
      // algorithmic bytes: every substructure's S once per apply
      for (int p = 0; p < np; ++p) {
        if (!active[p]) continue;
        for (int side = 0; side < 2; ++side) {
          const int sub = (int)qp[(size_t)p * Q_NPAIRF + (side ? Q_T : Q_S)];
          if (seen[sub]) continue;
          seen[sub] = 1;
          tm.fam_bytes[AMB_FAM_LOBOP] += (double)sizeof(T) * L.ng[sub] * L.ng[sub];
        }
      }
    }
    if (nullproj) {
      k_lob_nullproj<<<2 * np, 256, 0, st>>>(Q, QPd, cin, cout, m, dptr<int>(act_d), dptr<int64_t>(nqoff),
                                             dptr<double>(nQ), dptr<double>(nT), nr,
                                             cin == 1 ? dptr<int>(nw_d) : nullptr);
      AMB_LAUNCHED();
    }
    project(Q, Q_OQ, cout * m, m);
  };
  // W slot = M * (R in the temp panel, columns 0..m)
  auto applyM = [&](int cout) {
    project(dptr<V>(Tp), Q_OT, 0, m);
    to_op(dptr<V>(Tp), Q_OT, 0);
    zero_block(dptr<T>(Oout), Q_OO, 0, m);
    std::vector<GemmDesc> d1, d2, d3, d4, d5, dc1, dc2, dpi;
    // Neumann: per substructure, z = L_D^{-1} r_D; q = Y^T z; l = Ginv q;
    // z -= Y l; out_D = L_D^{-T} z, on the active pair-sides side by side
    std::vector<int> nsd(L.ns, 0);
    for (int p = 0; p < np; ++p) {
      if (!active[p]) continue;
      ++nsd[qp[(size_t)p * Q_NPAIRF + Q_S]];
      ++nsd[qp[(size_t)p * Q_NPAIRF + Q_T]];
    }
    std::vector<int64_t> xo(L.ns, 0), qo2(L.ns, 0);
    int64_t ox = 0, oq = 0;
    for (int s2 = 0; s2 < L.ns; ++s2) {
      xo[s2] = ox;
      qo2[s2] = oq;
      ox += (int64_t)L.nd[s2] * m * nsd[s2];
      oq += (int64_t)2 * L.ncp[s2] * m * nsd[s2];
    }
    std::vector<NeuMap> nmap;
    std::vector<int> used(L.ns, 0);
    for (int p = 0; p < np; ++p) {
      const int64_t* q = &qp[(size_t)p * Q_NPAIRF];
      if (!active[p]) continue;
      for (int side = 0; side < 2; ++side) {
        const int sub = (int)(side ? q[Q_T] : q[Q_S]);
        const int64_t r0 = side ? q[Q_NS] : 0;
        nmap.push_back(NeuMap{q[Q_OO] + r0, xo[sub] + (int64_t)used[sub] * m * L.nd[sub], (int)q[Q_N], L.nd[sub]});
        ++used[sub];
      }
    }
    for (int s2 = 0; s2 < L.ns; ++s2) {
      if (nsd[s2] == 0 || L.nd[s2] == 0) continue;
      const int nd = L.nd[s2], ncp = L.ncp[s2], wd = m * nsd[s2];
      const int ldd = std::max(nd, 1), ldc = std::max(ncp, 1);
      const int64_t zo = xo[s2], qo = qo2[s2];
      d1.push_back(GemmDesc{nd, wd, nd, ldd, ldd, ldd, L.pLD.off[s2], zo, zo});
      d2.push_back(GemmDesc{ncp, wd, nd, ldd, ldd, ldc, L.pY.off[s2], zo, qo});
      d3.push_back(GemmDesc{ncp, wd, ncp, ldc, ldc, ldc, L.pG.off[s2], qo, qo + (int64_t)ncp * wd});
      d4.push_back(GemmDesc{nd, wd, ncp, ldd, ldc, ldd, L.pY.off[s2], qo + (int64_t)ncp * wd, zo});
      d5.push_back(GemmDesc{nd, wd, nd, ldd, ldd, ldd, L.pLD.off[s2], zo, zo});
    }
    if (!nmap.empty()) {
      const NeuMap* dmap = static_cast<const NeuMap*>(ring.push(nmap.data(), nmap.size() * sizeof(NeuMap), st));
      const unsigned gx = (unsigned)std::min<int64_t>(nblk((int64_t)imax(L.nd) * m), 64);
      k_lob_neu_move<T><<<dim3(gx, (unsigned)nmap.size()), 256, 0, st>>>(dptr<T>(Xs), dptr<T>(Oin), dmap, m, 1);
      AMB_LAUNCHED();
      if constexpr (std::is_same<T, double>::value) {
        // FP64 form: the two triangular products with L_D^-1 (the bulk of the
        // Neumann solve) from exact slice products on the tensor cores:
        // C = A B^T with B(j, k) = Xs(k, j) (K-major), A = L_D^-1 (lower) or
        // its transpose (K-major reads, upper)
        std::vector<TcGemm> t1, t5;
        for (const auto& g : d1) t1.push_back(TcGemm{g.a, g.b, g.c, g.lda, g.ldb, g.ldc, g.m, g.n, g.k, 0, 1, 1});
        for (const auto& g : d5) t5.push_back(TcGemm{g.a, g.b, g.c, g.lda, g.ldb, g.ldc, g.m, g.n, g.k, 1, 1, 2});
        tc_gemm_f64(st, ring, t1, 1.0, 0.0, dptr<double>(L.LinvD), dptr<double>(Xs), dptr<double>(Zb), dptr<int>(status));
        gemm_batched<T>(st, ring, d2, G_TRANS_A | G_TUNE, one, zero, dptr<T>(L.Y), dptr<T>(Zb), dptr<T>(Qc));
        gemm_batched<T>(st, ring, d3, 0, one, zero, dptr<T>(L.Ginv), dptr<T>(Qc), dptr<T>(Qc));
        gemm_batched<T>(st, ring, d4, 0, T(-1), one, dptr<T>(L.Y), dptr<T>(Qc), dptr<T>(Zb));
        tc_gemm_f64(st, ring, t5, 1.0, 0.0, dptr<double>(L.LinvD), dptr<double>(Zb), dptr<double>(Xs), dptr<int>(status));
      } else {
        gemm_batched<T>(st, ring, d1, G_TRI_A_LOWER | G_TUNE, one, zero, dptr<T>(L.LinvD), dptr<T>(Xs), dptr<T>(Zb));
        gemm_batched<T>(st, ring, d2, G_TRANS_A | G_TUNE, one, zero, dptr<T>(L.Y), dptr<T>(Zb), dptr<T>(Qc));
        gemm_batched<T>(st, ring, d3, 0, one, zero, dptr<T>(L.Ginv), dptr<T>(Qc), dptr<T>(Qc));
        gemm_batched<T>(st, ring, d4, 0, T(-1), one, dptr<T>(L.Y), dptr<T>(Qc), dptr<T>(Zb));
        gemm_batched<T>(st, ring, d5, G_TRANS_A | G_TRI_A_UPPER | G_TUNE, one, zero, dptr<T>(L.LinvD), dptr<T>(Zb),
                        dptr<T>(Xs));
      }
      k_lob_neu_move<T><<<dim3(gx, (unsigned)nmap.size()), 256, 0, st>>>(dptr<T>(Oout), dptr<T>(Xs), dmap, m, 0);
      AMB_LAUNCHED();
    }
    // coarse: c = Psi^T r per pair-side ; later out += Psi u
    for (int p = 0; p < np; ++p) {
      const int64_t* q = &qp[(size_t)p * Q_NPAIRF];
      if (!active[p]) continue;
      const int64_t N = q[Q_N];
      int64_t co = q[Q_OC];
      for (int side = 0; side < 2; ++side) {
        const int sub = (int)(side ? q[Q_T] : q[Q_S]);
        const int nc = L.nc[sub], ng = L.ng[sub];
        const int64_t rin = q[Q_OO] + (side ? q[Q_NS] : 0);
        dc1.push_back(GemmDesc{nc, m, ng, std::max(ng, 1), (int)N, std::max(nc, 1), L.pPsi.off[sub], rin, co});
        co += (int64_t)nc * m;
      }
    }
    gemm_batched<T>(st, ring, dc1, G_TRANS_A | G_TUNE, one, zero, dptr<T>(L.Psi), dptr<T>(Oin), dptr<T>(Cb));
    k_lob_cgather<T><<<np, 256, 0, st>>>(dptr<T>(Cb), QPd, m, dptr<int32_t>(dcms), dptr<int32_t>(dcmt));
    AMB_LAUNCHED();
    for (int p = 0; p < np; ++p) {
      const int64_t* q = &qp[(size_t)p * Q_NPAIRF];
      if (!active[p]) continue;
      const int ncpr = (int)q[Q_NCP];
      const int64_t cp = q[Q_OC] + (q[Q_NCS] + q[Q_NCT]) * m;
      dpi.push_back(GemmDesc{ncpr, m, ncpr, std::max(ncpr, 1), std::max(ncpr, 1), std::max(ncpr, 1), q[Q_OPI], cp,
                             cp + (int64_t)ncpr * m});
    }
    gemm_batched<T>(st, ring, dpi, 0, one, zero, dptr<T>(Pinv), dptr<T>(Cb), dptr<T>(Cb));
    k_lob_cscatter<T><<<np, 256, 0, st>>>(dptr<T>(Cb), QPd, m, dptr<int32_t>(dcms), dptr<int32_t>(dcmt));
    AMB_LAUNCHED();
    for (int p = 0; p < np; ++p) {
      const int64_t* q = &qp[(size_t)p * Q_NPAIRF];
      if (!active[p]) continue;
      const int64_t N = q[Q_N];
      const int64_t us = q[Q_OC] + (q[Q_NCS] + q[Q_NCT] + 2 * q[Q_NCP]) * m;
      int64_t uo = us;
      for (int side = 0; side < 2; ++side) {
        const int sub = (int)(side ? q[Q_T] : q[Q_S]);
        const int nc = L.nc[sub], ng = L.ng[sub];
        const int64_t r0 = side ? q[Q_NS] : 0;
        dc2.push_back(GemmDesc{ng, m, nc, std::max(ng, 1), std::max(nc, 1), (int)N, L.pPsi.off[sub], uo,
                               q[Q_OO] + r0});
        uo += (int64_t)nc * m;
      }
    }
    gemm_batched<T>(st, ring, dc2, 0, one, one, dptr<T>(L.Psi), dptr<T>(Cb), dptr<T>(Oout));
    from_op(cout);
    project(Q, Q_OQ, cout * m, m);
  };
  auto rayleigh_ritz = [&](int w) {
    k_lob_gram_part<V><<<dim3(np, 2, ngchunk), 320, 0, st>>>(dptr<double>(Gpart), Q, QPd, m, w, dptr<int>(act_d),
                                                            ngchunk, dptr<int>(nw_d));
    AMB_LAUNCHED();
    k_lob_gram_sum<<<dim3(np, 2), 256, 0, st>>>(dptr<double>(Gr), dptr<double>(Gpart), QPd, m, w, dptr<int>(act_d),
                                               ngchunk, dptr<int>(nw_d));
    AMB_LAUNCHED();
    const int wl = w + (w & 1);
    const size_t smem = (size_t)(5 * wl * wl + wl) * sizeof(double);
    // one 1024-thread CTA per pair while the pairs fit on the SMs at once
    // (latency of one pair); with more pairs, two 512-thread CTAs per SM, so
    // that one pair's barriers and FP64 latency overlap another's work
    if (np <= n_sms) {
      AMB_CUDA(cudaFuncSetAttribute(k_lob_rr<V, kJacobiThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_lob_rr<V, kJacobiThreads><<<np, kJacobiThreads, smem, st>>>(dptr<V>(Cc), dptr<double>(lam), dptr<double>(Gr), QPd,
                                                                   dptr<int>(act_d), m, w, svqb_drop, dptr<int>(nw_d));
    } else {
      AMB_CUDA(cudaFuncSetAttribute(k_lob_rr<V, kJacobiThreads / 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      AMB_CUDA(cudaFuncSetAttribute(k_lob_rr<V, kJacobiThreads / 2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    cudaSharedmemCarveoutMaxShared));
      k_lob_rr<V, kJacobiThreads / 2><<<np, kJacobiThreads / 2, smem, st>>>(dptr<V>(Cc), dptr<double>(lam), dptr<double>(Gr),
                                                                           QPd, dptr<int>(act_d), m, w, svqb_drop,
                                                                           dptr<int>(nw_d));
    }
    AMB_LAUNCHED();
    // [Xn Pn] = U [Cx | Cp] with Cp = Cx with the X rows zeroed, so
    // Pn = U(:, m:w) Cx(m:w, :) and Xn = U(:, 0:m) Cx(0:m, :) + Pn: two
    // products of N x m x (w-m) and N x m x m instead of N x 2m x w (the sum
    // is formed in the copy-back).  Same for AU and BU.
    // Rows of the soft-locked W and P columns are zero in Cx.  The FP32 form
    // multiplies only the active rows: Pn = W(:, 0:nw) Cx(W rows) and then
    // += P(:, 0:nw) Cx(P rows).  The FP64 form (no soft locking) keeps the W
    // and P parts in one product, one accumulation chain per entry, as the
    // plain method.
    std::vector<GemmDesc> dp, dpp, dx;
    const bool split = sizeof(T) == sizeof(float) && w > 2 * m;
    for (int p = 0; p < np; ++p) {
      const int64_t* q = &qp[(size_t)p * Q_NPAIRF];
      if (!active[p]) continue;
      const int64_t N = q[Q_N];
      const int nwp = std::min(nwh[p], m);
      for (int g = 0; g < 3; ++g) {
        const int64_t u = q[Q_OQ] + (int64_t)3 * g * m * N, t = q[Q_OT] + (int64_t)2 * g * m * N;
        if (split) {
          dp.push_back(GemmDesc{(int)N, m, nwp, (int)N, m3, (int)N, u + (int64_t)m * N, q[Q_OCC] + m,
                                t + (int64_t)m * N});
          dpp.push_back(GemmDesc{(int)N, m, nwp, (int)N, m3, (int)N, u + (int64_t)2 * m * N, q[Q_OCC] + 2 * m,
                                 t + (int64_t)m * N});
        } else {
          dp.push_back(GemmDesc{(int)N, m, w - m, (int)N, m3, (int)N, u + (int64_t)m * N, q[Q_OCC] + m,
                                t + (int64_t)m * N});
        }
        dx.push_back(GemmDesc{(int)N, m, m, (int)N, m3, (int)N, u, q[Q_OCC], t});
      }
    }
    gemm_batched<V>(st, ring, dp, G_TUNE, 1.0, 0.0, Q, dptr<V>(Cc), dptr<V>(Tp));
    if (!dpp.empty()) gemm_batched<V>(st, ring, dpp, 0, 1.0, 1.0, Q, dptr<V>(Cc), dptr<V>(Tp));
    gemm_batched<V>(st, ring, dx, G_TUNE, 1.0, 0.0, Q, dptr<V>(Cc), dptr<V>(Tp));
    k_lob_copyback<V><<<dim3(nblk(maxN * 6 * m), np), 256, 0, st>>>(Q, dptr<V>(Tp), QPd, m, dptr<int>(act_d));
    AMB_LAUNCHED();
  };

  // ------------------------------------------------ LOBPCG
  // the factor space: the pair rigid modes out of a slot's leading columns
  auto deflate = [&](int slot, const int* ncol) {
    if (!pairdefl) return;
    k_lob_deflate<<<np, 256, 0, st>>>(Q, QPd, slot, m, dptr<int>(act_d), dptr<int64_t>(pqoff), dptr<double>(pQ), nr,
                                      ncol);
    AMB_LAUNCHED();
  };
  k_lob_random<V><<<dim3(nblk(maxN * 9 * m), np), 256, 0, st>>>(Q, QPd, m, cfg.opt.seed + 7919ull * lvl);
  AMB_LAUNCHED();
  AMB_CUDA(cudaMemcpyAsync(act_d.p, active.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
  project(Q, Q_OQ, 0, m);
  deflate(0, nullptr);
  applyA(0, 3);
  applyB(0, 6);
  rayleigh_ritz(m);
  std::vector<double> hl((size_t)np * m), hr((size_t)np * m), hb((size_t)np * m);
  const double tol = cfg.opt.lobpcg_tol;
  const int maxit = std::max(1, cfg.opt.lobpcg_maxit);
  const double tau = cfg.tau;
  std::vector<double> resid(np, 0.0), best(np, 1e300), prev((size_t)np * m, -1e300);
  std::vector<int> since(np, 0), stable(np, 0);
  // Convergence: every used column's residual at most tol, or every used
  // Ritz value still to kRitzTol (relative) for kRitzStable iterations in a
  // row.  The columns of very large eigenvalues (a stiff inclusion across
  // the face, lambda ~ 1e5 tau) have a residual floor far above tol: their
  // eigenvector's B-energy is tiny against its Euclidean norm, so the
  // residual's components along B's large eigenvalues dominate it, while
  // the Ritz value converges (quadratically in the eigenvector's error) to
  // the pencil's.  Iterating on after that lets rounding in [X W P] bring
  // spurious directions back into the basis.
  // Stagnation: far from tol, kStall iterations without halving the worst
  // used residual; within kFloor x tol (the residual floor of the operator
  // products, reached by some pairs of the FP32 form), kFloorStall.
  // FP64 form: a used Ritz value that still rises by more than tol (relative)
  // also counts as progress.  Ritz values of the FP32 form carry the FP32
  // pencil's noise, so that form keeps the residual rule alone there.
  constexpr int kStall = 20, kFloorStall = 3, kRitzStable = 2;
  constexpr double kFloor = 10.0, kRitzTol = 1e-10;
  constexpr bool kRitzProgress = sizeof(T) == sizeof(double);
  auto check = [&]() {
    k_lob_resid<V><<<dim3(np, m), 256, 0, st>>>(Q, dptr<double>(rn), dptr<double>(bn), dptr<double>(lam), QPd, m, dptr<int>(act_d));
    AMB_LAUNCHED();
    AMB_CUDA(cudaMemcpyAsync(hl.data(), lam.p, hl.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    AMB_CUDA(cudaMemcpyAsync(hr.data(), rn.p, hr.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    AMB_CUDA(cudaMemcpyAsync(hb.data(), bn.p, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    AMB_CUDA(cudaStreamSynchronize(st));
    int nact = 0;
    for (int p = 0; p < np; ++p) {
      bool ok = true;
      const double lref = 0.1 * tau;
      // the columns the method uses: the selected ones (lambda > tau, at most
      // max_adaptive_per_face) and the next one, lambda_{k+1}, the indicator
      int kuse = 0;
      while (kuse < m && kuse < maxad && hl[(size_t)p * m + kuse] > tau) ++kuse;
      kuse = std::min(m, kuse + 1);
      nwh[p] = std::min(m, kuse + kGuard);
      double worst = 0.0;
      bool rising = false, still = true;
      for (int k = 0; k < kuse; ++k) {
        const double l = hl[(size_t)p * m + k];
        const double b = hb[(size_t)p * m + k];
        if (kRitzProgress && l - prev[(size_t)p * m + k] > tol * std::max(std::fabs(l), lref)) rising = true;
        if (!(std::fabs(l - prev[(size_t)p * m + k]) <= kRitzTol * std::max(std::fabs(l), lref))) still = false;
        if (b == 0.0) continue;   // dropped direction (rank-deficient pair space)
        const double ratio = hr[(size_t)p * m + k] / (std::max(std::fabs(l), lref) * b);
        worst = std::max(worst, std::isfinite(ratio) ? ratio : 1e300);
        if (!(ratio <= tol)) ok = false;
      }
      resid[p] = worst;
      stable[p] = still ? stable[p] + 1 : 0;
      ok = ok || stable[p] >= kRitzStable;
      conv[p] = ok ? 1 : 0;
      // a stagnating pair stops iterating (reported as not converged, with
      // its residual)
      for (int k = 0; k < m; ++k) prev[(size_t)p * m + k] = hl[(size_t)p * m + k];
      if (worst < 0.5 * best[p]) {
        best[p] = worst;
        since[p] = 0;
      } else if (rising) {
        since[p] = 0;
      } else {
        ++since[p];
      }
      const bool stalled = since[p] >= kStall || (worst <= kFloor * tol && since[p] >= kFloorStall);
      active[p] = (ok || stalled) ? 0 : 1;
      nact += active[p];
    }
    return nact;
  };
  int it = 0;
  for (; it < maxit; ++it) {
    const int nact = check();
    if (nact == 0) break;
    for (int p = 0; p < np; ++p) iters[p] += active[p];
    AMB_CUDA(cudaMemcpyAsync(act_d.p, active.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    AMB_CUDA(cudaMemcpyAsync(nw_d.p, nwh.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    // R (W slot) -> temp panel columns 0..m, then W = M R
    k_lob_copy_w<V><<<dim3(nblk(maxN * m), np), 256, 0, st>>>(dptr<V>(Tp), Q, QPd, m, dptr<int>(act_d),
                                                             dptr<int>(nw_d));
    AMB_LAUNCHED();
    applyM(1);
    deflate(1, dptr<int>(nw_d));
    applyA(1, 4);
    applyB(1, 7);
    rayleigh_ritz(it == 0 ? 2 * m : 3 * m);
  }
  // consistency refresh: A X and B X are carried by the same coefficient
  // recurrence as X, and with a near-dependent [X W P] the coefficients are
  // large enough for them to drift from the products of the current X.
  // Recompute both for every pair and finish with Rayleigh-Ritz on X alone,
  // so that the reported eigenvalues are Rayleigh quotients of the vectors
  // and the rows below come from fresh A X.
  std::fill(active.begin(), active.end(), 1);
  AMB_CUDA(cudaMemcpyAsync(act_d.p, active.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
  applyA(0, 3);
  applyB(0, 6);
  rayleigh_ritz(m);
  check();
  // ------------------------------------------------ selection and rows
  std::vector<int> nsel(np, 0);
  double om = 0.0;
  for (int p = 0; p < np; ++p) {
    int k = 0;
    while (k < m && k < maxad && hl[(size_t)p * m + k] > tau) ++k;
    nsel[p] = k;
    const double next = k < m ? hl[(size_t)p * m + k] : 0.0;
    om = std::max(om, next);
  }
  AMB_CUDA(cudaMemcpyAsync(nsel_d.p, nsel.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
  k_lob_rows<V><<<np, 256, 0, st>>>(dptr<double>(rows), dptr<int>(kept), Q, QPd, dptr<int>(nsel_d), dptr<int32_t>(dps),
                                    dptr<int32_t>(dface), m);
  AMB_LAUNCHED();
  std::vector<double> hrows(std::max<int64_t>(oR, 1));
  std::vector<int> hkept(np);
  AMB_CUDA(cudaMemcpyAsync(hrows.data(), rows.p, hrows.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  AMB_CUDA(cudaMemcpyAsync(hkept.data(), kept.p, np * sizeof(int), cudaMemcpyDeviceToHost, st));
  AMB_CUDA(cudaStreamSynchronize(st));
  check_status("pair coarse pseudo-inverse", AMB_EASSUMPTION);
  int total = 0;
  L.pair_rows.assign(np, {});
  for (int p = 0; p < np; ++p) {
    const PairTopo& P = tp.pairs[p];
    const int64_t nfc = (int64_t)P.face.size();
    const int64_t o = qp[(size_t)p * Q_NPAIRF + Q_OR];
    std::vector<std::vector<double>> rr;
    for (int l = 0; l < hkept[p]; ++l)
      rr.emplace_back(hrows.begin() + o + l * nfc, hrows.begin() + o + (l + 1) * nfc);
    PairReportH rep;
    rep.level = lvl;
    rep.s = P.s;
    rep.t = P.t;
    rep.n_computed = m;
    rep.n_selected = nsel[p];
    rep.n_rows = hkept[p];
    rep.converged = conv[p];
    rep.iterations = iters[p];
    rep.residual = resid[p];
    rep.lambda.assign(hl.begin() + (size_t)p * m, hl.begin() + (size_t)(p + 1) * m);
    reports.push_back(rep);
    total += hkept[p];
    L.pair_rows[p] = rr;
  }
  for (int p = 0; p < np; ++p)
    if (!L.pair_rows[p].empty()) add_adaptive_rows(tp, p, L.pair_rows[p]);
  number_coarse(tp);
  omega.push_back(om);
  nadapt.push_back(total);
}

template void Engine<float>::adapt_level(LevelData<float>&);
template void Engine<double>::adapt_level(LevelData<double>&);

}  // namespace amb
