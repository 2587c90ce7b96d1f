/*
 * amb.h -- C ABI of the GB300 batched substructure engine for
 * Adaptive-Multilevel BDDC (Sousedik, Sistek, Mandel, arXiv:1301.0191).
 *
 * The library solves A u = f (Sec. 2, eq. problem-full-space-algebraic) for
 * a Q1 hexahedral discretization of a scalar diffusion or a linear
 * elasticity problem on a structured grid, with PCG preconditioned by one
 * application of Multilevel BDDC (Algorithm 1), whose constraints are
 * selected adaptively on every level (Algorithm 3, Sec. 4 to 6).
 *
 * Conventions shared by every entry point
 *  - Every call returns an int status: AMB_OK (0) or one of the AMB_E*
 *    codes below.  Nothing is thrown across the ABI.  amb_last_error()
 *    returns a NUL-terminated message for the last failing call on a
 *    context (owned by the context, valid until its next call).
 *  - Vectors on the mesh are "full-grid nodal": length
 *    n_nodes * dofs_per_node, dof = node * dofs_per_node + component,
 *    node (i,j,k) = i + (nx+1)*(j + (ny+1)*k).  Entries of Dirichlet nodes
 *    are ignored on input and written as 0 on output.
 *  - Element arrays: element (i,j,k) = i + nx*(j + ny*k).
 *  - Pointer arguments marked [host|device] may point to host memory or to
 *    device memory of the context's GPU; the library detects which with
 *    cudaPointerGetAttributes and copies host data itself.  The caller owns
 *    every input and output buffer; the library copies what it keeps.
 *  - All device work is issued on amb_options.cuda_stream (NULL = the
 *    legacy default stream); calls return after that stream has finished
 *    the call's work, so outputs are ready on return.
 *  - A context is not thread-safe: use one context per host thread.
 *  - Beside the contexts' own memory, each host thread that calls the
 *    library keeps device workspaces for its tensor-core products (the
 *    operand slabs of the current Cholesky panel or product chunk; in the
 *    FP64 form eight FP32 digit slices per operand entry, 3.4 GB for the
 *    48^3 workload's largest update).  They grow to the largest need seen,
 *    are reused by later calls of the same thread and freed when the thread
 *    ends.  They live on the first GPU the thread works on: a thread that
 *    later serves a context on another GPU gets AMB_EINVAL (serve each GPU's
 *    contexts from threads of their own).  The set-up's host combinatorics run on up to 16 threads of
 *    their own, which end before the call returns; the environment variable
 *    AMB_HOST_THREADS (read once) caps them (1: the calling thread only).
 *    Their results do not depend on the number of threads.
 */
#ifndef AMB_H
#define AMB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define AMB_OK           0
#define AMB_EINVAL       1   /* invalid argument or size */
#define AMB_ENOMEM       2   /* device or host allocation failed */
#define AMB_ENOTSPD      3   /* non-positive pivot in a Cholesky factorization */
#define AMB_EASSUMPTION  4   /* Assumption 1 violated: a constrained local problem is singular */
#define AMB_ENOCONV      5   /* PCG did not reach the tolerance within pcg_maxit */
#define AMB_ETIMEOUT     6   /* a bounded device wait gave up */
#define AMB_ECUDA        7   /* a CUDA runtime call failed */

/* precision of the substructure factors and preconditioner applies; the
 * outer PCG, its residuals and dot products, the Rayleigh-Ritz projections
 * and the coarsest factorization are always FP64 */
#define AMB_FP64 0
#define AMB_FP32 1

/* initial constraints (Sec. 7.1) */
#define AMB_CORNERS        1   /* corners only */
#define AMB_CORNERS_EDGES  2   /* corners + arithmetic edge averages (paper default) */
#define AMB_CORNERS_EDGES_FACES 3 /* + arithmetic face averages, one per face and component: the
                                     non-adaptive "c+e+f" of Sec. 8.2 (Table 6); requires adaptive = 0 */

/* quantity of interest for amb_grad */
#define AMB_QOI_COMPLIANCE 0   /* q = f^T u, adjoint = u */
#define AMB_QOI_GENERAL    1   /* dq/du supplied by the caller */

#define AMB_MAX_EIG 16
#define AMB_MAX_LEVELS 8

typedef struct amb_ctx amb_ctx;   /* opaque, owned by the library */

/* Structured hexahedral mesh of [0, nx*h] x [0, ny*h] x [0, nz*h] (Sec. 2). */
typedef struct {
  int32_t nx, ny, nz;          /* elements per axis, each >= 1 */
  double h;                    /* element edge length (cubic elements) */
  int32_t dofs_per_node;       /* 1 = scalar diffusion, 3 = linear elasticity */
  const uint8_t* dirichlet_node_mask; /* [host] (nx+1)(ny+1)(nz+1); 1 = all dofs of the node fixed to 0 */
} amb_mesh;

/* Per-element material: element matrix = coeff[e] * Khat (Q1, 2x2x2 Gauss). */
typedef struct {
  const double* coeff;         /* [host|device] n_el: kappa (diffusion) or Young's modulus (elasticity), > 0 */
  double poisson_ratio;        /* elasticity only, in (-1, 0.5) */
} amb_coeffs;

/* Decomposition hierarchy (Sec. 3): level-1 substructure of every element,
 * then the level-(i+1) substructure of every level-i substructure.  Every
 * substructure must be a box of elements (tensor-product partitions), so
 * that corners follow the box-vertex rule. */
typedef struct {
  const int32_t* elem_to_sub;            /* [host] n_el, values 0..n_sub1-1 */
  int32_t n_sub1;
  const int32_t* const* sub_to_parent;   /* [host] levels-2 arrays */
  const int32_t* n_sub;                  /* [host] levels-2 counts: n_sub[i] = #substructures on level i+2 */
} amb_partition;

typedef struct {
  int32_t precision;            /* AMB_FP64 | AMB_FP32 */
  int32_t initial_constraints;  /* AMB_CORNERS | AMB_CORNERS_EDGES | AMB_CORNERS_EDGES_FACES */
  int32_t adaptive;             /* 1 = adaptive face constraints (Algorithm 3), 0 = initial constraints only */
  int32_t max_adaptive_per_face;/* at most this many rows per face (paper: 10) */
  int32_t lobpcg_maxit;         /* LOBPCG iteration cap (paper mode 15) */
  double lobpcg_tol;            /* residual tolerance ||Ax - lam Bx|| <= tol * lam * ||Bx|| */
  double pcg_rtol;              /* stop at ||r||_2 <= pcg_rtol ||f||_2 */
  int32_t pcg_maxit;
  uint64_t seed;                /* LOBPCG start vectors */
  void* cuda_stream;            /* cudaStream_t or NULL */
  int32_t timing_events;        /* 1 = CUDA-event timing of the kernel families (amb_stats) */
} amb_options;

typedef struct {
  int32_t iterations;           /* PCG iterations k with ||r_k|| <= rtol ||f|| */
  double rel_residual;          /* ||r_k|| / ||f|| of the recursive residual */
  double true_rel_residual;     /* ||f - A u|| / ||f|| recomputed at exit */
  double cond_estimate;         /* Lanczos estimate from the CG coefficients */
  double ms;                    /* device time of the call */
} amb_solve_info;

typedef struct {
  int32_t level, s, t;          /* level (1-based) and the pair s < t */
  int32_t n_computed;           /* eigenpairs computed (<= AMB_MAX_EIG) */
  int32_t n_selected;           /* rows added: lambda > tau, at most max_adaptive_per_face */
  int32_t n_rows;               /* rows kept after QR */
  int32_t converged;            /* 1 if every residual met lobpcg_tol */
  int32_t iterations;           /* LOBPCG iterations */
  double lambda[AMB_MAX_EIG];   /* computed eigenvalues, descending; where the pair space has fewer
                                   than n_computed directions of non-negligible B-norm, the
                                   columns beyond them report 0 */
  double residual;              /* max over the used columns (selected + next) of
                                   ||A x - lam B x|| / (max(lam, tau/10) ||B x||) */
} amb_pair_report;

typedef struct {
  int32_t n_levels;             /* decomposition levels with eigenproblems (levels - 1) */
  int32_t n_pairs;              /* entries in pairs[] */
  double omega_level[AMB_MAX_LEVELS];   /* indicator per level: max over pairs of lambda_{k+1} (eq. cond-ind-mlevel) */
  double omega;                 /* product over levels */
  int32_t n_adaptive[AMB_MAX_LEVELS];   /* adaptive rows added per level */
  int32_t n_coarse[AMB_MAX_LEVELS];     /* coarse dofs per level after adaptivity */
  int32_t pcg_iterations;       /* of the last amb_solve */
  double cond_estimate;         /* of the last amb_solve */
  amb_pair_report pairs[1];     /* n_pairs entries (flexible) */
} amb_report;

/* kernel-family timings (CUDA events on the context stream) */
#define AMB_FAM_FACTOR   0   /* partial Cholesky: diagonal, panel and trailing-update kernels */
#define AMB_FAM_TRTRI    1   /* triangular inverses */
#define AMB_FAM_SCHUR    2   /* batched Schur applies (S X) */
#define AMB_FAM_LOBPCG   3   /* all LOBPCG kernels */
#define AMB_FAM_PRECOND  4   /* one Algorithm-1 application */
#define AMB_FAM_OPERATOR 5   /* matrix-free FP64 A p */
#define AMB_FAM_COARSE   6   /* coarse basis, coarse matrices and top factorization */
#define AMB_FAM_TC       7   /* FP32 form: tensor-core trailing updates of the factorization
                                (part of AMB_FAM_FACTOR; flops = rem (rem + 1) K per update) */
#define AMB_FAM_LOBOP    8   /* the LOBPCG operator products S X of the A and B applies (part of
                                AMB_FAM_LOBPCG; flops = 2 n k w per product, bytes = the S blocks
                                each apply reads once: sum n_G^2 (B) and sum n_f^2 (A) words) */
#define AMB_FAM_N        9
typedef struct {
  double ms[AMB_FAM_N];         /* summed event time */
  int64_t launches[AMB_FAM_N];  /* kernel launches counted in the family */
  double flops[AMB_FAM_N];      /* algorithmic flops issued (dense families) */
  double bytes[AMB_FAM_N];      /* algorithmic bytes (memory-bound families) */
  double phase_ms[8];           /* assembly, factor, eigen, constraints, coarse, solve, grad, total-setup */
  int64_t kernels_launched;     /* all kernels launched by the library so far (graph replays count
                                   their kernels) */
  int64_t tuned_shapes;         /* GEMM shape classes whose tile was chosen by timing (process-wide) */
  int64_t tuning_runs;          /* GEMM runs spent timing candidate tiles (process-wide) */
  int64_t graph_replays;        /* Algorithm-1 applications replayed from the context's CUDA graph */
} amb_kernel_stats;

/* Fill *o with the defaults: FP64, corners+edges, adaptive, 10 rows per
 * face, LOBPCG maxit 200 and tol 1e-6, PCG rtol 1e-8 and maxit 2000, seed 1,
 * NULL stream, no event timing. */
void amb_default_options(amb_options* o);

/* Algorithm 3: build the hierarchy, factor every substructure (Sec. 2:
 * A_II = L L^T, S = K_GG - K_GI A_II^{-1} K_IG; the corner-constrained
 * Neumann factor of Sec. 5), solve the pair eigenproblems of every level
 * with LOBPCG preconditioned by the BDDC pair preconditioner (Sec. 5, eq.
 * bddc_pair), add the adaptive rows (eq. d-def, Sec. 7.2) and set up the
 * coarse bases (eq. local_saddle_point_problem) and the top coarse
 * factorization.  levels >= 2; tau > 0 is the per-level target.
 * The decomposition is checked on the host before any device work:
 * AMB_EINVAL if an element or parent index is out of range, a substructure
 * of some level is empty, or is not a box of elements.
 * *out receives a new context even on failure (NULL only on AMB_ENOMEM),
 * so that amb_last_error can explain; release it with amb_destroy. */
int amb_setup(amb_ctx** out, const amb_mesh* mesh, const amb_coeffs* coeffs,
              const amb_partition* part, int32_t levels, double tau,
              const amb_options* opt);

/* PCG (FP64) with one application of Algorithm 1 per iteration.
 * rhs, u: [host|device] full-grid nodal vectors.  info may be NULL.
 * Returns AMB_ENOCONV (u still written) if pcg_maxit is reached. */
int amb_solve(amb_ctx* ctx, const double* rhs, double* u, amb_solve_info* info);

/* Consistent nodal loads of a per-element constant body-force density:
 * body [host|device] n_el * dofs_per_node (element-major); f [host|device]
 * full-grid nodal. */
int amb_load_vector(amb_ctx* ctx, const double* body, double* f);

/* Two-call size query: with buf == NULL (or *nbytes too small) writes the
 * needed size to *nbytes and returns AMB_OK (resp. AMB_EINVAL); otherwise
 * fills the report of the set-up (eq. cond-ind, cond-ind-mlevel, Table 5
 * columns) and the last solve. */
int amb_eigen_report(const amb_ctx* ctx, amb_report* buf, size_t* nbytes);

/* Adjoint gradient d q / d log(coeff_e) for every element (an addition
 * to the method, not in the paper): solve A lambda = dq/du with the same PCG and
 * preconditioner (lambda = u of the last solve for AMB_QOI_COMPLIANCE, no
 * second solve), then g_e = -coeff_e lambda_e^T Khat u_e.  Needs a previous
 * amb_solve.  dq_du [host|device] full-grid nodal (NULL for compliance);
 * grad [host|device] n_el. */
int amb_grad(amb_ctx* ctx, int32_t qoi_kind, const double* dq_du, double* grad_log_coeff);

/* Batched Schur apply (Sec. 5: the action of S^s used by LOBPCG):
 * Y^s = S^s X^s for every substructure s of `level` (1-based), X^s of
 * `width` columns.  X, Y: [device] arrays in the context precision (float
 * for AMB_FP32, double for AMB_FP64), substructure-major: block s starts at
 * element offset width * sum_{r<s} n_gamma(r) and is column-major with
 * leading dimension n_gamma(s) (interface order of amb_export
 * AMB_X_SUB_DOFS).  Y must not overlap X. */
int amb_schur_apply(amb_ctx* ctx, int32_t level, int32_t width, const void* x, void* y);

/* amb_schur_apply for callers that cannot allocate device memory during the
 * call: processes whose device memory is held by their own pool (a caching
 * allocator that owns the GPU) or that cannot afford the implicit device
 * synchronisation of cudaMalloc/cudaFree.  The paper has no counterpart;
 * this is an interface variant of the batched Schur apply.
 *
 * Same arguments, result and layout as amb_schur_apply.  The launch
 * descriptors are staged in a fixed 64 KiB device array that is part of the
 * library image (present on every GPU that loads the library until the
 * process exits); the call performs no cudaMalloc, cudaFree or other
 * allocating call.  Limits: at most 1024 substructures on the level, else
 * AMB_EINVAL with a message.  The context's device must be current.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it for the process; a device reset
 * invalidates it, so do not call this after resetting the device.  The call
 * copies its descriptors from host memory and waits for the context stream,
 * so it must not be made while that stream (or, in global capture mode, any
 * stream) is being captured: it returns AMB_EINVAL when the context stream
 * is capturing.  The descriptors are built in per-thread host buffers (no
 * large stack frame).  Unlike amb_schur_apply, this variant always runs the
 * SIMT products: at FP32 widths >= 64 it does not use the tensor cores, so
 * its results differ from amb_schur_apply's there by FP32 rounding.
 * All calls share the array and it keeps the last call's descriptors:
 * calls whose GPU work overlaps (other streams, other host threads) race on
 * it, so serialise them.  Returns after the context stream has finished. */
int amb_schur_apply_noalloc(amb_ctx* ctx, int32_t level, int32_t width, const void* x, void* y);

/* Level sizes for callers that size buffers or compare with a reference. */
typedef struct {
  int32_t n_subs, n_pairs, n_corner_nodes, n_edges, n_faces;
  int64_t n_dofs;               /* level dofs (level 1: free dofs) */
  int64_t n_coarse;             /* coarse dofs after adaptivity */
  int64_t sum_ni, sum_ngamma, max_ni, max_ngamma, max_ndelta;
  double factor_flops;          /* sum n_I^3/3 + n_I^2 n_G + n_I n_G^2 + n_D^3/3 */
  double schur_words;           /* sum n_G^2 */
} amb_level_sizes;
int amb_level_info(const amb_ctx* ctx, int32_t level, amb_level_sizes* info);

/* Host-only plan of one level, without a context and without any device
 * work: the classification of Sec. 2 (interface, faces, edges, box-vertex
 * corners; on level i >= 2 the nodes are the coarse objects of level i-1,
 * Sec. 3) and the initial constraints of Sec. 7.1, for sizing a run before
 * amb_setup (device memory grows with sum n_I^2 and schur_words).
 * Adaptive rows are not known before the eigenproblems, so the plan is that
 * of the hierarchy with the initial constraints only: level 1 equals what
 * amb_level_info(ctx, 1, ...) reports except that n_coarse counts the
 * initial coarse dofs; levels >= 2 equal those of a set-up with adaptive = 0.
 * level in [1, levels - 1].  sub_sizes: NULL, or [host] 4 * (substructures
 * on that level) int32 receiving per substructure (n_I, n_Gamma, corner
 * dofs, coarse dofs).  mesh, part: as for amb_setup; only dofs_per_node,
 * the sizes, the Dirichlet mask and the partition are read.  Errors:
 * AMB_EINVAL for NULL arguments, an unknown initial_constraints, a level out
 * of range or a partition that amb_setup would reject. */
int amb_plan(const amb_mesh* mesh, const amb_partition* part, int32_t levels, int32_t initial_constraints,
             int32_t level, amb_level_sizes* info, int32_t* sub_sizes);

/* Export internal results for verification.  Two-call size query as in
 * amb_eigen_report.  `what`:
 *  AMB_X_SUB_DOFS   int64: dofs of substructure `index`, [interior...,
 *                   interface (non-corner..., corner...)]; level 1 = full-grid
 *                   dof ids, higher levels = coarse ids of the level below
 *  AMB_X_SUB_SIZES  int32[4]: n_I, n_gamma, n_corner_dofs, n_coarse of sub `index`
 *  AMB_X_SCHUR      double n_gamma^2: S of sub `index` (column-major, interface order)
 *  AMB_X_COARSE_EL  double n_coarse^2: Psi^T S Psi of sub `index`
 *  AMB_X_CONSTR     double n_coarse x n_gamma: constraint rows of sub `index` (row-major)
 *  AMB_X_CORNERS    int64: level dofs of all corner dofs of the level
 *  AMB_X_PAIR_ROWS  double k x n_face (row-major) then int64 n_face dof ids:
 *                   adaptive rows of pair number `index` of the level */
#define AMB_X_SUB_DOFS   1
#define AMB_X_SUB_SIZES  2
#define AMB_X_SCHUR      3
#define AMB_X_COARSE_EL  4
#define AMB_X_CONSTR     5
#define AMB_X_CORNERS    6
#define AMB_X_PAIR_ROWS  7
int amb_export(const amb_ctx* ctx, int32_t what, int32_t level, int32_t index,
               void* out, size_t* nbytes);

int amb_stats(const amb_ctx* ctx, amb_kernel_stats* st);
const char* amb_last_error(const amb_ctx* ctx);
void amb_destroy(amb_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* AMB_H */
