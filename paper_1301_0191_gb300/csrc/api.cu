// C ABI of the substructure engine (include/amb.h): context management,
// PCG (Sec. 8: CG preconditioned by one application of Algorithm 1, with
// the Lanczos condition estimate), the adjoint gradient and exports.
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "ctx.h"
#include "fem.h"
#include "kernels.h"

using namespace amb;

namespace {

void copy_in(DevBuf& dst, const void* src, size_t bytes, cudaStream_t st) {
  if (dst.bytes < bytes) dst.alloc(bytes);
  AMB_CUDA(cudaMemcpyAsync(dst.p, src, bytes, is_device(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
}

void copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  AMB_CUDA(cudaMemcpyAsync(dst, src, bytes, is_device(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  AMB_CUDA(cudaStreamSynchronize(st));
}

double dotd(amb_ctx* c, const double* a, const double* b, int64_t n) {
  dot(c->st, dptr<double>(c->dscal), a, b, n, dptr<double>(c->partial));
  double h = 0;
  AMB_CUDA(cudaMemcpyAsync(&h, c->dscal.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  AMB_CUDA(cudaStreamSynchronize(c->st));
  return h;
}

// PCG on full-grid nodal vectors: solves A x = b (b in c->f), x in c->u.
int pcg(amb_ctx* c, double* info_rel, double* info_cond) {
  const Mesh& m = c->mesh;
  const int64_t n = m.ndof;
  cudaStream_t st = c->st;
  const bool flexible = c->opt.precision == AMB_FP32;
  double* f = dptr<double>(c->f);
  double* u = dptr<double>(c->u);
  double* r = dptr<double>(c->r);
  double* z = dptr<double>(c->z);
  double* p = dptr<double>(c->p);
  double* q = dptr<double>(c->q);
  double* ro = dptr<double>(c->rold);
  mask_dirichlet(st, f, dptr<uint8_t>(m.dir), m.nnodes, m.dpn);
  AMB_CUDA(cudaMemsetAsync(u, 0, n * sizeof(double), st));
  AMB_CUDA(cudaMemcpyAsync(r, f, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const double nf = std::sqrt(dotd(c, f, f, n));
  AMB_CHECK(std::isfinite(nf), AMB_EINVAL, "right-hand side contains non-finite values");
  std::vector<double> alphas, betas;
  int its = 0;
  double rel = 0.0;
  if (nf > 0) {
    {
      FamTimer ft(st, &c->tm, AMB_FAM_PRECOND, c->opt.timing_events != 0);
      c->eng->precond(r, z);
    }
    double rz = dotd(c, r, z, n);
    AMB_CUDA(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    rel = 1.0;
    while (its < c->opt.pcg_maxit) {
      {
        FamTimer ft(st, &c->tm, AMB_FAM_OPERATOR, c->opt.timing_events != 0);
        matvec(st, q, p, dptr<double>(m.coeff), dptr<double>(m.khat), dptr<uint8_t>(m.dir), m.nx, m.ny, m.nz, m.dpn);
      }
      const double pq = dotd(c, p, q, n);
      AMB_CHECK(pq > 0.0 && std::isfinite(pq), AMB_EINVAL, "PCG breakdown: p^T A p <= 0 (operator not SPD?)");
      const double alpha = rz / pq;
      if (flexible) AMB_CUDA(cudaMemcpyAsync(ro, r, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      axpy2(st, u, r, p, q, alpha, n);
      ++its;
      alphas.push_back(alpha);
      rel = std::sqrt(dotd(c, r, r, n)) / nf;
      if (!std::isfinite(rel)) throw Error(AMB_EINVAL, "PCG produced a non-finite residual");
      if (rel <= c->opt.pcg_rtol) break;
      {
        FamTimer ft(st, &c->tm, AMB_FAM_PRECOND, c->opt.timing_events != 0);
        c->eng->precond(r, z);
      }
      const double rz_new = dotd(c, r, z, n);
      double beta = rz_new / rz;
      if (flexible) beta = (rz_new - dotd(c, ro, z, n)) / rz;   // Polak-Ribiere: tolerates a slightly variable preconditioner
      betas.push_back(beta);
      xpby(st, p, z, beta, n);
      rz = rz_new;
    }
  }
  double cond = 1.0;
  if (!alphas.empty()) {
    std::vector<double> ab(alphas);
    ab.insert(ab.end(), betas.begin(), betas.end());
    ab.push_back(0.0);
    c->ab.alloc(ab.size() * sizeof(double));
    AMB_CUDA(cudaMemcpyAsync(c->ab.p, ab.data(), ab.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    tridiag_extremes(st, dptr<double>(c->dscal), dptr<double>(c->ab), dptr<double>(c->ab) + alphas.size(),
                     (int)alphas.size());
    double ex[2];
    AMB_CUDA(cudaMemcpyAsync(ex, c->dscal.p, sizeof(ex), cudaMemcpyDeviceToHost, st));
    AMB_CUDA(cudaStreamSynchronize(st));
    cond = ex[0] > 0 ? ex[1] / ex[0] : INFINITY;
  }
  *info_rel = rel;
  *info_cond = cond;
  return its;
}

void alloc_vectors(amb_ctx* c) {
  const size_t b = c->mesh.ndof * sizeof(double);
  for (DevBuf* v : {&c->f, &c->u, &c->r, &c->z, &c->p, &c->q, &c->rold, &c->tmp, &c->lam})
    if (v->bytes < b) v->alloc(b);
  if (c->partial.bytes < 1024 * sizeof(double)) c->partial.alloc(1024 * sizeof(double));
  if (c->dscal.bytes < 4 * sizeof(double)) c->dscal.alloc(4 * sizeof(double));
}

}  // namespace

extern "C" {

void amb_default_options(amb_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = AMB_FP64;
  o->initial_constraints = AMB_CORNERS_EDGES;
  o->adaptive = 1;
  o->max_adaptive_per_face = 10;
  o->lobpcg_maxit = 200;
  o->lobpcg_tol = 1e-6;
  o->pcg_rtol = 1e-8;
  o->pcg_maxit = 2000;
  o->seed = 1;
  o->cuda_stream = nullptr;
  o->timing_events = 0;
}

int amb_setup(amb_ctx** out, const amb_mesh* mesh, const amb_coeffs* coeffs, const amb_partition* part,
              int32_t levels, double tau, const amb_options* opt) {
  if (!out) return AMB_EINVAL;
  amb_ctx* c = new (std::nothrow) amb_ctx();
  *out = c;
  if (!c) return AMB_ENOMEM;
  return guarded(c, [&]() {
    AMB_CHECK(mesh && coeffs && part && opt, AMB_EINVAL, "NULL argument");
    AMB_CHECK(mesh->nx >= 1 && mesh->ny >= 1 && mesh->nz >= 1 && mesh->h > 0, AMB_EINVAL, "invalid mesh size");
    AMB_CHECK(mesh->dofs_per_node == 1 || mesh->dofs_per_node == 3, AMB_EINVAL, "dofs_per_node must be 1 or 3");
    AMB_CHECK(levels >= 2 && levels <= AMB_MAX_LEVELS, AMB_EINVAL, "levels must be in [2, 8]");
    AMB_CHECK(tau > 0, AMB_EINVAL, "tau must be positive");
    AMB_CHECK(opt->precision == AMB_FP64 || opt->precision == AMB_FP32, AMB_EINVAL, "unknown precision");
    AMB_CHECK(opt->initial_constraints == AMB_CORNERS || opt->initial_constraints == AMB_CORNERS_EDGES ||
                  opt->initial_constraints == AMB_CORNERS_EDGES_FACES,
              AMB_EINVAL, "unknown initial constraints");
    AMB_CHECK(opt->initial_constraints != AMB_CORNERS_EDGES_FACES || opt->adaptive == 0, AMB_EINVAL,
              "face averages are initial constraints of the non-adaptive method (c+e+f); set adaptive = 0");
    AMB_CHECK(opt->max_adaptive_per_face >= 0 && opt->max_adaptive_per_face < AMB_MAX_EIG, AMB_EINVAL,
              "max_adaptive_per_face must be in [0, 15]");
    AMB_CHECK(mesh->dirichlet_node_mask && part->elem_to_sub && coeffs->coeff, AMB_EINVAL, "NULL array");
    AMB_CHECK(mesh->dofs_per_node == 1 || (coeffs->poisson_ratio > -1.0 && coeffs->poisson_ratio < 0.5), AMB_EINVAL,
              "poisson_ratio out of range");
    // the decomposition hierarchy is checked on the host before any device work
    AMB_CHECK(!is_device(mesh->dirichlet_node_mask) && !is_device(part->elem_to_sub), AMB_EINVAL,
              "dirichlet_node_mask and the partition must be host arrays");
    AMB_CHECK(part->n_sub1 >= 1, AMB_EINVAL, "n_sub1 must be >= 1");
    c->cfg.nsubs.push_back(part->n_sub1);
    for (int i = 0; i < levels - 2; ++i) {
      AMB_CHECK(part->sub_to_parent && part->n_sub && part->sub_to_parent[i], AMB_EINVAL,
                "sub_to_parent required for levels > 2");
      AMB_CHECK(!is_device(part->sub_to_parent[i]), AMB_EINVAL, "sub_to_parent must be host arrays");
      const int nprev = c->cfg.nsubs.back();
      c->cfg.parents.emplace_back(part->sub_to_parent[i], part->sub_to_parent[i] + nprev);
      c->cfg.nsubs.push_back(part->n_sub[i]);
    }
    validate_partition(mesh->nx, mesh->ny, mesh->nz, part->elem_to_sub, c->cfg.parents, c->cfg.nsubs);
    c->opt = *opt;
    c->st = static_cast<cudaStream_t>(opt->cuda_stream);
    alloc_stream() = c->st;
    AMB_CUDA(cudaGetDevice(&c->device));
    Mesh& m = c->mesh;
    m.nx = mesh->nx;
    m.ny = mesh->ny;
    m.nz = mesh->nz;
    m.dpn = mesh->dofs_per_node;
    m.h = mesh->h;
    m.nu = coeffs->poisson_ratio;
    m.nel = (int64_t)m.nx * m.ny * m.nz;
    m.nnodes = (int64_t)(m.nx + 1) * (m.ny + 1) * (m.nz + 1);
    m.ndof = m.nnodes * m.dpn;
    m.dir_h.assign(mesh->dirichlet_node_mask, mesh->dirichlet_node_mask + m.nnodes);
    m.elem_sub_h.assign(part->elem_to_sub, part->elem_to_sub + m.nel);
    c->ring.init(64 << 20);
    c->status.alloc(4 * sizeof(int));
    AMB_CUDA(cudaMemsetAsync(c->status.p, 0, 4 * sizeof(int), c->st));
    copy_in(m.coeff, coeffs->coeff, m.nel * sizeof(double), c->st);
    std::vector<double> ch(m.nel);
    AMB_CUDA(cudaMemcpyAsync(ch.data(), m.coeff.p, m.nel * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    AMB_CUDA(cudaStreamSynchronize(c->st));
    for (double v : ch) AMB_CHECK(v > 0.0 && std::isfinite(v), AMB_EINVAL, "coefficients must be positive and finite");
    upload(m.dir, m.dir_h, c->st);
    upload(m.elem_sub, m.elem_sub_h, c->st);
    m.khat.alloc(576 * sizeof(double));
    compute_khat(c->st, dptr<double>(m.khat), m.dpn, m.h, m.nu);
    c->cfg.opt = *opt;
    c->cfg.levels = levels;
    c->cfg.tau = tau;
    alloc_vectors(c);
    EventPair ev;
    ev.start(c->st);
    c->eng = make_engine(opt->precision, m, c->cfg, c->st, c->ring, c->tm, c->reports, c->omega, c->nadapt, c->status);
    c->eng->setup();
    const float ms = ev.lap(c->st);
    c->tm.phase_ms[7] += ms;
    c->setup_ms = ms;
  });
}

int amb_solve(amb_ctx* c, const double* rhs, double* u, amb_solve_info* info) {
  int conv_status = AMB_OK;
  int st = guarded(c, [&]() {
    AMB_CHECK(c->eng, AMB_EINVAL, "context has no successful set-up");
    AMB_CHECK(rhs && u, AMB_EINVAL, "NULL vector");
    const int64_t n = c->mesh.ndof;
    EventPair ev;
    ev.start(c->st);
    copy_in(c->f, rhs, n * sizeof(double), c->st);
    double rel = 0, cond = 1;
    const int its = pcg(c, &rel, &cond);
    // true residual
    matvec(c->st, dptr<double>(c->tmp), dptr<double>(c->u), dptr<double>(c->mesh.coeff), dptr<double>(c->mesh.khat),
           dptr<uint8_t>(c->mesh.dir), c->mesh.nx, c->mesh.ny, c->mesh.nz, c->mesh.dpn);
    sub_vec(c->st, dptr<double>(c->tmp), dptr<double>(c->f), dptr<double>(c->tmp), n);
    // Dirichlet entries of f are not part of the system: zero them in the residual
    const double nf = std::sqrt(dotd(c, dptr<double>(c->f), dptr<double>(c->f), n));
    const double nr = std::sqrt(dotd(c, dptr<double>(c->tmp), dptr<double>(c->tmp), n));
    copy_out(u, c->u.p, n * sizeof(double), c->st);
    const float ms = ev.lap(c->st);
    c->tm.phase_ms[5] += ms;
    c->last_its = its;
    c->last_cond = cond;
    c->last_rel = rel;
    c->have_solution = true;
    if (info) {
      info->iterations = its;
      info->rel_residual = rel;
      info->true_rel_residual = nf > 0 ? nr / nf : 0.0;
      info->cond_estimate = cond;
      info->ms = ms;
    }
    if (!(rel <= c->opt.pcg_rtol)) {
      conv_status = AMB_ENOCONV;
      c->err = "PCG reached pcg_maxit = " + std::to_string(c->opt.pcg_maxit) + " with relative residual " +
               std::to_string(rel);
    }
  });
  if (st == AMB_OK && conv_status != AMB_OK) return conv_status;
  return st;
}

int amb_load_vector(amb_ctx* c, const double* body, double* f) {
  return guarded(c, [&]() {
    AMB_CHECK(body && f, AMB_EINVAL, "NULL vector");
    const Mesh& m = c->mesh;
    copy_in(c->body, body, m.nel * m.dpn * sizeof(double), c->st);
    load_vector(c->st, dptr<double>(c->tmp), dptr<double>(c->body), dptr<uint8_t>(m.dir), m.nx, m.ny, m.nz, m.dpn, m.h);
    copy_out(f, c->tmp.p, m.ndof * sizeof(double), c->st);
  });
}

int amb_eigen_report(const amb_ctx* cc, amb_report* buf, size_t* nbytes) {
  amb_ctx* c = const_cast<amb_ctx*>(cc);
  if (!c || !nbytes) return AMB_EINVAL;
  const size_t np = c->reports.size();
  const size_t need = offsetof(amb_report, pairs) + std::max<size_t>(np, 1) * sizeof(amb_pair_report);
  if (!buf) {
    *nbytes = need;
    return AMB_OK;
  }
  if (*nbytes < need) {
    *nbytes = need;
    c->err = "eigen report buffer too small";
    return AMB_EINVAL;
  }
  memset(buf, 0, need);
  buf->n_levels = (int32_t)c->omega.size();
  buf->n_pairs = (int32_t)np;
  double om = 1.0;
  for (size_t i = 0; i < c->omega.size() && i < AMB_MAX_LEVELS; ++i) {
    buf->omega_level[i] = c->omega[i];
    buf->n_adaptive[i] = c->nadapt[i];
    om *= c->omega[i];
    if (c->eng && (int)i < c->eng->n_levels()) buf->n_coarse[i] = (int32_t)c->eng->topo((int)i + 1).n_coarse;
  }
  buf->omega = c->omega.empty() ? 0.0 : om;
  buf->pcg_iterations = c->last_its;
  buf->cond_estimate = c->last_cond;
  for (size_t k = 0; k < np; ++k) {
    const PairReportH& r = c->reports[k];
    amb_pair_report& o = buf->pairs[k];
    o.level = r.level;
    o.s = r.s;
    o.t = r.t;
    o.n_computed = r.n_computed;
    o.n_selected = r.n_selected;
    o.n_rows = r.n_rows;
    o.converged = r.converged;
    o.iterations = r.iterations;
    o.residual = r.residual;
    for (size_t j = 0; j < r.lambda.size() && j < AMB_MAX_EIG; ++j) o.lambda[j] = r.lambda[j];
  }
  *nbytes = need;
  return AMB_OK;
}

int amb_grad(amb_ctx* c, int32_t qoi_kind, const double* dq_du, double* grad) {
  return guarded(c, [&]() {
    AMB_CHECK(c->eng, AMB_EINVAL, "context has no successful set-up");
    AMB_CHECK(c->have_solution, AMB_EINVAL, "amb_grad needs a previous amb_solve");
    AMB_CHECK(grad, AMB_EINVAL, "NULL gradient buffer");
    const Mesh& m = c->mesh;
    const int64_t n = m.ndof;
    EventPair ev;
    ev.start(c->st);
    // keep the primal solution: lam buffer receives u, adjoint overwrites u/f
    AMB_CUDA(cudaMemcpyAsync(c->lam.p, c->u.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    const double* lam = dptr<double>(c->lam);
    if (qoi_kind == AMB_QOI_GENERAL) {
      AMB_CHECK(dq_du, AMB_EINVAL, "dq_du required for AMB_QOI_GENERAL");
      DevBuf keep;
      keep.alloc(n * sizeof(double));
      AMB_CUDA(cudaMemcpyAsync(keep.p, c->u.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      copy_in(c->f, dq_du, n * sizeof(double), c->st);
      double rel, cond;
      pcg(c, &rel, &cond);
      AMB_CHECK(rel <= c->opt.pcg_rtol, AMB_ENOCONV, "adjoint PCG did not converge");
      // lam := adjoint solution, u := primal again
      AMB_CUDA(cudaMemcpyAsync(c->lam.p, c->u.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      AMB_CUDA(cudaMemcpyAsync(c->u.p, keep.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      AMB_CUDA(cudaStreamSynchronize(c->st));
    } else {
      AMB_CHECK(qoi_kind == AMB_QOI_COMPLIANCE, AMB_EINVAL, "unknown qoi_kind");
    }
    if (c->grad.bytes < m.nel * sizeof(double)) c->grad.alloc(m.nel * sizeof(double));
    element_gradient(c->st, dptr<double>(c->grad), dptr<double>(c->u), lam, dptr<double>(m.coeff), dptr<double>(m.khat),
                     dptr<uint8_t>(m.dir), m.nx, m.ny, m.nz, m.dpn);
    copy_out(grad, c->grad.p, m.nel * sizeof(double), c->st);
    c->tm.phase_ms[6] += ev.lap(c->st);
  });
}

int amb_schur_apply(amb_ctx* c, int32_t level, int32_t width, const void* x, void* y) {
  return guarded(c, [&]() {
    AMB_CHECK(c->eng, AMB_EINVAL, "context has no successful set-up");
    AMB_CHECK(is_device(x) && is_device(y), AMB_EINVAL, "x and y must be device arrays");
    c->eng->schur_apply(level, width, x, y);
    AMB_CUDA(cudaStreamSynchronize(c->st));
  });
}

namespace {
// sizes of one level; n_dofs is passed in (level 1: free dofs of the mesh)
void fill_sizes(const amb::LevelTopo& tp, int64_t n_dofs, amb_level_sizes* info) {
  memset(info, 0, sizeof(*info));
  info->n_subs = tp.n_subs;
  info->n_pairs = (int32_t)tp.pairs.size();
  info->n_corner_nodes = tp.n_corner_nodes;
  info->n_edges = tp.n_edges;
  info->n_faces = tp.n_faces;
  info->n_dofs = n_dofs;
  info->n_coarse = tp.n_coarse;
  for (const auto& sb : tp.subs) {
    const double ni = sb.n_i, ng = sb.n_g, ndl = sb.n_d();
    info->sum_ni += sb.n_i;
    info->sum_ngamma += sb.n_g;
    info->max_ni = std::max<int64_t>(info->max_ni, sb.n_i);
    info->max_ngamma = std::max<int64_t>(info->max_ngamma, sb.n_g);
    info->max_ndelta = std::max<int64_t>(info->max_ndelta, sb.n_d());
    info->factor_flops += ni * ni * ni / 3.0 + ni * ni * ng + ni * ng * ng + ndl * ndl * ndl / 3.0;
    info->schur_words += ng * ng;
  }
}

int64_t free_dofs(const uint8_t* dir, int64_t nnodes, int dpn) {
  int64_t nd = 0;
  for (int64_t i = 0; i < nnodes; ++i) nd += dir[i] ? 0 : 1;
  return nd * dpn;
}
}  // namespace

int amb_level_info(const amb_ctx* cc, int32_t level, amb_level_sizes* info) {
  amb_ctx* c = const_cast<amb_ctx*>(cc);
  return guarded(c, [&]() {
    AMB_CHECK(c->eng && info, AMB_EINVAL, "no set-up or NULL info");
    AMB_CHECK(level >= 1 && level <= c->eng->n_levels(), AMB_EINVAL, "level out of range");
    const LevelTopo& tp = c->eng->topo(level);
    const int64_t nd = level == 1 ? free_dofs(c->mesh.dir_h.data(), (int64_t)c->mesh.dir_h.size(), c->mesh.dpn)
                                  : tp.n_dofs;
    fill_sizes(tp, nd, info);
  });
}

int amb_plan(const amb_mesh* mesh, const amb_partition* part, int32_t levels, int32_t initial_constraints,
             int32_t level, amb_level_sizes* info, int32_t* sub_sizes) {
  try {
    AMB_CHECK(mesh && part && info, AMB_EINVAL, "NULL argument");
    AMB_CHECK(mesh->nx >= 1 && mesh->ny >= 1 && mesh->nz >= 1, AMB_EINVAL, "invalid mesh size");
    AMB_CHECK(mesh->dofs_per_node == 1 || mesh->dofs_per_node == 3, AMB_EINVAL, "dofs_per_node must be 1 or 3");
    AMB_CHECK(levels >= 2 && levels <= AMB_MAX_LEVELS, AMB_EINVAL, "levels must be in [2, 8]");
    AMB_CHECK(level >= 1 && level <= levels - 1, AMB_EINVAL, "level out of range");
    AMB_CHECK(initial_constraints == AMB_CORNERS || initial_constraints == AMB_CORNERS_EDGES ||
                  initial_constraints == AMB_CORNERS_EDGES_FACES,
              AMB_EINVAL, "unknown initial constraints");
    AMB_CHECK(mesh->dirichlet_node_mask && part->elem_to_sub, AMB_EINVAL, "NULL array");
    AMB_CHECK(part->n_sub1 >= 1, AMB_EINVAL, "n_sub1 must be >= 1");
    std::vector<int> nsubs{part->n_sub1};
    std::vector<std::vector<int32_t>> parents;
    for (int i = 0; i < levels - 2; ++i) {
      AMB_CHECK(part->sub_to_parent && part->n_sub && part->sub_to_parent[i], AMB_EINVAL,
                "sub_to_parent required for levels > 2");
      parents.emplace_back(part->sub_to_parent[i], part->sub_to_parent[i] + nsubs.back());
      nsubs.push_back(part->n_sub[i]);
    }
    validate_partition(mesh->nx, mesh->ny, mesh->nz, part->elem_to_sub, parents, nsubs);
    std::vector<int32_t> loc;
    LevelTopo tp = build_level_one(mesh->nx, mesh->ny, mesh->nz, mesh->dofs_per_node, mesh->dirichlet_node_mask,
                                   part->elem_to_sub, part->n_sub1, initial_constraints, loc);
    for (int l = 2; l <= level; ++l) {
      LevelTopo next = build_level_next(tp, parents[l - 2].data(), nsubs[l - 1], initial_constraints, loc);
      tp = std::move(next);
    }
    const int64_t nnodes = (int64_t)(mesh->nx + 1) * (mesh->ny + 1) * (mesh->nz + 1);
    fill_sizes(tp, level == 1 ? free_dofs(mesh->dirichlet_node_mask, nnodes, mesh->dofs_per_node) : tp.n_dofs, info);
    if (sub_sizes)
      for (int s = 0; s < tp.n_subs; ++s) {
        const SubTopo& sb = tp.subs[s];
        sub_sizes[4 * s + 0] = sb.n_i;
        sub_sizes[4 * s + 1] = sb.n_g;
        sub_sizes[4 * s + 2] = sb.n_crn;
        sub_sizes[4 * s + 3] = sb.n_c();
      }
    return AMB_OK;
  } catch (const Error& e) {
    return e.status;
  } catch (const std::bad_alloc&) {
    return AMB_ENOMEM;
  } catch (...) {
    return AMB_EINVAL;
  }
}

int amb_export(const amb_ctx* cc, int32_t what, int32_t level, int32_t index, void* out, size_t* nbytes) {
  amb_ctx* c = const_cast<amb_ctx*>(cc);
  return guarded(c, [&]() {
    AMB_CHECK(c->eng && nbytes, AMB_EINVAL, "no set-up or NULL size");
    std::vector<char> data;
    c->eng->export_sub(what, level, index, data);
    if (!out) {
      *nbytes = data.size();
      return;
    }
    if (*nbytes < data.size()) {
      *nbytes = data.size();
      throw Error(AMB_EINVAL, "export buffer too small");
    }
    memcpy(out, data.data(), data.size());
    *nbytes = data.size();
  });
}

int amb_stats(const amb_ctx* cc, amb_kernel_stats* st) {
  amb_ctx* c = const_cast<amb_ctx*>(cc);
  if (!c || !st) return AMB_EINVAL;
  memset(st, 0, sizeof(*st));
  for (int i = 0; i < AMB_FAM_N; ++i) {
    st->ms[i] = c->tm.fam_ms[i];
    st->launches[i] = c->tm.fam_launches[i];
    st->flops[i] = c->tm.fam_flops[i];
    st->bytes[i] = c->tm.fam_bytes[i];
  }
  for (int i = 0; i < 8; ++i) st->phase_ms[i] = c->tm.phase_ms[i];
  st->kernels_launched = c->launches_total;
  st->tuned_shapes = (int64_t)gemm_tune_entries();
  st->tuning_runs = gemm_tune_runs();
  st->graph_replays = c->eng ? c->eng->graph_replays() : 0;
  return AMB_OK;
}

const char* amb_last_error(const amb_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

void amb_destroy(amb_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  alloc_stream() = c->st;
  delete c;
}

}  // extern "C"
