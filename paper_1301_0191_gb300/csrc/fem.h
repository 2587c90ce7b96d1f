// Finite-element kernels (fem.cu).
#pragma once

#include <vector>

#include "common.h"

namespace amb {

void compute_khat(cudaStream_t st, double* khat, int dpn, double h, double nu);

// Deterministic assembly (no atomics): 8 colour passes over the elements.
template <typename T>
void assemble_level1(cudaStream_t st, T* M, const int64_t* sub_off, const int32_t* sub_n, const int32_t* elem_sub,
                     const int32_t* elem_local, const double* coeff, const double* khat, int nd, int nx, int ny,
                     int nz);

// One pass per sibling rank: child[pass_beg[r] .. pass_beg[r+1]) are the
// children of rank r; ent_off (device) / ent_h (host) the running entry
// offsets of their coarse matrices over the whole child list.
template <typename T>
void assemble_next(cudaStream_t st, T* M, const int64_t* par_off, const int32_t* par_n, const int32_t* parent,
                   const int64_t* ac_off, const int32_t* nc, const int64_t* loc_off, const int32_t* loc,
                   const double* ac, const int32_t* child, const int64_t* ent_off, const std::vector<int>& pass_beg,
                   const std::vector<int64_t>& ent_h);

void matvec(cudaStream_t st, double* y, const double* x, const double* coeff, const double* khat, const uint8_t* dir,
            int nx, int ny, int nz, int dpn);

void load_vector(cudaStream_t st, double* f, const double* body, const uint8_t* dir, int nx, int ny, int nz, int dpn,
                 double h);

void mask_dirichlet(cudaStream_t st, double* v, const uint8_t* dir, int64_t nnodes, int dpn);

void element_gradient(cudaStream_t st, double* g, const double* u, const double* lam, const double* coeff,
                      const double* khat, const uint8_t* dir, int nx, int ny, int nz, int dpn);

}  // namespace amb
