// Finite-element kernels (fem.cu).
#pragma once

#include "common.h"

namespace amb {

void compute_khat(cudaStream_t st, double* khat, int dpn, double h, double nu);

template <typename T>
void assemble_level1(cudaStream_t st, T* M, const int64_t* sub_off, const int32_t* sub_n, const int32_t* elem_sub,
                     const int32_t* elem_local, const double* coeff, const double* khat, int nd, int64_t nel);

template <typename T>
void assemble_next(cudaStream_t st, T* M, const int64_t* par_off, const int32_t* par_n, const int32_t* parent,
                   const int64_t* ac_off, const int32_t* nc, const int64_t* loc_off, const int32_t* loc,
                   const double* ac, const int64_t* ent_off, int nchild, int64_t total);

void matvec(cudaStream_t st, double* y, const double* x, const double* coeff, const double* khat, const uint8_t* dir,
            int nx, int ny, int nz, int dpn);

void load_vector(cudaStream_t st, double* f, const double* body, const uint8_t* dir, int nx, int ny, int nz, int dpn,
                 double h);

void mask_dirichlet(cudaStream_t st, double* v, const uint8_t* dir, int64_t nnodes, int dpn);

void element_gradient(cudaStream_t st, double* g, const double* u, const double* lam, const double* coeff,
                      const double* khat, const uint8_t* dir, int nx, int ny, int nz, int dpn);

}  // namespace amb
