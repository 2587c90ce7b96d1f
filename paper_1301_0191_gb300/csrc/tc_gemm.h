// Tensor-core (tcgen05) kernels (tc_gemm.cu): 3xTF32 products of the FP32 form
// and exact slice products of the FP64 form.
#pragma once

#include <vector>

#include "common.h"

namespace amb {

constexpr int kTcKMax = 256;   // widest K of one trailing update (the outer Cholesky block)
constexpr int kTcSchurWidth = 64;  // FP32 Schur applies of at least this many columns use the tensor cores

// One trailing update C(lower) -= P P^T of a substructure matrix: P is rem x
// k at element offset p (column-major, ld), C is rem x rem at offset c.
struct TcSyrk {
  int64_t p, c;
  int32_t ld, rem, k, pad;
};

// One product C = beta C + alpha A B^T (C m x n column-major, ldc).  A(i, k)
// sits at a + i + k*lda (column form) or a + k + i*lda (K-major form), B(j, k)
// likewise.  a_tri: 0 dense, 1 lower (A(i, k) = 0 for k > i), 2 upper
// (A(i, k) = 0 for k < i); the entries outside the triangle are not read.
struct TcGemm {
  int64_t a, b, c;
  int32_t lda, ldb, ldc, m, n, k;
  int32_t a_kmajor, b_kmajor, a_tri;
};

// split pass: a rows x cols source block -> slab rows [row0, row0 + rpad),
// entries outside it (and outside the triangle) zero; src points to FP32 data
// (FP32 form) or FP64 data (FP64 form)
struct TcSplitDesc {
  const float* src;
  int64_t row0;
  int32_t ld, rows, cols, rpad;
  int32_t kmajor, tri, diag, pad;             // tri as in TcGemm; diag = global row - global k at (0, 0)
};

// one tile job list entry: C rows at c (element offset) from A slab rows arow,
// B slab rows brow; lower: only the lower triangle of a square C.  tri/ioff
// narrow each row tile's K range (ioff = global row of row 0 - global k of
// slab column 0); first: beta applies (else the chunk accumulates onto C).
struct TcDesc {
  int64_t c, arow, brow;
  int32_t m, n, k, ldc, lower, tri, ioff, first;
};

struct TcTileArgs {
  const TcDesc* desc;
  const int* prefix;
  int ndesc, kp;
  float alpha, beta;
  const float *ah, *al, *bh, *bl;
  float* c;
  int* status;
};

int tc_tile_count(const TcDesc& x);

// C(lower) = beta C + alpha P P^T for every entry of d (FP32 data in base).
void tc_syrk_lower(cudaStream_t st, DescRing& ring, const std::vector<TcSyrk>& d, float alpha, float beta,
                   float* base, int* status);

// C = beta C + alpha A B^T for every entry of d (A from abase, B from bbase,
// C in cbase), K in chunks of kTcKMax accumulated in FP32 through C.
void tc_gemm(cudaStream_t st, DescRing& ring, const std::vector<TcGemm>& d, float alpha, float beta,
             const float* abase, const float* bbase, float* cbase, int* status);

// FP64 form: C(lower) = beta C + alpha P P^T for every entry of d (FP64 data in
// base) on the tensor cores, with FP64 accuracy from exact slice products:
// every row of P is scaled by a power of two to |P(r, :)| < 1 and cut into
// kOzSlices integer slices of 7 bits (exact in TF32); the products of slices
// p and q with p + q < kOzSlices are summed per level p + q in FP32 TMEM
// accumulators, where every partial sum is an integer below 2^24 and hence
// exact; the levels are combined exactly in 64-bit integers, rounded to FP64
// once and added to C with one FP64 multiply-add.
constexpr int kOzSlices = 8;
void tc_syrk_lower_f64(cudaStream_t st, DescRing& ring, const std::vector<TcSyrk>& d, double alpha, double beta,
                       double* base, int* status);

// FP64 form: C = beta C + alpha A B^T for every entry of d, as tc_gemm, with
// the exact slice products of tc_syrk_lower_f64 per K chunk of kTcKMax
// (each chunk rounded to FP64 once and added to C in FP64).  akey
// (optional, one per entry): entries with the same key >= 0 share one dense
// A, split once per chunk.
void tc_gemm_f64(cudaStream_t st, DescRing& ring, const std::vector<TcGemm>& d, double alpha, double beta,
                 const double* abase, const double* bbase, double* cbase, int* status,
                 const std::vector<int>* akey = nullptr);

}  // namespace amb
