// Tensor-core (tcgen05, 3xTF32) kernels of the FP32 form (tc_gemm.cu).
#pragma once

#include <vector>

#include "common.h"

namespace amb {

constexpr int kTcKMax = 256;   // widest K of one trailing update (the outer Cholesky block)

// One trailing update C(lower) -= P P^T of a substructure matrix: P is rem x
// k at element offset p (column-major, ld), C is rem x rem at offset c.
struct TcSyrk {
  int64_t p, c;
  int32_t ld, rem, k, pad;
};

// split pass: source block (column-major) -> slab rows [row0, row0 + rpad)
struct TcSplitDesc {
  int64_t src, row0;
  int32_t ld, rows, cols, rpad;
};

// one product C = beta C + alpha A B^T with A rows at slab row arow, B rows at brow
struct TcDesc {
  int64_t c, arow, brow;
  int32_t m, n, k, ldc, lower, pad;
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

}  // namespace amb
