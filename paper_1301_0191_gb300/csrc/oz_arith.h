// Integer arithmetic of the FP64 form's exact slice products (tc_gemm.cu):
// the base-128 digit split of an operand entry and the single rounding of
// an exact level sum to FP64.  The functions compile for the device (the
// kernels) and for the host (tests/test_slice_arith.py builds a harness
// from this header with the host compiler and checks them against exact
// rational arithmetic).
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define OZ_HD __host__ __device__ __forceinline__
#else
#define OZ_HD inline
#endif

namespace amb {
namespace oz {

constexpr int kSlices = 8;   // digits of 7 bits: 56 bits of every operand entry

OZ_HD int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

OZ_HD uint64_t bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}

OZ_HD double double_of(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  std::memcpy(&x, &u, sizeof x);
  return x;
#endif
}

// |x| as an ordered integer (the IEEE bit pattern without the sign)
OZ_HD uint64_t absbits(double x) { return bits_of(x) & 0x7FFFFFFFFFFFFFFFull; }

// e with 2^(e-1) <= |x| < 2^e from the bits of |x| (x != 0, finite)
OZ_HD int exponent(uint64_t ab) {
  const int bex = (int)(ab >> 52);
  const uint64_t mant = (ab & 0xFFFFFFFFFFFFFull) | (bex ? (1ull << 52) : 0ull);
  return (64 - clz64(mant)) + (bex > 1 ? bex : 1) - 1075;
}

// the kSlices balanced base-128 digits of x 2^-e (|x| < 2^e): F = x 2^(56-e)
// rounded to an integer (|F| < 2^56), taken apart least significant digit
// first, each digit into [-63, 64] with a carry into the next; the leading
// digit is the rest (0 .. 128), all with the sign of x.  So
// x = 2^e sum_p dig[p] 2^-7(p+1) up to 2^-57 2^e.
OZ_HD void digits(double x, int e, float* dig) {
  const uint64_t bits = bits_of(x);
  const uint64_t ab = bits & 0x7FFFFFFFFFFFFFFFull;
  const int bex = (int)(ab >> 52);
  const uint64_t mant = (ab & 0xFFFFFFFFFFFFFull) | (bex ? (1ull << 52) : 0ull);
  const int sh = (bex > 1 ? bex : 1) - 1075 + 56 - e;   // <= 3 since |x| < 2^e
  int64_t F;
  if (sh >= 0) F = (int64_t)(mant << sh);
  else if (sh > -64) F = (int64_t)((mant + (1ull << (-sh - 1))) >> (-sh));
  else F = 0;
  const float sg = (bits >> 63) ? -1.f : 1.f;
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int p = kSlices - 1; p > 0; --p) {
    int dd = (int)(F & 127);
    F >>= 7;
    if (dd > 64) {
      dd -= 128;
      F += 1;
    }
    dig[p] = sg * (float)dd;
  }
  dig[0] = sg * (float)F;
}

// (H 2^28 + L) 2^s rounded to the nearest double (ties to even), |H|, |L| <
// 2^46, in 64-bit integer arithmetic: the exact value is written as
// +-(a 2^28 + b) with a >= 0, 0 <= b < 2^28; its top 53 bits are rounded
// once, however H and L cancel.  Results outside the normal range go
// through ldexp.
OZ_HD double round_sum(int64_t H, int64_t L, int s) {
  int64_t hi = H + (L >> 28);   // floor division: L = (L >> 28) 2^28 + lo
  uint64_t lo = (uint64_t)(L & ((1ll << 28) - 1));
  const bool neg = hi < 0;
  uint64_t a;
  if (neg) {
    // -(hi 2^28 + lo) = (-hi - 1) 2^28 + (2^28 - lo), or -hi 2^28 when lo == 0
    a = lo ? (uint64_t)(-hi - 1) : (uint64_t)(-hi);
    lo = lo ? (1ull << 28) - lo : 0ull;
  } else {
    a = (uint64_t)hi;
  }
  if (a == 0 && lo == 0) return 0.0;
  uint64_t m;
  int nb;   // bit length of a 2^28 + lo
  if (a < (1ull << 25)) {
    m = (a << 28) | lo;   // exact: below 2^53
    nb = 64 - clz64(m);
    m <<= 53 - nb;
  } else {
    const int la = 64 - clz64(a);
    const int sh = la - 25;   // 1 .. 22: the bits of lo below the 53 kept ones
    nb = la + 28;
    m = (a << (28 - sh)) | (lo >> sh);
    const uint64_t rem = lo & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1))) ++m;
    if (m >> 53) {
      m >>= 1;
      ++nb;
    }
  }
  const int E = nb - 1 + s;   // exponent of the result
  if (E < -1022 || E > 1023) return ldexp(neg ? -(double)m : (double)m, E - 52);
  return double_of(((uint64_t)(E + 1023) << 52) | (m & ((1ull << 52) - 1)) | (neg ? (1ull << 63) : 0ull));
}

}  // namespace oz
}  // namespace amb
