// Batched dense kernels of the substructure engine: variable-size batched
// GEMM (with triangular operands and lower-only output, tile shape chosen by
// timing for repeatable calls), batched GEMV, blocked right-looking partial
// Cholesky and recursive-doubling triangular inverse.  Device memory comes
// from the stream-ordered pool (pool_init).  These carry the factorizations of Sec. 2 / Sec. 5 (A_II = L L^T,
// S = K_GG - X^T X with X = L^{-1} K_IG, and the corner-constrained Neumann
// factor S_DD = L_D L_D^T) and every solve with those factors.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "common.h"
#include "tc_gemm.h"
#include "timers.h"

namespace amb {

thread_local int64_t g_launches = 0;

void pool_init() {
  static thread_local int done_dev = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev == done_dev) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  done_dev = dev;
}

// ------------------------------------------------------------------ GEMM

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec2<double> { using type = double2; static constexpr int W = 2; };

template <typename T, typename TA>
struct GemmArgs {
  const GemmDesc* desc;
  const int* prefix;   // ndesc+1 tile prefix sums
  int ndesc;
  int flags;
  T alpha, beta;
  const TA* A;
  const T* B;
  T* C;
};

template <typename T, typename TA, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm(GemmArgs<T, TA> g) {
  constexpr int NTX = BM / TM, NTY = BN / TN, NT = NTX * NTY;
  constexpr int PAD = 16 / sizeof(T);
  constexpr int LA = BM * BK / NT, LB = BK * BN / NT;
  static_assert(LA * NT == BM * BK && LB * NT == BK * BN, "tile/thread mismatch");
  __shared__ __align__(16) T As[2][BK][BM + PAD];
  __shared__ __align__(16) T Bs[2][BK][BN + PAD];

  const int bid = blockIdx.x;
  int lo = 0, hi = g.ndesc - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (g.prefix[mid] <= bid) lo = mid; else hi = mid - 1;
  }
  const GemmDesc d = g.desc[lo];
  const int t = bid - g.prefix[lo];
  const int tn = (d.n + BN - 1) / BN;
  const int i0 = (t / tn) * BM, j0 = (t % tn) * BN;
  const int fl = g.flags;
  if ((fl & G_OUT_LOWER) && j0 > i0 + BM - 1) return;

  int kbeg = 0, kend = d.k;
  if (fl & G_TRI_A_LOWER) kend = min(kend, i0 + BM);
  if (fl & G_TRI_B_UPPER) kend = min(kend, j0 + BN);
  if (fl & G_TRI_A_UPPER) kbeg = max(kbeg, (i0 / BK) * BK);
  if (fl & G_TRI_B_LOWER) kbeg = max(kbeg, (j0 / BK) * BK);

  const TA* A = g.A + d.a;   // may alias C (in-place panel update)
  const T* __restrict__ B = g.B + d.b;
  const bool ta = fl & G_TRANS_A, tb = fl & G_TRANS_B;
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;

  T ra[LA], rb[LB];
  auto load = [&](int kt) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      int idx = tid + q * NT;
      int r, c;
      if (!ta) { r = idx % BM; c = idx / BM; } else { c = idx % BK; r = idx / BK; }
      int gi = i0 + r, gk = kt + c;
      bool ok = gi < d.m && gk < kend && gk >= 0;
      if ((fl & G_TRI_A_LOWER) && gk > gi) ok = false;
      if ((fl & G_TRI_A_UPPER) && gk < gi) ok = false;
      T v = T(0);
      if (ok) v = (T)(ta ? A[gk + (int64_t)gi * d.lda] : A[gi + (int64_t)gk * d.lda]);
      ra[q] = v;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      int idx = tid + q * NT;
      int c, j;
      if (!tb) { c = idx % BK; j = idx / BK; } else { j = idx % BN; c = idx / BN; }
      int gk = kt + c, gj = j0 + j;
      bool ok = gj < d.n && gk < kend && gk >= 0;
      if ((fl & G_TRI_B_LOWER) && gk < gj) ok = false;
      if ((fl & G_TRI_B_UPPER) && gk > gj) ok = false;
      T v = T(0);
      if (ok) v = tb ? B[gj + (int64_t)gk * d.ldb] : B[gk + (int64_t)gj * d.ldb];
      rb[q] = v;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      int idx = tid + q * NT;
      int r, c;
      if (!ta) { r = idx % BM; c = idx / BM; } else { c = idx % BK; r = idx / BK; }
      As[buf][c][r] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      int idx = tid + q * NT;
      int c, j;
      if (!tb) { c = idx % BK; j = idx / BK; } else { j = idx % BN; c = idx / BN; }
      Bs[buf][c][j] = rb[q];
    }
  };

  T acc[TM][TN];
#pragma unroll
  for (int p = 0; p < TM; ++p)
#pragma unroll
    for (int q = 0; q < TN; ++q) acc[p][q] = T(0);

  using V = typename Vec2<T>::type;
  constexpr int W = Vec2<T>::W;
  int buf = 0;
  if (kbeg < kend) {
    load(kbeg);
    store(0);
    __syncthreads();
    for (int kt = kbeg; kt < kend; kt += BK) {
      const bool more = kt + BK < kend;
      if (more) load(kt + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[TM], b[TN];
#pragma unroll
        for (int p = 0; p < TM; p += W) {
          V v = *reinterpret_cast<const V*>(&As[buf][kk][tx * TM + p]);
          memcpy(&a[p], &v, sizeof(V));
        }
        if constexpr (TN % W == 0) {
#pragma unroll
          for (int q = 0; q < TN; q += W) {
            V v = *reinterpret_cast<const V*>(&Bs[buf][kk][ty * TN + q]);
            memcpy(&b[q], &v, sizeof(V));
          }
        } else {
#pragma unroll
          for (int q = 0; q < TN; ++q) b[q] = Bs[buf][kk][ty * TN + q];
        }
#pragma unroll
        for (int p = 0; p < TM; ++p)
#pragma unroll
          for (int q = 0; q < TN; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
      }
      if (more) {
        store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }

  T* C = g.C + d.c;
  const bool lower = fl & G_OUT_LOWER;
#pragma unroll
  for (int q = 0; q < TN; ++q) {
    int j = j0 + ty * TN + q;
    if (j >= d.n) continue;
#pragma unroll
    for (int p = 0; p < TM; ++p) {
      int i = i0 + tx * TM + p;
      if (i >= d.m || (lower && i < j)) continue;
      int64_t o = i + (int64_t)j * d.ldc;
      T v = g.alpha * acc[p][q];
      if (g.beta != T(0)) v = fma(g.beta, C[o], v);
      C[o] = v;
    }
  }
}

// ------------------------------------------------------------------ GEMM, FP32 operands, extended accumulation
// C (FP64) = alpha op(A) op(B) + beta C with A stored in FP32 and B in FP64.
// FP64 arithmetic runs at 1/64 of the FP32 rate on this GPU, so the sum is
// carried in FP32 pairs instead: every product a*b_hi is split exactly into
// p + e with an FMA, added to (hi, lo) by Knuth's TwoSum, and a*b_lo (b =
// b_hi + b_lo, both FP32) goes into lo.  The result hi + lo has about 44
// significant bits, enough for the FP64-consistent Rayleigh-Ritz of the
// pair eigenproblems; plain FP32 accumulation is not (see lobpcg.cu).
// Tiles with at most 8 outputs per thread are held to 64 registers (1024
// resident threads per SM): the TwoSum chains are dependent, so the kernel
// needs warps to hide their latency (96 registers left 20 warps per SM and
// the FMA pipe half idle).  The 16-output tile would spill at 64.
template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN), TM * TN <= 8 ? 1024 / ((BM / TM) * (BN / TN)) : 1)
k_gemm_df(GemmArgs<double, float> g) {
  constexpr int NTX = BM / TM, NTY = BN / TN, NT = NTX * NTY;
  constexpr int LA = BM * BK / NT, LB = BK * BN / NT;
  static_assert(LA * NT == BM * BK && LB * NT == BK * BN, "tile/thread mismatch");
  __shared__ float As[BK][BM + 4];
  __shared__ float2 Bs[BK][BN + 2];
  const int bid = blockIdx.x;
  int lo = 0, hi = g.ndesc - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (g.prefix[mid] <= bid) lo = mid; else hi = mid - 1;
  }
  const GemmDesc d = g.desc[lo];
  const int t = bid - g.prefix[lo];
  const int tn = (d.n + BN - 1) / BN;
  const int i0 = (t / tn) * BM, j0 = (t % tn) * BN;
  const int fl = g.flags;
  const bool ta = fl & G_TRANS_A, tb = fl & G_TRANS_B;
  int kbeg = 0, kend = d.k;
  if (fl & G_TRI_A_LOWER) kend = min(kend, i0 + BM);
  if (fl & G_TRI_B_UPPER) kend = min(kend, j0 + BN);
  if (fl & G_TRI_A_UPPER) kbeg = max(kbeg, (i0 / BK) * BK);
  if (fl & G_TRI_B_LOWER) kbeg = max(kbeg, (j0 / BK) * BK);
  const float* __restrict__ A = g.A + d.a;
  const double* __restrict__ B = g.B + d.b;
  const int tid = threadIdx.x, tx = tid % NTX, ty = tid / NTX;
  float ah[TM][TN], al[TM][TN];
#pragma unroll
  for (int p = 0; p < TM; ++p)
#pragma unroll
    for (int q = 0; q < TN; ++q) ah[p][q] = al[p][q] = 0.f;
  for (int kt = kbeg; kt < kend; kt += BK) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      int idx = tid + q * NT, r, c;
      if (!ta) { r = idx % BM; c = idx / BM; } else { c = idx % BK; r = idx / BK; }
      int gi = i0 + r, gk = kt + c;
      bool ok = gi < d.m && gk < kend;
      if ((fl & G_TRI_A_LOWER) && gk > gi) ok = false;
      if ((fl & G_TRI_A_UPPER) && gk < gi) ok = false;
      float v = 0.f;
      if (ok) v = ta ? A[gk + (int64_t)gi * d.lda] : A[gi + (int64_t)gk * d.lda];
      As[c][r] = v;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      int idx = tid + q * NT, c, j;
      if (!tb) { c = idx % BK; j = idx / BK; } else { j = idx % BN; c = idx / BN; }
      int gk = kt + c, gj = j0 + j;
      bool ok = gj < d.n && gk < kend;
      if ((fl & G_TRI_B_LOWER) && gk < gj) ok = false;
      if ((fl & G_TRI_B_UPPER) && gk > gj) ok = false;
      double v = 0.0;
      if (ok) v = tb ? B[gj + (int64_t)gk * d.ldb] : B[gk + (int64_t)gj * d.ldb];
      const float vh = (float)v;
      Bs[c][j] = make_float2(vh, (float)(v - (double)vh));
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[TM];
      float2 b[TN];
#pragma unroll
      for (int p = 0; p < TM; ++p) a[p] = As[kk][tx * TM + p];
#pragma unroll
      for (int q = 0; q < TN; ++q) b[q] = Bs[kk][ty * TN + q];
#pragma unroll
      for (int p = 0; p < TM; ++p)
#pragma unroll
        for (int q = 0; q < TN; ++q) {
          // explicit _rn intrinsics: never contracted into FMAs, so the
          // error-free transformations stay exact
          const float pr = __fmul_rn(a[p], b[q].x);
          const float e = fmaf(a[p], b[q].x, -pr);
          const float s = __fadd_rn(ah[p][q], pr);
          const float bb = __fsub_rn(s, ah[p][q]);
          const float er = __fadd_rn(__fsub_rn(ah[p][q], __fsub_rn(s, bb)), __fsub_rn(pr, bb));
          ah[p][q] = s;
          al[p][q] = fmaf(a[p], b[q].y, __fadd_rn(al[p][q], __fadd_rn(er, e)));
        }
    }
    __syncthreads();
  }
  double* C = g.C + d.c;
#pragma unroll
  for (int q = 0; q < TN; ++q) {
    int j = j0 + ty * TN + q;
    if (j >= d.n) continue;
#pragma unroll
    for (int p = 0; p < TM; ++p) {
      int i = i0 + tx * TM + p;
      if (i >= d.m) continue;
      int64_t o = i + (int64_t)j * d.ldc;
      double v = g.alpha * ((double)ah[p][q] + (double)al[p][q]);
      if (g.beta != 0.0) v = fma(g.beta, C[o], v);
      C[o] = v;
    }
  }
}

template <typename T> struct GemmTile;
template <> struct GemmTile<double> { static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4; };
template <> struct GemmTile<float> { static constexpr int BM = 128, BN = 128, BK = 16, TM = 8, TN = 8; };

// Tile shapes: a thin one (8 columns) for the soft-locked LOBPCG blocks, whose
// active width is mostly the used columns plus a few guards;
template <typename T> struct GemmThin;
template <> struct GemmThin<double> { static constexpr int BM = 64, BN = 8, BK = 16, TM = 4, TN = 2; };
template <> struct GemmThin<float> { static constexpr int BM = 128, BN = 8, BK = 16, TM = 8, TN = 2; };
// a wide one, and a skinny one for products whose right-hand
// block has at most 16 columns (the LOBPCG blocks and the Neumann solves of
// the pair preconditioner), which would otherwise waste most of a wide tile.
template <typename T> struct GemmSkinny;
template <> struct GemmSkinny<double> { static constexpr int BM = 64, BN = 16, BK = 16, TM = 4, TN = 2; };
template <> struct GemmSkinny<float> { static constexpr int BM = 128, BN = 16, BK = 16, TM = 8, TN = 2; };
// ... and a medium one for 17..32 columns (the Rayleigh-Ritz updates)
template <typename T> struct GemmMedium;
template <> struct GemmMedium<double> { static constexpr int BM = 64, BN = 32, BK = 16, TM = 4, TN = 2; };
template <> struct GemmMedium<float> { static constexpr int BM = 128, BN = 32, BK = 16, TM = 8, TN = 2; };
// ... and a half-wide one (FP32) for 33..64 columns (the Cholesky strip and
// panel updates; an in-place panel update needs one CTA to own whole rows,
// which holds because the tile is at least as wide as the product)
struct GemmHalfF { static constexpr int BM = 128, BN = 64, BK = 16, TM = 8, TN = 4; };

template <typename T, typename TA, typename TL>
static void gemm_run(cudaStream_t st, DescRing& ring, const std::vector<GemmDesc>& d, int flags, T alpha, T beta,
                     const TA* A, const T* B, T* C) {
  std::vector<GemmDesc> dd;
  std::vector<int> prefix;
  dd.reserve(d.size());
  prefix.reserve(d.size() + 1);
  int64_t total = 0;
  for (const auto& x : d) {
    if (x.m <= 0 || x.n <= 0) continue;
    dd.push_back(x);
    prefix.push_back((int)total);
    total += (int64_t)((x.m + TL::BM - 1) / TL::BM) * ((x.n + TL::BN - 1) / TL::BN);
  }
  if (dd.empty()) return;
  AMB_CHECK(total < (int64_t)1 << 31, AMB_EINVAL, "GEMM batch too large");
  prefix.push_back((int)total);
  // one staging push: descriptors then prefix
  std::vector<char> blob(dd.size() * sizeof(GemmDesc) + prefix.size() * sizeof(int));
  memcpy(blob.data(), dd.data(), dd.size() * sizeof(GemmDesc));
  memcpy(blob.data() + dd.size() * sizeof(GemmDesc), prefix.data(), prefix.size() * sizeof(int));
  char* dev = static_cast<char*>(ring.push(blob.data(), blob.size(), st));
  GemmArgs<T, TA> g;
  g.desc = reinterpret_cast<const GemmDesc*>(dev);
  g.prefix = reinterpret_cast<const int*>(dev + dd.size() * sizeof(GemmDesc));
  g.ndesc = (int)dd.size();
  g.flags = flags;
  g.alpha = alpha;
  g.beta = beta;
  g.A = A;
  g.B = B;
  g.C = C;
  constexpr int NT = (TL::BM / TL::TM) * (TL::BN / TL::TN);
  if constexpr (std::is_same<T, double>::value && std::is_same<TA, float>::value) {
    if ((flags & G_OUT_LOWER) == 0) {   // extended-precision FP32 path
      k_gemm_df<TL::BM, TL::BN, TL::BK, TL::TM, TL::TN><<<(unsigned)total, NT, 0, st>>>(g);
      AMB_LAUNCHED();
      return;
    }
  }
  k_gemm<T, TA, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN><<<(unsigned)total, NT, 0, st>>>(g);
  AMB_LAUNCHED();
}

// Tile autotuner.  A product flagged G_TUNE is run once with every tile
// shape the first time its shape class is seen (types, flags, the widest
// right-hand block exactly, and powers of two of the batch size, the
// longest and the summed rows and the longest K, so that the shrinking
// batches of an iteration reuse one entry); the fastest by CUDA events is
// kept for the process.  Every shape accumulates each output over k in the
// same order, so the choice does not change the result.  Products without
// the flag, and products issued while the stream is being captured into a
// graph, take the static rule (narrowest tile that covers the columns).
namespace {

enum TileChoice { TILE_THIN = 0, TILE_SKINNY = 1, TILE_MEDIUM = 2, TILE_HALF = 3, TILE_WIDE = 4 };

struct TuneKey {
  int type, flags, ndesc, mmax, nmax, kmax;
  int64_t msum, nsum, ksum;
  bool operator==(const TuneKey& o) const {
    return type == o.type && flags == o.flags && ndesc == o.ndesc && mmax == o.mmax && nmax == o.nmax &&
           kmax == o.kmax && msum == o.msum && nsum == o.nsum && ksum == o.ksum;
  }
};
struct TuneKeyHash {
  size_t operator()(const TuneKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int64_t v : {(int64_t)k.type, (int64_t)k.flags, (int64_t)k.ndesc, (int64_t)k.mmax, (int64_t)k.nmax,
                      (int64_t)k.kmax, k.msum, k.nsum, k.ksum})
      h = (h ^ (uint64_t)v) * 1099511628211ull;
    return (size_t)h;
  }
};

std::mutex g_tune_mu;
std::unordered_map<TuneKey, int, TuneKeyHash> g_tune;
std::atomic<int64_t> g_tune_runs{0};   // products run for tuning

template <typename T, typename TA>
void run_choice(int c, cudaStream_t st, DescRing& ring, const std::vector<GemmDesc>& d, int flags, T alpha, T beta,
                const TA* A, const T* B, T* C) {
  switch (c) {
    case TILE_THIN: gemm_run<T, TA, GemmThin<T>>(st, ring, d, flags, alpha, beta, A, B, C); break;
    case TILE_SKINNY: gemm_run<T, TA, GemmSkinny<T>>(st, ring, d, flags, alpha, beta, A, B, C); break;
    case TILE_MEDIUM: gemm_run<T, TA, GemmMedium<T>>(st, ring, d, flags, alpha, beta, A, B, C); break;
    case TILE_HALF:
      if constexpr (std::is_same<T, float>::value) {
        gemm_run<T, TA, GemmHalfF>(st, ring, d, flags, alpha, beta, A, B, C);
        break;
      }
      [[fallthrough]];
    default: gemm_run<T, TA, GemmTile<T>>(st, ring, d, flags, alpha, beta, A, B, C); break;
  }
}

}  // namespace

int64_t gemm_tune_runs() { return g_tune_runs.load(); }
size_t gemm_tune_entries() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune.size();
}

template <typename T, typename TA>
void gemm_batched(cudaStream_t st, DescRing& ring, const std::vector<GemmDesc>& d, int flags,
                  T alpha, T beta, const TA* A, const T* B, T* C) {
  int nmax = 0, mmax = 0, kmax = 0, nd = 0;
  int64_t msum = 0, nsum = 0, ksum = 0;
  for (const auto& x : d) {
    if (x.m <= 0 || x.n <= 0) continue;
    ++nd;
    nmax = std::max(nmax, x.n);
    mmax = std::max(mmax, x.m);
    kmax = std::max(kmax, x.k);
    msum += x.m;
    nsum += x.n;
    ksum += x.k;
  }
  if (nd == 0) return;
  const bool narrow_ok = !(flags & G_OUT_LOWER);
  // static rule
  int choice = TILE_WIDE;
  if (narrow_ok && nmax <= 8) choice = TILE_THIN;
  else if (narrow_ok && nmax <= 16) choice = TILE_SKINNY;
  else if (narrow_ok && nmax <= 32) choice = TILE_MEDIUM;
  else if (std::is_same<T, float>::value && narrow_ok && nmax <= 64) choice = TILE_HALF;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  AMB_CUDA(cudaStreamIsCapturing(st, &cap));
  if (!(flags & G_TUNE) || !narrow_ok || beta != T(0) || cap != cudaStreamCaptureStatusNone) {
    run_choice<T, TA>(choice, st, ring, d, flags, alpha, beta, A, B, C);
    return;
  }
  auto lg = [](int64_t v) {
    int b = 0;
    while (v > 1) v >>= 1, ++b;
    return b;
  };
  const int type = (int)sizeof(T) * 16 + (int)sizeof(TA);
  const TuneKey key{type, flags, lg(nd), lg(mmax), nmax, lg(kmax), lg(msum), 0, 0};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      run_choice<T, TA>(it->second, st, ring, d, flags, alpha, beta, A, B, C);
      return;
    }
  }
  // candidates: every shape from the narrowest that covers the columns up
  // to the widest (a narrower tile than the columns runs more column tiles)
  std::vector<int> cand;
  for (int c = TILE_THIN; c <= TILE_WIDE; ++c) {
    if (c == TILE_HALF && !std::is_same<T, float>::value) continue;
    cand.push_back(c);
  }
  cudaEvent_t e0, e1;
  AMB_CUDA(cudaEventCreate(&e0));
  AMB_CUDA(cudaEventCreate(&e1));
  int best = choice;
  float best_ms = 1e30f;
  for (int c : cand) {
    AMB_CUDA(cudaEventRecord(e0, st));
    run_choice<T, TA>(c, st, ring, d, flags, alpha, beta, A, B, C);
    AMB_CUDA(cudaEventRecord(e1, st));
    AMB_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    ++g_tune_runs;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
}

template <typename T>
int gemm_ctas(const GemmDesc& x) {
  using TL = GemmTile<T>;
  if (x.m <= 0 || x.n <= 0) return 0;
  return ((x.m + TL::BM - 1) / TL::BM) * ((x.n + TL::BN - 1) / TL::BN);
}
template int gemm_ctas<float>(const GemmDesc&);
template int gemm_ctas<double>(const GemmDesc&);

template <typename T>
void gemm_launch_prepared(cudaStream_t st, const GemmDesc* d_desc, const int* d_prefix, int ndesc, int total,
                          int flags, T alpha, T beta, const T* A, const T* B, T* C) {
  using TL = GemmTile<T>;
  if (ndesc <= 0 || total <= 0) return;
  GemmArgs<T, T> g;
  g.desc = d_desc;
  g.prefix = d_prefix;
  g.ndesc = ndesc;
  g.flags = flags;
  g.alpha = alpha;
  g.beta = beta;
  g.A = A;
  g.B = B;
  g.C = C;
  constexpr int NT = (TL::BM / TL::TM) * (TL::BN / TL::TN);
  k_gemm<T, T, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN><<<(unsigned)total, NT, 0, st>>>(g);
  AMB_LAUNCHED();
}
template void gemm_launch_prepared<float>(cudaStream_t, const GemmDesc*, const int*, int, int, int, float, float,
                                          const float*, const float*, float*);
template void gemm_launch_prepared<double>(cudaStream_t, const GemmDesc*, const int*, int, int, int, double, double,
                                           const double*, const double*, double*);

template void gemm_batched<float, float>(cudaStream_t, DescRing&, const std::vector<GemmDesc>&, int, float, float,
                                         const float*, const float*, float*);
template void gemm_batched<double, double>(cudaStream_t, DescRing&, const std::vector<GemmDesc>&, int, double,
                                           double, const double*, const double*, double*);
template void gemm_batched<double, float>(cudaStream_t, DescRing&, const std::vector<GemmDesc>&, int, double,
                                          double, const float*, const double*, double*);

// ------------------------------------------------------------------ GEMV
// y = alpha op(A) x + beta y, one vector per descriptor; every launch
// streams its matrices from HBM once, so the kernels are built for bytes in
// flight.  No-transpose: a CTA owns 32 rows (one per lane) and its warps take
// interleaved 32-column chunks, each warp issuing its chunk's 32 column loads
// back to back (x broadcast by shuffle); the warps' partial sums are merged
// in a fixed order.  Transpose: one warp per output column, x staged in
// shared memory, loads unrolled by 8.

template <typename T>
struct GemvArgs {
  const GemvDesc* desc;
  const int* prefix;
  int ndesc, flags;
  T alpha, beta;
  const T* A;
  const T* X;
  T* Y;
};

constexpr int kGemvRows = 32;    // rows per CTA (no-transpose)
constexpr int kGemvWarps = 8;    // warps per CTA
constexpr int kGemvCols = 8;     // outputs per CTA (transpose): one warp each
constexpr int kGemvXChunk = 2048;   // staged x entries (transpose)

template <typename T>
__device__ inline int gemv_find(const GemvArgs<T>& g, int bid) {
  int lo = 0, hi = g.ndesc - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (g.prefix[mid] <= bid) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Compensated accumulation for FP32 matrix-vector products: (hi, lo) holds
// the running sum, products are split exactly by FMA and added by TwoSum
// (explicit _rn intrinsics: never contracted, so the transformations stay
// exact).  The extra FP32 instructions hide behind the memory stream.
struct DF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float pr = __fmul_rn(a, b);
    const float e = fmaf(a, b, -pr);
    const float s = __fadd_rn(hi, pr);
    const float bb = __fsub_rn(s, hi);
    const float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(pr, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(er, e));
  }
  __device__ __forceinline__ void merge(const DF& o) {
    const float s = __fadd_rn(hi, o.hi);
    const float bb = __fsub_rn(s, hi);
    const float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(o.hi, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(er, o.lo));
  }
  __device__ __forceinline__ void shfl_merge(int o) {
    DF t;
    t.hi = __shfl_xor_sync(0xffffffffu, hi, o);
    t.lo = __shfl_xor_sync(0xffffffffu, lo, o);
    merge(t);
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(hi, lo); }
};

// Plain FP64 accumulation with the same interface.
struct D64 {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ void merge(const D64& o) { v += o.v; }
  __device__ __forceinline__ void shfl_merge(int o) { v += __shfl_xor_sync(0xffffffffu, v, o); }
  __device__ __forceinline__ double value() const { return v; }
};

template <typename T> struct GemvAcc;
template <> struct GemvAcc<float> { using type = DF; };
template <> struct GemvAcc<double> { using type = D64; };

template <typename T>
__global__ void __launch_bounds__(32 * kGemvWarps) k_gemv_n(GemvArgs<T> g) {
  using Acc = typename GemvAcc<T>::type;
  __shared__ Acc red[kGemvWarps][32];
  const int di = gemv_find(g, blockIdx.x);
  const GemvDesc d = g.desc[di];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = (blockIdx.x - g.prefix[di]) * kGemvRows, i = i0 + lane;
  const bool row_ok = i < d.m;
  const bool lower = g.flags & G_TRI_A_LOWER, upper = g.flags & G_TRI_A_UPPER;
  int cbeg = 0, cend = d.n;
  if (lower) cend = min(d.n, i0 + kGemvRows);
  if (upper) cbeg = min(d.n, i0);
  const T* __restrict__ A = g.A + d.a + (row_ok ? i : i0);
  const T* __restrict__ x = g.X + d.x;
  Acc s;
  for (int c0 = cbeg + warp * 32; c0 < cend; c0 += 32 * kGemvWarps) {
    const int cn = min(32, cend - c0);
    const T xr = lane < cn ? x[c0 + lane] : T(0);
    const T* __restrict__ col = A + (int64_t)c0 * d.lda;
    // the chunk touches the diagonal: mask the other triangle per element
    const bool diag = (lower && c0 + 31 > i0) || (upper && c0 < i0 + 31);
    if (cn == 32 && !diag) {
      T a[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) a[j] = col[(int64_t)j * d.lda];
#pragma unroll
      for (int j = 0; j < 32; ++j) s.add(a[j], __shfl_sync(0xffffffffu, xr, j));
    } else {
      for (int j = 0; j < cn; ++j) {
        const int c = c0 + j;
        T a = col[(int64_t)j * d.lda];
        if ((lower && c > i) || (upper && c < i)) a = T(0);
        s.add(a, __shfl_sync(0xffffffffu, xr, j));
      }
    }
  }
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && row_ok) {
    Acc t = red[0][lane];
#pragma unroll
    for (int w = 1; w < kGemvWarps; ++w) t.merge(red[w][lane]);
    T v = g.alpha * (T)t.value();
    T* y = g.Y + d.y;
    if (g.beta != T(0)) v = fma(g.beta, y[i], v);
    y[i] = v;
  }
}

template <typename T>
__global__ void __launch_bounds__(32 * kGemvCols) k_gemv_t(GemvArgs<T> g) {
  using Acc = typename GemvAcc<T>::type;
  __shared__ T xs[kGemvXChunk];
  const int di = gemv_find(g, blockIdx.x);
  const GemvDesc d = g.desc[di];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = (blockIdx.x - g.prefix[di]) * kGemvCols;
  const int j = j0 + warp;   // output index = column of A
  const bool lower = g.flags & G_TRI_A_LOWER, upper = g.flags & G_TRI_A_UPPER;
  // rows of column j: op(A) = A^T upper <=> rows i >= j; lower <=> rows i <= j
  int ib = 0, ie = d.m;
  if (upper) ib = min(j, d.m);
  if (lower) ie = min(d.m, j + 1);
  // rows any column of this CTA reads
  int cb = 0, ce = d.m;
  if (upper) cb = min(j0, d.m);
  if (lower) ce = min(d.m, j0 + kGemvCols);
  const T* __restrict__ col = g.A + d.a + (int64_t)min(j, d.n - 1) * d.lda;
  const T* __restrict__ x = g.X + d.x;
  Acc s;
  for (int r0 = cb; r0 < ce; r0 += kGemvXChunk) {
    const int rn = min(kGemvXChunk, ce - r0);
    __syncthreads();
    for (int q = threadIdx.x; q < rn; q += blockDim.x) xs[q] = x[r0 + q];
    __syncthreads();
    if (j < d.n) {
      const int lo = max(ib, r0), hi = min(ie, r0 + rn);
      int r = lo + lane;
      for (; r + 7 * 32 < hi; r += 8 * 32) {
        T a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = col[r + u * 32];
#pragma unroll
        for (int u = 0; u < 8; ++u) s.add(a[u], xs[r + u * 32 - r0]);
      }
      for (; r < hi; r += 32) s.add(col[r], xs[r - r0]);
    }
  }
  if (j >= d.n) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s.shfl_merge(o);
  if (lane == 0) {
    T v = g.alpha * (T)s.value();
    T* y = g.Y + d.y;
    if (g.beta != T(0)) v = fma(g.beta, y[j], v);
    y[j] = v;
  }
}

// No-transpose product with few columns (a coarse basis, the constraint
// block): a thread per row, columns in order.  The 8-warp column split of
// k_gemv_n leaves most warps idle there.
constexpr int kGemvNarrowCols = 96;   // widest product that takes this kernel
constexpr int kGemvNarrowRows = 128;  // rows (threads) per CTA

template <typename T>
__global__ void __launch_bounds__(kGemvNarrowRows) k_gemv_nr(GemvArgs<T> g) {
  using Acc = typename GemvAcc<T>::type;
  const int di = gemv_find(g, blockIdx.x);
  const GemvDesc d = g.desc[di];
  const int i = (blockIdx.x - g.prefix[di]) * kGemvNarrowRows + threadIdx.x;
  if (i >= d.m) return;
  const T* __restrict__ a = g.A + d.a + i;
  const T* __restrict__ x = g.X + d.x;
  Acc s;
  int j = 0;
  for (; j + 8 <= d.n; j += 8) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = a[(int64_t)(j + u) * d.lda];
#pragma unroll
    for (int u = 0; u < 8; ++u) s.add(v[u], x[j + u]);
  }
  for (; j < d.n; ++j) s.add(a[(int64_t)j * d.lda], x[j]);
  T v = g.alpha * (T)s.value();
  T* y = g.Y + d.y;
  if (g.beta != T(0)) v = fma(g.beta, y[i], v);
  y[i] = v;
}

// FP32 products use compensated accumulation, FP64 plain FMA chains.
template <typename T>
static void launch_gemv(cudaStream_t st, const GemvArgs<T>& g, unsigned total, bool trans) {
  if (trans) k_gemv_t<T><<<total, 32 * kGemvCols, 0, st>>>(g);
  else k_gemv_n<T><<<total, 32 * kGemvWarps, 0, st>>>(g);
}

template <typename T>
void gemv_batched(cudaStream_t st, DescRing& ring, const std::vector<GemvDesc>& d, int flags,
                  T alpha, T beta, const T* A, const T* X, T* Y) {
  const bool trans = flags & G_TRANS_A;
  int nmax = 0;
  for (const auto& x : d) nmax = std::max(nmax, x.n);
  const bool narrow = !trans && !(flags & (G_TRI_A_LOWER | G_TRI_A_UPPER)) && nmax <= kGemvNarrowCols;
  const int rows_per_cta = narrow ? kGemvNarrowRows : kGemvRows;
  std::vector<GemvDesc> dd;
  std::vector<int> prefix;
  int64_t total = 0;
  for (const auto& x : d) {
    int outs = trans ? x.n : x.m;
    if (outs <= 0) continue;
    dd.push_back(x);
    prefix.push_back((int)total);
    total += trans ? (outs + kGemvCols - 1) / kGemvCols : (outs + rows_per_cta - 1) / rows_per_cta;
  }
  if (dd.empty()) return;
  prefix.push_back((int)total);
  std::vector<char> blob(dd.size() * sizeof(GemvDesc) + prefix.size() * sizeof(int));
  memcpy(blob.data(), dd.data(), dd.size() * sizeof(GemvDesc));
  memcpy(blob.data() + dd.size() * sizeof(GemvDesc), prefix.data(), prefix.size() * sizeof(int));
  char* dev = static_cast<char*>(ring.push(blob.data(), blob.size(), st));
  GemvArgs<T> g{reinterpret_cast<const GemvDesc*>(dev),
                reinterpret_cast<const int*>(dev + dd.size() * sizeof(GemvDesc)),
                (int)dd.size(), flags, alpha, beta, A, X, Y};
  if (narrow) k_gemv_nr<T><<<(unsigned)total, kGemvNarrowRows, 0, st>>>(g);
  else launch_gemv<T>(st, g, (unsigned)total, trans);
  AMB_LAUNCHED();
}

int gemv_ctas(const GemvDesc& x, bool trans) {
  const int outs = trans ? x.n : x.m;
  if (outs <= 0) return 0;
  return trans ? (outs + kGemvCols - 1) / kGemvCols : (outs + kGemvRows - 1) / kGemvRows;
}

template <typename T>
void gemv_launch_prepared(cudaStream_t st, const GemvDesc* d_desc, const int* d_prefix, int ndesc, int total,
                          int flags, T alpha, T beta, const T* A, const T* X, T* Y) {
  if (ndesc <= 0 || total <= 0) return;
  GemvArgs<T> g{d_desc, d_prefix, ndesc, flags, alpha, beta, A, X, Y};
  launch_gemv<T>(st, g, (unsigned)total, (flags & G_TRANS_A) != 0);

  AMB_LAUNCHED();
}
template void gemv_launch_prepared<float>(cudaStream_t, const GemvDesc*, const int*, int, int, int, float, float,
                                          const float*, const float*, float*);
template void gemv_launch_prepared<double>(cudaStream_t, const GemvDesc*, const int*, int, int, int, double, double,
                                           const double*, const double*, double*);

template void gemv_batched<float>(cudaStream_t, DescRing&, const std::vector<GemvDesc>&, int, float, float,
                                  const float*, const float*, float*);
template void gemv_batched<double>(cudaStream_t, DescRing&, const std::vector<GemvDesc>&, int, double, double,
                                   const double*, const double*, double*);

// ------------------------------------------------------------------ Cholesky
// Diagonal block: unblocked Cholesky in FP64 shared memory (whatever the
// storage type), then the explicit inverse of the block.  A non-positive
// pivot is recorded (status[0] = AMB_ENOTSPD, status[1] = id, status[2] =
// global column) and replaced by 1 so that the factorization stays finite.

struct DiagDesc {
  int64_t blk;      // offset of the diagonal block in the matrix buffer
  int64_t zblk;     // offset of the inverse block in the Z buffer (-1: none)
  int64_t scratch;  // offset (elements) of the nb x nb inverse in the scratch buffer
  int32_t ld, zld, jb, id, col;
};

template <typename T>
__global__ void __launch_bounds__(256) k_chol_diag(const DiagDesc* descs, T* base, T* zbase, T* scratch, int* status) {
  __shared__ double a[kNB][kNB + 1];
  const DiagDesc d = descs[blockIdx.x];
  const int jb = d.jb, tid = threadIdx.x;
  T* blk = base + d.blk;
  for (int idx = tid; idx < jb * jb; idx += blockDim.x) {
    int r = idx % jb, c = idx / jb;
    a[r][c] = (r >= c) ? (double)blk[r + (int64_t)c * d.ld] : 0.0;
  }
  __syncthreads();
  // FP64 divisions are long instruction sequences on this GPU's slow FP64
  // pipe: each pivot's reciprocal is formed once and multiplied
  __shared__ double dinv[kNB];
  for (int c = 0; c < jb; ++c) {
    if (tid == 0) {
      double p = a[c][c];
      if (!(p > 0.0)) {
        if (atomicCAS(status, 0, AMB_ENOTSPD) == 0) {
          status[1] = d.id;
          status[2] = d.col + c;
        }
        p = 1.0;
      }
      a[c][c] = sqrt(p);
      dinv[c] = 1.0 / a[c][c];
    }
    __syncthreads();
    const double rpiv = dinv[c];
    for (int r = c + 1 + tid; r < jb; r += blockDim.x) a[r][c] *= rpiv;
    __syncthreads();
    const int m = jb - c - 1;
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
      int r = c + 1 + idx % m, q = c + 1 + idx / m;
      if (r >= q) a[r][q] -= a[r][c] * a[q][c];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < jb * jb; idx += blockDim.x) {
    int r = idx % jb, c = idx / jb;
    if (r >= c) blk[r + (int64_t)c * d.ld] = (T)a[r][c];
  }
  // Inverse of the lower-triangular block by forward substitution, one
  // column per thread; entry (i, j), i > j, of the inverse is kept in the
  // unused upper triangle a[j][i], its diagonal in dinv[] (the reciprocals
  // of the pivots, formed above).
  if (tid < jb) {
    const int j = tid;
    for (int i = j + 1; i < jb; ++i) {
      double s = a[i][j] * dinv[j];
      for (int l = j + 1; l < i; ++l) s += a[i][l] * a[j][l];
      a[j][i] = -s * dinv[i];
    }
  }
  __syncthreads();
  T* sc = scratch + d.scratch;
  for (int idx = tid; idx < kNB * kNB; idx += blockDim.x) {
    int r = idx % kNB, c = idx / kNB;
    double v = 0.0;
    if (r < jb && c < jb) v = (r > c) ? a[c][r] : (r == c ? dinv[r] : 0.0);
    sc[r + c * kNB] = (T)v;
    if (d.zblk >= 0 && r < jb && c < jb) zbase[d.zblk + r + (int64_t)c * d.zld] = (T)v;
  }
}

// scratch space for the diagonal inverses, grown on demand
template <typename T>
static T* diag_scratch(size_t nblocks) {
  check_workspace_device();
  static thread_local DevBuf buf;
  size_t need = nblocks * kNB * kNB * sizeof(T);
  if (buf.bytes < need) {
    AMB_CUDA(cudaDeviceSynchronize());   // earlier factorizations may still read the old buffer
    buf.alloc(need);
  }
  return dptr<T>(buf);
}

template <typename T>
void partial_cholesky(cudaStream_t st, DescRing& ring, const std::vector<CholDesc>& d, T* base,
                      T* zbase, int* status, double* flops, Timers* tm, bool timing) {
  // Two-level blocking: inner panels of kNB columns (diagonal factor +
  // inverse, panel solve) inside outer blocks of kOuter columns.  Inside an
  // outer block the next panel's columns are brought up to date from the
  // previous panels of the block (left-looking strip update); the trailing
  // matrix is updated once per outer block with K = kOuter, which cuts the
  // passes over the trailing matrix (and its memory traffic) by kOuter/kNB.
  constexpr int kOuter = 4 * kNB;
  static_assert(kOuter <= kTcKMax, "outer block wider than the tensor-core slab");
  if (d.empty()) return;
  int maxouter = 0;
  for (const auto& x : d) maxouter = std::max(maxouter, (x.c1 - x.c0 + kOuter - 1) / kOuter);
  T* scratch = diag_scratch<T>(d.size());
  for (int ob = 0; ob < maxouter; ++ob) {
    for (int q = 0; q < kOuter / kNB; ++q) {
      std::vector<DiagDesc> dg;
      std::vector<GemmDesc> strip, panel;
      for (size_t i = 0; i < d.size(); ++i) {
        const CholDesc& x = d[i];
        const int J0 = x.c0 + ob * kOuter;
        if (J0 >= x.c1) continue;
        const int J1 = std::min(J0 + kOuter, x.c1);
        const int j0 = J0 + q * kNB;
        if (j0 >= J1) continue;
        const int jb = std::min(kNB, J1 - j0);
        const int rem0 = x.n - j0;   // rows from the diagonal block down
        if (j0 > J0) {
          // A[j0:, j0:j0+jb] -= A[j0:, J0:j0] A[j0:j0+jb, J0:j0]^T
          strip.push_back(GemmDesc{rem0, jb, j0 - J0, x.ld, x.ld, x.ld, x.off + j0 + (int64_t)J0 * x.ld,
                                   x.off + j0 + (int64_t)J0 * x.ld, x.off + j0 + (int64_t)j0 * x.ld});
          if (flops) *flops += 2.0 * rem0 * jb * (j0 - J0);
        }
        DiagDesc g;
        g.blk = x.off + j0 + (int64_t)j0 * x.ld;
        g.zblk = zbase ? x.zoff + (int64_t)(j0 - x.c0) * (x.zld + 1) : -1;
        g.scratch = (int64_t)i * kNB * kNB;
        g.ld = x.ld;
        g.zld = x.zld;
        g.jb = jb;
        g.id = x.id;
        g.col = j0;
        dg.push_back(g);
        const int r0 = j0 + jb, rem = x.n - r0;
        if (rem > 0) {
          panel.push_back(GemmDesc{rem, jb, jb, x.ld, kNB, x.ld, x.off + r0 + (int64_t)j0 * x.ld, (int64_t)i * kNB * kNB,
                                   x.off + r0 + (int64_t)j0 * x.ld});
          if (flops) *flops += (double)rem * jb * jb;
        }
        if (flops) *flops += (double)jb * jb * jb / 3.0;
      }
      if (dg.empty()) continue;
      // FP64 form: the strips and panels (C = A B^T, both operands in
      // column form; the diagonal inverse is stored with its zero upper
      // triangle) from exact slice products on the tensor cores.  (In the
      // FP32 form the SIMT tiles are faster at these 64-column widths than
      // the 128-wide 3xTF32 tiles with their split passes: 116 against
      // 127 ms for the 48^3 factorizations.)
      auto to_tc = [](const std::vector<GemmDesc>& g) {
        std::vector<TcGemm> t;
        t.reserve(g.size());
        for (const auto& x : g) t.push_back(TcGemm{x.a, x.b, x.c, x.lda, x.ldb, x.ldc, x.m, x.n, x.k, 0, 0, 0});
        return t;
      };
      if (!strip.empty()) {
        if constexpr (std::is_same<T, double>::value)
          tc_gemm_f64(st, ring, to_tc(strip), -1.0, 1.0, base, base, base, status);
        else
          gemm_batched<T>(st, ring, strip, G_TRANS_B, T(-1), T(1), base, base, base);
      }
      const DiagDesc* ddev = static_cast<const DiagDesc*>(ring.push(dg.data(), dg.size() * sizeof(DiagDesc), st));
      k_chol_diag<T><<<(unsigned)dg.size(), 256, 0, st>>>(ddev, base, zbase, scratch, status);
      AMB_LAUNCHED();
      if (!panel.empty()) {
        if constexpr (std::is_same<T, double>::value)
          tc_gemm_f64(st, ring, to_tc(panel), 1.0, 0.0, base, scratch, base, status);
        else
          gemm_batched<T>(st, ring, panel, G_TRANS_B | G_TRI_B_UPPER, T(1), T(0), base, scratch, base);
      }
    }
    // trailing update with the whole outer block: C(lower) -= P P^T
    std::vector<GemmDesc> trail;
    for (const auto& x : d) {
      const int J0 = x.c0 + ob * kOuter;
      if (J0 >= x.c1) continue;
      const int J1 = std::min(J0 + kOuter, x.c1);
      const int rem = x.n - J1;
      if (rem <= 0) continue;
      trail.push_back(GemmDesc{rem, rem, J1 - J0, x.ld, x.ld, x.ld, x.off + J1 + (int64_t)J0 * x.ld,
                               x.off + J1 + (int64_t)J0 * x.ld, x.off + J1 + (int64_t)J1 * x.ld});
      if (flops) *flops += (double)rem * (rem + 1) * (J1 - J0);
    }
    if (trail.empty()) continue;
    // on the tensor cores: 3xTF32 (FP32 accuracy) in the FP32 form, exact
    // slice products (FP64 accuracy) in the FP64 form
    std::vector<TcSyrk> tc;
    tc.reserve(trail.size());
    double tfl = 0.0;
    for (const auto& g : trail) {
      tc.push_back(TcSyrk{g.a, g.c, g.lda, g.m, g.k, 0});
      tfl += (double)g.m * (g.m + 1) * g.k;
    }
    auto run = [&] {
      if constexpr (std::is_same<T, float>::value)
        tc_syrk_lower(st, ring, tc, -1.f, 1.f, base, status);
      else
        tc_syrk_lower_f64(st, ring, tc, -1.0, 1.0, base, status);
    };
    if (tm) {
      FamTimer ft(st, tm, AMB_FAM_TC, timing);
      run();
      tm->fam_flops[AMB_FAM_TC] += tfl;
    } else {
      run();
    }
  }
}

template void partial_cholesky<float>(cudaStream_t, DescRing&, const std::vector<CholDesc>&, float*, float*, int*, double*,
                                       Timers*, bool);
template void partial_cholesky<double>(cudaStream_t, DescRing&, const std::vector<CholDesc>&, double*, double*, int*, double*,
                                        Timers*, bool);

// ------------------------------------------------------------------ TRTRI
// [L11 0; L21 L22]^{-1} = [Z11 0; -Z22 L21 Z11, Z22], merged bottom-up from
// the nb x nb diagonal inverses.  The upper block Z12 (unused by a lower
// inverse) holds the intermediate (L21 Z11)^T.

template <typename T>
void trtri_from_blocks(cudaStream_t st, DescRing& ring, const std::vector<TrtriDesc>& d, const T* lbase,
                       T* zbase, double* flops, int* status) {
  int maxn = 0;
  for (const auto& x : d) maxn = std::max(maxn, x.n);
  for (int half = kNB; half < maxn; half *= 2) {
    const int b = 2 * half;
    std::vector<GemmDesc> sa, sb;
    std::vector<TcGemm> ta, tb;
    // on the tensor cores: FP32-form merges with K >= the chunk width as 3xTF32
    // products (K in chunks, accumulated in FP32 through C), every FP64-form
    // merge from exact slice products (K in chunks, accumulated in FP64)
    const bool tc = std::is_same<T, float>::value ? half >= kTcKMax : true;
    for (const auto& x : d) {
      for (int p0 = 0; p0 + half < x.n; p0 += b) {
        const int h = p0 + half;
        const int r2 = std::min(p0 + b, x.n) - h;
        const int c1 = half;
        if (tc) {
          // Z12(i, j) = sum_k Z11(k, i) L21(j, k): A = Z11^T (K-major reads of Z11, upper), B = L21 (column form)
          ta.push_back(TcGemm{x.z + p0 + (int64_t)p0 * x.zld, x.l + h + (int64_t)p0 * x.ld, x.z + p0 + (int64_t)h * x.zld,
                              x.zld, x.ld, x.zld, c1, r2, c1, 1, 0, 2});
          // Z21(i, j) = -sum_k Z22(i, k) Z12(j, k): A = Z22 (lower), B = Z12 (column form)
          tb.push_back(TcGemm{x.z + h + (int64_t)h * x.zld, x.z + p0 + (int64_t)h * x.zld, x.z + h + (int64_t)p0 * x.zld,
                              x.zld, x.zld, x.zld, r2, c1, r2, 0, 0, 1});
        } else {
          // Z12 (c1 x r2) := Z11^T (upper) * L21^T
          sa.push_back(GemmDesc{c1, r2, c1, x.zld, x.ld, x.zld, x.z + p0 + (int64_t)p0 * x.zld,
                                x.l + h + (int64_t)p0 * x.ld, x.z + p0 + (int64_t)h * x.zld});
          // Z21 (r2 x c1) := -Z22 (lower) * Z12^T
          sb.push_back(GemmDesc{r2, c1, r2, x.zld, x.zld, x.zld, x.z + h + (int64_t)h * x.zld,
                                x.z + p0 + (int64_t)h * x.zld, x.z + h + (int64_t)p0 * x.zld});
        }
        if (flops) *flops += (double)c1 * c1 * r2 + (double)r2 * r2 * c1;
      }
    }
    if (tc) {
      if (ta.empty()) continue;
      if constexpr (std::is_same<T, float>::value) {
        tc_gemm(st, ring, ta, 1.f, 0.f, zbase, lbase, zbase, status);
        tc_gemm(st, ring, tb, -1.f, 0.f, zbase, zbase, zbase, status);
      } else {
        tc_gemm_f64(st, ring, ta, 1.0, 0.0, zbase, lbase, zbase, status);
        tc_gemm_f64(st, ring, tb, -1.0, 0.0, zbase, zbase, zbase, status);
      }
      continue;
    }
    if (sa.empty()) continue;
    gemm_batched<T>(st, ring, sa, G_TRANS_A | G_TRI_A_UPPER | G_TRANS_B | G_TUNE, T(1), T(0), zbase, lbase, zbase);
    gemm_batched<T>(st, ring, sb, G_TRI_A_LOWER | G_TRANS_B | G_TUNE, T(-1), T(0), zbase, zbase, zbase);
  }
}

template void trtri_from_blocks<float>(cudaStream_t, DescRing&, const std::vector<TrtriDesc>&, const float*, float*, double*,
                                        int*);
template void trtri_from_blocks<double>(cudaStream_t, DescRing&, const std::vector<TrtriDesc>&, const double*, double*,
                                         double*, int*);

}  // namespace amb
