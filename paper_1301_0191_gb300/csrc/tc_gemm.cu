// Dense products of the FP32 form on the 5th-generation tensor cores:
//
// - the trailing update of the blocked Cholesky (Sec. 2: A_II = L L^T and,
//   through the same elimination, S = K_GG - X^T X),
//     C(lower) = beta C + alpha P P^T,   P = rem x K (K <= 256);
// - general products C = beta C + alpha A B^T with an optionally triangular
//   A (the merges of the explicit triangular inverses), K taken in chunks of
//   256 whose partial products are added into C in FP32.
//
// Both in FP32 accuracy from three TF32 products (P = P_h + P_l, both
// TF32-exact: P P^T ~ P_h P_h^T + P_h P_l^T + P_l P_h^T, the P_l P_l^T term
// is below FP32 rounding).  A split pass writes the operands' high and low
// parts row-major (K contiguous, the K-major operand layout of tcgen05.mma
// kind::tf32) into a workspace slab, rows padded to a multiple of 128 and K
// to a multiple of 32 with zeros (entries outside a triangular operand's
// triangle are zero too); a row tile of a triangular A runs only over the
// K blocks that hold its entries.
//
// The tile kernel is persistent (one CTA per SM, 128 x 128 output tiles
// taken round-robin) and warp-specialized: warp 0 loads 128 x 32 operand
// tiles with TMA (128-byte swizzle) into a 3-stage shared-memory ring, warp 1
// owns the TMEM accumulators and issues the MMAs (one thread), and warps 2-5
// drain the accumulators with tcgen05.ld (lane = row), hand TMEM back to the
// MMA warp and then update C, so the next tile's MMAs overlap the epilogue's
// C traffic.  The C update goes 64 columns at a time (all loads, then all
// stores) with addresses formed by increments: with the 128 accumulator
// registers live, per-column 64-bit offsets spilled and made the update
// 2.3x slower.  Stage hand-offs use mbarriers: TMA completion (expect_tx),
// MMA completion (tcgen05.commit), TMEM full / TMEM empty.
//
// Accuracy: the tensor cores' FP32 accumulation rounds toward zero, so a
// single accumulator collecting all three products drifts on sums of like
// sign (the diagonal of P P^T): about 10x the error of an FP32 FMA chain at
// K = 256.  The K = 8 steps of P_h P_h^T therefore rotate over three TMEM
// accumulators, the small cross terms go to a fourth, and the epilogue adds
// the four with round-to-nearest; measured against exact sums this is as
// accurate as an FP32 FMA chain (rms 2.4e-8 vs 2.8e-8 relative to sum |terms|
// for random signs, 4.0e-7 vs 2.5e-7 for positive terms, K = 256).  Every wait
// is bounded: a wait that runs out sets AMB_ETIMEOUT in the status word and
// raises a CTA-wide abort flag; every role then leaves its loop, the TMA
// copies and MMAs already started are waited for (bounded again), and TMEM
// is released.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <unordered_map>

#include "common.h"
#include "oz_arith.h"
#include "tc_gemm.h"

namespace amb {

namespace {

constexpr int kTM = 128, kTN = 128, kTK = 32, kStages = 3;
constexpr int kTileBytes = kTM * kTK * 4;        // one operand tile (16 KB)
constexpr int kStageBytes = 4 * kTileBytes;      // A_h, A_l, B_h, B_l
constexpr int kSmemBytes = kStages * kStageBytes + 1024;
constexpr int kAccCols = 4 * kTN;                  // three P_h P_h^T accumulators + one for the cross terms
constexpr long kSpinLimit = 1L << 22;            // polls per wait (~0.5 s with backoff)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void mma_tf32(uint32_t tacc, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tacc),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// source block (rows x cols; column form: (r, k) at src + r + k*ld, K-major
// form: src + k + r*ld) -> slab rows [row0, row0 + rpad), K-contiguous,
// stride kp; entries outside rows x cols or outside the triangle are zero.
// A CTA moves a 128-row x 32-column tile through shared memory: the reads
// are coalesced along the source's contiguous direction, and each thread
// writes four consecutive K values of one slab row with a 16-byte store
// (slab rows are 1 KB apart, K blocks 128 B).
constexpr int kSplitRows = 128;

__global__ void __launch_bounds__(256) k_tc_split(const TcSplitDesc* d, int kp, float* sh, float* sl) {
  __shared__ float t[32][kSplitRows + 1];   // [k][r]
  const TcSplitDesc x = d[blockIdx.z];
  const int r0 = blockIdx.x * kSplitRows, k0 = blockIdx.y * 32;
  if (r0 >= x.rpad || k0 >= kp) return;
  const int tid = threadIdx.x;
  if (x.kmajor) {
    // lane = k: 32 consecutive k of one row per warp instruction
    const int k = k0 + (tid & 31);
    for (int rr = tid >> 5; rr < kSplitRows; rr += 8) {
      const int r = r0 + rr;
      bool ok = r < x.rows && k < x.cols;
      if (x.tri == 1 && k - r > x.diag) ok = false;
      if (x.tri == 2 && k - r < x.diag) ok = false;
      t[tid & 31][rr] = ok ? x.src[k + (int64_t)r * x.ld] : 0.f;
    }
  } else {
    // lane = row: 128 consecutive rows of one column per 4 warp instructions
    for (int idx = tid; idx < 32 * kSplitRows; idx += 256) {
      const int rr = idx % kSplitRows, kk = idx / kSplitRows;
      const int r = r0 + rr, k = k0 + kk;
      bool ok = r < x.rows && k < x.cols;
      if (x.tri == 1 && k - r > x.diag) ok = false;
      if (x.tri == 2 && k - r < x.diag) ok = false;
      t[kk][rr] = ok ? x.src[r + (int64_t)k * x.ld] : 0.f;
    }
  }
  __syncthreads();
  // 128 rows x 8 groups of 4 k: thread -> (row, k group)
  for (int idx = tid; idx < kSplitRows * 8; idx += 256) {
    const int g = idx & 7, rr = idx >> 3;
    float4 h, l;
    float v = t[4 * g + 0][rr];
    h.x = tf32_round(v);
    l.x = tf32_round(v - h.x);
    v = t[4 * g + 1][rr];
    h.y = tf32_round(v);
    l.y = tf32_round(v - h.y);
    v = t[4 * g + 2][rr];
    h.z = tf32_round(v);
    l.z = tf32_round(v - h.z);
    v = t[4 * g + 3][rr];
    h.w = tf32_round(v);
    l.w = tf32_round(v - h.w);
    const int64_t o = (x.row0 + r0 + rr) * (int64_t)kp + k0 + 4 * g;
    *reinterpret_cast<float4*>(sh + o) = h;
    *reinterpret_cast<float4*>(sl + o) = l;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// shared-memory descriptor of a K-major tile written by TMA with 128-byte
// swizzle: 8 rows x 128 B swizzle atoms, 1024 B between 8-row groups
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// bounded wait that also gives up when another role has aborted.  try_wait
// itself suspends the thread for a while before it reports false, so the
// loop polls without sleeping for its first 4096 rounds (a sleep can
// overshoot by microseconds, which the single MMA-issuing thread cannot
// afford between pipeline stages) and backs off only after that.
__device__ __forceinline__ bool role_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  for (long it = 0; it < kSpinLimit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (it > 4096) __nanosleep(64);
  }
  *abort_flag = 1;
  if (status) atomicCAS(status, 0, AMB_ETIMEOUT);
  return false;
}

// bounded wait without the abort test, for the drain after an abort
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity, int* status) {
  for (long it = 0; it < kSpinLimit; ++it) {
    if (mbar_try(bar, parity)) return;
    if (it > 4096) __nanosleep(64);
  }
  if (status) atomicCAS(status, 0, AMB_ETIMEOUT);
}

// After an abort the CTA must not exit while TMA copies it started still
// write its shared memory: wait for the last phase the producer started on
// each of the n stage barriers (issued loads so far; load i went to stage
// i % n as its use i / n).
__device__ __forceinline__ void drain_loads(const uint64_t* full, int n, uint32_t issued, int* status) {
  for (int s = 0; s < n; ++s)
    if (issued > (uint32_t)s) drain_wait(smem_u32(&full[s]), ((issued - 1 - (uint32_t)s) / (uint32_t)n) & 1u, status);
}

// ... nor while MMAs it issued still run: one more commit, to its own
// barrier, arrives once all of them have completed
__device__ __forceinline__ void drain_mmas(uint64_t* done, int* status) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(done))
               : "memory");
  drain_wait(smem_u32(done), 0, status);
}

__device__ __forceinline__ void tile_coords(const TcTileArgs& g, int tile, TcDesc& d, int& ti, int& tj) {
  int lo = 0, hi = g.ndesc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g.prefix[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  d = g.desc[lo];
  const int t = tile - g.prefix[lo];
  if (d.lower) {
    ti = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    tj = t - ti * (ti + 1) / 2;
  } else {
    const int tn = (d.n + kTN - 1) / kTN;
    ti = t / tn;
    tj = t % tn;
  }
}

// K blocks [kb, ke) of a tile: a triangular A has no entries in part of the
// chunk for a given row block
__device__ __forceinline__ void tile_krange(const TcDesc& d, int ti, int& kb, int& ke) {
  kb = 0;
  ke = d.k / kTK;
  const int ib = d.ioff + ti * kTM;   // global row - chunk k of the tile's first row
  if (d.tri == 1) ke = min(ke, max(0, (ib + kTM + kTK - 1) / kTK));
  if (d.tri == 2) kb = max(kb, ib / kTK);
  if (kb > ke) kb = ke;
}

__global__ void __launch_bounds__(192, 1) k_tc_syrk(const __grid_constant__ CUtensorMap map_h,
                                                   const __grid_constant__ CUtensorMap map_l, TcTileArgs g) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], tfull, tempty, mdone;
  __shared__ uint32_t tbase;
  __shared__ volatile int abort_sh;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                 "r"(kAccCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(1) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])), "r"(1) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tfull)), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tempty)), "r"(4) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mdone)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_h) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_l) : "memory");
    abort_sh = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tacc = tbase;
  const int ntiles = g.prefix[g.ndesc];

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      uint32_t it = 0;
      for (int tile = blockIdx.x; tile < ntiles && !abort_sh; tile += gridDim.x) {
        TcDesc d;
        int ti, tj;
        tile_coords(g, tile, d, ti, tj);
        const int ya = (int)(d.arow + (int64_t)ti * kTM), yb = (int)(d.brow + (int64_t)tj * kTN);
        int kb, ke;
        tile_krange(d, ti, kb, ke);
        for (int kt = kb; kt < ke; ++kt, ++it) {
          const int s = it % kStages;
          if (!role_wait(smem_u32(&empty[s]), ((it / kStages) & 1) ^ 1, &abort_sh, g.status)) break;
          const uint32_t sb = smem_u32(smem + s * kStageBytes), fb = smem_u32(&full[s]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kStageBytes) : "memory");
          tma_load_2d(sb, &map_h, kt * kTK, ya, fb);
          tma_load_2d(sb + kTileBytes, &map_l, kt * kTK, ya, fb);
          tma_load_2d(sb + 2 * kTileBytes, &map_h, kt * kTK, yb, fb);
          tma_load_2d(sb + 3 * kTileBytes, &map_l, kt * kTK, yb, fb);
        }
      }
      if (abort_sh) drain_loads(full, kStages, it, g.status);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t it = 0, tl = 0;
      for (int tile = blockIdx.x; tile < ntiles && !abort_sh; tile += gridDim.x, ++tl) {
        TcDesc d;
        int ti, tj;
        tile_coords(g, tile, d, ti, tj);
        int kb, ke;
        tile_krange(d, ti, kb, ke);
        if (!role_wait(smem_u32(&tempty), (tl & 1) ^ 1, &abort_sh, g.status)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int kt = kb; kt < ke; ++kt, ++it) {
          const int s = it % kStages;
          if (!role_wait(smem_u32(&full[s]), (it / kStages) & 1, &abort_sh, g.status)) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sb = smem_u32(smem + s * kStageBytes);
#pragma unroll
          for (int kk = 0; kk < kTK / 8; ++kk) {
            const uint32_t ko = kk * 32;   // K = 8 per MMA: 32 bytes along the swizzled row
            const uint64_t dah = smem_desc_sw128(sb + ko), dal = smem_desc_sw128(sb + kTileBytes + ko);
            const uint64_t dbh = smem_desc_sw128(sb + 2 * kTileBytes + ko), dbl = smem_desc_sw128(sb + 3 * kTileBytes + ko);
            const int step = (kt - kb) * (kTK / 8) + kk;
            mma_tf32(tacc + (uint32_t)((step % 3) * kTN), dah, dbh, step >= 3 ? 1u : 0u);
            mma_tf32(tacc + (uint32_t)(3 * kTN), dah, dbl, step >= 1 ? 1u : 0u);
            mma_tf32(tacc + (uint32_t)(3 * kTN), dal, dbh, 1u);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&empty[s]))
                       : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&tfull))
                     : "memory");
      }
      if (abort_sh) drain_mmas(&mdone, g.status);
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 2..5)
    const int quad = warp & 3;   // TMEM lanes 32*quad .. 32*quad + 31
    uint32_t tl = 0;
    for (int tile = blockIdx.x; tile < ntiles && !abort_sh; tile += gridDim.x, ++tl) {
      TcDesc d;
      int ti, tj;
      tile_coords(g, tile, d, ti, tj);
      int kb, ke;
      tile_krange(d, ti, kb, ke);
      const int nsteps = (ke - kb) * (kTK / 8);
      if (!role_wait(smem_u32(&tfull), tl & 1, &abort_sh, g.status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float acc[kTN];
      // drain: per 16-column slice, the four accumulators' loads go out together, one wait
#pragma unroll
      for (int h = 0; h < kTN / 16; ++h) {
        uint32_t r[4][16];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const uint32_t ta = tacc + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * kTN + h * 16);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(r[a][0]), "=r"(r[a][1]), "=r"(r[a][2]), "=r"(r[a][3]), "=r"(r[a][4]), "=r"(r[a][5]),
                "=r"(r[a][6]), "=r"(r[a][7]), "=r"(r[a][8]), "=r"(r[a][9]), "=r"(r[a][10]), "=r"(r[a][11]),
                "=r"(r[a][12]), "=r"(r[a][13]), "=r"(r[a][14]), "=r"(r[a][15])
              : "r"(ta));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // accumulators not yet written (fewer than three K = 8 steps) hold no data
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          float v = 0.f;
          if (nsteps > 0) v = __uint_as_float(r[3][q]) + __uint_as_float(r[0][q]);
          if (nsteps > 1) v += __uint_as_float(r[1][q]);
          if (nsteps > 2) v += __uint_as_float(r[2][q]);
          acc[h * 16 + q] = v;
        }
      }
      // TMEM back to the MMA warp before the C traffic
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty)) : "memory");
      const int i = ti * kTM + quad * 32 + lane;   // row of C within the product
      const float beta = d.first ? g.beta : 1.f;
      if (i < d.m) {
        // 64 columns at a time: the loads first, then the stores; addresses
        // by increments so that no per-column 64-bit offsets stay live
        const int64_t ldc = d.ldc;
        const int jlast = min(d.n, d.lower ? i + 1 : d.n) - 1;   // last column this row updates
        float* const p0 = g.c + d.c + i + (int64_t)tj * kTN * ldc;
#pragma unroll
        for (int cb = 0; cb < kTN / 64; ++cb) {
          const int j0 = tj * kTN + cb * 64;
          float cv[64];
          const float* p = p0 + (int64_t)cb * 64 * ldc;
#pragma unroll
          for (int q = 0; q < 64; ++q) {
            cv[q] = (j0 + q <= jlast && beta != 0.f) ? __ldcg(p) : 0.f;
            p += ldc;
          }
          float* o = p0 + (int64_t)cb * 64 * ldc;
#pragma unroll
          for (int q = 0; q < 64; ++q) {
            if (j0 + q <= jlast) *o = fmaf(beta, cv[q], g.alpha * acc[cb * 64 + q]);
            o += ldc;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tacc), "r"(kAccCols) : "memory");
}

// ---------------------------------------------------------------- FP64 form: exact slice products
//
// C = beta C + alpha A B^T in FP64 accuracy on the TF32 tensor cores (the
// Cholesky trailing updates, C lower and B = A; the Cholesky strips and
// panels; the triangular-inverse merges; the LOBPCG B products and the
// triangular products of the pair preconditioner).  The integer arithmetic
// is in oz_arith.h.  Every row r of an operand chunk (K <= 256) is scaled by 2^-e_r,
// e_r the exponent of its largest entry (|X(r, k)| < 2^e_r), rounded to the
// 56-bit integer F = X(r, k) 2^(56 - e_r) and written in balanced base-128
// digits: X(r, k) = 2^e_r sum_p m_p 2^-7(p+1) up to 2^-57 of 2^e_r, with
// |m_0| <= 128 and |m_p| <= 64 for p >= 1 (integer arithmetic only).  These small
// integers are exact in TF32 and so are their products; the products of
// slices p and q with p + q = l go to TMEM accumulator l.  Per K step a
// level collects at most 2^14 + (l - 1) 2^12 (l >= 1) or 2^14 (l = 0), so
// over K = 256 every partial sum is an integer below 10 * 2^20 < 2^24: exact
// in the FP32 accumulator whatever its rounding mode.  Products with
// p + q >= kOzSlices are dropped (below 2^-49 of 2^(e_i + e_j) each).  The
// epilogue forms sum_l L_l 2^(7 (7 - l)) as an exact integer and rounds
// it times 2^(e_i + e_j - 63) to FP64 once; the C update is one FP64 FMA.
//
// Tiles are 128 x 64 (M x N): the eight accumulators of a tile fill the 512
// TMEM columns.  Per K step of 32 the B rows of all slices (8 x 8 KB) sit in
// one of two B buffers, and the A rows of one slice at a time (16 KB) in one
// of four A stages: each slice tile is read from L2 once per K step.

constexpr int kOzTN = 64, kOzBBufs = 2, kOzAStages = 4;
constexpr int kOzATile = kTM * kTK * 4;                     // 16 KB
constexpr int kOzBTile = kOzTN * kTK * 4;                   // 8 KB
constexpr int kOzBBytes = kOzSlices * kOzBTile;             // 64 KB
constexpr int kOzSmemBytes = kOzBBufs * kOzBBytes + kOzAStages * kOzATile + 1024;
static_assert(kOzSlices * kOzTN <= 512, "the level accumulators must fit TMEM");
static_assert(kOzSlices == oz::kSlices, "one digit count for the split and the products");
static_assert(kOzSmemBytes <= 227 * 1024, "shared memory");

// kind::tf32 instruction descriptor for M = 128 and N columns
__host__ __device__ constexpr uint32_t oz_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32_idesc(uint32_t tacc, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tacc),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// FP64 source block (rows x cols; column form: (r, k) at src + r + k*ld,
// K-major form: src + k + r*ld; triangle masks as in the FP32 split) -> the
// slices of slab rows [row0, row0 + rpad) (slice p at slab row p * R + row),
// K contiguous with stride kp, and the row exponents ex[row].  A CTA takes
// 128 rows through shared memory in 32-column tiles (reads coalesced along
// the source's contiguous direction) twice: once for the row maxima, once
// to cut the slices; eight threads write one slab row's 128 bytes per slice.
__device__ __forceinline__ void oz_load_tile(const TcSplitDesc& x, int r0, int k0, int tid, double (*t)[kSplitRows + 1]) {
  const double* src = reinterpret_cast<const double*>(x.src);
  if (x.kmajor) {
    const int k = k0 + (tid & 31);
    for (int rr = tid >> 5; rr < kSplitRows; rr += 8) {
      const int r = r0 + rr;
      bool ok = r < x.rows && k < x.cols;
      if (x.tri == 1 && k - r > x.diag) ok = false;
      if (x.tri == 2 && k - r < x.diag) ok = false;
      t[tid & 31][rr] = ok ? src[k + (int64_t)r * x.ld] : 0.0;
    }
  } else {
    for (int idx = tid; idx < 32 * kSplitRows; idx += 256) {
      const int rr = idx % kSplitRows, kk = idx / kSplitRows;
      const int r = r0 + rr, k = k0 + kk;
      bool ok = r < x.rows && k < x.cols;
      if (x.tri == 1 && k - r > x.diag) ok = false;
      if (x.tri == 2 && k - r < x.diag) ok = false;
      t[kk][rr] = ok ? src[r + (int64_t)k * x.ld] : 0.0;
    }
  }
}

__global__ void __launch_bounds__(256) k_oz_split(const TcSplitDesc* d, int kp, int64_t R, float* slab, int* ex) {
  __shared__ double t[32][kSplitRows + 1];   // [k][r]
  __shared__ int esh[kSplitRows];
  const TcSplitDesc x = d[blockIdx.y];
  const int r0 = blockIdx.x * kSplitRows;
  if (r0 >= x.rpad) return;
  const int tid = threadIdx.x;
  const int kc = (x.cols + kTK - 1) / kTK * kTK;   // the K range the tiles read
  uint64_t mx = 0;
  for (int k0 = 0; k0 < kc; k0 += 32) {
    oz_load_tile(x, r0, k0, tid, t);
    __syncthreads();
    if (tid < kSplitRows)
      for (int kk = 0; kk < 32; ++kk) mx = max(mx, oz::absbits(t[kk][tid]));
    __syncthreads();
  }
  if (tid < kSplitRows) {
    const int e = mx ? oz::exponent(mx) : 0;
    esh[tid] = e;
    ex[x.row0 + r0 + tid] = e;
  }
  __syncthreads();
  for (int k0 = 0; k0 < kc; k0 += 32) {
    oz_load_tile(x, r0, k0, tid, t);
    __syncthreads();
    // 128 rows x 8 groups of 4 k: thread -> (row, k group)
    for (int idx = tid; idx < kSplitRows * 8; idx += 256) {
      const int g = idx & 7, rr = idx >> 3;
      const int e = esh[rr];
      float sl[4][kOzSlices];
#pragma unroll
      for (int u = 0; u < 4; ++u) oz::digits(t[4 * g + u][rr], e, sl[u]);
#pragma unroll
      for (int p = 0; p < kOzSlices; ++p)
        *reinterpret_cast<float4*>(slab + (p * R + x.row0 + r0 + rr) * (int64_t)kp + k0 + 4 * g) =
            make_float4(sl[0][p], sl[1][p], sl[2][p], sl[3][p]);
    }
    __syncthreads();
  }
}

// tile t of a descriptor: lower (square C, 128 x 64 tiles, row tile ti has
// min(2 ti + 2, tn) column tiles) or dense (row-major over tm x tn tiles)
__device__ __forceinline__ void oz_tile(const TcTileArgs& g, int tile, TcDesc& d, int& ti, int& tj) {
  int lo = 0, hi = g.ndesc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g.prefix[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  d = g.desc[lo];
  const int t = tile - g.prefix[lo];
  if (d.lower) {
    ti = (int)((sqrtf(4.f * t + 1.f) - 1.f) * 0.5f);
    while (ti * (ti + 1) > t) --ti;
    while ((ti + 1) * (ti + 2) <= t) ++ti;
    tj = t - ti * (ti + 1);
  } else {
    const int tn = (d.n + kOzTN - 1) / kOzTN;
    ti = t / tn;
    tj = t % tn;
  }
}

struct OzArgs {
  const TcDesc* desc;
  const int* prefix;
  int ndesc;
  int64_t R;
  double alpha, beta;
  double* c;
  const int* ex;
  int* status;
};

__global__ void __launch_bounds__(192, 1) k_oz_gemm(const __grid_constant__ CUtensorMap map_a,
                                                   const __grid_constant__ CUtensorMap map_b, OzArgs ga) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bfull[kOzBBufs], bempty[kOzBBufs], afull[kOzAStages], aempty[kOzAStages], tfull,
      tempty, mdone;
  __shared__ uint32_t tbase;
  __shared__ volatile int abort_sh;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  TcTileArgs g;
  g.desc = ga.desc;
  g.prefix = ga.prefix;
  g.ndesc = ga.ndesc;
  g.status = ga.status;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kOzBBufs; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bfull[s])), "r"(1) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bempty[s])), "r"(1) : "memory");
    }
    for (int s = 0; s < kOzAStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&afull[s])), "r"(1) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&aempty[s])), "r"(1) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tfull)), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tempty)), "r"(4) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mdone)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_a) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map_b) : "memory");
    abort_sh = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tacc = tbase;
  const int ntiles = g.prefix[g.ndesc];
  const int64_t R = ga.R;

  uint8_t* const bbuf = smem;
  uint8_t* const abuf = smem + kOzBBufs * kOzBBytes;
  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      uint32_t ib = 0, ia = 0;
      for (int tile = blockIdx.x; tile < ntiles && !abort_sh; tile += gridDim.x) {
        TcDesc d;
        int ti, tj;
        oz_tile(g, tile, d, ti, tj);
        const int64_t ya = d.arow + (int64_t)ti * kTM, yb = d.brow + (int64_t)tj * kOzTN;
        int kb, ke;
        tile_krange(d, ti, kb, ke);
        bool ok = true;
        for (int kt = kb; kt < ke && ok; ++kt, ++ib) {
          const int sb = ib % kOzBBufs;
          if (!role_wait(smem_u32(&bempty[sb]), ((ib / kOzBBufs) & 1) ^ 1, &abort_sh, g.status)) break;
          const uint32_t bdst = smem_u32(bbuf + sb * kOzBBytes), bfb = smem_u32(&bfull[sb]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bfb), "r"(kOzBBytes) : "memory");
          for (int q = 0; q < kOzSlices; ++q) tma_load_2d(bdst + q * kOzBTile, &map_b, kt * kTK, (int)(q * R + yb), bfb);
          for (int p = 0; p < kOzSlices; ++p, ++ia) {
            const int sa = ia % kOzAStages;
            if (!role_wait(smem_u32(&aempty[sa]), ((ia / kOzAStages) & 1) ^ 1, &abort_sh, g.status)) {
              ok = false;
              break;
            }
            const uint32_t afb = smem_u32(&afull[sa]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(afb), "r"(kOzATile) : "memory");
            tma_load_2d(smem_u32(abuf + sa * kOzATile), &map_a, kt * kTK, (int)(p * R + ya), afb);
          }
        }
      }
      if (abort_sh) {
        drain_loads(bfull, kOzBBufs, ib, g.status);
        drain_loads(afull, kOzAStages, ia, g.status);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t ib = 0, ia = 0, tl = 0;
      for (int tile = blockIdx.x; tile < ntiles && !abort_sh; tile += gridDim.x, ++tl) {
        TcDesc d;
        int ti, tj;
        oz_tile(g, tile, d, ti, tj);
        int kb, ke;
        tile_krange(d, ti, kb, ke);
        if (!role_wait(smem_u32(&tempty), (tl & 1) ^ 1, &abort_sh, g.status)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        bool ok = true;
        for (int kt = kb; kt < ke && ok; ++kt, ++ib) {
          const int sb = ib % kOzBBufs;
          if (!role_wait(smem_u32(&bfull[sb]), (ib / kOzBBufs) & 1, &abort_sh, g.status)) break;
          // descriptors advance by (byte offset >> 4) in their address field:
          // a slice tile is kOzBTile bytes, a K step of 8 is 32 bytes
          const uint64_t db0 = smem_desc_sw128(smem_u32(bbuf + sb * kOzBBytes));
          const uint32_t first = kt > kb ? 1u : 0u;
#pragma unroll
          for (int p = 0; p < kOzSlices; ++p) {
            const int sa = (int)((ia + p) % kOzAStages);
            if (!role_wait(smem_u32(&afull[sa]), ((ia + p) / kOzAStages) & 1, &abort_sh, g.status)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da0 = smem_desc_sw128(smem_u32(abuf + sa * kOzATile));
            // The B slices sit one after another in shared memory with the
            // same 8-row group stride, and level p + q of slice q's product
            // is TMEM column block p + q: so slices q = 0..3 (and 4..7-p)
            // go in one MMA of N = 64 x (their count), written to the
            // consecutive level blocks from p (and p + 4) on.  Level l is
            // started by the first product into it, p = 0 and kk = 0 of the
            // tile's first K step.
            const int nq = kOzSlices - p, n1 = nq < 4 ? nq : 4, n2 = nq - n1;
#pragma unroll
            for (int kk = 0; kk < kTK / 8; ++kk) {
              const uint32_t acc = (p > 0 || kk > 0) ? 1u : first;
              mma_tf32_idesc(tacc + (uint32_t)(p * kOzTN), da0 + (uint64_t)(kk * 2), db0 + (uint64_t)(kk * 2),
                             oz_idesc(n1 * kOzTN), acc);
              if (n2 > 0)
                mma_tf32_idesc(tacc + (uint32_t)((p + 4) * kOzTN), da0 + (uint64_t)(kk * 2),
                               db0 + (uint64_t)(4 * (kOzBTile >> 4) + kk * 2), oz_idesc(n2 * kOzTN), acc);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&aempty[sa]))
                         : "memory");
          }
          ia += kOzSlices;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&bempty[sb]))
                       : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&tfull))
                     : "memory");
      }
      if (abort_sh) drain_mmas(&mdone, g.status);
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 2..5)
    const int quad = warp & 3;   // TMEM lanes 32*quad .. 32*quad + 31
    uint32_t tl = 0;
    for (int tile = blockIdx.x; tile < ntiles && !abort_sh; tile += gridDim.x, ++tl) {
      TcDesc d;
      int ti, tj;
      oz_tile(g, tile, d, ti, tj);
      int kb, ke;
      tile_krange(d, ti, kb, ke);
      const int i = ti * kTM + quad * 32 + lane;   // row of C within the product
      const int jlast = min(d.n, d.lower ? i + 1 : d.n) - 1 - tj * kOzTN;   // last tile column this row updates
      const double beta = d.first ? ga.beta : 1.0;
      double* const crow = ga.c + d.c + i + (int64_t)tj * kOzTN * d.ldc;
      // C's lines into L2 while the tile's products run
      if (i < d.m && beta != 0.0)
        for (int q = 0; q <= min(jlast, kOzTN - 1); ++q)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(crow + (int64_t)q * d.ldc));
      const int ei = ga.ex[d.arow + i];
      if (!role_wait(smem_u32(&tfull), tl & 1, &abort_sh, g.status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      double v[kOzTN];
#pragma unroll
      for (int h = 0; h < kOzTN / 16; ++h) {
        // levels 0..3 -> H, levels 4..7 -> L: the product is (H 2^28 + L) 2^-63
        // in units of 2^(e_i + e_j), both parts exact in int64 (below 2^46)
        int64_t part[2][16];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          uint32_t r[4][16];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const uint32_t ta =
                tacc + ((uint32_t)(quad * 32) << 16) + (uint32_t)((half * 4 + a) * kOzTN + h * 16);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[a][0]), "=r"(r[a][1]), "=r"(r[a][2]), "=r"(r[a][3]), "=r"(r[a][4]), "=r"(r[a][5]),
                  "=r"(r[a][6]), "=r"(r[a][7]), "=r"(r[a][8]), "=r"(r[a][9]), "=r"(r[a][10]), "=r"(r[a][11]),
                  "=r"(r[a][12]), "=r"(r[a][13]), "=r"(r[a][14]), "=r"(r[a][15])
                : "r"(ta));
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            int64_t w = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a) w = w * 128 + (int64_t)__float2int_rn(__uint_as_float(r[a][q]));
            part[half][q] = w;
          }
        }
        int ej[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = tj * kOzTN + h * 16 + q;
          ej[q] = j < d.n ? __ldg(ga.ex + d.brow + j) : 0;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = tj * kOzTN + h * 16 + q;
          // a tile without K steps (a triangular operand with no entries in
          // this chunk) has no accumulator data: its product is zero
          v[h * 16 + q] = (kb < ke && j < d.n) ? oz::round_sum(part[0][q], part[1][q], ei + ej[q] - 63) : 0.0;
        }
      }
      // TMEM back to the MMA warp before the C traffic
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty)) : "memory");
      if (i < d.m) {
        // 16 columns at a time: the loads first, then the stores
#pragma unroll
        for (int cb = 0; cb < kOzTN / 16; ++cb) {
          double cv[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int jj = cb * 16 + q;
            cv[q] = (jj <= jlast && beta != 0.0) ? __ldcg(crow + (int64_t)jj * d.ldc) : 0.0;
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int jj = cb * 16 + q;
            if (jj <= jlast) crow[(int64_t)jj * d.ldc] = beta == 1.0 ? fma(ga.alpha, v[jj], cv[q])
                                                                     : fma(ga.alpha, v[jj], beta * cv[q]);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tacc), "r"(512) : "memory");
}

// cuTensorMapEncodeTiled through the runtime's driver entry point
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    AMB_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    AMB_CHECK(p != nullptr && q == cudaDriverEntryPointSuccess, AMB_ECUDA, "cuTensorMapEncodeTiled not available");
    return (EncodeTiledFn)p;
  }();
  return fn;
}

// 2-D map over a slab (rows x kp FP32, row-major) with box_rows x 32 boxes, 128-byte swizzle
CUtensorMap slab_map(float* base, int64_t rows, int kp, int box_rows = kTM) {
  CUtensorMap m;
  const cuuint64_t dim[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)kp * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)box_rows}, estr[2] = {1, 1};
  const CUresult r = encode_tiled()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dim, stride, box, estr,
                                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  AMB_CHECK(r == CUDA_SUCCESS, AMB_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

// workspace slab for the split operands, grown on demand
float* tc_slab(size_t floats) {
  check_workspace_device();
  static thread_local DevBuf buf;
  const size_t need = 2 * floats * sizeof(float);
  if (buf.bytes < need) {
    AMB_CUDA(cudaDeviceSynchronize());   // earlier launches may still read the old slab
    buf.alloc(need);
  }
  return dptr<float>(buf);
}

}  // namespace

int tc_tile_count(const TcDesc& x) {
  const int tm = (x.m + kTM - 1) / kTM;
  if (x.m <= 0 || x.n <= 0) return 0;
  if (x.lower) return tm * (tm + 1) / 2;
  return tm * ((x.n + kTN - 1) / kTN);
}

namespace {

// one split launch over sp, then one persistent tile launch over td
void run_tiles(cudaStream_t st, DescRing& ring, const std::vector<TcSplitDesc>& sp, const std::vector<TcDesc>& td,
               std::vector<int> prefix, int64_t rows, int maxr, int64_t tiles, float alpha, float beta, float* cbase,
               int* status) {
  static thread_local bool attr = false;
  if (!attr) {
    AMB_CUDA(cudaFuncSetAttribute(k_tc_syrk, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    attr = true;
  }
  constexpr int kp = kTcKMax;
  AMB_CHECK(tiles < (1LL << 31) && rows < (1LL << 31) && sp.size() < 65536, AMB_EINVAL,
            "tensor-core batch too large");
  prefix.push_back((int)tiles);
  std::vector<TcSplitDesc> spr(sp);
  float* sh = tc_slab((size_t)rows * kp);
  float* sl = sh + (size_t)rows * kp;
  const TcSplitDesc* dsp = static_cast<const TcSplitDesc*>(ring.push(spr.data(), spr.size() * sizeof(TcSplitDesc), st));
  static_assert(kTM % kSplitRows == 0, "slab row padding must cover whole split tiles");
  k_tc_split<<<dim3((unsigned)(maxr / kSplitRows), kp / 32, (unsigned)spr.size()), 256, 0, st>>>(dsp, kp, sh, sl);
  AMB_LAUNCHED();
  std::vector<char> blob(td.size() * sizeof(TcDesc) + prefix.size() * sizeof(int));
  memcpy(blob.data(), td.data(), td.size() * sizeof(TcDesc));
  memcpy(blob.data() + td.size() * sizeof(TcDesc), prefix.data(), prefix.size() * sizeof(int));
  char* dev = static_cast<char*>(ring.push(blob.data(), blob.size(), st));
  TcTileArgs g;
  g.desc = reinterpret_cast<const TcDesc*>(dev);
  g.prefix = reinterpret_cast<const int*>(dev + td.size() * sizeof(TcDesc));
  g.ndesc = (int)td.size();
  g.kp = kp;
  g.alpha = alpha;
  g.beta = beta;
  g.ah = sh;
  g.al = sl;
  g.bh = sh;
  g.bl = sl;
  g.c = cbase;
  g.status = status;
  static thread_local int nsm = 0;
  if (nsm == 0) {
    int devid = 0;
    AMB_CUDA(cudaGetDevice(&devid));
    AMB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, devid));
  }
  const CUtensorMap mh = slab_map(sh, rows, kp), ml = slab_map(sl, rows, kp);
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, nsm);
  k_tc_syrk<<<grid, 192, kSmemBytes, st>>>(mh, ml, g);
  AMB_LAUNCHED();
}

int pad_rows(int r) { return (r + kTM - 1) / kTM * kTM; }

}  // namespace

void tc_syrk_lower(cudaStream_t st, DescRing& ring, const std::vector<TcSyrk>& d, float alpha, float beta,
                   float* base, int* status) {
  if (d.empty()) return;
  constexpr int kp = kTcKMax;
  std::vector<TcSplitDesc> sp;
  std::vector<TcDesc> td;
  std::vector<int> prefix;
  int64_t rows = 0, tiles = 0;
  int maxr = 0;
  for (const auto& x : d) {
    AMB_CHECK(x.k >= 0 && x.k <= kp, AMB_EINVAL, "tensor-core trailing update with K above the slab width");
    if (x.rem <= 0 || x.k <= 0) continue;
    const int rpad = pad_rows(x.rem);
    sp.push_back(TcSplitDesc{base + x.p, rows, x.ld, x.rem, x.k, rpad, 0, 0, 0, 0});
    TcDesc t{x.c, rows, rows, x.rem, x.rem, (x.k + kTK - 1) / kTK * kTK, x.ld, 1, 0, 0, 1};
    prefix.push_back((int)tiles);
    tiles += tc_tile_count(t);
    td.push_back(t);
    rows += rpad;
    maxr = std::max(maxr, rpad);
  }
  if (td.empty()) return;
  run_tiles(st, ring, sp, td, prefix, rows, maxr, tiles, alpha, beta, base, status);
}

namespace {

int oz_tile_count(const TcDesc& x) {
  if (x.m <= 0 || x.n <= 0) return 0;
  const int tm = (x.m + kTM - 1) / kTM, tn = (x.n + kOzTN - 1) / kOzTN;
  if (x.lower) return tm * (tm + 1) - (2 * tm - tn);   // row tile ti holds min(2 ti + 2, tn) column tiles
  return tm * tn;
}

// one split launch over sp, then one persistent tile launch over td (FP64 data)
void run_oz(cudaStream_t st, DescRing& ring, const std::vector<TcSplitDesc>& sp, const std::vector<TcDesc>& td,
            std::vector<int> prefix, int64_t rows, int maxr, int64_t tiles, double alpha, double beta, double* cbase,
            int* status) {
  constexpr int kp = kTcKMax;
  AMB_CHECK(tiles < (1LL << 31) && rows * kOzSlices < (1LL << 31) && sp.size() < 65536, AMB_EINVAL,
            "tensor-core batch too large");
  static thread_local bool attr = false;
  if (!attr) {
    AMB_CUDA(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmemBytes));
    attr = true;
  }
  check_workspace_device();
  static thread_local DevBuf slab_buf, ex_buf;
  const size_t need = (size_t)kOzSlices * rows * kp * sizeof(float);
  if (slab_buf.bytes < need || ex_buf.bytes < (size_t)rows * sizeof(int)) {
    AMB_CUDA(cudaDeviceSynchronize());   // earlier launches may still read the old slab
    if (slab_buf.bytes < need) slab_buf.alloc(need);
    if (ex_buf.bytes < (size_t)rows * sizeof(int)) ex_buf.alloc((size_t)rows * sizeof(int));
  }
  float* slab = dptr<float>(slab_buf);
  int* ex = dptr<int>(ex_buf);
  prefix.push_back((int)tiles);
  const TcSplitDesc* dsp = static_cast<const TcSplitDesc*>(ring.push(sp.data(), sp.size() * sizeof(TcSplitDesc), st));
  static_assert(kTM % kSplitRows == 0, "slab row padding must cover whole split tiles");
  k_oz_split<<<dim3((unsigned)(maxr / kSplitRows), (unsigned)sp.size()), 256, 0, st>>>(dsp, kp, rows, slab, ex);
  AMB_LAUNCHED();
  std::vector<char> blob(td.size() * sizeof(TcDesc) + prefix.size() * sizeof(int));
  memcpy(blob.data(), td.data(), td.size() * sizeof(TcDesc));
  memcpy(blob.data() + td.size() * sizeof(TcDesc), prefix.data(), prefix.size() * sizeof(int));
  char* dev = static_cast<char*>(ring.push(blob.data(), blob.size(), st));
  OzArgs ga;
  ga.desc = reinterpret_cast<const TcDesc*>(dev);
  ga.prefix = reinterpret_cast<const int*>(dev + td.size() * sizeof(TcDesc));
  ga.ndesc = (int)td.size();
  ga.R = rows;
  ga.alpha = alpha;
  ga.beta = beta;
  ga.c = cbase;
  ga.ex = ex;
  ga.status = status;
  static thread_local int nsm = 0;
  if (nsm == 0) {
    int devid = 0;
    AMB_CUDA(cudaGetDevice(&devid));
    AMB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, devid));
  }
  const CUtensorMap ma = slab_map(slab, rows * kOzSlices, kp, kTM), mb = slab_map(slab, rows * kOzSlices, kp, kOzTN);
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, nsm);
  k_oz_gemm<<<grid, 192, kOzSmemBytes, st>>>(ma, mb, ga);
  AMB_LAUNCHED();
}

// C = beta C + alpha A B^T for every entry of d, K in chunks of kTcKMax: per
// chunk the split descriptors (B rows, then the A row ranges that have
// entries in the chunk) and the tile descriptors, handed to run(...)
// akey (optional): products with the same key >= 0 share one dense A (same
// offset, leading dimension, m, k and form), which is split once per chunk
template <typename E, class Count, class Run>
void gemm_chunks(const std::vector<TcGemm>& d, const E* abase, const E* bbase, Count count, Run run,
                 const std::vector<int>* akey = nullptr) {
  AMB_CHECK(!akey || akey->size() == d.size(), AMB_EINVAL, "tensor-core product keys do not match the products");
  constexpr int kp = kTcKMax;
  int kmax = 0;
  for (const auto& x : d) {
    AMB_CHECK(x.m >= 0 && x.n >= 0 && x.k >= 0 && x.a_tri >= 0 && x.a_tri <= 2, AMB_EINVAL, "bad tensor-core product");
    // rows of an upper-triangular A beyond K would never be written
    AMB_CHECK(x.a_tri != 2 || x.m <= x.k, AMB_EINVAL, "upper-triangular tensor-core operand with m > k");
    if (x.m > 0 && x.n > 0) kmax = std::max(kmax, x.k);
  }
  if (akey) {
    // a shared split is only valid for products whose A is the same matrix
    std::unordered_map<int, size_t> first;
    for (size_t di = 0; di < d.size(); ++di) {
      const int key = (*akey)[di];
      const TcGemm& x = d[di];
      if (key < 0 || x.a_tri != 0 || x.m <= 0 || x.n <= 0) continue;
      auto it = first.emplace(key, di).first;
      const TcGemm& y = d[it->second];
      AMB_CHECK(x.a == y.a && x.lda == y.lda && x.m == y.m && x.k == y.k && x.a_kmajor == y.a_kmajor, AMB_EINVAL,
                "tensor-core products with one key have different A operands");
    }
  }
  for (int k0 = 0; k0 < kmax || (k0 == 0 && kmax == 0); k0 += kp) {
    std::vector<TcSplitDesc> sp;
    std::vector<TcDesc> td;
    std::vector<int> prefix;
    int64_t rows = 0, tiles = 0;
    int maxr = 0;
    std::unordered_map<int, int64_t> shared_arow;   // key -> slab row of its split A in this chunk
    for (size_t di = 0; di < d.size(); ++di) {
      const TcGemm& x = d[di];
      if (x.m <= 0 || x.n <= 0) continue;
      if (x.k <= 0) {
        // an empty sum: C = beta C, as one chunk with no K steps
        if (k0 > 0) continue;
      } else if (k0 >= x.k) {
        continue;
      }
      const int key = (akey && x.a_tri == 0) ? (*akey)[di] : -1;
      const int k1 = std::min(x.k, k0 + kp), kc = std::max(0, k1 - k0);
      // row ranges of A with entries in [k0, k1), and whether beta applies
      // (the chunk is the first that reaches those rows)
      int rr[2][3];
      int nr = 0;
      if (x.a_tri == 2) {
        const int hi = std::min(x.m, std::max(k1, 1));
        if (k0 > 0 && std::min(k0, x.m) > 0) rr[nr][0] = 0, rr[nr][1] = std::min(k0, x.m), rr[nr][2] = 0, ++nr;
        if (hi > k0) rr[nr][0] = k0, rr[nr][1] = hi, rr[nr][2] = 1, ++nr;
      } else if (x.a_tri == 1) {
        if (k0 == 0) rr[nr][0] = 0, rr[nr][1] = x.m, rr[nr][2] = 1, ++nr;
        else if (k0 < x.m) rr[nr][0] = k0, rr[nr][1] = x.m, rr[nr][2] = 0, ++nr;
      } else {
        rr[nr][0] = 0, rr[nr][1] = x.m, rr[nr][2] = k0 == 0, ++nr;
      }
      if (nr == 0) continue;
      // B rows (all n) for this chunk
      const int npad = pad_rows(x.n);
      const int64_t brow = rows;
      sp.push_back(TcSplitDesc{reinterpret_cast<const float*>(bbase + x.b + (x.b_kmajor ? (int64_t)k0 : (int64_t)k0 * x.ldb)),
                               brow, x.ldb, x.n, kc, npad, x.b_kmajor, 0, 0, 0});
      rows += npad;
      maxr = std::max(maxr, npad);
      for (int q = 0; q < nr; ++q) {
        const int r0 = rr[q][0], r1 = rr[q][1];
        const int mpad = pad_rows(r1 - r0);
        int64_t arow = rows;
        auto hit = key >= 0 ? shared_arow.find(key) : shared_arow.end();
        if (hit != shared_arow.end()) {
          arow = hit->second;
        } else {
          const int64_t aoff = x.a_kmajor ? (int64_t)k0 + (int64_t)r0 * x.lda : (int64_t)r0 + (int64_t)k0 * x.lda;
          sp.push_back(TcSplitDesc{reinterpret_cast<const float*>(abase + x.a + aoff), rows, x.lda, r1 - r0, kc, mpad,
                                   x.a_kmajor, x.a_tri, r0 - k0, 0});
          if (key >= 0) shared_arow[key] = rows;
          rows += mpad;
          maxr = std::max(maxr, mpad);
        }
        TcDesc t{x.c + r0, arow, brow, r1 - r0, x.n, (kc + kTK - 1) / kTK * kTK, x.ldc, 0, x.a_tri, r0 - k0, rr[q][2]};
        prefix.push_back((int)tiles);
        tiles += count(t);
        td.push_back(t);
      }
    }
    if (td.empty()) break;
    run(sp, td, prefix, rows, maxr, tiles);
    if (kmax == 0) break;
  }
}

}  // namespace

void tc_syrk_lower_f64(cudaStream_t st, DescRing& ring, const std::vector<TcSyrk>& d, double alpha, double beta,
                       double* base, int* status) {
  if (d.empty()) return;
  constexpr int kp = kTcKMax;
  std::vector<TcSplitDesc> sp;
  std::vector<TcDesc> td;
  std::vector<int> prefix;
  int64_t rows = 0, tiles = 0;
  int maxr = 0;
  for (const auto& x : d) {
    AMB_CHECK(x.k >= 0 && x.k <= kp, AMB_EINVAL, "tensor-core trailing update with K above the slab width");
    if (x.rem <= 0 || x.k <= 0) continue;
    const int rpad = pad_rows(x.rem);
    // the split pass reads the FP64 source through the descriptor's pointer
    sp.push_back(TcSplitDesc{reinterpret_cast<const float*>(base + x.p), rows, x.ld, x.rem, x.k, rpad, 0, 0, 0, 0});
    TcDesc t{x.c, rows, rows, x.rem, x.rem, (x.k + kTK - 1) / kTK * kTK, x.ld, 1, 0, 0, 1};
    prefix.push_back((int)tiles);
    tiles += oz_tile_count(t);
    td.push_back(t);
    rows += rpad;
    maxr = std::max(maxr, rpad);
  }
  if (td.empty()) return;
  run_oz(st, ring, sp, td, prefix, rows, maxr, tiles, alpha, beta, base, status);
}

void tc_gemm_f64(cudaStream_t st, DescRing& ring, const std::vector<TcGemm>& d, double alpha, double beta,
                 const double* abase, const double* bbase, double* cbase, int* status, const std::vector<int>* akey) {
  gemm_chunks(d, abase, bbase, oz_tile_count,
              [&](const std::vector<TcSplitDesc>& sp, const std::vector<TcDesc>& td, const std::vector<int>& prefix,
                  int64_t rows, int maxr, int64_t tiles) {
                run_oz(st, ring, sp, td, prefix, rows, maxr, tiles, alpha, beta, cbase, status);
              },
              akey);
}

void tc_gemm(cudaStream_t st, DescRing& ring, const std::vector<TcGemm>& d, float alpha, float beta,
             const float* abase, const float* bbase, float* cbase, int* status) {
  gemm_chunks(d, abase, bbase, tc_tile_count,
              [&](const std::vector<TcSplitDesc>& sp, const std::vector<TcDesc>& td, const std::vector<int>& prefix,
                  int64_t rows, int maxr, int64_t tiles) {
                run_tiles(st, ring, sp, td, prefix, rows, maxr, tiles, alpha, beta, cbase, status);
              });
}

}  // namespace amb
