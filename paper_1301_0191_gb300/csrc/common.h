// Internal helpers shared by the translation units of libamb.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "amb.h"

namespace amb {

// Errors raised inside the library carry an AMB_E* status; the C ABI
// catches them and stores the message in the context.
struct Error : public std::runtime_error {
  int status;
  Error(int st, const std::string& m) : std::runtime_error(m), status(st) {}
};

#define AMB_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      throw ::amb::Error(AMB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_) + \
                                        " at " + __FILE__ + ":" + std::to_string(__LINE__)); \
  } while (0)

#define AMB_CHECK(cond, st, msg)                      \
  do {                                                \
    if (!(cond)) throw ::amb::Error((st), (msg));     \
  } while (0)

// Launch bookkeeping: every kernel launch goes through AMB_LAUNCHED so the
// context can report how many of its kernels ran.
extern thread_local int64_t g_launches;
#define AMB_LAUNCHED()                       \
  do {                                       \
    ++::amb::g_launches;                     \
    AMB_CUDA(cudaGetLastError());            \
  } while (0)

// Device memory comes from the device's stream-ordered pool (cudaMallocAsync)
// with no release threshold: buffers freed by one context are reused by the
// next without returning to the CUDA driver, and a free does not synchronize the
// device (cudaFree does).  Allocations and frees are ordered on the stream of
// the context that the calling thread is serving (set at every ABI entry).
inline cudaStream_t& alloc_stream() {
  static thread_local cudaStream_t s = nullptr;
  return s;
}
void pool_init();

// Owned device allocation.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, alloc_stream());
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t n) {
    release();
    if (n == 0) n = 16;
    pool_init();
    cudaError_t e = cudaMallocAsync(&p, n, alloc_stream());
    if (e != cudaSuccess) {
      p = nullptr;
      (void)cudaGetLastError();
      throw Error(AMB_ENOMEM, "device allocation of " + std::to_string(n) + " bytes failed: " + cudaGetErrorString(e));
    }
    bytes = n;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

template <typename T>
inline T* dptr(const DevBuf& b) { return static_cast<T*>(b.p); }

// A host thread's device workspaces (operand slabs of the tensor-core
// products, scratch of the diagonal blocks: grown on demand and kept for the
// thread's life) are allocated on the first device the thread works on.
// A later call of the same thread on another device is refused here rather
// than handing that device a pointer into another GPU's memory.
inline void check_workspace_device() {
  static thread_local int dev = -1;
  int d = 0;
  AMB_CUDA(cudaGetDevice(&d));
  if (dev < 0) dev = d;
  AMB_CHECK(d == dev, AMB_EINVAL,
            "this host thread holds device workspaces on another GPU: serve each GPU's contexts from its own threads");
}

template <typename T>
inline void upload(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
  b.alloc(v.size() * sizeof(T));
  if (!v.empty()) AMB_CUDA(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}

// Ring of pinned staging memory for small per-launch descriptor arrays.
// push() copies host data into pinned memory and enqueues an async H2D
// copy on the stream; the returned device pointer is valid for kernels
// launched afterwards on the same stream.  On wrap-around the stream is
// synchronized before pinned memory is reused.
class DescRing {
 public:
  void init(size_t bytes) {
    if (host_) return;
    AMB_CUDA(cudaMallocHost(&host_, bytes));
    dev_.alloc(bytes);
    cap_ = bytes;
  }
  ~DescRing() {
    if (host_) cudaFreeHost(host_);
  }
  // a ring that must not wrap (the staging of a captured graph): allocated
  // once, rewound to the start
  void reset(size_t bytes) {
    init(bytes);
    pos_ = 0;
    no_wrap_ = true;
  }
  void* push(const void* src, size_t bytes, cudaStream_t st) {
    size_t need = (bytes + 255) & ~size_t(255);
    AMB_CHECK(need <= cap_, AMB_EINVAL, "descriptor batch larger than the staging ring");
    if (pos_ + need > cap_) {
      AMB_CHECK(!no_wrap_, AMB_EINVAL, "graph descriptor staging ring too small");
      AMB_CUDA(cudaStreamSynchronize(st));
      pos_ = 0;
    }
    char* h = static_cast<char*>(host_) + pos_;
    char* d = static_cast<char*>(dev_.p) + pos_;
    memcpy(h, src, bytes);
    AMB_CUDA(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st));
    pos_ += need;
    return d;
  }

 private:
  void* host_ = nullptr;
  DevBuf dev_;
  size_t cap_ = 0, pos_ = 0;
  bool no_wrap_ = false;
};

constexpr size_t kGraphRingBytes = size_t(16) << 20;   // descriptor staging of the preconditioner graph

// tile autotuner bookkeeping (dense.cu): shape classes decided, runs spent timing
size_t gemm_tune_entries();
int64_t gemm_tune_runs();

// One matrix product C = alpha op(A) op(B) + beta C of a batch; offsets are
// element offsets from the launch's base pointers; matrices column-major.
struct GemmDesc {
  int32_t m, n, k;
  int32_t lda, ldb, ldc;
  int64_t a, b, c;
};

enum GemmFlags : int {
  G_TRANS_A = 1,
  G_TRANS_B = 2,
  G_TRI_A_LOWER = 4,   // op(A) lower triangular: op(A)(i,l) = 0 for l > i (not read)
  G_TRI_A_UPPER = 8,   // op(A) upper triangular: op(A)(i,l) = 0 for l < i
  G_TRI_B_LOWER = 16,  // op(B)(l,j) = 0 for l < j
  G_TRI_B_UPPER = 32,  // op(B)(l,j) = 0 for l > j
  G_OUT_LOWER = 64,    // write only C(i,j) with i >= j
  // the caller guarantees that running the product twice gives the same C
  // (beta = 0, C overlaps neither A nor B): its tile shape may be autotuned
  G_TUNE = 128,
};

// Batched product driver (dense.cu).  A may be stored in a narrower type
// TA than the compute/accumulate type T (e.g. FP32 Schur complements times
// FP64 block vectors with FP64 accumulation).
template <typename T, typename TA = T>
void gemm_batched(cudaStream_t st, DescRing& ring, const std::vector<GemmDesc>& d, int flags,
                  T alpha, T beta, const TA* A, const T* B, T* C);

// Gather/scatter descriptor for batched matrix-vector work (dense.cu).
struct GemvDesc {
  int32_t m, n, lda, pad;
  int64_t a, x, y;
};
template <typename T>
void gemv_batched(cudaStream_t st, DescRing& ring, const std::vector<GemvDesc>& d, int flags,
                  T alpha, T beta, const T* A, const T* X, T* Y);

// Launches on descriptor arrays already resident in device memory
// (d_desc[ndesc], d_prefix[ndesc+1] = per-descriptor CTA prefix sums, total
// = d_prefix[ndesc]); the *_ctas helpers give the CTA count of one
// descriptor so callers can build the prefix sums themselves.
template <typename T>
int gemm_ctas(const GemmDesc& d);
int gemv_ctas(const GemvDesc& d, bool trans);
template <typename T>
void gemm_launch_prepared(cudaStream_t st, const GemmDesc* d_desc, const int* d_prefix, int ndesc, int total,
                          int flags, T alpha, T beta, const T* A, const T* B, T* C);
template <typename T>
void gemv_launch_prepared(cudaStream_t st, const GemvDesc* d_desc, const int* d_prefix, int ndesc, int total,
                          int flags, T alpha, T beta, const T* A, const T* X, T* Y);

// Partial blocked Cholesky of a batch of column-major matrices (dense.cu):
// factor columns [c0, c1) of every matrix (lower), trailing updates applied
// to the whole remaining lower triangle.  Diagonal-block inverses are
// written into `zinv` (lower-triangular explicit inverse buffer, same block
// positions, leading dimension zld) when zinv != nullptr.
struct CholDesc {
  int64_t off;      // matrix offset (elements) in the base buffer
  int32_t ld;       // leading dimension (= order of the full matrix)
  int32_t n;        // order of the full matrix
  int32_t c0, c1;   // columns to factor
  int64_t zoff;     // offset of the inverse buffer block for column c0
  int32_t zld;
  int32_t id;       // substructure id for error reports
};
struct Timers;
template <typename T>
void partial_cholesky(cudaStream_t st, DescRing& ring, const std::vector<CholDesc>& d, T* base,
                      T* zbase, int* status, double* flops, Timers* tm = nullptr, bool timing = false);

// Explicit inverse of the lower-triangular factor of order n stored at
// L (ld) into Z (zld), whose nb x nb diagonal blocks already hold the
// inverses of L's diagonal blocks (written by partial_cholesky).
struct TrtriDesc {
  int64_t l, z;
  int32_t ld, zld, n, pad;
};
// status: the tensor-core products of the FP32 form report a bounded wait
// that ran out there (AMB_ETIMEOUT); may be null for the FP64 form.
template <typename T>
void trtri_from_blocks(cudaStream_t st, DescRing& ring, const std::vector<TrtriDesc>& d, const T* lbase,
                       T* zbase, double* flops, int* status = nullptr);

constexpr int kNB = 64;   // Cholesky / triangular-inverse block size

}  // namespace amb
