// amb_schur_apply_noalloc: the batched Schur apply of amb_schur_apply for
// callers that must not allocate device memory during the call.
//
// The only device memory the product needs besides its inputs and outputs
// is a small array of launch descriptors (one per substructure, plus CTA
// prefix sums).  amb_schur_apply stages them in memory the context
// allocated; this variant stages them in a fixed array that is part of the
// library image (file scope below), so the call itself never allocates.
#include <mutex>

#include "ctx.h"

namespace {

// 64 KiB: room for kStagedMaxDesc GEMM descriptors and their prefix sums.
constexpr size_t kNoAllocScratchBytes = 64 * 1024;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

}  // namespace

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_schur_noalloc_scratch[kNoAllocScratchBytes];

namespace {

// Device address of the scratch array on the current device.  Host code
// only knows a host-side stand-in for the symbol, so the real address is
// queried once per device (with that device current) and cached for the
// life of the process.  A device reset (cudaDeviceReset, or a reset of the
// primary context) reloads the module and invalidates the cached address:
// processes that reset a device must not call this entry point afterwards.
void* scratch_address(int dev) {
  AMB_CHECK(dev >= 0 && dev < kMaxDevices, AMB_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_schur_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      throw amb::Error(AMB_ECUDA, std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") +
                                      cudaGetErrorString(e));
    }
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

static_assert(sizeof(amb::GemmDesc) * amb::kStagedMaxDesc + 256 + (amb::kStagedMaxDesc + 1) * sizeof(int) <=
                  kNoAllocScratchBytes,
              "scratch array too small for the descriptor limit");

}  // namespace

extern "C" int amb_schur_apply_noalloc(amb_ctx* c, int32_t level, int32_t width, const void* x, void* y) {
  return amb::guarded(c, [&]() {
    AMB_CHECK(c->eng, AMB_EINVAL, "context has no successful set-up");
    AMB_CHECK(amb::is_device(x) && amb::is_device(y), AMB_EINVAL, "x and y must be device arrays");
    int dev = -1;
    AMB_CUDA(cudaGetDevice(&dev));
    AMB_CHECK(dev == c->device, AMB_EINVAL, "the context's device must be current");
    // the call copies its descriptors from host memory and waits for the
    // stream: it cannot be recorded into a CUDA graph
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    AMB_CUDA(cudaStreamIsCapturing(c->st, &cs));
    AMB_CHECK(cs == cudaStreamCaptureStatusNone, AMB_EINVAL,
              "amb_schur_apply_noalloc called while the context stream is being captured");
    void* scratch = scratch_address(dev);
    c->eng->schur_apply_staged(level, width, x, y, scratch, kNoAllocScratchBytes);
    AMB_CUDA(cudaStreamSynchronize(c->st));
  });
}
