// The opaque context behind the C ABI and helpers shared by its entry points.
#pragma once

#include <memory>
#include <new>
#include <string>
#include <vector>

#include "engine.h"

struct amb_ctx {
  std::string err;
  amb_options opt;
  cudaStream_t st = nullptr;
  int device = 0;
  amb::Mesh mesh;
  amb::EngineConfig cfg;
  amb::DescRing ring;
  amb::Timers tm;
  std::vector<amb::PairReportH> reports;
  std::vector<double> omega;
  std::vector<int> nadapt;
  amb::DevBuf status;
  std::unique_ptr<amb::EngineBase> eng;
  amb::DevBuf f, u, r, z, p, q, rold, tmp, partial, dscal, ab, lam, grad, body;
  bool have_solution = false;
  int last_its = 0;
  double last_cond = 0, last_rel = 0;
  int64_t launches_total = 0;
  double setup_ms = 0;
};

namespace amb {

inline bool is_device(const void* ptr) {
  if (!ptr) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Run fn, translating library errors into status codes and messages.
template <typename F>
int guarded(amb_ctx* c, F&& fn) {
  if (!c) return AMB_EINVAL;
  const int64_t l0 = g_launches;
  alloc_stream() = c->st;
  try {
    c->err.clear();
    fn();
    c->launches_total += g_launches - l0;
    return AMB_OK;
  } catch (const Error& e) {
    c->err = e.what();
    c->launches_total += g_launches - l0;
    return e.status;
  } catch (const std::bad_alloc& e) {
    c->err = std::string("host allocation failed: ") + e.what();
    c->launches_total += g_launches - l0;
    return AMB_ENOMEM;
  } catch (const std::exception& e) {
    c->err = e.what();
    c->launches_total += g_launches - l0;
    return AMB_EINVAL;
  } catch (...) {
    // nothing may cross the C boundary
    c->err = "unknown exception";
    c->launches_total += g_launches - l0;
    return AMB_EINVAL;
  }
}

}  // namespace amb
