// Per-family kernel timing of a context (CUDA events, enabled on request).
#pragma once

#include "amb.h"
#include "common.h"

namespace amb {

struct Timers {
  double phase_ms[8] = {0};
  double fam_ms[AMB_FAM_N] = {0};
  int64_t fam_launches[AMB_FAM_N] = {0};
  double fam_flops[AMB_FAM_N] = {0};
  double fam_bytes[AMB_FAM_N] = {0};
};

// Two events that time a section of work on one stream, destroyed on every
// exit path (an error thrown inside the section included).  start() records
// the first, lap() records the second, waits for it and returns the elapsed
// milliseconds; lap() may be followed by start() for the next section.
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() = default;
  EventPair(const EventPair&) = delete;
  EventPair& operator=(const EventPair&) = delete;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  void start(cudaStream_t st) {
    if (!a) AMB_CUDA(cudaEventCreate(&a));
    if (!b) AMB_CUDA(cudaEventCreate(&b));
    AMB_CUDA(cudaEventRecord(a, st));
  }
  float lap(cudaStream_t st) {
    AMB_CUDA(cudaEventRecord(b, st));
    AMB_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
};

// Event pair around a kernel family section (only when timing is enabled).
struct FamTimer {
  cudaStream_t st;
  Timers* tm;
  int fam;
  bool on;
  cudaEvent_t a = nullptr, b = nullptr;
  int64_t l0;
  FamTimer(cudaStream_t s, Timers* t, int f, bool enabled) : st(s), tm(t), fam(f), on(enabled), l0(g_launches) {
    if (on) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, st);
    }
  }
  ~FamTimer() {
    tm->fam_launches[fam] += g_launches - l0;
    if (on) {
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      tm->fam_ms[fam] += ms;
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  }
};

}  // namespace amb
