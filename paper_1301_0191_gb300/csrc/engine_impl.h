// Typed engine (one instantiation per factor precision).  Shared by
// engine.cu (set-up, Algorithm 1) and lobpcg.cu (adaptive constraints).
#pragma once

#include <algorithm>
#include <cstring>

#include "engine.h"
#include "fem.h"

namespace amb {

template <typename T>
class Engine : public EngineBase {
 public:
  Engine(Mesh& m, const EngineConfig& c, cudaStream_t s, DescRing& r, Timers& t, std::vector<PairReportH>& rep,
         std::vector<double>& om, std::vector<int>& na, DevBuf& stat)
      : mesh(m), cfg(c), st(s), ring(r), tm(t), reports(rep), omega(om), nadapt(na), status(stat) {}

  ~Engine() override {
    drop_graph();
    if (cstream) cudaStreamDestroy(cstream);
  }
  void setup() override;
  // Algorithm 1 on all levels as one CUDA graph: captured on the first call
  // for a given (r, z) pair of device vectors, replayed afterwards
  void precond(const double* r, double* z) override;
  void schur_apply(int level, int width, const void* x, void* y) override;
  void schur_apply_staged(int level, int width, const void* x, void* y, void* scratch, size_t bytes) override;
  const LevelTopo& topo(int level) const override { return lv[level - 1]->topo; }
  int n_levels() const override { return (int)lv.size(); }
  void export_sub(int what, int level, int idx, std::vector<char>& out) override;
  double level_factor_flops(int level) const override { return lv[level - 1]->factor_flops; }
  int64_t graph_replays() const override { return pg_replays; }

  // set-up pieces
  void alloc_level(LevelData<T>& L);
  void upload_par(LevelData<T>& L);
  void assemble(LevelData<T>& L, const LevelData<T>* prev, const std::vector<int32_t>& loc);
  void factor_level(LevelData<T>& L);
  void coarse_basis(LevelData<T>& L);
  void adapt_level(LevelData<T>& L);     // lobpcg.cu
  void setup_top();
  void apply_level(int i, const double* r, double* u);
  void drop_graph();
  void check_status(const char* what, int code);
  bool timing() const { return cfg.opt.timing_events != 0; }

  Mesh& mesh;
  EngineConfig cfg;
  cudaStream_t st;
  DescRing& ring;
  DescRing* aring = nullptr;               // descriptor staging of apply_level (the graph's own ring while capturing)
  DescRing gring;                          // staging of the captured graph: written once, kept with the graph
  cudaGraphExec_t pgraph = nullptr;
  cudaStream_t cstream = nullptr;          // capture stream of the graph
  const double* pg_r = nullptr;
  double* pg_z = nullptr;
  int64_t pg_kernels = 0;                  // kernel launches inside the graph
  int64_t pg_replays = 0;
  Timers& tm;
  std::vector<PairReportH>& reports;
  std::vector<double>& omega;
  std::vector<int>& nadapt;
  DevBuf& status;
  std::vector<std::unique_ptr<LevelData<T>>> lv;
  int64_t nC = 0;
  DevBuf AC, LinvC, topT;
};

// helpers for host-built descriptors
inline int imax(const std::vector<int>& v) {
  int m = 0;
  for (int x : v) m = std::max(m, x);
  return m;
}

}  // namespace amb
