// The batched substructure engine (one context, one GPU).
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "common.h"
#include "timers.h"
#include "kernels.h"
#include "level.h"
#include "topology.h"

namespace amb {

struct Mesh {
  int nx = 0, ny = 0, nz = 0, dpn = 1;
  double h = 1.0, nu = 0.3;
  int64_t nel = 0, nnodes = 0, ndof = 0;   // ndof = nnodes * dpn (full grid)
  std::vector<uint8_t> dir_h;
  std::vector<int32_t> elem_sub_h;
  DevBuf coeff, dir, khat, elem_sub, elem_local;
};

struct PairReportH {
  int level, s, t, n_computed, n_selected, n_rows, converged, iterations;
  std::vector<double> lambda;
  double residual = 0.0;
};

class EngineBase {
 public:
  virtual ~EngineBase() = default;
  virtual void setup() = 0;
  virtual void precond(const double* r, double* z) = 0;   // device full-grid vectors
  virtual void schur_apply(int level, int width, const void* x, void* y) = 0;
  // Same product, with the launch descriptors staged in caller-provided
  // device memory `scratch` (bytes) instead of the context's staging ring.
  virtual void schur_apply_staged(int level, int width, const void* x, void* y, void* scratch, size_t bytes) = 0;
  virtual const LevelTopo& topo(int level) const = 0;
  virtual int n_levels() const = 0;
  virtual void export_sub(int what, int level, int idx, std::vector<char>& out) = 0;
  virtual double level_factor_flops(int level) const = 0;
  virtual int64_t graph_replays() const = 0;
};

// Largest number of substructures per level the staged Schur apply accepts.
constexpr int kStagedMaxDesc = 1024;

struct EngineConfig {
  amb_options opt;
  int levels = 2;
  double tau = 10.0;
  std::vector<std::vector<int32_t>> parents;
  std::vector<int> nsubs;   // per level (index 0 = level 1)
};

std::unique_ptr<EngineBase> make_engine(int precision, Mesh& mesh, const EngineConfig& cfg, cudaStream_t st,
                                        DescRing& ring, Timers& tm, std::vector<PairReportH>& reports,
                                        std::vector<double>& omega, std::vector<int>& nadapt, DevBuf& status);

}  // namespace amb
