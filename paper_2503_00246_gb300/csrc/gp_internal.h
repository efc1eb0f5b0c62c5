// Internal declarations shared by the C-ABI translation units.
#pragma once

#include <string>
#include <vector>

#include "gp.h"
#include "gp_launch.h"
#include "gp_plan.h"

struct gp_ctx {
  gp::Plan plan;
  int device = -1;
  bool on_device = false;
  size_t elem = 8;
  int32_t* d_frows = nullptr;
  int32_t* d_lwin = nullptr;
  int32_t* d_lrow = nullptr;
  int2* d_zruns = nullptr;
  void* d_tp = nullptr;          // per-face outputs W_F (scratch)
  void* d_xh = nullptr;          // gp_apply_host staging
  void* d_yh = nullptr;
  gp::Tiles tiles{};             // tile shape of the face and lift launches (0: defaults)
  std::string err;
  // tracing: one event triple per traced apply
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  int64_t nprof = 0;
};

namespace gpi {

// Makes `dev` current for the lifetime of the guard and restores the caller's device.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Records `m` as the last error of `c` (or of the calling thread when c is NULL).
gp_status fail(const gp_ctx* c, gp_status s, const std::string& m);

// Enqueues y = G x (add = 0) or y += G x (add = 1) for context c; `scratch` replaces the
// context's face-output buffer when given; `trace` = false never records events.
// `tiles` overrides the context's tile shape; `which` (bit 0 face, bit 1 lift) drops a
// kernel (the autotuner times them apart).
gp_status launch(gp_ctx* c, const void* x, void* y, int add, cudaStream_t st, void* scratch = nullptr,
                 bool trace = true, const gp::Tiles* tiles = nullptr, int which = 3);

// Tile-shape helpers for the context's (dimension, arithmetic).
gp::TileOps tile_ops(int dim, int precision);

// Process-wide table of tuned tile shapes, keyed by (device, dimension, degree, precision);
// gp_setup starts every context from the entry of its key, if there is one.
bool tiles_lookup(int device, int dim, int k, int precision, gp::Tiles* out);
void tiles_record(int device, int dim, int k, int precision, const gp::Tiles& t);

}  // namespace gpi
