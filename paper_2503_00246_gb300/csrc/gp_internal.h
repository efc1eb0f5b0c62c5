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
gp_status launch(gp_ctx* c, const void* x, void* y, int add, cudaStream_t st, void* scratch = nullptr,
                 bool trace = true);

}  // namespace gpi
