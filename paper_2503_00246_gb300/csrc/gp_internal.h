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
  void* d_tp = nullptr;          // per-face outputs W_F (scratch of the face + lift path)
  // brick path (gp_brick.cuh): tables and the partial grids of the plane nodes (scratch)
  bool use_brick = false;
  int32_t* d_bdesc = nullptr;
  int32_t* d_bcell = nullptr;
  int32_t* d_bccoord = nullptr;
  uint32_t* d_bface = nullptr;
  int32_t* d_rowtab = nullptr;
  int32_t* d_pnode = nullptr;
  int32_t* d_poff = nullptr;
  int32_t* d_pslot = nullptr;
  void* d_part = nullptr;
  bool no_scratch = false;
  void* d_xh = nullptr;          // gp_apply_host staging
  void* d_yh = nullptr;
  int2* d_truns = nullptr;       // gp_apply_host: runs (c0, len) of the touched DoFs
  int32_t ntruns = -1;           // -1: not built yet
  int64_t host_bytes[2] = {0, 0};  // bytes the last gp_apply_host moved host -> device, device -> host
  // gp_apply_host with a page-locked y: a slab pipeline whose finished parts of y go back on a
  // second stream while later slabs compute (built on first use)
  bool hpipe_built = false;
  std::vector<int32_t> hslabs;   // slab table (gp::slab_table)
  std::vector<int64_t> hbounds;  // y chunk of slab s: [hbounds[s], hbounds[s + 1])
  std::vector<cudaEvent_t> hev;  // one per slab, recorded after its lift
  cudaStream_t hcopy = nullptr;  // the D2H stream
  std::vector<int2> htruns;      // host copy of d_truns
  std::vector<int32_t> hxrun;    // touched runs gathered for slab s: [hxrun[s], hxrun[s + 1])
  std::vector<cudaEvent_t> hgev; // one per slab, recorded after its gather
  cudaStream_t hin = nullptr;    // the gather stream
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
// A slab pipeline for one launch: a slab table (SLAB ints per slab) and an event per slab.
struct SlabRun {
  const int32_t* table = nullptr;
  int n = 0;
  cudaEvent_t* events = nullptr;   // recorded after each slab's lift
  cudaEvent_t* inputs = nullptr;   // waited for before each slab's face launch (or nullptr)
};
gp_status launch(gp_ctx* c, const void* x, void* y, int add, cudaStream_t st, void* scratch = nullptr,
                 bool trace = true, const gp::Tiles* tiles = nullptr, int which = 3, const SlabRun* run = nullptr);

// Slab pipeline of the face + lift path (gp_opts.slabs): at most MAX_SLABS slabs.
static_assert(gp::SLAB == gp::SLAB_INTS, "the plan's and the launcher's slab records differ");
constexpr int MAX_SLABS = 64;
// gp_apply_host: the device address of a page-locked host buffer (nullptr for other memory),
// the runs of touched DoFs (built on first use), and the copy of those runs of x.
const void* device_view(const void* host);
cudaError_t ensure_touched_runs(gp_ctx* c);
// The host-apply slab pipeline of c (host_slabs slabs; none when the plan has too few owners):
// 8 for FP32, 16 for the FP64 forms (measured best on the 128^3 gyroid at k = 4: FP32 35.7 /
// 38.3 / 37.6 GDoF/s end to end with 16 / 8 / 4 slabs, FP64 19.7 / 19.1 / 17.4).
inline int host_slabs(int precision) { return precision == GP_FP32 ? 8 : 16; }
cudaError_t ensure_host_pipeline(gp_ctx* c);
cudaError_t gather_runs(const void* src, void* dst, const int2* runs, int nruns, int elem, cudaStream_t st);
// Default faces per chunk of the brick kernel (about 256 threads).
int brick_default_fb(int dim, int k);
// Bytes of the brick path's partial grids (its scratch) for context c.
size_t brick_scratch_bytes(const gp_ctx* c);
// Allocates the face-output buffer W of the face + lift path if the context has none (the
// model system and the autotuner's face + lift timings need it).
gp_status ensure_face_outputs(gp_ctx* c);

// Tile-shape helpers for the context's (dimension, arithmetic).
gp::TileOps tile_ops(int dim, int precision);

// Process-wide table of tuned tile shapes, keyed by (device, dimension, degree, precision);
// gp_setup starts every context from the entry of its key, if there is one.
bool tiles_lookup(int device, int dim, int k, int precision, gp::Tiles* out);
void tiles_record(int device, int dim, int k, int precision, const gp::Tiles& t);
// The same for brick-path contexts (faces per chunk), filled by gp_autotune.
bool brick_tiles_lookup(int device, int dim, int k, int precision, gp::Tiles* out);

}  // namespace gpi
