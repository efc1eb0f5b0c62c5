// C ABI of the ghost-penalty operator (declarations and contracts in gp.h).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "gp_internal.h"

namespace gp {
size_t noalloc_scratch_bytes();
cudaError_t noalloc_scratch(int device, void** out);
}  // namespace gp



namespace {
thread_local std::string g_err;

// dst[c0 + i] = src[c0 + i] over the runs (c0, len): one warp per run, consecutive lanes on
// consecutive elements (src: a device view of page-locked host memory)
template <typename T>
__global__ void __launch_bounds__(256) gather_runs_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                         const int2* __restrict__ runs, const int nruns) {
  const int lane = threadIdx.x & 31;
  const int w0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int r = w0; r < nruns; r += nw) {
    const int2 run = __ldg(runs + r);
    for (int i = lane; i < run.y; i += 32) dst[run.x + i] = src[run.x + i];
  }
}
}  // namespace

namespace gpi {
cudaError_t gather_runs(const void* src, void* dst, const int2* runs, int nruns, int elem, cudaStream_t st) {
  if (nruns <= 0) return cudaSuccess;
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = std::max(1, std::min((nruns + 7) / 8, 8 * nsm));
  if (elem == 4)
    gather_runs_kernel<float><<<blocks, 256, 0, st>>>((const float*)src, (float*)dst, runs, nruns);
  else
    gather_runs_kernel<double><<<blocks, 256, 0, st>>>((const double*)src, (double*)dst, runs, nruns);
  return cudaGetLastError();
}
}  // namespace gpi

namespace gpi {

gp_status fail(const gp_ctx* c, gp_status s, const std::string& m) {
  if (c) const_cast<gp_ctx*>(c)->err = m;
  else g_err = m;
  return s;
}

const void* device_view(const void* host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();   // clear the error of an unknown pointer
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

cudaError_t ensure_touched_runs(gp_ctx* c) {
  if (c->ntruns >= 0) return cudaSuccess;
  // the touched DoFs are the active DoFs outside the zero runs (which are sorted and disjoint)
  constexpr int32_t RUN_MAX = 1024;
  const gp::Plan& p = c->plan;
  std::vector<int2> runs;
  auto emit = [&](int64_t a, int64_t b) {
    for (; a < b; a += RUN_MAX) runs.push_back(make_int2((int)a, (int)std::min<int64_t>(RUN_MAX, b - a)));
  };
  int64_t pos = 0;
  for (int64_t r = 0; r < p.num_zero_runs(); ++r) {
    emit(pos, p.zruns[2 * r]);
    pos = (int64_t)p.zruns[2 * r] + p.zruns[2 * r + 1];
  }
  emit(pos, p.n_active);
  cudaError_t e = cudaSuccess;
  if (!runs.empty()) {
    e = cudaMalloc(&c->d_truns, runs.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_truns, runs.data(), runs.size() * sizeof(int2), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    c->ntruns = (int32_t)runs.size();
    c->htruns.swap(runs);
  }
  return e;
}

cudaError_t ensure_host_pipeline(gp_ctx* c) {
  if (c->hpipe_built) return cudaSuccess;
  cudaError_t e = ensure_touched_runs(c);
  if (e != cudaSuccess) return e;
  if (!c->use_brick) {
    c->hslabs = gp::slab_table(c->plan, host_slabs(c->plan.precision));
    c->hbounds = gp::slab_y_bounds(c->plan, c->hslabs);
    // the touched runs slab s gathers: those that start below the x its face launch reads and
    // were not gathered for an earlier slab (the last slab takes the rest)
    const std::vector<int64_t> xb = gp::slab_x_bounds(c->plan, c->hslabs);
    const int ns = (int)xb.size();
    c->hxrun.assign(ns + 1, 0);
    int32_t r = 0;
    for (int s = 0; s < ns; ++s) {
      while (r < c->ntruns && (s == ns - 1 || c->htruns[r].x < xb[s])) ++r;
      c->hxrun[s + 1] = r;
    }
  }
  const size_t ns = c->hslabs.size() / gp::SLAB;
  while (e == cudaSuccess && c->hev.size() < ns) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) c->hev.push_back(ev);
  }
  while (e == cudaSuccess && c->hgev.size() < ns) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) c->hgev.push_back(ev);
  }
  if (e == cudaSuccess && ns > 1 && !c->hcopy) e = cudaStreamCreateWithFlags(&c->hcopy, cudaStreamNonBlocking);
  if (e == cudaSuccess && ns > 1 && !c->hin) e = cudaStreamCreateWithFlags(&c->hin, cudaStreamNonBlocking);
  if (e == cudaSuccess) c->hpipe_built = true;
  return e;
}

size_t brick_scratch_bytes(const gp_ctx* c) {
  const gp::Plan& p = c->plan;
  return (size_t)p.num_bricks() * (size_t)p.pgrid * (p.precision == GP_FP32 ? 4 : 8);
}

int brick_default_fb(int dim, int k) {
  const int L = dim == 3 ? (k + 1) * (k + 1) : k + 1;
  const int fb = 256 / L;
  return fb > 0 ? fb : 1;
}

gp_status ensure_face_outputs(gp_ctx* c) {
  if (c->d_tp || c->plan.num_faces() == 0) return GP_OK;
  if (c->no_scratch) return fail(c, GP_EINVAL, "the context was created with no_scratch = 1");
  const gp::Plan& p = c->plan;
  const size_t bytes = (size_t)p.num_faces() * p.L * (2 * p.k + 1) * (p.precision == GP_FP32 ? 4 : 8);
  DeviceGuard g(c->device);
  const cudaError_t e = cudaMalloc(&c->d_tp, bytes);
  if (e != cudaSuccess)
    return fail(c, e == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA,
                std::string("face outputs: ") + cudaGetErrorString(e));
  return GP_OK;
}

}  // namespace gpi

using gpi::DeviceGuard;
using gpi::fail;

namespace {



template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  *dst = nullptr;
  if (src.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)dst, src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

void free_device(gp_ctx* c) {
  void* ptrs[] = {c->d_frows, c->d_lwin, c->d_lrow, c->d_zruns, c->d_tp, c->d_xh, c->d_yh, c->d_truns,
                  c->d_bdesc, c->d_bcell, c->d_bccoord, c->d_bface, c->d_rowtab,
                  c->d_pnode, c->d_poff, c->d_pslot, c->d_part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  c->d_frows = c->d_lwin = c->d_lrow = nullptr;
  c->d_zruns = nullptr;
  c->d_tp = c->d_xh = c->d_yh = nullptr;
  c->d_truns = nullptr;
  c->ntruns = -1;
  c->d_bdesc = c->d_bcell = c->d_bccoord = c->d_rowtab = nullptr;
  c->d_pnode = c->d_poff = c->d_pslot = nullptr;
  c->d_bface = nullptr;
  c->d_part = nullptr;
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  for (cudaEvent_t e : c->hev) cudaEventDestroy(e);
  c->hev.clear();
  for (cudaEvent_t e : c->hgev) cudaEventDestroy(e);
  c->hgev.clear();
  if (c->hcopy) cudaStreamDestroy(c->hcopy);
  if (c->hin) cudaStreamDestroy(c->hin);
  c->hcopy = c->hin = nullptr;
  c->hpipe_built = false;
}

#define GP_CUDA(ctx, call)                                                            \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

}  // namespace

gp_status gpi::launch(gp_ctx* c, const void* x, void* y, int add, cudaStream_t st, void* scratch, bool trace,
                      const gp::Tiles* tiles, int which, const SlabRun* run) {
  const gp::Plan& p = c->plan;
  const bool brick = c->use_brick && which == 3;
  if (!scratch && p.num_faces() > 0 && (brick ? (!c->d_part && p.num_plane_nodes() > 0) : !c->d_tp))
    return fail(c, GP_EINVAL,
                c->no_scratch ? "the context was created with no_scratch = 1: only gp_apply_noalloc can apply it"
                              : "internal: the context has no face-output buffer");
  gp::ApplyArgs a;
  a.dim = p.dim;
  a.k = p.k;
  a.x = x;
  a.y = y;
  a.tp = scratch ? scratch : c->d_tp;
  a.add = add;
  a.frows = c->d_frows;
  for (int i = 0; i < 4; ++i) a.rbase[i] = p.rbase[i];
  for (int i = 0; i < 4; ++i) a.fstart[i] = p.fstart[i];
  a.la.lwin = c->d_lwin;
  a.la.lrow = c->d_lrow;
  a.la.nlift = (int32_t)p.num_lift_cells();
  a.la.n_active = (int32_t)p.n_active;
  a.zruns = c->d_zruns;
  a.nzruns = add ? 0 : (int32_t)p.num_zero_runs();
  a.g = p.jumps.data();
  a.m = p.mass.data();
  a.s = p.scale.data();
  cudaEvent_t* ev = nullptr;
  if (c->prof && trace) {
    const size_t need = 3 * (size_t)(c->nprof + 1);
    while (c->ev.size() < need) {
      cudaEvent_t e;
      GP_CUDA(c, cudaEventCreate(&e));
      c->ev.push_back(e);
    }
    ev = &c->ev[3 * c->nprof];
    c->nprof++;
  }
  a.ev = ev;
  a.tiles = tiles ? *tiles : c->tiles;
  a.which = which;
  a.slabs = run ? run->table : p.slabs.data();
  a.nslab = run ? run->n : p.num_slabs();
  a.slab_events = run ? run->events : nullptr;
  a.slab_inputs = run ? run->inputs : nullptr;
  if (brick) {
    a.brick = true;
    gp::BrickArgs& ba = a.ba;
    ba.bdesc = c->d_bdesc;
    ba.bcell = c->d_bcell;
    ba.bccoord = c->d_bccoord;
    ba.bface = c->d_bface;
    ba.rowtab = c->d_rowtab;
    ba.part = scratch ? scratch : c->d_part;
    ba.nbricks = (int32_t)p.num_bricks();
    ba.n = p.n;
    ba.pgrid = p.pgrid;
    ba.maxcell = p.bmax_cell;
    ba.maxown = p.bmax_own;
    for (int ax = 0; ax < 3; ++ax) {
      ba.bdim[ax] = p.bdim[ax];
      ba.gstride[ax] = p.gstride[ax];
      for (int side = 0; side < 2; ++side) ba.goff[ax][side] = p.goff[ax][side];
    }
    gp::PlaneArgs& pa = a.pa;
    pa.pnode = c->d_pnode;
    pa.poff = c->d_poff;
    pa.pslot = c->d_pslot;
    pa.nplane = (int32_t)p.num_plane_nodes();
    pa.part = ba.part;
  }
  cudaError_t e;
  if (p.precision == GP_FP64)
    e = p.dim == 2 ? gp::apply_f64_d2(a, st) : gp::apply_f64_d3(a, st);
  else if (p.precision == GP_FP64_FF)
    e = p.dim == 2 ? gp::apply_ff_d2(a, st) : gp::apply_ff_d3(a, st);
  else
    e = p.dim == 2 ? gp::apply_f32_d2(a, st) : gp::apply_f32_d3(a, st);
  if (e != cudaSuccess) return fail(c, GP_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return GP_OK;
}

// gp_apply_batched's batches, one per (contexts, nrhs) list; gp_destroy drops those of a context
struct BatchedKey {
  std::vector<gp_ctx*> ctxs;
  int nrhs;
  bool operator<(const BatchedKey& o) const { return nrhs != o.nrhs ? nrhs < o.nrhs : ctxs < o.ctxs; }
};
std::mutex g_batched_mu;
std::map<BatchedKey, gp_batch*> g_batched;

namespace {
using gpi::launch;

gp_status check_apply(const gp_ctx* c, const void* x, const void* y) {
  if (!c) return fail(nullptr, GP_EINVAL, "null context");
  if (!c->on_device) return fail(c, GP_EDEVICE, "context was built host-only (device = -1)");
  if (c->plan.n_active > 0 && (!x || !y)) return fail(c, GP_EINVAL, "null x or y");
  if (x == y && x != nullptr) return fail(c, GP_EINVAL, "x and y must not alias");
  return GP_OK;
}

}  // namespace

extern "C" {

const char* gp_version(void) { return "gp-gb300 0.2 (sm_103a)"; }

const char* gp_last_error(const gp_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

gp_status gp_setup(const gp_mesh* mesh, const gp_levelset* ls, const gp_opts* opts, gp_ctx** out) {
  if (!out) return fail(nullptr, GP_EINVAL, "null output pointer");
  *out = nullptr;
  gp_ctx* c = nullptr;
  try {
    c = new gp_ctx();
    std::string err;
    gp_status s = gp::build_plan(mesh, ls, opts, c->plan, err);
    if (s != GP_OK) {
      delete c;
      return fail(nullptr, s, err);
    }
  } catch (const std::bad_alloc&) {
    delete c;
    return fail(nullptr, GP_ENOMEM, "host allocation failed while building the plan");
  }
  c->elem = c->plan.precision == GP_FP32 ? 4 : 8;   // element size of x and y
  c->device = opts->device;
  c->no_scratch = opts->no_scratch != 0;
  {
    // kernel path: the brick path when a brick shape fits the shared-memory budget
    gp::Plan& p = c->plan;
    const size_t vbytes = p.precision == GP_FP32 ? 4 : 8;
    if (opts->kernel_path == GP_PATH_BRICK && p.num_faces() > 0 && !p.partitioned) {
      const size_t budget = opts->brick_smem > 0 ? (size_t)opts->brick_smem : (size_t)100 * 1024;
      const int fb = gpi::brick_default_fb(p.dim, p.k);
      const size_t extra = (size_t)(p.dim == 3 ? 2 : 1) * fb * p.k * p.L * vbytes;   // jump planes
      try {
        c->use_brick = gp::build_bricks(p, (int)vbytes, (int)vbytes, extra, std::min(budget, gp::BRICK_MAX_SMEM));
      } catch (const std::bad_alloc&) {
        delete c;
        return fail(nullptr, GP_ENOMEM, "host allocation failed while building the brick tables");
      }
    }
    if (opts->kernel_path == GP_PATH_BRICK && !c->use_brick && p.num_faces() > 0) {
      delete c;
      return fail(nullptr, GP_EUNSUPPORTED, "no brick shape fits the shared-memory budget (use GP_PATH_AUTO)");
    }
    if (!c->use_brick) {
      if (opts->slabs < 0) {
        delete c;
        return fail(nullptr, GP_EINVAL, "slabs must be >= 0");
      }
      try {
        gp::build_slabs(p, std::min(opts->slabs, gpi::MAX_SLABS));
      } catch (const std::bad_alloc&) {
        delete c;
        return fail(nullptr, GP_ENOMEM, "host allocation failed while building the slab pipeline");
      }
    }
  }
  if (opts->device >= 0) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      delete c;
      return fail(nullptr, GP_EDEVICE, "no CUDA device available");
    }
    if (opts->device >= ndev) {
      delete c;
      return fail(nullptr, GP_EINVAL, "device ordinal out of range");
    }
    DeviceGuard g(opts->device);
    cudaError_t e = g.ok ? cudaSuccess : cudaErrorInvalidDevice;
    const gp::Plan& p = c->plan;
    std::vector<int2> zruns(p.zruns.size() / 2);
    std::memcpy(zruns.data(), p.zruns.data(), p.zruns.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = upload(&c->d_frows, p.frows);
    if (e == cudaSuccess) e = upload(&c->d_lwin, p.lwin);
    if (e == cudaSuccess) e = upload(&c->d_lrow, p.lrow);
    if (e == cudaSuccess) e = upload(&c->d_zruns, zruns);
    const size_t vbytes = p.precision == GP_FP32 ? 4 : 8;
    if (c->use_brick) {
      if (e == cudaSuccess) e = upload(&c->d_bdesc, p.bdesc);
      if (e == cudaSuccess) e = upload(&c->d_bcell, p.bcell);
      if (e == cudaSuccess) e = upload(&c->d_bccoord, p.bccoord);
      if (e == cudaSuccess) e = upload(&c->d_bface, p.bface);
      if (e == cudaSuccess) e = upload(&c->d_rowtab, p.rowtab);
      if (e == cudaSuccess) e = upload(&c->d_pnode, p.pnode);
      if (e == cudaSuccess) e = upload(&c->d_poff, p.poff);
      if (e == cudaSuccess) e = upload(&c->d_pslot, p.pslot);
      const size_t part_bytes = gpi::brick_scratch_bytes(c);
      if (e == cudaSuccess && part_bytes > 0 && !opts->no_scratch) e = cudaMalloc(&c->d_part, part_bytes);
    }
    // face outputs W_F of the face + lift path: float, double, or a (hi, lo) float pair per value
    const size_t tp_bytes = (size_t)p.num_faces() * p.L * (2 * p.k + 1) * vbytes;
    if (e == cudaSuccess && tp_bytes > 0 && !opts->no_scratch && !c->use_brick) e = cudaMalloc(&c->d_tp, tp_bytes);
    if (e != cudaSuccess) {
      std::string m = std::string("device setup: ") + cudaGetErrorString(e);
      free_device(c);
      delete c;
      return fail(nullptr, e == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA, m);
    }
    c->on_device = true;
    if (c->use_brick) gpi::brick_tiles_lookup(c->device, c->plan.dim, c->plan.k, c->plan.precision, &c->tiles);
    else gpi::tiles_lookup(c->device, c->plan.dim, c->plan.k, c->plan.precision, &c->tiles);
  }
  *out = c;
  return GP_OK;
}

void gp_destroy(gp_ctx* ctx) {
  if (!ctx) return;
  {
    // release the cached gp_apply_batched batches that hold this context
    std::lock_guard<std::mutex> lock(g_batched_mu);
    for (auto it = g_batched.begin(); it != g_batched.end();) {
      if (std::find(it->first.ctxs.begin(), it->first.ctxs.end(), ctx) != it->first.ctxs.end()) {
        gp_batch_destroy(it->second);
        it = g_batched.erase(it);
      } else {
        ++it;
      }
    }
  }
  if (ctx->on_device) {
    DeviceGuard g(ctx->device);
    free_device(ctx);
  }
  delete ctx;
}

gp_status gp_num_active_dofs(const gp_ctx* ctx, int64_t* n) {
  if (!ctx || !n) return fail(ctx, GP_EINVAL, "null argument");
  *n = ctx->plan.n_active;
  return GP_OK;
}

gp_status gp_num_ghost_faces(const gp_ctx* ctx, int64_t* nf) {
  if (!ctx || !nf) return fail(ctx, GP_EINVAL, "null argument");
  *nf = ctx->plan.num_faces();
  return GP_OK;
}

gp_status gp_num_touched_dofs(const gp_ctx* ctx, int64_t* n) {
  if (!ctx || !n) return fail(ctx, GP_EINVAL, "null argument");
  *n = ctx->plan.n_touched;
  return GP_OK;
}

gp_status gp_cell_counts(const gp_ctx* ctx, int64_t counts[3]) {
  if (!ctx || !counts) return fail(ctx, GP_EINVAL, "null argument");
  for (int i = 0; i < 3; ++i) counts[i] = ctx->plan.cell_counts[i];
  return GP_OK;
}

gp_status gp_active_dof_coords(const gp_ctx* ctx, double* xyz) {
  if (!ctx || !xyz) return fail(ctx, GP_EINVAL, "null argument");
  gp::active_coords(ctx->plan, xyz);
  return GP_OK;
}

gp_status gp_ghost_faces(const gp_ctx* ctx, int32_t* axis, int64_t* cell) {
  if (!ctx || !axis || !cell) return fail(ctx, GP_EINVAL, "null argument");
  const gp::Plan& p = ctx->plan;
  for (int a = 0; a < p.dim; ++a)
    for (int64_t f = p.fstart[a]; f < p.fstart[a + 1]; ++f) {
      axis[f] = a;
      cell[f] = p.face_cell[f];
    }
  return GP_OK;
}

gp_status gp_cell_classes(const gp_ctx* ctx, int8_t* cls) {
  if (!ctx || !cls) return fail(ctx, GP_EINVAL, "null argument");
  std::memcpy(cls, ctx->plan.cls.data(), ctx->plan.cls.size());
  return GP_OK;
}

gp_status gp_partition_info(const gp_ctx* ctx, gp_partition* out) {
  if (!ctx || !out) return fail(ctx, GP_EINVAL, "null argument");
  const gp::Plan& p = ctx->plan;
  out->layer_lo = p.part_lo;
  out->layer_hi = p.part_hi;
  out->offset = p.g_offset;
  out->n_local = p.n_active;
  out->n_owned = p.n_owned;
  out->n_lower = p.n_lower;
  out->n_global = p.n_global;
  return GP_OK;
}

gp_status gp_partition_slabs(const gp_mesh* mesh, const gp_levelset* ls, const gp_opts* opts, int nparts,
                             int32_t* bounds) {
  try {
    std::string err;
    gp_status s = gp::partition_slabs(mesh, ls, opts, nparts, bounds, err);
    if (s != GP_OK) return fail(nullptr, s, err);
    return GP_OK;
  } catch (const std::exception& e) {
    return fail(nullptr, GP_ENOMEM, e.what());
  }
}

gp_status gp_kernel_path(const gp_ctx* ctx, int* path, int32_t* bdim, int64_t* counts) {
  if (!ctx || !path) return fail(ctx, GP_EINVAL, "null argument");
  const gp::Plan& p = ctx->plan;
  *path = ctx->use_brick ? GP_PATH_BRICK : GP_PATH_FACE_LIFT;
  if (bdim)
    for (int a = 0; a < 3; ++a) bdim[a] = ctx->use_brick ? p.bdim[a] : 0;
  if (counts) {
    counts[0] = ctx->use_brick ? p.num_bricks() : std::max(1, p.num_slabs());
    counts[1] = ctx->use_brick ? p.num_plane_nodes() : 0;
    counts[2] = ctx->use_brick ? (int64_t)gpi::brick_scratch_bytes(ctx)
                               : p.num_faces() * p.L * (2 * p.k + 1) * (p.precision == GP_FP32 ? 4 : 8);
  }
  return GP_OK;
}

gp_status gp_reference_1d(const gp_ctx* ctx, double* mass, double* jumps, double* scale) {
  if (!ctx || !mass || !jumps || !scale) return fail(ctx, GP_EINVAL, "null argument");
  const gp::Plan& p = ctx->plan;
  std::memcpy(mass, p.mass.data(), p.mass.size() * sizeof(double));
  std::memcpy(jumps, p.jumps.data(), p.jumps.size() * sizeof(double));
  std::memcpy(scale, p.scale.data(), p.scale.size() * sizeof(double));
  return GP_OK;
}

gp_status gp_profile_enable(gp_ctx* ctx, int enable) {
  if (!ctx) return fail(nullptr, GP_EINVAL, "null context");
  if (!ctx->on_device) return fail(ctx, GP_EDEVICE, "context was built host-only (device = -1)");
  ctx->prof = enable != 0;
  ctx->nprof = 0;
  return GP_OK;
}

gp_status gp_profile_read(gp_ctx* ctx, double ms[2], int64_t* calls) {
  if (!ctx || !ms || !calls) return fail(ctx, GP_EINVAL, "null argument");
  DeviceGuard g(ctx->device);
  ms[0] = ms[1] = 0.0;
  for (int64_t i = 0; i < ctx->nprof; ++i) {
    cudaEvent_t* e = &ctx->ev[3 * i];
    GP_CUDA(ctx, cudaEventSynchronize(e[2]));
    float a = 0.f, b = 0.f;
    GP_CUDA(ctx, cudaEventElapsedTime(&a, e[0], e[1]));
    GP_CUDA(ctx, cudaEventElapsedTime(&b, e[1], e[2]));
    ms[0] += a;
    ms[1] += b;
  }
  *calls = ctx->nprof;
  return GP_OK;
}

gp_status gp_apply(gp_ctx* ctx, const void* x, void* y, void* stream) {
  gp_status s = check_apply(ctx, x, y);
  if (s != GP_OK) return s;
  if (ctx->plan.n_active == 0) return GP_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, GP_ECUDA, "cudaSetDevice failed");
  return launch(ctx, x, y, 0, (cudaStream_t)stream);
}

gp_status gp_apply_noalloc(gp_ctx* ctx, const void* x, void* y, void* stream) {
  gp_status s = check_apply(ctx, x, y);
  if (s != GP_OK) return s;
  const gp::Plan& p = ctx->plan;
  const size_t vbytes = p.precision == GP_FP32 ? 4 : 8;
  // the scratch of the context's kernel path: partial grids (brick) or face outputs (face + lift)
  const size_t need = ctx->use_brick ? gpi::brick_scratch_bytes(ctx)
                                     : (size_t)p.num_faces() * p.L * (2 * p.k + 1) * vbytes;
  if (need > gp::noalloc_scratch_bytes())
    return fail(ctx, GP_EINVAL,
                std::string("gp_apply_noalloc: the ") + (ctx->use_brick ? "plane partial sums" : "face outputs") +
                    " need " + std::to_string(need) + " bytes, more than the fixed scratch of " +
                    std::to_string(gp::noalloc_scratch_bytes()) + " bytes; use gp_apply");
  if (p.n_active == 0) return GP_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, GP_ECUDA, "cudaSetDevice failed");
  void* scratch = nullptr;
  const cudaError_t e = gp::noalloc_scratch(ctx->device, &scratch);
  if (e != cudaSuccess)
    return fail(ctx, GP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  return launch(ctx, x, y, 0, (cudaStream_t)stream, scratch, false);
}

gp_status gp_apply_add(gp_ctx* ctx, const void* x, void* y, void* stream) {
  gp_status s = check_apply(ctx, x, y);
  if (s != GP_OK) return s;
  if (ctx->plan.n_active == 0 || ctx->plan.num_faces() == 0) return GP_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, GP_ECUDA, "cudaSetDevice failed");
  return launch(ctx, x, y, 1, (cudaStream_t)stream);
}

gp_status gp_apply_host(gp_ctx* ctx, const void* x_host, void* y_host, void* stream) {
  if (!ctx) return fail(nullptr, GP_EINVAL, "null context");
  if (!ctx->on_device) return fail(ctx, GP_EDEVICE, "context was built host-only (device = -1)");
  const int64_t n = ctx->plan.n_active;
  ctx->host_bytes[0] = ctx->host_bytes[1] = 0;
  if (n == 0) return GP_OK;
  if (!x_host || !y_host) return fail(ctx, GP_EINVAL, "null x or y");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, GP_ECUDA, "cudaSetDevice failed");
  const size_t bytes = (size_t)n * ctx->elem;
  if (!ctx->d_xh) GP_CUDA(ctx, cudaMalloc(&ctx->d_xh, bytes));
  cudaStream_t st = (cudaStream_t)stream;
  if (!ctx->d_yh) GP_CUDA(ctx, cudaMalloc(&ctx->d_yh, bytes));
  ctx->host_bytes[1] = (int64_t)bytes;
  // a page-locked x is read by a gather kernel on the touched DoFs only (the only entries the
  // face kernel reads); other memory is copied whole
  const void* xdev = gpi::device_view(x_host);
  if (xdev) {
    GP_CUDA(ctx, gpi::ensure_touched_runs(ctx));
    ctx->host_bytes[0] = ctx->plan.n_touched * ctx->elem;
  } else {
    ctx->host_bytes[0] = (int64_t)bytes;
  }
  if (gpi::device_view(y_host)) {
    // a page-locked y: the apply runs as a slab pipeline; each slab's part of x is gathered on
    // one stream before its face launch, and each slab's finished part of y goes back on another
    // while the later slabs compute
    GP_CUDA(ctx, gpi::ensure_host_pipeline(ctx));
    const int ns = (int)(ctx->hslabs.size() / gp::SLAB);
    if (ns > 1) {
      gpi::SlabRun run;
      run.table = ctx->hslabs.data();
      run.n = ns;
      run.events = ctx->hev.data();
      if (xdev) {
        for (int sl = 0; sl < ns; ++sl) {
          const int32_t r0 = ctx->hxrun[sl], r1 = ctx->hxrun[sl + 1];
          GP_CUDA(ctx, gpi::gather_runs(xdev, ctx->d_xh, ctx->d_truns + r0, r1 - r0, ctx->elem, ctx->hin));
          GP_CUDA(ctx, cudaEventRecord(ctx->hgev[sl], ctx->hin));
        }
        run.inputs = ctx->hgev.data();
      } else {
        GP_CUDA(ctx, cudaMemcpyAsync(ctx->d_xh, x_host, bytes, cudaMemcpyHostToDevice, st));
      }
      gp_status s = launch(ctx, ctx->d_xh, ctx->d_yh, 0, st, nullptr, false, nullptr, 3, &run);
      if (s != GP_OK) return s;
      for (int sl = 0; sl < ns; ++sl) {
        const int64_t lo = ctx->hbounds[sl], hi = ctx->hbounds[sl + 1];
        GP_CUDA(ctx, cudaStreamWaitEvent(ctx->hcopy, ctx->hev[sl], 0));
        if (hi > lo)
          GP_CUDA(ctx, cudaMemcpyAsync((char*)y_host + lo * ctx->elem, (const char*)ctx->d_yh + lo * ctx->elem,
                                       (size_t)(hi - lo) * ctx->elem, cudaMemcpyDeviceToHost, ctx->hcopy));
      }
      GP_CUDA(ctx, cudaStreamSynchronize(ctx->hcopy));
      GP_CUDA(ctx, cudaStreamSynchronize(ctx->hin));
      GP_CUDA(ctx, cudaStreamSynchronize(st));
      return GP_OK;
    }
  }
  if (xdev) GP_CUDA(ctx, gpi::gather_runs(xdev, ctx->d_xh, ctx->d_truns, ctx->ntruns, ctx->elem, st));
  else GP_CUDA(ctx, cudaMemcpyAsync(ctx->d_xh, x_host, bytes, cudaMemcpyHostToDevice, st));
  gp_status s = launch(ctx, ctx->d_xh, ctx->d_yh, 0, st);
  if (s != GP_OK) return s;
  GP_CUDA(ctx, cudaMemcpyAsync(y_host, ctx->d_yh, bytes, cudaMemcpyDeviceToHost, st));
  GP_CUDA(ctx, cudaStreamSynchronize(st));
  return GP_OK;
}

gp_status gp_apply_host_bytes(const gp_ctx* ctx, int64_t* h2d, int64_t* d2h) {
  if (!ctx || !h2d || !d2h) return fail(ctx, GP_EINVAL, "null argument");
  *h2d = ctx->host_bytes[0];
  *d2h = ctx->host_bytes[1];
  return GP_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches --
struct gp_batch {
  int device = -1, nprob = 0, nrhs = 0;
  std::vector<gp_ctx*> ctxs;
  struct Group {
    int dim = 0, k = 0, prec = 0;
    std::vector<int> prob, rhs;        // segment -> problem, right-hand side
    void* d_fsegs = nullptr;
    void* d_lsegs = nullptr;
    void* d_ptrs[2] = {nullptr, nullptr};
    void* h_ptrs[2] = {nullptr, nullptr};  // pinned: read by the graph's copy node at replay
    int face_blocks = 0, lift_blocks = 0;
    gp::BatchOps ops{};
    gp::Tiles tiles{};                 // the tile shape of the group's first context
  };
  std::vector<Group> groups;
  void* d_w = nullptr;
  void* d_gs = nullptr;                // per problem: the scaled jump vectors s_j g_j
  size_t w_bytes = 0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  bool pending[2] = {false, false};
  int slot = 0;
  int64_t launches = 0;   // graph replays made through gp_apply_batched
  std::string err;
};

namespace {

gp::BatchOps ops_for(int prec, int dim) {
  if (prec == GP_FP64) return dim == 2 ? gp::batch_ops_f64_d2() : gp::batch_ops_f64_d3();
  if (prec == GP_FP64_FF) return dim == 2 ? gp::batch_ops_ff_d2() : gp::batch_ops_ff_d3();
  return dim == 2 ? gp::batch_ops_f32_d2() : gp::batch_ops_f32_d3();
}

void batch_free(gp_batch* b) {
  for (int i = 0; i < 2; ++i) {
    if (b->pending[i] && b->done[i]) cudaEventSynchronize(b->done[i]);
    if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
    if (b->graph[i]) cudaGraphDestroy(b->graph[i]);
    if (b->done[i]) cudaEventDestroy(b->done[i]);
  }
  for (auto& g : b->groups) {
    if (g.d_fsegs) cudaFree(g.d_fsegs);
    if (g.d_lsegs) cudaFree(g.d_lsegs);
    for (int i = 0; i < 2; ++i) {
      if (g.d_ptrs[i]) cudaFree(g.d_ptrs[i]);
      if (g.h_ptrs[i]) cudaFreeHost(g.h_ptrs[i]);
    }
  }
  if (b->d_w) cudaFree(b->d_w);
  if (b->d_gs) cudaFree(b->d_gs);
  if (b->cap) cudaStreamDestroy(b->cap);
}

}  // namespace

extern "C" {

gp_status gp_batch_create(gp_ctx* const* ctxs, int nprob, int nrhs, gp_batch** out) {
  if (!out) return fail(nullptr, GP_EINVAL, "null output pointer");
  *out = nullptr;
  if (nprob < 1 || nrhs < 1 || !ctxs) return fail(nullptr, GP_EINVAL, "bad batch arguments");
  for (int p = 0; p < nprob; ++p) {
    if (!ctxs[p] || !ctxs[p]->on_device) return fail(nullptr, GP_EINVAL, "every context must be on a device");
    if (ctxs[p]->device != ctxs[0]->device) return fail(nullptr, GP_EINVAL, "all contexts must share a device");
  }
  gp_batch* b = new (std::nothrow) gp_batch();
  if (!b) return fail(nullptr, GP_ENOMEM, "host allocation failed");
  b->device = ctxs[0]->device;
  b->nprob = nprob;
  b->nrhs = nrhs;
  b->ctxs.assign(ctxs, ctxs + nprob);
  DeviceGuard dg(b->device);
  // group problems by (dimension, degree, arithmetic, stabilisation)
  std::map<std::tuple<int, int, int, int>, int> key;   // (d, k, arithmetic, stabilisation): one set of 1D data
  for (int p = 0; p < nprob; ++p) {
    const gp::Plan& pl = ctxs[p]->plan;
    auto kk = std::make_tuple(pl.dim, pl.k, pl.precision, pl.stabilization);
    auto it = key.find(kk);
    int gi;
    if (it == key.end()) {
      gi = (int)b->groups.size();
      key[kk] = gi;
      b->groups.emplace_back();
      b->groups[gi].dim = pl.dim;
      b->groups[gi].k = pl.k;
      b->groups[gi].prec = pl.precision;
      b->groups[gi].ops = ops_for(pl.precision, pl.dim);
      b->groups[gi].tiles = ctxs[p]->tiles;
    } else {
      gi = it->second;
    }
    for (int r = 0; r < nrhs; ++r) {
      b->groups[gi].prob.push_back(p);
      b->groups[gi].rhs.push_back(r);
    }
  }
  // face-output buffers, one per segment, 256-byte aligned in one allocation
  std::vector<std::vector<size_t>> woff(b->groups.size());
  size_t total = 0;
  for (size_t gi = 0; gi < b->groups.size(); ++gi)
    for (int p : b->groups[gi].prob) {
      const gp::Plan& pl = ctxs[p]->plan;
      const size_t vb = pl.precision == GP_FP32 ? 4 : 8;
      woff[gi].push_back(total);
      total += ((size_t)pl.num_faces() * pl.L * (2 * pl.k + 1) * vb + 255) / 256 * 256;
    }
  cudaError_t e = cudaSuccess;
  if (total > 0) e = cudaMalloc(&b->d_w, total);
  b->w_bytes = total;
  // the scaled jump vectors of every problem, in its group's arithmetic (256-byte aligned)
  std::vector<size_t> gs_off(nprob, 0);
  {
    std::vector<unsigned char> all, one;
    for (size_t gi = 0; gi < b->groups.size(); ++gi)
      for (size_t i = 0; i < b->groups[gi].prob.size(); ++i) {
        const int pi = b->groups[gi].prob[i];
        if (b->groups[gi].rhs[i] != 0) continue;
        const gp::Plan& pl = ctxs[pi]->plan;
        b->groups[gi].ops.jumps(pl.k, pl.jumps.data(), pl.scale.data(), one);
        gs_off[pi] = all.size();
        all.insert(all.end(), one.begin(), one.end());
        all.resize((all.size() + 255) / 256 * 256, 0);
      }
    if (e == cudaSuccess && !all.empty()) e = cudaMalloc(&b->d_gs, all.size());
    if (e == cudaSuccess && !all.empty()) e = cudaMemcpy(b->d_gs, all.data(), all.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
    auto& g = b->groups[gi];
    std::vector<gp::SegSpec> specs(g.prob.size());
    for (size_t i = 0; i < g.prob.size(); ++i) {
      const gp_ctx* c = ctxs[g.prob[i]];
      const gp::Plan& pl = c->plan;
      gp::SegSpec& sp = specs[i];
      sp.fa.frows = c->d_frows;
      for (int a = 0; a < 4; ++a) {
        sp.fa.rbase[a] = pl.rbase[a];
        sp.fa.fstart[a] = pl.fstart[a];
      }
      sp.fa.zruns = c->d_zruns;
      sp.fa.nzruns = (int32_t)pl.num_zero_runs();
      sp.la.lwin = c->d_lwin;
      sp.la.lrow = c->d_lrow;
      sp.la.nlift = (int32_t)pl.num_lift_cells();
      sp.la.n_active = (int32_t)pl.n_active;
      sp.wp = (char*)b->d_w + woff[gi][i];
      sp.gs = (const char*)b->d_gs + gs_off[g.prob[i]];
      for (int j = 0; j < pl.k; ++j) sp.s[j] = pl.scale[j];
    }
    std::vector<unsigned char> fs, ls;
    if (!g.ops.pack(g.k, specs, g.tiles, fs, ls, g.face_blocks, g.lift_blocks)) {
      e = cudaErrorInvalidConfiguration;
      break;
    }
    e = cudaMalloc(&g.d_fsegs, fs.size());
    if (e == cudaSuccess) e = cudaMemcpy(g.d_fsegs, fs.data(), fs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&g.d_lsegs, ls.size());
    if (e == cudaSuccess) e = cudaMemcpy(g.d_lsegs, ls.data(), ls.size(), cudaMemcpyHostToDevice);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = cudaMalloc(&g.d_ptrs[i], g.prob.size() * 2 * sizeof(void*));
      if (e == cudaSuccess) e = cudaMallocHost(&g.h_ptrs[i], g.prob.size() * 2 * sizeof(void*));
      if (e == cudaSuccess) std::memset(g.h_ptrs[i], 0, g.prob.size() * 2 * sizeof(void*));
    }
  }
  // one graph per slot: copy the pointer table, then each group's face and lift launches
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    for (auto& g : b->groups) {
      if (e != cudaSuccess) break;
      const gp::Plan& pl0 = ctxs[g.prob[0]]->plan;
      e = cudaMemcpyAsync(g.d_ptrs[i], g.h_ptrs[i], g.prob.size() * 2 * sizeof(void*), cudaMemcpyHostToDevice,
                          b->cap);
      if (e == cudaSuccess)
        e = g.ops.run(g.k, g.d_fsegs, g.d_lsegs, g.d_ptrs[i], (int)g.prob.size(), g.face_blocks, g.lift_blocks,
                      pl0.jumps.data(), pl0.mass.data(), g.tiles, b->cap);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e == cudaSuccess) e = e2;
    b->graph[i] = graph;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[i], graph, 0);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    std::string m = std::string("batch setup: ") + cudaGetErrorString(e);
    batch_free(b);
    delete b;
    return fail(nullptr, e == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA, m);
  }
  *out = b;
  return GP_OK;
}

gp_status gp_batch_apply(gp_batch* b, const void* const* x, void* const* y, void* stream) {
  if (!b || !x || !y) return fail(nullptr, GP_EINVAL, "null argument");
  for (int p = 0; p < b->nprob; ++p)
    if ((!x[p] || !y[p]) && b->ctxs[p]->plan.n_active > 0) return fail(nullptr, GP_EINVAL, "null x or y");
  DeviceGuard dg(b->device);
  const int s = b->slot;
  b->slot ^= 1;
  // the slot's pinned table is read by the graph launched two applies ago
  if (b->pending[s]) {
    const cudaError_t e = cudaEventSynchronize(b->done[s]);
    if (e != cudaSuccess) return fail(nullptr, GP_ECUDA, std::string("batch: ") + cudaGetErrorString(e));
  }
  for (auto& g : b->groups) {
    void** tab = (void**)g.h_ptrs[s];
    for (size_t i = 0; i < g.prob.size(); ++i) {
      const gp_ctx* c = b->ctxs[g.prob[i]];
      const size_t off = (size_t)g.rhs[i] * c->plan.n_active * c->elem;
      tab[2 * i] = (void*)((const char*)x[g.prob[i]] + off);
      tab[2 * i + 1] = (void*)((char*)y[g.prob[i]] + off);
    }
  }
  cudaError_t e = cudaGraphLaunch(b->exec[s], (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaEventRecord(b->done[s], (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, GP_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  b->pending[s] = true;
  return GP_OK;
}

gp_status gp_batch_info(const gp_batch* b, int64_t* ngroups, int64_t* scratch_bytes) {
  if (!b || !ngroups || !scratch_bytes) return fail(nullptr, GP_EINVAL, "null argument");
  *ngroups = (int64_t)b->groups.size();
  *scratch_bytes = (int64_t)b->w_bytes;
  return GP_OK;
}

void gp_batch_destroy(gp_batch* b) {
  if (!b) return;
  DeviceGuard dg(b->device);
  batch_free(b);
  delete b;
}

}  // extern "C"

// ---------------------------------------------- gp_apply_batched (cached batches) --
extern "C" {

gp_status gp_apply_batched(gp_ctx* const* ctxs, int nprob, int nrhs, const void* const* x,
                           void* const* y, void* stream) {
  if (nprob < 0 || nrhs < 1 || (nprob > 0 && (!ctxs || !x || !y)))
    return fail(nullptr, GP_EINVAL, "bad batched arguments");
  if (nprob == 0) return GP_OK;
  const int prec = ctxs[0] ? ctxs[0]->plan.precision : -1;
  const int dev = ctxs[0] ? ctxs[0]->device : -1;
  for (int p = 0; p < nprob; ++p) {
    gp_status s = check_apply(ctxs[p], x[p], y[p]);
    if (s != GP_OK) return fail(nullptr, s, std::string("problem ") + std::to_string(p) + ": " +
                                               (ctxs[p] ? ctxs[p]->err : std::string("null context")));
    if (ctxs[p]->plan.precision != prec || ctxs[p]->device != dev)
      return fail(nullptr, GP_EINVAL, "all contexts must share precision and device");
  }
  // the graph-replayed batch of this (contexts, nrhs) list: built on the first call, replayed after
  gp_batch* b = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_batched_mu);
    const BatchedKey key{std::vector<gp_ctx*>(ctxs, ctxs + nprob), nrhs};
    auto it = g_batched.find(key);
    if (it != g_batched.end()) {
      b = it->second;
    } else {
      const gp_status s = gp_batch_create(ctxs, nprob, nrhs, &b);
      if (s != GP_OK) return s;
      g_batched[key] = b;
    }
  }
  gp_status s = gp_batch_apply(b, x, y, stream);
  if (s == GP_OK) b->launches++;
  return s;
}

gp_status gp_apply_batched_info(gp_ctx* const* ctxs, int nprob, int nrhs, int64_t* graph_launches) {
  if (!graph_launches || nprob < 1 || !ctxs) return fail(nullptr, GP_EINVAL, "bad arguments");
  std::lock_guard<std::mutex> lock(g_batched_mu);
  auto it = g_batched.find(BatchedKey{std::vector<gp_ctx*>(ctxs, ctxs + nprob), nrhs});
  if (it == g_batched.end()) return fail(nullptr, GP_EINVAL, "no batch of these contexts has been applied");
  *graph_launches = it->second->launches;
  return GP_OK;
}

}  // extern "C"
