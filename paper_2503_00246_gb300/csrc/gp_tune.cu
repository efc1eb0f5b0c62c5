// Tile shapes of the face and lift launches and their autotuner.
//
// The tile shape is (faces per face CTA, owner cells per lift CTA, lift threads); on the
// brick path only the first field counts (faces per chunk of the brick kernel), and the
// autotuner times whole applies for it.
// gp_autotune times each candidate on the context's own tables with CUDA events,
// with the L2 flushed before every timed launch (the operator's operands are
// read from HBM in a real solve), and keeps the fastest face and lift shapes.
// The choice is recorded in a process-wide table keyed by (device, dimension,
// degree, arithmetic); gp_setup starts new contexts from that table, and a
// batch takes the shape of each group's first context.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gp_internal.h"

namespace {

std::mutex g_tiles_mu;
std::map<std::tuple<int, int, int, int>, gp::Tiles> g_tiles;        // face + lift path
std::map<std::tuple<int, int, int, int>, gp::Tiles> g_brick_tiles;  // brick path (fb only)

}  // namespace

namespace gpi {

gp::TileOps tile_ops(int dim, int precision) {
  if (precision == GP_FP64) return dim == 2 ? gp::tile_ops_f64_d2() : gp::tile_ops_f64_d3();
  if (precision == GP_FP64_FF) return dim == 2 ? gp::tile_ops_ff_d2() : gp::tile_ops_ff_d3();
  return dim == 2 ? gp::tile_ops_f32_d2() : gp::tile_ops_f32_d3();
}

bool tiles_lookup(int device, int dim, int k, int precision, gp::Tiles* out) {
  std::lock_guard<std::mutex> lk(g_tiles_mu);
  auto it = g_tiles.find(std::make_tuple(device, dim, k, precision));
  if (it == g_tiles.end()) return false;
  *out = it->second;
  return true;
}

void tiles_record(int device, int dim, int k, int precision, const gp::Tiles& t) {
  std::lock_guard<std::mutex> lk(g_tiles_mu);
  g_tiles[std::make_tuple(device, dim, k, precision)] = t;
}

bool brick_tiles_lookup(int device, int dim, int k, int precision, gp::Tiles* out) {
  std::lock_guard<std::mutex> lk(g_tiles_mu);
  auto it = g_brick_tiles.find(std::make_tuple(device, dim, k, precision));
  if (it == g_brick_tiles.end()) return false;
  *out = it->second;
  return true;
}

}  // namespace gpi

using gpi::DeviceGuard;
using gpi::fail;

namespace {

gp::Tiles from_abi(const gp_tiles& t) {
  gp::Tiles r;
  r.fb = t.faces_per_cta;
  r.lcb = t.lift_cells_per_cta;
  r.lnt = t.lift_threads;
  return r;
}

gp_tiles to_abi(const gp::Tiles& t) {
  gp_tiles r;
  r.faces_per_cta = t.fb;
  r.lift_cells_per_cta = t.lcb;
  r.lift_threads = t.lnt;
  return r;
}

int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}

// Candidate shapes: face CTAs of about 64..512 threads; lift CTAs of 64..512 threads
// with one or two rows per thread.
void candidates(const gp::Plan& p, const gp::TileOps& ops, std::vector<gp::Tiles>& face,
                std::vector<gp::Tiles>& lift) {
  const gp::Tiles d = ops.defaults(p.k);
  const int L = p.L, KR = (int)ipow(p.k, p.dim - 1);
  face.clear();
  lift.clear();
  for (int T : {64, 96, 128, 192, 256, 384, 512}) {
    gp::Tiles t = d;
    t.fb = std::max(1, T / L);
    bool dup = false;
    for (const auto& u : face) dup = dup || u.fb == t.fb;
    if (!dup && ops.resolve(p.k, t)) face.push_back(t);
  }
  for (int T : {64, 128, 256, 512})
    for (int depth : {1, 2}) {
      gp::Tiles t = d;
      t.lnt = T;
      t.lcb = std::max(1, depth * T / KR);
      bool dup = false;
      for (const auto& u : lift) dup = dup || (u.lnt == t.lnt && u.lcb == t.lcb);
      if (!dup && ops.resolve(p.k, t)) lift.push_back(t);
    }
}

}  // namespace

extern "C" {

gp_status gp_get_tiles(const gp_ctx* ctx, gp_tiles* out) {
  if (!ctx || !out) return fail(ctx, GP_EINVAL, "null argument");
  gp::Tiles t = ctx->tiles;
  if (!gpi::tile_ops(ctx->plan.dim, ctx->plan.precision).resolve(ctx->plan.k, t))
    return fail(ctx, GP_EINVAL, "the context holds an invalid tile shape");
  *out = to_abi(t);
  return GP_OK;
}

gp_status gp_set_tiles(gp_ctx* ctx, const gp_tiles* tiles) {
  if (!ctx || !tiles) return fail(ctx, GP_EINVAL, "null argument");
  gp::Tiles t = from_abi(*tiles);
  if (!gpi::tile_ops(ctx->plan.dim, ctx->plan.precision).resolve(ctx->plan.k, t))
    return fail(ctx, GP_EINVAL, "tile shape out of range (threads per CTA, shared memory or lift threads)");
  ctx->tiles = from_abi(*tiles);
  return GP_OK;
}

gp_status gp_tiles_record(int device, int dim, int degree, int precision, const gp_tiles* tiles) {
  if (!tiles) return fail(nullptr, GP_EINVAL, "null argument");
  if ((dim != 2 && dim != 3) || degree < 1 || degree > gp::KMAX ||
      (precision != GP_FP64 && precision != GP_FP32 && precision != GP_FP64_FF))
    return fail(nullptr, GP_EINVAL, "bad (dim, degree, precision)");
  gp::Tiles t = from_abi(*tiles);
  if (!gpi::tile_ops(dim, precision).resolve(degree, t)) return fail(nullptr, GP_EINVAL, "tile shape out of range");
  gpi::tiles_record(device, dim, degree, precision, from_abi(*tiles));
  return GP_OK;
}

gp_status gp_tiles_lookup(int device, int dim, int degree, int precision, gp_tiles* out) {
  if (!out) return fail(nullptr, GP_EINVAL, "null argument");
  gp::Tiles t;
  if (!gpi::tiles_lookup(device, dim, degree, precision, &t)) return fail(nullptr, GP_EINVAL, "no entry");
  *out = to_abi(t);
  return GP_OK;
}

gp_status gp_autotune(gp_ctx* ctx, int reps, gp_tiles* best, double* ms) {
  if (!ctx) return fail(nullptr, GP_EINVAL, "null context");
  if (!ctx->on_device) return fail(ctx, GP_EDEVICE, "context was built host-only (device = -1)");
  if (reps < 1) return fail(ctx, GP_EINVAL, "reps must be >= 1");
  const gp::Plan& p = ctx->plan;
  const gp::TileOps ops = gpi::tile_ops(p.dim, p.precision);
  std::vector<gp::Tiles> face, lift;
  candidates(p, ops, face, lift);
  gp::Tiles cur = ctx->tiles;
  if (!ops.resolve(p.k, cur)) cur = ops.defaults(p.k);
  if (p.num_faces() == 0 || face.empty() || lift.empty()) {
    if (best) *best = to_abi(cur);
    if (ms) ms[0] = ms[1] = 0.0;
    return GP_OK;
  }
  DeviceGuard dg(ctx->device);
  // operands of the timed launches and a buffer larger than the L2 to flush it
  const size_t vb = (size_t)p.n_active * ctx->elem;
  const size_t flush_bytes = (size_t)256 << 20;
  void *x = nullptr, *y = nullptr, *fl = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&x, std::max<size_t>(vb, 16));
  if (e == cudaSuccess) e = cudaMalloc(&y, std::max<size_t>(vb, 16));
  if (e == cudaSuccess) e = cudaMalloc(&fl, flush_bytes);
  if (e == cudaSuccess) e = cudaMemset(x, 0, std::max<size_t>(vb, 16));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  gp_status status = GP_OK;
  // mean time of one kernel (which = 1 face, 2 lift) over reps cold-L2 launches
  auto time_one = [&](const gp::Tiles& t, int which, double& out_ms) -> bool {
    double total = 0;
    for (int r = -1; r < reps && e == cudaSuccess; ++r) {   // r = -1: untimed warm-up
      e = cudaMemsetAsync(fl, r & 0xff, flush_bytes, st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      if (e == cudaSuccess && gpi::launch(ctx, x, y, 0, st, nullptr, false, &t, which) != GP_OK) {
        status = GP_ECUDA;
        return false;
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float m = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&m, e0, e1);
      if (r >= 0) total += m;
    }
    out_ms = total / reps;
    return e == cudaSuccess;
  };
  gp::Tiles bf = cur, bl = cur;
  double tf = 1e30, tl = 1e30;
  if (ctx->use_brick) {
    // brick path: faces per chunk of the brick kernel, timed over whole applies
    for (const gp::Tiles& t : face) {
      double m;
      if (!time_one(t, 3, m)) break;
      if (m < tf) { tf = m; bf = t; }
    }
    tl = 0.0;
  }
  for (const gp::Tiles& t : face) {
    if (ctx->use_brick) break;
    double m;
    if (!time_one(t, 1, m)) break;
    if (m < tf) { tf = m; bf = t; }
  }
  // the lift reads the face outputs of the best face shape
  if (!ctx->use_brick && e == cudaSuccess && status == GP_OK &&
      gpi::launch(ctx, x, y, 0, st, nullptr, false, &bf, 1) != GP_OK)
    status = GP_ECUDA;
  for (const gp::Tiles& t : lift) {
    if (ctx->use_brick || e != cudaSuccess || status != GP_OK) break;
    double m;
    if (!time_one(t, 2, m)) break;
    if (m < tl) { tl = m; bl = t; }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (x) cudaFree(x);
  if (y) cudaFree(y);
  if (fl) cudaFree(fl);
  if (status != GP_OK) return status;   // message set by launch
  if (e != cudaSuccess)
    return fail(ctx, e == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA,
                std::string("autotune: ") + cudaGetErrorString(e));
  gp::Tiles chosen;
  chosen.fb = bf.fb;
  chosen.lcb = bl.lcb;
  chosen.lnt = bl.lnt;
  ctx->tiles = chosen;
  if (ctx->use_brick) {
    std::lock_guard<std::mutex> lk(g_tiles_mu);
    g_brick_tiles[std::make_tuple(ctx->device, p.dim, p.k, p.precision)] = chosen;
  } else {
    gpi::tiles_record(ctx->device, p.dim, p.k, p.precision, chosen);
  }
  if (best) *best = to_abi(chosen);
  if (ms) {
    ms[0] = tf;
    ms[1] = tl;
  }
  return GP_OK;
}

}  // extern "C"
