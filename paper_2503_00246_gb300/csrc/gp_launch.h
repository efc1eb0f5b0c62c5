// Host-side launch interface between the C ABI and the templated kernels.
#pragma once

#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>

#include "gp_brick.cuh"
#include "gp_cell.cuh"
#include "gp_kernels.cuh"

namespace gp {

struct ApplyArgs {
  int dim = 0, k = 0;
  const void* x = nullptr;   // device, n_active elements
  void* y = nullptr;         // device, n_active elements
  void* tp = nullptr;        // device scratch: face outputs, nf * (2k+1) * L values
  int add = 0;               // 0: y = Gx, 1: y += Gx
  const int32_t* frows = nullptr;
  int64_t rbase[4] = {0, 0, 0, 0};
  int32_t fstart[4] = {0, 0, 0, 0};
  LiftArgs la{};
  const int2* zruns = nullptr;
  int32_t nzruns = 0;        // zero runs to fill (0 for the add form)
  const double* g = nullptr; // host FP64: k x (2k+1)
  const double* m = nullptr; // host FP64: (k+1)^2
  const double* s = nullptr; // host FP64: k
  cudaEvent_t* ev = nullptr;  // optional: 3 events recorded around the two kernels
  Tiles tiles{};              // 0 fields: the defaults of default_tiles
  int which = 3;              // bit 0: face kernel, bit 1: lift kernel (the autotuner times them apart)
  const int32_t* slabs = nullptr;  // host: SLAB ints per slab (see Plan::slabs); nslab > 1: slab pipeline
  int nslab = 0;
  cudaEvent_t* slab_events = nullptr;  // host, nslab events: recorded after each slab's lift (the
                                       // face launches then follow them in plain stream order)
  cudaEvent_t* slab_inputs = nullptr;  // host, nslab events (with slab_events): the face launch of
                                       // slab s waits for slab_inputs[s] (its part of x is in place)
  bool brick = false;         // the brick path (brick kernel + plane fixup) instead of face + lift
  BrickArgs ba{};             // brick tables (zero-run fields are filled by the launcher)
  PlaneArgs pa{};             // plane-fixup tables
};

// Default tile shape: about 256 threads per CTA, one item per thread.
template <int D, int K>
Tiles default_tiles_t() {
  Tiles t;
  t.fb = Shape<D, K>::FB;
  t.lcb = LiftShape<D, K>::CB;
  t.lnt = LiftShape<D, K>::NT;
  return t;
}

// Fills zero fields of t with the defaults and checks the limits of the kernels
// (threads per CTA <= MAX_CTA_THREADS, lift threads a multiple of 32, dynamic
// shared memory <= MAX_DYN_SMEM).  Returns false if t is out of range.
template <int D, int K, typename V>
bool resolve_tiles(Tiles& t) {
  const Tiles d = default_tiles_t<D, K>();
  if (t.fb == 0) t.fb = d.fb;
  if (t.lcb == 0) t.lcb = d.lcb;
  if (t.lnt == 0) t.lnt = d.lnt;
  if (t.fb < 1 || t.fb * Shape<D, K>::L > MAX_CTA_THREADS || face_smem<D, K, V>(t.fb) > MAX_DYN_SMEM) return false;
  if (t.lnt < 32 || t.lnt > MAX_CTA_THREADS || t.lnt % 32 != 0) return false;
  if (t.lcb < 1 || lift_smem<D, K>(t.lcb) > MAX_DYN_SMEM) return false;
  return true;
}

// Per (arithmetic, dimension): default tiles and range check for degree k.
struct TileOps {
  Tiles (*defaults)(int k);
  bool (*resolve)(int k, Tiles& t);
};
TileOps tile_ops_f64_d2();
TileOps tile_ops_f64_d3();
TileOps tile_ops_f32_d2();
TileOps tile_ops_f32_d3();
TileOps tile_ops_ff_d2();
TileOps tile_ops_ff_d3();

#define GP_TILE_CASE(D, A, K) \
  case K: return resolve_tiles<D, K, typename A::V>(t);
#define GP_TILE_OPS(D, A)                                                                     \
  TileOps ops;                                                                                \
  ops.defaults = [](int k) -> Tiles {                                                         \
    switch (k) {                                                                              \
      case 1: return default_tiles_t<D, 1>();                                                 \
      case 2: return default_tiles_t<D, 2>();                                                 \
      case 3: return default_tiles_t<D, 3>();                                                 \
      case 4: return default_tiles_t<D, 4>();                                                 \
      case 5: return default_tiles_t<D, 5>();                                                 \
      case 6: return default_tiles_t<D, 6>();                                                 \
      case 7: return default_tiles_t<D, 7>();                                                 \
      default: return default_tiles_t<D, 8>();                                                \
    }                                                                                         \
  };                                                                                          \
  ops.resolve = [](int k, Tiles& t) -> bool {                                                 \
    switch (k) {                                                                              \
      GP_TILE_CASE(D, A, 1) GP_TILE_CASE(D, A, 2) GP_TILE_CASE(D, A, 3) GP_TILE_CASE(D, A, 4) \
      GP_TILE_CASE(D, A, 5) GP_TILE_CASE(D, A, 6) GP_TILE_CASE(D, A, 7) GP_TILE_CASE(D, A, 8) \
      default: return false;                                                                  \
    }                                                                                         \
  };                                                                                          \
  return ops;

// One entry point per (arithmetic, dimension); each dispatches on k = 1..8.
cudaError_t apply_f64_d2(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_f64_d3(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_f32_d2(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_f32_d3(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_ff_d2(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_ff_d3(const ApplyArgs& a, cudaStream_t st);

// Faces per chunk of the brick kernel: the tile's fb, else about 256 threads.
template <int D, int K>
inline int brick_fb(const Tiles& t) {
  constexpr int L = Shape<D, K>::L;
  const int fb = t.fb > 0 ? t.fb : Shape<D, K>::FB;
  return fb * L <= MAX_CTA_THREADS ? fb : MAX_CTA_THREADS / L;
}

constexpr size_t BRICK_MAX_SMEM = 200 * 1024;   // dynamic shared memory the brick kernel may ask for

// The brick path: brick kernel (zero-fill CTAs first), then the plane fixup as its
// programmatic dependent.  Ar.ev (3 events) brackets the two kernels when given.
template <int D, int K, class A>
cudaError_t run_brick(const ApplyArgs& Ar, const Consts<typename A::V, K>& c, cudaStream_t st) {
  using V = typename A::V;
  using IO = typename A::IO;
  constexpr int L = Shape<D, K>::L;
  const int fb = brick_fb<D, K>(Ar.tiles);
  BrickArgs ba = Ar.ba;
  ba.zruns = Ar.zruns;
  ba.nzruns = Ar.nzruns;
  ba.nzblocks = (Ar.nzruns + ZGROUP - 1) / ZGROUP;
  const size_t smem = brick_smem<D, K, V>(ba.maxown, ba.maxcell, fb);
  if (smem > BRICK_MAX_SMEM) return cudaErrorInvalidConfiguration;
  // the opt-in limit covers static + dynamic shared memory: raise it once per instantiation
  // and device, whatever this launch needs
  static bool smem_raised[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !smem_raised[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(brick_kernel<D, K, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)BRICK_MAX_SMEM);
    if (e != cudaSuccess) return e;
    smem_raised[dev] = true;
  }
  const int grid = ba.nzblocks + ba.nbricks;
  if (Ar.ev) cudaEventRecord(Ar.ev[0], st);
  if (grid > 0) brick_kernel<D, K, A><<<grid, fb * L, smem, st>>>((const IO*)Ar.x, (IO*)Ar.y, Ar.add, ba, fb, c);
  if (Ar.ev) cudaEventRecord(Ar.ev[1], st);
  if (Ar.pa.nplane > 0 && ba.nbricks > 0) {
    const int nb = (Ar.pa.nplane + 255) / 256;
    if (Ar.ev) {
      plane_fixup_kernel<A><<<nb, 256, 0, st>>>((IO*)Ar.y, Ar.add, Ar.pa);
    } else {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)nb);
      cfg.blockDim = dim3(256u);
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      const cudaError_t e = cudaLaunchKernelEx(&cfg, plane_fixup_kernel<A>, (IO*)Ar.y, Ar.add, Ar.pa);
      if (e != cudaSuccess) return e;
    }
  }
  if (Ar.ev) cudaEventRecord(Ar.ev[2], st);
  return cudaGetLastError();
}

// ints per slab of the slab pipeline: owner range [lo, hi), then per axis the face range [lo, hi)
constexpr int SLAB_INTS = 8;

// Launches kernel with programmatic stream serialization (it may start when its predecessor
// signals griddepcontrol.launch_dependents).
template <typename... P, typename... Args>
cudaError_t launch_pdl(void (*kernel)(P...), int grid, int threads, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// The face + lift path as a pipeline of slabs along the last axis, so that the face outputs of a
// slab are still in L2 when its lift reads them: face(0), lift(0), face(1), lift(1), ...  Slab s
// holds a range of owner cells and the faces that range needs and no earlier range needed.
// lift(s) waits for face(s) before it reads W; face(s + 1) starts once every CTA of lift(s) has
// passed that wait, overlaps lift(s) (it writes other face outputs and reads only x), and waits for
// lift(s) only before it exits, so that each grid completes after all earlier ones (the last lift
// completes last).  The first face launch also zero-fills.  With slab_events, an event is
// recorded after every lift (another stream can then take the slab's finished part of y) and
// each face launch follows it in plain stream order.
template <int D, int K, class A>
cudaError_t run_slabs(const ApplyArgs& Ar, const Consts<typename A::V, K>& c, const Tiles& t, cudaStream_t st) {
  using S = Shape<D, K>;
  using V = typename A::V;
  using IO = typename A::IO;
  const int R[3] = {S::L, (D == 3) ? S::NN * (K + 1) : S::NN, S::NN * (K + 1)};   // row entries per face
  constexpr int KR = LiftShape<D, K>::KR, NW = LiftShape<D, K>::NW;
  for (int s = 0; s < Ar.nslab; ++s) {
    const int32_t* sl = Ar.slabs + (size_t)s * SLAB_INTS;
    FaceArgs fa;
    fa.frows = Ar.frows;
    fa.zruns = Ar.zruns;
    fa.nzruns = s == 0 ? Ar.nzruns : 0;
    fa.nzblocks = (fa.nzruns + ZGROUP - 1) / ZGROUP;
    fa.tail_wait = s > 0 && !Ar.slab_events;
    int32_t nb = fa.nzblocks;
    for (int a = 0; a < 4; ++a) {
      const bool in = a < D;
      fa.fstart[a] = in ? sl[2 + 2 * a] : 0;
      fa.fend[a] = in ? sl[3 + 2 * a] : 0;
      fa.rbase[a] = in ? Ar.rbase[a] + (int64_t)(fa.fstart[a] - Ar.fstart[a]) * R[a] : 0;
    }
    for (int a = 0; a < D; ++a) {
      fa.bstart[a] = nb;
      nb += (fa.fend[a] - fa.fstart[a] + t.fb - 1) / t.fb;
    }
    for (int a = D; a < 4; ++a) fa.bstart[a] = nb;
    if (Ar.slab_inputs) {
      const cudaError_t e = cudaStreamWaitEvent(st, Ar.slab_inputs[s], 0);
      if (e != cudaSuccess) return e;
    }
    if (nb > 0) {
      const cudaError_t e =
          (s == 0 || Ar.slab_events)
              ? (face_kernel<D, K, A><<<nb, t.fb * S::L, face_smem<D, K, V>(t.fb), st>>>((const IO*)Ar.x, (V*)Ar.tp,
                                                                                     (IO*)Ar.y, fa, t.fb, c),
                 cudaGetLastError())
              : launch_pdl(face_kernel<D, K, A>, nb, t.fb * S::L, face_smem<D, K, V>(t.fb), st, (const IO*)Ar.x,
                           (V*)Ar.tp, (IO*)Ar.y, fa, (int)t.fb, c);
      if (e != cudaSuccess) return e;
    }
    LiftArgs la = Ar.la;
    la.lwin = Ar.la.lwin + (size_t)sl[0] * NW;
    la.lrow = Ar.la.lrow + (size_t)sl[0] * KR;
    la.nlift = sl[1] - sl[0];
    const int32_t nlb = (la.nlift + t.lcb - 1) / t.lcb;
    if (nlb > 0) {
      // programmatic dependent of this slab's face launch (a plain launch after an event)
      const cudaError_t e =
          (nb > 0 || !Ar.slab_events)
              ? launch_pdl(lift_kernel<D, K, A>, nlb, t.lnt, lift_smem<D, K>(t.lcb), st, (const V*)Ar.tp, (IO*)Ar.y,
                           Ar.add, la, (int)t.lcb)
              : (lift_kernel<D, K, A><<<nlb, t.lnt, lift_smem<D, K>(t.lcb), st>>>((const V*)Ar.tp, (IO*)Ar.y, Ar.add, la,
                                                                                 t.lcb),
                 cudaGetLastError());
      if (e != cudaSuccess) return e;
    }
    if (Ar.slab_events) {
      const cudaError_t e = cudaEventRecord(Ar.slab_events[s], st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

template <int D, int K, class A>
cudaError_t run_apply(const ApplyArgs& Ar, cudaStream_t st) {
  using S = Shape<D, K>;
  using V = typename A::V;
  using IO = typename A::IO;
  Consts<V, K> c;
  for (int j = 0; j < K; ++j)
    for (int b = 0; b < 2 * K + 1; ++b) c.g[j][b] = from_host<V>(Ar.g[j * (2 * K + 1) + b]);
  for (int j = 0; j < K; ++j) {
    c.s[j] = from_host<V>(Ar.s[j]);
    for (int b = 0; b < 2 * K + 1; ++b) c.gs[j][b] = from_host<V>(Ar.s[j] * Ar.g[j * (2 * K + 1) + b]);
  }
  for (int p = 0; p < K + 1; ++p)
    for (int q = 0; q < K + 1; ++q) c.m[p][q] = from_host<V>(Ar.m[p * (K + 1) + q]);
  mass_halves<V, K>(Ar.m, c);
  if (Ar.brick) return run_brick<D, K, A>(Ar, c, st);
  Tiles t = Ar.tiles;
  if (!resolve_tiles<D, K, V>(t)) return cudaErrorInvalidConfiguration;
  if (Ar.nslab > 1 && !Ar.ev && Ar.which == 3) return run_slabs<D, K, A>(Ar, c, t, st);
  FaceArgs fa;
  fa.frows = Ar.frows;
  for (int a = 0; a < 4; ++a) fa.rbase[a] = Ar.rbase[a];
  fa.zruns = Ar.zruns;
  fa.nzruns = Ar.nzruns;
  fa.nzblocks = (Ar.nzruns + ZGROUP - 1) / ZGROUP;
  fa.tail_wait = 0;
  int32_t nb = fa.nzblocks;
  for (int a = 0; a < 4; ++a) fa.fstart[a] = Ar.fstart[a];
  for (int a = 0; a < 4; ++a) fa.fend[a] = a < D ? Ar.fstart[a + 1] : Ar.fstart[D];
  for (int a = 0; a < D; ++a) {
    fa.bstart[a] = nb;
    nb += (Ar.fstart[a + 1] - Ar.fstart[a] + t.fb - 1) / t.fb;
  }
  for (int a = D; a < 4; ++a) fa.bstart[a] = nb;
  const bool faces = Ar.fstart[D] > 0;
  const int32_t nlb = (Ar.la.nlift + t.lcb - 1) / t.lcb;
  if (Ar.ev) cudaEventRecord(Ar.ev[0], st);
  if (nb > 0 && (Ar.which & 1))
    face_kernel<D, K, A><<<nb, t.fb * S::L, face_smem<D, K, V>(t.fb), st>>>((const IO*)Ar.x, (V*)Ar.tp,
                                                                          (IO*)Ar.y, fa, t.fb, c);
  if (Ar.ev) cudaEventRecord(Ar.ev[1], st);
  if (nlb > 0 && faces && (Ar.which & 2)) {
    if (Ar.ev || !(Ar.which & 1)) {
      lift_kernel<D, K, A><<<nlb, t.lnt, lift_smem<D, K>(t.lcb), st>>>((const V*)Ar.tp, (IO*)Ar.y, Ar.add, Ar.la,
                                                                       t.lcb);
    } else {
      // programmatic dependent launch: the lift's CTAs start while the face grid drains
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)nlb);
      cfg.blockDim = dim3((unsigned)t.lnt);
      cfg.dynamicSmemBytes = lift_smem<D, K>(t.lcb);
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      const cudaError_t e = cudaLaunchKernelEx(&cfg, lift_kernel<D, K, A>, (const V*)Ar.tp, (IO*)Ar.y, Ar.add, Ar.la,
                                               (int)t.lcb);
      if (e != cudaSuccess) return e;
    }
  }
  if (Ar.ev) cudaEventRecord(Ar.ev[2], st);
  return cudaGetLastError();
}

// ------------------------------------------------------------- batches --
// Host description of one batch segment (one problem, one right-hand side).
struct SegSpec {
  FaceArgs fa;          // frows, rbase, fstart, zruns, nzruns of the segment's problem
  LiftArgs la;
  void* wp = nullptr;   // the segment's face-output buffer
  const void* gs = nullptr;   // device: K x (2K+1) scaled jump vectors of the segment's problem
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // the problem's s_j
};

// Packs the segments of one (d, k, arithmetic) group into the device layouts of
// FaceSeg<V, K> and LiftSeg, with the CTA offsets of both launches.
template <int D, int K, class A>
bool pack_batch(const std::vector<SegSpec>& in, Tiles& t, std::vector<unsigned char>& fsegs,
                std::vector<unsigned char>& lsegs, int& face_blocks, int& lift_blocks) {
  using V = typename A::V;
  if (!resolve_tiles<D, K, V>(t)) return false;
  fsegs.assign(in.size() * sizeof(FaceSeg<V, K>), 0);
  lsegs.assign(in.size() * sizeof(LiftSeg), 0);
  int fb = 0, lb = 0;
  for (size_t i = 0; i < in.size(); ++i) {
    FaceSeg<V, K> fs;
    fs.fa = in[i].fa;
    fs.fa.nzblocks = (fs.fa.nzruns + ZGROUP - 1) / ZGROUP;
    fs.fa.tail_wait = 0;
    for (int a = 0; a < 4; ++a) fs.fa.fend[a] = a < D ? fs.fa.fstart[a + 1] : fs.fa.fstart[D];
    int32_t nb = fs.fa.nzblocks;
    for (int a = 0; a < D; ++a) {
      fs.fa.bstart[a] = nb;
      nb += (fs.fa.fstart[a + 1] - fs.fa.fstart[a] + t.fb - 1) / t.fb;
    }
    for (int a = D; a < 4; ++a) fs.fa.bstart[a] = nb;
    fs.wp = (V*)in[i].wp;
    fs.gs = (const V*)in[i].gs;
    for (int j = 0; j < K; ++j) fs.s[j] = from_host<V>(in[i].s[j]);
    fs.block0 = fb;
    fb += nb;
    LiftSeg ls;
    ls.la = in[i].la;
    ls.block0 = lb;
    if (fs.fa.fstart[D] > 0) lb += (ls.la.nlift + t.lcb - 1) / t.lcb;
    std::memcpy(&fsegs[i * sizeof(FaceSeg<V, K>)], &fs, sizeof(fs));
    std::memcpy(&lsegs[i * sizeof(LiftSeg)], &ls, sizeof(ls));
  }
  face_blocks = fb;
  lift_blocks = lb;
  return true;
}

template <int D, int K, class A>
cudaError_t run_batch(const void* fsegs, const void* lsegs, const void* ptrs, int nseg, int face_blocks,
                      int lift_blocks, const double* g, const double* m, Tiles t, cudaStream_t st) {
  using V = typename A::V;
  using IO = typename A::IO;
  using S = Shape<D, K>;
  if (!resolve_tiles<D, K, V>(t)) return cudaErrorInvalidConfiguration;
  Consts<V, K> c;
  for (int j = 0; j < K; ++j)
    for (int b = 0; b < 2 * K + 1; ++b) c.g[j][b] = from_host<V>(g[j * (2 * K + 1) + b]);
  for (int p = 0; p < K + 1; ++p)
    for (int q = 0; q < K + 1; ++q) c.m[p][q] = from_host<V>(m[p * (K + 1) + q]);
  mass_halves<V, K>(m, c);
  for (int j = 0; j < K; ++j) {
    c.s[j] = vzero<V>();                                          // per segment: FaceSeg::s
    for (int b = 0; b < 2 * K + 1; ++b) c.gs[j][b] = vzero<V>();  // per segment: FaceSeg::gs
  }
  if (face_blocks > 0)
    face_kernel_batched<D, K, A><<<face_blocks, t.fb * S::L, face_smem<D, K, V>(t.fb), st>>>(
        (const FaceSeg<V, K>*)fsegs, nseg, (const SegPtrs<IO>*)ptrs, t.fb, c);
  if (lift_blocks > 0)
    lift_kernel_batched<D, K, A><<<lift_blocks, t.lnt, lift_smem<D, K>(t.lcb), st>>>(
        (const LiftSeg*)lsegs, (const FaceSeg<V, K>*)fsegs, nseg, (const SegPtrs<IO>*)ptrs, t.lcb);
  return cudaGetLastError();
}

// The scaled jump vectors s_j g_j[b] (k x (2k+1)) of one problem in the value type of the
// arithmetic (4 or 8 bytes per value), as the face kernels use them.
template <class A>
void scaled_jumps(int k, const double* g, const double* s, std::vector<unsigned char>& out) {
  using V = typename A::V;
  out.assign((size_t)k * (2 * k + 1) * sizeof(V), 0);
  V* o = reinterpret_cast<V*>(out.data());
  for (int j = 0; j < k; ++j)
    for (int b = 0; b < 2 * k + 1; ++b) o[j * (2 * k + 1) + b] = from_host<V>(s[j] * g[j * (2 * k + 1) + b]);
}

// Per translation unit: batch packing and launch for one (arithmetic, dimension).
struct BatchOps {
  bool (*pack)(int k, const std::vector<SegSpec>&, Tiles&, std::vector<unsigned char>&,
               std::vector<unsigned char>&, int&, int&);
  void (*jumps)(int k, const double* g, const double* s, std::vector<unsigned char>& out);
  cudaError_t (*run)(int k, const void*, const void*, const void*, int, int, int, const double*, const double*,
                     Tiles, cudaStream_t);
};
BatchOps batch_ops_f64_d2();
BatchOps batch_ops_f64_d3();
BatchOps batch_ops_f32_d2();
BatchOps batch_ops_f32_d3();
BatchOps batch_ops_ff_d2();
BatchOps batch_ops_ff_d3();

#define GP_BATCH_OPS(D, A)                                                                              \
  BatchOps ops;                                                                                         \
  ops.jumps = scaled_jumps<A>;                                                                          \
  ops.pack = [](int k, const std::vector<SegSpec>& in, Tiles& t, std::vector<unsigned char>& fs,       \
                std::vector<unsigned char>& ls, int& fb, int& lb) -> bool {                             \
    switch (k) {                                                                                        \
      case 1: return pack_batch<D, 1, A>(in, t, fs, ls, fb, lb);                                        \
      case 2: return pack_batch<D, 2, A>(in, t, fs, ls, fb, lb);                                        \
      case 3: return pack_batch<D, 3, A>(in, t, fs, ls, fb, lb);                                        \
      case 4: return pack_batch<D, 4, A>(in, t, fs, ls, fb, lb);                                        \
      case 5: return pack_batch<D, 5, A>(in, t, fs, ls, fb, lb);                                        \
      case 6: return pack_batch<D, 6, A>(in, t, fs, ls, fb, lb);                                        \
      case 7: return pack_batch<D, 7, A>(in, t, fs, ls, fb, lb);                                        \
      case 8: return pack_batch<D, 8, A>(in, t, fs, ls, fb, lb);                                        \
      default: return false;                                                                            \
    }                                                                                                   \
  };                                                                                                    \
  ops.run = [](int k, const void* fs, const void* ls, const void* pt, int ns, int fb, int lb,          \
               const double* g, const double* m, Tiles t, cudaStream_t st) -> cudaError_t {             \
    switch (k) {                                                                                        \
      case 1: return run_batch<D, 1, A>(fs, ls, pt, ns, fb, lb, g, m, t, st);                           \
      case 2: return run_batch<D, 2, A>(fs, ls, pt, ns, fb, lb, g, m, t, st);                           \
      case 3: return run_batch<D, 3, A>(fs, ls, pt, ns, fb, lb, g, m, t, st);                           \
      case 4: return run_batch<D, 4, A>(fs, ls, pt, ns, fb, lb, g, m, t, st);                           \
      case 5: return run_batch<D, 5, A>(fs, ls, pt, ns, fb, lb, g, m, t, st);                           \
      case 6: return run_batch<D, 6, A>(fs, ls, pt, ns, fb, lb, g, m, t, st);                           \
      case 7: return run_batch<D, 7, A>(fs, ls, pt, ns, fb, lb, g, m, t, st);                           \
      case 8: return run_batch<D, 8, A>(fs, ls, pt, ns, fb, lb, g, m, t, st);                           \
      default: return cudaErrorInvalidValue;                                                            \
    }                                                                                                   \
  };                                                                                                    \
  return ops;

// y (+)= (wm M_active + ws K_active) x over the active cells (cell kernel + gather; add = 1:
// onto y, 0: overwrite the nodes of active cells).  first = 1: the cell kernel is the first
// kernel of the call and is launched normally (it reads x before any dependency wait, so it must
// not start early under the previous kernel on the stream); 0: it follows the face kernel of
// the same call and starts as that kernel's programmatic dependent.
using CellsFn = cudaError_t (*)(int k, const void* x, void* y, const CellTabs& ct, const double* m, const double* s,
                                double h, double wm, double ws, int add, int first, cudaStream_t st);
CellsFn cells_f64_d2();
CellsFn cells_f64_d3();
CellsFn cells_f32_d2();
CellsFn cells_f32_d3();
CellsFn cells_ff_d2();
CellsFn cells_ff_d3();

#define GP_CELLS_CASE(D, A, K) \
  case K: return run_cells<D, K, A>(x, y, ct, m, s, h, wm, ws, add, first, st);
#define GP_CELLS_FN(D, A)                                                                                 \
  return [](int k, const void* x, void* y, const CellTabs& ct, const double* m, const double* s, double h, \
            double wm, double ws, int add, int first, cudaStream_t st) -> cudaError_t {                  \
    switch (k) {                                                                                          \
      GP_CELLS_CASE(D, A, 1) GP_CELLS_CASE(D, A, 2) GP_CELLS_CASE(D, A, 3) GP_CELLS_CASE(D, A, 4)         \
      GP_CELLS_CASE(D, A, 5) GP_CELLS_CASE(D, A, 6) GP_CELLS_CASE(D, A, 7) GP_CELLS_CASE(D, A, 8)         \
      default: return cudaErrorInvalidValue;                                                              \
    }                                                                                                     \
  };

#define GP_DISPATCH_K(D, A, Ar, st)                    \
  switch ((Ar).k) {                                    \
    case 1: return run_apply<D, 1, A>(Ar, st);         \
    case 2: return run_apply<D, 2, A>(Ar, st);         \
    case 3: return run_apply<D, 3, A>(Ar, st);         \
    case 4: return run_apply<D, 4, A>(Ar, st);         \
    case 5: return run_apply<D, 5, A>(Ar, st);         \
    case 6: return run_apply<D, 6, A>(Ar, st);         \
    case 7: return run_apply<D, 7, A>(Ar, st);         \
    case 8: return run_apply<D, 8, A>(Ar, st);         \
    default: return cudaErrorInvalidValue;             \
  }

}  // namespace gp
