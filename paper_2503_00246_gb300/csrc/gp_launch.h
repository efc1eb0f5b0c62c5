// Host-side launch interface between the C ABI and the templated kernels.
#pragma once

#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>

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
};

// One entry point per (arithmetic, dimension); each dispatches on k = 1..8.
cudaError_t apply_f64_d2(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_f64_d3(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_f32_d2(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_f32_d3(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_ff_d2(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_ff_d3(const ApplyArgs& a, cudaStream_t st);

template <int D, int K, class A>
cudaError_t run_apply(const ApplyArgs& Ar, cudaStream_t st) {
  using S = Shape<D, K>;
  using V = typename A::V;
  using IO = typename A::IO;
  Consts<V, K> c;
  for (int j = 0; j < K; ++j)
    for (int b = 0; b < 2 * K + 1; ++b) c.g[j][b] = from_host<V>(Ar.g[j * (2 * K + 1) + b]);
  for (int p = 0; p < K + 1; ++p)
    for (int q = 0; q < K + 1; ++q) c.m[p][q] = from_host<V>(Ar.m[p * (K + 1) + q]);
  for (int j = 0; j < K; ++j) c.s[j] = from_host<V>(Ar.s[j]);
  FaceArgs fa;
  fa.frows = Ar.frows;
  for (int a = 0; a < 4; ++a) fa.rbase[a] = Ar.rbase[a];
  fa.zruns = Ar.zruns;
  fa.nzruns = Ar.nzruns;
  fa.nzblocks = (Ar.nzruns + ZGROUP - 1) / ZGROUP;
  int32_t nb = fa.nzblocks;
  for (int a = 0; a < 4; ++a) fa.fstart[a] = Ar.fstart[a];
  for (int a = 0; a < D; ++a) {
    fa.bstart[a] = nb;
    nb += (Ar.fstart[a + 1] - Ar.fstart[a] + S::FB - 1) / S::FB;
  }
  for (int a = D; a < 4; ++a) fa.bstart[a] = nb;
  const bool faces = Ar.fstart[D] > 0;
  using LS = LiftShape<D, K>;
  const int32_t nlb = (Ar.la.nlift + LS::CB - 1) / LS::CB;
  if (Ar.ev) cudaEventRecord(Ar.ev[0], st);
  if (nb > 0)
    face_kernel<D, K, A><<<nb, S::NT, 0, st>>>((const IO*)Ar.x, (V*)Ar.tp, (IO*)Ar.y, fa, c);
  if (Ar.ev) cudaEventRecord(Ar.ev[1], st);
  if (nlb > 0 && faces)
    lift_kernel<D, K, A><<<nlb, LS::NT, 0, st>>>((const V*)Ar.tp, (IO*)Ar.y, Ar.add, Ar.la);
  if (Ar.ev) cudaEventRecord(Ar.ev[2], st);
  return cudaGetLastError();
}

// ------------------------------------------------------------- batches --
// Host description of one batch segment (one problem, one right-hand side).
struct SegSpec {
  FaceArgs fa;          // frows, rbase, fstart, zruns, nzruns of the segment's problem
  LiftArgs la;
  void* wp = nullptr;   // the segment's face-output buffer
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

// Packs the segments of one (d, k, arithmetic) group into the device layouts of
// FaceSeg<V, K> and LiftSeg, with the CTA offsets of both launches.
template <int D, int K, class A>
void pack_batch(const std::vector<SegSpec>& in, std::vector<unsigned char>& fsegs,
                std::vector<unsigned char>& lsegs, int& face_blocks, int& lift_blocks) {
  using V = typename A::V;
  using S = Shape<D, K>;
  using LS = LiftShape<D, K>;
  fsegs.assign(in.size() * sizeof(FaceSeg<V, K>), 0);
  lsegs.assign(in.size() * sizeof(LiftSeg), 0);
  int fb = 0, lb = 0;
  for (size_t i = 0; i < in.size(); ++i) {
    FaceSeg<V, K> fs;
    fs.fa = in[i].fa;
    fs.fa.nzblocks = (fs.fa.nzruns + ZGROUP - 1) / ZGROUP;
    int32_t nb = fs.fa.nzblocks;
    for (int a = 0; a < D; ++a) {
      fs.fa.bstart[a] = nb;
      nb += (fs.fa.fstart[a + 1] - fs.fa.fstart[a] + S::FB - 1) / S::FB;
    }
    for (int a = D; a < 4; ++a) fs.fa.bstart[a] = nb;
    fs.wp = (V*)in[i].wp;
    for (int j = 0; j < K; ++j) fs.s[j] = from_host<V>(in[i].s[j]);
    fs.block0 = fb;
    fb += nb;
    LiftSeg ls;
    ls.la = in[i].la;
    ls.block0 = lb;
    if (fs.fa.fstart[D] > 0) lb += (ls.la.nlift + LS::CB - 1) / LS::CB;
    std::memcpy(&fsegs[i * sizeof(FaceSeg<V, K>)], &fs, sizeof(fs));
    std::memcpy(&lsegs[i * sizeof(LiftSeg)], &ls, sizeof(ls));
  }
  face_blocks = fb;
  lift_blocks = lb;
}

template <int D, int K, class A>
cudaError_t run_batch(const void* fsegs, const void* lsegs, const void* ptrs, int nseg, int face_blocks,
                      int lift_blocks, const double* g, const double* m, cudaStream_t st) {
  using V = typename A::V;
  using IO = typename A::IO;
  using S = Shape<D, K>;
  Consts<V, K> c;
  for (int j = 0; j < K; ++j)
    for (int b = 0; b < 2 * K + 1; ++b) c.g[j][b] = from_host<V>(g[j * (2 * K + 1) + b]);
  for (int p = 0; p < K + 1; ++p)
    for (int q = 0; q < K + 1; ++q) c.m[p][q] = from_host<V>(m[p * (K + 1) + q]);
  for (int j = 0; j < K; ++j) c.s[j] = vzero<V>();   // per segment, in FaceSeg
  if (face_blocks > 0)
    face_kernel_batched<D, K, A><<<face_blocks, S::NT, 0, st>>>((const FaceSeg<V, K>*)fsegs, nseg,
                                                               (const SegPtrs<IO>*)ptrs, c);
  if (lift_blocks > 0)
    lift_kernel_batched<D, K, A><<<lift_blocks, LiftShape<D, K>::NT, 0, st>>>(
        (const LiftSeg*)lsegs, (const FaceSeg<V, K>*)fsegs, nseg, (const SegPtrs<IO>*)ptrs);
  return cudaGetLastError();
}

// Per translation unit: batch packing and launch for one (arithmetic, dimension).
struct BatchOps {
  void (*pack)(int k, const std::vector<SegSpec>&, std::vector<unsigned char>&, std::vector<unsigned char>&,
               int&, int&);
  cudaError_t (*run)(int k, const void*, const void*, const void*, int, int, int, const double*, const double*,
                     cudaStream_t);
};
BatchOps batch_ops_f64_d2();
BatchOps batch_ops_f64_d3();
BatchOps batch_ops_f32_d2();
BatchOps batch_ops_f32_d3();
BatchOps batch_ops_ff_d2();
BatchOps batch_ops_ff_d3();

#define GP_BATCH_OPS(D, A)                                                                              \
  BatchOps ops;                                                                                         \
  ops.pack = [](int k, const std::vector<SegSpec>& in, std::vector<unsigned char>& fs,                  \
                std::vector<unsigned char>& ls, int& fb, int& lb) {                                     \
    switch (k) {                                                                                        \
      case 1: pack_batch<D, 1, A>(in, fs, ls, fb, lb); break;                                           \
      case 2: pack_batch<D, 2, A>(in, fs, ls, fb, lb); break;                                           \
      case 3: pack_batch<D, 3, A>(in, fs, ls, fb, lb); break;                                           \
      case 4: pack_batch<D, 4, A>(in, fs, ls, fb, lb); break;                                           \
      case 5: pack_batch<D, 5, A>(in, fs, ls, fb, lb); break;                                           \
      case 6: pack_batch<D, 6, A>(in, fs, ls, fb, lb); break;                                           \
      case 7: pack_batch<D, 7, A>(in, fs, ls, fb, lb); break;                                           \
      default: pack_batch<D, 8, A>(in, fs, ls, fb, lb); break;                                          \
    }                                                                                                   \
  };                                                                                                    \
  ops.run = [](int k, const void* fs, const void* ls, const void* pt, int ns, int fb, int lb,          \
               const double* g, const double* m, cudaStream_t st) -> cudaError_t {                      \
    switch (k) {                                                                                        \
      case 1: return run_batch<D, 1, A>(fs, ls, pt, ns, fb, lb, g, m, st);                              \
      case 2: return run_batch<D, 2, A>(fs, ls, pt, ns, fb, lb, g, m, st);                              \
      case 3: return run_batch<D, 3, A>(fs, ls, pt, ns, fb, lb, g, m, st);                              \
      case 4: return run_batch<D, 4, A>(fs, ls, pt, ns, fb, lb, g, m, st);                              \
      case 5: return run_batch<D, 5, A>(fs, ls, pt, ns, fb, lb, g, m, st);                              \
      case 6: return run_batch<D, 6, A>(fs, ls, pt, ns, fb, lb, g, m, st);                              \
      case 7: return run_batch<D, 7, A>(fs, ls, pt, ns, fb, lb, g, m, st);                              \
      case 8: return run_batch<D, 8, A>(fs, ls, pt, ns, fb, lb, g, m, st);                              \
      default: return cudaErrorInvalidValue;                                                            \
    }                                                                                                   \
  };                                                                                                    \
  return ops;

// y += (M_active + K_active) x over the active cells (parity colours in order).
using CellsFn = cudaError_t (*)(int k, const void* x, void* y, const int32_t* crow, const int32_t* cstart,
                                const double* m, const double* s, double h, cudaStream_t st);
CellsFn cells_f64_d2();
CellsFn cells_f64_d3();
CellsFn cells_f32_d2();
CellsFn cells_f32_d3();
CellsFn cells_ff_d2();
CellsFn cells_ff_d3();

#define GP_CELLS_FN(D, A)                                                                               \
  return [](int k, const void* x, void* y, const int32_t* crow, const int32_t* cstart, const double* m, \
            const double* s, double h, cudaStream_t st) -> cudaError_t {                                \
    switch (k) {                                                                                        \
      case 1: return run_cells<D, 1, A>(x, y, crow, cstart, m, s, h, st);                               \
      case 2: return run_cells<D, 2, A>(x, y, crow, cstart, m, s, h, st);                               \
      case 3: return run_cells<D, 3, A>(x, y, crow, cstart, m, s, h, st);                               \
      case 4: return run_cells<D, 4, A>(x, y, crow, cstart, m, s, h, st);                               \
      case 5: return run_cells<D, 5, A>(x, y, crow, cstart, m, s, h, st);                               \
      case 6: return run_cells<D, 6, A>(x, y, crow, cstart, m, s, h, st);                               \
      case 7: return run_cells<D, 7, A>(x, y, crow, cstart, m, s, h, st);                               \
      case 8: return run_cells<D, 8, A>(x, y, crow, cstart, m, s, h, st);                               \
      default: return cudaErrorInvalidValue;                                                            \
    }                                                                                                   \
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
