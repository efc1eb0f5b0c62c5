// Host-side launch interface between the C ABI and the templated kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gp_kernels.cuh"

namespace gp {

struct ApplyArgs {
  int dim = 0, k = 0;
  const void* x = nullptr;   // device, n_active elements
  void* y = nullptr;         // device, n_active elements
  void* tp = nullptr;        // device scratch, nf * L * k elements
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

// One entry point per (precision, dimension); each dispatches on k = 1..8.
cudaError_t apply_f64_d2(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_f64_d3(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_f32_d2(const ApplyArgs& a, cudaStream_t st);
cudaError_t apply_f32_d3(const ApplyArgs& a, cudaStream_t st);

template <int D, int K, typename T>
cudaError_t run_apply(const ApplyArgs& A, cudaStream_t st) {
  using S = Shape<D, K>;
  Consts<T, K> c;
  for (int j = 0; j < K; ++j)
    for (int b = 0; b < 2 * K + 1; ++b) c.g[j][b] = (T)A.g[j * (2 * K + 1) + b];
  for (int p = 0; p < K + 1; ++p)
    for (int q = 0; q < K + 1; ++q) c.m[p][q] = (T)A.m[p * (K + 1) + q];
  for (int j = 0; j < K; ++j) c.s[j] = (T)A.s[j];
  FaceArgs fa;
  fa.frows = A.frows;
  for (int a = 0; a < 4; ++a) fa.rbase[a] = A.rbase[a];
  fa.zruns = A.zruns;
  fa.nzruns = A.nzruns;
  fa.nzblocks = (A.nzruns + ZGROUP - 1) / ZGROUP;
  int32_t nb = fa.nzblocks;
  for (int a = 0; a < 4; ++a) fa.fstart[a] = A.fstart[a];
  for (int a = 0; a < D; ++a) {
    fa.bstart[a] = nb;
    nb += (A.fstart[a + 1] - A.fstart[a] + S::FB - 1) / S::FB;
  }
  for (int a = D; a < 4; ++a) fa.bstart[a] = nb;
  const int32_t nblk = nb;
  const bool faces = A.fstart[D] > 0;
  using LS = LiftShape<D, K>;
  const int32_t nlb = (A.la.nlift + LS::CB - 1) / LS::CB;
  if (A.ev) cudaEventRecord(A.ev[0], st);
  if (nblk > 0)
    jump_kernel<D, K, T><<<nblk, S::NT, 0, st>>>((const T*)A.x, (T*)A.tp, (T*)A.y, fa, c);
  if (A.ev) cudaEventRecord(A.ev[1], st);
  if (nlb > 0 && faces)
    lift_kernel<D, K, T><<<nlb, LS::NT, 0, st>>>((const T*)A.tp, (T*)A.y, A.add, A.la, c);
  if (A.ev) cudaEventRecord(A.ev[2], st);
  return cudaGetLastError();
}

#define GP_DISPATCH_K(D, T, A, st)                     \
  switch ((A).k) {                                     \
    case 1: return run_apply<D, 1, T>(A, st);          \
    case 2: return run_apply<D, 2, T>(A, st);          \
    case 3: return run_apply<D, 3, T>(A, st);          \
    case 4: return run_apply<D, 4, T>(A, st);          \
    case 5: return run_apply<D, 5, T>(A, st);          \
    case 6: return run_apply<D, 6, T>(A, st);          \
    case 7: return run_apply<D, 7, T>(A, st);          \
    case 8: return run_apply<D, 8, T>(A, st);          \
    default: return cudaErrorInvalidValue;             \
  }

}  // namespace gp
