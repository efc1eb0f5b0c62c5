// Batched applies of many independent problems with several right-hand sides (the batched
// workload: meshes of uneven n, k and geometry), as two persistent launches per (dimension,
// degree, arithmetic, stabilisation): one face launch and one lift launch over a static work
// list.
//
// A work item of the face launch is up to fb faces of one normal axis of one problem (or a
// group of zero runs); of the lift launch up to cb owner cells of one problem.  The CTAs of a
// launch walk its list with a fixed stride (no inter-CTA waits).  One launch per degree: a
// launch that dispatched on the degree of each item took the registers of its largest degree
// (128 per thread with spills in FP32) for every item, and ran the batched workload at 60% of
// the speed of per-degree launches.  Each item runs
// all nrhs right-hand sides of its problem: the face item reads its row starts once and the
// lift item its candidate windows and row starts once, so the tables are read once per item
// instead of once per right-hand side.  The per-line arithmetic is that of the single-problem
// face and lift kernels (gp_kernels.cuh), in the same order: a batch gives the same bits as
// single applies.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gp_kernels.cuh"

namespace gp {

// one problem of a batch group (device copy)
template <typename V, typename IO>
struct PBProb {
  const int32_t* frows;   // per-face row starts of the patch
  const int32_t* lwin;    // lift candidate windows
  const int32_t* lrow;    // lift row starts
  const int2* zruns;      // zero runs
  V* wp;                  // face outputs of right-hand side 0; side r at wp + r wstride
  const V* gs;            // k x (2k+1) scaled jump vectors s_j g_j
  int64_t rbase[4];
  int64_t wstride;
  int32_t fstart[4];
  int32_t nlift, n_active, k, pad;
};

struct PBArgs {
  const void* probs;      // PBProb<V, IO>[nprob]
  const int4* items;      // {problem, kind (0..2 face axis, 3 zero runs; lift: 0), first, count}
  const void* ptrs;       // SegPtrs<IO>[nprob]: x and y of right-hand side 0 (side r at + r n_active)
  int32_t nitems;
  int32_t nrhs;
};

// dynamic shared memory of a face item of degree k: fb + 1 jump planes (two in 3D)
template <int D, int K, typename V>
__host__ __device__ constexpr size_t pb_face_smem(int face_threads);
// faces per face item and owner cells per lift item of degree k for the batch's block sizes
template <int D, int K>
__host__ __device__ constexpr int pb_fb(int face_threads) {
  return face_threads / Shape<D, K>::L > 0 ? face_threads / Shape<D, K>::L : 1;
}
template <int D, int K>
__host__ __device__ constexpr int pb_cb(int lift_threads) {
  return (2 * lift_threads) / LiftShape<D, K>::KR > 0 ? (2 * lift_threads) / LiftShape<D, K>::KR : 1;
}

template <int D, int K, typename V>
__host__ __device__ constexpr size_t pb_face_smem(int face_threads) {
  return (size_t)((D == 3) ? 2 : 1) * (pb_fb<D, K>(face_threads) + 1) * K * Shape<D, K>::L * sizeof(V);
}
template <int D, int K>
__host__ __device__ constexpr size_t pb_lift_smem(int lift_threads) {
  return (size_t)pb_cb<D, K>(lift_threads) * (LiftShape<D, K>::NW + 1) * sizeof(int);
}

// ------------------------------------------------------------------ face --
template <int D, int K, class A>
__device__ __forceinline__ void pb_face_item(const PBProb<typename A::V, typename A::IO>& pr,
                                             const SegPtrs<typename A::IO>& sp, const int4 it, const int nrhs,
                                             const Consts<typename A::V, K>& c, unsigned char* dsm) {
  using S = Shape<D, K>;
  using V = typename A::V;
  using IO = typename A::IO;
  constexpr int L = S::L, NN = S::NN, K1 = K + 1;
  typedef V Plane[K][L];
  const int t = threadIdx.x, nt = (int)blockDim.x;
  const int fb = pb_fb<D, K>(nt);
  // fb planes for the faces and one more for the threads past fb L (nt < (fb + 1) L): they run
  // the same code on that spare plane, so every thread meets every barrier
  Plane* buf = reinterpret_cast<Plane*>(dsm);
  Plane* sb2 = buf + fb + 1;
  __shared__ V sm[K1][K1];
  __shared__ V sg[K][NN];
  for (int i = t; i < K1 * K1; i += nt) sm[i / K1][i % K1] = c.m[i / K1][i % K1];
  for (int i = t; i < K * NN; i += nt) sg[i / NN][i % NN] = pr.gs[i];
  __syncthreads();
  const int axis = it.y, f0 = it.z, nf = it.w;
  const int fl = t / L, tau = t - fl * L;      // fl == fb: a thread on the spare plane
  const bool valid = fl < nf;
  const int f = f0 + fl;
  const int fbase = pr.fstart[axis];
  const int64_t rbase = pr.rbase[axis];
  // this thread's row starts, read once for all right-hand sides
  int32_t rs[NN];
  int tx = 0;
  if (valid) {
    if (axis == 0) {
      rs[0] = __ldg(pr.frows + rbase + (int64_t)(f - fbase) * L + tau);
    } else {
      constexpr int R = (D == 3) ? NN * K1 : NN;
      tx = (D == 3) ? tau % K1 : tau;
      const int tr = (D == 3) ? tau / K1 : 0;
      const int32_t* rows = pr.frows + rbase + (int64_t)(f - fbase) * R + NN * tr;
#pragma unroll
      for (int b = 0; b < NN; ++b) rs[b] = __ldg(rows + b);
    }
  }
  int pos0, pstride;
  if (axis == 0) {
    pos0 = NN * tau;
    pstride = 1;
  } else if (D == 2 || axis == 1) {
    const int tz = (D == 3) ? tau / K1 : 0;
    pos0 = ((D == 3) ? tau % K1 : tau) + K1 * NN * tz;
    pstride = K1;
  } else {
    pos0 = tau;
    pstride = K1 * K1;
  }
  for (int r = 0; r < nrhs; ++r) {
    const IO* x = sp.x + (size_t)r * pr.n_active;
    V v[NN];
    if (valid) {
      if (axis == 0) {
#pragma unroll
        for (int b = 0; b < NN; ++b) v[b] = from_io(__ldg(x + rs[0] + b), (V*)nullptr);
      } else {
#pragma unroll
        for (int b = 0; b < NN; ++b) v[b] = from_io(__ldg(x + rs[b] + tx), (V*)nullptr);
      }
    } else {
#pragma unroll
      for (int b = 0; b < NN; ++b) v[b] = vzero<V>();
    }
    {
      V tj[K];
      line_jumps<K, V>(v, sg, tj);
#pragma unroll
      for (int j = 0; j < K; ++j) buf[fl][j][tau] = tj[j];
    }
    __syncthreads();
    V out[K];
    if constexpr (std::is_same<V, ff64>::value) line_tangential_eo<D, K, V, L>(buf[fl], sb2[fl], c, tau, out);
    else line_tangential<D, K, V, L>(buf[fl], sb2[fl], sm, tau, out);
    if (valid) {
      V w[NN];
      line_expand<K, V>(c, out, w);
      V* dst = pr.wp + (size_t)r * pr.wstride + (size_t)f * S::P;
#pragma unroll
      for (int bb = 0; bb < NN; ++bb) dst[pos0 + pstride * bb] = w[bb];
    }
    __syncthreads();            // the planes are reused by the next right-hand side
  }
}

// zero runs [first, first + count) of a problem, every right-hand side
template <class A>
__device__ __forceinline__ void pb_zero_item(const PBProb<typename A::V, typename A::IO>& pr,
                                             const SegPtrs<typename A::IO>& sp, const int4 it, const int nrhs) {
  using IO = typename A::IO;
  const int t = threadIdx.x, nt = (int)blockDim.x;
  for (int q = 0; q < it.w; ++q) {
    const int2 run = __ldg(pr.zruns + it.z + q);
    for (int r = 0; r < nrhs; ++r) {
      IO* y = sp.y + (size_t)r * pr.n_active;
      for (int i = t; i < run.y; i += nt) __stcs(y + run.x + i, IO(0));
    }
  }
}

template <int D, int K, class A>
__global__ void __launch_bounds__(MAX_CTA_THREADS)
face_kernel_pb(const PBArgs a, const __grid_constant__ Consts<typename A::V, K> c) {
  using V = typename A::V;
  using IO = typename A::IO;
  __shared__ PBProb<V, IO> pr;
  __shared__ SegPtrs<IO> sp;
  __shared__ int4 it;
  extern __shared__ __align__(16) unsigned char pb_dyn_smem[];
  for (int item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    if (threadIdx.x == 0) {
      it = a.items[item];
      pr = reinterpret_cast<const PBProb<V, IO>*>(a.probs)[it.x];
      sp = reinterpret_cast<const SegPtrs<IO>*>(a.ptrs)[it.x];
    }
    __syncthreads();
    if (it.y == 3) pb_zero_item<A>(pr, sp, it, a.nrhs);
    else pb_face_item<D, K, A>(pr, sp, it, a.nrhs, c, pb_dyn_smem);
    __syncthreads();            // the next item rewrites pr, sp, it
  }
}

// ------------------------------------------------------------------ lift --
template <int D, int K, class A>
__device__ __forceinline__ void pb_lift_item(const PBProb<typename A::V, typename A::IO>& pr,
                                             const SegPtrs<typename A::IO>& sp, const int4 it, const int nrhs,
                                             unsigned char* dsm) {
  using S = LiftShape<D, K>;
  using V = typename A::V;
  using IO = typename A::IO;
  constexpr int NW = S::NW;
  typedef int Win[NW + 1];
  Win* win = reinterpret_cast<Win*>(dsm);
  const int t = threadIdx.x, nt = (int)blockDim.x;
  const int cell0 = it.z, cb = it.w;
  for (int idx = t; idx < NW * cb; idx += nt) {
    const int ln = idx / NW, w = idx - ln * NW;
    win[ln][w] = __ldg(pr.lwin + (size_t)cell0 * NW + idx);
  }
  __syncthreads();
  const int E1 = cb * S::count(0);
  const int E2 = E1 + cb * S::count(1);
  const int E3 = E2 + cb * S::count(2);
  const int ITEMS = cb * S::KR;
  for (int g = t; g < ITEMS; g += nt) {
    int m, local;
    if (g < E1) { m = 0; local = g; }
    else if (g < E2 || S::NTYPE == 2) { m = 1; local = g - E1; }
    else if (g < E3) { m = 2; local = g - E2; }
    else { m = 3; local = g - E3; }
    const int cnt = S::count(m);
    const int ci = local / cnt;
    int rem = local - ci * cnt;
    const int cell = cell0 + ci;
    int q = 0, r = 0;
    if constexpr (K > 1) {
      if (!(m & 1)) { q = 1 + rem % (K - 1); rem /= (K - 1); }
      if (D == 3 && !(m & 2)) { r = 1 + rem % (K - 1); }
    }
    const int row = q + (D == 3 ? K * r : 0);
    const int base = __ldg(pr.lrow + (size_t)cell * S::KR + row);
    if (base < 0) continue;
    for (int rh = 0; rh < nrhs; ++rh) {
      const V* wp = pr.wp + (size_t)rh * pr.wstride;
      IO* y = sp.y + (size_t)rh * pr.n_active;
      Sum<V> acc[K];
#pragma unroll
      for (int p = 0; p < K; ++p) acc[p] = sum_zero<V>();
      unsigned found = 0;
      switch (m) {
        case 0: lift_row<D, K, A, 0>(wp, win[ci], q, r, acc, found); break;
        case 1: lift_row<D, K, A, 1>(wp, win[ci], q, r, acc, found); break;
        case 2: lift_row<D, K, A, 2>(wp, win[ci], q, r, acc, found); break;
        default: lift_row<D, K, A, 3>(wp, win[ci], q, r, acc, found); break;
      }
#pragma unroll
      for (int p = 0; p < K; ++p) {
        if (!((found >> p) & 1u)) continue;
        const int idx = base + p;
        if (idx >= pr.n_active) continue;
        y[idx] = to_io(dot_value(acc[p]), (IO*)nullptr);
      }
    }
  }
}

template <int D, int K, class A>
__global__ void __launch_bounds__(MAX_CTA_THREADS)
lift_kernel_pb(const PBArgs a) {
  using V = typename A::V;
  using IO = typename A::IO;
  __shared__ PBProb<V, IO> pr;
  __shared__ SegPtrs<IO> sp;
  __shared__ int4 it;
  extern __shared__ __align__(16) unsigned char pb_dyn_smem[];
  for (int item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    if (threadIdx.x == 0) {
      it = a.items[item];
      pr = reinterpret_cast<const PBProb<V, IO>*>(a.probs)[it.x];
      sp = reinterpret_cast<const SegPtrs<IO>*>(a.ptrs)[it.x];
    }
    __syncthreads();
    pb_lift_item<D, K, A>(pr, sp, it, a.nrhs, pb_dyn_smem);
    __syncthreads();
  }
}

}  // namespace gp
