// Brick kernels of y = G x: the face loop and the gather fused, with the cell blocks staged in
// shared memory (the "copy both cells into one array" step of the face apply, Sec. 2.5.1,
// done once per brick of cells instead of once per face).
//
// The mesh is cut into bricks of bdim cells.  One CTA takes one brick that holds involved
// cells (cells that are K- or K+ of a ghost face):
//   1. it copies the (k+1)^d x values of every involved cell of the brick ("own" cells) and of
//      every cell outside the brick that shares a ghost face with one ("halo" cells) into
//      shared memory;
//   2. it evaluates every ghost face with at least one own cell (a face between two bricks is
//      evaluated by both), one thread per normal line, with the three one-dimensional steps
//      of the face kernel (gp_kernels.cuh), and adds the face output W_F to per-cell output
//      blocks of its own cells: W_F[b], b < k, to K- and W_F[b], b >= k, to K+ (the shared
//      node plane b = k belongs to K+), so every entry of W_F lands in exactly one cell block
//      of exactly one brick.  Per cell the contributions arrive in the fixed order
//      (axis 0: lower face, upper face; axis 1: ...; axis 2: ...), whatever the chunking;
//   3. every node of an own cell sums the output blocks of the own cells that contain it (in
//      increasing local cell index).  A node inside the brick has then its complete value and
//      is written to y once; a node on a boundary plane between two bricks (inside the mesh)
//      has contributions in every brick that owns a cell containing it, so each such brick
//      writes its partial sum to a dense grid per box face of the brick (brick slot x pgrid
//      values, box face (a, side) at goff[a][side]; a node on several box faces uses the one
//      of the lowest axis).
// plane_fixup_kernel then adds, for every plane node, the partials of the bricks holding
// involved cells that contain it, in increasing brick index (the host lists their grid
// entries per node), and writes y.  No atomics: bitwise reproducible, and independent of the
// faces per chunk.
// Extra CTAs at the front of the brick grid zero-fill the active DoFs no face touches.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gp_kernels.cuh"

namespace gp {

constexpr int BRICK_DESC = 10;  // ints per brick descriptor (BDESC of gp_plan.h)
constexpr int BRICK_CMAP = 256; // cells per brick at most (bdim[0] bdim[1] bdim[2])

struct BrickArgs {
  const int32_t* bdesc;    // per brick: first local cell, own cells, local cells, first face, faces, bx, by, bz,
                           // first face of axis 1, of axis 2 (within the brick's faces, sorted by axis)
  const int32_t* bcell;    // involved-cell index of every local cell (own first)
  const int32_t* bccoord;  // packed local coords cx | cy << 8 | cz << 16 of the own cells
  const uint32_t* bface;   // packed faces: axis | K- << 2 | K+ << 12 | K- own << 22 | K+ own << 23
  const int32_t* rowtab;   // per involved cell: compact index of node (ci k, row t), t < L
  void* part;              // partial grids, V values
  const int2* zruns;       // zero runs (overwrite form)
  int32_t nzruns, nzblocks;
  int32_t nbricks;
  int32_t bdim[3];
  int32_t n;               // cells per axis
  int64_t pgrid;           // partial entries per brick
  int32_t goff[3][2];      // offset of box face (axis, side) in a brick's partial grid
  int32_t gstride[3];      // row stride of box face a's grid: bdim[u0] k + 1, u0 the first other axis
  int32_t maxcell, maxown; // shared-memory sizing (largest brick)
};

struct PlaneArgs {
  const int32_t* pnode;    // per plane node: compact index of the DoF
  const int32_t* poff;     // plane nodes + 1: offsets into pslot
  const int32_t* pslot;    // partial-grid entries to add, per node in increasing brick index
  int32_t nplane;
  const void* part;        // partial grids, V values
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }

// dynamic shared memory of the brick kernel: per-cell output accumulators of the own cells,
// the staged x blocks of all local cells, the own cells' coordinates, and one region that
// holds first the local cells' row starts (staging), then the jump planes of fb faces (face
// loop), then the own cells' row starts (output)
template <int D, int K, typename V>
__host__ __device__ constexpr size_t brick_smem_region(int maxcell, int fb) {
  const size_t planes = (size_t)((D == 3) ? 2 : 1) * fb * K * Shape<D, K>::L * sizeof(V);
  const size_t rows = (size_t)maxcell * Shape<D, K>::L * sizeof(int32_t);
  return planes > rows ? planes : rows;
}
template <int D, int K, typename V>
__host__ __device__ constexpr size_t brick_smem(int maxown, int maxcell, int fb) {
  constexpr int NB = (D == 3) ? (K + 1) * (K + 1) * (K + 1) : (K + 1) * (K + 1);
  return align16((size_t)maxown * NB * sizeof(Sum<V>)) + align16((size_t)maxcell * NB * sizeof(V)) +
         align16((size_t)maxown * sizeof(int32_t)) + brick_smem_region<D, K, V>(maxcell, fb);
}

// Row starts of `count` local cells (from local cell `first`): rows[i] = rowtab of the cell's
// involved index, i < count * L; four independent loads in flight per thread.
template <int L>
__device__ __forceinline__ void load_rows(int32_t* rows, const int32_t* __restrict__ bcell,
                                          const int32_t* __restrict__ rowtab, const int count, const int t,
                                          const int nt) {
  const int total = count * L;
  for (int base = t; base < total; base += 4 * nt) {
    int32_t inv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = base + u * nt;
      inv[u] = i < total ? __ldg(bcell + i / L) : 0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = base + u * nt;
      if (i < total) rows[i] = __ldg(rowtab + (size_t)inv[u] * L + (i % L));
    }
  }
}

// position of node (normal index bn, tangential index tau) of a face with normal `axis` in a
// cell block (x fastest); tau = t1 + (k+1) t2 with t1, t2 the tangential axes in increasing order
template <int D, int K>
__device__ __forceinline__ int block_pos(const int axis, const int bn, const int tau) {
  constexpr int K1 = K + 1;
  if (axis == 0) return bn + K1 * tau;
  if (D == 2) return tau + K1 * bn;
  if (axis == 1) return (tau % K1) + K1 * bn + K1 * K1 * (tau / K1);
  return tau + K1 * K1 * bn;
}

// One chunk of faces [f0, min(f0 + fb, f1)) with normal AX: thread (fl, tau) gathers its
// normal line from the staged x blocks, runs the three one-dimensional steps and adds the line's
// outputs to the own cells' accumulators: the K+ parts (b = k..2k) of every face, a barrier, then
// the K- parts (b < k).  Every thread of the CTA calls it (it synchronises).
template <int D, int K, class A, int AX>
__device__ __forceinline__ void brick_chunk(const uint32_t* __restrict__ bface, const int f0, const int f1,
                                            const int fl, const int tau, const int fb, const typename A::V* xs,
                                            Sum<typename A::V>* ys,
                                            typename A::V (*buf)[K][Shape<D, K>::L],
                                            typename A::V (*sb2)[K][Shape<D, K>::L],
                                            const Consts<typename A::V, K>& c) {
  using V = typename A::V;
  constexpr int L = Shape<D, K>::L, NN = 2 * K + 1, K1 = K + 1;
  constexpr int NB = (D == 3) ? K1 * K1 * K1 : K1 * K1;
  const int f = f0 + fl;
  const bool valid = f < f1;
  const uint32_t rec = valid ? __ldg(bface + f) : 0u;
  const int lo = (int)((rec >> 2) & 1023u), hi = (int)((rec >> 12) & 1023u);
  const bool lo_own = (rec >> 22) & 1u, hi_own = (rec >> 23) & 1u;
  V v[NN];
  if (valid) {
#pragma unroll
    for (int b = 0; b <= K; ++b) v[b] = xs[lo * NB + block_pos<D, K>(AX, b, tau)];
#pragma unroll
    for (int b = 1; b <= K; ++b) v[K + b] = xs[hi * NB + block_pos<D, K>(AX, b, tau)];
  } else {
#pragma unroll
    for (int b = 0; b < NN; ++b) v[b] = vzero<V>();
  }
  {
    V tj[K];
    line_jumps<K, V>(v, FoldScale<V>::value ? c.gs : c.g, tj);
#pragma unroll
    for (int j = 0; j < K; ++j) buf[fl][j][tau] = tj[j];
  }
  __syncthreads();
  V out[K];
  line_tangential_eo<D, K, V, L>(buf, sb2, fb, c, fl, tau, out);
  V w[NN];
  if (valid) {
    if constexpr (!FoldScale<V>::value) {
#pragma unroll
      for (int j = 0; j < K; ++j) out[j] = vmul(c.s[j], out[j]);
    }
    line_expand<K, V>(c, out, w);
  }
  if (valid && hi_own) {
#pragma unroll
    for (int b = 0; b <= K; ++b) sum_add(ys[hi * NB + block_pos<D, K>(AX, b, tau)], w[K + b]);
  }
  __syncthreads();
  if (valid && lo_own) {
#pragma unroll
    for (int b = 0; b < K; ++b) sum_add(ys[lo * NB + block_pos<D, K>(AX, b, tau)], w[b]);
  }
  __syncthreads();
}

template <int D, int K, class A>
__global__ void __launch_bounds__(MAX_CTA_THREADS)
brick_kernel(const typename A::IO* __restrict__ x, typename A::IO* __restrict__ y, const int add,
             const BrickArgs ba, const int fb, const __grid_constant__ Consts<typename A::V, K> c) {
  using V = typename A::V;
  using IO = typename A::IO;
  constexpr int L = Shape<D, K>::L, K1 = K + 1;
  constexpr int NB = (D == 3) ? K1 * K1 * K1 : K1 * K1;
  typedef V Plane[K][L];
  const int t = threadIdx.x, nt = (int)blockDim.x;
  // the plane fixup may take its prologue while the bricks run (it waits for this grid)
  asm volatile("griddepcontrol.launch_dependents;");

  if ((int)blockIdx.x < ba.nzblocks) {
    // zero fill of the active DoFs outside every face patch (overwrite form only)
    __shared__ int2 zr[ZGROUP];
    const int r0 = blockIdx.x * ZGROUP;
    const int nr = min(ZGROUP, ba.nzruns - r0);
    for (int i = t; i < nr; i += nt) zr[i] = __ldg(ba.zruns + r0 + i);
    __syncthreads();
    for (int r = 0; r < nr; ++r) {
      const int2 run = zr[r];
      for (int i = t; i < run.y; i += nt) __stcs(y + run.x + i, IO(0));   // not read again: streaming
    }
    return;
  }
  const int brick = (int)blockIdx.x - ba.nzblocks;
  __shared__ int sd[BRICK_DESC];
  __shared__ short cmap[BRICK_CMAP];
  for (int i = t; i < BRICK_DESC; i += nt) sd[i] = __ldg(ba.bdesc + (size_t)brick * BRICK_DESC + i);
  for (int i = t; i < BRICK_CMAP; i += nt) cmap[i] = -1;
  __syncthreads();
  const int cell_off = sd[0], nown = sd[1], ncell = sd[2], face_off = sd[3], nface = sd[4];
  const int BX = ba.bdim[0], BY = ba.bdim[1], BZ = ba.bdim[2];
  extern __shared__ __align__(16) unsigned char gp_dyn_smem[];
  unsigned char* p0 = gp_dyn_smem;
  Sum<V>* ys = reinterpret_cast<Sum<V>*>(p0);
  p0 += align16((size_t)ba.maxown * NB * sizeof(Sum<V>));
  V* xs = reinterpret_cast<V*>(p0);
  p0 += align16((size_t)ba.maxcell * NB * sizeof(V));
  int32_t* scc = reinterpret_cast<int32_t*>(p0);
  p0 += align16((size_t)ba.maxown * sizeof(int32_t));
  int32_t* srow = reinterpret_cast<int32_t*>(p0);          // region: row starts ...
  Plane* buf = reinterpret_cast<Plane*>(p0);               // ... or jump planes
  Plane* sb2 = buf + fb;

  // ---- own-cell map and coordinates, zero accumulators, row starts, staged x blocks
  for (int i = t; i < nown; i += nt) {
    const int cc = __ldg(ba.bccoord + cell_off + i);
    scc[i] = cc;
    cmap[(cc & 255) + BX * (((cc >> 8) & 255) + BY * (cc >> 16))] = (short)i;
  }
  for (int i = t; i < nown * NB; i += nt) ys[i] = sum_zero<V>();
  load_rows<L>(srow, ba.bcell + cell_off, ba.rowtab, ncell, t, nt);
  __syncthreads();
  {
    const int total = ncell * NB;
    for (int base = t; base < total; base += 8 * nt) {
      IO v8[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = base + u * nt;
        if (i < total) {
          const int lc = i / NB, e = i - lc * NB;
          v8[u] = __ldg(x + srow[lc * L + e / K1] + (e % K1));
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = base + u * nt;
        if (i < total) xs[i] = from_io(v8[u], (V*)nullptr);
      }
    }
  }
  __syncthreads();

  // ---- faces, axis by axis, fb per chunk, one thread per normal line
  {
    const int fl = t / L, tau = t - fl * L;
    const uint32_t* bf = ba.bface + face_off;
    const int a1 = sd[8], a2 = (D == 3) ? sd[9] : nface;
    for (int f0 = 0; f0 < a1; f0 += fb) brick_chunk<D, K, A, 0>(bf, f0, a1, fl, tau, fb, xs, ys, buf, sb2, c);
    for (int f0 = a1; f0 < a2; f0 += fb) brick_chunk<D, K, A, 1>(bf, f0, a2, fl, tau, fb, xs, ys, buf, sb2, c);
    if constexpr (D == 3) {
      for (int f0 = a2; f0 < nface; f0 += fb)
        brick_chunk<D, K, A, 2>(bf, f0, nface, fl, tau, fb, xs, ys, buf, sb2, c);
    }
  }

  // ---- nodes of the own cells: sum of the blocks of the own cells that contain the node
  load_rows<L>(srow, ba.bcell + cell_off, ba.rowtab, nown, t, nt);   // the face loop has ended
  __syncthreads();
  const int bc[3] = {sd[5] * BX, sd[6] * BY, sd[7] * BZ};   // first cell of the brick
  const int bd[3] = {BX, BY, BZ};
  for (int i = t; i < nown * NB; i += nt) {
    const int lc = i / NB, e = i - lc * NB;
    const int pc[3] = {e % K1, (e / K1) % K1, (D == 3) ? e / (K1 * K1) : 0};
    const int cc = scc[lc];
    const int cl[3] = {cc & 255, (cc >> 8) & 255, cc >> 16};
    // local cells that contain the node: per axis cl - 1 (p = 0), cl, cl + 1 (p = k)
    int lo3[3], hi3[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      lo3[u] = (u < D && pc[u] == 0 && cl[u] > 0) ? cl[u] - 1 : cl[u];
      hi3[u] = (u < D && pc[u] == K && cl[u] + 1 < bd[u]) ? cl[u] + 1 : cl[u];
    }
    // the own cell of largest local index among them writes the node
    int best = -1;
    for (int z = lo3[2]; z <= hi3[2]; ++z)
      for (int yy = lo3[1]; yy <= hi3[1]; ++yy)
        for (int xx = lo3[0]; xx <= hi3[0]; ++xx)
          if (cmap[xx + BX * (yy + BY * z)] >= 0) best = xx + BX * (yy + BY * z);
    if (best != cl[0] + BX * (cl[1] + BY * cl[2])) continue;
    Sum<V> s = sum_zero<V>();
    for (int z = lo3[2]; z <= hi3[2]; ++z)
      for (int yy = lo3[1]; yy <= hi3[1]; ++yy)
        for (int xx = lo3[0]; xx <= hi3[0]; ++xx) {
          const int l2 = cmap[xx + BX * (yy + BY * z)];
          if (l2 < 0) continue;
          const int q3[3] = {pc[0] + K * (cl[0] - xx), pc[1] + K * (cl[1] - yy), pc[2] + K * (cl[2] - z)};
          sum_merge(s, ys[l2 * NB + q3[0] + K1 * (q3[1] + K1 * q3[2])]);
        }
    const V val = dot_value(s);
    // lattice coordinates; the lowest axis on which the node lies on a brick boundary inside the mesh
    int X[3], pa = -1;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      X[u] = (bc[u] + cl[u]) * K + pc[u];
      if (u < D && pa < 0 && X[u] % (bd[u] * K) == 0 && X[u] > 0 && X[u] < ba.n * K) pa = u;
    }
    if (pa < 0) {
      const int row = (D == 3) ? pc[1] + K1 * pc[2] : pc[1];
      const int32_t dst = srow[lc * L + row] + pc[0];
      y[dst] = to_io(add ? vadd(from_io(y[dst], (V*)nullptr), val) : val, (IO*)nullptr);
    } else {
      const int side = X[pa] == bc[pa] * K ? 0 : 1;
      const int u0 = pa == 0 ? 1 : 0, u1 = pa == 2 ? 1 : 2;
      const int g = (X[u0] - bc[u0] * K) + ((D == 3) ? ba.gstride[pa] * (X[u1] - bc[u1] * K) : 0);
      reinterpret_cast<V*>(ba.part)[(size_t)brick * ba.pgrid + ba.goff[pa][side] + g] = val;
    }
  }
}

// One thread per plane node: the partials of the bricks holding involved cells that contain
// the node, summed in increasing brick index, into y.
template <class A>
__global__ void __launch_bounds__(256)
plane_fixup_kernel(typename A::IO* __restrict__ y, const int add, const PlaneArgs pa) {
  using V = typename A::V;
  using IO = typename A::IO;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int ci = 0, s0 = 0, s1 = 0;
  if (i < pa.nplane) {
    ci = __ldg(pa.pnode + i);
    s0 = __ldg(pa.poff + i);
    s1 = __ldg(pa.poff + i + 1);
  }
  // the brick kernel's partials and y writes are complete after this wait
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (i >= pa.nplane) return;
  const V* part = reinterpret_cast<const V*>(pa.part);
  V s = part[__ldg(pa.pslot + s0)];
  for (int j = s0 + 1; j < s1; ++j) s = vadd(s, part[__ldg(pa.pslot + j)]);
  y[ci] = to_io(add ? vadd(from_io(y[ci], (V*)nullptr), s) : s, (IO*)nullptr);
}

}  // namespace gp
