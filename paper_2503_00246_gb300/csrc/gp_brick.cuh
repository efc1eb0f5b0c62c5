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
// involved cells that contain it, in increasing brick index, and writes y.  No atomics:
// bitwise reproducible, and independent of the faces per chunk.
// Extra CTAs at the front of the brick grid zero-fill the active DoFs no face touches.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gp_kernels.cuh"

namespace gp {

constexpr int BRICK_DESC = 8;   // ints per brick descriptor (BDESC of gp_plan.h)
constexpr int BRICK_CMAP = 256; // cells per brick at most (bdim[0] bdim[1] bdim[2])

struct BrickArgs {
  const int32_t* bdesc;    // per brick: first local cell, own cells, local cells, first face, faces, bx, by, bz
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
  const int4* pnode;       // plane nodes: compact index, lattice X, Y, Z
  int32_t nplane;
  const void* part;        // partial grids, V values
  const int32_t* bslot;    // dense brick index -> slot (-1: empty)
  const int8_t* invmask;   // per cell: involved
  int32_t n;
  int32_t bdim[3], nbx[3];
  int64_t pgrid;
  int32_t goff[3][2];
  int32_t gstride[3];
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }

// dynamic shared memory of the brick kernel: per-cell output accumulators of the own cells,
// the staged x blocks of all local cells, and the jump planes of fb faces
template <int D, int K, typename V>
__host__ __device__ constexpr size_t brick_smem(int maxown, int maxcell, int fb) {
  constexpr int NB = (D == 3) ? (K + 1) * (K + 1) * (K + 1) : (K + 1) * (K + 1);
  return align16((size_t)maxown * NB * sizeof(Sum<V>)) + align16((size_t)maxcell * NB * sizeof(V)) +
         (size_t)((D == 3) ? 2 : 1) * fb * K * Shape<D, K>::L * sizeof(V);
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

template <int D, int K, class A>
__global__ void __launch_bounds__(MAX_CTA_THREADS)
brick_kernel(const typename A::IO* __restrict__ x, typename A::IO* __restrict__ y, const int add,
             const BrickArgs ba, const int fb, const __grid_constant__ Consts<typename A::V, K> c) {
  using V = typename A::V;
  using IO = typename A::IO;
  constexpr int L = Shape<D, K>::L, NN = 2 * K + 1, K1 = K + 1;
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
      for (int i = t; i < run.y; i += nt) y[run.x + i] = IO(0);
    }
    return;
  }
  const int brick = (int)blockIdx.x - ba.nzblocks;
  __shared__ int sd[BRICK_DESC];
  __shared__ V sm[K1][K1];
  __shared__ short cmap[BRICK_CMAP];
  if (t < BRICK_DESC) sd[t] = __ldg(ba.bdesc + (size_t)brick * BRICK_DESC + t);
  for (int i = t; i < K1 * K1; i += nt) sm[i / K1][i % K1] = c.m[i / K1][i % K1];
  for (int i = t; i < BRICK_CMAP; i += nt) cmap[i] = -1;
  __syncthreads();
  const int cell_off = sd[0], nown = sd[1], ncell = sd[2], face_off = sd[3], nface = sd[4];
  const int BX = ba.bdim[0], BY = ba.bdim[1], BZ = ba.bdim[2];
  extern __shared__ __align__(16) unsigned char gp_dyn_smem[];
  Sum<V>* ys = reinterpret_cast<Sum<V>*>(gp_dyn_smem);
  V* xs = reinterpret_cast<V*>(gp_dyn_smem + align16((size_t)ba.maxown * NB * sizeof(Sum<V>)));
  Plane* buf = reinterpret_cast<Plane*>(reinterpret_cast<unsigned char*>(xs) +
                                        align16((size_t)ba.maxcell * NB * sizeof(V)));
  Plane* sb2 = buf + fb;

  // ---- own-cell map, zero accumulators, staged x blocks
  for (int i = t; i < nown; i += nt) {
    const int cc = __ldg(ba.bccoord + cell_off + i);
    cmap[(cc & 255) + BX * (((cc >> 8) & 255) + BY * (cc >> 16))] = (short)i;
  }
  for (int i = t; i < nown * NB; i += nt) ys[i] = sum_zero<V>();
  for (int i = t; i < ncell * NB; i += nt) {
    const int lc = i / NB, e = i - lc * NB;
    const int p = e % K1, row = e / K1;
    const int32_t start = __ldg(ba.rowtab + (size_t)__ldg(ba.bcell + cell_off + lc) * L + row);
    xs[i] = from_io(__ldg(x + start + p), (V*)nullptr);
  }
  __syncthreads();

  // ---- faces, fb per chunk, one thread per normal line
  const int fl = t / L, tau = t - fl * L;
  const int fls = fl < fb ? fl : 0;
  for (int f0 = 0; f0 < nface; f0 += fb) {
    const int f = f0 + fl;
    const bool valid = fl < fb && f < nface;
    const uint32_t rec = valid ? __ldg(ba.bface + face_off + f) : 0u;
    const int axis = (int)(rec & 3u);
    const int lo = (int)((rec >> 2) & 1023u), hi = (int)((rec >> 12) & 1023u);
    const bool lo_own = (rec >> 22) & 1u, hi_own = (rec >> 23) & 1u;
    V v[NN];
    if (valid) {
#pragma unroll
      for (int b = 0; b <= K; ++b) v[b] = xs[lo * NB + block_pos<D, K>(axis, b, tau)];
#pragma unroll
      for (int b = 1; b <= K; ++b) v[K + b] = xs[hi * NB + block_pos<D, K>(axis, b, tau)];
    } else {
#pragma unroll
      for (int b = 0; b < NN; ++b) v[b] = vzero<V>();
    }
    {
      V tj[K];
      line_jumps<K, V>(v, c, tj);
      if (fl < fb) {
#pragma unroll
        for (int j = 0; j < K; ++j) buf[fl][j][tau] = tj[j];
      }
    }
    __syncthreads();
    V out[K];
    line_tangential<D, K, V, L>(buf[fls], sb2[fls], sm, tau, out);
    V w[NN];
    if (valid) {
      V sj[K];
#pragma unroll
      for (int j = 0; j < K; ++j) sj[j] = vmul(c.s[j], out[j]);
      line_expand<K, V>(c, sj, w);
    }
    // add to the cell blocks, per axis: K+ parts (b = k..2k), then K- parts (b < k)
    const int fend = min(nface, f0 + fb) - 1;
    const int amin = (int)(__ldg(ba.bface + face_off + f0) & 3u);
    const int amax = (int)(__ldg(ba.bface + face_off + fend) & 3u);
    for (int a = amin; a <= amax; ++a) {
      if (valid && axis == a && hi_own) {
#pragma unroll
        for (int b = 0; b <= K; ++b) sum_add(ys[hi * NB + block_pos<D, K>(a, b, tau)], w[K + b]);
      }
      __syncthreads();
      if (valid && axis == a && lo_own) {
#pragma unroll
        for (int b = 0; b < K; ++b) sum_add(ys[lo * NB + block_pos<D, K>(a, b, tau)], w[b]);
      }
      __syncthreads();
    }
  }

  // ---- nodes of the own cells: sum of the blocks of the own cells that contain the node
  const int bc[3] = {sd[5] * BX, sd[6] * BY, sd[7] * BZ};   // first cell of the brick
  const int bd[3] = {BX, BY, BZ};
  for (int i = t; i < nown * NB; i += nt) {
    const int lc = i / NB, e = i - lc * NB;
    const int pc[3] = {e % K1, (e / K1) % K1, (D == 3) ? e / (K1 * K1) : 0};
    const int cc = __ldg(ba.bccoord + cell_off + lc);
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
      const int32_t dst = __ldg(ba.rowtab + (size_t)__ldg(ba.bcell + cell_off + lc) * L + row) + pc[0];
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
template <int D, class A>
__global__ void __launch_bounds__(256)
plane_fixup_kernel(typename A::IO* __restrict__ y, const int add, const PlaneArgs pa, const int k) {
  using V = typename A::V;
  using IO = typename A::IO;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int4 rec = make_int4(0, 0, 0, 0);
  if (i < pa.nplane) rec = __ldg(pa.pnode + i);
  // the brick kernel's partials and y writes are complete after this wait
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (i >= pa.nplane) return;
  const int X[3] = {rec.y, rec.z, rec.w};
  int c0[3], c1[3], b0[3], b1[3], axis = -1;
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    if (u < D) {
      const bool on = X[u] % k == 0;
      c0[u] = on ? max(X[u] / k - 1, 0) : X[u] / k;
      c1[u] = on ? min(X[u] / k, pa.n - 1) : X[u] / k;
      if (axis < 0 && X[u] % (pa.bdim[u] * k) == 0 && X[u] > 0 && X[u] < pa.n * k) axis = u;
    } else {
      c0[u] = c1[u] = 0;
    }
    b0[u] = c0[u] / pa.bdim[u];
    b1[u] = c1[u] / pa.bdim[u];
  }
  const int u0 = axis == 0 ? 1 : 0, u1 = axis == 2 ? 1 : 2;
  const V* part = reinterpret_cast<const V*>(pa.part);
  V s = vzero<V>();
  bool first = true;
  for (int bz = b0[2]; bz <= b1[2]; ++bz)
    for (int by = b0[1]; by <= b1[1]; ++by)
      for (int bx = b0[0]; bx <= b1[0]; ++bx) {
        const int bb[3] = {bx, by, bz};
        bool found = false;
        for (int cz = c0[2]; cz <= c1[2]; ++cz)
          for (int cy = c0[1]; cy <= c1[1]; ++cy)
            for (int cx = c0[0]; cx <= c1[0]; ++cx)
              if (cx / pa.bdim[0] == bx && cy / pa.bdim[1] == by && cz / pa.bdim[2] == bz &&
                  __ldg(pa.invmask + cx + (size_t)pa.n * (cy + (size_t)(D == 3 ? pa.n : 0) * cz)))
                found = true;
        if (!found) continue;
        const int slot = __ldg(pa.bslot + bx + (size_t)pa.nbx[0] * (by + (size_t)pa.nbx[1] * bz));
        const int side = X[axis] == bb[axis] * pa.bdim[axis] * k ? 0 : 1;
        const int g = (X[u0] - bb[u0] * pa.bdim[u0] * k) +
                      ((D == 3) ? pa.gstride[axis] * (X[u1] - bb[u1] * pa.bdim[u1] * k) : 0);
        const V v = part[(size_t)slot * pa.pgrid + pa.goff[axis][side] + g];
        s = first ? v : vadd(s, v);
        first = false;
      }
  const int ci = rec.x;
  y[ci] = to_io(add ? vadd(from_io(y[ci], (V*)nullptr), s) : s, (IO*)nullptr);
}

}  // namespace gp
