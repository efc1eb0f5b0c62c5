// Face kernels of the ghost-penalty operator y = G x on sm_103a.
//
// Per face F with normal axis a (Sec. 2.4), G_F = h^{d-2} (M^ x ... x G^) with
// G^ = sum_j c_j g_j g_j^T of rank k.  The face kernel computes the face output
//
//   t_F[j, tau] = g_j . x_F(:, tau)                    normal lines (k jump values)
//   T_F[tau, j] = s_j (M^ x M^) t_F[j, .]              tangential reference masses
//   W_F[b, tau] = sum_j g_j[b] T_F[tau, j]             normal expansion
//
// i.e. the three-step face apply of Sec. 2.5.1 with the normal step split in
// two around the tangential masses (G^ has rank k), and stores W_F in the
// patch's lexicographic order.  The lift kernel then adds, for every touched
// DoF, the W_F entries of the faces that contain it in a fixed order: a
// gather, so no atomics and bitwise reproducible.  For the overwrite form,
// extra CTAs of the face launch write the zeros of the untouched active DoFs.
//
// Template parameter A (gp_arith.cuh) picks the arithmetic: FP32, FP64, or
// float-float on FP64 data.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "gp_arith.cuh"

namespace gp {

template <int D, int K>
struct Shape {
  static constexpr int L = (D == 2) ? (K + 1) : (K + 1) * (K + 1);  // tangential nodes per face
  static constexpr int NN = 2 * K + 1;                               // nodes on a normal line
  static constexpr int P = NN * L;                                   // patch nodes per face
  static constexpr int FB = (256 / L) > 0 ? (256 / L) : 1;           // default faces per CTA
};

// Tile shape of one (d, k, arithmetic) apply, picked per GPU by the autotuner:
// faces per face CTA (fb * L threads), owner cells per lift CTA and lift threads.
struct Tiles {
  int32_t fb = 0;
  int32_t lcb = 0;
  int32_t lnt = 0;
};

constexpr int MAX_CTA_THREADS = 512;
constexpr size_t MAX_DYN_SMEM = 46 * 1024;   // plus < 2 KB of static shared memory: under the 48 KB default

// dynamic shared memory of the face kernel: the k jump planes (and the first
// tangential pass in 3D) of fb faces
template <int D, int K, typename V>
__host__ __device__ constexpr size_t face_smem(int fb) {
  return (size_t)((D == 3) ? 2 : 1) * fb * K * Shape<D, K>::L * sizeof(V);
}

// Kernel constants (passed by value; they sit in the constant bank).  In FP64 and float-float
// the per-order factor s_j = c_j h^{d-2} is folded into the jump vectors of the first step
// (gs = s_j g_j), so no line multiplies by s_j; FP32 multiplies each line's k tangential results
// by s_j instead (its face kernel is bound by memory instructions, and a batch then needs no
// per-problem table).
template <typename V>
struct FoldScale {
  static constexpr bool value = !std::is_same<V, float>::value;
};
template <typename V, int K>
struct Consts {
  V g[K][2 * K + 1];   // jump of the j-th derivative of patch basis b (row j-1)
  V gs[K][2 * K + 1];  // s_j g_j[b], the jump vectors of the first step (FP64, float-float)
  V s[K];              // s_j (FP32)
  V m[K + 1][K + 1];   // reference mass matrix
  // even and odd halves of the centrosymmetric mass matrix (M^[N-1-p][N-1-i] = M^[p][i], N = k+1):
  // me[p][i] = (M^[p][i] + M^[p][N-1-i]) / 2 (M^[p][i] for the middle i), mo[p][i] = (M^[p][i] - M^[p][N-1-i]) / 2
  V me[(K + 2) / 2][(K + 2) / 2];
  V mo[(K + 1) / 2][(K + 1) / 2];
};

// Fills the even / odd halves of the mass matrix m (row-major, (k+1)^2) into c.
template <typename V, int K>
void mass_halves(const double* m, Consts<V, K>& c) {
  constexpr int N = K + 1, NE = (K + 2) / 2, H = (K + 1) / 2;
  for (int p = 0; p < NE; ++p)
    for (int i = 0; i < NE; ++i) {
      const bool mid = 2 * i == N - 1;
      c.me[p][i] = from_host<V>(mid ? m[p * N + i] : 0.5 * (m[p * N + i] + m[p * N + N - 1 - i]));
    }
  for (int p = 0; p < H; ++p)
    for (int i = 0; i < H; ++i) c.mo[p][i] = from_host<V>(0.5 * (m[p * N + i] - m[p * N + N - 1 - i]));
}

struct FaceArgs {
  const int32_t* frows;   // per-face row starts of the patch (see rbase)
  int64_t rbase[4];       // row entry of face fstart[a] of each axis
  int32_t fstart[4];      // first face of each axis in this launch
  int32_t fend[4];        // one past the last face of each axis in this launch
  int32_t bstart[4];      // first CTA of each axis (after the zero-fill CTAs); bstart[D] = grid
  const int2* zruns;      // (c0, len <= 256) runs of untouched active DoFs
  int32_t nzruns;         // 0 for the add form
  int32_t nzblocks;       // zero-fill CTAs at the front of the grid
  int32_t tail_wait;      // 1: before exiting, wait for the grid this launch programmatically
                          // depends on (slab pipeline: so that this grid completes after it)
};

constexpr int ZGROUP = 16;  // zero runs per zero-fill CTA

struct LiftArgs {
  const int32_t* lwin;    // [nlift][NW] candidate face ids of each owner cell (-1 if none)
  const int32_t* lrow;    // [nlift][KR] compact index of node (ci k, cj k + q, cl k + r)
  int32_t nlift;
  int32_t n_active;
};

// ------------------------------------------------- one normal line's steps --
// The three one-dimensional steps of the face apply for one normal line, shared by the
// face kernel and the brick kernel (gp_brick.cuh).

// Jump values t_j = g_j . v of the line (j = 1..k; row j - 1 of g).  Mirroring the patch
// about the face maps basis b to 2k - b, K- to K+ and d/dn to -d/dn, so
// g_j[2k - b] = (-1)^(j+1) g_j[b]: odd orders see v[b] + v[2k-b], even orders
// v[b] - v[2k-b], and only odd orders see the shared node b = k.
template <int K, typename V>
__device__ __forceinline__ void line_jumps(const V (&v)[2 * K + 1], const V (*g)[2 * K + 1], V (&t)[K]) {
  constexpr int NN = 2 * K + 1;
  V vp[K], vm[K];
#pragma unroll
  for (int b = 0; b < K; ++b) {
    vp[b] = vadd_loose(v[b], v[NN - 1 - b]);
    vm[b] = vsub_loose(v[b], v[NN - 1 - b]);
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const bool odd = (j % 2) == 0;   // order j + 1
    Dot<V> acc = dot_first(g[j][0], odd ? vp[0] : vm[0]);
#pragma unroll
    for (int b = 1; b < K; ++b) dot_fma(acc, g[j][b], odd ? vp[b] : vm[b]);
    if (odd) dot_fma(acc, g[j][K], v[K]);
    t[j] = dot_value(acc);
  }
}

// The mass matrix applied to one line of N = k+1 values u through its even and odd halves:
// y[p] = E_p + O_p and y[N-1-p] = E_p - O_p, E_p = sum_i me[p][i] (u[i] + u[N-1-i]) (the middle
// value once), O_p = sum_i mo[p][i] (u[i] - u[N-1-i]): (N/2)^2 + (N/2 rounded up)^2 terms and
// 2 (N/2) folds and merges instead of N^2 terms.
template <int K, typename V>
__device__ __forceinline__ void mass_line_eo(const Consts<V, K>& c, const V (&u)[K + 1], V (&y)[K + 1]) {
  constexpr int N = K + 1, NE = (K + 2) / 2, H = (K + 1) / 2;
  V e[NE], o[H > 0 ? H : 1];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    e[i] = vadd_loose(u[i], u[N - 1 - i]);
    o[i] = vsub_loose(u[i], u[N - 1 - i]);
  }
  if (N % 2 == 1) e[NE - 1] = u[NE - 1];
#pragma unroll
  for (int p = 0; p < NE; ++p) {
    Dot<V> ev = dot_first(c.me[p][0], e[0]);
#pragma unroll
    for (int i = 1; i < NE; ++i) dot_fma(ev, c.me[p][i], e[i]);
    if (p < H) {
      Dot<V> ov = dot_first(c.mo[p][0], o[0]);
#pragma unroll
      for (int i = 1; i < H; ++i) dot_fma(ov, c.mo[p][i], o[i]);
      y[p] = dot_merge<false>(ev, ov);
      y[N - 1 - p] = dot_merge<true>(ev, ov);
    } else {
      y[p] = dot_value(ev);
    }
  }
}

// The tangential masses applied line by line through the even / odd halves of M^: a task is
// one (face, order j, tangential line of k+1 values); the tasks of the CTA's fb faces are
// spread over its threads in order (task u on thread u), so the busy threads fill whole warps
// and the rest of the CTA idles at the barriers.  Each task moves 2 (k+1) shared-memory values
// instead of the (k+1)^2 of one output per thread, and does (k+1)^2 / 2 + O(k) instead of
// (k+1)^2 multiply-adds.  3D: pass 1 along t1 from `plane` into `plane2`, pass 2 along t2 back
// into `plane`; 2D: one pass, in place (the 2D kernels hold one plane per face).  Thread
// (fl, tau) then reads out[j] = plane[fl][j][tau].  Every thread of the CTA must call it (it
// synchronises); nt >= fb L.
template <int D, int K, typename V, int L>
__device__ __forceinline__ void line_tangential_eo(V (*plane)[K][L], V (*plane2)[K][L], const int fb,
                                                   const Consts<V, K>& c, const int fl, const int tau,
                                                   V (&out)[K]) {
  constexpr int N = K + 1;
  constexpr int T = (D == 3) ? K * N : K;     // tasks per face and pass
  const int u = threadIdx.x;
  const bool task = u < fb * T;
  const int tf = u / T, w = u - tf * T;
  const int j = (D == 3) ? w / N : w, tr = (D == 3) ? w % N : 0;
  if (task) {       // first pass: along t1 within the line t2 = tr (2D: the only pass)
    V uu[N], yv[N];
#pragma unroll
    for (int q = 0; q < N; ++q) uu[q] = plane[tf][j][q + N * tr];
    mass_line_eo<K, V>(c, uu, yv);
    V (*dst)[K][L] = (D == 3) ? plane2 : plane;   // 2D: the task owns row j of its face's plane
#pragma unroll
    for (int i = 0; i < N; ++i) dst[tf][j][i + N * tr] = yv[i];
  }
  __syncthreads();
  if constexpr (D == 3) {
    if (task) {     // second pass: along t2 within the line t1 = tr
      V uu[N], yv[N];
#pragma unroll
      for (int q = 0; q < N; ++q) uu[q] = plane2[tf][j][tr + N * q];
      mass_line_eo<K, V>(c, uu, yv);
#pragma unroll
      for (int i = 0; i < N; ++i) plane[tf][j][tr + N * i] = yv[i];
    }
    __syncthreads();
  }
#pragma unroll
  for (int jj = 0; jj < K; ++jj) out[jj] = plane[fl][jj][tau];
}

// Normal expansion w[b] = sum_j g_j[b] sj[j] (sj: the tangential results of the line):
// w[b] = E_b + O_b and w[2k-b] = E_b - O_b, with E_b (O_b) the sum over odd (even) orders of
// g_j[b] sj[j]; w[k] = E_k.
template <int K, typename V>
__device__ __forceinline__ void line_expand(const Consts<V, K>& c, const V (&sj)[K], V (&w)[2 * K + 1]) {
  constexpr int NN = 2 * K + 1;
#pragma unroll
  for (int b = 0; b <= K; ++b) {
    Dot<V> ev = dot_first(c.g[0][b], sj[0]);
#pragma unroll
    for (int j = 2; j < K; j += 2) dot_fma(ev, c.g[j][b], sj[j]);
    if (b == K || K == 1) {
      const V e = dot_value(ev);
      w[b] = e;
      if (b < K) w[NN - 1 - b] = e;
    } else {
      Dot<V> ov = dot_first(c.g[K > 1 ? 1 : 0][b], sj[K > 1 ? 1 : 0]);
#pragma unroll
      for (int j = 3; j < K; j += 2) dot_fma(ov, c.g[j][b], sj[j]);
      w[b] = dot_merge<false>(ev, ov);
      w[NN - 1 - b] = dot_merge<true>(ev, ov);
    }
  }
}

// ----------------------------------------------------------------- face --
// One thread per (face, normal line tau); fb faces per CTA (blockDim.x = fb L).
// `blk` is the CTA's index within its problem; `gs` holds the jump vectors of the first step
// (FP64, float-float: the scaled s_j g_j, c.gs or a batch segment's copy in shared memory;
// FP32: the plain c.g) and `sc` the k factors s_j (FP32 only); `dsm` is the
// face_smem<D, K, V>(fb) bytes of dynamic shared memory.
template <int D, int K, class A>
__device__ __forceinline__ void face_body(const typename A::IO* __restrict__ x, typename A::V* __restrict__ wp,
                                          typename A::IO* __restrict__ y, const FaceArgs& fa,
                                          const Consts<typename A::V, K>& c, const typename A::V (*gs)[2 * K + 1],
                                          const typename A::V* sc, const int blk, const int fb, unsigned char* dsm) {
  using S = Shape<D, K>;
  using V = typename A::V;
  using IO = typename A::IO;
  constexpr int L = S::L, NN = S::NN, K1 = K + 1;
  typedef V Plane[K][L];
  Plane* buf = reinterpret_cast<Plane*>(dsm);            // [fb][K][L]
  Plane* sb2 = buf + fb;                                  // [fb][K][L], 3D only
  const int nt = (int)blockDim.x;
  // the lift may start its prologue as soon as every face CTA is running (programmatic
  // dependent launch; it waits for this grid's completion before it reads W)
  asm volatile("griddepcontrol.launch_dependents;");

  if (blk < fa.nzblocks) {
    // zero fill of the active DoFs outside every face patch (overwrite form only):
    // ZGROUP runs of <= 256 elements, descriptors fetched in parallel
    __shared__ int2 zr[ZGROUP];
    const int r0 = blk * ZGROUP;
    const int nr = min(ZGROUP, fa.nzruns - r0);
    for (int i = threadIdx.x; i < nr; i += nt) zr[i] = __ldg(fa.zruns + r0 + i);   // nt may be < ZGROUP
    __syncthreads();
    for (int r = 0; r < nr; ++r) {
      const int2 run = zr[r];
      // streaming stores: the zeros are not read again, so they should not push x out of L2
      for (int i = threadIdx.x; i < run.y; i += nt) __stcs(y + run.x + i, IO(0));
    }
    return;
  }
  // axis of this CTA's faces (constant indices only: no local-memory copy of fa)
  int axis = 0, fbase = fa.fstart[0], fend = fa.fend[0], bbase = fa.bstart[0];
  int64_t rbase = fa.rbase[0];
  if (D >= 2 && blk >= fa.bstart[1]) {
    axis = 1; fbase = fa.fstart[1]; fend = fa.fend[1]; bbase = fa.bstart[1]; rbase = fa.rbase[1];
  }
  if (D >= 3 && blk >= fa.bstart[2]) {
    axis = 2; fbase = fa.fstart[2]; fend = fa.fend[2]; bbase = fa.bstart[2]; rbase = fa.rbase[2];
  }
  const int f0 = fbase + (blk - bbase) * fb;
  const int t = threadIdx.x;
  const int fl = t / L, tau = t - fl * L;
  const int f = f0 + fl;
  const bool valid = f < fend;

  // ---- gather this thread's normal line (2k+1 values)
  V v[NN];
  if (valid) {
    if (axis == 0) {
      const int32_t base = __ldg(fa.frows + rbase + (int64_t)(f - fbase) * L + tau);
#pragma unroll
      for (int b = 0; b < NN; ++b) v[b] = from_io(__ldg(x + base + b), (V*)nullptr);
    } else {
      // tau = tx + (K+1) tr; row b of the patch at outer tangential index tr
      constexpr int R = (D == 3) ? NN * K1 : NN;
      const int tx = (D == 3) ? tau % K1 : tau;
      const int tr = (D == 3) ? tau / K1 : 0;
      const int32_t* rows = fa.frows + rbase + (int64_t)(f - fbase) * R + NN * tr;
#pragma unroll
      for (int b = 0; b < NN; ++b) v[b] = from_io(__ldg(x + __ldg(rows + b) + tx), (V*)nullptr);
    }
  } else {
#pragma unroll
    for (int b = 0; b < NN; ++b) v[b] = vzero<V>();
  }
  // ---- contract with the k jump vectors, then the tangential reference masses
  {
    V t[K];
    line_jumps<K, V>(v, gs, t);
#pragma unroll
    for (int j = 0; j < K; ++j) buf[fl][j][tau] = t[j];
  }
  __syncthreads();
  V out[K];
  line_tangential_eo<D, K, V, L>(buf, sb2, fb, c, fl, tau, out);

  // ---- normal expansion W_F[b, tau] = sum_j g_j[b] s_j out[j], stored at tau + L b (the
  // lanes of a face store neighbouring values)
  if (valid) {
    V* dst = wp + (size_t)f * S::P + tau;
    if constexpr (!FoldScale<V>::value) {
#pragma unroll
      for (int j = 0; j < K; ++j) out[j] = vmul(sc[j], out[j]);
    }
    V w[NN];
    line_expand<K, V>(c, out, w);
#pragma unroll
    for (int bb = 0; bb < NN; ++bb) dst[L * bb] = w[bb];
  }
}

extern __shared__ __align__(16) unsigned char gp_dyn_smem[];

template <int D, int K, class A>
__global__ void __launch_bounds__(MAX_CTA_THREADS)
face_kernel(const typename A::IO* __restrict__ x, typename A::V* __restrict__ wp,
            typename A::IO* __restrict__ y, const FaceArgs fa, const int fb,
            const __grid_constant__ Consts<typename A::V, K> c) {
  face_body<D, K, A>(x, wp, y, fa, c, FoldScale<typename A::V>::value ? c.gs : c.g, c.s, blockIdx.x, fb, gp_dyn_smem);
  if (fa.tail_wait) asm volatile("griddepcontrol.wait;" ::: "memory");
}

// --------------------------------------------------------------- batches --
// A batch segment is one (problem, right-hand side) pair of a group of problems
// with the same dimension, degree and arithmetic.  Its x and y pointers live in
// a separate table the host rewrites for every apply.
template <typename V, int K>
struct FaceSeg {
  FaceArgs fa;
  V* wp;           // this segment's face outputs
  const V* gs;     // FP64, float-float: K x (2K+1) scaled jump vectors s_j g_j of the problem
  V s[K];          // FP32: s_j of the problem
  int32_t block0;  // first CTA of the segment in the group's face launch
};

struct LiftSeg {
  LiftArgs la;
  int32_t block0;  // first CTA of the segment in the group's lift launch
};

template <typename IO>
struct SegPtrs {
  const IO* x;
  IO* y;
};

// index of the segment holding CTA `blk`: the last segment whose block0 <= blk
template <typename Seg>
__device__ __forceinline__ int find_segment(const Seg* segs, const int nseg, const int blk) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&segs[mid].block0) <= blk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int D, int K, class A>
__global__ void __launch_bounds__(MAX_CTA_THREADS)
face_kernel_batched(const FaceSeg<typename A::V, K>* __restrict__ segs, const int nseg,
                    const SegPtrs<typename A::IO>* __restrict__ ptrs, const int fb,
                    const __grid_constant__ Consts<typename A::V, K> c) {
  using V = typename A::V;
  __shared__ FaceSeg<V, K> seg;
  __shared__ SegPtrs<typename A::IO> sp;
  __shared__ V sg[K][2 * K + 1];
  if (threadIdx.x == 0) {
    const int s = find_segment(segs, nseg, (int)blockIdx.x);
    seg = segs[s];
    sp = ptrs[s];
  }
  __syncthreads();
  if constexpr (FoldScale<V>::value) {
    for (int i = threadIdx.x; i < K * (2 * K + 1); i += blockDim.x) sg[i / (2 * K + 1)][i % (2 * K + 1)] = seg.gs[i];
    __syncthreads();
    face_body<D, K, A>(sp.x, seg.wp, sp.y, seg.fa, c, sg, seg.s, (int)blockIdx.x - seg.block0, fb, gp_dyn_smem);
  } else {
    face_body<D, K, A>(sp.x, seg.wp, sp.y, seg.fa, c, c.g, seg.s, (int)blockIdx.x - seg.block0, fb, gp_dyn_smem);
  }
}

// ----------------------------------------------------------------- lift --
// Owner cell c = (ci, cj, cl) holds the lattice nodes (ci k + p, cj k + q, cl k + r),
// p, q, r in [0, k).  The faces with normal a whose patch holds such a node have
// lower cell c + (s_a - 2) e_a + (s_1 - 1) e_t1 + (s_2 - 1) e_t2 with s_a in {0,1,2}
// (0 only when p_a = 0) and s_t in {0,1} (0 only when p_t = 0); the node sits at
// normal index b = p_a + (2 - s_a) k and tangential index tau_t = p_t + (1 - s_t) k.
//
// One thread takes one x-row (q, r) of an owner cell: its k nodes p = 0..k-1 are
// contiguous in y.  Face outputs are stored as W_F[b][tau] (tau + L b, x the fastest
// tangential index), so the row's nodes read entries L apart in a face of normal x and
// contiguous entries in the other faces.  The row type
// (q == 0, r == 0) fixes at compile time which of the 36 candidate faces can reach
// the row (p = 0 is the only node on the lower x face).  Each node sums its
// contributions in the fixed order (axis, s_a, s_1, s_2): bitwise reproducible.
template <int D, int K>
struct LiftShape {
  static constexpr int KR = (D == 3) ? K * K : K;   // x-rows per owner cell
  static constexpr int CB0 = 256 / KR;
  static constexpr int CB = CB0 < 1 ? 1 : CB0;      // default owner cells per CTA
  static constexpr int NT = 256;                    // default threads per CTA
  static constexpr int NW = (D == 3) ? 36 : 12;     // candidate faces per cell
  static constexpr int NTYPE = (D == 3) ? 4 : 2;
  // rows of type m (bit 0: q == 0, bit 1: r == 0)
  __host__ __device__ static constexpr int count(int m) {
    int c = 1;
    for (int i = 0; i < D - 1; ++i)
      if (!((m >> i) & 1)) c *= (K - 1);
    return c;
  }
};

// Native FP64: the adds of a missing face are skipped (FP64 issue is the scarce
// resource on GB300; the host groups owner cells with the same candidate-face
// pattern so that the skips are warp-uniform).  FP32 and float-float: branch-free
// (a missing face reads face 0 and adds zeros), with the loads of each (axis, s_a)
// group of up to four faces issued before their adds, so they are in flight together.
// Either way each node adds its contributions in the order (axis, s_a, s_1, s_2).
template <int D, int K, class A, int M>
__device__ __forceinline__ void lift_row(const typename A::V* __restrict__ wp, const int* win, const int q,
                                         const int r, Sum<typename A::V> (&acc)[K], unsigned& found) {
  using V = typename A::V;
  constexpr int K1 = K + 1;
  constexpr int P = Shape<D, K>::P, L = Shape<D, K>::L;
  constexpr bool SKIP = std::is_same<V, double>::value;
  constexpr bool QZ = (M & 1) != 0;   // q == 0
  constexpr bool RZ = (M & 2) != 0;   // r == 0 (3D)
  constexpr unsigned ALL = (1u << K) - 1u;
  // patch position of node p = 0 of this row in the face (a, s_a, s_1, s_2), and how
  // many of the row's k nodes that face reaches
  auto where = [&](const int a, const int sa, const int s1, const int s2, int& cnt) -> int {
    if (a == 0) {             // b = p + (2 - s_a) k on the x-line (q', r') of the face (stride L)
      cnt = (sa == 0) ? 1 : K;
      const int tq = q + (1 - s1) * K;
      const int tr = (D == 3) ? r + (1 - s2) * K : 0;
      return (2 - sa) * K * L + (tq + K1 * tr);
    }
    cnt = (s1 == 0) ? 1 : K;
    if (a == 1) {             // x index p + (1 - s1) k, z index r + (1 - s2) k, b = q + (2 - s_a) k
      const int bb = q + (2 - sa) * K;
      const int tz = (D == 3) ? r + (1 - s2) * K : 0;
      return (1 - s1) * K + K1 * tz + L * bb;
    }
    const int ty = q + (1 - s2) * K;   // normal z: x index p + (1 - s1) k, y index q + (1 - s2) k
    const int bb = r + (2 - sa) * K;
    return (1 - s1) * K + K1 * ty + L * bb;
  };
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int ps = (a == 0) ? L : 1;   // patch stride between the row's nodes
    // zero-ness of the normal coordinate and of the two tangential coordinates
    const bool nz = (a == 0) ? true : ((a == 1) ? QZ : RZ);
    const bool xz = (a == 0) ? QZ : true;         // first tangential: y (a = 0) or x
    const bool yz = (a == 0) ? RZ : ((a == 1) ? RZ : QZ);
#pragma unroll
    for (int sa = 0; sa < 3; ++sa) {
      if (a != 0 && sa == 0 && !nz) continue;
      if constexpr (SKIP) {
        // native FP64: skip the adds of a missing face (warp-uniform by the host's cell order)
#pragma unroll
        for (int s1 = 0; s1 < 2; ++s1) {
          if (s1 == 0 && !xz) continue;
#pragma unroll
          for (int s2 = 0; s2 < ((D == 3) ? 2 : 1); ++s2) {
            if (D == 3 && s2 == 0 && !yz) continue;
            const int f = win[(D == 3) ? a * 12 + sa * 4 + s1 * 2 + s2 : a * 6 + sa * 2 + s1];
            if (f < 0) continue;
            int cnt;
            const int pos = where(a, sa, s1, s2, cnt);
            const V* src = wp + (size_t)f * P + pos;
            // the first contribution of a node sets its sum (no add with zero)
#pragma unroll
            for (int p = 0; p < K; ++p)
              if (p < cnt) {
                if ((found >> p) & 1u) sum_add(acc[p], src[p * ps]);
                else sum_set(acc[p], src[p * ps]);
              }
            found |= (cnt == 1) ? 1u : ALL;
          }
        }
      } else {
        // FP32 and float-float: branch-free.  All loads of the (up to 4) faces of this
        // (a, s_a) are issued before their adds; a missing face reads face 0 and adds 0.
        V ld[4 * K];
        int n = 0;
#pragma unroll
        for (int s1 = 0; s1 < 2; ++s1) {
          if (s1 == 0 && !xz) continue;
#pragma unroll
          for (int s2 = 0; s2 < ((D == 3) ? 2 : 1); ++s2) {
            if (D == 3 && s2 == 0 && !yz) continue;
            const int f = win[(D == 3) ? a * 12 + sa * 4 + s1 * 2 + s2 : a * 6 + sa * 2 + s1];
            const bool ok = f >= 0;
            int cnt;
            const int pos = where(a, sa, s1, s2, cnt);
            const V* src = wp + (size_t)(ok ? f : 0) * P + (ok ? pos : 0);
#pragma unroll
            for (int p = 0; p < K; ++p)
              if (p < cnt) {
                const V v = src[p * ps];
                ld[n++] = ok ? v : vzero<V>();
              }
            if (ok) found |= (cnt == 1) ? 1u : ALL;
          }
        }
        n = 0;
#pragma unroll
        for (int s1 = 0; s1 < 2; ++s1) {
          if (s1 == 0 && !xz) continue;
#pragma unroll
          for (int s2 = 0; s2 < ((D == 3) ? 2 : 1); ++s2) {
            if (D == 3 && s2 == 0 && !yz) continue;
            const int cnt = (a == 0) ? ((sa == 0) ? 1 : K) : ((s1 == 0) ? 1 : K);
#pragma unroll
            for (int p = 0; p < K; ++p)
              if (p < cnt) sum_add(acc[p], ld[n++]);
          }
        }
      }
    }
  }
}

// dynamic shared memory of the lift kernel: the candidate windows of cb cells
template <int D, int K>
__host__ __device__ constexpr size_t lift_smem(int cb) {
  return (size_t)cb * (LiftShape<D, K>::NW + 1) * sizeof(int);
}

// cb owner cells per CTA; each of the blockDim.x threads takes the items g, g + nt, ...
// of the cb * KR rows.
template <int D, int K, class A>
__device__ __forceinline__ void lift_body(const typename A::V* __restrict__ wp, typename A::IO* __restrict__ y,
                                          const int add, const LiftArgs& la, const int blk, const int cb,
                                          unsigned char* dsm) {
  using S = LiftShape<D, K>;
  using V = typename A::V;
  using IO = typename A::IO;
  constexpr int NW = S::NW;
  typedef int Win[NW + 1];
  Win* win = reinterpret_cast<Win*>(dsm);                // [cb][NW + 1]
  const int cell0 = blk * cb;
  const int t = threadIdx.x, nt = (int)blockDim.x;
  for (int idx = t; idx < NW * cb; idx += nt) {
    const int ln = idx / NW, w = idx - ln * NW;
    win[ln][w] = (cell0 + ln < la.nlift) ? __ldg(la.lwin + (size_t)cell0 * NW + idx) : -1;
  }
  __syncthreads();
  // wait for the face kernel (a no-op unless launched as its programmatic dependent), and
  // let a programmatic dependent of this grid start (the cell operator of the model system)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  // one pass: item -> (row type m, cell, row of that type); items sorted by type
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
    if (cell >= la.nlift) continue;
    int q = 0, r = 0;
    if constexpr (K > 1) {
      if (!(m & 1)) { q = 1 + rem % (K - 1); rem /= (K - 1); }
      if (D == 3 && !(m & 2)) { r = 1 + rem % (K - 1); }
    }
    const int row = q + (D == 3 ? K * r : 0);
    const int base = __ldg(la.lrow + (size_t)cell * S::KR + row);
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
    if (base < 0) continue;
#pragma unroll
    for (int p = 0; p < K; ++p) {
      if (!((found >> p) & 1u)) continue;
      const int idx = base + p;
      if (idx >= la.n_active) continue;
      const V sv = dot_value(acc[p]);
      const V outv = add ? vadd(from_io(y[idx], (V*)nullptr), sv) : sv;
      y[idx] = to_io(outv, (IO*)nullptr);
    }
  }
}

template <int D, int K, class A>
__global__ void __launch_bounds__(MAX_CTA_THREADS)
lift_kernel(const typename A::V* __restrict__ wp, typename A::IO* __restrict__ y, const int add,
            const LiftArgs la, const int cb) {
  lift_body<D, K, A>(wp, y, add, la, blockIdx.x, cb, gp_dyn_smem);
}

template <int D, int K, class A>
__global__ void __launch_bounds__(MAX_CTA_THREADS)
lift_kernel_batched(const LiftSeg* __restrict__ segs, const FaceSeg<typename A::V, K>* __restrict__ fsegs,
                    const int nseg, const SegPtrs<typename A::IO>* __restrict__ ptrs, const int cb) {
  __shared__ LiftSeg seg;
  __shared__ typename A::V* wp;
  __shared__ typename A::IO* y;
  if (threadIdx.x == 0) {
    const int s = find_segment(segs, nseg, (int)blockIdx.x);
    seg = segs[s];
    wp = fsegs[s].wp;
    y = ptrs[s].y;
  }
  __syncthreads();
  lift_body<D, K, A>(wp, y, 0, seg.la, (int)blockIdx.x - seg.block0, cb, gp_dyn_smem);
}

}  // namespace gp
