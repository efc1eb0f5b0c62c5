// Mass + Laplace stiffness of the active cells, y (+)= (wm M_active + ws K_active) x, for
// the model SPD system (M_active + K_active + G) u = b of the defect-correction
// solver.  Every active cell is integrated as a full cube (no cut quadrature):
// the interior-cell evaluation of Sec. 2.5.2, with the k+1 Gauss points per
// direction folded into the 1D reference mass M^ and stiffness S^, so that
//
//   A_K = h^d  M^ x M^ x M^  +  h^(d-2) (S^ x M^ x M^ + M^ x S^ x M^ + M^ x M^ x S^)
//
// is applied by sum factorisation: a = M^ x, b = S^ x along x; c = M^ a, d = S^ a,
// e = M^ b along y; y_K = M^ (h^3 c + h (d + e)) + S^ (h c) along z (3D), or
// y_K = M^ (h^2 a + b) + S^ a along y (2D).  One thread per x-line of a cell; the y
// and z passes go through shared memory.  Every 1D application uses the even / odd
// halves of the centrosymmetric M^ and S^ (about half the multiply-adds; CellConsts).  The float-float form renormalises after every
// operation here (the model system's outer residual needs the full accuracy).
//
// Two launches, like the face operator: cell_kernel stores every cell's (k+1)^d
// outputs, and cell_gather adds, for every node, the outputs of the (up to 2^d) active
// cells that hold it, in a fixed order: no atomics, no colour phases, bitwise
// reproducible.  In the model system's apply the gather first adds the ghost-face
// outputs of the node (the lift's row code) and so writes y = (M + K + G) x once.  Both
// are programmatic dependents of the kernel before them: cell_kernel reads only x and
// the tables, so it runs while the ghost-penalty face kernel drains and waits for it
// only before it exits; cell_gather waits for cell_kernel before it touches y.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gp_arith.cuh"
#include "gp_kernels.cuh"

namespace gp {

template <int D, int K>
struct CellShape {
  static constexpr int K1 = K + 1;
  static constexpr int R = (D == 3) ? K1 * K1 : K1;        // x-lines per cell
  static constexpr int NODES = R * K1;                      // nodes per cell
  static constexpr int CB = (256 / R) > 0 ? 256 / R : 1;   // cells per CTA
  static constexpr int NT = CB * R;
  static constexpr int NWC = (D == 3) ? 8 : 4;              // cells holding a node
  static constexpr int KR = (D == 3) ? K * K : K;           // x-rows per owner cell
};

// Even / odd halves of a centrosymmetric (N x N) matrix A (A[N-1-p][N-1-q] = A[p][q]; the 1D
// reference mass and stiffness on the Gauss-Lobatto nodes, which are symmetric about the
// cell centre).  With the folded input e[i] = x[i] + x[N-1-i], o[i] = x[i] - x[N-1-i]
// (i < N/2) and e[N/2] = x[N/2] for odd N,
//   y[p] = E_p + O_p,  y[N-1-p] = E_p - O_p  (p < N/2),  y[N/2] = E_{N/2}  (odd N),
//   E_p = sum_i ae[p][i] e[i],  O_p = sum_i ao[p][i] o[i],
// with ae[p][i] = (A[p][i] + A[p][N-1-i]) / 2, ae[p][N/2] = A[p][N/2] and
// ao[p][i] = (A[p][i] - A[p][N-1-i]) / 2: (N/2 + 1)(N+1)/2 + (N/2)^2 multiply-adds instead
// of N^2.
template <typename V, int K>
struct CellConsts {
  static constexpr int N = K + 1, H = N / 2, NE = (N + 1) / 2;
  V me[NE][NE];  // reference mass, even half
  V mo[H][H];    // reference mass, odd half
  V se[NE][NE];  // reference stiffness, even half
  V so[H][H];    // reference stiffness, odd half
  V hm;          // wm h^d
  V hs;          // ws h^(d-2)
};

template <int N, class V>
__device__ __forceinline__ void eo_fold(const V (&x)[N], V (&e)[(N + 1) / 2], V (&o)[N / 2]) {
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    e[i] = vadd(x[i], x[N - 1 - i]);
    o[i] = vsub(x[i], x[N - 1 - i]);
  }
  if constexpr (N % 2 == 1) e[N / 2] = x[N / 2];
}

// the even (E) or odd (O) partial sum of output p: sum_i a[p][i] v[i]
template <int M, class V>
__device__ __forceinline__ V eo_row(const V (&a)[M], const V (&v)[M]) {
  V acc = vmul(a[0], v[0]);
#pragma unroll
  for (int i = 1; i < M; ++i) acc = vfma(a[i], v[i], acc);
  return acc;
}
template <int M, class V>
__device__ __forceinline__ V eo_row2(const V (&a)[M], const V (&v)[M], const V (&b)[M], const V (&w)[M]) {
  V acc = vmul(a[0], v[0]);
#pragma unroll
  for (int i = 1; i < M; ++i) acc = vfma(a[i], v[i], acc);
#pragma unroll
  for (int i = 0; i < M; ++i) acc = vfma(b[i], w[i], acc);
  return acc;
}

// Device tables of the cell operator (see Plan::crow, cwin, corow).
struct CellTabs {
  const int32_t* crow = nullptr;   // [ncact][R] compact index of each x-line start
  int32_t ncact = 0;
  const int32_t* cwin = nullptr;   // [ncown][NWC] active-cell index of (ci - s_x, cj - s_y, cl - s_z)
  const int32_t* corow = nullptr;  // [ncown][KR] compact index of node (ci k, cj k + q, cl k + r)
  int32_t ncown = 0;
  int32_t n_active = 0;
  void* wc = nullptr;              // [ncact][NODES] cell outputs (scratch)
  // optional fused inner product for CG: per gather CTA, sum over its nodes of
  // dotp[i] * y[i] (the stored result) into dotpart[blockIdx.x] (fixed order)
  const void* dotp = nullptr;
  double* dotpart = nullptr;
  // optional fused ghost penalty (the model system's M + K + G in one gather): the face
  // kernel's outputs, its candidate-face windows per lift owner cell, and per owner cell of
  // this table its lift owner index (-1: no ghost face reaches it)
  const void* wf = nullptr;
  const int32_t* fwin = nullptr;
  const int32_t* own2lift = nullptr;
};

constexpr int GATHER_THREADS = 256;

// the two fields of a pass kept side by side in shared memory, so that one access
// moves both (half the shared-memory instructions)
template <typename V>
struct alignas(2 * sizeof(V)) VPair {
  V a, b;
};

template <int D, int K, class A>
__global__ void __launch_bounds__(CellShape<D, K>::NT)
cell_kernel(const typename A::IO* __restrict__ x, typename A::V* __restrict__ wc, const int32_t* __restrict__ crow,
            const int32_t ncact, const __grid_constant__ CellConsts<typename A::V, K> c) {
  using S = CellShape<D, K>;
  using V = typename A::V;
  constexpr int K1 = S::K1, R = S::R, NODES = S::NODES, CB = S::CB;
  constexpr int H = K1 / 2, NE = (K1 + 1) / 2;
  __shared__ VPair<V> sab[CB][NODES];
  const int t = threadIdx.x;
  const int cl = t / R, line = t - cl * R;
  const int cell = blockIdx.x * CB + cl;
  const bool valid = cell < ncact;
  const int32_t row = valid ? __ldg(crow + (size_t)cell * R + line) : 0;
  asm volatile("griddepcontrol.launch_dependents;");

  // ---- x pass: a = M^ x, b = S^ x on this thread's x-line
  {
    V xl[K1], e[NE], o[H];
#pragma unroll
    for (int i = 0; i < K1; ++i) xl[i] = valid ? from_io(__ldg(x + row + i), (V*)nullptr) : vzero<V>();
    eo_fold<K1>(xl, e, o);
#pragma unroll
    for (int p = 0; p < NE; ++p) {
      const V ae = eo_row<NE>(c.me[p], e), be = eo_row<NE>(c.se[p], e);
      if (p < H) {
        const V ao = eo_row<H>(c.mo[p], o), bo = eo_row<H>(c.so[p], o);
        sab[cl][p + K1 * line] = VPair<V>{vadd(ae, ao), vadd(be, bo)};
        sab[cl][K1 - 1 - p + K1 * line] = VPair<V>{vsub(ae, ao), vsub(be, bo)};
      } else {
        sab[cl][p + K1 * line] = VPair<V>{ae, be};
      }
    }
  }
  __syncthreads();

  V yout[K1];
  if constexpr (D == 3) {
    // ---- y pass on the line (i1, i3): f = h^3 M^ a + h (S^ a + M^ b), g = h M^ a
    {
      const int i1 = line % K1, i3 = line / K1;
      V ay[K1], by[K1], ae[NE], ao[H], be[NE], bo[H];
#pragma unroll
      for (int q = 0; q < K1; ++q) {
        const VPair<V> v = sab[cl][i1 + K1 * (q + K1 * i3)];
        ay[q] = v.a;
        by[q] = v.b;
      }
      eo_fold<K1>(ay, ae, ao);
      eo_fold<K1>(by, be, bo);
#pragma unroll
      for (int p = 0; p < NE; ++p) {
        const V cE = eo_row<NE>(c.me[p], ae), tE = eo_row2<NE>(c.se[p], ae, c.me[p], be);
        if (p < H) {
          const V cO = eo_row<H>(c.mo[p], ao), tO = eo_row2<H>(c.so[p], ao, c.mo[p], bo);
          const V c0 = vadd(cE, cO), c1 = vsub(cE, cO), t0 = vadd(tE, tO), t1 = vsub(tE, tO);
          sab[cl][i1 + K1 * (p + K1 * i3)] = VPair<V>{vfma(c.hm, c0, vmul(c.hs, t0)), vmul(c.hs, c0)};
          sab[cl][i1 + K1 * (K1 - 1 - p + K1 * i3)] = VPair<V>{vfma(c.hm, c1, vmul(c.hs, t1)), vmul(c.hs, c1)};
        } else {
          sab[cl][i1 + K1 * (p + K1 * i3)] = VPair<V>{vfma(c.hm, cE, vmul(c.hs, tE)), vmul(c.hs, cE)};
        }
      }
    }
    __syncthreads();
    // ---- z pass on the line (i1, i2): y = M^ f + S^ g, stored along z
    {
      const int i1 = line % K1, i2 = line / K1;
      V fz[K1], gz[K1], fe[NE], fo[H], ge[NE], go[H];
#pragma unroll
      for (int q = 0; q < K1; ++q) {
        const VPair<V> v = sab[cl][i1 + K1 * (i2 + K1 * q)];
        fz[q] = v.a;
        gz[q] = v.b;
      }
      eo_fold<K1>(fz, fe, fo);
      eo_fold<K1>(gz, ge, go);
#pragma unroll
      for (int p = 0; p < NE; ++p) {
        const V yE = eo_row2<NE>(c.me[p], fe, c.se[p], ge);
        if (p < H) {
          const V yO = eo_row2<H>(c.mo[p], fo, c.so[p], go);
          yout[p] = vadd(yE, yO);
          yout[K1 - 1 - p] = vsub(yE, yO);
        } else {
          yout[p] = yE;
        }
      }
      if (valid) {
        V* dst = wc + (size_t)cell * NODES;
#pragma unroll
        for (int p = 0; p < K1; ++p) dst[i1 + K1 * (i2 + K1 * p)] = yout[p];
      }
    }
    // the completion of this grid stands for the completion of the kernel before it
    asm volatile("griddepcontrol.wait;" ::: "memory");
  } else {
    // ---- y pass on the line i1: y = M^ (h^2 a + b) + S^ a
    V f[K1], g[K1], fe[NE], fo[H], ge[NE], go[H];
#pragma unroll
    for (int q = 0; q < K1; ++q) {
      const VPair<V> v = sab[cl][line + K1 * q];
      const V ay = v.a, by = v.b;
      f[q] = vfma(c.hm, ay, vmul(c.hs, by));
      g[q] = vmul(c.hs, ay);
    }
    eo_fold<K1>(f, fe, fo);
    eo_fold<K1>(g, ge, go);
#pragma unroll
    for (int p = 0; p < NE; ++p) {
      const V yE = eo_row2<NE>(c.me[p], fe, c.se[p], ge);
      if (p < H) {
        const V yO = eo_row2<H>(c.mo[p], fo, c.so[p], go);
        yout[p] = vadd(yE, yO);
        yout[K1 - 1 - p] = vsub(yE, yO);
      } else {
        yout[p] = yE;
      }
    }
    if (valid) {
      V* dst = wc + (size_t)cell * NODES;
#pragma unroll
      for (int p = 0; p < K1; ++p) dst[line + K1 * p] = yout[p];
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
  }
}

// One thread per x-row (q, r) of an owner cell: its k nodes p add the outputs of the cells
// (ci - s_x, cj - s_y, cl - s_z) that hold them (s_y = 1 only for q = 0, s_z = 1 only for
// r = 0, s_x = 1 only for p = 0), in the order w = s_x + 2 s_y + 4 s_z.
template <int D, int K, class A>
__device__ __forceinline__ void gather_row(const typename A::V* __restrict__ wc, typename A::IO* __restrict__ y,
                                           const int add, const CellTabs& ct, const int own, const int t,
                                           const int base, IoDot<typename A::IO>& dot) {
  using S = CellShape<D, K>;
  using V = typename A::V;
  using IO = typename A::IO;
  constexpr int K1 = S::K1, NODES = S::NODES, NWC = S::NWC;
  const int q = t % K, r = (D == 3) ? t / K : 0;
  Sum<V> acc[K];
#pragma unroll
  for (int p = 0; p < K; ++p) acc[p] = sum_zero<V>();
  bool any0 = false, anyp = false;
  if (ct.wf) {
    // the ghost penalty first: the faces whose patch holds this row, in the lift's order
    const int li = __ldg(ct.own2lift + own);
    if (li >= 0) {
      const int* win = ct.fwin + (size_t)li * LiftShape<D, K>::NW;
      const V* wf = (const V*)ct.wf;
      unsigned found = 0;
      const int m = (q == 0 ? 1 : 0) + (r == 0 && D == 3 ? 2 : 0);
      switch (m) {
        case 0: lift_row<D, K, A, 0>(wf, win, q, r, acc, found); break;
        case 1: lift_row<D, K, A, 1>(wf, win, q, r, acc, found); break;
        case 2: lift_row<D, K, A, 2>(wf, win, q, r, acc, found); break;
        default: lift_row<D, K, A, 3>(wf, win, q, r, acc, found); break;
      }
    }
  }
  // the owner's window (2^d cell indices, one vector load), then per group of four
  // windows (s_z fixed) every cell-output load of the row before the first add; the adds
  // run in the window order w = s_x + 2 s_y + 4 s_z
  int cw[NWC];
  {
    const int4* wv = reinterpret_cast<const int4*>(ct.cwin + (size_t)own * NWC);
#pragma unroll
    for (int i = 0; i < NWC / 4; ++i) {
      const int4 v4 = __ldg(wv + i);
      cw[4 * i] = v4.x;
      cw[4 * i + 1] = v4.y;
      cw[4 * i + 2] = v4.z;
      cw[4 * i + 3] = v4.w;
    }
  }
#pragma unroll
  for (int sz = 0; sz < (D == 3 ? 2 : 1); ++sz) {
    if (sz && r != 0) break;
    V v0[2][K], v1[2];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int w = u + 4 * sz, sx = u & 1, sy = u >> 1;
      ok[u] = cw[w] >= 0 && !(sy && q != 0);
      // in-bounds address even where the window is unused (cell 0, row 0)
      const int ly = ok[u] ? q + sy * K : 0, lz = ok[u] ? r + sz * K : 0;
      const V* src = wc + (size_t)(ok[u] ? cw[w] : 0) * NODES + K1 * (ly + (D == 3 ? K1 * lz : 0));
      if (sx == 0) {
#pragma unroll
        for (int p = 0; p < K; ++p) v0[sy][p] = ok[u] ? src[p] : vzero<V>();
      } else {
        v1[sy] = ok[u] ? src[K] : vzero<V>();
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!ok[u]) continue;
      if ((u & 1) == 0) {
#pragma unroll
        for (int p = 0; p < K; ++p) sum_add(acc[p], v0[u >> 1][p]);
        any0 = anyp = true;
      } else {
        sum_add(acc[0], v1[u >> 1]);
        any0 = true;
      }
    }
  }
#pragma unroll
  for (int p = 0; p < K; ++p) {
    if (p == 0 ? !any0 : !anyp) continue;
    const int idx = base + p;
    if (idx >= ct.n_active) break;
    const V sv = dot_value(acc[p]);
    const V outv = add ? vadd(from_io(y[idx], (V*)nullptr), sv) : sv;
    const IO o = to_io(outv, (IO*)nullptr);
    y[idx] = o;
    if (ct.dotp) dot.add(((const IO*)ct.dotp)[idx], o);
  }
}

// A gather CTA takes GATHER_THREADS / KR whole owner cells.  Its threads are ordered
// by row type (q == 0, r == 0) first, so that a warp's rows take the same path through
// the row code (the candidate ghost faces and cell windows depend on the type): 3D
// rows (0, 0), then (0, r > 0), (q > 0, 0), (q > 0, r > 0); 2D rows q = 0, then q > 0.
// Within a type, owner-major.
__host__ __device__ constexpr int gather_owners_per_cta(int dim, int k) {
  return (dim == 3 ? k * k : k) >= GATHER_THREADS ? 1 : GATHER_THREADS / (dim == 3 ? k * k : k);
}
inline int64_t gather_ctas(int dim, int k, int64_t ncown) {
  const int opc = gather_owners_per_cta(dim, k);
  return (ncown + opc - 1) / opc;
}

template <int D, int K>
__host__ __device__ __forceinline__ bool gather_slot(const int u, int& o, int& q, int& r) {
  constexpr int OPC = gather_owners_per_cta(D, K);
  constexpr int C1 = K - 1;                 // rows per owner with exactly one of q, r zero (each)
  if (u >= OPC * CellShape<D, K>::KR) return false;
  if (u < OPC) {
    o = u;
    q = r = 0;
    return true;
  }
  if constexpr (K == 1) {
    return false;
  } else if constexpr (D == 2) {
    const int v = u - OPC;
    o = v / C1;
    q = 1 + (v - o * C1);
    r = 0;
  } else {
    int v = u - OPC;
    if (v < OPC * C1) {
      o = v / C1;
      q = 0;
      r = 1 + (v - o * C1);
      return true;
    }
    v -= OPC * C1;
    if (v < OPC * C1) {
      o = v / C1;
      q = 1 + (v - o * C1);
      r = 0;
      return true;
    }
    v -= OPC * C1;
    o = v / (C1 * C1);
    const int j = v - o * C1 * C1;
    q = 1 + j % C1;
    r = 1 + j / C1;
  }
  return true;
}

template <int D, int K, class A>
__global__ void __launch_bounds__(GATHER_THREADS)
cell_gather(const typename A::V* __restrict__ wc, typename A::IO* __restrict__ y, const int add, const CellTabs ct) {
  using S = CellShape<D, K>;
  constexpr int KR = S::KR;
  int o = 0, q = 0, r = 0;
  const bool slot = gather_slot<D, K>((int)threadIdx.x, o, q, r);
  const int own = (int)blockIdx.x * gather_owners_per_cta(D, K) + o;
  const bool live = slot && own < ct.ncown;
  const int t = q + K * r;
  const int base = live ? __ldg(ct.corow + (size_t)own * KR + t) : -1;
  asm volatile("griddepcontrol.wait;" ::: "memory");   // cell outputs and y are complete
  IoDot<typename A::IO> dot;
  if (base >= 0) gather_row<D, K, A>(wc, y, add, ct, own, t, base, dot);
  if (ct.dotpart) {
    // the CTA's partial sum in a fixed order: a shuffle tree per warp, then the warps in
    // order, in the accumulator's own arithmetic (no FP64 work for FP32 vectors)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot.merge(dot.shfl_down(o));
    __shared__ IoDot<typename A::IO> wsum[GATHER_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = dot;
    __syncthreads();
    if (threadIdx.x == 0) {
      IoDot<typename A::IO> tot = wsum[0];
      for (int w = 1; w < GATHER_THREADS / 32; ++w) tot.merge(wsum[w]);
      ct.dotpart[blockIdx.x] = tot.value();
    }
  }
}

// CTAs of the gather (the number of fused inner-product partials)
template <int D, int K>
inline int gather_blocks(const CellTabs& ct) {
  return (int)gather_ctas(D, K, ct.ncown);
}

// y (+)= (wm M_active + ws K_active) x: the cell kernel, then the gather (add = 1: onto y).
template <int D, int K, class A>
cudaError_t run_cells(const void* x, void* y, const CellTabs& ct, const double* m, const double* s, double h,
                      double wm, double ws, int add, int first, cudaStream_t st) {
  using S = CellShape<D, K>;
  using V = typename A::V;
  using IO = typename A::IO;
  using C = CellConsts<V, K>;
  constexpr int N = C::N, H = C::H, NE = C::NE;
  C c;
  // even / odd halves of the centrosymmetric reference matrices (see CellConsts)
  for (int p = 0; p < NE; ++p)
    for (int i = 0; i < NE; ++i) {
      const bool mid = 2 * i == N - 1;
      c.me[p][i] = from_host<V>(mid ? m[p * N + i] : 0.5 * (m[p * N + i] + m[p * N + N - 1 - i]));
      c.se[p][i] = from_host<V>(mid ? s[p * N + i] : 0.5 * (s[p * N + i] + s[p * N + N - 1 - i]));
    }
  for (int p = 0; p < H; ++p)
    for (int i = 0; i < H; ++i) {
      c.mo[p][i] = from_host<V>(0.5 * (m[p * N + i] - m[p * N + N - 1 - i]));
      c.so[p][i] = from_host<V>(0.5 * (s[p * N + i] - s[p * N + N - 1 - i]));
    }
  c.hm = from_host<V>(wm * (D == 3 ? h * h * h : h * h));
  c.hs = from_host<V>(ws * (D == 3 ? h : 1.0));
  if (ct.ncact <= 0) return cudaSuccess;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((ct.ncact + S::CB - 1) / S::CB));
  cfg.blockDim = dim3((unsigned)S::NT);
  cfg.stream = st;
  cfg.attrs = attr;
  // the cell kernel loads x before its dependency wait: as the first kernel of a call it runs
  // only after everything earlier on the stream has completed
  cfg.numAttrs = first ? 0 : 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, cell_kernel<D, K, A>, (const IO*)x, (V*)ct.wc, ct.crow, ct.ncact, c);
  if (e != cudaSuccess) return e;
  cfg.numAttrs = 1;
  const int64_t rows = (int64_t)ct.ncown * S::KR;
  if (rows > 0) {
    cfg.gridDim = dim3((unsigned)gather_blocks<D, K>(ct));
    cfg.blockDim = dim3((unsigned)GATHER_THREADS);
    e = cudaLaunchKernelEx(&cfg, cell_gather<D, K, A>, (const V*)ct.wc, (IO*)y, add, ct);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace gp
