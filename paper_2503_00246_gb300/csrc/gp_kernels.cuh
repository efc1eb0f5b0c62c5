// Face kernels of the ghost-penalty operator y = G x on sm_103a.
//
// Per face F with normal axis a (Sec. 2.4), G_F = h^{d-2} (M^ x ... x G^) with
// G^ = sum_j c_j g_j g_j^T of rank k.  The apply is split as G = J^T W J:
//
//   jump kernel (J, then W):  t_F[j, tau] = g_j . x_F(:, tau)            normal lines
//                             T_F[tau, j] = s_j (M^ x M^) t_F[j, .]      tangential mass
//   lift kernel (J^T):        y_I = sum_{F contains I} sum_j g_j[b_F(I)] T_F[tau_F(I), j]
//
// which reorders the three-step face apply of Sec. 2.5.1 (normal G, then the
// two tangential masses) so the normal contraction acts through the k jump
// vectors on both sides of the tangential step.  The lift is a gather: every
// active DoF is written by exactly one thread, which sums the contributions of
// the faces that contain it in a fixed order.  No atomics, bitwise
// reproducible, and the zero fill of y for the overwrite form rides along.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gp {

template <int D, int K>
struct Shape {
  static constexpr int L = (D == 2) ? (K + 1) : (K + 1) * (K + 1);  // tangential nodes per face
  static constexpr int NN = 2 * K + 1;                               // nodes on a normal line
  static constexpr int FB = (256 / L) > 0 ? (256 / L) : 1;           // faces per CTA
  static constexpr int NT = FB * L;                                  // threads per CTA
};

// Kernel constants (passed by value; they sit in the constant bank).
template <typename T, int K>
struct Consts {
  T g[K][2 * K + 1];  // jump of the j-th derivative of patch basis b (row j-1)
  T m[K + 1][K + 1];  // reference mass matrix
  T s[K];             // c_j h^{d-2}
};

struct FaceArgs {
  const int32_t* rowtab;  // [ninv][L] compact index of each x-row start of a cell
  const int32_t* fcell;   // [nf][2] involved-cell index of K-, K+
  int32_t fstart[4];      // first face of each axis; fstart[D] = nf
  int32_t bstart[4];      // first CTA of each axis; bstart[D] = grid size
};

struct LiftArgs {
  const int4* segs;       // (c0, X0, row, len | touched << 16)
  const int2* tiles;      // (first segment, count), <= 256 nodes each
  const int32_t* face_of; // [D][ncell] face id or -1
  int32_t n;              // cells per axis
  int32_t nl;             // lattice nodes per axis
  int64_t ncell;
};

// ----------------------------------------------------------------- jump --
template <int D, int K, typename T>
__global__ void __launch_bounds__(Shape<D, K>::NT)
jump_kernel(const T* __restrict__ x, T* __restrict__ tp, const FaceArgs fa,
            const __grid_constant__ Consts<T, K> c) {
  using S = Shape<D, K>;
  constexpr int L = S::L, FB = S::FB, NN = S::NN, K1 = K + 1;
  __shared__ T buf[FB][K][L];

  // axis of this CTA's faces (constant indices only: no local-memory copy of fa)
  const int blk = blockIdx.x;
  int axis = 0, fbase = fa.fstart[0], fend = fa.fstart[1], bbase = fa.bstart[0];
  if (D >= 2 && blk >= fa.bstart[1]) { axis = 1; fbase = fa.fstart[1]; fend = fa.fstart[2]; bbase = fa.bstart[1]; }
  if (D >= 3 && blk >= fa.bstart[2]) { axis = 2; fbase = fa.fstart[2]; fend = fa.fstart[3]; bbase = fa.bstart[2]; }
  const int f0 = fbase + (blk - bbase) * FB;
  const int t = threadIdx.x;
  const int fl = t / L, tau = t - fl * L;
  const int f = f0 + fl;

  // ---- normal lines: gather 2k+1 values, contract with the k jump vectors
  if (f < fend) {
    const int lo = __ldg(fa.fcell + 2 * f), hi = __ldg(fa.fcell + 2 * f + 1);
    const int32_t* rlo = fa.rowtab + (size_t)lo * L;
    const int32_t* rhi = fa.rowtab + (size_t)hi * L;
    T v[NN];
    if (axis == 0) {
      const int32_t base = __ldg(rlo + tau);
#pragma unroll
      for (int b = 0; b < NN; ++b) v[b] = __ldg(x + base + b);
    } else {
      // tau = tx + (K+1) tr; the normal index b selects the row of K- (b <= k) or K+ (b > k)
      const int tx = (D == 3) ? tau % K1 : tau;
      const int tr = (D == 3) ? tau / K1 : 0;
      const int rstride = (D == 3 && axis == 2) ? K1 : 1;
      const int roff = (D == 3) ? ((axis == 1) ? K1 * tr : tr) : 0;
#pragma unroll
      for (int b = 0; b < NN; ++b) {
        const int32_t* rt = (b <= K) ? rlo : rhi;
        const int bc = (b <= K) ? b : b - K;
        v[b] = __ldg(x + __ldg(rt + roff + rstride * bc) + tx);
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
      T acc = T(0);
#pragma unroll
      for (int b = 0; b < NN; ++b) acc = fma(c.g[j][b], v[b], acc);
      buf[fl][j][tau] = acc;
    }
  }
  __syncthreads();

  // ---- tangential reference masses, one 1D line per thread
  if constexpr (D == 3) {
    constexpr int NL = FB * K * K1;
    // along the first tangential index: lines (fl, j, t2)
    for (int ln = t; ln < NL; ln += S::NT) {
      const int ff = ln / (K * K1), rem = ln - ff * (K * K1);
      const int j = rem / K1, t2 = rem - j * K1;
      T u[K1];
#pragma unroll
      for (int q = 0; q < K1; ++q) u[q] = buf[ff][j][q + K1 * t2];
#pragma unroll
      for (int p = 0; p < K1; ++p) {
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < K1; ++q) acc = fma(c.m[p][q], u[q], acc);
        buf[ff][j][p + K1 * t2] = acc;
      }
    }
    __syncthreads();
    // along the second tangential index: lines (fl, j, t1)
    for (int ln = t; ln < NL; ln += S::NT) {
      const int ff = ln / (K * K1), rem = ln - ff * (K * K1);
      const int j = rem / K1, t1 = rem - j * K1;
      T u[K1];
#pragma unroll
      for (int q = 0; q < K1; ++q) u[q] = buf[ff][j][t1 + K1 * q];
#pragma unroll
      for (int p = 0; p < K1; ++p) {
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < K1; ++q) acc = fma(c.m[p][q], u[q], acc);
        buf[ff][j][t1 + K1 * p] = acc;
      }
    }
    __syncthreads();
  } else {
    constexpr int NL = FB * K;
    for (int ln = t; ln < NL; ln += S::NT) {
      const int ff = ln / K, j = ln - ff * K;
      T u[K1];
#pragma unroll
      for (int q = 0; q < K1; ++q) u[q] = buf[ff][j][q];
#pragma unroll
      for (int p = 0; p < K1; ++p) {
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < K1; ++q) acc = fma(c.m[p][q], u[q], acc);
        buf[ff][j][p] = acc;
      }
    }
    __syncthreads();
  }

  // ---- scaled jumps T_F[tau][j], k contiguous values per thread
  if (f < fend) {
    T* out = tp + ((size_t)f * L + tau) * K;
#pragma unroll
    for (int j = 0; j < K; ++j) out[j] = c.s[j] * buf[fl][j][tau];
  }
}

// ----------------------------------------------------------------- lift --
template <int D, int K, typename T>
__global__ void __launch_bounds__(256)
lift_kernel(const T* __restrict__ tp, T* __restrict__ y, const int add, const LiftArgs la,
            const __grid_constant__ Consts<T, K> c) {
  constexpr int L = Shape<D, K>::L, K1 = K + 1;
  __shared__ int4 sseg[256];
  __shared__ int spre[257];
  const int2 tile = la.tiles[blockIdx.x];
  const int ns = tile.y;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) sseg[i] = la.segs[tile.x + i];
  __syncthreads();
  if (threadIdx.x < 32) {
    // exclusive prefix of segment lengths (one warp, ns <= 256)
    int carry = 0;
    for (int base = 0; base < ns; base += 32) {
      const int i = base + threadIdx.x;
      int v = (i < ns) ? (sseg[i].w & 0xffff) : 0;
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)threadIdx.x >= o) incl += u;
      }
      if (i < ns) spre[i] = carry + incl - v;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (threadIdx.x == 0) spre[ns] = carry;
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t >= spre[ns]) return;
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (spre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const int4 s = sseg[lo];
  const int o = t - spre[lo];
  const int ci = s.x + o;
  if (((s.w >> 16) & 1) == 0) {  // DoF outside every face patch
    y[ci] = T(0);
    return;
  }
  int P[3];
  P[0] = s.y + o;
  if (D == 3) {
    P[1] = s.z % la.nl;
    P[2] = s.z / la.nl;
  } else {
    P[1] = s.z;
    P[2] = 0;
  }
  const int n = la.n;
  T acc = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int t1 = (a == 0) ? 1 : 0;
    const int t2 = (a == 2) ? 1 : 2;
    // faces with normal a whose patch holds this node: lower cell ia with
    // ia*k <= P[a] <= ia*k + 2k, tangential cells it with it*k <= P[t] <= it*k + k
    const int ca = P[a] / K, pa = P[a] - ca * K;
    const int ia0 = (pa == 0) ? ca - 2 : ca - 1;
    const int c1 = P[t1] / K, p1 = P[t1] - c1 * K;
    const int j10 = (p1 == 0) ? c1 - 1 : c1;
    int j20 = 0, j21 = 0, c2 = 0;
    if (D == 3) {
      c2 = P[t2] / K;
      const int p2 = P[t2] - c2 * K;
      j20 = (p2 == 0) ? c2 - 1 : c2;
      j21 = c2;
    }
    for (int ia = ia0; ia <= ca; ++ia) {
      if (ia < 0 || ia > n - 2) continue;
      const int b = P[a] - ia * K;
      for (int i1 = j10; i1 <= c1; ++i1) {
        if (i1 < 0 || i1 > n - 1) continue;
        const int tau1 = P[t1] - i1 * K;
        for (int i2 = j20; i2 <= j21; ++i2) {
          if (D == 3 && (i2 < 0 || i2 > n - 1)) continue;
          const int tau2 = (D == 3) ? P[t2] - i2 * K : 0;
          int cc[3];
          cc[a] = ia;
          cc[t1] = i1;
          if (D == 3) cc[t2] = i2;
          int64_t lin = cc[0] + (int64_t)n * cc[1];
          if (D == 3) lin += (int64_t)n * n * cc[2];
          const int f = __ldg(la.face_of + a * la.ncell + lin);
          if (f < 0) continue;
          const T* src = tp + ((size_t)f * L + tau1 + K1 * tau2) * K;
#pragma unroll
          for (int j = 0; j < K; ++j) acc = fma(c.g[j][b], __ldg(src + j), acc);
        }
      }
    }
  }
  y[ci] = add ? y[ci] + acc : acc;
}

}  // namespace gp
