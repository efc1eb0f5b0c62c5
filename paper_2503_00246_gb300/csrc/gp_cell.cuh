// Mass + Laplace stiffness of the active cells, y += (M_active + K_active) x, for
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
// and z passes go through shared memory in place.  Cells of one parity colour share
// no node, so the launch for a colour adds its cells' results with plain
// read-modify-writes; the colours run in a fixed order (bitwise reproducible).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gp_arith.cuh"

namespace gp {

template <int D, int K>
struct CellShape {
  static constexpr int K1 = K + 1;
  static constexpr int R = (D == 3) ? K1 * K1 : K1;        // x-lines per cell
  static constexpr int NODES = R * K1;                      // nodes per cell
  static constexpr int CB = (256 / R) > 0 ? 256 / R : 1;   // cells per CTA
  static constexpr int NT = CB * R;
};

template <typename V, int K>
struct CellConsts {
  V m[K + 1][K + 1];  // reference mass
  V s[K + 1][K + 1];  // reference stiffness
  V hm;               // h^d
  V hs;               // h^(d-2)
};

struct CellArgs {
  const int32_t* crow;  // [ncell][R] compact index of each x-line start
  int32_t c0, c1;       // cells [c0, c1) of one colour
};

template <int D, int K, class A>
__global__ void __launch_bounds__(CellShape<D, K>::NT)
cell_kernel(const typename A::IO* __restrict__ x, typename A::IO* __restrict__ y, const CellArgs ca,
            const __grid_constant__ CellConsts<typename A::V, K> c) {
  using S = CellShape<D, K>;
  using V = typename A::V;
  using IO = typename A::IO;
  constexpr int K1 = S::K1, R = S::R, NODES = S::NODES, CB = S::CB;
  __shared__ V sa[CB][NODES];
  __shared__ V sb[CB][NODES];
  const int t = threadIdx.x;
  const int cl = t / R, line = t - cl * R;
  const int cell = ca.c0 + blockIdx.x * CB + cl;
  const bool valid = cell < ca.c1;
  const int32_t row = valid ? __ldg(ca.crow + (size_t)cell * R + line) : 0;

  // ---- x pass: a = M^ x, b = S^ x on this thread's x-line
  V xl[K1];
#pragma unroll
  for (int i = 0; i < K1; ++i) xl[i] = valid ? from_io(__ldg(x + row + i), (V*)nullptr) : vzero<V>();
#pragma unroll
  for (int p = 0; p < K1; ++p) {
    V a = vzero<V>(), b = vzero<V>();
#pragma unroll
    for (int q = 0; q < K1; ++q) {
      a = vfma(c.m[p][q], xl[q], a);
      b = vfma(c.s[p][q], xl[q], b);
    }
    sa[cl][p + K1 * line] = a;
    sb[cl][p + K1 * line] = b;
  }
  __syncthreads();

  if constexpr (D == 3) {
    // ---- y pass on the line (i1, i3): f = h^3 M^ a + h (S^ a + M^ b), g = h M^ a
    {
      const int i1 = line % K1, i3 = line / K1;
      V ay[K1], by[K1];
#pragma unroll
      for (int q = 0; q < K1; ++q) {
        ay[q] = sa[cl][i1 + K1 * (q + K1 * i3)];
        by[q] = sb[cl][i1 + K1 * (q + K1 * i3)];
      }
#pragma unroll
      for (int p = 0; p < K1; ++p) {
        V cc = vzero<V>(), dd = vzero<V>(), ee = vzero<V>();
#pragma unroll
        for (int q = 0; q < K1; ++q) {
          cc = vfma(c.m[p][q], ay[q], cc);
          dd = vfma(c.s[p][q], ay[q], dd);
          ee = vfma(c.m[p][q], by[q], ee);
        }
        sa[cl][i1 + K1 * (p + K1 * i3)] = vfma(c.hm, cc, vfma(c.hs, vadd(dd, ee), vzero<V>()));
        sb[cl][i1 + K1 * (p + K1 * i3)] = vfma(c.hs, cc, vzero<V>());
      }
    }
    __syncthreads();
    // ---- z pass on the line (i1, i2): y = M^ f + S^ g
    {
      const int i1 = line % K1, i2 = line / K1;
      V fz[K1], gz[K1];
#pragma unroll
      for (int q = 0; q < K1; ++q) {
        fz[q] = sa[cl][i1 + K1 * (i2 + K1 * q)];
        gz[q] = sb[cl][i1 + K1 * (i2 + K1 * q)];
      }
#pragma unroll
      for (int p = 0; p < K1; ++p) {
        V yv = vzero<V>();
#pragma unroll
        for (int q = 0; q < K1; ++q) yv = vfma(c.s[p][q], gz[q], vfma(c.m[p][q], fz[q], yv));
        sa[cl][i1 + K1 * (i2 + K1 * p)] = yv;
      }
    }
    __syncthreads();
  } else {
    // ---- y pass on the line i1: y = M^ (h^2 a + b) + S^ a
    V ay[K1], by[K1];
#pragma unroll
    for (int q = 0; q < K1; ++q) {
      ay[q] = sa[cl][line + K1 * q];
      by[q] = sb[cl][line + K1 * q];
    }
#pragma unroll
    for (int p = 0; p < K1; ++p) {
      V yv = vzero<V>();
#pragma unroll
      for (int q = 0; q < K1; ++q) {
        const V f = vfma(c.hm, ay[q], vfma(c.hs, by[q], vzero<V>()));
        yv = vfma(c.m[p][q], f, yv);
        yv = vfma(c.s[p][q], vfma(c.hs, ay[q], vzero<V>()), yv);
      }
      sa[cl][line + K1 * p] = yv;
    }
    __syncthreads();
  }

  // ---- add the cell's result on this thread's x-line
  if (valid) {
#pragma unroll
    for (int i = 0; i < K1; ++i) {
      const int idx = row + i;
      y[idx] = to_io(vadd(from_io(y[idx], (V*)nullptr), sa[cl][i + K1 * line]), (IO*)nullptr);
    }
  }
}

// Launches the parity colours in order; y += (wm M_active + ws K_active) x.
template <int D, int K, class A>
cudaError_t run_cells(const void* x, void* y, const int32_t* crow, const int32_t* cstart, const double* m,
                      const double* s, double h, double wm, double ws, cudaStream_t st) {
  using S = CellShape<D, K>;
  using V = typename A::V;
  using IO = typename A::IO;
  CellConsts<V, K> c;
  for (int p = 0; p < K + 1; ++p)
    for (int q = 0; q < K + 1; ++q) {
      c.m[p][q] = from_host<V>(m[p * (K + 1) + q]);
      c.s[p][q] = from_host<V>(s[p * (K + 1) + q]);
    }
  c.hm = from_host<V>(wm * (D == 3 ? h * h * h : h * h));
  c.hs = from_host<V>(ws * (D == 3 ? h : 1.0));
  const int ncol = D == 3 ? 8 : 4;
  for (int col = 0; col < ncol; ++col) {
    CellArgs ca;
    ca.crow = crow;
    ca.c0 = cstart[col];
    ca.c1 = cstart[col + 1];
    const int ncell = ca.c1 - ca.c0;
    if (ncell <= 0) continue;
    cell_kernel<D, K, A><<<(ncell + S::CB - 1) / S::CB, S::NT, 0, st>>>((const IO*)x, (IO*)y, ca, c);
  }
  return cudaGetLastError();
}

}  // namespace gp
