// Host plan of the ghost-penalty operator (built once per mesh, degree, level set).
//
//  * cell classification from the level set phi (> 0 inside), Sec. 2;
//  * ghost faces: interior faces between two active cells with at least one
//    cut cell (Sec. 2.2 and the figure of intersected cells);
//  * active DoFs: FE_Q lattice nodes of active cells, lexicographic with x
//    fastest (Sec. 2.4, i = i1 + i2 N1 + i3 N1 N2), compacted;
//  * 1D reference matrices in FP64 (Sec. 2.4, M^1 and G^1_k with their h
//    scaling), computed here with a collocation differentiation matrix;
//  * tables for the kernels: per involved cell the compact index of each of
//    its x-rows, per face its two cells, per (axis, cell) the face id, and
//    the lift owner cells and the zero runs of the active DoFs.
//
// Compile with -ffp-contract=off: the classification must round exactly as
// written so that every implementation of the same rule agrees cell by cell.
#include "gp_plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

namespace gp {

// ---------------------------------------------------------------- 1D data --

// All 1D quantities are computed in long double (80-bit on x86-64, binary128 on
// aarch64) and rounded once to double: powers of the differentiation matrix
// lose about 1e-12 of relative accuracy at k = 8 in plain double.
using R = long double;

// Legendre P_n and P_n' at t in (-1, 1) by the three-term recurrence.
static void legendre(int n, R t, R& p, R& dp) {
  R p0 = 1, p1 = t;
  if (n == 0) { p = 1; dp = 0; return; }
  for (int m = 2; m <= n; ++m) {
    R p2 = ((2 * m - 1) * t * p1 - (m - 1) * p0) / m;
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  dp = n * (t * p1 - p0) / (t * t - 1);  // P_n' = n (t P_n - P_{n-1}) / (t^2 - 1)
}

static void gauss_lobatto_01_r(int k, std::vector<R>& x) {
  x.assign(k + 1, R(0));
  x[k] = 1;
  const R pi = 3.141592653589793238462643383279502884L;
  for (int i = 1; i < k; ++i) {
    // interior points: roots of P_k', Newton from the Chebyshev-Lobatto guess;
    // P_k'' from the Legendre equation (1-t^2) P'' = 2 t P' - k(k+1) P
    R t = -std::cos(pi * i / k);
    for (int it = 0; it < 200; ++it) {
      R p, dp;
      legendre(k, t, p, dp);
      R d2p = (2 * t * dp - R(k) * (k + 1) * p) / (1 - t * t);
      R dt = dp / d2p;
      t -= dt;
      if (std::fabs(dt) <= 4 * std::numeric_limits<R>::epsilon() * std::fabs(t)) break;
    }
    x[i] = (t + 1) / 2;
  }
}

void gauss_lobatto_01(int k, std::vector<double>& x) {
  std::vector<R> xr;
  gauss_lobatto_01_r(k, xr);
  x.assign(xr.begin(), xr.end());
}

static void gauss_legendre_01(int nq, std::vector<R>& x, std::vector<R>& w) {
  x.assign(nq, R(0));
  w.assign(nq, R(0));
  const R pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < nq; ++i) {
    R t = -std::cos(pi * (i + R(0.75)) / (nq + R(0.5)));
    R p = 0, dp = 1;
    for (int it = 0; it < 200; ++it) {
      legendre(nq, t, p, dp);
      R dt = p / dp;
      t -= dt;
      if (std::fabs(dt) <= 4 * std::numeric_limits<R>::epsilon()) break;
    }
    legendre(nq, t, p, dp);
    x[i] = (t + 1) / 2;
    w[i] = 1 / ((1 - t * t) * dp * dp);  // 2/((1-t^2)P'^2) scaled to [0,1]
  }
}

// M^[a][b] = int_0^1 l_a l_b (Gauss rule with k+1 points, exact for degree 2k),
// g_j[b] = jump of d^j/dx^j of patch basis b at the face of [0,1] u [1,2]:
//   b <= k: l_b on K- (evaluated at x = 1), b >= k: l_{b-k} on K+ (at x = 0 of K+).
// Derivatives come from powers of the collocation differentiation matrix
// D[i][m] = l_m'(x_i) (barycentric form), so (D^j)[i][m] = l_m^(j)(x_i).
void reference_1d(int k, const std::vector<double>& /*gl*/, std::vector<double>& mass,
                  std::vector<double>& jumps) {
  const int N = k + 1;
  std::vector<R> gl;
  gauss_lobatto_01_r(k, gl);
  std::vector<R> bw(N, R(1));
  for (int i = 0; i < N; ++i)
    for (int m = 0; m < N; ++m)
      if (m != i) bw[i] /= (gl[i] - gl[m]);
  std::vector<R> D(N * N, R(0));
  for (int i = 0; i < N; ++i) {
    R diag = 0;
    for (int m = 0; m < N; ++m) {
      if (m == i) continue;
      R v = (bw[m] / bw[i]) / (gl[i] - gl[m]);
      D[i * N + m] = v;
      diag -= v;
    }
    D[i * N + i] = diag;
  }
  jumps.assign(k * (2 * k + 1), 0.0);
  std::vector<R> Dj(D), tmp(N * N);
  for (int j = 1; j <= k; ++j) {
    for (int b = 0; b <= 2 * k; ++b) {
      R v = 0;
      if (b <= k) v += Dj[k * N + b];        // l_b^(j) at the right end of K-
      if (b >= k) v -= Dj[0 * N + (b - k)];  // l_{b-k}^(j) at the left end of K+
      jumps[(j - 1) * (2 * k + 1) + b] = (double)v;
    }
    for (int i = 0; i < N; ++i)
      for (int m = 0; m < N; ++m) {
        R s = 0;
        for (int q = 0; q < N; ++q) s += Dj[i * N + q] * D[q * N + m];
        tmp[i * N + m] = s;
      }
    Dj.swap(tmp);
  }
  std::vector<R> xq, wq;
  gauss_legendre_01(N, xq, wq);
  std::vector<R> V(N * N);  // V[q][m] = l_m(x_q), product form
  for (int q = 0; q < N; ++q)
    for (int m = 0; m < N; ++m) {
      R v = 1;
      for (int i = 0; i < N; ++i)
        if (i != m) v *= (xq[q] - gl[i]) / (gl[m] - gl[i]);
      V[q * N + m] = v;
    }
  mass.assign(N * N, 0.0);
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      R s = 0;
      for (int q = 0; q < N; ++q) s += wq[q] * V[q * N + a] * V[q * N + b];
      mass[a * N + b] = (double)s;
    }
}

// Macro-patch stabilisation (the alternative named in Sec. 2.2): on the two-cell patch
// [0,1] u [1,2] of a face, the difference between the polynomial on one cell and the
// extension of the neighbour's polynomial into it, squared and integrated over both cells:
//   G^mp = sum_q w_q (d_q d_q^T + e_q e_q^T),
//   d_q[b] = [b >= k] l_{b-k}(t_q) - [b <= k] l_b(1 + t_q)       (K+, the K- polynomial extended),
//   e_q[b] = [b <= k] l_b(t_q) - [b >= k] l_{b-k}(t_q - 1)       (K-, the K+ polynomial extended),
// with the k+1 Gauss points t_q of [0,1] (exact: the integrands have degree 2k).  G^mp is
// mirror symmetric and vanishes exactly on the patch interpolants of global polynomials of
// degree <= k, the null space of the ghost-penalty matrix, so it has rank k and the same range:
// G^mp = sum_j lambda_j v_j v_j^T with eigenvectors of alternating parity, odd orders (j = 1,
// 3, ...) mirror symmetric and even orders antisymmetric, like the jump vectors g_j.  The face
// kernels then apply it unchanged with v_j in place of g_j and lambda_j in place of c_j.
// Eigenvectors by cyclic Jacobi rotations in long double.
static R lagrange_at(const std::vector<R>& gl, int m, R x) {
  R v = 1;
  for (size_t i = 0; i < gl.size(); ++i)
    if ((int)i != m) v *= (x - gl[i]) / (gl[m] - gl[i]);
  return v;
}

bool macro_patch_1d(int k, std::vector<double>& vecs, std::vector<double>& lambda) {
  const int N = k + 1, NN = 2 * k + 1;
  std::vector<R> gl, tq, wq;
  gauss_lobatto_01_r(k, gl);
  gauss_legendre_01(N, tq, wq);
  std::vector<R> A(NN * NN, R(0)), d(NN), e(NN);
  for (int q = 0; q < N; ++q) {
    for (int b = 0; b < NN; ++b) {
      d[b] = (b >= k ? lagrange_at(gl, b - k, tq[q]) : R(0)) - (b <= k ? lagrange_at(gl, b, 1 + tq[q]) : R(0));
      e[b] = (b <= k ? lagrange_at(gl, b, tq[q]) : R(0)) - (b >= k ? lagrange_at(gl, b - k, tq[q] - 1) : R(0));
    }
    for (int a = 0; a < NN; ++a)
      for (int b = 0; b < NN; ++b) A[a * NN + b] += wq[q] * (d[a] * d[b] + e[a] * e[b]);
  }
  // cyclic Jacobi: A = V diag(ev) V^T
  std::vector<R> V(NN * NN, R(0));
  for (int i = 0; i < NN; ++i) V[i * NN + i] = 1;
  for (int sweep = 0; sweep < 100; ++sweep) {
    R off = 0, tot = 0;
    for (int a = 0; a < NN; ++a)
      for (int b = 0; b < NN; ++b) {
        tot += A[a * NN + b] * A[a * NN + b];
        if (a != b) off += A[a * NN + b] * A[a * NN + b];
      }
    if (off <= tot * R(1e-36)) break;
    for (int p = 0; p < NN; ++p)
      for (int q = p + 1; q < NN; ++q) {
        const R apq = A[p * NN + q];
        if (apq == 0) continue;
        const R theta = (A[q * NN + q] - A[p * NN + p]) / (2 * apq);
        const R t = (theta >= 0 ? 1 : -1) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
        const R c = 1 / std::sqrt(t * t + 1), sn = t * c;
        for (int r = 0; r < NN; ++r) {          // A <- J^T A J, V <- V J
          const R arp = A[r * NN + p], arq = A[r * NN + q];
          A[r * NN + p] = c * arp - sn * arq;
          A[r * NN + q] = sn * arp + c * arq;
        }
        for (int r = 0; r < NN; ++r) {
          const R apr = A[p * NN + r], aqr = A[q * NN + r];
          A[p * NN + r] = c * apr - sn * aqr;
          A[q * NN + r] = sn * apr + c * aqr;
        }
        for (int r = 0; r < NN; ++r) {
          const R vrp = V[r * NN + p], vrq = V[r * NN + q];
          V[r * NN + p] = c * vrp - sn * vrq;
          V[r * NN + q] = sn * vrp + c * vrq;
        }
      }
  }
  // the k largest eigenvalues; parity of each eigenvector
  std::vector<int> order(NN);
  for (int i = 0; i < NN; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return A[a * NN + a] > A[b * NN + b]; });
  R top = A[order[0] * NN + order[0]];
  std::vector<int> sym, anti;
  for (int r = 0; r < k; ++r) {
    const int c = order[r];
    R ds = 0, da = 0;
    for (int b = 0; b < NN; ++b) {
      ds += std::fabs(V[b * NN + c] - V[(NN - 1 - b) * NN + c]);
      da += std::fabs(V[b * NN + c] + V[(NN - 1 - b) * NN + c]);
    }
    (ds < da ? sym : anti).push_back(c);
  }
  // a rank-k matrix: the (k+1)-th eigenvalue is rounding noise
  if (k < NN && A[order[k] * NN + order[k]] > top * R(1e-12)) return false;
  if ((int)sym.size() != (k + 1) / 2 || (int)anti.size() != k / 2) return false;
  vecs.assign((size_t)k * NN, 0.0);
  lambda.assign(k, 0.0);
  for (int j = 0; j < k; ++j) {
    const int c = (j % 2 == 0) ? sym[j / 2] : anti[j / 2];
    lambda[j] = (double)A[c * NN + c];
    for (int b = 0; b < NN; ++b) {
      // exact mirror symmetry, so that the kernels' even-odd split is exact
      const R v = V[b * NN + c], w = V[(NN - 1 - b) * NN + c];
      vecs[(size_t)j * NN + b] = (double)((j % 2 == 0) ? (v + w) / 2 : (v - w) / 2);
    }
  }
  return true;
}

// S^[a][b] = int_0^1 l_a' l_b' with k+1 Gauss points (exact for degree 2k-2); the
// derivative of l_m is evaluated as sum_i 1/(x_m - x_i) prod_{l != m, i} (x - x_l)/(x_m - x_l),
// which stays finite when a Gauss point coincides with a node.
void reference_stiffness(int k, std::vector<double>& stiff) {
  const int N = k + 1;
  std::vector<R> gl, xq, wq;
  gauss_lobatto_01_r(k, gl);
  gauss_legendre_01(N, xq, wq);
  std::vector<R> Dv(N * N);  // Dv[q][m] = l_m'(x_q)
  for (int q = 0; q < N; ++q)
    for (int m = 0; m < N; ++m) {
      R sum = 0;
      for (int i = 0; i < N; ++i) {
        if (i == m) continue;
        R prod = 1 / (gl[m] - gl[i]);
        for (int l = 0; l < N; ++l)
          if (l != m && l != i) prod *= (xq[q] - gl[l]) / (gl[m] - gl[l]);
        sum += prod;
      }
      Dv[q * N + m] = sum;
    }
  stiff.assign(N * N, 0.0);
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      R s = 0;
      for (int q = 0; q < N; ++q) s += wq[q] * Dv[q * N + a] * Dv[q * N + b];
      stiff[a * N + b] = (double)s;
    }
}

void build_cell_table(Plan& p) {
  const int d = p.dim, n = p.n, k = p.k;
  const int R1 = d == 3 ? (k + 1) * (k + 1) : k + 1;
  const int n1 = n + 1;
  // active cells, lexicographic; x-line starts of each
  std::vector<int32_t> act_of(p.ncell, -1);
  p.ncact = 0;
  for (int64_t c = 0; c < p.ncell; ++c)
    if (p.cls[c] != OUTSIDE) act_of[c] = (int32_t)p.ncact++;
  p.crow.assign((size_t)p.ncact * R1, 0);
  for (int64_t c = 0; c < p.ncell; ++c) {
    const int32_t a = act_of[c];
    if (a < 0) continue;
    const int ci = (int)(c % n), cj = (int)((c / n) % n), cl = d == 3 ? (int)(c / ((int64_t)n * n)) : 0;
    for (int t = 0; t < R1; ++t) {
      const int q = t % (k + 1), r = t / (k + 1);
      const int64_t row = (int64_t)(cj * k + q) + (d == 3 ? (int64_t)p.nl * (cl * k + r) : 0);
      p.crow[(size_t)a * R1 + t] = (int32_t)p.compact(ci * k, row);
    }
  }
  // owner cells (coordinates in [0, n]) of the active nodes; their window of
  // the 2^d cells (ci - s_x, cj - s_y, cl - s_z), s in {0,1}^d, that hold their nodes
  std::vector<uint8_t> own((size_t)n1 * n1 * (d == 3 ? n1 : 1), 0);
  for (int64_t c = 0; c < p.ncell; ++c) {
    if (act_of[c] < 0) continue;
    const int ci = (int)(c % n), cj = (int)((c / n) % n), cl = d == 3 ? (int)(c / ((int64_t)n * n)) : 0;
    for (int dz = 0; dz <= (d == 3 ? 1 : 0); ++dz)
      for (int dy = 0; dy <= 1; ++dy)
        for (int dx = 0; dx <= 1; ++dx)
          own[(ci + dx) + (size_t)n1 * ((cj + dy) + (size_t)n1 * (cl + dz))] = 1;
  }
  const int NWC = d == 3 ? 8 : 4;
  const int KR = d == 3 ? k * k : k;
  p.cwin.clear();
  // order: the owners that some ghost face reaches first, in the lift's order (so that the
  // fused gather's warps do face work together), then the others, lexicographic
  std::vector<int64_t> owners;
  std::vector<uint8_t> taken(own.size(), 0);
  for (int64_t i = 0; i < p.num_lift_cells(); ++i) {
    const int32_t* c = &p.lcell[4 * i];
    const size_t o = c[0] + (size_t)n1 * (c[1] + (size_t)n1 * c[2]);
    if (o < own.size() && own[o] && !taken[o]) {
      owners.push_back((int64_t)o);
      taken[o] = 1;
    }
  }
  for (size_t o = 0; o < own.size(); ++o)
    if (own[o] && !taken[o]) owners.push_back((int64_t)o);
  p.ncown = (int64_t)owners.size();
  p.cown.assign(owners.begin(), owners.end());
  p.cwin.assign((size_t)p.ncown * NWC, -1);
  p.corow.assign((size_t)KR * p.ncown, -1);
  for (int64_t i = 0; i < p.ncown; ++i) {
    const int64_t o = owners[i];
    const int ci = (int)(o % n1), cj = (int)((o / n1) % n1), cl = d == 3 ? (int)(o / ((int64_t)n1 * n1)) : 0;
    for (int w = 0; w < NWC; ++w) {
      const int sx = w & 1, sy = (w >> 1) & 1, sz = (w >> 2) & 1;
      const int x = ci - sx, y = cj - sy, z = cl - sz;
      if (x < 0 || x >= n || y < 0 || y >= n || (d == 3 && (z < 0 || z >= n))) continue;
      p.cwin[(size_t)i * NWC + w] = act_of[x + (int64_t)n * (y + (int64_t)n * z)];
    }
    for (int t = 0; t < KR; ++t) {
      const int q = t % k, r = t / k;
      const int X = ci * k, Y = cj * k + q, Z = cl * k + r;
      int64_t cidx = -1;
      if (X < p.nl && Y < p.nl && (d == 2 || Z < p.nl)) {
        const int64_t row = (int64_t)Y + (d == 3 ? (int64_t)p.nl * Z : 0);
        cidx = p.compact(X, row);
      }
      p.corow[(size_t)i * KR + t] = (int32_t)cidx;
    }
  }
}

std::vector<int32_t> owner_lift_index(const Plan& cells, const Plan& faces) {
  const int n1 = cells.n + 1;
  std::vector<int32_t> at((size_t)n1 * n1 * (cells.dim == 3 ? n1 : 1), -1);
  const int64_t nl = faces.num_lift_cells();
  for (int64_t i = 0; i < nl; ++i) {
    const int32_t* c = &faces.lcell[4 * i];
    at[c[0] + (size_t)n1 * (c[1] + (size_t)n1 * c[2])] = (int32_t)i;
  }
  std::vector<int32_t> out(cells.cown.size());
  for (size_t i = 0; i < cells.cown.size(); ++i) out[i] = at[(size_t)cells.cown[i]];
  return out;
}

bool check_cell_table(const Plan& p) {
  const int64_t na = p.n_active, K1 = p.k + 1;
  for (int32_t r : p.crow)
    if (r < 0 || r + K1 > na) return false;
  for (int32_t c : p.cwin)
    if (c < -1 || c >= p.ncact) return false;
  for (int32_t r : p.corow)
    if (r < -1 || r >= na) return false;
  return true;
}

// Diagonal of the model system: per active cell h^d M_ii M_jj M_kk + h^(d-2) (S_ii M_jj M_kk +
// M_ii S_jj M_kk + M_ii M_jj S_kk) at local node (i, j, k); per ghost face
// sum_j s_j g_j[b]^2 times the tangential M^ diagonals at patch node (b, tau).
void build_diagonal(const Plan& p, std::vector<double>& diag) {
  const int d = p.dim, k = p.k, K1 = k + 1, NN = 2 * k + 1;
  const int R1 = d == 3 ? K1 * K1 : K1;
  diag.assign(p.n_active, 0.0);
  const double hm = d == 3 ? p.h * p.h * p.h : p.h * p.h, hs = d == 3 ? p.h : 1.0;
  auto M = [&](int a) { return p.mass[a * K1 + a]; };
  auto S = [&](int a) { return p.stiff[a * K1 + a]; };
  for (int64_t c = 0; c < p.ncact; ++c)
    for (int t = 0; t < R1; ++t) {
      const int j = t % K1, l = d == 3 ? t / K1 : 0;
      const int64_t base = p.crow[(size_t)c * R1 + t];
      for (int i = 0; i < K1; ++i) {
        double v;
        if (d == 3)
          v = hm * M(i) * M(j) * M(l) + hs * (S(i) * M(j) * M(l) + M(i) * S(j) * M(l) + M(i) * M(j) * S(l));
        else
          v = hm * M(i) * M(j) + hs * (S(i) * M(j) + M(i) * S(j));
        diag[base + i] += v;
      }
    }
  std::vector<double> gb(NN, 0.0);  // sum_j s_j g_j[b]^2
  for (int b = 0; b < NN; ++b)
    for (int j = 0; j < k; ++j) gb[b] += p.scale[j] * p.jumps[j * NN + b] * p.jumps[j * NN + b];
  const int L = p.L, R = d == 3 ? NN * K1 : NN;
  for (int a = 0; a < d; ++a)
    for (int64_t f = p.fstart[a]; f < p.fstart[a + 1]; ++f)
      for (int tau = 0; tau < L; ++tau) {
        const int t1 = d == 3 ? tau % K1 : tau, t2 = d == 3 ? tau / K1 : 0;
        const double mt = M(t1) * (d == 3 ? M(t2) : 1.0);
        for (int b = 0; b < NN; ++b) {
          int64_t idx;
          if (a == 0) idx = p.frows[p.rbase[0] + (f - p.fstart[0]) * L + tau] + b;
          else idx = p.frows[p.rbase[a] + (f - p.fstart[a]) * R + b + NN * t2] + t1;
          diag[idx] += gb[b] * mt;
        }
      }
}

// -------------------------------------------------------- classification --

static int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}

static void classify_balls(const Plan& p, const gp_levelset* ls, int n, std::vector<int8_t>& cls) {
  const int d = p.dim;
  const double h = p.h;
  int64_t nc = p.ncell;
  std::vector<uint8_t> any_in(nc, 0), all_out(nc, 1);
  for (int bidx = 0; bidx < ls->nballs; ++bidx) {
    const double* c = ls->centers + 3 * bidx;
    const double r = ls->radii[bidx];
    const double r2 = r * r;
    // per-axis squared near/far distances
    std::vector<double> n2[3], f2[3];
    for (int a = 0; a < d; ++a) {
      n2[a].resize(n);
      f2[a].resize(n);
      for (int i = 0; i < n; ++i) {
        double lo = p.lo[a] + i * h;
        double hi = p.lo[a] + (i + 1.0) * h;
        double near = std::max(std::max(lo - c[a], c[a] - hi), 0.0);
        double far = std::max(std::fabs(lo - c[a]), std::fabs(hi - c[a]));
        n2[a][i] = near * near;
        f2[a][i] = far * far;
      }
    }
    for (int64_t cell = 0; cell < nc; ++cell) {
      int ix = (int)(cell % n), iy = (int)((cell / n) % n), iz = (int)(cell / ((int64_t)n * n));
      double dmin2 = n2[0][ix] + n2[1][iy];
      double dmax2 = f2[0][ix] + f2[1][iy];
      if (d == 3) {
        dmin2 = dmin2 + n2[2][iz];
        dmax2 = dmax2 + f2[2][iz];
      }
      if (dmax2 < r2) any_in[cell] = 1;
      if (!(dmin2 >= r2)) all_out[cell] = 0;
    }
  }
  for (int64_t cell = 0; cell < nc; ++cell)
    cls[cell] = any_in[cell] ? INSIDE : (all_out[cell] ? OUTSIDE : CUT);
}

// Sampled classification with a Lipschitz margin: phi on an (m+1)^d lattice
// per cell; inside if min > margin, outside if max < -margin, else cut.
static bool classify_sampled(const Plan& p, const gp_levelset* ls, int n, double domain_hi0,
                             std::vector<int8_t>& cls) {
  const int d = p.dim;
  const int m = ls->samples > 0 ? ls->samples : 4;
  const double hs = (domain_hi0 - p.lo[0]) / ((double)n * m);
  const int ns = n * m + 1;
  double lip = ls->kind == GP_LS_GYROID ? std::sqrt(6.0) : ls->lipschitz;
  const double margin = lip * hs * std::sqrt((double)d) / 2.0;
  std::vector<double> co[3];
  for (int a = 0; a < d; ++a) {
    co[a].resize(ns);
    for (int s = 0; s < ns; ++s) co[a][s] = p.lo[a] + s * hs;
  }
  std::vector<double> sn[3], cs[3];
  if (ls->kind == GP_LS_GYROID) {
    for (int a = 0; a < 3; ++a) {
      sn[a].resize(ns);
      cs[a].resize(ns);
      for (int s = 0; s < ns; ++s) {
        sn[a][s] = std::sin(co[a][s]);
        cs[a][s] = std::cos(co[a][s]);
      }
    }
  }
  auto phi = [&](int sx, int sy, int sz) -> double {
    if (ls->kind == GP_LS_GYROID)
      return ((sn[0][sx] * cs[1][sy] + sn[1][sy] * cs[2][sz]) + sn[2][sz] * cs[0][sx]) - ls->iso;
    double pt[3] = {co[0][sx], co[1][sy], d == 3 ? co[2][sz] : 0.0};
    return ls->fn(pt, ls->user);
  };
  const int64_t nc = p.ncell;
  for (int64_t cell = 0; cell < nc; ++cell) {
    int ix = (int)(cell % n), iy = (int)((cell / n) % n), iz = d == 3 ? (int)(cell / ((int64_t)n * n)) : 0;
    double mn = std::numeric_limits<double>::infinity(), mx = -mn;
    int zr = d == 3 ? m : 0;
    for (int c = 0; c <= zr; ++c)
      for (int b = 0; b <= m; ++b)
        for (int a = 0; a <= m; ++a) {
          double v = phi(ix * m + a, iy * m + b, iz * m + c);
          if (!std::isfinite(v)) return false;
          mn = std::min(mn, v);
          mx = std::max(mx, v);
        }
    cls[cell] = (mx < -margin) ? OUTSIDE : ((mn > margin) ? INSIDE : CUT);
  }
  return true;
}

// ----------------------------------------------------------- numbering --

void build_slabs(Plan& p, int nslab) { p.slabs = slab_table(p, nslab); }

std::vector<int64_t> slab_y_bounds(const Plan& p, const std::vector<int32_t>& table) {
  const int ns = (int)(table.size() / SLAB);
  const int KR = p.num_lift_cells() > 0 ? (int)(p.lrow.size() / p.num_lift_cells()) : 0;
  std::vector<int64_t> b(ns + 1, 0);
  b[ns] = p.n_active;
  // b[s] = the smallest compact index a lift owner of slab s or later writes (each of its rows
  // writes base .. base + k - 1), so every index below it is final once slab s - 1 is lifted
  int64_t lo = p.n_active;
  for (int s = ns - 1; s >= 1; --s) {
    for (int64_t o = table[(size_t)s * SLAB]; o < table[(size_t)s * SLAB + 1]; ++o)
      for (int r = 0; r < KR; ++r) {
        const int32_t base = p.lrow[(size_t)o * KR + r];
        if (base >= 0) lo = std::min<int64_t>(lo, base);
      }
    b[s] = lo;
  }
  for (int s = 1; s <= ns; ++s) b[s] = std::max(b[s], b[s - 1]);
  return b;
}

std::vector<int64_t> slab_x_bounds(const Plan& p, const std::vector<int32_t>& table) {
  const int ns = (int)(table.size() / SLAB);
  const int k = p.k, d = p.dim, L = p.L, NN = 2 * k + 1, K1 = k + 1;
  const int R1 = d == 3 ? NN * K1 : NN;
  std::vector<int64_t> b(ns, 0);
  int64_t hi = 0;
  for (int s = 0; s < ns; ++s) {
    for (int a = 0; a < d; ++a) {
      const int rows = a == 0 ? L : R1, span = a == 0 ? NN : K1;
      for (int64_t f = table[(size_t)s * SLAB + 2 + 2 * a]; f < table[(size_t)s * SLAB + 3 + 2 * a]; ++f) {
        const int32_t* r = &p.frows[p.rbase[a] + (f - p.fstart[a]) * rows];
        for (int i = 0; i < rows; ++i) hi = std::max<int64_t>(hi, (int64_t)r[i] + span);
      }
    }
    b[s] = hi;
  }
  return b;
}

std::vector<int32_t> slab_table(const Plan& p, int nslab) {
  std::vector<int32_t> table;
  const int64_t nlift = p.num_lift_cells(), ngroup = (nlift + SLAB_GROUP - 1) / SLAB_GROUP;
  if (nslab <= 1 || ngroup < 2 || p.num_faces() == 0) return table;
  nslab = (int)std::min<int64_t>(nslab, ngroup);
  const int d = p.dim, nw = p.lwin_width / d;
  int32_t done[3] = {p.fstart[0], p.fstart[1], p.fstart[2]};   // faces of earlier slabs: [fstart, done)
  for (int s = 0; s < nslab; ++s) {
    const int64_t lo = std::min(nlift, (ngroup * s / nslab) * SLAB_GROUP);
    const int64_t hi = s == nslab - 1 ? nlift : std::min(nlift, (ngroup * (s + 1) / nslab) * SLAB_GROUP);
    int32_t need[3] = {done[0], done[1], done[2]};
    for (int64_t i = lo; i < hi; ++i)
      for (int a = 0; a < d; ++a)
        for (int w = 0; w < nw; ++w) {
          const int32_t f = p.lwin[(size_t)p.lwin_width * i + a * nw + w];
          if (f >= 0) need[a] = std::max(need[a], f + 1);
        }
    int32_t sl[SLAB] = {(int32_t)lo, (int32_t)hi, 0, 0, 0, 0, 0, 0};
    for (int a = 0; a < d; ++a) {
      const int32_t end = s == nslab - 1 ? p.fstart[a + 1] : need[a];
      sl[2 + 2 * a] = done[a];
      sl[3 + 2 * a] = end;
      done[a] = end;
    }
    table.insert(table.end(), sl, sl + SLAB);
  }
  return table;
}

int64_t Plan::compact(int X, int64_t row) const {
  int64_t base = row_start[row];
  for (int r = run_off[row]; r < run_off[row + 1]; ++r) {
    int X0 = runs[2 * r], X1 = runs[2 * r + 1];
    if (X >= X0 && X <= X1) return base + (X - X0);
    if (X > X1) base += X1 - X0 + 1;
  }
  return -1;
}

// cell indices along one axis whose closure contains lattice coordinate Y
static int adjacent_cells(int Y, int k, int n, int out[2]) {
  int c = Y / k, cnt = 0;
  if (Y % k == 0 && c - 1 >= 0) out[cnt++] = c - 1;
  if (c < n) out[cnt++] = c;
  return cnt;
}

// Per lattice row: x-runs of nodes that belong to a cell flagged in `mask`.
static void row_runs(const Plan& p, const std::vector<uint8_t>& mask, int64_t row,
                     std::vector<int>& out) {
  const int n = p.n, k = p.k;
  int Y = (int)(row % p.nl), Z = p.dim == 3 ? (int)(row / p.nl) : 0;
  int cy[2], cz[2] = {0, 0};
  int ny = adjacent_cells(Y, k, n, cy);
  int nz = p.dim == 3 ? adjacent_cells(Z, k, n, cz) : 1;
  out.clear();
  int open0 = -1, open1 = -1;
  for (int ci = 0; ci < n; ++ci) {
    bool on = false;
    for (int a = 0; a < ny && !on; ++a)
      for (int b = 0; b < nz && !on; ++b) {
        int64_t cell = ci + (int64_t)n * (cy[a] + (int64_t)n * cz[b]);
        on = mask[cell] != 0;
      }
    if (!on) continue;
    int X0 = ci * k, X1 = ci * k + k;
    if (open0 >= 0 && X0 <= open1) {
      open1 = X1;
    } else {
      if (open0 >= 0) { out.push_back(open0); out.push_back(open1); }
      open0 = X0;
      open1 = X1;
    }
  }
  if (open0 >= 0) { out.push_back(open0); out.push_back(open1); }
}

void active_coords(const Plan& p, double* xyz) {
  const int d = p.dim, k = p.k;
  int64_t c = 0;
  auto coord = [&](int a, int X) {
    int ci = X / k, q = X % k;
    return p.lo[a] + (ci + p.gl[q]) * p.h;
  };
  for (int64_t row = 0; row < p.nrows; ++row) {
    int Y = (int)(row % p.nl), Z = d == 3 ? (int)(row / p.nl) : 0;
    for (int r = p.run_off[row]; r < p.run_off[row + 1]; ++r)
      for (int X = p.runs[2 * r]; X <= p.runs[2 * r + 1]; ++X) {
        xyz[c * d + 0] = coord(0, X);
        xyz[c * d + 1] = coord(1, Y);
        if (d == 3) xyz[c * d + 2] = coord(2, Z);
        ++c;
      }
  }
}

// ---------------------------------------------------------------- plan --

// Checks the arguments and classifies the cells (fills the mesh fields and cls).
static gp_status classify_mesh(const gp_mesh* mesh, const gp_levelset* ls, const gp_opts* opts, Plan& p,
                               std::string& err) {
  if (!mesh || !ls || !opts) { err = "null argument"; return GP_EINVAL; }
  const int d = mesh->dim;
  if (d != 2 && d != 3) { err = "dim must be 2 or 3"; return GP_EINVAL; }
  const int k = opts->degree;
  if (k < 1) { err = "degree must be >= 1"; return GP_EINVAL; }
  if (k > KMAX) { err = "degree > 8 is not built"; return GP_EUNSUPPORTED; }
  if (opts->precision != GP_FP64 && opts->precision != GP_FP32 && opts->precision != GP_FP64_FF) {
    err = "bad precision";
    return GP_EINVAL;
  }
  const int n = mesh->n[0];
  for (int a = 0; a < d; ++a) {
    if (mesh->n[a] != n) { err = "the mesh must have the same number of cells per axis"; return GP_EINVAL; }
    if (!(mesh->hi[a] > mesh->lo[a])) { err = "empty mesh box"; return GP_EINVAL; }
  }
  if (n < 1 || (int64_t)n * k + 1 > (1 << 24)) { err = "bad cell count"; return GP_EINVAL; }
  const double h = (mesh->hi[0] - mesh->lo[0]) / n;
  for (int a = 1; a < d; ++a) {
    double ha = (mesh->hi[a] - mesh->lo[a]) / n;
    if (std::fabs(ha - h) > 1e-12 * h) { err = "cells must be squares/cubes (equal h per axis)"; return GP_EINVAL; }
  }
  if (opts->nweights != 0 && opts->nweights != k) { err = "nweights must be 0 or k"; return GP_EINVAL; }
  if (opts->nweights == k && !opts->weights) { err = "weights is NULL"; return GP_EINVAL; }

  p.dim = d;
  p.n = n;
  p.k = k;
  p.precision = opts->precision;
  for (int a = 0; a < 3; ++a) p.lo[a] = a < d ? mesh->lo[a] : 0.0;
  p.h = h;
  p.nl = n * k + 1;
  p.ncell = ipow(n, d);
  p.nrows = ipow(p.nl, d - 1);
  p.L = (int)ipow(k + 1, d - 1);
  if (p.ncell > (int64_t)1 << 31) { err = "too many cells"; return GP_EINVAL; }

  // ---- classification
  p.cls.assign(p.ncell, OUTSIDE);
  switch (ls->kind) {
    case GP_LS_CONST:
      std::fill(p.cls.begin(), p.cls.end(), ls->value > 0 ? INSIDE : OUTSIDE);
      break;
    case GP_LS_BALLS:
      if (ls->nballs < 1 || !ls->centers || !ls->radii) { err = "balls need centers and radii"; return GP_EINVAL; }
      classify_balls(p, ls, n, p.cls);
      break;
    case GP_LS_GYROID:
      if (d != 3) { err = "the gyroid level set is 3D"; return GP_EINVAL; }
      if (!classify_sampled(p, ls, n, mesh->hi[0], p.cls)) { err = "the level set is not finite"; return GP_EINVAL; }
      break;
    case GP_LS_CALLBACK:
      if (!ls->fn || !(ls->lipschitz > 0)) { err = "callback level set needs fn and lipschitz > 0"; return GP_EINVAL; }
      if (!classify_sampled(p, ls, n, mesh->hi[0], p.cls)) {
        err = "the level-set callback returned a value that is not finite";
        return GP_EINVAL;
      }
      break;
    default:
      err = "unknown level-set kind";
      return GP_EINVAL;
  }
  for (int c = 0; c < 3; ++c) p.cell_counts[c] = 0;
  for (int64_t c = 0; c < p.ncell; ++c) p.cell_counts[(int)p.cls[c]]++;
  return GP_OK;
}

// Cell weights for the load balance of Sec. 2.7: 0 outside, 1 inside, k^(d-1) cut.
// Layer l (cells with last coordinate l) weighs C_{l+1} - C_l.  Boundary b_p is the
// first layer boundary with C_b * nparts >= p * C_n, clamped to [2p, n - 2(nparts - p)]
// and pushed up to b_{p-1} + 2: every partition holds at least two layers, so the halo
// of a partition never reaches beyond its neighbour.
gp_status partition_slabs(const gp_mesh* mesh, const gp_levelset* ls, const gp_opts* opts, int nparts,
                          int32_t* bounds, std::string& err) {
  if (!bounds) { err = "null argument"; return GP_EINVAL; }
  if (nparts < 1) { err = "nparts must be >= 1"; return GP_EINVAL; }
  Plan p;
  gp_status st = classify_mesh(mesh, ls, opts, p, err);
  if (st != GP_OK) return st;
  const int n = p.n;
  if (nparts > 1 && n < 2 * nparts) { err = "fewer than two cell layers per partition"; return GP_EINVAL; }
  const int64_t layer = p.ncell / n;
  const int64_t wcut = ipow(p.k, p.dim - 1);
  std::vector<int64_t> C(n + 1, 0);
  for (int l = 0; l < n; ++l) {
    int64_t w = 0;
    for (int64_t c = (int64_t)l * layer; c < (int64_t)(l + 1) * layer; ++c)
      w += p.cls[c] == INSIDE ? 1 : (p.cls[c] == CUT ? wcut : 0);
    C[l + 1] = C[l] + w;
  }
  bounds[0] = 0;
  bounds[nparts] = n;
  for (int q = 1; q < nparts; ++q) {
    int b = 0;
    while (b < n && C[b] * nparts < q * C[n]) ++b;
    b = std::max(b, 2 * q);
    b = std::min(b, n - 2 * (nparts - q));
    b = std::max(b, bounds[q - 1] + 2);
    bounds[q] = b;
  }
  return GP_OK;
}

gp_status build_plan(const gp_mesh* mesh, const gp_levelset* ls, const gp_opts* opts, Plan& p,
                     std::string& err) {
  gp_status st = classify_mesh(mesh, ls, opts, p, err);
  if (st != GP_OK) return st;
  const int d = p.dim, n = p.n, k = p.k;
  const double h = p.h;

  // ---- partition (Sec. 2.7): layers [part_lo, part_hi) of the last axis
  p.partitioned = opts->part_lo != 0 || opts->part_hi != 0;
  p.part_lo = p.partitioned ? opts->part_lo : 0;
  p.part_hi = p.partitioned ? opts->part_hi : n;
  if (p.partitioned) {
    if (p.part_lo < 0 || p.part_hi > n || p.part_hi <= p.part_lo) { err = "bad partition layers"; return GP_EINVAL; }
    if (p.part_lo > 0 && p.part_hi < n && p.part_hi - p.part_lo < 2) {
      err = "a partition between two others needs at least two cell layers";
      return GP_EINVAL;
    }
  }
  const int64_t layer_cells = p.ncell / n;

  // ---- ghost faces, sorted by axis then lower cell.  A face belongs to the partition of
  // its lower cell: the lower rank of the two for a face across a partition boundary.
  p.face_cell.clear();
  const int64_t stride[3] = {1, n, (int64_t)n * n};
  for (int a = 0; a < d; ++a) {
    p.fstart[a] = (int32_t)p.face_cell.size();
    for (int64_t c = 0; c < p.ncell; ++c) {
      int ia = (int)((c / stride[a]) % n);
      if (ia + 1 >= n) continue;
      const int64_t lay = c / layer_cells;
      if (lay < p.part_lo || lay >= p.part_hi) continue;
      int8_t c0 = p.cls[c], c1 = p.cls[c + stride[a]];
      if (c0 == OUTSIDE || c1 == OUTSIDE) continue;
      if (opts->all_faces || c0 == CUT || c1 == CUT) p.face_cell.push_back(c);
    }
  }
  p.fstart[d] = (int32_t)p.face_cell.size();
  for (int a = d + 1; a < 4; ++a) p.fstart[a] = p.fstart[d];
  const int64_t nf = p.num_faces();
  if (nf > (int64_t)1 << 30) { err = "too many faces"; return GP_EINVAL; }

  // ---- involved cells (the two cells of every face)
  std::vector<int32_t> inv_of(p.ncell, -1);
  std::vector<uint8_t> involved(p.ncell, 0);
  for (int a = 0; a < d; ++a)
    for (int64_t f = p.fstart[a]; f < p.fstart[a + 1]; ++f) {
      involved[p.face_cell[f]] = 1;
      involved[p.face_cell[f] + stride[a]] = 1;
    }
  p.inv_cells.clear();
  for (int64_t c = 0; c < p.ncell; ++c)
    if (involved[c]) {
      inv_of[c] = (int32_t)p.inv_cells.size();
      p.inv_cells.push_back(c);
    }
  p.face_inv.resize(2 * nf);
  p.face_of.assign((size_t)d * p.ncell, -1);
  for (int a = 0; a < d; ++a)
    for (int64_t f = p.fstart[a]; f < p.fstart[a + 1]; ++f) {
      int64_t c = p.face_cell[f];
      p.face_inv[2 * f] = inv_of[c];
      p.face_inv[2 * f + 1] = inv_of[c + stride[a]];
      p.face_of[(size_t)a * p.ncell + c] = (int32_t)f;
    }

  // ---- numbering: active runs per lattice row
  std::vector<uint8_t> active(p.ncell);
  for (int64_t c = 0; c < p.ncell; ++c) active[c] = p.cls[c] != OUTSIDE;
  p.row_start.assign(p.nrows, 0);
  p.run_off.assign(p.nrows + 1, 0);
  p.runs.clear();
  std::vector<int> tmp;
  int64_t total = 0;
  for (int64_t row = 0; row < p.nrows; ++row) {
    row_runs(p, active, row, tmp);
    p.row_start[row] = total;
    for (size_t i = 0; i < tmp.size(); i += 2) {
      p.runs.push_back(tmp[i]);
      p.runs.push_back(tmp[i + 1]);
      total += tmp[i + 1] - tmp[i] + 1;
    }
    p.run_off[row + 1] = (int32_t)(p.runs.size() / 2);
  }
  if (total >= ((int64_t)1 << 31) - 1) { err = "too many active DoFs for 32-bit indices"; return GP_EUNSUPPORTED; }
  p.n_global = total;
  p.n_active = total;
  p.g_offset = 0;
  p.n_owned = total;
  p.n_lower = 0;
  if (p.partitioned) {
    // keep the lattice planes [W0, W1] of the last axis, renumbered from 0
    const int64_t rpp = d == 3 ? p.nl : 1;                 // lattice rows per plane
    auto plane_start = [&](int64_t Z) { return Z * rpp < p.nrows ? p.row_start[Z * rpp] : total; };
    const int64_t W0 = (int64_t)p.part_lo * k, W1 = (int64_t)std::min(p.part_hi + 1, n) * k;
    p.g_offset = plane_start(W0);
    p.n_active = plane_start(W1 + 1) - p.g_offset;
    p.n_owned = (p.part_hi < n ? plane_start((int64_t)p.part_hi * k) : total) - p.g_offset;
    p.n_lower = p.part_lo > 0 ? plane_start((int64_t)(p.part_lo + 1) * k + 1) - p.g_offset : 0;
    std::vector<int32_t> runs2, off2(p.nrows + 1, 0);
    for (int64_t row = 0; row < p.nrows; ++row) {
      const int64_t Z = row / rpp;
      if (Z >= W0 && Z <= W1) {
        for (int r = p.run_off[row]; r < p.run_off[row + 1]; ++r) {
          runs2.push_back(p.runs[2 * r]);
          runs2.push_back(p.runs[2 * r + 1]);
        }
        p.row_start[row] -= p.g_offset;
      } else {
        p.row_start[row] = 0;
      }
      off2[row + 1] = (int32_t)(runs2.size() / 2);
    }
    p.runs.swap(runs2);
    p.run_off.swap(off2);
  }

  // ---- row table of the involved cells
  const int L = p.L;
  const int64_t ninv = (int64_t)p.inv_cells.size();
  p.rowtab.resize((size_t)ninv * L);
  for (int64_t i = 0; i < ninv; ++i) {
    int64_t c = p.inv_cells[i];
    int ci = (int)(c % n), cj = (int)((c / n) % n), cl = d == 3 ? (int)(c / ((int64_t)n * n)) : 0;
    for (int t = 0; t < L; ++t) {
      int ty = t % (k + 1), tz = t / (k + 1);
      int64_t row = (int64_t)(cj * k + ty) + (d == 3 ? (int64_t)p.nl * (cl * k + tz) : 0);
      int64_t cidx = p.compact(ci * k, row);
      if (cidx < 0) { err = "internal: involved cell node not active"; return GP_EINVAL; }
      p.rowtab[(size_t)i * L + t] = (int32_t)cidx;
    }
  }

  // ---- per-face row starts (the gather reads them with one coalesced load per face)
  {
    const int K1 = k + 1, NN = 2 * k + 1;
    const int R0 = L, R1 = d == 3 ? NN * K1 : NN;
    int64_t off = 0;
    for (int a = 0; a < d; ++a) {
      p.rbase[a] = off;
      off += (int64_t)(p.fstart[a + 1] - p.fstart[a]) * (a == 0 ? R0 : R1);
    }
    for (int a = d; a < 4; ++a) p.rbase[a] = off;
    p.frows.assign(off, 0);
    for (int a = 0; a < d; ++a)
      for (int64_t f = p.fstart[a]; f < p.fstart[a + 1]; ++f) {
        const int32_t* rlo = &p.rowtab[(size_t)p.face_inv[2 * f] * L];
        const int32_t* rhi = &p.rowtab[(size_t)p.face_inv[2 * f + 1] * L];
        if (a == 0) {
          int32_t* dst = &p.frows[p.rbase[0] + (f - p.fstart[0]) * R0];
          for (int t = 0; t < L; ++t) dst[t] = rlo[t];
        } else {
          int32_t* dst = &p.frows[p.rbase[a] + (f - p.fstart[a]) * R1];
          const int outer = d == 3 ? K1 : 1;
          for (int tr = 0; tr < outer; ++tr)
            for (int b = 0; b < NN; ++b) {
              const int32_t* rt = b <= k ? rlo : rhi;
              const int bc = b <= k ? b : b - k;
              // a = 1: rows (b, tz) -> b + K1 tz ; a = 2: rows (ty, b) -> ty + K1 b
              const int ri = d == 2 ? bc : (a == 1 ? bc + K1 * tr : tr + K1 * bc);
              dst[b + NN * tr] = rt[ri];
            }
        }
      }
  }

  // ---- touched DoFs (nodes of involved cells) and the zero runs (active, untouched)
  std::vector<int> trun;
  int64_t touched = 0;
  p.zruns.clear();
  for (int64_t row = 0; row < p.nrows; ++row) {
    if (p.run_off[row] == p.run_off[row + 1]) continue;
    row_runs(p, involved, row, trun);
    int64_t c = p.row_start[row];
    size_t tr = 0;
    for (int r = p.run_off[row]; r < p.run_off[row + 1]; ++r) {
      int X = p.runs[2 * r], X1 = p.runs[2 * r + 1];
      while (X <= X1) {
        while (tr < trun.size() && trun[tr + 1] < X) tr += 2;
        int e;
        if (tr < trun.size() && trun[tr] <= X) {
          e = std::min(X1, trun[tr + 1]);
          touched += e - X + 1;
        } else {
          e = (tr < trun.size()) ? std::min(X1, trun[tr] - 1) : X1;
          int64_t c0 = c;
          int len = e - X + 1;
          // extend the previous run when contiguous in compact order, then split at ZRUN_MAX
          while (len > 0) {
            if (!p.zruns.empty() && (int64_t)p.zruns[p.zruns.size() - 2] + p.zruns.back() == c0 &&
                p.zruns.back() < ZRUN_MAX) {
              int l = std::min(len, ZRUN_MAX - p.zruns.back());
              p.zruns.back() += l;
              c0 += l;
              len -= l;
            } else {
              int l = std::min(len, ZRUN_MAX);
              p.zruns.push_back((int32_t)c0);
              p.zruns.push_back(l);
              c0 += l;
              len -= l;
            }
          }
        }
        c += e - X + 1;
        X = e + 1;
      }
    }
  }
  p.n_touched = touched;
  // ---- lift cells: owners floor(X/k) of the touched nodes, coordinates in [0, n]
  {
    const int n1 = n + 1;
    const int64_t nown = ipow(n1, d);
    std::vector<uint8_t> own(nown, 0);
    for (int64_t i = 0; i < ninv; ++i) {
      int64_t c = p.inv_cells[i];
      int ci = (int)(c % n), cj = (int)((c / n) % n), cl = d == 3 ? (int)(c / ((int64_t)n * n)) : 0;
      for (int dz = 0; dz <= (d == 3 ? 1 : 0); ++dz)
        for (int dy = 0; dy <= 1; ++dy)
          for (int dx = 0; dx <= 1; ++dx)
            own[(ci + dx) + (int64_t)n1 * ((cj + dy) + (int64_t)n1 * (cl + dz))] = 1;
    }
    // candidate-face pattern of an owner cell c: bit (a, s_a, s_1, s_2) set when the face with
    // normal a and lower cell c + (s_a-2) e_a + (s_1-1) e_t1 + (s_2-1) e_t2 exists
    const int nw = d == 3 ? 12 : 6;
    p.lwin_width = d * nw;
    auto window = [&](const int co0[3], int32_t* out) {
      for (int a = 0; a < d; ++a) {
        const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
        for (int w = 0; w < nw; ++w) {
          int sa = d == 3 ? w / 4 : w / 2, s1 = d == 3 ? (w % 4) / 2 : w % 2, s2 = d == 3 ? w % 2 : 1;
          int co[3] = {co0[0], co0[1], co0[2]};
          co[a] += sa - 2;
          co[t1] += s1 - 1;
          if (d == 3) co[t2] += s2 - 1;
          bool ok = co[a] >= 0 && co[a] <= n - 2 && co[t1] >= 0 && co[t1] <= n - 1;
          if (d == 3) ok = ok && co[t2] >= 0 && co[t2] <= n - 1;
          int32_t f = -1;
          if (ok) {
            int64_t lin = co[0] + (int64_t)n * co[1] + (d == 3 ? (int64_t)n * n * co[2] : 0);
            f = p.face_of[(size_t)a * p.ncell + lin];
          }
          out[a * nw + w] = f;
        }
      }
    };
    auto pattern = [&](const int co0[3]) -> uint64_t {
      int32_t win[36];
      window(co0, win);
      uint64_t m = 0;
      for (int i = 0; i < d * nw; ++i)
        if (win[i] >= 0) m |= (uint64_t)1 << i;
      return m;
    };
    std::vector<std::pair<uint64_t, int64_t>> order;
    for (int64_t o = 0; o < nown; ++o) {
      if (!own[o]) continue;
      int co[3] = {(int)(o % n1), (int)((o / n1) % n1), d == 3 ? (int)(o / ((int64_t)n1 * n1)) : 0};
      order.emplace_back(pattern(co), o);
    }
    // FP64: same-pattern cells share a warp, so the lift issues (almost) only useful FP64
    // work; the cells are sorted by pattern only within consecutive groups of LIFT_SORT_GROUP
    // owners of the lexicographic order, so that the lift still reads the face outputs of one
    // region of the mesh at a time (a global pattern sort scattered those reads: 6.5 times the
    // face-output bytes came from DRAM on the 128^3 gyroid).  FP32 and float-float: keep the
    // lexicographic order, so a warp's loads and stores stay in neighbouring memory (FP32 issue
    // is cheap on this GPU).
    if (opts->precision == GP_FP64) {
      constexpr size_t LIFT_SORT_GROUP = SLAB_GROUP;
      for (size_t g0 = 0; g0 < order.size(); g0 += LIFT_SORT_GROUP)
        std::stable_sort(order.begin() + g0, order.begin() + std::min(order.size(), g0 + LIFT_SORT_GROUP),
                         [](const std::pair<uint64_t, int64_t>& x, const std::pair<uint64_t, int64_t>& y) {
                           return x.first < y.first;
                         });
    }
    const int KR = (int)ipow(k, d - 1);   // rows q (, r) in [0, k) of an owner cell
    const int64_t nlift = (int64_t)order.size();
    p.lcell.assign(4 * nlift, 0);
    p.lrow.assign((size_t)KR * nlift, -1);
    p.lwin.assign((size_t)p.lwin_width * nlift, -1);
    for (int64_t i = 0; i < nlift; ++i) {
      int64_t o = order[i].second;
      int ci = (int)(o % n1), cj = (int)((o / n1) % n1), cl = d == 3 ? (int)(o / ((int64_t)n1 * n1)) : 0;
      p.lcell[4 * i + 0] = ci;
      p.lcell[4 * i + 1] = cj;
      p.lcell[4 * i + 2] = cl;
      const int co[3] = {ci, cj, cl};
      window(co, &p.lwin[(size_t)p.lwin_width * i]);
      for (int t = 0; t < KR; ++t) {
        int q = t % k, r = t / k;
        int Y = cj * k + q, Z = cl * k + r, X = ci * k;
        int64_t cidx = -1;
        if (Y < p.nl && (d == 2 || Z < p.nl) && X < p.nl) {
          int64_t row = (int64_t)Y + (d == 3 ? (int64_t)p.nl * Z : 0);
          cidx = p.compact(X, row);
        }
        p.lrow[(size_t)i * KR + t] = (int32_t)cidx;
      }
    }
  }

  // ---- bounds of every index the kernels read or write (the GPU has no bounds checker here)
  {
    const int64_t na = p.n_active, K1 = k + 1, NN = 2 * k + 1;
    const int R1 = d == 3 ? (int)(NN * K1) : (int)NN;
    for (int a = 0; a < d; ++a) {
      const int64_t rows = (int64_t)(p.fstart[a + 1] - p.fstart[a]) * (a == 0 ? L : R1);
      const int64_t span = a == 0 ? NN : K1;          // contiguous values read from each row start
      for (int64_t i = 0; i < rows; ++i) {
        const int64_t r = p.frows[p.rbase[a] + i];
        if (r < 0 || r + span > na) { err = "internal: face row outside the active DoFs"; return GP_EINVAL; }
      }
    }
    for (int32_t f : p.lwin)
      if (f < -1 || f >= (int32_t)nf) { err = "internal: lift window outside the face list"; return GP_EINVAL; }
    for (int32_t r : p.lrow)
      if (r < -1 || r >= na) { err = "internal: lift row outside the active DoFs"; return GP_EINVAL; }
    for (size_t i = 0; i + 1 < p.zruns.size(); i += 2)
      if (p.zruns[i] < 0 || p.zruns[i + 1] < 1 || p.zruns[i + 1] > ZRUN_MAX || p.zruns[i] + p.zruns[i + 1] > na) {
        err = "internal: zero run outside the active DoFs";
        return GP_EINVAL;
      }
  }

  // ---- 1D reference data and the per-order scale c_j h^(d-2)
  gauss_lobatto_01(k, p.gl);
  reference_1d(k, p.gl, p.mass, p.jumps);
  reference_stiffness(k, p.stiff);
  p.scale.resize(k);
  p.stabilization = opts->stabilization;
  if (opts->stabilization == GP_STAB_MACRO) {
    // macro patch: gamma h^d sum_j lambda_j (M^ x ... x v_j v_j^T)  (volume integral: h per direction)
    std::vector<double> lam;
    if (!macro_patch_1d(k, p.jumps, lam)) { err = "internal: macro-patch matrix not of rank k"; return GP_EINVAL; }
    const double hv = d == 3 ? h * h * h : h * h;
    for (int j = 0; j < k; ++j) {
      p.scale[j] = opts->gamma * lam[j] * hv;
      const double a = std::fabs(p.scale[j]);
      if (opts->precision == GP_FP64_FF && a != 0.0 && !(a >= 0x1p-90 && a <= 0x1p90)) {
        err = "GP_FP64_FF: a macro-patch scale factor lies outside [2^-90, 2^90]; use GP_FP64";
        return GP_EINVAL;
      }
    }
    return GP_OK;
  }
  if (opts->stabilization != GP_STAB_GHOST) { err = "unknown stabilization"; return GP_EINVAL; }
  const double hd = d == 3 ? h : 1.0;
  for (int j = 0; j < k; ++j) {
    double c = opts->nweights == k ? opts->weights[j] : opts->gamma;
    p.scale[j] = c * hd;
    // float-float keeps float's exponent range: the scale factors must stay well inside it
    const double a = std::fabs(p.scale[j]);
    if (opts->precision == GP_FP64_FF && a != 0.0 && !(a >= 0x1p-90 && a <= 0x1p90)) {
      err = "GP_FP64_FF: the scale factor c_j h^(d-2) of order " + std::to_string(j + 1) +
            " lies outside [2^-90, 2^90]; use GP_FP64";
      return GP_EINVAL;
    }
  }
  return GP_OK;
}

}  // namespace gp
