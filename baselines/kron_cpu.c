/* The paper's own evaluation of y = G x on the CPU: the factorised face operator
 * (Sec. 2.4) applied in one-dimensional steps (Sec. 2.5.1), FP64, OpenMP over faces.
 *
 * TEST INFRASTRUCTURE ONLY: the paper-like CPU baseline that bench.py times beside the
 * oracle.  It is not the oracle (which never factorises), shares no code with the CUDA
 * path, and is checked against the oracle by tests/test_oracle_kronecker.py.
 *
 * Per face with normal a: gather the (2k+1) x (k+1)^(d-1) patch values (x fastest),
 * apply the reference penalty G^ along the normal and the reference mass M^ along each
 * tangential direction, scale by h^(d-2), and add the result into y, one colour class of
 * faces after another (within a class no two faces share a node): deterministic, with no
 * atomics.  Portable C99 + OpenMP: no architecture-specific code. */
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* out = A applied along direction `dir` of an ext[0] x ext[1] x ext[2] box (x fastest);
 * A is ext[dir] x ext[dir] row-major.  The innermost loop runs along x where it can. */
static void along(const double* in, double* out, const int ext[3], int dir, const double* A) {
  const int nx = ext[0], ny = ext[1], nz = ext[2];
  if (dir == 0) {
    for (int l = 0; l < ny * nz; ++l) {
      const double* src = in + l * nx;
      double* dst = out + l * nx;
      for (int i = 0; i < nx; ++i) {
        double s = 0.0;
        for (int m = 0; m < nx; ++m) s += A[i * nx + m] * src[m];
        dst[i] = s;
      }
    }
  } else if (dir == 1) {
    for (int z = 0; z < nz; ++z)
      for (int i = 0; i < ny; ++i) {
        double* dst = out + nx * (i + ny * z);
        for (int x = 0; x < nx; ++x) dst[x] = 0.0;
        for (int m = 0; m < ny; ++m) {
          const double a = A[i * ny + m];
          const double* src = in + nx * (m + ny * z);
          for (int x = 0; x < nx; ++x) dst[x] += a * src[x];
        }
      }
  } else {
    const int plane = nx * ny;
    for (int i = 0; i < nz; ++i) {
      double* dst = out + plane * i;
      for (int e = 0; e < plane; ++e) dst[e] = 0.0;
      for (int m = 0; m < nz; ++m) {
        const double a = A[i * nz + m];
        const double* src = in + plane * m;
        for (int e = 0; e < plane; ++e) dst[e] += a * src[e];
      }
    }
  }
}

/* dim 2 or 3, degree k; per axis a: nf[a] faces with patch indices idx[a] (nf[a] x P int64,
 * patch order x fastest with 2k+1 nodes along a), sorted by colour, and the colour offsets
 * coff[a] (13 int64: faces [coff[a][c], coff[a][c+1]) have colour c).  Colour of a face with
 * lower cell i: (i_a mod 3) + 3 (i_t1 mod 2) + 6 (i_t2 mod 2); faces of one colour share no
 * node (their patches are at least three cells apart along a and two along the others), so
 * each colour adds into y without conflicts, and the colours run in order.  M (k+1)^2 and
 * G (2k+1)^2 row-major; scale = h^(d-2); x, y of length n (y overwritten).  Returns 0, or -1
 * on bad arguments. */
int kron_apply(int dim, int k, const int64_t* nf, const int64_t* const* idx, const int64_t* const* coff,
               const double* M, const double* G, double scale, const double* x, double* y, int64_t n,
               int nthreads) {
  if ((dim != 2 && dim != 3) || k < 1 || k > 8 || n < 0 || nthreads < 1) return -1;
  const int K1 = k + 1, NN = 2 * k + 1;
  const int P = NN * (dim == 3 ? K1 * K1 : K1);
#ifdef _OPENMP
  omp_set_num_threads(nthreads);
#endif
  memset(y, 0, (size_t)n * sizeof(double));
  for (int a = 0; a < dim; ++a) {
    int ext[3] = {K1, K1, dim == 3 ? K1 : 1};
    ext[a] = NN;
    const int64_t* ia = idx[a];
    if (coff[a][12] != nf[a]) return -1;
    for (int c = 0; c < 12; ++c) {
      const int64_t f0 = coff[a][c], f1 = coff[a][c + 1];
#pragma omp parallel
      {
        double u[17 * 81], v[17 * 81];
#pragma omp for schedule(static)
        for (int64_t f = f0; f < f1; ++f) {
          const int64_t* pi = ia + f * P;
          for (int i = 0; i < P; ++i) u[i] = x[pi[i]];
          along(u, v, ext, 0, a == 0 ? G : M);
          along(v, u, ext, 1, a == 1 ? G : M);
          if (dim == 3) {
            along(u, v, ext, 2, a == 2 ? G : M);
            for (int i = 0; i < P; ++i) y[pi[i]] += scale * v[i];
          } else {
            for (int i = 0; i < P; ++i) y[pi[i]] += scale * u[i];
          }
        }
      }
    }
  }
  return 0;
}
