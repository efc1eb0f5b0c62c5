// Model SPD system (M_active + K_active + G) u = b and its solvers.
//
// The system couples the ghost penalty G with the mass and Laplace stiffness of
// every active cell integrated as a full cell (Sec. 2.5.2 for the interior-cell
// evaluation).  The paper leaves the solver to future work (Sec. 1); this file
// provides the defect-correction scheme of mixed-precision solvers: residuals,
// updates and inner products in FP64, the inner correction solved by CG with the
// FP32 operator, next to plain CG with the FP64 operator for comparison.  The inner
// CG's FP32 vectors have their inner products summed from exact float products in
// compensated float-float arithmetic and combined in FP64 (IoDot), which keeps the
// FP64 pipe (2 FMAs per clock per SM on GB300) out of the per-element work.
//
// Every reduction has a fixed order (fixed grid, fixed tree), so a solve is
// bitwise reproducible.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "gp_arith.cuh"
#include "gp_internal.h"

struct gp_system {
  gp_ctx* hi = nullptr;   // FP64 or float-float operator
  gp_ctx* lo = nullptr;   // FP32 operator (optional)
  int device = -1;
  int64_t n = 0;
  int32_t* d_crow = nullptr;
  int32_t* d_cwin = nullptr;
  int32_t* d_corow = nullptr;
  void* d_wc = nullptr;     // cell outputs (scratch, 8 bytes per value)
  int32_t* d_o2l_hi = nullptr;  // per owner cell: lift owner index in hi's / lo's face plan
  int32_t* d_o2l_lo = nullptr;
  gp::CellTabs ct{};
  int nparts = 0;           // CTAs of the cell gather (fused inner-product partials)
  int nblk = 0;             // CTAs of the vector reductions: 4 per SM
  int nvec = 0;             // CTAs of the element-wise vector kernels: 8 per SM
  gp::CellsFn cells_hi = nullptr, cells_lo = nullptr;
  // solver vectors
  double *r = nullptr, *p = nullptr, *q = nullptr, *dd = nullptr, *z = nullptr, *ri = nullptr;
  float *r32 = nullptr, *d32 = nullptr, *ri32 = nullptr, *p32 = nullptr, *q32 = nullptr, *z32 = nullptr;
  double* dinv = nullptr;   // 1 / diag(A) (Jacobi)
  float* dinv32 = nullptr;
  double* part = nullptr;   // dot partials + result
  double* h_res = nullptr;  // pinned copy of the dot result
  void* d_cg = nullptr;     // CgScalars of the running CG (device)
  void* h_cg = nullptr;     // pinned copy
  cudaStream_t st = nullptr;
  std::string err;
};

namespace {

using gpi::DeviceGuard;
using gpi::fail;

constexpr int kDotPerSm = 4;   // reduction CTAs per SM (the grid is a multiple of the SM count)
constexpr int kThreads = 256;
constexpr int kVecPerSm = 8;   // CTAs per SM of the element-wise vector kernels

template <typename T>
__global__ void __launch_bounds__(kThreads) dot_partial(const T* __restrict__ a, const T* __restrict__ b,
                                                        int64_t n, double* __restrict__ part) {
  __shared__ double sh[kThreads];
  gp::IoDot<T> acc;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    acc.add(a[i], b[i]);
  sh[threadIdx.x] = acc.value();
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kThreads) dot_final(const double* __restrict__ part, const int nblk,
                                                      double* __restrict__ out) {
  __shared__ double sh[kThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += kThreads) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < (n); i += (int64_t)gridDim.x * kThreads)

// vector updates in the vectors' own precision (FP32 vectors: FP32 arithmetic)
template <typename T>
__global__ void axpy_k(T* __restrict__ y, const T* __restrict__ x, double a, int64_t n) {
  const T at = (T)a;
  GRID_STRIDE(i, n) y[i] = fma(at, x[i], y[i]);
}
template <typename T>
__global__ void xpay_k(T* __restrict__ p, const T* __restrict__ r, double beta, int64_t n) {
  const T bt = (T)beta;
  GRID_STRIDE(i, n) p[i] = fma(bt, p[i], r[i]);
}
__global__ void resid_k(double* __restrict__ r, const double* __restrict__ b, const double* __restrict__ q,
                        int64_t n) {
  GRID_STRIDE(i, n) r[i] = b[i] - q[i];
}
__global__ void to32_k(float* __restrict__ o, const double* __restrict__ v, int64_t n) {
  GRID_STRIDE(i, n) o[i] = (float)v[i];
}
__global__ void add32_k(double* __restrict__ u, const float* __restrict__ d, int64_t n) {
  GRID_STRIDE(i, n) u[i] += (double)d[i];
}
template <typename T>
__global__ void scale_k(T* __restrict__ z, const T* __restrict__ dinv, const T* __restrict__ r, int64_t n) {
  GRID_STRIDE(i, n) z[i] = dinv[i] * r[i];
}
__global__ void add64_k(double* __restrict__ u, const double* __restrict__ d, int64_t n) {
  GRID_STRIDE(i, n) u[i] += d[i];
}

template <typename T>
cudaError_t dot(gp_system* s, const T* a, const T* b, double* out) {
  dot_partial<T><<<s->nblk, kThreads, 0, s->st>>>(a, b, s->n, s->part);
  dot_final<<<1, kThreads, 0, s->st>>>(s->part, s->nblk, s->part + 2 * s->nblk);
  cudaError_t e =
      cudaMemcpyAsync(s->h_res, s->part + 2 * s->nblk, sizeof(double), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  *out = *s->h_res;
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// y = A x with the operator of context c in three launches: the ghost-penalty face
// kernel (face outputs only), the cell kernel (cell outputs; it overlaps the face kernel
// as its programmatic dependent), and one gather that adds, per node, the face outputs
// and then the cell outputs and writes y once.  With dotp, the gather also leaves the
// partial sums of dotp . y (one per gather CTA, s->nparts of them) in s->part.
gp_status sys_apply(gp_system* s, gp_ctx* c, gp::CellsFn cells, const void* x, void* y, cudaStream_t st,
                    const void* dotp = nullptr) {
  gp_status g = gpi::launch(c, x, y, 1, st, nullptr, false, nullptr, 1);   // face kernel alone
  if (g != GP_OK) return g;
  const gp::Plan& p = c->plan;
  gp::CellTabs ct = s->ct;
  ct.dotp = dotp;
  ct.dotpart = dotp ? s->part : nullptr;
  ct.wf = c->d_tp;
  ct.fwin = c->d_lwin;
  ct.own2lift = c == s->hi ? s->d_o2l_hi : s->d_o2l_lo;
  const cudaError_t e = cells(p.k, x, y, ct, p.mass.data(), p.stiff.data(), p.h, 1.0, 1.0, 0, 0, st);
  if (e != cudaSuccess) return fail(c, GP_ECUDA, std::string("cell kernels: ") + cudaGetErrorString(e));
  return GP_OK;
}

gp::CellsFn cells_for(const gp::Plan& p) {
  if (p.precision == GP_FP64) return p.dim == 2 ? gp::cells_f64_d2() : gp::cells_f64_d3();
  if (p.precision == GP_FP64_FF) return p.dim == 2 ? gp::cells_ff_d2() : gp::cells_ff_d3();
  return p.dim == 2 ? gp::cells_f32_d2() : gp::cells_f32_d3();
}

void sys_free(gp_system* s) {
  void* ptrs[] = {s->d_crow, s->d_cwin, s->d_corow, s->d_wc, s->d_o2l_hi, s->d_o2l_lo, s->r, s->p, s->q, s->dd,
                  s->z, s->ri, s->r32,
                  s->d32, s->ri32, s->p32, s->q32, s->z32, s->dinv, s->dinv32, s->part, s->d_cg};
  for (void* v : ptrs)
    if (v) cudaFree(v);
  if (s->h_res) cudaFreeHost(s->h_res);
  if (s->h_cg) cudaFreeHost(s->h_cg);
  if (s->st) cudaStreamDestroy(s->st);
}

#define SYS_CUDA(call)                                                                           \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      s->err = std::string(#call) + ": " + cudaGetErrorString(e_);                               \
      return fail(nullptr, e_ == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA, s->err);      \
    }                                                                                            \
  } while (0)

// ---- CG with its scalars on the device --------------------------------------------
// One iteration is enqueued without a host round trip: q = A p; alpha = rz / (p.q);
// d += alpha p, r -= alpha q, z = D^-1 r together with the partial sums of r.r and r.z;
// beta = rz' / rz; p = z + beta p.  A block of kCgBlock iterations is captured once as a
// CUDA graph and replayed; the host reads the scalars (converged, iterations) after
// each replay.  Iterations after convergence leave d and r unchanged (alpha = 0).
// Every reduction has a fixed grid and tree: bitwise reproducible.
struct CgScalars {
  double rz, rr, stop, alpha, beta;
  int done, iters, maxit, breakdown;
};

constexpr int kCgBlock = 16;

__global__ void __launch_bounds__(kThreads) cg_init_final(const double* __restrict__ part, const int nblk,
                                                          CgScalars* sc, double tol, int maxit) {
  __shared__ double sa[kThreads], sb[kThreads];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblk; i += kThreads) {
    a += part[i];
    b += part[nblk + i];
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double rr0 = sa[0];
    sc->rr = rr0;
    sc->rz = sb[0];
    sc->stop = tol * tol * rr0;
    sc->iters = 0;
    sc->maxit = maxit;
    sc->breakdown = 0;
    sc->alpha = sc->beta = 0.0;
    sc->done = (maxit <= 0 || !(rr0 > sc->stop) || !(rr0 > 0.0)) ? 1 : 0;
  }
}

// alpha = rz / (p.q) from the nparts partial sums of p.q
__global__ void __launch_bounds__(kThreads) cg_alpha(const double* __restrict__ part, const int nparts,
                                                     CgScalars* sc) {
  __shared__ double sh[kThreads];
  double a = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kThreads) a += part[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double pq = sh[0];
    double alpha = 0.0;
    if (!sc->done) {
      if (pq > 0.0) alpha = sc->rz / pq;
      else { sc->done = 1; sc->breakdown = 1; }
    }
    sc->alpha = alpha;
  }
}

// Four consecutive vector elements, loaded and stored as one 16-byte (FP32) or
// 32-byte (FP64) access.  The solver's vectors are its own allocations (256-byte
// aligned), so the n / 4 leading quads are aligned; the n % 4 tail is scalar.
template <typename T>
struct alignas(4 * sizeof(T)) Quad {
  T v[4];
};

// the two block sums of a thread's (a, b) partials: a into part[blockIdx.x], b into
// part[gridDim.x + blockIdx.x] (fixed tree)
__device__ __forceinline__ void block_sums2(double a, double b, double* __restrict__ part) {
  __shared__ double sa[kThreads], sb[kThreads];
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sa[0];
    part[gridDim.x + blockIdx.x] = sb[0];
  }
}

// d += alpha p, r -= alpha q, z = dinv r (when dinv), and the partial sums of r.r, r.z
template <typename T>
__global__ void __launch_bounds__(kThreads) cg_update(T* __restrict__ d, T* __restrict__ r, const T* __restrict__ p,
                                                      const T* __restrict__ q, T* __restrict__ z,
                                                      const T* __restrict__ dinv, const CgScalars* __restrict__ sc,
                                                      int64_t n, double* __restrict__ part) {
  if (sc->done) return;
  const T a = (T)sc->alpha;
  gp::IoDot<T> rr, rz;
  const int64_t tid = (int64_t)blockIdx.x * kThreads + threadIdx.x, stride = (int64_t)gridDim.x * kThreads;
  const int64_t n4 = n >> 2;
  for (int64_t j = tid; j < n4; j += stride) {
    Quad<T> dq = reinterpret_cast<const Quad<T>*>(d)[j];
    Quad<T> rq = reinterpret_cast<const Quad<T>*>(r)[j];
    const Quad<T> pq = reinterpret_cast<const Quad<T>*>(p)[j];
    const Quad<T> qq = reinterpret_cast<const Quad<T>*>(q)[j];
    Quad<T> zq;
    if (dinv) zq = reinterpret_cast<const Quad<T>*>(dinv)[j];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      dq.v[e] = fma(a, pq.v[e], dq.v[e]);
      const T ri = fma(-a, qq.v[e], rq.v[e]);
      rq.v[e] = ri;
      const T zi = dinv ? zq.v[e] * ri : ri;
      zq.v[e] = zi;
      rr.add(ri, ri);
      rz.add(ri, zi);
    }
    reinterpret_cast<Quad<T>*>(d)[j] = dq;
    reinterpret_cast<Quad<T>*>(r)[j] = rq;
    if (dinv) reinterpret_cast<Quad<T>*>(z)[j] = zq;
  }
  for (int64_t i = 4 * n4 + tid; i < n; i += stride) {
    d[i] = fma(a, p[i], d[i]);
    const T ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    T zi = ri;
    if (dinv) {
      zi = dinv[i] * ri;
      z[i] = zi;
    }
    rr.add(ri, ri);
    rz.add(ri, zi);
  }
  block_sums2(rr.value(), rz.value(), part);
}

// beta = rz' / rz, the convergence test and the iteration count
__global__ void __launch_bounds__(kThreads) cg_beta(const double* __restrict__ part, const int nblk,
                                                    CgScalars* sc) {
  __shared__ double sa[kThreads], sb[kThreads];
  __shared__ int done;
  if (threadIdx.x == 0) done = sc->done;
  __syncthreads();
  if (done) return;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblk; i += kThreads) {
    a += part[i];
    b += part[nblk + i];
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double rr = sa[0], rz1 = sb[0];
    sc->beta = rz1 / sc->rz;
    sc->rz = rz1;
    sc->rr = rr;
    sc->iters += 1;
    if (!(rr > sc->stop) || !(rr > 0.0) || sc->iters >= sc->maxit) sc->done = 1;
  }
}

// p = z + beta p
template <typename T>
__global__ void __launch_bounds__(kThreads, kVecPerSm)
cg_direction(T* __restrict__ p, const T* __restrict__ z, const CgScalars* __restrict__ sc, int64_t n) {
  if (sc->done) return;
  const T bt = (T)sc->beta;
  const int64_t tid = (int64_t)blockIdx.x * kThreads + threadIdx.x, stride = (int64_t)gridDim.x * kThreads;
  const int64_t n4 = n >> 2;
  for (int64_t j = tid; j < n4; j += stride) {
    Quad<T> pq = reinterpret_cast<const Quad<T>*>(p)[j];
    const Quad<T> zq = reinterpret_cast<const Quad<T>*>(z)[j];
#pragma unroll
    for (int e = 0; e < 4; ++e) pq.v[e] = fma(bt, pq.v[e], zq.v[e]);
    reinterpret_cast<Quad<T>*>(p)[j] = pq;
  }
  for (int64_t i = 4 * n4 + tid; i < n; i += stride) p[i] = fma(bt, p[i], z[i]);
}

// the partial sums of a.b and c.e (one per CTA each) into part
template <typename T>
__global__ void __launch_bounds__(kThreads) dot2_partial(const T* __restrict__ a, const T* __restrict__ b,
                                                         const T* __restrict__ c, const T* __restrict__ e,
                                                         int64_t n, double* __restrict__ part) {
  gp::IoDot<T> x, w;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    x.add(a[i], b[i]);
    w.add(c[i], e[i]);
  }
  block_sums2(x.value(), w.value(), part);
}

// Preconditioned CG (Jacobi when dinv is given) on A d = rhs from d = 0, until
// ||r|| <= tol * ||rhs|| or maxit iterations.
template <typename T>
gp_status cg(gp_system* s, gp_ctx* c, gp::CellsFn cells, const T* rhs, T* d, T* r, T* p, T* q, T* z,
             const T* dinv, double tol, int maxit, int* iters, int* applies) {
  const int64_t n = s->n;
  CgScalars* sc = (CgScalars*)s->d_cg;
  CgScalars* hs = (CgScalars*)s->h_cg;
  T* zz = dinv ? z : r;
  SYS_CUDA(cudaMemsetAsync(d, 0, n * sizeof(T), s->st));
  SYS_CUDA(cudaMemcpyAsync(r, rhs, n * sizeof(T), cudaMemcpyDeviceToDevice, s->st));
  if (dinv) scale_k<T><<<s->nvec, kThreads, 0, s->st>>>(z, dinv, r, n);
  SYS_CUDA(cudaMemcpyAsync(p, zz, n * sizeof(T), cudaMemcpyDeviceToDevice, s->st));
  dot2_partial<T><<<s->nblk, kThreads, 0, s->st>>>(r, r, r, zz, n, s->part);
  cg_init_final<<<1, kThreads, 0, s->st>>>(s->part, s->nblk, sc, tol, maxit);
  SYS_CUDA(cudaGetLastError());
  // one block of iterations, captured once and replayed
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  SYS_CUDA(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
  gp_status g = GP_OK;
  for (int i = 0; i < kCgBlock && g == GP_OK; ++i) {
    g = sys_apply(s, c, cells, p, q, s->st, p);   // q = A p and the partial sums of p . q
    if (g != GP_OK) break;
    cg_alpha<<<1, kThreads, 0, s->st>>>(s->part, s->nparts, sc);
    cg_update<T><<<s->nblk, kThreads, 0, s->st>>>(d, r, p, q, z, dinv, sc, n, s->part);
    cg_beta<<<1, kThreads, 0, s->st>>>(s->part, s->nblk, sc);
    cg_direction<T><<<s->nvec, kThreads, 0, s->st>>>(p, zz, sc, n);
  }
  const cudaError_t ec = cudaStreamEndCapture(s->st, &graph);
  if (g != GP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return g;
  }
  SYS_CUDA(ec);
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  int blocks = 0;
  while (e == cudaSuccess) {
    e = cudaMemcpyAsync(hs, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess || hs->done) break;
    e = cudaGraphLaunch(exec, s->st);
    ++blocks;
  }
  if (exec) cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  SYS_CUDA(e);
  *iters = hs->iters;
  *applies += blocks * kCgBlock;
  return GP_OK;
}

}  // namespace

extern "C" {

gp_status gp_system_create(gp_ctx* hi, gp_ctx* lo, gp_system** out) {
  if (!out) return fail(nullptr, GP_EINVAL, "null output pointer");
  *out = nullptr;
  if (!hi || !hi->on_device) return fail(nullptr, GP_EINVAL, "the high-precision context must be on a device");
  if (hi->plan.precision == GP_FP32) return fail(nullptr, GP_EINVAL, "hi must be GP_FP64 or GP_FP64_FF");
  if (hi->plan.partitioned || (lo && lo->plan.partitioned))
    return fail(nullptr, GP_EUNSUPPORTED, "the model system is built for whole meshes only");
  if (hi->no_scratch || (lo && lo->no_scratch))
    return fail(nullptr, GP_EINVAL, "the model system needs contexts created with no_scratch = 0");
  // the system's fused gather reads the face kernel's outputs W_F: give brick-path contexts one
  if (gpi::ensure_face_outputs(hi) != GP_OK) return fail(nullptr, GP_ENOMEM, hi->err);
  if (lo && gpi::ensure_face_outputs(lo) != GP_OK) return fail(nullptr, GP_ENOMEM, lo->err);
  if (lo) {
    if (!lo->on_device || lo->device != hi->device) return fail(nullptr, GP_EINVAL, "lo must be on hi's device");
    if (lo->plan.precision != GP_FP32) return fail(nullptr, GP_EINVAL, "lo must be GP_FP32");
    const gp::Plan &a = hi->plan, &b = lo->plan;
    if (a.dim != b.dim || a.n != b.n || a.k != b.k || a.n_active != b.n_active || a.num_faces() != b.num_faces() ||
        a.h != b.h)
      return fail(nullptr, GP_EINVAL, "hi and lo must describe the same mesh, degree and level set");
  }
  gp_system* s = new (std::nothrow) gp_system();
  if (!s) return fail(nullptr, GP_ENOMEM, "host allocation failed");
  s->hi = hi;
  s->lo = lo;
  s->device = hi->device;
  s->n = hi->plan.n_active;
  DeviceGuard dg(s->device);
  gp::Plan& p = hi->plan;
  if (p.crow.empty() && p.n_active > 0) gp::build_cell_table(p);
  if (!gp::check_cell_table(p)) {
    delete s;
    return fail(nullptr, GP_EINVAL, "internal: cell table outside the active DoFs");
  }
  // the cell kernel applies M^ and S^ through their even / odd halves, which needs
  // A[k-p][k-q] = A[p][q] (Gauss-Lobatto nodes symmetric about the cell centre)
  {
    const int N = p.k + 1;
    double dev = 0.0, mx = 0.0;
    for (int a = 0; a < N; ++a)
      for (int b = 0; b < N; ++b)
        for (const std::vector<double>* A : {&p.mass, &p.stiff}) {
          dev = std::max(dev, std::fabs((*A)[a * N + b] - (*A)[(N - 1 - a) * N + N - 1 - b]));
          mx = std::max(mx, std::fabs((*A)[a * N + b]));
        }
    if (!(dev <= 1e-13 * mx)) {
      delete s;
      return fail(nullptr, GP_EINVAL, "internal: reference mass / stiffness not centrosymmetric");
    }
  }
  s->cells_hi = cells_for(p);
  if (lo) s->cells_lo = cells_for(lo->plan);
  auto cleanup = [&](cudaError_t e) {
    std::string m = std::string("system setup: ") + cudaGetErrorString(e);
    sys_free(s);
    delete s;
    return fail(nullptr, e == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA, m);
  };
  cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  s->nblk = kDotPerSm * std::max(sms, 1);
  s->nvec = kVecPerSm * std::max(sms, 1);
  auto upload = [](int32_t** dst, const std::vector<int32_t>& v) -> cudaError_t {
    if (v.empty()) return cudaSuccess;
    cudaError_t r = cudaMalloc((void**)dst, v.size() * sizeof(int32_t));
    if (r == cudaSuccess) r = cudaMemcpy(*dst, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    return r;
  };
  if (e == cudaSuccess) e = upload(&s->d_crow, p.crow);
  if (e == cudaSuccess) e = upload(&s->d_cwin, p.cwin);
  if (e == cudaSuccess) e = upload(&s->d_corow, p.corow);
  if (e == cudaSuccess) e = upload(&s->d_o2l_hi, gp::owner_lift_index(p, hi->plan));
  if (e == cudaSuccess && lo) e = upload(&s->d_o2l_lo, gp::owner_lift_index(p, lo->plan));
  const size_t nodes = (size_t)gp::ipow_host(p.k + 1, p.dim);
  if (e == cudaSuccess && p.ncact > 0) e = cudaMalloc(&s->d_wc, (size_t)p.ncact * nodes * 8);
  s->ct.crow = s->d_crow;
  s->ct.ncact = (int32_t)p.ncact;
  s->ct.cwin = s->d_cwin;
  s->ct.corow = s->d_corow;
  s->ct.ncown = (int32_t)p.ncown;
  s->ct.n_active = (int32_t)p.n_active;
  s->ct.wc = s->d_wc;
  const size_t n8 = (size_t)std::max<int64_t>(s->n, 1) * 8, n4 = (size_t)std::max<int64_t>(s->n, 1) * 4;
  if (e == cudaSuccess) e = cudaMalloc(&s->r, n8);
  if (e == cudaSuccess) e = cudaMalloc(&s->p, n8);
  if (e == cudaSuccess) e = cudaMalloc(&s->q, n8);
  if (e == cudaSuccess) e = cudaMalloc(&s->dd, n8);
  if (e == cudaSuccess) e = cudaMalloc(&s->z, n8);
  if (e == cudaSuccess) e = cudaMalloc(&s->ri, n8);
  if (e == cudaSuccess) e = cudaMalloc(&s->dinv, n8);
  if (e == cudaSuccess && lo) e = cudaMalloc(&s->z32, n4);
  if (e == cudaSuccess && lo) e = cudaMalloc(&s->dinv32, n4);
  if (e == cudaSuccess && s->n > 0) {
    // Jacobi: inverse diagonal of the model system, computed on the host in FP64
    std::vector<double> diag;
    gp::build_diagonal(p, diag);
    std::vector<double> inv(diag.size());
    std::vector<float> inv32(diag.size());
    for (size_t i = 0; i < diag.size(); ++i) {
      inv[i] = diag[i] > 0 ? 1.0 / diag[i] : 1.0;
      inv32[i] = (float)inv[i];
    }
    e = cudaMemcpy(s->dinv, inv.data(), n8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && lo) e = cudaMemcpy(s->dinv32, inv32.data(), n4, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && lo) e = cudaMalloc(&s->r32, n4);
  if (e == cudaSuccess && lo) e = cudaMalloc(&s->d32, n4);
  if (e == cudaSuccess && lo) e = cudaMalloc(&s->ri32, n4);
  if (e == cudaSuccess && lo) e = cudaMalloc(&s->p32, n4);
  if (e == cudaSuccess && lo) e = cudaMalloc(&s->q32, n4);
  s->nparts = (int)gp::gather_ctas(p.dim, p.k, p.ncown);
  if (e == cudaSuccess)
    e = cudaMalloc(&s->part, (size_t)std::max<int64_t>(2 * s->nblk + 1, s->nparts) * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_res, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_cg, sizeof(CgScalars));
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_cg, sizeof(CgScalars));
  if (e != cudaSuccess) return cleanup(e);
  *out = s;
  return GP_OK;
}

gp_status gp_system_apply(gp_system* s, int which, const void* x, void* y, void* stream) {
  if (!s) return fail(nullptr, GP_EINVAL, "null system");
  gp_ctx* c = which == 0 ? s->hi : s->lo;
  if (!c) return fail(nullptr, GP_EINVAL, "this system has no FP32 operator");
  if (s->n > 0 && (!x || !y || x == y)) return fail(nullptr, GP_EINVAL, "bad x or y");
  if (s->n == 0) return GP_OK;
  DeviceGuard dg(s->device);
  return sys_apply(s, c, which == 0 ? s->cells_hi : s->cells_lo, x, y, (cudaStream_t)stream);
}

gp_status gp_system_cells(gp_system* s, int which, double mass_weight, double stiff_weight, const void* x, void* y,
                          void* stream) {
  if (!s) return fail(nullptr, GP_EINVAL, "null system");
  gp_ctx* c = which == 0 ? s->hi : s->lo;
  if (!c) return fail(nullptr, GP_EINVAL, "this system has no FP32 operator");
  if (s->n > 0 && (!x || !y || x == y)) return fail(nullptr, GP_EINVAL, "bad x or y");
  if (s->n == 0) return GP_OK;
  DeviceGuard dg(s->device);
  const gp::Plan& p = c->plan;
  const cudaStream_t st = (cudaStream_t)stream;
  // the gather overwrites every active DoF (each is a node of an active cell)
  const cudaError_t e = (which == 0 ? s->cells_hi : s->cells_lo)(p.k, x, y, s->ct, p.mass.data(), p.stiff.data(),
                                                                 p.h, mass_weight, stiff_weight, 0, 1, st);
  if (e != cudaSuccess) return fail(c, GP_ECUDA, std::string("cell kernels: ") + cudaGetErrorString(e));
  return GP_OK;
}

gp_status gp_system_solve(gp_system* s, const double* b, double* u, const gp_solve_opts* o, gp_solve_stats* stats) {
  if (!s || !b || !u || !o || !stats) return fail(nullptr, GP_EINVAL, "null argument");
  if (o->mode == 0 && !s->lo) return fail(nullptr, GP_EINVAL, "defect correction needs the FP32 operator");
  std::memset(stats, 0, sizeof(*stats));
  DeviceGuard dg(s->device);
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = s->n;
  const bool jac = o->precond == 1;
  gp_status g = GP_OK;
  // outer loop on the true FP64 residual r = b - A_hi u; the correction A d = r is
  // solved by FP32 PCG (mode 0, to inner_rtol) or FP64 PCG (mode 1, to what rtol needs)
  SYS_CUDA(cudaMemsetAsync(u, 0, n * sizeof(double), s->st));
  SYS_CUDA(cudaMemcpyAsync(s->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
  double bb = 0.0;
  SYS_CUDA(dot<double>(s, b, b, &bb));
  const double nb = std::sqrt(bb);
  int outer = 0;
  double rn = nb;
  while (outer < o->max_outer) {
    double rr = 0.0;
    SYS_CUDA(dot<double>(s, s->r, s->r, &rr));
    rn = std::sqrt(rr);
    if (rn <= o->rtol * nb || rr == 0.0) break;
    int it = 0, applies = 0;
    if (o->mode == 0) {
      to32_k<<<s->nvec, kThreads, 0, s->st>>>(s->r32, s->r, n);
      g = cg<float>(s, s->lo, s->cells_lo, s->r32, s->d32, s->ri32, s->p32, s->q32, s->z32,
                    jac ? s->dinv32 : nullptr, o->inner_rtol, o->max_inner, &it, &applies);
      if (g != GP_OK) return g;
      stats->lo_applies += applies;
      add32_k<<<s->nvec, kThreads, 0, s->st>>>(u, s->d32, n);
    } else {
      const double tol = std::max(0.5 * o->rtol * nb / rn, 1e-15);
      g = cg<double>(s, s->hi, s->cells_hi, s->r, s->dd, s->ri, s->p, s->q, s->z, jac ? s->dinv : nullptr, tol,
                     o->max_inner, &it, &applies);
      if (g != GP_OK) return g;
      stats->hi_applies += applies;
      add64_k<<<s->nvec, kThreads, 0, s->st>>>(u, s->dd, n);
    }
    stats->inner += it;
    g = sys_apply(s, s->hi, s->cells_hi, u, s->q, s->st);
    if (g != GP_OK) return g;
    stats->hi_applies++;
    resid_k<<<s->nvec, kThreads, 0, s->st>>>(s->r, b, s->q, n);
    ++outer;
  }
  double rr = 0.0;
  SYS_CUDA(dot<double>(s, s->r, s->r, &rr));
  stats->outer = outer;
  stats->rel_residual = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return GP_OK;
}

void gp_system_destroy(gp_system* s) {
  if (!s) return;
  DeviceGuard dg(s->device);
  if (s->st) cudaStreamSynchronize(s->st);
  sys_free(s);
  delete s;
}

}  // extern "C"
