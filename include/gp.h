/*
 * gp.h -- C ABI of the GB300 matrix-free ghost-penalty operator.
 *
 * Operation (Sec. 2.2, ghost penalty g_h; Sec. 2.4, tensor-product face
 * matrix; Sec. 2.5.1, face loop of the operator application):
 *
 *   y = G x,   G = sum_{F in F_h} sum_{j=1..k} c_j h^{2j-1} (integral over F of
 *                  [d_n^j u] [d_n^j v]),
 *
 * on an axis-aligned Cartesian mesh of 2D squares / 3D cubes of edge h with
 * continuous FE_Q(k) elements on Gauss-Lobatto points, for the faces F_h
 * between two active cells of which at least one is cut by the level set
 * (phi > 0 inside).  Per face, the matrix factorises as
 * h^{d-2} (M^ x ... x G^) with the 1D reference mass M^ along the tangential
 * directions and the 1D penalty G^ = sum_j c_j g_j g_j^T along the normal
 * (Eq. of G_F = M^h x M^h x G^h_k and its h-scaling).
 *
 * Conventions shared by every call
 *   - Vectors live on the active DoFs: the FE_Q lattice nodes (n*k+1 per
 *     axis) that belong to at least one active cell, numbered
 *     lexicographically with x fastest, then compacted
 *     (gp_active_dof_coords returns their coordinates).
 *   - x and y are caller-owned DEVICE pointers to contiguous arrays of
 *     n_active elements (double for GP_FP64 and GP_FP64_FF, float for GP_FP32), on the
 *     device that was current during gp_setup.  x and y must not alias.
 *   - stream is a cudaStream_t (0 = legacy default stream).  Calls only
 *     enqueue work; they do not synchronise.
 *   - Every call returns a gp_status and never aborts.  On error,
 *     gp_last_error() gives a message for that context (or for the calling
 *     thread when ctx is NULL).
 *   - A context is not thread-safe: one host thread (or external locking)
 *     per context.  Concurrent applies on different streams that share a
 *     context race on its scratch buffer.
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gp_ctx gp_ctx;

typedef enum {
  GP_OK = 0,
  GP_EINVAL = 1,        /* bad argument (null pointer, size, degree, mesh) */
  GP_ENOMEM = 2,        /* host or device allocation failed */
  GP_ECUDA = 3,         /* a CUDA runtime call failed (message has the error) */
  GP_EDEVICE = 4,       /* no usable CUDA device, or context built host-only */
  GP_EUNSUPPORTED = 5   /* valid request outside this build (e.g. k > 8) */
} gp_status;

/* Arithmetic of the operator.  GP_FP64: x, y double, FP64 arithmetic.
 * GP_FP32: x, y float, FP32 arithmetic.  GP_FP64_FF: x, y double, computed in
 * float-float pairs (hi + lo, about 2^-48 relative per operation) on the FP32
 * pipes.  The pairs have the exponent range of float, not of double:
 *   - FP64-level accuracy (1e-12 relative to the largest output) holds when every
 *     non-zero |x_i| lies in [2^-97, 2^127) and every output |y_i| stays below
 *     2^127 (about 1.7e38); besides that relative error, every value carries an
 *     absolute error of up to a few 2^-126 (about 1e-38: float cannot hold the low
 *     part of a smaller value), which matters only for outputs below about 2^-80;
 *   - an entry with 2^-126 <= |x_i| < 2^-97 keeps only its leading 24 bits (the
 *     low float would be subnormal), |x_i| < 2^-126 reads as 0, and |x_i| >= 2^128
 *     reads as infinity (y is then not finite on the DoFs its faces reach);
 *   - the operator is linear: scale x by a power of two into that range (and y
 *     back) when the data lie outside it, or use GP_FP64.
 * gp_setup refuses (GP_EINVAL) a GP_FP64_FF context whose per-order scale factors
 * c_j h^(d-2) lie outside [2^-90, 2^90]. */
enum { GP_FP64 = 0, GP_FP32 = 1, GP_FP64_FF = 2 };

/* level-set kinds; phi > 0 inside the domain (Sec. 2) */
enum {
  GP_LS_BALLS = 1,      /* union of balls, phi = max_b (r_b - |x - c_b|) */
  GP_LS_GYROID = 2,     /* phi = sin x cos y + sin y cos z + sin z cos x - iso (3D) */
  GP_LS_CALLBACK = 3,   /* user function, sampled with a Lipschitz margin */
  GP_LS_CONST = 4       /* phi = value everywhere */
};

typedef double (*gp_levelset_fn)(const double* x, void* user);

/* Uniform Cartesian mesh of n[a] cells on [lo[a], hi[a]], a < dim; the cell
 * edge h = (hi[a]-lo[a])/n[a] must be the same on every axis (Sec. 2: squares
 * or cubes of size h). */
typedef struct {
  int dim;              /* 2 or 3 */
  int n[3];
  double lo[3];
  double hi[3];
} gp_mesh;

typedef struct {
  int kind;                 /* GP_LS_* */
  int nballs;               /* GP_LS_BALLS */
  const double* centers;    /* nballs x 3 (z ignored in 2D), host memory */
  const double* radii;      /* nballs, host memory */
  double iso;               /* GP_LS_GYROID */
  double value;             /* GP_LS_CONST */
  gp_levelset_fn fn;        /* GP_LS_CALLBACK */
  void* user;
  double lipschitz;         /* GP_LS_CALLBACK: bound on |grad phi| */
  int samples;              /* sub-intervals per cell edge for sampled kinds (<=0: 4) */
} gp_levelset;

/* Options of gp_setup.  Zero-initialise the struct (memset, or = {0} in C) and set the fields you
 * need: 0 selects the default of every field (precision GP_FP64, device 0, the whole mesh, the
 * ghost penalty, automatic kernel path, ...) except degree, which must be set, and gamma, whose 0
 * gives G = 0 unless weights are given. */
typedef struct {
  int degree;               /* k, 1 <= k <= 8 */
  int nweights;             /* 0, or k: per-order weights c_1..c_k */
  const double* weights;    /* NULL -> c_j = gamma for every order j */
  double gamma;             /* default weight */
  int precision;            /* GP_FP64, GP_FP32 or GP_FP64_FF */
  int all_faces;            /* 1: penalise every interior face of the active mesh */
  int device;               /* CUDA device ordinal; -1 = build the host plan only */
  int part_lo, part_hi;     /* 0, 0: the whole mesh.  Otherwise this context is the slab
                               partition of cell layers [part_lo, part_hi) along the last
                               axis (y in 2D, z in 3D); see gp_partition_info */
  int stabilization;        /* GP_STAB_GHOST (0, the ghost penalty) or GP_STAB_MACRO */
  int no_scratch;           /* 1: allocate no face-output scratch; only gp_apply_noalloc can
                               apply the context (the other applies, the autotuner, batches and
                               the model system return GP_EINVAL) */
  int kernel_path;          /* GP_PATH_AUTO (0), GP_PATH_FACE_LIFT or GP_PATH_BRICK */
  int brick_smem;           /* brick path: shared-memory budget in bytes that picks the brick
                               shape (0: 100 KB) */
  int slabs;                /* face + lift path: 0 or 1 = one face and one lift launch; n > 1 =
                               a pipeline of about n slabs along the last axis (a face and a
                               lift launch per slab, so that a slab's face outputs are still in
                               L2 when its lift reads them).  Results are identical; on the
                               128^3 gyroid (k = 4) every n > 1 measured slower on GB300. */
} gp_opts;

/* Kernel paths of gp_apply / gp_apply_add (same operator, same accuracy, rounding may differ):
 *   GP_PATH_FACE_LIFT  a face kernel writes every face output W_F to a buffer of
 *                      n_faces (2k+1)(k+1)^(d-1) values and a lift kernel gathers them per DoF;
 *   GP_PATH_BRICK      the mesh is cut into bricks of cells; one CTA per brick stages the x
 *                      blocks of its involved cells in shared memory, evaluates the faces of
 *                      its cells, sums the outputs per DoF in shared memory and writes y once
 *                      (DoFs on the boundary planes between bricks go through a small buffer of
 *                      partial sums and a second kernel); GP_EUNSUPPORTED from gp_setup when no
 *                      brick shape fits the shared-memory budget;
 *   GP_PATH_AUTO       the path this build measured fastest on the benchmark workloads:
 *                      face + lift.
 * Both are deterministic: repeated applies are bitwise identical. */
enum { GP_PATH_AUTO = 0, GP_PATH_FACE_LIFT = 1, GP_PATH_BRICK = 2 };

/* Stabilisations.  GP_STAB_MACRO is the macro-patch alternative the paper names next to the
 * ghost penalty (Sec. 2.2): per ghost face, gamma times the integral over each of its two
 * cells of the square of (the function there - the extension of the neighbour cell's
 * polynomial into it).  On the Cartesian patch it has the same Kronecker form,
 * gamma h^d (M^ x ... x G^mp), with a 1D matrix G^mp of rank k; weights and nweights are
 * ignored. */
enum { GP_STAB_GHOST = 0, GP_STAB_MACRO = 1 };

/* Classify cells, collect the ghost faces, number the active DoFs, build the
 * 1D matrices in FP64 and upload the face tables (Sec. 2, Sec. 2.4, Sec. 2.7).
 * mesh, ls and opts are read during the call only.  *out receives a new
 * context owned by the caller (release with gp_destroy). */
gp_status gp_setup(const gp_mesh* mesh, const gp_levelset* ls, const gp_opts* opts,
                   gp_ctx** out);

/* Release a context and its device memory.  NULL is ignored. */
void gp_destroy(gp_ctx* ctx);

/* Sizes: active DoFs, ghost faces, DoFs touched by some ghost face, and
 * number of cells in each class (outside, cut, inside). */
gp_status gp_num_active_dofs(const gp_ctx* ctx, int64_t* n);
gp_status gp_num_ghost_faces(const gp_ctx* ctx, int64_t* nf);
gp_status gp_num_touched_dofs(const gp_ctx* ctx, int64_t* n);
gp_status gp_cell_counts(const gp_ctx* ctx, int64_t counts[3]);

/* Host copies of the plan, for checks.  Caller-owned host buffers:
 *   xyz   n_active * dim doubles, coordinates of the active DoFs in order;
 *   axis / cell  nf entries: normal axis and lexicographic (x fastest)
 *          index of the lower cell of every ghost face, in face order;
 *   cls   n_cells int8: 0 outside, 1 cut, 2 inside (lexicographic). */
gp_status gp_active_dof_coords(const gp_ctx* ctx, double* xyz);
gp_status gp_ghost_faces(const gp_ctx* ctx, int32_t* axis, int64_t* cell);
gp_status gp_cell_classes(const gp_ctx* ctx, int8_t* cls);

/* ---- Slab partitions (Sec. 2.7 and Algorithm 1: distributed evaluation) ----
 *
 * The paper distributes the cells over MPI ranks with a weighted load balance,
 * gives a face shared by two ranks to the lower rank, imports the ghost values
 * of u before the face loop and adds the ghost contributions of w afterwards.
 * Here a partition is a slab of whole cell layers [part_lo, part_hi) along the
 * last axis (y in 2D, z in 3D), so that every exchange is one contiguous block:
 *   - its faces are the ghost faces whose lower cell lies in the slab (the face
 *     between two slabs belongs to the lower one);
 *   - its vector holds, in global order, the active DoFs on the lattice planes
 *     [part_lo k, min(part_hi + 1, n) k] of the last axis (one cell of halo above);
 *   - entries [0, n_owned) are owned; [n_owned, n_local) is the halo, equal to the
 *     first n_lower entries of the partition above; the first n_lower entries are
 *     the halo of the partition below (n_lower = 0 for the first slab).
 * One application: copy x[0, n_lower) of every partition to the halo of the one
 * below, apply (gp_apply), then add y[n_owned, n_local) of every partition into
 * y[0, n_lower) of the one above.  y[0, n_owned) is then the global result.  A slab
 * with a neighbour on both sides needs at least two layers (GP_EINVAL otherwise).
 * The model system (gp_system_create) takes whole meshes only. */
typedef struct {
  int32_t layer_lo, layer_hi;  /* cell layers of the slab */
  int64_t offset;              /* global index of local entry 0 */
  int64_t n_local;             /* local vector length (== gp_num_active_dofs) */
  int64_t n_owned;             /* owned entries [0, n_owned) */
  int64_t n_lower;             /* entries shared with the partition below */
  int64_t n_global;            /* active DoFs of the whole mesh */
} gp_partition;

/* Partition layout of a context (a whole-mesh context reports one slab with
 * offset 0 and n_owned == n_local == n_global). */
gp_status gp_partition_info(const gp_ctx* ctx, gp_partition* out);

/* Weighted slab partition for nparts processes: cell weight 0 outside, 1 inside,
 * k^(d-1) cut (Sec. 2.7).  bounds (host, nparts + 1 entries, caller-owned)
 * receives layer boundaries 0 = b_0 < ... < b_nparts = n: b_p is the first layer
 * boundary where the prefix weight reaches p / nparts of the total, clamped so
 * that every slab has at least two layers.  Needs n >= 2 nparts (GP_EINVAL
 * otherwise).  opts->part_lo / part_hi and opts->device are ignored. */
gp_status gp_partition_slabs(const gp_mesh* mesh, const gp_levelset* ls, const gp_opts* opts,
                             int nparts, int32_t* bounds);

/* ---- Tile shapes and the autotuner (no counterpart in the paper) ----
 *
 * The face kernel runs faces_per_cta faces per CTA (faces_per_cta * (k+1)^(d-1)
 * threads, one per normal line); the lift kernel runs lift_threads threads per CTA
 * over the rows of lift_cells_per_cta owner cells.  A field 0 means the default
 * (about 256 threads, one row per thread).  Limits: at most 512 threads per CTA,
 * lift_threads a multiple of 32, and at most 46 KB of dynamic shared memory per CTA
 * (GP_EINVAL otherwise).  The shape changes the speed, never the result: every
 * DoF is summed in the same fixed order. */
typedef struct {
  int faces_per_cta;
  int lift_cells_per_cta;
  int lift_threads;
} gp_tiles;

/* The context's current shape (defaults resolved). */
gp_status gp_get_tiles(const gp_ctx* ctx, gp_tiles* out);
/* Sets the context's shape (checked against the limits above). */
gp_status gp_set_tiles(gp_ctx* ctx, const gp_tiles* tiles);

/* Times every candidate shape of the face kernel (about 64 to 512 threads per
 * CTA) and of the lift kernel (64 to 512 threads, one or two rows per thread)
 * on this context's own tables: reps launches each, L2 flushed before every
 * timed launch, CUDA events on a private stream.  Keeps the fastest face shape
 * and the fastest lift shape in the context and records them in a
 * process-wide table keyed by (device, d, k, precision), which gp_setup reads
 * for every new context.  best (may be NULL) receives the shape, ms (may be
 * NULL, 2 doubles) the mean face and lift kernel times in milliseconds.
 * Allocates and frees two vectors and a 256 MB flush buffer; synchronises. */
gp_status gp_autotune(gp_ctx* ctx, int reps, gp_tiles* best, double* ms);

/* The process-wide table: record a shape (e.g. one read back from a cache
 * file) or look one up (GP_EINVAL if absent). */
gp_status gp_tiles_record(int device, int dim, int degree, int precision, const gp_tiles* tiles);
gp_status gp_tiles_lookup(int device, int dim, int degree, int precision, gp_tiles* out);

/* The FP64 1D reference matrices of this context (Sec. 2.4, M^1 and G^1_k):
 *   mass  (k+1)^2 doubles, M^[a][b] = integral_0^1 phi_a phi_b;
 *   jumps k*(2k+1) doubles, g_j[b] = jump of the j-th derivative of patch
 *         basis function b across the face of the patch [0,1] u [1,2];
 *   scale k doubles, s_j = c_j h^{d-2} (the one FP64 factor per order). */
gp_status gp_reference_1d(const gp_ctx* ctx, double* mass, double* jumps, double* scale);

/* y = G x (y is overwritten on every active DoF).  Stream-ordered: work launched
 * normally on the same stream afterwards sees the complete y.  The second kernel lets
 * programmatic dependents start early (programmatic dependent launch): a kernel of the
 * caller launched with programmatic stream serialization right after this call must
 * wait for its prerequisite grid (griddepcontrol.wait) before it reads y. */
gp_status gp_apply(gp_ctx* ctx, const void* x, void* y, void* stream);

/* y += G x (only DoFs touched by a ghost face are read and written). */
gp_status gp_apply_add(gp_ctx* ctx, const void* x, void* y, void* stream);

/* Allocation-free y = G x (no counterpart in the paper).  For callers that
 * cannot allocate device memory when they apply the operator: code whose device
 * memory is owned by another allocator (a framework pool that reserves the GPU
 * up front), or latency-critical loops where a cudaMalloc/cudaFree pair would
 * synchronise the device.  Same result as gp_apply, but the face outputs go to a
 * fixed scratch array of GP_NOALLOC_SCRATCH_BYTES compiled into the library (every
 * GPU that loads the library holds it until the process exits) instead of the
 * context's buffer.  The call allocates nothing and records no trace events.
 *   - The scratch must hold n_faces * (2k+1) * (k+1)^(d-1) values (4 bytes for
 *     GP_FP32, 8 otherwise); larger problems get GP_EINVAL and a message.
 *   - The first call on a device looks the array's device address up with
 *     cudaGetSymbolAddress and keeps it for the life of the process; make that
 *     first call before any stream capture.  A device reset (cudaDeviceReset)
 *     invalidates the kept address: do not call gp_apply_noalloc after one.
 *   - A context created with gp_opts.no_scratch = 1 holds no face-output buffer
 *     of its own, so that a caller who only uses this entry point pays for no
 *     device allocation beyond the plan's tables.
 *   - All calls share the array and it keeps the last call's contents (every
 *     value the operator reads is rewritten first, so nothing needs clearing);
 *     calls whose kernels overlap on the GPU race on it.
 * x, y, stream and errors as for gp_apply. */
#define GP_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
gp_status gp_apply_noalloc(gp_ctx* ctx, const void* x, void* y, void* stream);

/* Kernel path of a context: *path receives GP_PATH_BRICK or GP_PATH_FACE_LIFT; on the brick
 * path bdim (3 ints, may be NULL) receives the brick shape in cells and counts (3 int64, may
 * be NULL) the bricks that hold faces, the plane nodes shared by several bricks and the bytes
 * of the partial sums (the path's scratch).  On the face + lift path bdim receives zeros and
 * counts the slabs of gp_apply's launch pipeline (1: one face and one lift launch), 0 and the
 * bytes of the face outputs. */
gp_status gp_kernel_path(const gp_ctx* ctx, int* path, int32_t* bdim, int64_t* counts);

/* End-to-end form with HOST buffers (n_active elements of the context's precision each):
 * y = G x, waiting for completion.  A page-locked x (cudaHostAlloc, cudaHostRegister, torch
 * pin_memory) is read by a gather kernel on the DoFs some face patch touches only (the only
 * entries the face kernel reads); other host memory is copied whole.  y is computed in a device
 * buffer owned by the context; a page-locked y comes back in chunks on a second stream while the
 * apply runs as a pipeline of up to 16 slabs (8 in FP32; each chunk as soon as the slabs that write it are
 * done; x is then gathered slab by slab on a third stream, each slab's face launch waiting for
 * its part), any other y in one copy at the end.  The device buffers, streams and events belong
 * to ctx: calls on one context must not overlap. */
gp_status gp_apply_host(gp_ctx* ctx, const void* x_host, void* y_host, void* stream);

/* Bytes the last gp_apply_host of ctx moved from host to device and from device to host. */
gp_status gp_apply_host_bytes(const gp_ctx* ctx, int64_t* h2d, int64_t* d2h);

/* Several independent problems, nrhs right-hand sides each (the batched workload
 * of many meshes of uneven n, k and geometry): x[p] and y[p] point to nrhs
 * contiguous vectors of n_active(p) elements (layout [nrhs][n_active]).  All
 * contexts must share one precision and device.  y[p] is overwritten.
 * The first call with a given list of contexts and nrhs builds a gp_batch for it
 * (gp_batch_create below: device allocations and a CUDA graph capture, so make
 * that first call outside any stream capture) and keeps it until one of the
 * contexts is destroyed; every call then replays that batch's graph once
 * (gp_batch_apply).  gp_apply_batched_info returns the number of graph replays
 * made so far for the list (GP_EINVAL if it was never applied). */
gp_status gp_apply_batched(gp_ctx* const* ctxs, int nprob, int nrhs,
                           const void* const* x, void* const* y, void* stream);
gp_status gp_apply_batched_info(gp_ctx* const* ctxs, int nprob, int nrhs, int64_t* graph_launches);

/* Kernel tracing.  While enabled, every apply on ctx records CUDA events on
 * its stream before the jump kernel, between the two kernels and after the
 * lift kernel (Sec. 3.1 times each component of the operator separately).
 * gp_profile_read waits for the recorded events and returns the summed
 * device time of each kernel in milliseconds (ms[0] jump, ms[1] lift) and the
 * number of traced applies since the last enable; enabling again resets. */
gp_status gp_profile_enable(gp_ctx* ctx, int enable);
gp_status gp_profile_read(gp_ctx* ctx, double ms[2], int64_t* calls);

/* Batched form: several independent problems, nrhs right-hand sides each, replayed
 * as one CUDA graph (the batched workload of many meshes of uneven n, k and
 * geometry).  gp_batch_create groups the problems by (dimension, degree,
 * arithmetic, stabilisation); every (problem, right-hand side) pair gets its own face-output
 * buffer, and one face launch plus one lift launch per group cover all pairs.  The
 * graph also holds the host-to-device copy of the table of x / y pointers, so each
 * gp_batch_apply writes that table (pinned host memory) and launches the graph.
 *   ctxs: contexts on one device; they must outlive the batch.
 *   x[p], y[p]: device arrays of nrhs * n_active(p) elements, layout [nrhs][n_active];
 *   y[p] is overwritten.  An apply waits for the apply issued two calls earlier
 *   (the pointer tables are double-buffered). */
typedef struct gp_batch gp_batch;
gp_status gp_batch_create(gp_ctx* const* ctxs, int nprob, int nrhs, gp_batch** out);
gp_status gp_batch_apply(gp_batch* batch, const void* const* x, void* const* y, void* stream);
gp_status gp_batch_info(const gp_batch* batch, int64_t* ngroups, int64_t* scratch_bytes);
void gp_batch_destroy(gp_batch* batch);

/* Model SPD system (M_active + K_active + G) u = b: the mass and Laplace
 * stiffness of every active cell integrated over the whole cell (the interior-cell
 * evaluation of Sec. 2.5.2 applied to all active cells; no cut quadrature) plus the
 * ghost penalty.  hi: a GP_FP64 or GP_FP64_FF context; lo: a GP_FP32 context of the
 * same mesh, degree and level set, or NULL.  Both must outlive the system. */
typedef struct gp_system gp_system;
gp_status gp_system_create(gp_ctx* hi, gp_ctx* lo, gp_system** out);

/* y = A x with the hi (which = 0; x, y double) or lo (which = 1; float) operator,
 * y overwritten.  Three launches on `stream`: the ghost-penalty face kernel, the cell
 * kernel, and one gather that adds per node the ghost-face outputs and then the cell
 * outputs in a fixed order (no atomics: bitwise reproducible) and writes y once. */
gp_status gp_system_apply(gp_system* sys, int which, const void* x, void* y, void* stream);

/* y = (mass_weight M_active + stiff_weight K_active) x with the hi (which = 0) or lo
 * (which = 1) arithmetic, y overwritten: the interior-cell evaluation of Sec. 2.5.2 on
 * every active cell (mass 0, stiffness 1 is the Laplace operator of the paper's cell loop,
 * Algorithm 1).  Same argument rules as gp_system_apply. */
gp_status gp_system_cells(gp_system* sys, int which, double mass_weight, double stiff_weight, const void* x,
                          void* y, void* stream);

/* Solvers (the paper leaves the solver open, Sec. 1).  mode 0, defect correction:
 * r = b - A_hi u and all updates in FP64; each correction A_lo d = r solved by CG
 * with the FP32 operator to relative residual inner_rtol; its inner products sum
 * the exact products of the FP32 entries with compensated float-float sums and
 * combine the per-thread sums in FP64 (about FP64 accuracy, no FP64 work per element)
 * (at most max_inner iterations); at most max_outer corrections; stops when
 * ||b - A_hi u|| <= rtol ||b||.  mode 1: the same outer loop with FP64 CG on the hi
 * operator as the inner solver (tolerance chosen to reach rtol), i.e. plain FP64 CG
 * with a true-residual check.  precond 1: Jacobi (diag(A) computed in FP64 on the
 * host), 0: none.  b, u: device arrays of n_active doubles; u is overwritten (the
 * solve starts from u = 0).  The call synchronises. */
typedef struct {
  double rtol;
  double inner_rtol;
  int max_outer;
  int max_inner;
  int mode;
  int precond;
} gp_solve_opts;
typedef struct {
  int outer;            /* outer corrections */
  int inner;            /* CG iterations in total */
  int hi_applies;
  int lo_applies;
  double rel_residual;  /* ||b - A_hi u|| / ||b|| at return */
  double seconds;
} gp_solve_stats;
gp_status gp_system_solve(gp_system* sys, const double* b, double* u, const gp_solve_opts* opts,
                          gp_solve_stats* stats);
void gp_system_destroy(gp_system* sys);

/* Last error message of ctx (or of the calling thread when ctx is NULL). */
const char* gp_last_error(const gp_ctx* ctx);

/* Library version string. */
const char* gp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GP_H */
