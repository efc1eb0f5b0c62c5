"""Thin Python binding of the C ABI in include/gp.h (ctypes).

Argument marshalling only: every step of y = G x runs in libgp.so.  The
functions keep the C names.  Device vectors are passed as torch CUDA tensors
(or raw device pointers); the library never sees a torch type.  Importing
this module loads the in-tree library and fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgp.so")

GP_OK, GP_EINVAL, GP_ENOMEM, GP_ECUDA, GP_EDEVICE, GP_EUNSUPPORTED = range(6)
GP_FP64, GP_FP32, GP_FP64_FF = 0, 1, 2
GP_LS_BALLS, GP_LS_GYROID, GP_LS_CALLBACK, GP_LS_CONST = 1, 2, 3, 4
GP_STAB_GHOST, GP_STAB_MACRO = 0, 1
GP_PATH_AUTO, GP_PATH_FACE_LIFT, GP_PATH_BRICK = 0, 1, 2
_STATUS = {0: "GP_OK", 1: "GP_EINVAL", 2: "GP_ENOMEM", 3: "GP_ECUDA", 4: "GP_EDEVICE",
           5: "GP_EUNSUPPORTED"}


class GpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class gp_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


LEVELSET_FN = C.CFUNCTYPE(C.c_double, C.POINTER(C.c_double), C.c_void_p)


class gp_levelset(C.Structure):
    _fields_ = [("kind", C.c_int), ("nballs", C.c_int), ("centers", C.POINTER(C.c_double)),
                ("radii", C.POINTER(C.c_double)), ("iso", C.c_double), ("value", C.c_double),
                ("fn", LEVELSET_FN), ("user", C.c_void_p), ("lipschitz", C.c_double),
                ("samples", C.c_int)]


class gp_solve_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("inner_rtol", C.c_double), ("max_outer", C.c_int),
                ("max_inner", C.c_int), ("mode", C.c_int), ("precond", C.c_int)]


class gp_solve_stats(C.Structure):
    _fields_ = [("outer", C.c_int), ("inner", C.c_int), ("hi_applies", C.c_int), ("lo_applies", C.c_int),
                ("rel_residual", C.c_double), ("seconds", C.c_double)]


class gp_opts(C.Structure):
    _fields_ = [("degree", C.c_int), ("nweights", C.c_int), ("weights", C.POINTER(C.c_double)),
                ("gamma", C.c_double), ("precision", C.c_int), ("all_faces", C.c_int),
                ("device", C.c_int), ("part_lo", C.c_int), ("part_hi", C.c_int), ("stabilization", C.c_int),
                ("no_scratch", C.c_int), ("kernel_path", C.c_int), ("brick_smem", C.c_int),
                ("slabs", C.c_int)]


class gp_tiles(C.Structure):
    _fields_ = [("faces_per_cta", C.c_int), ("lift_cells_per_cta", C.c_int), ("lift_threads", C.c_int)]


class gp_partition(C.Structure):
    _fields_ = [("layer_lo", C.c_int32), ("layer_hi", C.c_int32), ("offset", C.c_int64),
                ("n_local", C.c_int64), ("n_owned", C.c_int64), ("n_lower", C.c_int64),
                ("n_global", C.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgp.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                          "or python -m paper_2503_00246_gb300.build")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    i64p = C.POINTER(C.c_int64)
    sig = {
        "gp_setup": ([C.POINTER(gp_mesh), C.POINTER(gp_levelset), C.POINTER(gp_opts), C.POINTER(P)], C.c_int),
        "gp_destroy": ([P], None),
        "gp_num_active_dofs": ([P, i64p], C.c_int),
        "gp_num_ghost_faces": ([P, i64p], C.c_int),
        "gp_num_touched_dofs": ([P, i64p], C.c_int),
        "gp_cell_counts": ([P, i64p], C.c_int),
        "gp_active_dof_coords": ([P, C.POINTER(C.c_double)], C.c_int),
        "gp_ghost_faces": ([P, C.POINTER(C.c_int32), i64p], C.c_int),
        "gp_cell_classes": ([P, C.POINTER(C.c_int8)], C.c_int),
        "gp_get_tiles": ([P, C.POINTER(gp_tiles)], C.c_int),
        "gp_set_tiles": ([P, C.POINTER(gp_tiles)], C.c_int),
        "gp_autotune": ([P, C.c_int, C.POINTER(gp_tiles), C.POINTER(C.c_double)], C.c_int),
        "gp_tiles_record": ([C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(gp_tiles)], C.c_int),
        "gp_tiles_lookup": ([C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(gp_tiles)], C.c_int),
        "gp_partition_info": ([P, C.POINTER(gp_partition)], C.c_int),
        "gp_partition_slabs": ([C.POINTER(gp_mesh), C.POINTER(gp_levelset), C.POINTER(gp_opts), C.c_int,
                                C.POINTER(C.c_int32)], C.c_int),
        "gp_reference_1d": ([P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
        "gp_apply": ([P, P, P, P], C.c_int),
        "gp_apply_add": ([P, P, P, P], C.c_int),
        "gp_apply_noalloc": ([P, P, P, P], C.c_int),
        "gp_apply_host": ([P, P, P, P], C.c_int),
        "gp_apply_host_bytes": ([P, i64p, i64p], C.c_int),
        "gp_apply_batched": ([C.POINTER(P), C.c_int, C.c_int, C.POINTER(P), C.POINTER(P), P], C.c_int),
        "gp_apply_batched_info": ([C.POINTER(P), C.c_int, C.c_int, i64p], C.c_int),
        "gp_kernel_path": ([P, C.POINTER(C.c_int), C.POINTER(C.c_int32), i64p], C.c_int),
        "gp_batch_create": ([C.POINTER(P), C.c_int, C.c_int, C.POINTER(P)], C.c_int),
        "gp_batch_apply": ([P, C.POINTER(P), C.POINTER(P), P], C.c_int),
        "gp_batch_info": ([P, i64p, i64p], C.c_int),
        "gp_batch_destroy": ([P], None),
        "gp_system_create": ([P, P, C.POINTER(P)], C.c_int),
        "gp_system_apply": ([P, C.c_int, P, P, P], C.c_int),
        "gp_system_cells": ([P, C.c_int, C.c_double, C.c_double, P, P, P], C.c_int),
        "gp_system_solve": ([P, P, P, C.POINTER(gp_solve_opts), C.POINTER(gp_solve_stats)], C.c_int),
        "gp_system_destroy": ([P], None),
        "gp_profile_enable": ([P, C.c_int], C.c_int),
        "gp_profile_read": ([P, C.POINTER(C.c_double), i64p], C.c_int),
        "gp_last_error": ([P], C.c_char_p),
        "gp_version": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()

# names declared in include/gp.h, used by the tests to check the exports
ABI_SYMBOLS = ("gp_setup", "gp_destroy", "gp_num_active_dofs", "gp_num_ghost_faces",
               "gp_num_touched_dofs", "gp_cell_counts", "gp_active_dof_coords", "gp_ghost_faces",
               "gp_cell_classes", "gp_reference_1d", "gp_apply", "gp_apply_add", "gp_apply_host",
               "gp_apply_batched", "gp_profile_enable", "gp_profile_read", "gp_last_error",
               "gp_version", "gp_apply_noalloc", "gp_batch_create", "gp_batch_apply", "gp_batch_info",
               "gp_batch_destroy", "gp_system_create", "gp_system_apply", "gp_system_solve",
               "gp_system_destroy", "gp_partition_info", "gp_partition_slabs", "gp_get_tiles",
               "gp_set_tiles", "gp_autotune", "gp_tiles_record", "gp_tiles_lookup", "gp_system_cells",
               "gp_apply_batched_info", "gp_kernel_path", "gp_apply_host_bytes")
NOALLOC_SCRATCH_BYTES = 32 << 20


def _check(status, ctx=None):
    if status != GP_OK:
        msg = lib.gp_last_error(ctx.handle if ctx is not None else None)
        raise GpError(status, (msg or b"").decode())


class Context:
    """Owns a gp_ctx handle (gp_destroy on close / garbage collection)."""

    def __init__(self, handle, precision, dim, degree, device=0):
        self.handle = handle
        self.precision = precision
        self.dim = dim
        self.degree = degree
        self.device = device
        n = C.c_int64()
        _check(lib.gp_num_active_dofs(handle, C.byref(n)), self)
        self.n_active = n.value
        _check(lib.gp_num_ghost_faces(handle, C.byref(n)), self)
        self.n_faces = n.value
        _check(lib.gp_num_touched_dofs(handle, C.byref(n)), self)
        self.n_touched = n.value

    def close(self):
        if self.handle:
            lib.gp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dtype_np(self):
        return np.float32 if self.precision == GP_FP32 else np.float64


def gp_setup(mesh: gp_mesh, levelset: gp_levelset, opts: gp_opts) -> Context:
    h = C.c_void_p()
    _check(lib.gp_setup(C.byref(mesh), C.byref(levelset), C.byref(opts), C.byref(h)))
    return Context(h.value, opts.precision, mesh.dim, opts.degree, opts.device)


def gp_destroy(ctx: Context):
    ctx.close()


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _check_vec(ctx, t, nrhs=1):
    if isinstance(t, int):
        return
    import torch
    want = torch.float32 if ctx.precision == GP_FP32 else torch.float64
    if t.dtype != want or not t.is_cuda or not t.is_contiguous() or t.numel() != nrhs * ctx.n_active:
        raise GpError(GP_EINVAL, f"expected a contiguous CUDA {want} tensor of {nrhs * ctx.n_active} "
                                 f"elements, got {t.dtype} {tuple(t.shape)} on {t.device}")


def gp_apply(ctx: Context, x, y, stream=None):
    _check_vec(ctx, x)
    _check_vec(ctx, y)
    _check(lib.gp_apply(ctx.handle, _ptr(x), _ptr(y), _stream(stream)), ctx)


def gp_apply_noalloc(ctx: Context, x, y, stream=None):
    """y = G x without any device allocation: the face outputs use the library's fixed
    32 MiB scratch (see gp.h).  For callers whose device memory is owned by another
    allocator, or whose loop must not pay for cudaMalloc/cudaFree."""
    _check_vec(ctx, x)
    _check_vec(ctx, y)
    _check(lib.gp_apply_noalloc(ctx.handle, _ptr(x), _ptr(y), _stream(stream)), ctx)


def gp_apply_add(ctx: Context, x, y, stream=None):
    _check_vec(ctx, x)
    _check_vec(ctx, y)
    _check(lib.gp_apply_add(ctx.handle, _ptr(x), _ptr(y), _stream(stream)), ctx)


def gp_apply_host(ctx: Context, x: np.ndarray, y: np.ndarray | None = None, stream=0):
    """End-to-end apply on host arrays (numpy or pinned torch CPU tensors)."""
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x, dtype=ctx.dtype_np)
        if y is None:
            y = np.empty_like(x)
        assert x.size == ctx.n_active and y.size == ctx.n_active and y.dtype == x.dtype
        xp, yp = x.ctypes.data, y.ctypes.data
    else:
        xp, yp = x.data_ptr(), y.data_ptr()
    _check(lib.gp_apply_host(ctx.handle, xp, yp, stream if isinstance(stream, int) else stream.cuda_stream), ctx)
    return y


def gp_apply_host_bytes(ctx: Context):
    """(host -> device, device -> host) bytes the last gp_apply_host of ctx moved."""
    a, b = C.c_int64(), C.c_int64()
    _check(lib.gp_apply_host_bytes(ctx.handle, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def gp_apply_batched(ctxs, nrhs, xs, ys, stream=None):
    """y_p = G_p x_p for every problem and right-hand side: one graph replay of the batch the
    library keeps for this list of contexts (built on the first call)."""
    n = len(ctxs)
    for c, x, y in zip(ctxs, xs, ys):
        _check_vec(c, x, nrhs)
        _check_vec(c, y, nrhs)
    H = (C.c_void_p * n)(*[c.handle for c in ctxs])
    X = (C.c_void_p * n)(*[_ptr(x) for x in xs])
    Y = (C.c_void_p * n)(*[_ptr(y) for y in ys])
    _check(lib.gp_apply_batched(H, n, nrhs, X, Y, _stream(stream)))


def gp_apply_batched_info(ctxs, nrhs) -> int:
    """Graph replays made by gp_apply_batched for this list of contexts."""
    n = len(ctxs)
    H = (C.c_void_p * n)(*[c.handle for c in ctxs])
    v = C.c_int64()
    _check(lib.gp_apply_batched_info(H, n, nrhs, C.byref(v)))
    return v.value


class Batch:
    """Owns a gp_batch handle; keeps its contexts alive."""

    def __init__(self, handle, ctxs, nrhs):
        self.handle = handle
        self.ctxs = list(ctxs)
        self.nrhs = nrhs

    def close(self):
        if self.handle:
            lib.gp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gp_batch_create(ctxs, nrhs) -> Batch:
    n = len(ctxs)
    H = (C.c_void_p * n)(*[c.handle for c in ctxs])
    h = C.c_void_p()
    _check(lib.gp_batch_create(H, n, nrhs, C.byref(h)))
    return Batch(h.value, ctxs, nrhs)


def gp_batch_apply(batch: Batch, xs, ys, stream=None):
    for c, x, y in zip(batch.ctxs, xs, ys):
        _check_vec(c, x, batch.nrhs)
        _check_vec(c, y, batch.nrhs)
    n = len(batch.ctxs)
    X = (C.c_void_p * n)(*[_ptr(x) for x in xs])
    Y = (C.c_void_p * n)(*[_ptr(y) for y in ys])
    _check(lib.gp_batch_apply(batch.handle, X, Y, _stream(stream)))


def gp_batch_info(batch: Batch):
    a, b = C.c_int64(), C.c_int64()
    _check(lib.gp_batch_info(batch.handle, C.byref(a), C.byref(b)))
    return a.value, b.value


def gp_batch_destroy(batch: Batch):
    batch.close()


class System:
    """Owns a gp_system handle; keeps its contexts alive."""

    def __init__(self, handle, hi, lo):
        self.handle, self.hi, self.lo = handle, hi, lo

    def close(self):
        if self.handle:
            lib.gp_system_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gp_system_create(hi: Context, lo: Context | None = None) -> System:
    h = C.c_void_p()
    _check(lib.gp_system_create(hi.handle, lo.handle if lo is not None else None, C.byref(h)))
    return System(h.value, hi, lo)


def gp_system_apply(sys: System, which: int, x, y, stream=None):
    ctx = sys.hi if which == 0 else sys.lo
    _check_vec(ctx, x)
    _check_vec(ctx, y)
    _check(lib.gp_system_apply(sys.handle, which, _ptr(x), _ptr(y), _stream(stream)))


def gp_system_cells(sys: System, which: int, x, y, mass: float = 1.0, stiff: float = 1.0, stream=None):
    """y = (mass M_active + stiff K_active) x with the hi (0) or lo (1) arithmetic."""
    ctx = sys.hi if which == 0 else sys.lo
    _check_vec(ctx, x)
    _check_vec(ctx, y)
    _check(lib.gp_system_cells(sys.handle, int(which), float(mass), float(stiff), _ptr(x), _ptr(y), _stream(stream)))


def gp_system_solve(sys: System, b, u, rtol=1e-10, inner_rtol=1e-4, max_outer=50, max_inner=20000, mode=0,
                    precond=1):
    """Solve (M+K+G) u = b; returns the gp_solve_stats as a dict."""
    _check_vec(sys.hi, b)
    _check_vec(sys.hi, u)
    o = gp_solve_opts(rtol, inner_rtol, max_outer, max_inner, mode, precond)
    st = gp_solve_stats()
    _check(lib.gp_system_solve(sys.handle, _ptr(b), _ptr(u), C.byref(o), C.byref(st)))
    return {f: getattr(st, f) for f, _ in gp_solve_stats._fields_}


def gp_system_destroy(sys: System):
    sys.close()


def gp_num_active_dofs(ctx: Context) -> int:
    return ctx.n_active


def gp_num_ghost_faces(ctx: Context) -> int:
    return ctx.n_faces


def gp_num_touched_dofs(ctx: Context) -> int:
    return ctx.n_touched


def gp_cell_counts(ctx: Context) -> np.ndarray:
    out = np.zeros(3, dtype=np.int64)
    _check(lib.gp_cell_counts(ctx.handle, out.ctypes.data_as(C.POINTER(C.c_int64))), ctx)
    return out


def gp_active_dof_coords(ctx: Context) -> np.ndarray:
    out = np.zeros((ctx.n_active, ctx.dim), dtype=np.float64)
    _check(lib.gp_active_dof_coords(ctx.handle, out.ctypes.data_as(C.POINTER(C.c_double))), ctx)
    return out


def gp_ghost_faces(ctx: Context):
    axis = np.zeros(ctx.n_faces, dtype=np.int32)
    cell = np.zeros(ctx.n_faces, dtype=np.int64)
    _check(lib.gp_ghost_faces(ctx.handle, axis.ctypes.data_as(C.POINTER(C.c_int32)),
                              cell.ctypes.data_as(C.POINTER(C.c_int64))), ctx)
    return axis, cell


def gp_cell_classes(ctx: Context, n_cells: int) -> np.ndarray:
    out = np.zeros(n_cells, dtype=np.int8)
    _check(lib.gp_cell_classes(ctx.handle, out.ctypes.data_as(C.POINTER(C.c_int8))), ctx)
    return out


def _tiles_dict(t: gp_tiles) -> dict:
    return {f: getattr(t, f) for f, _ in gp_tiles._fields_}


def _tiles_struct(d: dict) -> gp_tiles:
    t = gp_tiles()
    for f, _ in gp_tiles._fields_:
        setattr(t, f, int(d.get(f, 0)))
    return t


def gp_get_tiles(ctx: Context) -> dict:
    """faces_per_cta, lift_cells_per_cta, lift_threads of the context."""
    t = gp_tiles()
    _check(lib.gp_get_tiles(ctx.handle, C.byref(t)), ctx)
    return _tiles_dict(t)


def gp_set_tiles(ctx: Context, tiles: dict):
    _check(lib.gp_set_tiles(ctx.handle, C.byref(_tiles_struct(tiles))), ctx)


def gp_autotune(ctx: Context, reps: int = 10):
    """Times the candidate tile shapes on the context; returns (tiles, (face_ms, lift_ms))."""
    t = gp_tiles()
    ms = (C.c_double * 2)()
    _check(lib.gp_autotune(ctx.handle, int(reps), C.byref(t), ms), ctx)
    return _tiles_dict(t), (ms[0], ms[1])


def gp_tiles_record(device: int, dim: int, degree: int, precision: int, tiles: dict):
    _check(lib.gp_tiles_record(device, dim, degree, precision, C.byref(_tiles_struct(tiles))))


def gp_tiles_lookup(device: int, dim: int, degree: int, precision: int):
    """The process-wide entry for the key, or None."""
    t = gp_tiles()
    if lib.gp_tiles_lookup(device, dim, degree, precision, C.byref(t)) != GP_OK:
        return None
    return _tiles_dict(t)


def tiles_cache_path() -> str:
    """The autotuner's cache file: $GP_TILES_CACHE, else ~/.cache/gp_gb300/tiles.json."""
    return os.environ.get("GP_TILES_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "gp_gb300",
                                                             "tiles.json")


def autotune_cached(ctx: Context, reps: int = 10, path: str | None = None) -> dict:
    """Tile shapes for ctx from the cache file, keyed by (GPU name, d, k, precision, path); on a miss
    gp_autotune times the candidates and the result is written back.  Either way the shape is
    set on ctx and recorded in the library's table for new contexts."""
    import json
    import torch
    path = path or tiles_cache_path()
    kpath = gp_kernel_path(ctx)["path"]
    key = f"{torch.cuda.get_device_name(ctx.device)}|d{ctx.dim}|k{ctx.degree}|p{ctx.precision}|path{kpath}"
    cache = {}
    if os.path.exists(path):
        with open(path) as fh:
            cache = json.load(fh)
    if key in cache:
        tiles = cache[key]
        gp_set_tiles(ctx, tiles)
        if kpath == GP_PATH_FACE_LIFT:
            gp_tiles_record(ctx.device, ctx.dim, ctx.degree, ctx.precision, tiles)
        return tiles
    tiles, _ = gp_autotune(ctx, reps)
    cache[key] = tiles
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return tiles


def gp_partition_info(ctx: Context) -> dict:
    """Layout of a slab partition: layer_lo, layer_hi, offset, n_local, n_owned, n_lower, n_global."""
    out = gp_partition()
    _check(lib.gp_partition_info(ctx.handle, C.byref(out)), ctx)
    return {f: getattr(out, f) for f, _ in gp_partition._fields_}


def gp_partition_slabs(mesh: gp_mesh, levelset: gp_levelset, opts: gp_opts, nparts: int) -> np.ndarray:
    """Layer boundaries (nparts + 1 int32) of the weighted slab partition."""
    b = np.zeros(nparts + 1, dtype=np.int32)
    _check(lib.gp_partition_slabs(C.byref(mesh), C.byref(levelset), C.byref(opts), int(nparts),
                                  b.ctypes.data_as(C.POINTER(C.c_int32))))
    return b


def gp_kernel_path(ctx: Context) -> dict:
    """{"path": GP_PATH_*, "bdim": brick shape, "bricks", "plane_nodes", "scratch_bytes", "slabs"}
    (bricks and plane_nodes 0 on the face + lift path, slabs 0 on the brick path)."""
    path = C.c_int()
    bd = (C.c_int32 * 3)()
    cn = (C.c_int64 * 3)()
    _check(lib.gp_kernel_path(ctx.handle, C.byref(path), bd, cn), ctx)
    brick = path.value == GP_PATH_BRICK
    return {"path": path.value, "bdim": list(bd), "bricks": cn[0] if brick else 0,
            "plane_nodes": cn[1], "scratch_bytes": cn[2], "slabs": 0 if brick else cn[0]}


def gp_reference_1d(ctx: Context):
    k = ctx.degree
    m = np.zeros((k + 1) * (k + 1))
    g = np.zeros(k * (2 * k + 1))
    s = np.zeros(k)
    dp = C.POINTER(C.c_double)
    _check(lib.gp_reference_1d(ctx.handle, m.ctypes.data_as(dp), g.ctypes.data_as(dp),
                               s.ctypes.data_as(dp)), ctx)
    return m.reshape(k + 1, k + 1), g.reshape(k, 2 * k + 1), s


def gp_profile_enable(ctx: Context, enable: bool = True):
    _check(lib.gp_profile_enable(ctx.handle, 1 if enable else 0), ctx)


def gp_profile_read(ctx: Context):
    """(ms_jump, ms_lift, calls): summed kernel times of the traced applies."""
    ms = (C.c_double * 2)()
    calls = C.c_int64()
    _check(lib.gp_profile_read(ctx.handle, ms, C.byref(calls)), ctx)
    return ms[0], ms[1], calls.value


def gp_last_error(ctx: Context | None = None) -> str:
    return (lib.gp_last_error(ctx.handle if ctx else None) or b"").decode()


def gp_version() -> str:
    return lib.gp_version().decode()


# ------------------------------------------------------------ marshalling --

def structs_for(pr: W.Problem, precision: int = GP_FP64, device: int = 0, part=None, path: int = GP_PATH_AUTO,
                slabs: int = 0):
    """gp_mesh / gp_levelset / gp_opts for a workloads.Problem (kept alive in the tuple);
    path is the kernel path (GP_PATH_*), slabs gp_opts.slabs."""
    mesh = gp_mesh()
    mesh.dim = pr.dim
    for a in range(3):
        mesh.n[a] = pr.n if a < pr.dim else 1
        mesh.lo[a] = pr.lo if a < pr.dim else 0.0
        mesh.hi[a] = pr.hi if a < pr.dim else 1.0
    ls = gp_levelset()
    ls.kind = pr.ls_kind
    keep = []
    if pr.ls_kind == GP_LS_BALLS:
        cen = np.ascontiguousarray(np.asarray(pr.centers, dtype=np.float64).reshape(-1, 3))
        rad = np.ascontiguousarray(np.asarray(pr.radii, dtype=np.float64))
        keep += [cen, rad]
        ls.nballs = rad.size
        ls.centers = cen.ctypes.data_as(C.POINTER(C.c_double))
        ls.radii = rad.ctypes.data_as(C.POINTER(C.c_double))
    ls.iso = pr.iso
    ls.value = pr.ls_value
    ls.samples = 4
    opts = gp_opts()
    opts.degree = pr.degree
    opts.gamma = pr.gamma
    if pr.weights is not None:
        w = np.ascontiguousarray(np.asarray(pr.weights, dtype=np.float64))
        keep.append(w)
        opts.nweights = w.size
        opts.weights = w.ctypes.data_as(C.POINTER(C.c_double))
    opts.precision = precision
    opts.all_faces = 1 if pr.all_faces else 0
    opts.device = device
    opts.stabilization = int(getattr(pr, "stabilization", 0))
    if part is not None:
        opts.part_lo, opts.part_hi = int(part[0]), int(part[1])
    opts.kernel_path = int(path)
    opts.slabs = int(slabs)
    return mesh, ls, opts, keep


def setup_problem(pr: W.Problem, precision: int = GP_FP64, device: int = 0, part=None,
                  path: int = GP_PATH_AUTO, slabs: int = 0) -> Context:
    """Context for a workloads.Problem; part = (layer_lo, layer_hi) selects a slab partition,
    path the kernel path (GP_PATH_AUTO, GP_PATH_FACE_LIFT, GP_PATH_BRICK), slabs the face + lift
    launch pipeline (gp_opts.slabs: 0 or 1 off, n about n slabs)."""
    mesh, ls, opts, keep = structs_for(pr, precision, device, part, path, slabs)
    return gp_setup(mesh, ls, opts)


def partition_problem(pr: W.Problem, nparts: int) -> np.ndarray:
    """Layer boundaries of the weighted slab partition of a workloads.Problem."""
    mesh, ls, opts, keep = structs_for(pr, GP_FP64, -1)
    return gp_partition_slabs(mesh, ls, opts, nparts)
