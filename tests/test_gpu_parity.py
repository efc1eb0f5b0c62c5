"""GPU parity: y = G x through the C ABI against the FP64 CPU oracle.

Tolerances (the operator's stated accuracy targets):
  FP64 path  ||y - y_ref|| / ||y_ref|| <= 1e-12 and |y_i - y_ref,i| <= 1e-12 ||y_ref||_inf
  FP32 path  ||y - y_ref|| / ||y_ref|| <= 1e-5  and |y_i - y_ref,i| <= 1e-5  ||y_ref||_inf
  float-float path (FP64 data, FP32 pairs): the FP64 tolerances
The FP32 path is compared with the oracle applied to x rounded to FP32, so the
check measures the operator, not the rounding of its input.
"""
import numpy as np
import pytest

from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-12}
PRECS = [0, 1, 2]


def _dev(torch, x, prec):
    dt = torch.float32 if prec == 1 else torch.float64
    return torch.tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")


def _apply(gp, torch, ctx, x, prec, add_to=None):
    xd = _dev(torch, x, prec)
    if add_to is None:
        yd = torch.full_like(xd, float("nan"))   # every active DoF must be written
        gp.gp_apply(ctx, xd, yd)
    else:
        yd = _dev(torch, add_to, prec)
        gp.gp_apply_add(ctx, xd, yd)
    torch.cuda.synchronize()
    return yd.double().cpu().numpy()


def _ref_input(x, prec):
    return x if prec != 1 else x.astype(np.float32).astype(np.float64)


def _close(y, ref, prec):
    tol = TOL[prec]
    assert np.all(np.isfinite(y))
    nr = np.linalg.norm(ref)
    assert np.linalg.norm(y - ref) <= tol * nr, np.linalg.norm(y - ref) / nr
    assert np.abs(y - ref).max() <= tol * np.abs(ref).max()


SMALL = [(2, k, 16) for k in range(1, 9)] + [(3, k, 9) for k in range(1, 6)] + [(3, 6, 7), (3, 7, 6),
                                                                              (3, 8, 6)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dim,k,n", SMALL)
def test_small_meshes_all_degrees(gplib, cuda, dim, k, n, prec):
    pr = W.small_ball(dim, n, k, radius=0.62, seed=100 + 10 * dim + k)
    o = Oracle(pr)
    ctx = gplib.setup_problem(pr, precision=prec)
    assert (ctx.n_active, ctx.n_faces) == (o.n_active, o.n_faces) and o.n_faces > 0
    x = W.x_vectors(pr, ctx.n_active)[0]
    y = _apply(gplib, cuda, ctx, x, prec)
    _close(y, o.apply(_ref_input(x, prec)), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_paper_weights_and_multiple_balls(gplib, cuda, prec):
    pr = W.small_ball(3, 12, 4, seed=7, weights=W.paper_weights(0.5, 4))
    pr.centers = np.array([[-0.3, 0.1, 0.0], [0.35, -0.2, 0.1]])
    pr.radii = np.array([0.45, 0.4])
    o = Oracle(pr)
    ctx = gplib.setup_problem(pr, precision=prec)
    x = W.x_vectors(pr, ctx.n_active)[0]
    _close(_apply(gplib, cuda, ctx, x, prec), o.apply(_ref_input(x, prec)), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_disc_2d_k2(gplib, cuda, prec):
    pr = W.disc_2d()
    o = Oracle(pr)
    ctx = gplib.setup_problem(pr, precision=prec)
    x = W.x_vectors(pr, ctx.n_active)[0]
    _close(_apply(gplib, cuda, ctx, x, prec), o.apply(_ref_input(x, prec)), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_ball_3d_k3_full(gplib, cuda, prec):
    """64^3 ball, k = 3: every output compared (the benchmark's launch configuration)."""
    pr = W.ball_3d()
    o = Oracle(pr)
    ctx = gplib.setup_problem(pr, precision=prec)
    x = W.x_vectors(pr, ctx.n_active)[0]
    _close(_apply(gplib, cuda, ctx, x, prec), o.apply(_ref_input(x, prec)), prec)
    if prec != 1:
        # annihilation of a seeded global polynomial of degree <= k (||G|| from power iteration)
        ex, co = W.poly_coeffs(pr)
        xp = W.poly_eval(ex, co, gplib.gp_active_dof_coords(ctx))
        v = np.random.default_rng(0).standard_normal(ctx.n_active)
        for _ in range(30):
            w = _apply(gplib, cuda, ctx, v, prec)
            gn = np.linalg.norm(w)
            v = w / gn
        r = np.linalg.norm(_apply(gplib, cuda, ctx, xp, prec))
        assert r <= 1e-10 * gn * np.linalg.norm(xp), r / (gn * np.linalg.norm(xp))


@pytest.mark.parametrize("prec", PRECS)
def test_apply_add_and_determinism(gplib, cuda, prec):
    pr = W.small_ball(3, 16, 3, seed=8)
    o = Oracle(pr)
    ctx = gplib.setup_problem(pr, precision=prec)
    rng = np.random.default_rng(4)
    x = W.x_vectors(pr, ctx.n_active)[0]
    y0 = rng.uniform(-1, 1, ctx.n_active)
    y = _apply(gplib, cuda, ctx, x, prec, add_to=y0)
    ref = _ref_input(y0, prec) + o.apply(_ref_input(x, prec))
    tol = TOL[prec]
    assert np.abs(y - ref).max() <= tol * np.abs(ref).max()
    a = _apply(gplib, cuda, ctx, x, prec)
    b = _apply(gplib, cuda, ctx, x, prec)
    assert np.array_equal(a, b)   # fixed summation order: bitwise reproducible


@pytest.mark.parametrize("dim,k,m", [(2, 3, 2), (3, 2, 1), (3, 3, 3)])
def test_kink_energy_on_gpu(gplib, cuda, dim, k, m):
    """x^T G x of u = ((x_a - x_P)_+)^m * 1 equals c_m h^(2m-1) (m!)^2 |plane| (no oracle)."""
    import math
    n, h = 6, 0.3
    pr = W.box_problem(dim, n, k, all_faces=True, lo=0.0, hi=n * h)
    ctx = gplib.setup_problem(pr, precision=0)
    xyz = gplib.gp_active_dof_coords(ctx)
    u = np.maximum(xyz[:, dim - 1] - 3 * h, 0.0) ** m
    y = _apply(gplib, cuda, ctx, u, 0)
    ref = 0.5 * h ** (2 * m - 1) * math.factorial(m) ** 2 * (n * h) ** (dim - 1)
    assert abs(u @ y - ref) <= 1e-11 * ref


def test_no_ghost_faces(gplib, cuda):
    pr = W.box_problem(3, 4, 2, all_faces=False)      # every cell inside: nothing to penalise
    ctx = gplib.setup_problem(pr, precision=0)
    assert ctx.n_faces == 0 and ctx.n_active == 9 ** 3
    x = np.ones(ctx.n_active)
    assert np.array_equal(_apply(gplib, cuda, ctx, x, 0), np.zeros(ctx.n_active))
    y0 = np.arange(ctx.n_active, dtype=np.float64)
    assert np.array_equal(_apply(gplib, cuda, ctx, x, 0, add_to=y0), y0)


@pytest.mark.parametrize("prec", PRECS)
def test_empty_domain(gplib, cuda, prec):
    """A level set negative everywhere: no active DoF, no face.  Every apply is a no-op that
    returns GP_OK (device, add, no-alloc, host buffers), and so is the autotuner."""
    pr = W.box_problem(3, 4, 2, all_faces=False)
    pr.ls_value = -1.0
    ctx = gplib.setup_problem(pr, precision=prec)
    assert ctx.n_active == 0 and ctx.n_faces == 0
    dt = cuda.float32 if prec == 1 else cuda.float64
    xd = cuda.zeros(1, dtype=dt, device="cuda")
    yd = cuda.zeros(1, dtype=dt, device="cuda")
    for fn in (gplib.lib.gp_apply, gplib.lib.gp_apply_add, gplib.lib.gp_apply_noalloc):
        assert fn(ctx.handle, xd.data_ptr(), yd.data_ptr(), None) == gplib.GP_OK
    xh = cuda.zeros(1, dtype=dt).pin_memory()
    yh = cuda.zeros(1, dtype=dt).pin_memory()
    assert gplib.lib.gp_apply_host(ctx.handle, xh.data_ptr(), yh.data_ptr(), None) == gplib.GP_OK
    assert gplib.gp_apply_host_bytes(ctx) == (0, 0)
    gplib.gp_autotune(ctx, 1)
    cuda.cuda.synchronize()


def test_single_face_mesh(gplib, cuda):
    pr = W.box_problem(3, 2, 4, all_faces=True)        # 2x2x2 cells, 12 faces
    o = Oracle(pr)
    ctx = gplib.setup_problem(pr, precision=0)
    x = W.x_vectors(pr, ctx.n_active)[0]
    _close(_apply(gplib, cuda, ctx, x, 0), o.apply(x), 0)


def test_host_buffers_end_to_end(gplib, cuda):
    pr = W.small_ball(3, 12, 2, seed=9)
    ctx = gplib.setup_problem(pr, precision=0)
    x = W.x_vectors(pr, ctx.n_active)[0]
    y_host = gplib.gp_apply_host(ctx, x)
    y_dev = _apply(gplib, cuda, ctx, x, 0)
    assert np.array_equal(y_host, y_dev)


@pytest.mark.parametrize("prec", PRECS)
def test_host_buffers_page_locked(gplib, cuda, prec):
    """Page-locked host buffers: the GPU gathers x on the touched DoFs only, and y comes back in
    slab chunks while later slabs compute (the third problem has 8 slabs; y starts as NaN, so
    every entry must come back); bitwise equal to the device apply and to the copy path of
    pageable buffers, with the bytes each path moves."""
    dt = cuda.float32 if prec == 1 else cuda.float64
    for pr in (W.small_ball(3, 12, 2, seed=9), W.small_ball(2, 30, 3, seed=10), W.small_ball(3, 24, 3, seed=12)):
        ctx = gplib.setup_problem(pr, precision=prec)
        x = W.x_vectors(pr, ctx.n_active)[0]
        y_dev = _apply(gplib, cuda, ctx, x, prec)
        xh = cuda.tensor(x, dtype=dt).pin_memory()
        yh = cuda.full((ctx.n_active,), float("nan"), dtype=dt).pin_memory()
        gplib.gp_apply_host(ctx, xh, yh)
        assert np.array_equal(yh.double().numpy(), y_dev)
        w = xh.element_size()
        assert gplib.gp_apply_host_bytes(ctx) == (ctx.n_touched * w, ctx.n_active * w)
        yh.fill_(float("nan"))
        gplib.gp_apply_host(ctx, xh, yh)                   # again: the pipeline's second use
        assert np.array_equal(yh.double().numpy(), y_dev)
        y_pageable = gplib.gp_apply_host(ctx, xh.numpy().copy())
        assert np.array_equal(y_pageable.astype(np.float64), y_dev)
        assert gplib.gp_apply_host_bytes(ctx) == (ctx.n_active * w, ctx.n_active * w)
        # mixed: page-locked x with pageable y, and pageable x with page-locked y
        yp = cuda.full((ctx.n_active,), float("nan"), dtype=dt)
        gplib.gp_apply_host(ctx, xh, yp)
        assert np.array_equal(yp.double().numpy(), y_dev)
        assert gplib.gp_apply_host_bytes(ctx) == (ctx.n_touched * w, ctx.n_active * w)
        xp = cuda.tensor(x, dtype=dt)                     # pageable
        yh.fill_(float("nan"))
        gplib.gp_apply_host(ctx, xp, yh)
        assert np.array_equal(yh.double().numpy(), y_dev)
        assert gplib.gp_apply_host_bytes(ctx) == (ctx.n_active * w, ctx.n_active * w)
    # no ghost faces: nothing to gather, y is all zeros
    pr = W.box_problem(3, 4, 2, all_faces=False)      # every cell inside
    ctx = gplib.setup_problem(pr, precision=prec)
    assert ctx.n_faces == 0
    xh = cuda.ones(ctx.n_active, dtype=dt).pin_memory()
    yh = cuda.full((ctx.n_active,), float("nan"), dtype=dt).pin_memory()
    gplib.gp_apply_host(ctx, xh, yh)
    assert not yh.any().item() and gplib.gp_apply_host_bytes(ctx)[0] == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_host_buffers_full_size_gyroid(gplib, cuda, prec):
    """The 128^3 gyroid at k = 4 (the end-to-end workload of bench.py): the pipelined host apply
    equals the device apply bit for bit."""
    pr = W.gyroid_3d(k=4, n=128)
    ctx = gplib.setup_problem(pr, precision=prec)
    dt = cuda.float32 if prec == 1 else cuda.float64
    x = W.x_vectors(pr, ctx.n_active)[0]
    xd = cuda.tensor(x, dtype=dt, device="cuda")
    yd = cuda.empty_like(xd)
    gplib.gp_apply(ctx, xd, yd)
    xh = xd.cpu().pin_memory()
    yh = cuda.full((ctx.n_active,), float("nan"), dtype=dt).pin_memory()
    for _ in range(2):
        gplib.gp_apply_host(ctx, xh, yh)
        assert cuda.equal(yh, yd.cpu())


def _batched_c(gplib):
    """gp_apply_batched as the exported C symbol (ctypes.CDLL on the library file)."""
    import ctypes
    fn = ctypes.CDLL(gplib.LIB_PATH).gp_apply_batched
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int

    def call(ctxs, nrhs, xs, ys, stream):
        import ctypes as C
        n = len(ctxs)
        H = (C.c_void_p * n)(*[c.handle for c in ctxs])
        X = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
        Y = (C.c_void_p * n)(*[y.data_ptr() for y in ys])
        return fn(H, n, nrhs, X, Y, stream)
    return call


@pytest.mark.parametrize("prec", PRECS)
def test_batched(gplib, cuda, prec):
    """gp_apply_batched through the C symbol: two calls with fresh inputs replay the cached
    batch's graph once each, and match the oracle."""
    probs = [W.small_ball(3, 10, 2, seed=21), W.small_ball(3, 13, 4, seed=22),
             W.small_ball(3, 8, 6, seed=23), W.small_ball(2, 18, 3, seed=24)]
    nrhs = 2
    # the batch runs the face + lift kernels: its outputs equal those of face + lift contexts
    ctxs = [gplib.setup_problem(p, precision=prec, path=gplib.GP_PATH_FACE_LIFT) for p in probs]
    call = _batched_c(gplib)
    oracles = [Oracle(p) for p in probs]
    stream = cuda.cuda.current_stream().cuda_stream
    for rep in range(2):
        xs = [W.x_vectors(p, c.n_active, nrhs + rep)[rep:] for p, c in zip(probs, ctxs)]
        xd = [_dev(cuda, x.ravel(), prec) for x in xs]
        yd = [cuda.full_like(a, float("nan")) for a in xd]
        assert call(ctxs, nrhs, xd, yd, stream) == gplib.GP_OK, gplib.gp_last_error()
        cuda.cuda.synchronize()
        assert gplib.gp_apply_batched_info(ctxs, nrhs) == rep + 1     # one graph launch per call
        for o, c, x, y in zip(oracles, ctxs, xs, yd):
            yy = y.double().cpu().numpy().reshape(nrhs, -1)
            for r in range(nrhs):
                _close(yy[r], o.apply(_ref_input(x[r], prec)), prec)
                assert np.array_equal(yy[r], _apply(gplib, cuda, c, x[r], prec))


@pytest.mark.parametrize("prec", PRECS)
def test_batched_workload_full_size(gplib, cuda, prec):
    """The batched workload at its stated size: 64 independent 3D balls (n ~ U{16..96},
    k ~ U{2..6}), 4 right-hand sides, one gp_apply_batched call.  Every output vector equals a
    single gp_apply bit for bit; the oracle checks sampled rows of 8 problems (the smallest,
    the largest and one of every degree)."""
    probs = W.batched_3d()
    nrhs = 4
    ctxs = [gplib.setup_problem(p, precision=prec, path=gplib.GP_PATH_FACE_LIFT) for p in probs]
    dt = cuda.float32 if prec == 1 else cuda.float64
    gen = cuda.Generator(device="cuda")
    gen.manual_seed(W.BASE_SEED + 5000)
    xs = [cuda.rand(nrhs * c.n_active, generator=gen, dtype=dt, device="cuda") * 2 - 1 for c in ctxs]
    ys = [cuda.full_like(x, float("nan")) for x in xs]
    call = _batched_c(gplib)
    assert call(ctxs, nrhs, xs, ys, cuda.cuda.current_stream().cuda_stream) == gplib.GP_OK, gplib.gp_last_error()
    cuda.cuda.synchronize()
    for c, x, y in zip(ctxs, xs, ys):
        n = c.n_active
        one = cuda.empty(n, dtype=dt, device="cuda")
        for r in range(nrhs):
            gplib.gp_apply(c, x[r * n:(r + 1) * n], one)
            assert cuda.equal(y[r * n:(r + 1) * n], one)
    pick = {int(np.argmin([c.n_active for c in ctxs])), int(np.argmax([c.n_active for c in ctxs]))}
    for k in sorted({p.degree for p in probs}):
        pick.add(next(i for i, p in enumerate(probs) if p.degree == k))
    rng = np.random.default_rng(31)
    for i in sorted(pick):
        o = Oracle(probs[i])
        n = ctxs[i].n_active
        assert (n, ctxs[i].n_faces) == (o.n_active, o.n_faces)
        r = int(rng.integers(0, nrhs))
        x = xs[i][r * n:(r + 1) * n].double().cpu().numpy()
        y = ys[i][r * n:(r + 1) * n].double().cpu().numpy()
        touched = np.unique(o.patch_index(0)[rng.integers(0, o.faces[0].shape[0], 100)].ravel())
        rows = np.unique(np.concatenate([rng.integers(0, n, 1500), touched]))
        ref = o.apply_rows(x, rows)
        assert np.abs(y[rows] - ref).max() <= TOL[prec] * np.abs(ref).max(), i


def test_argument_errors(gplib, cuda):
    pr = W.small_ball(2, 8, 2)
    ctx = gplib.setup_problem(pr, precision=0)
    xd = cuda.zeros(ctx.n_active, dtype=cuda.float64, device="cuda")
    assert gplib.lib.gp_apply(ctx.handle, xd.data_ptr(), xd.data_ptr(), None) == gplib.GP_EINVAL
    assert gplib.lib.gp_apply(ctx.handle, None, xd.data_ptr(), None) == gplib.GP_EINVAL
    with pytest.raises(gplib.GpError):
        gplib.gp_apply(ctx, xd.float(), xd)


_ORACLE = {}


def _oracle_once(key, pr):
    """The oracle of the last large workload (built once for the three arithmetic forms)."""
    if key not in _ORACLE:
        _ORACLE.clear()
        _ORACLE[key] = Oracle(pr)
    return _ORACLE[key]


def _sampled(gplib, cuda, pr, prec, nsample=3000, key=None):
    o = _oracle_once(key, pr) if key is not None else Oracle(pr)
    ctx = gplib.setup_problem(pr, precision=prec)
    assert (ctx.n_active, ctx.n_faces) == (o.n_active, o.n_faces)
    x = W.x_vectors(pr, ctx.n_active)[0]
    y = _apply(gplib, cuda, ctx, x, prec)
    rng = np.random.default_rng(12)
    touched = np.unique(o.patch_index(0)[rng.integers(0, o.faces[0].shape[0], 400)].ravel())
    rows = np.unique(np.concatenate([rng.integers(0, ctx.n_active, nsample), touched]))
    ref = o.apply_rows(_ref_input(x, prec), rows)
    tol = TOL[prec]
    scale = np.abs(ref).max()
    assert np.abs(y[rows] - ref).max() <= tol * scale
    assert np.all(np.isfinite(y))
    return y


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("k", range(1, 9))
def test_ball_96_sampled_every_degree(gplib, cuda, k, prec):
    """The degree sweep at its stated size: 96^3 ball, k = 1..8, every arithmetic form."""
    _sampled(gplib, cuda, W.ball_3d_sweep(k), prec, key=("ball96", k))


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("k", [5, 6])
def test_ball_96_annihilation(gplib, cuda, k, prec):
    """Consistency of the penalty (Sec. 2.2): G annihilates the interpolant of a seeded global
    polynomial of degree <= k, here on the 96^3 mesh at k = 5, 6 (||G|| by 30 power iterations)."""
    pr = W.ball_3d_sweep(k)
    ctx = gplib.setup_problem(pr, precision=prec)
    ex, co = W.poly_coeffs(pr, k)
    xp = W.poly_eval(ex, co, gplib.gp_active_dof_coords(ctx))
    xd = _dev(cuda, xp, prec)
    yd = cuda.empty_like(xd)
    v = cuda.tensor(np.random.default_rng(0).standard_normal(ctx.n_active), dtype=cuda.float64, device="cuda")
    w = cuda.empty_like(v)
    for _ in range(30):
        gplib.gp_apply(ctx, v, w)
        gn = float(cuda.linalg.norm(w))
        v = w / gn
    gplib.gp_apply(ctx, xd, yd)
    r = float(cuda.linalg.norm(yd))
    bound = 1e-10 * gn * float(cuda.linalg.norm(xd))
    assert np.isfinite(r) and r <= bound, r / (gn * float(cuda.linalg.norm(xd)))


@pytest.mark.parametrize("prec", PRECS)
def test_gyroid_128_k4_sampled(gplib, cuda, prec):
    _sampled(gplib, cuda, W.gyroid_3d(), prec, key="gyroid128")


@pytest.mark.parametrize("prec", PRECS)
def test_batch_graph_replays(gplib, cuda, prec):
    """gp_batch_*: problems of mixed k and dimension, 3 right-hand sides, three graph replays
    with fresh inputs; every vector equals gp_apply's bitwise (face + lift contexts: the batch
    runs the same kernels) and the oracle within tolerance."""
    probs = [W.small_ball(3, 10, 2, seed=31), W.small_ball(3, 12, 3, seed=32), W.small_ball(3, 8, 5, seed=33),
             W.small_ball(2, 16, 4, seed=34), W.small_ball(3, 11, 3, seed=35), W.small_ball(3, 9, 2, seed=36)]
    nrhs = 3
    ctxs = [gplib.setup_problem(p, precision=prec, path=gplib.GP_PATH_FACE_LIFT) for p in probs]
    batch = gplib.gp_batch_create(ctxs, nrhs)
    ngroups, scratch = gplib.gp_batch_info(batch)
    assert ngroups == 4 and scratch > 0     # (3D,k2) x2, (3D,k3) x2, (3D,k5), (2D,k4)
    oracles = [Oracle(p) for p in probs]
    rng = np.random.default_rng(17)
    for call in range(3):
        xs = [rng.uniform(-1, 1, (nrhs, c.n_active)) for c in ctxs]
        xd = [_dev(cuda, x.ravel(), prec) for x in xs]
        yd = [cuda.full_like(a, float("nan")) for a in xd]
        gplib.gp_batch_apply(batch, xd, yd)
        cuda.cuda.synchronize()
        for p, c, x, y in zip(range(len(probs)), ctxs, xs, yd):
            yy = y.double().cpu().numpy().reshape(nrhs, -1)
            for r in range(nrhs):
                single = _apply(gplib, cuda, c, x[r], prec)
                assert np.array_equal(yy[r], single), (p, r)
                if call == 0:
                    _close(yy[r], oracles[p].apply(_ref_input(x[r], prec)), prec)
    batch.close()
