"""Tile shapes and the autotuner on the GPU: the shape changes the speed, never the
result (every DoF sums its face contributions in one fixed order), so every shape
must give a bitwise-equal y on both kernel paths (face + lift, brick), and so must a
batch built from tuned contexts."""
import numpy as np
import pytest

from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [
    {"faces_per_cta": 1, "lift_cells_per_cta": 1, "lift_threads": 32},
    {"faces_per_cta": 4, "lift_cells_per_cta": 3, "lift_threads": 64},
    {"faces_per_cta": 8, "lift_cells_per_cta": 14, "lift_threads": 128},
    {"faces_per_cta": 0, "lift_cells_per_cta": 0, "lift_threads": 0},
    {"faces_per_cta": 32, "lift_cells_per_cta": 56, "lift_threads": 512},
]


def _run(gp, torch, ctx, x, prec, add=False):
    dt = torch.float32 if prec == 1 else torch.float64
    xd = torch.tensor(x, dtype=dt, device="cuda")
    yd = torch.full_like(xd, float("nan")) if not add else torch.ones_like(xd)
    (gp.gp_apply_add if add else gp.gp_apply)(ctx, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("dim,n,k", [(3, 14, 3), (2, 40, 4), (3, 10, 1), (3, 8, 6)])
def test_every_shape_is_bitwise_equal(gplib, cuda, prec, dim, n, k, path):
    pr = W.small_ball(dim, n, k, seed=40 + k)
    try:
        ctx = gplib.setup_problem(pr, precision=prec, path=path)
    except gplib.GpError as e:          # the brick path does not fit every (k, precision)
        assert path == gplib.GP_PATH_BRICK and e.status == gplib.GP_EUNSUPPORTED
        pytest.skip("no brick shape fits")
    x = W.x_vectors(pr, ctx.n_active)[0]
    ref = _run(gplib, cuda, ctx, x, prec)
    ref_add = _run(gplib, cuda, ctx, x, prec, add=True)
    o = Oracle(pr)
    xr = x if prec != 1 else x.astype(np.float32).astype(np.float64)
    yo = o.apply(xr)
    tol = 1e-5 if prec == 1 else 1e-12
    assert np.abs(ref - yo).max() <= tol * np.abs(yo).max()
    L = (k + 1) ** (dim - 1)
    vb = 4 if prec == 1 else 8
    fb_max = min(512 // L, (46 * 1024) // ((2 if dim == 3 else 1) * k * L * vb))
    for sh in SHAPES:
        sh = dict(sh)
        sh["faces_per_cta"] = min(sh["faces_per_cta"], fb_max)
        gplib.gp_set_tiles(ctx, sh)
        assert np.array_equal(_run(gplib, cuda, ctx, x, prec), ref), sh
        assert np.array_equal(_run(gplib, cuda, ctx, x, prec, add=True), ref_add), sh


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_autotune_records_and_keeps_result(gplib, cuda, prec):
    pr = W.small_ball(3, 24, 3, seed=5)
    ctx = gplib.setup_problem(pr, precision=prec, path=gplib.GP_PATH_FACE_LIFT)
    x = W.x_vectors(pr, ctx.n_active)[0]
    ref = _run(gplib, cuda, ctx, x, prec)
    tiles, (tf, tl) = gplib.gp_autotune(ctx, reps=3)
    assert tf > 0 and tl > 0
    assert gplib.gp_get_tiles(ctx) == tiles
    assert gplib.gp_tiles_lookup(0, 3, 3, prec) == tiles
    assert np.array_equal(_run(gplib, cuda, ctx, x, prec), ref)
    # a new context of the same (d, k, precision) starts from the table
    ctx2 = gplib.setup_problem(W.small_ball(3, 16, 3, seed=6), precision=prec, path=gplib.GP_PATH_FACE_LIFT)
    assert gplib.gp_get_tiles(ctx2) == tiles
    # brick path: the autotuner picks the faces per chunk over whole applies; the result stays
    cb = gplib.setup_problem(pr, precision=prec, path=gplib.GP_PATH_BRICK)
    yb = _run(gplib, cuda, cb, x, prec)
    tb, (tbf, tbl) = gplib.gp_autotune(cb, reps=3)
    assert tbf > 0 and tbl == 0.0 and gplib.gp_get_tiles(cb) == tb
    assert np.array_equal(_run(gplib, cuda, cb, x, prec), yb)
    cb2 = gplib.setup_problem(W.small_ball(3, 16, 3, seed=6), precision=prec, path=gplib.GP_PATH_BRICK)
    assert gplib.gp_get_tiles(cb2)["faces_per_cta"] == tb["faces_per_cta"]


def test_batch_with_tuned_groups_equals_single_applies(gplib, cuda):
    probs = [W.small_ball(3, 12 + 2 * i, 2 + i % 3, seed=60 + i) for i in range(6)]
    ctxs = [gplib.setup_problem(pr, precision=1, path=gplib.GP_PATH_FACE_LIFT) for pr in probs]
    gplib.gp_set_tiles(ctxs[0], {"faces_per_cta": 3, "lift_cells_per_cta": 5, "lift_threads": 64})
    gplib.gp_set_tiles(ctxs[1], {"faces_per_cta": 20, "lift_cells_per_cta": 60, "lift_threads": 512})
    nrhs = 2
    xs = [cuda.tensor(W.x_vectors(pr, c.n_active, nrhs).ravel(), dtype=cuda.float32, device="cuda")
          for pr, c in zip(probs, ctxs)]
    ys = [cuda.full_like(x, float("nan")) for x in xs]
    b = gplib.gp_batch_create(ctxs, nrhs)
    gplib.gp_batch_apply(b, xs, ys)
    cuda.cuda.synchronize()
    for c, x, y in zip(ctxs, xs, ys):
        for r in range(nrhs):
            s = slice(r * c.n_active, (r + 1) * c.n_active)
            yr = cuda.empty(c.n_active, dtype=cuda.float32, device="cuda")
            gplib.gp_apply(c, x[s].contiguous(), yr)
            cuda.cuda.synchronize()
            assert cuda.equal(y[s], yr)
    gplib.gp_batch_destroy(b)


def test_autotune_cache_file(gplib, cuda, tmp_path):
    import json
    path = str(tmp_path / "tiles.json")
    pr = W.small_ball(3, 16, 2, seed=12)
    ctx = gplib.setup_problem(pr, precision=1, path=gplib.GP_PATH_FACE_LIFT)
    t1 = gplib.autotune_cached(ctx, reps=2, path=path)
    data = json.load(open(path))
    assert len(data) == 1 and list(data.values())[0] == t1 and "|d3|k2|p1|path1" in list(data)[0]
    # a hit sets the stored shape without timing
    data[list(data)[0]] = {"faces_per_cta": 5, "lift_cells_per_cta": 7, "lift_threads": 96}
    json.dump(data, open(path, "w"))
    ctx2 = gplib.setup_problem(pr, precision=1, path=gplib.GP_PATH_FACE_LIFT)
    assert gplib.autotune_cached(ctx2, path=path) == {"faces_per_cta": 5, "lift_cells_per_cta": 7, "lift_threads": 96}
    assert gplib.gp_get_tiles(ctx2) == {"faces_per_cta": 5, "lift_cells_per_cta": 7, "lift_threads": 96}
