"""GPU: the brick path (gp_opts.kernel_path = GP_PATH_BRICK) against the oracle and against
the face + lift path.

The brick kernel stages the cell blocks of a brick of cells in shared memory, evaluates every
ghost face with a cell in the brick, sums the face outputs per cell and per node in shared
memory, and writes interior nodes once; nodes on the planes between bricks go through partial
sums and a fixup kernel.  Checked: element-wise parity with the oracle (FP64 and float-float
1e-12, FP32 1e-5) for d = 2, 3 and the degrees whose bricks fit in shared memory, with large
and small bricks (many plane nodes, edges and corners shared by up to 8 bricks); the add form;
bitwise reproducibility; bitwise independence of the faces per chunk; agreement with the face +
lift path; the full-size 64^3 and 128^3 workloads.
"""
import numpy as np
import pytest

from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-12}


def _ctx(gp, pr, prec, path, smem=0):
    mesh, ls, opts, keep = gp.structs_for(pr, prec, 0)
    opts.kernel_path = path
    opts.brick_smem = smem
    return gp.gp_setup(mesh, ls, opts)


def _apply(gp, torch, ctx, x, prec, add_to=None, tiles=None):
    dt = torch.float32 if prec == 1 else torch.float64
    xd = torch.tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")
    if tiles is not None:
        gp.gp_set_tiles(ctx, tiles)
    if add_to is None:
        yd = torch.full_like(xd, float("nan"))
        gp.gp_apply(ctx, xd, yd)
    else:
        yd = torch.tensor(np.ascontiguousarray(add_to), dtype=dt, device="cuda")
        gp.gp_apply_add(ctx, xd, yd)
    torch.cuda.synchronize()
    return yd.double().cpu().numpy()


def _ref_in(x, prec):
    return x if prec != 1 else x.astype(np.float32).astype(np.float64)


def _close(y, ref, prec):
    assert np.all(np.isfinite(y))
    assert np.abs(y - ref).max() <= TOL[prec] * np.abs(ref).max(), np.abs(y - ref).max() / np.abs(ref).max()


CASES = [(2, k, 24) for k in (1, 2, 3, 4, 5, 6, 7, 8)] + [(3, k, 10) for k in (1, 2, 3, 4)] + [(3, 5, 8), (3, 6, 7)]


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("dim,k,n", CASES)
def test_brick_matches_oracle(gplib, cuda, dim, k, n, prec):
    pr = W.small_ball(dim, n, k, radius=0.62, seed=300 + 10 * dim + k)
    o = Oracle(pr)
    try:
        ctx = _ctx(gplib, pr, prec, gplib.GP_PATH_BRICK)
    except gplib.GpError as e:
        assert e.status == gplib.GP_EUNSUPPORTED
        pytest.skip("no brick shape fits")
    x = W.x_vectors(pr, ctx.n_active)[0]
    _close(_apply(gplib, cuda, ctx, x, prec), o.apply(_ref_in(x, prec)), prec)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("smem", [16 * 1024, 40 * 1024, 0])
def test_brick_shapes_and_add_form(gplib, cuda, prec, smem):
    """Smaller budgets pick smaller bricks: more plane nodes (edges and corners of up to 8
    bricks).  Also the add form y += G x, reproducibility, and the faces per chunk."""
    pr = W.small_ball(3, 14, 2, radius=0.66, seed=351)
    o = Oracle(pr)
    ctx = _ctx(gplib, pr, prec, gplib.GP_PATH_BRICK, smem)
    info = gplib.gp_kernel_path(ctx)
    assert info["path"] == gplib.GP_PATH_BRICK and info["plane_nodes"] > 0
    x = W.x_vectors(pr, ctx.n_active)[0]
    ref = o.apply(_ref_in(x, prec))
    y = _apply(gplib, cuda, ctx, x, prec)
    _close(y, ref, prec)
    assert np.array_equal(y, _apply(gplib, cuda, ctx, x, prec))           # bitwise reproducible
    for fb in (1, 3, 7, 20):                                               # chunking does not matter
        assert np.array_equal(y, _apply(gplib, cuda, ctx, x, prec, tiles={"faces_per_cta": fb}))
    y0 = np.random.default_rng(3).uniform(-1, 1, ctx.n_active)
    ya = _apply(gplib, cuda, ctx, x, prec, add_to=y0)
    _close(ya, _ref_in(y0, prec) + ref, prec)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_brick_and_face_lift_agree(gplib, cuda, prec):
    pr = W.ball_3d()
    cb = _ctx(gplib, pr, prec, gplib.GP_PATH_BRICK)
    cf = _ctx(gplib, pr, prec, gplib.GP_PATH_FACE_LIFT)
    x = W.x_vectors(pr, cb.n_active)[0]
    yb = _apply(gplib, cuda, cb, x, prec)
    yf = _apply(gplib, cuda, cf, x, prec)
    assert np.abs(yb - yf).max() <= 2 * TOL[prec] * np.abs(yf).max()
    o = Oracle(pr)
    _close(yb, o.apply(_ref_in(x, prec)), prec)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_brick_gyroid_128_sampled(gplib, cuda, prec):
    pr = W.gyroid_3d()
    o = Oracle(pr)
    ctx = _ctx(gplib, pr, prec, gplib.GP_PATH_BRICK)
    x = W.x_vectors(pr, ctx.n_active)[0]
    y = _apply(gplib, cuda, ctx, x, prec)
    rng = np.random.default_rng(12)
    touched = np.unique(np.concatenate([o.patch_index(a)[rng.integers(0, o.faces[a].shape[0], 150)].ravel()
                                        for a in range(3)]))
    rows = np.unique(np.concatenate([rng.integers(0, ctx.n_active, 3000), touched]))
    ref = o.apply_rows(_ref_in(x, prec), rows)
    assert np.all(np.isfinite(y))
    assert np.abs(y[rows] - ref).max() <= TOL[prec] * np.abs(ref).max()
