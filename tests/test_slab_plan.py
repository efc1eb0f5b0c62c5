"""Host checks of the slab pipeline's plan (no GPU): gp_opts.slabs and gp_kernel_path.

The lift owners are the cells (coordinates in [0, n]) c + s, s in {0, 1}^d, of the involved
cells c (the two cells of each ghost face); the pipeline cuts them into ranges of whole groups
of 256 owners, so it has min(requested, ceil(owners / 256), 64) slabs, and none (one launch
pair) when fewer than two groups exist or slabs is 0 or 1.  Recomputed here with numpy from
the face list.
"""
import numpy as np
import pytest

from paper_2503_00246_gb300 import workloads as W


def _ctx(gp, pr, prec, slabs, path=0):
    mesh, ls, opts, keep = gp.structs_for(pr, prec, -1, path=path, slabs=slabs)
    return gp.gp_setup(mesh, ls, opts)


def _owners(gp, ctx, pr):
    d, n = pr.dim, pr.n
    axis, cell = gp.gp_ghost_faces(ctx)
    C = np.stack([(cell // n ** a) % n for a in range(d)], 1)
    U = C.copy()
    U[np.arange(len(axis)), axis] += 1
    inv = np.unique(np.concatenate([C, U]), axis=0)
    shifts = np.array(np.meshgrid(*[np.arange(2)] * d, indexing="ij")).reshape(d, -1).T
    own = (inv[:, None, :] + shifts[None, :, :]).reshape(-1, d)
    return len(np.unique(own, axis=0))


CASES = [lambda: W.small_ball(3, 14, 2, radius=0.66, seed=351), lambda: W.small_ball(2, 200, 3, seed=352),
         lambda: W.small_ball(3, 24, 1, radius=0.7, seed=353)]


@pytest.mark.parametrize("make", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_slab_counts(gplib, make, prec):
    pr = make()
    groups = -(-_owners(gplib, _ctx(gplib, pr, prec, 1), pr) // 256)
    assert groups >= 3
    for req in (0, 1, 2, 3, 7, 64, 1000):
        ctx = _ctx(gplib, pr, prec, req)
        info = gplib.gp_kernel_path(ctx)
        assert info["path"] == gplib.GP_PATH_FACE_LIFT
        want = 1 if req <= 1 or groups < 2 else min(req, groups, 64)
        assert info["slabs"] == want, (req, groups)


def test_face_output_bytes_and_default(gplib):
    pr = W.small_ball(3, 14, 2, radius=0.66, seed=351)
    for prec, vb in ((0, 8), (1, 4), (2, 8)):
        ctx = _ctx(gplib, pr, prec, 0)
        info = gplib.gp_kernel_path(ctx)
        k, L = pr.degree, (pr.degree + 1) ** 2
        assert info["scratch_bytes"] == ctx.n_faces * L * (2 * k + 1) * vb
        assert info["slabs"] == 1
    g = W.gyroid_3d(k=4, n=128)
    for prec, vb in ((1, 4), (0, 8)):
        info = gplib.gp_kernel_path(_ctx(gplib, g, prec, 0))
        assert info["scratch_bytes"] == 335664 * 25 * 9 * vb and info["slabs"] == 1


def test_negative_slabs_rejected_and_brick_has_none(gplib):
    pr = W.small_ball(3, 14, 2, radius=0.66, seed=351)
    with pytest.raises(gplib.GpError) as e:
        _ctx(gplib, pr, 0, -1)
    assert e.value.status == gplib.GP_EINVAL
    info = gplib.gp_kernel_path(_ctx(gplib, pr, 1, 5, path=gplib.GP_PATH_BRICK))
    assert info["path"] == gplib.GP_PATH_BRICK and info["slabs"] == 0
