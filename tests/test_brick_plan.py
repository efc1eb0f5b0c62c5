"""Host checks of the brick planner (no GPU): the brick shape, the bricks that hold faces and
the plane nodes follow from their definitions, recomputed here with numpy from the face list.

A brick of bdim cells holds a face when one of the face's two cells lies in it; a plane node is
a DoF of an involved cell (a cell of some ghost face) whose lattice coordinate along some axis
is a multiple of bdim[a] k strictly inside the mesh (it is shared by the bricks on both sides).
"""
import numpy as np
import pytest

from paper_2503_00246_gb300 import workloads as W


def _ctx(gp, pr, prec, path=0, smem=0):
    mesh, ls, opts, keep = gp.structs_for(pr, prec, -1)
    opts.kernel_path = path
    opts.brick_smem = smem
    return gp.gp_setup(mesh, ls, opts)


CASES = [lambda: W.small_ball(3, 14, 2, radius=0.66, seed=351), lambda: W.small_ball(2, 30, 3, seed=352),
         lambda: W.ball_3d(), lambda: W.gyroid_3d(k=2, n=24)]


@pytest.mark.parametrize("make", CASES)
@pytest.mark.parametrize("smem", [16 * 1024, 0])
def test_bricks_and_plane_nodes(gplib, make, smem):
    pr = make()
    ctx = _ctx(gplib, pr, 1, gplib.GP_PATH_BRICK, smem)
    info = gplib.gp_kernel_path(ctx)
    assert info["path"] == gplib.GP_PATH_BRICK
    d, n, k = pr.dim, pr.n, pr.degree
    B = np.array(info["bdim"][:d])
    assert np.all(B >= 1)
    axis, cell = gplib.gp_ghost_faces(ctx)
    C = np.stack([(cell // n ** a) % n for a in range(d)], 1)
    U = C.copy()
    U[np.arange(len(axis)), axis] += 1
    nb = (n + B - 1) // B
    lin = lambda c: sum((c[:, a] // B[a]) * int(np.prod(nb[:a])) for a in range(d))
    assert len(np.unique(np.concatenate([lin(C), lin(U)]))) == info["bricks"]
    # plane nodes: DoFs of involved cells on an interior brick plane
    inv = np.unique(np.concatenate([C, U]), axis=0)
    offs = np.array(np.meshgrid(*[np.arange(k + 1)] * d, indexing="ij")).reshape(d, -1).T
    nodes = np.unique((inv[:, None, :] * k + offs[None, :, :]).reshape(-1, d), axis=0)
    on = np.zeros(len(nodes), dtype=bool)
    for a in range(d):
        X = nodes[:, a]
        on |= (X % (B[a] * k) == 0) & (X > 0) & (X < n * k)
    assert on.sum() == info["plane_nodes"]
    assert info["scratch_bytes"] > 0


def test_smaller_budget_gives_smaller_bricks(gplib):
    pr = W.ball_3d()
    big = gplib.gp_kernel_path(_ctx(gplib, pr, 1, gplib.GP_PATH_BRICK))
    small = gplib.gp_kernel_path(_ctx(gplib, pr, 1, gplib.GP_PATH_BRICK, 16 * 1024))
    assert np.prod(small["bdim"]) < np.prod(big["bdim"]) and small["bricks"] > big["bricks"]
    face_lift = gplib.gp_kernel_path(_ctx(gplib, pr, 1, gplib.GP_PATH_FACE_LIFT))
    assert face_lift["path"] == gplib.GP_PATH_FACE_LIFT and face_lift["bricks"] == 0
    with pytest.raises(gplib.GpError) as e:                     # nothing fits 1 KB
        _ctx(gplib, pr, 1, gplib.GP_PATH_BRICK, 1024)
    assert e.value.status == gplib.GP_EUNSUPPORTED
