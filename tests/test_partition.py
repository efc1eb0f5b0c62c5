"""Slab partitions through the C-ABI host plan (no GPU) and the halo exchange of
paper_2503_00246_gb300.halo on gloo ranks (world sizes 2 and 3, CPU).

Sec. 2.7: weighted load balance, faces across a partition boundary evaluated by
the lower rank, ghost values of u imported before the face loop and ghost
contributions of w added on their owners afterwards (Algorithm 1).  On the CPU
ranks the face loop of each rank is the oracle restricted to the faces the
rank's context lists; the exchange is the product's.
"""
import os
import socket

import numpy as np
import pytest

import oracle.partition as opart
from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W

CASES = [
    (lambda: W.small_ball(3, 12, 2, radius=0.6, seed=3), 2),
    (lambda: W.small_ball(3, 12, 2, radius=0.6, seed=3), 3),
    (lambda: W.small_ball(2, 20, 3, radius=0.7, seed=4), 2),
    (lambda: W.small_ball(3, 10, 3, radius=0.8, seed=5), 4),
    (lambda: W.gyroid_3d(k=2, n=16), 3),
    (lambda: W.box_problem(3, 6, 2, all_faces=True), 3),
]


def _face_mask(o, ax, cell):
    """Per-axis masks of the oracle faces listed by a context (axis, lower-cell index)."""
    fl = o.face_list()
    keys = set(zip(ax.tolist(), cell.tolist()))
    sel = np.array([(int(a), int(c)) in keys for a, c in fl], dtype=bool)
    out, pos = [], 0
    for a in range(o.pr.dim):
        m = o.faces[a].shape[0]
        out.append(sel[pos:pos + m])
        pos += m
    return out


@pytest.mark.parametrize("make,P", CASES)
def test_slab_bounds_match_oracle(gplib, make, P):
    pr = make()
    assert gplib.partition_problem(pr, P).tolist() == opart.slab_bounds(pr, P).tolist()


@pytest.mark.parametrize("make,P", CASES)
def test_partition_plans_match_oracle(gplib, make, P):
    pr = make()
    o = Oracle(pr)
    b = gplib.partition_problem(pr, P)
    owners = opart.face_owner(pr, o.faces, b)
    coords = o.num.coords()
    fl = o.face_list()
    own_all = np.concatenate(owners) if owners else np.zeros(0, dtype=np.int64)
    nf = 0
    for r in range(P):
        ctx = gplib.setup_problem(pr, device=-1, part=(b[r], b[r + 1]))
        info = gplib.gp_partition_info(ctx)
        assert info == opart.window(pr, o.num, b, r)
        assert ctx.n_active == info["n_local"]
        ax, cell = gplib.gp_ghost_faces(ctx)
        assert np.array_equal(np.stack([ax, cell], 1), fl[own_all == r])
        nf += ctx.n_faces
        s = slice(info["offset"], info["offset"] + info["n_local"])
        np.testing.assert_allclose(gplib.gp_active_dof_coords(ctx), coords[s], rtol=0, atol=1e-14 * 4)
        mask = [ow == r for ow in owners]
        pidx = [o.patch_index(a)[mask[a]].ravel() for a in range(pr.dim)]
        touched = np.unique(np.concatenate(pidx)) if pidx else np.zeros(0)
        assert ctx.n_touched == touched.size
    assert nf == o.n_faces


def test_whole_mesh_partition_info(gplib):
    ctx = gplib.setup_problem(W.small_ball(3, 8, 2, seed=2), device=-1)
    info = gplib.gp_partition_info(ctx)
    assert info["offset"] == 0 and info["n_lower"] == 0
    assert info["n_local"] == info["n_owned"] == info["n_global"] == ctx.n_active
    assert (info["layer_lo"], info["layer_hi"]) == (0, 8)


def test_partition_argument_errors(gplib):
    pr = W.small_ball(3, 10, 2, seed=2)
    for part in [(3, 4), (-1, 4), (4, 11), (5, 5), (6, 2)]:
        with pytest.raises(gplib.GpError) as e:
            gplib.setup_problem(pr, device=-1, part=part)
        assert e.value.status == gplib.GP_EINVAL
    # one layer is allowed at either end of the mesh
    for part in [(0, 1), (9, 10)]:
        gplib.setup_problem(pr, device=-1, part=part)
    with pytest.raises(gplib.GpError):
        gplib.partition_problem(pr, 6)
    with pytest.raises(gplib.GpError):
        gplib.partition_problem(pr, 0)


# ------------------------------------------------------------- gloo ranks --

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, case, dtype_name):
    import torch
    import torch.distributed as dist
    from paper_2503_00246_gb300 import gp, halo

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        make, _ = CASES[case]
        pr = make()
        dtype = getattr(torch, dtype_name)
        o = Oracle(pr)
        b = gp.partition_problem(pr, ws)
        ctx = gp.setup_problem(pr, device=-1, part=(b[rank], b[rank + 1]))
        info = gp.gp_partition_info(ctx)
        x = W.x_vectors(pr, o.n_active)[0]
        s = slice(info["offset"], info["offset"] + info["n_local"])
        x_loc = torch.full((info["n_local"],), float("nan"), dtype=dtype)
        x_loc[:info["n_owned"]] = torch.from_numpy(x[s][:info["n_owned"]]).to(dtype)
        halo.import_halo(x_loc, info)
        assert torch.equal(x_loc, torch.from_numpy(x[s]).to(dtype)), "halo import"
        # this rank's face loop: the oracle on the faces its context lists, with only the
        # window of x known (zeros elsewhere)
        ax, cell = gp.gp_ghost_faces(ctx)
        xg = np.zeros(o.n_active)
        xg[s] = x_loc.double().numpy()
        y_loc = torch.from_numpy(o.apply(xg, _face_mask(o, ax, cell))[s].copy()).to(dtype)
        halo.export_add(y_loc, info)
        y_ref = o.apply(x)[s][:info["n_owned"]]
        got = y_loc[:info["n_owned"]].double().numpy()
        tol = 1e-13 if dtype == torch.float64 else 1e-6
        scale = max(np.abs(o.apply(x)).max(), 1e-300)
        assert np.abs(got - y_ref).max() <= tol * scale, (rank, np.abs(got - y_ref).max() / scale)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", [1, 2, 3, 4])
@pytest.mark.parametrize("dtype_name", ["float64", "float32"])
def test_gloo_ranks_halo_exchange(gplib, case, dtype_name):
    import torch.multiprocessing as mp
    ws = CASES[case][1]
    mp.start_processes(_rank_main, args=(ws, _free_port(), case, dtype_name), nprocs=ws,
                       join=True, start_method="spawn")
