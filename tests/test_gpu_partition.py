"""Slab partitions on one GPU: every partition's context applies its own faces on
its window of x (one cell of halo above), the contributions to the halo are added
into the partition above, and the owned blocks must give G x (Sec. 2.7 and the
two exchange steps of Algorithm 1).  The exchange between the partitions is done
here with device copies on one GPU, as the ranks of halo.SlabOperator do it with
point-to-point messages.

Tolerances: those of the whole-mesh parity tests (FP64 and float-float 1e-12,
FP32 1e-5 relative to the FP64 oracle); the partitioned result also agrees with
the whole-mesh apply of the same precision to a few units of its rounding.
"""
import socket

import numpy as np
import pytest

import oracle.partition as opart
from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-12}
SELF = {0: 1e-14, 1: 1e-6, 2: 1e-14}


def _partitioned_apply(gp, torch, pr, prec, P, x):
    dt = torch.float32 if prec == 1 else torch.float64
    xd = torch.tensor(x, dtype=dt, device="cuda")
    b = gp.partition_problem(pr, P)
    parts = []
    for r in range(P):
        ctx = gp.setup_problem(pr, precision=prec, part=(b[r], b[r + 1]))
        info = gp.gp_partition_info(ctx)
        xl = xd[info["offset"]:info["offset"] + info["n_local"]]     # owned block + halo above
        yl = torch.full_like(xl, float("nan"))
        gp.gp_apply(ctx, xl, yl)
        parts.append((info, yl))
    for r in range(P - 1):                                          # export / add of the halo
        info, yl = parts[r]
        nxt, yn = parts[r + 1]
        assert info["n_local"] - info["n_owned"] == nxt["n_lower"]
        yn[:nxt["n_lower"]] += yl[info["n_owned"]:]
    y = torch.cat([yl[:info["n_owned"]] for info, yl in parts])
    torch.cuda.synchronize()
    return y.double().cpu().numpy(), b


def _close(y, ref, tol):
    assert np.all(np.isfinite(y))
    nr = np.linalg.norm(ref)
    assert np.linalg.norm(y - ref) <= tol * nr, np.linalg.norm(y - ref) / nr
    assert np.abs(y - ref).max() <= tol * np.abs(ref).max()


CASES = [
    (lambda: W.small_ball(3, 12, 3, radius=0.6, seed=3), 3),
    (lambda: W.small_ball(3, 14, 5, radius=0.7, seed=8), 2),
    (lambda: W.disc_2d(), 4),
    (lambda: W.gyroid_3d(k=2, n=16), 3),
    (lambda: W.box_problem(3, 8, 4, all_faces=True), 4),
]


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_partitions_match_oracle(gplib, cuda, case, prec):
    make, P = CASES[case]
    pr = make()
    o = Oracle(pr)
    x = W.x_vectors(pr, o.n_active)[0]
    if prec == 1:
        x = x.astype(np.float32).astype(np.float64)
    y, b = _partitioned_apply(gplib, cuda, pr, prec, P, x)
    assert b.tolist() == opart.slab_bounds(pr, P, o.cls).tolist()
    _close(y, o.apply(x), TOL[prec])


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("P", [2, 4, 7])
def test_partitions_ball64_k3_match_whole_mesh(gplib, cuda, prec, P):
    pr = W.ball_3d()
    whole = gplib.setup_problem(pr, precision=prec)
    x = W.x_vectors(pr, whole.n_active)[0]
    if prec == 1:
        x = x.astype(np.float32).astype(np.float64)
    dt = cuda.float32 if prec == 1 else cuda.float64
    xd = cuda.tensor(x, dtype=dt, device="cuda")
    yd = cuda.empty_like(xd)
    gplib.gp_apply(whole, xd, yd)
    y_whole = yd.double().cpu().numpy()
    y, _ = _partitioned_apply(gplib, cuda, pr, prec, P, x)
    _close(y, y_whole, SELF[prec])


def test_partition_refused_by_model_system(gplib, cuda):
    pr = W.small_ball(3, 10, 2, seed=2)
    ctx = gplib.setup_problem(pr, precision=0, part=(0, 5))
    with pytest.raises(gplib.GpError) as e:
        gplib.gp_system_create(ctx)
    assert e.value.status == gplib.GP_EUNSUPPORTED


def test_slab_operator_single_rank(gplib, cuda):
    # halo.SlabOperator on a one-rank group: the whole mesh as one partition
    import torch.distributed as dist
    from paper_2503_00246_gb300 import halo
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        pr = W.small_ball(3, 12, 3, seed=9)
        o = Oracle(pr)
        op = halo.SlabOperator(pr, precision=0)
        assert op.bounds.tolist() == [0, 12]
        assert op.info["n_local"] == op.info["n_owned"] == o.n_active
        x = W.x_vectors(pr, o.n_active)[0]
        xd = cuda.tensor(x, dtype=cuda.float64, device="cuda")
        yd = cuda.empty_like(xd)
        op.apply(xd, yd)
        cuda.cuda.synchronize()
        _close(yd.cpu().numpy(), o.apply(x), TOL[0])
    finally:
        dist.destroy_process_group()
