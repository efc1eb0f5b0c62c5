"""GPU parity of the macro-patch stabilisation (Sec. 2.2's alternative to the ghost penalty,
the same Kronecker form with a rank-k 1D matrix): y = S x against the oracle's explicit
macro-patch face matrices, in the three arithmetic forms, alone and in a batch together
with ghost-penalty problems of the same degree (they must not share 1D data)."""
import numpy as np
import pytest

from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-12}


def _close(y, ref, tol):
    assert np.all(np.isfinite(y))
    assert np.linalg.norm(y - ref) <= tol * np.linalg.norm(ref), np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert np.abs(y - ref).max() <= tol * np.abs(ref).max()


def _macro(pr):
    pr.stabilization = 1
    return pr


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("dim,n,k", [(2, 20, 1), (2, 16, 3), (2, 12, 8), (3, 10, 1), (3, 9, 2), (3, 8, 4),
                                     (3, 6, 6)])
def test_macro_patch_matches_oracle(gplib, cuda, dim, n, k, prec):
    pr = _macro(W.small_ball(dim, n, k, radius=0.62, seed=200 + k))
    o = Oracle(pr)
    ctx = gplib.setup_problem(pr, precision=prec)
    x = W.x_vectors(pr, ctx.n_active)[0]
    if prec == 1:
        x = x.astype(np.float32).astype(np.float64)
    dt = cuda.float32 if prec == 1 else cuda.float64
    xd = cuda.tensor(x, dtype=dt, device="cuda")
    yd = cuda.full_like(xd, float("nan"))
    gplib.gp_apply(ctx, xd, yd)
    cuda.cuda.synchronize()
    _close(yd.double().cpu().numpy(), o.apply(x), TOL[prec])


def test_macro_patch_ball64_k3(gplib, cuda):
    pr = _macro(W.ball_3d())
    o = Oracle(pr)
    for prec in (2, 1):
        ctx = gplib.setup_problem(pr, precision=prec)
        x = W.x_vectors(pr, ctx.n_active)[0]
        if prec == 1:
            x = x.astype(np.float32).astype(np.float64)
        dt = cuda.float32 if prec == 1 else cuda.float64
        xd = cuda.tensor(x, dtype=dt, device="cuda")
        yd = cuda.empty_like(xd)
        gplib.gp_apply(ctx, xd, yd)
        cuda.cuda.synchronize()
        _close(yd.double().cpu().numpy(), o.apply(x), TOL[prec])


def test_batch_keeps_stabilisations_apart(gplib, cuda):
    probs = [W.small_ball(3, 10, 3, seed=300), _macro(W.small_ball(3, 11, 3, seed=301)),
             W.small_ball(3, 12, 3, seed=302), _macro(W.small_ball(3, 9, 3, seed=303))]
    ctxs = [gplib.setup_problem(pr, precision=2) for pr in probs]
    xs = [cuda.tensor(W.x_vectors(pr, c.n_active)[0], dtype=cuda.float64, device="cuda") for pr, c in zip(probs, ctxs)]
    ys = [cuda.full_like(x, float("nan")) for x in xs]
    b = gplib.gp_batch_create(ctxs, 1)
    ngroups, _ = gplib.gp_batch_info(b)
    assert ngroups == 2
    gplib.gp_batch_apply(b, xs, ys)
    cuda.cuda.synchronize()
    for pr, x, y in zip(probs, xs, ys):
        _close(y.cpu().numpy(), Oracle(pr).apply(x.cpu().numpy()), TOL[2])
    gplib.gp_batch_destroy(b)
