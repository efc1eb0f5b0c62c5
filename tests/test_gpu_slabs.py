"""GPU: the slab pipeline of the face + lift path (gp_opts.slabs).

With slabs = n > 1 an apply runs a face and a lift launch per slab of lift owners (about n
ranges of whole groups of 256 owners along the last axis), each lift overlapping the next face
launch.  Every face output and every DoF is computed by the same code in the same order as with
one face and one lift launch, so the results must agree bit for bit.  Checked: bitwise equality
with slabs = 1 for the three arithmetics, d = 2 and 3, several slab counts (including more slabs
than owner groups), the overwrite and the add form; consecutive applies on one stream (each
apply's first launch waits for the previous apply's last lift); the model system's apply
followed by its cell operator; the solver's captured graphs; the full-size 128^3 gyroid
k = 4 workload; element-wise parity with the oracle of one slabbed case.
"""
import numpy as np
import pytest

from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-12}


def _dev(torch, x, prec):
    dt = torch.float32 if prec == 1 else torch.float64
    return torch.tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")


def _run(gp, torch, ctx, x, prec, y0=None, reps=1):
    """y = G x (y0 None) or y = y0 + G x, then reps - 1 further y += G x, on one stream."""
    xd = _dev(torch, x, prec)
    if y0 is None:
        yd = torch.full_like(xd, float("nan"))
        gp.gp_apply(ctx, xd, yd)
    else:
        yd = _dev(torch, y0, prec)
        gp.gp_apply_add(ctx, xd, yd)
    for _ in range(reps - 1):
        gp.gp_apply_add(ctx, xd, yd)
    torch.cuda.synchronize()
    return yd.double().cpu().numpy()


CASES = [(3, 2, 14, 0.66), (3, 4, 12, 0.6), (2, 3, 200, 0.7), (3, 1, 24, 0.7)]


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("dim,k,n,r", CASES)
def test_slabs_bitwise_equal_to_one_launch_pair(gplib, cuda, prec, dim, k, n, r):
    pr = W.small_ball(dim, n, k, radius=r, seed=400 + 10 * dim + k)
    one = gplib.setup_problem(pr, precision=prec, slabs=1)
    assert gplib.gp_kernel_path(one)["slabs"] == 1
    x, y0 = W.x_vectors(pr, one.n_active, 2)
    ref = _run(gplib, cuda, one, x, prec)
    ref_add = _run(gplib, cuda, one, x, prec, y0=y0, reps=3)
    seen = set()
    for ns in (2, 3, 7, 64):
        ctx = gplib.setup_problem(pr, precision=prec, slabs=ns)
        got = gplib.gp_kernel_path(ctx)["slabs"]
        assert 1 <= got <= ns
        seen.add(got)
        y = _run(gplib, cuda, ctx, x, prec)
        assert np.array_equal(y, ref), (ns, got)
        y = _run(gplib, cuda, ctx, x, prec, y0=y0, reps=3)
        assert np.array_equal(y, ref_add), (ns, got)
    assert max(seen) >= 3        # the cases span several owner groups


def test_slabbed_apply_matches_oracle(gplib, cuda):
    pr = W.small_ball(3, 18, 2, radius=0.66, seed=442)
    o = Oracle(pr)
    for prec in (0, 1, 2):
        ctx = gplib.setup_problem(pr, precision=prec, slabs=5)
        assert gplib.gp_kernel_path(ctx)["slabs"] == 5
        x = W.x_vectors(pr, ctx.n_active)[0]
        xin = x if prec != 1 else x.astype(np.float32).astype(np.float64)
        ref = o.apply(xin)
        y = _run(gplib, cuda, ctx, x, prec)
        assert np.abs(y - ref).max() <= TOL[prec] * np.abs(ref).max()


@pytest.mark.parametrize("hi", [0, 2])
def test_system_apply_and_cells_with_slabs(gplib, cuda, hi):
    """The model system applies G (slabbed) and then its cell operator as a programmatic
    dependent of the last lift: y = (M + K + G) x must not depend on the slab count."""
    pr = W.small_ball(3, 16, 3, radius=0.6, seed=443)
    out = []
    for ns in (1, 4):
        chi = gplib.setup_problem(pr, precision=hi, slabs=ns)
        clo = gplib.setup_problem(pr, precision=1, slabs=ns)
        sysm = gplib.gp_system_create(chi, clo)
        x = W.x_vectors(pr, chi.n_active)[0]
        res = []
        for which, prec in ((0, hi), (1, 1)):
            xd = _dev(cuda, x, prec)
            yd = cuda.full_like(xd, float("nan"))
            gplib.gp_system_apply(sysm, which, xd, yd)
            cuda.cuda.synchronize()
            res.append(yd.double().cpu().numpy())
        out.append(res)
        sysm.close()
    for a, b in zip(out[0], out[1]):
        assert np.all(np.isfinite(a)) and np.array_equal(a, b)


@pytest.mark.parametrize("prec", [1, 0])
def test_full_size_gyroid_slabs(gplib, cuda, prec):
    """128^3 gyroid, k = 4 (face outputs of 0.3 / 0.6 GB): ten slabs against one launch pair,
    bit for bit, overwrite and add form."""
    pr = W.gyroid_3d(k=4, n=128)
    auto = gplib.setup_problem(pr, precision=prec, slabs=10)
    assert gplib.gp_kernel_path(auto)["slabs"] == 10
    x = W.x_vectors(pr, auto.n_active)[0]
    y_auto = _run(gplib, cuda, auto, x, prec, reps=2)
    auto.close()
    one = gplib.setup_problem(pr, precision=prec, slabs=1)
    y_one = _run(gplib, cuda, one, x, prec, reps=2)
    assert np.all(np.isfinite(y_one)) and np.array_equal(y_auto, y_one)


@pytest.mark.parametrize("hi", [0, 2])
def test_solver_graph_with_slabs(gplib, cuda, hi):
    """The solver captures its iterations (applies included) in a CUDA graph; with slabbed
    contexts the programmatic launches of the pipeline become graph edges.  Defect correction
    and PCG must give the same iterates, bit for bit, as with one launch pair."""
    pr = W.small_ball(3, 16, 3, radius=0.62, seed=91)
    b = W.rhs_vector(pr, gplib.setup_problem(pr, precision=hi, device=-1).n_active)
    res = []
    for ns in (1, 4):
        chi = gplib.setup_problem(pr, precision=hi, slabs=ns)
        clo = gplib.setup_problem(pr, precision=1, slabs=ns)
        assert gplib.gp_kernel_path(chi)["slabs"] == ns and gplib.gp_kernel_path(clo)["slabs"] == ns
        sysm = gplib.gp_system_create(chi, clo)
        bd = cuda.tensor(b, dtype=cuda.float64, device="cuda")
        u_dc, u_cg = cuda.zeros_like(bd), cuda.zeros_like(bd)
        st_dc = gplib.gp_system_solve(sysm, bd, u_dc, rtol=1e-9, inner_rtol=1e-4, mode=0)
        st_cg = gplib.gp_system_solve(sysm, bd, u_cg, rtol=1e-9, mode=1)
        assert st_dc["rel_residual"] <= 1e-9 and st_cg["rel_residual"] <= 1e-9
        res.append((st_dc["inner"], st_cg["inner"], u_dc.cpu().numpy(), u_cg.cpu().numpy()))
        sysm.close()
    (i0, j0, a0, c0), (i1, j1, a1, c1) = res
    assert (i0, j0) == (i1, j1)
    assert np.array_equal(a0, a1) and np.array_equal(c0, c1)
