"""The float-float form (GP_FP64_FF) at the edges of its exponent range.

The pairs (hi, lo) of floats carry about 48 significant bits but only float's
exponent range; gp.h states the behaviour this file checks on the 16^3 ball, k = 3:
  * non-zero |x_i| in [2^-97, 2^127): the FP64 tolerance (1e-12) holds, here for x
    scaled by 1e-20 and 1e30;
  * 2^-126 <= |x_i| < 2^-97: only the leading 24 bits of x_i are used (x ~ 1e-30), and
    values below 2^-126 (low parts of small outputs) are lost: an absolute error floor of
    a few 2^-126;
  * |x_i| < 2^-126 reads as 0;
  * |x_i| >= 2^128 reads as infinity and makes y non-finite where its faces reach.
gp_setup's refusal of scale factors outside [2^-90, 2^90] is checked on the host
(tests/test_abi_host.py).
"""
import numpy as np
import pytest

from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _apply(gp, torch, ctx, x):
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.full_like(xd, float("nan"))
    gp.gp_apply(ctx, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _trunc24(x):
    """x with its significand cut to the leading 24 bits (toward zero)."""
    b = x.view(np.uint64) & ~np.uint64((1 << 29) - 1)
    return b.view(np.float64)


@pytest.fixture(scope="module")
def case(gplib):
    pr = W.small_ball(3, 16, 3, seed=61)
    return pr, Oracle(pr)


@pytest.mark.parametrize("scale", [1e-20, 1e30])
def test_full_accuracy_inside_the_range(gplib, cuda, case, scale):
    pr, o = case
    ctx = gplib.setup_problem(pr, precision=2)
    x = W.x_vectors(pr, ctx.n_active)[0] * scale
    y = _apply(gplib, cuda, ctx, x)
    ref = o.apply(x)
    assert np.all(np.isfinite(y))
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


def test_below_2_pow_minus_97_keeps_24_bits(gplib, cuda, case):
    pr, o = case
    ctx = gplib.setup_problem(pr, precision=2)
    x = W.x_vectors(pr, ctx.n_active)[0] * 1e-30
    assert np.abs(x[x != 0]).max() < 2.0 ** -97
    y = _apply(gplib, cuda, ctx, x)
    ref = o.apply(_trunc24(x))
    # outputs near 1e-31 have low parts below 2^-126, which float does not hold: an absolute
    # error floor of a few 2^-126 besides the relative 1e-12
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max() + 4 * 2.0 ** -126
    assert np.abs(y - o.apply(x)).max() > 1e-9 * np.abs(ref).max()    # the low bits of x are gone


def test_tiny_and_huge_entries(gplib, cuda, case):
    pr, o = case
    ctx = gplib.setup_problem(pr, precision=2)
    x = W.x_vectors(pr, ctx.n_active)[0]
    tiny = np.arange(0, ctx.n_active, 7)
    x[tiny] = 1e-40                                        # below 2^-126: read as 0
    y = _apply(gplib, cuda, ctx, x)
    x0 = x.copy()
    x0[tiny] = 0.0
    ref = o.apply(x0)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    touched = np.flatnonzero(ref != 0.0)
    x[touched[len(touched) // 2]] = 1e39                   # at or above 2^128: infinity
    y = _apply(gplib, cuda, ctx, x)
    assert not np.all(np.isfinite(y))

