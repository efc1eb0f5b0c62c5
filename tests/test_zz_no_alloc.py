"""The allocation-free apply, gp_apply_noalloc, against gp_apply.

gp_apply_noalloc serves callers that cannot allocate device memory when they
apply the operator (a framework allocator owns the GPU's memory, or a tight
loop must not pay for cudaMalloc/cudaFree).  It must give gp_apply's result
while keeping the face outputs in the library's fixed 32 MiB scratch: checked
through the C ABI on two calls in a row (the scratch keeps the previous call's
contents), in all three arithmetic forms, and an oversized problem must be
refused with a clear error.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2503_00246_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-12}


def _run(gp, torch, ctx, x, prec, fn):
    dt = torch.float32 if prec == 1 else torch.float64
    xd = torch.tensor(x, dtype=dt, device="cuda")
    yd = torch.full_like(xd, float("nan"))
    st = fn(ctx.handle, xd.data_ptr(), yd.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == gp.GP_OK, gp.gp_last_error(ctx)
    return yd.double().cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_matches_apply_twice(gplib, cuda, prec):
    lib = ctypes.CDLL(gplib.LIB_PATH)        # call the exported C symbol directly
    fn = lib.gp_apply_noalloc
    fn.argtypes = [ctypes.c_void_p] * 4
    fn.restype = ctypes.c_int
    problems = [W.ball_3d(), W.small_ball(2, 20, 5, seed=3)]
    for pr in problems:
        ctx = gplib.setup_problem(pr, precision=prec)
        for call in range(2):                # second call: scratch holds the first call's data
            x = W.x_vectors(pr, ctx.n_active, 2)[call]
            ref = _run(gplib, cuda, ctx, x, prec, gplib.lib.gp_apply)
            got = _run(gplib, cuda, ctx, x, prec, fn)
            assert np.all(np.isfinite(got))
            assert np.abs(got - ref).max() <= TOL[prec] * np.abs(ref).max()
        ctx.close()


def test_noalloc_refuses_oversized_problem(gplib, cuda):
    pr = W.ball_3d_sweep(4)                  # 96^3 ball, k = 4: face outputs need ~145 MB in FP64
    ctx = gplib.setup_problem(pr, precision=0)
    need = ctx.n_faces * 9 * 25 * 8
    assert need > gplib.NOALLOC_SCRATCH_BYTES
    x = cuda.zeros(ctx.n_active, dtype=cuda.float64, device="cuda")
    y = cuda.zeros_like(x)
    with pytest.raises(gplib.GpError) as e:
        gplib.gp_apply_noalloc(ctx, x, y)
    assert e.value.status == gplib.GP_EINVAL and "fixed scratch" in str(e.value)
