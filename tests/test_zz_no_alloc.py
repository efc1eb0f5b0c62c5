"""The allocation-free apply, gp_apply_noalloc, against gp_apply.

gp_apply_noalloc serves callers that cannot allocate device memory when they
apply the operator (a framework allocator owns the GPU's memory, or a tight
loop must not pay for cudaMalloc/cudaFree).  It runs the same kernels in the
same order as gp_apply, with the face outputs in the library's fixed 32 MiB
scratch instead of the context's buffer, so its result must equal gp_apply's
bit for bit: checked through the C ABI on two calls in a row (the scratch keeps
the previous call's contents), in all three arithmetic forms, for a context
with its own scratch and for one created with no_scratch = 1 (which allocates
none).  An oversized problem must be refused with a clear error.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2503_00246_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(gp, torch, ctx, x, prec, fn):
    dt = torch.float32 if prec == 1 else torch.float64
    xd = torch.tensor(x, dtype=dt, device="cuda")
    yd = torch.full_like(xd, float("nan"))
    st = fn(ctx.handle, xd.data_ptr(), yd.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == gp.GP_OK, gp.gp_last_error(ctx)
    return yd.double().cpu().numpy()


def _setup(gp, pr, prec, no_scratch):
    mesh, ls, opts, keep = gp.structs_for(pr, prec, 0)
    opts.no_scratch = no_scratch
    return gp.gp_setup(mesh, ls, opts)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_matches_apply_twice(gplib, cuda, prec):
    lib = ctypes.CDLL(gplib.LIB_PATH)        # call the exported C symbol directly
    fn = lib.gp_apply_noalloc
    fn.argtypes = [ctypes.c_void_p] * 4
    fn.restype = ctypes.c_int
    problems = [W.ball_3d(), W.small_ball(2, 20, 5, seed=3)]
    for pr in problems:
        ctx = gplib.setup_problem(pr, precision=prec)
        bare = _setup(gplib, pr, prec, 1)
        for call in range(2):                # second call: scratch holds the first call's data
            x = W.x_vectors(pr, ctx.n_active, 2)[call]
            ref = _run(gplib, cuda, ctx, x, prec, gplib.lib.gp_apply)
            got = _run(gplib, cuda, ctx, x, prec, fn)
            got_bare = _run(gplib, cuda, bare, x, prec, fn)
            assert np.all(np.isfinite(got))
            assert np.array_equal(got, ref)        # same kernels, same order: bitwise
            assert np.array_equal(got_bare, ref)
        xd = cuda.zeros(ctx.n_active, dtype=cuda.float32 if prec == 1 else cuda.float64, device="cuda")
        with pytest.raises(gplib.GpError) as e:    # a no_scratch context has no buffer for gp_apply
            gplib.gp_apply(bare, xd, cuda.zeros_like(xd))
        assert e.value.status == gplib.GP_EINVAL and "no_scratch" in str(e.value)
        bare.close()
        ctx.close()


def test_noalloc_refuses_oversized_problem(gplib, cuda):
    # face + lift path: the 96^3 ball at k = 4 has ~114 MB of face outputs in FP64
    pr = W.ball_3d_sweep(4)
    ctx = gplib.setup_problem(pr, precision=0, path=gplib.GP_PATH_FACE_LIFT)
    need = ctx.n_faces * 9 * 25 * 8
    assert need > gplib.NOALLOC_SCRATCH_BYTES
    x = cuda.zeros(ctx.n_active, dtype=cuda.float64, device="cuda")
    y = cuda.zeros_like(x)
    with pytest.raises(gplib.GpError) as e:
        gplib.gp_apply_noalloc(ctx, x, y)
    assert e.value.status == gplib.GP_EINVAL and "fixed scratch" in str(e.value)
    # brick path: the partial sums of the 128^3 gyroid's plane nodes exceed 32 MiB in FP64
    ctx = gplib.setup_problem(W.gyroid_3d(), precision=0, path=gplib.GP_PATH_BRICK)
    assert gplib.gp_kernel_path(ctx)["scratch_bytes"] > gplib.NOALLOC_SCRATCH_BYTES
    x = cuda.zeros(ctx.n_active, dtype=cuda.float64, device="cuda")
    y = cuda.zeros_like(x)
    with pytest.raises(gplib.GpError) as e:
        gplib.gp_apply_noalloc(ctx, x, y)
    assert e.value.status == gplib.GP_EINVAL and "fixed scratch" in str(e.value)
