"""C-ABI library checks that need no GPU: exports, host plan vs the oracle,
1D reference data vs an independent construction, argument errors."""
import ctypes
import os
import re

import numpy as np
import pytest
from numpy.polynomial import Legendre

from oracle.basis import gauss_lobatto_nodes
from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "gp.h")


def test_library_exports_every_declared_symbol(gplib):
    src = open(HEADER).read()
    declared = set(re.findall(r"^\s*(?:gp_status|void|const char\*)\s+(gp_\w+)\s*\(", src, re.M))
    assert declared == set(gplib.ABI_SYMBOLS)
    lib = ctypes.CDLL(gplib.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert "sm_103a" in gplib.gp_version()


PROBLEMS = [
    lambda: W.disc_2d(),
    lambda: W.small_ball(2, 24, 5, seed=3),
    lambda: W.small_ball(3, 9, 2, seed=5),
    lambda: W.small_ball(3, 14, 1, radius=0.45, seed=6),
    lambda: W.ball_3d(),
    lambda: W.gyroid_3d(k=2, n=24),
    lambda: W.box_problem(3, 4, 2, all_faces=True),
    lambda: W.box_problem(2, 5, 3, all_faces=False),
]


@pytest.mark.parametrize("make", PROBLEMS)
def test_host_plan_matches_oracle(gplib, make):
    pr = make()
    ctx = gplib.setup_problem(pr, device=-1)
    o = Oracle(pr)
    assert ctx.n_active == o.n_active
    assert ctx.n_faces == o.n_faces
    ax, cell = gplib.gp_ghost_faces(ctx)
    assert np.array_equal(np.stack([ax, cell], 1), o.face_list())
    cls = gplib.gp_cell_classes(ctx, pr.n ** pr.dim)
    assert np.array_equal(cls, o.cls.transpose().ravel())
    np.testing.assert_allclose(gplib.gp_active_dof_coords(ctx), o.num.coords(), rtol=0, atol=1e-14 * max(abs(pr.lo), abs(pr.hi)))
    counts = gplib.gp_cell_counts(ctx)
    assert list(counts) == [int((o.cls == c).sum()) for c in range(3)]
    if o.n_faces:
        touched = np.unique(np.concatenate([o.patch_index(a).ravel() for a in range(pr.dim)]))
        assert ctx.n_touched == touched.size
    else:
        assert ctx.n_touched == 0


@pytest.mark.parametrize("k", range(1, 9))
def test_reference_1d_against_independent_fits(gplib, k):
    pr = W.small_ball(3, 6, k, seed=2, weights=W.paper_weights(0.5, k))
    ctx = gplib.setup_problem(pr, device=-1)
    M, g, s = gplib.gp_reference_1d(ctx)
    xi = gauss_lobatto_nodes(k)
    polys = []
    for m in range(k + 1):
        e = np.zeros(k + 1)
        e[m] = 1
        polys.append(Legendre.fit(xi, e, k, domain=[0, 1]))
    Mref = np.array([[((pa * pb).integ()(1.0) - (pa * pb).integ()(0.0)) for pb in polys] for pa in polys])
    np.testing.assert_allclose(M, Mref, rtol=1e-12, atol=1e-14)
    hi = [Legendre.fit(1 + xi, np.eye(k + 1)[m], k, domain=[1, 2]) for m in range(k + 1)]
    for j in range(1, k + 1):
        gref = np.zeros(2 * k + 1)
        for b in range(2 * k + 1):
            if b <= k:
                gref[b] += polys[b].deriv(j)(1.0)
            if b >= k:
                gref[b] -= hi[b - k].deriv(j)(1.0)
        np.testing.assert_allclose(g[j - 1], gref, rtol=1e-9, atol=1e-9 * np.abs(gref).max())
        # symmetry of the patch under reflection about the face: g_j[2k-b] = (-1)^(j+1) g_j[b]
        np.testing.assert_allclose(g[j - 1][::-1], (-1) ** (j + 1) * g[j - 1],
                                   rtol=1e-10, atol=1e-10 * np.abs(g[j - 1]).max())
    np.testing.assert_allclose(s, np.array(W.paper_weights(0.5, k)) * pr.h, rtol=1e-15)


def test_setup_errors(gplib):
    pr = W.small_ball(3, 6, 3)
    mesh, ls, opts, keep = gplib.structs_for(pr, device=-1)
    for field, val, status in (("degree", 9, gplib.GP_EUNSUPPORTED), ("degree", 0, gplib.GP_EINVAL),
                               ("precision", 7, gplib.GP_EINVAL), ("nweights", 2, gplib.GP_EINVAL)):
        old = getattr(opts, field)
        setattr(opts, field, val)
        with pytest.raises(gplib.GpError) as e:
            gplib.gp_setup(mesh, ls, opts)
        assert e.value.status == status
        setattr(opts, field, old)
    mesh.dim = 4
    with pytest.raises(gplib.GpError):
        gplib.gp_setup(mesh, ls, opts)
    mesh.dim = 3
    mesh.hi[1] = 3.0  # non-cubic cells
    with pytest.raises(gplib.GpError):
        gplib.gp_setup(mesh, ls, opts)


def test_host_only_context_refuses_apply(gplib):
    ctx = gplib.setup_problem(W.small_ball(2, 8, 2), device=-1)
    st = gplib.lib.gp_apply(ctx.handle, 16, 32, None)
    assert st == gplib.GP_EDEVICE
    assert "host-only" in gplib.gp_last_error(ctx)


@pytest.mark.parametrize("k", [2, 4, 6, 8])
def test_reference_1d_high_precision(gplib, k):
    """Jumps g_j and mass M^ within 2e-15 (relative per row) of a 60-digit evaluation."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    xi = gauss_lobatto_nodes(k)
    xm = []
    for v in xi:
        if v in (0.0, 1.0):
            xm.append(mp.mpf(v))
            continue
        f = lambda s: mp.diff(lambda u: mp.legendre(k, u), s)   # noqa: E731
        xm.append((mp.findroot(f, mp.mpf(2 * v - 1)) + 1) / 2)

    def lag(nodes, m):
        coef = [mp.mpf(1)]
        for i, xq in enumerate(nodes):
            if i == m:
                continue
            a0, a1 = -xq / (nodes[m] - xq), 1 / (nodes[m] - xq)
            new = [mp.mpf(0)] * (len(coef) + 1)
            for p, c in enumerate(coef):
                new[p] += c * a0
                new[p + 1] += c * a1
            coef = new
        return coef                                              # monomial coefficients

    def deriv(coef, x, j):
        return sum(mp.factorial(p) / mp.factorial(p - j) * c * x ** (p - j)
                   for p, c in enumerate(coef) if p >= j)

    lo = [lag(xm, m) for m in range(k + 1)]
    hi = [lag([1 + u for u in xm], m) for m in range(k + 1)]
    ctx = gplib.setup_problem(W.small_ball(3, 6, k, seed=2), device=-1)
    M, g, _ = gplib.gp_reference_1d(ctx)
    for j in range(1, k + 1):
        ref = np.array([float((deriv(lo[b], 1, j) if b <= k else 0) - (deriv(hi[b - k], 1, j) if b >= k else 0))
                        for b in range(2 * k + 1)])
        assert np.abs(g[j - 1] - ref).max() <= 2e-15 * np.abs(ref).max(), j
    Mref = np.zeros((k + 1, k + 1))
    for a in range(k + 1):
        for b in range(k + 1):
            prod = [mp.mpf(0)] * (2 * k + 1)
            for p, ca in enumerate(lo[a]):
                for q, cb in enumerate(lo[b]):
                    prod[p + q] += ca * cb
            Mref[a, b] = float(sum(c / (p + 1) for p, c in enumerate(prod)))
    assert np.abs(M - Mref).max() <= 2e-15 * np.abs(Mref).max()


def test_tile_shapes_host(gplib):
    # defaults, range checks and the process-wide table (no kernel runs)
    ctx = gplib.setup_problem(W.small_ball(3, 8, 3, seed=2), precision=2, device=-1)
    t = gplib.gp_get_tiles(ctx)
    assert t["faces_per_cta"] * 16 <= 512 and t["lift_threads"] % 32 == 0
    good = {"faces_per_cta": 32, "lift_cells_per_cta": 8, "lift_threads": 128}
    gplib.gp_set_tiles(ctx, good)
    assert gplib.gp_get_tiles(ctx) == good
    for bad in [{"faces_per_cta": 33}, {"lift_threads": 100}, {"lift_threads": 1024},
                {"lift_cells_per_cta": 1000}, {"faces_per_cta": -1}]:
        with pytest.raises(gplib.GpError):
            gplib.gp_set_tiles(ctx, bad)
    assert gplib.gp_get_tiles(ctx) == good
    with pytest.raises(gplib.GpError):
        gplib.gp_tiles_record(0, 4, 3, 0, good)
    with pytest.raises(gplib.GpError):
        gplib.gp_autotune(ctx)                      # host-only context
    gplib.gp_tiles_record(-1, 2, 7, 1, {"faces_per_cta": 4})
    assert gplib.gp_tiles_lookup(-1, 2, 7, 1) == {"faces_per_cta": 4, "lift_cells_per_cta": 0, "lift_threads": 0}
    assert gplib.gp_tiles_lookup(-1, 2, 6, 1) is None


@pytest.mark.parametrize("k", range(1, 9))
def test_jump_vectors_mirror_symmetry(gplib, k):
    # Reflecting the patch about the face swaps K- and K+, maps basis b to 2k - b and
    # flips d/dn: g_j[2k - b] = (-1)^(j+1) g_j[b], so g_j[k] = 0 for even j.  The face
    # kernel uses only b <= k of each g_j and relies on this.
    ctx = gplib.setup_problem(W.small_ball(3, 6, k), device=-1)
    _, g, _ = gplib.gp_reference_1d(ctx)
    g = np.asarray(g).reshape(k, 2 * k + 1)
    for j in range(1, k + 1):
        row = g[j - 1]
        scale = np.abs(row).max()
        assert np.abs(row[::-1] * (-1) ** (j + 1) - row).max() <= 1e-14 * scale
        if j % 2 == 0:
            assert abs(row[k]) <= 1e-14 * scale


@pytest.mark.parametrize("k", range(1, 9))
def test_reference_mass_centrosymmetric(gplib, k):
    # The Gauss-Lobatto nodes are symmetric about the cell centre, so reversing the node
    # order maps M^ to itself: M^[k-a][k-b] = M^[a][b].  The cell kernel of the model system
    # applies M^ (and S^, which the library checks when a system is created) through its
    # even and odd halves and relies on this.
    ctx = gplib.setup_problem(W.small_ball(3, 6, k), device=-1)
    m, _, _ = gplib.gp_reference_1d(ctx)
    m = np.asarray(m)
    assert np.abs(m[::-1, ::-1] - m).max() <= 1e-15 * np.abs(m).max()


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 4), (2, 8), (3, 2), (3, 3), (3, 5)])
def test_macro_patch_1d_data_matches_oracle(gplib, dim, k):
    # the host's rank-k form gamma h^d sum_j lambda_j (M^ x ... x v_j v_j^T) against the oracle's
    # explicit macro-patch face matrix (no factorisation there)
    from oracle.macro_patch import face_matrix_macro
    pr = W.small_ball(dim, 8, k, seed=4)
    pr.stabilization = gplib.GP_STAB_MACRO
    ctx = gplib.setup_problem(pr, device=-1)
    mass, g, s = gplib.gp_reference_1d(ctx)
    M = np.asarray(mass).reshape(k + 1, k + 1)
    g = np.asarray(g).reshape(k, 2 * k + 1)
    s = np.asarray(s)
    G = sum(s[j] * np.outer(g[j], g[j]) for j in range(k))
    # mirror parities alternate (odd orders symmetric), as the face kernel's even-odd split assumes
    for j in range(k):
        assert np.abs(g[j][::-1] * (1 if j % 2 == 0 else -1) - g[j]).max() <= 1e-15 * np.abs(g[j]).max()
    for axis in range(dim):
        fac = [G if a == axis else M for a in range(dim)]
        K = fac[-1]
        for f in reversed(fac[:-1]):
            K = np.kron(K, f)
        A = face_matrix_macro(dim, k, pr.h, axis, pr.gamma)
        assert np.abs(A - K).max() <= 1e-11 * np.abs(A).max(), axis


def test_callback_level_set_and_non_finite_values(gplib):
    # a callback ball phi = r - |x - c| (Lipschitz 1) classifies like the exact ball test up to
    # the sampling margin: every exactly inside/outside cell keeps its class or becomes cut
    import math
    pr = W.small_ball(3, 12, 2, radius=0.6, seed=9)
    c = np.asarray(pr.centers, dtype=np.float64).reshape(-1, 3)[0]
    exact = gplib.setup_problem(pr, device=-1)
    mesh, ls, opts, keep = gplib.structs_for(pr, device=-1)

    def ball(xp, user):
        return 0.6 - math.sqrt(sum((xp[a] - c[a]) ** 2 for a in range(3)))
    fn = gplib.LEVELSET_FN(ball)
    ls.kind = gplib.GP_LS_CALLBACK
    ls.fn = fn
    ls.lipschitz = 1.0
    ctx = gplib.gp_setup(mesh, ls, opts)
    ce = gplib.gp_cell_classes(exact, 12 ** 3)
    cc = gplib.gp_cell_classes(ctx, 12 ** 3)
    assert np.all((cc == ce) | (cc == 1))
    assert np.count_nonzero(cc == 2) > 0 and np.count_nonzero(cc == 0) > 0

    def bad(xp, user):
        return float("nan") if xp[0] > 0.5 else 1.0
    ls.fn = gplib.LEVELSET_FN(bad)
    with pytest.raises(gplib.GpError) as e:
        gplib.gp_setup(mesh, ls, opts)
    assert e.value.status == gplib.GP_EINVAL and "finite" in str(e.value)


def test_noalloc_limit_and_struct_layout_match_header(gplib):
    """The binding's copy of GP_NOALLOC_SCRATCH_BYTES and of gp_opts' fields follow gp.h."""
    src = open(HEADER).read()
    m = re.search(r"#define GP_NOALLOC_SCRATCH_BYTES \(\(size_t\)(\d+) << (\d+)\)", src)
    assert m and int(m.group(1)) << int(m.group(2)) == gplib.NOALLOC_SCRATCH_BYTES
    body = re.search(r"typedef struct \{([^{}]*?)\} gp_opts;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        if decl.strip():
            names += [part.replace("*", " ").split()[-1] for part in decl.split(",")]
    assert names == [f for f, _ in gplib.gp_opts._fields_]


def test_ff_setup_refuses_extreme_scale_factors(gplib):
    """GP_FP64_FF keeps float's exponent range: gp_setup refuses scale factors c_j h^(d-2)
    outside [2^-90, 2^90] (native FP64 accepts them)."""
    pr = W.small_ball(3, 8, 2, seed=62)
    pr.weights = [1e30, 0.5]                               # c_1 h = 1e30 * 0.25 > 2^90
    with pytest.raises(gplib.GpError) as e:
        gplib.setup_problem(pr, precision=2, device=-1)
    assert e.value.status == gplib.GP_EINVAL and "2^90" in str(e.value)
    gplib.setup_problem(pr, precision=0, device=-1).close()    # native FP64 accepts it
