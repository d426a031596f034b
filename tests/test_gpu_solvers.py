"""HODLR preconditioner and GMRES on the GPU, checked against the FP64 oracle.

Tolerances: GMRES stops on the FP64 residual of the DAFMM operator, which
differs from the oracle's A by ~1e-11 relative (the matvec parity), so the
oracle residual of the returned solution is checked at tol + 1e-10.  The HODLR
apply is an exact (Woodbury) inverse of the exported A~, so it is checked
against a dense LU solve of A~ at 1e-10 in FP64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2204_00326_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    import paper_2204_00326_gb300 as pkg

    pkg.build()
    from paper_2204_00326_gb300 import native

    return native


@pytest.fixture(scope="module")
def grid32(N):
    from paper_2204_00326_gb300.operator import DafmmOperator

    w = W.GRID32_K8
    op = DafmmOperator(w.n_side, w.kappa, lambda xy: W.contrast(w, xy))
    A = O.dense_A(O.K_dense(w.n_side, w.kappa), op.q, w.kappa)
    f = -w.kappa ** 2 * op.q * W.plane_waves(w.kappa, op.xy)[:, 0]
    yield w, op, A, f
    op.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_hodlr_full_rank_is_A(N, grid32):
    w, op, A, f = grid32
    M = N.hodlr_factor(op.ops, rank=512, leaf_size=64)
    info = N.hodlr_info(M)
    assert info["levels"] == 4 and info["leaf_size"] == 64
    At = N.hodlr_export(M, w.N)
    assert np.abs(At - A).max() < 1e-12 * np.abs(A).max()
    b = W.random_vector(w.N, 1, seed=4)[:, 0]
    x = torch.empty(w.N, dtype=torch.complex128, device="cuda")
    N.hodlr_solve(M, torch.as_tensor(b, device="cuda"), x, N.DAFMM_FP64)
    assert _rel(x.cpu().numpy(), O.lu_solve(A, b)) < 1e-10
    N.hodlr_destroy(M)


@pytest.mark.parametrize("rank", [5, 15])
def test_hodlr_apply_is_inverse_of_exported_matrix(N, grid32, rank):
    w, op, A, f = grid32
    M = N.hodlr_factor(op.ops, rank=rank, leaf_size=64)
    At = N.hodlr_export(M, w.N)
    b = W.random_vector(w.N, 1, seed=5)[:, 0]
    ref = O.lu_solve(At, b)
    bd = torch.as_tensor(b, device="cuda")
    x = torch.empty_like(bd)
    N.hodlr_solve(M, bd, x, N.DAFMM_FP64)
    assert _rel(x.cpu().numpy(), ref) < 1e-10
    N.hodlr_solve(M, bd, x, N.DAFMM_MIXED)
    assert _rel(x.cpu().numpy(), ref) < 1e-4
    # in place
    y = bd.clone()
    N.hodlr_solve(M, y, y, N.DAFMM_FP64)
    assert _rel(y.cpu().numpy(), ref) < 1e-10
    # the low-rank approximation is close to A
    assert np.linalg.norm(At - A) / np.linalg.norm(A) < 0.05
    N.hodlr_destroy(M)


@pytest.mark.parametrize("leaf,ctas", [(32, 1), (32, 4), (32, 32), (64, 2), (64, 16), (256, 4), (512, 1), (512, 2)])
def test_hodlr_apply_every_launch_width(N, grid32, leaf, ctas):
    """One CTA may own several nodes of a level, exactly one, or part of one
    (then the last CTA to finish the node forms s); leaves larger than the
    CTA's thread count take several rows per thread.  Every width gives the
    Woodbury inverse of the exported A~."""
    w, op, A, f = grid32
    M = N.hodlr_factor(op.ops, rank=12, leaf_size=leaf)
    try:
        At = N.hodlr_export(M, w.N)
        b = W.random_vector(w.N, 1, seed=6)[:, 0]
        ref = O.lu_solve(At, b)
        bd = torch.as_tensor(b, device="cuda")
        N.hodlr_set_ctas(M, ctas)
        x = torch.empty_like(bd)
        N.hodlr_solve(M, bd, x, N.DAFMM_FP64)
        N.hodlr_sync(M)
        assert _rel(x.cpu().numpy(), ref) < 1e-10
        N.hodlr_solve(M, bd, x, N.DAFMM_MIXED)
        N.hodlr_sync(M)
        assert _rel(x.cpu().numpy(), ref) < 1e-4
        N.hodlr_set_ctas(M, 0)
    finally:
        N.hodlr_destroy(M)


def test_hodlr_width_argument_errors(N, grid32):
    w, op, A, f = grid32
    M = N.hodlr_factor(op.ops, rank=5, leaf_size=64)
    try:
        for bad in (3, -2, 2 * w.N // 64):
            with pytest.raises(N.DafmmError):
                N.hodlr_set_ctas(M, bad)
    finally:
        N.hodlr_destroy(M)


def test_hodlr_barrier_timeout_is_reported_and_the_handle_recovers(N, grid32):
    """A launch told to wait for one CTA more than it has gives up its first
    grid barrier after about 0.2 s; hodlr_sync reports DAFMM_ETIMEOUT and the
    next application is correct again."""
    w, op, A, f = grid32
    M = N.hodlr_factor(op.ops, rank=5, leaf_size=64)
    try:
        At = N.hodlr_export(M, w.N)
        b = W.random_vector(w.N, 1, seed=7)[:, 0]
        ref = O.lu_solve(At, b)
        bd = torch.as_tensor(b, device="cuda")
        x = torch.empty_like(bd)
        N.hodlr_debug_stall(M)
        N.hodlr_solve(M, bd, x, N.DAFMM_MIXED)
        with pytest.raises(N.DafmmError) as e:
            N.hodlr_sync(M)
        assert e.value.code == N.DAFMM_ETIMEOUT
        N.hodlr_solve(M, bd, x, N.DAFMM_FP64)
        N.hodlr_sync(M)
        assert _rel(x.cpu().numpy(), ref) < 1e-10
    finally:
        N.hodlr_destroy(M)


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_hodlr_direct_solver(N, grid32, tol):
    """HODLR as a direct solver (the paper's third solver): ACA to a tolerance,
    the Woodbury inverse applied once, no GMRES.  The residual against the
    oracle's dense A follows the compression tolerance."""
    w, op, A, f = grid32
    M = N.hodlr_factor(op.ops, rank=0, tol=tol, leaf_size=64)
    try:
        fd = torch.as_tensor(f, device="cuda")
        x = torch.empty_like(fd)
        N.hodlr_solve(M, fd, x, N.DAFMM_FP64)
        N.hodlr_sync(M)
        xh = x.cpu().numpy()
        res = np.linalg.norm(A @ xh - f) / np.linalg.norm(f)
        assert res < 100 * tol, res
        assert _rel(xh, O.lu_solve(A, f)) < 1e3 * tol
    finally:
        N.hodlr_destroy(M)


def _solve(N, op, f, **kw):
    x = torch.zeros(op.N, dtype=torch.complex128, device="cuda")
    rc, st, hist = N.gmres_solve(op.ops, torch.as_tensor(f, device="cuda"), x, **kw)
    return rc, st, x.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gmres_grid32_matches_dense_lu(N, grid32, precision):
    w, op, A, f = grid32
    prec = N.DAFMM_FP64 if precision == "fp64" else N.DAFMM_MIXED
    rc, st, x = _solve(N, op, f, tol=1e-10, precision=prec, restart=50, max_iters=500)
    assert rc == N.DAFMM_OK and st.converged == 1 and st.rel_residual <= 1e-10
    assert np.linalg.norm(A @ x - f) / np.linalg.norm(f) < 1e-10 + 1e-10
    psi = O.lu_solve(A, f)
    assert _rel(x, psi) < 1e-7
    if precision == "mixed":
        assert st.outer_iterations >= 1


def test_gmres_hodlr_preconditioned_needs_fewer_iterations(N, grid32):
    w, op, A, f = grid32
    M = N.hodlr_factor(op.ops, rank=15, leaf_size=64)
    rc0, st0, x0 = _solve(N, op, f, tol=1e-10)
    rc1, st1, x1 = _solve(N, op, f, tol=1e-10, M=M)
    assert rc0 == N.DAFMM_OK and rc1 == N.DAFMM_OK
    assert st1.precond_applies > 0
    assert st1.iterations < st0.iterations
    assert np.linalg.norm(A @ x1 - f) / np.linalg.norm(f) < 2e-10
    N.hodlr_destroy(M)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gmres_left_preconditioning_matches_dense_lu(N, grid32, precision):
    """The paper's side (M^{-1} A x = M^{-1} f, Eq. hybrid): the same FP64
    true-residual stopping rule, the same solution as the dense LU solve, and
    HODLR still cuts the iteration count."""
    w, op, A, f = grid32
    prec = N.DAFMM_FP64 if precision == "fp64" else N.DAFMM_MIXED
    M = N.hodlr_factor(op.ops, rank=15, leaf_size=64)
    try:
        rc, st, x = _solve(N, op, f, tol=1e-10, precision=prec, M=M, side=N.DAFMM_PREC_LEFT, max_iters=500)
        assert rc == N.DAFMM_OK and st.converged == 1 and st.rel_residual <= 1e-10
        assert np.linalg.norm(A @ x - f) / np.linalg.norm(f) < 1e-10 + 1e-10
        assert _rel(x, O.lu_solve(A, f)) < 1e-7
        rc0, st0, _ = _solve(N, op, f, tol=1e-10, precision=prec, max_iters=500)
        assert st.iterations < st0.iterations
        assert st.precond_applies >= st.iterations
    finally:
        N.hodlr_destroy(M)


def test_gmres_side_argument_checked(N, grid32):
    w, op, A, f = grid32
    with pytest.raises(N.DafmmError):
        _solve(N, op, f, tol=1e-8, side=2)


def test_gmres_reports_not_converged(N, grid32):
    w, op, A, f = grid32
    rc, st, x = _solve(N, op, f, tol=1e-12, max_iters=3, restart=3)
    assert rc == N.DAFMM_ENOTCONV and st.converged == 0 and st.iterations == 3
    assert 0 < st.rel_residual < 1.0


def test_gmres_grid128_mixed_and_fp64(N):
    """The 128 x 128, kappa = 40 workload to 1e-8: FP64 and mixed + refinement."""
    from paper_2204_00326_gb300.operator import DafmmOperator

    w = W.GRID128_K40
    op = DafmmOperator(w.n_side, w.kappa, lambda xy: W.contrast(w, xy))
    f = -w.kappa ** 2 * op.q * W.plane_waves(w.kappa, op.xy)[:, 0]
    sols = {}
    for name, prec in (("fp64", N.DAFMM_FP64), ("mixed", N.DAFMM_MIXED)):
        rc, st, x = _solve(N, op, f, tol=1e-8, precision=prec, restart=50, max_iters=2000)
        assert rc == N.DAFMM_OK and st.rel_residual <= 1e-8
        sols[name] = x
    # the two agree to the tolerance, and sampled rows of the oracle's residual are small
    assert _rel(sols["mixed"], sols["fp64"]) < 1e-6
    rows = np.sort(np.random.default_rng(3).choice(w.N, 48, replace=False))
    r = O.matvec_rows(w.n_side, w.kappa, op.q, sols["fp64"], rows) - f[rows]
    assert np.linalg.norm(r) / np.linalg.norm(f[rows]) < 1e-7
    op.close()
