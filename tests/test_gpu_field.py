"""Fields at arbitrary points (Section 6.1): the interpolant psi(x) of Eq. 7 and
its volume potential u(x) = V[psi](x), by dafmm_field_eval, against the
oracle; and the error function E(x) of a solution.

Tolerances: u(x) from the library's near/far quadrature against the oracle's
adaptive one at 1e-10 relative (both resolve the integrals to ~1e-13; the
points include targets 1e-6 from a leaf edge, on edges and at nodes);
psi(x) is the same finite sum on both sides, 1e-12.  E(x) is the paper's
"true" error: solver error plus discretisation error, the latter O(h^p), so
it falls by about 2^p between the 32^2 and 64^2 grids of one problem.
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


def _op(n, kappa, contrast):
    from paper_2204_00326_gb300.operator import DafmmOperator

    return DafmmOperator(n, kappa, contrast)


def _points(n, rng, k=24):
    """Random interior points, points 1e-6 off a leaf edge, on a leaf edge, at
    a corner of the domain, at grid nodes, and outside the domain."""
    h = 2.0 / (n // 4)  # leaf width
    pts = list(rng.uniform(-1, 1, size=(k, 2)))
    e = -1.0 + 3 * h
    pts += [[e + 1e-6, 0.1], [e - 1e-6, -0.3], [e, 0.37], [0.2, e], [-1.0, -1.0], [1.0, 0.5]]
    xy = O.grid_nodes(n)
    pts += list(xy[[0, n * n // 2 + 7]])
    pts += [[1.3, 0.2], [-0.4, -1.5], [2.5, 2.5]]
    return np.array(pts)


@pytest.mark.parametrize("n,kappa", [(32, 8.0), (64, 20.0)])
def test_fields_match_the_oracle(N, n, kappa):
    w = W.GRID32_K8
    op = _op(n, kappa, lambda xy: W.contrast(w, xy))
    try:
        rng = np.random.default_rng(n)
        psi = W.random_vector(op.N, 1, seed=70)[:, 0]
        pts = _points(n, rng)
        u, pa = N.dafmm_field_eval(op.ops, torch.as_tensor(psi, device="cuda"), torch.as_tensor(pts, device="cuda"))
        ur, par = O.field_eval(n, kappa, psi, pts)
        u, pa = u.cpu().numpy(), pa.cpu().numpy()
        assert np.linalg.norm(u - ur) / np.linalg.norm(ur) < 1e-10
        assert np.abs(u - ur).max() < 1e-10 * np.abs(ur).max()
        assert np.abs(pa - par).max() < 1e-12 * np.abs(par).max()
        assert np.all(pa[-3:] == 0)
    finally:
        op.close()


def _error_function(N, n, kappa, w):
    """Solve the configuration's problem on an n x n grid (FP64 GMRES to
    1e-12), then E(x) = |psi(x) + kappa^2 q(x) u(x) - f(x)| / kappa^2 at
    fixed points, f = -kappa^2 q u_inc evaluated exactly (not from the grid)."""
    op = _op(n, kappa, lambda xy: W.contrast(w, xy))
    try:
        f = -kappa ** 2 * op.q * W.plane_waves(kappa, op.xy)[:, 0]
        x = torch.zeros(op.N, dtype=torch.complex128, device="cuda")
        rc, st, _ = N.gmres_solve(op.ops, torch.as_tensor(f, device="cuda"), x, tol=1e-12, max_iters=2000)
        assert rc == N.DAFMM_OK
        pts = np.random.default_rng(71).uniform(-0.8, 0.8, size=(32, 2))
        u, pa = N.dafmm_field_eval(op.ops, x, torch.as_tensor(pts, device="cuda"))
        u, pa = u.cpu().numpy(), pa.cpu().numpy()
        q = W.contrast(w, pts)
        fx = -kappa ** 2 * q * W.plane_waves(kappa, pts)[:, 0]
        E = np.abs(pa + kappa ** 2 * q * u - fx) / kappa ** 2
        return E, np.abs(fx).max() / kappa ** 2, x.cpu().numpy(), pts, u
    finally:
        op.close()


def test_error_function_falls_with_the_grid(N):
    """Config 1's problem (kappa = 8, truncated Gaussian contrast) solved on
    32^2 and 64^2 grids: E(x) is small against |f| / kappa^2 and falls at
    about the order p = 4 of the discretisation."""
    w = W.GRID32_K8
    E32, fs, psi32, pts, u32 = _error_function(N, 32, w.kappa, w)
    E64, _, _, _, _ = _error_function(N, 64, w.kappa, w)
    r32, r64 = np.sqrt(np.mean(E32 ** 2)), np.sqrt(np.mean(E64 ** 2))
    print(f"E(x) rms: 32^2 {r32:.3e}, 64^2 {r64:.3e}, |f|/kappa^2 {fs:.3e}")
    assert r32 < 1e-2 * fs
    assert r32 / r64 > 8.0
    # the library's u at these points against the oracle's
    ur, _ = O.field_eval(32, w.kappa, psi32, pts[:6])
    assert np.linalg.norm(u32[:6] - ur) / np.linalg.norm(ur) < 1e-10


def test_fields_grid128_sampled_points(N):
    """The 128^2, kappa = 40 workload: 12 points against the oracle."""
    w = W.GRID128_K40
    op = _op(w.n_side, w.kappa, lambda xy: W.contrast(w, xy))
    try:
        psi = W.random_vector(op.N, 1, seed=72)[:, 0]
        pts = _points(w.n_side, np.random.default_rng(73), k=6)
        u, pa = N.dafmm_field_eval(op.ops, torch.as_tensor(psi, device="cuda"), torch.as_tensor(pts, device="cuda"))
        ur, par = O.field_eval(w.n_side, w.kappa, psi, pts)
        assert np.linalg.norm(u.cpu().numpy() - ur) / np.linalg.norm(ur) < 1e-10
        assert np.abs(pa.cpu().numpy() - par).max() < 1e-12 * np.abs(par).max()
    finally:
        op.close()


def test_field_eval_argument_errors(N):
    w = W.GRID32_K8
    op = _op(32, w.kappa, lambda xy: W.contrast(w, xy))
    try:
        assert N.lib.dafmm_field_eval(op.ops, None, 1, None, None, None, None) == N.DAFMM_EBADARG
        psi = torch.zeros(op.N, dtype=torch.complex128, device="cuda")
        u, pa = N.dafmm_field_eval(op.ops, psi, torch.zeros(0, 2, dtype=torch.float64, device="cuda"))
        assert u.numel() == 0
    finally:
        op.close()
