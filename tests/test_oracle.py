"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test ties one oracle function to something other than itself: a library
routine (numpy, scipy), a textbook table, a closed form, an invariant of the
discretisation, or the exact solution of a manufactured problem.  A plausible
slip anywhere in the oracle -- a dropped beta^2, a sign of G, a transposed
Q^+, a wrong node order, a mis-scaled quadrature -- fails at least one of them.
"""
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O
from paper_2204_00326_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gauss_legendre_matches_numpy():
    for m in (1, 2, 7, 16, 20, 24):
        x, w = O.gauss_legendre(m)
        xr, wr = np.polynomial.legendre.leggauss(m)
        idx = np.argsort(x)
        assert np.allclose(x[idx], xr, rtol=0, atol=1e-15)
        assert np.allclose(w[idx], wr, rtol=0, atol=2e-15)


def test_cheb_nodes_are_roots_of_T_p_ascending():
    for p in (2, 4, 6, 8):
        z = O.cheb_nodes(p)
        assert np.all(np.diff(z) > 0)
        for zk in z:
            assert abs(O.cheb_T(p, zk)) < 1e-14
            assert abs(O.cheb_T(p, zk) - np.cos(p * np.arccos(zk))) < 1e-13


def test_basis_count_and_degrees():
    for p in (1, 3, 4, 6):
        a, b = O.basis_degrees(p)
        assert len(a) == p * (p + 1) // 2
        assert np.all(a + b < p)
        assert len(set(zip(a.tolist(), b.tolist()))) == len(a)


@pytest.mark.parametrize("p", [2, 4, 6])
def test_qpinv_is_pseudo_inverse(p):
    Q = O.qmatrix(p)
    Qp = O.qpinv(p)
    # library routine
    assert np.abs(Qp - np.linalg.pinv(Q)).max() < 1e-13
    # left inverse of a full-column-rank matrix
    assert np.abs(Qp @ Q - np.eye(Q.shape[1])).max() < 1e-13
    # closed form from the discrete orthogonality of T_a at first-kind nodes
    a, b = O.basis_degrees(p)
    z = O.cheb_nodes(p)
    c = lambda k: p if k == 0 else p / 2.0
    T = lambda n, x: np.cos(n * np.arccos(x))
    closed = np.zeros_like(Qp)
    for l in range(len(a)):
        for k2 in range(p):
            for k1 in range(p):
                closed[l, k1 + p * k2] = T(a[l], z[k1]) * T(b[l], z[k2]) / (c(a[l]) * c(b[l]))
    assert np.abs(Qp - closed).max() < 1e-14


def test_hankel_matches_scipy_and_textbook_table():
    for z in (1e-6, 1e-3, 0.1, 0.5, 0.8935769662791675, 1.0, 2.4048255576957727, 3.9576784193148579, 10.0, 50.0, 321.7):
        assert abs(O.hankel0(z) - special.hankel1(0, z)) < 1e-14 * max(1.0, abs(special.hankel1(0, z)))
    rows = np.loadtxt(os.path.join(GOLDEN, "bessel_abramowitz_stegun_table9_1.txt"))
    for x, j, y in rows:
        h = O.hankel0(x)
        assert abs(h.real - j) < 6e-11 and abs(h.imag - y) < 6e-11


def _dblquad_basis(p, kb, t, l):
    """Reference integral by scipy's adaptive QUADPACK, split at the target."""
    a, b = O.basis_degrees(p)
    T = lambda n, x: np.cos(n * np.arccos(np.clip(x, -1.0, 1.0)))

    def f(y2, y1, part):
        r = np.hypot(y1 - t[0], y2 - t[1])
        g = 0.25j * special.hankel1(0, kb * r) * T(a[l], y1) * T(b[l], y2)
        return g.real if part == 0 else g.imag

    xs = sorted({-1.0, 1.0} | ({t[0]} if -1 < t[0] < 1 else set()))
    ys = sorted({-1.0, 1.0} | ({t[1]} if -1 < t[1] < 1 else set()))
    out = 0j
    for part in (0, 1):
        s = 0.0
        for i in range(len(xs) - 1):
            for j in range(len(ys) - 1):
                s += integrate.dblquad(lambda y2, y1: f(y2, y1, part), xs[i], xs[i + 1], ys[j], ys[j + 1],
                                       epsabs=1e-14, epsrel=1e-13)[0]
        out += s if part == 0 else 1j * s
    return out


@pytest.mark.parametrize("case", ["self", "edge", "corner", "far"])
def test_basis_integrals_match_adaptive_quadpack(case):
    p, kb = 4, 1.25
    z = O.cheb_nodes(p)
    t = {"self": (z[0], z[1]), "edge": (2 + z[0], z[3]), "corner": (2 + z[0], 2 + z[0]),
         "far": (4 + z[2], z[1])}[case]
    I = O.basis_integrals(p, kb, t)
    for l in (0, 2, 4, 9):
        ref = _dblquad_basis(p, kb, t, l)
        assert abs(I[l] - ref) < 5e-14, (case, l, abs(I[l] - ref))


def test_basis_integrals_converged_in_rule_parameters():
    p = 4
    z = O.cheb_nodes(p)
    for kb in (0.3, 1.25, 2.5):
        for t in ((z[1], z[2]), (2 + z[0], z[3]), (-2 - z[0], 2 + z[1]), (6 + z[3], -4 + z[0])):
            a = O.basis_integrals(p, kb, t, m=20, dmin=2e-6)
            b = O.basis_integrals(p, kb, t, m=28, dmin=1e-8)
            assert np.abs(a - b).max() < 1e-12 * max(1.0, np.abs(b).max())


def _manufactured(kappa, R=0.8, k=10):
    """phi compactly supported in |x|<R and psi = -(Laplacian + kappa^2) phi,
    so that V[psi] = phi exactly (G is the radiating fundamental solution)."""
    def phi(xy):
        r2 = (xy ** 2).sum(1)
        s = np.clip(1 - r2 / R ** 2, 0, None)
        return s ** k

    def psi(xy):
        r2 = (xy ** 2).sum(1)
        s = np.clip(1 - r2 / R ** 2, 0, None)
        lap = 4 * k * (k - 1) * s ** (k - 2) * r2 / R ** 4 - 4 * k * s ** (k - 1) / R ** 2
        lap = np.where(r2 < R * R, lap, 0.0)
        return -(lap + kappa ** 2 * s ** k)

    return phi, psi


def test_manufactured_solution_converges_at_order_p():
    """K psi -> phi with the local least-squares error O(h^p), p = 4 (Eq. 11-13)."""
    kappa = 8.0
    phi, psi = _manufactured(kappa)
    rng = np.random.default_rng(0)
    errs = []
    for n in (32, 64):
        xy = O.grid_nodes(n)
        rows = rng.choice(n * n, size=40, replace=False)
        u = O.K_rows(n, kappa, rows) @ psi(xy)
        errs.append(np.linalg.norm(u - phi(xy[rows])) / np.linalg.norm(phi(xy[rows])))
    assert errs[1] < 2e-4
    assert errs[0] / errs[1] > 12.0  # order close to 4


def test_known_solution_residual_small():
    """With f := psi + kappa^2 q phi, the exact psi nearly solves A psi = f (Eq. 12a)."""
    kappa, n = 8.0, 64
    phi, psi = _manufactured(kappa)
    xy = O.grid_nodes(n)
    q = W.contrast(W.GRID32_K8, xy)
    f = psi(xy) + kappa ** 2 * q * phi(xy)
    rows = np.random.default_rng(1).choice(n * n, size=32, replace=False)
    Apsi = O.matvec_rows(n, kappa, q, psi(xy).astype(complex), rows)
    assert np.linalg.norm(Apsi - f[rows]) / np.linalg.norm(f[rows]) < 1e-4


def test_polynomial_density_reproduced_exactly():
    """A global polynomial of degree < p is fitted exactly on every leaf, so
    (K psi)_i equals the integral of G(x_i, .) psi over the whole domain."""
    n, kappa = 8, 3.0
    xy = O.grid_nodes(n)
    psi = xy[:, 0] + 0.5 * xy[:, 1] ** 2 - 0.25 * xy[:, 0] * xy[:, 1]
    i = 37
    Krow = O.K_rows(n, kappa, [i])[0]
    xi = xy[i]
    dens = lambda y1, y2: y1 + 0.5 * y2 ** 2 - 0.25 * y1 * y2

    def f(y2, y1, part):
        g = 0.25j * special.hankel1(0, kappa * np.hypot(y1 - xi[0], y2 - xi[1])) * dens(y1, y2)
        return g.real if part == 0 else g.imag

    ref = 0j
    for part in (0, 1):
        s = 0.0
        for (a0, a1) in ((-1, xi[0]), (xi[0], 1)):
            for (b0, b1) in ((-1, xi[1]), (xi[1], 1)):
                s += integrate.dblquad(lambda y2, y1: f(y2, y1, part), a0, a1, b0, b1, epsabs=1e-13, epsrel=1e-12)[0]
        ref += s if part == 0 else 1j * s
    assert abs(Krow @ psi - ref) < 1e-11 * abs(ref)


def test_K_invariant_under_grid_symmetries():
    """Reflections of the square map nodes onto nodes and leave G invariant,
    so K[s(i), s(j)] = K[i, j] for each symmetry s."""
    n, kappa = 8, 5.0
    K = O.K_dense(n, kappa)
    xy = O.grid_nodes(n)
    key = {tuple(np.round(v, 12)): i for i, v in enumerate(xy)}
    for T in (lambda v: (-v[0], v[1]), lambda v: (v[0], -v[1]), lambda v: (v[1], v[0])):
        s = np.array([key[tuple(np.round(T(v), 12))] for v in xy])
        assert np.abs(K[np.ix_(s, s)] - K).max() < 1e-13 * np.abs(K).max()
    # K is not symmetric (cardinal functions versus point values), and that is expected
    assert np.abs(K - K.T).max() > 1e-6


def test_K_rows_consistent_with_matvec_rows():
    n, kappa = 8, 5.0
    xy = O.grid_nodes(n)
    q = W.contrast(W.GRID32_K8, xy)
    v = W.random_vector(n * n, 2, seed=3)
    K = O.K_dense(n, kappa)
    A = O.dense_A(K, q, kappa)
    rows = np.arange(0, n * n, 5)
    got = O.matvec_rows(n, kappa, q, v, rows)
    assert np.abs(got - (A @ v)[rows]).max() < 1e-12 * np.abs(A @ v).max()


def test_lu_solve_matches_numpy():
    rng = np.random.default_rng(5)
    for n in (1, 7, 64):
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
        b = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
        x = O.lu_solve(A, b)
        assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-12


def test_solution_satisfies_lippmann_schwinger_identity():
    """At the discrete solution psi = -kappa^2 q (u_inc + K psi) (Eq. 6, 12a)."""
    w = W.GRID32_K8
    n = 16
    xy = O.grid_nodes(n)
    q = W.contrast(w, xy)
    uinc = W.plane_waves(w.kappa, xy)[:, 0]
    f = -w.kappa ** 2 * q * uinc
    K = O.K_dense(n, w.kappa)
    A = O.dense_A(K, q, w.kappa)
    psi = O.lu_solve(A, f)
    assert np.linalg.norm(A @ psi - f) / np.linalg.norm(f) < 1e-13
    rhs = -w.kappa ** 2 * q * (uinc + K @ psi)
    assert np.linalg.norm(psi - rhs) < 1e-12 * np.linalg.norm(psi)


def test_nbody_rows_match_scipy_direct_sum():
    """Experiment 1's potential u_i = sum_{j != i} (i/4) H0(kappa |p_i - p_j|) v_j
    against a direct numpy sum with scipy's Hankel function, several
    right-hand sides, on a 8 x 8 grid."""
    from scipy.special import hankel1

    n, kappa = 8, 5.0
    xy = O.grid_nodes(n)
    rng = np.random.default_rng(3)
    v = rng.standard_normal((n * n, 3)) + 1j * rng.standard_normal((n * n, 3))
    d = np.hypot(xy[:, None, 0] - xy[None, :, 0], xy[:, None, 1] - xy[None, :, 1])
    np.fill_diagonal(d, 1.0)
    G = 0.25j * hankel1(0, kappa * d)
    np.fill_diagonal(G, 0.0)
    rows = np.array([0, 5, 17, 63])
    got = O.nbody_rows(n, kappa, v, rows)
    ref = (G @ v)[rows]
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_nbody_matrix_is_symmetric_with_zero_diagonal():
    """G(p_a, p_b) = G(p_b, p_a) bitwise, and the j = i term is left out."""
    n, kappa = 8, 7.0
    N = n * n
    for a, b in ((3, 40), (0, 63), (12, 13)):
        ea = np.zeros(N, complex)
        eb = np.zeros(N, complex)
        ea[a] = 1.0
        eb[b] = 1.0
        assert O.nbody_rows(n, kappa, eb, [a])[0] == O.nbody_rows(n, kappa, ea, [b])[0]
        assert O.nbody_rows(n, kappa, ea, [a])[0] == 0.0


def test_field_eval_at_the_nodes_equals_rows_of_K():
    """At a grid node the off-grid field is the row of K applied to psi."""
    n, kappa = 16, 8.0
    xy = O.grid_nodes(n)
    rng = np.random.default_rng(5)
    psi = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
    rows = np.array([0, 37, 200, 255])
    u, _ = O.field_eval(n, kappa, psi, xy[rows])
    ref = O.K_rows(n, kappa, rows) @ psi
    assert np.abs(u - ref).max() < 1e-13 * np.abs(ref).max()


def test_field_eval_interpolant_reproduces_polynomials():
    """Eq. 7's interpolant is exact for a global polynomial of total degree
    < p, at any point of the domain, and zero outside it."""
    n = 16
    xy = O.grid_nodes(n)

    def g(p):
        x, y = p[:, 0], p[:, 1]
        return 1.0 + 2.0 * x - 0.5 * y + x * y - 1.5 * y ** 2 + 0.7 * x ** 3 - 0.2 * x * y ** 2

    pts = np.random.default_rng(6).uniform(-1, 1, size=(50, 2))
    _, pa = O.field_eval(n, 3.0, g(xy).astype(complex), np.vstack([pts, [[1.5, 0.0], [0.0, -1.2]]]))
    assert np.abs(pa[:50] - g(pts)).max() < 1e-12
    assert pa[50] == 0 and pa[51] == 0


def test_field_eval_manufactured_solution_off_the_grid():
    """psi = -(Laplacian + kappa^2) phi gives V[psi] = phi exactly; at points
    off the grid the error of the discretised potential falls at order ~p."""
    kappa = 8.0
    phi, psi = _manufactured(kappa)
    pts = np.random.default_rng(7).uniform(-0.9, 0.9, size=(12, 2))
    errs = []
    for n in (16, 32):
        u, _ = O.field_eval(n, kappa, psi(O.grid_nodes(n)).astype(complex), pts)
        errs.append(np.linalg.norm(u - phi(pts)) / np.linalg.norm(phi(pts)))
    assert errs[1] < 5e-3
    assert errs[0] / errs[1] > 8.0
