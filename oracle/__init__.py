"""FP64 CPU oracle for the discretised Lippmann-Schwinger operator (arXiv 2204.00326).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library; the two meet only through seeded inputs and through the
index conventions (Morton leaf order, ``i' = k1 + p*k2``, ascending first-kind
Chebyshev nodes).

The arithmetic lives in ``oracle.c`` (plain C, double precision).  This module
compiles it with gcc on first use and wraps it with ctypes.  Every function
cites the passage of the paper it follows:

* ``cheb_nodes``, ``qmatrix``, ``qpinv`` -- Section 2.2, Eq. 7-10;
* ``basis_integrals`` -- Section 2.3 (integrals of G times the basis);
* ``K_rows`` / ``K_dense`` -- Eq. 13 without the ``kappa^2 q`` factor;
* ``matvec_rows`` -- ``(A v)_i`` of Eq. 12a-13 with entries made on the fly;
* ``dense_A`` -- ``A = I + kappa^2 diag(q) K`` (Eq. 13);
* ``lu_solve`` -- dense Gaussian elimination for ``A psi = f`` (Eq. 12a).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
        P = ctypes.c_void_p
        lib.or_gauss_legendre.argtypes = [i, P, P]
        lib.or_cheb_T.argtypes = [i, d]
        lib.or_cheb_T.restype = d
        lib.or_cheb_nodes.argtypes = [i, P]
        lib.or_basis_count.argtypes = [i]
        lib.or_basis_degrees.argtypes = [i, P, P]
        lib.or_qmatrix.argtypes = [i, P]
        lib.or_qpinv.argtypes = [i, P]
        lib.or_hankel0.argtypes = [d, P, P]
        lib.or_basis_integrals.argtypes = [i, d, d, d, i, d, P]
        lib.or_grid_nodes.argtypes = [i, d, d, i, P]
        lib.or_K_rows.argtypes = [i, d, d, i, d, l, P, P]
        lib.or_matvec_rows.argtypes = [i, d, d, i, d, P, i, P, l, P, P]
        lib.or_nbody_rows.argtypes = [i, d, d, i, d, i, P, l, P, P]
        lib.or_field_eval.argtypes = [i, d, d, i, d, P, l, P, P, P]
        lib.or_lu_solve.argtypes = [l, P, i, P]
        lib.or_num_threads.argtypes = []
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(st: int, what: str):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def num_threads() -> int:
    """Threads the oracle's OpenMP loops use."""
    return int(_load().or_num_threads())


def gauss_legendre(m: int):
    """m-point Gauss-Legendre nodes and weights on [-1, 1]."""
    x = np.zeros(m)
    w = np.zeros(m)
    _check(_load().or_gauss_legendre(m, _ptr(x), _ptr(w)), "gauss_legendre")
    return x, w


def cheb_T(n: int, x: float) -> float:
    return float(_load().or_cheb_T(n, x))


def cheb_nodes(p: int) -> np.ndarray:
    """First-kind Chebyshev nodes, ascending (Section 2, p x p leaf grid)."""
    z = np.zeros(p)
    _load().or_cheb_nodes(p, _ptr(z))
    return z


def basis_degrees(p: int):
    """(a, b) degree pairs of b_l = T_a(x) T_b(y), a + b < p (Section 2.2)."""
    n = _load().or_basis_count(p)
    a = np.zeros(n, dtype=np.int32)
    b = np.zeros(n, dtype=np.int32)
    _load().or_basis_degrees(p, _ptr(a), _ptr(b))
    return a, b


def qmatrix(p: int) -> np.ndarray:
    """Interpolation matrix Q (p^2 x N_p), Eq. 9b."""
    n = _load().or_basis_count(p)
    Q = np.zeros((p * p, n))
    _check(_load().or_qmatrix(p, _ptr(Q)), "qmatrix")
    return Q


def qpinv(p: int) -> np.ndarray:
    """Q^+ = (Q^T Q)^{-1} Q^T (N_p x p^2), Eq. 10."""
    n = _load().or_basis_count(p)
    Qp = np.zeros((n, p * p))
    _check(_load().or_qpinv(p, _ptr(Qp)), "qpinv")
    return Qp


def hankel0(z: float) -> complex:
    """H0^(1)(z) = J0(z) + i Y0(z) (Eq. 6's Green's function uses it)."""
    re = np.zeros(1)
    im = np.zeros(1)
    _load().or_hankel0(float(z), _ptr(re), _ptr(im))
    return complex(re[0], im[0])


def basis_integrals(p: int, kb: float, t, m: int = 20, dmin: float = 2e-6) -> np.ndarray:
    """I_l = int_{[-1,1]^2} (i/4) H0(kb |t - eta|) b_l(eta) d eta (Section 2.3)."""
    n = _load().or_basis_count(p)
    out = np.zeros(2 * n)
    st = _load().or_basis_integrals(p, float(kb), float(t[0]), float(t[1]), m, dmin, _ptr(out))
    _check(st, "basis_integrals")
    return out[0::2] + 1j * out[1::2]


def grid_nodes(n_side: int, x0: float = -1.0, x1: float = 1.0, p: int = 4) -> np.ndarray:
    """Coordinates (N x 2) of the unknowns: Morton leaves, i' = k1 + p*k2."""
    xy = np.zeros((n_side * n_side, 2))
    _check(_load().or_grid_nodes(n_side, x0, x1, p, _ptr(xy)), "grid_nodes")
    return xy


def K_rows(n_side: int, kappa: float, rows, x0: float = -1.0, x1: float = 1.0, p: int = 4) -> np.ndarray:
    """Rows of K_ij = int_{B(j)} G(x_i, y) L_{j'}(y) dy (Eq. 13 without kappa^2 q)."""
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    N = n_side * n_side
    out = np.zeros((len(rows), N, 2))
    st = _load().or_K_rows(n_side, x0, x1, p, float(kappa), len(rows), _ptr(rows), _ptr(out))
    _check(st, "K_rows")
    return out[..., 0] + 1j * out[..., 1]


def K_dense(n_side: int, kappa: float, x0: float = -1.0, x1: float = 1.0, p: int = 4) -> np.ndarray:
    """The full N x N matrix K of Eq. 13 (without the kappa^2 q factor)."""
    return K_rows(n_side, kappa, np.arange(n_side * n_side), x0, x1, p)


def dense_A(K: np.ndarray, q: np.ndarray, kappa: float) -> np.ndarray:
    """A = I + kappa^2 diag(q) K (Eq. 13)."""
    A = (kappa * kappa) * (np.asarray(q, dtype=np.float64)[:, None] * K)
    A[np.diag_indices_from(A)] += 1.0
    return A


def matvec_rows(n_side: int, kappa: float, q, v, rows, x0: float = -1.0, x1: float = 1.0, p: int = 4) -> np.ndarray:
    """(A v)_i for the listed rows, entries generated on the fly (Eq. 12a-13).

    ``v`` is (N,) or (N, nrhs) complex; returns (len(rows),) or (len(rows), nrhs).
    """
    v = np.asarray(v, dtype=np.complex128)
    squeeze = v.ndim == 1
    v2 = v.reshape(v.shape[0], -1)
    nrhs = v2.shape[1]
    if nrhs > 64:
        raise ValueError("oracle matvec_rows handles at most 64 right-hand sides")
    vv = np.ascontiguousarray(np.stack([v2.real, v2.imag], axis=-1))
    qq = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros((len(rows), nrhs, 2))
    st = _load().or_matvec_rows(n_side, x0, x1, p, float(kappa), _ptr(qq), nrhs, _ptr(vv), len(rows), _ptr(rows), _ptr(out))
    _check(st, "matvec_rows")
    res = out[..., 0] + 1j * out[..., 1]
    return res[:, 0] if squeeze else res


def field_eval(n_side: int, kappa: float, psi, pts, x0: float = -1.0, x1: float = 1.0, p: int = 4):
    """(u, psi_at) at the points pts (m x 2): the volume potential of the
    interpolant of the grid values psi (Eq. 5, 7) and the interpolant itself
    (zero outside the domain), the ingredients of E(x) (Section 6.1)."""
    psi = np.asarray(psi, dtype=np.complex128)
    pv = np.ascontiguousarray(np.stack([psi.real, psi.imag], axis=-1))
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float64))
    m = pts.shape[0]
    u = np.zeros((m, 2))
    pa = np.zeros((m, 2))
    _check(_load().or_field_eval(n_side, x0, x1, p, float(kappa), _ptr(pv), m, _ptr(pts), _ptr(u), _ptr(pa)), "field_eval")
    return u[:, 0] + 1j * u[:, 1], pa[:, 0] + 1j * pa[:, 1]


def nbody_rows(n_side: int, kappa: float, v, rows, x0: float = -1.0, x1: float = 1.0, p: int = 4) -> np.ndarray:
    """u_i = sum_{j != i} G(p_i, p_j) v_j at the grid nodes for the listed rows
    (Experiment 1's N-body potential, Section 6.2), by direct summation.

    ``v`` is (N,) or (N, nrhs) complex; returns (len(rows),) or (len(rows), nrhs).
    """
    v = np.asarray(v, dtype=np.complex128)
    squeeze = v.ndim == 1
    v2 = v.reshape(v.shape[0], -1)
    nrhs = v2.shape[1]
    if nrhs > 64:
        raise ValueError("oracle nbody_rows handles at most 64 right-hand sides")
    vv = np.ascontiguousarray(np.stack([v2.real, v2.imag], axis=-1))
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros((len(rows), nrhs, 2))
    _check(_load().or_nbody_rows(n_side, x0, x1, p, float(kappa), nrhs, _ptr(vv), len(rows), _ptr(rows), _ptr(out)), "nbody_rows")
    res = out[..., 0] + 1j * out[..., 1]
    return res[:, 0] if squeeze else res


def lu_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve A x = b by Gaussian elimination with partial pivoting (Eq. 12a)."""
    n = A.shape[0]
    Ac = np.ascontiguousarray(np.stack([A.real, A.imag], axis=-1))
    b = np.asarray(b, dtype=np.complex128)
    squeeze = b.ndim == 1
    b2 = b.reshape(n, -1)
    bc = np.ascontiguousarray(np.stack([b2.real, b2.imag], axis=-1))
    _check(_load().or_lu_solve(n, _ptr(Ac), b2.shape[1], _ptr(bc)), "lu_solve")
    x = bc[..., 0] + 1j * bc[..., 1]
    return x[:, 0] if squeeze else x
