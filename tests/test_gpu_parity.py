"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances: FP64 mode 1e-10 relative 2-norm against the oracle's operator A
(the DAFMM is an approximation of A to about eps_nca = 1e-12 per block, and
the two quadratures agree to ~1e-13).  The single-right-hand-side FP64
launch computes in double-float (float pairs, unit roundoff u = 2^-48 =
3.6e-15), and so does the several-right-hand-side path; with the same
|U| |V| ~ 1e2 amplification as below, the rounding (seen in the linearity
defect and between the two paths) stays under ~1e-12, checked at
DF_TOL = 1e-11.  Mixed mode (complex64 operators and
FP32 accumulation) is checked at 2e-5: complex64 rounds each stored operator
entry to 6e-8 relative, and the realised NCA factors amplify that by the
norms of the interpolation operators (|U|, |V| up to ~1e2), giving a few 1e-6
on the matvec; refinement in FP64 removes it in the solver.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2204_00326_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 2e-5
DF_TOL = 1e-11  # rounding of the double-float single-right-hand-side FP64 launch (see above)


@pytest.fixture(scope="module")
def N():
    import paper_2204_00326_gb300 as pkg

    pkg.build()
    from paper_2204_00326_gb300 import native

    return native


def _op(n_side, kappa, contrast, **kw):
    from paper_2204_00326_gb300.operator import DafmmOperator

    return DafmmOperator(n_side, kappa, contrast, **kw)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_entry_table_matches_oracle_entries(N):
    w = W.GRID32_K8
    op = _op(w.n_side, w.kappa, lambda xy: W.contrast(w, xy))
    rng = np.random.default_rng(0)
    rows = np.concatenate([np.arange(16), rng.choice(w.N, 24, replace=False)])
    Kr = O.K_rows(w.n_side, w.kappa, rows)
    got = op.entries(rows, np.arange(w.N))
    # self, adjacent and far leaves all appear in these rows
    assert np.abs(got - Kr).max() < 1e-12 * np.abs(Kr).max()
    op.close()


@pytest.mark.parametrize("n_side,kappa", [(4, 3.0), (8, 8.0), (16, 8.0), (32, 8.0)])
def test_fp64_matvec_matches_dense_oracle(N, n_side, kappa):
    w = W.GRID32_K8
    op = _op(n_side, kappa, lambda xy: W.contrast(w, xy))
    K = O.K_dense(n_side, kappa)
    A = O.dense_A(K, op.q, kappa)
    for seed in (1, 2):
        v = W.random_vector(n_side * n_side, 1, seed=seed)[:, 0]
        out = op.matvec(torch.as_tensor(v, device="cuda"), precision=N.DAFMM_FP64).cpu().numpy()
        assert _rel(out, A @ v) < FP64_TOL
    # the configuration's own right-hand side: f = -kappa^2 q u_inc
    f = -kappa ** 2 * op.q * W.plane_waves(kappa, op.xy)[:, 0]
    out = op.matvec(torch.as_tensor(f, device="cuda"), precision=N.DAFMM_FP64).cpu().numpy()
    assert _rel(out, A @ f) < FP64_TOL
    op.close()


def test_mixed_matvec_matches_dense_oracle(N):
    w = W.GRID32_K8
    op = _op(w.n_side, w.kappa, lambda xy: W.contrast(w, xy))
    A = O.dense_A(O.K_dense(w.n_side, w.kappa), op.q, w.kappa)
    v = W.random_vector(w.N, 1, seed=3)[:, 0]
    out = op.matvec(torch.as_tensor(v, device="cuda"), precision=N.DAFMM_MIXED).cpu().numpy()
    err = _rel(out, A @ v)
    assert err < MIXED_TOL
    # mixed is a different (coarser) computation, not a copy of the FP64 path
    out64 = op.matvec(torch.as_tensor(v, device="cuda"), precision=N.DAFMM_FP64).cpu().numpy()
    assert _rel(out64, A @ v) < err
    op.close()


@pytest.fixture(scope="module")
def op128(N):
    w = W.GRID128_K40
    op = _op(w.n_side, w.kappa, lambda xy: W.contrast(w, xy))
    yield op
    op.close()


def test_grid128_directional_tree_shape(op128):
    info = op128.info()
    assert info.top == 3 and info.hf[3] == 1 and info.cones[3] == 32
    st = op128.stats()
    assert st.slots[3] > 0 and st.rank_in_max[5] <= 16 and st.rank_out_max[5] <= 10


def test_fp64_matvec_grid128_sampled_rows(N, op128):
    """Full-size workload (N = 16384, directional level): sampled rows of A v."""
    w = W.GRID128_K40
    rng = np.random.default_rng(11)
    rows = np.sort(rng.choice(w.N, 96, replace=False))
    for v in (W.random_vector(w.N, 1, seed=5)[:, 0], -w.kappa ** 2 * op128.q * W.plane_waves(w.kappa, op128.xy)[:, 0]):
        out = op128.matvec(torch.as_tensor(v, device="cuda"), precision=N.DAFMM_FP64).cpu().numpy()
        ref = O.matvec_rows(w.n_side, w.kappa, op128.q, v, rows)
        assert _rel(out[rows], ref) < FP64_TOL


def test_mixed_matvec_grid128_sampled_rows(N, op128):
    w = W.GRID128_K40
    rows = np.sort(np.random.default_rng(12).choice(w.N, 64, replace=False))
    v = W.random_vector(w.N, 1, seed=6)[:, 0]
    out = op128.matvec(torch.as_tensor(v, device="cuda"), precision=N.DAFMM_MIXED).cpu().numpy()
    ref = O.matvec_rows(w.n_side, w.kappa, op128.q, v, rows)
    assert _rel(out[rows], ref) < MIXED_TOL


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("mixed", MIXED_TOL)])
def test_potential_matches_oracle_rows(N, op128, precision, tol):
    """dafmm_potential is K v (the scattered field V[psi] at the nodes): the
    oracle's A with q = 1/kappa^2 is I + K, so (A v - v) on sampled rows is the
    reference; and the operator application is v + kappa^2 q (K v)."""
    w = W.GRID128_K40
    prec = N.DAFMM_FP64 if precision == "fp64" else N.DAFMM_MIXED
    rows = np.sort(np.random.default_rng(14).choice(w.N, 48, replace=False))
    v = W.random_vector(w.N, 1, seed=15)[:, 0]
    vd = torch.as_tensor(v, device="cuda")
    kv = torch.empty_like(vd)
    N.dafmm_potential(op128.ops, vd, kv, prec)
    kvh = kv.cpu().numpy()
    ref = O.matvec_rows(w.n_side, w.kappa, np.full(w.N, 1.0 / w.kappa ** 2), v, rows) - v[rows]
    assert _rel(kvh[rows], ref) < tol
    av = op128.matvec(vd, precision=prec).cpu().numpy()
    assert _rel(av, v + w.kappa ** 2 * op128.q * kvh) < (1e-12 if precision == "fp64" else 1e-6)
    op128.sync()


def test_matvec_is_linear_and_repeatable(N, op128):
    w = W.GRID128_K40
    a = torch.as_tensor(W.random_vector(w.N, 1, seed=8)[:, 0], device="cuda")
    b = torch.as_tensor(W.random_vector(w.N, 1, seed=9)[:, 0], device="cuda")
    for prec in (N.DAFMM_FP64, N.DAFMM_MIXED):
        ya = op128.matvec(a, precision=prec)
        yb = op128.matvec(b, precision=prec)
        yab = op128.matvec(a + 2.5j * b, precision=prec)
        tol = DF_TOL if prec == N.DAFMM_FP64 else 1e-5
        assert (torch.linalg.norm(yab - (ya + 2.5j * yb)) / torch.linalg.norm(yab)).item() < tol
        assert torch.equal(op128.matvec(a, precision=prec), ya)
    op128.sync()  # no device-side wait gave up


def test_matvec_argument_errors(N, op128):
    v = torch.zeros(op128.N, dtype=torch.complex128, device="cuda")
    with pytest.raises(N.DafmmError):
        N.dafmm_matvec(op128.ops, v, v)
    with pytest.raises(N.DafmmError):
        N.dafmm_matvec(op128.ops, v, torch.empty_like(v), precision=7)
    with pytest.raises(ValueError):
        N.dafmm_matvec(op128.ops, v.to(torch.complex64), torch.empty_like(v))


def test_profile_records_passes(N, op128):
    v = torch.as_tensor(W.random_vector(op128.N, 1, seed=2)[:, 0], device="cuda")
    plain = op128.matvec(v, precision=N.DAFMM_MIXED)
    N.dafmm_profile(op128.ops, True)
    for _ in range(3):
        marked = op128.matvec(v, precision=N.DAFMM_MIXED)
    p = N.dafmm_profile_read(op128.ops)
    N.dafmm_profile(op128.ops, False)
    # the profiled calls replay a graph with event nodes at the pass marks: same kernels, same result
    assert torch.equal(marked, plain)
    assert torch.equal(op128.matvec(v, precision=N.DAFMM_MIXED), plain)
    # one right-hand side: every tree pass is one kernel, reported as the far field only
    assert p.calls == 3 and p.ms_far > 0 and p.ms_leaf > 0
    assert p.ms_up == 0 and p.ms_m2l == 0 and p.ms_down == 0
    assert abs(p.ms_total - (p.ms_far + p.ms_leaf)) < 1e-6
    # several right-hand sides: the passes are launched separately
    V = torch.as_tensor(W.random_vector(op128.N, 4, seed=3), device="cuda").contiguous()
    N.dafmm_profile(op128.ops, True)
    op128.matvec(V, precision=N.DAFMM_MIXED)
    p = N.dafmm_profile_read(op128.ops)
    N.dafmm_profile(op128.ops, False)
    assert p.calls == 1 and p.ms_m2l > 0 and p.ms_up > 0 and p.ms_down > 0
    assert abs(p.ms_far - (p.ms_up + p.ms_m2l + p.ms_down)) < 1e-6
    assert abs(p.ms_total - (p.ms_far + p.ms_leaf)) < 1e-6


def test_graph_replay_follows_new_pointers(N, op128):
    """The captured application is re-pointed when the caller's vectors change."""
    vs = [torch.as_tensor(W.random_vector(op128.N, 1, seed=40 + k)[:, 0], device="cuda") for k in range(3)]
    outs = [op128.matvec(v, precision=N.DAFMM_MIXED) for v in vs]
    again = [op128.matvec(v, precision=N.DAFMM_MIXED) for v in reversed(vs)]
    for o, a in zip(outs, reversed(again)):
        assert torch.equal(o, a)
    assert not torch.equal(outs[0], outs[1])
    op128.sync()


def test_capture_by_the_caller(N, op128):
    """Inside the caller's own stream capture the kernels join the caller's graph."""
    v = torch.as_tensor(W.random_vector(op128.N, 1, seed=50)[:, 0], device="cuda")
    ref = op128.matvec(v, precision=N.DAFMM_FP64)
    out = torch.empty_like(v)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        N.dafmm_matvec(op128.ops, v, out, N.DAFMM_FP64, s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


@pytest.mark.parametrize("nrhs", [2, 16, 37, 64])
def test_batched_matvec_matches_single(N, op128, nrhs):
    """Several right-hand sides in one application equal one-at-a-time applications."""
    w = W.GRID128_K40
    V = torch.as_tensor(W.random_vector(w.N, nrhs, seed=60 + nrhs), device="cuda").contiguous()
    # sums grouped differently in the two paths: compare at the mixed
    # tolerance, and at the double-float rounding bound in FP64
    for prec, tol in ((N.DAFMM_FP64, DF_TOL), (N.DAFMM_MIXED, MIXED_TOL)):
        Y = op128.matvec(V, precision=prec)
        for k in sorted({0, nrhs // 2, nrhs - 1}):
            yk = op128.matvec(V[:, k].contiguous(), precision=prec)
            assert (torch.linalg.norm(Y[:, k] - yk) / torch.linalg.norm(yk)).item() < tol
    op128.sync()


def test_batched_matvec_against_oracle_rows(N, op128):
    w = W.GRID128_K40
    nrhs = 8
    V = W.plane_waves(w.kappa, op128.xy, nrhs) * (-w.kappa ** 2 * op128.q)[:, None]
    Y = op128.matvec(torch.as_tensor(V, device="cuda").contiguous(), precision=N.DAFMM_FP64).cpu().numpy()
    rows = np.sort(np.random.default_rng(13).choice(w.N, 32, replace=False))
    ref = O.matvec_rows(w.n_side, w.kappa, op128.q, V, rows)
    assert _rel(Y[rows], ref) < FP64_TOL


def test_batched_rejects_too_many_rhs(N, op128):
    V = torch.zeros(op128.N, 65, dtype=torch.complex128, device="cuda")
    with pytest.raises(N.DafmmError):
        op128.matvec(V)


def test_stalled_pass_times_out_and_handle_recovers(N, op128):
    """A tree pass that never completes: the bounded waits give up, the host
    reads DAFMM_ETIMEOUT, and the next application is correct again."""
    v = torch.as_tensor(W.random_vector(op128.N, 1, seed=77)[:, 0], device="cuda")
    ref = op128.matvec(v, precision=N.DAFMM_MIXED)
    op128.sync()
    with pytest.raises(N.DafmmError):
        N.dafmm_debug_stall(op128.ops, 10 ** 6)
    N.dafmm_debug_stall(op128.ops, 0)
    out = torch.empty_like(v)
    t0 = time.perf_counter()
    N.dafmm_matvec(op128.ops, v, out, N.DAFMM_MIXED)
    with pytest.raises(N.DafmmError) as e:
        op128.sync()
    assert e.value.code == N.DAFMM_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    again = op128.matvec(v, precision=N.DAFMM_MIXED)
    op128.sync()
    assert torch.equal(again, ref)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_leaf_staging_and_global_path_agree(N, op128, precision):
    """The leaf kernel's far-field blocks staged in shared memory (the planned
    path) or read from global memory (the fallback for larger operators):
    the same products in the same order, so the same result bit for bit, and
    the oracle's rows at the usual bars."""
    prec = N.DAFMM_MIXED if precision == "mixed" else N.DAFMM_FP64
    v = torch.as_tensor(W.random_vector(op128.N, 1, seed=78)[:, 0], device="cuda")
    staged = op128.matvec(v, precision=prec)
    N.dafmm_debug_leaf_staging(op128.ops, False)
    try:
        plain = op128.matvec(v, precision=prec)
        again = op128.matvec(v, precision=prec)
    finally:
        N.dafmm_debug_leaf_staging(op128.ops, True)
    op128.sync()
    assert torch.equal(plain, staged) and torch.equal(again, staged)
    assert torch.equal(op128.matvec(v, precision=prec), staged)
    with pytest.raises(N.DafmmError):
        N._check(N.lib.dafmm_debug_leaf_staging(op128.ops, 2))
