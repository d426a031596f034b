"""The complex64 several-right-hand-side tree passes on the tensor cores
(tcgen05.mma kind::tf32, every value split into two tf32 parts), against the
CUDA-core kernel and the FP64 oracle.

Tolerances: the mixed-precision bar of test_gpu_parity.py, 2e-5 relative
2-norm against the oracle's A on sampled rows.  The three-part tf32 split
represents every FP32 operand exactly and keeps every partial product down
to 2^-33, and each chunk's short MMA chain is drained into FP32 registers
with rounded additions, so the tensor-core result differs from the
CUDA-core kernel's by FP32 rounding in a different order; the two are
compared at 1e-5 (measured 2e-6; the NCA factors amplify FP32 rounding by
~50 as in the complex64 path; a wrong operand layout or a lost term shows as
O(1)).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2204_00326_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

MIXED_TOL = 2e-5
KERNELS_TOL = 1e-5


@pytest.fixture(scope="module")
def N():
    import paper_2204_00326_gb300 as pkg

    pkg.build()
    from paper_2204_00326_gb300 import native

    return native


def _make(w, eps_nca=1e-12):
    from paper_2204_00326_gb300.operator import DafmmOperator

    return DafmmOperator(w.n_side, w.kappa, lambda xy: W.contrast(w, xy), eps_nca=eps_nca)


@pytest.fixture(scope="module")
def op128(N):
    op = _make(W.GRID128_K40)
    yield op
    op.close()


def _cols_rel(a, b):
    return (torch.linalg.norm(a - b, dim=0) / torch.linalg.norm(b, dim=0)).max().item()


def _apply(N, op, V, mode, prec=None):
    N.dafmm_set_batched_kernel(op.ops, mode)
    try:
        return op.matvec(V, precision=N.DAFMM_MIXED if prec is None else prec)
    finally:
        N.dafmm_set_batched_kernel(op.ops, N.BATCHED_AUTO)


@pytest.mark.parametrize("nrhs", [2, 3, 8, 16, 37, 64])
def test_tensor_cores_match_cuda_cores(N, op128, nrhs):
    """Odd counts take the gathered (not bulk-copied) input path."""
    V = torch.as_tensor(W.random_vector(op128.N, nrhs, seed=200 + nrhs), device="cuda").contiguous()
    y_tc = _apply(N, op128, V, N.BATCHED_TENSOR_CORES)
    y_cc = _apply(N, op128, V, N.BATCHED_CUDA_CORES)
    assert torch.isfinite(torch.view_as_real(y_tc)).all()
    d = _cols_rel(y_tc, y_cc)
    print(f"nrhs {nrhs}: tensor vs CUDA cores {d:.2e}")
    assert d < KERNELS_TOL
    # repeatable (fixed summation order)
    assert torch.equal(_apply(N, op128, V, N.BATCHED_TENSOR_CORES), y_tc)
    op128.sync()


def test_automatic_mode_uses_cuda_cores(N, op128):
    """At these chunk shapes the CUDA-core kernel is the faster one (measured
    0.74 vs 1.33 ms for 64 right-hand sides at N = 16384), so automatic mode
    picks it; the tensor-core kernel is chosen explicitly."""
    for nrhs in (4, 64):
        V = torch.as_tensor(W.random_vector(op128.N, nrhs, seed=300 + nrhs), device="cuda").contiguous()
        assert torch.equal(op128.matvec(V, precision=N.DAFMM_MIXED), _apply(N, op128, V, N.BATCHED_CUDA_CORES))


@pytest.mark.parametrize("w,eps", [(W.GRID128_K40, 1e-12), (W.Workload("grid128_k80_bumps4", 128, 80.0, "bumps", nbumps=4, seed=0), 1e-13),
                                   (W.GRID256_K80, 1e-13)], ids=["kappa40", "kappa80", "disc256"])
def test_tensor_cores_against_oracle_rows(N, w, eps):
    """64 plane waves and 64 random vectors in one application, each column
    against the oracle's rows (at kappa = 80 two high-frequency levels carry
    interaction lists, so the cone-to-cone transfers run on the tensor cores
    too)."""
    op = _make(w, eps)
    try:
        rows = np.sort(np.random.default_rng(41).choice(w.N, 32, replace=False))
        F = W.plane_waves(w.kappa, op.xy, 64) * (-w.kappa ** 2 * op.q)[:, None]
        for V in (F, W.random_vector(w.N, 64, seed=42)):
            Y = _apply(N, op, torch.as_tensor(V, device="cuda").contiguous(), N.BATCHED_TENSOR_CORES).cpu().numpy()
            ref = O.matvec_rows(w.n_side, w.kappa, op.q, V, rows)
            err = np.linalg.norm(Y[rows] - ref, axis=0) / np.linalg.norm(ref, axis=0)
            Yc = _apply(N, op, torch.as_tensor(V, device="cuda").contiguous(), N.BATCHED_CUDA_CORES).cpu().numpy()
            errc = np.linalg.norm(Yc[rows] - ref, axis=0) / np.linalg.norm(ref, axis=0)
            print(f"{w.name}: tensor cores vs oracle {err.max():.2e}, CUDA cores vs oracle {errc.max():.2e}")
            assert err.max() < MIXED_TOL, err.max()
        op.sync()
    finally:
        op.close()


def test_tensor_cores_potential(N, op128):
    """dafmm_potential (K v, no epilogue) through the same passes."""
    V = torch.as_tensor(W.random_vector(op128.N, 16, seed=43), device="cuda").contiguous()
    out = {}
    for mode in (N.BATCHED_TENSOR_CORES, N.BATCHED_CUDA_CORES):
        N.dafmm_set_batched_kernel(op128.ops, mode)
        o = torch.empty_like(V)
        N.dafmm_potential(op128.ops, V, o, N.DAFMM_MIXED)
        out[mode] = o
    N.dafmm_set_batched_kernel(op128.ops, N.BATCHED_AUTO)
    assert _cols_rel(out[N.BATCHED_TENSOR_CORES], out[N.BATCHED_CUDA_CORES]) < KERNELS_TOL


def test_fp64_ignores_the_mode(N, op128):
    V = torch.as_tensor(W.random_vector(op128.N, 8, seed=44), device="cuda").contiguous()
    assert torch.equal(_apply(N, op128, V, N.BATCHED_TENSOR_CORES, N.DAFMM_FP64), _apply(N, op128, V, N.BATCHED_CUDA_CORES, N.DAFMM_FP64))


def test_mode_argument_errors(N, op128):
    for bad in (-1, 3):
        with pytest.raises(N.DafmmError):
            N.dafmm_set_batched_kernel(op128.ops, bad)
