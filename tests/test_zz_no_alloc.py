"""dafmm_matvec_noalloc: the allocation-free variant of dafmm_matvec.

Some callers cannot have device memory allocated for them at call time (their
device memory belongs to their own pool, or their loop cannot absorb
cudaMalloc's implicit synchronisation, or their deployment fixes all memory
up front).  The variant keeps its scratch in a static device array; these
tests call it through the C-ABI twice in a row (the array keeps the previous
call's contents) and compare with dafmm_matvec at the parity tolerances.
This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2204_00326_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 2e-5


def _rel(a, b):
    return (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()


@pytest.mark.parametrize("w", [W.GRID32_K8, W.GRID128_K40], ids=lambda w: w.name)
def test_noalloc_matches_matvec_on_consecutive_calls(w):
    import paper_2204_00326_gb300 as pkg

    pkg.build()
    from paper_2204_00326_gb300 import native as N
    from paper_2204_00326_gb300.operator import DafmmOperator

    op = DafmmOperator(w.n_side, w.kappa, lambda xy: W.contrast(w, xy))
    for prec, tol in ((N.DAFMM_FP64, FP64_TOL), (N.DAFMM_MIXED, MIXED_TOL)):
        for seed in (31, 32):  # two calls in a row, different inputs
            v = torch.as_tensor(W.random_vector(w.N, 1, seed=seed)[:, 0], device="cuda")
            ref = torch.empty_like(v)
            got = torch.full_like(v, complex(np.nan, np.nan))
            N.dafmm_matvec(op.ops, v, ref, prec)
            N.dafmm_matvec_noalloc(op.ops, v, got, prec)
            torch.cuda.synchronize()
            assert torch.isfinite(torch.view_as_real(got)).all()
            assert _rel(got, ref) < tol
    op.close()


def test_noalloc_argument_errors():
    import paper_2204_00326_gb300 as pkg

    pkg.build()
    from paper_2204_00326_gb300 import native as N
    from paper_2204_00326_gb300.operator import DafmmOperator

    assert N.lib.dafmm_matvec_noalloc(None, None, None, 0, None) == N.DAFMM_EBADARG
    w = W.GRID32_K8
    op = DafmmOperator(w.n_side, w.kappa, lambda xy: W.contrast(w, xy))
    v = torch.as_tensor(W.random_vector(w.N, 1, seed=33)[:, 0], device="cuda")
    out = torch.empty_like(v)
    with pytest.raises(N.DafmmError) as e:  # unknown precision
        N.dafmm_matvec_noalloc(op.ops, v, out, 7)
    assert e.value.code == N.DAFMM_EBADARG
    with pytest.raises(N.DafmmError) as e:  # input and output alias
        N.dafmm_matvec_noalloc(op.ops, v, v, N.DAFMM_FP64)
    assert e.value.code == N.DAFMM_EBADARG
    op.close()


def test_noalloc_rejects_problems_larger_than_its_scratch():
    """A problem whose coefficients do not fit the static array is refused
    with DAFMM_EBADARG before any work is queued, and the output is left as
    it was.  Smaller problems on the way give the same result as
    dafmm_matvec."""
    import paper_2204_00326_gb300 as pkg

    pkg.build()
    from paper_2204_00326_gb300 import native as N
    from paper_2204_00326_gb300.operator import DafmmOperator

    rejected = None
    for w in (W.GRID256_K80, W.GRID512_K160):
        op = DafmmOperator(w.n_side, w.kappa, lambda xy: W.contrast(w, xy))
        try:
            v = torch.as_tensor(W.random_vector(w.N, 1, seed=34)[:, 0], device="cuda")
            got = torch.full_like(v, complex(1.5, -2.5))
            try:
                N.dafmm_matvec_noalloc(op.ops, v, got, N.DAFMM_MIXED)
            except N.DafmmError as e:
                torch.cuda.synchronize()
                assert e.code == N.DAFMM_EBADARG
                assert str(N.NOALLOC_SCRATCH_BYTES) in str(e)
                assert bool((got == complex(1.5, -2.5)).all())
                rejected = w.name
                break
            ref = torch.empty_like(v)
            N.dafmm_matvec(op.ops, v, ref, N.DAFMM_MIXED)
            torch.cuda.synchronize()
            assert _rel(got, ref) < MIXED_TOL
        finally:
            op.close()
    assert rejected is not None
