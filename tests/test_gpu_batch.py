"""Several problems of different sizes applied in one captured graph
(dafmm_batch_matvec) and the tuner of the several-right-hand-side passes
(dafmm_tune_batched): the mixed-size batch of problems with kappa =
0.3 sqrt(N), Gaussian-bump or disc contrasts and 8 plane waves each.

Tolerances: the batch runs each problem's own kernels, so its outputs equal
the problems' own applications bit for bit; against the oracle's rows the
FP64 bar is 1e-10 and the mixed one 2e-5 (as in test_gpu_parity.py).  A
tuned configuration changes the kernel or the grid, so it is compared with
the untuned result at the mixed bar.
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
def problems(N):
    from paper_2204_00326_gb300.operator import DafmmOperator

    ws = W.mixed_size_batch(count=5, sizes=(64, 128, 256), seed=11)
    assert len({w.n_side for w in ws}) >= 2  # mixed sizes
    ops = [DafmmOperator(w.n_side, w.kappa, lambda xy, w=w: W.contrast(w, xy)) for w in ws]
    yield ws, ops
    for op in ops:
        op.close()


def _inputs(ws, ops):
    return [torch.as_tensor(W.plane_waves(w.kappa, op.xy, 8) * (-w.kappa ** 2 * op.q)[:, None], device="cuda").contiguous()
            for w, op in zip(ws, ops)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_batch_equals_each_problem_and_the_oracle(N, problems, precision, tol):
    ws, ops = problems
    prec = N.DAFMM_FP64 if precision == "fp64" else N.DAFMM_MIXED
    vs = _inputs(ws, ops)
    outs = [torch.empty_like(v) for v in vs]
    b = N.Batch([op.ops for op in ops])
    try:
        b.matvec(vs, outs, prec)
        b.matvec(vs, outs, prec)  # replay of the captured graph
        torch.cuda.synchronize()
        for w, op, v, o in zip(ws, ops, vs, outs):
            own = op.matvec(v, precision=prec)
            assert torch.equal(o, own), w.name
            rows = np.sort(np.random.default_rng(w.n_side).choice(w.N, 12, replace=False))
            ref = O.matvec_rows(w.n_side, w.kappa, op.q, v.cpu().numpy(), rows)
            got = o.cpu().numpy()[rows]
            err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
            assert err.max() < tol, (w.name, err.max())
        # new vectors: a new capture, the same results
        vs2 = [v.clone() for v in vs]
        outs2 = [torch.empty_like(v) for v in vs]
        b.matvec(vs2, outs2, prec)
        torch.cuda.synchronize()
        for o, o2 in zip(outs, outs2):
            assert torch.equal(o, o2)
    finally:
        b.close()
    for op in ops:
        op.sync()


def test_batch_with_one_rhs(N, problems):
    """One right-hand side: the problems run in order inside the graph."""
    ws, ops = problems
    vs = [torch.as_tensor(W.random_vector(w.N, 1, seed=80 + k)[:, 0], device="cuda") for k, w in enumerate(ws)]
    outs = [torch.empty_like(v) for v in vs]
    b = N.Batch([op.ops for op in ops])
    try:
        for prec in (N.DAFMM_MIXED, N.DAFMM_FP64):
            b.matvec(vs, outs, prec)
            torch.cuda.synchronize()
            for op, v, o in zip(ops, vs, outs):
                assert torch.equal(o, op.matvec(v, precision=prec))
    finally:
        b.close()
    for op in ops:
        op.sync()


def test_tuner_records_and_applies_its_choice(N, problems):
    ws, ops = problems
    k = max(range(len(ws)), key=lambda i: ws[i].N)
    op = ops[k]
    v = _inputs([ws[k]], [op])[0]
    before = op.matvec(v, precision=N.DAFMM_MIXED)
    t = N.dafmm_tune_batched(op.ops, 8, N.DAFMM_MIXED)
    try:
        assert t["nrhs"] == 8 and t["precision"] == "mixed" and len(t["candidates"]) == 5
        assert t["best_ms"] == min(c["ms"] for c in t["candidates"]) and t["best_ms"] > 0
        assert {"kernel": t["kernel"], "ctas_per_sm": t["ctas_per_sm"], "ms": t["best_ms"]} in t["candidates"]
        after = op.matvec(v, precision=N.DAFMM_MIXED)
        assert (torch.linalg.norm(after - before) / torch.linalg.norm(before)).item() < 2e-5
        t64 = N.dafmm_tune_batched(op.ops, 8, N.DAFMM_FP64)
        assert len(t64["candidates"]) == 4 and t64["kernel"] == "cuda_cores"
    finally:
        N.dafmm_set_batched_kernel(op.ops, N.BATCHED_AUTO)
        N.dafmm_set_batched_grid(op.ops, 0)
    with pytest.raises(N.DafmmError):
        N.dafmm_tune_batched(op.ops, 1, N.DAFMM_MIXED)
    with pytest.raises(N.DafmmError):
        N.dafmm_set_batched_grid(op.ops, 33)
