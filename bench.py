#!/usr/bin/env python
"""DAFMM matrix-vector product throughput on GB300 (Munknowns/s).

One step = one application of the DAFMM operator A = I + kappa^2 diag(q) K~
(upward pass, M2L, downward pass, near field, epilogue) to one synthetic
right-hand side of the 128 x 128 grid, kappa = 40, 4-bump contrast
(N = 16384), through the C-ABI call dafmm_matvec.  The headline value is the
mixed-precision application (complex64 operators, FP32 arithmetic); the FP64
application is timed in the same run and reported beside it.

--impl reference times the FP64 CPU oracle (test infrastructure) on the
same workload, a bounded sample of rows per step, on the host cores.

Multi-GPU runs (torchrun) run one independent replica per rank: a single
problem has no data-parallel split (it would exchange multipoles at every
level), so value = all ranks' unknowns / max-over-ranks time and scaling is
"weak".
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2204_00326_gb300 import replicas  # noqa: E402
from paper_2204_00326_gb300 import workloads as W  # noqa: E402

METRIC = "DAFMM matvec Munknowns/s; time-to-1e-8 residual, mixed vs FP64 on GB300"
FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=W.GRID128_K40.name, choices=sorted(W.WORKLOADS))
    ap.add_argument("--eps-nca", type=float, default=1e-12)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip the time-to-residual solves")
    ap.add_argument("--no-nbody", action="store_true", help="skip Experiment 1's N-body measurement")
    ap.add_argument("--no-mixed-batch", action="store_true", help="skip the mixed-size batch of problems")
    ap.add_argument("--no-batched-solve", action="store_true",
                    help="skip the 64-plane-wave solve on the 256 x 256, kappa = 80 disc workload")
    ap.add_argument("--nrhs", type=int, default=64, help="right-hand sides of the batched measurement (1 = skip)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--learned", action="store_true",
                    help="instead of the matvec line: train the initial-guess network and compare solves from its guess "
                         "and from zero on --workload (default grid512_k160_bumps8)")
    ap.add_argument("--learned-train", type=int, default=2000, help="training problems (solved at 64 x 64)")
    ap.add_argument("--learned-steps", type=int, default=6000, help="Adam steps")
    ap.add_argument("--learned-base", type=int, default=32)
    ap.add_argument("--learned-levels", type=int, default=4)
    return ap.parse_args()


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def _bf16_peak():
    """Dense bf16 TFLOP/s (burst): measured, else the fallback figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f).get("bf16_tflops", 1900.0), "measured"
    return 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        exe = shutil.which("nvidia-smi")
        if exe:
            self.proc = subprocess.Popen([exe, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                                          "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons), "samples": len(sm)}


def _traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None when the kernel source changed since that capture."""
    import hashlib

    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    src = os.path.join(ROOT, t["source"])
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return t["dram_bytes_per_launch"] if h == t["source_sha256_16"] else None


def cpu_baseline(w, target_s: float, seed: int = 21):
    """The FP64 oracle's row-by-row matvec on a bounded sample of rows."""
    import oracle

    xy = oracle.grid_nodes(w.n_side)
    q = W.contrast(w, xy)
    v = W.random_vector(w.N, 1, seed=seed)[:, 0]
    rng = np.random.default_rng(seed)
    probe = np.sort(rng.choice(w.N, 16, replace=False))
    t0 = time.perf_counter()
    oracle.matvec_rows(w.n_side, w.kappa, q, v, probe)
    tp = time.perf_counter() - t0
    nrows = int(min(w.N, max(16, 16 * target_s / max(tp, 1e-6))))
    rows = np.sort(rng.choice(w.N, nrows, replace=False))
    t0 = time.perf_counter()
    oracle.matvec_rows(w.n_side, w.kappa, q, v, rows)
    dt = time.perf_counter() - t0
    return {"value": nrows / dt / 1e6, "unit": "Munknowns/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{nrows} of {w.N} rows of A v (entries generated by quadrature, FP64), {dt:.1f} s"}


def run_reference(a, w):
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    import oracle

    xy = oracle.grid_nodes(w.n_side)
    q = W.contrast(w, xy)
    v = W.random_vector(w.N, 1, seed=21)[:, 0]
    rng = np.random.default_rng(21)
    probe = np.sort(rng.choice(w.N, 8, replace=False))
    t0 = time.perf_counter()
    oracle.matvec_rows(w.n_side, w.kappa, q, v, probe)
    tp = (time.perf_counter() - t0) / 8
    per_step = max(1.0, 150.0 / max(1, a.steps + a.warmup))  # whole run within a few minutes
    nrows = int(min(w.N, max(8, per_step / max(tp, 1e-9))))
    for _ in range(a.warmup):
        oracle.matvec_rows(w.n_side, w.kappa, q, v, rng.choice(w.N, nrows, replace=False))
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle.matvec_rows(w.n_side, w.kappa, q, v, rng.choice(w.N, nrows, replace=False))
    dt = time.perf_counter() - t0
    value = a.steps * nrows / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Munknowns/s", "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n_side": w.n_side, "N": w.N, "kappa": w.kappa, "precision": "fp64 oracle",
                       "rows_per_step": nrows},
            "cpu_baseline": {"value": value, "unit": "Munknowns/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{nrows} of {w.N} rows of A v per step"},
            "e2e": {"value": value, "unit": "Munknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_learned(a):
    """Learned initial guess on the target workload: train at 64 x 64 with the
    same points per wavelength, then HODLR-preconditioned GMRES (mixed
    precision, FP64 residual) to 1e-8 from zero and from the guess."""
    import torch

    import paper_2204_00326_gb300 as pkg

    pkg.build()
    from paper_2204_00326_gb300 import learned as Lr
    from paper_2204_00326_gb300 import native as N
    from paper_2204_00326_gb300.operator import DafmmOperator

    name = a.workload if "--workload" in sys.argv else W.GRID512_K160.name
    w = W.WORKLOADS[name]
    n_t = 64
    k_t = w.kappa * n_t / w.n_side
    X, Y, t_gen = Lr.generate(n_t, k_t, count=a.learned_train, seed=100000)
    net = N.unet_create(levels=a.learned_levels, base=a.learned_base, seed=1)
    losses, t_train = Lr.train(net, X, Y, steps=a.learned_steps, batch=16, lr=1e-3, lr_final=5e-5)
    del X, Y
    result = {"mode": "learned_guess", "workload": w.name, "n_side": w.n_side, "N": w.N, "kappa": w.kappa,
              "train": {"grid": n_t, "kappa": k_t, "problems": a.learned_train, "steps": a.learned_steps, "batch": 16,
                        "levels": a.learned_levels, "base": a.learned_base, "params": N.unet_num_params(net),
                        "solve_seconds": t_gen, "train_seconds": t_train,
                        "loss_first": float(np.mean(losses[:50])), "loss_last": float(np.mean(losses[-50:]))}}
    # in-distribution check at the training size
    op_t = DafmmOperator(n_t, k_t, np.zeros(n_t * n_t))
    q, f = Lr.problem(op_t.xy, k_t, 8, seed=999999)
    N.dafmm_set_contrast(op_t.ops, torch.as_tensor(q, device="cuda"))
    M = N.hodlr_factor(op_t.ops, rank=15, leaf_size=64)
    result["train_size"] = Lr.compare(op_t, net, f, M)
    N.hodlr_destroy(M)
    op_t.close()
    # the target workload
    t0 = time.perf_counter()
    op = DafmmOperator(w.n_side, w.kappa, lambda xy: W.contrast(w, xy))
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    M = N.hodlr_factor(op.ops, rank=15, leaf_size=64)
    t_factor = time.perf_counter() - t0
    f = -w.kappa ** 2 * op.q * W.plane_waves(w.kappa, op.xy)[:, 0]
    Lr.compare(op, net, f, M)  # warm-up (graph capture, workspaces)
    result["target"] = Lr.compare(op, net, f, M)
    result["target"]["setup_seconds"] = setup
    result["target"]["hodlr_factor_seconds"] = t_factor
    # network inference on the target grid
    fd = torch.as_tensor(f, device="cuda")
    xg = torch.empty_like(fd)
    for _ in range(3):
        N.unet_guess(net, op.ops, fd, xg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        N.unet_guess(net, op.ops, fd, xg)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 10
    flops = Lr.forward_flops(a.learned_levels, a.learned_base, w.n_side, w.n_side)
    result["inference"] = {"ms": ms, "gflop": flops / 1e9, "tflops": flops / (ms * 1e-3) / 1e12,
                           "peak_tflops": 152 * 128 * 2 * 2.07e9 / 1e12, "peak_kind": "FP32 FMA lanes x clock (CUDA cores)"}
    N.hodlr_destroy(M)
    op.close()
    N.unet_destroy(net)
    print(json.dumps(result), flush=True)


def batched_solve(N, DafmmOperator, nrhs=64, rank=15, singles=4):
    """Time to 1e-8 for nrhs plane waves (theta_k = 2 pi k / nrhs) solved
    together on the 256 x 256, kappa = 80 disc workload: HODLR-preconditioned
    GMRES (rank `rank`), one batched application and one batched HODLR apply
    per step, FP64 and mixed precision with FP64 refinement.  A few columns
    solved one at a time give the per-right-hand-side cost without batching."""
    import torch

    w = W.GRID256_K80
    t0 = time.perf_counter()
    op = DafmmOperator(w.n_side, w.kappa, lambda xy: W.contrast(w, xy))
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    M = N.hodlr_factor(op.ops, rank=rank, leaf_size=64)
    t_factor = time.perf_counter() - t0
    F = torch.as_tensor(W.plane_waves(w.kappa, op.xy, nrhs) * (-w.kappa ** 2 * op.q)[:, None], device="cuda").contiguous()
    out = {"workload": w.name, "N": w.N, "nrhs": nrhs, "tol": 1e-8, "hodlr_rank": rank, "setup_s": setup,
           "hodlr_factor_s": t_factor, "setup_excluded": True}
    for name, prec in (("fp64", N.DAFMM_FP64), ("mixed", N.DAFMM_MIXED)):
        for rep in range(2):  # the first solve warms up (workspaces, graph capture)
            X = torch.zeros_like(F)
            rc, sts, _ = N.gmres_solve(op.ops, F, X, tol=1e-8, precision=prec, restart=50, max_iters=2000, M=M)
        its = [s.iterations for s in sts]
        out[name] = {"seconds": sts[0].seconds, "converged": all(s.converged for s in sts),
                     "worst_rel_residual": max(s.rel_residual for s in sts), "steps": sts[0].matvecs,
                     "iterations_max": max(its), "iterations_mean": float(np.mean(its)),
                     "munknowns_rhs_per_s": w.N * nrhs / sts[0].seconds / 1e6}
    # the same columns one at a time (mixed), for the per-right-hand-side cost without batching
    f1 = F[:, 0].contiguous()
    x1 = torch.zeros_like(f1)
    N.gmres_solve(op.ops, f1, x1, tol=1e-8, precision=N.DAFMM_MIXED, restart=50, max_iters=2000, M=M)
    secs, its = [], []
    for k in range(singles):
        fk = F[:, k * (nrhs // singles)].contiguous()
        xk = torch.zeros_like(fk)
        rc, st, _ = N.gmres_solve(op.ops, fk, xk, tol=1e-8, precision=N.DAFMM_MIXED, restart=50, max_iters=2000, M=M)
        secs.append(st.seconds)
        its.append(st.iterations)
    out["mixed_one_at_a_time"] = {"columns": singles, "seconds_per_rhs": float(np.mean(secs)), "iterations_mean": float(np.mean(its))}
    out["mixed_batched_seconds_per_rhs"] = out["mixed"]["seconds"] / nrhs
    out["mixed_vs_fp64_speedup"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    N.hodlr_destroy(M)
    op.close()
    return out


def mixed_size_batch(N, DafmmOperator, count=8, sizes=(64, 128, 256), nrhs=8, reps=10):
    """The mixed-size batch (kappa = 0.3 sqrt(N), bump or disc contrasts, 8
    plane waves each): every problem's several-right-hand-side passes tuned
    (dafmm_tune_batched, choice recorded), then the whole batch applied in
    one captured graph (dafmm_batch_matvec), against the same applications
    launched one problem after another.  Grids up to 256^2: a 1024^2 problem
    alone holds tens of GB of operators and needs a long host setup."""
    import torch

    ws = W.mixed_size_batch(count=count, sizes=sizes, seed=5, nrhs=nrhs)
    t0 = time.perf_counter()
    ops = [DafmmOperator(w.n_side, w.kappa, lambda xy, w=w: W.contrast(w, xy)) for w in ws]
    setup = time.perf_counter() - t0
    vs = [torch.as_tensor(W.plane_waves(w.kappa, op.xy, nrhs) * (-w.kappa ** 2 * op.q)[:, None], device="cuda").contiguous()
          for w, op in zip(ws, ops)]
    outs = [torch.empty_like(v) for v in vs]
    total = sum(w.N for w in ws) * nrhs
    out = {"problems": [w.name for w in ws], "nrhs": nrhs, "unknowns_x_rhs": total, "setup_s": setup,
           "sizes_note": "grids drawn from 64^2, 128^2, 256^2"}
    out["tuning"] = {w.name: N.dafmm_tune_batched(op.ops, nrhs, N.DAFMM_MIXED) for w, op in zip(ws, ops)}
    b = N.Batch([op.ops for op in ops])
    for name, prec in (("mixed", N.DAFMM_MIXED), ("fp64", N.DAFMM_FP64)):
        for _ in range(3):
            b.matvec(vs, outs, prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.matvec(vs, outs, prec)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        e0.record()
        for _ in range(reps):
            for op, v, o in zip(ops, vs, outs):
                op.matvec(v, o, prec)
        e1.record()
        torch.cuda.synchronize()
        ms_seq = e0.elapsed_time(e1) / reps
        out[name] = {"ms_per_batch": ms, "munknowns_rhs_per_s": total / (ms * 1e-3) / 1e6,
                     "ms_one_problem_after_another": ms_seq}
    b.close()
    for op in ops:
        op.close()
    return out


def experiment1(N, DafmmOperator, reps=10):
    """Experiment 1 (Section 6.2): the point N-body potential of random
    charges at the 256 x 256 Chebyshev nodes (N = 65536, kappa = 50) by the
    DAFMM (dafmm_potential, FP64 and mixed) and by direct summation on the
    GPU; relative errors against the direct sum for three eps_nca (the
    paper's error against eps_nca), apply times with CUDA events."""
    import torch

    w = W.NBODY256_K50
    f = torch.as_tensor(W.random_vector(w.N, 1, seed=65)[:, 0], device="cuda")
    out = {"workload": w.name, "N": w.N, "kappa": w.kappa, "p": 4}
    direct = torch.empty_like(f)
    tree_op = None
    rows = []
    for eps in (1e-6, 1e-9, 1e-12):
        t0 = time.perf_counter()
        op = DafmmOperator(w.n_side, w.kappa, np.zeros(w.N), eps_nca=eps, kernel=N.DAFMM_KERNEL_POINTS)
        setup = time.perf_counter() - t0
        if tree_op is None:
            N.dafmm_nbody_direct(op.tree, f, direct)  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            N.dafmm_nbody_direct(op.tree, f, direct)
            e1.record()
            torch.cuda.synchronize()
            out["direct_ms"] = e0.elapsed_time(e1)
            tree_op = True
        rec = {"eps_nca": eps, "setup_s": setup}
        for name, prec in (("fp64", N.DAFMM_FP64), ("mixed", N.DAFMM_MIXED)):
            u = op.potential(f, precision=prec)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                op.potential(f, u, precision=prec)
            e1.record()
            torch.cuda.synchronize()
            rec[name] = {"ms": e0.elapsed_time(e1) / reps,
                         "rel_error_vs_direct": (torch.linalg.norm(u - direct) / torch.linalg.norm(direct)).item()}
        rows.append(rec)
        op.close()
    out["by_eps_nca"] = rows
    return out


def main():
    a = _args()
    w = W.WORKLOADS[a.workload]
    if a.impl == "reference":
        run_reference(a, w)
        return
    if a.learned:
        run_learned(a)
        return
    rank, world, local = _dist_env()
    import torch

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    import paper_2204_00326_gb300 as pkg

    pkg.build()
    from paper_2204_00326_gb300 import native as N
    from paper_2204_00326_gb300.operator import DafmmOperator

    t0 = time.perf_counter()
    op = DafmmOperator(w.n_side, w.kappa, lambda xy: W.contrast(w, xy), eps_nca=a.eps_nca)
    setup_s = time.perf_counter() - t0
    st = op.stats()
    stream = torch.cuda.current_stream()
    v = torch.as_tensor(W.random_vector(w.N, 1, seed=1 + rank)[:, 0], device="cuda")
    out = torch.empty_like(v)
    # L2 flush between timed steps: a read of 256 MiB (twice the L2) evicts every
    # line the previous step touched.  A write of the buffer would do the same but
    # leave up to 129 MB of dirty lines, whose write-back the next timed kernel
    # would pay (measured: far field 102 us after a write, 96.5 us after a read,
    # 94.6 us without any flush; the operators alone, 266 MB, exceed the L2).
    flush_buf = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    flush_sink = torch.empty((), dtype=torch.float32, device="cuda")

    def flush_l2():
        torch.sum(flush_buf, dim=0, out=flush_sink)

    def timed(prec, steps, profile):
        for _ in range(a.warmup):
            flush_l2()
            op.matvec(v, out, prec)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        if profile:
            N.dafmm_profile(op.ops, True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in evs:
            flush_l2()  # L2 flush between timed steps, outside the events
            e0.record(stream)
            op.matvec(v, out, prec)
            e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
        prof = None
        if profile:
            prof = N.dafmm_profile_read(op.ops)
            N.dafmm_profile(op.ops, False)
        return replicas.max_over_ranks(ms, device="cuda"), prof

    clk = ClockSampler(local).__enter__()
    # the step times unprofiled (the user's path); the pass times from a second
    # run whose graphs carry event-record nodes at the pass marks (each adds
    # about 2.5 us of latency, so those intervals are conservative)
    ms_mixed, _ = timed(N.DAFMM_MIXED, a.steps, False)
    ms_fp64, _ = timed(N.DAFMM_FP64, a.steps, False)
    _, prof_mixed = timed(N.DAFMM_MIXED, a.steps, True)
    _, prof_fp64 = timed(N.DAFMM_FP64, a.steps, True)

    # end to end: pinned host input -> device -> matvec -> pinned host output
    vh = v.cpu().pin_memory()
    oh = torch.empty_like(vh).pin_memory()
    vd = torch.empty_like(v)
    for _ in range(a.warmup):
        vd.copy_(vh, non_blocking=True)
        op.matvec(vd, out, N.DAFMM_MIXED)
        oh.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        vd.copy_(vh, non_blocking=True)
        op.matvec(vd, out, N.DAFMM_MIXED)
        oh.copy_(out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = replicas.max_over_ranks(e0.elapsed_time(e1), device="cuda")

    value = replicas.job_throughput(float(w.N) * a.steps, world, ms_mixed)
    value64 = replicas.job_throughput(float(w.N) * a.steps, world, ms_fp64)
    e2e = replicas.job_throughput(float(w.N) * a.steps, world, ms_e2e)

    hbm, peak_kind = _peaks()
    # dominant kernel: the fused far field (every tree pass in one cooperative launch)
    calls = max(1, prof_mixed.calls)
    ms_far = prof_mixed.ms_far / calls
    cmacs_far = st.cmacs_far_fused  # realised entries the kernel streams (its operators, see dafmm_stats_t)
    # operators read once (complex64), coefficients written and read once (complex64), the input read (complex128)
    bytes_far = cmacs_far * 8.0 + st.coef_bytes_per_rhs / 2.0 + 16.0 * w.N
    achieved = bytes_far / (ms_far * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": _traffic(), "kernel": "stream_kernel<float>: P2M, M2M, M2L, L2L of every level, one launch",
                "peak_kind": f"{peak_kind} HBM copy bandwidth", "algorithmic_bytes_per_launch": bytes_far,
                "ms_per_launch": ms_far,
                "pass_ms": {"far": ms_far, "leaf": prof_mixed.ms_leaf / calls}}
    calls64 = max(1, prof_fp64.calls)
    ms_far64 = prof_fp64.ms_far / calls64
    # complex128 leg: the operators as float pairs (16 bytes an entry) read once,
    # complex128 coefficients written and read once, the input read
    bytes_far64 = cmacs_far * 16.0 + st.coef_bytes_per_rhs + 16.0 * w.N
    achieved64 = bytes_far64 / (ms_far64 * 1e-3) / 1e9
    roof64 = {"bound": "hbm", "achieved": achieved64, "peak": hbm, "unit": "GB/s", "frac": achieved64 / hbm,
              "kernel": "stream_kernel<double>: every tree pass, one launch, double-float arithmetic",
              "peak_kind": f"{peak_kind} HBM copy bandwidth", "algorithmic_bytes_per_launch": bytes_far64,
              "ms_per_launch": ms_far64,
              "pass_ms": {"far": ms_far64, "leaf": prof_fp64.ms_leaf / calls64}}

    # several right-hand sides in one application: nrhs plane waves
    batched = None
    if a.nrhs > 1:
        Vb = torch.as_tensor(W.plane_waves(w.kappa, op.xy, a.nrhs), device="cuda").contiguous()
        Yb = torch.empty_like(Vb)
        batched = {"nrhs": a.nrhs}
        for name, prec in (("mixed", N.DAFMM_MIXED), ("fp64", N.DAFMM_FP64)):
            for _ in range(a.warmup):
                flush_l2()
                op.matvec(Vb, Yb, prec)
            torch.cuda.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
            for e0b, e1b in evs:
                flush_l2()
                e0b.record(stream)
                op.matvec(Vb, Yb, prec)
                e1b.record(stream)
            torch.cuda.synchronize()
            msb = sum(x.elapsed_time(y) for x, y in evs) / a.steps
            batched[name] = {"value": w.N * a.nrhs / (msb * 1e-3) / 1e6, "unit": "Munknowns/s (unknowns x rhs)",
                             "ms_per_step": msb}
        cm = st.cmacs_per_rhs * a.nrhs
        batched["mixed"]["achieved_tflops"] = 8.0 * cm / (batched["mixed"]["ms_per_step"] * 1e-3) / 1e12
        # the same application with the tree passes on the tensor cores (opt-in kernel)
        N.dafmm_set_batched_kernel(op.ops, N.BATCHED_TENSOR_CORES)
        for _ in range(a.warmup):
            flush_l2()
            op.matvec(Vb, Yb, N.DAFMM_MIXED)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        for e0b, e1b in evs:
            flush_l2()
            e0b.record(stream)
            op.matvec(Vb, Yb, N.DAFMM_MIXED)
            e1b.record(stream)
        torch.cuda.synchronize()
        N.dafmm_set_batched_kernel(op.ops, N.BATCHED_AUTO)
        mst = sum(x.elapsed_time(y) for x, y in evs) / a.steps
        cm_tree = (st.cmacs_up + st.cmacs_m2l + st.cmacs_down) * a.nrhs
        issued = 64.0 * cm_tree  # tensor flops issued per complex MAC: 8 (real embedding) x 2 (stacked rows) x 4 (MMAs)
        batched["mixed_tensor_cores"] = {
            "value": w.N * a.nrhs / (mst * 1e-3) / 1e6, "unit": "Munknowns/s (unknowns x rhs)", "ms_per_step": mst,
            "kernel": "stream_batched_tc_kernel: tcgen05.mma kind::tf32, three-part tf32 split, per-chunk accumulators",
            "issued_tensor_tflops_upper_bound": issued / (mst * 1e-3) / 1e12,
            "bf16_peak_tflops": _bf16_peak()[0], "peak_kind": _bf16_peak()[1] + " bf16 (tf32 runs at half the bf16 rate)",
            "note": "not the default: slower than the CUDA-core kernel at these chunk shapes"}
        del Vb, Yb

    # time to relative residual 1e-8 (FP64 residual), f = -kappa^2 q u_inc
    ttr = None
    if not a.no_solve:
        f = torch.as_tensor(-w.kappa ** 2 * op.q * W.plane_waves(w.kappa, op.xy)[:, 0], device="cuda")
        t0 = time.perf_counter()
        M = N.hodlr_factor(op.ops, rank=15, leaf_size=64)
        t_factor = time.perf_counter() - t0
        # a tolerance-based HODLR (ranks to 1e-3) trades factor time for iterations
        t0 = time.perf_counter()
        Mt = N.hodlr_factor(op.ops, rank=0, tol=1e-3, leaf_size=64)
        t_factor_t = time.perf_counter() - t0
        ttr = {"tol": 1e-8, "rhs": "plane wave exp(i kappa x1)", "hodlr_factor_s": t_factor,
               "hodlr_tol1e-3_factor_s": t_factor_t, "hodlr_tol1e-3_rank_max": N.hodlr_info(Mt)["rank_max"],
               "setup_excluded": True}
        for name, prec, pre in (("fp64", N.DAFMM_FP64, None), ("mixed", N.DAFMM_MIXED, None),
                                ("fp64_hodlr15", N.DAFMM_FP64, M), ("mixed_hodlr15", N.DAFMM_MIXED, M),
                                ("fp64_hodlr_tol1e-3", N.DAFMM_FP64, Mt), ("mixed_hodlr_tol1e-3", N.DAFMM_MIXED, Mt)):
            for rep in range(2):  # the first solve warms up (graph capture, workspace)
                x = torch.zeros_like(f)
                rc, gs, _ = N.gmres_solve(op.ops, f, x, tol=1e-8, precision=prec, restart=50, max_iters=3000, M=pre)
            ttr[name] = {"seconds": gs.seconds, "iterations": gs.iterations, "outer_iterations": gs.outer_iterations,
                         "matvecs": gs.matvecs, "rel_residual": gs.rel_residual, "converged": bool(gs.converged)}
        N.hodlr_destroy(M)
        N.hodlr_destroy(Mt)

    ttr_b = None
    if not a.no_batched_solve and world == 1:
        ttr_b = batched_solve(N, DafmmOperator)
    exp1 = None
    if not a.no_nbody and world == 1:
        exp1 = experiment1(N, DafmmOperator)
    mbatch = None
    if not a.no_mixed_batch and world == 1:
        mbatch = mixed_size_batch(N, DafmmOperator)

    clk.__exit__(None, None, None)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(w, a.cpu_seconds)

    line = {
        "metric": METRIC, "value": value, "unit": "Munknowns/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms_mixed / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64", "data": "synthetic",
        "config": {"workload": w.name, "n_side": w.n_side, "N": w.N, "kappa": w.kappa, "contrast": w.contrast,
                   "nbumps": w.nbumps, "nrhs": 1, "precision": "mixed (complex64 operators, FP32 math)",
                   "eps_nca": a.eps_nca, "l2": "flushed: 256 MiB read between timed steps (operators streamed per step: 266 MB, larger than the L2)", "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": "Munknowns/s", "h2d_bytes_per_step": w.N * 16, "d2h_bytes_per_step": w.N * 16},
        "gpu_launches": int(st.launches_per_call * a.steps),
        "clocks": clk.summary(),
        "fp64": {"value": value64, "unit": "Munknowns/s", "ms_per_step": ms_fp64 / a.steps,
                 "dtype": "c128 (far field in double-float: float pairs, u = 2^-48)", "roofline": roof64,
                 "gpu_launches": int(st.launches_per_call_fp64 * a.steps)},
        "batched": batched,
        "time_to_residual": ttr,
        "time_to_residual_batched": ttr_b,
        "experiment1_nbody": exp1,
        "mixed_size_batch": mbatch,
        "setup_s": {"total": setup_s, "entry_table": st.setup_seconds_table, "nca": st.setup_seconds_nca},
        "operator": {"bytes_fp32": st.operator_bytes_fp32, "bytes_fp64": st.operator_bytes_fp64,
                     "cmacs_per_rhs": st.cmacs_per_rhs},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    op.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
