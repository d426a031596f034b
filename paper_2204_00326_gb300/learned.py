"""Learned initial guess: training data from the library's own solver, the
training loop and the evaluation (argument marshalling over the C-ABI; every
network step runs in the library's kernels).

Problems follow the bump-mixture recipe of the workloads (centres, widths and
amplitudes drawn from a seeded PCG64), with a plane wave of random direction;
the right-hand side is f = -kappa^2 q u_inc and the target the solution psi
of A psi = f (Eq. 12a), computed by HODLR-preconditioned GMRES to 1e-10.  A
network trained on an n_t x n_t grid is applied on n x n grids with the same
number of points per wavelength (kappa_t = kappa n_t / n).

Images: the node grid as an n_side x n_side picture (pixel (x, y) holds node
(4 lx + k1, 4 ly + k2) of Morton leaf (lx, ly), local index k1 + 4 k2),
channels (q, Re f / s, Im f / s) in, (Re psi / s, Im psi / s) out, s = max|f|.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import native as N
from .operator import DafmmOperator


def node_pixels(n_side: int) -> np.ndarray:
    """Pixel index y * n_side + x of every node (Morton leaf order)."""
    N_ = n_side * n_side
    n = np.arange(N_)
    leaf, k = n >> 4, n & 15
    lx = np.zeros(N_, dtype=np.int64)
    ly = np.zeros(N_, dtype=np.int64)
    for b in range(31):
        lx |= ((leaf >> (2 * b)) & 1) << b
        ly |= ((leaf >> (2 * b + 1)) & 1) << b
    return (4 * ly + (k >> 2)) * n_side + 4 * lx + (k & 3)


def bump_contrast(xy: np.ndarray, nbumps: int, rng: np.random.Generator) -> np.ndarray:
    """Sum of nbumps Gaussian bumps (centres, then widths, then amplitudes)."""
    centres = rng.uniform(-0.6, 0.6, size=(nbumps, 2))
    widths = rng.uniform(0.1, 0.3, size=nbumps)
    amps = rng.uniform(0.5, 2.0, size=nbumps)
    q = np.zeros(len(xy))
    for c, s, a in zip(centres, widths, amps):
        q += a * np.exp(-((xy[:, 0] - c[0]) ** 2 + (xy[:, 1] - c[1]) ** 2) / (s * s))
    return q


def problem(xy: np.ndarray, kappa: float, nbumps: int, seed: int):
    """(q, f) of one random problem: bump contrast, plane wave of random direction."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = bump_contrast(xy, nbumps, rng)
    th = rng.uniform(0.0, 2.0 * np.pi)
    u = np.exp(1j * kappa * (xy[:, 0] * np.cos(th) + xy[:, 1] * np.sin(th)))
    return q, -kappa * kappa * q * u


def to_image(n_side: int, pix: np.ndarray, q: np.ndarray, v: np.ndarray, s: float) -> np.ndarray:
    img = np.zeros((n_side * n_side, 3), np.float32)
    img[pix, 0] = q
    img[pix, 1] = v.real / s
    img[pix, 2] = v.imag / s
    return img.reshape(n_side, n_side, 3)


def to_target(n_side: int, pix: np.ndarray, psi: np.ndarray, s: float) -> np.ndarray:
    img = np.zeros((n_side * n_side, 2), np.float32)
    img[pix, 0] = psi.real / s
    img[pix, 1] = psi.imag / s
    return img.reshape(n_side, n_side, 2)


def generate(n_side: int, kappa: float, count: int, nbumps: int = 8, seed: int = 1000, rank: int = 15, tol: float = 1e-10):
    """count (input, target) image pairs solved by HODLR-preconditioned GMRES.

    One tree and one NCA operator serve every contrast (dafmm_set_contrast);
    the HODLR preconditioner is refactored per contrast.  Returns float32
    tensors [count, n, n, 3] and [count, n, n, 2] on the GPU and the seconds.
    """
    t0 = time.perf_counter()
    op = DafmmOperator(n_side, kappa, np.zeros(n_side * n_side))
    pix = node_pixels(n_side)
    X = np.zeros((count, n_side, n_side, 3), np.float32)
    Y = np.zeros((count, n_side, n_side, 2), np.float32)
    try:
        for k in range(count):
            q, f = problem(op.xy, kappa, nbumps, seed + k)
            N.dafmm_set_contrast(op.ops, torch.as_tensor(q, device="cuda"))
            M = N.hodlr_factor(op.ops, rank=rank, leaf_size=64)
            try:
                fd = torch.as_tensor(f, device="cuda")
                x = torch.zeros_like(fd)
                rc, st, _ = N.gmres_solve(op.ops, fd, x, tol=tol, precision=N.DAFMM_MIXED, M=M, max_iters=2000)
                if rc != N.DAFMM_OK:
                    raise RuntimeError(f"training solve {k} did not converge: {st.rel_residual}")
            finally:
                N.hodlr_destroy(M)
            s = float(np.abs(f).max()) or 1.0
            X[k] = to_image(n_side, pix, q, f, s)
            Y[k] = to_target(n_side, pix, x.cpu().numpy(), s)
    finally:
        op.close()
    return torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda"), time.perf_counter() - t0


def train(net: int, X: torch.Tensor, Y: torch.Tensor, steps: int, batch: int = 16, lr: float = 1e-3, seed: int = 0,
          lr_final: float = 1e-4):
    """Adam on random minibatches (learning rate decaying geometrically to lr_final).

    Returns the loss of every step and the seconds.
    """
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    t0 = time.perf_counter()
    out = torch.empty((batch,) + tuple(Y.shape[1:]), dtype=torch.float32, device=X.device)
    for k in range(steps):
        idx = torch.randint(0, X.shape[0], (batch,), generator=g).to(X.device)
        xb = X.index_select(0, idx).contiguous()
        yb = Y.index_select(0, idx).contiguous()
        loss, _ = N.unet_backward(net, xb, yb, out)
        rate = lr * (lr_final / lr) ** (k / max(1, steps - 1))
        N.unet_adam(net, rate)
        losses.append(loss)
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0


def compare(op: DafmmOperator, net: int, f: np.ndarray, M: int | None, tol: float = 1e-8, precision: int = N.DAFMM_MIXED,
            restart: int = 50, max_iters: int = 3000):
    """GMRES from x0 = 0 against GMRES from the network's guess (acceptance rule applied)."""
    fd = torch.as_tensor(f, device="cuda")
    res = {}
    x = torch.zeros_like(fd)
    t0 = time.perf_counter()
    rc, st, _ = N.gmres_solve(op.ops, fd, x, tol=tol, precision=precision, M=M, restart=restart, max_iters=max_iters)
    res["zero_guess"] = {"converged": rc == N.DAFMM_OK, "iterations": st.iterations, "matvecs": st.matvecs,
                         "seconds": time.perf_counter() - t0, "rel_residual": st.rel_residual}
    x = torch.zeros_like(fd)
    t0 = time.perf_counter()
    rc, st, ls = N.gmres_solve_learned(op.ops, net, fd, x, flags=1, tol=tol, precision=precision, M=M, restart=restart,
                                       max_iters=max_iters)
    res["learned_guess"] = {"converged": rc == N.DAFMM_OK, "iterations": st.iterations, "matvecs": st.matvecs,
                            "seconds": time.perf_counter() - t0, "rel_residual": st.rel_residual,
                            "guess_used": bool(ls.guess_used), "guess_residual": ls.guess_residual}
    return res


def forward_flops(levels: int, base: int, height: int, width: int, batch: int = 1) -> float:
    """Multiply-add operations x 2 of one forward pass (convolutions only)."""
    c = [base << l for l in range(levels)]
    px = [batch * (height >> l) * (width >> l) for l in range(levels)]
    f = 0.0
    for l in range(levels):
        f += 2.0 * 9 * (3 if l == 0 else c[l - 1]) * c[l] * px[l] + 2.0 * 9 * c[l] * c[l] * px[l]
    for l in range(levels - 1):
        f += 2.0 * 9 * px[l] * (c[l + 1] * c[l] + 2 * c[l] * c[l] + c[l] * c[l])
    return f + 2.0 * c[0] * 2 * px[0]

