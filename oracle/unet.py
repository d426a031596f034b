"""Plain FP64 reference of the learned-guess network (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's baseline legs use this
module; the product path never imports it.  It shares no code with the CUDA
implementation.

The network is not part of the paper: it maps (q, Re f / s, Im f / s) on the
node grid to (Re psi / s, Im psi / s), psi the solution of Eq. 13.  Every
layer is written out directly, in float64 numpy:

* convolution (cross-correlation with zero padding):
  out[b, y, x, o] = bias[o] + sum_{ky, kx, i} in[b, y + ky - R, x + kx - R, i] w[ky, kx, i, o],
  one einsum per kernel tap over the padded input;
* its adjoints: d_in by scattering every tap's einsum back into the padded
  gradient, d_w[ky, kx] = einsum of the tap's input window with d, d_bias = sum of d;
* ReLU, 2 x 2 average pooling, nearest 2x upsampling, channel concatenation
  and the mean squared error, each with its adjoint.

Architecture and the flat parameter layout are those of the C-ABI
(unet_params): for each convolution in the order (encoder level 0..L-1:
first, second), (decoder level L-2..0: up, first, second), (output 1x1),
the weights [ky][kx][c_in][c_out] then the bias [c_out].

Pinned in tests/test_unet_oracle.py by scipy's correlate2d (forward
convolution) and by central finite differences of the loss (every adjoint).
"""
from __future__ import annotations

import numpy as np


def conv_specs(levels: int, base: int, in_ch: int = 3, out_ch: int = 2):
    """(c_in, c_out, K) of every convolution, in parameter order."""
    c = [base << l for l in range(levels)]
    specs = []
    for l in range(levels):
        specs.append((in_ch if l == 0 else c[l - 1], c[l], 3))
        specs.append((c[l], c[l], 3))
    for l in range(levels - 2, -1, -1):
        specs.append((c[l + 1], c[l], 3))
        specs.append((2 * c[l], c[l], 3))
        specs.append((c[l], c[l], 3))
    specs.append((c[0], out_ch, 1))
    return specs


def num_params(levels: int, base: int) -> int:
    return sum(K * K * ci * co + co for ci, co, K in conv_specs(levels, base))


def unpack(theta: np.ndarray, levels: int, base: int):
    """List of (w [K, K, c_in, c_out], bias [c_out]) views of the flat vector."""
    out, off = [], 0
    for ci, co, K in conv_specs(levels, base):
        n = K * K * ci * co
        w = theta[off:off + n].reshape(K, K, ci, co)
        off += n
        b = theta[off:off + co]
        off += co
        out.append((w, b))
    assert off == theta.size
    return out


def conv(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    K = w.shape[0]
    R = K // 2
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (R, R), (R, R), (0, 0)))
    out = np.zeros((B, H, W, w.shape[3]))
    for ky in range(K):
        for kx in range(K):
            out += np.einsum("byxi,io->byxo", xp[:, ky:ky + H, kx:kx + W, :], w[ky, kx])
    return out + b


def conv_back(x: np.ndarray, w: np.ndarray, d: np.ndarray):
    """(d_x, d_w, d_b) of conv(x, w, b) for the output gradient d."""
    K = w.shape[0]
    R = K // 2
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (R, R), (R, R), (0, 0)))
    gp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(K):
        for kx in range(K):
            gp[:, ky:ky + H, kx:kx + W, :] += np.einsum("byxo,io->byxi", d, w[ky, kx])
            dw[ky, kx] = np.einsum("byxi,byxo->io", xp[:, ky:ky + H, kx:kx + W, :], d)
    return gp[:, R:R + H, R:R + W, :], dw, d.sum(axis=(0, 1, 2))


def relu(x):
    return np.maximum(x, 0.0)


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_back(d):
    return np.repeat(np.repeat(d, 2, axis=1), 2, axis=2) * 0.25


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_back(d):
    B, H, W, C = d.shape
    return d.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def forward(theta: np.ndarray, x: np.ndarray, levels: int, base: int, keep: bool = False):
    """Network output for images x [B, H, W, 3]; with keep, also the intermediates."""
    P = unpack(theta, levels, base)
    L = levels
    cache = {}
    h = x
    skips = []
    for l in range(L):
        inp = h
        a = relu(conv(inp, *P[2 * l]))
        e = relu(conv(a, *P[2 * l + 1]))
        cache[("enc", l)] = (inp, a, e)
        skips.append(e)
        h = pool(e) if l < L - 1 else e
    for l in range(L - 2, -1, -1):
        k = 2 * L + 3 * (L - 2 - l)
        u = up(h)
        uc = relu(conv(u, *P[k]))
        cat = np.concatenate([skips[l], uc], axis=3)
        da = relu(conv(cat, *P[k + 1]))
        db = relu(conv(da, *P[k + 2]))
        cache[("dec", l)] = (u, uc, cat, da, db)
        h = db
    y = conv(h, *P[-1])
    cache["top"] = h
    return (y, cache) if keep else y


def loss_and_grad(theta: np.ndarray, x: np.ndarray, target: np.ndarray, levels: int, base: int):
    """Mean squared error of the output against target and its gradient in theta."""
    P = unpack(theta, levels, base)
    L = levels
    y, cache = forward(theta, x, levels, base, keep=True)
    n = y.size
    loss = float(((y - target) ** 2).sum() / n)
    dy = 2.0 * (y - target) / n
    grads = [None] * len(P)
    dh, dw, db = conv_back(cache["top"], P[-1][0], dy)
    grads[-1] = (dw, db)
    dskip = [None] * L
    for l in range(0, L - 1):
        k = 2 * L + 3 * (L - 2 - l)
        u, uc, cat, da, db_ = cache[("dec", l)]
        g = dh * (db_ > 0)
        dda, dw, db = conv_back(da, P[k + 2][0], g)
        grads[k + 2] = (dw, db)
        g = dda * (da > 0)
        dcat, dw, db = conv_back(cat, P[k + 1][0], g)
        grads[k + 1] = (dw, db)
        c = cat.shape[3] // 2
        dskip[l] = dcat[..., :c]
        g = dcat[..., c:] * (uc > 0)
        du, dw, db = conv_back(u, P[k][0], g)
        grads[k] = (dw, db)
        dh = up_back(du)
    # dh: gradient of the bottom encoder output
    for l in range(L - 1, -1, -1):
        inp, a, e = cache[("enc", l)]
        ge = dh if l == L - 1 else dskip[l] + pool_back(dh)
        g = ge * (e > 0)
        da_, dw, db = conv_back(a, P[2 * l + 1][0], g)
        grads[2 * l + 1] = (dw, db)
        g = da_ * (a > 0)
        dinp, dw, db = conv_back(inp, P[2 * l][0], g)
        grads[2 * l] = (dw, db)
        dh = dinp
    flat = np.concatenate([np.concatenate([dw.ravel(), db.ravel()]) for dw, db in grads])
    return loss, flat


def init(levels: int, base: int, seed: int = 0) -> np.ndarray:
    """He-normal weights (numpy PCG64), small random biases, as a flat vector."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for ci, co, K in conv_specs(levels, base):
        parts.append(rng.standard_normal(K * K * ci * co) * np.sqrt(2.0 / (K * K * ci)))
        parts.append(0.05 * rng.standard_normal(co))
    return np.concatenate(parts)
