"""The double-float scheme of the complex128 paths, emulated in numpy float32.

The CUDA kernels carry complex128 values as float pairs (hi + lo) and form
sums of products with an exact product error (an FMA: a*b - fl(a*b)), the
cross terms, and a two-sum into the high word (Knuth; error to the low word).
This test pins the scheme itself, not the kernels (the GPU parity tests pin
those against the FP64 oracle): over sums of a few hundred complex products
of split FP64 numbers the relative error stays near 2^-46, far below FP64
parity's 1e-10 and far above FP32's 2^-24.  float32 products of float32
values are exact in float64 (48 significant bits), which gives the exact
FMA error term here.
"""
import numpy as np

f32 = np.float32


def split(x):
    """A double as a float pair: hi its nearest float, lo the nearest float of the rest."""
    hi = f32(x)
    return hi, f32(x - np.float64(hi))


def two_sum(a, b):
    s = f32(a + b)
    v = f32(s - a)
    return s, f32(f32(a - f32(s - v)) + f32(b - v))


def mac(sh, sl, ah, al, bh, bl):
    """(sh, sl) += (ah + al)(bh + bl) as in the kernels' df_mac."""
    p = f32(ah * bh)
    e = f32(np.float64(ah) * np.float64(bh) - np.float64(p))  # fma(ah, bh, -p): exact
    e = f32(np.float64(ah) * np.float64(bl) + np.float64(e))  # fma(ah, bl, e)
    e = f32(np.float64(al) * np.float64(bh) + np.float64(e))  # fma(al, bh, e)
    t, err = two_sum(sh, p)
    return t, f32(sl + f32(err + e))


def cdot(m, x):
    """sum_k m_k x_k for complex128 vectors, in float pairs (two accumulators per part)."""
    rh = rl = ih = il = f32(0.0)
    for a, b in zip(m, x):
        arh, arl = split(a.real)
        aih, ail = split(a.imag)
        brh, brl = split(b.real)
        bih, bil = split(b.imag)
        rh, rl = mac(rh, rl, arh, arl, brh, brl)
        rh, rl = mac(rh, rl, -aih, -ail, bih, bil)
        ih, il = mac(ih, il, arh, arl, bih, bil)
        ih, il = mac(ih, il, aih, ail, brh, brl)
    return complex(np.float64(rh) + np.float64(rl), np.float64(ih) + np.float64(il))


def test_double_float_dot_products_keep_about_48_bits():
    rng = np.random.default_rng(3)
    worst = 0.0
    for n in (16, 64, 256):
        for _ in range(6):
            m = rng.standard_normal(n) + 1j * rng.standard_normal(n)
            x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
            got = cdot(m, x)
            # reference: the exact sum of the split inputs' products, evaluated in long
            # double where available and otherwise in double (both far beyond 2^-46 here)
            ref = np.sum(m.astype(np.clongdouble) * x.astype(np.clongdouble))
            scale = np.sum(np.abs(m) * np.abs(x))
            worst = max(worst, float(abs(got - complex(ref)) / scale))
    assert worst < 2.0 ** -44, worst
    assert worst < 1e-12  # the FP64 parity bound is 1e-10


def test_single_float_accumulation_would_not_do():
    """The same sums in plain float32 lose ~1e-7: why the low word is carried."""
    rng = np.random.default_rng(4)
    m = rng.standard_normal(256) + 1j * rng.standard_normal(256)
    x = rng.standard_normal(256) + 1j * rng.standard_normal(256)
    plain = np.sum(m.astype(np.complex64) * x.astype(np.complex64))
    ref = np.sum(m * x)
    assert abs(plain - ref) / np.sum(np.abs(m) * np.abs(x)) > 1e-9
    assert abs(cdot(m, x) - ref) / np.sum(np.abs(m) * np.abs(x)) < 1e-13
