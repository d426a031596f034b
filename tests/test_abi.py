"""C-ABI library: loads, exports what include/dafmm.h declares, host-side
tree logic and argument checking (CPU only; no compute call needs a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2204_00326_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pkg.build()
from paper_2204_00326_gb300 import native as N  # noqa: E402
from paper_2204_00326_gb300 import workloads as W  # noqa: E402


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*int\s+(\w+)\s*\(", txt, flags=re.M)
    return names


def test_every_declared_symbol_is_exported_and_bound():
    names = _declared()
    assert "dafmm_matvec" in names and "build_tree" in names and "build_nca_operators" in names
    lib = ctypes.CDLL(N.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
        assert n in N.EXPORTS, n


def _tree(n_side, kappa, **kw):
    return N.build_tree(N.make_params(kappa, **kw), n_side)


def test_regimes_and_cones_of_the_grid128_workload():
    t = _tree(128, 40.0)
    info = N.tree_info(t)
    assert info.N == 16384 and info.levels == 6
    # kappa w = 40, 20, 10, 5, 2.5, 1.25 at levels 0..5; HF iff (kappa w)^2 > 16
    assert [info.hf[k] for k in range(6)] == [1, 1, 1, 1, 0, 0]
    # 2 pi kappa w = 31.4 at level 3 -> 32 cones, doubling upwards
    assert [info.cones[k] for k in range(4)] == [256, 128, 64, 32]
    assert info.top == 3
    assert info.il_pairs[5] > 0 and info.il_pairs[4] > 0 and info.il_pairs[3] > 0
    N.tree_destroy(t)


@pytest.mark.parametrize("n_side,kappa", [(4, 3.0), (8, 8.0), (16, 8.0), (32, 8.0), (64, 20.0), (128, 40.0), (64, 40.0)])
def test_near_plus_interaction_lists_cover_each_pair_once(n_side, kappa):
    t = _tree(n_side, kappa)
    assert N.tree_check(t) == 0
    N.tree_destroy(t)


def test_nodes_follow_the_documented_order():
    t = _tree(8, 2.0)
    xy = N.tree_nodes(t, 64)
    z = -np.cos((2 * np.arange(4) + 1) * np.pi / 8)
    beta = 0.5
    # leaf 1 in Morton order is (bx, by) = (1, 0); node i' = k1 + 4 k2
    assert np.allclose(xy[16 + 1 + 4 * 2], [-1 + 3 * beta + beta * z[1], -1 + beta + beta * z[2]])
    assert np.allclose(xy[2 * 16], [-1 + beta + beta * z[0], -1 + 3 * beta + beta * z[0]])
    N.tree_destroy(t)


@pytest.mark.parametrize("kw,n_side,msg", [
    (dict(p=5), 20, "p = 4"),
    (dict(), 24, "power of two"),
    (dict(), 6, "multiple of p"),
    (dict(eps_nca=0.0), 16, "eps_nca"),
    (dict(T=-1.0), 16, "T must"),
])
def test_bad_arguments_are_rejected(kw, n_side, msg):
    with pytest.raises(N.DafmmError) as e:
        _tree(n_side, 4.0, **kw)
    assert e.value.code == N.DAFMM_EBADARG and msg in str(e.value)


def test_high_frequency_leaves_are_rejected():
    with pytest.raises(N.DafmmError) as e:
        _tree(16, 40.0)  # leaf kappa w = 10
    assert "high-frequency" in str(e.value)


def test_null_and_device_errors_are_status_codes():
    lib = N.lib
    assert lib.build_tree(None, 16, -1.0, 1.0, None) == N.DAFMM_EBADARG
    assert lib.dafmm_matvec(None, 1, None, None, 0, None) == N.DAFMM_EBADARG
    assert lib.dafmm_potential(None, 1, None, None, 0, None) == N.DAFMM_EBADARG
    assert lib.hodlr_sync(None, None) == N.DAFMM_EBADARG
    assert lib.hodlr_set_ctas(None, 0) == N.DAFMM_EBADARG
    assert lib.hodlr_debug_stall(None) == N.DAFMM_EBADARG
    assert lib.hodlr_solve(None, 1, None, None, 0, None) == N.DAFMM_EBADARG
    assert lib.gmres_solve(None, None, 1, None, None, None, None, None) == N.DAFMM_EBADARG
    assert lib.dafmm_set_batched_kernel(None, 0) == N.DAFMM_EBADARG
    assert lib.dafmm_debug_leaf_staging(None, 1) == N.DAFMM_EBADARG
    buf = ctypes.create_string_buffer(256)
    assert lib.dafmm_last_error(buf, 256) == N.DAFMM_EBADARG
    assert b"NULL" in buf.value
    import torch

    if not torch.cuda.is_available():
        t = _tree(16, 8.0)
        h = ctypes.c_void_p()
        q = np.zeros(256)
        st = lib.build_nca_operators(t, q.ctypes.data, None, ctypes.byref(h))
        assert st == N.DAFMM_ECUDA
        N.tree_destroy(t)
