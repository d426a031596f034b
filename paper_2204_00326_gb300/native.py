"""ctypes binding of the C-ABI in ``include/dafmm.h`` (argument marshalling only).

Every function has the name of the C entry point it wraps.  Device arrays are
torch CUDA tensors (complex128 vectors, float64 contrast); streams are torch
CUDA streams.  A nonzero status raises :class:`DafmmError` with the library's
message.  There is no fallback: if ``libdafmm.so`` cannot be loaded the import
of this module fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdafmm.so")

DAFMM_OK = 0
DAFMM_EBADARG = 1
DAFMM_ENOMEM = 2
DAFMM_ENOTCONV = 3
DAFMM_EBREAKDOWN = 4
DAFMM_ETIMEOUT = 5
DAFMM_ECUDA = 6
DAFMM_PREC_RIGHT = 0
DAFMM_PREC_LEFT = 1
DAFMM_FP64 = 0
DAFMM_MIXED = 1

_NAMES = {0: "OK", 1: "EBADARG", 2: "ENOMEM", 3: "ENOTCONV", 4: "EBREAKDOWN", 5: "ETIMEOUT", 6: "ECUDA"}


class DafmmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"DAFMM_{_NAMES.get(code, code)}: {msg}")
        self.code = code


class dafmm_params(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_int),
        ("kappa", ctypes.c_double),
        ("T", ctypes.c_double),
        ("eps_nca", ctypes.c_double),
        ("max_rank", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("reserved", ctypes.c_int * 6),
    ]


class dafmm_tuning(ctypes.Structure):
    _fields_ = [
        ("nrhs", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("best_ms", ctypes.c_double),
        ("ncand", ctypes.c_int),
        ("cand_kernel", ctypes.c_int * 16),
        ("cand_ctas", ctypes.c_int * 16),
        ("cand_ms", ctypes.c_double * 16),
        ("reserved", ctypes.c_int * 8),
    ]


class dafmm_tree_info(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_long),
        ("n_side", ctypes.c_int),
        ("levels", ctypes.c_int),
        ("top", ctypes.c_int),
        ("hf", ctypes.c_int * 32),
        ("cones", ctypes.c_int * 32),
        ("il_pairs", ctypes.c_long * 32),
    ]


class dafmm_stats_t(ctypes.Structure):
    _fields_ = [
        ("rank_in_max", ctypes.c_int * 32),
        ("rank_out_max", ctypes.c_int * 32),
        ("rank_in_mean", ctypes.c_double * 32),
        ("rank_out_mean", ctypes.c_double * 32),
        ("slots", ctypes.c_long * 32),
        ("operator_bytes_fp64", ctypes.c_double),
        ("operator_bytes_fp32", ctypes.c_double),
        ("vector_bytes_per_rhs", ctypes.c_double),
        ("cmacs_per_rhs", ctypes.c_double),
        ("setup_seconds_table", ctypes.c_double),
        ("setup_seconds_nca", ctypes.c_double),
        ("p2p_cmacs_per_rhs", ctypes.c_long),
        ("cmacs_up", ctypes.c_double),
        ("cmacs_m2l", ctypes.c_double),
        ("cmacs_down", ctypes.c_double),
        ("cmacs_leaf", ctypes.c_double),
        ("coef_bytes_per_rhs", ctypes.c_double),
        ("launches_per_call", ctypes.c_int),
        ("launches_per_call_fp64", ctypes.c_int),
        ("cmacs_far_fused", ctypes.c_double),
        ("cmacs_leaf_fused", ctypes.c_double),
    ]


class dafmm_profile_t(ctypes.Structure):
    _fields_ = [
        ("calls", ctypes.c_long),
        ("ms_total", ctypes.c_double),
        ("ms_up", ctypes.c_double),
        ("ms_m2l", ctypes.c_double),
        ("ms_down", ctypes.c_double),
        ("ms_leaf", ctypes.c_double),
        ("ms_far", ctypes.c_double),
    ]


class gmres_opts(ctypes.Structure):
    _fields_ = [
        ("restart", ctypes.c_int),
        ("max_iters", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
        ("history", ctypes.POINTER(ctypes.c_double)),
        ("history_len", ctypes.c_int),
        ("side", ctypes.c_int),
        ("reserved", ctypes.c_int * 5),
    ]


class gmres_stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("outer_iterations", ctypes.c_int),
        ("matvecs", ctypes.c_int),
        ("precond_applies", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("rel_residual", ctypes.c_double),
        ("seconds", ctypes.c_double),
    ]


class unet_params(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int),
        ("base", ctypes.c_int),
        ("in_ch", ctypes.c_int),
        ("out_ch", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("reserved", ctypes.c_int * 8),
    ]


class learned_stats(ctypes.Structure):
    _fields_ = [
        ("guess_used", ctypes.c_int),
        ("guess_residual", ctypes.c_double),
        ("corrections", ctypes.c_int),
    ]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2204_00326_gb300.build()")
lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_sig = {
    "dafmm_last_error": ([ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
    "build_tree": ([ctypes.POINTER(dafmm_params), ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_P)], ctypes.c_int),
    "tree_nodes": ([_P, _P], ctypes.c_int),
    "tree_info": ([_P, ctypes.POINTER(dafmm_tree_info)], ctypes.c_int),
    "tree_check": ([_P, ctypes.POINTER(ctypes.c_long)], ctypes.c_int),
    "tree_destroy": ([_P], ctypes.c_int),
    "build_nca_operators": ([_P, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "dafmm_matvec": ([_P, ctypes.c_int, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "dafmm_matvec_noalloc": ([_P, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "dafmm_set_batched_kernel": ([_P, ctypes.c_int], ctypes.c_int),
    "dafmm_nbody_direct": ([_P, _P, _P, _P], ctypes.c_int),
    "tree_nodes_dev": ([_P, _P, _P], ctypes.c_int),
    "dafmm_field_eval": ([_P, _P, ctypes.c_long, _P, _P, _P, _P], ctypes.c_int),
    "dafmm_tune_batched": ([_P, ctypes.c_int, ctypes.c_int, _P], ctypes.c_int),
    "dafmm_set_batched_grid": ([_P, ctypes.c_int], ctypes.c_int),
    "dafmm_batch_create": ([ctypes.c_int, _P, _P], ctypes.c_int),
    "dafmm_batch_matvec": ([_P, ctypes.c_int, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "dafmm_batch_destroy": ([_P], ctypes.c_int),
    "dafmm_sync": ([_P, _P], ctypes.c_int),
    "dafmm_debug_stall": ([_P, ctypes.c_int], ctypes.c_int),
    "dafmm_debug_leaf_staging": ([_P, ctypes.c_int], ctypes.c_int),
    "dafmm_potential": ([_P, ctypes.c_int, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "dafmm_set_contrast": ([_P, _P, _P], ctypes.c_int),
    "gmres_solve": ([_P, _P, ctypes.c_int, _P, _P, ctypes.POINTER(gmres_opts), ctypes.POINTER(gmres_stats), _P], ctypes.c_int),
    "hodlr_factor": ([_P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
    "hodlr_solve": ([_P, ctypes.c_int, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "hodlr_sync": ([_P, _P], ctypes.c_int),
    "hodlr_debug_stall": ([_P], ctypes.c_int),
    "hodlr_set_ctas": ([_P, ctypes.c_int], ctypes.c_int),
    "hodlr_export": ([_P, _P], ctypes.c_int),
    "hodlr_info": ([_P, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "hodlr_destroy": ([_P], ctypes.c_int),
    "dafmm_stats": ([_P, ctypes.POINTER(dafmm_stats_t)], ctypes.c_int),
    "dafmm_entries": ([_P, ctypes.c_long, _P, ctypes.c_long, _P, _P], ctypes.c_int),
    "dafmm_profile": ([_P, ctypes.c_int], ctypes.c_int),
    "dafmm_profile_read": ([_P, ctypes.POINTER(dafmm_profile_t)], ctypes.c_int),
    "ops_destroy": ([_P], ctypes.c_int),
    "unet_create": ([ctypes.POINTER(unet_params), ctypes.POINTER(_P)], ctypes.c_int),
    "unet_destroy": ([_P], ctypes.c_int),
    "unet_num_params": ([_P, ctypes.POINTER(ctypes.c_long)], ctypes.c_int),
    "unet_get_params": ([_P, _P], ctypes.c_int),
    "unet_set_params": ([_P, _P], ctypes.c_int),
    "unet_forward": ([_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P], ctypes.c_int),
    "unet_backward": ([_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "unet_get_grads": ([_P, _P], ctypes.c_int),
    "unet_adam": ([_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P], ctypes.c_int),
    "unet_guess": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "gmres_solve_learned": ([_P, _P, _P, ctypes.c_int, ctypes.c_double, _P, _P, ctypes.POINTER(gmres_opts),
                             ctypes.POINTER(gmres_stats), ctypes.POINTER(learned_stats), _P], ctypes.c_int),
}
EXPORTS = tuple(_sig)
for _name, (_args, _res) in _sig.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def _check(st: int):
    if st != DAFMM_OK:
        buf = ctypes.create_string_buffer(1024)
        lib.dafmm_last_error(buf, 1024)
        raise DafmmError(st, buf.value.decode(errors="replace"))


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dptr(t, dtype_name: str) -> int:
    import torch

    if not t.is_cuda:
        raise ValueError(f"expected a CUDA tensor of {dtype_name}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    want = {"complex128": torch.complex128, "float64": torch.float64, "float32": torch.float32}[dtype_name]
    if t.dtype != want:
        raise ValueError(f"expected dtype {want}, got {t.dtype}")
    return int(t.data_ptr())


DAFMM_KERNEL_LS, DAFMM_KERNEL_POINTS = 0, 1


def make_params(kappa: float, eps_nca: float = 1e-12, T: float = 16.0, p: int = 4, max_rank: int = 0,
                kernel: int = DAFMM_KERNEL_LS) -> dafmm_params:
    prm = dafmm_params()
    prm.p = p
    prm.kappa = kappa
    prm.T = T
    prm.eps_nca = eps_nca
    prm.max_rank = max_rank
    prm.kernel = kernel
    return prm


def build_tree(params: dafmm_params, n_side: int, x0: float = -1.0, x1: float = 1.0) -> int:
    h = _P()
    _check(lib.build_tree(ctypes.byref(params), n_side, x0, x1, ctypes.byref(h)))
    return h.value


def tree_nodes_dev(tree: int, xy, stream=None) -> None:
    """Node coordinates into a (N, 2) float64 CUDA tensor."""
    _check(lib.tree_nodes_dev(tree, _dptr(xy, "float64"), _stream_ptr(stream)))


def tree_nodes(tree: int, N: int) -> np.ndarray:
    xy = np.zeros((N, 2))
    _check(lib.tree_nodes(tree, xy.ctypes.data))
    return xy


def tree_info(tree: int) -> dafmm_tree_info:
    info = dafmm_tree_info()
    _check(lib.tree_info(tree, ctypes.byref(info)))
    return info


def tree_check(tree: int) -> int:
    bad = ctypes.c_long()
    _check(lib.tree_check(tree, ctypes.byref(bad)))
    return bad.value


def tree_destroy(tree: int) -> None:
    _check(lib.tree_destroy(tree))


def build_nca_operators(tree: int, q, stream=None) -> int:
    h = _P()
    _check(lib.build_nca_operators(tree, _dptr(q, "float64"), _stream_ptr(stream), ctypes.byref(h)))
    return h.value


def dafmm_matvec(ops: int, v, out, precision: int = DAFMM_FP64, stream=None) -> None:
    nrhs = 1 if v.dim() == 1 else v.shape[1]
    if out.shape != v.shape:
        raise ValueError("v and out must have the same shape")
    _check(lib.dafmm_matvec(ops, nrhs, _dptr(v, "complex128"), _dptr(out, "complex128"), precision, _stream_ptr(stream)))


def dafmm_potential(ops: int, v, out, precision: int = DAFMM_FP64, stream=None) -> None:
    """out = K v: the volume potential at the nodes (the scattered field from psi)."""
    nrhs = 1 if v.dim() == 1 else v.shape[1]
    if out.shape != v.shape:
        raise ValueError("v and out must have the same shape")
    _check(lib.dafmm_potential(ops, nrhs, _dptr(v, "complex128"), _dptr(out, "complex128"), precision, _stream_ptr(stream)))


NOALLOC_SCRATCH_BYTES = 32 << 20


def dafmm_matvec_noalloc(ops: int, v, out, precision: int = DAFMM_FP64, stream=None) -> None:
    """dafmm_matvec for one right-hand side with the library's static scratch
    (for callers that cannot allocate device memory at call time)."""
    if v.dim() != 1 or out.shape != v.shape:
        raise ValueError("one right-hand side: v and out are (N,) vectors")
    _check(lib.dafmm_matvec_noalloc(ops, _dptr(v, "complex128"), _dptr(out, "complex128"), precision, _stream_ptr(stream)))


def dafmm_field_eval(ops: int, psi, pts, want_psi: bool = True, stream=None):
    """(u, psi_at): the volume potential V[psi](x) and the interpolant psi(x)
    (Eq. 7) at the points pts ((m, 2) float64 CUDA tensor)."""
    import torch

    if pts.dim() != 2 or pts.shape[1] != 2:
        raise ValueError("pts is an (m, 2) tensor")
    m = pts.shape[0]
    u = torch.empty(m, dtype=torch.complex128, device=pts.device)
    pa = torch.empty_like(u) if want_psi else None
    _check(lib.dafmm_field_eval(ops, _dptr(psi, "complex128"), m, _dptr(pts.contiguous(), "float64"), _dptr(u, "complex128"),
                                _dptr(pa, "complex128") if pa is not None else None, _stream_ptr(stream)))
    return u, pa


def dafmm_nbody_direct(tree: int, v, out, stream=None) -> None:
    """u_i = sum_{j != i} G(x_i, x_j) v_j by direct summation on the device."""
    if v.dim() != 1 or out.shape != v.shape:
        raise ValueError("v and out are (N,) vectors")
    _check(lib.dafmm_nbody_direct(tree, _dptr(v, "complex128"), _dptr(out, "complex128"), _stream_ptr(stream)))


def dafmm_tune_batched(ops: int, nrhs: int, precision: int) -> dict:
    """Time the several-right-hand-side pass configurations, keep the fastest;
    returns the choice and every candidate's time (ms per application)."""
    r = dafmm_tuning()
    _check(lib.dafmm_tune_batched(ops, int(nrhs), int(precision), ctypes.byref(r)))
    kinds = {1: "cuda_cores", 2: "tensor_cores"}
    return {"nrhs": r.nrhs, "precision": "fp64" if r.precision == DAFMM_FP64 else "mixed", "kernel": kinds[r.kernel],
            "ctas_per_sm": r.ctas_per_sm, "best_ms": r.best_ms,
            "candidates": [{"kernel": kinds[r.cand_kernel[k]], "ctas_per_sm": r.cand_ctas[k], "ms": r.cand_ms[k]} for k in range(r.ncand)]}


def dafmm_set_batched_grid(ops: int, ctas_per_sm: int) -> None:
    _check(lib.dafmm_set_batched_grid(ops, int(ctas_per_sm)))


class Batch:
    """Several operators applied together in one captured CUDA graph
    (dafmm_batch_create / dafmm_batch_matvec)."""

    def __init__(self, ops_handles):
        self.n = len(ops_handles)
        arr = (_P * self.n)(*ops_handles)
        h = _P()
        _check(lib.dafmm_batch_create(self.n, arr, ctypes.byref(h)))
        self.h = h.value

    def matvec(self, vs, outs, precision: int = DAFMM_FP64, stream=None) -> None:
        if len(vs) != self.n or len(outs) != self.n:
            raise ValueError("one input and one output per problem")
        nrhs = 1 if vs[0].dim() == 1 else vs[0].shape[1]
        for v, o in zip(vs, outs):
            if o.shape != v.shape or (1 if v.dim() == 1 else v.shape[1]) != nrhs:
                raise ValueError("every problem takes the same number of right-hand sides")
        va = (_P * self.n)(*[_dptr(v, "complex128") for v in vs])
        oa = (_P * self.n)(*[_dptr(o, "complex128") for o in outs])
        _check(lib.dafmm_batch_matvec(self.h, nrhs, va, oa, precision, _stream_ptr(stream)))

    def close(self) -> None:
        if getattr(self, "h", None):
            lib.dafmm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


BATCHED_AUTO, BATCHED_CUDA_CORES, BATCHED_TENSOR_CORES = 0, 1, 2


def dafmm_set_batched_kernel(ops: int, mode: int) -> None:
    """Kernel of the complex64 tree passes with several right-hand sides:
    0 automatic, 1 CUDA cores, 2 tensor cores (tcgen05, split tf32)."""
    _check(lib.dafmm_set_batched_kernel(ops, int(mode)))


def dafmm_sync(ops: int, stream=None) -> None:
    """Synchronise and raise DafmmError(DAFMM_ETIMEOUT) if a device wait gave up."""
    _check(lib.dafmm_sync(ops, _stream_ptr(stream)))


def dafmm_set_contrast(ops: int, q, stream=None) -> None:
    """Replace the operator's contrast (N float64 on the device)."""
    _check(lib.dafmm_set_contrast(ops, _dptr(q, "float64"), _stream_ptr(stream)))


def dafmm_debug_stall(ops: int, pass_index: int) -> None:
    """Test support: the next single-RHS application waits for a row of tree
    pass `pass_index` that is never written (bounded), so dafmm_sync reports
    DAFMM_ETIMEOUT.  -1 cancels."""
    _check(lib.dafmm_debug_stall(ops, int(pass_index)))


def dafmm_debug_leaf_staging(ops: int, enable: bool) -> None:
    """Test support: the leaf kernel's far-field blocks staged in shared
    memory (True, the planned path) or read from global memory (False)."""
    _check(lib.dafmm_debug_leaf_staging(ops, 1 if enable else 0))


def dafmm_stats(ops: int) -> dafmm_stats_t:
    st = dafmm_stats_t()
    _check(lib.dafmm_stats(ops, ctypes.byref(st)))
    return st


def dafmm_entries(ops: int, rows, cols) -> np.ndarray:
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    cols = np.ascontiguousarray(np.asarray(cols, dtype=np.int64))
    out = np.zeros((len(rows), len(cols), 2))
    _check(lib.dafmm_entries(ops, len(rows), rows.ctypes.data, len(cols), cols.ctypes.data, out.ctypes.data))
    return out[..., 0] + 1j * out[..., 1]


def dafmm_profile(ops: int, enable: bool) -> None:
    _check(lib.dafmm_profile(ops, 1 if enable else 0))


def dafmm_profile_read(ops: int) -> dafmm_profile_t:
    p = dafmm_profile_t()
    _check(lib.dafmm_profile_read(ops, ctypes.byref(p)))
    return p


def gmres_solve(ops: int, f, x, tol: float = 1e-8, precision: int = DAFMM_FP64, restart: int = 50, max_iters: int = 1000,
                inner_tol: float = 1e-5, M: int | None = None, stream=None, history_len: int = 0, side: int = 0):
    """Solve A x = f (x holds the initial guess on entry).  Returns (status, stats, history).

    f and x are (N,) or (N, nrhs) complex128 (nrhs <= 64, right-hand side
    fastest); with several right-hand sides the columns are solved together
    (one batched application per step) and stats is a list of nrhs entries.
    side: DAFMM_PREC_RIGHT (0) or DAFMM_PREC_LEFT (1) preconditioning by M.
    status is DAFMM_OK or DAFMM_ENOTCONV (not converged within max_iters); other
    failures raise DafmmError.
    """
    nrhs = 1 if f.dim() == 1 else f.shape[1]
    if x.shape != f.shape:
        raise ValueError("f and x must have the same shape")
    o = gmres_opts()
    o.side = side
    o.restart = restart
    o.max_iters = max_iters
    o.tol = tol
    o.precision = precision
    o.inner_tol = inner_tol
    hist = None
    if history_len > 0:
        hist = (ctypes.c_double * history_len)()
        o.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
        o.history_len = history_len
    sts = (gmres_stats * nrhs)()
    rc = lib.gmres_solve(ops, M, nrhs, _dptr(f, "complex128"), _dptr(x, "complex128"), ctypes.byref(o), sts, _stream_ptr(stream))
    if rc not in (DAFMM_OK, DAFMM_ENOTCONV):
        _check(rc)
    n_hist = max(s.iterations + s.outer_iterations + 1 for s in sts)
    h = list(hist)[: min(history_len, n_hist)] if hist is not None else None
    return rc, (sts[0] if nrhs == 1 else list(sts)), h


def hodlr_factor(ops: int, rank: int = 15, tol: float = 0.0, leaf_size: int = 64) -> int:
    h = _P()
    _check(lib.hodlr_factor(ops, rank, tol, leaf_size, ctypes.byref(h)))
    return h.value


def hodlr_solve(M: int, b, x, precision: int = DAFMM_FP64, stream=None) -> None:
    """x = A~^{-1} b for (N,) or (N, nrhs) complex128 (nrhs <= 64, right-hand side fastest)."""
    nrhs = 1 if b.dim() == 1 else b.shape[1]
    if x.shape != b.shape:
        raise ValueError("b and x must have the same shape")
    _check(lib.hodlr_solve(M, nrhs, _dptr(b, "complex128"), _dptr(x, "complex128"), precision, _stream_ptr(stream)))


def hodlr_sync(M: int, stream=None) -> None:
    """Synchronise; raises DafmmError (DAFMM_ETIMEOUT) if an application gave up a wait."""
    _check(lib.hodlr_sync(M, _stream_ptr(stream)))


def hodlr_debug_stall(M: int) -> None:
    _check(lib.hodlr_debug_stall(M))


def hodlr_set_ctas(M: int, ctas: int) -> None:
    _check(lib.hodlr_set_ctas(M, int(ctas)))


def hodlr_export(M: int, N: int) -> np.ndarray:
    out = np.zeros((N, N, 2))
    _check(lib.hodlr_export(M, out.ctypes.data))
    return out[..., 0] + 1j * out[..., 1]


def hodlr_info(M: int) -> dict:
    N, lv, lf, rk, sec = ctypes.c_long(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib.hodlr_info(M, ctypes.byref(N), ctypes.byref(lv), ctypes.byref(lf), ctypes.byref(rk), ctypes.byref(sec)))
    return {"N": N.value, "levels": lv.value, "leaf_size": lf.value, "rank_max": rk.value, "factor_seconds": sec.value}


def hodlr_destroy(M: int) -> None:
    _check(lib.hodlr_destroy(M))


def ops_destroy(ops: int) -> None:
    _check(lib.ops_destroy(ops))


# --- learned guess ---------------------------------------------------------
def unet_create(levels: int = 4, base: int = 32, seed: int = 0) -> int:
    p = unet_params()
    p.levels = levels
    p.base = base
    p.in_ch = 3
    p.out_ch = 2
    p.seed = seed
    h = _P()
    _check(lib.unet_create(ctypes.byref(p), ctypes.byref(h)))
    return h.value


def unet_destroy(net: int) -> None:
    _check(lib.unet_destroy(net))


def unet_num_params(net: int) -> int:
    n = ctypes.c_long()
    _check(lib.unet_num_params(net, ctypes.byref(n)))
    return n.value


def unet_get_params(net: int) -> np.ndarray:
    a = np.zeros(unet_num_params(net), np.float32)
    _check(lib.unet_get_params(net, a.ctypes.data))
    return a


def unet_set_params(net: int, params: np.ndarray) -> None:
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != unet_num_params(net):
        raise ValueError("wrong number of parameters")
    _check(lib.unet_set_params(net, a.ctypes.data))


def unet_forward(net: int, x, out=None, stream=None):
    """x: [batch, height, width, 3] float32 CUDA tensor; returns [batch, height, width, 2]."""
    import torch

    b, h, w, _ = x.shape
    if out is None:
        out = torch.empty((b, h, w, 2), dtype=torch.float32, device=x.device)
    _check(lib.unet_forward(net, b, h, w, _dptr(x, "float32"), _dptr(out, "float32"), _stream_ptr(stream)))
    return out


def unet_backward(net: int, x, target, out=None, stream=None):
    """Forward, mean squared error against target, parameter gradients. Returns (loss, out)."""
    import torch

    b, h, w, _ = x.shape
    if out is None:
        out = torch.empty((b, h, w, 2), dtype=torch.float32, device=x.device)
    loss = ctypes.c_double()
    _check(lib.unet_backward(net, b, h, w, _dptr(x, "float32"), _dptr(target, "float32"), _dptr(out, "float32"),
                             ctypes.byref(loss), _stream_ptr(stream)))
    return loss.value, out


def unet_get_grads(net: int) -> np.ndarray:
    a = np.zeros(unet_num_params(net), np.float32)
    _check(lib.unet_get_grads(net, a.ctypes.data))
    return a


def unet_adam(net: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None) -> None:
    _check(lib.unet_adam(net, lr, beta1, beta2, eps, _stream_ptr(stream)))


def unet_guess(net: int, ops: int, f, x, stream=None) -> None:
    _check(lib.unet_guess(net, ops, _dptr(f, "complex128"), _dptr(x, "complex128"), _stream_ptr(stream)))


def gmres_solve_learned(ops: int, net: int, f, x, flags: int = 1, alpha: float = 1.0, tol: float = 1e-8,
                        precision: int = DAFMM_FP64, restart: int = 50, max_iters: int = 1000, inner_tol: float = 1e-5,
                        M: int | None = None, stream=None):
    """gmres_solve with the network's initial guess (flags bit 0) and/or coarse
    correction (bit 1).  Returns (status, gmres_stats, learned_stats)."""
    o = gmres_opts()
    o.restart = restart
    o.max_iters = max_iters
    o.tol = tol
    o.precision = precision
    o.inner_tol = inner_tol
    st = gmres_stats()
    ls = learned_stats()
    rc = lib.gmres_solve_learned(ops, M, net, flags, alpha, _dptr(f, "complex128"), _dptr(x, "complex128"), ctypes.byref(o),
                                 ctypes.byref(st), ctypes.byref(ls), _stream_ptr(stream))
    if rc not in (DAFMM_OK, DAFMM_ENOTCONV):
        _check(rc)
    return rc, st, ls

