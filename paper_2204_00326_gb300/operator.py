"""Owner of a tree + NCA operator pair built through the C-ABI."""
from __future__ import annotations

import numpy as np
import torch

from . import native as N


class DafmmOperator:
    """A = I + kappa^2 diag(q) K on a uniform n_side x n_side grid (Eq. 12a-13).

    ``contrast`` is either an array of q at the nodes or a callable taking the
    (N, 2) node coordinates.  Setup runs build_tree and build_nca_operators;
    :meth:`matvec` calls dafmm_matvec on torch CUDA tensors.
    """

    def __init__(self, n_side: int, kappa: float, contrast, eps_nca: float = 1e-12, T: float = 16.0,
                 x0: float = -1.0, x1: float = 1.0, stream=None, kernel: int = N.DAFMM_KERNEL_LS):
        self.n_side = n_side
        self.kappa = kappa
        self.N = n_side * n_side
        self.params = N.make_params(kappa, eps_nca=eps_nca, T=T, kernel=kernel)
        self.tree = N.build_tree(self.params, n_side, x0, x1)
        self.ops = None
        self.xy = N.tree_nodes(self.tree, self.N)
        q = contrast(self.xy) if callable(contrast) else np.asarray(contrast, dtype=np.float64)
        self.q = np.ascontiguousarray(q, dtype=np.float64)
        q_dev = torch.as_tensor(self.q, device="cuda")
        self.ops = N.build_nca_operators(self.tree, q_dev, stream)

    def potential(self, v: torch.Tensor, out: torch.Tensor | None = None, precision: int = N.DAFMM_FP64, stream=None):
        """K v: the volume potential (or, with the point kernel, the N-body potential)."""
        if out is None:
            out = torch.empty_like(v)
        N.dafmm_potential(self.ops, v, out, precision, stream)
        return out

    def matvec(self, v: torch.Tensor, out: torch.Tensor | None = None, precision: int = N.DAFMM_FP64, stream=None):
        if out is None:
            out = torch.empty_like(v)
        N.dafmm_matvec(self.ops, v, out, precision, stream)
        return out

    def sync(self, stream=None):
        N.dafmm_sync(self.ops, stream)

    def stats(self):
        return N.dafmm_stats(self.ops)

    def info(self):
        return N.tree_info(self.tree)

    def entries(self, rows, cols):
        return N.dafmm_entries(self.ops, rows, cols)

    def close(self):
        if getattr(self, "ops", None):
            N.ops_destroy(self.ops)
            self.ops = None
        if getattr(self, "tree", None):
            N.tree_destroy(self.tree)
            self.tree = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
