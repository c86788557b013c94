"""Tensor-train form of a HOBO tensor (Sec. VI) and its contraction.

``tt_svd`` decomposes a dense tensor by successive SVDs on the host (the
decomposition of Sec. VI, here swept from the last index to the first);
``TensorTrain`` holds the cores on the GPU and contracts them with batches
of states in the library's kernel (hobo_tt_energy).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .binding import _check, _ptr, _stream, load_library


def tt_svd(T: np.ndarray, rel_tol: float = 1e-10, max_rank: int = 256) -> list:
    """Cores G_c [r_{c-1}, n_c, r_c] of a dense tensor by successive SVDs
    (Sec. VI), taken from the last index to the first: the part of the
    tensor not yet split off, reshaped to (n_1...n_{c-1}) x (n_c r_c), is
    factored as U S V*; V* (singular values above rel_tol * the largest, at
    most max_rank of them) becomes core c and U S is carried to the left.
    Without truncation the ranks are those of the tensor's unfoldings, the
    same as a first-to-last sweep gives."""
    T = np.asarray(T, dtype=np.float64)
    d, n = T.ndim, T.shape
    cores = [None] * d
    r_right = 1
    left = T.reshape(-1, n[d - 1])
    for c in range(d - 1, 0, -1):
        left = left.reshape(-1, n[c] * r_right)
        U, s, Vt = np.linalg.svd(left, full_matrices=False)
        keep = 1 if not s.size or s[0] == 0 else int(np.count_nonzero(s > rel_tol * s[0]))
        keep = max(1, min(keep, max_rank))
        cores[c] = Vt[:keep].reshape(keep, n[c], r_right)
        left = U[:, :keep] * s[:keep]
        r_right = keep
    cores[0] = left.reshape(1, n[0], r_right)
    return cores


class TensorTrain:
    """A train of cores on the current GPU (hobo_tt_*)."""

    def __init__(self, cores):
        cores = [np.asarray(G, dtype=np.float32) for G in cores]
        if not cores or any(G.ndim != 3 for G in cores):
            raise ValueError("cores must be 3-d arrays [r_prev, N, r_next]")
        self.order, self.N = len(cores), cores[0].shape[1]
        ranks = np.array([cores[0].shape[0]] + [G.shape[2] for G in cores], dtype=np.int32)
        for c, G in enumerate(cores):
            if G.shape[1] != self.N or G.shape[0] != ranks[c]:
                raise ValueError("core shapes do not chain")
        flat = np.ascontiguousarray(np.concatenate([G.reshape(-1) for G in cores]))
        h = C.c_void_p()
        _check(load_library().hobo_tt_create(C.byref(h), self.order, self.N, ranks.ctypes.data_as(C.c_void_p),
                                             flat.ctypes.data_as(C.c_void_p)))
        self._h = h
        self.ranks = ranks.tolist()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().hobo_tt_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def energy(self, X, stream=None):
        """Energies (float32 CUDA [B]) of packed states X (int32 CUDA [B, W])."""
        import torch
        E = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _check(load_library().hobo_tt_energy(self._h, _ptr(X), X.shape[0], _ptr(E), _stream(stream)))
        return E
