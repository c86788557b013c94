"""Thin Python binding of the libhobo C ABI (include/hobo.h).

Argument marshalling only: every step of the energy contraction and of the
annealer runs in the library's CUDA kernels.  PyTorch supplies device
memory and the current CUDA stream.  If the compiled library is missing the
binding raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhobo.so")

HOBO_OK = 0
HOBO_ERR_ARG = -1
HOBO_ERR_ORDER = -2
HOBO_ERR_NOT_EXACT = -3
HOBO_ERR_OOM = -4
HOBO_ERR_CUDA = -5
HOBO_ERR_TIMEOUT = -6
HOBO_ERR_UNSUPPORTED = -7

HOBO_INTEGER = 1
HOBO_FORCE_SPARSE = 2
HOBO_FORCE_DENSE = 4
HOBO_SPLIT3 = 8
HOBO_SPLIT2 = 16
HOBO_RESCORE_CUDA_CORES = 32

HOBO_ANNEAL_TUNED = 0
HOBO_ANNEAL_PLAIN = 1

PATH_AUTO, PATH_TERMS, PATH_TENSOR_CORE, PATH_TENSOR_CORE_F32ACC = 0, 1, 2, 3

HOBO_MAX_ORDER = 8
HOBO_NOALLOC_MAX_B = 65536


class HoboError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hobo error {code}: {msg}")
        self.code = code


class hobo_info_t(C.Structure):
    _fields_ = [("N", C.c_int), ("order", C.c_int), ("words", C.c_int), ("dense", C.c_int),
                ("integer", C.c_int), ("terms", C.c_int64 * (HOBO_MAX_ORDER + 1)),
                ("abs_sum", C.c_double), ("tc_limbs", C.c_int)]


HOBO_BATCH_GRAPH = 0
HOBO_BATCH_PER_INSTANCE_TUNED = 1
HOBO_BATCH_PER_INSTANCE_PLAIN = 2


class hobo_batch_opts(C.Structure):
    _fields_ = [("mode", C.c_int), ("no_autotune", C.c_int), ("warps_per_cta", C.c_int),
                ("ctas_per_sm", C.c_int), ("accepts", C.c_void_p), ("X_out", C.c_void_p),
                ("E_out", C.c_void_p), ("ev_begin", C.c_void_p), ("ev_end", C.c_void_p)]


class hobo_learned_opts(C.Structure):
    _fields_ = [("plain_every", C.c_int), ("select", C.c_int), ("top_frac", C.c_float), ("threshold", C.c_float),
                ("table_size", C.c_int),
                ("vmax", C.c_float), ("rec_every", C.c_int), ("rec_states", C.c_int),
                ("rec_F", C.c_void_p), ("rec_y", C.c_void_p), ("X_out", C.c_void_p), ("E_out", C.c_void_p),
                ("accepts", C.c_void_p), ("ev_begin", C.c_void_p), ("ev_end", C.c_void_p)]


class hobo_anneal_opts(C.Structure):
    _fields_ = [("mode", C.c_int), ("states_per_block", C.c_int), ("sweep0", C.c_int),
                ("resume", C.c_int), ("X_io", C.c_void_p), ("bestE32_io", C.c_void_p),
                ("E_io", C.c_void_p), ("g_io", C.c_void_p), ("accepts", C.c_void_p), ("coef_bytes", C.c_void_p), ("ev_sweep_begin", C.c_void_p),
                ("ev_sweep_end", C.c_void_p), ("state0", C.c_uint64)]


_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libhobo.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libhobo.so not built ({path}); run paper_2407_19987_gb300/build.py")
    L = C.CDLL(path)
    P, I, I64, U64 = C.c_void_p, C.c_int, C.c_int64, C.c_uint64
    L.hobo_create.argtypes = [C.POINTER(P), P, I, I, C.c_uint]
    L.hobo_create_terms.argtypes = [C.POINTER(P), P, P, I64, I, I, C.c_uint]
    L.hobo_destroy.argtypes = [P]
    L.hobo_destroy.restype = None
    L.hobo_info.argtypes = [P, C.POINTER(hobo_info_t)]
    L.hobo_energy.argtypes = [P, P, I, P, P, P]
    L.hobo_energy_path.argtypes = [P, P, I, P, P, I, P]
    L.hobo_energy_fp64.argtypes = [P, P, I, P, P]
    L.hobo_anneal.argtypes = [P, U64, I, P, I, P, P, C.POINTER(hobo_anneal_opts), P]
    L.hobo_check.argtypes = [P, P]
    L.hobo_tt_create.argtypes = [C.POINTER(P), I, I, P, P]
    L.hobo_tt_create.restype = I
    L.hobo_tt_destroy.argtypes = [P]
    L.hobo_tt_destroy.restype = None
    L.hobo_tt_energy.argtypes = [P, P, I, P, P]
    L.hobo_tt_energy.restype = I
    L.hobo_aggregate.argtypes = [I, P, P, I, P, P, P, P, P, P]
    L.hobo_aggregate.restype = I
    L.hobo_selftest_timeout.argtypes = [P, U64, P]
    L.hobo_selftest_timeout.restype = I
    L.hobo_selftest_philox.argtypes = [P, P, I64, P, P, P]
    L.hobo_selftest_philox.restype = I
    L.hobo_probe_l2_read.argtypes = [P, I64, I, P]
    L.hobo_probe_l2_read.restype = I
    L.hobo_energy_fp64_noalloc.argtypes = [P, P, I, P, P]
    L.hobo_energy_fp64_noalloc.restype = I
    L.hobo_batch_create.argtypes = [C.POINTER(P), P, I, P]
    L.hobo_batch_destroy.argtypes = [P]
    L.hobo_batch_destroy.restype = None
    L.hobo_batch_layout.argtypes = [P, P, P]
    L.hobo_batch_anneal.argtypes = [P, P, P, I, P, P, C.POINTER(hobo_batch_opts), P]
    L.hobo_batch_launch_shape.argtypes = [P, I, C.POINTER(I), C.POINTER(I)]
    for name in ("hobo_batch_create", "hobo_batch_layout", "hobo_batch_anneal", "hobo_batch_launch_shape"):
        getattr(L, name).restype = I
    L.hobo_mlp_create.argtypes = [C.POINTER(P), I, U64]
    L.hobo_mlp_destroy.argtypes = [P]
    L.hobo_mlp_destroy.restype = None
    L.hobo_mlp_num_params.argtypes = [P]
    L.hobo_mlp_num_params.restype = I64
    L.hobo_mlp_get.argtypes = [P, P, I]
    L.hobo_mlp_set.argtypes = [P, P]
    L.hobo_mlp_forward.argtypes = [P, P, I64, P, P]
    L.hobo_mlp_set_tensor_cores.argtypes = [P, I]
    L.hobo_mlp_check.argtypes = [P, P]
    L.hobo_mlp_score_tables.argtypes = [P, P, I, I, C.c_float, P, P]
    L.hobo_mlp_loss_grad.argtypes = [P, P, P, I64, P, P, P]
    L.hobo_mlp_train_step.argtypes = [P, P, P, I64, C.c_float, P, P]
    L.hobo_mlp_save.argtypes = [P, C.c_char_p]
    L.hobo_mlp_load.argtypes = [C.POINTER(P), C.c_char_p]
    L.hobo_anneal_learned.argtypes = [P, P, U64, I, P, I, P, P, C.POINTER(hobo_learned_opts), P]
    for name in ("hobo_mlp_create", "hobo_mlp_get", "hobo_mlp_set", "hobo_mlp_forward", "hobo_mlp_set_tensor_cores",
                 "hobo_mlp_check", "hobo_mlp_score_tables", "hobo_mlp_loss_grad",
                 "hobo_mlp_train_step", "hobo_mlp_save", "hobo_mlp_load", "hobo_anneal_learned"):
        getattr(L, name).restype = I
    L.hobo_last_error.restype = C.c_char_p
    L.hobo_version.restype = C.c_char_p
    for name in ("hobo_create", "hobo_create_terms", "hobo_info", "hobo_energy", "hobo_energy_path",
                 "hobo_energy_fp64", "hobo_anneal", "hobo_check"):
        getattr(L, name).restype = I
    _lib = L
    return L


def _check(rc: int):
    if rc != HOBO_OK:
        raise HoboError(rc, load_library().hobo_last_error().decode())


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream=None) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def words(N: int) -> int:
    return (N + 31) // 32


class Instance:
    """A HOBO instance resident on the current CUDA device (hobo_create)."""

    def __init__(self, handle: int, N: int, order: int):
        self._h = C.c_void_p(handle)
        self.N = N
        self.order = order
        self.W = words(N)

    @classmethod
    def from_dense(cls, T: np.ndarray, flags: int = 0) -> "Instance":
        T = np.ascontiguousarray(T, dtype=np.float32)
        order, N = T.ndim, T.shape[0]
        if any(s != N for s in T.shape):
            raise ValueError("dense tensor must have shape (N,)*order")
        h = C.c_void_p()
        _check(load_library().hobo_create(C.byref(h), T.ctypes.data_as(C.c_void_p), order, N, flags))
        return cls(h.value, N, order)

    @classmethod
    def from_terms(cls, idx: np.ndarray, coef: np.ndarray, N: int, flags: int = 0) -> "Instance":
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        coef = np.ascontiguousarray(coef, dtype=np.float32)
        nnz, order = idx.shape
        h = C.c_void_p()
        _check(load_library().hobo_create_terms(C.byref(h), idx.ctypes.data_as(C.c_void_p),
                                                coef.ctypes.data_as(C.c_void_p), nnz, order, N, flags))
        return cls(h.value, N, order)

    def close(self):
        if self._h is not None and self._h.value:
            load_library().hobo_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    def info(self) -> dict:
        inf = hobo_info_t()
        _check(load_library().hobo_info(self._h, C.byref(inf)))
        return dict(N=inf.N, order=inf.order, words=inf.words, dense=bool(inf.dense),
                    integer=bool(inf.integer), terms=list(inf.terms), abs_sum=inf.abs_sum,
                    tc_limbs=inf.tc_limbs)

    def energy(self, X, with_delta: bool = True, path: int = PATH_AUTO, stream=None):
        """X: int32 CUDA tensor [B, W] of packed states.  Returns (E [B] f32,
        dE [B, N] f32 or None)."""
        import torch
        B = X.shape[0]
        E = torch.empty(B, dtype=torch.float32, device=X.device)
        dE = torch.empty((B, self.N), dtype=torch.float32, device=X.device) if with_delta else None
        self.energy_into(X, E, dE, path, stream)
        return E, dE

    def energy_into(self, X, E, dE=None, path: int = PATH_AUTO, stream=None):
        """hobo_energy_path into caller buffers: E float32 CUDA [B], dE float32
        CUDA [B, N] or None (no flip deltas)."""
        _check(load_library().hobo_energy_path(self._h, _ptr(X), X.shape[0], _ptr(E), _ptr(dE), path,
                                               _stream(stream)))

    def check(self, stream=None):
        """Synchronize the stream and raise HoboError(HOBO_ERR_TIMEOUT) if a
        kernel of this instance gave up a bounded wait."""
        _check(load_library().hobo_check(self._h, _stream(stream)))

    def selftest_timeout(self, limit_ns: int = 10_000_000, stream=None):
        """hobo_selftest_timeout: a bounded device wait that runs out; the
        next check() raises HoboError(HOBO_ERR_TIMEOUT)."""
        _check(load_library().hobo_selftest_timeout(self._h, C.c_uint64(limit_ns), _stream(stream)))

    def energy_fp64_noalloc(self, X, E=None, stream=None):
        """hobo_energy_fp64_noalloc: float64 re-score using the library's fixed
        device scratch (no allocation in the library; at most
        HOBO_NOALLOC_MAX_B states).  E: optional preallocated f64 output."""
        import torch
        B = X.shape[0]
        if E is None:
            E = torch.empty(B, dtype=torch.float64, device=X.device)
        _check(load_library().hobo_energy_fp64_noalloc(self._h, _ptr(X), B, _ptr(E), _stream(stream)))
        return E

    def energy_fp64(self, X, stream=None):
        import torch
        B = X.shape[0]
        E = torch.empty(B, dtype=torch.float64, device=X.device)
        _check(load_library().hobo_energy_fp64(self._h, _ptr(X), B, _ptr(E), _stream(stream)))
        return E

    def anneal(self, seed: int, B: int, betas: np.ndarray, *, mode: int = HOBO_ANNEAL_TUNED,
               states_per_block: int = 0, sweep0: int = 0, resume: bool = False, X=None,
               bestX=None, bestE32=None, E=None, g=None, want_final: bool = False,
               want_fields: bool = False, want_accepts: bool = False, want_bytes: bool = False,
               device=None, stream=None, sweep_events=None, state0: int = 0) -> dict:
        """Batched annealing (hobo_anneal).  betas: host float32 [sweeps];
        state0: global index of the first state (random streams).
        Returns a dict of CUDA tensors: bestX [B, W] int32, bestE [B] f64, and
        when asked X (final), E (final f32), bestE32, accepts."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        betas = np.ascontiguousarray(betas, dtype=np.float32)
        if bestX is None:
            bestX = torch.zeros((B, self.W), dtype=torch.int32, device=dev)
        bestE = torch.empty(B, dtype=torch.float64, device=dev)
        if X is None and (want_final or resume):
            X = torch.zeros((B, self.W), dtype=torch.int32, device=dev)
        if bestE32 is None:
            bestE32 = torch.empty(B, dtype=torch.float32, device=dev)
        if E is None and (want_final or want_fields):
            E = torch.empty(B, dtype=torch.float32, device=dev)
        if g is None and want_fields:
            g = torch.empty((B, self.N), dtype=torch.float32, device=dev)
        acc = torch.zeros(B, dtype=torch.int64, device=dev) if want_accepts else None
        cb = torch.zeros(B, dtype=torch.int64, device=dev) if want_bytes else None
        ev0 = ev1 = None
        if sweep_events is not None:
            for e in sweep_events:          # torch creates its events lazily
                if not e.cuda_event:
                    e.record()
            ev0, ev1 = sweep_events[0].cuda_event, sweep_events[1].cuda_event
        o = hobo_anneal_opts(mode, states_per_block, sweep0, 1 if resume else 0,
                             _ptr(X), _ptr(bestE32), _ptr(E), _ptr(g), _ptr(acc), _ptr(cb), ev0, ev1,
                             int(state0) & (2 ** 64 - 1))
        _check(load_library().hobo_anneal(self._h, C.c_uint64(seed & (2 ** 64 - 1)), B,
                                          betas.ctypes.data_as(C.c_void_p), betas.shape[0],
                                          _ptr(bestX), _ptr(bestE), C.byref(o), _stream(stream)))
        out = dict(bestX=bestX, bestE=bestE, bestE32=bestE32)
        if X is not None:
            out["X"] = X
        if E is not None:
            out["E"] = E
        if g is not None:
            out["g"] = g
        if acc is not None:
            out["accepts"] = acc
        if cb is not None:
            out["coef_bytes"] = cb
        return out


def version() -> str:
    return load_library().hobo_version().decode()


def _event_handle(e):
    if e is None:
        return None
    if not e.cuda_event:          # torch creates its events lazily
        e.record()
    return e.cuda_event


class Batch:
    """A batch plan over several instances (hobo_batch_create): instance t
    contributes B[t] states; outputs are laid out instance after instance."""

    def __init__(self, instances, B):
        self.instances = list(instances)     # kept alive while the plan exists
        self.B = [int(b) for b in B]
        n = len(self.instances)
        arr = (C.c_void_p * n)(*[i.handle.value for i in self.instances])
        bs = np.ascontiguousarray(np.array(self.B, dtype=np.int32))
        h = C.c_void_p()
        _check(load_library().hobo_batch_create(C.byref(h), arr, n, bs.ctypes.data_as(C.c_void_p)))
        self._h = h
        so = np.zeros(n, np.int64)
        wo = np.zeros(n, np.int64)
        _check(load_library().hobo_batch_layout(self._h, so.ctypes.data_as(C.c_void_p), wo.ctypes.data_as(C.c_void_p)))
        self.state_offset = so
        self.word_offset = wo
        self.total = int(sum(self.B))
        self.words = int(sum(b * inst.W for b, inst in zip(self.B, self.instances)))

    def close(self):
        if self._h is not None and self._h.value:
            load_library().hobo_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def anneal(self, seeds, betas, *, mode: int = HOBO_BATCH_GRAPH, no_autotune: bool = False,
               warps_per_cta: int = 0, ctas_per_sm: int = 0, want_final: bool = False,
               want_accepts: bool = False, events=None, stream=None) -> dict:
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        seeds = np.ascontiguousarray(np.array(seeds, dtype=np.uint64))
        betas = np.ascontiguousarray(betas, dtype=np.float32)
        bestX = torch.zeros(self.words, dtype=torch.int32, device=dev)
        bestE = torch.empty(self.total, dtype=torch.float64, device=dev)
        X = torch.zeros(self.words, dtype=torch.int32, device=dev) if want_final else None
        E = torch.empty(self.total, dtype=torch.float32, device=dev) if want_final else None
        acc = torch.zeros(self.total, dtype=torch.int64, device=dev) if want_accepts else None
        ev0, ev1 = (None, None) if events is None else (_event_handle(events[0]), _event_handle(events[1]))
        o = hobo_batch_opts(mode, 1 if no_autotune else 0, warps_per_cta, ctas_per_sm, _ptr(acc), _ptr(X),
                            _ptr(E), ev0, ev1)
        _check(load_library().hobo_batch_anneal(self._h, seeds.ctypes.data_as(C.c_void_p),
                                                betas.ctypes.data_as(C.c_void_p), betas.shape[0],
                                                _ptr(bestX), _ptr(bestE), C.byref(o), _stream(stream)))
        out = dict(bestX=bestX, bestE=bestE)
        if X is not None:
            out["X"], out["E"] = X, E
        if acc is not None:
            out["accepts"] = acc
        return out

    def rows(self, flat, t):
        """View of instance t's block of a state-indexed or word-indexed output."""
        inst = self.instances[t]
        if flat.numel() == self.total:
            o = int(self.state_offset[t])
            return flat[o:o + self.B[t]]
        o = int(self.word_offset[t])
        return flat[o:o + self.B[t] * inst.W].view(self.B[t], inst.W)

    def launch_shape(self, group: int = 0):
        w = C.c_int()
        c = C.c_int()
        _check(load_library().hobo_batch_launch_shape(self._h, group, C.byref(w), C.byref(c)))
        return w.value, c.value


class MLP:
    """The learned flip-proposal network (hobo_mlp_*): 3 -> H -> H -> 1,
    bf16 weights, trained by the library's kernels."""

    def __init__(self, hidden: int = 256, seed: int = 0, _handle=None):
        if _handle is None:
            h = C.c_void_p()
            _check(load_library().hobo_mlp_create(C.byref(h), hidden, C.c_uint64(seed)))
            _handle = h
        self._h = _handle
        self.nparam = int(load_library().hobo_mlp_num_params(self._h))
        self.hidden = hidden

    @classmethod
    def load(cls, path: str) -> "MLP":
        h = C.c_void_p()
        _check(load_library().hobo_mlp_load(C.byref(h), path.encode()))
        m = cls(_handle=h)
        m.hidden = (int(np.sqrt(36 + 4 * (m.nparam - 1))) - 6) // 2
        return m

    def close(self):
        if self._h is not None and self._h.value:
            load_library().hobo_mlp_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def params(self, rounded: bool = True) -> np.ndarray:
        out = np.zeros(self.nparam, np.float32)
        _check(load_library().hobo_mlp_get(self._h, out.ctypes.data_as(C.c_void_p), 1 if rounded else 0))
        return out

    def set_params(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        _check(load_library().hobo_mlp_set(self._h, flat.ctypes.data_as(C.c_void_p)))

    def unpack(self, flat: np.ndarray) -> dict:
        H = self.hidden
        o = 0
        out = {}
        for k, shape in (("W1", (H, 3)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))):
            n = int(np.prod(shape))
            out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
            o += n
        return out

    def set_tensor_cores(self, on: bool):
        """Forward passes and score tables on the tensor cores (default for
        hidden widths 64..256, multiples of 64) or on CUDA cores."""
        _check(load_library().hobo_mlp_set_tensor_cores(self._h, 1 if on else 0))

    def check(self, stream=None):
        """Raise HoboError if a network kernel gave up a bounded wait."""
        _check(load_library().hobo_mlp_check(self._h, _stream(stream)))

    def score_tables(self, beta, G: int = 256, vmax: float = 32.0, stream=None):
        """The learned sweep's score tables [S, 2, G] for the device betas
        [S] (hobo_mlp_score_tables)."""
        import torch
        beta = beta.contiguous()
        out = torch.empty((beta.shape[0], 2, G), dtype=torch.float32, device=beta.device)
        _check(load_library().hobo_mlp_score_tables(self._h, _ptr(beta), beta.shape[0], G, C.c_float(vmax),
                                                    _ptr(out), _stream(stream)))
        return out

    def forward(self, F, stream=None):
        import torch
        logit = torch.empty(F.shape[0], dtype=torch.float32, device=F.device)
        _check(load_library().hobo_mlp_forward(self._h, _ptr(F), F.shape[0], _ptr(logit), _stream(stream)))
        return logit

    def loss_grad(self, F, y, stream=None):
        import torch
        g = torch.empty(self.nparam, dtype=torch.float32, device=F.device)
        loss = torch.empty(1, dtype=torch.float32, device=F.device)
        _check(load_library().hobo_mlp_loss_grad(self._h, _ptr(F), _ptr(y), F.shape[0], _ptr(g), _ptr(loss),
                                                 _stream(stream)))
        return loss, g

    def train_step(self, F, y, lr: float, loss=None, stream=None):
        _check(load_library().hobo_mlp_train_step(self._h, _ptr(F), _ptr(y), F.shape[0], C.c_float(lr),
                                                  _ptr(loss), _stream(stream)))

    def save(self, path: str):
        _check(load_library().hobo_mlp_save(self._h, path.encode()))


SELECT_ORDER, SELECT_THRESHOLD = 0, 1


def anneal_learned(inst: Instance, mlp, seed: int, B: int, betas: np.ndarray, *, plain_every: int = 4,
                   select: int = SELECT_ORDER, top_frac: float = 1.0, threshold: float = 0.0,
                   table_size: int = 0, vmax: float = 0.0, rec_every: int = 0,
                   rec_states: int = 0, want_final: bool = False, want_accepts: bool = False, events=None,
                   stream=None) -> dict:
    """hobo_anneal_learned through the C ABI; returns CUDA tensors."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    betas = np.ascontiguousarray(betas, dtype=np.float32)
    S = betas.shape[0]
    bestX = torch.zeros((B, inst.W), dtype=torch.int32, device=dev)
    bestE = torch.empty(B, dtype=torch.float64, device=dev)
    X = torch.zeros((B, inst.W), dtype=torch.int32, device=dev) if want_final else None
    E = torch.empty(B, dtype=torch.float32, device=dev) if want_final else None
    acc = torch.zeros(B, dtype=torch.int64, device=dev) if want_accepts else None
    recF = recy = None
    if rec_every > 0 and rec_states > 0:
        nr = ((S + rec_every - 1) // rec_every) * min(rec_states, B) * inst.N
        recF = torch.zeros((nr, 3), dtype=torch.float32, device=dev)
        recy = torch.zeros(nr, dtype=torch.float32, device=dev)
    ev0, ev1 = (None, None) if events is None else (_event_handle(events[0]), _event_handle(events[1]))
    o = hobo_learned_opts(plain_every, select, top_frac, threshold, table_size, vmax, rec_every, rec_states,
                          _ptr(recF), _ptr(recy),
                          _ptr(X), _ptr(E), _ptr(acc), ev0, ev1)
    _check(load_library().hobo_anneal_learned(inst.handle, None if mlp is None else mlp.handle,
                                              C.c_uint64(seed & (2 ** 64 - 1)), B,
                                              betas.ctypes.data_as(C.c_void_p), S, _ptr(bestX), _ptr(bestE),
                                              C.byref(o), _stream(stream)))
    out = dict(bestX=bestX, bestE=bestE)
    if X is not None:
        out["X"], out["E"] = X, E
    if acc is not None:
        out["accepts"] = acc
    if recF is not None:
        out["rec_F"], out["rec_y"] = recF, recy
    return out


def aggregate(X, E, stream=None) -> dict:
    """hobo_aggregate: distinct states of X (int32 CUDA [B, W]) with energies
    E (float64 CUDA [B]), sorted by energy then first index.  Returns CUDA
    tensors states [K, W], energy [K], count [K], first [K]."""
    import torch
    B, W = X.shape
    dev = X.device
    U = torch.empty((max(B, 1), W), dtype=torch.int32, device=dev)
    UE = torch.empty(max(B, 1), dtype=torch.float64, device=dev)
    cnt = torch.empty(max(B, 1), dtype=torch.int64, device=dev)
    first = torch.empty(max(B, 1), dtype=torch.int32, device=dev)
    K = torch.zeros(1, dtype=torch.int32, device=dev)
    _check(load_library().hobo_aggregate(W, _ptr(X), _ptr(E), B, _ptr(U), _ptr(UE), _ptr(cnt), _ptr(first),
                                         _ptr(K), _stream(stream)))
    k = int(K.item())
    return {"states": U[:k], "energy": UE[:k], "count": cnt[:k], "first": first[:k]}


def selftest_philox(ctr, key, stream=None):
    """hobo_selftest_philox: the library's Philox4x32-10 blocks and those of
    the cuRAND device header for counters ctr (uint32 CUDA [n, 4], as int32)
    and keys key ([n, 2]).  Returns (ours, ref), int32 CUDA [n, 4]."""
    import torch
    n = ctr.shape[0]
    ours = torch.empty((n, 4), dtype=torch.int32, device=ctr.device)
    ref = torch.empty((n, 4), dtype=torch.int32, device=ctr.device)
    _check(load_library().hobo_selftest_philox(_ptr(ctr), _ptr(key), n, _ptr(ours), _ptr(ref), _stream(stream)))
    return ours, ref


def probe_l2_read(buf, reps: int, stream=None):
    """hobo_probe_l2_read: one launch reading the CUDA buffer `buf` reps
    times (16-byte loads cached in L2 only); time it with CUDA events."""
    _check(load_library().hobo_probe_l2_read(_ptr(buf), buf.numel() * buf.element_size(), reps, _stream(stream)))
