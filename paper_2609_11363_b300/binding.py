"""ctypes binding of libsinv (argument marshalling only).

Numeric calls take CUDA tensors (float64, contiguous) and run on the current
torch stream unless a stream is given.  Index arrays for the symbolic call are
host numpy arrays (the symbolic analysis runs on the host).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsinv.so")
_lib = None


def use_checked_library():
    """Load the checked build (libsinv_checked.so: out-of-range plan or map indices
    are reported as SINV_ERR_CUDA 'index out of range' instead of being used) in
    place of the regular one; call before anything loads the library."""
    global _LIB_PATH
    if _lib is not None:
        raise RuntimeError("the library is already loaded")
    _LIB_PATH = os.path.join(_HERE, "libsinv_checked.so")

PREC = {"fp64": 0, "fp32": 1, "fp32x2": 2, "tf32": 3, "bf16": 4}
STATUS = {
    0: "SINV_OK", 1: "SINV_ERR_INVALID_ARG", 2: "SINV_ERR_PATTERN", 3: "SINV_ERR_SINGULAR_PIVOT",
    4: "SINV_ERR_OOM", 5: "SINV_ERR_CUDA", 6: "SINV_ERR_TIMEOUT", 7: "SINV_ERR_UNSUPPORTED",
}

# every symbol include/sinv.h declares
EXPORTS = [
    "sinv_symbolic", "sinv_get_pattern", "sinv_get_pattern_host", "sinv_selinv", "sinv_ninv", "sinv_mix",
    "sinv_lowrank_correct", "sinv_sync_status", "sinv_get_stats", "sinv_get_supernodes",
    "sinv_status_string", "sinv_last_error", "sinv_destroy", "sinv_debug_wait_timeout",
    "sinv_trace_enable", "sinv_trace_read", "sinv_lowrank_correct_noalloc",
    "sinv_batch_symbolic", "sinv_batch_layout", "sinv_ninv_stack", "sinv_ninv_drop",
    "sinv_spai_analyse", "sinv_spai_pattern", "sinv_spai", "sinv_einv_analyse", "sinv_einv_lanczos",
    "sinv_mlp_param_count", "sinv_mlp_create", "sinv_mlp_destroy", "sinv_mlp_get_params", "sinv_mlp_set_params",
    "sinv_mlp_features", "sinv_mlp_targets", "sinv_mlp_grad", "sinv_mlp_train_step", "sinv_mlp_predict",
    "sinv_mlp_sync_status", "sinv_timeline_enable", "sinv_timeline_read", "sinv_batch_run",
    "sinv_einv_set_solver", "sinv_ninv_own", "sinv_ninv_own_size", "sinv_ninv_own_copy",
    "sinv_selinv_scan_counts", "sinv_mix_own", "sinv_mix_own_size", "sinv_mix_own_copy",
    "sinv_lowrank_correct_mix_own", "sinv_spai_analyse_mix_own", "sinv_spai_mix_own", "sinv_debug_corrupt_plan",
    "sinv_mlp_get_state", "sinv_mlp_set_state",
]


class SinvError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = int(status)
        self.name = STATUS.get(self.status, str(status))
        super().__init__("%s: %s" % (self.name, msg))


class _Opts(ctypes.Structure):
    _fields_ = [("supernode_cap", ctypes.c_int32), ("device", ctypes.c_int32), ("wait_limit", ctypes.c_int64),
                ("big_pairs", ctypes.c_int64), ("ninv_index_bytes", ctypes.c_int64),
                ("selinv_pair_bytes", ctypes.c_int64)]


class _KTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("n", "nnz_L", "nnz_S_lo", "n_blocks", "n_2x2", "n_supernodes",
                                              "n_levels", "max_c", "hit_pairs", "max_width", "nnz_W")] + [
        ("ninv_m", ctypes.c_int32), ("pad", ctypes.c_int32), ("horner_products", ctypes.c_int64),
        ("product_stream", ctypes.c_int64), ("selinv_flops", ctypes.c_int64), ("selinv_bytes", ctypes.c_int64),
        ("ninv_index_bytes", ctypes.c_int64), ("product_hits", ctypes.c_int64), ("spai_entries", ctypes.c_int64),
        ("spai_cols_warp", ctypes.c_int64), ("spai_cols_cta", ctypes.c_int64), ("spai_nnz_P", ctypes.c_int64),
        ("einv_levels_fwd", ctypes.c_int64), ("einv_levels_bwd", ctypes.c_int64), ("tc_levels", ctypes.c_int64),
        ("tc_supernodes", ctypes.c_int64), ("tc_pairs", ctypes.c_int64), ("tc_mirror_bytes", ctypes.c_int64),
        ("selinv_scan", ctypes.c_int64), ("scan_rows_total", ctypes.c_int64)]


def lib_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libsinv.so (build it first with ``paper_2609_11363_b300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libsinv.so not built at %s (run __graft_entry__.build())" % _LIB_PATH)
    lib = ctypes.CDLL(_LIB_PATH)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    H = ctypes.c_void_p
    lib.sinv_symbolic.argtypes = [I64, P, P, P, ctypes.POINTER(_Opts), ctypes.POINTER(H)]
    lib.sinv_get_pattern.argtypes = [H, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(I64)]
    lib.sinv_get_pattern_host.argtypes = [H, P, P]
    lib.sinv_selinv.argtypes = [H, P, P, ctypes.c_int, P, P]
    lib.sinv_ninv.argtypes = [H, P, P, ctypes.c_int, ctypes.c_int, P, P]
    lib.sinv_ninv_drop.argtypes = [H, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_int, P, P]
    lib.sinv_mix.argtypes = [H, P, P, D, P, P]
    lib.sinv_spai_analyse.argtypes = [H, I64, P, P, ctypes.c_int, ctypes.c_int]
    lib.sinv_spai_pattern.argtypes = [H, P, P]
    lib.sinv_einv_analyse.argtypes = [H, I64, P, P]
    lib.sinv_einv_lanczos.argtypes = [H, P, P, P, P, P, ctypes.c_int, D, ctypes.c_int, ctypes.c_int, P, P, P, P]
    lib.sinv_spai.argtypes = [H, P, P, ctypes.c_int, P, P]
    lib.sinv_lowrank_correct.argtypes = [H, ctypes.c_int, P, P, ctypes.c_int, P, P]
    lib.sinv_sync_status.argtypes = [H, P]
    lib.sinv_get_stats.argtypes = [H, ctypes.POINTER(_Stats)]
    lib.sinv_get_supernodes.argtypes = [H, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(I64)]
    lib.sinv_status_string.argtypes = [ctypes.c_int]
    lib.sinv_status_string.restype = ctypes.c_char_p
    lib.sinv_last_error.argtypes = [H, ctypes.c_char_p, ctypes.c_size_t]
    lib.sinv_destroy.argtypes = [H]
    lib.sinv_destroy.restype = None
    lib.sinv_debug_wait_timeout.argtypes = [H, P]
    lib.sinv_ninv_stack.argtypes = [H, P, P, ctypes.c_int, ctypes.c_int, P, P]
    lib.sinv_mlp_create.argtypes = [ctypes.c_int32, ctypes.c_uint64, I64, ctypes.POINTER(H)]
    lib.sinv_mlp_destroy.argtypes = [H]
    lib.sinv_mlp_get_params.argtypes = [H, P]
    lib.sinv_mlp_set_params.argtypes = [H, P]
    lib.sinv_mlp_get_state.argtypes = [H, P, P, P, ctypes.POINTER(I64)]
    lib.sinv_mlp_set_state.argtypes = [H, P, P, P, I64]
    lib.sinv_mlp_features.argtypes = [H, P, ctypes.c_int, P, P, P, P, P]
    lib.sinv_mlp_targets.argtypes = [H, I64, P, P, P, P, P]
    lib.sinv_mlp_grad.argtypes = [H, P, P, P, I64, P, P, P]
    lib.sinv_mlp_train_step.argtypes = [H, P, P, P, I64, ctypes.c_float, P, P]
    lib.sinv_mlp_predict.argtypes = [H, P, P, P, I64, P, P]
    lib.sinv_mlp_sync_status.argtypes = [H, P]
    lib.sinv_timeline_enable.argtypes = [H, ctypes.c_int]
    lib.sinv_timeline_read.argtypes = [H, P, I64, P]
    lib.sinv_selinv_scan_counts.argtypes = [H, ctypes.POINTER(I64), ctypes.POINTER(I64), P]
    lib.sinv_debug_corrupt_plan.argtypes = [H]
    lib.sinv_batch_run.argtypes = [H, ctypes.c_int32, P, P, ctypes.c_int, P, ctypes.c_int, P, P]
    lib.sinv_einv_set_solver.argtypes = [H, ctypes.c_int32]
    lib.sinv_ninv_own.argtypes = [H, P, P, ctypes.c_int, ctypes.c_double, P]
    lib.sinv_ninv_own_size.argtypes = [H, ctypes.POINTER(I64), P, ctypes.c_int32]
    lib.sinv_ninv_own_copy.argtypes = [H, P, P, P, P]
    lib.sinv_mix_own.argtypes = [H, P, ctypes.c_double, P]
    lib.sinv_mix_own_size.argtypes = [H, ctypes.POINTER(I64)]
    lib.sinv_mix_own_copy.argtypes = [H, P, P, P, P]
    lib.sinv_lowrank_correct_mix_own.argtypes = [H, ctypes.c_int, P, P, ctypes.c_int, P]
    lib.sinv_spai_analyse_mix_own.argtypes = [H, I64, P, P, ctypes.c_int]
    lib.sinv_spai_mix_own.argtypes = [H, P, P, ctypes.c_int, P, P]
    lib.sinv_batch_symbolic.argtypes = [ctypes.c_int32, P, P, P, P, ctypes.POINTER(_Opts), ctypes.POINTER(H)]
    lib.sinv_batch_layout.argtypes = [H, ctypes.POINTER(ctypes.c_int32), P, P, P, P]
    lib.sinv_lowrank_correct_noalloc.argtypes = [I64, P, P, ctypes.c_int, P, P, P, P]
    lib.sinv_trace_enable.argtypes = [H, ctypes.c_int]
    lib.sinv_trace_read.argtypes = [H, ctypes.POINTER(_KTime), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                    ctypes.c_int]
    for name in EXPORTS:
        f = getattr(lib, name)
        if name not in ("sinv_status_string", "sinv_destroy", "sinv_mlp_destroy"):
            f.restype = ctypes.c_int
    lib.sinv_mlp_destroy.restype = None
    _lib = lib
    return lib


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check_tensor(t, name, numel=None, dtype=torch.float64, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if device is not None and t.device != device:
        raise ValueError("%s is on %s, the handle on %s" % (name, t.device, device))
    if t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if numel is not None and t.numel() != numel:
        raise ValueError("%s has %d entries, expected %d" % (name, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream, device=None):
    if stream is None:
        if not torch.cuda.is_available():
            return ctypes.c_void_p(0)  # host-only handles: the library rejects the call itself
        stream = torch.cuda.current_stream(device)
    elif device is not None and stream.device != device:
        raise ValueError("the stream is on %s, the handle on %s" % (stream.device, device))
    return ctypes.c_void_p(stream.cuda_stream)


MLP_F = 16
MLP_H = 64


class Mlp:
    """The learned NInv -> SelInv correction network (weights live on the GPU)."""

    def __init__(self, seed=0, max_batch=1 << 16, device=0):
        self._lib = load_library()
        self._m = ctypes.c_void_p()
        self.device = torch.device("cuda", int(device))
        self.max_batch = int(max_batch)
        st = self._lib.sinv_mlp_create(int(device), ctypes.c_uint64(int(seed)), self.max_batch, ctypes.byref(self._m))
        if st != 0:
            raise SinvError(st, "sinv_mlp_create")
        self.n_params = int(self._lib.sinv_mlp_param_count())
        self._loss = torch.zeros(1, dtype=torch.float32, device=self.device)

    def _t(self, t, name, numel=None, dtype=torch.float64):
        """A CUDA tensor of this object's device (else ValueError), as a pointer."""
        return _check_tensor(t, name, numel, dtype, self.device)

    def _s(self, stream):
        """The given stream (on this object's device) or that device's current one."""
        return _stream_ptr(stream, self.device)

    def close(self):
        if getattr(self, "_m", None):
            self._lib.sinv_mlp_destroy(self._m)
            self._m = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st, what):
        if st != 0:
            raise SinvError(st, what)

    def get_params(self) -> np.ndarray:
        th = np.empty(self.n_params, dtype=np.float32)
        self._chk(self._lib.sinv_mlp_get_params(self._m, _np_ptr(th)), "get_params")
        return th

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        assert th.size == self.n_params
        self._chk(self._lib.sinv_mlp_set_params(self._m, _np_ptr(th)), "set_params")

    def get_state(self) -> dict:
        """The training state (weights, Adam moments, step count) as host arrays."""
        th, m1, m2 = (np.empty(self.n_params, dtype=np.float32) for _ in range(3))
        step = ctypes.c_int64()
        self._chk(self._lib.sinv_mlp_get_state(self._m, _np_ptr(th), _np_ptr(m1), _np_ptr(m2), ctypes.byref(step)),
                  "get_state")
        return {"theta": th, "mom1": m1, "mom2": m2, "step": int(step.value)}

    def set_state(self, state):
        """Restore a state from get_state: training continues where it stopped."""
        arrs = [np.ascontiguousarray(state[k], dtype=np.float32) for k in ("theta", "mom1", "mom2")]
        if any(a.size != self.n_params for a in arrs):
            raise ValueError("a state holds %d floats per array" % self.n_params)
        self._chk(self._lib.sinv_mlp_set_state(self._m, *[_np_ptr(a) for a in arrs], int(state["step"])),
                  "set_state")

    def save(self, path):
        """Checkpoint the training state to an .npz file."""
        st = self.get_state()
        np.savez(path, theta=st["theta"], mom1=st["mom1"], mom2=st["mom2"], step=np.int64(st["step"]))

    def load(self, path):
        """Restore a checkpoint written by save()."""
        with np.load(path) as z:
            self.set_state({"theta": z["theta"], "mom1": z["mom1"], "mom2": z["mom2"], "step": int(z["step"])})

    def targets(self, G, N, scale, stream=None):
        y = torch.empty(G.numel(), dtype=torch.float32, device=self.device)
        self._chk(self._lib.sinv_mlp_targets(self._m, G.numel(), self._t(G, "G"), self._t(N, "N"),
                                             self._t(scale, "scale", None, torch.float32),
                                             self._t(y, "y", None, torch.float32), self._s(stream)),
                  "targets")
        return y

    def grad(self, X, y, idx=None, stream=None):
        """(gradient [n_params] float32 tensor, loss tensor) over the entries idx (or all)."""
        count = int(idx.numel()) if idx is not None else int(X.shape[0])
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        self._chk(self._lib.sinv_mlp_grad(self._m, self._t(X, "X", None, torch.bfloat16),
                                          self._t(y, "y", None, torch.float32),
                                          self._t(idx, "idx", None, torch.int64) if idx is not None else None,
                                          count, self._t(g, "grad", None, torch.float32),
                                          self._t(self._loss, "loss", None, torch.float32), self._s(stream)),
                  "grad")
        return g, self._loss

    def train_step(self, X, y, idx, lr, stream=None):
        self._chk(self._lib.sinv_mlp_train_step(self._m, self._t(X, "X", None, torch.bfloat16),
                                                self._t(y, "y", None, torch.float32),
                                                self._t(idx, "idx", None, torch.int64), int(idx.numel()),
                                                ctypes.c_float(lr), self._t(self._loss, "loss", None,
                                                                                  torch.float32),
                                                self._s(stream)), "train_step")
        return self._loss

    def predict(self, X, scale, N, out=None, stream=None):
        if out is None:
            out = torch.empty_like(N)
        self._chk(self._lib.sinv_mlp_predict(self._m, self._t(X, "X", None, torch.bfloat16),
                                             self._t(scale, "scale", None, torch.float32),
                                             self._t(N, "N"), int(N.numel()), self._t(out, "out"),
                                             self._s(stream)), "predict")
        return out

    def sync_status(self, stream=None):
        """Synchronize and raise on a device error of the asynchronous calls."""
        self._chk(self._lib.sinv_mlp_sync_status(self._m, self._s(stream)), "sync_status")


LOWRANK_NOALLOC_MAX = 1 << 22  # n*k + k floats of the library's built-in working array
LOWRANK_NOALLOC_KMAX = 256     # largest rank k of the low-rank correction


def lowrank_correct_noalloc(S_rowptr, S_col, V, lam, X, stream=None):
    """FP32 low-rank correction on S through the allocation-free entry point.

    For callers that cannot allocate device memory: no handle, the working copy
    lives in the library's fixed 16 MiB array.  S_rowptr (int64, n+1) and S_col
    (int32) are the pattern on the device; V (n x k, float64), lam (k) and the
    in/out X (float64) are CUDA tensors, all on one device; the call runs with
    that device current.  Raises SinvError(SINV_ERR_UNSUPPORTED) when k > 256 or
    n*k + k exceeds LOWRANK_NOALLOC_MAX.
    """
    lib = load_library()
    tensors = (S_rowptr, S_col, V, lam, X)
    dev = V.device
    if dev.type != "cuda" or any(t.device != dev for t in tensors):
        raise ValueError("S_rowptr, S_col, V, lam and X must be CUDA tensors on one device")
    n = int(S_rowptr.numel()) - 1
    k = int(lam.numel())
    with torch.cuda.device(dev):
        st = lib.sinv_lowrank_correct_noalloc(
            n, _check_tensor(S_rowptr, "S_rowptr", n + 1, torch.int64),
            _check_tensor(S_col, "S_col", None, torch.int32), k, _check_tensor(V, "V", n * k),
            _check_tensor(lam, "lambda", k), _check_tensor(X, "X_S", int(S_col.numel())), _stream_ptr(stream))
    if st != 0:
        if st == 7:
            msg = "k = %d (limit %d) or n*k + k = %d (limit %d) too large" % (
                k, LOWRANK_NOALLOC_KMAX, n * k + k, LOWRANK_NOALLOC_MAX)
        else:
            msg = "invalid argument" if st == 1 else "launch failed"
        raise SinvError(st, msg)
    return X


class Handle:
    """Symbolic analysis of one factor pattern; numeric calls reuse it.

    ``L_rowptr`` (int64, n+1), ``L_col`` (int32), ``pivot_start`` (int8, n) are
    host arrays describing strictly lower CSR L and the 1x1/2x2 pivot layout.
    """

    def __init__(self, n, L_rowptr, L_col, pivot_start, supernode_cap=0, device=0, wait_limit=0, big_pairs=0,
                 ninv_index_bytes=0, selinv_pair_bytes=0, _batch=None):
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        opts = _Opts(int(supernode_cap), int(device), int(wait_limit), int(big_pairs), int(ninv_index_bytes),
                     int(selinv_pair_bytes))
        self.device = torch.device("cuda", int(device)) if int(device) >= 0 else None
        if _batch is None:
            self.n = int(n)
            rp = np.ascontiguousarray(L_rowptr, dtype=np.int64)
            col = np.ascontiguousarray(L_col, dtype=np.int32)
            ps = np.ascontiguousarray(pivot_start, dtype=np.int8)
            if rp.shape != (self.n + 1,) or ps.shape != (self.n,):
                raise ValueError("L_rowptr must have n+1 and pivot_start n entries")
            st = self._lib.sinv_symbolic(self.n, _np_ptr(rp), _np_ptr(col), _np_ptr(ps), ctypes.byref(opts),
                                         ctypes.byref(self._h))
        else:
            ns, rps, cols, pss = _batch
            nmat = len(ns)
            keep = [np.ascontiguousarray(x, dtype=dt) for xs, dt in ((rps, np.int64), (cols, np.int32), (pss, np.int8))
                    for x in xs]
            rps_a, cols_a, pss_a = keep[:nmat], keep[nmat:2 * nmat], keep[2 * nmat:]
            n_arr = np.ascontiguousarray(ns, dtype=np.int64)
            arr = lambda xs: (ctypes.c_void_p * max(nmat, 1))(*[x.ctypes.data for x in xs])  # noqa: E731
            prp, pcol, pps = arr(rps_a), arr(cols_a), arr(pss_a)
            self.n = int(n_arr.sum())
            st = self._lib.sinv_batch_symbolic(nmat, _np_ptr(n_arr), ctypes.cast(prp, ctypes.c_void_p),
                                               ctypes.cast(pcol, ctypes.c_void_p), ctypes.cast(pps, ctypes.c_void_p),
                                               ctypes.byref(opts), ctypes.byref(self._h))
        if st != 0:
            msg = self.last_error()
            self.close()
            raise SinvError(st, msg)
        s = self.stats()
        self.nnz_S = s["nnz_S_lo"]
        self.nnz_L = s["nnz_L"]
        self.nD = self.n + s["n_2x2"]

    @classmethod
    def batch(cls, factors, **kw):
        """One handle over several matrices (block-diagonal concatenation).

        ``factors``: sequence of objects with n, L_rowptr, L_col, pivot_start.
        Value arrays are concatenated in matrix order; ``layout()`` gives the offsets.
        """
        fs = list(factors)
        return cls(None, None, None, None, _batch=([f.n for f in fs], [f.L_rowptr for f in fs],
                                                   [f.L_col for f in fs], [f.pivot_start for f in fs]), **kw)

    def layout(self):
        """{'n', 'L', 'D', 'S'}: nmat+1 offsets each (empty for a single-matrix handle)."""
        nmat = ctypes.c_int32()
        self._check(self._lib.sinv_batch_layout(self._h, ctypes.byref(nmat), None, None, None, None))
        k = nmat.value
        if k == 0:
            return {}
        arrs = [np.zeros(k + 1, dtype=np.int64) for _ in range(4)]
        self._check(self._lib.sinv_batch_layout(self._h, ctypes.byref(nmat), *[_np_ptr(a) for a in arrs]))
        return dict(zip(("n", "L", "D", "S"), arrs))

    def batch_run(self, L_vals, D_vals, prec="fp64", G_outs=None, m=0, N_outs=None, stream=None):
        """sinv_batch_run: SelInv (into G_outs) and / or NInv with m terms (into N_outs)
        for every matrix of a batch handle, each in its own CUDA tensors."""
        k = len(L_vals)

        def ptrs(ts, name, dtype=torch.float64):
            arr = (ctypes.c_void_p * k)()
            for b, t in enumerate(ts):
                arr[b] = self._t(t, name, None, dtype).value if t is not None else None
            return arr

        Lp, Dp = ptrs(L_vals, "L_val"), ptrs(D_vals, "D_val")
        Gp = ptrs(G_outs, "G_out") if G_outs is not None else None
        Np = ptrs(N_outs, "N_out") if N_outs is not None else None
        self._check(self._lib.sinv_batch_run(self._h, k, Lp, Dp, PREC[prec], Gp, int(m), Np, self._s(stream)))

    # -- helpers -----------------------------------------------------------
    def last_error(self) -> str:
        if not self._h:
            return ""
        buf = ctypes.create_string_buffer(4096)
        self._lib.sinv_last_error(self._h, buf, len(buf))
        return buf.value.decode(errors="replace")

    def _check(self, st):
        if st != 0:
            raise SinvError(st, self.last_error())

    def _t(self, t, name, numel=None, dtype=torch.float64):
        """A CUDA tensor of this object's device (else ValueError), as a pointer."""
        return _check_tensor(t, name, numel, dtype, self.device)

    def _s(self, stream):
        """The given stream (on this object's device) or that device's current one."""
        return _stream_ptr(stream, self.device)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sinv_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        s = _Stats()
        self._check(self._lib.sinv_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in _Stats._fields_}

    def pattern_host(self):
        rp = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(max(self.nnz_S, 1), dtype=np.int32)
        self._check(self._lib.sinv_get_pattern_host(self._h, _np_ptr(rp), _np_ptr(col)))
        return rp, col[: self.nnz_S]

    def pattern_device_ptrs(self):
        rp, col, nnz = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
        self._check(self._lib.sinv_get_pattern(self._h, ctypes.byref(rp), ctypes.byref(col), ctypes.byref(nnz)))
        return rp.value, col.value, nnz.value

    def supernodes(self):
        a, b, c = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
        self._check(self._lib.sinv_get_supernodes(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        ns = c.value
        start = np.ctypeslib.as_array(ctypes.cast(a, ctypes.POINTER(ctypes.c_int32)), shape=(ns + 1,)).copy()
        level = np.ctypeslib.as_array(ctypes.cast(b, ctypes.POINTER(ctypes.c_int32)), shape=(max(ns, 1),))[:ns].copy()
        return start, level

    def _out(self, out):
        if out is None:
            out = torch.empty(self.nnz_S, dtype=torch.float64, device=self.device)
        return out

    # -- numeric calls -----------------------------------------------------
    def selinv(self, L_val, D_val, prec="fp64", out=None, stream=None):
        out = self._out(out)
        self._check(self._lib.sinv_selinv(self._h, self._t(L_val, "L_val", self.nnz_L),
                                          self._t(D_val, "D_val", self.nD), PREC[prec],
                                          self._t(out, "G_S", self.nnz_S), self._s(stream)))
        return out

    def ninv(self, L_val, D_val, m, prec="fp64", out=None, stream=None, delta=0.0):
        """NInv on S; delta > 0 drops off-diagonal |w| < delta after every Horner step."""
        out = self._out(out)
        Lp = self._t(L_val, "L_val", self.nnz_L)
        Dp = self._t(D_val, "D_val", self.nD)
        Np = self._t(out, "N_S", self.nnz_S)
        if delta:
            st = self._lib.sinv_ninv_drop(self._h, Lp, Dp, int(m), float(delta), PREC[prec], Np, self._s(stream))
        else:
            st = self._lib.sinv_ninv(self._h, Lp, Dp, int(m), PREC[prec], Np, self._s(stream))
        self._check(st)
        return out

    def mix(self, G, N, eps, out=None, stream=None):
        out = self._out(out)
        self._check(self._lib.sinv_mix(self._h, self._t(G, "G_S", self.nnz_S),
                                       self._t(N, "N_S", self.nnz_S), float(eps),
                                       self._t(out, "M_S", self.nnz_S), self._s(stream)))
        return out

    def spai_analyse(self, A, power=0, warp_entries=0):
        """Analyse the pattern of the symmetric matrix A (scipy sparse) for spai(): the
        refinement pattern P = S widened to graph distance <= power in A.  Returns the
        CSR A (int64 rowptr, int32 indices) whose value order spai() takes.
        warp_entries: cap on the entries of a warp-solved column (0 = default)."""
        import scipy.sparse as sp
        A = sp.csr_matrix(A)
        A.sum_duplicates()
        rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
        col = np.ascontiguousarray(A.indices, dtype=np.int32)
        self._check(self._lib.sinv_spai_analyse(self._h, int(A.nnz), _np_ptr(rp), _np_ptr(col), int(power),
                                                int(warp_entries)))
        self._spai_nnzA = int(A.nnz)
        self.nnz_P = self.stats()["spai_nnz_P"]
        return sp.csr_matrix((A.data, col, rp), shape=A.shape)

    def spai_pattern(self):
        """(rowptr int64[n+1], col int32[|P_lo|]) of the SPAI pattern P_lo (host)."""
        rp = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(max(self.nnz_P, 1), dtype=np.int32)
        self._check(self._lib.sinv_spai_pattern(self._h, _np_ptr(rp), _np_ptr(col)))
        return rp, col[: self.nnz_P]

    def spai(self, A_val, X, iters, out=None, stream=None):
        """SPAI refinement of X (on S) over the analysed pattern P: result on P_lo
        (Mix-SPAI when X is Mix).  A_val in the order of the matrix spai_analyse returned."""
        nP = getattr(self, "nnz_P", None)
        if out is None:
            out = torch.empty(nP or 0, dtype=torch.float64, device=self.device)
        self._check(self._lib.sinv_spai(self._h, self._t(A_val, "A_val", getattr(self, "_spai_nnzA", None)),
                                        self._t(X, "X_S", self.nnz_S), int(iters),
                                        self._t(out, "Y_P", nP), self._s(stream)))
        return out

    def spai_analyse_mix_own(self, A, warp_entries=0):
        """Analyse A (scipy sparse) for spai_mix_own(): the refinement pattern is the one
        of the current mix_own result.  Returns the CSR A whose value order it takes."""
        import scipy.sparse as sp
        A = sp.csr_matrix(A)
        A.sum_duplicates()
        rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
        col = np.ascontiguousarray(A.indices, dtype=np.int32)
        self._check(self._lib.sinv_spai_analyse_mix_own(self._h, int(A.nnz), _np_ptr(rp), _np_ptr(col),
                                                        int(warp_entries)))
        self._spai_nnzA = int(A.nnz)
        self.nnz_P = self.stats()["spai_nnz_P"]
        return sp.csr_matrix((A.data, col, rp), shape=A.shape)

    def spai_mix_own(self, A_val, iters, X=None, out=None, stream=None):
        """Mix-SPAI over the pattern of the current mix_own result, from its values (or
        from X, given in the order of mix_own_result): result on P_lo."""
        nP = getattr(self, "nnz_P", None)
        if out is None:
            out = torch.empty(nP or 0, dtype=torch.float64, device=self.device)
        xp = None if X is None else self._t(X, "X_M")
        self._check(self._lib.sinv_spai_mix_own(self._h, self._t(A_val, "A_val",
                                                                       getattr(self, "_spai_nnzA", None)),
                                                xp, int(iters), self._t(out, "Y_P", nP), self._s(stream)))
        return out

    def einv_analyse(self, A):
        """Analyse the pattern of the symmetric matrix A (scipy sparse) for einv_lanczos();
        returns the CSR A whose value order einv_lanczos() takes."""
        import scipy.sparse as sp
        A = sp.csr_matrix(A)
        A.sum_duplicates()
        rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
        col = np.ascontiguousarray(A.indices, dtype=np.int32)
        self._check(self._lib.sinv_einv_analyse(self._h, int(A.nnz), _np_ptr(rp), _np_ptr(col)))
        self._einv_nnzA = int(A.nnz)
        return sp.csr_matrix((A.data, col, rp), shape=A.shape)

    def einv_set_solver(self, solver, grid_solve=False):
        """Inner solver of einv_lanczos: "cg" (A SPD) or "minres" (L |D| L^T, indefinite A);
        grid_solve forces the persistent multi-CTA triangular solves."""
        self._check(self._lib.sinv_einv_set_solver(self._h, {"cg": 0, "minres": 1}[solver] | (2 if grid_solve else 0)))

    def einv_lanczos(self, A_val, L_val, D_val, X, q0, k, steps, cg_tol=1e-12, cg_maxit=1000, stream=None):
        """k dominant eigenpairs of E_inv = A^{-1} - A^inv (A^inv = X on S): returns
        (lambda numpy[k], V tensor [n, k], info dict)."""
        lam = np.zeros(int(k), dtype=np.float64)
        info = np.zeros(3, dtype=np.int32)
        V = torch.empty((self.n, int(k)), dtype=torch.float64, device=self.device)
        self._check(self._lib.sinv_einv_lanczos(
            self._h, self._t(A_val, "A_val", getattr(self, "_einv_nnzA", None)),
            self._t(L_val, "L_val", self.nnz_L), self._t(D_val, "D_val", self.nD),
            self._t(X, "X_S", self.nnz_S), self._t(q0, "q0", self.n), int(steps), float(cg_tol),
            int(cg_maxit), int(k), _np_ptr(lam), self._t(V, "V", self.n * int(k)), _np_ptr(info),
            self._s(stream)))
        return lam, V, {"steps": int(info[0]), "cg_iterations": int(info[1]), "cg_unconverged": int(info[2])}

    def lowrank_correct(self, V, lam, X, prec="fp64", stream=None):
        k = int(lam.numel())
        self._check(self._lib.sinv_lowrank_correct(self._h, k, self._t(V, "V", self.n * k),
                                                   self._t(lam, "lambda", k), PREC[prec],
                                                   self._t(X, "X_S", self.nnz_S), self._s(stream)))
        return X

    def ninv_own(self, L_val, D_val, m, delta, stream=None, copy=True):
        """NInv on its own pattern: (colptr, rows, values) of the lower triangle in CSC
        (CUDA tensors) and the nnz of W after every Horner step; copy=False leaves the
        result in the handle and returns (None, None, None, steps)."""
        self._check(self._lib.sinv_ninv_own(self._h, self._t(L_val, "L_val"), self._t(D_val, "D_val"),
                                            int(m), float(delta), self._s(stream)))
        nnz = ctypes.c_int64()
        steps = np.zeros(int(m) + 1, dtype=np.int64)
        self._check(self._lib.sinv_ninv_own_size(self._h, ctypes.byref(nnz), _np_ptr(steps), int(m) + 1))
        if not copy:
            self.own_nnz = int(nnz.value)
            return None, None, None, steps
        cp = torch.empty(self.n + 1, dtype=torch.int64, device=self.device)
        rows = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=self.device)
        vals = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=self.device)
        self._check(self._lib.sinv_ninv_own_copy(self._h, self._t(cp, "colptr", None, torch.int64),
                                                 self._t(rows, "rows", None, torch.int32),
                                                 self._t(vals, "vals"), self._s(stream)))
        return cp, rows[:nnz.value], vals[:nnz.value], steps

    def mix_own(self, G, eps, stream=None, copy=True):
        """Mix on the pattern of the last ninv_own: (colptr, rows, values) of the lower
        triangle in CSC (CUDA tensors); copy=False leaves the result in the handle."""
        self._check(self._lib.sinv_mix_own(self._h, self._t(G, "G", self.nnz_S), float(eps),
                                           self._s(stream)))
        return self.mix_own_result(stream) if copy else None

    def mix_own_nnz(self) -> int:
        nnz = ctypes.c_int64()
        self._check(self._lib.sinv_mix_own_size(self._h, ctypes.byref(nnz)))
        return int(nnz.value)

    def mix_own_result(self, stream=None):
        """The handle's current Mix on the own pattern (copies): (colptr, rows, values)."""
        nnz = ctypes.c_int64()
        self._check(self._lib.sinv_mix_own_size(self._h, ctypes.byref(nnz)))
        cp = torch.empty(self.n + 1, dtype=torch.int64, device=self.device)
        rows = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=self.device)
        vals = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=self.device)
        self._check(self._lib.sinv_mix_own_copy(self._h, self._t(cp, "colptr", None, torch.int64),
                                                self._t(rows, "rows", None, torch.int32),
                                                self._t(vals, "vals"), self._s(stream)))
        return cp, rows[:nnz.value], vals[:nnz.value]

    def lowrank_correct_mix_own(self, V, lam, prec="fp64", stream=None):
        """Add V diag(lam) V^T on the pattern of the last mix_own result (in place)."""
        k = int(lam.numel())
        self._check(self._lib.sinv_lowrank_correct_mix_own(self._h, k, self._t(V, "V", self.n * k),
                                                           self._t(lam, "lambda", k), PREC[prec],
                                                           self._s(stream)))

    def ninv_stack(self, L_val, D_val, m, prec="fp64", out=None, stream=None):
        """NInv on S for the truncations after 0..m terms: tensor [(m+1), |S_lo|]."""
        if out is None:
            out = torch.empty((m + 1) * self.nnz_S, dtype=torch.float64, device=self.device)
        self._check(self._lib.sinv_ninv_stack(self._h, self._t(L_val, "L_val", self.nnz_L),
                                              self._t(D_val, "D_val", self.nD), int(m), PREC[prec],
                                              self._t(out, "N_stack", (m + 1) * self.nnz_S),
                                              self._s(stream)))
        return out.view(m + 1, self.nnz_S)

    def mlp_features(self, N_stack, m, L_val, D_val, stream=None):
        """(X [|S_lo| x 16] bfloat16, scale [|S_lo|] float32) for the learned correction."""
        X = torch.empty((self.nnz_S, MLP_F), dtype=torch.bfloat16, device=self.device)
        sc = torch.empty(self.nnz_S, dtype=torch.float32, device=self.device)
        self._check(self._lib.sinv_mlp_features(
            self._h, self._t(N_stack.reshape(-1), "N_stack", (m + 1) * self.nnz_S), int(m),
            self._t(L_val, "L_val", self.nnz_L), self._t(D_val, "D_val", self.nD),
            self._t(X, "X", None, torch.bfloat16), self._t(sc, "scale", None, torch.float32),
            self._s(stream)))
        return X, sc

    def sync_status(self, stream=None):
        self._check(self._lib.sinv_sync_status(self._h, self._s(stream)))

    def trace(self, enable=True):
        """Turn per-kernel event timing on or off."""
        self._check(self._lib.sinv_trace_enable(self._h, int(bool(enable))))

    def trace_read(self, reset=True) -> dict:
        """{kernel name: (launches, total ms)} since the last reset (waits for the events)."""
        buf = (_KTime * 64)()
        cnt = ctypes.c_int()
        self._check(self._lib.sinv_trace_read(self._h, buf, 64, ctypes.byref(cnt), int(bool(reset))))
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(cnt.value)}

    def timeline(self, enable=True):
        """Record the per-supernode timeline of the following selinv calls."""
        self._check(self._lib.sinv_timeline_enable(self._h, 1 if enable else 0))

    def timeline_read(self, stream=None) -> np.ndarray:
        """[n_supernodes, 4] uint64 globaltimer stamps (ns) of the last selinv: start,
        dependencies published, contraction done, published."""
        ns = int(self.stats()["n_supernodes"])
        out = np.zeros((ns, 4), dtype=np.uint64)
        self._check(self._lib.sinv_timeline_read(self._h, _np_ptr(out), ns, self._s(stream)))
        return out

    def selinv_scan_counts(self, stream=None):
        """(lookups, pairs) of the last selinv run with the timeline enabled (scan form)."""
        lk, pr = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.sinv_selinv_scan_counts(self._h, ctypes.byref(lk), ctypes.byref(pr),
                                                      self._s(stream)))
        return int(lk.value), int(pr.value)

    def debug_corrupt_plan(self) -> int:
        """Checked build only: plant an out-of-range SelInv pair position (status code)."""
        return int(self._lib.sinv_debug_corrupt_plan(self._h))

    def debug_wait_timeout(self, stream=None) -> int:
        return int(self._lib.sinv_debug_wait_timeout(self._h, self._s(stream)))
