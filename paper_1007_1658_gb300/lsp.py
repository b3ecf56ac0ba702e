"""ctypes binding of ``liblsp.so`` (include/lsp.h), argument marshalling only.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they are passed to
the C ABI as raw pointers.  Device tensors go through the library's
asynchronous device path on the current torch stream (or the stream given to
``Context``); host arrays go through its host path, which copies them in and
the result out.  Every step of the computation runs in the library's CUDA
kernels.  If the library has not been built, loading fails loudly: there is
no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblsp.so")
_lib = None
_lock = threading.Lock()

OK, ERR_INVALID_ARG, ERR_DEGENERATE, ERR_NONFINITE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NO_MODEL, \
    ERR_UNSUPPORTED = range(9)
SINCOS_AUTO, SINCOS_MUFU, SINCOS_RECUR, SINCOS_RECUR3, SINCOS_RECUR3_X2 = 0, 1, 2, 3, 4
PHASE_FIXED64, PHASE_NAIVE_FP32 = 0, 1

_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "DEGENERATE", 3: "NONFINITE", 4: "OOM", 5: "CUDA",
          6: "TIMEOUT", 7: "NO_MODEL", 8: "UNSUPPORTED"}


class LspError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_NAMES.get(status, status), msg))
        self.status = status


class lsp_options(ctypes.Structure):
    _fields_ = [("sincos_mode", ctypes.c_int32), ("phase_mode", ctypes.c_int32),
                ("freqs_per_thread", ctypes.c_int32), ("split", ctypes.c_int32),
                ("timing", ctypes.c_int32), ("mlp_fp32", ctypes.c_int32), ("batch_rhs", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


class lsp_pipe_rates(ctypes.Structure):
    _fields_ = [("sms", ctypes.c_int32), ("sm_mhz", ctypes.c_double), ("sincos_per_clk_sm", ctypes.c_double),
                ("ffma_per_clk_sm", ctypes.c_double), ("ffma2_lanes_per_clk_sm", ctypes.c_double)]


class lsp_train_report(ctypes.Structure):
    _fields_ = [("best_step", ctypes.c_int32), ("evaluations", ctypes.c_int32), ("val_loss_initial", ctypes.c_float),
                ("val_loss_best", ctypes.c_float), ("train_loss_last", ctypes.c_float), ("gpu_ms", ctypes.c_float)]


class lsp_train_opts(ctypes.Structure):
    _fields_ = [("n_pat", ctypes.c_int32), ("n_rows", ctypes.c_int32), ("features", ctypes.c_void_p),
                ("counts", ctypes.c_void_p), ("targets", ctypes.c_void_p), ("n_val_pat", ctypes.c_int32),
                ("n_val_real", ctypes.c_int32), ("val_features", ctypes.c_void_p), ("val_counts", ctypes.c_void_p),
                ("val_targets", ctypes.c_void_p), ("steps", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("warmup_steps", ctypes.c_int32), ("eval_every", ctypes.c_int32), ("lr", ctypes.c_float),
                ("lr_final", ctypes.c_float), ("weight_decay", ctypes.c_float), ("reserved0", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("val_history", ctypes.c_void_p), ("train_history", ctypes.c_void_p),
                ("report", ctypes.POINTER(lsp_train_report))]


def load():
    """Open liblsp.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblsp.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        p, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.lsp_default_options.argtypes = [ctypes.POINTER(lsp_options)]
        lib.lsp_default_options.restype = None
        lib.lsp_create.argtypes = [ctypes.POINTER(p), ctypes.c_int, ctypes.POINTER(lsp_options), p]
        lib.lsp_set_options.argtypes = [p, ctypes.POINTER(lsp_options)]
        lib.lsp_set_stream.argtypes = [p, p]
        lib.lsp_periodogram.argtypes = [p, p, p, i64, d, d, i64, p]
        lib.lsp_periodogram_gls.argtypes = [p, p, p, p, i64, d, d, i64, p]
        lib.lsp_press_rybicki.argtypes = [p, p, p, i64, d, d, i64, i32, p]
        lib.lsp_batch_gls.argtypes = [p, i32, p, p, p, p, p, p, p, p, p, p, p]
        lib.lsp_grid.argtypes = [d, d, i64, d, d, p, p, p]
        lib.lsp_sync.argtypes = [p, d]
        lib.lsp_last_timing.argtypes = [p, p, p, p]
        lib.lsp_last_launch_count.argtypes = [p]
        lib.lsp_last_launch_count.restype = i32
        lib.lsp_last_error.argtypes = [p]
        lib.lsp_last_error.restype = ctypes.c_char_p
        lib.lsp_destroy.argtypes = [p]
        lib.lsp_destroy.restype = None
        for name in ("lsp_create", "lsp_set_options", "lsp_set_stream", "lsp_periodogram", "lsp_grid",
                     "lsp_sync", "lsp_last_timing"):
            getattr(lib, name).restype = ctypes.c_int
        _extra_prototypes(lib)
        _lib = lib
        return lib


def _extra_prototypes(lib):
    """Prototypes of entry points added beside the single-curve path."""
    p, i32, i64, d, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
    if hasattr(lib, "lsp_periodogram_noalloc"):
        lib.lsp_periodogram_noalloc.argtypes = [p, p, i64, d, d, i64, p, p]
        lib.lsp_periodogram_noalloc.restype = ctypes.c_int
    if hasattr(lib, "lsp_batch"):
        lib.lsp_batch.argtypes = [p, i32, p, p, p, u64, i32, p, p, p, p, p, p, p]
        lib.lsp_batch.restype = ctypes.c_int
    if hasattr(lib, "lsp_batch_gls_noise"):
        lib.lsp_batch_gls_noise.argtypes = [p, i32, p, p, p, u64, i32, p, p, p, p, p, p, p]
        lib.lsp_batch_gls_noise.restype = ctypes.c_int
    if hasattr(lib, "lsp_fap_features"):
        lib.lsp_fap_features.argtypes = [p, i32, p, p, p, p, p, p]
        lib.lsp_fap_init.argtypes = [p, i32, u64, i32, p]
        lib.lsp_fap_train_step.argtypes = [p, i32, p, i32, p, p, p, ctypes.c_float, p]
        lib.lsp_fap_train.argtypes = [p, ctypes.POINTER(lsp_train_opts)]
        lib.lsp_fap_train.restype = ctypes.c_int
        lib.lsp_fap_gradients.argtypes = [p, i32, p, p, p, p, p]
        lib.lsp_fap_eval.argtypes = [p, i32, p, p, p]
        lib.lsp_fap_predict.argtypes = [p, i32, p, p, p, p, p, p]
        lib.lsp_fap_get_params.argtypes = [p, p, i64, ctypes.POINTER(ctypes.c_int64)]
        lib.lsp_fap_set_params.argtypes = [p, i32, p, i64]
        lib.lsp_fap_save.argtypes = [p, ctypes.c_char_p]
        lib.lsp_fap_load.argtypes = [p, ctypes.c_char_p]
        for name in ("lsp_fap_features", "lsp_fap_init", "lsp_fap_train_step", "lsp_fap_gradients", "lsp_fap_eval",
                     "lsp_fap_predict", "lsp_fap_get_params", "lsp_fap_set_params", "lsp_fap_save", "lsp_fap_load"):
            getattr(lib, name).restype = ctypes.c_int
    if hasattr(lib, "lsp_autotune"):
        lib.lsp_autotune.argtypes = [p, i64, i64, ctypes.POINTER(lsp_options)]
        lib.lsp_autotune.restype = ctypes.c_int
        lib.lsp_autotune_batch.argtypes = [p, i32, p, p, p, p, p, i32, ctypes.POINTER(lsp_options)]
        lib.lsp_autotune_batch.restype = ctypes.c_int
        lib.lsp_tune_save.argtypes = [p, ctypes.c_char_p]
        lib.lsp_tune_save.restype = ctypes.c_int
        lib.lsp_tune_load.argtypes = [p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32)]
        lib.lsp_tune_load.restype = ctypes.c_int
    if hasattr(lib, "lsp_probe_pipes"):
        lib.lsp_probe_pipes.argtypes = [p, ctypes.POINTER(lsp_pipe_rates)]
        lib.lsp_probe_pipes.restype = ctypes.c_int
    if hasattr(lib, "lsp_noise"):
        lib.lsp_noise.argtypes = [p, u64, i32, i32, i64, p]
        lib.lsp_noise.restype = ctypes.c_int
    if hasattr(lib, "lsp_test_pointer_kind"):
        lib.lsp_test_pointer_kind.argtypes = [i32, i32, i32]
        lib.lsp_test_pointer_kind.restype = i32
        lib.lsp_test_fail_allocation.argtypes = [p, i32]
        lib.lsp_test_fail_allocation.restype = ctypes.c_int
        lib.lsp_test_last_batch_shape.argtypes = [p, p]
        lib.lsp_test_last_batch_shape.restype = ctypes.c_int


def options(**kw) -> lsp_options:
    o = lsp_options()
    load().lsp_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


def _like(ref, shape, dtype):
    """An output array on the same side (device tensor / numpy) as `ref`."""
    if hasattr(ref, "data_ptr"):
        import torch
        return torch.empty(shape, dtype={np.float32: torch.float32, np.int32: torch.int32}[dtype], device=ref.device)
    return np.empty(shape, dtype=dtype)


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("array must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(a))


class Context:
    """Owns an lsp_ctx.  ``stream``: a torch.cuda.Stream, a raw cudaStream_t
    (int), or None for the current torch stream at each call."""

    def __init__(self, device: int = 0, stream=None, **opts):
        self._lib = load()
        self.device = int(device)
        self._stream = stream
        h = ctypes.c_void_p()
        o = options(**opts)
        st = self._lib.lsp_create(ctypes.byref(h), self.device, ctypes.byref(o), self._raw_stream())
        if st != OK:
            raise LspError(st, "lsp_create failed")
        self.h = h

    def _raw_stream(self):
        s = self._stream
        if s is None:
            try:
                import torch
                if torch.cuda.is_available():
                    s = torch.cuda.current_stream(self.device)
            except Exception:
                s = None
            if s is None:
                return None
        h = s.cuda_stream if hasattr(s, "cuda_stream") else int(s)
        # handle 0 is the legacy default stream; pass it as cudaStreamLegacy
        # (0x1) because a NULL stream means "the context's own stream"
        return ctypes.c_void_p(h if h else 1)

    def _check(self, st):
        if st != OK:
            raise LspError(st, self._lib.lsp_last_error(self.h).decode())

    def _bind_stream(self):
        self._check(self._lib.lsp_set_stream(self.h, self._raw_stream()))

    def set_options(self, **opts):
        o = options(**opts)
        self._check(self._lib.lsp_set_options(self.h, ctypes.byref(o)))

    def periodogram(self, t, X, f0, df, nf, out=None):
        """P[k] = P_n(f0 + k df), k < nf (Eq. 1-2 via Eq. 5-8)."""
        nf = int(nf)
        if out is None:
            if hasattr(t, "data_ptr"):
                import torch
                out = torch.empty(nf, dtype=torch.float32, device=t.device)
            else:
                out = np.empty(nf, dtype=np.float32)
        self._bind_stream()
        n = t.numel() if hasattr(t, "numel") else t.size
        self._check(self._lib.lsp_periodogram(self.h, _ptr(t), _ptr(X), int(n), float(f0), float(df), nf,
                                              _ptr(out)))
        return out

    def periodogram_gls(self, t, X, f0, df, nf, dy=None, out=None):
        """Floating-mean periodogram, P[k] = (N_t/2) p(f0 + k df) with weights 1/dy^2
        (equal weights when dy is None); lsp_periodogram_gls."""
        nf = int(nf)
        if out is None:
            if hasattr(t, "data_ptr"):
                import torch
                out = torch.empty(nf, dtype=torch.float32, device=t.device)
            else:
                out = np.empty(nf, dtype=np.float32)
        self._bind_stream()
        n = t.numel() if hasattr(t, "numel") else t.size
        self._check(self._lib.lsp_periodogram_gls(self.h, _ptr(t), _ptr(X), _ptr(dy), int(n), float(f0), float(df),
                                                  nf, _ptr(out)))
        return out

    def press_rybicki(self, t, X, f0, df, nf, macc=4, out=None):
        """Press-Rybicki fast approximate P_n at f0 + k df (f0 a multiple of df)."""
        nf = int(nf)
        if out is None:
            if hasattr(t, "data_ptr"):
                import torch
                out = torch.empty(nf, dtype=torch.float32, device=t.device)
            else:
                out = np.empty(nf, dtype=np.float32)
        self._bind_stream()
        n = t.numel() if hasattr(t, "numel") else t.size
        self._check(self._lib.lsp_press_rybicki(self.h, _ptr(t), _ptr(X), int(n), float(f0), float(df), nf,
                                                int(macc), _ptr(out)))
        return out

    def batch_gls(self, t_off, t, X, f0, df, nf, dy=None, P_out=None, P_off=None, maxP=None, argmax=None):
        """lsp_batch_gls: floating-mean periodograms of many curves (CSR t_off/t/X/dy,
        per-curve grids).  A missing maxP/argmax is allocated like t and returned."""
        n = int(nf.numel() if hasattr(nf, "numel") else len(nf))
        if maxP is None and argmax is None and P_out is None:
            maxP = _like(t, (n,), np.float32)
            argmax = _like(t, (n,), np.int32)
        self._bind_stream()
        self._check(self._lib.lsp_batch_gls(self.h, n, _ptr(t_off), _ptr(t), _ptr(X), _ptr(dy), _ptr(f0), _ptr(df),
                                            _ptr(nf), _ptr(P_out), _ptr(P_off), _ptr(maxP), _ptr(argmax)))
        return maxP, argmax

    def batch_gls_noise(self, t_off, t, f0, df, nf, dy=None, seed=0, n_real=1, P_out=None, P_off=None,
                        maxP=None, argmax=None):
        """lsp_batch_gls_noise: n_real floating-mean noise periodograms per curve
        (X = dy z, z the Philox N(0,1) values of lsp_batch).  A missing maxP/argmax
        is allocated like t and returned."""
        n = int(nf.numel() if hasattr(nf, "numel") else len(nf))
        if maxP is None and argmax is None and P_out is None:
            maxP = _like(t, (n_real * n,), np.float32)
            argmax = _like(t, (n_real * n,), np.int32)
        self._bind_stream()
        self._check(self._lib.lsp_batch_gls_noise(self.h, n, _ptr(t_off), _ptr(t), _ptr(dy), ctypes.c_uint64(int(seed)),
                                                  int(n_real), _ptr(f0), _ptr(df), _ptr(nf), _ptr(P_out),
                                                  _ptr(P_off), _ptr(maxP), _ptr(argmax)))
        return maxP, argmax

    def batch(self, t_off, t, f0, df, nf, X=None, seed=0, n_real=1, P_out=None, P_off=None,
              maxP=None, argmax=None):
        """lsp_batch: many curves (CSR t_off/t), per-curve grids f0/df/nf; X None =
        Philox noise (n_real realizations).  Outputs are filled in place; a
        missing maxP/argmax is allocated on t's device (or host) and returned."""
        n = int(nf.numel() if hasattr(nf, "numel") else len(nf))
        if maxP is None and argmax is None and P_out is None:
            if hasattr(t, "data_ptr"):
                import torch
                maxP = torch.empty(n_real * n, dtype=torch.float32, device=t.device)
                argmax = torch.empty(n_real * n, dtype=torch.int32, device=t.device)
            else:
                maxP = np.empty(n_real * n, dtype=np.float32)
                argmax = np.empty(n_real * n, dtype=np.int32)
        self._bind_stream()
        self._check(self._lib.lsp_batch(self.h, n, _ptr(t_off), _ptr(t), _ptr(X), ctypes.c_uint64(int(seed)),
                                        int(n_real), _ptr(f0), _ptr(df), _ptr(nf), _ptr(P_out), _ptr(P_off),
                                        _ptr(maxP), _ptr(argmax)))
        return maxP, argmax

    def noise(self, seed, curve, real, n, out=None):
        """lsp_noise: the raw N(0,1) values lsp_batch draws for (seed, curve, real)."""
        if out is None:
            out = np.empty(int(n), dtype=np.float32)
        self._bind_stream()
        self._check(self._lib.lsp_noise(self.h, ctypes.c_uint64(int(seed)), int(curve), int(real), int(n), _ptr(out)))
        return out

    def autotune(self, n_t, n_f):
        """lsp_autotune: returns the chosen options as a dict."""
        o = lsp_options()
        self._bind_stream()
        self._check(self._lib.lsp_autotune(self.h, int(n_t), int(n_f), ctypes.byref(o)))
        return {"sincos_mode": o.sincos_mode, "freqs_per_thread": o.freqs_per_thread, "split": o.split}

    def autotune_batch(self, t_off, t, f0, df, nf, n_real=1):
        """lsp_autotune_batch on this batch description: the chosen options as a dict."""
        o = lsp_options()
        n = int(nf.numel() if hasattr(nf, "numel") else len(nf))
        self._bind_stream()
        self._check(self._lib.lsp_autotune_batch(self.h, n, _ptr(t_off), _ptr(t), _ptr(f0), _ptr(df), _ptr(nf),
                                                 int(n_real), ctypes.byref(o)))
        return {"sincos_mode": o.sincos_mode, "freqs_per_thread": o.freqs_per_thread, "batch_rhs": o.batch_rhs}

    def tune_save(self, path):
        """lsp_tune_save: the tuning table as JSON."""
        self._check(self._lib.lsp_tune_save(self.h, str(path).encode()))

    def tune_load(self, path):
        """lsp_tune_load: merge a tuning file; returns the number of entries taken."""
        n = ctypes.c_int32(0)
        self._check(self._lib.lsp_tune_load(self.h, str(path).encode(), ctypes.byref(n)))
        return int(n.value)

    def test_last_batch_shape(self):
        """lsp_test_last_batch_shape: (mode, F, R, tail F, tile) of the last batch plan."""
        a = np.zeros(5, dtype=np.int32)
        self._check(self._lib.lsp_test_last_batch_shape(self.h, _ptr(a)))
        return tuple(int(x) for x in a)

    def probe_pipes(self):
        """lsp_probe_pipes: measured per-SM, per-clock pipe rates as a dict."""
        r = lsp_pipe_rates()
        self._bind_stream()
        self._check(self._lib.lsp_probe_pipes(self.h, ctypes.byref(r)))
        return {k: getattr(r, k) for k, _ in lsp_pipe_rates._fields_}

    # ---- learned false-alarm surrogate ----
    def fap_features(self, t_off, t, f0, df, nf, out=None):
        n = int(nf.numel() if hasattr(nf, "numel") else len(nf))
        if out is None:
            out = _like(t, (n, 32), np.float32)
        self._bind_stream()
        self._check(self._lib.lsp_fap_features(self.h, n, _ptr(t_off), _ptr(t), _ptr(f0), _ptr(df), _ptr(nf),
                                               _ptr(out)))
        return out

    def fap_init(self, features, hidden=256, seed=0):
        n = int(features.shape[0])
        self._bind_stream()
        self._check(self._lib.lsp_fap_init(self.h, int(hidden), ctypes.c_uint64(int(seed)), n, _ptr(features)))

    def fap_train_step(self, rows, features, counts, targets, lr, loss_out=None):
        self._bind_stream()
        self._check(self._lib.lsp_fap_train_step(self.h, int(rows.numel()), _ptr(rows), int(features.shape[0]),
                                                 _ptr(features), _ptr(counts), _ptr(targets), float(lr),
                                                 _ptr(loss_out)))

    def fap_train(self, features, counts, targets, val_features, val_counts, val_targets, steps, batch=4096,
                  lr=1e-3, lr_final=0.05, warmup_steps=0, weight_decay=0.0, eval_every=100, seed=0):
        """lsp_fap_train: the whole training loop in the library.  features/counts
        [n_pat][32]/[n_pat][2], targets [n_rows] (row r -> pattern r % n_pat),
        val_targets [n_val_real][n_val_pat]; all device tensors.  Returns the
        report as a dict with the validation and training-loss histories."""
        n_val_real = int(val_targets.shape[0]) if val_targets.dim() == 2 else 1
        passes = 2 + (int(steps) - 1) // int(eval_every) if eval_every > 0 else 2
        vh = np.full(passes, np.nan, dtype=np.float32)
        th = np.full(passes, np.nan, dtype=np.float32)
        rep = lsp_train_report()
        o = lsp_train_opts(n_pat=int(features.shape[0]), n_rows=int(targets.numel()), features=_ptr(features),
                           counts=_ptr(counts), targets=_ptr(targets), n_val_pat=int(val_features.shape[0]),
                           n_val_real=n_val_real, val_features=_ptr(val_features), val_counts=_ptr(val_counts),
                           val_targets=_ptr(val_targets), steps=int(steps), batch=int(batch),
                           warmup_steps=int(warmup_steps), eval_every=int(eval_every), lr=float(lr),
                           lr_final=float(lr_final), weight_decay=float(weight_decay), reserved0=0, seed=int(seed),
                           val_history=_ptr(vh), train_history=_ptr(th), report=ctypes.pointer(rep))
        self._bind_stream()
        self._check(self._lib.lsp_fap_train(self.h, ctypes.byref(o)))
        e = rep.evaluations
        d = {k: getattr(rep, k) for k, _ in lsp_train_report._fields_}
        d["val_history"] = vh[:e].tolist()
        d["train_history"] = th[:e].tolist()
        return d

    def fap_gradients(self, features, counts, targets):
        B = int(features.shape[0])
        n = ctypes.c_int64()
        self._check(self._lib.lsp_fap_get_params(self.h, None, 0, ctypes.byref(n)))
        g = np.empty(int(n.value) - 64, dtype=np.float32)
        loss = np.empty(1, dtype=np.float32)
        self._bind_stream()
        self._check(self._lib.lsp_fap_gradients(self.h, B, _ptr(features), _ptr(counts), _ptr(targets), _ptr(g),
                                                _ptr(loss)))
        return g, float(loss[0])

    def fap_eval(self, features, counts, out=None):
        B = int(features.shape[0])
        if out is None:
            out = _like(features, (B, 9), np.float32)
        self._bind_stream()
        self._check(self._lib.lsp_fap_eval(self.h, B, _ptr(features), _ptr(counts), _ptr(out)))
        return out

    def fap_predict(self, t_off, t, f0, df, nf, out=None):
        n = int(nf.numel() if hasattr(nf, "numel") else len(nf))
        if out is None:
            out = _like(t, (n, 9), np.float32)
        self._bind_stream()
        self._check(self._lib.lsp_fap_predict(self.h, n, _ptr(t_off), _ptr(t), _ptr(f0), _ptr(df), _ptr(nf),
                                              _ptr(out)))
        return out

    def fap_get_params(self):
        n = ctypes.c_int64()
        self._check(self._lib.lsp_fap_get_params(self.h, None, 0, ctypes.byref(n)))
        out = np.empty(int(n.value), dtype=np.float32)
        self._check(self._lib.lsp_fap_get_params(self.h, _ptr(out), out.size, ctypes.byref(n)))
        return out

    def fap_set_params(self, flat, hidden=256):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(self._lib.lsp_fap_set_params(self.h, int(hidden), _ptr(flat), flat.size))

    def fap_save(self, path):
        self._check(self._lib.lsp_fap_save(self.h, str(path).encode()))

    def fap_load(self, path):
        self._check(self._lib.lsp_fap_load(self.h, str(path).encode()))

    def test_fail_allocation(self, n):
        """lsp_test_fail_allocation: the n-th workspace allocation from now fails (0 cancels)."""
        self._check(self._lib.lsp_test_fail_allocation(self.h, int(n)))

    def sync(self, timeout_s: float = -1.0):
        self._check(self._lib.lsp_sync(self.h, float(timeout_s)))

    def last_timing(self):
        a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        self._check(self._lib.lsp_last_timing(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def last_launch_count(self) -> int:
        return int(self._lib.lsp_last_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self._lib.lsp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def periodogram_noalloc(t, X, f0, df, nf, out, stream=None):
    """lsp_periodogram_noalloc: device tensors only, no context, nothing allocated
    by the library (the caller provides `out`).  Queued on `stream` (a
    torch.cuda.Stream or raw handle; None = current torch stream)."""
    lib = load()
    if stream is None:
        import torch
        raw = torch.cuda.current_stream().cuda_stream
    else:
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    raw = raw if raw else 1  # the legacy default stream
    st = lib.lsp_periodogram_noalloc(_ptr(t), _ptr(X), int(t.numel()), float(f0), float(df), int(nf), _ptr(out),
                                     ctypes.c_void_p(raw))
    if st != OK:
        raise LspError(st, "lsp_periodogram_noalloc")
    return out


def pointer_kind(memory_type, pointer_device, device):
    """lsp_test_pointer_kind: 0 host (staged), 1 used in place, 2 another GPU (refused)."""
    return int(load().lsp_test_pointer_kind(int(memory_type), int(pointer_device), int(device)))


def grid(t_min, t_max, n, f_over, f_high):
    """Eq. 9-11 grid: (f0, df, nf) with f0 = df."""
    f0, df, nf = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    st = load().lsp_grid(float(t_min), float(t_max), int(n), float(f_over), float(f_high),
                         ctypes.byref(f0), ctypes.byref(df), ctypes.byref(nf))
    if st != OK:
        raise LspError(st, "lsp_grid")
    return f0.value, df.value, nf.value
