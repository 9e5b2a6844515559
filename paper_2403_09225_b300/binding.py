"""ctypes binding of libpwa (include/pwa.h): argument marshalling only.

Every function of the C ABI is exposed under its own name; ``Likelihood`` is a
thin owner of one handle.  All arithmetic of the likelihood runs in the CUDA
library; there is no Python or CPU fallback: importing this module on a
machine without the built library raises, and every call checks the status
the library returns.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpwa.so")

PWA_OK, PWA_EINVAL, PWA_ENOMEM, PWA_ECUDA, PWA_ENONFINITE, PWA_ENOCONV, PWA_ETIMEOUT = range(7)
STATUS_NAMES = {0: "PWA_OK", 1: "PWA_EINVAL", 2: "PWA_ENOMEM", 3: "PWA_ECUDA", 4: "PWA_ENONFINITE",
                5: "PWA_ENOCONV", 6: "PWA_ETIMEOUT"}
FIT_STATUS_NAMES = ("xtol", "gtol", "maxiter", "time_limit", "linesearch_failed", "precision_limit", "error")


class pwa_events(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m2", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("F", ctypes.c_void_p), ("on_device", ctypes.c_int)]


class pwa_resonance(ctypes.Structure):
    _fields_ = [("channel", ctypes.c_int), ("spin", ctypes.c_int), ("mass", ctypes.c_double),
                ("width", ctypes.c_double), ("mag", ctypes.c_double), ("phase", ctypes.c_double),
                ("fix_coupling", ctypes.c_int), ("fix_mass", ctypes.c_int), ("fix_width", ctypes.c_int)]


class pwa_fit_iter(ctypes.Structure):
    _fields_ = [("nll", ctypes.c_double), ("grad_max", ctypes.c_double), ("cg_eps", ctypes.c_double),
                ("cg_res", ctypes.c_double), ("step", ctypes.c_double), ("dir_deriv", ctypes.c_double),
                ("cg_iters", ctypes.c_int), ("cg_exit", ctypes.c_int), ("n_fev", ctypes.c_int),
                ("hessian", ctypes.c_int)]


class pwa_fit_opts(ctypes.Structure):
    _fields_ = [("xtol", ctypes.c_double), ("gtol", ctypes.c_double), ("maxiter", ctypes.c_int),
                ("cg_maxiter", ctypes.c_int), ("time_limit_s", ctypes.c_double), ("matrix_free", ctypes.c_int),
                ("method", ctypes.c_int), ("trace_cap", ctypes.c_int), ("trace", ctypes.POINTER(pwa_fit_iter)),
                ("one_launch", ctypes.c_int)]


class pwa_lineshape(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ma", ctypes.c_double), ("mb", ctypes.c_double), ("mc", ctypes.c_double),
                ("md", ctypes.c_double), ("radius", ctypes.c_double), ("width2", ctypes.c_double)]


class pwa_fit_result(ctypes.Structure):
    _fields_ = [("nll", ctypes.c_double), ("grad_max", ctypes.c_double), ("iters", ctypes.c_int),
                ("n_hvp", ctypes.c_int), ("n_fev", ctypes.c_int), ("status", ctypes.c_int),
                ("elapsed_s", ctypes.c_double), ("n_trace", ctypes.c_int), ("n_hess", ctypes.c_int)]


_TRACE_KEYS = ("nll", "grad_max", "cg_eps", "cg_res", "step", "dir_deriv", "cg_iters", "cg_exit", "n_fev",
               "hessian")


def _attach_trace(opts: pwa_fit_opts, n_fits: int, cap: int):
    """Give opts a per-fit trace buffer of cap records (kept alive by the return value)."""
    if cap <= 0:
        return None
    buf = (pwa_fit_iter * (n_fits * cap))()
    opts.trace_cap = cap
    opts.trace = ctypes.cast(buf, ctypes.POINTER(pwa_fit_iter))
    return buf


def _read_trace(buf, cap: int, row: int, n: int):
    if buf is None:
        return None
    return [{k: getattr(buf[row * cap + i], k) for k in _TRACE_KEYS} for i in range(n)]


class PwaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


#: every symbol include/pwa.h declares
EXPORTS = ("pwa_create", "pwa_last_create_error", "pwa_num_params", "pwa_nll", "pwa_grad", "pwa_hvp", "pwa_hessian",
           "pwa_hessian_batch",
           "pwa_hvp_reuse", "pwa_hvp_reuse_device", "pwa_eval_multi_device", "pwa_set_hessian_cuda_cores",
           "pwa_release_event_copies",
           "pwa_device_bytes",
           "pwa_eval", "pwa_eval_device", "pwa_eval_device_noalloc", "pwa_eval_batch", "pwa_eval_batch_device",
           "pwa_sync", "pwa_event_intensity", "pwa_newton_cg_fit", "pwa_newton_cg_fit_batch",
           "pwa_newton_cg_fit_multi", "pwa_autotune", "pwa_coupling_create", "pwa_coupling_num_params",
           "pwa_coupling_integral_matrix", "pwa_coupling_eval", "pwa_coupling_fit", "pwa_coupling_destroy",
           "pwa_fit_opts_default", "pwa_set_stream", "pwa_set_tiling", "pwa_get_tiling",
           "pwa_selftest_bounded_wait", "pwa_last_error", "pwa_destroy", "pwa_mlp_create", "pwa_mlp_forward",
           "pwa_mlp_gradients", "pwa_mlp_train_step", "pwa_mlp_params", "pwa_mlp_gemm_check",
           "pwa_mlp_last_error", "pwa_mlp_destroy", "pwa_accept_reject", "pwa_dalitz_histogram",
           "pwa_gather_events", "pwa_last_generate_error", "pwa_variant_create", "pwa_variant_num_params",
           "pwa_variant_eval", "pwa_variant_eval_batch", "pwa_variant_fit", "pwa_variant_set_shapes", "pwa_variant_coupling_num_params",
           "pwa_variant_coupling_eval", "pwa_variant_coupling_fit", "pwa_variant_last_error", "pwa_variant_destroy")


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError("libpwa is not built (%s missing); run paper_2403_09225_b300/build.py" % path)
    lib = ctypes.CDLL(path)
    H, vp, dp, ip, i = ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), \
        ctypes.POINTER(ctypes.c_int), ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    st = ctypes.c_int
    sig = {
        "pwa_create": (st, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(pwa_events),
                            ctypes.POINTER(pwa_events), ctypes.POINTER(pwa_resonance), i, i, vp]),
        "pwa_last_create_error": (ctypes.c_char_p, []),
        "pwa_num_params": (i, [H]),
        "pwa_nll": (st, [H, dp, dp]),
        "pwa_grad": (st, [H, dp, dp, dp]),
        "pwa_hvp": (st, [H, dp, dp, dp]),
        "pwa_eval": (st, [H, dp, dp, dp, dp, dp]),
        "pwa_hessian": (st, [H, dp, dp, dp, dp]),
        "pwa_hessian_batch": (st, [H, i, dp, dp, dp, dp, ip]),
        "pwa_hvp_reuse": (st, [H, dp, dp, dp]),
        "pwa_eval_multi_device": (st, [i, ctypes.POINTER(ctypes.c_void_p), ip, ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), i, i, vp]),
        "pwa_hvp_reuse_device": (st, [H, vp, vp, vp]),
        "pwa_release_event_copies": (st, [H]),
        "pwa_set_hessian_cuda_cores": (st, [H, i]),
        "pwa_device_bytes": (st, [H, ctypes.POINTER(ctypes.c_longlong)]),
        "pwa_eval_device": (st, [H, vp, vp, vp, i, i]),
        "pwa_eval_device_noalloc": (st, [H, vp, vp, vp, i, i]),
        "pwa_eval_batch": (st, [H, i, dp, dp, dp, dp, dp]),
        "pwa_eval_batch_device": (st, [H, i, vp, vp, vp, i, i]),
        "pwa_sync": (st, [H]),
        "pwa_event_intensity": (st, [H, i, dp, vp, i]),
        "pwa_newton_cg_fit": (st, [H, dp, ctypes.POINTER(pwa_fit_opts), dp, ctypes.POINTER(pwa_fit_result)]),
        "pwa_newton_cg_fit_batch": (st, [H, i, dp, ctypes.POINTER(pwa_fit_opts), dp, ctypes.POINTER(pwa_fit_result)]),
        "pwa_newton_cg_fit_multi": (st, [i, ctypes.POINTER(ctypes.c_void_p), ip, ctypes.POINTER(dp),
                                         ctypes.POINTER(pwa_fit_opts), ctypes.POINTER(dp),
                                         ctypes.POINTER(ctypes.POINTER(pwa_fit_result))]),
        "pwa_autotune": (st, [H, dp, i, ip]),
        "pwa_coupling_create": (st, [H, dp, ctypes.POINTER(ctypes.c_void_p)]),
        "pwa_coupling_num_params": (i, [vp]),
        "pwa_coupling_integral_matrix": (st, [vp, dp]),
        "pwa_coupling_eval": (st, [vp, i, dp, dp, dp, dp, dp]),
        "pwa_coupling_fit": (st, [vp, i, dp, ctypes.POINTER(pwa_fit_opts), dp, ctypes.POINTER(pwa_fit_result)]),
        "pwa_coupling_destroy": (None, [vp]),
        "pwa_fit_opts_default": (None, [ctypes.POINTER(pwa_fit_opts)]),
        "pwa_set_stream": (st, [H, vp]),
        "pwa_set_tiling": (st, [H, i, i, i]),
        "pwa_get_tiling": (st, [H, ip]),
        "pwa_selftest_bounded_wait": (st, [ctypes.c_double]),
        "pwa_last_error": (ctypes.c_char_p, [H]),
        "pwa_destroy": (None, [H]),
        "pwa_mlp_create": (st, [i, i, i, i, i, ctypes.c_ulonglong, ip, fp, vp, ctypes.POINTER(ctypes.c_void_p)]),
        "pwa_mlp_forward": (st, [vp, i, vp, vp]),
        "pwa_mlp_gradients": (st, [vp, i, vp, vp, dp]),
        "pwa_mlp_train_step": (st, [vp, i, vp, vp, ctypes.c_float, dp]),
        "pwa_mlp_params": (st, [vp, i, i, fp, i]),
        "pwa_mlp_gemm_check": (st, [vp, i, i, i, fp, fp, fp]),
        "pwa_mlp_last_error": (ctypes.c_char_p, [vp]),
        "pwa_mlp_destroy": (None, [vp]),
        "pwa_accept_reject": (st, [vp, ctypes.c_longlong, ctypes.c_double, ctypes.c_ulonglong, ctypes.c_longlong, i,
                                   vp, ip, dp, vp]),
        "pwa_dalitz_histogram": (st, [vp, ctypes.c_longlong, vp, i, i, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, i, vp, vp]),
        "pwa_gather_events": (st, [vp, ctypes.c_longlong, vp, i, vp, i, vp, vp, vp]),
        "pwa_last_generate_error": (ctypes.c_char_p, []),
        "pwa_variant_create": (st, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(pwa_events),
                                    ctypes.POINTER(pwa_events), ctypes.POINTER(pwa_resonance),
                                    ctypes.POINTER(pwa_lineshape), i, i, i, vp]),
        "pwa_variant_num_params": (i, [vp]),
        "pwa_variant_eval": (st, [vp, dp, dp, dp, dp, dp]),
        "pwa_variant_eval_batch": (st, [vp, i, dp, dp, dp, dp, dp, ip]),
        "pwa_variant_fit": (st, [vp, i, dp, ctypes.POINTER(pwa_fit_opts), dp, ctypes.POINTER(pwa_fit_result)]),
        "pwa_variant_set_shapes": (st, [vp, dp, dp]),
        "pwa_variant_coupling_num_params": (i, [vp]),
        "pwa_variant_coupling_eval": (st, [vp, dp, dp, dp, dp, dp]),
        "pwa_variant_coupling_fit": (st, [vp, i, dp, ctypes.POINTER(pwa_fit_opts), dp, ctypes.POINTER(pwa_fit_result)]),
        "pwa_variant_last_error": (ctypes.c_char_p, [vp]),
        "pwa_variant_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(x, n: Optional[int] = None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _events(m2, F, w, keep: list) -> pwa_events:
    """pwa_events for numpy arrays (host) or torch CUDA tensors (device)."""
    if _is_torch(m2):
        import torch
        m2 = m2.contiguous().to(torch.float32)
        Fr = torch.view_as_real(F.contiguous()) if F.is_complex() else F.contiguous()
        Fr = Fr.to(torch.float32)
        wt = None if w is None else w.contiguous().to(torch.float32)
        keep.extend([m2, Fr, wt])
        dev = 1 if m2.is_cuda else 0
        return pwa_events(int(m2.shape[1]), m2.data_ptr(), 0 if wt is None else wt.data_ptr(), Fr.data_ptr(), dev)
    m2 = np.ascontiguousarray(m2, dtype=np.float32)
    Fv = np.ascontiguousarray(F)
    Fv = Fv.view(np.float32) if np.iscomplexobj(Fv) else np.ascontiguousarray(Fv, dtype=np.float32)
    wv = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    keep.extend([m2, Fv, wv])
    return pwa_events(int(m2.shape[1]), m2.ctypes.data, 0 if wv is None else wv.ctypes.data, Fv.ctypes.data, 0)


def resonance_table(table: Sequence) -> ctypes.Array:
    """pwa_resonance[K] from objects with channel, spin, mass, width, mag,
    phase, fix_coupling, fix_mass, fix_width attributes."""
    arr = (pwa_resonance * len(table))()
    for k, r in enumerate(table):
        arr[k] = pwa_resonance(int(r.channel), int(r.spin), float(r.mass), float(r.width), float(r.mag),
                               float(r.phase), int(bool(r.fix_coupling)), int(bool(r.fix_mass)),
                               int(bool(r.fix_width)))
    return arr


class Likelihood:
    """One libpwa handle: data + MC events and a resonance table."""

    def __init__(self, data, mc, table, K: int, S: int, stream: int = 0):
        """data, mc: objects with m2 [3, n], F [n, K, S] complex and w ([n] or
        None) as numpy arrays or torch CUDA tensors."""
        keep: list = []
        de = _events(data.m2, data.F, getattr(data, "w", None), keep)
        me = _events(mc.m2, mc.F, None, keep)
        tab = resonance_table(table)
        h = ctypes.c_void_p()
        st = lib().pwa_create(ctypes.byref(h), ctypes.byref(de), ctypes.byref(me), tab, int(K), int(S),
                              ctypes.c_void_p(stream))
        if st != PWA_OK:
            raise PwaError(st, lib().pwa_last_create_error().decode())
        self._h = h
        self.K, self.S = int(K), int(S)
        self.P = lib().pwa_num_params(h)
        self._n = (int(de.n), int(me.n))

    # -- plumbing --
    def _check(self, st: int):
        if st != PWA_OK:
            raise PwaError(st, lib().pwa_last_error(self._h).decode())

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().pwa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- evaluation (host vectors) --
    def nll(self, theta) -> float:
        th = _f64(theta, self.P)
        f = ctypes.c_double()
        self._check(lib().pwa_nll(self._h, _dptr(th), ctypes.byref(f)))
        return f.value

    def grad(self, theta):
        th = _f64(theta, self.P)
        f = ctypes.c_double()
        g = np.empty(self.P)
        self._check(lib().pwa_grad(self._h, _dptr(th), ctypes.byref(f), _dptr(g)))
        return f.value, g

    def hvp(self, theta, v) -> np.ndarray:
        th, vv = _f64(theta, self.P), _f64(v, self.P)
        hv = np.empty(self.P)
        self._check(lib().pwa_hvp(self._h, _dptr(th), _dptr(vv), _dptr(hv)))
        return hv

    def set_hessian_cuda_cores(self, on: bool):
        """Hessian Gram matrices on the CUDA cores even where tensor cores apply."""
        self._check(lib().pwa_set_hessian_cuda_cores(self._h, int(on)))

    def release_event_copies(self):
        """Free the caller-layout event copies (the tiling becomes fixed)."""
        self._check(lib().pwa_release_event_copies(self._h))

    def device_bytes(self) -> int:
        out = ctypes.c_longlong()
        self._check(lib().pwa_device_bytes(self._h, ctypes.byref(out)))
        return out.value

    def hvp_reuse(self, theta, v) -> np.ndarray:
        """H v reusing the sums of the last full H v pass at the same theta."""
        th = _f64(theta, self.P)
        vv = _f64(v, self.P)
        hv = np.empty(self.P)
        self._check(lib().pwa_hvp_reuse(self._h, _dptr(th), _dptr(vv), _dptr(hv)))
        return hv

    def hvp_reuse_device(self, d_theta: int, d_v: int, d_out: int):
        self._check(lib().pwa_hvp_reuse_device(self._h, d_theta, d_v, d_out))

    def hessian(self, theta):
        """(NLL, gradient [P], Hessian [P, P]) at theta from one Hessian pass."""
        th = _f64(theta, self.P)
        f = ctypes.c_double()
        g = np.empty(self.P)
        H = np.empty((self.P, self.P))
        self._check(lib().pwa_hessian(self._h, _dptr(th), ctypes.byref(f), _dptr(g), _dptr(H)))
        return f.value, g, H

    def hessian_batch(self, thetas):
        """(NLL [B], gradient [B, P], Hessian [B, P, P], status [B]) of B
        parameter vectors from one batched Hessian pass; status[b] is
        PWA_ENONFINITE for a vector with a non-finite intensity (its rows are
        then not written)."""
        th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(-1, self.P))
        B = th.shape[0]
        f = np.full(B, np.nan)
        g = np.full((B, self.P), np.nan)
        H = np.full((B, self.P, self.P), np.nan)
        stat = np.zeros(B, dtype=np.int32)
        self._check(lib().pwa_hessian_batch(self._h, B, _dptr(th), _dptr(f), _dptr(g), _dptr(H),
                                            stat.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return f, g, H, stat

    def eval(self, theta, v=None):
        """(NLL, grad, H v) from one fused pass; H v is None when v is None."""
        th = _f64(theta, self.P)
        f = ctypes.c_double()
        g = np.empty(self.P)
        if v is None:
            self._check(lib().pwa_eval(self._h, _dptr(th), None, ctypes.byref(f), _dptr(g), None))
            return f.value, g, None
        vv = _f64(v, self.P)
        hv = np.empty(self.P)
        self._check(lib().pwa_eval(self._h, _dptr(th), _dptr(vv), ctypes.byref(f), _dptr(g), _dptr(hv)))
        return f.value, g, hv

    def eval_batch(self, thetas, vs=None):
        """(NLL [B], grad [B, P], H v [B, P] or None) for B parameter vectors
        (rows of thetas) in one batched pass."""
        th = _f64(thetas).reshape(-1, self.P)
        B = th.shape[0]
        f = np.empty(B)
        g = np.empty((B, self.P))
        if vs is None:
            self._check(lib().pwa_eval_batch(self._h, B, _dptr(th), None, _dptr(f), _dptr(g), None))
            return f, g, None
        vv = _f64(vs).reshape(B, self.P)
        hv = np.empty((B, self.P))
        self._check(lib().pwa_eval_batch(self._h, B, _dptr(th), _dptr(vv), _dptr(f), _dptr(g), _dptr(hv)))
        return f, g, hv

    def eval_batch_device(self, B: int, d_theta: int, d_v: int, d_out: int, want_grad: bool = True,
                          want_hv: bool = True):
        """Asynchronous batched pass on device pointers (theta [B][P], v [B][P], out [B][1 + 2P])."""
        self._check(lib().pwa_eval_batch_device(self._h, int(B), ctypes.c_void_p(d_theta), ctypes.c_void_p(d_v),
                                                ctypes.c_void_p(d_out), int(want_grad), int(want_hv)))

    def eval_device(self, d_theta: int, d_v: int, d_out: int, want_grad: bool = True, want_hv: bool = True):
        """Asynchronous fused pass on device pointers (theta [P], v [P], out [1 + 2P])."""
        self._check(lib().pwa_eval_device(self._h, ctypes.c_void_p(d_theta), ctypes.c_void_p(d_v),
                                          ctypes.c_void_p(d_out), int(want_grad), int(want_hv)))

    def eval_device_noalloc(self, d_theta: int, d_v: int, d_out: int, want_grad: bool = True,
                            want_hv: bool = True):
        """eval_device with the reduction scratch in the library's static
        device array: allocates nothing (see include/pwa.h)."""
        self._check(lib().pwa_eval_device_noalloc(self._h, ctypes.c_void_p(d_theta), ctypes.c_void_p(d_v),
                                                  ctypes.c_void_p(d_out), int(want_grad), int(want_hv)))

    def sync(self):
        self._check(lib().pwa_sync(self._h))

    def set_stream(self, stream: int):
        self._check(lib().pwa_set_stream(self._h, ctypes.c_void_p(stream)))

    def intensity(self, theta, sample: int = 1, out=None) -> np.ndarray:
        """I(e) of the data (sample 0) or MC (sample 1) events, FP32.  With out
        a torch CUDA tensor the result is written there on the device."""
        th = _f64(theta, self.P)
        if out is not None and _is_torch(out):
            self._check(lib().pwa_event_intensity(self._h, int(sample), _dptr(th), ctypes.c_void_p(out.data_ptr()), 1))
            return out
        n = self.n_events(sample)
        res = np.empty(n, dtype=np.float32)
        self._check(lib().pwa_event_intensity(self._h, int(sample), _dptr(th), ctypes.c_void_p(res.ctypes.data), 0))
        return res

    def n_events(self, sample: int) -> int:
        return self._n[sample]

    # -- fitting --
    def fit(self, theta0, xtol: float = 1e-8, gtol: float = 0.0, maxiter: int = 0, cg_maxiter: int = 0,
            time_limit_s: float = 0.0, trace: int = 0, matrix_free: bool = False, method: int = 0):
        """Newton-CG fit from theta0; with trace > 0 the info dict carries the
        first `trace` outer iterations' records under "trace".  matrix_free:
        every CG step is one fused H v pass instead of a product with the
        outer iteration's Hessian (pwa_hessian).  method: 0 line search
        (the paper's), 1 trust region."""
        th = _f64(theta0, self.P)
        out = np.empty(self.P)
        opts = pwa_fit_opts(xtol, gtol, maxiter, cg_maxiter, time_limit_s, int(matrix_free), int(method))
        tbuf = _attach_trace(opts, 1, trace)
        res = pwa_fit_result()
        st = lib().pwa_newton_cg_fit(self._h, _dptr(th), ctypes.byref(opts), _dptr(out), ctypes.byref(res))
        if st not in (PWA_OK, PWA_ENOCONV):
            self._check(st)
        info = {"nll": res.nll, "grad_max": res.grad_max, "iters": res.iters, "n_hvp": res.n_hvp,
                "n_fev": res.n_fev, "n_hess": res.n_hess, "status": FIT_STATUS_NAMES[res.status], "elapsed_s": res.elapsed_s,
                "converged": st == PWA_OK}
        if tbuf is not None:
            info["trace"] = _read_trace(tbuf, trace, 0, res.n_trace)
        return out, info

    def fit_batch(self, thetas0, xtol: float = 1e-8, gtol: float = 0.0, maxiter: int = 0, cg_maxiter: int = 0,
                  time_limit_s: float = 0.0, trace: int = 0, matrix_free: bool = False, method: int = 0):
        """B fits (rows of thetas0) in lockstep with batched passes; returns
        (theta [B, P], list of per-fit info dicts, converged-or-time-limit for all)."""
        th = _f64(thetas0).reshape(-1, self.P)
        B = th.shape[0]
        out = np.empty((B, self.P))
        opts = pwa_fit_opts(xtol, gtol, maxiter, cg_maxiter, time_limit_s, int(matrix_free), int(method))
        tbuf = _attach_trace(opts, B, trace)
        res = (pwa_fit_result * B)()
        st = lib().pwa_newton_cg_fit_batch(self._h, B, _dptr(th), ctypes.byref(opts), _dptr(out), res)
        if st not in (PWA_OK, PWA_ENOCONV):
            self._check(st)
        infos = [{"nll": r.nll, "grad_max": r.grad_max, "iters": r.iters, "n_hvp": r.n_hvp, "n_fev": r.n_fev,
                  "n_hess": r.n_hess, "status": FIT_STATUS_NAMES[r.status], "elapsed_s": r.elapsed_s} for r in res]
        if tbuf is not None:
            for b, (r, info) in enumerate(zip(res, infos)):
                info["trace"] = _read_trace(tbuf, trace, b, r.n_trace)
        return out, infos, st == PWA_OK

    # -- tiling --
    def set_tiling(self, warps: int, stages: int = 2, blocks_per_sm: int = 0):
        self._check(lib().pwa_set_tiling(self._h, warps, stages, blocks_per_sm))

    def autotune(self, theta, batch: int = 1) -> dict:
        """Pick the fastest tiling for batched HVP passes of `batch` vectors at theta."""
        th = _f64(theta, self.P)
        out = (ctypes.c_int * 3)()
        self._check(lib().pwa_autotune(self._h, _dptr(th), int(batch), out))
        return self.get_tiling()

    def get_tiling(self) -> dict:
        out = (ctypes.c_int * 6)()
        self._check(lib().pwa_get_tiling(self._h, out))
        keys = ("warps", "stages", "blocks_per_sm", "events_per_tile", "grid_blocks", "smem_bytes")
        return dict(zip(keys, list(out)))


class Coupling:
    """The fixed-mass coupling sub-problem of a likelihood (tensor-core GEMMs
    over U = BW F tiles and the K x K integral matrix; see include/pwa.h).
    Its parameters are the first Pc entries of theta (free magnitudes, then
    free phases); masses, widths and fixed couplings come from `theta`."""

    def __init__(self, L: "Likelihood", theta):
        th = _f64(theta, L.P)
        h = ctypes.c_void_p()
        st = lib().pwa_coupling_create(L._h, _dptr(th), ctypes.byref(h))
        if st != PWA_OK:
            raise PwaError(st, lib().pwa_last_error(L._h).decode())
        self._L = L
        self._h = h
        self.K = L.K
        self.Pc = lib().pwa_coupling_num_params(h)

    def _check(self, st: int):
        if st != PWA_OK:
            raise PwaError(st, lib().pwa_last_error(self._L._h).decode())

    def integral_matrix(self) -> np.ndarray:
        out = np.empty(2 * self.K * self.K)
        self._check(lib().pwa_coupling_integral_matrix(self._h, _dptr(out)))
        return (out[0::2] + 1j * out[1::2]).reshape(self.K, self.K)

    def eval(self, thetas_c, vs=None):
        """(NLL [C], grad [C, Pc], H v [C, Pc] or None) for C coupling vectors."""
        th = _f64(thetas_c).reshape(-1, self.Pc)
        C = th.shape[0]
        f = np.empty(C)
        g = np.empty((C, self.Pc))
        if vs is None:
            self._check(lib().pwa_coupling_eval(self._h, C, _dptr(th), None, _dptr(f), _dptr(g), None))
            return f, g, None
        vv = _f64(vs).reshape(C, self.Pc)
        hv = np.empty((C, self.Pc))
        self._check(lib().pwa_coupling_eval(self._h, C, _dptr(th), _dptr(vv), _dptr(f), _dptr(g), _dptr(hv)))
        return f, g, hv

    def fit(self, thetas_c0, xtol: float = 1e-8, gtol: float = 0.0, maxiter: int = 0, cg_maxiter: int = 0,
            time_limit_s: float = 0.0):
        """C coupling-only fits in lockstep; returns (theta_c [C, Pc], infos, all converged)."""
        th = _f64(thetas_c0).reshape(-1, self.Pc)
        C = th.shape[0]
        out = np.empty((C, self.Pc))
        opts = pwa_fit_opts(xtol, gtol, maxiter, cg_maxiter, time_limit_s)
        res = (pwa_fit_result * C)()
        st = lib().pwa_coupling_fit(self._h, C, _dptr(th), ctypes.byref(opts), _dptr(out), res)
        if st not in (PWA_OK, PWA_ENOCONV):
            self._check(st)
        infos = [{"nll": r.nll, "grad_max": r.grad_max, "iters": r.iters, "n_hvp": r.n_hvp, "n_fev": r.n_fev,
                  "n_hess": r.n_hess, "status": FIT_STATUS_NAMES[r.status], "elapsed_s": r.elapsed_s} for r in res]
        return out, infos, st == PWA_OK

    def close(self):
        if getattr(self, "_h", None):
            lib().pwa_coupling_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fit_multi(likelihoods, thetas0, xtol: float = 1e-8, gtol: float = 0.0, maxiter: int = 0,
              cg_maxiter: int = 0, time_limit_s: float = 0.0, matrix_free: bool = False, method: int = 0,
              one_launch: bool = False):
    """Lockstep fits over several likelihoods (one group of starts per
    likelihood; their batched passes run concurrently, or with one_launch as
    one launch over all likelihoods per round).  thetas0[i]: [B_i, P_i].
    Returns ([theta [B_i, P_i]], [[info per fit]], all converged-or-time-limit)."""
    n = len(likelihoods)
    ths = [_f64(t).reshape(-1, L.P) for L, t in zip(likelihoods, thetas0)]
    outs = [np.empty_like(t) for t in ths]
    Bs = (ctypes.c_int * n)(*[t.shape[0] for t in ths])
    res = [(pwa_fit_result * t.shape[0])() for t in ths]
    hs = (ctypes.c_void_p * n)(*[L._h.value for L in likelihoods])
    dpp = ctypes.POINTER(ctypes.c_double)
    th_p = (dpp * n)(*[_dptr(t) for t in ths])
    out_p = (dpp * n)(*[_dptr(o) for o in outs])
    res_p = (ctypes.POINTER(pwa_fit_result) * n)(*[ctypes.cast(r, ctypes.POINTER(pwa_fit_result)) for r in res])
    opts = pwa_fit_opts(xtol, gtol, maxiter, cg_maxiter, time_limit_s, int(matrix_free), int(method))
    opts.one_launch = int(one_launch)
    st = lib().pwa_newton_cg_fit_multi(n, hs, Bs, th_p, ctypes.byref(opts), out_p, res_p)
    if st not in (PWA_OK, PWA_ENOCONV):
        msgs = "; ".join(filter(None, (lib().pwa_last_error(L._h).decode() for L in likelihoods)))
        raise PwaError(st, msgs)
    infos = [[{"nll": r.nll, "grad_max": r.grad_max, "iters": r.iters, "n_hvp": r.n_hvp, "n_fev": r.n_fev,
               "n_hess": r.n_hess, "status": FIT_STATUS_NAMES[r.status], "elapsed_s": r.elapsed_s} for r in rr] for rr in res]
    return outs, infos, st == PWA_OK


def eval_multi(likelihoods, thetas, vs=None):
    """One launch over several likelihoods (pwa_eval_multi_device): thetas[i]
    [B_i, P_i] (and vs[i] for H v) -> per likelihood (nll [B_i], grad
    [B_i, P_i], hv [B_i, P_i] or None).  Device buffers are torch tensors;
    the launch runs on torch's current stream."""
    import torch
    n = len(likelihoods)
    want_hv = vs is not None
    th = [torch.as_tensor(np.asarray(t, dtype=np.float64).reshape(-1, L.P), device="cuda")
          for L, t in zip(likelihoods, thetas)]
    vv = [torch.as_tensor(np.asarray(v, dtype=np.float64).reshape(-1, L.P), device="cuda")
          for L, v in zip(likelihoods, vs)] if want_hv else None
    out = [torch.empty((t.shape[0], 1 + 2 * L.P), dtype=torch.float64, device="cuda") for L, t in zip(likelihoods, th)]
    hs = (ctypes.c_void_p * n)(*[L._h.value for L in likelihoods])
    Bs = (ctypes.c_int * n)(*[t.shape[0] for t in th])
    ptr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
    stream = torch.cuda.current_stream()
    st = lib().pwa_eval_multi_device(n, hs, Bs, ptr(th), ptr(vv) if want_hv else None, ptr(out), 1, int(want_hv),
                                     stream.cuda_stream)
    if st != PWA_OK:
        msgs = "; ".join(filter(None, (lib().pwa_last_error(L._h).decode() for L in likelihoods)))
        raise PwaError(st, msgs)
    stream.synchronize()
    for L in likelihoods:
        L.sync()
    res = []
    for L, o in zip(likelihoods, out):
        o = o.cpu().numpy()
        res.append((o[:, 0].copy(), o[:, 1:1 + L.P].copy(), o[:, 1 + L.P:].copy() if want_hv else None))
    return res


SHAPE_CONSTANT, SHAPE_MASS_DEPENDENT, SHAPE_FLATTE = 0, 1, 2


class Variant:
    """A physics-variant likelihood (see include/pwa.h): line shapes per
    resonance (objects with kind, ma, mb, mc, md, radius, width2 attributes,
    or None for constant widths) and one coupling per resonance or per
    (resonance, projection)."""

    def __init__(self, data, mc, table, K: int, S: int, shapes=None, per_projection: bool = False,
                 stream: int = 0):
        keep: list = []
        de = _events(data.m2, data.F, getattr(data, "w", None), keep)
        me = _events(mc.m2, mc.F, None, keep)
        tab = resonance_table(table)
        shp = None
        if shapes is not None:
            shp = (pwa_lineshape * K)()
            for k, sh in enumerate(shapes):
                shp[k] = pwa_lineshape(int(sh.kind), float(sh.ma), float(sh.mb), float(sh.mc), float(sh.md),
                                       float(sh.radius), float(sh.width2))
        h = ctypes.c_void_p()
        st = lib().pwa_variant_create(ctypes.byref(h), ctypes.byref(de), ctypes.byref(me), tab, shp, int(K), int(S),
                                      int(bool(per_projection)), ctypes.c_void_p(stream))
        if st != PWA_OK:
            raise PwaError(st, lib().pwa_variant_last_error(None).decode())
        self._h = h
        self.K, self.S = int(K), int(S)
        self.P = lib().pwa_variant_num_params(h)

    @staticmethod
    def initial_theta(table, shapes, S: int, per_projection: bool = False) -> np.ndarray:
        """theta in the variant's order from the table's values (width2 of
        the Flatte shapes for gamma2), as pwa_variant_create lays it out."""
        ns = S if per_projection else 1
        K = len(table)
        kind = [0 if shapes is None else int(shapes[k].kind) for k in range(K)]
        th = [r.mag for r in table if not r.fix_coupling for _ in range(ns)]
        th += [r.phase for r in table if not r.fix_coupling for _ in range(ns)]
        th += [r.mass for r in table if not r.fix_mass]
        th += [r.width for r in table if not r.fix_width]
        th += [shapes[k].width2 for k, r in enumerate(table) if not r.fix_width and kind[k] == SHAPE_FLATTE]
        return np.array(th, dtype=np.float64)

    def _check(self, st: int):
        if st != PWA_OK:
            raise PwaError(st, lib().pwa_variant_last_error(self._h).decode())

    def nll(self, theta) -> float:
        th = _f64(theta, self.P)
        f = ctypes.c_double()
        self._check(lib().pwa_variant_eval(self._h, _dptr(th), None, ctypes.byref(f), None, None))
        return f.value

    def eval(self, theta, v=None):
        """(NLL, grad, H v or None) from one pass."""
        th = _f64(theta, self.P)
        f = ctypes.c_double()
        g = np.empty(self.P)
        if v is None:
            self._check(lib().pwa_variant_eval(self._h, _dptr(th), None, ctypes.byref(f), _dptr(g), None))
            return f.value, g, None
        vv = _f64(v, self.P)
        hv = np.empty(self.P)
        self._check(lib().pwa_variant_eval(self._h, _dptr(th), _dptr(vv), ctypes.byref(f), _dptr(g), _dptr(hv)))
        return f.value, g, hv

    def eval_batch(self, thetas, vs=None):
        """(NLL [B], grad [B, P], H v [B, P] or None, status [B]) of B
        parameter vectors in one launch; a vector outside the model's domain
        or with a non-finite intensity has a non-zero status (its rows are NaN)."""
        th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(-1, self.P))
        B = th.shape[0]
        f = np.full(B, np.nan)
        g = np.full((B, self.P), np.nan)
        stat = np.zeros(B, dtype=np.int32)
        sp = stat.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        if vs is None:
            self._check(lib().pwa_variant_eval_batch(self._h, B, _dptr(th), None, _dptr(f), _dptr(g), None, sp))
            return f, g, None, stat
        vv = np.ascontiguousarray(np.asarray(vs, dtype=np.float64).reshape(B, self.P))
        hv = np.full((B, self.P), np.nan)
        self._check(lib().pwa_variant_eval_batch(self._h, B, _dptr(th), _dptr(vv), _dptr(f), _dptr(g), _dptr(hv),
                                                 sp))
        return f, g, hv, stat

    def fit(self, thetas0, xtol: float = 1e-8, gtol: float = 0.0, maxiter: int = 0, cg_maxiter: int = 0,
            time_limit_s: float = 0.0):
        """B fits (rows of thetas0) in lockstep; returns (theta [B, P], infos, all converged)."""
        th = _f64(thetas0).reshape(-1, self.P)
        B = th.shape[0]
        out = np.empty((B, self.P))
        opts = pwa_fit_opts(xtol, gtol, maxiter, cg_maxiter, time_limit_s)
        res = (pwa_fit_result * B)()
        st = lib().pwa_variant_fit(self._h, B, _dptr(th), ctypes.byref(opts), _dptr(out), res)
        if st not in (PWA_OK, PWA_ENOCONV):
            self._check(st)
        infos = [{"nll": r.nll, "grad_max": r.grad_max, "iters": r.iters, "n_hvp": r.n_hvp, "n_fev": r.n_fev,
                  "n_hess": r.n_hess, "status": FIT_STATUS_NAMES[r.status], "elapsed_s": r.elapsed_s} for r in res]
        return out, infos, st == PWA_OK

    # -- couplings only, at fixed line shapes (integral matrices of the MC events) --
    def set_shapes(self, theta) -> np.ndarray:
        """Fix the line shapes at theta's masses and widths; returns the MC
        integral matrices Phi [S, K, K] (complex)."""
        th = _f64(theta, self.P)
        out = np.empty(2 * self.S * self.K * self.K)
        self._check(lib().pwa_variant_set_shapes(self._h, _dptr(th), _dptr(out)))
        self.Pc = lib().pwa_variant_coupling_num_params(self._h)
        return (out[0::2] + 1j * out[1::2]).reshape(self.S, self.K, self.K)

    def coupling_eval(self, theta_c, v=None):
        """(NLL, grad [Pc], H v [Pc] or None) in the coupling parameters."""
        Pc = lib().pwa_variant_coupling_num_params(self._h)
        th = _f64(theta_c, Pc)
        f = ctypes.c_double()
        g = np.empty(Pc)
        if v is None:
            self._check(lib().pwa_variant_coupling_eval(self._h, _dptr(th), None, ctypes.byref(f), _dptr(g), None))
            return f.value, g, None
        vv = _f64(v, Pc)
        hv = np.empty(Pc)
        self._check(lib().pwa_variant_coupling_eval(self._h, _dptr(th), _dptr(vv), ctypes.byref(f), _dptr(g),
                                                    _dptr(hv)))
        return f.value, g, hv

    def coupling_fit(self, thetas_c0, xtol: float = 1e-8, gtol: float = 0.0, maxiter: int = 0, cg_maxiter: int = 0,
                     time_limit_s: float = 0.0):
        """B coupling-only fits in lockstep; returns (theta_c [B, Pc], infos, all converged)."""
        Pc = lib().pwa_variant_coupling_num_params(self._h)
        th = _f64(thetas_c0).reshape(-1, Pc)
        B = th.shape[0]
        out = np.empty((B, Pc))
        opts = pwa_fit_opts(xtol, gtol, maxiter, cg_maxiter, time_limit_s)
        res = (pwa_fit_result * B)()
        st = lib().pwa_variant_coupling_fit(self._h, B, _dptr(th), ctypes.byref(opts), _dptr(out), res)
        if st not in (PWA_OK, PWA_ENOCONV):
            self._check(st)
        infos = [{"nll": r.nll, "grad_max": r.grad_max, "iters": r.iters, "n_hvp": r.n_hvp, "n_fev": r.n_fev,
                  "n_hess": r.n_hess, "status": FIT_STATUS_NAMES[r.status], "elapsed_s": r.elapsed_s} for r in res]
        return out, infos, st == PWA_OK

    def close(self):
        if getattr(self, "_h", None):
            lib().pwa_variant_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _gen_check(st: int):
    if st != PWA_OK:
        raise PwaError(st, lib().pwa_last_generate_error().decode())


def _cuda_f32(t, what: str):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("%s: expected a contiguous CUDA float32 tensor" % what)
    return ctypes.c_void_p(t.data_ptr())


def accept_reject(I, seed: int, start: int, n_target: int, C: float = 0.0, stream: int = 0):
    """Counter-based accept-reject over a pool's intensities I (CUDA float32
    [n]); returns (pool indices as a CUDA int32 tensor [n_kept], C used)."""
    import torch
    idx = torch.empty(max(1, n_target), dtype=torch.int32, device=I.device)
    n_out = ctypes.c_int()
    c_used = ctypes.c_double()
    _gen_check(lib().pwa_accept_reject(_cuda_f32(I, "I"), int(I.numel()), float(C), ctypes.c_ulonglong(seed),
                                       int(start), int(n_target), ctypes.c_void_p(idx.data_ptr()),
                                       ctypes.byref(n_out), ctypes.byref(c_used), ctypes.c_void_p(stream)))
    return idx[:n_out.value], c_used.value


def dalitz_histogram(m2, idx, nb: int, bounds, log_scale: bool = True, out=None, stream: int = 0):
    """nb x nb histogram of (m12^2, m23^2) over the pool events idx (CUDA int32);
    m2: CUDA float32 [3, ld]; returns CUDA float32 [nb * nb] (or fills out)."""
    import torch
    if out is None:
        out = torch.empty(nb * nb, dtype=torch.float32, device=m2.device)
    x0, x1, y0, y1 = bounds
    _gen_check(lib().pwa_dalitz_histogram(_cuda_f32(m2, "m2"), int(m2.shape[1]), ctypes.c_void_p(idx.data_ptr()),
                                          int(idx.numel()), int(nb), x0, x1, y0, y1, int(bool(log_scale)),
                                          _cuda_f32(out, "out"), ctypes.c_void_p(stream)))
    return out


def gather_events(m2, F, idx, stream: int = 0):
    """Sample arrays (m2 [3, n], F [n, K, S] complex as float32 [..., 2]) of the
    pool events idx; m2: CUDA float32 [3, ld], F: CUDA float32 [ld, K, S, 2]."""
    import torch
    n = int(idx.numel())
    KS = int(F.shape[1] * F.shape[2])
    m2o = torch.empty((3, max(n, 1)), dtype=torch.float32, device=m2.device)
    Fo = torch.empty((max(n, 1),) + tuple(F.shape[1:]), dtype=torch.float32, device=m2.device)
    _gen_check(lib().pwa_gather_events(_cuda_f32(m2, "m2"), int(m2.shape[1]), _cuda_f32(F, "F"), KS,
                                       ctypes.c_void_p(idx.data_ptr()), n, _cuda_f32(m2o, "m2_out"),
                                       _cuda_f32(Fo, "F_out"), ctypes.c_void_p(stream)))
    return m2o[:, :n], Fo[:n]


class ProposalMLP:
    """The learned starting-point proposal network (see include/pwa.h):
    in -> `layers` x hidden (GELU) -> out, BF16 tensor-core products, Adam.
    Inputs and targets are torch CUDA float32 tensors [B, in] / [B, out] with
    B a multiple of 128; parameters move through host numpy arrays."""

    def __init__(self, n_in: int, hidden: int, layers: int, n_out: int, max_batch: int, seed: int = 1,
                 periodic=None, loss_weight=None, stream: int = 0):
        per = None if periodic is None else (ctypes.c_int * n_out)(*[int(bool(x)) for x in periodic])
        wg = None if loss_weight is None else (ctypes.c_float * n_out)(*[float(x) for x in loss_weight])
        h = ctypes.c_void_p()
        st = lib().pwa_mlp_create(n_in, hidden, layers, n_out, max_batch, ctypes.c_ulonglong(seed),
                                  ctypes.cast(per, ctypes.POINTER(ctypes.c_int)) if per is not None else None,
                                  ctypes.cast(wg, ctypes.POINTER(ctypes.c_float)) if wg is not None else None,
                                  ctypes.c_void_p(stream), ctypes.byref(h))
        if st != PWA_OK:
            raise PwaError(st, lib().pwa_mlp_last_error(None).decode())
        self._h = h
        self.n_in, self.hidden, self.layers, self.n_out, self.max_batch = n_in, hidden, layers, n_out, max_batch

    def _check(self, st: int):
        if st != PWA_OK:
            raise PwaError(st, lib().pwa_mlp_last_error(self._h).decode())

    @staticmethod
    def _dev(t, cols: int):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                and t.dim() == 2 and t.shape[1] == cols):
            raise ValueError("expected a contiguous CUDA float32 tensor [B, %d]" % cols)
        return ctypes.c_void_p(t.data_ptr())

    def forward(self, x):
        import torch
        y = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device=x.device)
        self._check(lib().pwa_mlp_forward(self._h, int(x.shape[0]), self._dev(x, self.n_in), self._dev(y, self.n_out)))
        return y

    def gradients(self, x, t) -> float:
        loss = ctypes.c_double()
        self._check(lib().pwa_mlp_gradients(self._h, int(x.shape[0]), self._dev(x, self.n_in),
                                            self._dev(t, self.n_out), ctypes.byref(loss)))
        return loss.value

    def train_step(self, x, t, lr: float) -> float:
        loss = ctypes.c_double()
        self._check(lib().pwa_mlp_train_step(self._h, int(x.shape[0]), self._dev(x, self.n_in),
                                             self._dev(t, self.n_out), ctypes.c_float(lr), ctypes.byref(loss)))
        return loss.value

    def _shape(self, layer: int, which: int):
        fi = self.n_in if layer == 0 else self.hidden
        fo = self.n_out if layer == self.layers else self.hidden
        return (fo, fi) if which in (0, 2) else (fo,)

    def get(self, layer: int, which: int) -> np.ndarray:
        """which: 0 W, 1 bias, 2 last weight gradient, 3 last bias gradient."""
        a = np.empty(self._shape(layer, which), dtype=np.float32)
        self._check(lib().pwa_mlp_params(self._h, layer, which, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 0))
        return a

    def set(self, layer: int, which: int, values):
        a = np.ascontiguousarray(np.asarray(values, dtype=np.float32).reshape(self._shape(layer, which)))
        self._check(lib().pwa_mlp_params(self._h, layer, which, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 1))

    def params(self):
        """[(W, b)] per layer as float64 arrays."""
        return [(self.get(l, 0).astype(np.float64), self.get(l, 1).astype(np.float64))
                for l in range(self.layers + 1)]

    def gemm_check(self, A, B) -> np.ndarray:
        """C = bf16(A) bf16(B)^T on the tensor cores (FP32 accumulation)."""
        A = np.ascontiguousarray(A, dtype=np.float32)
        B = np.ascontiguousarray(B, dtype=np.float32)
        C = np.empty((A.shape[0], B.shape[0]), dtype=np.float32)
        fpp = ctypes.POINTER(ctypes.c_float)
        self._check(lib().pwa_mlp_gemm_check(self._h, A.shape[0], B.shape[0], A.shape[1], A.ctypes.data_as(fpp),
                                             B.ctypes.data_as(fpp), C.ctypes.data_as(fpp)))
        return C

    def close(self):
        if getattr(self, "_h", None):
            lib().pwa_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_likelihood(workload, stream: int = 0, device_inputs: bool = False) -> Likelihood:
    """Likelihood for a workload.Workload (host inputs, or torch CUDA tensors
    when device_inputs is True)."""
    data, mc = workload.data, workload.mc
    if device_inputs:
        import torch
        from types import SimpleNamespace
        dev = torch.device("cuda")
        data = SimpleNamespace(m2=torch.from_numpy(data.m2).to(dev), F=torch.from_numpy(data.F).to(dev),
                               w=None if data.w is None else torch.from_numpy(data.w).to(dev))
        mc = SimpleNamespace(m2=torch.from_numpy(mc.m2).to(dev), F=torch.from_numpy(mc.F).to(dev), w=None)
    return Likelihood(data, mc, workload.table, workload.K, workload.S, stream)
