"""CPU FP64 oracle for the PWACG likelihood (arXiv:2403.09225) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports, links or runs it, and shares no code with it.

``pwa_oracle.c`` holds the arithmetic (plain single-threaded loops in FP64);
this module only marshals arrays through ctypes and maps the free-parameter
vector theta onto the full per-resonance parameter list.  ``newton_cg.py`` is
the textbook line-search Newton-CG used as the reference fit.

Functions and the passages they follow:
  intensity        I(e) = sum_s |A_s|^2                     Eq. 1
  nll              -ln L                                    Eq. 3 (negated)
  nll_grad_hvp     -ln L, its gradient and H v              Eqs. 4, 6, 7
  sample_sums      per-shard F_m, G_m and derivatives       Eq. 5
  hessian          full Hessian of -ln L                    Eq. 7
  sharded_*        the same over event shards in workers    Eqs. 4-5 (shard sums add up)
  integral_matrix  Phi_kk' = sum_e sum_s conj(U_ks) U_k's   Eq. 1 (couplings factored out)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from concurrent.futures import ProcessPoolExecutor, as_completed
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pwa_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, strict IEEE: no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp, fp, ip = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float),
                      ctypes.POINTER(ctypes.c_int))
        L, I = ctypes.c_long, ctypes.c_int
        lib.or_intensity.argtypes = [I, I, ip, dp, L, fp, fp, dp]
        lib.or_intensity.restype = L
        lib.or_sample_sums.argtypes = [I, I, ip, dp, dp, L, fp, fp, fp, I, dp]
        lib.or_sample_sums.restype = L
        lib.or_sample_hessian.argtypes = [I, I, ip, dp, L, fp, fp, fp, I, dp]
        lib.or_sample_hessian.restype = L
        lib.or_nll.argtypes = [I, I, ip, dp, dp, L, fp, fp, fp, L, fp, fp, dp, dp, dp]
        lib.or_nll.restype = L
        lib.or_integral_matrix.argtypes = [I, I, ip, dp, L, fp, fp, dp]
        lib.or_integral_matrix.restype = L
        lib.or_hessian.argtypes = [I, I, ip, dp, L, fp, fp, fp, L, fp, fp, dp]
        lib.or_hessian.restype = L
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if a is not None else None


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _events(m2, F, w=None):
    m2 = np.ascontiguousarray(m2, dtype=np.float32)
    F = np.ascontiguousarray(F, dtype=np.complex64).view(np.float32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    return m2, F, w


class OracleError(RuntimeError):
    """An event's intensity is not finite (or not positive for data)."""

    def __init__(self, index: int):
        super().__init__("non-finite or non-positive intensity at event %d" % index)
        self.index = index


class Model:
    """Resonance channels plus the map between theta (free parameters) and the
    full parameter list par[4K] = (rho_0..rho_{K-1}, phi_.., M_.., Gamma_..).

    theta order: free magnitudes, free phases, free masses, free widths, each
    block in resonance order (the library uses the same order)."""

    def __init__(self, channels: Sequence[int], mag, phase, mass, width,
                 fix_coupling, fix_mass, fix_width, S: int):
        self.K = len(channels)
        self.S = int(S)
        self.channels = np.ascontiguousarray(channels, dtype=np.int32)
        self.par0 = np.concatenate([mag, phase, mass, width]).astype(np.float64)
        K = self.K
        fixed = np.zeros(4 * K, dtype=bool)
        fixed[0:K] = fix_coupling
        fixed[K:2 * K] = fix_coupling
        fixed[2 * K:3 * K] = fix_mass
        fixed[3 * K:4 * K] = fix_width
        self.free_index = np.flatnonzero(~fixed)
        self.P = int(self.free_index.size)

    @classmethod
    def from_table(cls, table, S: int) -> "Model":
        return cls([r.channel for r in table], [r.mag for r in table], [r.phase for r in table],
                   [r.mass for r in table], [r.width for r in table],
                   [r.fix_coupling for r in table], [r.fix_mass for r in table],
                   [r.fix_width for r in table], S)

    def full(self, theta) -> np.ndarray:
        par = self.par0.copy()
        par[self.free_index] = np.asarray(theta, dtype=np.float64)
        return par

    def embed(self, v) -> np.ndarray:
        """A free-parameter direction as a full-order vector (zero on fixed)."""
        out = np.zeros(4 * self.K)
        out[self.free_index] = np.asarray(v, dtype=np.float64)
        return out

    def restrict(self, full_vec) -> np.ndarray:
        return np.asarray(full_vec)[..., self.free_index]


def intensity(model: Model, theta, m2, F) -> np.ndarray:
    """I(e) per event (Eq. 1)."""
    lib = _load()
    m2, Fv, _ = _events(m2, F)
    n = m2.shape[1]
    out = np.empty(n)
    par = model.full(theta)
    lib.or_intensity(model.K, model.S, _i(model.channels), _d(par), n, _f(m2), _f(Fv), _d(out))
    return out


def integral_matrix(model: Model, theta, m2, F) -> np.ndarray:
    """Phi [K, K] complex at theta's masses and widths: sum over the events of
    sum_s conj(U_ks) U_k's with U = BW F, so that sum_e I(e) = g^H Phi g for
    the couplings g_k = rho_k e^{i phi_k} (Eq. 1 with the couplings factored out)."""
    lib = _load()
    m2, Fv, _ = _events(m2, F)
    out = np.empty(2 * model.K * model.K)
    rc = lib.or_integral_matrix(model.K, model.S, _i(model.channels), _d(model.full(theta)), m2.shape[1],
                                _f(m2), _f(Fv), _d(out))
    if rc != -1:
        raise MemoryError("or_integral_matrix")
    return (out[0::2] + 1j * out[1::2]).reshape(model.K, model.K)


def couplings(model: Model, theta) -> np.ndarray:
    """g_k = rho_k e^{i phi_k} of every resonance (fixed ones included)."""
    par = model.full(theta)
    K = model.K
    return par[:K] * np.exp(1j * par[K:2 * K])


def intensity_full(K, S, channels, par_full, m2, F) -> np.ndarray:
    """I(e) for a full-order parameter vector."""
    lib = _load()
    m2, Fv, _ = _events(m2, F)
    ch = np.ascontiguousarray(channels, dtype=np.int32)
    par = np.ascontiguousarray(par_full, dtype=np.float64)
    out = np.empty(m2.shape[1])
    lib.or_intensity(K, S, _i(ch), _d(par), m2.shape[1], _f(m2), _f(Fv), _d(out))
    return out


def sample_sums(model: Model, theta, v, m2, F, w, is_data: bool) -> np.ndarray:
    """Eq. 5 shard sums over one sample, full order (see pwa_oracle.c)."""
    lib = _load()
    m2, Fv, w = _events(m2, F, w)
    K = model.K
    out = np.empty(2 + 8 * K + 1)
    par = model.full(theta)
    vf = None if v is None else model.embed(v)
    bad = lib.or_sample_sums(K, model.S, _i(model.channels), _d(par), _d(vf), m2.shape[1],
                             _f(m2), _f(w), _f(Fv), int(bool(is_data)), _d(out))
    if bad >= 0:
        raise OracleError(int(bad))
    return out


def combine(model: Model, sd: np.ndarray, sm: np.ndarray, n_mc: int):
    """Eqs. 4, 6, 7 from the data and MC shard sums (restricted to theta)."""
    K = model.K
    P4 = 4 * K
    Fsum, Nd, G = sd[0], sd[1], sm[0]
    nll = -Fsum + Nd * math.log(G / n_mc)
    grad = -sd[2:2 + P4] + Nd * sm[2:2 + P4] / G
    dGv = sm[2 + 2 * P4]
    hv = -sd[2 + P4:2 + 2 * P4] + Nd * (sm[2 + P4:2 + 2 * P4] / G - sm[2:2 + P4] * dGv / (G * G))
    return nll, model.restrict(grad), model.restrict(hv)


def nll_grad_hvp(model: Model, theta, v, data, mc):
    """(NLL, grad, H v) at theta; v may be None (then H v is zeros)."""
    sd = sample_sums(model, theta, v, data.m2, data.F, data.w, True)
    try:
        sm = sample_sums(model, theta, v, mc.m2, mc.F, None, False)
    except OracleError as e:  # MC events are numbered after the data events
        raise OracleError(data.n + e.index) from None
    return combine(model, sd, sm, mc.n)


def nll(model: Model, theta, data, mc) -> float:
    return nll_grad_hvp(model, theta, None, data, mc)[0]


def nll_grad(model: Model, theta, data, mc):
    f, g, _ = nll_grad_hvp(model, theta, None, data, mc)
    return f, g


def hessian(model: Model, theta, data, mc) -> np.ndarray:
    """Full P x P Hessian of NLL (Eq. 7), for small cases."""
    lib = _load()
    m2d, Fd, wd = _events(data.m2, data.F, data.w)
    m2m, Fm, _ = _events(mc.m2, mc.F)
    K = model.K
    H = np.empty((4 * K, 4 * K))
    bad = lib.or_hessian(K, model.S, _i(model.channels), _d(model.full(theta)), m2d.shape[1],
                         _f(m2d), _f(wd), _f(Fd), m2m.shape[1], _f(m2m), _f(Fm), _d(H))
    if bad >= 0:
        raise OracleError(int(bad))
    idx = model.free_index
    return H[np.ix_(idx, idx)]


# ---------------------------------------------------------------------------
# shard-parallel evaluation for large samples (Eqs. 4-5: sums over disjoint
# event subsets add up; the shards are combined in a fixed order in FP64)
# ---------------------------------------------------------------------------

def _shard_job(args):
    model, theta, v, m2, F, w, is_data = args
    return sample_sums(model, theta, v, m2, F, w, is_data)


def sharded_nll_grad_hvp(model: Model, theta, v, data, mc, workers: int = 8, shard: int = 250_000,
                         pool: Optional[ProcessPoolExecutor] = None):
    """nll_grad_hvp over event shards evaluated in worker processes (spawned)."""
    jobs = []
    for s, is_data in ((data, True), (mc, False)):
        for a in range(0, s.n, shard):
            b = min(s.n, a + shard)
            w = None if s.w is None else s.w[a:b]
            jobs.append((model, np.asarray(theta), None if v is None else np.asarray(v),
                         np.ascontiguousarray(s.m2[:, a:b]), np.ascontiguousarray(s.F[a:b]), w, is_data))
    own = pool is None
    if own:
        import multiprocessing as mp
        pool = ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    try:
        # at most 2 x workers shards in flight (each submitted shard holds a
        # pickled copy of its events); results are kept in shard order
        parts = [None] * len(jobs)
        pending = {}
        nxt = 0
        while nxt < len(jobs) or pending:
            while nxt < len(jobs) and len(pending) < 2 * workers:
                pending[pool.submit(_shard_job, jobs[nxt])] = nxt
                nxt += 1
            done = next(iter(as_completed(list(pending))))
            parts[pending.pop(done)] = done.result()
    finally:
        if own:
            pool.shutdown()
    nd_jobs = sum(1 for j in jobs if j[6])
    sd = np.sum(parts[:nd_jobs], axis=0) if nd_jobs else np.zeros(2 + 8 * model.K + 1)
    sm = np.sum(parts[nd_jobs:], axis=0)
    return combine(model, sd, sm, mc.n)


def sample_hessian(model: Model, theta, m2, F, w, is_data: bool) -> np.ndarray:
    """Per-shard second-derivative sums (full 4K x 4K order): d2F_m for data
    (sum w [d2I / I - dI dI^T / I^2]) and d2G_m for MC (sum d2I), Eq. 7."""
    lib = _load()
    m2, Fv, w = _events(m2, F, w)
    K = model.K
    out = np.empty((4 * K, 4 * K))
    bad = lib.or_sample_hessian(K, model.S, _i(model.channels), _d(model.full(theta)), m2.shape[1], _f(m2), _f(w),
                                _f(Fv), int(bool(is_data)), _d(out))
    if bad >= 0:
        raise OracleError(int(bad))
    return out


def _shard_hessian_job(args):
    model, theta, m2, F, w, is_data = args
    return sample_sums(model, theta, None, m2, F, w, is_data), sample_hessian(model, theta, m2, F, w, is_data)


def sharded_hessian(model: Model, theta, data, mc, workers: int = 8, shard: int = 20_000,
                    pool: Optional[ProcessPoolExecutor] = None):
    """(NLL, grad, full Hessian) over event shards in spawned worker processes:
    the shard sums add up (Eqs. 4-5) and Eq. 7 combines them,
    H = -d2F + N_d [d2G / G - dG dG^T / G^2] (the combination or_hessian makes)."""
    jobs = []
    for s, is_data in ((data, True), (mc, False)):
        for a in range(0, s.n, shard):
            b = min(s.n, a + shard)
            w = None if s.w is None else s.w[a:b]
            jobs.append((model, np.asarray(theta), np.ascontiguousarray(s.m2[:, a:b]),
                         np.ascontiguousarray(s.F[a:b]), w, is_data))
    own = pool is None
    if own:
        import multiprocessing as mp
        pool = ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    try:
        parts = list(pool.map(_shard_hessian_job, jobs))
    finally:
        if own:
            pool.shutdown()
    nd_jobs = sum(1 for j in jobs if j[5])
    sd = np.sum([p[0] for p in parts[:nd_jobs]], axis=0)
    sm = np.sum([p[0] for p in parts[nd_jobs:]], axis=0)
    Hd = np.sum([p[1] for p in parts[:nd_jobs]], axis=0)
    Hm = np.sum([p[1] for p in parts[nd_jobs:]], axis=0)
    nll, grad, _ = combine(model, sd, sm, mc.n)
    P4 = 4 * model.K
    Nd, G = sd[1], sm[0]
    dG = sm[2:2 + P4]
    H = -Hd + Nd * (Hm / G - np.outer(dG, dG) / (G * G))
    idx = model.free_index
    return nll, grad, H[np.ix_(idx, idx)]


def parameter_errors(H: np.ndarray) -> np.ndarray:
    """sigma_i = sqrt(diag(H^-1)) with H the Hessian of NLL at the minimum."""
    return np.sqrt(np.diag(np.linalg.inv(H)))


def canonical(model: Model, theta) -> np.ndarray:
    """Map equivalent minima to one representative: rho > 0, phi in (-pi, pi]
    ((rho, phi) and (-rho, phi + pi) give the same coupling)."""
    par = model.full(theta)
    K = model.K
    rho, phi = par[0:K], par[K:2 * K]
    neg = rho < 0
    rho[neg] = -rho[neg]
    phi[neg] += math.pi
    phi[:] = math.pi - np.mod(math.pi - phi, 2 * math.pi)
    return model.restrict(par)
