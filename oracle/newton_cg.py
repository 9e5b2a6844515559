"""Textbook line-search Newton-CG -- the oracle's reference minimiser.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper fits with the truncated-Newton method of scipy ("Newton-CG", paper
Sec. 3) driven by exact gradients and Hessian-vector products.  This file
restates the method from Nocedal & Wright, *Numerical Optimization* (2nd ed.):
  * Algorithm 7.1 (line-search Newton-CG): inner CG on H p = -g from z = 0,
    forcing term eta = min(0.5, sqrt(|g|)) |g|, exit on negative curvature
    (steepest descent if it happens on the first inner iteration);
  * Algorithms 3.5/3.6 (line search for the strong Wolfe conditions, with
    zoom by safeguarded cubic interpolation), c1 = 1e-4, c2 = 0.9, alpha0 = 1.
Termination (the paper's xtol, Sec. 3, default 1e-8): mean |delta theta| of an
outer step <= xtol; or |g|_inf <= gtol; or maxiter outer iterations; or a
wall-clock limit (the paper's early stopping at 500 s).  When the line search
fails while the predicted decrease |g.p| is below the resolution of f
(1e3 x machine epsilon x |f|), the fit stops with "precision_limit": the
objective cannot resolve a further step, which counts as converged.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Callable, Optional

import numpy as np

CONVERGED_XTOL, CONVERGED_GTOL, MAXITER, TIME_LIMIT, LINESEARCH_FAILED, PRECISION_LIMIT = range(6)
STATUS_NAMES = ("xtol", "gtol", "maxiter", "time_limit", "linesearch_failed", "precision_limit")
#: statuses that mean "at a minimum to the resolution asked for or available"
CONVERGED = (CONVERGED_XTOL, CONVERGED_GTOL, PRECISION_LIMIT)


@dataclasses.dataclass
class FitResult:
    x: np.ndarray
    fun: float
    grad: np.ndarray
    status: int
    iters: int
    n_fev: int
    n_gev: int
    n_hvp: int
    elapsed: float

    @property
    def status_name(self) -> str:
        return STATUS_NAMES[self.status]


def _cubic_min(a, fa, dfa, b, fb, dfb):
    """Minimiser of the cubic interpolating f and f' at a and b (N&W Eq. 3.59)."""
    d1 = dfa + dfb - 3 * (fa - fb) / (a - b)
    disc = d1 * d1 - dfa * dfb
    if disc < 0:
        return None
    d2 = math.copysign(math.sqrt(disc), b - a)
    denom = dfb - dfa + 2 * d2
    if denom == 0:
        return None
    return b - (b - a) * (dfb + d2 - d1) / denom


def wolfe_line_search(phi: Callable[[float], tuple[float, float]], f0: float, df0: float,
                      c1: float = 1e-4, c2: float = 0.9, alpha1: float = 1.0,
                      alpha_max: float = 1e3, max_iter: int = 30):
    """Strong-Wolfe step length (N&W Algorithm 3.5 with zoom, Algorithm 3.6).

    phi(alpha) returns (f, f') along the search direction.  Returns
    (alpha, f, df) or None when no acceptable step was found."""

    def zoom(lo, flo, dflo, hi, fhi, dfhi):
        for _ in range(max_iter):
            a = _cubic_min(lo, flo, dflo, hi, fhi, dfhi)
            left, right = min(lo, hi), max(lo, hi)
            width = right - left
            if a is None or not (left + 0.1 * width <= a <= right - 0.1 * width):
                a = 0.5 * (lo + hi)
            fa, dfa = phi(a)
            if fa > f0 + c1 * a * df0 or fa >= flo:
                hi, fhi, dfhi = a, fa, dfa
            else:
                if abs(dfa) <= -c2 * df0:
                    return a, fa, dfa
                if dfa * (hi - lo) >= 0:
                    hi, fhi, dfhi = lo, flo, dflo
                lo, flo, dflo = a, fa, dfa
            if abs(hi - lo) < 1e-14 * max(1.0, abs(lo)):
                break
        return None

    a_prev, f_prev, df_prev = 0.0, f0, df0
    a = alpha1
    for i in range(max_iter):
        fa, dfa = phi(a)
        if not math.isfinite(fa):
            # step left the region where the objective is defined: shrink
            a = 0.5 * (a_prev + a)
            continue
        if fa > f0 + c1 * a * df0 or (i > 0 and fa >= f_prev):
            return zoom(a_prev, f_prev, df_prev, a, fa, dfa)
        if abs(dfa) <= -c2 * df0:
            return a, fa, dfa
        if dfa >= 0:
            return zoom(a, fa, dfa, a_prev, f_prev, df_prev)
        a_prev, f_prev, df_prev = a, fa, dfa
        a = min(2 * a, alpha_max)
    return None


def inner_cg(hessp_d: Callable[[np.ndarray], np.ndarray], g: np.ndarray, eps: float, maxiter: int):
    """Inner loop of N&W Algorithm 7.1: CG on B p = -g from z = 0, stopped at
    |r| < eps, or at negative curvature (then -g on the first iteration, else
    the current iterate).  Returns (p, number of Hessian-vector products)."""
    n = g.size
    z = np.zeros(n)
    r = g.copy()
    d = -r
    rr = float(r @ r)
    for j in range(maxiter):
        Bd = np.asarray(hessp_d(d), dtype=np.float64)
        curv = float(d @ Bd)
        if curv <= 0:
            return (-g if j == 0 else z), j + 1
        alpha = rr / curv
        z = z + alpha * d
        r = r + alpha * Bd
        rr_new = float(r @ r)
        if math.sqrt(rr_new) < eps:
            return z, j + 1
        d = -r + (rr_new / rr) * d
        rr = rr_new
    return z, maxiter


def newton_cg(fun_grad: Callable[[np.ndarray], tuple[float, np.ndarray]],
              hessp: Callable[[np.ndarray, np.ndarray], np.ndarray],
              x0, xtol: float = 1e-8, gtol: float = 0.0, maxiter: Optional[int] = None,
              cg_maxiter: Optional[int] = None, time_limit: Optional[float] = None) -> FitResult:
    """Minimise f with exact gradients and Hessian-vector products
    (N&W Algorithm 7.1 with a strong-Wolfe line search).  A Newton step whose
    mean absolute size is already below xtol ends the fit before its line
    search (the remaining change is below the requested resolution)."""
    t0 = time.perf_counter()
    x = np.array(x0, dtype=np.float64)
    n = x.size
    maxiter = 200 * n if maxiter is None else maxiter
    cg_maxiter = 20 * n if cg_maxiter is None else cg_maxiter
    counts = {"f": 0, "h": 0}

    def fg(xx):
        counts["f"] += 1
        f, g = fun_grad(xx)
        return float(f), np.asarray(g, dtype=np.float64)

    f, g = fg(x)
    status, k = MAXITER, 0
    while k < maxiter:
        if gtol > 0 and np.max(np.abs(g)) <= gtol:
            status = CONVERGED_GTOL
            break
        gnorm = float(np.linalg.norm(g))
        eps = min(0.5, math.sqrt(gnorm)) * gnorm
        p, nh = inner_cg(lambda d: hessp(x, d), g, eps, cg_maxiter)
        counts["h"] += nh
        k += 1
        if np.mean(np.abs(p)) <= xtol:
            status = CONVERGED_XTOL
            break
        df0 = float(g @ p)
        if df0 >= 0:  # not a descent direction (round-off): fall back to -g
            p = -g
            df0 = float(g @ p)
        cache = {}

        def phi(a):
            xa = x + a * p
            fa, ga = fg(xa)
            cache[a] = (xa, fa, ga)
            return fa, float(ga @ p)

        ls = wolfe_line_search(phi, f, df0)
        if ls is None:
            resolution = 1e3 * np.finfo(np.float64).eps * max(1.0, abs(f))
            status = PRECISION_LIMIT if abs(df0) <= resolution else LINESEARCH_FAILED
            break
        a, _, _ = ls
        xa, fa, ga = cache[a]
        step = xa - x
        x, f, g = xa, fa, ga
        if np.mean(np.abs(step)) <= xtol:
            status = CONVERGED_XTOL
            break
        if time_limit is not None and time.perf_counter() - t0 > time_limit:
            status = TIME_LIMIT
            break
    return FitResult(x=x, fun=f, grad=g, status=status, iters=k, n_fev=counts["f"],
                     n_gev=counts["f"], n_hvp=counts["h"], elapsed=time.perf_counter() - t0)
