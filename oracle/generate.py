"""CPU oracle of the pseudo-experiment generator -- TEST INFRASTRUCTURE.

Accept-reject from a pool by the model intensity (paper Sec. 3 draws its test
samples from the PWA model itself), written out from the definitions:
  * u_j = (z >> 11) 2^-53 with z output j + 1 of splitmix64 started at the
    seed (Steele, Lea and Flood 2014: state += 0x9E3779B97F4A7C15, then the
    two xor-shift-multiply rounds and a final xor-shift);
  * event j kept when u_j C < I_j (double precision), taken in the order
    start, start + 1, ..., n - 1, 0, ..., start - 1, the first n_target kept;
  * the binned Dalitz plot of the kept events, bin
    floor((x - x0) nb / (x1 - x0)) clamped, and log(1 + count nb^2 / n).
Nothing here is imported by the library.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, j: np.ndarray) -> np.ndarray:
    """Output j + 1 (j = 0, 1, ...) of splitmix64 started at `seed`."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(j, dtype=np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniforms(seed: int, j: np.ndarray) -> np.ndarray:
    return (splitmix64(seed, j) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def accept_reject(I: np.ndarray, C: float, seed: int, start: int, n_target: int):
    """(pool indices of the first n_target kept events, C applied)."""
    I = np.asarray(I, dtype=np.float32).astype(np.float64)
    n = I.size
    if C <= 0:
        C = float(I.max())
    order = (start + np.arange(n)) % n
    keep = uniforms(seed, order) * C < I[order]
    return order[keep][:n_target].astype(np.int64), C


def dalitz_histogram(m2: np.ndarray, idx: np.ndarray, nb: int, bounds, log_scale: bool = True) -> np.ndarray:
    """[nb * nb] at bx * nb + by for x = m12^2 = m2[0], y = m23^2 = m2[2]."""
    x0, x1, y0, y1 = bounds
    x = np.asarray(m2[0], dtype=np.float32)[idx].astype(np.float64)
    y = np.asarray(m2[2], dtype=np.float32)[idx].astype(np.float64)
    bx = np.clip(np.floor((x - x0) * nb / (x1 - x0)), 0, nb - 1).astype(np.int64)
    by = np.clip(np.floor((y - y0) * nb / (y1 - y0)), 0, nb - 1).astype(np.int64)
    h = np.bincount(bx * nb + by, minlength=nb * nb).astype(np.float64)
    if log_scale:
        h = np.log1p(h * (nb * nb / len(idx))) if len(idx) else h
    return h
