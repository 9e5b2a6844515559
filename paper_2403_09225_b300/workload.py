"""Seeded synthetic workloads for the PWA likelihood (input generation only).

This module is the one piece shared by the CPU oracle and the CUDA library:
it draws events, builds the parameter-free amplitude tensor F and samples
resonance parameters.  It holds none of the likelihood arithmetic.  Where a
data sample has to follow the model intensity I(e; theta_true) (accept-reject,
paper Sec. 3: the test sample is generated from the PWA model itself), the
intensity is supplied by the caller as a function, so the oracle and the GPU
path each bring their own.

Kinematics (the decay studied in paper Sec. 3 is a three-body decay; the
synthetic stand-in keeps a three-body topology):
  parent mass 3.097 GeV, daughters 0.1396, 0.1396, 1.0195 GeV,
  channels ch = 0 (m12), 1 (m13), 2 (m23), events uniform in the Dalitz plot.
Amplitude projections (the parameter-free U of Eq. 1, precomputed once):
  F_{k,s}(e) = P_J(cos theta_ch) * B_J(q_ch) * exp(i s phi_ch),   s = 0..S-1,
  with P_J the Legendre polynomial of the resonance spin, B_J the
  Blatt-Weisskopf barrier factor (von Hippel-Quigg form, z = (q r)^2,
  r = 3 GeV^-1), theta_ch the helicity angle of the lower-index daughter of the
  pair in the pair rest frame and phi_ch the azimuth of the pair direction in
  the parent frame after an isotropic random orientation of each event.

Random numbers: numpy's Philox counter-based generator, one independent stream
per purpose (table, MC, data, starts) derived from (seed, stream id).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

PARENT_MASS = 3.097
DAUGHTER_MASSES = (0.1396, 0.1396, 1.0195)
BARRIER_RADIUS = 3.0  # GeV^-1
#: channel -> (a, b, spectator) daughter indices; ch 0 = m12, 1 = m13, 2 = m23
CHANNEL_PAIRS = ((0, 1, 2), (0, 2, 1), (1, 2, 0))
BASE_SEED = 20240314

STREAM_TABLE, STREAM_MC, STREAM_DATA, STREAM_STARTS, STREAM_POOL = range(5)


def rng_stream(seed: int, stream: int) -> np.random.Generator:
    """Independent Philox stream for (seed, stream id)."""
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(stream)])))


def channel_mass_range(ch: int) -> tuple[float, float]:
    a, b, c = CHANNEL_PAIRS[ch]
    return (DAUGHTER_MASSES[a] + DAUGHTER_MASSES[b], PARENT_MASS - DAUGHTER_MASSES[c])


def _other_range(u: np.ndarray, a: int, b: int, c: int):
    """Range of m_bc^2 given m_ab^2 = u (standard Dalitz-plot boundary)."""
    M = PARENT_MASS
    ma, mb, mc = DAUGHTER_MASSES[a], DAUGHTER_MASSES[b], DAUGHTER_MASSES[c]
    su = np.sqrt(u)
    Eb = (u - ma * ma + mb * mb) / (2 * su)
    Ec = (M * M - u - mc * mc) / (2 * su)
    pb = np.sqrt(np.maximum(Eb * Eb - mb * mb, 0.0))
    pc = np.sqrt(np.maximum(Ec * Ec - mc * mc, 0.0))
    s = (Eb + Ec) ** 2
    return s - (pb + pc) ** 2, s - (pb - pc) ** 2


def _sum_m2() -> float:
    return PARENT_MASS ** 2 + sum(m * m for m in DAUGHTER_MASSES)


# ---------------------------------------------------------------------------
# resonance table and the parameter prior
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Resonance:
    channel: int
    spin: int
    mass: float
    width: float
    mag: float
    phase: float
    fix_coupling: bool = False
    fix_mass: bool = False
    fix_width: bool = False


WIDTH_PRIOR = (0.02, 0.3)
MAG_PRIOR = (0.5, 2.0)


def sample_table(rng: np.random.Generator, K: int, j_max: int, all_m12: bool) -> list[Resonance]:
    """Resonance table from the prior: channel = k mod 3 (or all m12),
    M ~ U(channel mass range), Gamma ~ U[0.02, 0.3], rho ~ U[0.5, 2],
    phi ~ U(-pi, pi], spin ~ U{0..j_max}; resonance 0 has its coupling fixed
    to 1 (the overall scale and phase of the couplings are not observable)."""
    table = []
    for k in range(K):
        ch = 0 if all_m12 else k % 3
        lo, hi = channel_mass_range(ch)
        spin = int(rng.integers(0, j_max + 1))
        mass = float(rng.uniform(lo, hi))
        width = float(rng.uniform(*WIDTH_PRIOR))
        mag = float(rng.uniform(*MAG_PRIOR))
        phase = float(math.pi - rng.uniform(0.0, 2 * math.pi))
        if k == 0:
            mag, phase = 1.0, 0.0
        table.append(Resonance(ch, spin, mass, width, mag, phase, fix_coupling=(k == 0)))
    return table


def free_parameter_vector(table: list[Resonance]) -> np.ndarray:
    """theta in the library's order: free magnitudes, free phases, free masses,
    free widths, each block in resonance order."""
    rho = [r.mag for r in table if not r.fix_coupling]
    phi = [r.phase for r in table if not r.fix_coupling]
    M = [r.mass for r in table if not r.fix_mass]
    G = [r.width for r in table if not r.fix_width]
    return np.array(rho + phi + M + G, dtype=np.float64)


def sample_start(rng: np.random.Generator, table: list[Resonance]) -> np.ndarray:
    """A random starting point drawn from the same prior, in theta order."""
    rho, phi, M, G = [], [], [], []
    for r in table:
        if not r.fix_coupling:
            rho.append(rng.uniform(*MAG_PRIOR))
            phi.append(math.pi - rng.uniform(0.0, 2 * math.pi))
        if not r.fix_mass:
            M.append(rng.uniform(*channel_mass_range(r.channel)))
        if not r.fix_width:
            G.append(rng.uniform(*WIDTH_PRIOR))
    return np.array(rho + phi + M + G, dtype=np.float64)


# ---------------------------------------------------------------------------
# phase space and amplitude projections
# ---------------------------------------------------------------------------

def dalitz_bounds() -> tuple[float, float, float, float]:
    """Bounding box (x = m12^2, y = m23^2)."""
    lo12, hi12 = channel_mass_range(0)
    lo23, hi23 = channel_mass_range(2)
    return lo12 ** 2, hi12 ** 2, lo23 ** 2, hi23 ** 2


def inside_dalitz(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    ylo, yhi = _other_range(x, 0, 1, 2)
    return (y >= ylo) & (y <= yhi)


def uniform_dalitz(rng: np.random.Generator, n: int) -> tuple[np.ndarray, np.ndarray]:
    """n points uniform over the Dalitz region by rejection from the box."""
    x0, x1, y0, y1 = dalitz_bounds()
    xs, ys, have = [], [], 0
    while have < n:
        m = max(1024, int((n - have) * 1.6))
        x = rng.uniform(x0, x1, m)
        y = rng.uniform(y0, y1, m)
        ok = inside_dalitz(x, y)
        xs.append(x[ok]); ys.append(y[ok]); have += int(ok.sum())
    return np.concatenate(xs)[:n], np.concatenate(ys)[:n]


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices (unit quaternions, Shoemake 1992)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    qx, qy = a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2)
    qz, qw = b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (qy * qy + qz * qz); R[:, 0, 1] = 2 * (qx * qy - qz * qw); R[:, 0, 2] = 2 * (qx * qz + qy * qw)
    R[:, 1, 0] = 2 * (qx * qy + qz * qw); R[:, 1, 1] = 1 - 2 * (qx * qx + qz * qz); R[:, 1, 2] = 2 * (qy * qz - qx * qw)
    R[:, 2, 0] = 2 * (qx * qz - qy * qw); R[:, 2, 1] = 2 * (qy * qz + qx * qw); R[:, 2, 2] = 1 - 2 * (qx * qx + qy * qy)
    return R


@dataclasses.dataclass
class Kinematics:
    m2: np.ndarray     # [3, n] float64: m12^2, m13^2, m23^2
    cos: np.ndarray    # [3, n] helicity cosine per channel
    phi: np.ndarray    # [3, n] azimuth of the pair direction per channel
    q: np.ndarray      # [3, n] breakup momentum per channel

    @property
    def n(self) -> int:
        return self.m2.shape[1]


def kinematics(rng: np.random.Generator, x: np.ndarray, y: np.ndarray) -> Kinematics:
    """Angles and momenta for Dalitz points (x = m12^2, y = m23^2), each event
    given an isotropic random orientation drawn from rng."""
    n = x.shape[0]
    M = PARENT_MASS
    m = DAUGHTER_MASSES
    z = _sum_m2() - x - y  # m13^2
    m2 = np.stack([x, z, y])  # channel order m12, m13, m23
    # momenta in the parent rest frame: p3 along +z, p1 in the xz plane
    # E_i = (M^2 + m_i^2 - m_jk^2) / 2M with (jk) the pair that excludes daughter i
    pair_of = {0: 2, 1: 1, 2: 0}  # daughter i -> channel whose pair excludes i
    E = [(M * M + m[i] ** 2 - m2[pair_of[i]]) / (2 * M) for i in range(3)]
    p = [np.sqrt(np.maximum(E[i] ** 2 - m[i] ** 2, 0.0)) for i in range(3)]
    # p1.p3 from m13^2 = m1^2 + m3^2 + 2 (E1 E3 - p1.p3)
    dot13 = (m[0] ** 2 + m[2] ** 2 + 2 * E[0] * E[2] - m2[1]) / 2
    cosa = np.clip(dot13 / np.maximum(p[0] * p[2], 1e-300), -1.0, 1.0)
    sina = np.sqrt(1 - cosa * cosa)
    P = np.zeros((3, n, 3))
    P[2, :, 2] = p[2]
    P[0, :, 0] = p[0] * sina
    P[0, :, 2] = p[0] * cosa
    P[1] = -P[0] - P[2]
    R = _random_rotations(rng, n)
    Prot = np.einsum('nij,dnj->dni', R, P)
    cos = np.empty((3, n)); phi = np.empty((3, n)); q = np.empty((3, n))
    for ch, (a, b, c) in enumerate(CHANNEL_PAIRS):
        u = m2[ch]
        su = np.sqrt(u)
        ma, mb, mc = m[a], m[b], m[c]
        # pair rest frame: energy/momentum of daughter a and of the spectator c
        Ea = (u + ma * ma - mb * mb) / (2 * su)
        Ec = (M * M - u - mc * mc) / (2 * su)
        pa = np.sqrt(np.maximum(Ea * Ea - ma * ma, 0.0))
        pc = np.sqrt(np.maximum(Ec * Ec - mc * mc, 0.0))
        # m_ac^2 from the other channel: invariant of (a, c)
        ch_ac = [i for i, pr in enumerate(CHANNEL_PAIRS) if set(pr[:2]) == {a, c}][0]
        mac2 = m2[ch_ac]
        # angle between a and the pair direction (= -p_c in the pair frame)
        cos[ch] = np.clip((mac2 - ma * ma - mc * mc - 2 * Ea * Ec) / np.maximum(2 * pa * pc, 1e-300), -1.0, 1.0)
        d = -Prot[c]
        phi[ch] = np.arctan2(d[:, 1], d[:, 0])
        q[ch] = pa
    return Kinematics(m2=m2, cos=cos, phi=phi, q=q)


def legendre(J: int, x: np.ndarray) -> np.ndarray:
    if J == 0:
        return np.ones_like(x)
    if J == 1:
        return x
    if J == 2:
        return 0.5 * (3 * x * x - 1)
    if J == 3:
        return 0.5 * (5 * x ** 3 - 3 * x)
    if J == 4:
        return (35 * x ** 4 - 30 * x * x + 3) / 8
    raise ValueError("spin must be 0..4")


def blatt_weisskopf(J: int, q: np.ndarray) -> np.ndarray:
    """Unnormalised Blatt-Weisskopf barrier factor, z = (q r)^2."""
    z = (q * BARRIER_RADIUS) ** 2
    if J == 0:
        return np.ones_like(z)
    if J == 1:
        return np.sqrt(2 * z / (1 + z))
    if J == 2:
        return np.sqrt(13 * z * z / ((z - 3) ** 2 + 9 * z))
    if J == 3:
        return np.sqrt(277 * z ** 3 / (z * (z - 15) ** 2 + 9 * (2 * z - 5) ** 2))
    if J == 4:
        return np.sqrt(12746 * z ** 4 / ((z * z - 45 * z + 105) ** 2 + 25 * z * (2 * z - 21) ** 2))
    raise ValueError("spin must be 0..4")


def amplitudes(kin: Kinematics, table: list[Resonance], S: int) -> np.ndarray:
    """F[n, K, S] complex64 (interleaved re/im when viewed as float32)."""
    n = kin.n
    spins = sorted({r.spin for r in table})
    # radial part P_J(cos) B_J(q) per (channel, spin), phase e^{i s phi} per (channel, s)
    radial = np.empty((n, 3, max(spins) + 1), dtype=np.float32)
    for ch in range(3):
        for J in spins:
            radial[:, ch, J] = legendre(J, kin.cos[ch]) * blatt_weisskopf(J, kin.q[ch])
    phase = np.empty((n, 3, S), dtype=np.complex64)
    for ch in range(3):
        e1 = np.exp(1j * kin.phi[ch])
        p = np.ones(n, dtype=np.complex128)
        for s in range(S):
            phase[:, ch, s] = p
            p = p * e1
    ch = np.array([r.channel for r in table])
    J = np.array([r.spin for r in table])
    return radial[:, ch, J][:, :, None] * phase[:, ch, :]


# ---------------------------------------------------------------------------
# samples
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Sample:
    """One event sample in the library's input layout."""
    m2: np.ndarray                 # [3, n] float32, channel-major
    F: np.ndarray                  # [n, K, S] complex64
    w: Optional[np.ndarray] = None  # [n] float32 or None (= 1)

    @property
    def n(self) -> int:
        return self.m2.shape[1]


def _phase_space_chunk(args):
    seed, n, table, S = args
    rng = np.random.Generator(np.random.Philox(seed))
    x, y = uniform_dalitz(rng, n)
    kin = kinematics(rng, x, y)
    return kin.m2.astype(np.float32), amplitudes(kin, table, S)


def phase_space_sample(rng: np.random.Generator, n: int, table: list[Resonance], S: int,
                       chunk: int = 1 << 17, threads: int = 8) -> Sample:
    """n phase-space events (the MC sample; efficiency = 1, paper Eq. 2).
    Chunks draw from their own Philox streams seeded from rng, so the result
    does not depend on the number of threads."""
    from concurrent.futures import ThreadPoolExecutor
    m2 = np.empty((3, n), dtype=np.float32)
    F = np.empty((n, len(table), S), dtype=np.complex64)
    starts = list(range(0, n, chunk))
    seeds = rng.integers(0, 2 ** 63 - 1, size=len(starts))
    jobs = [(int(sd), min(n, a + chunk) - a, table, S) for sd, a in zip(seeds, starts)]

    def run(i):
        a = starts[i]
        cm2, cF = _phase_space_chunk(jobs[i])
        m2[:, a:a + cm2.shape[1]] = cm2
        F[a:a + cm2.shape[1]] = cF

    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        list(ex.map(run, range(len(jobs))))
    return Sample(m2=m2, F=F)


IntensityFn = Callable[[np.ndarray, np.ndarray], np.ndarray]


class Proposal:
    """Candidate density for accept-reject sampling of data events: a mixture
    of the uniform Dalitz density and, per resonance k, a density that is a
    truncated Cauchy (Breit-Wigner shape) in the channel invariant u times a
    density proportional to P_J(c)^2 + delta in the helicity cosine c, which is
    linear in the other Dalitz variable at fixed u.  density() is the exact
    normalised density over the Dalitz region, so any bound C >= I/q yields an
    unbiased sample."""

    DELTA = 0.1

    def __init__(self, table: list[Resonance], uniform_weight: float = 0.1):
        from scipy import integrate
        self.table = table
        x0, x1, _, _ = dalitz_bounds()
        self.area = integrate.quad(lambda x: float(np.diff(_other_range(np.array(x), 0, 1, 2))[0]),
                                   x0, x1, limit=200, epsabs=0, epsrel=1e-12)[0]
        self.comp = []
        mass_w = []
        for r in table:
            lo, hi = channel_mass_range(r.channel)
            mu, gam = r.mass ** 2, r.mass * r.width
            t0, t1 = math.atan((lo * lo - mu) / gam), math.atan((hi * hi - mu) / gam)
            self.comp.append((r.channel, r.spin, mu, gam, t0, t1))
            # expected share of the intensity: peak area x barrier^2 x <P_J^2> x range
            u = np.array([min(max(mu, lo * lo * 1.0001), hi * hi * 0.9999)])
            _, _, olo, ohi = self._u_and_other(r.channel, *self._point(r.channel, u, 0.5))
            a, b, c = CHANNEL_PAIRS[r.channel]
            su = np.sqrt(u)
            Ea = (u + DAUGHTER_MASSES[a] ** 2 - DAUGHTER_MASSES[b] ** 2) / (2 * su)
            q = np.sqrt(np.maximum(Ea * Ea - DAUGHTER_MASSES[a] ** 2, 0.0))
            bw2 = float(blatt_weisskopf(r.spin, q)[0] ** 2)
            mass_w.append(r.mag ** 2 * bw2 * (t1 - t0) * float((ohi - olo)[0])
                          / ((2 * r.spin + 1) * r.mass * r.width))
        mass_w = np.array(mass_w)
        self.weights = np.concatenate([[uniform_weight], (1 - uniform_weight) * mass_w / mass_w.sum()])

    @staticmethod
    def _u_and_other(ch: int, x, y):
        """(channel invariant u, the other sampled coordinate, its range)."""
        if ch == 0:
            lo, hi = _other_range(x, 0, 1, 2)
            return x, y, lo, hi
        if ch == 2:
            lo, hi = _other_range(y, 2, 1, 0)
            return y, x, lo, hi
        u = _sum_m2() - x - y
        lo, hi = _other_range(u, 2, 0, 1)
        return u, x, lo, hi

    @staticmethod
    def _point(ch: int, u, frac):
        """Dalitz point (x, y) for channel invariant u and the other variable
        at fraction frac of its allowed range."""
        if ch == 0:
            lo, hi = _other_range(u, 0, 1, 2)
            return u, lo + frac * (hi - lo)
        if ch == 2:
            lo, hi = _other_range(u, 2, 1, 0)
            return lo + frac * (hi - lo), u
        lo, hi = _other_range(u, 2, 0, 1)
        xx = lo + frac * (hi - lo)
        return xx, _sum_m2() - xx - u

    def _angular(self, J: int, c):
        return (legendre(J, c) ** 2 + self.DELTA) / (2.0 / (2 * J + 1) + 2 * self.DELTA)

    def density(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        q = np.full_like(x, self.weights[0] / self.area)
        for wk, (ch, J, mu, gam, t0, t1) in zip(self.weights[1:], self.comp):
            u, other, lo, hi = self._u_and_other(ch, x, y)
            L = np.maximum(hi - lo, 1e-300)
            c = np.clip(2 * (other - lo) / L - 1, -1.0, 1.0)
            cauchy = gam / (np.pi * ((u - mu) ** 2 + gam * gam)) / ((t1 - t0) / np.pi)
            q += wk * cauchy * self._angular(J, c) * 2.0 / L
        return q

    def _sample_cos(self, rng: np.random.Generator, J: int, n: int) -> np.ndarray:
        out, have = [], 0
        while have < n:
            m = max(256, 2 * (n - have) * (2 * J + 1))
            c = rng.uniform(-1.0, 1.0, m)
            keep = rng.random(m) * (1 + self.DELTA) < legendre(J, c) ** 2 + self.DELTA
            out.append(c[keep]); have += int(keep.sum())
        return np.concatenate(out)[:n]

    def sample(self, rng: np.random.Generator, n: int) -> tuple[np.ndarray, np.ndarray]:
        which = rng.choice(len(self.weights), size=n, p=self.weights)
        x = np.empty(n); y = np.empty(n)
        sel = which == 0
        x[sel], y[sel] = uniform_dalitz(rng, int(sel.sum()))
        for k, (ch, J, mu, gam, t0, t1) in enumerate(self.comp):
            sel = which == k + 1
            m = int(sel.sum())
            if m == 0:
                continue
            u = mu + gam * np.tan(rng.uniform(t0, t1, m))
            frac = 0.5 * (self._sample_cos(rng, J, m) + 1)
            x[sel], y[sel] = self._point(ch, u, frac)
        return x, y


def accept_reject_sample(rng: np.random.Generator, n: int, table: list[Resonance], S: int,
                         intensity: IntensityFn, pool: int = 200_000, safety: float = 1.5,
                         chunk: int = 1 << 19) -> tuple[Sample, dict]:
    """n data events distributed as I(e; table) over phase space.

    Candidates come from Proposal; a candidate is kept when u * C * q < I with
    u ~ U[0,1) and C = safety * max(I/q) over a pool of candidates.  Every
    candidate whose I/q exceeds C is counted; if any appears, C is raised and
    the acceptance restarts from the first chunk with the same random draws.
    """
    prop = Proposal(table)
    px, py = prop.sample(rng, pool)
    pk = kinematics(rng, px, py)
    ratio = intensity(pk.m2.astype(np.float32), amplitudes(pk, table, S)) / prop.density(px, py)
    C = safety * float(np.max(ratio))
    stats = {"pool": pool, "C": C, "candidates": 0, "restarts": 0}
    # candidates per chunk: enough for the whole sample at the pool's mean acceptance
    accept = float(np.mean(ratio)) / C
    chunk = int(min(chunk, max(16384, 1.3 * n / max(accept, 1e-6))))
    state = rng.bit_generator.state
    while True:
        rng.bit_generator.state = state
        m2s, Fs, have, exceeded = [], [], 0, 0.0
        cand = kept = 0
        while have < n:
            x, y = prop.sample(rng, chunk)
            kin = kinematics(rng, x, y)
            m2 = kin.m2.astype(np.float32)
            F = amplitudes(kin, table, S)
            I = intensity(m2, F)
            r = I / prop.density(x, y)
            u = rng.random(chunk)
            cand += chunk
            exceeded = max(exceeded, float(r.max()))
            if exceeded > C:
                break
            keep = u * C < r
            kept += int(keep.sum())
            m2s.append(m2[:, keep]); Fs.append(F[keep]); have += int(keep.sum())
        if exceeded > C:
            C = safety * exceeded
            stats["restarts"] += 1
            continue
        stats.update(C=C, candidates=cand, efficiency=kept / cand)
        m2 = np.concatenate(m2s, axis=1)[:, :n]
        F = np.concatenate(Fs)[:n]
        return Sample(m2=np.ascontiguousarray(m2), F=np.ascontiguousarray(F), w=None), stats


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Config:
    name: str
    K: int
    S: int
    n_data: int
    n_mc: int
    j_max: int
    all_m12: bool
    seed_offset: int


CONFIGS = {
    # K=3 resonances in m12, spins 0..2, S=2, 2e4 data + 1e5 MC
    "tiny": Config("tiny", 3, 2, 20_000, 100_000, 2, True, 0),
    # the same with K=4 (14 real parameters)
    "tiny_k4": Config("tiny_k4", 4, 2, 20_000, 100_000, 2, True, 0),
    # K=20 over the three channels, spins 0..4, S=4, 1e6 data + 5e6 MC
    "paper": Config("paper", 20, 4, 1_000_000, 5_000_000, 4, False, 1),
    # K=40, S=4, 2e6 data + 1e7 MC
    "diff": Config("diff", 40, 4, 2_000_000, 10_000_000, 4, False, 2),
}


@dataclasses.dataclass
class Workload:
    config: Config
    table: list[Resonance]
    theta_true: np.ndarray
    data: Sample
    mc: Sample
    stats: dict

    @property
    def K(self) -> int:
        return self.config.K

    @property
    def S(self) -> int:
        return self.config.S

    @property
    def channels(self) -> np.ndarray:
        return np.array([r.channel for r in self.table], dtype=np.int32)


def make_table(config: Config, seed: int = BASE_SEED) -> list[Resonance]:
    return sample_table(rng_stream(seed + config.seed_offset, STREAM_TABLE), config.K,
                        config.j_max, config.all_m12)


def make_workload(config: Config | str, intensity: Optional[IntensityFn] = None,
                  n_data: Optional[int] = None, n_mc: Optional[int] = None,
                  seed: int = BASE_SEED) -> Workload:
    """Build a workload.  With intensity=None the data sample is drawn from
    phase space (unweighted), which keeps every property the likelihood needs
    but not the resonance structure of real data."""
    if isinstance(config, str):
        config = CONFIGS[config]
    s = seed + config.seed_offset
    table = make_table(config, seed)
    nd = config.n_data if n_data is None else n_data
    nm = config.n_mc if n_mc is None else n_mc
    mc = phase_space_sample(rng_stream(s, STREAM_MC), nm, table, config.S)
    if intensity is None:
        data = phase_space_sample(rng_stream(s, STREAM_DATA), nd, table, config.S)
        stats = {"data": "phase space"}
    else:
        data, stats = accept_reject_sample(rng_stream(s, STREAM_DATA), nd, table, config.S, intensity)
    return Workload(config, table, free_parameter_vector(table), data, mc, stats)


def random_starts(workload: Workload, count: int, seed: int = BASE_SEED) -> np.ndarray:
    rng = rng_stream(seed + workload.config.seed_offset, STREAM_STARTS)
    return np.stack([sample_start(rng, workload.table) for _ in range(count)])
