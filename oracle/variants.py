"""CPU oracle of the physics variants -- TEST INFRASTRUCTURE.

Nothing in the library imports this module; the tests compare the library's
variant kernels against it.

Model (paper Sec. 2.2, Eq. 1, with Eq. 3 for the likelihood): the intensity
I(e) = sum_s |A_s(e)|^2 with A_s = sum_k g_ks BW_k(m_e) F_ks(e), where the
coupling g_ks = rho_ks e^{i phi_ks} is one per resonance (g_ks = g_k, the
form Eq. 1 writes) or one per (resonance, projection) (each partial wave of a
resonance with its own coupling), and BW_k = 1 / D_k is one of three line
shapes of the resonance's pair mass m (m^2 = the channel's invariant):
  constant width     D = M^2 - m^2 - i M Gamma
  mass-dependent     D = M^2 - m^2 - i M Gamma(m),
                     Gamma(m) = Gamma0 (q(m) / q(M)) (M / m) (F_L(q(m)) / F_L(q(M)))^2
                     (q the pair's breakup momentum, F_L the von Hippel-Quigg
                     barrier factor of the resonance's spin L, z = (q r)^2)
  Flatte             D = M^2 - m^2 - i (gamma1 rho1(m) + gamma2 rho2(m)),
                     rho_i = 2 q_i(m) / m with q_i the breakup momentum for the
                     i-th channel's masses, q_i = i sqrt(-q_i^2) below its
                     threshold.
NLL = -sum_data w ln I + N_d ln((1 / N_mc) sum_mc I) (Eq. 3, N_d = sum w).

theta order: free magnitudes (resonance-major, then projection when the
couplings are per projection), free phases (same order), free masses, free
first width parameters (Gamma, Gamma0 or gamma1), free gamma2 (Flatte
resonances).  fix_coupling fixes all couplings of a resonance, fix_width
both width parameters.

Derivatives are exact: the NLL is evaluated in hyper-dual arithmetic (Fike
and Alonso, AIAA 2011-886): with theta + e1 v + e2 u, e1^2 = e2^2 = 0, the e2
part of the NLL is grad . u and the e1 e2 part is u^T H v, so P evaluations
with u the unit vectors give the gradient and H v.  That is the plain
definition of both, independent of the adjoint formulas the kernels use.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np

KIND_CONSTANT, KIND_MASS_DEPENDENT, KIND_FLATTE = 0, 1, 2


class HD:
    """Hyper-dual number a + b e1 + c e2 + d e1 e2 over numpy arrays (real or complex)."""
    __slots__ = ("a", "b", "c", "d")

    def __init__(self, a, b=0.0, c=0.0, d=0.0):
        self.a, self.b, self.c, self.d = a, b, c, d

    @staticmethod
    def lift(x):
        return x if isinstance(x, HD) else HD(x)

    def __add__(self, o):
        o = HD.lift(o)
        return HD(self.a + o.a, self.b + o.b, self.c + o.c, self.d + o.d)

    __radd__ = __add__

    def __neg__(self):
        return HD(-self.a, -self.b, -self.c, -self.d)

    def __sub__(self, o):
        return self + (-HD.lift(o))

    def __rsub__(self, o):
        return HD.lift(o) + (-self)

    def __mul__(self, o):
        o = HD.lift(o)
        return HD(self.a * o.a, self.a * o.b + self.b * o.a, self.a * o.c + self.c * o.a,
                  self.a * o.d + self.b * o.c + self.c * o.b + self.d * o.a)

    __rmul__ = __mul__

    def _chain(self, f0, f1, f2):
        """f(self) for a function with value f0, first derivative f1 and second f2 at self.a."""
        return HD(f0, f1 * self.b, f1 * self.c, f1 * self.d + f2 * self.b * self.c)

    def inv(self):
        r = 1.0 / self.a
        return self._chain(r, -r * r, 2 * r * r * r)

    def __truediv__(self, o):
        return self * HD.lift(o).inv()

    def __rtruediv__(self, o):
        return HD.lift(o) * self.inv()

    def conj(self):
        return HD(np.conj(self.a), np.conj(self.b), np.conj(self.c), np.conj(self.d))

    def real(self):
        return HD(np.real(self.a), np.real(self.b), np.real(self.c), np.real(self.d))

    def log(self):
        return self._chain(np.log(self.a), 1.0 / self.a, -1.0 / (self.a * self.a))

    def sqrt(self):
        r = np.sqrt(self.a)
        return self._chain(r, 0.5 / r, -0.25 / (r * self.a))

    def exp_i(self):
        """e^{i self} for real self."""
        e = np.exp(1j * self.a)
        return self._chain(e, 1j * e, -e)

    def sum(self):
        return HD(np.sum(self.a), np.sum(self.b), np.sum(self.c), np.sum(self.d))


@dataclasses.dataclass
class Shape:
    """Line shape of one resonance (the arguments of the library's
    pwa_lineshape): kind, the pair's daughter masses (ma, mb) (Flatte:
    channel 1), the Flatte channel 2 masses (mc, md), the barrier radius for
    the mass-dependent width, and gamma2's initial value."""
    kind: int = KIND_CONSTANT
    ma: float = 0.0
    mb: float = 0.0
    mc: float = 0.0
    md: float = 0.0
    radius: float = 3.0
    width2: float = 0.0


@dataclasses.dataclass
class VariantModel:
    channels: np.ndarray
    spins: np.ndarray
    S: int
    per_projection: bool
    shapes: list
    mag: np.ndarray          # [K] initial / fixed magnitude (all projections)
    phase: np.ndarray
    mass: np.ndarray
    width: np.ndarray        # Gamma, Gamma0 or gamma1
    fix_coupling: np.ndarray
    fix_mass: np.ndarray
    fix_width: np.ndarray

    @classmethod
    def from_table(cls, table, S: int, shapes: Optional[Sequence[Shape]] = None, per_projection: bool = False):
        K = len(table)
        shapes = list(shapes) if shapes is not None else [Shape() for _ in range(K)]
        return cls(np.array([r.channel for r in table]), np.array([r.spin for r in table]), S, per_projection,
                   shapes, np.array([r.mag for r in table], float), np.array([r.phase for r in table], float),
                   np.array([r.mass for r in table], float), np.array([r.width for r in table], float),
                   np.array([r.fix_coupling for r in table], bool), np.array([r.fix_mass for r in table], bool),
                   np.array([r.fix_width for r in table], bool))

    @property
    def K(self) -> int:
        return len(self.channels)

    def layout(self):
        """Lists of (name, k, s) in theta order."""
        K, S = self.K, self.S
        ns = S if self.per_projection else 1
        out = []
        for name in ("mag", "phase"):
            for k in range(K):
                if not self.fix_coupling[k]:
                    out += [(name, k, s) for s in range(ns)]
        out += [("mass", k, 0) for k in range(K) if not self.fix_mass[k]]
        out += [("w1", k, 0) for k in range(K) if not self.fix_width[k]]
        out += [("w2", k, 0) for k in range(K) if not self.fix_width[k] and self.shapes[k].kind == KIND_FLATTE]
        return out

    @property
    def P(self) -> int:
        return len(self.layout())

    def theta0(self) -> np.ndarray:
        vals = []
        for name, k, s in self.layout():
            vals.append({"mag": self.mag[k], "phase": self.phase[k], "mass": self.mass[k], "w1": self.width[k],
                         "w2": self.shapes[k].width2}[name])
        return np.array(vals)


def breakup_q2(m2, ma: float, mb: float):
    """q^2 of a pair of masses (ma, mb) at invariant mass^2 m2."""
    return (m2 - (ma + mb) ** 2) * (m2 - (ma - mb) ** 2) / (4.0 * m2)


def barrier_sq(L: int, z):
    """F_L(z)^2, von Hippel-Quigg form (unnormalised), z = (q r)^2."""
    if L == 0:
        return 1.0 + 0.0 * z
    if L == 1:
        return 2 * z / (1 + z)
    if L == 2:
        return 13 * z * z / ((z - 3) * (z - 3) + 9 * z)
    if L == 3:
        return 277 * z * z * z / (z * (z - 15) * (z - 15) + 9 * (2 * z - 5) * (2 * z - 5))
    if L == 4:
        return 12746 * z ** 4 / ((z * z - 45 * z + 105) ** 2 + 25 * z * (2 * z - 21) ** 2)
    raise ValueError("spin must be 0..4")


def _hd_pair(M, ma, mb):
    """q^2 at m^2 = M^2 for a hyper-dual mass M."""
    M2 = M * M
    return (M2 - (ma + mb) ** 2) * (M2 - (ma - mb) ** 2) / (4.0 * M2)


def _barrier_sq_hd(L: int, z: HD) -> HD:
    if L == 0:
        return HD(1.0)
    if L == 1:
        return 2 * z / (1 + z)
    if L == 2:
        return 13 * z * z / ((z - 3) * (z - 3) + 9 * z)
    if L == 3:
        return 277 * z * z * z / (z * (z - 15) * (z - 15) + 9 * (2 * z - 5) * (2 * z - 5))
    if L == 4:
        z2 = z * z
        a = z2 - 45 * z + 105
        b = 2 * z - 21
        return 12746 * z2 * z2 / (a * a + 25 * z * b * b)
    raise ValueError("spin must be 0..4")


def _rho_flatte(m2, ma, mb):
    """2 q / m, analytically continued below threshold (complex array)."""
    q2 = breakup_q2(m2, ma, mb)
    q = np.where(q2 >= 0, np.sqrt(np.abs(q2)) + 0j, 1j * np.sqrt(np.abs(q2)))
    return 2 * q / np.sqrt(m2)


def breit_wigner(model: VariantModel, k: int, m2, M: HD, w1: HD, w2: HD) -> HD:
    """BW_k = 1 / D_k over events with pair mass^2 m2 (float64 array)."""
    sh = model.shapes[k]
    m2 = np.asarray(m2, dtype=np.float64)
    if sh.kind == KIND_CONSTANT:
        D = M * M - m2 - 1j * (M * w1)
    elif sh.kind == KIND_MASS_DEPENDENT:
        L = int(model.spins[k])
        r2 = sh.radius ** 2
        q2 = breakup_q2(m2, sh.ma, sh.mb)
        q = np.sqrt(np.maximum(q2, 0.0))
        rho = q * barrier_sq(L, q2 * r2) / np.sqrt(m2)
        q02 = _hd_pair(M, sh.ma, sh.mb)
        h = M * M / (q02.sqrt() * _barrier_sq_hd(L, q02 * r2))
        D = M * M - m2 - 1j * (w1 * h * rho)
    elif sh.kind == KIND_FLATTE:
        D = M * M - m2 - 1j * (w1 * _rho_flatte(m2, sh.ma, sh.mb) + w2 * _rho_flatte(m2, sh.mc, sh.md))
    else:
        raise ValueError("unknown line shape")
    return D.inv()


def _params(model: VariantModel, theta, v=None, u=None):
    """Hyper-dual parameters: value theta, e1 part v, e2 part u (both optional)."""
    th = np.asarray(theta, dtype=np.float64)
    P = model.P
    vv = np.zeros(P) if v is None else np.asarray(v, dtype=np.float64)
    uu = np.zeros(P) if u is None else np.asarray(u, dtype=np.float64)
    K = model.K
    ns = model.S if model.per_projection else 1
    mag = [[HD(model.mag[k]) for _ in range(ns)] for k in range(K)]
    phase = [[HD(model.phase[k]) for _ in range(ns)] for k in range(K)]
    mass = [HD(model.mass[k]) for k in range(K)]
    w1 = [HD(model.width[k]) for k in range(K)]
    w2 = [HD(model.shapes[k].width2) for k in range(K)]
    for i, (name, k, s) in enumerate(model.layout()):
        x = HD(th[i], vv[i], uu[i], 0.0)
        if name == "mag":
            mag[k][s] = x
        elif name == "phase":
            phase[k][s] = x
        elif name == "mass":
            mass[k] = x
        elif name == "w1":
            w1[k] = x
        else:
            w2[k] = x
    return mag, phase, mass, w1, w2


def intensity_hd(model: VariantModel, pars, m2, F) -> HD:
    """I(e) over a sample (m2 [3][n], F [n][K][S] complex) as a hyper-dual array."""
    mag, phase, mass, w1, w2 = pars
    K, S = model.K, model.S
    A = [HD(np.zeros(F.shape[0], dtype=np.complex128)) for _ in range(S)]
    for k in range(K):
        bw = breit_wigner(model, k, np.asarray(m2[model.channels[k]], dtype=np.float64), mass[k], w1[k], w2[k])
        for s in range(S):
            j = s if model.per_projection else 0
            g = mag[k][j] * phase[k][j].exp_i()
            A[s] = A[s] + (g * bw) * np.asarray(F[:, k, s], dtype=np.complex128)
    I = HD(0.0)
    for s in range(S):
        I = I + (A[s] * A[s].conj()).real()
    return I


def nll_hd(model: VariantModel, theta, data, mc, v=None, u=None) -> HD:
    pars = _params(model, theta, v, u)
    w = np.ones(data.m2.shape[1]) if getattr(data, "w", None) is None else np.asarray(data.w, dtype=np.float64)
    Id = intensity_hd(model, pars, data.m2, data.F)
    Im = intensity_hd(model, pars, mc.m2, mc.F)
    Nd = float(np.sum(w))
    Nmc = mc.m2.shape[1]
    return -(Id.log() * w).sum() + Nd * (Im.sum() / Nmc).log()


def nll(model: VariantModel, theta, data, mc) -> float:
    return float(np.real(nll_hd(model, theta, data, mc).a))


def nll_grad_hvp(model: VariantModel, theta, v, data, mc):
    """(NLL, gradient, H v): P hyper-dual evaluations with u = e_j."""
    P = model.P
    g = np.empty(P)
    hv = np.empty(P)
    f = None
    for j in range(P):
        u = np.zeros(P)
        u[j] = 1.0
        r = nll_hd(model, theta, data, mc, v=v, u=u)
        f = float(np.real(r.a))
        g[j] = float(np.real(r.c))
        hv[j] = float(np.real(r.d))
    return f, g, hv


def intensity(model: VariantModel, theta, m2, F) -> np.ndarray:
    return np.real(intensity_hd(model, _params(model, theta), m2, F).a)


def integral_matrices(model: VariantModel, theta, m2, F) -> np.ndarray:
    """Phi [S][K][K] complex: Phi_s,kk' = sum over the sample of
    conj(U_ks) U_k's with U_ks = BW_k F_ks at the line-shape parameters of
    theta (Eq. 1 written as sum_s g_s^H Phi_s g_s over the events)."""
    pars = _params(model, theta)
    _, _, mass, w1, w2 = pars
    K, S = model.K, model.S
    U = np.empty((F.shape[0], K, S), dtype=np.complex128)
    for k in range(K):
        bw = breit_wigner(model, k, np.asarray(m2[model.channels[k]], dtype=np.float64), mass[k], w1[k], w2[k]).a
        U[:, k, :] = bw[:, None] * np.asarray(F[:, k, :], dtype=np.complex128)
    return np.einsum("eks,ejs->skj", np.conj(U), U)


def coupling_count(model: VariantModel) -> int:
    """Number of coupling parameters (magnitudes and phases) at the head of theta."""
    return sum(1 for name, _, _ in model.layout() if name in ("mag", "phase"))
