"""Learned starting points for Newton-CG (no counterpart in the paper).

A proposal network maps the binned Dalitz plot of a data set to a starting
theta.  It is trained on pseudo-experiments that the method generates itself:
theta drawn from the prior, events accept-rejected from I(e; theta) (the
paper's Sec. 3 makes its test samples from the model the same way), the
sample fitted by Newton-CG from theta (the label).  Every step with
arithmetic runs in libpwa: the intensities of the pool (pwa_event_intensity),
the accept-reject selection, histogram and gather (generate.cu), the fits
(pwa_newton_cg_fit_multi) and the network's forward, backward and Adam
kernels (mlp.cu).  This module only moves arrays and keeps the bookkeeping.

Label switching: resonances that share a (channel, spin) and have free
couplings, masses and widths enter I through the same F columns, so permuting
their (rho, phi, M, Gamma) leaves I unchanged; a label is made canonical by
sorting those groups by mass.  (rho, phi) and (-rho, phi + pi) give the same
coupling: rho >= 0 and phi in (-pi, pi] are taken.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Optional, Sequence

import numpy as np

from . import binding
from . import workload as W

HIST_BINS = 64


def _torch():
    import torch
    return torch


def _device_sample(sample):
    torch = _torch()
    dev = torch.device("cuda")
    m2 = torch.from_numpy(np.ascontiguousarray(sample.m2, dtype=np.float32)).to(dev)
    F = torch.from_numpy(np.ascontiguousarray(sample.F).view(np.float32).reshape(sample.F.shape + (2,))).to(dev)
    return m2, F


@dataclasses.dataclass
class Layout:
    """Where each resonance's parameters sit in theta (-1: fixed)."""
    rho: np.ndarray
    phi: np.ndarray
    mass: np.ndarray
    width: np.ndarray
    P: int

    @classmethod
    def of(cls, table) -> "Layout":
        K = len(table)
        rho, phi, mass, width = (np.full(K, -1) for _ in range(4))
        kc = [k for k, r in enumerate(table) if not r.fix_coupling]
        km = [k for k, r in enumerate(table) if not r.fix_mass]
        kw = [k for k, r in enumerate(table) if not r.fix_width]
        for i, k in enumerate(kc):
            rho[k] = i
            phi[k] = len(kc) + i
        for i, k in enumerate(km):
            mass[k] = 2 * len(kc) + i
        for i, k in enumerate(kw):
            width[k] = 2 * len(kc) + len(km) + i
        return cls(rho, phi, mass, width, 2 * len(kc) + len(km) + len(kw))

    def periodic(self) -> np.ndarray:
        out = np.zeros(self.P, dtype=bool)
        out[self.phi[self.phi >= 0]] = True
        return out


def exchangeable_groups(table) -> list:
    """Lists of resonances (two or more) with the same (channel, spin) whose
    coupling, mass and width are all free."""
    groups: dict = {}
    for k, r in enumerate(table):
        if not (r.fix_coupling or r.fix_mass or r.fix_width):
            groups.setdefault((r.channel, r.spin), []).append(k)
    return [g for g in groups.values() if len(g) > 1]


def canonical(table, theta) -> np.ndarray:
    """theta with rho >= 0, phi in (-pi, pi] and every exchangeable group
    ordered by increasing mass."""
    lay = Layout.of(table)
    th = np.array(theta, dtype=np.float64)
    single = th.ndim == 1
    th = np.atleast_2d(th).copy()
    for k in range(len(table)):
        if lay.rho[k] >= 0:
            neg = th[:, lay.rho[k]] < 0
            th[neg, lay.rho[k]] *= -1
            th[neg, lay.phi[k]] += math.pi
            th[:, lay.phi[k]] = math.pi - np.mod(math.pi - th[:, lay.phi[k]], 2 * math.pi)
    for g in exchangeable_groups(table):
        g = np.asarray(g)
        cols = np.stack([lay.rho[g], lay.phi[g], lay.mass[g], lay.width[g]])  # [4, |g|]
        order = np.argsort(th[:, lay.mass[g]], axis=1, kind="stable")           # [B, |g|]
        for row in range(th.shape[0]):
            vals = th[row][cols]                                               # [4, |g|]
            th[row, cols] = vals[:, order[row]]
    return th[0] if single else th


class Codec:
    """Network targets from theta: (x - mean) / std per parameter for
    magnitudes, masses and widths, the raw phase for phases (their loss is
    1 - cos of the difference).  decode() maps outputs back into the prior's
    box (masses into the channel's range, widths and magnitudes positive)."""

    def __init__(self, table, labels: np.ndarray):
        self.table = table
        self.lay = Layout.of(table)
        self.periodic = self.lay.periodic()
        self.mean = np.where(self.periodic, 0.0, labels.mean(axis=0))
        self.std = np.where(self.periodic, 1.0, np.maximum(labels.std(axis=0), 1e-6))
        self.lo = np.full(self.lay.P, -np.inf)
        self.hi = np.full(self.lay.P, np.inf)
        for k, r in enumerate(table):
            if self.lay.mass[k] >= 0:
                lo, hi = W.channel_mass_range(r.channel)
                self.lo[self.lay.mass[k]], self.hi[self.lay.mass[k]] = lo + 1e-3, hi - 1e-3
            if self.lay.width[k] >= 0:
                self.lo[self.lay.width[k]], self.hi[self.lay.width[k]] = 0.005, 1.0
            if self.lay.rho[k] >= 0:
                self.lo[self.lay.rho[k]] = 0.01

    def encode(self, theta: np.ndarray) -> np.ndarray:
        return ((np.asarray(theta) - self.mean) / self.std).astype(np.float32)

    def decode(self, out: np.ndarray) -> np.ndarray:
        th = np.asarray(out, dtype=np.float64) * self.std + self.mean
        th = np.clip(th, self.lo, self.hi)
        ph = self.periodic
        th[..., ph] = math.pi - np.mod(math.pi - th[..., ph], 2 * math.pi)
        return th


class Generator:
    """Pseudo-experiments of one resonance table: a pool of phase-space events
    resident on the device (raw arrays for the gather, and a likelihood handle
    whose MC sample is the pool, for I(e; theta)), plus the shared MC sample of
    every pseudo-experiment's likelihood."""

    def __init__(self, table, S: int, pool_size: int, n_mc: int, seed: int = W.BASE_SEED, nb: int = HIST_BINS):
        torch = _torch()
        self.table, self.S, self.K, self.nb = table, S, len(table), nb
        self.seed = int(seed)
        pool = W.phase_space_sample(W.rng_stream(seed, W.STREAM_POOL), pool_size, table, S)
        mc = W.phase_space_sample(W.rng_stream(seed, W.STREAM_MC), n_mc, table, S)
        self.pool_m2, self.pool_F = _device_sample(pool)
        self.mc_m2, self.mc_F = _device_sample(mc)
        del pool, mc
        small = _Sample(self.pool_m2[:, :1024].contiguous(), self.pool_F[:1024].contiguous())
        self.pool_L = binding.Likelihood(small, _Sample(self.pool_m2, self.pool_F), table, self.K, S)
        self.P = self.pool_L.P
        self.I = torch.empty(pool_size, dtype=torch.float32, device="cuda")
        self.bounds = W.dalitz_bounds()
        self.pool_size = pool_size

    def draw(self, theta, n_events: int, seed: int):
        """Pool indices (CUDA int32) of a pseudo-experiment of up to n_events
        events from I(e; theta)."""
        self.pool_L.intensity(theta, sample=1, out=self.I)
        start = int(np.random.default_rng(seed).integers(self.pool_size))
        idx, _ = binding.accept_reject(self.I, seed=seed, start=start, n_target=n_events)
        return idx

    def features(self, idx, out=None):
        return binding.dalitz_histogram(self.pool_m2, idx, self.nb, self.bounds, log_scale=True, out=out)

    def likelihood(self, idx) -> binding.Likelihood:
        m2, F = binding.gather_events(self.pool_m2, self.pool_F, idx)
        return binding.Likelihood(_Sample(m2, F), _Sample(self.mc_m2, self.mc_F), self.table, self.K, self.S)

    def close(self):
        self.pool_L.close()


@dataclasses.dataclass
class _Sample:
    m2: object
    F: object
    w: object = None


@dataclasses.dataclass
class Experiments:
    """Pseudo-experiments: features [N, nb^2] (CUDA float32), generating and
    fitted theta, kept event counts and the labelling fits' statistics."""
    X: object
    theta_true: np.ndarray
    theta_fit: np.ndarray
    n_events: np.ndarray
    seeds: np.ndarray
    fit_s: float
    gen_s: float


def make_experiments(gen: Generator, count: int, n_events: int, seed: int, group: int = 16,
                     label_fit: bool = True, fit_opts: Optional[dict] = None, keep_idx: bool = False):
    """count pseudo-experiments with theta from the prior; labels from
    Newton-CG fits started at the generating theta, `group` likelihoods at a
    time in lockstep (pwa_newton_cg_fit_multi)."""
    torch = _torch()
    rng = W.rng_stream(seed, W.STREAM_STARTS)
    # a label needs the minimum near theta only to well within the network's
    # own error: capped Newton and CG iterations
    opts = dict(xtol=1e-5, maxiter=30, cg_maxiter=gen.P)
    opts.update(fit_opts or {})
    X = torch.empty((count, gen.nb * gen.nb), dtype=torch.float32, device="cuda")
    th_true = np.stack([W.sample_start(rng, gen.table) for _ in range(count)])
    th_fit = th_true.copy()
    n_ev = np.zeros(count, dtype=np.int64)
    seeds = np.array([(seed * 1_000_003 + i) & ((1 << 62) - 1) for i in range(count)], dtype=np.int64)
    idxs = [] if keep_idx else None
    fit_s = gen_s = 0.0
    for g0 in range(0, count, group):
        rows = range(g0, min(count, g0 + group))
        Ls = []
        t0 = time.perf_counter()
        for i in rows:
            idx = gen.draw(th_true[i], n_events, int(seeds[i]))
            gen.features(idx, out=X[i])
            n_ev[i] = idx.numel()
            if keep_idx:
                idxs.append(idx.clone())
            if label_fit:
                Ls.append(gen.likelihood(idx))
        torch.cuda.synchronize()
        gen_s += time.perf_counter() - t0
        if label_fit:
            t0 = time.perf_counter()
            outs, _, _ = binding.fit_multi(Ls, [th_true[i][None] for i in rows], **opts)
            fit_s += time.perf_counter() - t0
            for j, i in enumerate(rows):
                th_fit[i] = outs[j][0]
            for L in Ls:
                L.close()
    ex = Experiments(X, th_true, canonical(gen.table, th_fit), n_ev, seeds, fit_s, gen_s)
    return (ex, idxs) if keep_idx else ex


def train(ex: Experiments, table, hidden: int = 512, layers: int = 3, batch: int = 128, epochs: int = 20,
          lr: float = 1e-3, lr_final: float = 1e-5, seed: int = 1, log=None):
    """Train a ProposalMLP on the experiments (rows in the stored order,
    mini-batches of `batch` consecutive rows visited in a seeded random order
    each epoch; the learning rate falls from lr to lr_final on a cosine).
    Returns (net, codec, mean loss per epoch)."""
    torch = _torch()
    codec = Codec(table, ex.theta_fit)
    N = (ex.X.shape[0] // batch) * batch
    T = torch.from_numpy(codec.encode(ex.theta_fit[:N])).cuda()
    weight = np.ones(codec.lay.P, dtype=np.float32)
    net = binding.ProposalMLP(ex.X.shape[1], hidden, layers, codec.lay.P, batch, seed=seed,
                              periodic=codec.periodic, loss_weight=weight)
    rng = np.random.default_rng(seed)
    nbatch = N // batch
    steps = max(1, epochs * nbatch)
    hist = []
    step = 0
    for ep in range(epochs):
        tot = 0.0
        for b in rng.permutation(nbatch):
            a = int(b) * batch
            rate = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * step / steps))
            tot += net.train_step(ex.X[a:a + batch], T[a:a + batch], rate)
            step += 1
        hist.append(tot / nbatch)
        if log:
            log("epoch %d loss %.4f" % (ep, hist[-1]))
    return net, codec, hist


def propose(net, codec: Codec, X) -> np.ndarray:
    """Starting points for the rows of X (CUDA float32 [N, nb^2]); N is padded
    to the network's batch with zero rows."""
    torch = _torch()
    N = X.shape[0]
    B = net.max_batch
    out = []
    for a in range(0, N, B):
        xb = X[a:a + B]
        if xb.shape[0] < B:
            pad = torch.zeros((B, X.shape[1]), dtype=torch.float32, device=X.device)
            pad[:xb.shape[0]].copy_(xb)
            xb = pad
        out.append(net.forward(xb).cpu().numpy()[:min(B, N - a)])
    return codec.decode(np.concatenate(out))


def perturbed_starts(codec: Codec, start: np.ndarray, count: int, rng, scale: float = 0.3) -> np.ndarray:
    """The start itself and count - 1 draws around it: Gaussian steps of
    `scale` in the network's standardised target space (radians for phases)."""
    t = codec.encode(start[None])[0].astype(np.float64)
    rows = [t] + [t + scale * rng.standard_normal(t.size) for _ in range(count - 1)]
    return codec.decode(np.stack(rows))


def polish_couplings(L, starts: np.ndarray, opts: Optional[dict] = None) -> np.ndarray:
    """Each start with its couplings replaced by the coupling-only Newton-CG
    fit at its own masses and widths (the tensor-core coupling object of
    binding.Coupling: the data events as U = BW F tiles, the MC events as the
    integral matrix)."""
    out = np.array(starts, dtype=np.float64, copy=True)
    o = dict(xtol=1e-6, maxiter=50)
    o.update(opts or {})
    for i in range(out.shape[0]):
        try:
            cp = binding.Coupling(L, out[i])
        except binding.PwaError:
            continue  # a start the coupling object refuses keeps its couplings
        try:
            c, _, _ = cp.fit(out[i, :cp.Pc][None], **o)
            if np.all(np.isfinite(c[0])):
                out[i, :cp.Pc] = c[0]
        except binding.PwaError:
            pass
        finally:
            cp.close()
    return out


def evaluate(gen: Generator, net, codec: Codec, count: int, n_events: int, n_random: int, seed: int,
             fit_opts: Optional[dict] = None, tol: float = 0.01, n_learned: int = 4, polish: bool = False):
    """Held-out pseudo-experiments, three ways with the same fit options:
    one fit from the network's start; one batched call from the network's
    start and n_learned - 1 draws around it; one batched call from n_random
    prior starts.  With polish, also the first two with their starts'
    couplings fitted first at the starts' masses and widths
    (polish_couplings; its time counts).  The global minimum of an experiment is the lowest NLL any
    of its fits reached; a fit reaches it when its NLL is within `tol`.
    Returns per-experiment records and the summary of summarize()."""
    opts = dict(xtol=1e-8, maxiter=0)
    opts.update(fit_opts or {})
    ex, idxs = make_experiments(gen, count, n_events, seed, label_fit=False, keep_idx=True)
    starts = propose(net, codec, ex.X)
    rng = W.rng_stream(seed + 1, W.STREAM_STARTS)
    prng = np.random.default_rng(seed + 2)
    recs = []
    for i in range(count):
        L = gen.likelihood(idxs[i])
        rnd = np.stack([W.sample_start(rng, gen.table) for _ in range(n_random)])
        t0 = time.perf_counter()
        _, info_m = L.fit(starts[i], **opts)
        t_m = time.perf_counter() - t0
        lb = perturbed_starts(codec, starts[i], n_learned, prng)
        t0 = time.perf_counter()
        _, info_b, _ = L.fit_batch(lb, **opts)
        t_b = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, info_r, _ = L.fit_batch(rnd, **opts)
        t_r = time.perf_counter() - t0
        extra = {}
        if polish:
            # the same starts with their couplings fitted at their masses and widths first
            t0 = time.perf_counter()
            ps = polish_couplings(L, starts[i][None])[0]
            _, info_p = L.fit(ps, **opts)
            t_p = time.perf_counter() - t0
            t0 = time.perf_counter()
            pb = polish_couplings(L, lb)
            _, info_pb, _ = L.fit_batch(pb, **opts)
            t_pb = time.perf_counter() - t0
            extra = dict(nll_polish=info_p["nll"], t_polish=t_p,
                         nll_polish_batch=[d["nll"] for d in info_pb], t_polish_batch=t_pb)
        f_true = L.nll(ex.theta_true[i])
        L.close()
        nll_r = np.array([d["nll"] for d in info_r])
        nll_b = np.array([d["nll"] for d in info_b])
        cands = [info_m["nll"], float(np.min(nll_b)), float(np.min(nll_r))]
        if polish:
            cands += [extra["nll_polish"], float(np.min(extra["nll_polish_batch"]))]
        best = min(cands)
        rec = dict(n_events=int(ex.n_events[i]), nll_mlp=info_m["nll"], nll_learned_batch=nll_b.tolist(),
                   nll_random=nll_r.tolist(), nll_true=f_true, best=best, t_mlp=t_m, t_learned_batch=t_b,
                   t_random=t_r, mlp_hit=bool(info_m["nll"] <= best + tol),
                   learned_batch_hit=bool(np.min(nll_b) <= best + tol),
                   random_hits=int(np.sum(nll_r <= best + tol)))
        if polish:
            rec.update(extra, polish_hit=bool(extra["nll_polish"] <= best + tol),
                       polish_batch_hit=bool(min(extra["nll_polish_batch"]) <= best + tol))
        recs.append(rec)
    return recs, summarize(recs, n_random, n_learned)


def summarize(recs: Sequence[dict], n_random: int, n_learned: int = 1) -> dict:
    """Expected GPU-seconds until an experiment's global minimum is found.
    Random multi-start runs batches of n_random prior starts until one hits:
    with p the pooled hit rate of a start and T the mean time of a batched
    call, E = T / (1 - (1 - p)^n_random).  Learned: the time of the fit from
    the network's start (or of the batched call from it and the draws around
    it), plus E when that misses (random multi-start remains the fallback)."""
    t_rand = float(np.mean([r["t_random"] for r in recs]))
    hits = sum(r["random_hits"] for r in recs)
    p = hits / max(1, n_random * len(recs))
    q = 1.0 - (1.0 - p) ** n_random
    e_rand = t_rand / q if q > 0 else float("inf")
    learned = [r["t_mlp"] + (0.0 if r["mlp_hit"] else e_rand) for r in recs]
    out = dict(experiments=len(recs), random_starts=n_random,
               mlp_hit_rate=float(np.mean([r["mlp_hit"] for r in recs])), random_hit_rate=p,
               random_s_to_min=e_rand, learned_s_to_min=float(np.mean(learned)),
               mean_t_mlp_fit=float(np.mean([r["t_mlp"] for r in recs])), mean_t_random_batch=t_rand,
               mean_dnll_mlp=float(np.mean([r["nll_mlp"] - r["best"] for r in recs])),
               mean_dnll_random=float(np.mean([np.mean(np.asarray(r["nll_random"]) - r["best"]) for r in recs])))
    if recs and "t_learned_batch" in recs[0]:
        lb = [r["t_learned_batch"] + (0.0 if r["learned_batch_hit"] else e_rand) for r in recs]
        out.update(learned_starts=n_learned,
                   learned_batch_hit_rate=float(np.mean([r["learned_batch_hit"] for r in recs])),
                   learned_batch_s_to_min=float(np.mean(lb)),
                   mean_t_learned_batch=float(np.mean([r["t_learned_batch"] for r in recs])))
    if recs and "t_polish" in recs[0]:
        lp = [r["t_polish"] + (0.0 if r["polish_hit"] else e_rand) for r in recs]
        lpb = [r["t_polish_batch"] + (0.0 if r["polish_batch_hit"] else e_rand) for r in recs]
        out.update(polish_hit_rate=float(np.mean([r["polish_hit"] for r in recs])),
                   polish_s_to_min=float(np.mean(lp)),
                   polish_batch_hit_rate=float(np.mean([r["polish_batch_hit"] for r in recs])),
                   polish_batch_s_to_min=float(np.mean(lpb)),
                   mean_t_polish=float(np.mean([r["t_polish"] for r in recs])),
                   mean_t_polish_batch=float(np.mean([r["t_polish_batch"] for r in recs])))
    return out
