#!/usr/bin/env python
"""Throughput benchmark of the fused NLL + gradient + HVP pass.

Workload: the paper-scale configuration -- a three-body decay (parent
3.097 GeV; daughters 0.1396, 0.1396, 1.0195 GeV) with K = 20 Breit-Wigner
resonances over the three channels (spins 0..4), S = 4 complex FP32 amplitude
projections per resonance, 1e6 data events drawn from I(theta_true) by
accept-reject and 5e6 phase-space MC events; 78 real parameters.  All inputs
are synthetic and seeded (the paper's psi(3686) -> phi K+ K- sample is not
available).

One step = one fused pass over all events (parameter unpack, Breit-Wigner,
coherent sums, adjoint gradient sweep, forward-over-reverse HVP, FP64
reductions and the Eq. 4-7 combination), i.e. one Newton-CG inner iteration.
Metric: event-amplitude evaluations per second, (N_data + N_MC) * K / time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the path is not sharded: replicas only); value = all ranks' units / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NLL+grad+HVP event-amplitude evaluations/s (fused pass)"
#: identifies the kernel version the committed DRAM-traffic summary was taken on
KERNEL_REVISION = "paired-projection tiles, paired butterfly, twosum folds, shared block body"
UNIT = "event*amp/s"
CONFIG_NAME = "paper"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def bf16_peak():
    """Dense BF16 tensor peak: the measured burst figure, or the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1800.0, "fallback"


def units_per_pass(nd, nm, K):
    return (nd + nm) * K


def bytes_per_pass(nd, nm, K, S):
    """Algorithmic HBM bytes of one pass: F (8 S bytes per event-amplitude),
    three m^2 values per event, one weight per data event."""
    return nd * (8 * K * S + 12 + 4) + nm * (8 * K * S + 12)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        time.sleep(0.2)
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_intensity_fn(table, K, S):
    """I(e) at the table's parameter values computed by the library (used to
    accept-reject the data sample)."""
    from types import SimpleNamespace
    from paper_2403_09225_b300 import binding
    from paper_2403_09225_b300 import workload as W
    theta = W.free_parameter_vector(table)
    one = SimpleNamespace(m2=np.full((3, 1), 1.0, np.float32), F=np.ones((1, K, S), np.complex64), w=None)

    def fn(m2, F):
        L = binding.Likelihood(one, SimpleNamespace(m2=m2, F=F, w=None), table, K, S)
        try:
            return L.intensity(theta, sample=1).astype(np.float64)
        finally:
            L.close()
    return fn


def build_workload(scale: float = 1.0):
    from paper_2403_09225_b300 import workload as W
    cfg = W.CONFIGS[CONFIG_NAME]
    table = W.make_table(cfg)
    return W.make_workload(cfg, intensity=gpu_intensity_fn(table, cfg.K, cfg.S),
                           n_data=int(round(cfg.n_data * scale)), n_mc=int(round(cfg.n_mc * scale)))


def run_reference(args, rank, world):
    """The CPU oracle (FP64, one thread) on a bounded sample of the workload."""
    if rank != 0:
        return None
    import oracle
    from paper_2403_09225_b300 import workload as W
    cfg = W.CONFIGS[CONFIG_NAME]
    table = W.make_table(cfg)
    model = oracle.Model.from_table(table, cfg.S)
    frac = 1.0 / 60.0
    nd, nm = int(cfg.n_data * frac), int(cfg.n_mc * frac)
    wl = W.make_workload(cfg, intensity=None, n_data=nd, n_mc=nm)
    th = W.random_starts(wl, 1)[0]
    v = np.linspace(-1.0, 1.0, model.P)
    warm = max(0, min(args.warmup, 5))  # each oracle step is a bounded sample (about a second)
    for _ in range(warm):
        oracle.nll_grad_hvp(model, th, v, wl.data, wl.mc)
    steps = max(1, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.nll_grad_hvp(model, th, v, wl.data, wl.mc)
    dt = time.perf_counter() - t0
    value = steps * (nd + nm) * cfg.K / dt
    sample = ("%d data + %d MC phase-space events (1/60 of the workload), K=%d, S=%d, %d steps"
              % (nd, nm, cfg.K, cfg.S, steps))
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": dt / steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "paper-scale K=20 S=4 (bounded CPU sample)",
                                        "n_data": nd, "n_mc": nm, "K": cfg.K, "S": cfg.S},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def cpu_baseline_leg():
    """The oracle as it stands, single-threaded, on a bounded sample."""
    import oracle
    from paper_2403_09225_b300 import workload as W
    cfg = W.CONFIGS[CONFIG_NAME]
    table = W.make_table(cfg)
    model = oracle.Model.from_table(table, cfg.S)
    nd, nm = cfg.n_data // 60, cfg.n_mc // 60
    wl = W.make_workload(cfg, intensity=None, n_data=nd, n_mc=nm)
    th = W.random_starts(wl, 1)[0]
    v = np.linspace(-1.0, 1.0, model.P)
    reps, dt = 0, 0.0
    t0 = time.perf_counter()
    while reps < 2 or dt < 12.0:  # about 12 s of single-core work
        oracle.nll_grad_hvp(model, th, v, wl.data, wl.mc)
        reps += 1
        dt = time.perf_counter() - t0
    out = {"value": reps * (nd + nm) * cfg.K / dt, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
           "kind": "oracle", "pass_s_sample": dt / reps,
           "sample": "%d data + %d MC events (1/60 of the workload), K=%d, S=%d, %d fused evaluations, "
                     "%.1f s" % (nd, nm, cfg.K, cfg.S, reps, dt)}
    out["other_configs"] = _oracle_other_configs()
    return out


def _oracle_eval_rate(name: str, frac: float):
    """One oracle NLL + gradient + H v evaluation on (a fraction of) a configuration."""
    import oracle
    from paper_2403_09225_b300 import workload as W
    cfg = W.CONFIGS[name]
    model = oracle.Model.from_table(W.make_table(cfg), cfg.S)
    nd, nm = max(1, int(cfg.n_data * frac)), max(1, int(cfg.n_mc * frac))
    wl = W.make_workload(cfg, intensity=None, n_data=nd, n_mc=nm)
    th = W.random_starts(wl, 1)[0]
    v = np.linspace(-1.0, 1.0, model.P)
    t0 = time.perf_counter()
    oracle.nll_grad_hvp(model, th, v, wl.data, wl.mc)
    dt = time.perf_counter() - t0
    return {"events": nd + nm, "fraction_of_config": frac, "K": cfg.K, "S": cfg.S, "eval_s": dt,
            "event_amps_per_s": (nd + nm) * cfg.K / dt}


def _oracle_other_configs():
    """The oracle on the other configurations (single core): one fused
    evaluation on the full tiny configuration and on 1/600 of the
    differentiation one, and a full Newton-CG fit (its own FP64 iteration,
    matrix-free) on 1/4 of tiny, data accept-rejected from the model."""
    import oracle
    from oracle import newton_cg as ncg
    from paper_2403_09225_b300 import workload as W
    out = {"tiny": _oracle_eval_rate("tiny", 1.0), "diff": _oracle_eval_rate("diff", 1.0 / 600)}
    cfg = W.CONFIGS["tiny"]
    table = W.make_table(cfg)
    model = oracle.Model.from_table(table, cfg.S)
    fn = lambda m2, F: oracle.intensity_full(cfg.K, cfg.S, model.channels, model.par0, m2, F)
    nd, nm = cfg.n_data // 4, cfg.n_mc // 4
    wl = W.make_workload(cfg, intensity=fn, n_data=nd, n_mc=nm)
    x0 = W.random_starts(wl, 1)[0]
    fg = lambda x: oracle.nll_grad(model, x, wl.data, wl.mc)
    hp = lambda x, v: oracle.nll_grad_hvp(model, x, v, wl.data, wl.mc)[2]
    r = ncg.newton_cg(fg, hp, x0, xtol=1e-8, time_limit=30.0)
    out["tiny_fit"] = {"events": nd + nm, "fraction_of_config": 0.25, "seconds": r.elapsed, "iters": r.iters,
                       "n_fev": r.n_fev, "n_hvp": r.n_hvp, "status": r.status_name, "time_limit_s": 30.0}
    return out


def _fit_runs(L, wl, starts, time_limit: float, batched: bool = False, method: int = 0,
              matrix_free: bool = False, best_extra=()):
    """Fits from `starts`: one after another (plain multi-start), or all in
    lockstep with batched passes (pwa_newton_cg_fit_batch).  GPU seconds are
    the wall time of the fits (the device is busy or waiting on the host
    between passes; nothing else runs)."""
    kw = dict(xtol=1e-8, time_limit_s=time_limit, method=method, matrix_free=matrix_free)
    t0 = time.perf_counter()
    if batched:
        _, results, _ = L.fit_batch(np.array(starts), **kw)
    else:
        results = [L.fit(s, **kw)[1] for s in starts]
    total = time.perf_counter() - t0
    return {"starts": len(starts), "gpu_seconds": total, "nll": [r["nll"] for r in results],
            "grad_max": [r["grad_max"] for r in results], "status_per_fit": [r["status"] for r in results],
            "iters": [r["iters"] for r in results], "statuses": sorted({r["status"] for r in results}),
            "passes": int(sum(r["n_fev"] + r["n_hvp"] + r["n_hess"] for r in results)),
            "hessian_passes": int(sum(r["n_hess"] for r in results)), "time_limit_s": time_limit,
            "method": "trust-region" if method == 1 else "line-search",
            "hessian": "matrix-free H v passes" if matrix_free else "one Hessian pass per outer iteration"}


def _score(arms: dict, best: float, tol: float = 0.01):
    """Hits (NLL within tol of the best seen) and hits per GPU-second per arm."""
    for a in arms.values():
        ok = sum(1 for f in a["nll"] if f <= best + tol)
        a["reached_global_min"] = ok
        a["fits_to_global_min_per_s"] = ok / a["gpu_seconds"] if a["gpu_seconds"] > 0 else 0.0
        a["dnll_median"] = float(np.median(np.asarray(a["nll"]) - best))


def fit_metric(L, wl, n_starts: int, time_limit: float):
    """Newton-CG fits (xtol 1e-8) from random starts of the prior, every
    outer iteration driven by one Hessian pass.  A fit reaches the global
    minimum when its NLL is within 0.01 of the best NLL seen over all fits of
    that workload (including fits from theta_true).  Paper scale: the paper's
    line-search Newton-CG one start after another, and half of the starts with
    the trust-region Newton-CG.  The tiny configuration (K = 3, 2e4 + 1e5
    events) shows the rate on a model whose random starts often find the
    minimum, also in lockstep (one batched f, g launch per round)."""
    from paper_2403_09225_b300 import binding
    from paper_2403_09225_b300 import workload as W
    starts = W.random_starts(wl, n_starts)
    ref_infos = [L.fit(wl.theta_true, xtol=1e-8, time_limit_s=time_limit, method=m)[1] for m in (0, 1)]
    refs = [r["nll"] for r in ref_infos]
    paper = {"line_search": _fit_runs(L, wl, starts, time_limit),
             "trust_region": _fit_runs(L, wl, starts[:max(1, n_starts // 2)], time_limit, method=1)}
    best = min(refs + [f for a in paper.values() for f in a["nll"]])
    _score(paper, best)
    paper["best_nll"] = best
    paper["nll_from_theta_true"] = refs
    paper["from_theta_true"] = [{"method": m, "nll": r["nll"], "grad_max": r["grad_max"], "iters": r["iters"],
                                 "status": r["status"]} for m, r in zip(("line-search", "trust-region"), ref_infos)]
    out = {"xtol": 1e-8, "paper": paper}
    cfg = W.CONFIGS["tiny"]
    table = W.make_table(cfg)
    tiny_wl = W.make_workload(cfg, intensity=gpu_intensity_fn(table, cfg.K, cfg.S))
    Lt = binding.make_likelihood(tiny_wl)
    try:
        ts = W.random_starts(tiny_wl, 32)
        tref = Lt.fit(tiny_wl.theta_true, xtol=1e-8, time_limit_s=time_limit)[1]["nll"]
        tiny = {"line_search": _fit_runs(Lt, tiny_wl, ts, time_limit),
                "line_search_lockstep": _fit_runs(Lt, tiny_wl, ts, time_limit * 32, batched=True),
                "trust_region": _fit_runs(Lt, tiny_wl, ts, time_limit, method=1)}
        tbest = min([tref] + [f for a in tiny.values() for f in a["nll"]])
        _score(tiny, tbest)
        tiny["best_nll"] = tbest
        out["tiny"] = tiny
    finally:
        Lt.close()
    return out


def batching_metric(n_toys: int, n_starts: int, time_limit: float, seed: int = 7):
    """Toy fits of uneven size and model, plain against batched.  Each toy
    draws data events log-uniform in [1e4, 1e5] (MC = 5 x data), K uniform in
    5..30 and S uniform in 2..4 (the batching configuration's distributions,
    with data sizes capped at 1e5 to keep a run to minutes), accept-rejects its
    data from I at its own generating point, and is fitted from n_starts
    random starts.  Plain: every fit of every toy one after another.  Batched:
    all fits of all toys in lockstep (pwa_newton_cg_fit_multi: every round is
    one batched pass per toy, each on its own stream, and one batched Hessian
    pass per toy), and the same with each round's f, g requests in one
    persistent launch over all toys (captured into a CUDA graph once its
    shape repeats).  (A
    matrix-free lockstep, every inner CG product a row of the shared launch,
    took 7x the GPU time in a measured run: fit_multi(..., matrix_free=True).)  A
    fit reaches the global minimum when its NLL is within 0.01 of the best NLL
    of its toy (over both arms and a fit from the generating point)."""
    from paper_2403_09225_b300 import binding
    from paper_2403_09225_b300 import workload as W
    rng = np.random.default_rng(seed)
    toys, Ls = [], []
    for i in range(n_toys):
        nd = int(round(10 ** rng.uniform(4, 5)))
        cfg = W.Config("toy%d" % i, int(rng.integers(5, 31)), int(rng.integers(2, 5)), nd, 5 * nd, 4, False,
                       100 + i)
        table = W.make_table(cfg)
        wl = W.make_workload(cfg, intensity=gpu_intensity_fn(table, cfg.K, cfg.S))
        toys.append(wl)
        Ls.append(binding.make_likelihood(wl))
    try:
        starts = [W.random_starts(wl, n_starts) for wl in toys]
        best = [L.fit(wl.theta_true, xtol=1e-8, time_limit_s=time_limit)[1]["nll"] for L, wl in zip(Ls, toys)]
        t0 = time.perf_counter()
        plain = [[L.fit(s, xtol=1e-8, time_limit_s=time_limit)[1] for s in st] for L, st in zip(Ls, starts)]
        t_plain = time.perf_counter() - t0
        # in lockstep every fit advances once per round, so a fit's wall-clock
        # limit is scaled by the number of fits sharing the rounds: both arms
        # then grant a fit the same GPU time at most
        t0 = time.perf_counter()
        _, batched, _ = binding.fit_multi(Ls, starts, xtol=1e-8, time_limit_s=time_limit * n_toys * n_starts)
        t_batched = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, one, _ = binding.fit_multi(Ls, starts, xtol=1e-8, time_limit_s=time_limit * n_toys * n_starts,
                                      one_launch=True)
        t_one = time.perf_counter() - t0
        for i in range(n_toys):
            best[i] = min([best[i]] + [r["nll"] for r in plain[i]] + [r["nll"] for r in batched[i]] +
                          [r["nll"] for r in one[i]])

        def arm(results, seconds):
            ok = sum(1 for i in range(n_toys) for r in results[i] if r["nll"] <= best[i] + 0.01)
            return {"fits": n_toys * n_starts, "reached_global_min": ok, "gpu_seconds": seconds,
                    "fits_to_global_min_per_s": ok / seconds if seconds > 0 else 0.0,
                    "passes": int(sum(r["n_fev"] + r["n_hvp"] + r["n_hess"] for rr in results for r in rr)),
                    "statuses": sorted({r["status"] for rr in results for r in rr})}
        return {"toys": n_toys, "starts_per_toy": n_starts, "time_limit_s_per_fit": time_limit,
                "K": [wl.K for wl in toys], "S": [wl.S for wl in toys], "n_data": [wl.data.n for wl in toys],
                "plain": arm(plain, t_plain), "batched": arm(batched, t_batched),
                "batched_one_launch": arm(one, t_one),
                "arms": {"plain": "one fit after another, one Hessian pass per outer iteration",
                         "batched": "all fits of all toys in lockstep: per round one batched pass per toy for the "
                                    "f, g requests (each toy on its own stream) and one batched Hessian pass per toy",
                         "batched_one_launch": "the same with each round's f, g requests in one launch over "
                                               "every toy (pwa_eval_multi_device)"}}
    finally:
        for L in Ls:
            L.close()


def coupling_metric(L, wl, reps: int = 20):
    """The fixed-mass coupling sub-problem at the paper scale: NLL, gradient
    and H v in the coupling parameters for 16 coupling vectors per call
    (tcgen05 GEMMs on three-part BF16 splits of U = BW F tiles of the data
    events plus the K x K integral matrix for the MC term), against one fused
    pass per vector.
    Times are host-synchronous calls (upload, launches, download)."""
    from paper_2403_09225_b300 import binding
    th0 = wl.theta_true
    t0 = time.perf_counter()
    cp = binding.Coupling(L, th0)
    create_s = time.perf_counter() - t0
    try:
        rng = np.random.default_rng(3)
        C = 16
        rows = th0[:cp.Pc] * (1 + 0.05 * rng.standard_normal((C, cp.Pc)))
        vs = rng.standard_normal((C, cp.Pc))
        cp.eval(rows, vs)
        t0 = time.perf_counter()
        for _ in range(reps):
            cp.eval(rows, vs)
        ms = (time.perf_counter() - t0) / reps * 1e3
        v = np.linspace(-1.0, 1.0, L.P)
        L.eval(th0, v)
        t0 = time.perf_counter()
        for _ in range(reps):
            L.eval(th0, v)
        fused_ms = (time.perf_counter() - t0) / reps * 1e3
        rows_per_call = wl.data.n * wl.S
        # useful flops per (event, projection) row: two real GEMMs of 2K x 4C
        flops = 2 * 2.0 * (2 * wl.K) * (4 * C) * rows_per_call
        tpk, tkind = bf16_peak()
        achieved = flops / (ms * 1e-3) / 1e12
        return {"vectors_per_call": C, "ms_per_call": ms, "us_per_vector": ms * 1e3 / C,
                "fused_pass_us_per_vector": fused_ms * 1e3, "speedup_per_vector": fused_ms * C / ms,
                "create_s": create_s, "K": wl.K, "S": wl.S, "data_events": wl.data.n,
                "roofline": {"bound": "tensor", "achieved": achieved, "unit": "TFLOP/s",
                             "peak": tpk, "frac": achieved / tpk, "peak_kind": tkind,
                             "flops_per_call": flops, "note": "useful flops of the two GEMMs; the BF16 "
                             "three-part split issues 6 products (split terms i + j <= 2) per useful one"}}
    finally:
        cp.close()


def learned_metric(n_train: int, n_eval: int, n_random: int, time_limit: float, pool: int = 10_000_000,
                   n_events: int = 100_000, n_mc: int = 500_000, epochs: int = 60, polish: bool = False,
                   main=None):
    """The learned starting-point proposal on the paper-scale model (K = 20,
    S = 4, 78 parameters): n_train pseudo-experiments (theta from the prior,
    up to n_events events accept-rejected from a pool of phase-space events,
    labels from capped Newton-CG fits started at theta), the 4096 -> 3 x 512
    -> 78 network trained with the library's BF16 kernels, then n_eval
    held-out experiments fitted from the network's start and from n_random
    prior starts (one batched call) with the same options.  With main =
    (likelihood, workload, best NLL of the fit leg or None, fit time limit,
    the fit leg's line-search record or None), also the benchmark's own
    paper-scale workload (1e6 data events): the network's start for its data
    histogram, fitted alone and as a batch with three draws around it,
    against the fit leg's random starts."""
    import torch
    from paper_2403_09225_b300 import proposal, workload as W
    cfg = W.CONFIGS["paper"]
    table = W.make_table(cfg)
    t0 = time.perf_counter()
    gen = proposal.Generator(table, cfg.S, pool_size=pool, n_mc=n_mc, seed=7)
    gen_setup_s = time.perf_counter() - t0
    try:
        t0 = time.perf_counter()
        ex = proposal.make_experiments(gen, n_train, n_events, seed=100)
        make_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        net, codec, hist = proposal.train(ex, table, epochs=epochs, batch=128, lr=1e-3)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        # one training step's tensor-core throughput (forward + backward products: 6 B fan_in fan_out)
        sizes = [(net.n_in, net.hidden)] + [(net.hidden, net.hidden)] * (net.layers - 1) + \
                [(net.hidden, 128 * ((net.n_out + 127) // 128))]
        flops = 6.0 * 128 * sum(a * b for a, b in sizes)
        T = torch.from_numpy(codec.encode(ex.theta_fit[:128])).cuda()
        stream = torch.cuda.current_stream()
        for _ in range(5):
            net.gradients(ex.X[:128], T)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 50
        e0.record(stream)
        for _ in range(reps):
            net.gradients(ex.X[:128], T)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / reps
        peak, kind = bf16_peak()
        t0 = time.perf_counter()
        recs, summ = proposal.evaluate(gen, net, codec, n_eval, n_events, n_random, seed=999,
                                       fit_opts=dict(time_limit_s=time_limit), polish=polish)
        eval_s = time.perf_counter() - t0
        paper_scale = None
        if main is not None:
            paper_scale = _learned_paper_scale(net, codec, gen, *main)
        net.close()
        return {"paper_scale": paper_scale, "model": "paper-scale table: K=20, S=4, P=78", "train_experiments": n_train,
                "eval_experiments": n_eval, "events_per_experiment": n_events, "pool_events": pool,
                "mc_events": n_mc, "kept_events_min_mean": [int(ex.n_events.min()), float(ex.n_events.mean())],
                "label_fit_s": ex.fit_s, "generate_s": ex.gen_s, "setup_s": gen_setup_s, "make_s": make_s,
                "epochs": epochs, "train_s": train_s, "loss_first_last": [hist[0], hist[-1]],
                "fit_time_limit_s": time_limit, "eval_s": eval_s, **summ,
                "gradient_step": {"batch": 128, "ms": step_ms, "flops": flops,
                                  "roofline": {"bound": "tensor", "achieved": flops / (step_ms * 1e-3) / 1e12,
                                               "unit": "TFLOP/s", "peak": peak,
                                               "frac": flops / (step_ms * 1e-3) / 1e12 / peak,
                                               "peak_kind": kind}}}
    finally:
        gen.close()


def _learned_paper_scale(net, codec, gen, L, wl, best_fit, time_limit, random_runs):
    """The trained network on the benchmark's own workload: its start for the
    data sample's histogram, one fit from it and one batched call from it and
    three draws around it (the learned leg's batched form); a fit reaches the
    global minimum when its NLL is within 0.01 of the best NLL seen (these
    fits, the fit leg's random starts and its fits from theta_true)."""
    import torch
    from paper_2403_09225_b300 import binding, proposal
    m2 = torch.from_numpy(np.ascontiguousarray(wl.data.m2, dtype=np.float32)).cuda()
    idx = torch.arange(wl.data.n, dtype=torch.int32, device="cuda")
    X = binding.dalitz_histogram(m2, idx, gen.nb, gen.bounds, log_scale=True)[None]
    start = proposal.propose(net, codec, X)[0]
    t0 = time.perf_counter()
    _, info = L.fit(start, xtol=1e-8, time_limit_s=time_limit)
    t_one = time.perf_counter() - t0
    starts = proposal.perturbed_starts(codec, start, 4, np.random.default_rng(5))
    t0 = time.perf_counter()
    _, infos, _ = L.fit_batch(starts, xtol=1e-8, time_limit_s=time_limit * 4)
    t_batch = time.perf_counter() - t0
    nll_b = [d["nll"] for d in infos]
    best = min([info["nll"]] + nll_b + ([best_fit] if best_fit is not None else []))
    out = {"events": int(wl.data.n + wl.mc.n), "nll_learned": info["nll"], "t_learned": t_one,
           "status_learned": info["status"], "nll_learned_batch": nll_b, "t_learned_batch": t_batch,
           "best_nll": best, "learned_hit": bool(info["nll"] <= best + 0.01),
           "learned_batch_hit": bool(min(nll_b) <= best + 0.01)}
    if random_runs is not None:
        hits = sum(1 for f in random_runs["nll"] if f <= best + 0.01)
        out["random"] = {"starts": len(random_runs["nll"]), "gpu_seconds": random_runs["gpu_seconds"],
                         "hits": hits, "dnll_closest": min(random_runs["nll"]) - best}
    # how close each form came (the 0.01 criterion is finer than an FP32 pass resolves at |NLL| ~ 1.5e6)
    out["dnll_closest"] = {"learned": info["nll"] - best, "learned_batch": min(nll_b) - best}
    out["fits_to_global_min_per_s"] = {
        "learned": (1.0 if out["learned_hit"] else 0.0) / t_one,
        "learned_batch": (1.0 if out["learned_batch_hit"] else 0.0) / t_batch,
        "random": (out["random"]["hits"] / out["random"]["gpu_seconds"]) if random_runs else None}
    return out


def mlp_step_metric(batches=(128, 512, 1024), reps: int = 50):
    """The learned proposal's network (4096 -> 3 x 512 GELU -> 78) alone: one
    gradient step (forward, loss, backward on the tcgen05 products; replayed
    as a CUDA graph after its first calls) per batch size, CUDA events over
    `reps` host-synchronous calls, useful flops 6 B sum fan_in fan_out."""
    import torch
    from paper_2403_09225_b300 import binding
    peak, kind = bf16_peak()
    sizes = [(4096, 512), (512, 512), (512, 512), (512, 128)]
    out = {"network": "4096 -> 3 x 512 GELU -> 78 (output padded to 128 in the products)"}
    for B in batches:
        net = binding.ProposalMLP(4096, 512, 3, 78, B, seed=1)
        try:
            g = torch.Generator(device="cuda").manual_seed(B)
            x = torch.randn(B, 4096, device="cuda", generator=g)
            t = torch.randn(B, 78, device="cuda", generator=g)
            for _ in range(5):
                net.gradients(x, t)
            stream = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                net.gradients(x, t)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            flops = 6.0 * B * sum(a * b for a, b in sizes)
            out["batch_%d" % B] = {"ms": ms, "tflops": flops / (ms * 1e-3) / 1e12,
                                   "frac": flops / (ms * 1e-3) / 1e12 / peak, "peak": peak, "peak_kind": kind}
        finally:
            net.close()
    return out


def variant_shapes(table):
    """The benchmark's variant model: every third resonance (k = 1, 4, ...)
    with a mass-dependent width, resonance 6 (a pi pi resonance) Flatte with a
    K K second channel, the rest constant width."""
    from types import SimpleNamespace
    from paper_2403_09225_b300 import binding, workload as W
    out = []
    for k, r in enumerate(table):
        a, b, _ = W.CHANNEL_PAIRS[r.channel]
        ma, mb = W.DAUGHTER_MASSES[a], W.DAUGHTER_MASSES[b]
        if k == 6:
            out.append(SimpleNamespace(kind=binding.SHAPE_FLATTE, ma=ma, mb=mb, mc=0.4937, md=0.4937, radius=3.0,
                                       width2=0.25))
        elif k % 3 == 1:
            out.append(SimpleNamespace(kind=binding.SHAPE_MASS_DEPENDENT, ma=ma, mb=mb, mc=0.0, md=0.0, radius=3.0,
                                       width2=0.0))
        else:
            out.append(SimpleNamespace(kind=binding.SHAPE_CONSTANT, ma=0.0, mb=0.0, mc=0.0, md=0.0, radius=3.0,
                                       width2=0.0))
    return out


def variant_metric(wl, reps: int = 10):
    """The physics variants at the paper scale (same events): one fused
    NLL + gradient + H v pass of the variant kernel per call, with one coupling
    per resonance and with one per (resonance, projection).  Host-synchronous
    calls, timed with CUDA events on the calling stream over `reps` calls."""
    import torch
    from paper_2403_09225_b300 import binding
    shapes = variant_shapes(wl.table)
    nd, nm, K, S = wl.data.n, wl.mc.n, wl.K, wl.S
    stream = torch.cuda.current_stream()
    peak, kind = peaks()
    out = {"model": "paper-scale table, every third resonance with a mass-dependent width, one Flatte",
           "events": nd + nm}
    for pp in (False, True):
        Lv = binding.Variant(wl.data, wl.mc, wl.table, K, S, shapes=shapes, per_projection=pp,
                             stream=stream.cuda_stream)
        try:
            th = binding.Variant.initial_theta(wl.table, shapes, S, pp)
            v = np.linspace(-1.0, 1.0, Lv.P)
            for _ in range(3):
                Lv.eval(th, v)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                Lv.eval(th, v)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            bpp = bytes_per_pass(nd, nm, K, S)
            achieved = bpp / (ms * 1e-3) / 1e9
            rec = {"P": Lv.P, "ms_per_pass": ms, "event_amps_per_s": (nd + nm) * K / (ms * 1e-3),
                   "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                "frac": achieved / peak, "peak_kind": kind, "algorithmic_bytes_per_launch": bpp}}
            if pp:
                # couplings only at fixed line shapes: the MC integral matrices once, then
                # one pass over the data events per call
                t0 = time.perf_counter()
                Lv.set_shapes(th)
                torch.cuda.synchronize()
                setup_s = time.perf_counter() - t0
                Pc = Lv.Pc
                vc = v[:Pc]
                for _ in range(3):
                    Lv.coupling_eval(th[:Pc], vc)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(reps):
                    Lv.coupling_eval(th[:Pc], vc)
                e1.record(stream)
                torch.cuda.synchronize()
                cms = e0.elapsed_time(e1) / reps
                rec["couplings_only"] = {"Pc": Pc, "set_shapes_s": setup_s, "ms_per_call": cms,
                                         "speedup_vs_full_pass": ms / cms,
                                         "data_bytes_per_call": nd * (8 * K * S + 16)}
            out["per_projection" if pp else "per_resonance"] = rec
        finally:
            Lv.close()
    return out


def hessian_metric(L, wl, reps: int = 10):
    """The Hessian pass (pwa_hessian: NLL, gradient and the full P x P
    Hessian from one pass over F) on the benchmark's workload: host calls
    timed with CUDA events on the handle's stream, plus the Gram-matrix
    flops it performs (X^T X over the (event, projection) rows of 4K
    columns for data and MC, z^T z over the data events)."""
    import torch
    th = wl.theta_true
    stream = torch.cuda.current_stream()

    def timed():
        for _ in range(2):
            L.hessian(th)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            L.hessian(th)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    C = 4 * wl.K
    rows = (wl.data.n + wl.mc.n) * wl.S
    # useful flops of the Gram matrices (full C x C: what the contraction computes)
    flops = 2.0 * rows * C * C + 2.0 * wl.data.n * C * C
    ms = timed()
    L.set_hessian_cuda_cores(True)
    ms_cc = timed()
    L.set_hessian_cuda_cores(False)
    peak, kind = bf16_peak()
    out = {"ms_per_call": ms, "P": L.P, "gram_flops_per_call": flops, "cuda_cores_ms_per_call": ms_cc,
           "fused_passes_per_hessian": None}
    if wl.K <= 32:
        out["gram_tflops"] = flops / (ms * 1e-3) / 1e12
        out["roofline"] = {"bound": "tensor", "achieved": out["gram_tflops"], "unit": "TFLOP/s", "peak": peak,
                           "frac": out["gram_tflops"] / peak, "peak_kind": kind,
                           "note": "useful Gram flops over the host call's time; the BF16 hi/lo split issues 2 "
                                   "products per useful one (hi^T hi, hi^T 2lo), and the event phase (Breit-Wigner, "
                                   "coherent sums, operand split) runs on the CUDA cores while the tiles' MMAs run"}
    return out


def diff_metric(reps: int = 20):
    """The differentiation configuration at full size: K = 40, S = 4, 2e6
    data + 1e7 MC phase-space events (15.4 GB of F), its caller-layout copy
    released after tiling (tiles only on the device).  The fused NLL +
    gradient + H v pass over device-resident parameters, CUDA events over
    `reps` back-to-back passes; the Hessian pass once (host-synchronous)."""
    import torch
    from paper_2403_09225_b300 import binding, workload as W
    cfg = W.CONFIGS["diff"]
    t0 = time.perf_counter()
    wl = W.make_workload(cfg, intensity=None)
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    L = binding.make_likelihood(wl, stream=stream.cuda_stream)
    try:
        before = L.device_bytes()
        L.release_event_copies()
        after = L.device_bytes()
        P = L.P
        th = W.random_starts(wl, 1)[0]
        d_th = torch.tensor(th, dtype=torch.float64, device="cuda")
        d_v = torch.tensor(np.linspace(-1.0, 1.0, P), dtype=torch.float64, device="cuda")
        d_out = torch.empty(1 + 2 * P, dtype=torch.float64, device="cuda")
        for _ in range(3):
            L.eval_device(d_th.data_ptr(), d_v.data_ptr(), d_out.data_ptr(), True, True)
        L.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            L.eval_device(d_th.data_ptr(), d_v.data_ptr(), d_out.data_ptr(), True, True)
        e1.record(stream)
        torch.cuda.synchronize()
        L.sync()
        ms = e0.elapsed_time(e1) / reps
        nd, nm = wl.data.n, wl.mc.n
        bpp = bytes_per_pass(nd, nm, cfg.K, cfg.S)
        peak, kind = peaks()
        achieved = bpp / (ms * 1e-3) / 1e9
        L.hessian(th)
        t0 = time.perf_counter()
        L.hessian(th)
        hess_ms = (time.perf_counter() - t0) * 1e3
        return {"workload": "differentiation: K=40, S=4, 2e6 data + 1e7 MC (phase space), P=%d" % P,
                "generate_s": gen_s, "ms_per_pass": ms, "event_amps_per_s": (nd + nm) * cfg.K / (ms * 1e-3),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_kind": kind, "algorithmic_bytes_per_launch": bpp},
                "device_bytes_with_copies": before, "device_bytes_after_release": after,
                "f_bytes": (nd + nm) * cfg.K * cfg.S * 8, "hessian_call_ms": hess_ms}
    finally:
        L.close()


def measured_traffic(tiling: dict):
    """DRAM bytes per launch of the fused HVP pass from the committed ncu
    summary, when it was taken with the tiling in use (else None)."""
    path = os.path.join(ROOT, "profiles", "pass_kernel_hvp_paper_traffic.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_revision") != KERNEL_REVISION or kv.get("tiling") != "%d,%d" % (
                tiling["warps"], tiling["stages"]):
            return None
        return float(kv["dram_bytes_per_launch_full"])
    except (OSError, KeyError, ValueError):
        return None


def aggregate_replicas(ms: float, units: float, dist=None, device="cuda"):
    """Whole-job throughput of independent replicas: every rank processed
    `units` in `ms` milliseconds; the job takes the slowest rank's time."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * units / (ms * 1e-3), ms


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fits", type=int, default=16, help="random-start fits for the fit metric (0: skip)")
    ap.add_argument("--fit-time-limit", type=float, default=60.0, help="seconds per fit (early stopping)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tiling", default="", help="warps,lanes_per_event,stages[,blocks_per_sm] (default: library's)")
    ap.add_argument("--no-coupling", action="store_true", help="skip the fixed-mass coupling sub-problem leg")
    ap.add_argument("--no-variants", action="store_true", help="skip the physics-variant leg")
    ap.add_argument("--no-diff", action="store_true", help="skip the full-size differentiation configuration leg")
    ap.add_argument("--mlp-timing", action="store_true",
                    help="also time the learned proposal's network (gradient step at batches 128, 512, 1024)")
    ap.add_argument("--batching", default="12,16", metavar="TOYS,STARTS",
                    help="uneven-size toy-fit comparison (plain vs batched); 0 to skip")
    ap.add_argument("--learned", default="8192,48,16", metavar="TRAIN,EVAL,STARTS",
                    help="train and evaluate the learned starting-point proposal; 0 to skip")
    ap.add_argument("--learned-time-limit", type=float, default=20.0, help="seconds per fit call in the learned leg")
    ap.add_argument("--learned-polish", action="store_true",
                    help="in the learned leg, also fit each learned start's couplings first (coupling object)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="event counts relative to the workload (profiling captures only; default 1)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2403_09225_b300 import binding
    wl = build_workload(args.scale)
    K, S, nd, nm = wl.K, wl.S, wl.data.n, wl.mc.n
    stream = torch.cuda.current_stream()
    L = binding.make_likelihood(wl, stream=stream.cuda_stream)
    if args.tiling:
        L.set_tiling(*[int(x) for x in args.tiling.split(",")])
    P = L.P
    rng = np.random.default_rng(1)
    th = wl.theta_true + 0.01 * rng.standard_normal(P)
    v = rng.standard_normal(P)
    d_th = torch.tensor(th, dtype=torch.float64, device="cuda")
    d_v = torch.tensor(v, dtype=torch.float64, device="cuda")
    d_out = torch.empty(1 + 2 * P, dtype=torch.float64, device="cuda")

    # ---- device-resident timing: K back-to-back fused passes ----
    for _ in range(max(3, args.warmup)):
        L.eval_device(d_th.data_ptr(), d_v.data_ptr(), d_out.data_ptr(), True, True)
    torch.cuda.synchronize()
    L.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            L.eval_device(d_th.data_ptr(), d_v.data_ptr(), d_out.data_ptr(), True, True)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    L.sync()
    units = (nd + nm) * K
    value, ms = aggregate_replicas(e0.elapsed_time(e1) / args.steps, units, dist)
    bpp = bytes_per_pass(nd, nm, K, S)
    peak, peak_kind = peaks()
    achieved = bpp / (ms * 1e-3) / 1e9

    # ---- the conjugate-gradient product: H v passes reusing the full pass's sums at th ----
    L.eval_device(d_th.data_ptr(), d_v.data_ptr(), d_out.data_ptr(), True, True)  # full pass keeps the sums
    for _ in range(3):
        L.hvp_reuse_device(d_th.data_ptr(), d_v.data_ptr(), d_out.data_ptr())
    torch.cuda.synchronize()
    L.sync()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(args.steps):
        L.hvp_reuse_device(d_th.data_ptr(), d_v.data_ptr(), d_out.data_ptr())
    r1.record(stream)
    torch.cuda.synchronize()
    L.sync()
    reuse_ms = r0.elapsed_time(r1) / args.steps
    reuse = {"ms_per_pass": reuse_ms, "event_amps_per_s": units_per_pass(nd, nm, K) / (reuse_ms * 1e-3),
             "roofline": {"bound": "hbm", "achieved": bytes_per_pass(nd, nm, K, S) / (reuse_ms * 1e-3) / 1e9,
                          "peak": peaks()[0], "unit": "GB/s",
                          "frac": bytes_per_pass(nd, nm, K, S) / (reuse_ms * 1e-3) / 1e9 / peaks()[0],
                          "peak_kind": peaks()[1], "algorithmic_bytes_per_launch": bytes_per_pass(nd, nm, K, S)},
             "note": "H v at the theta of the last full pass: Q sums, G and the gradient reused, P1, P2 and "
                     "Gdot formed (one inner CG iteration of a matrix-free Newton-CG solve)"}

    # ---- end to end through the C ABI with host vectors (pinned staging inside) ----
    e2e_steps = max(1, args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        L.eval(th, v)
    e2e_dt = time.perf_counter() - t0
    e2e_value, e2e_ms = aggregate_replicas(e2e_dt / e2e_steps * 1e3, units, dist)

    hess = None
    if rank == 0:
        hess = hessian_metric(L, wl)
        hess["fused_passes_per_hessian"] = hess["ms_per_call"] / ms

    fit = None
    if args.fits > 0 and rank == 0:
        t0 = time.perf_counter()
        fit = fit_metric(L, wl, args.fits, time_limit=args.fit_time_limit)
        fit["leg_s"] = time.perf_counter() - t0

    coupling = None
    if rank == 0 and not args.no_coupling:
        coupling = coupling_metric(L, wl)

    batching = None
    if args.batching not in ("", "0") and rank == 0:
        n_toys, n_starts = (int(x) for x in args.batching.split(","))
        t0 = time.perf_counter()
        batching = batching_metric(n_toys, n_starts, time_limit=args.fit_time_limit)
        batching["leg_s"] = time.perf_counter() - t0

    variants = None
    if rank == 0 and not args.no_variants:
        variants = variant_metric(wl)

    diff = None
    if rank == 0 and not args.no_diff:
        diff = diff_metric()

    mlp_step = None
    if args.mlp_timing and rank == 0:
        mlp_step = mlp_step_metric()

    learned = None
    if args.learned not in ("", "0") and rank == 0:
        n_train, n_eval, n_rand = (int(x) for x in args.learned.split(","))
        t0 = time.perf_counter()
        main = (L, wl, fit["paper"]["best_nll"] if fit else None, args.fit_time_limit,
                fit["paper"]["line_search"] if fit else None)
        learned = learned_metric(n_train, n_eval, n_rand, time_limit=args.learned_time_limit,
                                 polish=args.learned_polish, main=main)
        learned["leg_s"] = time.perf_counter() - t0

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg()
        if fit is not None:
            # the oracle on a paper-scale fit of the GPU fits' length, extrapolated: its full-scale
            # pass time (the 1/60 sample's x 60) times the GPU fits' f, g evaluations per fit (a
            # lower bound: the oracle's matrix-free CG adds one H v pass per inner iteration)
            ls = fit["paper"]["line_search"]
            fev = (ls["passes"] - ls["hessian_passes"]) / max(1, ls["starts"])
            cpu["paper_fit_extrapolated"] = {"pass_s_full_scale": 60.0 * cpu["pass_s_sample"],
                                             "fg_evaluations_per_gpu_fit": fev,
                                             "seconds_lower_bound": fev * 60.0 * cpu["pass_s_sample"],
                                             "gpu_seconds_per_fit": ls["gpu_seconds"] / max(1, ls["starts"])}

    til = L.get_tiling()
    traffic = measured_traffic(til)

    if rank == 0:
        res = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper-scale: K=20, S=4, 1e6 data (accept-reject from I) + 5e6 MC, P=78"
                       + ("" if args.scale == 1.0 else " (scaled x%g for profiling)" % args.scale),
                       "n_data": nd, "n_mc": nm, "K": K, "S": S, "P": P, "parallelism": "replicas" if world > 1
                       else "single", "l2": "inputs (%.2f GB) larger than L2, no flush" % (bpp / 1e9),
                       "tiling": til},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": bpp},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * P * 8,
                    "d2h_bytes_per_step": (1 + 2 * P) * 8 + 12, "ms_per_step": e2e_ms},
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
        }
        res["hvp_reuse"] = reuse
        if hess is not None:
            res["hessian"] = hess
        if cpu is not None:
            res["cpu_baseline"] = cpu
        if fit is not None:
            res["fit"] = fit
        if batching is not None:
            res["batching"] = batching
        if coupling is not None:
            res["coupling"] = coupling
        if variants is not None:
            res["variants"] = variants
        if diff is not None:
            res["diff"] = diff
        if mlp_step is not None:
            res["mlp_step"] = mlp_step
        if learned is not None:
            res["learned"] = learned
        print(json.dumps(res))
    L.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
