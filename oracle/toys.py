"""Toy fits for the recovery pin of the oracle -- TEST INFRASTRUCTURE ONLY.

A toy draws a data sample from I(theta_true) (accept-reject with the oracle's
own intensity), fits it with the oracle's Newton-CG from theta_true and
returns the pulls (theta_hat - theta_true) / sigma, sigma from the oracle's
Hessian at the minimum.  Toys are independent, so they run in spawned worker
processes.
"""
from __future__ import annotations

import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np

import oracle
from oracle import newton_cg as ncg


def _one_toy(args):
    from paper_2403_09225_b300 import workload as W
    config_name, toy_seed, n_data, n_mc, mc_seed = args
    cfg = W.CONFIGS[config_name]
    table = W.make_table(cfg)
    model = oracle.Model.from_table(table, cfg.S)
    th_true = W.free_parameter_vector(table)
    mc = W.phase_space_sample(W.rng_stream(mc_seed, W.STREAM_MC), n_mc, table, cfg.S)
    fn = lambda m2, F: oracle.intensity_full(cfg.K, cfg.S, model.channels, model.par0, m2, F)
    data, _ = W.accept_reject_sample(W.rng_stream(toy_seed, W.STREAM_DATA), n_data, table, cfg.S,
                                     fn, pool=20_000)
    fg = lambda x: oracle.nll_grad(model, x, data, mc)
    hp = lambda x, v: oracle.nll_grad_hvp(model, x, v, data, mc)[2]
    res = ncg.newton_cg(fg, hp, th_true, xtol=1e-9, maxiter=100)
    sig = oracle.parameter_errors(oracle.hessian(model, res.x, data, mc))
    return res.status, (oracle.canonical(model, res.x) - th_true) / sig


def toy_pulls(config_name: str, n_toys: int, n_data: int, n_mc: int, workers: int = 8,
              first_seed: int = 1000, mc_seed: int = 99):
    """(statuses, pulls[n_toys, P]) for n_toys independent toys."""
    jobs = [(config_name, first_seed + t, n_data, n_mc, mc_seed) for t in range(n_toys)]
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as pool:
        out = list(pool.map(_one_toy, jobs))
    return [o[0] for o in out], np.array([o[1] for o in out])
