"""Write fit_k20.npz: the oracle's Newton-CG minimum for the paper-scale model
(K = 20, S = 4, P = 78) on a reduced sample, for the GPU fit-parity test.

Inputs: 2e4 data events accept-rejected from I at theta_true with the
oracle's FP64 intensity, 1e5 phase-space MC events (the seeded generator of
the workload module), start theta0 = theta_true (1 + 0.01 N(0, 1)) with
numpy's default_rng(8).  The fit is the oracle's textbook Newton-CG
(Nocedal & Wright Alg. 7.1 with a strong-Wolfe line search, xtol 1e-10);
its inner products H v come from the oracle's full Hessian (Eq. 7) at each
outer point, summed over event shards in worker processes (Eqs. 4-5).
That path takes some 180 Newton iterations across a multimodal surface, so
where it ends depends on rounding (an FP32 evaluation of the same path can
end in another local minimum).  The parity start is therefore a second one,
theta1 = minimum + 0.2 sigma N(0, 1) (default_rng(9)), inside the minimum's
basin; the oracle fit from theta1 gives the stored minimum.
Only the oracle runs here.  Stored: theta0, theta1, the minimum from theta1,
its NLL, the parameter errors sqrt(diag(H^-1)) there, the statuses, and a
SHA-256 of the sample's bytes (the test checks that it regenerates the same
events).

Usage: python tests/golden/make_fit_k20.py   (about 5 minutes on 8 cores)
"""
import hashlib
import multiprocessing as mp
import os
import sys
from concurrent.futures import ProcessPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

N_DATA, N_MC = 20_000, 100_000


def sample_hash(wl) -> str:
    h = hashlib.sha256()
    for a in (wl.data.m2, wl.data.F, wl.mc.m2, wl.mc.F):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def start(wl, P):
    rng = np.random.default_rng(8)
    return wl.theta_true * (1 + 0.01 * rng.standard_normal(P))


def basin_start(theta_min, sigma):
    rng = np.random.default_rng(9)
    return theta_min + 0.2 * sigma * rng.standard_normal(theta_min.size)


def main():
    import oracle
    from oracle import newton_cg as ncg
    from conftest import small_workload
    pool = ProcessPoolExecutor(max_workers=max(2, min(32, os.cpu_count() or 2)), mp_context=mp.get_context("spawn"))
    try:
        wl, model = small_workload("paper", N_DATA, N_MC)
        th0 = start(wl, model.P)
        cache = {}

        def hess(x):
            key = x.tobytes()
            if key not in cache:
                cache.clear()
                cache[key] = oracle.sharded_hessian(model, x, wl.data, wl.mc, pool=pool, shard=5000)[2]
            return cache[key]

        fg = lambda x: oracle.sharded_nll_grad_hvp(model, x, None, wl.data, wl.mc, pool=pool, shard=10000)[:2]
        hp = lambda x, v: hess(x) @ v
        ref0 = ncg.newton_cg(fg, hp, th0, xtol=1e-10, maxiter=400)
        th1 = basin_start(ref0.x, oracle.parameter_errors(hess(ref0.x)))
        ref = ncg.newton_cg(fg, hp, th1, xtol=1e-10, maxiter=400)
        sig = oracle.parameter_errors(hess(ref.x))
        np.savez(os.path.join(HERE, "fit_k20.npz"), theta0=th0, theta1=th1, theta_min=ref.x, nll=ref.fun,
                 sigma=sig, status0=ref0.status_name, iters0=ref0.iters, nll0=ref0.fun, status=ref.status_name,
                 iters=ref.iters, sample_sha256=sample_hash(wl), n_data=N_DATA, n_mc=N_MC)
        print("from theta0:", ref0.status_name, ref0.iters, ref0.fun)
        print("from theta1:", ref.status_name, ref.iters, ref.fun)
    finally:
        pool.shutdown()


if __name__ == "__main__":
    main()
