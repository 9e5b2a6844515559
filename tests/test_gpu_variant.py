"""Physics variants on the GPU (pwa_variant_*) against the hyper-dual oracle
(oracle/variants.py): mass-dependent widths, Flatte line shapes, one coupling
per resonance or per (resonance, projection).  Bars as for the main path:
NLL within 1e-6 of max(|NLL|, sum w |ln I|) (the two terms of Eq. 3 nearly
cancel on small samples), gradient within 1e-5 and H v within 1e-4 of their
largest component, fitted theta within 1e-3 of the oracle's parameter errors."""
import numpy as np
import pytest

from oracle import newton_cg as ncg
from oracle import variants as V
from paper_2403_09225_b300 import workload as W

pytestmark = pytest.mark.gpu

PI, PHI, K_MASS = 0.1396, 1.0195, 0.4937
_CACHE = {}


def shapes_for(table, flatte_k=None, md_every=3):
    """Line shapes: every md_every-th resonance with a mass-dependent width (its
    channel's daughters), resonance flatte_k Flatte (pi pi / K K), else constant."""
    out = []
    for k, r in enumerate(table):
        a, b, _ = W.CHANNEL_PAIRS[r.channel]
        ma, mb = W.DAUGHTER_MASSES[a], W.DAUGHTER_MASSES[b]
        if k == flatte_k:
            out.append(V.Shape(V.KIND_FLATTE, ma=ma, mb=mb, mc=K_MASS, md=K_MASS, width2=0.25))
        elif k % md_every == 1:
            out.append(V.Shape(V.KIND_MASS_DEPENDENT, ma=ma, mb=mb, radius=3.0))
        else:
            out.append(V.Shape(V.KIND_CONSTANT))
    return out


def variant_case(name, per_projection):
    key = (name, per_projection)
    if key in _CACHE:
        return _CACHE[key]
    if name == "tiny":
        cfg, nd, nm, fk = W.CONFIGS["tiny"], 2003, 6011, 2
    elif name == "k7s3":
        cfg, nd, nm, fk = W.Config("k7s3", 7, 3, 0, 0, 4, False, 5), 1501, 4507, 3
    else:
        cfg, nd, nm, fk = W.CONFIGS["paper"], 1203, 3001, 6
    table = W.make_table(cfg)
    if name == "tiny":
        table[0].channel = 0
    vm = V.VariantModel.from_table(table, cfg.S, shapes_for(table, fk), per_projection)
    th_gen = vm.theta0()
    fn = lambda m2, F: V.intensity(vm, th_gen, m2, F)
    wl = W.make_workload(cfg, intensity=fn, n_data=nd, n_mc=nm)
    _CACHE[key] = (cfg, table, vm, wl)
    return _CACHE[key]


def make_variant(cfg, table, vm, wl):
    from paper_2403_09225_b300 import binding
    return binding.Variant(wl.data, wl.mc, table, cfg.K, cfg.S, shapes=vm.shapes, per_projection=vm.per_projection)


@pytest.mark.parametrize("name,per_projection", [("tiny", False), ("tiny", True), ("k7s3", False),
                                                 ("k7s3", True), ("paper", False), ("paper", True)])
def test_variant_matches_oracle(name, per_projection):
    cfg, table, vm, wl = variant_case(name, per_projection)
    Lv = make_variant(cfg, table, vm, wl)
    assert Lv.P == vm.P
    rng = np.random.default_rng(7)
    th = vm.theta0() * (1 + 0.02 * rng.standard_normal(vm.P))
    v = rng.standard_normal(vm.P)
    f, g, hv = Lv.eval(th, v)
    fo, go, hvo = V.nll_grad_hvp(vm, th, v, wl.data, wl.mc)
    I = V.intensity(vm, th, wl.data.m2, wl.data.F)
    scale = max(abs(fo), float(np.sum(np.abs(np.log(I)))))
    assert abs(f - fo) <= 1e-6 * scale, (f, fo)
    eg = np.max(np.abs(g - go)) / np.max(np.abs(go))
    eh = np.max(np.abs(hv - hvo)) / np.max(np.abs(hvo))
    print("%s per_projection=%s P=%d: grad %.2e, H v %.2e" % (name, per_projection, vm.P, eg, eh))
    assert eg <= 1e-5 and eh <= 1e-4, (eg, eh)
    # the NLL-only and gradient-only kernels (other instances, other FP32
    # operation order) agree with the oracle at the same bars
    assert abs(Lv.nll(th) - fo) <= 1e-6 * scale
    f2, g2, _ = Lv.eval(th)
    assert abs(f2 - fo) <= 1e-6 * scale
    assert np.max(np.abs(g2 - go)) <= 1e-5 * np.max(np.abs(go))
    # the library's table-order start point is the oracle's
    from paper_2403_09225_b300 import binding
    assert np.allclose(binding.Variant.initial_theta(table, vm.shapes, cfg.S, per_projection), vm.theta0())
    Lv.close()


def test_constant_width_variant_equals_the_main_path():
    """With constant widths and one coupling per resonance the variant is the
    main path's model: both GPU evaluations agree (and both match the oracle
    elsewhere)."""
    from paper_2403_09225_b300 import binding
    cfg = W.CONFIGS["paper"]
    table = W.make_table(cfg)
    wl = W.make_workload(cfg, n_data=4001, n_mc=12003)
    Lv = binding.Variant(wl.data, wl.mc, table, cfg.K, cfg.S)
    L = binding.make_likelihood(wl)
    rng = np.random.default_rng(3)
    th = wl.theta_true * (1 + 0.02 * rng.standard_normal(L.P))
    v = rng.standard_normal(L.P)
    f, g, hv = Lv.eval(th, v)
    fm, gm, hvm = L.eval(th, v)
    assert abs(f - fm) <= 1e-6 * max(abs(fm), 1.0)
    assert np.max(np.abs(g - gm)) <= 1e-5 * np.max(np.abs(gm))
    assert np.max(np.abs(hv - hvm)) <= 1e-4 * np.max(np.abs(hvm))
    Lv.close()
    L.close()


def test_variant_rejects_a_mass_below_its_threshold():
    from paper_2403_09225_b300 import binding
    cfg, table, vm, wl = variant_case("tiny", False)
    Lv = make_variant(cfg, table, vm, wl)
    th = vm.theta0()
    lay = vm.layout()
    k_md = [k for k, sh in enumerate(vm.shapes) if sh.kind == V.KIND_MASS_DEPENDENT][0]
    i = [j for j, (n, k, _) in enumerate(lay) if n == "mass" and k == k_md][0]
    th[i] = 0.2  # below pi pi threshold 0.279
    with pytest.raises(binding.PwaError):
        Lv.eval(th)
    Lv.close()


@pytest.mark.parametrize("name,per_projection", [("tiny", False), ("k7s3", True)])
def test_variant_batch_equals_single_evaluations(name, per_projection):
    """B vectors in one launch: every vector runs the single evaluation's
    blocks, so NLL, gradient and H v equal pwa_variant_eval's bit for bit; a
    vector with a mass below its pair threshold gets PWA_EINVAL and one with
    an overflowing intensity PWA_ENONFINITE, without disturbing the others."""
    from paper_2403_09225_b300 import binding
    cfg, table, vm, wl = variant_case(name, per_projection)
    Lv = make_variant(cfg, table, vm, wl)
    rng = np.random.default_rng(3)
    P = vm.P
    ths = np.array([vm.theta0() * (1 + 0.02 * rng.standard_normal(P)) for _ in range(6)])
    vs = rng.standard_normal((6, P))
    lay = vm.layout()
    k_md = [k for k, sh in enumerate(vm.shapes) if sh.kind == V.KIND_MASS_DEPENDENT][0]
    i_m = [j for j, (n, k, _) in enumerate(lay) if n == "mass" and k == k_md][0]
    i_mag = [j for j, (n, _, _) in enumerate(lay) if n == "mag"][0]
    sh = vm.shapes[k_md]
    ths[2, i_m] = max(sh.ma, sh.mb)  # between |ma - mb| and ma + mb: q^2 < 0, outside the model's domain
    ths[4, i_mag] = 1e30  # the intensity overflows FP32
    for with_v in (False, True):
        f, g, hv, st = Lv.eval_batch(ths, vs if with_v else None)
        assert st[2] == binding.PWA_EINVAL and st[4] == binding.PWA_ENONFINITE
        for b in (0, 1, 3, 5):
            assert st[b] == binding.PWA_OK
            f1, g1, hv1 = Lv.eval(ths[b], vs[b] if with_v else None)
            assert f[b] == f1 and np.array_equal(g[b], g1)
            if with_v:
                assert np.array_equal(hv[b], hv1)
    Lv.close()


def _canonical(vm, th):
    th = np.array(th, dtype=float)
    lay = vm.layout()
    for i, (n, k, s) in enumerate(lay):
        if n == "mag" and th[i] < 0:
            th[i] = -th[i]
            j = [q for q, (n2, k2, s2) in enumerate(lay) if n2 == "phase" and k2 == k and s2 == s][0]
            th[j] += np.pi
    for i, (n, k, s) in enumerate(lay):
        if n == "phase":
            th[i] = np.pi - np.mod(np.pi - th[i], 2 * np.pi)
    return th


def test_variant_fit_matches_oracle_fit():
    cfg, table, vm, wl = variant_case("tiny", False)
    rng = np.random.default_rng(5)
    th0 = vm.theta0() * (1 + 0.03 * rng.standard_normal(vm.P))

    def fg(x):
        f, g, _ = V.nll_grad_hvp(vm, x, np.zeros(vm.P), wl.data, wl.mc)
        return f, g

    hp = lambda x, v: V.nll_grad_hvp(vm, x, v, wl.data, wl.mc)[2]
    ref = ncg.newton_cg(fg, hp, th0, xtol=1e-10, maxiter=200)
    assert ref.status in ncg.CONVERGED, ref.status_name
    Lv = make_variant(cfg, table, vm, wl)
    th, infos, ok = Lv.fit(th0[None], xtol=1e-10)
    assert ok, infos
    H = np.stack([hp(ref.x, e) for e in np.eye(vm.P)])
    sig = np.sqrt(np.diag(np.linalg.inv(0.5 * (H + H.T))))
    pull = (_canonical(vm, th[0]) - _canonical(vm, ref.x)) / sig
    assert np.max(np.abs(pull)) <= 1e-3, (pull, infos)
    assert abs(infos[0]["nll"] - ref.fun) <= 1e-6 * max(abs(ref.fun), 1.0)
    Lv.close()


@pytest.mark.parametrize("name,per_projection", [("tiny", True), ("k7s3", True), ("paper", False), ("paper", True)])
def test_coupling_only_matches_oracle(name, per_projection):
    """Fixed line shapes: the integral matrices Phi_s against the oracle's, and
    the coupling-only NLL, gradient and H v (data pass + Phi) against the
    oracle's full evaluation restricted to the couplings."""
    cfg, table, vm, wl = variant_case(name, per_projection)
    Lv = make_variant(cfg, table, vm, wl)
    rng = np.random.default_rng(11)
    th = vm.theta0() * (1 + 0.02 * rng.standard_normal(vm.P))
    phi = Lv.set_shapes(th)
    phio = V.integral_matrices(vm, th, wl.mc.m2, wl.mc.F)
    assert np.max(np.abs(phi - phio)) <= 1e-6 * np.max(np.abs(phio))
    Pc = V.coupling_count(vm)
    assert Lv.Pc == Pc
    v = np.zeros(vm.P)
    v[:Pc] = rng.standard_normal(Pc)
    f, g, hv = Lv.coupling_eval(th[:Pc], v[:Pc])
    fo, go, hvo = V.nll_grad_hvp(vm, th, v, wl.data, wl.mc)
    I = V.intensity(vm, th, wl.data.m2, wl.data.F)
    scale = max(abs(fo), float(np.sum(np.abs(np.log(I)))))
    assert abs(f - fo) <= 1e-6 * scale, (f, fo)
    eg = np.max(np.abs(g - go[:Pc])) / np.max(np.abs(go[:Pc]))
    eh = np.max(np.abs(hv - hvo[:Pc])) / np.max(np.abs(hvo[:Pc]))
    print("%s per_projection=%s Pc=%d: coupling-only grad %.2e, H v %.2e" % (name, per_projection, Pc, eg, eh))
    assert eg <= 1e-5 and eh <= 1e-4, (eg, eh)
    Lv.close()


def test_coupling_only_needs_the_shapes_first():
    from paper_2403_09225_b300 import binding
    cfg, table, vm, wl = variant_case("tiny", True)
    Lv = make_variant(cfg, table, vm, wl)
    with pytest.raises(binding.PwaError):
        Lv.coupling_eval(vm.theta0()[:V.coupling_count(vm)])
    Lv.close()


def test_coupling_only_fit_matches_oracle_fit():
    """Coupling-only Newton-CG (lockstep, on the data pass + Phi) against the
    oracle's Newton-CG on the couplings with the line shapes held fixed."""
    cfg, table, vm, wl = variant_case("tiny", True)
    Pc = V.coupling_count(vm)
    rng = np.random.default_rng(6)
    th_all = vm.theta0()
    shape = th_all[Pc:]
    c0 = th_all[:Pc] * (1 + 0.05 * rng.standard_normal(Pc))

    def full(c):
        return np.concatenate([c, shape])

    def fg(c):
        f, g, _ = V.nll_grad_hvp(vm, full(c), np.zeros(vm.P), wl.data, wl.mc)
        return f, g[:Pc]

    def hp(c, vc):
        return V.nll_grad_hvp(vm, full(c), np.concatenate([vc, np.zeros(vm.P - Pc)]), wl.data, wl.mc)[2][:Pc]

    ref = ncg.newton_cg(fg, hp, c0, xtol=1e-10, maxiter=200)
    assert ref.status in ncg.CONVERGED, ref.status_name
    Lv = make_variant(cfg, table, vm, wl)
    Lv.set_shapes(th_all)
    out, infos, ok = Lv.coupling_fit(c0[None], xtol=1e-10)
    assert ok, infos
    H = np.stack([hp(ref.x, e) for e in np.eye(Pc)])
    sig = np.sqrt(np.diag(np.linalg.inv(0.5 * (H + H.T))))
    pull = (_canonical(vm, full(out[0]))[:Pc] - _canonical(vm, full(ref.x))[:Pc]) / sig
    assert np.max(np.abs(pull)) <= 1e-3, (pull, infos)
    Lv.close()
