"""Argument validation of the C ABI, on the CPU: every call below must
refuse its arguments with PWA_EINVAL (and a message) before it touches the
device, so these run without a GPU."""
import ctypes

import numpy as np
import pytest

from paper_2403_09225_b300 import binding as B


@pytest.fixture(scope="module")
def lib():
    return B.load_library()


FAKE = ctypes.c_void_p(16)  # never dereferenced: the calls refuse their sizes first


@pytest.mark.parametrize("args", [
    dict(in_=63, hidden=128, layers=1, out=4, max_batch=128),     # in % 64
    dict(in_=64, hidden=100, layers=1, out=4, max_batch=128),     # hidden % 128
    dict(in_=64, hidden=128, layers=0, out=4, max_batch=128),     # no hidden layer
    dict(in_=64, hidden=128, layers=1, out=0, max_batch=128),     # no output
    dict(in_=64, hidden=128, layers=1, out=4, max_batch=100),     # batch % 128
])
def test_mlp_create_refuses_bad_sizes(lib, args):
    h = ctypes.c_void_p()
    st = lib.pwa_mlp_create(args["in_"], args["hidden"], args["layers"], args["out"], args["max_batch"],
                            ctypes.c_ulonglong(1), None, None, None, ctypes.byref(h))
    assert st == B.PWA_EINVAL and not h.value
    assert lib.pwa_mlp_last_error(None)


@pytest.mark.parametrize("n,start,n_target,C", [(0, 0, 1, 0.0), (10, 10, 1, 0.0), (10, -1, 1, 0.0),
                                                (10, 0, -1, 0.0), (10, 0, 1, float("nan")), (1 << 31, 0, 1, 0.0)])
def test_accept_reject_refuses_bad_arguments(lib, n, start, n_target, C):
    n_out = ctypes.c_int(-7)
    st = lib.pwa_accept_reject(FAKE, n, C, ctypes.c_ulonglong(1), start, n_target, FAKE, ctypes.byref(n_out),
                               None, None)
    assert st == B.PWA_EINVAL and n_out.value == -7
    assert lib.pwa_last_generate_error()


def test_histogram_and_gather_refuse_bad_arguments(lib):
    assert lib.pwa_dalitz_histogram(FAKE, 10, FAKE, 5, 0, 0.0, 1.0, 0.0, 1.0, 1, FAKE, None) == B.PWA_EINVAL
    assert lib.pwa_dalitz_histogram(FAKE, 10, FAKE, 5, 2048, 0.0, 1.0, 0.0, 1.0, 1, FAKE, None) == B.PWA_EINVAL
    assert lib.pwa_dalitz_histogram(FAKE, 10, FAKE, 5, 8, 1.0, 1.0, 0.0, 1.0, 1, FAKE, None) == B.PWA_EINVAL
    assert lib.pwa_dalitz_histogram(FAKE, 10, None, 5, 8, 0.0, 1.0, 0.0, 1.0, 1, FAKE, None) == B.PWA_EINVAL
    assert lib.pwa_gather_events(FAKE, 10, FAKE, 0, FAKE, 5, FAKE, FAKE, None) == B.PWA_EINVAL
    assert lib.pwa_gather_events(FAKE, 10, FAKE, 8, FAKE, -1, FAKE, FAKE, None) == B.PWA_EINVAL


def _events(n, K, S, w=False):
    m2 = np.full((3, n), 1.0, np.float32)
    F = np.ones((n, K, S, 2), np.float32)
    keep = [m2, F]
    wp = None
    if w:
        wv = np.ones(n, np.float32)
        keep.append(wv)
        wp = wv.ctypes.data
    return B.pwa_events(n, m2.ctypes.data, wp or 0, F.ctypes.data, 0), keep


def _table(K, **over):
    arr = (B.pwa_resonance * K)()
    for k in range(K):
        arr[k] = B.pwa_resonance(0, 0, 1.0, 0.1, 1.0, 0.0, int(k == 0), 0, 0)
    for k, kw in over.items():
        r = arr[int(k)]
        for name, v in kw.items():
            setattr(r, name, v)
    return arr


@pytest.mark.parametrize("case", ["K0", "K33", "S5", "channel", "kind", "radius", "mc_weights", "nan_m2", "inf_mass"])
def test_variant_create_refuses_bad_input(lib, case):
    K, S = 3, 2
    data, k1 = _events(4, K if case not in ("K0", "K33") else 3, S)
    mc, k2 = _events(4, K, S, w=(case == "mc_weights"))
    tab = _table(3)
    shapes = (B.pwa_lineshape * 3)()
    for k in range(3):
        shapes[k] = B.pwa_lineshape(0, 0.14, 0.14, 0.0, 0.0, 3.0, 0.0)
    Kc, Sc = K, S
    if case == "K0":
        Kc = 0
    elif case == "K33":
        Kc = 33
    elif case == "S5":
        Sc = 5
    elif case == "channel":
        tab[1].channel = 3
    elif case == "kind":
        shapes[2].kind = 7
    elif case == "radius":
        shapes[1].kind = B.SHAPE_MASS_DEPENDENT
        shapes[1].radius = 0.0
    elif case == "nan_m2":
        k1[0][1, 2] = np.nan
    elif case == "inf_mass":
        tab[2].mass = float("inf")
    h = ctypes.c_void_p()
    st = lib.pwa_variant_create(ctypes.byref(h), ctypes.byref(data), ctypes.byref(mc), tab, shapes, Kc, Sc, 0, None)
    assert st == B.PWA_EINVAL, (case, st, lib.pwa_variant_last_error(None))
    assert not h.value and lib.pwa_variant_last_error(None)
