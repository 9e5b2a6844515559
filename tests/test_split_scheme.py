"""The split-precision scheme of the tensor-core Gram matrices (the Hessian
pass), emulated in numpy: each FP32 value x = hi + lo with hi the nearest
BF16 of x and lo the nearest BF16 of x - hi, and per 16 rows the two
products hi^T hi + hi^T (2 lo), symmetrised afterwards.  The symmetric part
equals hi^T hi + hi^T lo + lo^T hi, which misses only lo^T lo and the
rounding of lo: the Gram matrix comes out within a few 2^-16 of |X|^T |X|
of the FP64 one, far inside the 1e-4 Hessian bar.  Dropping the factor 2 or
one product breaks the bound (checked), so the test pins the scheme's
algebra, independently of the kernels."""
import numpy as np


def bf16(x: np.ndarray) -> np.ndarray:
    """Nearest BF16 (ties to even) of FP32 values, returned as FP32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split(x: np.ndarray):
    x = x.astype(np.float32)
    hi = bf16(x)
    lo = bf16((x - hi).astype(np.float32))
    return hi, lo


def gram_scheme(X: np.ndarray, lo_factor: float = 2.0, products: int = 2) -> np.ndarray:
    hi, lo = split(X)
    h, l = hi.astype(np.float64), lo.astype(np.float64)
    D = h.T @ h
    if products >= 2:
        D = D + h.T @ (lo_factor * l)
    if products >= 3:
        D = D + l.T @ h
    return 0.5 * (D + D.T) if products == 2 else D


def scaled_error(D: np.ndarray, X: np.ndarray) -> float:
    ref = X.astype(np.float64).T @ X.astype(np.float64)
    mag = np.abs(X.astype(np.float64)).T @ np.abs(X.astype(np.float64))
    return float(np.max(np.abs(D - ref) / mag))


def test_bf16_rounding_is_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.0e-20, 1e30], dtype=np.float32)
    y = bf16(x)
    assert y[0] == 1.0
    assert y[1] == 1.0  # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even 1
    assert y[2] == np.float32(1.0 + 2 ** -7)
    assert y[3] == -2.5
    assert abs(y[4] - x[4]) <= abs(x[4]) * 2 ** -8 and abs(y[5] - x[5]) <= abs(x[5]) * 2 ** -8


def test_split_captures_sixteen_bits():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(10000) * np.exp(rng.uniform(-20, 20, 10000))).astype(np.float32)
    hi, lo = split(x)
    rel = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64)) / np.abs(x)
    assert rel.max() <= 2.0 ** -16


def test_two_symmetrised_products_reach_the_gram_matrix():
    rng = np.random.default_rng(11)
    # rows of wildly different scale (peaked line shapes) and mixed signs
    X = (rng.standard_normal((4096, 40)) * np.exp(rng.uniform(-6, 6, (4096, 1)))).astype(np.float32)
    err = scaled_error(gram_scheme(X), X)
    assert err <= 4 * 2.0 ** -16, err
    # the same result as the three-product form it replaces (hi^T hi + hi^T lo + lo^T hi)
    three = gram_scheme(X, lo_factor=1.0, products=3)
    assert abs(err - scaled_error(three, X)) <= 2.0 ** -30
    mag = np.abs(X.astype(np.float64)).T @ np.abs(X.astype(np.float64))
    assert np.max(np.abs(gram_scheme(X) - three) / mag) <= 2.0 ** -40


def test_the_scheme_fails_without_its_pieces():
    rng = np.random.default_rng(12)
    X = (rng.standard_normal((2048, 24)) * np.exp(rng.uniform(-4, 4, (2048, 1)))).astype(np.float32)
    good = scaled_error(gram_scheme(X), X)
    assert scaled_error(gram_scheme(X, lo_factor=1.0), X) > 8 * good  # lo not doubled: half the correction
    assert scaled_error(gram_scheme(X, products=1), X) > 8 * good     # hi^T hi alone: BF16 accuracy
