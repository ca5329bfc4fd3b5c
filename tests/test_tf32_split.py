"""The rounding model of the FP32 form's tensor-core products (three TF32
products of exact hi/lo splits, tests/parity.py U_TF32_PAIR), pinned on
emulated TF32 arithmetic in numpy: a TF32 operand is the FP32 word with its
low 13 mantissa bits cleared (10 explicit bits), the products are exact in
FP64.  These are statements about the arithmetic, independent of the GPU."""

import numpy as np

from tests.parity import U_TF32_PAIR

MASK = np.uint32(0xFFFFE000)


def tf32(v):
    """The TF32 value an MMA reads from FP32 words (truncation)."""
    return (np.asarray(v, np.float32).view(np.uint32) & MASK).view(np.float32)


def split(v):
    v = np.asarray(v, np.float32)
    h = tf32(v)
    return h, (v - h)  # FP32 subtraction


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    mag = np.exp2(rng.integers(-20, 20, n)).astype(np.float32)
    return (rng.standard_normal(n).astype(np.float32) * mag).astype(np.float32)


def test_split_is_exact():
    x = _samples(200000, 1)
    h, l = split(x)
    # v = v_h + v_l holds exactly (checked in FP64) and v_h is a TF32 value
    assert np.array_equal(h.astype(np.float64) + l.astype(np.float64), x.astype(np.float64))
    assert np.array_equal(tf32(h), h)
    # |v_l| < 2^-10 |v| (below one TF32 ulp of v)
    nz = x != 0
    assert np.all(np.abs(l[nz]).astype(np.float64) < 2.0 ** -10 * np.abs(x[nz]).astype(np.float64))


def test_three_product_error_terms():
    x = _samples(200000, 2)
    w = _samples(200000, 3)
    xh, xl = split(x)
    wh, wl = split(w)
    f = lambda a: tf32(a).astype(np.float64)
    approx = f(xh) * f(wh) + f(xh) * f(wl) + f(xl) * f(wh)
    exact = x.astype(np.float64) * w.astype(np.float64)
    nz = exact != 0
    rel = np.abs(approx - exact)[nz] / np.abs(exact[nz])
    # each of the three error terms is below 2^-20 |x w|
    assert rel.max() < 3 * 2.0 ** -20
    # the unit of the model is above the worst case, and far above the RMS
    assert U_TF32_PAIR >= 3 * 2.0 ** -20
    assert np.sqrt(np.mean(rel ** 2)) < 0.25 * U_TF32_PAIR
    # dropping a term breaks the bound: X_l W_h is needed (its size ~2^-11)
    partial = f(xh) * f(wh) + f(xh) * f(wl)
    assert (np.abs(partial - exact)[nz] / np.abs(exact[nz])).max() > 2.0 ** -14


def test_dot_products_within_the_model():
    rng = np.random.default_rng(4)
    K = 1024
    X = rng.standard_normal((64, K)).astype(np.float32)
    W = rng.standard_normal((K, 16)).astype(np.float32)
    Xh, Xl = split(X)
    Wh, Wl = split(W)
    f = lambda a: tf32(a).astype(np.float64)
    approx = f(Xh) @ f(Wh) + f(Xh) @ f(Wl) + f(Xl) @ f(Wh)
    exact = X.astype(np.float64) @ W.astype(np.float64)
    # Frobenius-relative error against the model's per-stage bound
    # unit * sqrt(K) * ||X|| ||W|| / ||X W|| (independent roundings)
    err = np.linalg.norm(approx - exact)
    bound = U_TF32_PAIR * np.sqrt(K) * np.linalg.norm(np.abs(X).astype(np.float64) @ np.abs(W).astype(np.float64))
    assert err <= bound
    assert err / np.linalg.norm(exact) < 1e-5
