"""Premises of the FP64-grade tensor-core squaring (GBE_PREC_FP64TC), checked on the CPU.

An Ozaki-type slicing (a published error-free splitting of matrix products into products
of short-mantissa pieces) carries an SP2 iterate x (spectrum in [0, 1], so |x_ij| <= 1) on
the 2^-50 grid as five fixed-point digits of 10 bits, x = t0 + 2^-10 t1 + 2^-20 t2 +
2^-30 t3 + 2^-40 t4 (digits rounded to nearest at each level), each exact in fp16, and
forms X^2 from fp16 products in four FP32 tensor-core accumulators.  On one squaring at
m = 256 (an SP2-like iterate: a random orthogonal basis, eigenvalues in [0, 1]):
  * the digits and their derived planes (u, v of t1 and the 2^-10-scaled copies) are exact
    in fp16 and rebuild x exactly;
  * grouping the 15 digit products by weight alone does not work: the weight-2^-20 group
    holds t1 t1, whose diagonal (a row's sum of squares, ~K/12 in units of 2^-20 times
    2^20) needs more than FP32's 24 bits, and one squaring is then off by > 1e-11;
  * the built grouping takes t1 t1 as u u + u v + v u + v v (u = t1 rounded to 2^-5) and
    moves u u into the 2^-10 accumulator (as u' u, u' = 2^-10 u): the three leading
    accumulators then stay below 16 in magnitude on their 2^-20 grid in every partial sum
    (so FP32 holds them exactly, whatever the order of the additions), and with the fourth
    accumulator rounded to FP32 one squaring is within 2e-14 of the exact product (a
    long-double reference), nearly all of it the dropped 2^-50 level: adding that level
    back leaves < 1e-15.  On the tensor cores the fourth accumulator is rounded once per
    MMA instead of once, which adds an error of the same order (measured: the GPU parity
    tests).
"""
import numpy as np
import pytest

M = 256


@pytest.fixture(scope="module")
def it():
    rng = np.random.default_rng(0)
    V, _ = np.linalg.qr(rng.normal(size=(M, M)))
    X = (V * rng.uniform(0.0, 1.0, M)) @ V.T
    X = np.rint(X * 2.0 ** 50) / 2.0 ** 50
    # digits by rounding to nearest at 2^-10, 2^-20, 2^-30, 2^-40 of the integer x 2^50
    Vi = np.rint(X * 2.0 ** 50).astype(np.int64)
    k = []
    rest = Vi
    for sh in (40, 30, 20, 10):
        q = (rest + (1 << (sh - 1))) >> sh
        k.append(q)
        rest = rest - (q << sh)
    k.append(rest)
    t = [q.astype(np.float64) * 2.0 ** -10 for q in k]
    ku = (k[1] + 16) >> 5
    u = ku * 2.0 ** -5
    v = (k[1] - 32 * ku) * 2.0 ** -10
    return dict(X=X, t=t, u=u, v=v)


def f16_exact(a):
    return np.array_equal(a.astype(np.float16).astype(np.float64), a)


def test_digit_planes_are_exact(it):
    t, u, v = it["t"], it["u"], it["v"]
    rebuilt = t[0] + t[1] * 2.0 ** -10 + t[2] * 2.0 ** -20 + t[3] * 2.0 ** -30 + t[4] * 2.0 ** -40
    assert np.array_equal(rebuilt, it["X"])
    assert np.abs(t[0]).max() <= 1.0 and all(np.abs(p).max() <= 0.5 for p in t[1:])
    assert np.array_equal(u + v, t[1]) and np.abs(v).max() <= 2.0 ** -6
    for p in t + [u, v, u * 2.0 ** -10, t[2] * 2.0 ** -10, t[3] * 2.0 ** -10, t[4] * 2.0 ** -10]:
        assert f16_exact(p)


def test_grouping_by_weight_alone_is_not_exact(it):
    t = it["t"]
    g2 = [(0, 2), (1, 1), (2, 0)]
    exact = sum(t[i] @ t[j] for i, j in g2)
    f32 = np.zeros((M, M), np.float32)
    for i, j in g2:
        f32 = f32 + t[i].astype(np.float32) @ t[j].astype(np.float32)
    assert not np.array_equal(exact, f32.astype(np.float64))
    assert (t[1] ** 2).sum(axis=1).max() * 2.0 ** 20 > 2.0 ** 24     # the Gram diagonal, in units of 2^-20


def accumulators(it):
    t, u, v = it["t"], it["u"], it["v"]
    up, t2p, t3p, t4p = u * 2.0 ** -10, t[2] * 2.0 ** -10, t[3] * 2.0 ** -10, t[4] * 2.0 ** -10
    return [[(t[0], t[0])],
            [(t[0], t[1]), (t[1], t[0]), (up, u)],
            [(t[0], t[2]), (t[2], t[0]), (u, v), (v, u), (v, v)],
            [(t[0], t[3]), (t[3], t[0]), (t[1], t[2]), (t[2], t[1]), (t[0], t4p), (t4p, t[0]), (t[1], t3p),
             (t3p, t[1]), (t[2], t2p)]]


def test_leading_accumulators_are_exact_in_fp32(it):
    for acc in accumulators(it)[:3]:
        # every partial sum of every product, in any order, is bounded by sum |a||b|
        bound = sum(np.abs(a) @ np.abs(b) for a, b in acc)
        assert bound.max() < 16.0
        exact = sum(a @ b for a, b in acc)
        f32 = np.zeros((M, M), np.float32)
        for a, b in acc:
            f32 = f32 + a.astype(np.float32) @ b.astype(np.float32)
        assert np.array_equal(exact, f32.astype(np.float64))
        assert np.array_equal(exact * 2.0 ** 20, np.rint(exact * 2.0 ** 20))   # on the 2^-20 grid


def test_one_squaring_is_fp64_grade(it):
    A = [sum(a @ b for a, b in acc) for acc in accumulators(it)]
    A[3] = A[3].astype(np.float32).astype(np.float64)
    S = A[0] + A[1] * 2.0 ** -10 + A[2] * 2.0 ** -20 + A[3] * 2.0 ** -30
    Xl = it["X"].astype(np.longdouble)
    ref = Xl @ Xl
    err = float(np.abs(S - ref).max())
    assert err < 2e-14, err
    # the dropped 2^-50 level is the remainder: adding it back leaves the FP64 sums' rounding
    t = it["t"]
    l5 = (t[1] @ t[4] + t[4] @ t[1] + t[2] @ t[3] + t[3] @ t[2]) * 2.0 ** -50
    assert float(np.abs(S + l5 - ref).max()) < 1e-15
