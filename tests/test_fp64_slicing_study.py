"""Why FP64-grade squarings on the tensor cores are not built (CPU study).

An Ozaki-type slicing (a published error-free splitting of matrix products) would carry an
SP2 iterate x (spectrum in [0, 1], on the 2^-50 grid) as five fixed-point digit planes of
10 bits, x = sum_i d_i 2^-10(i+1), each plane exact in fp16, and form X^2 from the 15 digit
products grouped by weight 2^-10k (k = 0..4), one FP32 tensor-core accumulator per group.
The study, on one squaring at m = 256:
  * the digits reconstruct x exactly and every plane is exact in fp16;
  * with exact accumulation the 15 products give X^2 to ~1e-14 (FP64-grade);
  * with FP32 accumulators the k = 2 group is not exact: it holds the Gram diagonal
    sum_k s1_ik^2, which in units of 2^-20 needs more than FP32's 24 bits, and one
    squaring is off by ~5e-11 -- too much for a 1e-10 bound after an SP2 run amplifies it.
Exactness would need that group split further (more products and planes), which is the
cost estimate behind leaving the FP64 path on the FP64 pipe.
"""
import numpy as np
import pytest

M = 256
GROUPS = [[(0, 0)], [(0, 1), (1, 0)], [(0, 2), (1, 1), (2, 0)], [(0, 3), (1, 2), (2, 1), (3, 0)],
          [(0, 4), (1, 3), (2, 2), (3, 1), (4, 0)]]


@pytest.fixture(scope="module")
def planes():
    rng = np.random.default_rng(0)
    V, _ = np.linalg.qr(rng.normal(size=(M, M)))
    X = (V * rng.uniform(0.0, 1.0, M)) @ V.T
    X = np.rint(X * 2.0 ** 50) / 2.0 ** 50
    s, r = [], X.copy()
    for i in range(5):
        sc = 2.0 ** (10 * (i + 1))
        d = np.rint(r * sc)
        r = r - d / sc
        s.append(d * 2.0 ** -10)
    return X, s, r


def group(s, k, f32):
    dt = np.float32 if f32 else np.float64
    acc = np.zeros((M, M), dtype=dt)
    for i, j in GROUPS[k]:
        acc = acc + s[i].astype(dt) @ s[j].astype(dt).T
    return acc.astype(np.float64)


def test_digit_planes_are_exact(planes):
    X, s, r = planes
    assert np.all(r == 0.0)
    for p in s:
        np.testing.assert_array_equal(p.astype(np.float16).astype(np.float64), p)
        assert np.abs(p).max() <= 1.0


def test_exact_accumulation_is_fp64_grade(planes):
    X, s, _ = planes
    S = sum(2.0 ** (-10 * k) * group(s, k, False) for k in range(5))
    assert np.abs(S - X @ X).max() < 1e-13


def test_fp32_accumulation_is_not(planes):
    X, s, _ = planes
    exact = [group(s, k, False) for k in range(5)]
    f32 = [group(s, k, True) for k in range(5)]
    assert np.array_equal(exact[0], f32[0]) and np.array_equal(exact[1], f32[1])
    assert not np.array_equal(exact[2], f32[2])
    gram = (s[1] ** 2).sum(axis=1).max() * 2.0 ** 20      # in units of 2^-20
    assert gram > 2.0 ** 24
    S = sum(2.0 ** (-10 * k) * f32[k] for k in range(5))
    assert np.abs(S - X @ X).max() > 1e-11
