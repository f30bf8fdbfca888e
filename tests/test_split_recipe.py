"""The arithmetic premises of the tensor-core squaring's split recipes, checked on the CPU
with IEEE round-to-nearest conversions (numpy float16/float32, torch bfloat16).

FP16X6: x = s0 + 2^-11 (s1 + s2), s0 = x on the fixed-point grid 2^-10, t = (x - s0) 2^11,
s1 = fp16(t), s2 = fp16(t - s1), plus s1s = fp16(x - s0); X^2 is taken as
s0 s0^T + 2^-11 (s0 s1^T + s1 s0^T + s1 s1s^T + s0 s2^T + s2 s0^T) with two FP32
accumulators.  The premises the GPU path's tolerance rests on:
  * an SP2 iterate has its spectrum in [0, 1], so |x_ij| <= 1 and s0 is exact in fp16;
  * the split represents x to about 2^-35;
  * the leading product s0 s0^T is exact in FP32 whatever the summation order (products
    are multiples of 2^-20 and every partial sum is bounded by the row norms, <= 1);
  * the six products give one squaring to ~1e-9 at m = 256, and each of the five
    correction products is needed (dropping any one costs at least 50x).
BF16X3 (hi hi + hi lo + lo hi, one FP32 accumulator) lands near 1e-5 per squaring, which
is why it cannot carry a 1e-6 bound over an SP2 run.
"""
import numpy as np
import pytest

M = 256


@pytest.fixture(scope="module")
def X():
    """A symmetric matrix with spectrum in [0, 1], like every SP2 iterate."""
    rng = np.random.default_rng(0)
    V, _ = np.linalg.qr(rng.normal(size=(M, M)))
    return (V * rng.uniform(0.0, 1.0, M)) @ V.T


def fp16(a):
    return np.asarray(a, dtype=np.float64).astype(np.float16).astype(np.float64)


def f32(a):
    return np.asarray(a, dtype=np.float32)


def split(X):
    s0 = np.round(X * 1024.0) / 1024.0
    t = (X - s0) * 2048.0
    s1 = fp16(t)
    s2 = fp16(t - s1)
    s1s = fp16(X - s0)
    return s0, s1, s2, s1s


def test_split_represents_x(X):
    assert np.abs(X).max() <= 1.0
    s0, s1, s2, _ = split(X)
    np.testing.assert_array_equal(fp16(s0), s0)              # exact in fp16
    assert np.abs(X - s0).max() <= 2.0 ** -11
    assert np.abs(X - s0 - (s1 + s2) / 2048.0).max() <= 2.0 ** -34


def test_leading_product_is_exact_in_fp32(X):
    s0, *_ = split(X)
    exact = s0 @ s0.T                                        # multiples of 2^-20: exact in FP64
    lead = f32(s0) @ f32(s0).T
    np.testing.assert_array_equal(lead.astype(np.float64), exact)
    # any summation order: a sequential FP32 sum over k gives the same bits
    i, j = 3, 17
    acc = np.float32(0.0)
    for k in range(M):
        acc = np.float32(acc + np.float32(s0[i, k]) * np.float32(s0[j, k]))
    assert float(acc) == exact[i, j]


def six_products(s0, s1, s2, s1s, drop=None):
    terms = {"s0s1": (s0, s1), "s1s0": (s1, s0), "s1s1s": (s1, s1s), "s0s2": (s0, s2), "s2s0": (s2, s0)}
    acc1 = np.zeros((M, M), dtype=np.float32)
    for name, (a, b) in terms.items():
        if name != drop:
            acc1 = acc1 + f32(a) @ f32(b).T
    return (f32(s0) @ f32(s0).T).astype(np.float64) + acc1.astype(np.float64) / 2048.0, terms


def test_six_products_give_one_squaring(X):
    parts = split(X)
    ref = X @ X
    P, terms = six_products(*parts)
    err = np.abs(P - ref).max()
    assert err <= 5e-9, err
    for name in terms:
        Pd, _ = six_products(*parts, drop=name)
        assert np.abs(Pd - ref).max() >= 50 * err, name


def test_bf16x3_one_squaring():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    V, _ = np.linalg.qr(rng.normal(size=(M, M)))
    X = (V * rng.uniform(0.0, 1.0, M)) @ V.T
    xt = torch.from_numpy(X)
    hi = xt.to(torch.bfloat16).float()
    lo = (xt - hi.double()).to(torch.bfloat16).float()
    P = (hi @ hi.T + hi @ lo.T + lo @ hi.T).double().numpy()
    err = np.abs(P - X @ X).max()
    assert 1e-6 < err < 2.0 ** -14, err
