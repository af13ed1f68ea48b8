"""The error model behind the tensor-core GEMM's element-wise tolerance
(tests/test_gpu_tc_gemm.py), checked on the CPU with the same split in numpy:
x_hi = x rounded to TF32 (10 fraction bits, ties away from zero),
x_lo = (x - x_hi) in FP32 rounded to TF32, D = A_hi B_hi^T + A_hi B_lo^T +
A_lo B_hi^T summed exactly (FP64; TF32 x TF32 products are exact there).

- the split: |x_lo| <= 2^-11 |x| and |x - x_hi - x_lo| <= 2^-23 |x|;
- the three products leave at most 2^-21 of |A| |B|^T per element (the
  dropped lo x lo term and the remainders), so the GPU test's bound
  (2^-20 + K 2^-23) |A| |B|^T keeps room for K FP32 roundings of 2^-24;
- dropping any one of the three products, or shifting a K index, breaks that
  bound on random data: the tolerance catches each of these mistakes."""
import numpy as np
import pytest


def round_tf32(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def split(x):
    x = np.asarray(x, dtype=np.float32)
    hi = round_tf32(x)
    lo = round_tf32((x - hi).astype(np.float32))
    return hi, lo


def _operands(seed, M=70, N=50, K=300):
    rng = np.random.default_rng(seed)
    scale = np.exp(rng.uniform(-8, 8, size=(M, K)))   # wide dynamic range
    a = (rng.standard_normal((M, K)) * scale).astype(np.float32)
    b = rng.standard_normal((N, K)).astype(np.float32)
    return a, b


def test_split_parts():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-30, 30, 200000))).astype(np.float32)
    hi, lo = split(x)
    x64, hi64, lo64 = (v.astype(np.float64) for v in (x, hi, lo))
    assert np.all(np.abs(lo64) <= 2.0 ** -11 * np.abs(x64))
    assert np.all(np.abs(x64 - hi64 - lo64) <= 2.0 ** -23 * np.abs(x64))
    # both parts are TF32 values: 13 low mantissa bits clear
    assert np.all((hi.view(np.uint32) & 0x1FFF) == 0) and np.all((lo.view(np.uint32) & 0x1FFF) == 0)


def _three_products(a, b, drop=None, shift=False):
    ah, al = (v.astype(np.float64) for v in split(a))
    bh, bl = (v.astype(np.float64) for v in split(b))
    if shift:
        bh, bl = np.roll(bh, 1, axis=1), np.roll(bl, 1, axis=1)
    terms = {'hh': ah @ bh.T, 'hl': ah @ bl.T, 'lh': al @ bh.T}
    return sum(v for k, v in terms.items() if k != drop)


@pytest.mark.parametrize('seed', [0, 1, 2])
def test_three_products_within_2_pow_minus_21(seed):
    a, b = _operands(seed)
    ref = a.astype(np.float64) @ b.astype(np.float64).T
    bound = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64).T
    err = np.abs(_three_products(a, b) - ref)
    assert np.max(err / bound) <= 2.0 ** -21
    # with K FP32 roundings on top, still inside the GPU test's bound
    K = a.shape[1]
    assert np.max(err / bound) + K * 2.0 ** -24 <= 2.0 ** -20 + K * 2.0 ** -23


@pytest.mark.parametrize('mistake', ['hh', 'hl', 'lh', 'shift'])
def test_tolerance_catches_mistakes(mistake):
    a, b = _operands(5)
    ref = a.astype(np.float64) @ b.astype(np.float64).T
    bound = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64).T
    K = a.shape[1]
    lim = (2.0 ** -20 + K * 2.0 ** -23) * bound
    if mistake == 'shift':
        got = _three_products(a, b, shift=True)
    else:
        got = _three_products(a, b, drop=mistake)
    assert np.max(np.abs(got - ref) / lim) > 1.0
