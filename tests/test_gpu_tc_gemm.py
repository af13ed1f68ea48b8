"""The split-TF32 tcgen05 GEMM of the fast-diagonalisation transforms
(igapw_tc_gemm) element by element against the FP64 product of the same FP32
operands: every combination of operand layout (unit stride along K, along
the rows, neither), pre-split operand, tile width, batch and ragged edges
(sizes that are not multiples of the 128 x bn x 32 tiles), K split over
several CTAs per tile (partials added by the tile's last CTA), and the
1032 x 1027 x 1032 shape of the 1024^2 Poisson transforms.

Bound per element: |D - A B^T| <= (2^-20 + K 2^-23) (|A| |B|^T), twice the
estimate: the split leaves each product with a relative error below 2^-21
(the dropped lo x lo term, at most 2^-22, and the split remainders, at most
2^-23 per operand), the FP32 accumulation adds at most K rounding errors of
2^-24.  Dropping one of the three products or mis-placing a K column gives
errors near 2^-11 of the terms and fails."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    from paper_1910_08535_gb300 import _build
    _build.build()


def _operand(rng, rows, K, layout, batch):
    """(batch, rows, K) float32 values stored with the given layout:
    'k' unit stride along K, 'm' unit stride along the rows, 'x' neither
    (a transposed view of a padded buffer, row stride not a multiple of 4)."""
    import torch
    v = rng.standard_normal((batch, rows, K)).astype(np.float32)
    if layout == 'k':
        t = torch.from_numpy(v).cuda()
    elif layout == 'm':
        t = torch.from_numpy(np.ascontiguousarray(v.transpose(0, 2, 1))).cuda().transpose(1, 2)
    else:
        buf = torch.zeros((batch, K, rows + 3), dtype=torch.float32, device='cuda')
        buf[:, :, :rows] = torch.from_numpy(np.ascontiguousarray(v.transpose(0, 2, 1))).cuda()
        t = buf[:, :, :rows].transpose(1, 2)
    return v, t


def _check(a, b, d):
    ref = np.einsum('bmk,bnk->bmn', a.astype(np.float64), b.astype(np.float64))
    bound = np.einsum('bmk,bnk->bmn', np.abs(a).astype(np.float64), np.abs(b).astype(np.float64))
    K = a.shape[2]
    err = np.abs(d.astype(np.float64) - ref)
    lim = (2.0 ** -20 + K * 2.0 ** -23) * bound
    worst = float(np.max(err / lim))
    assert worst <= 1.0, worst
    return worst


CASES = [(128, 64, 32, 1), (200, 150, 77, 1), (256, 96, 64, 3), (129, 257, 33, 2), (7, 5, 3, 1)]


@pytest.mark.parametrize('M,N,K,batch', CASES)
@pytest.mark.parametrize('la,lb', [('k', 'k'), ('m', 'm'), ('m', 'k'), ('x', 'x')])
@pytest.mark.parametrize('pre', [0, 1, 2])
def test_layouts_and_presplit(M, N, K, batch, la, lb, pre):
    import torch
    from paper_1910_08535_gb300 import igapw
    rng = np.random.Generator(np.random.PCG64(M * 7 + N + K + batch))
    a, ta = _operand(rng, M, K, la, batch)
    if pre == 2 or pre == 1:
        # a pre-split operand is one matrix shared by the batch
        if pre == 1:
            a = np.repeat(a[:1], batch, axis=0)
            ta = ta[0]
    b, tb = _operand(rng, N, K, lb, batch)
    if pre == 2:
        b = np.repeat(b[:1], batch, axis=0)
        tb = tb[0]
    if batch == 1 and pre == 0:
        ta, tb = ta[0], tb[0]
    d = igapw.tc_gemm(ta, tb, pre=pre)
    torch.cuda.synchronize()
    _check(a, b, d.cpu().numpy().reshape(batch, M, N))


@pytest.mark.parametrize('bn', [64, 96, 128])
@pytest.mark.parametrize('pre', [0, 1, 2])
@pytest.mark.parametrize('splits', [1, 3])
def test_tile_widths(bn, pre, splits):
    from paper_1910_08535_gb300 import igapw
    rng = np.random.Generator(np.random.PCG64(bn + pre))
    a, ta = _operand(rng, 300, 100, 'm', 1)
    b, tb = _operand(rng, 270, 100, 'k', 1)
    d = igapw.tc_gemm(ta[0], tb[0], pre=pre, bn=bn, splits=splits)
    _check(a, b, d.cpu().numpy()[None])


@pytest.mark.parametrize('splits', [2, 3, 4])
@pytest.mark.parametrize('pre,la,lb', [(0, 'k', 'm'), (1, 'm', 'k'), (2, 'm', 'm'), (1, 'x', 'x')])
def test_split_k(splits, pre, la, lb):
    """K = 200 (7 chunks, the last ragged) split into 2-4 ranges of chunks
    over a batch of 2 with ragged tiles in M and N; the same call twice gives
    bit-identical results (the partials are added in split order whichever
    CTA finishes last)."""
    import torch
    from paper_1910_08535_gb300 import igapw
    rng = np.random.Generator(np.random.PCG64(100 * splits + 10 * pre + len(la)))
    batch, M, N, K = 2, 300, 170, 200
    a, ta = _operand(rng, M, K, la, batch)
    b, tb = _operand(rng, N, K, lb, batch)
    if pre == 1:
        a = np.repeat(a[:1], batch, axis=0)
        ta = ta[0]
    if pre == 2:
        b = np.repeat(b[:1], batch, axis=0)
        tb = tb[0]
    d1 = igapw.tc_gemm(ta, tb, pre=pre, bn=64, splits=splits)
    d2 = igapw.tc_gemm(ta, tb, pre=pre, bn=64, splits=splits)
    torch.cuda.synchronize()
    assert torch.equal(d1, d2)
    _check(a, b, d1.cpu().numpy().reshape(batch, M, N))


def test_split_matches_unsplit_within_rounding():
    """Splitting K changes only the order of the FP32 additions of the chunk
    sums: the split and unsplit results agree to a few ulps of the terms."""
    from paper_1910_08535_gb300 import igapw
    rng = np.random.Generator(np.random.PCG64(77))
    a, ta = _operand(rng, 260, 1000, 'k', 1)
    b, tb = _operand(rng, 190, 1000, 'k', 1)
    d1 = igapw.tc_gemm(ta[0], tb[0], pre=1, bn=96, splits=1).cpu().numpy().astype(np.float64)
    d4 = igapw.tc_gemm(ta[0], tb[0], pre=1, bn=96, splits=4).cpu().numpy().astype(np.float64)
    bound = np.abs(a[0]).astype(np.float64) @ np.abs(b[0]).astype(np.float64).T
    assert np.max(np.abs(d1 - d4) / bound) < 64 * 2.0 ** -24
    _check(a, b, d4[None].astype(np.float32))


@pytest.mark.parametrize('pre,la,lb', [(1, 'm', 'k'), (2, 'm', 'm'), (0, 'k', 'k')])
@pytest.mark.parametrize('splits', [0, 1])
def test_poisson_transform_shape(pre, la, lb, splits):
    """1032 x 1027 x 1032: the x and y transforms of the 1024^2 p = 3 solve
    (the matrix operand pre-split, the data operand live), with the split of
    K the cost model picks for 99 tiles on the GPU's SMs and without."""
    from paper_1910_08535_gb300 import igapw
    rng = np.random.Generator(np.random.PCG64(11 + pre))
    a, ta = _operand(rng, 1032, 1032, la, 1)
    b, tb = _operand(rng, 1027, 1032, lb, 1)
    d = igapw.tc_gemm(ta[0], tb[0], pre=pre, splits=splits)
    _check(a, b, d.cpu().numpy()[None])


def test_rejects_bad_arguments():
    import torch
    from paper_1910_08535_gb300 import igapw
    x = torch.zeros((4, 4), dtype=torch.float32, device='cuda')
    with pytest.raises(igapw.IgapwError) as e:
        igapw.tc_gemm(x, x, bn=48)
    assert e.value.code == igapw.IGAPW_ERR_ARG
    with pytest.raises(igapw.IgapwError):
        igapw.tc_gemm(x, torch.zeros((4, 5), dtype=torch.float32, device='cuda'))
    y = torch.zeros((2, 4, 4), dtype=torch.float32, device='cuda')
    with pytest.raises(igapw.IgapwError) as e:
        igapw.tc_gemm(y, y, pre=1)   # pre-split operand with a batch stride
    assert e.value.code == igapw.IGAPW_ERR_ARG
    z = torch.zeros((4, 100), dtype=torch.float32, device='cuda')
    for splits in (-1, 5):   # outside 0 .. 4
        with pytest.raises(igapw.IgapwError) as e:
            igapw.tc_gemm(z, z, splits=splits)
        assert e.value.code == igapw.IGAPW_ERR_ARG
    with pytest.raises(igapw.IgapwError) as e:
        igapw.tc_gemm(x, x, splits=2)   # K = 4: one chunk of 32, nothing to split
    assert e.value.code == igapw.IGAPW_ERR_ARG
