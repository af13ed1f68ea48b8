"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/igapw.h declares; the binding's constants match the header."""
import re

import pytest


@pytest.fixture(scope='module')
def lib():
    from paper_1910_08535_gb300 import _build, igapw
    _build.build()
    return igapw.load()


def test_exports_every_declared_symbol(lib):
    from paper_1910_08535_gb300 import igapw
    names = igapw.header_symbols()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(igapw._SIGS), set(names) ^ set(igapw._SIGS)


def test_constants_match_header():
    from paper_1910_08535_gb300 import igapw
    txt = open(igapw.HEADER).read()
    defs = dict((m[0], int(m[1])) for m in re.findall(r'#define\s+(IGAPW_\w+)\s+(-?\d+)', txt))
    for name, val in defs.items():
        if hasattr(igapw, name):
            assert getattr(igapw, name) == val, name
    for name in ('IGAPW_PWCONST', 'IGAPW_FP32_REFINE', 'IGAPW_OP_POISSON', 'IGAPW_ERR_SINGULAR'):
        assert name in defs and hasattr(igapw, name)


def test_desc_layout_matches_header():
    """igapw_desc is eleven fields (thirteen ints) in the header's order."""
    from paper_1910_08535_gb300 import igapw
    txt = open(igapw.HEADER).read()
    body = re.search(r'typedef struct \{(.*?)\} igapw_desc;', txt, re.S).group(1)
    fields = re.findall(r'int\s+(\w+)(?:\[(\d)\])?;', body)
    assert [f[0] for f in fields] == [f[0] for f in igapw.igapw_desc._fields_]
    import ctypes
    assert ctypes.sizeof(igapw.igapw_desc) == 13 * 4


def test_missing_library_fails_loudly(tmp_path):
    from paper_1910_08535_gb300 import igapw
    saved = igapw._lib
    try:
        igapw._lib = None
        with pytest.raises(RuntimeError, match='not built'):
            igapw.load(str(tmp_path / 'nope.so'))
    finally:
        igapw._lib = saved


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor on a machine without a GPU."""

    def __init__(self, dtype, numel, contiguous=True):
        self.is_cuda, self.dtype, self._n, self._c = True, dtype, numel, contiguous

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c


def test_helper_argument_checks():
    """The Context helpers reject, with IGAPW_ERR_ARG and before any library
    call, tensors the kernels would address on the host, reinterpret or run
    past the end of; raw pointers pass unchecked."""
    import torch
    from paper_1910_08535_gb300 import igapw
    chk = igapw._check_tensor
    chk(_FakeDeviceTensor(torch.float32, 24), 'u', torch.float32, 24)
    chk(12345, 'u', torch.float32, 24)
    cases = [(torch.zeros(24, dtype=torch.float32), 'not on a CUDA device'),
             (_FakeDeviceTensor(torch.float64, 24), 'dtype'),
             (_FakeDeviceTensor(torch.float32, 24, contiguous=False), 'not contiguous'),
             (_FakeDeviceTensor(torch.float32, 23), '23 elements, expected 24')]
    for t, msg in cases:
        with pytest.raises(igapw.IgapwError, match=msg) as ei:
            chk(t, 'u', torch.float32, 24)
        assert ei.value.code == igapw.IGAPW_ERR_ARG


def test_batch_params_shape_checked(monkeypatch):
    """Batch.source_sine passes exactly instances x 3 doubles to the library
    (which reads that many from the host pointer); other shapes are rejected."""
    import numpy as np
    from paper_1910_08535_gb300 import igapw
    seen = []
    monkeypatch.setattr(igapw, 'igapw_batch_source_sine', lambda h, p: seen.append(p.shape))
    b = object.__new__(igapw.Batch)
    b.shapes, b.handle = [(8, 8, 2)] * 4, None
    b.source_sine(np.ones((4, 3)))
    for bad in (np.ones((3, 3)), np.ones(12), np.ones((4, 2))):
        with pytest.raises(igapw.IgapwError, match='source_sine'):
            b.source_sine(bad)
    assert seen == [(4, 3)]


def _bare_context(precision, ntot=24):
    from paper_1910_08535_gb300 import igapw
    c = object.__new__(igapw.Context)
    c.precision, c.ntot, c.ctx = precision, ntot, None
    return c


def test_step_host_checks_host_buffers(monkeypatch):
    """Context.step_host hands the library a host pointer only for a writable,
    C-contiguous host buffer of the context's dtype and size."""
    import numpy as np
    import torch
    from paper_1910_08535_gb300 import igapw
    seen = []
    monkeypatch.setattr(igapw, 'igapw_step_host', lambda ctx, dt, n, ptr: seen.append(ptr))
    c = _bare_context('fp32r')
    a = np.zeros((2, 24), dtype=np.float32)
    c.step_host(a, 1e-3, 2)
    t = torch.zeros(48, dtype=torch.float32)
    c.step_host(t, 1e-3, 2)
    assert seen == [a.ctypes.data, t.data_ptr()]
    bad = [np.zeros(48), np.zeros(47, dtype=np.float32), np.zeros((24, 4), dtype=np.float32)[:, ::2],
           _FakeDeviceTensor(torch.float32, 48), 12345]
    ro = np.zeros(48, dtype=np.float32)
    ro.flags.writeable = False
    bad.append(ro)
    for b in bad:
        with pytest.raises(igapw.IgapwError, match='step_host'):
            c.step_host(b, 1e-3, 2)
    assert len(seen) == 2
    c64 = _bare_context('fp64')
    c64.step_host(np.zeros(24), 1e-3, 1)
    with pytest.raises(igapw.IgapwError):
        c64.step_host(np.zeros(24, dtype=np.float32), 1e-3, 1)


def test_context_and_batch_close_on_exit(monkeypatch):
    from paper_1910_08535_gb300 import igapw
    closed = []
    monkeypatch.setattr(igapw, 'igapw_destroy', lambda ctx: closed.append('ctx'))
    monkeypatch.setattr(igapw, 'igapw_batch_destroy', lambda h: closed.append('batch'))
    c = _bare_context('fp64')
    c.ctx = object()
    with c as same:
        assert same is c
    assert c.ctx is None
    b = object.__new__(igapw.Batch)
    b.handle = object()
    with b:
        pass
    assert b.handle is None and closed == ['ctx', 'batch']
