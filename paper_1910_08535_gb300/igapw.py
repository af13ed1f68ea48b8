"""ctypes binding of libigapw (include/igapw.h): the same call names, argument
marshalling only.  Every step of the computation runs in the library's CUDA
kernels; nothing here computes on the host or falls back to a CPU path.

``Context`` wraps a context handle for torch users: it allocates coefficient
tensors of the layout the library expects and passes their device pointers and
torch's current CUDA stream.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, 'lib', 'libigapw.so')
HEADER = os.path.join(os.path.dirname(HERE), 'include', 'igapw.h')

# constants mirrored from include/igapw.h (checked against it by the tests)
IGAPW_OK, IGAPW_ERR_ARG, IGAPW_ERR_SINGULAR, IGAPW_ERR_OOM = 0, -1, -2, -3
IGAPW_ERR_CUDA, IGAPW_ERR_DEVICE_STATUS, IGAPW_ERR_TIMEOUT = -4, -5, -6
IGAPW_GALERKIN, IGAPW_PWCONST, IGAPW_REFINED = 0, 1, 2
IGAPW_BC_NONE, IGAPW_BC_DIRICHLET0 = 0, 1
IGAPW_FP64, IGAPW_FP32_REFINE = 0, 1
IGAPW_OP_MASS, IGAPW_OP_LAPLACE, IGAPW_OP_HEAT, IGAPW_OP_POISSON = 0, 1, 2, 3
IGAPW_FLAG_FP64_RESIDUAL, IGAPW_FLAG_STEP_RHS_SOLVE, IGAPW_FLAG_FDM_BF16X9, IGAPW_FLAG_FDM_CUBLAS = 1, 2, 4, 8

TESTS = {'galerkin': IGAPW_GALERKIN, 'pw': IGAPW_PWCONST, 'refined': IGAPW_REFINED}
BCS = {'none': IGAPW_BC_NONE, 'dirichlet0': IGAPW_BC_DIRICHLET0}
PRECISIONS = {'fp64': IGAPW_FP64, 'fp32r': IGAPW_FP32_REFINE}
OPS = {'mass': IGAPW_OP_MASS, 'laplace': IGAPW_OP_LAPLACE, 'heat': IGAPW_OP_HEAT, 'poisson': IGAPW_OP_POISSON}


class IgapwError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f'igapw error {code}: {msg}')
        self.code = code


class igapw_desc(ctypes.Structure):
    _fields_ = [('dim', ctypes.c_int), ('n_elem', ctypes.c_int * 3), ('degree', ctypes.c_int),
                ('nq', ctypes.c_int), ('test', ctypes.c_int), ('bc', ctypes.c_int),
                ('precision', ctypes.c_int), ('op', ctypes.c_int), ('flags', ctypes.c_int),
                ('neumann_axes', ctypes.c_int), ('refine', ctypes.c_int)]


_VP, _I, _D, _LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
_SIGS = {
    'igapw_create': (_I, [ctypes.POINTER(_VP), ctypes.POINTER(igapw_desc), _VP]),
    'igapw_set_knots': (_I, [_VP, _I, ctypes.POINTER(_D), _I]),
    'igapw_quad_points': (_I, [_VP, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    'igapw_basis_table': (_I, [_VP, _I, ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    'igapw_rhs_source': (_I, [_VP, _VP, _VP]),
    'igapw_rhs_source_noalloc': (_I, [_VP, _VP, _VP]),
    'igapw_rhs_source_sine': (_I, [_VP, _D, ctypes.POINTER(_D), _VP]),
    'igapw_rhs_neumann': (_I, [_VP, _I, _I, _VP, _VP]),
    'igapw_apply': (_I, [_VP, _I, _D, _VP, _VP]),
    'igapw_assemble_1d': (_I, [_VP, _I, _I, ctypes.POINTER(_D)]),
    'igapw_solve': (_I, [_VP, _VP, _VP]),
    'igapw_step': (_I, [_VP, _D, _I, _VP]),
    'igapw_step_host': (_I, [_VP, _D, _I, _VP]),
    'igapw_set_step_shape': (_I, [_VP, _I, _I, _I]),
    'igapw_get_step_shape': (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    'igapw_sync_status': (_I, [_VP]),
    'igapw_last_error': (ctypes.c_char_p, [_VP]),
    'igapw_size': (ctypes.c_longlong, [_VP, ctypes.POINTER(_I)]),
    'igapw_destroy': (_I, [_VP]),
    'igapw_batch_create': (_I, [ctypes.POINTER(_VP), ctypes.POINTER(igapw_desc), _I, _VP]),
    'igapw_batch_source_sine': (_I, [_VP, ctypes.POINTER(_D)]),
    'igapw_batch_solve': (_I, [_VP]),
    'igapw_tc_gemm': (_I, [_I, _I, _I, _I, _VP, _LL, _LL, _LL, _VP, _LL, _LL, _LL, _VP, _LL, _LL, _LL, _I, _I, _I, _VP]),
    'igapw_batch_sync_status': (_I, [_VP]),
    'igapw_batch_tensor': (_I, [_VP, _I, _I, ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_longlong)]),
    'igapw_batch_info': (_I, [_VP, ctypes.POINTER(_I)]),
    'igapw_batch_last_error': (ctypes.c_char_p, [_VP]),
    'igapw_batch_destroy': (_I, [_VP]),
}

_lib = None


def header_symbols(path=HEADER):
    """Names of the functions declared in include/igapw.h."""
    txt = open(path).read()
    return sorted(set(re.findall(r'^\s*(?:int|long long|const char\*)\s+(igapw_\w+)\s*\(', txt, re.M)))


def load(path=LIB_PATH):
    """Load libigapw.so (no CUDA context is created).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f'libigapw.so not built at {path}: run paper_1910_08535_gb300/_build.py '
                           '(there is no CPU fallback)')
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc, ctx=None):
    if rc != IGAPW_OK:
        msg = load().igapw_last_error(ctx)
        raise IgapwError(rc, msg.decode() if msg else '')


def _check_tensor(t, what, dtype, numel):
    """Argument check of the Context helpers: a torch tensor that the library
    would address on the host, reinterpret or run past the end of (not on a
    CUDA device, another dtype, not contiguous, another element count) raises
    IgapwError(IGAPW_ERR_ARG) before the call.  Raw pointers (ints) are the
    caller's responsibility and pass unchecked."""
    if not hasattr(t, 'is_cuda'):
        return
    if not t.is_cuda:
        problem = 'not on a CUDA device'
    elif t.dtype != dtype:
        problem = f'dtype {t.dtype}, expected {dtype}'
    elif not t.is_contiguous():
        problem = 'not contiguous'
    elif t.numel() != numel:
        problem = f'{t.numel()} elements, expected {numel}'
    else:
        return
    raise IgapwError(IGAPW_ERR_ARG, f'{what}: {problem}')


def _dptr(a):
    return ctypes.cast(ctypes.c_void_p(a.data_ptr() if hasattr(a, 'data_ptr') else int(a)), ctypes.c_void_p)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, 'cuda_stream') else int(stream))


# ---- the C ABI, same names -------------------------------------------------

def igapw_create(desc, stream=None):
    ctx = ctypes.c_void_p()
    rc = load().igapw_create(ctypes.byref(ctx), ctypes.byref(desc), _stream_handle(stream))
    _check(rc, None)
    return ctx


def igapw_set_knots(ctx, axis, knots):
    import numpy as np
    k = np.ascontiguousarray(knots, dtype=np.float64)
    _check(load().igapw_set_knots(ctx, axis, k.ctypes.data_as(ctypes.POINTER(_D)), len(k)), ctx)


def igapw_quad_points(ctx, axis):
    import numpy as np
    cnt = _I()
    _check(load().igapw_quad_points(ctx, axis, None, None, ctypes.byref(cnt)), ctx)
    x = np.empty(cnt.value)
    w = np.empty(cnt.value)
    _check(load().igapw_quad_points(ctx, axis, x.ctypes.data_as(ctypes.POINTER(_D)),
                                    w.ctypes.data_as(ctypes.POINTER(_D)), ctypes.byref(cnt)), ctx)
    return x, w


def igapw_basis_table(ctx, axis, p):
    import numpy as np
    x, _ = igapw_quad_points(ctx, axis)
    vals = np.empty((len(x), p + 1, 3))
    first = np.empty(len(x), dtype=np.int32)
    _check(load().igapw_basis_table(ctx, axis, vals.ctypes.data_as(ctypes.POINTER(_D)),
                                    first.ctypes.data_as(ctypes.POINTER(_I))), ctx)
    return vals, first


def igapw_rhs_source(ctx, f, b):
    _check(load().igapw_rhs_source(ctx, _dptr(f), _dptr(b)), ctx)


def igapw_rhs_source_noalloc(ctx, f, b):
    """Same result as igapw_rhs_source, with the intermediates in the library's
    static device array instead of memory allocated on first use (for callers
    that cannot let the library allocate; see include/igapw.h)."""
    _check(load().igapw_rhs_source_noalloc(ctx, _dptr(f), _dptr(b)), ctx)


def igapw_rhs_source_sine(ctx, amp, k, b):
    arr = (_D * len(k))(*[float(x) for x in k])
    _check(load().igapw_rhs_source_sine(ctx, float(amp), arr, _dptr(b)), ctx)


def igapw_rhs_neumann(ctx, axis, side, g, b):
    _check(load().igapw_rhs_neumann(ctx, int(axis), int(side), _dptr(g), _dptr(b)), ctx)


def igapw_apply(ctx, op, dt, u, r):
    _check(load().igapw_apply(ctx, op, float(dt), _dptr(u), _dptr(r)), ctx)


def igapw_assemble_1d(ctx, axis, which, n):
    import numpy as np
    out = np.empty((n, n))
    _check(load().igapw_assemble_1d(ctx, axis, which, out.ctypes.data_as(ctypes.POINTER(_D))), ctx)
    return out


def igapw_solve(ctx, r, u):
    _check(load().igapw_solve(ctx, _dptr(r), _dptr(u)), ctx)


def igapw_step(ctx, dt, nsteps, u):
    _check(load().igapw_step(ctx, float(dt), int(nsteps), _dptr(u)), ctx)


def igapw_step_host(ctx, dt, nsteps, u_host):
    _check(load().igapw_step_host(ctx, float(dt), int(nsteps), _dptr(u_host)), ctx)


def igapw_set_step_shape(ctx, axis, kind, lines):
    _check(load().igapw_set_step_shape(ctx, int(axis), int(kind), int(lines)), ctx)


def igapw_get_step_shape(ctx, axis):
    kind, lines = ctypes.c_int(), ctypes.c_int()
    _check(load().igapw_get_step_shape(ctx, int(axis), ctypes.byref(kind), ctypes.byref(lines)), ctx)
    return kind.value, lines.value


def igapw_sync_status(ctx):
    _check(load().igapw_sync_status(ctx), ctx)


def igapw_last_error(ctx):
    return load().igapw_last_error(ctx).decode()


def igapw_size(ctx):
    dims = (_I * 3)()
    n = load().igapw_size(ctx, dims)
    return n, tuple(dims)


def igapw_destroy(ctx):
    _check(load().igapw_destroy(ctx), None)


def igapw_tc_gemm(M, N, K, batch, A, sA, bA, B, sB, bB, D, sD, bD, pre=0, bn=0, splits=0, stream=None):
    """The library's tensor-core transform GEMM on device pointers:
    D(m, n) = sum_k A(m, k) B(n, k) per batch entry; sA = (s_m, s_k),
    sB = (s_n, s_k), sD = (s_m, s_n) element strides.  Synchronous."""
    _check(load().igapw_tc_gemm(M, N, K, batch, A, sA[0], sA[1], bA, B, sB[0], sB[1], bB, D, sD[0], sD[1], bD, pre, bn,
                                splits, _stream_handle(stream)), None)


def tc_gemm(a, b, out=None, pre=0, bn=0, splits=0):
    """Torch convenience form: D = A @ B^T for CUDA float32 tensors A (M x K)
    and B (N x K) of any strides (or batched, (batch, M, K) and (batch, N, K),
    a pre-split operand shared by the batch as a 2D tensor).  bn: tile width
    (0: chosen); splits: K split over CTAs (0: chosen, 1: none, 2-4)."""
    import torch
    if a.dtype != torch.float32 or b.dtype != torch.float32 or not (a.is_cuda and b.is_cuda):
        raise IgapwError(IGAPW_ERR_ARG, 'tc_gemm: CUDA float32 tensors required')
    batched = a.dim() == 3 or b.dim() == 3
    batch = a.shape[0] if a.dim() == 3 else (b.shape[0] if b.dim() == 3 else 1)
    M, K = a.shape[-2], a.shape[-1]
    N = b.shape[-2]
    if b.shape[-1] != K:
        raise IgapwError(IGAPW_ERR_ARG, f'tc_gemm: inner sizes {K} and {b.shape[-1]} differ')
    if out is None:
        out = torch.empty((batch, M, N) if batched else (M, N), dtype=torch.float32, device=a.device)
    sa = a.stride()
    sb = b.stride()
    so = out.stride()
    bA = sa[0] if a.dim() == 3 else 0
    bB = sb[0] if b.dim() == 3 else 0
    bD = so[0] if out.dim() == 3 else 0
    igapw_tc_gemm(M, N, K, batch, a.data_ptr(), sa[-2:], bA, b.data_ptr(), sb[-2:], bB, out.data_ptr(), so[-2:], bD,
                  pre, bn, splits, torch.cuda.current_stream())
    return out


def _bcheck(rc, b=None):
    if rc != IGAPW_OK:
        msg = load().igapw_batch_last_error(b)
        raise IgapwError(rc, msg.decode() if msg else '')


def igapw_batch_create(descs, stream=None):
    arr = (igapw_desc * len(descs))(*descs)
    b = ctypes.c_void_p()
    _bcheck(load().igapw_batch_create(ctypes.byref(b), arr, len(descs), _stream_handle(stream)), None)
    return b


def igapw_batch_source_sine(b, params):
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float64)
    _bcheck(load().igapw_batch_source_sine(b, p.ctypes.data_as(ctypes.POINTER(_D))), b)


def igapw_batch_solve(b):
    _bcheck(load().igapw_batch_solve(b), b)


def igapw_batch_sync_status(b):
    _bcheck(load().igapw_batch_sync_status(b), b)


def igapw_batch_tensor(b, i, which):
    ptr = ctypes.c_void_p()
    n = ctypes.c_longlong()
    _bcheck(load().igapw_batch_tensor(b, i, which, ctypes.byref(ptr), ctypes.byref(n)), b)
    return ptr.value, n.value


def igapw_batch_info(b):
    t = (_I * 4)()
    _bcheck(load().igapw_batch_info(b, t), b)
    return tuple(t)


def igapw_batch_last_error(b):
    return load().igapw_batch_last_error(b).decode()


def igapw_batch_destroy(b):
    _bcheck(load().igapw_batch_destroy(b), None)


# ---- torch convenience wrapper ----------------------------------------------

class Context:
    """One problem instance.  Coefficient tensors: float64 of shape
    (n_z, n_y, n_x)[-dim:] for precision 'fp64'; float32 of shape
    (2, n_z, n_y, n_x)[...] (hi plane, lo plane) for 'fp32r'."""

    def __init__(self, dim, n_elem, degree, nq, test='pw', bc='none', precision='fp64', op='heat',
                 flags=0, stream=None, neumann_axes=0, refine=0):
        import torch
        if isinstance(n_elem, int):
            n_elem = [n_elem] * dim
        d = igapw_desc()
        d.dim = dim
        for a in range(3):
            d.n_elem[a] = n_elem[a] if a < dim else 1
        d.degree, d.nq = degree, nq
        d.test, d.bc = TESTS[test], BCS[bc]
        d.precision, d.op, d.flags = PRECISIONS[precision], OPS[op], flags
        d.neumann_axes = neumann_axes
        d.refine = refine
        self.desc = d
        self.dim, self.p, self.precision = dim, degree, precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = igapw_create(d, self.stream)
        self.ntot, dims = igapw_size(self.ctx)
        self.n = dims                                   # (n_x, n_y, n_z)
        self.shape = tuple(reversed(dims[:dim]))        # (n_z, n_y, n_x)[-dim:]
        self._count_points()

    def _count_points(self):
        """Quadrature points per axis (the sample grid of rhs_source)."""
        self.q = []
        for a in range(self.dim):
            cnt = _I()
            _check(load().igapw_quad_points(self.ctx, a, None, None, ctypes.byref(cnt)), self.ctx)
            self.q.append(cnt.value)

    def _coefs(self, t, what):
        import torch
        if self.precision == 'fp64':
            _check_tensor(t, what, torch.float64, self.ntot)
        else:
            _check_tensor(t, what, torch.float32, 2 * self.ntot)
        return t

    def _samples(self, t, what, axes):
        import torch
        numel = 1
        for a in axes:
            numel *= self.q[a]
        _check_tensor(t, what, torch.float64 if self.precision == 'fp64' else torch.float32, numel)
        return t

    # tensors --------------------------------------------------------------
    def empty(self):
        import torch
        if self.precision == 'fp64':
            return torch.empty(self.shape, dtype=torch.float64, device='cuda')
        return torch.empty((2,) + self.shape, dtype=torch.float32, device='cuda')

    def from_numpy(self, u):
        """Device coefficient tensor from a float64 array (split into hi/lo for fp32r)."""
        import numpy as np
        import torch
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.shape)
        if self.precision == 'fp64':
            return torch.from_numpy(u).cuda()
        hi = u.astype(np.float32)
        lo = (u - hi.astype(np.float64)).astype(np.float32)
        return torch.from_numpy(np.stack([hi, lo])).cuda()

    def to_numpy(self, t):
        import numpy as np
        a = t.detach().cpu().numpy()
        if self.precision == 'fp64':
            return a.astype(np.float64)
        return a[0].astype(np.float64) + a[1].astype(np.float64)

    # calls -------------------------------------------------------------------
    def apply(self, op, u, dt=0.0, out=None):
        out = self.empty() if out is None else self._coefs(out, 'apply: out')
        igapw_apply(self.ctx, OPS[op], dt, self._coefs(u, 'apply: u'), out)
        return out

    def solve(self, r, out=None):
        out = self.empty() if out is None else self._coefs(out, 'solve: out')
        igapw_solve(self.ctx, self._coefs(r, 'solve: r'), out)
        return out

    def step(self, u, dt, nsteps):
        igapw_step(self.ctx, dt, nsteps, self._coefs(u, 'step: u'))
        return u

    STEP_KINDS = {'staged': 0, 'global': 1, 'staged16': 2, 'chunked': 3}

    def set_step_shape(self, axis, kind, lines=32):
        """igapw_set_step_shape: pin the split-step kernel of one axis
        ('staged', 'global', 'staged16', 'chunked', or None for the autotuner)."""
        k = -1 if kind is None else self.STEP_KINDS[kind]
        igapw_set_step_shape(self.ctx, axis, k, lines if k >= 0 else 0)

    def get_step_shape(self, axis):
        """(kind name or None, lines per block) in use on one axis."""
        k, nl = igapw_get_step_shape(self.ctx, axis)
        names = {v: n for n, v in self.STEP_KINDS.items()}
        return names.get(k), nl

    def step_host(self, u_host, dt, nsteps):
        """igapw_step_host: `nsteps` steps of a HOST state (numpy array or CPU
        tensor, C-contiguous, float64 / float32 pair planes as on the device;
        pinned memory makes the copies asynchronous), copied in and back,
        synchronised before returning."""
        import numpy as np
        fp64 = self.precision == 'fp64'
        numel = self.ntot if fp64 else 2 * self.ntot
        if isinstance(u_host, np.ndarray):
            ok = (u_host.dtype == (np.float64 if fp64 else np.float32) and u_host.flags.c_contiguous
                  and u_host.flags.writeable and u_host.size == numel)
            ptr = u_host.ctypes.data
        elif hasattr(u_host, 'is_cuda') and not u_host.is_cuda:
            import torch
            ok = (u_host.dtype == (torch.float64 if fp64 else torch.float32) and u_host.is_contiguous()
                  and u_host.numel() == numel)
            ptr = u_host.data_ptr()
        else:
            raise IgapwError(IGAPW_ERR_ARG, 'step_host: u_host must be a numpy array or a CPU tensor')
        if not ok:
            raise IgapwError(IGAPW_ERR_ARG, f'step_host: expected a writable C-contiguous '
                             f'{"float64" if fp64 else "float32"} buffer of {numel} elements')
        igapw_step_host(self.ctx, dt, nsteps, ptr)
        return u_host

    def rhs_source(self, f, out=None):
        out = self.empty() if out is None else self._coefs(out, 'rhs_source: out')
        igapw_rhs_source(self.ctx, self._samples(f, 'rhs_source: f', range(self.dim)), out)
        return out

    def rhs_source_sine(self, amp, k, out=None):
        """igapw_rhs_source_sine: b = T(amp prod_a sin(k_a pi x_a)), source evaluated on the device."""
        out = self.empty() if out is None else self._coefs(out, 'rhs_source_sine: out')
        if len(k) != self.dim:
            raise IgapwError(IGAPW_ERR_ARG, f'rhs_source_sine: {len(k)} wave numbers for dim {self.dim}')
        igapw_rhs_source_sine(self.ctx, amp, k, out)
        return out

    def rhs_neumann(self, axis, side, g, b):
        """b += the Neumann data term of the end face `side` of `axis` (in place)."""
        if 0 <= axis < self.dim:
            self._samples(g, 'rhs_neumann: g', [a for a in range(self.dim) if a != axis])
        igapw_rhs_neumann(self.ctx, axis, side, g, self._coefs(b, 'rhs_neumann: b'))
        return b

    def quad_points(self, axis):
        return igapw_quad_points(self.ctx, axis)

    def basis_table(self, axis):
        return igapw_basis_table(self.ctx, axis, self.p)

    def assemble_1d(self, axis, which):
        return igapw_assemble_1d(self.ctx, axis, OPS[which], self.n[axis])

    def set_knots(self, axis, knots):
        igapw_set_knots(self.ctx, axis, knots)
        self._count_points()

    def sync(self):
        igapw_sync_status(self.ctx)

    def close(self):
        if self.ctx:
            igapw_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _desc(dim, n_elem, degree, nq, test, bc, precision, op, flags=0):
    if isinstance(n_elem, int):
        n_elem = [n_elem] * dim
    d = igapw_desc()
    d.dim = dim
    for a in range(3):
        d.n_elem[a] = n_elem[a] if a < dim else 1
    d.degree, d.nq = degree, nq
    d.test, d.bc = TESTS[test], BCS[bc]
    d.precision, d.op, d.flags = PRECISIONS[precision], OPS[op], flags
    return d


class _DevArray:
    """A device buffer owned by the library, exposed to torch without a copy."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {'shape': (count,), 'typestr': '<f4', 'data': (ptr, False), 'version': 2}


class Batch:
    """Batched 2D Poisson instances (FP32 pairs): shapes is a list of
    (n_elem_x, n_elem_y, degree) tuples; tests PW or Galerkin.  gemm: 'tc'
    (the library's tensor-core transforms) or 'cublas'."""

    def __init__(self, shapes, test='pw', stream=None, gemm='tc'):
        import torch
        if gemm not in ('tc', 'cublas'):
            raise IgapwError(IGAPW_ERR_ARG, f"Batch: gemm must be 'tc' or 'cublas', not {gemm!r}")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.shapes = [tuple(s) for s in shapes]
        flags = IGAPW_FLAG_FDM_CUBLAS if gemm == 'cublas' else 0
        descs = [_desc(2, [nx, ny], p, p + 1, test, 'dirichlet0', 'fp32r', 'poisson', flags)
                 for nx, ny, p in self.shapes]
        self.handle = igapw_batch_create(descs, self.stream)

    def source_sine(self, params):
        """params: one row (amp, kx, ky) per instance; the library reads
        exactly instances x 3 doubles, so any other shape is rejected."""
        import numpy as np
        p = np.asarray(params, dtype=np.float64)
        if p.shape != (len(self.shapes), 3):
            raise IgapwError(IGAPW_ERR_ARG, f'source_sine: params of shape {p.shape}, expected ({len(self.shapes)}, 3)')
        igapw_batch_source_sine(self.handle, p)

    def solve(self):
        igapw_batch_solve(self.handle)

    def sync_status(self):
        """Waits for the batch stream; raises IgapwError if a tensor-core GEMM
        of a solve timed out."""
        igapw_batch_sync_status(self.handle)

    def tensor(self, i, which):
        """Instance i's RHS (which = 0) or solution (1) as a torch view of shape
        (2, n_y, n_x) (hi plane, lo plane), aliasing the batch's memory."""
        import torch
        ptr, n = igapw_batch_tensor(self.handle, i, which)
        nx, ny, p = self.shapes[i]
        t = torch.as_tensor(_DevArray(ptr, 2 * n), device='cuda')
        return t.view(2, ny + p, nx + p)

    def to_numpy(self, i, which):
        t = self.tensor(i, which).cpu().numpy().astype('float64')
        return t[0] + t[1]

    def tiles(self):
        return igapw_batch_info(self.handle)

    def close(self):
        if self.handle:
            igapw_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
