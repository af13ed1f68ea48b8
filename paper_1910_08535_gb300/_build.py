"""Builds libigapw.so in-tree for sm_103a: one nvcc process per translation
unit (run in parallel), then one link step.  No cmake, no torch extension
machinery; the library has a plain C ABI (include/igapw.h).

build(bounds=True) builds the debug variant lib/libigapw_bounds.so (objects
in _objs_bounds/): every kernel checks its global and shared indices, skips
an out-of-range access and records it, and igapw_sync_status reports it."""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, 'csrc')
OBJ = os.path.join(HERE, '_objs')
LIB = os.path.join(HERE, 'lib', 'libigapw.so')
OBJ_BOUNDS = os.path.join(HERE, '_objs_bounds')
LIB_BOUNDS = os.path.join(HERE, 'lib', 'libigapw_bounds.so')
SOURCES = ['setup.cpp', 'tables.cu', 'solve.cu', 'rhs.cu', 'api.cu', 'noalloc.cu', 'step.cu', 'poisson.cu', 'batch.cu',
           'step_f64_p2.cu', 'step_f64_p3.cu', 'step_f64_p4.cu', 'step_df_p2.cu', 'step_df_p3.cu', 'step_df_p4.cu',
           'chunkstep_p2.cu', 'chunkstep_p3.cu', 'chunkstep_p4.cu']
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC', '--expt-relaxed-constexpr',
         '-Xcompiler', '-Wall', '-Xcompiler', '-Wno-unused-function']


def nvcc():
    path = shutil.which('nvcc') or '/usr/local/cuda/bin/nvcc'
    if not os.path.exists(path):
        raise RuntimeError('nvcc not found: the CUDA toolkit is required to build libigapw')
    return path


def _extra():
    """Extra nvcc flags from IGAPW_NVCC_EXTRA (any additional defines)."""
    return os.environ.get('IGAPW_NVCC_EXTRA', '').split()


def _obj(src, objdir):
    return os.path.join(objdir, os.path.splitext(src)[0] + '.o')


def _deps(src, objdir):
    """Files the object of `src` depends on (from the .d file nvcc wrote with
    it), or None when unknown."""
    d = os.path.splitext(_obj(src, objdir))[0] + '.d'
    try:
        txt = open(d).read().replace('\\\n', ' ')
    except OSError:
        return None
    parts = txt.split(':', 1)
    return [f for f in parts[1].split() if f] if len(parts) == 2 else None


def _stale(src, objdir):
    out = _obj(src, objdir)
    if not os.path.exists(out):
        return True
    deps = _deps(src, objdir)
    if deps is None:
        return True
    t = os.path.getmtime(out)
    try:
        return any(os.path.getmtime(f) > t for f in deps + [os.path.join(CSRC, src)])
    except OSError:
        return True


def _compile(src, objdir, extra):
    out = _obj(src, objdir)
    dep = os.path.splitext(out)[0] + '.d'
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, '-MD', '-MF', dep, '-c', os.path.join(CSRC, src), '-o', out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, r.returncode, r.stdout + r.stderr, out


def build(verbose=False, force=False, bounds=False):
    """Compile (the units whose object is older than the unit or a header it
    includes; all with force) and link; returns the .so path."""
    objdir, lib = (OBJ_BOUNDS, LIB_BOUNDS) if bounds else (OBJ, LIB)
    extra = _extra() + (['-DIGAPW_BOUNDS_CHECK'] if bounds else [])
    if _extra():
        force = True
    os.makedirs(objdir, exist_ok=True)
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    todo = [s for s in SOURCES if force or _stale(s, objdir)]
    if not todo and os.path.exists(lib):
        newest = max(os.path.getmtime(_obj(s, objdir)) for s in SOURCES)
        if os.path.getmtime(lib) >= newest:
            return lib
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(todo))) as ex:
        results = list(ex.map(lambda s: _compile(s, objdir, extra), todo))
    failed = [r for r in results if r[1] != 0]
    for src, rc, log, _ in results:
        if verbose or rc != 0:
            sys.stderr.write(f'--- {src} (rc={rc})\n{log}')
    if failed:
        raise RuntimeError('nvcc failed for ' + ', '.join(f[0] for f in failed))
    objs = [_obj(s, objdir) for s in SOURCES]
    tmp = lib + '.tmp'
    libdir = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc()))), 'lib64')
    cmd = [nvcc(), *ARCH, '-shared', '-o', tmp, *objs, '-lcudart', '-lcublas', '-lcusolver',
           '-Xlinker', '-rpath=' + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('link failed:\n' + r.stdout + r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == '__main__':
    print(build(verbose='-v' in sys.argv, force='-f' in sys.argv, bounds='--bounds' in sys.argv))
