"""The public header is a C ABI: a plain C99 program (tests/c/abi_from_c.c)
compiles against include/igapw.h with warnings as errors, links
libigapw.so, and gets IGAPW_ERR_ARG with an error text from igapw_create's
argument checks (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which('gcc') is None, reason='gcc not available')
def test_plain_c_caller():
    from paper_1910_08535_gb300 import _build, igapw
    lib = _build.build()
    libdir = os.path.dirname(lib)
    out_dir = os.path.join(ROOT, 'tests', 'c', '_build')
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, 'abi_from_c')
    subprocess.run(['gcc', '-std=c99', '-Wall', '-Wextra', '-pedantic', '-Werror',
                    '-I', os.path.join(ROOT, 'include'), os.path.join(ROOT, 'tests', 'c', 'abi_from_c.c'),
                    '-L', libdir, '-ligapw', f'-Wl,-rpath,{libdir}', '-o', exe], check=True)
    res = subprocess.run([exe], check=True, capture_output=True, text=True)
    lines = [l.split(' ', 3) for l in res.stdout.strip().splitlines()]
    assert [l[0] for l in lines] == ['dim', 'degree', 'desc', 'out']
    for what, rc, cleared, msg in lines:
        assert int(rc) == igapw.IGAPW_ERR_ARG, (what, rc, msg)
        assert cleared == '1' and msg, (what, msg)
    assert 'dim' in lines[0][3] and 'degree' in lines[1][3] and 'NULL' in lines[2][3] and 'NULL' in lines[3][3]
