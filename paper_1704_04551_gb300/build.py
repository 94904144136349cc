"""Build the CUDA library ``libibmlbm.so`` in-tree with nvcc for sm_103a.

Each .cu file is compiled to an object in parallel, then linked into one
shared library next to this file. No CMake, no torch extension machinery.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, 'csrc')
INCLUDE = os.path.join(os.path.dirname(HERE), 'include')
BUILD = os.path.join(HERE, '_build')
LIB = os.path.join(HERE, 'libibmlbm.so')
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC', '--expt-relaxed-constexpr',
         '-Xptxas', '-warn-spills']


def nvcc() -> str:
    cand = os.environ.get('NVCC') or shutil.which('nvcc') or '/usr/local/cuda/bin/nvcc'
    if not os.path.exists(cand):
        raise RuntimeError('nvcc not found')
    return cand


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith('.cu'))


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(INCLUDE, 'ibm_lbm.h'))
    return out


def build(force: bool = False, verbose: bool = False, extra=(), out: str | None = None) -> str:
    """Compile (if sources are newer) and return the library path. ``out``
    and ``extra`` build a variant elsewhere with additional nvcc flags."""
    lib = out or LIB
    bdir = BUILD if out is None else out + '.build'
    os.makedirs(bdir, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _deps() + [__file__])
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    cc = nvcc()
    objs = []
    cmds = []
    for src in sources():
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + '.o')
        objs.append(obj)
        cmds.append([cc, *ARCH, *FLAGS, *extra, '-I', INCLUDE, '-c', src, '-o', obj])
    with cf.ThreadPoolExecutor(max_workers=min(8, len(cmds))) as ex:
        futs = [ex.submit(subprocess.run, c, capture_output=True, text=True) for c in cmds]
        for c, f in zip(cmds, futs):
            r = f.result()
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f'nvcc failed: {" ".join(c)}')
    tmp = lib + f'.{os.getpid()}.tmp'
    r = subprocess.run([cc, *ARCH, '-shared', '-o', tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError('link failed')
    os.replace(tmp, lib)
    return lib


if __name__ == '__main__':
    build(force='--force' in sys.argv, verbose='-v' in sys.argv,
          extra=['-Xptxas', '-v'] if '--ptxas' in sys.argv else ())
    print(LIB)
