"""Build the CUDA library libhdg_gb300.so in-tree with nvcc for sm_103a.

The translation units are compiled in parallel, then linked into one shared library next to
this file. No CMake; nvcc and a host C++ compiler only.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, 'csrc')
LIB = os.path.join(HERE, 'libhdg_gb300.so')
BUILD = os.path.join(HERE, '_build')
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
SOURCES = ['hdg_solver.cu', 'refelem.cpp', 'mesh.cpp', 'hdg_server.cpp']


def _nvcc():
    exe = shutil.which('nvcc')
    if exe is None:
        for cand in ('/usr/local/cuda/bin/nvcc',):
            if os.path.exists(cand):
                return cand
        raise RuntimeError('nvcc not found')
    return exe


def _newer(target, deps):
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def build_library(force=False, verbose=False):
    """Compile (if needed) and return the path of the shared library."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + \
           [os.path.join(HERE, '..', 'include', 'hdg.h')]
    if not force and _newer(LIB, deps + [__file__]):
        return LIB
    flags = ['-O3', '-std=c++17', '-lineinfo', '-Xcompiler', '-fPIC', '-Xcompiler', '-O3',
             '--expt-relaxed-constexpr'] + ARCH

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + '.o')
        cmd = [nvcc] + flags + ['-c', os.path.join(CSRC, src), '-o', obj]
        if verbose:
            cmd.append('-Xptxas=-v')
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f'nvcc failed for {src}:\n{r.stdout}\n{r.stderr}')
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    objs = [o for o, _ in results]
    tmp = LIB + '.tmp'
    r = subprocess.run([nvcc] + ARCH + ['-shared', '-o', tmp] + objs + ['-lcudart'],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f'link failed:\n{r.stdout}\n{r.stderr}')
    os.replace(tmp, LIB)
    if verbose:
        for _, log in results:
            print(log)
    return LIB


if __name__ == '__main__':
    print(build_library(force=True, verbose=True))
