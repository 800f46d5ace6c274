"""Build libevp.so in-tree for sm_103a with nvcc (no cmake, one -gencode).

Usage: python -m paper_1803_09563_gb300.build [--force] [--debug]
Each .cu translation unit is compiled in parallel, then linked into
paper_1803_09563_gb300/libevp.so next to this file.  --debug builds the
bounds-checked libevp_debug.so instead (-DEVP_DEBUG: the stencil kernels check
every staged copy and poison their shared memory with NaN; a failed check
raises EVP_ERR_BOUNDS at evp_sync).  The binding loads it when the environment
variable EVP_LIB names it.
"""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, 'csrc')
INCLUDE = os.path.join(ROOT, 'include')
OUT = os.path.join(HERE, 'libevp.so')
BUILD = os.path.join(HERE, '_build')
OUT_DEBUG = os.path.join(HERE, 'libevp_debug.so')
BUILD_DEBUG = os.path.join(HERE, '_build_debug')
# translation units that differ in the bounds-checked build; the others are shared
DEBUG_SOURCES = ('k_stress_f32.cu', 'k_stress_f64.cu', 'k_momentum.cu')
SOURCES = ['evp_abi.cu', 'evp_batch.cu', 'k_diag.cu', 'k_stress_f32.cu', 'k_stress_f64.cu', 'k_momentum.cu', 'k_poisson.cu', 'k_twophase.cu', 'evp_static.cu', 'k_selftest.cu', 'k_ibm.cu']

ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC', '-Xcompiler', '-O3',
         '-I', INCLUDE, '-I', CSRC]


def nvcc():
    for cand in (os.environ.get('NVCC'), '/usr/local/cuda/bin/nvcc', 'nvcc'):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return 'nvcc'


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(('.cuh', '.h'))]
    deps.append(os.path.join(INCLUDE, 'evp.h'))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, debug=False):
    bdir, out = (BUILD_DEBUG, OUT_DEBUG) if debug else (BUILD, OUT)
    flags = FLAGS + (['-DEVP_DEBUG'] if debug else [])
    os.makedirs(bdir, exist_ok=True)
    objs = []
    jobs = []
    if debug:
        build(force=force, verbose=verbose)      # the shared objects
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        own = not debug or src in DEBUG_SOURCES
        o = os.path.join(bdir if own else BUILD, src.replace('.cu', '.o'))
        objs.append(o)
        if own and (force or _stale(o, s)):
            jobs.append([nvcc()] + ARCH + flags + ['-c', s, '-o', o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError('nvcc failed:\n' + ' '.join(cmd) + '\n' + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return r

    with ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        list(ex.map(run, jobs))
    if jobs or force or not os.path.exists(out) or any(os.path.getmtime(o) > os.path.getmtime(out) for o in objs):
        run([nvcc()] + ARCH + ['-shared', '-o', out] + objs + ['-lcudart'])
    return out


if __name__ == '__main__':
    print(build(force='--force' in sys.argv, verbose='-v' in sys.argv, debug='--debug' in sys.argv))
