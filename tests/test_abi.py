"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/evp.h declares (no compute calls)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, 'include', 'evp.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    return sorted(set(re.findall(r'\b(evp_[a-z_0-9]+)\s*\(', src)))


@pytest.fixture(scope='module')
def libpath():
    from paper_1803_09563_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ('evp_init', 'evp_step', 'evp_project', 'evp_set_field', 'evp_get_field', 'evp_sync',
                 'evp_destroy', 'evp_poisson_solve', 'evp_stress_rhs', 'evp_last_error'):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(['nm', '-D', '--defined-only', libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r' T (evp_\w+)', out))
    assert set(declared_functions()) <= exported


def test_binding_resolves_declared_names(libpath):
    from paper_1803_09563_gb300 import evp
    assert set(evp.exported_symbols()) == set(declared_functions())
    lib = evp.load(libpath)
    assert lib.evp_num_kernels() >= 9
    assert lib.evp_kernel_name(0).decode() == 'stress_weno_update'


def test_state_bytes_validates_without_a_gpu(libpath):
    from paper_1803_09563_gb300 import evp
    evp.load(libpath)
    g = evp.make_grid(256, 128, 128, 4 * 3.141592653589793, 2.0, 2 * 3.141592653589793, True)
    p = evp.make_params(Re=100, Wi=1, beta=0.5, Bi=0.5, precision=evp.EVP_FP32)
    nb = evp.evp_state_bytes(g, evp.EVP_SARAMITO, p)
    N = 256 * 128 * 128
    assert 29 * N * 4 <= nb < 40 * N * 4
    bad = evp.make_grid(250, 128, 128, 1.0, 1.0, 1.0, True)
    assert evp.evp_state_bytes(bad, evp.EVP_SARAMITO, p) == 0


def test_state_bytes_count_the_summed_stress(libpath):
    """An RK3 state with a stress model holds six more fields than a Newtonian one:
    the summed stress tau^k + tau^{k-1} that the stress kernel hands to the momentum
    kernel (N * 4 bytes is a multiple of the 256-byte arena alignment here)."""
    from paper_1803_09563_gb300 import evp
    evp.load(libpath)
    g = evp.make_grid(64, 32, 32, 6.283185307179586, 2.0, 6.283185307179586, True)
    p = evp.make_params(Re=100, Wi=1, beta=0.5, Bi=0.5, precision=evp.EVP_FP32)
    N = 64 * 32 * 32
    assert evp.evp_state_bytes(g, evp.EVP_SARAMITO, p) - evp.evp_state_bytes(g, evp.EVP_NEWTONIAN, p) == 6 * N * 4


def test_batched_copies_reject_a_null_state(libpath):
    """evp_set_fields / evp_get_fields check their arguments before any CUDA call."""
    from paper_1803_09563_gb300 import evp
    lib = evp.load(libpath)
    ids = (ctypes.c_int * 1)(evp.EVP_U)
    bufs = (ctypes.c_void_p * 1)(None)
    assert lib.evp_set_fields(None, 1, ids, bufs, 0) == evp.EVP_ERR_ARG
    assert lib.evp_get_fields(None, 1, ids, bufs, 0) == evp.EVP_ERR_ARG
    assert b'null' in lib.evp_last_error()


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C layout: a small C
    program compiled against include/evp.h prints sizeof and every offsetof."""
    from paper_1803_09563_gb300 import evp
    structs = (('evp_grid', evp.evp_grid), ('evp_params', evp.evp_params), ('evp_diag', evp.evp_diag),
               ('evp_tile_config', evp.evp_tile_config))
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "evp.h"', 'int main(void) {']
    for cname, ct in structs:
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in ct._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['return 0;', '}']
    src = tmp_path / 'layout.c'
    src.write_text('\n'.join(lines))
    exe = tmp_path / 'layout'
    subprocess.run(['gcc', '-std=c99', '-I', os.path.join(ROOT, 'include'), str(src), '-o', str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, fname, val = line.split()
        got[(cname, fname)] = int(val)
    for cname, ct in structs:
        assert got[(cname, 'sizeof')] == ctypes.sizeof(ct), cname
        for fname, _ in ct._fields_:
            assert got[(cname, fname)] == getattr(ct, fname).offset, (cname, fname)
