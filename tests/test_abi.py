"""The C ABI library: builds, loads without a GPU, exports every function
include/lbm.h declares, and its ctypes mirror matches the C layout."""
import ctypes as C
import os
import re
import subprocess

import pytest

import paper_2609_25670_b300 as lbm
from paper_2609_25670_b300 import build as lbm_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    lbm_build.build()
    return lbm.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_header_declarations_are_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    out = subprocess.check_output(["nm", "-D", "--defined-only", lbm.LIB_PATH]).decode()
    exported = set(re.findall(r"\bT (lbm_\w+)", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)
    assert set(lbm.EXPORTED) <= exported


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\nint main(void){'
                    'printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(lbm_params), sizeof(lbm_seed), '
                    'sizeof(lbm_diag), offsetof(lbm_params, dt_base), offsetof(lbm_params, frozen_V), '
                    'offsetof(lbm_diag, tip), sizeof(lbm_allocator), offsetof(lbm_diag, R_M)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(lbm.lbm_params), C.sizeof(lbm.lbm_seed), C.sizeof(lbm.lbm_diag),
            lbm.lbm_params.dt_base.offset, lbm.lbm_params.frozen_V.offset, lbm.lbm_diag.tip.offset,
            C.sizeof(lbm.lbm_allocator), lbm.lbm_diag.R_M.offset]
    assert got == want


def _create(lib, p):
    h = C.c_void_p()
    st = lib.lbm_create(C.byref(p), 1, None, None, None, C.byref(h))
    return st, lib.lbm_last_error(None).decode()


@pytest.mark.parametrize("mutate,status", [
    (lambda p: setattr(p, "struct_version", 99), 1),
    (lambda p: setattr(p, "nx", 2), 1),
    (lambda p: setattr(p, "N_U", 0), 1),
    (lambda p: setattr(p, "precision", 7), 1),
    (lambda p: setattr(p, "q_scalar", 7), 1),
    (lambda p: setattr(p, "bc_flow_y", 2), 1),
    (lambda p: setattr(p, "fields", lbm.FIELD_T | lbm.FIELD_FROZEN_T), 1),
    (lambda p: setattr(p, "tip_cx", 1000), 1),
    (lambda p: setattr(p, "DL", 0.0), 2),
    (lambda p: setattr(p, "nu", -1.0), 2),
])
def test_create_rejects_bad_parameters_without_touching_the_gpu(lib, mutate, status):
    """Validation runs before any CUDA call, so it is checkable on the CPU."""
    import workloads as W
    p = lbm.make_params(W.thermosolutal_convection(n=64).params, "f32")
    mutate(p)
    st, msg = _create(lib, p)
    assert st == status, msg
    assert msg


def test_null_arguments(lib):
    assert lib.lbm_create(None, 1, None, None, None, None) == 1
    assert lib.lbm_advance(None, 1) == 1
    assert lib.lbm_last_error(None)
    lib.lbm_destroy(None)
