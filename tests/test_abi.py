"""The C-ABI library builds, loads and exports every entry point of include/isam.h;
struct layouts seen by the binding match the C compiler's; argument validation
works without touching a GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "isam.h")


@pytest.fixture(scope="module")
def isam():
    import __graft_entry__ as g
    g.build()
    from paper_1905_06058_gb300 import isam as B
    return B


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(isam_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(isam):
    names = declared_functions()
    assert "isam_plan_create" in names and "isam_solve" in names and len(names) >= 10
    lib = ctypes.CDLL(isam.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", isam.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (isam_\w+)", out))
    assert set(names) <= exported


def test_struct_layout_matches_c(isam):
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "isam.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("isam_params %zu\n", sizeof(isam_params));
  printf("isam_solve_opts %zu\n", sizeof(isam_solve_opts));
  printf("isam_solve_state %zu\n", sizeof(isam_solve_state));
  printf("isam_solve_info %zu\n", sizeof(isam_solve_info));
  printf("isam_tuning %zu\n", sizeof(isam_tuning));
  P(isam_tuning, stolt_table) P(isam_tuning, lateral_radix)
  P(isam_params, k_min) P(isam_params, dx) P(isam_params, z0) P(isam_params, n_disp)
  P(isam_params, disp) P(isam_params, precision) P(isam_params, nufft_os)
  P(isam_params, flags)
  P(isam_solve_opts, max_iter) P(isam_solve_opts, w_dev) P(isam_solve_opts, L)
  P(isam_solve_opts, eps) P(isam_solve_opts, prior) P(isam_solve_state, k) P(isam_solve_state, L)
  P(isam_solve_info, rr) P(isam_solve_info, status) P(isam_solve_info, objective)
  P(isam_solve_opts, objective) P(isam_solve_opts, prior_iters)
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in lines if line)
    types = {"isam_params": isam.IsamParams, "isam_solve_opts": isam.SolveOpts,
             "isam_solve_state": isam.SolveState, "isam_solve_info": isam.SolveInfo,
             "isam_tuning": isam.Tuning}
    for key, val in got.items():
        if "." in key:
            t, f = key.split(".")
            f = {"lambda": "lambda_"}.get(f, f)
            assert getattr(types[t], f).offset == int(val), key
        else:
            assert ctypes.sizeof(types[key]) == int(val), key


def test_status_strings(isam):
    lib = isam.lib()
    for code, text in isam.STATUS.items():
        assert lib.isam_status_string(code).decode() == text


def _params(isam, **kw):
    from paper_1905_06058_gb300 import inputs as I
    g = I.small_bscan(nx=8, nk=32).geom
    p = isam.make_params(g)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("field,value,status", [
    ("nx", 5, 1),            # neither 2^p nor 3 * 2^p
    ("nx", 12, 1),           # 3 * 2^p needs p >= 3
    ("ny", 40, 1),
    ("nk", 48, 1),
    ("nz", 16, 6),           # nz < nk
    ("nz", 4096, 6),         # beyond the 2048-row axial limit
    ("k_min", -1.0, 1),
    ("dx", 0.0, 1),
    ("n_disp", 5, 1),
    ("nufft_J", 5, 6),
    ("nufft_os", 3, 6),
    ("precision", 7, 1),
    ("flags", 2, 1),         # unknown flag bit
])
def test_plan_create_rejects_bad_parameters_before_any_device_call(isam, field, value, status):
    lib = isam.lib()
    p = _params(isam, **{field: value})
    h = ctypes.c_void_p()
    assert lib.isam_plan_create(ctypes.byref(p), None, ctypes.byref(h)) == status
    assert not h.value


def test_null_arguments(isam):
    lib = isam.lib()
    assert lib.isam_plan_create(None, None, None) == 1
    assert lib.isam_forward(None, None, None) == 1
    assert lib.isam_adjoint(None, None, None) == 1
    assert lib.isam_solve(None, None, None, None, None, None) == 1
    assert lib.isam_last_launch_count(None) == -1
    lib.isam_plan_destroy(None)
    a = isam._ALLOC_T(lambda n, c: None)
    assert lib.isam_set_allocator(ctypes.cast(a, ctypes.c_void_p), None, None) == 1   # half a pair
    assert lib.isam_set_allocator(None, None, None) == 0
    assert lib.isam_batch_create(None, 0, None, None, None, None, None) == 1
    assert lib.isam_batch_entry_ms(None, None) == 1
    assert lib.isam_data_fidelity(None, None, None, None, None) == 1
    assert lib.isam_autotune_ex(None, None) == 1
    assert lib.isam_get_tuning(None, None) == 1
    assert lib.isam_set_tuning(None, None) == 1
    assert lib.isam_set_filter(None, None) == 1
    assert lib.isam_unrolled_checkpoint_images(20, 5) == 8
    assert lib.isam_unrolled_checkpoint_images(0, 5) == -1
