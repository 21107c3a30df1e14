"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/sr_ot.h with the struct layout the binding assumes.
No compute call: these run without a GPU."""
import ctypes as ct
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sr_ot.h")


@pytest.fixture(scope="module")
def built():
    from paper_2103_05857_gb300 import build as B
    return B.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sr_ot_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sr_ot_create", "sr_ot_solve", "sr_ot_solve_batched", "sr_ot_grad", "sr_ot_gap",
                     "sr_ot_destroy", "sr_ot_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(built):
    lib = ct.CDLL(built)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sr_ot_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_matches_c_struct_layout(built):
    from paper_2103_05857_gb300 import sr_ot as S
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "sr_ot.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(sr_ot_options), sizeof(sr_ot_result),
         offsetof(sr_ot_options, seed), offsetof(sr_ot_options, trace),
         offsetof(sr_ot_options, trace_capacity), offsetof(sr_ot_result, status));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "layout.c")
        exe = os.path.join(td, "layout")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert vals[0] == ct.sizeof(S.Options)
    assert vals[1] == ct.sizeof(S.Result)
    assert vals[2] == S.Options.seed.offset
    assert vals[3] == S.Options.trace.offset
    assert vals[4] == S.Options.trace_capacity.offset
    assert vals[5] == S.Result.status.offset


def test_default_options(built):
    from paper_2103_05857_gb300 import sr_ot as S
    o = S.options()
    assert (o.variant, o.order, o.step, o.precision) == (S.BCFW, S.CYCLIC, S.DEC, S.FP32)
    assert o.rho == 10.0 and o.gap_every == 1 and o.max_epochs == 100


def test_create_fails_cleanly_without_a_gpu(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2103_05857_gb300 import sr_ot as S
    h = ct.c_void_p()
    st = S.lib.sr_ot_create(ct.byref(h), 0, None)
    assert st == S.ECUDA
    assert h.value is None
    assert b"CUDA" in S.lib.sr_ot_last_error(None) or len(S.lib.sr_ot_last_error(None)) > 0


def test_oracle_is_not_linked_into_the_library(built):
    out = subprocess.run(["nm", "-D", built], capture_output=True, text=True).stdout
    assert "srot_or_" not in out
