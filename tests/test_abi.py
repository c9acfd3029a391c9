"""The C ABI library: it loads, exports every symbol include/sf.h declares, and
its struct layouts match what a C compiler makes of the header. No GPU needed."""

import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_1610_07159_gb300 import build as B
from paper_1610_07159_gb300 import sf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sf.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return sf.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SF_API\s+[\w\s\*]+?\b(sf_\w+)\s*\(", text)))


def test_header_declares_what_the_binding_expects():
    assert declared_functions() == sorted(sf.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sf_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "sf.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(sf_params), offsetof(sf_params, F), offsetof(sf_params, gn_iters),
         offsetof(sf_params, wfeat_gain), offsetof(sf_params, use_graph), sizeof(sf_stats));
  printf("%zu %zu %zu %zu %zu %zu\n", offsetof(sf_stats, energy), offsetof(sf_stats, step_energy),
         offsetof(sf_stats, step_t), offsetof(sf_stats, step_excluded), offsetof(sf_stats, launches),
         offsetof(sf_params, profile_mask));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in out]
    P, S = sf.Params, sf.Stats
    assert vals[:6] == [ctypes.sizeof(P), P.F.offset, P.gn_iters.offset, P.wfeat_gain.offset, P.use_graph.offset,
                        ctypes.sizeof(S)]
    assert vals[6:] == [S.energy.offset, S.step_energy.offset, S.step_t.offset, S.step_excluded.offset,
                        S.launches.offset, P.profile_mask.offset]


def test_preset_is_table1(lib):
    import oracle
    for which, name in ((sf.PRESET_FIG2, "fig2"), (sf.PRESET_FIG568, "fig568"), (sf.PRESET_FIG79, "fig79")):
        p = sf.preset(which)
        for k, v in oracle.TABLE1[name].items():
            assert abs(getattr(p, k) - v) <= 1e-6 * abs(v), (name, k)
        assert p.w_smooth == 1.0 and p.w_mag == 1.0
    assert lib.sf_params_preset(ctypes.byref(sf.Params()), 7) == sf.ERR_ARG


@pytest.mark.parametrize("w,h,s,L", [(1, 10, 2, 1), (64, 48, 0, 2), (64, 48, 8, 9), (64, 48, 8, 4), (16, 16, 16, 1)])
def test_create_rejects_invalid_sizes_before_touching_the_gpu(lib, w, h, s, L):
    p = sf.preset()
    assert not lib.sf_create(w, h, s, L, ctypes.byref(p))
    assert lib.sf_last_error() == sf.ERR_ARG


def test_create_rejects_invalid_params(lib):
    p = sf.preset(eps=0.0)
    assert not lib.sf_create(64, 48, 4, 2, ctypes.byref(p))
    assert lib.sf_last_error() == sf.ERR_ARG
    p = sf.preset(w_photo=float("nan"))
    assert not lib.sf_create(64, 48, 4, 2, ctypes.byref(p))
    p = sf.preset(gn_iters=[17])
    assert not lib.sf_create(64, 48, 4, 2, ctypes.byref(p))


def test_null_arguments_are_errors(lib):
    assert lib.sf_solve(None, None, None, None, None, None, None) == sf.ERR_ARG
    assert lib.sf_get_stats(None, None) == sf.ERR_ARG
    assert lib.sf_status_string(sf.ERR_TIMEOUT) == b"device barrier timeout"
