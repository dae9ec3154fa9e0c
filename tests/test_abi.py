"""The C-ABI library builds, loads without a GPU, and exports what include/pico.h declares."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_2605_09590_gb300 as pico
from paper_2605_09590_gb300 import build as pico_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pico.h")


@pytest.fixture(scope="module")
def lib():
    pico_build.build()
    return pico.load_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pico_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for need in ("pico_init", "pico_apply_normal", "pico_cg_batch", "pico_variance_map", "pico_pmr",
                 "pico_sync", "pico_last_error", "pico_destroy"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", pico.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pico_[a-z_0-9]+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_null_arguments_are_rejected_without_a_gpu(lib):
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    assert lib.pico_init(None, None, 0, ctypes.byref(h)) == pico.PICO_E_INVALID
    assert lib.pico_sync(None) == pico.PICO_E_INVALID
    assert lib.pico_get_info(None, None) == pico.PICO_E_INVALID
    assert lib.pico_get_tuning(None, None) == pico.PICO_E_INVALID
    assert lib.pico_set_tuning(None, None) == pico.PICO_E_INVALID
    assert lib.pico_autotune(None, 0, None, None, 0) == pico.PICO_E_INVALID
    lib.pico_destroy(None)


def test_ctypes_structs_match_the_c_layout(lib):
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "pico.h"
#define P(T, f) printf(#T " " #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("pico_operator_desc size %zu\n", sizeof(pico_operator_desc));
  printf("pico_info size %zu\n", sizeof(pico_info));
  printf("pico_request size %zu\n", sizeof(pico_request));
  printf("pico_tuning size %zu\n", sizeof(pico_tuning));
  P(pico_operator_desc, smaps) P(pico_operator_desc, noise_cov) P(pico_operator_desc, mask)
  P(pico_operator_desc, mask_2d) P(pico_operator_desc, traj) P(pico_operator_desc, nsamp)
  P(pico_operator_desc, oversamp) P(pico_operator_desc, kb_width) P(pico_operator_desc, lambda)
  P(pico_operator_desc, power_iters) P(pico_operator_desc, power_margin) P(pico_operator_desc, max_batch)
  P(pico_operator_desc, max_iter_cap)
  P(pico_info, lambda_max) P(pico_info, lambda_phys) P(pico_info, kind) P(pico_info, nsamp) P(pico_info, device_bytes)
  P(pico_info, normal_op)
  P(pico_request, seed) P(pico_request, nprobes) P(pico_request, rtol) P(pico_request, pmr_sigma)
  P(pico_request, cs_data) P(pico_request, cs_lambda) P(pico_request, cs_iters) P(pico_request, cs_levels)
  P(pico_tuning, gram_min_batch) P(pico_tuning, gram_kc) P(pico_tuning, gram_a_tmem) P(pico_tuning, probe_batch)
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "layout")
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe])
        lines = subprocess.check_output([exe], text=True).split("\n")
    got = {}
    for ln in lines:
        if ln:
            t, f, v = ln.split()
            got[(t, f)] = int(v)
    assert got[("pico_operator_desc", "size")] == ctypes.sizeof(pico.pico_operator_desc)
    assert got[("pico_info", "size")] == ctypes.sizeof(pico.pico_info)
    assert got[("pico_request", "size")] == ctypes.sizeof(pico.pico_request)
    assert got[("pico_tuning", "size")] == ctypes.sizeof(pico.pico_tuning)
    classes = {"pico_operator_desc": pico.pico_operator_desc, "pico_info": pico.pico_info,
               "pico_request": pico.pico_request, "pico_tuning": pico.pico_tuning}
    for (t, f), v in got.items():
        if f == "size":
            continue
        cls = classes[t]
        name = "lambda_" if f == "lambda" else f
        assert getattr(cls, name).offset == v, (t, f)


def test_shard_range_partitions_exactly():
    for total in (0, 1, 7, 256, 1001):
        for world in (1, 2, 3, 8):
            spans = [pico.shard_range(total, world, r) for r in range(world)]
            assert sum(c for _, c in spans) == total
            pos = 0
            for b, c in spans:
                assert b == pos
                pos += c
