"""The C ABI library loads and exports every entry point include/gpeval.h
declares (CPU only: no CUDA call is made)."""
import ctypes
import os
import re

import paper_1601_00221_gb300 as gp

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "gpeval.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gp_eval_population", "gp_eval_population_bool", "gp_eval_outputs",
                 "gp_encode_tree", "gp_encode_population", "gp_set_config", "gp_shutdown"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(gp.build.LIB if os.path.exists(gp.build.LIB) else gp.build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a():
    # the build flags name exactly one architecture: sm_103a
    assert gp.build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_side_argument_checks_without_gpu():
    L = gp.lib()
    assert gp.version() >= 10000
    # argument errors are found on the host before any CUDA call
    rc = L.gp_eval_population(None, None, None, -1, None, 1, 10, None, None, None)
    assert rc == 1
    assert b"negative" in L.gp_error_string() or b"null" in L.gp_error_string()
    bad = gp.Config(variant=1, k=3, block=128, chunk_cases=0)
    assert L.gp_set_config(ctypes.byref(bad)) == 1
    assert b"k must be" in L.gp_error_string()
