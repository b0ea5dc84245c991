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


def test_eval_launches_argument_checks():
    """(answered before any device query)"""
    import pytest
    assert gp.eval_launches(0, 1000) == 0
    with pytest.raises(gp.GPError):
        gp.eval_launches(-1, 1000)
    with pytest.raises(gp.GPError):
        gp.eval_launches(10, -1)


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
    # the encoder's slot layout: count and pointers checked before the launch
    assert L.gp_encode_slots_device(None, -1, None, None) == 1
    assert b"negative" in L.gp_error_string()
    assert L.gp_encode_slots_device(None, 5, None, None) == 1
    assert b"null" in L.gp_error_string()
    assert L.gp_encode_slots_device(None, 0, None, None) == 0


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field
    offsets (the header compiled by the host C compiler)."""
    import subprocess
    import sys
    mirrors = {"gp_config": gp.Config, "gp_prog_info": gp._ProgInfo,
               "gp_server_opts": gp._ServerOpts, "gp_evolve_params": gp.EvolveParams,
               "gp_request_info": gp.RequestInfo, "gp_server_stats": gp.ServerStats}
    nested = {"gp_server_opts": {"variant", "k", "block", "chunk_cases", "fitness", "tile_inputs",
                                 "stack_registers", "max_instructions"}}

    def member(cname, fname):  # the binding flattens gp_server_opts.config
        return f"config.{fname}" if fname in nested.get(cname, ()) else fname
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {member(cname, fname)}));')
    lines.append("  return 0; }")
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-std=c11", str(src), "-o", str(exe)])
    out = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, py in mirrors.items():
        assert int(out[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(py, fname).offset, f"{cname}.{fname}"
