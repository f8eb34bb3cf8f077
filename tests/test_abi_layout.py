"""The Python binding mirrors include/mclg.h by hand; this compiles a small C
program against the header (gcc, CPU only) and checks that the parameter struct's
layout, the status codes and the flag, mode and sampler constants agree."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "mclg.h"
#define F(name) printf("off_" #name " %zu\n", offsetof(mclg_params, name));
int main(void) {
    printf("size %zu\n", sizeof(mclg_params));
    F(C) F(lambda_num) F(lambda_den) F(flags) F(mode) F(first_replica) F(sampler)
    F(slice_n_max) F(kernel_variant) F(node_offset)
    printf("NO_STREAM %u\nSTATS %u\nGALILEAN %u\nHALO %u\n", MCLG_NO_STREAM, MCLG_STATS,
           MCLG_GALILEAN, MCLG_HALO);
    printf("MODE_AUTO %u\nMODE_PLAIN %u\nMODE_PERSISTENT %u\nMODE_BATCHED %u\n",
           MCLG_MODE_AUTO, MCLG_MODE_PLAIN, MCLG_MODE_PERSISTENT, MCLG_MODE_BATCHED);
    printf("SAMPLER_SEQUENTIAL %u\nSAMPLER_SLICE %u\n", MCLG_SAMPLER_SEQUENTIAL, MCLG_SAMPLER_SLICE);
    printf("status_max %d\n", (int)MCLG_ERR_SAMPLER);
    printf("size2d %zu\n", sizeof(mclg2d_params));
#define F2(name) printf("off2d_" #name " %zu\n", offsetof(mclg2d_params, name));
    F2(C) F2(lambda_num) F2(lambda_den) F2(flags) F2(first_replica)
    return 0;
}
"""


@pytest.fixture(scope="module")
def header_values(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "probe.c", d / "probe"
    src.write_text(PROBE)
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


def mclg_module():
    # the binding's constants and ctypes struct need no GPU and no built library
    import importlib
    return importlib.import_module("paper_1706_01094_gb300.mclg")


def test_params_struct_layout_matches_header(header_values):
    m = mclg_module()
    assert ctypes.sizeof(m.Params) == header_values["size"]
    for name, _ in m.Params._fields_:
        assert getattr(m.Params, name).offset == header_values["off_" + name], name
    assert {n for n, _ in m.Params._fields_} == {k[4:] for k in header_values if k.startswith("off_")}
    assert ctypes.sizeof(m.Params2D) == header_values["size2d"]
    for name, _ in m.Params2D._fields_:
        assert getattr(m.Params2D, name).offset == header_values["off2d_" + name], name


def test_constants_match_header(header_values):
    m = mclg_module()
    for name in ("NO_STREAM", "STATS", "GALILEAN", "HALO", "MODE_AUTO", "MODE_PLAIN", "MODE_PERSISTENT",
                 "MODE_BATCHED", "SAMPLER_SEQUENTIAL", "SAMPLER_SLICE"):
        assert getattr(m, name) == header_values[name], name
    assert sorted(m.STATUS) == list(range(header_values["status_max"] + 1))
