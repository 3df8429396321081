"""Host side of the kernel timeline (paper_2602_14450_gb300/timeline.py): the
default build refuses to record, the kernel-site hash of the Python tool is
the one the device code computes, and block records group into launches."""

import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2602_14450_gb300 import build as B
from paper_2602_14450_gb300 import timeline as T
from paper_2602_14450_gb300 import wd


def test_default_build_refuses_recording():
    B.build()
    assert wd.lib().wd_timeline_set(None, None) == wd.WD_ERR_INVALID_ARG


def test_site_hash_matches_the_device_code():
    names = ["hop16_impl.cuh", "blas_impl.cuh", "hop_impl.cuh", "common.cuh"]
    src = ('#include "common.cuh"\n#include <cstdio>\n'
           "void wd::tl::register_unit(int (*)(void*, void*)) {}\n"
           "int main() {\n"
           + "".join(f'    std::printf("%u\\n", wd::tl::name_hash(wd::tl::base_name("/a/b/{n}", "/a/b/{n}")));\n'
                     for n in names)
           + "    return 0;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        cu, exe = os.path.join(d, "h.cu"), os.path.join(d, "h")
        with open(cu, "w") as f:
            f.write(src)
        r = subprocess.run([B.nvcc(), *B.ARCH, *B.FLAGS, "-DWD_TIMELINE", "-I", B.CSRC, cu, "-o", exe],
                           capture_output=True, text=True)
        if r.returncode != 0:
            pytest.fail(r.stderr)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == [T.name_hash(n) for n in names]


def test_block_records_group_into_launches():
    def rec(site, grid, sm, start, end):
        w = (site << 32) | (grid << 8) | sm
        return [w - (1 << 64) if w >= 1 << 63 else w, start - 5, start, end]

    a, b = (7 << 16) | 100, (0xFE20 << 16) | 200   # a file hash with the top bit set (negative as int64)
    rows = [
        rec(a, 2, 0, 0, 10), rec(a, 2, 1, 1, 12),       # launch 1: two blocks
        rec(b, 1, 0, 13, 20),                            # launch 2: another kernel
        rec(b, 1, 3, 25, 30),                            # launch 3: same kernel, starts after all ended
        rec(a, 2, 2, 31, 40), rec(a, 2, 0, 33, 41),      # launch 4
    ]
    ls = T.launches_of(np.array(rows[::-1], dtype=np.int64))   # records arrive in any order
    assert [(l["site"], l["grid"], l["blocks"], l["start"], l["end"]) for l in ls] == [
        (a, 2, 2, 0, 12), (b, 1, 1, 13, 20), (b, 1, 1, 25, 30), (a, 2, 2, 31, 41)]
    assert ls[0]["last_block"] == 2.0 and ls[1]["last_block"] == 0.0
