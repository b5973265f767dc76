"""Register budget of every kernel, read from ptxas (-Xptxas -v) on the host:
no kernel spills, except the fused kernel's one-slot, four-warp shape at
n <= 11. Its 72-register cap lets 7 CTAs of 128 threads share an SM, and
that shape may spill at most 16 bytes."""
import concurrent.futures as cf
import glob
import os
import re
import shutil

import pytest

from paper_2212_02224_gb300 import build

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists(
    "/usr/local/cuda/bin/nvcc"), reason="needs nvcc")

ENTRY = re.compile(r"Compiling entry function '(\S+)'")
SPILL = re.compile(r"(\d+) bytes spill stores, (\d+) bytes spill loads")


def _entries(src):
    out, name = [], None
    for line in build.ptxas_report(os.path.basename(src)).splitlines():
        m = ENTRY.search(line)
        if m:
            name = m.group(1)
            continue
        m = SPILL.search(line)
        if m and name:
            out.append((name, int(m.group(1)), int(m.group(2))))
            name = None
    return out


def test_no_kernel_spills_beyond_the_documented_shape():
    srcs = sorted(glob.glob(os.path.join(build.CSRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        reports = dict(zip(srcs, ex.map(_entries, srcs)))
    kernels = 0
    for src, entries in reports.items():
        for name, st, ld in entries:
            kernels += 1
            one_slot_four_warps = re.search(r"fused_kernelILi(8|11)ELi1ELi4E", name) is not None
            limit = 16 if one_slot_four_warps else 0
            assert st <= limit and ld <= limit, (os.path.basename(src), name, st, ld)
    assert kernels >= 50          # every translation unit was compiled and read
