"""Every shared-memory pass of every candidate plan stays inside the plan's
shared memory and never reads a region it writes (host-side, no GPU): the
plan builder's layout, including fused pairs of 2-way levels, checked by a
small C++ program linked against the library's own plan code."""
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2201_10473_gb300 import autotune

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2201_10473_gb300", "csrc")


@pytest.fixture(scope="module")
def checker():
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not available")
    exe = os.path.join(tempfile.mkdtemp(prefix="gf2x_layout_"), "layout_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    os.path.join(HERE, "layout_check.cpp"), os.path.join(CSRC, "plan_host.cpp"), "-o", exe],
                   check=True)
    return exe


@pytest.mark.parametrize("sizes", [(12323, 17669, 24659), (35851, 40973, 57637), (1000, 4096, 65536, 131072)])
def test_every_candidate_plan_layout(checker, sizes):
    lines = [f"{n} {s}" for n in sizes for s in autotune.candidate_specs(n, split_from=0)]
    r = subprocess.run([checker], input="\n".join(lines), capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-2000:]
    assert f"checked {len(lines)} plans" in r.stdout and " 0 problems" in r.stdout, r.stdout[-500:]
