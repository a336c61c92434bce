"""Host logic of the column-wave scheduler, on CPU: the scheduler source is
compiled with g++ together with a checker (tests/native/sched_check.cpp) and
run on single-grid and multi-grid cases; every (grid, tile, plane) unit must
be covered once, by a valid item of a CTA below the CTA count, and the
busiest CTA must carry no more than one item's worth of planes above an even
share."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2312_13094_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    gxx = shutil.which("g++")
    inc = _cuda_include()
    if not gxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("sched") / "sched_check")
    subprocess.check_call([gxx, "-std=c++17", "-O2", "-I", inc, "-I", CSRC, "-x", "c++",
                           os.path.join(CSRC, "fd_sched.cu"), "-x", "c++",
                           os.path.join(ROOT, "tests", "native", "sched_check.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True)
    rows = {}
    for line in out.stdout.split("\n"):
        if line.strip():
            name, used, items, busiest, bad = line.split()
            rows[name] = (int(used), int(items), int(busiest), int(bad))
    return out.returncode, rows


def test_every_unit_is_scheduled_exactly_once(results):
    rc, rows = results
    assert len(rows) == 10
    for name, (_, _, _, bad) in rows.items():
        assert bad == 0, name
    assert rc == 0


def test_schedules_fill_the_ctas_evenly(results):
    _, rows = results
    # all 740 columns fit in 760 CTAs: one whole column each
    assert rows["single_fits"][:3] == (740, 740, 592)
    # 370 columns on 304 CTAs: chunks, every CTA busy, the busiest CTA within
    # one chunk of the even share
    used, items, busiest, _ = rows["single_waves"]
    assert used == 304 and items > 370
    assert busiest <= 370 * 592 / 304 + 592 / (items // 370)
    assert rows["tiny"][0] == 3 and rows["one_cell"][:2] == (1, 1)
    assert rows["one_cta"][0] == 1 and rows["one_cta"][2] == 17 * 33
