"""Failure handling of the C ABI on the GPU, driven from the host: invalid
arguments, unstable time steps, non-finite data, an injected allocation
failure, and a bounded device wait that is made to run out (the load of one
plane is never issued), after which the grid keeps working."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2312_13094_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2312_13094_gb300 import build
    build.build()
    from paper_2312_13094_gb300 import binding
    return binding


def small(nt=20):
    w = wl.small_acoustic(24)
    w["nt"] = nt
    w["wavelet"] = w["wavelet"][:nt]
    return w


def test_bad_descriptor(fd):
    with pytest.raises(fd.FDError) as e:
        fd.Grid((10, 10, 10), 10.0, 7, 2, 1.0, 5)
    assert e.value.status == fd.FD_ERR_ARG
    with pytest.raises(fd.FDError) as e:
        fd.Grid((0, 10, 10), 10.0, 8, 2, 1.0, 5)
    assert e.value.status == fd.FD_ERR_ARG


def test_forward_before_model_is_a_state_error(fd):
    w = small()
    with fd.Grid.from_workload(w) as g:
        rec = np.zeros((w["nt"], len(w["rec"])), np.float32)
        assert g.forward(w["src"], w["wavelet"], w["rec"], rec) == fd.FD_ERR_STATE


def test_unstable_time_step_is_rejected(fd):
    w = small()
    w["dt"] = 0.6 * w["h"] / 1.5  # above the SO 4 limit 0.5
    with fd.Grid.from_workload(w) as g:
        with pytest.raises(fd.FDError) as e:
            g.set_model(w["v"])
        assert e.value.status == fd.FD_ERR_UNSTABLE
        assert g.info()["cfl_limit"] == pytest.approx(0.5, rel=1e-12)


def test_bad_model_values_are_rejected(fd):
    w = small()
    for bad in (np.nan, 0.0, -1.0, np.inf):
        v = w["v"].copy()
        v[3, 4, 5] = bad
        with fd.Grid.from_workload(w) as g:
            with pytest.raises(fd.FDError) as e:
                g.set_model(v)
            assert e.value.status == fd.FD_ERR_ARG


def test_points_outside_the_box_are_rejected(fd):
    w = small()
    with fd.Grid.from_workload(w) as g:
        g.set_model(w["v"])
        rec = np.zeros((w["nt"], 1), np.float32)
        edge = (w["n"][0] - 1) * w["h"]
        for bad in ([[edge + 0.01, 10, 10]], [[-0.01, 10, 10]], [[10, 10, edge * 2]]):
            assert g.forward(w["src"], w["wavelet"], bad, rec) == fd.FD_ERR_ARG
        # on the far face itself is inside
        assert g.forward(w["src"], w["wavelet"], [[edge, edge, edge]], rec) == fd.FD_OK


def test_non_finite_receivers_are_reported(fd):
    w = small()
    wav = w["wavelet"].copy()
    wav[3, 0] = np.inf
    with fd.Grid.from_workload(w) as g:
        g.set_model(w["v"])
        rec = np.zeros((w["nt"], len(w["rec"])), np.float32)
        assert g.forward(w["src"], wav, w["rec"], rec) == fd.FD_ERR_NONFINITE


def test_bounded_wait_times_out_and_grid_recovers(fd):
    w = small()
    with fd.Grid.from_workload(w) as g:
        g.set_model(w["v"])
        ref = np.zeros((w["nt"], len(w["rec"])), np.float32)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], ref), "clean run")
        g.set_debug(fd.FD_DEBUG_SPIN_LIMIT, 2_000_000)
        g.set_debug(fd.FD_DEBUG_SKIP_PLANE, 5)
        rec = np.zeros_like(ref)
        assert g.forward(w["src"], w["wavelet"], w["rec"], rec) == fd.FD_ERR_TIMEOUT
        msg = fd.fd_last_error().decode()
        assert "wait" in msg
        g.set_debug(fd.FD_DEBUG_SKIP_PLANE, -1)
        rec2 = np.zeros_like(ref)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec2), "after recovery")
        np.testing.assert_array_equal(rec2, ref)


def test_injected_allocation_failure_reports_oom(fd):
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2312_13094_gb300 import binding as fd\n"
            "try:\n"
            "    fd.Grid((16, 16, 16), 10.0, 8, 4, 1.0, 5)\n"
            "    print('created')\n"
            "except fd.FDError as e:\n"
            "    print('status', e.status)\n") % ROOT
    env = dict(os.environ, FD_FAULT_ALLOC_AT="2")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert "status 3" in out.stdout
