"""The allocation-free forward entry point (fd_forward_noalloc).

It serves callers that may not allocate device memory at call time (for
example under another framework's memory pool, or with a fixed device
footprint): its scratch lives in a static device array of the library.  Two
calls in a row must reproduce the regular entry point (fd_create_grid +
fd_set_model + fd_forward) within the parity tolerance of the other tests,
whether this file runs alone in a fresh process or after the rest.
"""
import ctypes

import numpy as np
import pytest

from paper_2312_13094_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def fd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2312_13094_gb300 import build
    build.build()
    from paper_2312_13094_gb300 import binding
    return binding


def _workload(so, n, nt, nbl):
    h = 10.0
    v = wl.layered_model(n, h, 31, vmin=1.5, vmax=3.0).astype(np.float32)
    dt = 0.35 * h / float(v.max())
    ext = [(d - 1) * h for d in n]
    src = np.array([[0.4 * ext[0], 0.55 * ext[1], 0.5 * ext[2]]])
    rec = np.array([[x, 0.5 * ext[1], 2.5 * h] for x in np.linspace(0.0, ext[0], 11)])
    return dict(n=n, h=h, space_order=so, nbl=nbl, dt=dt, nt=nt, v=v, src=src, rec=rec,
                wavelet=wl.ricker(nt, dt, 25.0).reshape(nt, 1))


def _regular(fd, w):
    with fd.Grid.from_workload(w) as g:
        g.set_model(w["v"])
        rec = np.zeros((w["nt"], len(w["rec"])), np.float32)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec), "fd_forward")
    return rec


def _noalloc(fd, w):
    import torch
    desc = fd.fd_grid_desc(*[int(x) for x in w["n"]], float(w["h"]), int(w["space_order"]),
                           int(w["nbl"]), float(w["dt"]), int(w["nt"]), 0, None)
    v = torch.from_numpy(w["v"]).cuda()
    wav = torch.from_numpy(np.ascontiguousarray(w["wavelet"])).cuda()
    out = torch.full((w["nt"], len(w["rec"])), float("nan"), device="cuda")
    s, r = fd.Points(w["src"]), fd.Points(w["rec"])
    st = fd.fd_forward_noalloc(ctypes.byref(desc), v.data_ptr(), fd.FD_MODEL_VP_KMS, s.ref(),
                               wav.data_ptr(), r.ref(), out.data_ptr())
    fd.check(st, "fd_forward_noalloc")
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("so,n,nt,nbl", [(8, (40, 33, 29), 60, 6), (4, (24, 24, 24), 40, 10)])
def test_two_calls_match_the_regular_entry_point(fd, so, n, nt, nbl):
    w = _workload(so, n, nt, nbl)
    ref = _regular(fd, w)
    for _ in range(2):
        got = _noalloc(fd, w)
        assert np.isfinite(got).all()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL


def test_grid_above_the_scratch_limit_is_rejected(fd):
    desc = fd.fd_grid_desc(400, 400, 400, 10.0, 8, 10, 1.0, 10, 0, None)
    import torch
    v = torch.full((400, 400, 400), 2.0, device="cuda")
    st = fd.fd_forward_noalloc(ctypes.byref(desc), v.data_ptr(), fd.FD_MODEL_VP_KMS, None, None,
                               None, None)
    assert st == fd.FD_ERR_ARG
    assert "limit" in fd.fd_last_error().decode()


def test_host_arrays_are_rejected(fd):
    w = _workload(4, (20, 20, 20), 10, 4)
    desc = fd.fd_grid_desc(20, 20, 20, 10.0, 4, 4, float(w["dt"]), 10, 0, None)
    st = fd.fd_forward_noalloc(ctypes.byref(desc), w["v"].ctypes.data, fd.FD_MODEL_VP_KMS, None,
                               None, None, None)
    assert st == fd.FD_ERR_ARG
