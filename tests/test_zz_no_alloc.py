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


def test_calls_allocate_nothing_on_a_caller_stream(fd):
    """Several sources and receivers on a stream the caller created: the
    entry point matches fd_forward on the same stream, its calls leave the
    library's device allocation count and the device's free memory
    unchanged, and a call made while the library's next allocation is set to
    fail (FD_FAULT_ALLOC_AT) still succeeds."""
    import os
    import torch
    w = _workload(8, (36, 30, 28), 50, 5)
    ext = [(d - 1) * w["h"] for d in w["n"]]
    w["src"] = np.array([[0.3 * ext[0], 0.4 * ext[1], 0.5 * ext[2]],
                         [0.71 * ext[0], 0.22 * ext[1], 0.35 * ext[2]],
                         [ext[0], 0.0, 0.8 * ext[2]]])
    f = [25.0, 18.0, 30.0]
    w["wavelet"] = np.ascontiguousarray(
        np.stack([wl.ricker(w["nt"], w["dt"], fh) for fh in f], 1), np.float32)
    w["rec"] = np.array([[x, y, 2.5 * w["h"]] for x in np.linspace(0.0, ext[0], 8)
                         for y in np.linspace(0.0, ext[1], 5)])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with fd.Grid.from_workload(w, stream=stream.cuda_stream) as g:
            g.set_model(w["v"])
            ref = np.zeros((w["nt"], len(w["rec"])), np.float32)
            fd.check(g.forward(w["src"], w["wavelet"], w["rec"], ref), "fd_forward")
        desc = fd.fd_grid_desc(*[int(x) for x in w["n"]], float(w["h"]), int(w["space_order"]),
                               int(w["nbl"]), float(w["dt"]), int(w["nt"]), 0,
                               stream.cuda_stream)
        v = torch.from_numpy(w["v"]).cuda()
        wav = torch.from_numpy(w["wavelet"]).cuda()
        outs = [torch.full((w["nt"], len(w["rec"])), float("nan"), device="cuda")
                for _ in range(3)]
        s, r = fd.Points(w["src"]), fd.Points(w["rec"])
        torch.cuda.synchronize()

        def call(out):
            st = fd.fd_forward_noalloc(ctypes.byref(desc), v.data_ptr(), fd.FD_MODEL_VP_KMS,
                                       s.ref(), wav.data_ptr(), r.ref(), out.data_ptr())
            fd.check(st, "fd_forward_noalloc")

        call(outs[0])  # loads the kernels the call uses (lazy module loading)
        torch.cuda.synchronize()
        allocs0 = fd.fd_alloc_count()
        free0 = torch.cuda.mem_get_info()[0]
        call(outs[1])
        key = "FD_FAULT_ALLOC_AT"
        old = os.environ.get(key)
        os.environ[key] = str(fd.fd_alloc_count() + 1)
        try:
            call(outs[2])
        finally:
            if old is None:
                del os.environ[key]
            else:
                os.environ[key] = old
        torch.cuda.synchronize()
        assert fd.fd_alloc_count() == allocs0
        assert torch.cuda.mem_get_info()[0] == free0
    for out in outs:
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL
