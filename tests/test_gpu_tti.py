"""GPU parity of the anisotropic acoustic (TTI) path (fd_tti_* through the C
ABI) against the FP64 oracle (oracle/tti.py) on the same seeded inputs.

Tolerance: relative L2 <= 1e-5 on receivers and wavefields (FP32 against
FP64), as for the isotropic path; a single step from a random state is
compared element by element."""
import numpy as np
import pytest

import oracle
from oracle import tti as otti
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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def ogrid(w):
    return oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=w["space_order"] // 2, nbl=w["nbl"])


def model(w):
    return w["v"], w["eps"], w["delta"], w["theta"], w["phi"]


def run_gpu(fd, w):
    with fd.TtiGrid.from_workload(w) as g:
        g.set_model(*model(w))
        rec = np.zeros((w["nt"], len(w["rec"])), np.float32)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec), "fd_tti_forward")
        shp = g.padded_shape
        p, q = np.zeros(shp, np.float32), np.zeros(shp, np.float32)
        g.get_state(p=p, q=q)
    return rec, p, q


@pytest.mark.parametrize("so", [2, 4, 8, 12, 16])
def test_forward_matches_the_oracle(fd, so):
    w = wl.tti_workload(n=(37, 29, 26), so=so, nbl=5, nt=45)
    rec, p, q = run_gpu(fd, w)
    ref = otti.forward(ogrid(w), *model(w), w["nt"], w["src"], w["wavelet"], w["rec"])
    assert np.abs(ref["rec"]).max() > 0
    assert rel(rec, ref["rec"]) <= TOL, rel(rec, ref["rec"])
    assert rel(p, ref["p"]) <= TOL, rel(p, ref["p"])
    assert rel(q, ref["q"]) <= TOL, rel(q, ref["q"])


@pytest.mark.parametrize("so", [4, 6, 8])
def test_tall_grid_in_several_z_chunks_matches_the_oracle(fd, so):
    """A grid tall enough that the launch cuts every tile column into several
    z chunks (each with its own 2R-plane prologue), ragged in x and y."""
    w = wl.tti_workload(n=(35, 21, 84), so=so, nbl=4, nt=40, seed=5)
    rec, p, q = run_gpu(fd, w)
    ref = otti.forward(ogrid(w), *model(w), w["nt"], w["src"], w["wavelet"], w["rec"])
    assert rel(rec, ref["rec"]) <= TOL, rel(rec, ref["rec"])
    assert rel(p, ref["p"]) <= TOL, rel(p, ref["p"])
    assert rel(q, ref["q"]) <= TOL, rel(q, ref["q"])


def test_single_step_from_random_state_elementwise(fd):
    w = wl.tti_workload(n=(41, 23, 35), so=8, nbl=6, nt=1)
    g0 = ogrid(w)
    shp = g0.padded_shape
    st = [wl.random_state(shp, 40 + i).astype(np.float32) for i in range(4)]
    ref = otti.forward(g0, *model(w), 1, np.zeros((0, 3)), np.zeros((1, 0)), np.zeros((0, 3)),
                       state=st)
    with fd.TtiGrid.from_workload(w) as g:
        g.set_model(*model(w))
        g.set_state(*st)
        fd.check(g.propagate(0, 1), "fd_tti_propagate")
        out = [np.zeros(shp, np.float32) for _ in range(4)]
        g.get_state(*out)
    np.testing.assert_array_equal(out[0], st[1])  # p^n becomes p^{n-1}
    np.testing.assert_array_equal(out[2], st[3])
    for got, want in ((out[1], ref["p"]), (out[3], ref["q"])):
        assert np.abs(got - want).max() <= 2e-6 * np.abs(want).max()


def test_isotropic_limit_matches_the_acoustic_kernel(fd):
    """eps = delta = 0 with any tilt: p follows the isotropic equation, so the
    TTI kernel and the acoustic kernel agree to FP32 rounding."""
    w = wl.tti_workload(n=(33, 30, 28), so=8, nbl=5, nt=50)
    zero = np.zeros_like(w["eps"])
    w["eps"], w["delta"] = zero, zero
    rec_t, p_t, _ = run_gpu(fd, w)
    with fd.Grid.from_workload(w) as g:
        g.set_model(w["v"])
        rec_a = np.zeros_like(rec_t)
        u = np.zeros(g.phys_shape, np.float32)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec_a, u), "fd_forward")
    nb = w["nbl"]
    assert rel(rec_t, rec_a) <= TOL
    assert rel(p_t[nb:-nb, nb:-nb, nb:-nb], u) <= TOL


def test_pieces_equal_one_run_and_host_device_buffers_agree(fd):
    import torch
    w = wl.tti_workload(n=(30, 28, 26), so=4, nbl=4, nt=30)
    rec, p, _ = run_gpu(fd, w)
    with fd.TtiGrid.from_workload(w) as g:
        g.set_model(*(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in model(w)))
        a = torch.zeros((12, len(w["rec"])), device="cuda")
        b = torch.zeros((18, len(w["rec"])), device="cuda")
        wav = torch.from_numpy(w["wavelet"]).cuda()
        fd.check(g.propagate(0, 12, w["src"], wav, w["rec"], a), "p1")
        fd.check(g.propagate(12, 18, w["src"], wav, w["rec"], b), "p2")
        p2 = torch.zeros(g.padded_shape, device="cuda")
        g.get_state(p=p2)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(torch.cat([a, b]).cpu().numpy(), rec)
    np.testing.assert_array_equal(p2.cpu().numpy(), p)


def test_errors(fd):
    w = wl.tti_workload(n=(20, 20, 20), so=8, nbl=2, nt=5)
    with fd.TtiGrid.from_workload(w) as g:
        rec = np.zeros((w["nt"], len(w["rec"])), np.float32)
        st = g.forward(w["src"], w["wavelet"], w["rec"], rec)
        assert st == fd.FD_ERR_STATE
        bad = w["eps"].copy()
        bad[3, 4, 5] = -0.6
        with pytest.raises(fd.FDError) as e:
            g.set_model(w["v"], bad, w["delta"], w["theta"], w["phi"])
        assert e.value.status == fd.FD_ERR_ARG
        with pytest.raises(fd.FDError) as e:
            g.set_model(w["v"] * 3.0, w["eps"], w["delta"], w["theta"], w["phi"])
        assert e.value.status == fd.FD_ERR_UNSTABLE
        g.set_model(*model(w))
        st = g.forward(np.array([[1e4, 0.0, 0.0]]), w["wavelet"], w["rec"], rec)
        assert st == fd.FD_ERR_ARG
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec), "fd_tti_forward")
