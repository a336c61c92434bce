"""GPU parts of the full-waveform-inversion loop: the device model update
(fd_descent_step) against its FP64 reference, and a few iterations of the loop
on libfd adjoint gradients."""
import numpy as np
import pytest

from oracle import fwi as ofwi
from paper_2312_13094_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2312_13094_gb300 import build
    build.build()
    from paper_2312_13094_gb300 import binding
    return binding


@pytest.mark.parametrize("n", [1, 7, 1000, 1234567])
def test_descent_step_matches_the_reference(fd, n):
    """FP32 update against the FP64 definition: within a few float roundings
    of the model's scale; bounds clip some entries on both sides."""
    import torch
    rng = np.random.default_rng(n)
    m = rng.uniform(0.05, 0.45, n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    lo, hi = 0.06, 0.44
    ref, alpha_ref = ofwi.descent_step(m, g, 0.1, lo, hi)
    md = torch.from_numpy(m).cuda()
    gd = torch.from_numpy(g).cuda()
    alpha = fd.descent_step(md, gd, 0.1, lo, hi)
    got = md.cpu().numpy()
    assert abs(alpha - alpha_ref) <= 1e-12 * alpha_ref
    assert np.abs(got - ref).max() <= 4e-7 * np.abs(m).max()
    assert got.min() >= np.float32(lo) and got.max() <= np.float32(hi)


def test_descent_step_edge_cases(fd):
    import torch
    m = torch.full((100,), 0.25, device="cuda")
    assert fd.descent_step(m, torch.zeros(100, device="cuda"), 0.1, 0.0, 1.0) == 0.0
    assert bool((m == 0.25).all())
    assert fd.descent_step(m, torch.ones(100, device="cuda"), 0.0, 0.0, 1.0) == 0.0
    assert bool((m == 0.25).all())
    g = torch.ones(100, device="cuda")
    g[17] = float("nan")
    with pytest.raises(fd.FDError) as e:
        fd.descent_step(m, g, 0.1, 0.0, 1.0)
    assert e.value.status == fd.FD_ERR_NONFINITE
    assert bool((m == 0.25).all())
    with pytest.raises(fd.FDError) as e:
        fd.descent_step(torch.zeros(10), torch.zeros(10), 0.1, 0.0, 1.0)  # host arrays
    assert e.value.status == fd.FD_ERR_ARG
    with pytest.raises(fd.FDError):
        fd.descent_step(m, g, 0.1, 1.0, 0.0)
    empty = torch.zeros(0, device="cuda")
    assert fd.descent_step(empty, empty, 0.1, 0.0, 1.0) == 0.0


def test_fwi_iterations_lower_the_misfit(fd):
    """Three shots through a Gaussian velocity anomaly (a small version of the
    adjoint workload): three accepted iterations, each lowering the summed
    misfit, the model moving towards the true anomaly."""
    import torch
    from paper_2312_13094_gb300 import fwi
    w = wl.adjoint_256(n=40, nt=160, nbl=10)
    w0 = wl.adjoint_256(n=40, nt=160, nbl=10, anomaly=False)
    h = w["h"]
    srcs = [np.array([[x * h, 20.0 * h, 8.0 * h]]) for x in (10.0, 20.0, 30.0)]
    wav = torch.from_numpy(np.ascontiguousarray(w["wavelet"])).cuda()
    with fd.Grid.from_workload(w) as g:
        m_true = torch.from_numpy(1.0 / w["v"].astype(np.float32) ** 2).cuda()
        d_obs = []
        for s in srcs:
            g.set_model(m_true, fd.FD_MODEL_M)
            d = torch.zeros((w["nt"], len(w["rec"])), device="cuda")
            fd.check(g.forward(s, wav, w["rec"], d), "observed data")
            d_obs.append(d)
        shots = fwi.AdjointShots(g, srcs, wav, w["rec"], d_obs, n_checkpoints=8)
        m0 = torch.from_numpy(1.0 / w0["v"].astype(np.float32) ** 2).cuda()
        vmin, vmax = 1.5, 3.0
        m, hist = fwi.fwi_loop(m0, len(srcs), shots,
                               fwi.device_update(1.0 / vmax ** 2, 1.0 / vmin ** 2),
                               iterations=3, step=0.01)
    loss = hist["loss"]
    assert len(loss) == 4 and all(b < a for a, b in zip(loss, loss[1:]))
    # inside the anomaly (away from the source and receiver spikes of the
    # gradient) the update points towards the true perturbation
    core = slice(15, 25)
    dm = (m - m0).double()[core, core, core]
    dtrue = (m_true - m0).double()[core, core, core]
    assert float((dm * dtrue).sum()) > 0
