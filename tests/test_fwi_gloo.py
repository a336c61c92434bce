"""Full-waveform-inversion loop (host logic) and the FP64 reference of its
model update, on CPU: properties of the normalised descent step, the
backtracking of the loop, and the loop over two gloo ranks with FP64 oracle
gradients equal to the serial loop."""
import socket

import numpy as np
import pytest

from oracle import fwi as ofwi
from paper_2312_13094_gb300 import fwi


def test_descent_step_moves_the_largest_entry_by_the_step():
    rng = np.random.default_rng(0)
    m = rng.uniform(0.1, 0.4, 500)
    g = rng.standard_normal(500)
    out, alpha = ofwi.descent_step(m, g, 0.03, 0.0, 1.0)
    d = out - m
    # the largest |change| is step * max|m| and sits where |g| is largest
    k = int(np.argmax(np.abs(g)))
    assert np.isclose(np.abs(d).max(), 0.03 * m.max(), rtol=1e-12)
    assert np.isclose(abs(d[k]), 0.03 * m.max(), rtol=1e-12)
    # every change points against the gradient, in proportion to it
    assert np.all(d * g <= 0)
    np.testing.assert_allclose(d, -alpha * g, rtol=1e-12, atol=1e-15)


def test_descent_step_bounds_zero_gradient_and_zero_step():
    m = np.array([0.2, 0.25, 0.3])
    g = np.array([10.0, -10.0, 0.0])
    out, _ = ofwi.descent_step(m, g, 0.5, 0.15, 0.33)
    assert out.min() >= 0.15 and out.max() <= 0.33
    assert out[0] == 0.15 and out[1] == 0.33 and out[2] == 0.3
    same, a0 = ofwi.descent_step(m, np.zeros(3), 0.5, 0.0, 1.0)
    assert a0 == 0.0 and np.array_equal(same, m)
    same, a0 = ofwi.descent_step(m, g, 0.0, 0.0, 1.0)
    assert a0 == 0.0 and np.array_equal(same, m)


def test_small_step_lowers_a_quadratic_misfit():
    rng = np.random.default_rng(1)
    target = rng.uniform(0.2, 0.3, 64)
    m = rng.uniform(0.2, 0.3, 64)
    J = 0.5 * np.sum((m - target) ** 2)
    out, _ = ofwi.descent_step(m, m - target, 0.01, 0.0, 1.0)
    assert 0.5 * np.sum((out - target) ** 2) < J


def _np_update(m, g, step):
    import torch
    out, _ = ofwi.descent_step(m.numpy(), g.numpy(), step, 0.0, 10.0)
    return torch.from_numpy(out)


def test_loop_backtracks_on_overshoot_and_stops_at_the_optimum():
    torch = pytest.importorskip("torch")
    target = torch.tensor([3.0, 1.0], dtype=torch.float64)

    def grad(s, m):  # one shot, J = 1/2 |m - target|^2
        return (m - target).clone(), float(0.5 * ((m - target) ** 2).sum())

    m0 = torch.tensor([1.0, 1.0], dtype=torch.float64)
    # step 2: alpha = 2 * max|m| / max|g| = 1 -> lands on target[0] exactly
    m, h = fwi.fwi_loop(m0, 1, grad, _np_update, iterations=3, step=2.0, dist=None)
    assert h["loss"][1] == 0.0 and h["step"] == [2.0]
    assert torch.equal(m, target)
    # from the optimum no step lowers the misfit: stop without accepting
    m2, h2 = fwi.fwi_loop(target, 1, grad, _np_update, iterations=3, step=0.1)
    assert h2["step"] == [] and torch.equal(m2, target) and h2["evals"] == 1 + 4
    # step 8 overshoots (alpha 4: misfit 18), step 4 only mirrors (alpha 2: misfit
    # unchanged, not accepted), step 2 lands on the target: two halvings
    m3, h3 = fwi.fwi_loop(m0, 1, grad, _np_update, iterations=1, step=8.0)
    assert h3["step"] == [2.0]
    assert h3["loss"][-1] < h3["loss"][0]


def _problem():
    from paper_2312_13094_gb300 import workloads as wl
    n = (10, 9, 8)
    h = 10.0
    v_true = wl.layered_model(n, h, 21, vmin=1.8, vmax=2.4)
    nt = 24
    dt = 0.3 * h / 2.6
    wav = wl.ricker(nt, dt, 40.0).reshape(nt, 1)
    rec = np.array([[x, 40.0, 60.0] for x in np.linspace(0.0, 90.0, 5)])
    return n, h, v_true, nt, dt, wav, rec


def _src(s):
    return np.array([[10.0 + 15.0 * s, 30.0 + 5.0 * s, 10.0]])


def _shots():
    import oracle
    n, h, v_true, nt, dt, wav, rec = _problem()
    og = oracle.Grid(n=n, h=h, dt=dt, R=2, nbl=3)
    m_true = 1.0 / v_true.astype(np.float64) ** 2
    d_obs = [oracle.forward(og, m_true, nt, _src(s), wav, rec)["rec"] for s in range(5)]

    def grad(s, m):
        import torch
        g, loss, _ = oracle.adjoint_gradient(og, m.numpy(), nt, _src(s), wav, rec,
                                             d_obs=d_obs[s])
        return torch.from_numpy(np.ascontiguousarray(g)), loss

    m0 = np.full(v_true.shape, 1.0 / 2.1 ** 2)
    return grad, m0, m_true


def _rank_main(rank, world, port):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            world_size=world, rank=rank)
    try:
        grad, m0, _ = _shots()
        m, h = fwi.fwi_loop(torch.from_numpy(m0), 5, grad, _np_update, iterations=3,
                            step=0.02, dist=dist)
        parts = [None] * world
        dist.all_gather_object(parts, (m.numpy(), h))
        if rank == 0:
            ref_m, ref_h = fwi.fwi_loop(torch.from_numpy(m0), 5, grad, _np_update,
                                        iterations=3, step=0.02, dist=None)
            for pm, ph in parts:
                np.testing.assert_array_equal(pm, parts[0][0])
                np.testing.assert_allclose(pm, ref_m.numpy(), rtol=1e-12, atol=0)
                assert ph["step"] == ref_h["step"]
                np.testing.assert_allclose(ph["loss"], ref_h["loss"], rtol=1e-12)
            losses = parts[0][1]["loss"]
            assert len(losses) == 4
            assert all(b < a for a, b in zip(losses, losses[1:]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_fwi_loop_over_two_gloo_ranks_equals_the_serial_loop():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    oracle.build()
    mp.spawn(_rank_main, args=(2, _free_port()), nprocs=2, join=True)
