"""Learned per-cell weights on the GPU: network inference, loss gradient and
Adam against the FP64 reference network; the per-cell stencil against the
oracle; and the trained network's gain over the plain coarse stencil.

Tolerances: inference and loss rel. 1e-5 (FP32 dense layers of width 64);
gradient rel. L2 1e-4 (FP32 sums over the samples of a batch).
"""
import os

import numpy as np
import pytest

import oracle
from oracle import mlp
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


@pytest.fixture(scope="module")
def learned(fd):
    from paper_2312_13094_gb300 import learned as lr
    return lr


def samples(n, seed):
    rng = np.random.default_rng(seed)
    X = mlp.features(rng.uniform(1.5, 4.5, n), 20.0, 1.6, 12.0)
    T = rng.standard_normal((n, 4))
    y = rng.standard_normal(n) * 0.3
    w = rng.uniform(0.5, 2.0, n)
    return np.ascontiguousarray(np.concatenate([X, T, y[:, None], w[:, None]], 1), np.float32)


def test_inference_matches_reference(learned):
    th = mlp.init_params(5, scale_out=0.8).astype(np.float32)
    net = learned.Network(th)
    X = mlp.features(np.linspace(1.5, 4.5, 301), 20.0, 1.6, 12.0).astype(np.float32)
    got = net.coefficients(X)
    ref = mlp.coefficients(th.astype(np.float64), X.astype(np.float64), oracle.fd_coefficients(4))
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    net.close()


@pytest.mark.parametrize("n", [1, 127, 1000, 5003])
def test_loss_gradient_matches_reference(learned, n):
    th = mlp.init_params(6, scale_out=0.8).astype(np.float32)
    net = learned.Network(th)
    S = samples(n, n)
    loss, g = net.loss_grad(S)
    rl, rg = mlp.loss_grad(th.astype(np.float64), S.astype(np.float64),
                           oracle.fd_coefficients(4))
    assert abs(loss - rl) <= 1e-5 * abs(rl)
    assert np.linalg.norm(g - rg) <= 1e-4 * np.linalg.norm(rg)
    net.close()


def test_adam_step_matches_reference(fd, learned):
    th = mlp.init_params(7, scale_out=0.8).astype(np.float32)
    net = learned.Network(th)
    S = samples(777, 8)
    ref = th.astype(np.float64)
    m = np.zeros_like(ref)
    v = np.zeros_like(ref)
    for t in range(1, 4):
        _, g = net.loss_grad(S)
        fd.check(fd.fd_mlp_adam_step(net.handle, 1e-3), "adam")
        _, rg = mlp.loss_grad(ref, S.astype(np.float64), oracle.fd_coefficients(4))
        ref, m, v = mlp.adam(ref, rg, m, v, t, lr=1e-3)
    assert np.abs(net.params() - ref).max() <= 2e-6
    net.close()


def _percell_workload(nt=40):
    n = (30, 26, 22)
    h = 20.0
    v = wl.layered_model(n, h, 23, vmin=1.5, vmax=4.5)
    dt = 0.3 * h / 4.5
    ext = [(d - 1) * h for d in n]
    src = np.array([[0.5 * ext[0], 0.5 * ext[1], 0.3 * ext[2]]])
    rec = np.array([[x, 0.5 * ext[1], 0.8 * ext[2]] for x in np.linspace(0, ext[0], 9)])
    return dict(n=n, h=h, space_order=8, nbl=6, dt=dt, nt=nt, v=v, src=src, rec=rec,
                wavelet=wl.ricker(nt, dt, 12.0).reshape(nt, 1), f0=12.0)


def _oracle_percell(w, c_pad):
    og = oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=4, nbl=w["nbl"])
    pc = np.zeros(og.padded_shape + (5,))
    pc[..., 1:] = c_pad
    pc[..., 0] = -2.0 * c_pad.sum(-1)
    out = oracle.forward(og, 1.0 / w["v"].astype(np.float64) ** 2, w["nt"], w["src"],
                         w["wavelet"], w["rec"], percell=pc.reshape(-1, 5))
    return og, out["rec"]


def test_per_cell_weights_match_oracle(fd):
    w = _percell_workload()
    rng = np.random.default_rng(1)
    cT = oracle.fd_coefficients(4)
    cphys = (cT[1:] * (1 + 0.2 * rng.uniform(-1, 1, w["v"].shape + (4,)))).astype(np.float32)
    with fd.Grid.from_workload(w) as g:
        g.set_model(w["v"])
        fd.check(fd.fd_set_coefficients(g.handle, cphys.ctypes.data, fd.FD_COEF_PER_CELL),
                 "per-cell")
        rec = np.zeros((w["nt"], len(w["rec"])), np.float32)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec), "fd_forward")
    og = oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=4, nbl=w["nbl"])
    Nz, Ny, Nx = og.padded_shape
    nb = w["nbl"]
    iz = np.clip(np.arange(Nz) - nb, 0, w["n"][2] - 1)
    iy = np.clip(np.arange(Ny) - nb, 0, w["n"][1] - 1)
    ix = np.clip(np.arange(Nx) - nb, 0, w["n"][0] - 1)
    c_pad = cphys.astype(np.float64)[iz][:, iy][:, :, ix]
    _, ref = _oracle_percell(w, c_pad)
    assert np.linalg.norm(rec - ref) / np.linalg.norm(ref) <= 1e-5


def test_learned_weights_on_a_grid_match_oracle(fd, learned):
    w = _percell_workload()
    th = mlp.init_params(9, scale_out=1.0).astype(np.float32)
    net = learned.Network(th)
    with fd.Grid.from_workload(w) as g:
        g.set_model(w["v"])
        fd.check(fd.fd_set_learned_coefficients(g.handle, net.handle, w["f0"]), "learned")
        rec = np.zeros((w["nt"], len(w["rec"])), np.float32)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec), "fd_forward")
    og = oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=4, nbl=w["nbl"])
    v_pad = 1.0 / np.sqrt(oracle.pad_model(og, 1.0 / w["v"].astype(np.float64) ** 2))
    X = mlp.features(v_pad, w["h"], w["dt"], w["f0"]).reshape(-1, 4)
    c_pad = mlp.coefficients(th.astype(np.float64), X, oracle.fd_coefficients(4))
    _, ref = _oracle_percell(w, c_pad.reshape(og.padded_shape + (4,)))
    assert np.linalg.norm(rec - ref) / np.linalg.norm(ref) <= 1e-5
    net.close()


@pytest.mark.parametrize("nodes", [2, 64, 256])
def test_learned_table_on_a_grid_matches_oracle(fd, learned, nodes):
    """Table mode: the network at `nodes` Courant numbers over the model's
    range, interpolated per point, against the oracle's per-cell forward with
    the FP64 table weights of every padded cell."""
    w = _percell_workload()
    th = mlp.init_params(9, scale_out=1.0).astype(np.float32)
    net = learned.Network(th)
    with fd.Grid.from_workload(w) as g:
        g.set_model(w["v"])
        fd.check(fd.fd_set_learned_table(g.handle, net.handle, w["f0"], nodes), "table")
        rec = np.zeros((w["nt"], len(w["rec"])), np.float32)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec), "fd_forward")
    og = oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=4, nbl=w["nbl"])
    v_pad = 1.0 / np.sqrt(oracle.pad_model(og, 1.0 / w["v"].astype(np.float64) ** 2))
    v = w["v"].astype(np.float64)
    lo, hi = v.min() * w["dt"] / w["h"], v.max() * w["dt"] / w["h"]
    c_pad = mlp.table_coefficients(th.astype(np.float64), v_pad * w["dt"] / w["h"], w["h"],
                                   w["dt"], w["f0"], nodes, lo, hi, oracle.fd_coefficients(4))
    _, ref = _oracle_percell(w, c_pad)
    assert np.linalg.norm(rec - ref) / np.linalg.norm(ref) <= 1e-5
    net.close()


def test_table_mode_schedules_tiles_and_tuner_agree_bitwise(fd, learned):
    """Table-weight steps on column waves and equal shares, on three tiles,
    and a long run that tunes the grid on its own (table) kernel: the same
    receivers bit for bit."""
    w = _percell_workload()
    net = learned.Network(mlp.init_params(9, scale_out=1.0).astype(np.float32))

    def rec_with(sched, tile, nt=None):
        ww = w if nt is None else _percell_workload(nt)
        with fd.Grid.from_workload(ww) as g:
            if tile is not None:
                g.set_tile(tile[0], tile[1], 0)
            g.set_schedule(sched)
            g.set_model(ww["v"])
            fd.check(fd.fd_set_learned_table(g.handle, net.handle, ww["f0"], 64), "table")
            rec = np.zeros((ww["nt"], len(ww["rec"])), np.float32)
            fd.check(g.forward(ww["src"], ww["wavelet"], ww["rec"], rec), "fd_forward")
            return rec

    ref = rec_with(fd.FD_SCHED_SHARES, None)
    assert np.abs(ref).max() > 0
    for sched, tile in ((fd.FD_SCHED_WAVES, (64, 16)), (fd.FD_SCHED_WAVES, (32, 8)),
                        (fd.FD_SCHED_WAVES, None)):
        np.testing.assert_array_equal(rec_with(sched, tile), ref)
    long_ref = rec_with(fd.FD_SCHED_SHARES, None, nt=420)
    np.testing.assert_array_equal(rec_with(fd.FD_SCHED_AUTO, None, nt=420), long_ref)
    net.close()


def test_table_mode_is_refused_by_the_adjoint_and_reset_by_plain_weights(fd, learned):
    w = _percell_workload()
    net = learned.Network(mlp.init_params(9, scale_out=1.0).astype(np.float32))
    with fd.Grid.from_workload(w) as g:
        g.set_model(w["v"])
        assert fd.fd_set_learned_table(g.handle, net.handle, w["f0"], 1) == fd.FD_ERR_ARG
        fd.check(fd.fd_set_learned_table(g.handle, net.handle, w["f0"], 16), "table")
        grad = np.zeros(g.phys_shape, np.float32)
        d = np.zeros((w["nt"], len(w["rec"])), np.float32)
        st, _ = g.adjoint_gradient(w["src"], w["wavelet"], w["rec"], d, 4, grad)
        assert st == fd.FD_ERR_STATE
        fd.check(fd.fd_set_coefficients(g.handle, None, fd.FD_COEF_TAYLOR), "taylor")
        plain = np.zeros((w["nt"], len(w["rec"])), np.float32)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], plain), "fd_forward")
    with fd.Grid.from_workload(w) as g2:
        g2.set_model(w["v"])
        ref = np.zeros_like(plain)
        fd.check(g2.forward(w["src"], w["wavelet"], w["rec"], ref), "fd_forward")
    np.testing.assert_array_equal(plain, ref)
    net.close()


def test_training_lowers_the_coarse_step_error_on_held_out_models(learned):
    """What the trained network gains over plain SO 8 weights: on fine-run
    samples of models it has not seen (fine 96^3 SO 16 vs coarse 48^3 at
    twice h and dt, 12 Hz), the coarse one-step error (the quantity the
    weights set) is lower than with the Taylor weights.  The receiver errors
    of plain and learned coarse solves are reported; in this small box they
    are dominated by boundary-layer differences near the surface receivers,
    which no per-cell weights can remove, so they are not asserted here (the
    512^3 / 256^3 workload measures them over km of propagation)."""
    import torch
    kw = dict(n=96, nt=700, nbl=16, f_hz=12.0, rec_every=4)

    def data(seeds):
        out = []
        for s in seeds:
            fine, coarse = learned.pair(s, **kw)
            out.append(learned.training_samples(fine, coarse, ncell=8192, ntimes=6, seed=s))
        S = torch.cat(out)
        g = torch.Generator().manual_seed(0)
        return S[torch.randperm(S.shape[0], generator=g).to(S.device)]

    train = data(range(100, 108))
    held = data((200, 201))
    net = learned.Network(learned.init_params(0, scale_out=0.0))
    plain_held = net.loss_grad(held)[0]
    l0 = net.loss_grad(train)[0]
    l1 = net.train(train, epochs=40, batch=16384, lr=5e-4)
    learned_held = net.loss_grad(held)[0]
    assert l1 < l0, (l0, l1)
    assert learned_held < 0.97 * plain_held, (plain_held, learned_held)
    rows = []
    for s in (200, 201):
        fine, coarse = learned.pair(s, **kw)
        ref = learned.run_forward(fine)[0][::2]
        rows.append((learned.rel_l2(learned.run_forward(coarse)[0], ref),
                     learned.rel_l2(learned.run_forward(coarse, net=net.handle)[0], ref)))
    print("one-step error plain/learned", plain_held, learned_held, "receivers", rows)
    assert all(np.isfinite(r).all() for r in rows)
    net.close()


NET = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2312_13094_gb300", "data", "learned_coarse_h20_so8_12hz.fdck")


@pytest.mark.skipif(not os.path.exists(NET), reason="trained network not stored")
def test_stored_network_meets_the_criterion_where_plain_fails(learned):
    """What the trained network gains at the receivers, at the configured
    size: the network shipped with the package (one-step training on 200
    models, then the rollout fine-tune of its output bias on six of them,
    `bench.py --workload learned --finetune 6`) on three held-out models
    (fine 512^3 h 10 m SO 16 dt 0.8 ms vs coarse 256^3 h 20 m SO 8 dt 1.6 ms,
    receiver relative L2 against the fine solve).  Model 10014 is the plain
    coarse solve's worst case, 10007 another that plain misses, 10011 one
    where plain is better than learned: every learned solve stays within
    1 %, plain misses it, and learned is better on the worst and the mean."""
    from paper_2312_13094_gb300 import checkpoint
    params, meta = checkpoint.load(NET)
    net = learned.Network(params)
    rows = []
    for s in (10014, 10007, 10011):
        fine, coarse = learned.pair(s)
        ref = learned.run_forward(fine, timed=False)[0][::2]
        plain = learned.rel_l2(learned.run_forward(coarse, timed=False)[0], ref)
        lrn = learned.rel_l2(learned.run_forward(coarse, net=net.handle, table=256,
                                                 timed=False)[0], ref)
        rows.append((s, plain, lrn))
    print("held-out receiver rel. L2 (seed, plain, learned):", rows)
    assert all(r[2] <= 0.01 for r in rows), rows
    assert max(r[1] for r in rows) > 0.01
    assert max(r[2] for r in rows) < max(r[1] for r in rows)
    assert np.mean([r[2] for r in rows]) < np.mean([r[1] for r in rows])
    net.close()
