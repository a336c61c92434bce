"""GPU runs of the column-wave schedule (FD_SCHED_WAVES) against the
equal-share sweep: every point takes the same arithmetic whichever CTA runs
its column chunk, so receivers and wavefields must agree bit for bit, on
single grids (columns fewer and more than the resident CTAs) and on batches
of uneven shots; the equal-share runs are themselves held to the FP64 oracle
by the forward and batch tests."""
import numpy as np
import pytest

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


def workload(so, n, nbl, nt, seed=9):
    h = 10.0
    v = wl.layered_model(n, h, seed, vmin=1.5, vmax=3.0)
    dt = 0.35 * h / float(v.max())
    ext = [(d - 1) * h for d in n]
    src = np.array([[0.37 * ext[0], 0.61 * ext[1], 0.45 * ext[2]],
                    [0.8 * ext[0], 0.2 * ext[1], 0.9 * ext[2]]])
    rec = np.array([[x, 0.33 * ext[1], z] for x in np.linspace(0.0, ext[0], 17)
                    for z in (2.5 * h, 0.5 * ext[2], ext[2])])
    wav = np.stack([wl.ricker(nt, dt, 25.0), 0.5 * wl.ricker(nt, dt, 18.0)], 1)
    return dict(n=n, h=h, space_order=so, nbl=nbl, dt=dt, nt=nt, v=v, src=src, rec=rec,
                wavelet=np.ascontiguousarray(wav, np.float32))


def run(fd, w, sched, tile=None):
    with fd.Grid.from_workload(w) as g:
        if tile is not None:
            g.set_tile(tile[0], tile[1], 0)
        g.set_schedule(sched)
        g.set_model(w["v"])
        rec = np.zeros((w["nt"], len(w["rec"])), np.float32)
        u = np.zeros(g.phys_shape, np.float32)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec, u), "fd_forward")
        assert g.info()["schedule"] == (fd.FD_SCHED_SHARES if sched != fd.FD_SCHED_WAVES
                                        else fd.FD_SCHED_WAVES)
        return rec, u


@pytest.mark.parametrize("so", [2, 4, 8, 16])
@pytest.mark.parametrize("tile", [(64, 16), (32, 8)])
def test_waves_match_shares_on_a_ragged_grid(fd, so, tile):
    w = workload(so, (70, 45, 41), 6, 40)
    a = run(fd, w, fd.FD_SCHED_SHARES, tile)
    b = run(fd, w, fd.FD_SCHED_WAVES, tile)
    assert np.abs(a[0]).max() > 0
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("so,tile", [(8, (32, 8)), (8, (128, 8)), (16, (32, 16))])
def test_waves_match_shares_with_more_columns_than_ctas(fd, so, tile):
    """A wide, shallow grid: thousands of tile columns, several waves of
    z chunks."""
    w = workload(so, (1200, 800, 40), 10, 12)
    a = run(fd, w, fd.FD_SCHED_SHARES, tile)
    b = run(fd, w, fd.FD_SCHED_WAVES, tile)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    c = run(fd, w, fd.FD_SCHED_AUTO, tile)
    np.testing.assert_array_equal(a[0], c[0])


def test_batched_shots_under_waves_match_shares(fd):
    import torch
    shots = wl.batched_shots(nshots=6, nt=30, lo=24, hi=60, nbl=6)
    outs = []
    for sched in (fd.FD_SCHED_SHARES, fd.FD_SCHED_WAVES):
        grids, spec = [], []
        for w in shots:
            g = fd.Grid.from_workload(w)
            g.set_model(w["v"])
            rec = torch.zeros((w["nt"], len(w["rec"])), device="cuda")
            spec.append((g, w["src"], w["wavelet"], w["rec"], rec))
            grids.append(g)
        grids[0].set_schedule(sched)
        fd.check(fd.batch_forward(spec, fd.FD_BATCH_GRAPH), "fd_batch_forward")
        assert grids[0].info()["schedule"] == sched
        outs.append([r.cpu().numpy() for (_, _, _, _, r) in spec])
        for g in grids:
            g.close()
    for a, b in zip(*outs):
        assert np.abs(a).max() > 0
        np.testing.assert_array_equal(a, b)


def test_unknown_schedule_is_rejected(fd):
    w = workload(4, (20, 20, 20), 2, 4)
    with fd.Grid.from_workload(w) as g:
        with pytest.raises(fd.FDError) as e:
            g.set_schedule(7)
        assert e.value.status == fd.FD_ERR_ARG


def test_tuner_keeps_the_bits_for_forward_and_adjoint_runs(fd):
    """A grid left on its default tile is tuned by its first long fd_forward:
    the pick is a compiled tile under one of the two schedules, the receivers
    and wavefield equal an untuned run on the default tile bit for bit, and a
    later adjoint gradient (run on the tuned tile and schedule) equals that of
    a grid that was never tuned."""
    import torch
    w = workload(8, (60, 50, 44), 6, 420)
    rec0 = np.zeros((w["nt"], len(w["rec"])), np.float32)
    u0 = np.zeros((44, 50, 60), np.float32)
    g0 = torch.zeros((44, 50, 60), device="cuda")
    with fd.Grid.from_workload(w) as g:
        i0 = g.info()
        g.set_tile(i0["tile_x"], i0["tile_y"], 0)  # tuning off, default tile
        g.set_model(w["v"])
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec0, u0), "fd_forward")
        assert g.info()["schedule"] == fd.FD_SCHED_SHARES
        st, loss0 = g.adjoint_gradient(w["src"], w["wavelet"], w["rec"], 0.5 * rec0, 5, g0)
        fd.check(st, "fd_adjoint_gradient")
    rec1 = np.zeros_like(rec0)
    u1 = np.zeros_like(u0)
    g1 = torch.zeros_like(g0)
    with fd.Grid.from_workload(w) as g:
        g.set_model(w["v"])
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec1, u1), "fd_forward")
        info = g.info()
        assert (info["tile_x"], info["tile_y"]) in [(64, 16), (128, 8), (32, 16), (64, 8),
                                                    (32, 8)]
        assert info["schedule"] in (fd.FD_SCHED_SHARES, fd.FD_SCHED_WAVES)
        st, loss1 = g.adjoint_gradient(w["src"], w["wavelet"], w["rec"], 0.5 * rec0, 5, g1)
        fd.check(st, "fd_adjoint_gradient")
        assert (g.info()["tile_x"], g.info()["tile_y"]) == (info["tile_x"], info["tile_y"])
        # the tuned pair serves the next forward run again
        rec2 = np.zeros_like(rec0)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec2), "fd_forward")
        assert (g.info()["tile_x"], g.info()["tile_y"]) == (info["tile_x"], info["tile_y"])
    np.testing.assert_array_equal(rec0, rec1)
    np.testing.assert_array_equal(u0, u1)
    np.testing.assert_array_equal(rec2, rec0)
    # the misfit is a double sum accumulated with atomics: equal up to the
    # order of the additions
    assert abs(loss0 - loss1) <= 1e-12 * abs(loss0)
    assert torch.equal(g0, g1)
