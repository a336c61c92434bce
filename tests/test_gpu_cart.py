"""GPU runs of the Cartesian domain decomposition (fd_set_topology: px x py x
pz boxes with ghost layers, stepped in one launch on column waves or equal
shares; six face messages packed after every step, and every ghost block,
faces, edges and corners, unpacked from them in one exchange, Sec. III)
through the C ABI.

Every point of a box run goes through the same arithmetic as in the
undecomposed run, so the two must agree bit for bit (receivers, final and
previous wavefields); the undecomposed run is itself held to the FP64 oracle,
and one decomposed run is checked against the oracle directly.
"""
import numpy as np
import pytest

import oracle
from paper_2312_13094_gb300 import decomp
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


def box_workload(so, n=(53, 41, 37), nbl=5, nt=50, seed=9):
    """Sources scattered through the box so that some sit next to every cut,
    receivers on lines along x, y and z through the middle (crossing every
    face of a 2 x 2 x 2 split) and on the corners."""
    h = 10.0
    v = wl.layered_model(n, h, seed, vmin=1.5, vmax=3.0)
    rng = np.random.default_rng(seed)
    v = (v * (1.0 + 0.05 * rng.uniform(-1, 1, v.shape))).astype(np.float32)
    dt = 0.35 * h / float(v.max())
    ext = np.array([(d - 1) * h for d in n])
    src = np.array([[0.49, 0.51, 0.5], [0.2, 0.8, 0.3], [0.75, 0.25, 0.7], [0.5, 0.1, 0.95],
                    [0.0, 0.5, 0.5], [1.0, 1.0, 0.0]]) * ext
    lines = []
    for a in range(3):
        t = np.arange(0.0, ext[a] + 1e-3, 0.5 * h)
        p = np.tile(0.5 * ext + np.array([0.3, 0.2, 0.1]) * h, (len(t), 1))
        p[:, a] = t
        lines.append(p)
    rec = np.concatenate(lines + [np.array([[0.0, 0.0, 0.0], ext, [ext[0], 0.0, ext[2]]])])
    wav = np.stack([(1.0 - 0.1 * i) * wl.ricker(nt, dt, 20.0 + 3 * i) for i in range(len(src))],
                   1)
    return dict(n=n, h=h, space_order=so, nbl=nbl, dt=dt, nt=nt, v=v, src=src, rec=rec,
                wavelet=np.ascontiguousarray(wav, np.float32))


def run(fd, w, topo=None, tile=None, no_graph=False, sched=None):
    with fd.Grid.from_workload(w) as g:
        if tile is not None:
            g.set_tile(tile[0], tile[1], 0)
        if sched is not None:
            g.set_schedule(sched)
        if topo is not None:
            g.set_topology(*topo)
        if no_graph:
            g.set_debug(fd.FD_DEBUG_NO_GRAPH, 1)
        g.set_model(w["v"])
        rec = np.zeros((w["nt"], len(w["rec"])), np.float32)
        u = np.zeros(g.phys_shape, np.float32)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec, u), "fd_forward")
        prev = np.zeros(g.padded_shape, np.float32)
        cur = np.zeros(g.padded_shape, np.float32)
        g.get_wavefield(prev, cur)
        return rec, u, prev, cur


@pytest.mark.parametrize("so", [2, 8, 16])
@pytest.mark.parametrize("topo", [(2, 2, 1), (1, 2, 2), (2, 1, 2), (2, 2, 2), (3, 2, 1)])
def test_boxes_match_the_whole_grid_bitwise(fd, so, topo):
    w = box_workload(so)
    ref = run(fd, w)
    got = run(fd, w, topo)
    assert np.abs(ref[0]).max() > 0
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("topo", [(2, 2, 1), (2, 2, 2), (1, 3, 2)])
def test_box_schedules_and_tiles_agree_bitwise(fd, topo):
    """Column waves over all boxes (the default) and equal shares, on three
    tiles: every point is computed the same way whatever CTA computes it."""
    w = box_workload(8, n=(70, 45, 39), nt=24)
    ref = run(fd, w)
    for sched, tile in ((fd.FD_SCHED_SHARES, None), (fd.FD_SCHED_WAVES, (64, 16)),
                        (fd.FD_SCHED_WAVES, (32, 8)), (fd.FD_SCHED_AUTO, (128, 8))):
        got = run(fd, w, topo, tile=tile, sched=sched)
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b)


def test_receivers_on_box_edges_and_corners(fd):
    """Receivers whose eight interpolation nodes straddle two and three cuts
    (they read edge and corner ghosts, which the stencil never does)."""
    w = box_workload(8, n=(44, 40, 36), nbl=4, nt=40)
    N = [d + 2 * w["nbl"] for d in w["n"]]
    cut = [n // 2 - w["nbl"] - 0.4 for n in N]  # just below each cut, fraction 0.6
    h = w["h"]
    w["rec"] = np.array([[cut[0] * h, cut[1] * h, 3.3 * h], [cut[0] * h, 7.1 * h, cut[2] * h],
                         [9.2 * h, cut[1] * h, cut[2] * h], [cut[0] * h, cut[1] * h, cut[2] * h]])
    ref = run(fd, w)
    for topo in [(2, 2, 1), (2, 1, 2), (1, 2, 2), (2, 2, 2)]:
        got = run(fd, w, topo)
        np.testing.assert_array_equal(got[0], ref[0])


def test_dims_create_topologies_tiles_and_direct_launches(fd):
    """Topologies chosen as MPI_Dims_create would for 4, 6 and 12 ranks, on
    two tile shapes, with and without the captured graph."""
    w = box_workload(4, n=(61, 47, 43), nt=36)
    ref = run(fd, w)
    for ranks in (4, 6, 12):
        topo = decomp.dims_create(ranks, 3)
        for kw in (dict(), dict(tile=(32, 8)), dict(tile=(128, 8), no_graph=True)):
            got = run(fd, w, topo, **kw)
            for a, b in zip(got, ref):
                np.testing.assert_array_equal(a, b)


def test_box_run_against_the_oracle(fd):
    w = box_workload(8, nt=45)
    rec, u, _, _ = run(fd, w, (2, 2, 2))
    og = oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=4, nbl=w["nbl"])
    out = oracle.forward(og, 1.0 / w["v"].astype(np.float64) ** 2, w["nt"], w["src"],
                         w["wavelet"], w["rec"])
    nb = w["nbl"]
    assert rel(rec, out["rec"]) <= TOL
    assert rel(u, out["u_cur"][nb:-nb, nb:-nb, nb:-nb]) <= TOL


def test_pieces_and_switching_between_slabs_and_boxes(fd):
    w = box_workload(8, nt=30)
    ref = run(fd, w)
    with fd.Grid.from_workload(w) as g:
        g.set_topology(2, 2, 1)
        g.set_model(w["v"])
        a = np.zeros((13, len(w["rec"])), np.float32)
        b = np.zeros((17, len(w["rec"])), np.float32)
        fd.check(g.propagate(0, 13, w["src"], w["wavelet"], w["rec"], a), "p1")
        g.set_decomposition(3, fd.FD_DMP_BASIC)  # replaces the boxes
        fd.check(g.propagate(13, 17, w["src"], w["wavelet"], w["rec"], b), "p2")
        cur = np.zeros(g.padded_shape, np.float32)
        g.get_wavefield(None, cur)
    np.testing.assert_array_equal(np.concatenate([a, b]), ref[0])
    np.testing.assert_array_equal(cur, ref[3])


def test_boxes_thinner_than_the_stencil_are_rejected(fd):
    w = box_workload(16, n=(20, 20, 20), nbl=2, nt=5)
    with fd.Grid.from_workload(w) as g:
        st = fd.fd_set_topology(g.handle, 4, 1, 1)  # 24 points into 4 boxes of 6 < 8
        assert st == fd.FD_ERR_ARG
        assert b"at least" in fd.fd_last_error()
