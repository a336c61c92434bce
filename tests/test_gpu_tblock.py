"""Temporal blocking (FD_SCHED_TEMPORAL): two leapfrog steps per pass over the
grid, the paper's named next optimisation (Discussion of Sec. IV).

Each point of both steps takes the single-step kernel's operations in the
same order, so a blocked run must equal the single-step run bit for bit:
receivers, final wavefield and previous wavefield, for even and odd step
counts, ragged grids, sources on tile seams and in the layer, grids without
a layer and grids smaller than one tile.  It is also compared with the FP64
oracle (relative L2 <= 1e-5).
"""
import numpy as np
import pytest

import oracle
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


def workload(so, n, nbl, nt, seed=7):
    h = 10.0
    v = wl.layered_model(n, h, seed, vmin=1.5, vmax=3.0)
    rng = np.random.default_rng(seed)
    v = (v * (1.0 + 0.05 * rng.uniform(-1, 1, v.shape))).astype(np.float32)
    dt = 0.35 * h / float(v.max())
    ext = [(d - 1) * h for d in n]
    # sources: interior, on a face, near an output-tile seam (x = 56, y = 24
    # padded cells) and inside the layer's reach of a corner
    src = np.array([[0.37 * ext[0], 0.61 * ext[1], 0.45 * ext[2]],
                    [0.0, ext[1], 0.2 * ext[2]],
                    [(55.5 - nbl) * h if n[0] > 60 else 0.5 * ext[0],
                     (23.7 - nbl) * h if n[1] > 30 else 0.3 * ext[1], 0.6 * ext[2]],
                    [0.02 * ext[0], 0.03 * ext[1], ext[2]]])
    rec = np.array([[0.0, 0.0, 0.0], [ext[0], ext[1], ext[2]]]
                   + [[x, 0.33 * ext[1], 2.5 * h] for x in np.linspace(0.2, ext[0] - 0.1, 17)]
                   + [[0.5 * ext[0], y, 0.5 * ext[2]] for y in np.linspace(0.0, ext[1], 9)])
    fr = [25.0, 18.0, 22.0, 30.0]
    wav = np.stack([wl.ricker(nt, dt, f) * (1.0 - 0.2 * i) for i, f in enumerate(fr)], 1)
    return dict(n=n, h=h, space_order=so, nbl=nbl, dt=dt, nt=nt, v=v, src=src, rec=rec,
                wavelet=np.ascontiguousarray(wav, np.float32))


def run(fd, w, sched, nt=None):
    nt = w["nt"] if nt is None else nt
    with fd.Grid.from_workload(w, nt=nt) as g:
        g.set_schedule(sched)
        g.set_model(w["v"])
        rec = np.zeros((nt, len(w["rec"])), np.float32)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec), "fd_forward")
        shp = g.padded_shape
        prev = np.zeros(shp, np.float32)
        cur = np.zeros(shp, np.float32)
        g.get_wavefield(prev, cur)
        info = g.info()
    return rec, prev, cur, info


CASES = [
    (8, (70, 45, 41), 6, 40),
    (8, (70, 45, 41), 6, 41),
    (4, (90, 61, 37), 8, 36),
    (4, (90, 61, 37), 8, 35),
    (8, (61, 50, 47), 0, 30),
    (8, (20, 17, 23), 3, 25),
    (4, (12, 14, 9), 4, 16),
]


@pytest.mark.parametrize("so,n,nbl,nt", CASES)
def test_blocked_run_equals_single_steps_bitwise(fd, so, n, nbl, nt):
    w = workload(so, n, nbl, nt)
    ref = run(fd, w, fd.FD_SCHED_SHARES)
    got = run(fd, w, fd.FD_SCHED_TEMPORAL)
    assert got[3]["schedule"] == fd.FD_SCHED_TEMPORAL
    assert ref[3]["schedule"] == fd.FD_SCHED_SHARES
    assert np.abs(ref[0]).max() > 0
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[2], ref[2])
    np.testing.assert_array_equal(got[1], ref[1])


@pytest.mark.parametrize("so", [4, 8])
def test_blocked_run_against_the_oracle(fd, so):
    w = workload(so, (66, 53, 45), 7, 60)
    rec, _, cur, _ = run(fd, w, fd.FD_SCHED_TEMPORAL)
    og = oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=so // 2, nbl=w["nbl"])
    out = oracle.forward(og, 1.0 / w["v"].astype(np.float64) ** 2, w["nt"], w["src"],
                         w["wavelet"], w["rec"])
    assert rel(rec, out["rec"]) <= TOL, rel(rec, out["rec"])
    assert rel(cur, out["u_cur"]) <= TOL, rel(cur, out["u_cur"])


def test_blocked_pieces_equal_one_run(fd):
    """fd_propagate in pieces of odd and even length (each ending on a single
    step when odd) continues the state exactly."""
    w = workload(8, (58, 40, 33), 5, 37)
    full = run(fd, w, fd.FD_SCHED_TEMPORAL)
    with fd.Grid.from_workload(w) as g:
        g.set_schedule(fd.FD_SCHED_TEMPORAL)
        g.set_model(w["v"])
        parts, n0 = [], 0
        for k in (7, 10, 1, 19):
            r = np.zeros((k, len(w["rec"])), np.float32)
            fd.check(g.propagate(n0, k, w["src"], w["wavelet"], w["rec"], r), "fd_propagate")
            parts.append(r)
            n0 += k
        cur = np.zeros(g.padded_shape, np.float32)
        g.get_wavefield(None, cur)
    np.testing.assert_array_equal(np.concatenate(parts), full[0])
    np.testing.assert_array_equal(cur, full[2])


def test_other_space_orders_fall_back_to_single_steps(fd):
    w = workload(6, (40, 33, 29), 5, 20)
    ref = run(fd, w, fd.FD_SCHED_SHARES)
    got = run(fd, w, fd.FD_SCHED_TEMPORAL)
    assert got[3]["schedule"] == fd.FD_SCHED_SHARES
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[2], ref[2])


def test_reduced_headline_blocked_against_the_oracle(fd):
    """The headline recipe at 128^3 (+40), SO 8, 450 steps in two-step passes."""
    w = wl.acoustic_512(n=128, nt=450)
    rec, _, cur, info = run(fd, w, fd.FD_SCHED_TEMPORAL)
    assert info["schedule"] == fd.FD_SCHED_TEMPORAL
    og = oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=4, nbl=w["nbl"])
    out = oracle.forward(og, 1.0 / w["v"].astype(np.float64) ** 2, w["nt"], w["src"],
                         w["wavelet"], w["rec"])
    e_rec, e_u = rel(rec, out["rec"]), rel(cur, out["u_cur"])
    print(f"two-step passes, 128^3 x 450: receivers {e_rec:.2e}, wavefield {e_u:.2e}")
    assert e_rec <= TOL and e_u <= TOL
