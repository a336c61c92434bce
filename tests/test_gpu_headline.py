"""Parity of the benchmarked launch at the headline workload's own recipe and
length (Eq. 1 of App. A, discretised as in Sec. IV-B, with the layer of
Sec. IV-C and the off-grid points of Sec. III "Sparse data").

* The headline recipe at reduced size (128^3 + 40-cell layer, SO 8, 450
  steps, long enough for the direct wave to pass the receivers: the
  two-layer model with its smooth perturbation, the centred
  15 Hz Ricker and the line of receivers at z = 2.5 cells), run in the exact
  launch configurations the benchmark's tuner picks on the full grid (64 x 16
  and 128 x 8 tiles on the column-wave schedule, i.e. ``sched_kernel``), and
  SO 16 on its tuned 32 x 16 tile: receivers and final wavefield against the
  FP64 oracle run, relative L2 <= 1e-5.
* The full headline run (592^3, 1000 steps) in the benchmark's own
  configuration (tile and schedule picked by the tuner): sampled cells of its
  last two wavefields (and its receivers) against the FP64 oracle's, written
  once by ``tests/golden/make_acoustic_512_golden.py`` (oracle only).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2312_13094_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "acoustic_512_so8_1000.npz")


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


@pytest.fixture(scope="module")
def reduced():
    """The headline recipe at 128^3 (+40), 450 steps, and its oracle run at
    SO 8 and SO 16 (each oracle run is shared by the launches compared)."""
    out = {}
    for so in (8, 16):
        w = wl.acoustic_512(n=128, nt=450)
        w["space_order"] = so
        og = oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=so // 2, nbl=w["nbl"])
        ref = oracle.forward(og, 1.0 / w["v"].astype(np.float64) ** 2, w["nt"], w["src"],
                             w["wavelet"], w["rec"])
        nb = w["nbl"]
        out[so] = (w, ref["rec"], ref["u_cur"][nb:-nb, nb:-nb, nb:-nb])
    return out


def run(fd, w, tile, sched):
    with fd.Grid.from_workload(w) as g:
        g.set_tile(tile[0], tile[1], 0)
        g.set_schedule(sched)
        g.set_model(w["v"])
        rec = np.zeros((w["nt"], len(w["rec"])), np.float32)
        u = np.zeros(g.phys_shape, np.float32)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], rec, u), "fd_forward")
        info = g.info()
    return rec, u, info


@pytest.mark.parametrize("so,tile", [(8, (64, 16)), (8, (128, 8)), (16, (32, 16))])
def test_reduced_headline_in_the_benchmark_launch(fd, reduced, so, tile):
    w, rrec, ru = reduced[so]
    rec, u, info = run(fd, w, tile, fd.FD_SCHED_WAVES)
    assert (info["tile_x"], info["tile_y"]) == tile
    assert info["schedule"] == fd.FD_SCHED_WAVES  # the sched_kernel launch ran
    e_rec, e_u = rel(rec, rrec), rel(u, ru)
    print(f"SO {so} tile {tile}: receivers {e_rec:.2e}, wavefield {e_u:.2e}")
    # the direct wave has reached the receivers: not a comparison of zeros
    assert np.abs(rrec).max() > 0.05 * np.abs(rrec[:150]).max() + 1e-3 * np.abs(ru).max()
    assert e_rec <= TOL and e_u <= TOL


def test_reduced_headline_schedules_agree_bitwise(fd, reduced):
    """Equal shares and column waves give the same bits on this recipe."""
    w = reduced[8][0]
    a = run(fd, w, (64, 16), fd.FD_SCHED_WAVES)
    b = run(fd, w, (64, 16), fd.FD_SCHED_SHARES)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="golden oracle run not written")
def test_full_headline_run_against_the_oracle(fd):
    """592^3, SO 8, 1000 steps in the benchmark's configuration (default tile
    and schedule, tuned by the first long run) against the stored FP64 oracle
    run: the final and previous wavefields at 18k sampled cells (random cells,
    the source's and the receiver line's neighbourhoods, corners, faces) within
    relative L2 1e-5.  The receivers sit 2.5 km from the source and the direct
    wave needs ~1.7 s to reach them, longer than the workload's 1.27 s: they
    hold only the stencil's numerical precursor (~1e-33), so they are held to
    the oracle's values within 1e-5 of the wavefield's amplitude instead of a
    relative norm."""
    import torch
    gold = np.load(GOLDEN)
    meta = json.loads(str(gold["meta"]))
    w = wl.acoustic_512()
    assert meta["workload"] == w["name"] and meta["nt"] == w["nt"]
    with fd.Grid.from_workload(w) as g:
        g.set_model(torch.from_numpy(w["v"]).cuda())
        rec = torch.zeros((w["nt"], len(w["rec"])), device="cuda")
        wav = torch.from_numpy(np.ascontiguousarray(w["wavelet"])).cuda()
        fd.check(g.forward(w["src"], wav, w["rec"], rec), "fd_forward")
        info = g.info()
        prev = torch.zeros(g.phys_shape, device="cuda")
        cur = torch.zeros(g.phys_shape, device="cuda")
        g.get_wavefield(prev, cur, fd.FD_REGION_PHYSICAL)
        torch.cuda.synchronize()
    pts = torch.from_numpy(gold["pts"].astype(np.int64)).cuda()
    got_u = cur[pts[:, 0], pts[:, 1], pts[:, 2]].cpu().numpy()
    got_p = prev[pts[:, 0], pts[:, 1], pts[:, 2]].cpu().numpy()
    rec = rec.cpu().numpy().astype(np.float64)
    e_u = rel(got_u, gold["u_last"])
    e_p = rel(got_p, gold["u_prev"])
    scale = np.abs(gold["u_last"]).max()
    e_rec = np.abs(rec - gold["rec"]).max() / scale
    print(f"592^3 x 1000 (tile {info['tile_x']}x{info['tile_y']}, schedule "
          f"{info['schedule']}): sampled u^1000 {e_u:.2e}, u^999 {e_p:.2e}; receivers "
          f"max |error| / max |u| {e_rec:.1e} (oracle receivers up to "
          f"{np.abs(gold['rec']).max():.1e})")
    assert e_u <= TOL and e_p <= TOL
    assert e_rec <= TOL
