"""Batched multi-shot forward (one persistent launch per step, CUDA graph,
autotuned tiles) against single-shot runs and the FP64 oracle."""
import numpy as np
import pytest

import oracle
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


def shots_small(nshots=5, nt=40):
    return wl.batched_shots(nshots=nshots, nt=nt, lo=24, hi=60, nbl=6)


def run_batch(fd, shots, flags):
    grids, outs, spec = [], [], []
    for w in shots:
        g = fd.Grid.from_workload(w)
        g.set_model(w["v"])
        out = np.zeros((w["nt"], len(w["rec"])), np.float32)
        grids.append(g)
        outs.append(out)
        spec.append((g, w["src"], w["wavelet"], w["rec"], out))
    fd.check(fd.batch_forward(spec, flags), "fd_batch_forward")
    return grids, outs


def test_batch_equals_single_shot_runs_bitwise(fd):
    shots = shots_small()
    grids, outs = run_batch(fd, shots, fd.FD_BATCH_GRAPH)
    for g, w, out in zip(grids, shots, outs):
        single = np.zeros_like(out)
        fd.check(g.forward(w["src"], w["wavelet"], w["rec"], single), "fd_forward")
        np.testing.assert_array_equal(out, single)
        g.close()


def test_batch_matches_oracle(fd):
    shots = shots_small(nshots=3, nt=30)
    grids, outs = run_batch(fd, shots, fd.FD_BATCH_GRAPH)
    for w, out in zip(shots, outs):
        og = oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=w["space_order"] // 2, nbl=w["nbl"])
        ref = oracle.forward(og, 1.0 / w["v"].astype(np.float64) ** 2, w["nt"], w["src"],
                             w["wavelet"], w["rec"])["rec"]
        assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-5
    for g in grids:
        g.close()


def test_graph_autotune_and_plain_launches_agree(fd):
    shots = shots_small(nshots=4, nt=25)
    _, plain = run_batch(fd, shots, 0)
    grids, tuned = run_batch(fd, shots, fd.FD_BATCH_GRAPH | fd.FD_BATCH_AUTOTUNE)
    for a, b in zip(plain, tuned):
        np.testing.assert_array_equal(a, b)
    info = grids[0].info()
    assert (info["tile_x"], info["tile_y"]) in [(64, 16), (128, 8), (32, 16), (64, 8), (32, 8)]
    # a second call reuses the cached pick and the captured graph
    _, again = run_batch(fd, shots, fd.FD_BATCH_GRAPH | fd.FD_BATCH_AUTOTUNE)
    for a, b in zip(tuned, again):
        np.testing.assert_array_equal(a, b)


def test_batch_rejects_mixed_space_orders(fd):
    shots = shots_small(nshots=2, nt=10)
    shots[1] = dict(shots[1], space_order=4)
    grids, specs = [], []
    for w in shots:
        g = fd.Grid.from_workload(w)
        g.set_model(w["v"])
        grids.append(g)
        specs.append((g, w["src"], w["wavelet"], w["rec"],
                      np.zeros((w["nt"], len(w["rec"])), np.float32)))
    assert fd.batch_forward(specs) == fd.FD_ERR_ARG


def test_batch_at_the_configured_sizes_against_the_oracle(fd):
    """The batched workload as configured (32 windows of 128..320 points per
    axis + 20-cell layer, SO 8, 600 steps, one graph-captured persistent
    launch per step with autotuned tiles): every shot equals its single-shot
    run bit for bit on two of them, and the receivers of the two smallest
    windows match the FP64 oracle run of the full 600 steps within 1e-5."""
    import torch
    shots = wl.batched_shots()
    assert len(shots) == 32 and min(min(w["n"]) for w in shots) >= 128
    grids, specs = [], []
    for w in shots:
        g = fd.Grid.from_workload(w)
        g.set_model(w["v"])
        out = torch.zeros((w["nt"], len(w["rec"])), device="cuda")
        wav = torch.from_numpy(np.ascontiguousarray(w["wavelet"])).cuda()
        grids.append(g)
        specs.append((g, w["src"], wav, w["rec"], out))
    fd.check(fd.batch_forward(specs, fd.FD_BATCH_GRAPH | fd.FD_BATCH_AUTOTUNE),
             "fd_batch_forward")
    torch.cuda.synchronize()
    size = [int(np.prod(w["n"])) for w in shots]
    pick = sorted(range(len(shots)), key=lambda i: size[i])[:2]
    for i in pick:
        w = shots[i]
        got = specs[i][4].cpu().numpy()
        single = np.zeros_like(got)
        fd.check(grids[i].forward(w["src"], w["wavelet"], w["rec"], single), "fd_forward")
        np.testing.assert_array_equal(got, single)
        og = oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=4, nbl=w["nbl"])
        ref = oracle.forward(og, 1.0 / w["v"].astype(np.float64) ** 2, w["nt"], w["src"],
                             w["wavelet"], w["rec"])["rec"]
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"shot {i} {w['n']} x {w['nt']} steps: receivers rel L2 {err:.2e}")
        assert err <= 1e-5
    for g in grids:
        g.close()
