"""Shot-parallel sharding over two CPU ranks (gloo): the shares cover every
shot once, and the summed gradient over ranks equals the serial sum of the
per-shot FP64 oracle gradients."""
import os
import socket

import numpy as np
import pytest

from paper_2312_13094_gb300 import shard


@pytest.mark.parametrize("nshots", [0, 1, 2, 7, 32, 33])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shot_ranges_partition_the_shots(nshots, world):
    seen = []
    sizes = []
    for r in range(world):
        rr = shard.shot_range(nshots, world, r)
        seen.extend(rr)
        sizes.append(len(rr))
    assert seen == list(range(nshots))
    assert max(sizes) - min(sizes) <= 1


def test_shot_range_rejects_bad_ranks():
    with pytest.raises(ValueError):
        shard.shot_range(4, 2, 2)
    with pytest.raises(ValueError):
        shard.shot_range(4, 0, 0)


def _problem():
    from paper_2312_13094_gb300 import workloads as wl
    n = (10, 9, 8)
    h = 10.0
    v = wl.layered_model(n, h, 21, vmin=1.8, vmax=2.4)
    nt = 24
    dt = 0.3 * h / float(v.max())
    wav = wl.ricker(nt, dt, 40.0).reshape(nt, 1)
    rec = np.array([[x, 40.0, 60.0] for x in np.linspace(0.0, 90.0, 4)])
    return n, h, v, nt, dt, wav, rec


def _shot_src(s):
    return np.array([[10.0 + 12.0 * s, 30.0 + 3.0 * s, 20.0]])


def _grad_of_shot(s):
    import oracle
    import torch
    n, h, v, nt, dt, wav, rec = _problem()
    og = oracle.Grid(n=n, h=h, dt=dt, R=2, nbl=3)
    m = 1.0 / v.astype(np.float64) ** 2
    d_obs = np.zeros((nt, len(rec)))
    g, loss, _ = oracle.adjoint_gradient(og, m, nt, _shot_src(s), wav, rec, d_obs=d_obs)
    return torch.from_numpy(np.ascontiguousarray(g)), loss


def _rank_main(rank, world, port, nshots):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            world_size=world, rank=rank)
    try:
        like = torch.zeros(_problem()[0][::-1], dtype=torch.float64)
        total, loss = shard.shot_parallel_gradient(nshots, _grad_of_shot, like, dist)
        t = torch.tensor([float(rank + 1)])
        shard.max_over_ranks(t, dist)
        assert float(t) == world
        if rank == 0:
            ref = torch.zeros_like(like)
            ref_loss = 0.0
            for s in range(nshots):
                g, l_s = _grad_of_shot(s)
                ref += g
                ref_loss += l_s
            assert float(ref.abs().max()) > 0
            np.testing.assert_allclose(total.numpy(), ref.numpy(), rtol=1e-12,
                                       atol=1e-14 * float(ref.abs().max()))
            assert abs(loss - ref_loss) <= 1e-12 * abs(ref_loss)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shot_parallel_gradient_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    oracle.build()
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    mp.spawn(_rank_main, args=(2, _free_port(), 5), nprocs=2, join=True)
