"""Domain decomposition along z over CPU ranks (gloo): each rank steps its own
slab of the padded grid with the FP64 reference step after an R-plane halo
exchange (basic mode), or steps its CORE planes while the exchange travels
and its REMAINDER planes after it (full mode); the gathered result equals
the undecomposed run bit for bit.  A rank that leaves before an exchange is
reported to its neighbour as an error within the process group's timeout
(failure made on the host)."""
import socket

import numpy as np
import pytest

import oracle
from paper_2312_13094_gb300 import decomp


@pytest.mark.parametrize("Nz,world", [(15, 1), (15, 2), (15, 3), (16, 5), (100, 7)])
def test_slab_ranges_partition_the_planes(Nz, world):
    seen, sizes = [], []
    for r in range(world):
        z0, n = decomp.slab_range(Nz, world, r)
        seen.extend(range(z0, z0 + n))
        sizes.append(n)
    assert seen == list(range(Nz))
    assert max(sizes) - min(sizes) <= 1


def test_slab_range_rejects_more_ranks_than_planes():
    with pytest.raises(ValueError):
        decomp.slab_range(3, 4, 0)


def _problem(R):
    from paper_2312_13094_gb300 import workloads as wl
    n = (12, 10, 9)
    h = 10.0
    v = wl.layered_model(n, h, 3, vmin=1.8, vmax=2.4)
    g = oracle.Grid(n=n, h=h, dt=0.3 * h / 2.4, R=R, nbl=3)
    shp = g.padded_shape
    m_pad = oracle.pad_model(g, 1.0 / v.astype(np.float64) ** 2)
    b = oracle.damping(g, float(v.max()))
    return g, m_pad, b, wl.random_state(shp, 1), wl.random_state(shp, 2)


@pytest.mark.parametrize("R", [2, 4])
def test_slab_step_over_the_whole_grid_is_the_full_step(R):
    g, m_pad, b, up, uc = _problem(R)
    zero = np.zeros((R,) + up.shape[1:])
    out = oracle.step_slab(g, m_pad, b, up, np.concatenate([zero, uc, zero]))
    ref, _ = oracle.step(g, m_pad, b, up, uc)
    np.testing.assert_array_equal(out, ref)


def _rank_main(rank, world, port, R, nt):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            world_size=world, rank=rank)
    try:
        g, m_pad, b, up, uc = _problem(R)
        z0, nzs = decomp.slab_range(g.padded_shape[0], world, rank)
        own = slice(z0, z0 + nzs)
        prev = up[own].copy()
        ux = torch.zeros((nzs + 2 * R,) + up.shape[1:], dtype=torch.float64)
        ux[R:R + nzs] = torch.from_numpy(uc[own])
        for _ in range(nt):
            decomp.exchange_halos(ux, R, dist, rank, world)
            nxt = oracle.step_slab(g, m_pad[own], b[own], prev, ux.numpy())
            prev = ux[R:R + nzs].numpy().copy()
            ux[R:R + nzs] = torch.from_numpy(nxt)
        parts = [None] * world
        dist.all_gather_object(parts, (z0, ux[R:R + nzs].numpy().copy()))
        if rank == 0:
            got = np.concatenate([p for _, p in sorted(parts, key=lambda t: t[0])])
            pu, cu = up, uc
            for _ in range(nt):
                nu, _ = oracle.step(g, m_pad, b, pu, cu)
                pu, cu = cu, nu
            np.testing.assert_array_equal(got, cu)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,R", [(2, 2), (3, 4)])
def test_decomposed_run_over_gloo_ranks_equals_the_undecomposed_run(world, R):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    oracle.build()
    mp.spawn(_rank_main, args=(world, _free_port(), R, 6), nprocs=world, join=True)


def _dead_rank_main(rank, world, port, q):
    """Rank 1 leaves before the exchange; rank 0 must get an error from its
    halo exchange within the process group's short timeout, not hang."""
    import datetime
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            world_size=world, rank=rank,
                            timeout=datetime.timedelta(seconds=4))
    if rank == 1:
        q.put((1, "left"))
        return  # never joins the exchange, never tears down the group
    ux = torch.zeros((6 + 2 * 2, 5, 5), dtype=torch.float64)
    try:
        decomp.exchange_halos(ux, 2, dist, rank, world)
        q.put((0, "no error"))
    except Exception as e:  # the missing neighbour surfaces as an error
        q.put((0, f"error: {type(e).__name__}"))


def test_a_rank_that_leaves_is_detected_by_its_neighbour():
    pytest.importorskip("torch")
    import multiprocessing as mpl
    ctx = mpl.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dead_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    import queue
    try:
        for _ in range(2):
            r, msg = q.get(timeout=90)
            got[r] = msg
    except queue.Empty:
        pass
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
            p.join()
    assert got.get(1) == "left"
    assert got.get(0, "").startswith("error"), got


def _full_mode_main(rank, world, port, R, nt):
    """The paper's full mode on z slabs: start the exchange, step the CORE
    planes while it travels, finish it, then step the REMAINDER planes."""
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            world_size=world, rank=rank)
    try:
        g, m_pad, b, up, uc = _problem(R)
        z0, nzs = decomp.slab_range(g.padded_shape[0], world, rank)
        own = slice(z0, z0 + nzs)
        prev = up[own].copy()
        ux = torch.full((nzs + 2 * R,) + up.shape[1:], float("nan"), dtype=torch.float64)
        ux[R:R + nzs] = torch.from_numpy(uc[own])
        core, rem = decomp.core_and_remainder(nzs, R, rank, world)
        for _ in range(nt):
            pend = decomp.halo_begin(ux, R, dist, rank, world)
            nxt = np.full(prev.shape, np.nan)

            def part(a, b_):
                # owned planes [a, b_) from extended planes [a, b_ + 2R)
                return oracle.step_slab(g, m_pad[own][a:b_], b[own][a:b_], prev[a:b_],
                                        ux.numpy()[a:b_ + 2 * R])

            if core[1] > core[0]:
                nxt[core[0]:core[1]] = part(*core)  # no ghost plane read yet
            decomp.halo_end(pend)
            for a, b_ in rem:
                nxt[a:b_] = part(a, b_)
            prev = ux[R:R + nzs].numpy().copy()
            ux[R:R + nzs] = torch.from_numpy(nxt)
        parts = [None] * world
        dist.all_gather_object(parts, (z0, ux[R:R + nzs].numpy().copy()))
        if rank == 0:
            got = np.concatenate([p for _, p in sorted(parts, key=lambda t: t[0])])
            pu, cu = up, uc
            for _ in range(nt):
                nu, _ = oracle.step(g, m_pad, b, pu, cu)
                pu, cu = cu, nu
            np.testing.assert_array_equal(got, cu)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,R", [(2, 2), (3, 4)])
def test_full_mode_core_then_remainder_equals_the_undecomposed_run(world, R):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    oracle.build()
    mp.spawn(_full_mode_main, args=(world, _free_port(), R, 5), nprocs=world, join=True)


@pytest.mark.parametrize("nzs,R,rank,world,core,rem", [
    (10, 2, 0, 1, (0, 10), []), (10, 2, 0, 3, (0, 8), [(8, 10)]),
    (10, 2, 1, 3, (2, 8), [(0, 2), (8, 10)]), (10, 2, 2, 3, (2, 10), [(0, 2)]),
    (4, 2, 1, 3, (0, 0), [(0, 2), (2, 4)])])
def test_core_and_remainder_ranges(nzs, R, rank, world, core, rem):
    assert decomp.core_and_remainder(nzs, R, rank, world) == (core, rem)
