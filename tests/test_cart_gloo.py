"""Cartesian domain decomposition over CPU ranks (gloo), the paper's basic
mode (Sec. III): a topology of px x py x pz ranks, each owning a box of the
padded grid and filling its R-wide ghost layers with six messages per step
(one synchronous exchange per axis, faces packed into contiguous buffers,
edges and corners carried by the later axes).  Gathered after several steps,
the boxes equal the undecomposed FP64 oracle run bit for bit, for the
isotropic star stencil (C oracle) and for the TTI stencil, whose cross
derivatives read the edge and corner ghosts."""
import socket

import numpy as np
import pytest

import oracle
from oracle import tti as otti
from paper_2312_13094_gb300 import decomp


@pytest.mark.parametrize("world,want", [(1, (1, 1, 1)), (2, (2, 1, 1)), (4, (2, 2, 1)),
                                        (6, (3, 2, 1)), (8, (2, 2, 2)), (12, (3, 2, 2)),
                                        (30, (5, 3, 2)), (64, (4, 4, 4)), (128, (8, 4, 4))])
def test_dims_create_is_balanced(world, want):
    """The split MPI_Dims_create gives for three axes (as close to a cube as
    the prime factors allow, in non-increasing order)."""
    assert decomp.dims_create(world) == want


def test_topology_ranks_boxes_and_neighbours():
    t = decomp.Topology((3, 2, 2), (17, 11, 9))
    owned = np.zeros((9, 11, 17), dtype=int)
    for r in range(t.world):
        c = t.coords(r)
        assert t.rank_of(c) == r
        (x0, nx), (y0, ny), (z0, nz) = t.box(r)
        owned[z0:z0 + nz, y0:y0 + ny, x0:x0 + nx] += 1
        for axis in range(3):
            for step in (-1, 1):
                nb = t.neighbour(r, axis, step)
                if nb is not None:
                    assert t.neighbour(nb, axis, -step) == r
                    cn = list(t.coords(nb))
                    cn[axis] -= step
                    assert tuple(cn) == c
    assert np.all(owned == 1)
    with pytest.raises(ValueError):
        decomp.Topology((4, 1, 1), (3, 5, 5))


def test_block_step_over_the_whole_grid_is_the_full_step():
    g, m_pad, b, up, uc = _acoustic_problem(2)
    R = g.R
    ux = np.zeros(tuple(s + 2 * R for s in up.shape))
    ux[R:-R, R:-R, R:-R] = uc
    np.testing.assert_array_equal(oracle.step_block(g, m_pad, b, up, ux),
                                  oracle.step(g, m_pad, b, up, uc)[0])


def _acoustic_problem(R):
    from paper_2312_13094_gb300 import workloads as wl
    n = (11, 9, 10)
    h = 10.0
    v = wl.layered_model(n, h, 3, vmin=1.8, vmax=2.4)
    g = oracle.Grid(n=n, h=h, dt=0.3 * h / 2.4, R=R, nbl=3)
    shp = g.padded_shape
    m_pad = oracle.pad_model(g, 1.0 / v.astype(np.float64) ** 2)
    b = oracle.damping(g, float(v.max()))
    return g, m_pad, b, wl.random_state(shp, 1), wl.random_state(shp, 2)


def _tti_problem():
    from paper_2312_13094_gb300 import workloads as wl
    w = wl.tti_workload(n=(10, 9, 8), so=4, nbl=2, nt=1)
    g = oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=2, nbl=w["nbl"])
    shp = g.padded_shape
    pads = [oracle.pad_model(g, np.asarray(a, np.float64))
            for a in (1.0 / w["v"].astype(np.float64) ** 2, w["eps"], w["delta"], w["theta"],
                      w["phi"])]
    vmax = float(np.max(w["v"] * np.sqrt(1.0 + 2.0 * w["eps"].astype(np.float64))))
    b = oracle.damping(g, vmax)
    st = [wl.random_state(shp, 11 + i) for i in range(4)]
    return g, pads, b, st


def _ext(a, box, R, fill):
    """The box of a padded (z, y, x) array with R layers around it, `fill`
    beyond the grid."""
    (x0, nx), (y0, ny), (z0, nz) = box
    out = np.full((nz + 2 * R, ny + 2 * R, nx + 2 * R), fill, dtype=a.dtype)
    Z, Y, X = a.shape
    zs, ys, xs = (slice(max(0, s0 - R), min(S, s0 + n + R))
                  for s0, n, S in ((z0, nz, Z), (y0, ny, Y), (x0, nx, X)))
    out[zs.start - (z0 - R):zs.stop - (z0 - R), ys.start - (y0 - R):ys.stop - (y0 - R),
        xs.start - (x0 - R):xs.stop - (x0 - R)] = a[zs, ys, xs]
    return out


def _own(a_x, R):
    return a_x[R:-R, R:-R, R:-R]


def _only_box(a, box, R):
    """The box of `a` with R layers of NaN around it: every ghost value a step
    reads must come from the exchange."""
    (x0, nx), (y0, ny), (z0, nz) = box
    out = np.full((nz + 2 * R, ny + 2 * R, nx + 2 * R), np.nan)
    out[R:-R, R:-R, R:-R] = a[z0:z0 + nz, y0:y0 + ny, x0:x0 + nx]
    return out


def _rank_main(rank, world, port, dims, kind, nt, mode="basic"):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            world_size=world, rank=rank)
    try:
        def exchange(u_x, R, topo):
            if mode == "diag":
                sent = decomp.exchange_halos_diag(u_x, R, dist, topo, rank)
                c = topo.coords(rank)
                # one message per existing neighbour among the 26 directions
                want = sum(1 for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                           if (dx, dy, dz) != (0, 0, 0) and
                           topo.rank_of((c[0] + dx, c[1] + dy, c[2] + dz)) is not None)
                assert sent == want
            else:
                decomp.exchange_halos_3d(u_x, R, dist, topo, rank)

        if kind == "acoustic":
            g, m_pad, b, up, uc = _acoustic_problem(2)
            R = g.R
            topo = decomp.Topology(dims, up.shape[::-1])
            box = topo.box(rank)
            (x0, nx), (y0, ny), (z0, nz) = box
            own = (slice(z0, z0 + nz), slice(y0, y0 + ny), slice(x0, x0 + nx))
            prev = up[own].copy()
            ux = torch.from_numpy(_only_box(uc, box, R))
            for _ in range(nt):
                exchange(ux, R, topo)
                nxt = oracle.step_block(g, m_pad[own], b[own], prev, ux.numpy())
                prev = _own(ux.numpy(), R).copy()
                ux[R:-R, R:-R, R:-R] = torch.from_numpy(nxt)
            mine = _own(ux.numpy(), R).copy()
            ref_full = None
            if rank == 0:
                pu, cu = up, uc
                for _ in range(nt):
                    nu, _ = oracle.step(g, m_pad, b, pu, cu)
                    pu, cu = cu, nu
                ref_full = cu
        else:
            g, pads, b, st = _tti_problem()
            R = g.R
            shp = st[0].shape
            topo = decomp.Topology(dims, shp[::-1])
            box = topo.box(rank)
            (x0, nx), (y0, ny), (z0, nz) = box
            coef = [_ext(a, box, R, 1.0) for a in pads]
            bx = _ext(b, box, R, 0.0)
            p_prev = _ext(st[0], box, R, 0.0)
            q_prev = _ext(st[2], box, R, 0.0)
            px = torch.from_numpy(_only_box(st[1], box, R))
            qx = torch.from_numpy(_only_box(st[3], box, R))
            for _ in range(nt):
                exchange(px, R, topo)
                exchange(qx, R, topo)
                pn, qn = otti.step(g, *coef, bx, p_prev, px.numpy(), q_prev, qx.numpy())
                p_prev, q_prev = px.numpy().copy(), qx.numpy().copy()
                px[R:-R, R:-R, R:-R] = torch.from_numpy(_own(pn, R))
                qx[R:-R, R:-R, R:-R] = torch.from_numpy(_own(qn, R))
            mine = np.stack([_own(px.numpy(), R), _own(qx.numpy(), R)])
            ref_full = None
            if rank == 0:
                a = st
                for _ in range(nt):
                    pn, qn = otti.step(g, *pads, b, a[0], a[1], a[2], a[3])
                    a = [a[1], pn, a[3], qn]
                ref_full = np.stack([a[1], a[3]])
        parts = [None] * world
        dist.all_gather_object(parts, (box, mine))
        if rank == 0:
            got = np.full(ref_full.shape, np.nan)
            for (bx0, by0, bz0), blk in parts:
                sl = (slice(bz0[0], bz0[0] + bz0[1]), slice(by0[0], by0[0] + by0[1]),
                      slice(bx0[0], bx0[0] + bx0[1]))
                got[(Ellipsis,) + sl] = blk
            np.testing.assert_array_equal(got, ref_full)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("dims,kind,mode", [((2, 2, 1), "acoustic", "basic"),
                                            ((1, 2, 3), "acoustic", "basic"),
                                            ((2, 2, 2), "tti", "basic"),
                                            ((2, 2, 2), "tti", "diag"),
                                            ((3, 1, 2), "acoustic", "diag")])
def test_cartesian_run_over_gloo_ranks_equals_the_undecomposed_run(dims, kind, mode):
    """Basic mode (three axis steps) and diagonal mode (one step, up to 26
    messages per rank) both give the undecomposed run's bits."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    oracle.build()
    world = dims[0] * dims[1] * dims[2]
    mp.spawn(_rank_main, args=(world, _free_port(), dims, kind, 4, mode), nprocs=world,
             join=True)
