"""Domain decomposition of one grid over ranks (the paper's Sec. III: each
subdomain exchanges an R-deep halo with its neighbours before every step).

This module holds the data movement of that scheme, not the step itself:
  * slabs along z: which padded z planes a rank owns (slab_range) and the
    exchange that fills the R ghost planes on either side (exchange_halos);
    the device runs the same split inside one GPU (fd_set_decomposition);
  * a Cartesian topology of px x py x pz ranks (dims_create, Topology) and the
    paper's basic-mode exchange on it (exchange_halos_3d): one synchronous
    step per axis, two packed face messages each, later axes carrying the
    edges and corners; and its diagonal mode (exchange_halos_diag): one step
    with up to 26 messages, faces, edges and corners at once;
  * the full mode on slabs (halo_begin, halo_end, core_and_remainder): the
    CORE planes are stepped while the exchange travels.
The CPU tests run these exchanges between gloo ranks around the FP64
reference step and compare with the undecomposed run bit for bit.

Layout of a rank's extended array: its owned points with R ghost layers
around them (along z only for slabs, along every axis for Cartesian blocks);
ghost layers beyond the global grid are zero (the read-only zero halo of
Sec. III).
"""
from __future__ import annotations


def slab_range(Nz: int, world: int, rank: int) -> tuple[int, int]:
    """(z0, nzs): rank's owned padded planes [z0, z0 + nzs), contiguous and
    balanced (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or Nz < world:
        raise ValueError(f"cannot split {Nz} planes over {world} ranks (rank {rank})")
    z0 = Nz * rank // world
    return z0, Nz * (rank + 1) // world - z0


def exchange_halos(u_x, R: int, dist, rank: int, world: int) -> None:
    """Fill the ghost planes of the extended slab `u_x` ([nzs + 2R, ...]
    tensor) in place: planes [0, R) from rank - 1's last R owned planes,
    planes [nzs + R, nzs + 2R) from rank + 1's first R owned planes; at the
    ends of the grid they are set to zero (the paper's basic mode: the whole
    exchange before the step).  Every rank must call this with the same R;
    each slab needs at least R owned planes."""
    halo_end(halo_begin(u_x, R, dist, rank, world))


def halo_begin(u_x, R: int, dist, rank: int, world: int):
    """Start the slab exchange of exchange_halos without waiting (the paper's
    "full" mode, Sec. III: the halo travels while the CORE planes, whose
    stencils stay inside the slab, are computed).  Returns the pending state
    for halo_end; ghost planes beyond the grid are zeroed at once."""
    nzs = u_x.shape[0] - 2 * R
    if nzs < R:
        raise ValueError(f"a slab of {nzs} planes cannot feed an {R}-plane halo")
    reqs, recv = [], []
    if rank > 0:
        reqs.append(dist.isend(u_x[R:2 * R].contiguous(), rank - 1, tag=1))
        lo = u_x.new_empty(u_x[0:R].shape)
        reqs.append(dist.irecv(lo, rank - 1, tag=2))
        recv.append((slice(0, R), lo))
    else:
        u_x[0:R].zero_()
    if rank + 1 < world:
        reqs.append(dist.isend(u_x[nzs:nzs + R].contiguous(), rank + 1, tag=2))
        hi = u_x.new_empty(u_x[nzs + R:].shape)
        reqs.append(dist.irecv(hi, rank + 1, tag=1))
        recv.append((slice(nzs + R, nzs + 2 * R), hi))
    else:
        u_x[nzs + R:].zero_()
    return u_x, reqs, recv


def halo_end(pending) -> None:
    """Wait for the messages of halo_begin and place the received ghost
    planes (the REMAINDER planes can then be computed)."""
    u_x, reqs, recv = pending
    for r in reqs:
        r.wait()
    for sl, buf in recv:
        u_x[sl] = buf


def core_and_remainder(nzs: int, R: int, rank: int, world: int):
    """Owned-plane ranges of a slab: the CORE planes, whose stencils read no
    ghost plane, and the REMAINDER planes beside an inner face (ranges are
    [a, b) in owned-plane numbering; a slab at the end of the grid has no
    remainder on that side, since its ghost planes there are zero)."""
    lo = R if rank > 0 else 0
    hi = R if rank + 1 < world else 0
    core = (lo, nzs - hi) if nzs - hi > lo else (0, 0)
    rem = [r for r in ((0, lo), (nzs - hi, nzs)) if r[1] > r[0]]
    return core, rem


# ---------------------------------------------------------------------------
# Cartesian topology (Sec. III: the grid is split over an MPI Cartesian
# topology of px x py x pz ranks, chosen by the library or given by the user
# as topology=(px, py, pz))
# ---------------------------------------------------------------------------

def dims_create(world: int, ndims: int = 3) -> tuple:
    """A balanced split of `world` ranks over `ndims` axes: the prime factors
    of world dealt largest first to the axis with the fewest ranks so far,
    returned in non-increasing order (as MPI_Dims_create does); axis order
    (x, y, z)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    f, n, p = [], world, 2
    while p * p <= n:
        while n % p == 0:
            f.append(p)
            n //= p
        p += 1
    if n > 1:
        f.append(n)
    dims = [1] * ndims
    for q in sorted(f, reverse=True):
        dims[dims.index(min(dims))] *= q
    return tuple(sorted(dims, reverse=True))


class Topology:
    """Rank layout of a Cartesian decomposition: dims = (px, py, pz), rank
    = (cz * py + cy) * px + cx (x fastest); each axis split into balanced
    contiguous ranges of the padded grid (slab_range per axis)."""

    def __init__(self, dims, shape_xyz):
        self.dims = tuple(int(d) for d in dims)
        self.shape = tuple(int(s) for s in shape_xyz)
        if len(self.dims) != 3 or min(self.dims) < 1:
            raise ValueError(f"bad topology {dims}")
        for d, s in zip(self.dims, self.shape):
            if d > s:
                raise ValueError(f"cannot split {s} points over {d} ranks")
        self.world = self.dims[0] * self.dims[1] * self.dims[2]

    def coords(self, rank: int) -> tuple:
        px, py, _ = self.dims
        if not 0 <= rank < self.world:
            raise ValueError(f"rank {rank} outside a world of {self.world}")
        return rank % px, (rank // px) % py, rank // (px * py)

    def rank_of(self, coords) -> int | None:
        """Rank at coords, or None outside the topology (the grid's edge)."""
        if any(c < 0 or c >= d for c, d in zip(coords, self.dims)):
            return None
        cx, cy, cz = coords
        return (cz * self.dims[1] + cy) * self.dims[0] + cx

    def box(self, rank: int) -> tuple:
        """((x0, nx), (y0, ny), (z0, nz)): the padded points a rank owns."""
        return tuple(slab_range(s, d, c) for s, d, c in zip(self.shape, self.dims,
                                                              self.coords(rank)))

    def neighbour(self, rank: int, axis: int, step: int) -> int | None:
        c = list(self.coords(rank))
        c[axis] += step
        return self.rank_of(c)


def exchange_halos_3d(u_x, R: int, dist, topo: Topology, rank: int) -> None:
    """Fill the R-wide ghost layers of the extended block `u_x`
    ([nz + 2R, ny + 2R, nx + 2R] tensor, the owned box in the middle) from the
    neighbours, in the paper's basic mode: one synchronous step per axis, x,
    then y, then z, two messages each (six in all).  A step sends the R owned
    layers next to each face, packed into a contiguous buffer; across the
    axes already exchanged the face includes their ghost layers, so edges and
    corners arrive too (what cross-derivative stencils such as TTI's need).
    Ghost layers beyond the grid are zero.  Every rank must call this."""
    nz, ny, nx = (s - 2 * R for s in u_x.shape)
    n = {0: nx, 1: ny, 2: nz}
    if min(n.values()) < R:
        raise ValueError("a block needs at least R points along every axis")
    done = []
    for axis in (0, 1, 2):  # x, y, z
        dim = 2 - axis      # tensor dimension of this axis
        idx = [slice(R, R + n[a]) if a not in done else slice(None) for a in (2, 1, 0)]
        # idx is in tensor order (z, y, x); the axis itself is set per face

        def face(lo, hi):
            sl = list(idx)
            sl[dim] = slice(lo, hi)
            return tuple(sl)

        reqs, recv = [], []
        for step, (own, ghost) in ((-1, ((R, 2 * R), (0, R))),
                                   (1, ((n[axis], n[axis] + R), (n[axis] + R, n[axis] + 2 * R)))):
            peer = topo.neighbour(rank, axis, step)
            gsl = face(*ghost)
            if peer is None:
                u_x[gsl] = 0
                continue
            reqs.append(dist.isend(u_x[face(*own)].contiguous(), peer, tag=10 * axis + (step + 1)))
            buf = u_x.new_empty(u_x[gsl].shape)
            reqs.append(dist.irecv(buf, peer, tag=10 * axis + (1 - step)))
            recv.append((gsl, buf))
        for r in reqs:
            r.wait()
        for gsl, buf in recv:
            u_x[gsl] = buf
        done.append(axis)


def exchange_halos_diag(u_x, R: int, dist, topo: Topology, rank: int) -> int:
    """The paper's diagonal mode on the same blocks: one step in which the
    block exchanges with all 26 face, edge and corner neighbours at once
    (each message the R-deep part of the owned box next to that neighbour),
    instead of three axis steps.  Ghost regions beyond the grid are zero.
    Returns the number of messages sent."""
    nz, ny, nx = (s - 2 * R for s in u_x.shape)
    n = (nx, ny, nz)
    if min(n) < R:
        raise ValueError("a block needs at least R points along every axis")

    def rng(axis, d, ghost):
        if d == 0:
            return slice(R, R + n[axis])
        if ghost:
            return slice(0, R) if d < 0 else slice(n[axis] + R, n[axis] + 2 * R)
        return slice(R, 2 * R) if d < 0 else slice(n[axis], n[axis] + R)

    def code(off):
        return (off[0] + 1) + 3 * (off[1] + 1) + 9 * (off[2] + 1)

    cx, cy, cz = topo.coords(rank)
    reqs, recv, sent = [], [], 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                off = (dx, dy, dz)
                if off == (0, 0, 0):
                    continue
                gsl = (rng(2, dz, True), rng(1, dy, True), rng(0, dx, True))
                peer = topo.rank_of((cx + dx, cy + dy, cz + dz))
                if peer is None:
                    u_x[gsl] = 0
                    continue
                osl = (rng(2, dz, False), rng(1, dy, False), rng(0, dx, False))
                reqs.append(dist.isend(u_x[osl].contiguous(), peer, tag=100 + code(off)))
                sent += 1
                buf = u_x.new_empty(u_x[gsl].shape)
                reqs.append(dist.irecv(buf, peer, tag=100 + code((-dx, -dy, -dz))))
                recv.append((gsl, buf))
    for r in reqs:
        r.wait()
    for gsl, buf in recv:
        u_x[gsl] = buf
    return sent
