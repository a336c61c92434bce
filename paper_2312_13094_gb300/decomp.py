"""Domain decomposition of one grid along z (the paper's basic mode, Sec. III:
each subdomain exchanges an R-deep halo with its neighbours before every step).

This module holds only the data movement of that scheme: which padded z planes
a rank owns, and the halo exchange that fills the R ghost planes on either
side of a rank's slab with its neighbours' edge planes.  The step itself is
whatever the caller computes on the slab (the FD kernels of libfd.so need a
slab with ghost planes of their own, which they do not have yet; the CPU tests
run the exchange between gloo ranks around the FP64 reference step).

Layout of a rank's extended array: [R ghost planes | nzs owned planes | R ghost
planes] along the first axis; ghost planes beyond the global grid stay zero
(the read-only zero halo of Sec. III).
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
    ends of the grid they are set to zero.  Every rank must call this with
    the same R; each slab needs at least R owned planes."""
    nzs = u_x.shape[0] - 2 * R
    if nzs < R:
        raise ValueError(f"a slab of {nzs} planes cannot feed an {R}-plane halo")
    reqs = []
    if rank > 0:
        reqs.append(dist.isend(u_x[R:2 * R].contiguous(), rank - 1, tag=1))
        lo = u_x.new_empty(u_x[0:R].shape)
        reqs.append(dist.irecv(lo, rank - 1, tag=2))
    else:
        lo = None
        u_x[0:R].zero_()
    if rank + 1 < world:
        reqs.append(dist.isend(u_x[nzs:nzs + R].contiguous(), rank + 1, tag=2))
        hi = u_x.new_empty(u_x[nzs + R:].shape)
        reqs.append(dist.irecv(hi, rank + 1, tag=1))
    else:
        hi = None
        u_x[nzs + R:].zero_()
    for r in reqs:
        r.wait()
    if lo is not None:
        u_x[0:R].copy_(lo)
    if hi is not None:
        u_x[nzs + R:].copy_(hi)
