"""Write the FP64 oracle's run of the full headline workload to tests/golden.

The headline workload (512^3 physical cells + 40-cell layer = 592^3, h 10 m,
SO 8, 1000 leapfrog steps, two-layer model with a seeded smooth perturbation,
15 Hz Ricker at the centre, 512 receivers at z = 2.5 cells) is stepped once by
the FP64 oracle (Eq. 1 of App. A discretised as in Sec. IV-B, the layer of
Sec. IV-C, the point weights of Sec. III "Sparse data").  The script imports
only ``oracle`` and the seeded input generators; nothing here comes from the
CUDA path.

Stored (``acoustic_512_so8_1000.npz``):
  rec        [1000][512] float32  receivers I(u^n), n = 0..999 (2.5 km from the
                                  source, they see no arrival within the 1.27 s
                                  simulated: only the stencil's precursor, ~1e-33)
  pts        [K][3]      int32    physical (z, y, x) of sampled cells
  u_last     [K]         float64  u^1000 at those cells
  u_prev     [K]         float64  u^999 at those cells
  and the run's metadata (workload name, steps, seconds, threads).

It took 4726 s on 6 host threads (x86) and ~12 GB of RAM:

    OMP_NUM_THREADS=8 python tests/golden/make_acoustic_512_golden.py
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2312_13094_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(HERE, "acoustic_512_so8_1000.npz")


def sample_points(n: int, seed: int = 7) -> np.ndarray:
    """Physical cells to keep: random cells everywhere, the receiver line's
    neighbourhood, the source's neighbourhood, the corners and the faces."""
    rng = np.random.default_rng(seed)
    pts = [rng.integers(0, n, size=(12000, 3))]
    half = n // 2
    zs = np.arange(0, 6)
    xs = rng.integers(0, n, 2000)
    pts.append(np.stack([rng.choice(zs, 2000), np.full(2000, half - 1) + rng.integers(0, 2, 2000),
                         xs], 1))
    pts.append(half - 4 + rng.integers(0, 8, size=(2000, 3)))
    corner = np.array([[z, y, x] for z in (0, n - 1) for y in (0, n - 1) for x in (0, n - 1)])
    pts.append(corner)
    face = rng.integers(0, n, size=(4000, 3))
    face[np.arange(4000), rng.integers(0, 3, 4000)] = rng.choice([0, 1, n - 2, n - 1], 4000)
    pts.append(face)
    return np.unique(np.concatenate(pts).astype(np.int32), axis=0)


def main():
    w = wl.acoustic_512()
    n, nbl = w["n"][0], w["nbl"]
    og = oracle.Grid(n=w["n"], h=w["h"], dt=w["dt"], R=w["space_order"] // 2, nbl=nbl)
    m = 1.0 / w["v"].astype(np.float64) ** 2
    del w["v"]
    t0 = time.time()
    out = oracle.forward(og, m, w["nt"], w["src"], w["wavelet"], w["rec"])
    seconds = time.time() - t0
    pts = sample_points(n)
    z, y, x = (pts[:, a] + nbl for a in range(3))
    meta = {"workload": w["name"], "nt": w["nt"], "padded": list(og.padded_shape),
            "seconds": seconds, "threads": os.environ.get("OMP_NUM_THREADS", "all")}
    np.savez_compressed(OUT, rec=out["rec"].astype(np.float32), pts=pts,
                        u_last=out["u_cur"][z, y, x], u_prev=out["u_prev"][z, y, x],
                        meta=json.dumps(meta))
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
