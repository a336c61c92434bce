"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module generates INPUT DATA only (velocity models, source and receiver
positions, source wavelets).  It holds none of the finite-difference method's
arithmetic, so the FP64 oracle and the CUDA path can both be fed from it
without sharing any part of the computation.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here so that the
draws are identical on every platform; Gaussian deviates use Box-Muller.

Units follow the usual seismic convention: h in m, dt in ms, velocity in km/s
(= m/ms), frequency given in Hz and converted to 1/ms.

Workloads (the paper's Sec. IV-C uses seeded synthetic models with a Ricker
source; no dataset is involved):
  * ``small_acoustic``   64^3, h 10 m, SO 4, 100 steps, v = 1.5, 10-cell layer
  * ``acoustic_512``     512^3, h 10 m, SO 8, 1000 steps, two layers
                         1.5/3.0 km/s x (1 + 5 % smooth noise), 40-cell layer
  * ``batched_shots``    32 windows 128^3..320^3, SO 8, 600 steps
  * ``adjoint_256``      256^3, SO 8, 500 steps, Gaussian anomaly
  * ``learned_pair``     fine 512^3 h 10 SO 16 / coarse 256^3 h 20 SO 8
  * ``tti_workload``     smooth TTI media (layered vp, eps, delta, tilt and
                         azimuth), ``tti_896`` the paper's 896^3 SO 8 grid
"""
from __future__ import annotations

import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` outputs of splitmix64 started from ``seed``; output k is the
    mix of state seed + (offset + k + 1) * golden."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in (0, 1) from the top 53 bits."""
    z = splitmix64(seed, count, offset) >> np.uint64(11)
    return (z.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal deviates by Box-Muller on pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    th = 2.0 * np.pi * u[1::2]
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(th)
    out[1::2] = r * np.sin(th)
    return out[:count]


def ricker(nt: int, dt_ms: float, f_hz: float, t0_ms: float | None = None,
           dtype=np.float32) -> np.ndarray:
    """Ricker wavelet q(t_n), t_n = n dt, amplitude 1, delay t0 = 1/f."""
    f = f_hz / 1000.0  # 1/ms
    t0 = 1.0 / f if t0_ms is None else t0_ms
    t = np.arange(nt, dtype=np.float64) * dt_ms - t0
    a = (np.pi * f * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(dtype)


def _gauss_smooth(x: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian smoothing (truncated at 4 sigma, edge mode
    'nearest'), applied to input noise only."""
    from scipy.ndimage import gaussian_filter1d
    out = x
    for ax in range(x.ndim):
        out = gaussian_filter1d(out, sigma, axis=ax, mode="nearest",
                                truncate=4.0)
    return out


def smooth_layers(n, h, interfaces_m, velocities, width_m=40.0):
    """Velocity column for horizontally layered media with tanh-smoothed
    interfaces (depth axis z = last axis of ``n``).  Returns v[nz]."""
    nz = n[2]
    z = np.arange(nz, dtype=np.float64) * h
    v = np.full(nz, velocities[0], dtype=np.float64)
    for zi, (va, vb) in zip(interfaces_m, zip(velocities[:-1], velocities[1:])):
        v += (vb - va) * 0.5 * (1.0 + np.tanh((z - zi) / (0.5 * width_m)))
    return v


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def small_acoustic(n: int = 64):
    """64^3 correctness workload: SO 4, 100 steps at CFL 0.4, v = 1.5 km/s,
    10-cell layer, 10 Hz Ricker at the centre, 64 receivers at z = 2 cells."""
    h, vmax = 10.0, 1.5
    dt = 0.4 * h / vmax
    nt = 100
    v = np.full((n, n, n), 1.5, dtype=np.float32)
    c = (n - 1) / 2.0 * h
    src = np.array([[c, c, c]])
    nrec = n
    rec = np.stack([np.arange(nrec) * h * (n - 1) / (nrec - 1),
                    np.full(nrec, c), np.full(nrec, 2.0 * h)], axis=1)
    return dict(name=f"acoustic {n}^3 SO4 h10 100 steps", n=(n, n, n), h=h,
                space_order=4, nbl=10, dt=dt, nt=nt, v=v, src=src, rec=rec,
                wavelet=ricker(nt, dt, 10.0).reshape(nt, 1), f0=10.0)


def acoustic_512(n: int = 512, nt: int = 1000, seed: int = 2, nbl: int = 40):
    """Headline workload: n^3 (+2*nbl layer) h 10 m SO 8, two layers
    1.5/3.0 km/s split at half depth, times (1 + p) with p seeded white noise
    smoothed by a sigma = 4-cell Gaussian and scaled to max |p| = 0.05;
    15 Hz Ricker at the centre, n receivers on a line at z = 2.5 cells."""
    h = 10.0
    half = n // 2
    vcol = np.where(np.arange(n) < half, 1.5, 3.0)
    p = normal(seed, n * n * n).reshape(n, n, n).astype(np.float32)
    p = _gauss_smooth(p, 4.0)
    p *= np.float32(0.05 / float(np.abs(p).max()))
    v = (vcol[:, None, None].astype(np.float32) * (1.0 + p)).astype(np.float32)
    vmax = 3.0 * 1.05
    dt = 0.4 * h / vmax
    c = (half - 0.5) * h
    src = np.array([[c, c, c]])
    nrec = n
    rec = np.stack([(0.5 + np.arange(nrec) * (n - 2) / (nrec - 1)) * h,
                    np.full(nrec, (half - 0.25) * h),
                    np.full(nrec, 2.5 * h)], axis=1)
    return dict(name=f"acoustic {n}^3 SO8 h10 {nt} steps", n=(n, n, n), h=h,
                space_order=8, nbl=nbl, dt=dt, nt=nt, v=v, src=src, rec=rec,
                wavelet=ricker(nt, dt, 15.0).reshape(nt, 1), f0=15.0)


def layered_model(n, h, seed: int, vmin=1.5, vmax=4.5, width_m=40.0, depth_m=None):
    """3-8 horizontal layers, velocities i.i.d. U[vmin, vmax], interface depths
    uniform in [0, depth_m) (default: the column, n_z h), interfaces
    tanh-smoothed.  The same seed and depth_m give the same medium sampled at
    any spacing h."""
    u = uniform(seed, 32)
    nl = 3 + int(u[0] * 6)  # 3..8
    vels = list(vmin + (vmax - vmin) * u[1:1 + nl])
    depth = n[2] * h if depth_m is None else depth_m
    ifs = sorted(depth * u[10:10 + nl - 1])
    col = smooth_layers(n, h, ifs, vels, width_m)
    v = np.broadcast_to(col[:, None, None].astype(np.float32),
                        (n[2], n[1], n[0])).copy()
    return v


def batched_shots(nshots: int = 32, nt: int = 600, seed: int = 3,
                  lo: int = 128, hi: int = 320, nbl: int = 20):
    """Shots with uneven windows: dims per axis i.i.d. uniform integers in
    [lo, hi] rounded to a multiple of 4, layered v in [1.5, 4.5] km/s, common
    dt = 0.4 h / 4.5, 15 Hz Ricker at the window centre, 128 receivers."""
    h = 10.0
    dt = 0.4 * h / 4.5
    u = uniform(seed, 3 * nshots)
    shots = []
    for s in range(nshots):
        dims = [int(round((lo + u[3 * s + a] * (hi - lo)) / 4.0)) * 4
                for a in range(3)]
        dims = [min(max(d, lo), hi) for d in dims]
        n = tuple(dims)
        v = layered_model(n, h, seed + 1 + s)
        cx, cy, cz = [(d - 1) / 2.0 * h for d in n]
        src = np.array([[cx, cy, cz]])
        nrec = 128
        rec = np.stack([np.linspace(0.0, (n[0] - 1) * h, nrec),
                        np.full(nrec, cy), np.full(nrec, 2.5 * h)], axis=1)
        shots.append(dict(name=f"shot {s}", n=n, h=h, space_order=8, nbl=nbl,
                          dt=dt, nt=nt, v=v, src=src, rec=rec,
                          wavelet=ricker(nt, dt, 15.0).reshape(nt, 1), f0=15.0))
    return shots


def adjoint_256(n: int = 256, nt: int = 500, nbl: int = 20, anomaly=True):
    """Gradient workload: v = 2.0 + 0.2 exp(-r^2 / (2 (20 h)^2)) centred
    (true model) or v = 2.0 (start model); 10 Hz Ricker at (n/2, n/2, n/4)h;
    32 x 32 receivers at z = 3n/4 cells."""
    h = 10.0
    dt = 0.4 * h / 2.2
    ax = np.arange(n, dtype=np.float64)
    c = (n - 1) / 2.0
    r2 = ((ax[None, None, :] - c) ** 2 + (ax[None, :, None] - c) ** 2
          + (ax[:, None, None] - c) ** 2)
    shape = np.exp(-r2 / (2.0 * (n / 12.8) ** 2))
    v = (2.0 + (0.2 * shape if anomaly else np.zeros_like(shape))).astype(np.float32)
    src = np.array([[n / 2 * h, n / 2 * h, n / 4 * h]])
    g = np.linspace(0.0, (n - 1) * h, 32)
    gx, gy = np.meshgrid(g, g, indexing="xy")
    rec = np.stack([gx.ravel(), gy.ravel(),
                    np.full(gx.size, 0.75 * n * h)], axis=1)
    return dict(name=f"adjoint {n}^3 SO8 h10 {nt} steps", n=(n, n, n), h=h,
                space_order=8, nbl=nbl, dt=dt, nt=nt, v=v, src=src, rec=rec,
                wavelet=ricker(nt, dt, 10.0).reshape(nt, 1), f0=10.0,
                shape=shape.astype(np.float32))


def random_state(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Uniform [-scale, scale) field for wavefield-state tests."""
    count = int(np.prod(shape))
    return ((uniform(seed, count) * 2.0 - 1.0) * scale).reshape(shape)


def cfl_dt(h: float, vmax: float, courant: float = 0.4) -> float:
    return courant * h / vmax


__all__ = [name for name in globals() if not name.startswith("_")
           and name not in ("annotations", "math", "np")]


def tti_model(n, h: float, seed: int, vmin: float = 1.5, vmax: float = 3.5):
    """Smooth anisotropic (TTI) medium on an n = (nx, ny, nz) grid, physical
    float32 arrays [nz][ny][nx]: a layered vp (3-6 layers, tanh interfaces),
    Thomsen eps in [0.05, 0.2] with delta = eps / 2, tilt theta in
    [0, 0.6] rad and azimuth phi in [0, 1.2] rad, each a product of seeded
    low-wavenumber sines along the three axes (cheap to build at any size)."""
    nx, ny, nz = n
    u = uniform(seed, 32)
    nl = 3 + int(u[0] * 4)
    depth = (nz - 1) * h
    zi = np.sort(u[1:nl] * depth)
    vel = np.sort(vmin + (vmax - vmin) * u[8:8 + nl])
    vz = smooth_layers(n, h, zi, vel).astype(np.float32)

    def field(k):
        ax = [np.sin(2 * np.pi * (0.5 + u[16 + 3 * k + a]) * np.arange(m) / max(m - 1, 1)
                     + 6.28 * u[16 + 3 * k + a] + 1.0).astype(np.float32)
              for a, m in enumerate((nx, ny, nz))]
        return 0.5 + 0.5 * (ax[2][:, None, None] * ax[1][None, :, None] * ax[0][None, None, :])

    shape = (nz, ny, nx)
    v = np.broadcast_to(vz[:, None, None], shape).astype(np.float32)
    eps = (0.05 + 0.15 * field(0)).astype(np.float32)
    delta = (0.5 * eps).astype(np.float32)
    theta = (0.6 * field(1)).astype(np.float32)
    phi = (1.2 * field(2)).astype(np.float32)
    return v, eps, delta, theta, phi


def tti_workload(n=(40, 36, 32), so: int = 8, nbl: int = 6, nt: int = 60, seed: int = 11,
                 courant: float = 0.35, f_hz: float = 15.0, name: str | None = None):
    """TTI modelling: tti_model medium, dt from the fastest speed
    v sqrt(1+2 eps), Ricker at the centre, a line of receivers at z = 2.5 h."""
    h = 10.0
    v, eps, delta, theta, phi = tti_model(n, h, seed)
    vfast = float(np.max(v[:, :1, :1] * np.sqrt(1.0 + 2.0 * eps.max())))
    dt = courant * h / vfast
    ext = [(d - 1) * h for d in n]
    src = np.array([[0.5 * ext[0], 0.5 * ext[1], 0.5 * ext[2]]])
    nrec = min(n[0], 128)
    rec = np.stack([np.linspace(0.0, ext[0], nrec), np.full(nrec, 0.5 * ext[1]),
                    np.full(nrec, min(2.5 * h, ext[2]))], axis=1)
    wav = ricker(nt, dt, f_hz).reshape(nt, 1)
    return dict(name=name or f"tti {n[0]}x{n[1]}x{n[2]} SO{so} h10 {nt} steps", n=tuple(n), h=h,
                space_order=so, nbl=nbl, dt=dt, nt=nt, v=v, eps=eps, delta=delta, theta=theta,
                phi=phi, src=src, rec=rec, wavelet=wav)


def tti_896(n: int = 896, nt: int = 100):
    """The paper's single-GPU TTI grid (Sec. IV-C: 896^3 with a 40-cell
    absorbing layer, SO 8), 15 Hz Ricker at the centre."""
    return tti_workload(n=(n, n, n), so=8, nbl=40, nt=nt, seed=12,
                        name=f"tti {n}^3 SO8 h10 {nt} steps")
