"""FP64 reference of the anisotropic acoustic (TTI) time step.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy on padded
(Nz, Ny, Nx) arrays, x fastest; one step is written out term by term.

Sec. IV-B ("Anisotropic acoustic") and App. A (Eq. rot) of the paper: the TTI
model couples two scalar fields through a rotated anisotropic Laplacian whose
x-bar component is G_xbar = D_xbar^T D_xbar with
D_xbar = cos(theta) cos(phi) d/dx + cos(theta) sin(phi) d/dy - sin(theta) d/dz,
theta the tilt and phi the azimuth (both per cell); the rest of the system is
left to the cited formulation (Zhang et al. 2011).  Readings taken here:

* Rotated frame: xbar = (cos t cos p, cos t sin p, -sin t) from Eq. rot,
  zbar = (sin t cos p, sin t sin p, cos t) (the symmetry axis) and
  ybar = zbar x xbar = (-sin p, cos p, 0); an orthonormal basis.
* Operators ("centred" form, pointwise angles): with D_ab the discrete second
  derivative along axes a, b,
      H_z u = sum_ab zbar_a zbar_b D_ab u,
      H_0 u = sum_ab (xbar_a xbar_b + ybar_a ybar_b) D_ab u,
  D_aa the centred order-2R second-derivative weights (as for the isotropic
  stencil), D_ab (a != b) the product of the centred order-2R first-derivative
  weights along a and b.  At space order 16 the stencil then touches the 769
  points of the paper's TTI stencil figure: the 49-point star and three
  16 x 16 squares (the xy, xz and yz planes through the point).
* System (pseudo-acoustic, Zhang et al. 2011):
      m p_tt + eta p_t = (1+2 eps) H_0 p + sqrt(1+2 delta) H_z q + s,
      m q_tt + eta q_t = sqrt(1+2 delta) H_0 p + H_z q + s,
  the source s injected into both fields, receivers interpolating p.
* Time stepping, damping layer, zero ghost, source scaling and point weights
  exactly as for the isotropic path (fd_oracle.c), with the layer strength
  taken from the fastest (horizontal) speed v sqrt(1+2 eps).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from . import Grid, damping, fd_coefficients, pad_model, point_weights

AXES = ("x", "y", "z")


def fd1_coefficients(R: int) -> np.ndarray:
    """Centred first-derivative weights of order 2R: d[j], j = 0..R (d[0] = 0,
    d[-j] = -d[j]); d_j = (-1)^(j+1) (R!)^2 / (j (R-j)! (R+j)!)."""
    d = np.zeros(R + 1)
    for j in range(1, R + 1):
        d[j] = float(Fraction((-1) ** (j + 1) * math.factorial(R) ** 2,
                              j * math.factorial(R - j) * math.factorial(R + j)))
    return d


def frame(theta, phi):
    """(xbar, ybar, zbar), each [..., 3] in (x, y, z) component order."""
    ct, st, cp, sp = np.cos(theta), np.sin(theta), np.cos(phi), np.sin(phi)
    xb = np.stack([ct * cp, ct * sp, -st], -1)
    zb = np.stack([st * cp, st * sp, ct], -1)
    yb = np.cross(zb, xb)
    return xb, yb, zb


def _shift(g: Grid, u, dx=0, dy=0, dz=0):
    """v[z, y, x] = u[z + dz, y + dy, x + dx]: zero beyond the padded grid, or
    wrapped around when the grid is periodic."""
    if g.periodic:
        return np.roll(u, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
    out = np.zeros_like(u)
    Nz, Ny, Nx = u.shape

    def rng(n, d):
        return slice(max(0, -d), min(n, n - d)), slice(max(0, d), min(n, n + d))

    (oz, iz), (oy, iy), (ox, ix) = rng(Nz, dz), rng(Ny, dy), rng(Nx, dx)
    out[oz, oy, ox] = u[iz, iy, ix]
    return out


def second_derivatives(g: Grid, u):
    """{(a, b): D_ab u} for the six axis pairs a <= b, in units of 1/h^2."""
    R = g.R
    c = fd_coefficients(R)
    d = fd1_coefficients(R)
    unit = {"x": (1, 0, 0), "y": (0, 1, 0), "z": (0, 0, 1)}
    D = {}
    for a in AXES:
        ea = unit[a]
        acc = c[0] * u
        for j in range(1, R + 1):
            acc = acc + c[j] * (_shift(g, u, *(j * e for e in ea)) +
                                _shift(g, u, *(-j * e for e in ea)))
        D[(a, a)] = acc / g.h ** 2
    for a, b in (("x", "y"), ("x", "z"), ("y", "z")):
        ea, eb = unit[a], unit[b]
        acc = np.zeros_like(u)
        for i in range(1, R + 1):
            for j in range(1, R + 1):
                def at(si, sj):
                    return _shift(g, u, *(si * i * p + sj * j * q for p, q in zip(ea, eb)))
                acc = acc + d[i] * d[j] * (at(1, 1) - at(-1, 1) - at(1, -1) + at(-1, -1))
        D[(a, b)] = acc / g.h ** 2
    return D


def operators(g: Grid, u, theta_pad, phi_pad):
    """(H_0 u, H_z u) on the padded grid with per-cell angles."""
    D = second_derivatives(g, u)
    xb, yb, zb = frame(theta_pad, phi_pad)
    h0 = np.zeros_like(u)
    hz = np.zeros_like(u)
    for ia, a in enumerate(AXES):
        for ib, b in enumerate(AXES):
            Dab = D[(a, b)] if (a, b) in D else D[(b, a)]
            hz = hz + zb[..., ia] * zb[..., ib] * Dab
            h0 = h0 + (xb[..., ia] * xb[..., ib] + yb[..., ia] * yb[..., ib]) * Dab
    return h0, hz


def step(g: Grid, m_pad, eps_pad, delta_pad, theta_pad, phi_pad, b, p_prev, p, q_prev, q,
         src=None):
    """One damped leapfrog step of the coupled system; src = (flat padded
    indices, values) of s^n (already q(t_n) w / h^3).  Returns (p_next,
    q_next)."""
    h0p, _ = operators(g, p, theta_pad, phi_pad)
    _, hzq = operators(g, q, theta_pad, phi_pad)
    s = np.zeros_like(p)
    if src is not None:
        np.add.at(s.reshape(-1), src[0], src[1])
    e2 = 1.0 + 2.0 * eps_pad
    dl = np.sqrt(1.0 + 2.0 * delta_pad)
    rp = e2 * h0p + dl * hzq + s
    rq = dl * h0p + hzq + s
    a = g.dt ** 2 / m_pad
    p_next = (2.0 * p - (1.0 - b) * p_prev + a * rp) / (1.0 + b)
    q_next = (2.0 * q - (1.0 - b) * q_prev + a * rq) / (1.0 + b)
    return p_next, q_next


def forward(g: Grid, vp, eps, delta, theta, phi, nt: int, src_xyz, wavelet, rec_xyz, *,
            state=None):
    """nt steps from rest (or from state = (p_prev, p, q_prev, q), padded).
    Physical [nz][ny][nx] models: vp in km/s, eps and delta (Thomsen), theta
    and phi in radians.  Returns rec [nt, nrec] = I(p^n) and the final state."""
    vp = np.asarray(vp, dtype=np.float64)
    m_pad = pad_model(g, 1.0 / vp ** 2)
    eps_pad = pad_model(g, np.asarray(eps, dtype=np.float64))
    delta_pad = pad_model(g, np.asarray(delta, dtype=np.float64))
    theta_pad = pad_model(g, np.asarray(theta, dtype=np.float64))
    phi_pad = pad_model(g, np.asarray(phi, dtype=np.float64))
    vmax = float(np.max(vp * np.sqrt(1.0 + 2.0 * np.asarray(eps, dtype=np.float64))))
    b = damping(g, vmax)
    shp = g.padded_shape
    if state is None:
        p_prev, p, q_prev, q = (np.zeros(shp) for _ in range(4))
    else:
        p_prev, p, q_prev, q = (np.array(s, dtype=np.float64) for s in state)
    src_xyz = np.asarray(src_xyz, dtype=np.float64).reshape(-1, 3)
    rec_xyz = np.asarray(rec_xyz, dtype=np.float64).reshape(-1, 3)
    wavelet = np.asarray(wavelet, dtype=np.float64).reshape(-1, max(len(src_xyz), 1))
    sw = [point_weights(g, s) for s in src_xyz]
    rw = [point_weights(g, r) for r in rec_xyz]
    if any(x is None for x in sw + rw):
        raise ValueError("source or receiver outside the physical box")
    rec = np.zeros((nt, len(rec_xyz)))
    for n in range(nt):
        flat = p.reshape(-1)
        for r, (idx, w) in enumerate(rw):
            rec[n, r] = np.dot(w, flat[idx])
        src = None
        if len(sw):
            idx = np.concatenate([i for i, _ in sw])
            val = np.concatenate([w * wavelet[n, s] / g.h ** 3 for s, (_, w) in enumerate(sw)])
            src = (idx, val)
        pn, qn = step(g, m_pad, eps_pad, delta_pad, theta_pad, phi_pad, b, p_prev, p, q_prev,
                      q, src)
        p_prev, p, q_prev, q = p, pn, q, qn
    return {"rec": rec, "p_prev": p_prev, "p": p, "q_prev": q_prev, "q": q}
