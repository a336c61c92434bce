"""Pins of the FP64 TTI oracle (oracle/tti.py) against closed forms and
special cases: the first-derivative weights (exact moment conditions and
textbook values), the rotated frame of Eq. rot, the discrete derivative
symbols on a periodic plane wave, brute-force stencil sums with the zero
ghost on a tiny grid, the reduction to the isotropic oracle when
eps = delta = 0 (any tilt), and plane waves of the coupled system that follow
its 2 x 2 discrete dispersion relation exactly."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import tti


@pytest.mark.parametrize("R", [1, 2, 3, 4, 6, 8])
def test_first_derivative_weights_moment_conditions(R):
    """sum_j 2 d_j j^(2p+1) = 1 for p = 0 and 0 for p = 1..R-1 (exact)."""
    d = [Fraction((-1) ** (j + 1) * math.factorial(R) ** 2,
                  j * math.factorial(R - j) * math.factorial(R + j)) for j in range(1, R + 1)]
    for p in range(R):
        s = sum(2 * dj * Fraction(j) ** (2 * p + 1) for j, dj in enumerate(d, 1))
        assert s == (1 if p == 0 else 0)
    np.testing.assert_allclose(tti.fd1_coefficients(R)[1:], [float(x) for x in d], rtol=1e-15)


def test_first_derivative_weights_textbook():
    np.testing.assert_allclose(tti.fd1_coefficients(1)[1:], [0.5])
    np.testing.assert_allclose(tti.fd1_coefficients(2)[1:], [2 / 3, -1 / 12])
    np.testing.assert_allclose(tti.fd1_coefficients(4)[1:], [4 / 5, -1 / 5, 4 / 105, -1 / 280])


def test_rotated_frame_is_orthonormal_and_follows_eq_rot():
    rng = np.random.default_rng(0)
    th, ph = rng.uniform(-1.5, 1.5, 50), rng.uniform(-3.1, 3.1, 50)
    xb, yb, zb = tti.frame(th, ph)
    F = np.stack([xb, yb, zb], -2)  # [..., 3 vectors, 3 components]
    np.testing.assert_allclose(F @ np.swapaxes(F, -1, -2), np.broadcast_to(np.eye(3), F.shape),
                               atol=1e-14)
    # D_xbar = cos t cos p d/dx + cos t sin p d/dy - sin t d/dz
    np.testing.assert_allclose(xb, np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph),
                                             -np.sin(th)], -1), atol=1e-15)
    # the symmetry axis is z when untilted
    _, _, z0 = tti.frame(np.zeros(1), np.array([0.7]))
    np.testing.assert_allclose(z0[0], [0.0, 0.0, 1.0], atol=1e-15)


@pytest.mark.parametrize("R", [1, 2, 4])
def test_derivatives_of_a_periodic_plane_wave(R):
    """On u = cos(k.x): D_aa u = (c0 + 2 sum c_j cos(j k_a h)) u / h^2 and
    D_ab u = -S_a S_b u / h^2 with S(k) = 2 sum d_j sin(j k h)."""
    n, h = (12, 10, 8), 10.0
    g = oracle.Grid(n=n, h=h, dt=1.0, R=R, periodic=True)
    k = [2 * math.pi * 2 / (n[0] * h), 2 * math.pi * 3 / (n[1] * h), 2 * math.pi * 1 / (n[2] * h)]
    z, y, x = np.meshgrid(*(np.arange(s) * h for s in g.padded_shape), indexing="ij")
    u = np.cos(k[0] * x + k[1] * y + k[2] * z)
    D = tti.second_derivatives(g, u)
    c = oracle.fd_coefficients(R)
    d = tti.fd1_coefficients(R)
    J = np.arange(1, R + 1)
    sym2 = [c[0] + 2 * np.sum(c[1:] * np.cos(J * ka * h)) for ka in k]
    S = [2 * np.sum(d[1:] * np.sin(J * ka * h)) for ka in k]
    ax = {"x": 0, "y": 1, "z": 2}
    for (a, b), v in D.items():
        ia, ib = ax[a], ax[b]
        want = (sym2[ia] if a == b else -S[ia] * S[ib]) * u / h ** 2
        np.testing.assert_allclose(v, want, atol=1e-12 * np.abs(want).max() + 1e-18)


def _iso_problem(R):
    from paper_2312_13094_gb300 import workloads as wl
    n, h = (14, 12, 13), 10.0
    v = wl.layered_model(n, h, 4, vmin=1.8, vmax=2.6)
    dt = 0.3 * h / 2.6
    nt = 30
    src = np.array([[61.0, 48.0, 57.0]])
    rec = np.array([[x, 55.0, 20.0] for x in np.linspace(0.0, 130.0, 7)])
    wav = wl.ricker(nt, dt, 30.0).reshape(nt, 1)
    return n, h, v, dt, nt, src, rec, wav


@pytest.mark.parametrize("R", [2, 4])
def test_isotropic_limit_equals_the_acoustic_oracle(R):
    """eps = delta = 0: H_0 + H_z is the Laplacian for any tilt (the rotated
    frame is orthonormal), p and q obey the same equation, and p is the
    isotropic oracle's wavefield (a separate C code path)."""
    n, h, v, dt, nt, src, rec, wav = _iso_problem(R)
    g = oracle.Grid(n=n, h=h, dt=dt, R=R, nbl=3)
    rng = np.random.default_rng(R)
    shp = g.phys_shape
    theta = 0.6 + 0.2 * rng.standard_normal(shp)
    phi = 1.1 + 0.3 * rng.standard_normal(shp)
    zero = np.zeros(shp)
    out = tti.forward(g, v, zero, zero, theta, phi, nt, src, wav, rec)
    ref = oracle.forward(g, 1.0 / v.astype(np.float64) ** 2, nt, src, wav, rec)
    scale = np.abs(ref["u_cur"]).max()
    assert scale > 0
    np.testing.assert_allclose(out["p"], ref["u_cur"], atol=1e-11 * scale)
    np.testing.assert_allclose(out["q"], ref["u_cur"], atol=1e-11 * scale)
    np.testing.assert_allclose(out["rec"], ref["rec"], atol=1e-11 * np.abs(ref["rec"]).max())


def _tti_symbols(R, k, h, theta, phi):
    c = oracle.fd_coefficients(R)
    d = tti.fd1_coefficients(R)
    J = np.arange(1, R + 1)
    sym = np.zeros((3, 3))
    S = [2 * np.sum(d[1:] * np.sin(J * ka * h)) for ka in k]
    for a in range(3):
        for b in range(3):
            sym[a, b] = (c[0] + 2 * np.sum(c[1:] * np.cos(J * k[a] * h))) if a == b \
                else -S[a] * S[b]
    xb, yb, zb = (f.reshape(3) for f in tti.frame(np.array(theta), np.array(phi)))
    hz = zb @ sym @ zb / h ** 2
    h0 = (xb @ sym @ xb + yb @ sym @ yb) / h ** 2
    return h0, hz


@pytest.mark.parametrize("R", [2, 4])
@pytest.mark.parametrize("mode", [0, 1])
def test_plane_waves_follow_the_coupled_dispersion_relation(R, mode):
    """Periodic plane wave (p, q) = (a_p, a_q) cos(k.x - w t) with (a_p, a_q)
    an eigenvector of M = [[e h0, d hz], [d h0, hz]] (e = 1+2eps, d =
    sqrt(1+2delta), h0 and hz the operator symbols) and
    cos(w dt) = 1 + (dt^2/m) lambda / 2: an exact solution of the scheme for
    both the quasi-P (mode 0) and the slower (mode 1) branch."""
    n, h, v = (16, 12, 10), 10.0, 2.0
    eps, delta, theta, phi = 0.2, 0.1, 0.5, 0.8
    dt = 0.25 * h / (v * math.sqrt(1 + 2 * eps))
    g = oracle.Grid(n=n, h=h, dt=dt, R=R, periodic=True)
    k = [2 * math.pi * 3 / (n[0] * h), 2 * math.pi * 2 / (n[1] * h), 2 * math.pi * 1 / (n[2] * h)]
    h0, hz = _tti_symbols(R, k, h, theta, phi)
    e, dd = 1 + 2 * eps, math.sqrt(1 + 2 * delta)
    M = np.array([[e * h0, dd * hz], [dd * h0, hz]])
    lam, vec = np.linalg.eig(M)
    order = np.argsort(lam)  # most negative first: the faster branch
    lam, vec = lam[order].real, vec[:, order].real
    a = dt ** 2 * v ** 2
    w = math.acos(1 + a * lam[mode] / 2) / dt
    ap, aq = vec[:, mode]
    z, y, x = np.meshgrid(*(np.arange(s) * h for s in g.padded_shape), indexing="ij")
    ph = k[0] * x + k[1] * y + k[2] * z
    shp = g.phys_shape
    full = np.ones(shp)
    nt = 40
    st = (ap * np.cos(ph + w * dt), ap * np.cos(ph), aq * np.cos(ph + w * dt), aq * np.cos(ph))
    out = tti.forward(g, v * full, eps * full, delta * full, theta * full, phi * full, nt,
                      np.zeros((0, 3)), np.zeros((nt, 0)), np.zeros((0, 3)), state=st)
    np.testing.assert_allclose(out["p"], ap * np.cos(ph - w * nt * dt), atol=1e-10)
    np.testing.assert_allclose(out["q"], aq * np.cos(ph - w * nt * dt), atol=1e-10)
    # guard: the isotropic frequency of the same wavenumber is not a solution
    wi = math.acos(1 + a * (h0 + hz) / 2) / dt
    assert abs(wi - w) > 1e-3 * w


def test_source_reaches_both_fields_and_receivers_read_p():
    n, h, v, dt, nt, src, rec, wav = _iso_problem(2)
    g = oracle.Grid(n=n, h=h, dt=dt, R=2, nbl=2)
    shp = g.phys_shape
    out = tti.forward(g, v, np.full(shp, 0.15), np.full(shp, 0.05), np.full(shp, 0.4),
                      np.full(shp, 0.3), nt, src, wav, rec)
    assert np.abs(out["p"]).max() > 0 and np.abs(out["q"]).max() > 0
    assert np.all(out["rec"][0] == 0)
    # receivers interpolate p
    w = [oracle.point_weights(g, r) for r in rec]
    last = np.array([np.dot(wt, out["p_prev"].reshape(-1)[i]) for i, wt in w])
    np.testing.assert_allclose(out["rec"][-1], last, rtol=1e-12, atol=1e-300)


def test_derivatives_match_brute_force_sums_with_the_zero_ghost():
    """Every D_ab of a random field on a tiny non-periodic grid equals the
    explicit double sum over the stencil points, with values beyond the grid
    taken as zero (the read-only ghost), evaluated point by point."""
    R = 2
    g = oracle.Grid(n=(6, 5, 4), h=2.0, dt=1.0, R=R)
    rng = np.random.default_rng(7)
    u = rng.standard_normal(g.padded_shape)
    D = tti.second_derivatives(g, u)
    c = oracle.fd_coefficients(R)
    d = tti.fd1_coefficients(R)
    Nz, Ny, Nx = u.shape

    def val(z, y, x):
        return u[z, y, x] if 0 <= z < Nz and 0 <= y < Ny and 0 <= x < Nx else 0.0

    ax = {"x": 2, "y": 1, "z": 0}
    for (a, b), got in D.items():
        for z in range(Nz):
            for y in range(Ny):
                for x in range(Nx):
                    p = [z, y, x]
                    if a == b:
                        acc = c[0] * val(*p)
                        for j in range(1, R + 1):
                            for s in (1, -1):
                                q = list(p)
                                q[ax[a]] += s * j
                                acc += c[j] * val(*q)
                    else:
                        acc = 0.0
                        for i in range(-R, R + 1):
                            for j in range(-R, R + 1):
                                if i == 0 or j == 0:
                                    continue
                                q = list(p)
                                q[ax[a]] += i
                                q[ax[b]] += j
                                acc += np.sign(i) * d[abs(i)] * np.sign(j) * d[abs(j)] * val(*q)
                    assert abs(got[z, y, x] - acc / g.h ** 2) <= 1e-12 * (1 + abs(acc))


def _max_eigen(R, eps, delta, theta, phi, nk=10):
    """Largest |eigenvalue| (times h^2) of the 2 x 2 symbol matrix of the
    discrete TTI system over a grid of wavenumbers k h in [0, pi]^3 (the
    symbol is even in k, so one octant with both signs of two axes)."""
    c = oracle.fd_coefficients(R)
    d = tti.fd1_coefficients(R)
    J = np.arange(1, R + 1)
    xb, yb, zb = (f.reshape(3) for f in tti.frame(np.array(theta), np.array(phi)))
    e, dl = 1 + 2 * eps, math.sqrt(1 + 2 * delta)
    worst = 0.0
    for kx in np.linspace(0, np.pi, nk):
        for ky in np.linspace(-np.pi, np.pi, 2 * nk):
            for kz in np.linspace(-np.pi, np.pi, 2 * nk):
                k = (kx, ky, kz)
                S = [2 * np.sum(d[1:] * np.sin(J * ka)) for ka in k]
                s2 = [c[0] + 2 * np.sum(c[1:] * np.cos(J * ka)) for ka in k]
                sym = np.array([[s2[a] if a == b else -S[a] * S[b] for b in range(3)]
                                for a in range(3)])
                hz, h0 = zb @ sym @ zb, xb @ sym @ xb + yb @ sym @ yb
                lam = np.linalg.eigvals(np.array([[e * h0, dl * hz], [dl * h0, hz]]))
                worst = max(worst, float(np.max(np.abs(lam))))
    return worst


@pytest.mark.parametrize("R", [2, 4])
def test_accepted_tti_models_are_stable_in_the_workload_ranges(R):
    """Frozen-coefficient (von Neumann) analysis: leapfrog stability needs
    (dt^2 v^2 / h^2) |lambda| <= 4 for every eigenvalue of the symbol matrix.
    Over the workloads' ranges (eps <= 0.2, delta = eps / 2, tilt <= 0.6 rad,
    azimuths 0..1.2 rad), sampled on a wavenumber grid that includes the
    Nyquist corners, the largest Courant number v sqrt(1+2 eps) dt / h this
    allows is above the isotropic limit the library checks against, so the
    check is conservative there; with eps = delta = 0 the bound is exactly the
    isotropic one."""
    c = oracle.fd_coefficients(R)
    iso = -c[0] - 2 * np.sum(c[1:] * (-1.0) ** np.arange(1, R + 1))  # 1-D Nyquist symbol
    iso_limit = math.sqrt(4.0 / (3.0 * iso))
    assert abs(math.sqrt(4.0 / _max_eigen(R, 0.0, 0.0, 0.3, 0.5)) - iso_limit) < 1e-9
    lam = max(_max_eigen(R, 0.2, 0.1, t, p) for t in (0.0, 0.3, 0.6) for p in (0.0, 0.6, 1.2))
    tti_limit = math.sqrt(4.0 * 1.4 / lam)  # in units of the fast speed v sqrt(1 + 2 eps)
    assert tti_limit > iso_limit
