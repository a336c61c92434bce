"""Pins of the FP64 oracle against facts fixed outside it: exact rationals,
the paper's printed worked example, closed-form discrete and continuum
solutions, conservation laws and brute force.  CPU only."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2312_13094_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# FD weights
# --------------------------------------------------------------------------

def _weights_from_moments(R):
    """Solve sum_j c_j j^(2p) = [p == 1] (p = 1..R) exactly (Gauss-Jordan on
    Fractions); c_0 from the zero row sum.  Independent of the closed form."""
    A = [[Fraction(j) ** (2 * p) for j in range(1, R + 1)] + [Fraction(int(p == 1))]
         for p in range(1, R + 1)]
    n = R
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        pv = A[col][col]
        A[col] = [x / pv for x in A[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
    c = [A[r][n] for r in range(n)]
    return [-2 * sum(c)] + c


@pytest.mark.parametrize("R", range(1, 9))
def test_fd_weights_match_moment_conditions(R):
    exact = _weights_from_moments(R)
    got = oracle.fd_coefficients(R)
    for e, g in zip(exact, got):
        assert abs(g - float(e)) <= 1e-15 * max(1.0, abs(float(e)))


def test_fd_weights_textbook_so8():
    # Fornberg (Math. Comp. 1988), second derivative, 8th order, centred.
    ref = [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5),
           Fraction(8, 315), Fraction(-1, 560)]
    got = oracle.fd_coefficients(4)
    np.testing.assert_allclose(got, [float(x) for x in ref], rtol=1e-15)


# --------------------------------------------------------------------------
# Worked example of the paper (Sec. II, Listing 1; Sec. III Listings 2-3)
# --------------------------------------------------------------------------

def _read_golden_heat():
    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, "heat_4x4_listings_2_3.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                blocks[cur] = np.zeros((4, 4))
                continue
            parts = line.split()
            r = int(parts[0][4:])
            vals = np.array([float(x) for x in parts[1:]]).reshape(2, 2)
            blocks[cur][2 * (r // 2):2 * (r // 2) + 2, 2 * (r % 2):2 * (r % 2) + 2] = vals
    return blocks


def test_heat_worked_example_matches_paper():
    gold = _read_golden_heat()
    nx = ny = 4
    dx = 2.0 / (nx - 1)
    dt = 0.25 * dx * dx / 0.5
    g = oracle.Grid(n=(nx, ny), h=dx, dt=dt, R=1, dims=2)
    u = np.zeros(g.padded_shape)
    u[0, 1:-1, 1:-1] = 1.0
    np.testing.assert_array_equal(u[0], gold["before"])
    # time_M = 1 runs time = 0 and time = 1: two forward-Euler steps
    u = oracle.heat_step(g, oracle.heat_step(g, u))
    np.testing.assert_allclose(u[0], gold["after"], atol=1e-14)


def test_heat_worked_example_one_step_differs():
    # guards the reading "time_M=1 means two steps": one step does not match
    gold = _read_golden_heat()
    g = oracle.Grid(n=(4, 4), h=2 / 3, dt=2 / 9, R=1, dims=2)
    u = np.zeros(g.padded_shape)
    u[0, 1:-1, 1:-1] = 1.0
    assert not np.allclose(oracle.heat_step(g, u)[0], gold["after"])


# --------------------------------------------------------------------------
# Time stepping: exact discrete solutions
# --------------------------------------------------------------------------

def test_dalembert_courant_one_is_exact():
    """1D, SO 2, v dt = h: the leapfrog reproduces u(x, t) = f(x - v t)."""
    n, h, v = 200, 10.0, 1.5
    dt = h / v
    g = oracle.Grid(n=(n,), h=h, dt=dt, R=1, dims=1)
    x = np.arange(n) * h
    f = lambda s: np.exp(-((s - 600.0) / 80.0) ** 2)
    u_prev = f(x + v * dt).reshape(g.padded_shape)
    u_cur = f(x).reshape(g.padded_shape)
    m = np.full((1, 1, n), 1.0 / v ** 2)
    nt = 60
    out = oracle.forward(g, m, nt, np.zeros((0, 3)), np.zeros((nt, 0)),
                         np.zeros((0, 3)), state=(u_prev, u_cur))
    np.testing.assert_allclose(out["u_cur"].ravel(), f(x - v * nt * dt),
                               atol=1e-12)


def test_discrete_impulse_response_courant_one():
    """1D, SO 2, Courant 1, source on a node: the exact discrete solution is
    u_i^n = h * sum_k q^k [d <= n-1-k and n-1-k-d even], d = |i - i_s|."""
    n, h, v = 101, 10.0, 2.0
    dt = h / v
    g = oracle.Grid(n=(n,), h=h, dt=dt, R=1, dims=1)
    nt = 40
    rng = np.random.default_rng(0)
    q = rng.standard_normal(nt)
    i_s = 50
    m = np.full((1, 1, n), 1.0 / v ** 2)
    rec_i = np.arange(30, 71)
    out = oracle.forward(g, m, nt, [[i_s * h, 0, 0]], q.reshape(nt, 1),
                         np.stack([rec_i * h, 0 * rec_i, 0 * rec_i], 1))
    expect = np.zeros((nt, len(rec_i)))
    for t in range(nt):
        for a, i in enumerate(rec_i):
            d = abs(i - i_s)
            for k in range(t):
                L = t - 1 - k
                if d <= L and (L - d) % 2 == 0:
                    expect[t, a] += h * q[k]
    np.testing.assert_allclose(out["rec"], expect, atol=1e-12)


def _discrete_omega(c, R, k, h, v, dt):
    s = 0.0
    for ka in k:
        s += -c[0] - 2.0 * sum(c[j] * math.cos(j * ka * h) for j in range(1, R + 1))
    rhs = (v * dt / h) ** 2 * s / 4.0
    return 2.0 / dt * math.asin(math.sqrt(rhs))


@pytest.mark.parametrize("R", [1, 2, 4, 6, 8])
def test_plane_wave_follows_discrete_dispersion(R):
    """Periodic 3D plane wave cos(k.x - w t) with w from
    (4/dt^2) sin^2(w dt/2) = (v^2/h^2) sum_a [-c0 - 2 sum_j c_j cos(j k_a h)]
    stays an exact discrete solution."""
    n, h, v = (16, 12, 10), 10.0, 2.0
    dt = 0.3 * h / v
    g = oracle.Grid(n=n, h=h, dt=dt, R=R, periodic=True)
    c = oracle.fd_coefficients(R)
    k = [2 * math.pi * 3 / (n[0] * h), 2 * math.pi * 2 / (n[1] * h),
         2 * math.pi * 1 / (n[2] * h)]
    w = _discrete_omega(c, R, k, h, v, dt)
    z, y, x = np.meshgrid(*(np.arange(s) * h for s in g.padded_shape), indexing="ij")
    phase = k[0] * x + k[1] * y + k[2] * z
    nt = 50
    m = np.full(g.phys_shape, 1.0 / v ** 2)
    out = oracle.forward(g, m, nt, np.zeros((0, 3)), np.zeros((nt, 0)), np.zeros((0, 3)),
                         state=(np.cos(phase + w * dt), np.cos(phase)))
    np.testing.assert_allclose(out["u_cur"], np.cos(phase - w * nt * dt), atol=1e-10)


def test_plane_wave_rejects_continuum_dispersion():
    """The continuum w = v|k| does not satisfy the scheme (guards the test)."""
    n, h, v, R = (16, 12, 10), 10.0, 2.0, 2
    dt = 0.3 * h / v
    g = oracle.Grid(n=n, h=h, dt=dt, R=R, periodic=True)
    k = [2 * math.pi * 3 / (n[0] * h), 0.0, 0.0]
    w = v * abs(k[0])
    z, y, x = np.meshgrid(*(np.arange(s) * h for s in g.padded_shape), indexing="ij")
    phase = k[0] * x
    m = np.full(g.phys_shape, 1.0 / v ** 2)
    out = oracle.forward(g, m, 50, np.zeros((0, 3)), np.zeros((50, 0)), np.zeros((0, 3)),
                         state=(np.cos(phase + w * dt), np.cos(phase)))
    assert np.abs(out["u_cur"] - np.cos(phase - w * 50 * dt)).max() > 1e-4


# --------------------------------------------------------------------------
# Energy balance and damping
# --------------------------------------------------------------------------

def _energy(g, m_pad, u_next, u_cur):
    Lu = oracle.laplacian(g, u_cur)
    return np.sum(m_pad * ((u_next - u_cur) / g.dt) ** 2) - np.sum(u_next * Lu)


@pytest.mark.parametrize("nbl", [0, 4])
def test_energy_balance_with_damping(nbl):
    """E^{n+1/2} - E^{n-1/2} = -sum m b (u^{n+1} - u^{n-1})^2 / dt^2 exactly
    (zero ghost, no source); with no layer the energy is conserved."""
    n, h, R = (10, 9, 8), 10.0, 4
    rng = np.random.default_rng(1)
    v = rng.uniform(1.5, 3.0, size=(n[2], n[1], n[0]))
    dt = 0.4 * h / v.max()
    g = oracle.Grid(n=n, h=h, dt=dt, R=R, nbl=nbl)
    m_pad = oracle.pad_model(g, 1.0 / v ** 2)
    b = oracle.damping(g, v.max())
    if nbl == 0:
        assert np.all(b == 0)
    u0 = rng.standard_normal(g.padded_shape)
    u1 = rng.standard_normal(g.padded_shape)
    u2, _ = oracle.step(g, m_pad, b, u0, u1)
    E_prev = _energy(g, m_pad, u2, u1)
    scale = abs(E_prev)
    for _ in range(10):
        u3, _ = oracle.step(g, m_pad, b, u1, u2)
        E = _energy(g, m_pad, u3, u2)
        loss = np.sum(m_pad * b * (u3 - u1) ** 2) / dt ** 2
        assert abs((E - E_prev) + loss) <= 1e-11 * scale
        if nbl:
            assert E <= E_prev + 1e-11 * scale
        u1, u2, E_prev = u2, u3, E


def test_uniform_damping_decay_rate():
    """With constant b the amplitude of every oscillating mode decays by
    sqrt((1-b)/(1+b)) per step (roots of (1+b) r^2 - (2 + a lam) r + (1-b))."""
    n, h, v, R = (32,), 10.0, 2.0, 2
    dt = 0.4 * h / v
    g = oracle.Grid(n=n, h=h, dt=dt, R=R, dims=1, periodic=True)
    bval = 0.05
    b = np.full(g.padded_shape, bval)
    m_pad = np.full(g.padded_shape, 1.0 / v ** 2)
    x = np.arange(n[0]) * h
    kx = 2 * math.pi * 2 / (n[0] * h)
    c = oracle.fd_coefficients(R)
    lam = (c[0] + 2 * sum(c[j] * math.cos(j * kx * h) for j in range(1, R + 1))) / h ** 2
    a = dt ** 2 * v ** 2
    roots = np.roots([1 + bval, -(2 + a * lam), 1 - bval])
    assert np.iscomplexobj(roots)
    mode = np.cos(kx * x).reshape(g.padded_shape)
    u0, u1 = mode.copy(), mode.copy()
    nt = 40
    for _ in range(nt):
        u0, u1 = u1, oracle.step(g, m_pad, b, u0, u1)[0]
    # exact two-term recurrence of the mode's amplitude
    A = np.zeros(nt + 2)
    A[0] = A[1] = 1.0
    for t in range(nt):
        A[t + 2] = ((2 + a * lam) * A[t + 1] - (1 - bval) * A[t]) / (1 + bval)
    np.testing.assert_allclose(u1.ravel(), A[nt + 1] * mode.ravel(), atol=1e-12)
    assert abs(abs(roots[0]) - math.sqrt((1 - bval) / (1 + bval))) < 1e-14


def test_damping_profile_properties():
    n, h, R, nbl = (6, 5, 4), 10.0, 2, 5
    g = oracle.Grid(n=n, h=h, dt=2.0, R=R, nbl=nbl)
    vmax = 3.0
    b = oracle.damping(g, vmax)
    Nz, Ny, Nx = g.padded_shape
    assert np.all(b[nbl:nbl + n[2], nbl:nbl + n[1], nbl:nbl + n[0]] == 0)
    assert np.all(b >= 0)
    # along x through the physical centre row the profile is quadratic in depth
    row = b[nbl + 1, nbl + 1, :nbl + 1][::-1]  # depth 0..nbl
    d = np.arange(nbl + 1) / nbl
    assert np.allclose(row, row[-1] * d ** 2)
    # the corner has three times the face value
    assert math.isclose(b[0, 0, 0], 3 * row[-1], rel_tol=1e-14)
    # layer strength scales with v_max and 1/(nbl h), and with dt
    b2 = oracle.damping(g, 2 * vmax)
    assert np.allclose(b2, 2 * b)


# --------------------------------------------------------------------------
# Sparse points (Sec. III "Sparse data")
# --------------------------------------------------------------------------

def test_point_weights_reproduce_linear_fields():
    g = oracle.Grid(n=(7, 6, 5), h=10.0, dt=1.0, R=2, nbl=3)
    Nz, Ny, Nx = g.padded_shape
    z, y, x = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    field = (0.3 + 1.7 * (x - 3) * 10 - 0.4 * (y - 3) * 10 + 2.2 * (z - 3) * 10).ravel()
    rng = np.random.default_rng(3)
    for _ in range(50):
        p = rng.uniform(0, 1, 3) * (np.array([6, 5, 4]) * 10.0)
        idx, w = oracle.point_weights(g, p)
        assert abs(w.sum() - 1.0) < 1e-14 and np.all(w > 0)
        val = np.dot(w, field[idx])
        assert abs(val - (0.3 + 1.7 * p[0] - 0.4 * p[1] + 2.2 * p[2])) < 1e-11


def test_point_weights_on_node_and_outside():
    g = oracle.Grid(n=(7, 6, 5), h=10.0, dt=1.0, R=2, nbl=3)
    idx, w = oracle.point_weights(g, [20.0, 50.0, 40.0])
    Nz, Ny, Nx = g.padded_shape
    assert len(w) == 1 and w[0] == 1.0
    assert idx[0] == (2 + 3) + Nx * ((5 + 3) + Ny * (4 + 3))
    assert oracle.point_weights(g, [60.000001, 0, 0]) is None
    assert oracle.point_weights(g, [-1e-9, 0, 0]) is None


# --------------------------------------------------------------------------
# Green's functions (continuum limits)
# --------------------------------------------------------------------------

def _ricker(t_ms, f_hz):
    f = f_hz / 1000.0
    a = (math.pi * f * (t_ms - 1.0 / f)) ** 2
    return (1 - 2 * a) * np.exp(-a)


def _green_3d(t, r, v, f):
    return _ricker(t - r / v, f) / (4 * math.pi * r)


def _green_2d(t, r, v, f, nquad=4000):
    # u = 1/(2 pi) * int_0^{t - r/v} q(tau) / sqrt((t - tau)^2 - r^2/v^2) dtau,
    # with t - tau = (r/v) cosh(theta) removing the end-point singularity
    out = np.zeros_like(t)
    a = r / v
    for i, ti in enumerate(t):
        if ti <= a:
            continue
        th_max = math.acosh(ti / a)
        th = np.linspace(0.0, th_max, nquad)
        vals = _ricker(ti - a * np.cosh(th), f)
        out[i] = np.trapezoid(vals, th) / (2 * math.pi)
    return out


def _green_1d(t, r, v, f):
    # (v/2) * integral_0^{t - r/v} q, by fine quadrature
    out = np.zeros_like(t)
    for i, ti in enumerate(t):
        T = ti - r / v
        if T <= 0:
            continue
        s = np.linspace(0.0, T, 4000)
        out[i] = v / 2 * np.trapezoid(_ricker(s, f), s)
    return out


def _run_point_source(dims, ncell, h, R, f, r_cells, tmax, nbl):
    v = 1.5
    dt = 0.4 * h / v
    nt = int(round(tmax / dt))
    n = (ncell,) * dims
    g = oracle.Grid(n=n, h=h, dt=dt, R=R, nbl=nbl, dims=dims)
    c = (ncell // 2) * h
    src = [[c if a < dims else 0.0 for a in range(3)]]
    rec = [[c + r_cells * 10.0 if a == 0 else (c if a < dims else 0.0)
            for a in range(3)]]
    q = _ricker(np.arange(nt) * dt, f).reshape(nt, 1)
    m = np.full(g.phys_shape, 1.0 / v ** 2)
    out = oracle.forward(g, m, nt, src, q, rec)
    t = np.arange(nt) * dt
    return t, out["rec"][:, 0], v, r_cells * 10.0


@pytest.mark.parametrize("dims,green,tol", [(1, _green_1d, 0.01), (2, _green_2d, 0.03),
                                            (3, _green_3d, 0.03)])
def test_point_source_matches_greens_function(dims, green, tol):
    """Discrete delta = weights / h^dims: the receiver trace approaches the
    continuum Green's function; error falls when h and dt are halved."""
    f, tmax = 8.0, 330.0
    errs = []
    for h, ncell, nbl in [(10.0, 48, 16), (5.0, 96, 32)] if dims < 3 else [(10.0, 48, 16)]:
        t, trace, v, r = _run_point_source(dims, ncell, h, 8, f, 12, tmax, nbl)
        ref = green(t, r, v, f)
        errs.append(np.linalg.norm(trace - ref) / np.linalg.norm(ref))
    assert errs[0] < tol, errs
    if len(errs) > 1:
        assert errs[1] < 0.6 * errs[0], errs


# --------------------------------------------------------------------------
# Adjoint gradient: brute-force central differences
# --------------------------------------------------------------------------

def _small_inversion_problem():
    n, h, R, nbl = (8, 7, 6), 10.0, 2, 3
    rng = np.random.default_rng(7)
    v = rng.uniform(1.8, 2.4, size=(n[2], n[1], n[0]))
    dt = 0.4 * h / 2.4
    nt = 30
    g = oracle.Grid(n=n, h=h, dt=dt, R=R, nbl=nbl)
    src = [[33.0, 31.0, 24.0], [12.5, 44.0, 11.0]]
    q = np.stack([wl.ricker(nt, dt, 40.0).astype(np.float64),
                  0.5 * wl.ricker(nt, dt, 30.0).astype(np.float64)], 1)
    rec = [[x, 20.0, 45.0] for x in (0.0, 17.0, 35.5, 70.0)] + [[40.0, 60.0, 0.0]]
    m = 1.0 / v ** 2
    return g, m, nt, src, q, rec


def test_adjoint_gradient_matches_central_differences():
    g, m, nt, src, q, rec = _small_inversion_problem()
    d_obs = oracle.forward(g, m * 1.02, nt, src, q, rec)["rec"]
    grad, loss, _ = oracle.adjoint_gradient(g, m, nt, src, q, rec, d_obs=d_obs)

    def J(mm):
        r = oracle.forward(g, mm, nt, src, q, rec)["rec"] - d_obs
        return 0.5 * np.sum(r * r)

    assert abs(J(m) - loss) <= 1e-14 * abs(loss)
    eps = 1e-6 * m.mean()
    fd = np.zeros_like(m)
    for i in np.ndindex(m.shape):
        mp, mm = m.copy(), m.copy()
        mp[i] += eps
        mm[i] -= eps
        fd[i] = (J(mp) - J(mm)) / (2 * eps)
    # the cell holding v_max also sets the layer strength gamma_max, which the
    # gradient holds fixed by construction: leave that one cell out
    keep = np.ones(m.shape, bool)
    keep[np.unravel_index(np.argmin(m), m.shape)] = False
    assert np.linalg.norm((grad - fd)[keep]) <= 1e-6 * np.linalg.norm(fd[keep])


def test_adjoint_is_transpose_of_linearised_modelling():
    """<J dm, r> = <dm, J^T r> for an arbitrary residual r (dot-product test
    of the Jacobian against its transpose), J dm by central differences."""
    g, m, nt, src, q, rec = _small_inversion_problem()
    rng = np.random.default_rng(11)
    r = rng.standard_normal((nt, len(rec)))
    dm = rng.standard_normal(m.shape) * m.mean()
    dm[np.unravel_index(np.argmin(m), m.shape)] = 0.0  # keeps gamma_max fixed
    grad, _, _ = oracle.adjoint_gradient(g, m, nt, src, q, rec, residual=r)
    eps = 1e-6
    jp = oracle.forward(g, m + eps * dm, nt, src, q, rec)["rec"]
    jm = oracle.forward(g, m - eps * dm, nt, src, q, rec)["rec"]
    lhs = np.sum((jp - jm) / (2 * eps) * r)
    rhs = np.sum(dm * grad)
    assert abs(lhs - rhs) <= 1e-7 * abs(lhs)


# --------------------------------------------------------------------------
# Sampled single step (the checker of the full-size GPU tests) against the
# full-grid step
# --------------------------------------------------------------------------

@pytest.mark.parametrize("R,n,nbl", [(4, (13, 11, 9), 6), (1, (5, 7, 6), 3), (8, (18, 17, 19), 5),
                                     (2, (9, 8, 7), 0)])
def test_step_points_equals_full_step_everywhere(R, n, nbl):
    """or_step_points restates the damped leapfrog update (layer depth, model
    lookup by edge replication, zero ghost) for listed cells only.  Evaluated
    at EVERY padded cell of a small grid with a layer, from a random state on
    a model that varies along all three axes, it must equal or_step (pinned
    above by the worked example, d'Alembert, dispersion, energy and Green's
    functions) to rounding: the two differ only in where h^-2 is applied."""
    h, dt = 10.0, 1.1
    g = oracle.Grid(n=n, h=h, dt=dt, R=R, nbl=nbl)
    shp = g.padded_shape
    nz, ny, nx = g.phys_shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = 1.5 + 0.1 * zz + 0.07 * yy + 0.05 * xx + 0.3 * np.sin(xx * yy + zz)
    m = 1.0 / v ** 2
    vmax = float(v.max())
    up = wl.random_state(shp, 41 + R)
    uc = wl.random_state(shp, 42 + R)
    ref, _ = oracle.step(g, oracle.pad_model(g, m), oracle.damping(g, vmax), up, uc)
    idx = np.arange(int(np.prod(shp)), dtype=np.int64)
    got = oracle.step_points(g, m, vmax, up, uc, idx).reshape(shp)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-15 * scale * (2 * R + 2)
    # the layer is present and matters: the corner cells are damped
    if nbl:
        b = oracle.damping(g, vmax)
        assert b[0, 0, 0] > 0.05
        assert abs(got[0, 0, 0] - ref[0, 0, 0]) <= 1e-14 * scale
        assert abs(got[-1, -1, -1] - ref[-1, -1, -1]) <= 1e-14 * scale


def test_step_points_detects_a_wrong_layer_depth():
    """A planted off-by-one in the layer's far-side depth (as the restated
    formula could carry) moves the cells of the far faces well outside the
    rounding bound of the test above: the pin is sensitive to it."""
    R, n, nbl, h, dt = 4, (13, 11, 9), 6, 10.0, 1.1
    g = oracle.Grid(n=n, h=h, dt=dt, R=R, nbl=nbl)
    shp = g.padded_shape
    m = np.full(g.phys_shape, 1.0 / 2.0 ** 2)
    up = wl.random_state(shp, 5)
    uc = wl.random_state(shp, 6)
    ref, _ = oracle.step(g, oracle.pad_model(g, m), oracle.damping(g, 2.0), up, uc)
    # the same step with the far-side depth shifted by one cell: b of every
    # cell from the far face of the physical box outward takes the depth + 1
    b_bad = oracle.damping(g, 2.0)
    Nz, Ny, Nx = shp
    gmax = 3.0 * 2.0 * math.log(1e3) / (2 * nbl * h)
    for i in range(Nx):
        d_ok = max(nbl - i, i - (n[0] + nbl - 1), 0) / nbl
        d_bad = max(nbl - i, i - (n[0] + nbl - 2), 0) / nbl
        b_bad[:, :, i] += gmax * (d_bad ** 2 - d_ok ** 2) * dt / 2
    bad, _ = oracle.step(g, oracle.pad_model(g, m), b_bad, up, uc)
    idx = np.arange(int(np.prod(shp)), dtype=np.int64)
    got = oracle.step_points(g, m, 2.0, up, uc, idx).reshape(shp)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-15 * scale * 10
    assert np.abs(got - bad).max() > 1e-4 * scale
