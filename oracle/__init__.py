"""FP64 CPU oracle for the finite-difference acoustic path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2312_13094_gb300``) and never imports it; the two
meet only through the seeded input generators.

Every function is a thin ctypes wrapper over ``fd_oracle.c`` (plain C, FP64),
whose header lists the paper passages it follows and the readings taken where
the paper is silent.  ``mlp.py`` holds the FP64 reference of the learned
coefficient network, ``fwi.py`` that of the inversion loop's model update.

Pinned: coefficients (moment conditions), the heat worked example (Sec. II,
Listings 1-3), d'Alembert at Courant 1, plane-wave dispersion, energy balance
with damping, Green's functions, multilinear weights, the adjoint gradient
(brute-force central differences), the MLP backward pass (central
differences) and the sampled step ``step_points`` (equal to the full-grid
step at every cell of a grid with a layer).  The absorbing-layer profile strength (gamma_max) is a reading,
checked only by its properties: parity unpinned for that constant.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_fd_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``fd_oracle.c`` with gcc (FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32), ("n", ctypes.c_int32 * 3),
                ("nbl", ctypes.c_int32), ("R", ctypes.c_int32),
                ("periodic", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("h", ctypes.c_double), ("dt", ctypes.c_double),
                ("rc", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        G = ctypes.POINTER(_Grid)
        lib.or_ncell.argtypes = [G]
        lib.or_ncell.restype = ctypes.c_int64
        lib.or_fd_coefficients.argtypes = [ctypes.c_int32, _D]
        lib.or_pad_model.argtypes = [G, _D, _D]
        lib.or_damping.argtypes = [G, ctypes.c_double, _D]
        lib.or_laplacian.argtypes = [G, _D, _D, _D, _D]
        lib.or_point_weights.argtypes = [G, _D, _I64, _D]
        lib.or_point_weights.restype = ctypes.c_int32
        lib.or_step.argtypes = [G, _D, _D, _D, _D, _D, _D, ctypes.c_int32,
                                _I64, _D, _D, _D, _D]
        lib.or_heat_step.argtypes = [G, _D, _D, _D]
        lib.or_forward.argtypes = [G, _D, _D, _D, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_int32, _D, _D,
                                   ctypes.c_int32, _D, _D, _D, _D, _D]
        lib.or_forward.restype = ctypes.c_int32
        lib.or_adjoint_gradient.argtypes = [G, _D, ctypes.c_int32,
                                            ctypes.c_int32, _D, _D,
                                            ctypes.c_int32, _D, _D, _D, _D,
                                            _D, _D]
        lib.or_adjoint_gradient.restype = ctypes.c_int32
        lib.or_step_slab.argtypes = [G, _D, _D, _D, _D, _D, ctypes.c_int64, _D]
        lib.or_step_slab.restype = ctypes.c_int32
        lib.or_step_block.argtypes = [G, _D, _D, _D, _D, _D, _I64, _D]
        lib.or_step_block.restype = ctypes.c_int32
        lib.or_step_points.argtypes = [G, _D, ctypes.c_double, _D, _D, _D,
                                       ctypes.c_int64, _I64, _D]
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Grid:
    """Oracle grid: ``n`` physical cells (x, y, z), ``nbl`` layer cells per
    active face, half width ``R`` (space order 2R), spacing ``h`` [m], step
    ``dt`` [ms]."""
    n: tuple
    h: float
    dt: float
    R: int
    nbl: int = 0
    dims: int = 3
    periodic: bool = False
    rc: float = 1e-3

    def c(self) -> _Grid:
        n = list(self.n) + [1] * (3 - len(self.n))
        return _Grid(self.dims, (ctypes.c_int32 * 3)(*n), self.nbl, self.R,
                     int(self.periodic), 0, self.h, self.dt, self.rc)

    @property
    def padded_shape(self):
        """(Nz, Ny, Nx) of the padded arrays (x fastest)."""
        n = list(self.n) + [1] * (3 - len(self.n))
        N = [n[a] + 2 * self.nbl if a < self.dims else 1 for a in range(3)]
        return (N[2], N[1], N[0])

    @property
    def phys_shape(self):
        n = list(self.n) + [1] * (3 - len(self.n))
        return (n[2], n[1], n[0])


def fd_coefficients(R: int) -> np.ndarray:
    c = np.zeros(R + 1)
    _load().or_fd_coefficients(R, _p(c))
    return c


def pad_model(g: Grid, m_phys) -> np.ndarray:
    m_phys = _f64(m_phys)
    out = np.zeros(g.padded_shape)
    gc = g.c()
    _load().or_pad_model(ctypes.byref(gc), _p(m_phys), _p(out))
    return out


def damping(g: Grid, vmax: float) -> np.ndarray:
    out = np.zeros(g.padded_shape)
    gc = g.c()
    _load().or_damping(ctypes.byref(gc), vmax, _p(out))
    return out


def laplacian(g: Grid, u, coef=None, percell=None) -> np.ndarray:
    u = _f64(u)
    coef = fd_coefficients(g.R) if coef is None and percell is None else _f64(coef)
    out = np.zeros(g.padded_shape)
    gc = g.c()
    _load().or_laplacian(ctypes.byref(gc), _p(coef), _p(_f64(percell)), _p(u),
                         _p(out))
    return out


def point_weights(g: Grid, xyz):
    """Multilinear (padded flat index, weight) pairs of one point, or None."""
    xyz = _f64(np.asarray(xyz, dtype=np.float64).reshape(3))
    idx = np.zeros(8, dtype=np.int64)
    w = np.zeros(8)
    gc = g.c()
    n = _load().or_point_weights(ctypes.byref(gc), _p(xyz),
                                 idx.ctypes.data_as(_I64), _p(w))
    if n < 0:
        return None
    return idx[:n].copy(), w[:n].copy()


def step(g: Grid, m_pad, b, u_prev, u_cur, *, coef=None, percell=None,
         src_idx=None, src_val=None):
    """One damped leapfrog step on padded arrays with explicit ``m_pad`` and
    ``b``; ``src_idx``/``src_val`` add point terms (already / h^dims, times
    q) to L u.  Returns (u_next, e) with e = (dt^2/m)(L u + s)."""
    if coef is None and percell is None:
        coef = fd_coefficients(g.R)
    shp = g.padded_shape
    L = np.zeros(shp)
    out = np.zeros(shp)
    e = np.zeros(shp)
    si = np.zeros(1, np.int64) if src_idx is None else np.ascontiguousarray(src_idx, np.int64)
    sv = np.zeros(1) if src_val is None else _f64(src_val)
    ns = 0 if src_idx is None else len(si)
    gc = g.c()
    _load().or_step(ctypes.byref(gc), _p(_f64(m_pad)), _p(_f64(b)), _p(_f64(coef)),
                    _p(_f64(percell)), _p(_f64(u_prev)), _p(_f64(u_cur)), ns,
                    si.ctypes.data_as(_I64), _p(sv), _p(L), _p(out), _p(e))
    return out, e


def step_slab(g: Grid, m_pad_s, b_s, u_prev_s, u_cur_x, coef=None):
    """One source-free step of the owned z planes of a slab (domain
    decomposition along z): ``u_cur_x`` holds the owned planes with R ghost
    planes before and after; the other arrays cover the owned planes."""
    coef = fd_coefficients(g.R) if coef is None else _f64(coef)
    u_prev_s = _f64(u_prev_s)
    nzs = u_prev_s.shape[0]
    assert u_cur_x.shape[0] == nzs + 2 * g.R
    out = np.zeros(u_prev_s.shape)
    gc = g.c()
    r = _load().or_step_slab(ctypes.byref(gc), _p(_f64(m_pad_s)), _p(_f64(b_s)), _p(coef),
                             _p(u_prev_s), _p(_f64(u_cur_x)), nzs, _p(out))
    if r != 0:
        raise ValueError("slab steps need a 3-D, non-periodic grid")
    return out


def step_block(g: Grid, m_pad_b, b_b, u_prev_b, u_cur_x, coef=None):
    """One source-free step of the owned box of a block of a Cartesian
    decomposition: ``u_cur_x`` holds the box with R ghost layers on every
    side; the other arrays cover the box ([nz][ny][nx])."""
    coef = fd_coefficients(g.R) if coef is None else _f64(coef)
    u_prev_b = _f64(u_prev_b)
    nz, ny, nx = u_prev_b.shape
    R = g.R
    assert u_cur_x.shape == (nz + 2 * R, ny + 2 * R, nx + 2 * R)
    nb = np.array([nx, ny, nz], dtype=np.int64)
    out = np.zeros(u_prev_b.shape)
    gc = g.c()
    r = _load().or_step_block(ctypes.byref(gc), _p(_f64(m_pad_b)), _p(_f64(b_b)), _p(coef),
                              _p(u_prev_b), _p(_f64(u_cur_x)), nb.ctypes.data_as(_I64),
                              _p(out))
    if r != 0:
        raise ValueError("block steps need a 3-D, non-periodic grid")
    return out


def step_points(g: Grid, m_phys, vmax: float, u_prev, u_cur, idx, coef=None):
    """One source-free step evaluated only at padded flat indices ``idx``."""
    coef = fd_coefficients(g.R) if coef is None else _f64(coef)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(len(idx))
    gc = g.c()
    _load().or_step_points(ctypes.byref(gc), _p(_f64(m_phys)), float(vmax), _p(coef),
                           _p(_f64(u_prev)), _p(_f64(u_cur)), len(idx),
                           idx.ctypes.data_as(_I64), _p(out))
    return out


def heat_step(g: Grid, u) -> np.ndarray:
    u = _f64(u)
    scratch = np.zeros(g.padded_shape)
    out = np.zeros(g.padded_shape)
    gc = g.c()
    _load().or_heat_step(ctypes.byref(gc), _p(u), _p(scratch), _p(out))
    return out


def forward(g: Grid, m_phys, nt: int, src_xyz, wavelet, rec_xyz, *,
            coef=None, percell=None, state=None, n0: int = 0,
            want_e: bool = False, want_hist: bool = False):
    """Run ``nt`` damped leapfrog steps (Eq. 1 discretised).

    Returns a dict with ``rec`` [nt, nrec], ``u_prev``/``u_cur`` (padded final
    state) and optionally ``e`` [nt, ...] and ``u_hist`` [nt+1, ...].
    ``state`` = (u_prev, u_cur) padded arrays to start from (default: rest).
    ``wavelet`` is [n0+nt, nsrc] (row n0+t feeds step t).
    """
    m_phys = _f64(m_phys)
    src_xyz = _f64(np.asarray(src_xyz, dtype=np.float64).reshape(-1, 3))
    rec_xyz = _f64(np.asarray(rec_xyz, dtype=np.float64).reshape(-1, 3))
    nsrc, nrec = src_xyz.shape[0], rec_xyz.shape[0]
    wavelet = _f64(np.asarray(wavelet, dtype=np.float64).reshape(-1, max(nsrc, 1)))
    if coef is None and percell is None:
        coef = fd_coefficients(g.R)
    coef = _f64(coef)
    percell = _f64(percell)
    shp = g.padded_shape
    st = np.zeros((2,) + shp)
    if state is not None:
        st[0] = state[0]
        st[1] = state[1]
    rec = np.zeros((nt, nrec))
    ncell = int(np.prod(shp))
    e = np.zeros((nt,) + shp) if want_e else None
    hist = np.zeros((nt + 1,) + shp) if want_hist else None
    gc = g.c()
    rc = _load().or_forward(ctypes.byref(gc), _p(m_phys), _p(coef), _p(percell),
                            n0, nt, nsrc, _p(src_xyz), _p(wavelet), nrec,
                            _p(rec_xyz), _p(rec), _p(st), _p(e), _p(hist))
    if rc != 0:
        raise ValueError("source or receiver outside the physical box")
    del ncell
    return {"rec": rec, "u_prev": st[0], "u_cur": st[1], "e": e, "u_hist": hist}


def adjoint_gradient(g: Grid, m_phys, nt: int, src_xyz, wavelet, rec_xyz, *,
                     d_obs=None, residual=None):
    """Gradient of 1/2 ||rec - d_obs||^2 w.r.t. the physical squared slowness
    (or of <rec, residual> when ``residual`` is given).  Small grids only.
    Returns (grad [phys shape], loss, residual)."""
    m_phys = _f64(m_phys)
    src_xyz = _f64(np.asarray(src_xyz, dtype=np.float64).reshape(-1, 3))
    rec_xyz = _f64(np.asarray(rec_xyz, dtype=np.float64).reshape(-1, 3))
    nsrc, nrec = src_xyz.shape[0], rec_xyz.shape[0]
    wavelet = _f64(np.asarray(wavelet, dtype=np.float64).reshape(-1, max(nsrc, 1)))
    grad = np.zeros(g.phys_shape)
    loss = ctypes.c_double(0.0)
    r = np.zeros((nt, nrec))
    gc = g.c()
    rc = _load().or_adjoint_gradient(
        ctypes.byref(gc), _p(m_phys), nt, nsrc, _p(src_xyz), _p(wavelet),
        nrec, _p(rec_xyz), _p(_f64(d_obs)), _p(_f64(residual)), _p(grad),
        ctypes.byref(loss), _p(r))
    if rc != 0:
        raise ValueError("source or receiver outside the physical box")
    return grad, loss.value, r
