"""ctypes binding of libfd.so (C ABI in include/fd.h).

Argument marshalling only: every step of the finite-difference path runs in
the library's CUDA kernels.  Functions keep the C names (``fd_create_grid``,
``fd_set_model``, ``fd_forward``, ``fd_propagate``, ``fd_adjoint_gradient``,
``fd_backward``, ``fd_batch_forward`` ...); ``Grid`` is a small convenience
wrapper that owns a handle and checks status codes.

Array arguments may be numpy arrays (host) or torch tensors (host or CUDA);
they must be C-contiguous float32.  If libfd.so is missing this module raises
on import: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
        "g.build()'` (or python paper_2312_13094_gb300/build.py); the finite-difference "
        "path has no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

FD_OK, FD_ERR_ARG, FD_ERR_CUDA, FD_ERR_OOM, FD_ERR_UNSTABLE, FD_ERR_STATE, \
    FD_ERR_TIMEOUT, FD_ERR_NONFINITE = range(8)
FD_MODEL_VP_KMS, FD_MODEL_M = 0, 1
FD_REGION_PHYSICAL, FD_REGION_PADDED = 0, 1
FD_BATCH_GRAPH, FD_BATCH_AUTOTUNE = 1, 2
FD_DEBUG_SKIP_PLANE, FD_DEBUG_SPIN_LIMIT, FD_DEBUG_NO_GRAPH = 1, 2, 3
FD_COEF_TAYLOR, FD_COEF_UNIFORM, FD_COEF_PER_CELL = 0, 1, 2
FD_MLP_NPARAM, FD_MLP_SAMPLE = 5000, 10
FD_DMP_BASIC, FD_DMP_OVERLAP = 0, 1
FD_SCHED_AUTO, FD_SCHED_SHARES, FD_SCHED_WAVES, FD_SCHED_TEMPORAL = 0, 1, 2, 3


class fd_grid_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("h", ctypes.c_double), ("space_order", ctypes.c_int32),
                ("nbl", ctypes.c_int32), ("dt", ctypes.c_double), ("nt", ctypes.c_int32),
                ("device", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class fd_points(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("xyz", ctypes.c_void_p)]


class fd_grid_info(ctypes.Structure):
    _fields_ = [("nx_pad", ctypes.c_int32), ("ny_pad", ctypes.c_int32),
                ("nz_pad", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32),
                ("ctas", ctypes.c_int32), ("v_max", ctypes.c_double),
                ("cfl_limit", ctypes.c_double), ("launches", ctypes.c_int64),
                ("step_ms", ctypes.c_double), ("steps_timed", ctypes.c_int64),
                ("schedule", ctypes.c_int32)]


class fd_shot(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_void_p), ("src", ctypes.POINTER(fd_points)),
                ("wavelet", ctypes.c_void_p), ("rec", ctypes.POINTER(fd_points)),
                ("rec_out", ctypes.c_void_p)]


_G = ctypes.c_void_p
_P = ctypes.c_void_p
_PTS = ctypes.POINTER(fd_points)
_S = ctypes.c_int

_SIGS = {
    "fd_create_grid": (_S, [ctypes.POINTER(fd_grid_desc), ctypes.POINTER(ctypes.c_void_p)]),
    "fd_destroy_grid": (_S, [_G]),
    "fd_set_model": (_S, [_G, _P, ctypes.c_int32]),
    "fd_forward": (_S, [_G, _PTS, _P, _PTS, _P, _P]),
    "fd_propagate": (_S, [_G, ctypes.c_int32, ctypes.c_int32, _PTS, _P, _PTS, _P]),
    "fd_set_wavefield": (_S, [_G, _P, _P, ctypes.c_int32]),
    "fd_get_wavefield": (_S, [_G, _P, _P, ctypes.c_int32]),
    "fd_adjoint_gradient": (_S, [_G, _PTS, _P, _PTS, _P, ctypes.c_int32, _P,
                                 ctypes.POINTER(ctypes.c_double)]),
    "fd_backward": (_S, [_G, _PTS, _P, _PTS, _P, ctypes.c_int32, _P]),
    "fd_batch_forward": (_S, [ctypes.c_int32, ctypes.POINTER(fd_shot), ctypes.c_int32]),
    "fd_set_coefficients": (_S, [_G, _P, ctypes.c_int32]),
    "fd_set_learned_coefficients": (_S, [_G, _G, ctypes.c_double]),
    "fd_set_learned_table": (_S, [_G, _G, ctypes.c_double, ctypes.c_int32]),
    "fd_mlp_create": (_S, [ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_void_p)]),
    "fd_mlp_destroy": (_S, [_G]),
    "fd_mlp_get_params": (_S, [_G, _P]),
    "fd_mlp_set_params": (_S, [_G, _P]),
    "fd_mlp_loss_grad": (_S, [_G, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "fd_mlp_adam_step": (_S, [_G, ctypes.c_float]),
    "fd_mlp_train": (_S, [_G, ctypes.c_int64, _P, ctypes.c_int32, ctypes.c_int32,
                          ctypes.c_float, ctypes.POINTER(ctypes.c_double)]),
    "fd_mlp_coefficients": (_S, [_G, ctypes.c_int64, _P, _P]),
    "fd_sample_stencil": (_S, [_G, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "fd_mlp_make_samples": (_S, [ctypes.c_int32, _P, _P, _P, _P, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, _P]),
    "fd_forward_noalloc": (_S, [ctypes.POINTER(fd_grid_desc), _P, ctypes.c_int32, _PTS, _P,
                                _PTS, _P]),
    "fd_tti_create": (_S, [ctypes.POINTER(fd_grid_desc), ctypes.POINTER(ctypes.c_void_p)]),
    "fd_tti_destroy": (_S, [_G]),
    "fd_tti_set_model": (_S, [_G, _P, _P, _P, _P, _P]),
    "fd_tti_forward": (_S, [_G, _PTS, _P, _PTS, _P]),
    "fd_tti_propagate": (_S, [_G, ctypes.c_int32, ctypes.c_int32, _PTS, _P, _PTS, _P]),
    "fd_tti_set_state": (_S, [_G, _P, _P, _P, _P]),
    "fd_tti_get_state": (_S, [_G, _P, _P, _P, _P]),
    "fd_tti_set_profiling": (_S, [_G, ctypes.c_int32]),
    "fd_tti_get_info": (_S, [_G, ctypes.POINTER(fd_grid_info)]),
    "fd_set_tile": (_S, [_G, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "fd_set_decomposition": (_S, [_G, ctypes.c_int32, ctypes.c_int32]),
    "fd_set_schedule": (_S, [_G, ctypes.c_int32]),
    "fd_set_topology": (_S, [_G, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "fd_descent_step": (_S, [ctypes.c_int64, _P, _P, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, _P, ctypes.POINTER(ctypes.c_double)]),
    "fd_set_debug": (_S, [_G, ctypes.c_int32, ctypes.c_int64]),
    "fd_get_info": (_S, [_G, ctypes.POINTER(fd_grid_info)]),
    "fd_set_profiling": (_S, [_G, ctypes.c_int32]),
    "fd_launch_count": (ctypes.c_int64, []),
    "fd_alloc_count": (ctypes.c_int64, []),
    "fd_status_string": (ctypes.c_char_p, [_S]),
    "fd_last_error": (ctypes.c_char_p, []),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = tuple(_SIGS)


class FDError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.fd_last_error().decode()
        super().__init__(f"{where}: {_lib.fd_status_string(status).decode()} "
                         f"(status {status}){': ' + msg if msg else ''}")


def check(status, where="libfd"):
    if status != FD_OK:
        raise FDError(status, where)
    return status


def _ptr(a):
    """Raw pointer of a C-contiguous float32 numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays passed to libfd must be C-contiguous float32")
        return a.ctypes.data
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise TypeError("tensors passed to libfd must be contiguous float32")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)!r}")


class Points:
    """Host coordinate table [n, 3] in metres (kept alive with the struct)."""

    def __init__(self, xyz):
        xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32).reshape(-1, 3))
        self.xyz = xyz
        self.c = fd_points(xyz.shape[0], xyz.ctypes.data if xyz.size else None)

    @property
    def n(self):
        return self.xyz.shape[0]

    def ref(self):
        return ctypes.byref(self.c)


class Grid:
    """Owns one fd_grid handle."""

    def __init__(self, n, h, space_order, nbl, dt, nt, device=0, stream=None):
        self.desc = fd_grid_desc(int(n[0]), int(n[1]), int(n[2]), float(h), int(space_order),
                                 int(nbl), float(dt), int(nt), int(device),
                                 ctypes.c_void_p(stream) if stream else None)
        self.n = tuple(int(x) for x in n)
        self.nt = int(nt)
        handle = ctypes.c_void_p()
        check(fd_create_grid(ctypes.byref(self.desc), ctypes.byref(handle)), "fd_create_grid")
        self.handle = handle

    @classmethod
    def from_workload(cls, w, device=0, stream=None, nt=None):
        return cls(w["n"], w["h"], w["space_order"], w["nbl"], w["dt"],
                   w["nt"] if nt is None else nt, device, stream)

    def close(self):
        if getattr(self, "handle", None):
            fd_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def phys_shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def info(self):
        i = fd_grid_info()
        check(fd_get_info(self.handle, ctypes.byref(i)), "fd_get_info")
        return {k: getattr(i, k) for k, _ in fd_grid_info._fields_}

    @property
    def padded_shape(self):
        i = self.info()
        return (i["nz_pad"], i["ny_pad"], i["nx_pad"])

    def set_model(self, data, kind=FD_MODEL_VP_KMS):
        check(fd_set_model(self.handle, _ptr(data), kind), "fd_set_model")

    def set_tile(self, tile_x, tile_y, ctas=0):
        check(fd_set_tile(self.handle, tile_x, tile_y, ctas), "fd_set_tile")

    def set_schedule(self, mode):
        check(fd_set_schedule(self.handle, mode), "fd_set_schedule")

    def set_decomposition(self, nsub, mode=FD_DMP_BASIC):
        check(fd_set_decomposition(self.handle, nsub, mode), "fd_set_decomposition")

    def set_topology(self, px, py, pz):
        check(fd_set_topology(self.handle, px, py, pz), "fd_set_topology")

    def set_debug(self, key, value):
        check(fd_set_debug(self.handle, key, value), "fd_set_debug")

    def set_profiling(self, on=True):
        check(fd_set_profiling(self.handle, int(on)), "fd_set_profiling")

    def forward(self, src, wavelet, rec, rec_out, u_out=None):
        s, r = Points(src), Points(rec)
        return fd_forward(self.handle, s.ref(), _ptr(wavelet), r.ref(), _ptr(rec_out),
                          _ptr(u_out))

    def propagate(self, n0, nsteps, src=None, wavelet=None, rec=None, rec_out=None):
        s = Points(src) if src is not None else None
        r = Points(rec) if rec is not None else None
        return fd_propagate(self.handle, n0, nsteps, s.ref() if s else None, _ptr(wavelet),
                            r.ref() if r else None, _ptr(rec_out))

    def set_wavefield(self, u_prev, u_cur, region=FD_REGION_PADDED):
        check(fd_set_wavefield(self.handle, _ptr(u_prev), _ptr(u_cur), region),
              "fd_set_wavefield")

    def get_wavefield(self, u_prev, u_cur, region=FD_REGION_PADDED):
        check(fd_get_wavefield(self.handle, _ptr(u_prev), _ptr(u_cur), region),
              "fd_get_wavefield")

    def adjoint_gradient(self, src, wavelet, rec, d_obs, n_checkpoints, grad_out):
        s, r = Points(src), Points(rec)
        loss = ctypes.c_double(0.0)
        st = fd_adjoint_gradient(self.handle, s.ref(), _ptr(wavelet), r.ref(), _ptr(d_obs),
                                 n_checkpoints, _ptr(grad_out), ctypes.byref(loss))
        return st, loss.value

    def backward(self, src, wavelet, rec, grad_rec, n_checkpoints, grad_out):
        s, r = Points(src), Points(rec)
        return fd_backward(self.handle, s.ref(), _ptr(wavelet), r.ref(), _ptr(grad_rec),
                           n_checkpoints, _ptr(grad_out))


class TtiGrid:
    """Owns one fd_tti handle (anisotropic acoustic propagation)."""

    def __init__(self, n, h, space_order, nbl, dt, nt, device=0, stream=None):
        self.desc = fd_grid_desc(int(n[0]), int(n[1]), int(n[2]), float(h), int(space_order),
                                 int(nbl), float(dt), int(nt), int(device),
                                 ctypes.c_void_p(stream) if stream else None)
        self.n = tuple(int(x) for x in n)
        self.nt = int(nt)
        handle = ctypes.c_void_p()
        check(fd_tti_create(ctypes.byref(self.desc), ctypes.byref(handle)), "fd_tti_create")
        self.handle = handle

    @classmethod
    def from_workload(cls, w, device=0, stream=None, nt=None):
        return cls(w["n"], w["h"], w["space_order"], w["nbl"], w["dt"],
                   w["nt"] if nt is None else nt, device, stream)

    def close(self):
        if getattr(self, "handle", None):
            fd_tti_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def phys_shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def info(self):
        i = fd_grid_info()
        check(fd_tti_get_info(self.handle, ctypes.byref(i)), "fd_tti_get_info")
        return {k: getattr(i, k) for k, _ in fd_grid_info._fields_}

    @property
    def padded_shape(self):
        i = self.info()
        return (i["nz_pad"], i["ny_pad"], i["nx_pad"])

    def set_model(self, vp, epsilon, delta, theta, phi):
        check(fd_tti_set_model(self.handle, _ptr(vp), _ptr(epsilon), _ptr(delta), _ptr(theta),
                               _ptr(phi)), "fd_tti_set_model")

    def set_profiling(self, on=True):
        check(fd_tti_set_profiling(self.handle, int(on)), "fd_tti_set_profiling")

    def forward(self, src, wavelet, rec, rec_out):
        s, r = Points(src), Points(rec)
        return fd_tti_forward(self.handle, s.ref(), _ptr(wavelet), r.ref(), _ptr(rec_out))

    def propagate(self, n0, nsteps, src=None, wavelet=None, rec=None, rec_out=None):
        s = Points(src) if src is not None else None
        r = Points(rec) if rec is not None else None
        return fd_tti_propagate(self.handle, n0, nsteps, s.ref() if s else None, _ptr(wavelet),
                                r.ref() if r else None, _ptr(rec_out))

    def set_state(self, p_prev=None, p=None, q_prev=None, q=None):
        check(fd_tti_set_state(self.handle, _ptr(p_prev), _ptr(p), _ptr(q_prev), _ptr(q)),
              "fd_tti_set_state")

    def get_state(self, p_prev=None, p=None, q_prev=None, q=None):
        check(fd_tti_get_state(self.handle, _ptr(p_prev), _ptr(p), _ptr(q_prev), _ptr(q)),
              "fd_tti_get_state")


def descent_step(m, grad, step, m_min, m_max, stream=None):
    """fd_descent_step on two device tensors of equal size (m in place);
    returns alpha."""
    if m.numel() != grad.numel():
        raise ValueError("m and grad differ in size")
    alpha = ctypes.c_double(0.0)
    check(fd_descent_step(m.numel(), _ptr(m), _ptr(grad), float(step), float(m_min),
                          float(m_max), stream, ctypes.byref(alpha)), "fd_descent_step")
    return alpha.value


def batch_forward(shots, flags=FD_BATCH_GRAPH):
    """shots: list of (Grid, src_xyz, wavelet, rec_xyz, rec_out)."""
    keep = []
    arr = (fd_shot * len(shots))()
    for i, (g, src, wav, rec, out) in enumerate(shots):
        s, r = Points(src), Points(rec)
        keep += [s, r]
        arr[i] = fd_shot(g.handle.value, ctypes.pointer(s.c), _ptr(wav), ctypes.pointer(r.c),
                         _ptr(out))
    return fd_batch_forward(len(shots), arr, flags)
