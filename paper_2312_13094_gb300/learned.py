"""Learned per-cell stencil weights: training data from fine-grid runs, GPU
training with the library's own kernels, and the coarse-vs-fine evaluation.

Every numerical step runs in libfd.so (fine and coarse propagation, stencil
sampling, sample assembly, network training and inference); this module only
schedules the calls and moves arrays.

Setting (coarse solve = every second fine node, twice the time step):
  fine    n^3 + nbl_f layer, h_f, space order 16, dt_f, nt_f steps
  coarse  (n/2)^3 + nbl_f/2, h_c = 2 h_f, space order 8 (plain or learned),
          dt_c = 2 dt_f, nt_c = nt_f / 2 steps; coarse rec[k] vs fine rec[2k].
Velocity models: 3-8 horizontal layers, v in [1.5, 4.5] km/s, interfaces
smoothed over 40 m, drawn with seeded splitmix64 streams.  The source and the
receivers sit on multiples of 4 h_f, which are grid nodes of every spacing
compared (h_f, 4/3 h_f, 2 h_f), so no configuration is scored on its point
interpolation.
"""
from __future__ import annotations

import time

import numpy as np

from . import binding as fd
from . import workloads as wl


def pair(seed: int, n: int = 512, h: float = 10.0, dt: float = 0.8, nt: int = 1250,
         nbl: int = 40, f_hz: float = 12.0, rec_every: int = 4):
    """Fine and coarse workloads on the same seeded layered model: the source
    near the centre in x/y at depth 8 h, receivers on a line along x every
    `rec_every` fine cells (a multiple of 4) through the source's y, at
    depth 4 h."""
    assert n % 2 == 0 and nt % 2 == 0 and nbl % 2 == 0 and rec_every % 4 == 0
    nf = (n, n, n)
    v = wl.layered_model(nf, h, seed)
    c = int(round(n / 2 / 4)) * 4
    src = np.array([[c * h, c * h, 8 * h]])
    xs = np.arange(0, n, rec_every) * h
    rec = np.stack([xs, np.full(len(xs), c * h), np.full(len(xs), 4 * h)], 1)
    wav_f = wl.ricker(nt, dt, f_hz).reshape(nt, 1)
    fine = dict(name=f"fine {n}^3 h{h:g} SO16", n=nf, h=h, space_order=16, nbl=nbl, dt=dt,
                nt=nt, v=v, src=src, rec=rec, wavelet=wav_f, f0=f_hz)
    vc = np.ascontiguousarray(v[::2, ::2, ::2])
    wav_c = wl.ricker(nt // 2, 2 * dt, f_hz).reshape(nt // 2, 1)
    coarse = dict(name=f"coarse {n // 2}^3 h{2 * h:g} SO8", n=(n // 2,) * 3, h=2 * h,
                  space_order=8, nbl=nbl // 2, dt=2 * dt, nt=nt // 2, v=vc, src=src,
                  rec=rec, wavelet=wav_c, f0=f_hz)
    return fine, coarse


# Plain configurations between the coarse and the fine grid, (h, space
# order, dt): dt is a multiple of the fine 0.8 ms so that receiver times
# coincide, and within each stencil's stability limit at v = 4.5 km/s.
LADDER = ((20.0, 8, 0.8), (40.0 / 3.0, 8, 0.8), (40.0 / 3.0, 16, 0.8), (10.0, 8, 0.8))


def plain_config(seed: int, h: float, space_order: int, dt: float, n: int = 512,
                 h_f: float = 10.0, dt_f: float = 0.8, nt_f: int = 1250, nbl_m: float = 400.0,
                 f_hz: float = 12.0):
    """The fine workload's medium, source and receivers on a plain grid of
    spacing h (the same physical box, sponge about nbl_m thick); its
    receivers sample the fine times k * dt."""
    fine, _ = pair(seed, n=n, h=h_f, dt=dt_f, nt=nt_f, f_hz=f_hz)
    ext = (n - 1) * h_f
    ns = int(np.ceil(ext / h - 1e-9)) + 1
    nd = (ns, ns, ns)
    v = wl.layered_model(nd, h, seed, depth_m=n * h_f)
    nt = int(round(nt_f * dt_f / dt))
    return dict(name=f"plain {ns}^3 h{h:.4g} SO{space_order}", n=nd, h=h,
                space_order=space_order, nbl=int(round(nbl_m / h)), dt=dt, nt=nt, v=v,
                src=fine["src"], rec=fine["rec"],
                wavelet=wl.ricker(nt, dt, f_hz).reshape(nt, 1), f0=f_hz,
                stride=int(round(dt / dt_f)))


def run_forward(w, device=0, net=None, space_order=None, timed=False, table=0):
    """Receivers of one forward run (and its device time in ms if timed).
    With a network: per-cell weight fields, or with table > 0 the network
    tabulated at that many Courant numbers (fd_set_learned_table)."""
    import torch
    so = w["space_order"] if space_order is None else space_order
    ww = dict(w, space_order=so)
    with fd.Grid.from_workload(ww, device=device) as g:
        g.set_model(w["v"])
        if net is not None and table:
            fd.check(fd.fd_set_learned_table(g.handle, net, float(w["f0"]), int(table)),
                     "fd_set_learned_table")
        elif net is not None:
            fd.check(fd.fd_set_learned_coefficients(g.handle, net, float(w["f0"])),
                     "fd_set_learned_coefficients")
        rec = torch.zeros((w["nt"], len(w["rec"])), device=f"cuda:{device}")
        wav = torch.from_numpy(np.ascontiguousarray(w["wavelet"])).to(f"cuda:{device}")
        ms = None
        if timed:
            fd.check(g.forward(w["src"], wav, w["rec"], rec), "warm-up")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        fd.check(g.forward(w["src"], wav, w["rec"], rec), "fd_forward")
        torch.cuda.synchronize()
        if timed:
            ms = (time.perf_counter() - t0) * 1e3
        return rec.cpu().numpy(), ms


def training_samples(fine, coarse, ncell: int = 16384, ntimes: int = 8, seed: int = 0,
                     min_src_dist: int = 5, device: int = 0):
    """Samples (device tensor [m, 10]) from one fine run: at `ntimes` coarse
    times in the second half of the run, `ncell` random coarse cells (at
    least `min_src_dist` coarse cells from the source), stencils taken at
    fine steps 2k-2, 2k, 2k+2 with stride 2."""
    import torch
    dev = f"cuda:{device}"
    nc = coarse["n"]
    nbl_f = fine["nbl"]
    rng = np.random.default_rng(seed)
    ntc = coarse["nt"]
    # coarse times at least two coarse steps apart, so that the fine-step
    # triples (2t-2, 2t, 2t+2) of different times never overlap
    cand = np.arange(ntc // 2, ntc - 1, 2)
    times = np.sort(rng.choice(cand, min(ntimes, len(cand)), replace=False))
    times = times[np.concatenate([[True], np.diff(times) >= 2])]
    src_c = np.round(np.asarray(coarse["src"][0]) / coarse["h"]).astype(int)
    vf = fine["v"]
    nf = vf.shape
    cells_c = []
    tries = 0
    while len(cells_c) < ncell and tries < 200:
        tries += 1
        c = rng.integers(0, nc[0], size=(ncell, 3))
        d = np.abs(c - src_c[None, :]).max(axis=1)
        c = c[d >= min_src_dist]
        # keep cells whose coarse stencil (radius 4) sees a homogeneous medium:
        # only there can a set of weights per cell reproduce the fine solution
        vc = vf[2 * c[:, 2], 2 * c[:, 1], 2 * c[:, 0]]
        ok = np.ones(len(c), bool)
        for a in range(3):
            for j in (-8, -4, 4, 8):
                p = 2 * c.copy()
                p[:, a] = np.clip(p[:, a] + j, 0, nf[2 - a] - 1)
                vn = vf[p[:, 2], p[:, 1], p[:, 0]]
                ok &= np.abs(vn - vc) <= 0.01 * vc
        cells_c.extend(c[ok].tolist())
    cells_c = np.array(cells_c[:ncell], dtype=np.int32).reshape(-1, 3)  # (x, y, z) coarse
    ncell = len(cells_c)
    if ncell == 0:
        raise ValueError("no homogeneous cells to sample")
    cells_f = np.ascontiguousarray(2 * cells_c + nbl_f, dtype=np.int32)  # padded fine
    vel = torch.from_numpy(np.ascontiguousarray(
        fine["v"][2 * cells_c[:, 2], 2 * cells_c[:, 1], 2 * cells_c[:, 0]],
        dtype=np.float32)).to(dev)
    width = 1 + 6 * 4
    out = []
    with fd.Grid.from_workload(fine, device=device) as g:
        g.set_model(fine["v"])
        wav = torch.from_numpy(np.ascontiguousarray(fine["wavelet"])).to(dev)
        step = 0
        for tk in times:
            snaps = []
            for fstep in (2 * tk - 2, 2 * tk, 2 * tk + 2):
                if fstep > step:
                    fd.check(g.propagate(step, fstep - step, fine["src"], wav), "fd_propagate")
                    step = fstep
                buf = torch.zeros((ncell, width), device=dev)
                fd.check(fd.fd_sample_stencil(g.handle, ncell, cells_f.ctypes.data, 2, 4,
                                              buf.data_ptr()), "fd_sample_stencil")
                snaps.append(buf)
            ms = float((snaps[1] ** 2).mean())
            s = torch.zeros((ncell, fd.FD_MLP_SAMPLE), device=dev)
            fd.check(fd.fd_mlp_make_samples(ncell, snaps[0].data_ptr(), snaps[1].data_ptr(),
                                            snaps[2].data_ptr(), vel.data_ptr(),
                                            coarse["h"], coarse["dt"], coarse["f0"],
                                            ms + 1e-30, s.data_ptr()),
                     "fd_mlp_make_samples")
            out.append(s)
    return torch.cat(out)


class Network:
    """Owns an fd_mlp handle."""

    def __init__(self, params=None, device=0):
        import ctypes
        h = ctypes.c_void_p()
        p = None if params is None else np.ascontiguousarray(params, np.float32)
        fd.check(fd.fd_mlp_create(device, None if p is None else p.ctypes.data,
                                  ctypes.byref(h)), "fd_mlp_create")
        self.handle = h

    def params(self):
        out = np.zeros(fd.FD_MLP_NPARAM, np.float32)
        fd.check(fd.fd_mlp_get_params(self.handle, out.ctypes.data), "fd_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        fd.check(fd.fd_mlp_set_params(self.handle, p.ctypes.data), "fd_mlp_set_params")

    def loss_grad(self, samples):
        import ctypes
        loss = ctypes.c_double()
        g = np.zeros(fd.FD_MLP_NPARAM, np.float32)
        fd.check(fd.fd_mlp_loss_grad(self.handle, samples.shape[0], fd._ptr(samples),
                                     ctypes.byref(loss), g.ctypes.data), "fd_mlp_loss_grad")
        return loss.value, g

    def train(self, samples, epochs, batch, lr):
        import ctypes
        loss = ctypes.c_double()
        fd.check(fd.fd_mlp_train(self.handle, samples.shape[0], fd._ptr(samples), epochs,
                                 batch, lr, ctypes.byref(loss)), "fd_mlp_train")
        return loss.value

    def coefficients(self, features):
        features = np.ascontiguousarray(features, np.float32)
        out = np.zeros((features.shape[0], 4), np.float32)
        fd.check(fd.fd_mlp_coefficients(self.handle, features.shape[0], features.ctypes.data,
                                        out.ctypes.data), "fd_mlp_coefficients")
        return out

    def close(self):
        if getattr(self, "handle", None):
            fd.fd_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def init_params(seed: int, scale_out: float = 0.1):
    """Seeded initial parameters (hidden layers He-scaled, output layer scaled
    by `scale_out`), drawn from splitmix64 normals."""
    H, NIN, NOUT = 64, 4, 8
    z = wl.normal(seed, H * NIN + H * H + NOUT * H)
    W1 = z[:H * NIN] * np.sqrt(2.0 / NIN)
    W2 = z[H * NIN:H * NIN + H * H] * np.sqrt(2.0 / H)
    W3 = z[H * NIN + H * H:] * np.sqrt(1.0 / H) * scale_out
    return np.concatenate([W1, np.zeros(H), W2, np.zeros(H), W3, np.zeros(NOUT)]).astype(
        np.float32)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


_FINE_CACHE = {}


def fine_receivers(seed, device=0, timed=True, **kw):
    """Receivers (and GPU time) of the fine SO 16 solve of one model (`kw` as
    for pair), kept for the process so that evaluations and the fine-tune
    share them."""
    key = (seed, tuple(sorted(kw.items())))
    if key not in _FINE_CACHE:
        fine, _ = pair(seed, **kw)
        _FINE_CACHE[key] = run_forward(fine, device, timed=timed)
    return _FINE_CACHE[key]


# the output-layer bias of the network: entries o_j and o_{j+4} of the 8
# outputs enter weight j only through their mean, so 4 directions matter
_B3 = 5000 - 8


def finetune_output_bias(net, seeds, device=0, iters=12, h0=0.05, table=256, **kw):
    """Rollout fine-tune of the network's output bias on the receiver misfit.

    The one-step training sets the weights from local fine-run samples; the
    quantity they are judged by is the receiver error of whole coarse runs.
    This stage moves the bias of output pair j (o_j, o_{j+4}) by beta_j to
    minimise the largest receiver relative L2, against the fine solve, over
    the training models `seeds`: each iteration estimates the gradient of
    that objective by central differences (step h) through coarse forward
    runs of the library and takes a backtracking step (`kw` as for pair).
    Returns the history of the objective and the bias shifts."""
    p0 = net.params().astype(np.float64)
    refs = {s: fine_receivers(s, device=device, **kw)[0][::2] for s in seeds}
    coarse = {s: pair(s, **kw)[1] for s in seeds}

    def objective(beta):
        p = p0.copy()
        for j in range(4):
            p[_B3 + j] += beta[j]
            p[_B3 + 4 + j] += beta[j]
        net.set_params(p.astype(np.float32))
        return max(rel_l2(run_forward(coarse[s], device, net=net.handle, table=table,
                                      timed=False)[0], refs[s]) for s in seeds)

    beta = np.zeros(4)
    f = objective(beta)
    hist = [f]
    h = h0
    for _ in range(iters):
        g = np.zeros(4)
        for j in range(4):
            e = np.zeros(4)
            e[j] = h
            g[j] = (objective(beta + e) - objective(beta - e)) / (2 * h)
        if not np.any(g):
            break
        step = 4 * h / np.abs(g).max()
        improved = False
        for _ in range(5):
            trial = beta - step * g
            ft = objective(trial)
            if ft < f:
                beta, f, improved = trial, ft, True
                break
            step *= 0.5
        hist.append(f)
        if not improved:
            h *= 0.5
    objective(beta)  # leave the network at the best bias
    return hist, beta


def evaluate(net, seeds, n=512, nt=1250, device=0, timed=True, ladder=False):
    """Per held-out model: receiver rel. L2 of coarse plain and coarse learned
    against the fine SO 16 solve (fine rec[2k]), and the GPU times; with
    ladder, also the plain configurations of LADDER."""
    rows = []
    for s in seeds:
        fine, coarse = pair(s, n=n, nt=nt)
        rf, tf = fine_receivers(s, device=device, timed=timed, n=n, nt=nt)
        ref = rf[::2]
        extra = {}
        if ladder:
            for (hh, so, dt) in LADDER:
                w = plain_config(s, hh, so, dt, n=n, nt_f=nt)
                r, t = run_forward(w, device, timed=timed)
                key = f"h{hh:.4g}_so{so}"
                extra[key] = rel_l2(r, rf[::w["stride"]][:len(r)])
                extra["ms_" + key] = t
        rp, tp = run_forward(coarse, device, timed=timed)
        r16, t16 = run_forward(coarse, device, space_order=16, timed=timed)
        rl, tlr = run_forward(coarse, device, net=net.handle, timed=timed)
        rt, ttb = run_forward(coarse, device, net=net.handle, timed=timed, table=256)
        rows.append(dict(seed=s, plain=rel_l2(rp, ref), plain16=rel_l2(r16, ref),
                         learned=rel_l2(rl, ref), learned_table=rel_l2(rt, ref), ms_fine=tf,
                         ms_plain=tp, ms_plain16=t16, ms_learned=tlr, ms_learned_table=ttb,
                         **extra))
    return rows
