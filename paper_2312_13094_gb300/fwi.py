"""Shot-parallel full-waveform inversion on top of the adjoint gradient.

The paper names full-waveform inversion (FWI) as a user of its propagators
(Sec. I and IV-B) without giving an algorithm.  The loop here lowers the
misfit J(m) = 1/2 sum_s ||rec_s(m) - d_s||^2 over the shots s with gradient
steps on the squared slowness m; the gradient is the sum of the per-shot
adjoint gradients (fd_adjoint_gradient).  Shots are independent, so each rank
evaluates a balanced share of them and one sum over ranks gives the total
(shard.shot_parallel_gradient); every rank then applies the same model update
to the same reduced gradient (fd_descent_step, a normalised steepest-descent
step run on the device), so the models stay identical without a broadcast.

A step whose misfit does not fall is retried with half the step, up to
`max_halvings` times; the loop stops early when no halving lowers the misfit.
Each accepted iteration costs one gradient evaluation of every shot (the
gradient at the new model comes with its misfit), each rejected step one more.
"""
from __future__ import annotations

from . import shard


def fwi_loop(m, nshots, grad_of_shot, update, iterations, step=0.05, max_halvings=3,
             dist=None):
    """Run `iterations` accepted steps from model `m` (not modified).

    grad_of_shot(s, m) -> (gradient tensor shaped like m, misfit of shot s)
    update(m, g, step) -> new model tensor (e.g. device_update below)
    Returns (m, history) with history["loss"] the misfit of every accepted
    model (the starting one first), history["step"] the step taken to reach
    each, and history["evals"] the number of gradient evaluations."""
    g, J = shard.shot_parallel_gradient(nshots, lambda s: grad_of_shot(s, m), m, dist)
    hist = {"loss": [J], "step": [], "evals": 1}
    for _ in range(iterations):
        st = step
        accepted = False
        for _ in range(max_halvings + 1):
            m_new = update(m, g, st)
            g_new, J_new = shard.shot_parallel_gradient(
                nshots, lambda s: grad_of_shot(s, m_new), m, dist)
            hist["evals"] += 1
            if J_new < J:
                accepted = True
                break
            st *= 0.5
        if not accepted:
            break
        m, g, J = m_new, g_new, J_new
        hist["loss"].append(J)
        hist["step"].append(st)
    return m, hist


class AdjointShots:
    """grad_of_shot backed by libfd: shot s fires source srcs[s] with the
    shared wavelet into one grid and is compared with d_obs[s] at the shared
    receivers.  m is the physical squared slowness (float32 device tensor)."""

    def __init__(self, grid, srcs, wavelet, rec, d_obs, n_checkpoints=25):
        self.grid, self.srcs, self.wavelet = grid, srcs, wavelet
        self.rec, self.d_obs, self.nc = rec, d_obs, n_checkpoints

    def __call__(self, s, m):
        import torch
        from . import binding as fd
        self.grid.set_model(m, fd.FD_MODEL_M)
        g = torch.zeros_like(m)
        st, loss = self.grid.adjoint_gradient(self.srcs[s], self.wavelet, self.rec,
                                              self.d_obs[s], self.nc, g)
        fd.check(st, "fd_adjoint_gradient")
        return g, loss


def device_update(m_min, m_max):
    """update() for fwi_loop: a copy of m advanced by fd_descent_step."""
    from . import binding as fd

    def update(m, g, step):
        m2 = m.clone()
        fd.descent_step(m2, g, step, m_min, m_max)
        return m2

    return update
