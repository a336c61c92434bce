"""FP64 reference of the full-waveform-inversion model update.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy.

The paper names full-waveform inversion as a user of the propagator (Sec. I
and IV-B) and gives no update rule.  The loop built on the adjoint gradient
takes normalised steepest-descent steps: with the summed shot gradient g of
the misfit J(m) = 1/2 sum_shots ||rec(m) - d_obs||^2,

    alpha = step * max|m| / max|g|,    m <- clip(m - alpha g, m_min, m_max),

so the largest change of a step is `step` times the model's scale; a zero
gradient leaves m unchanged.  A step whose misfit does not fall is retried
with half the step (backtracking).
"""
from __future__ import annotations

import numpy as np


def descent_step(m, g, step, m_min, m_max):
    """(new m, alpha) of one normalised steepest-descent step, in FP64."""
    m = np.asarray(m, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    gmax = float(np.abs(g).max()) if g.size else 0.0
    if gmax == 0.0 or step == 0.0:
        return m.copy(), 0.0
    alpha = step * float(np.abs(m).max()) / gmax
    return np.clip(m - alpha * g, m_min, m_max), alpha
