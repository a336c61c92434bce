"""FP64 reference of the learned stencil-coefficient network.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy: each
dense layer is a matrix product, the backward pass is the chain rule written
out layer by layer.

The paper has no learned component; this follows the learned-discretisation
idea of Bar-Sinai et al. (PNAS 2019): a small network maps local, scale-free
inputs to finite-difference weights, trained so that a coarse-grid update
reproduces a fine-grid solution.

Network: x (4) -> 64 -> ReLU -> 64 -> ReLU -> 8 outputs o.
Inputs per cell: x = [v dt / h, h / 10 m, dt / 1 ms, f / 10 Hz].
Coefficients (space order 8, R = 4): s_j = (o_{j} + o_{j+4}) / 2 for
j = 1..4 (outputs o_1..o_8), c_j = cT_j (1 + tanh(s_j) / 2), c_0 = -2 sum c_j,
where cT are the Taylor weights; so an all-zero network gives Taylor SO 8.
Prediction for a sample with stencil sums T_j = S_j - 6 u (S_j the sum of the
six neighbours at distance j): p = sum_j c_j T_j.  Loss over n samples
(x, T, y, w): L = (1/n) sum w (p - y)^2.

Parameter vector (5000 floats): W1[64][4], b1[64], W2[64][64], b2[64],
W3[8][64], b3[8].
"""
from __future__ import annotations

import numpy as np

H = 64
NIN = 4
NOUT = 8
R = 4
SHAPES = [("W1", (H, NIN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
          ("W3", (NOUT, H)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)
SAMPLE = NIN + R + 2  # x[4], T[4], y, w


def unpack(theta):
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shp)
        k += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def init_params(seed: int, scale_out: float = 0.0):
    """He-style init for the hidden layers from a seeded generator; the last
    layer is scaled by ``scale_out`` (0 gives exactly the Taylor weights)."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.standard_normal((H, NIN)) * np.sqrt(2.0 / NIN),
         "b1": np.zeros(H),
         "W2": rng.standard_normal((H, H)) * np.sqrt(2.0 / H),
         "b2": np.zeros(H),
         "W3": rng.standard_normal((NOUT, H)) * np.sqrt(1.0 / H) * scale_out,
         "b3": np.zeros(NOUT)}
    return pack(p)


def forward(theta, X):
    """Outputs o [n, 8] and the cache for the backward pass."""
    p = unpack(theta)
    X = np.asarray(X, np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    o = h2 @ p["W3"].T + p["b3"]
    return o, (X, z1, h1, z2, h2, p)


def coefficients(theta, X, c_taylor):
    """Applied weights c_1..c_4 [n, 4] (c_0 = -2 sum follows)."""
    o, _ = forward(theta, X)
    s = 0.5 * (o[:, :R] + o[:, R:])
    return np.asarray(c_taylor[1:R + 1])[None, :] * (1.0 + 0.5 * np.tanh(s))


def loss(theta, samples, c_taylor):
    S = np.asarray(samples, np.float64)
    c = coefficients(theta, S[:, :NIN], c_taylor)
    pred = np.sum(c * S[:, NIN:NIN + R], axis=1)
    r = pred - S[:, NIN + R]
    return float(np.mean(S[:, NIN + R + 1] * r * r))


def loss_grad(theta, samples, c_taylor):
    """(L, dL/dtheta) by the chain rule through the coefficient map and the
    three dense layers."""
    S = np.asarray(samples, np.float64)
    n = S.shape[0]
    X, T, y, w = S[:, :NIN], S[:, NIN:NIN + R], S[:, NIN + R], S[:, NIN + R + 1]
    o, (X, z1, h1, z2, h2, p) = forward(theta, X)
    s = 0.5 * (o[:, :R] + o[:, R:])
    th = np.tanh(s)
    cT = np.asarray(c_taylor[1:R + 1])[None, :]
    c = cT * (1.0 + 0.5 * th)
    r = np.sum(c * T, axis=1) - y
    L = float(np.mean(w * r * r))
    dpred = 2.0 * w * r / n                          # dL/dp
    dc = dpred[:, None] * T                          # dL/dc_j
    ds = dc * cT * 0.5 * (1.0 - th * th)             # dL/ds_j
    do = np.concatenate([0.5 * ds, 0.5 * ds], axis=1)  # dL/do
    g = {"W3": do.T @ h2, "b3": do.sum(0)}
    dh2 = do @ p["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return L, pack(g)


def adam(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, ICLR 2015), t = 1 for the first step."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def features(v_kms, h, dt, f_hz):
    """Network inputs for velocities v (any shape) -> [..., 4]."""
    v = np.asarray(v_kms, np.float64)
    x = np.empty(v.shape + (NIN,))
    x[..., 0] = v * dt / h
    x[..., 1] = h / 10.0
    x[..., 2] = dt / 1.0
    x[..., 3] = f_hz / 10.0
    return x


def table_coefficients(theta, courant, h, dt, f_hz, nodes, lo, hi, c_taylor):
    """Weights c_1..c_4 [..., 4] of points with Courant numbers `courant`
    (v dt / h, any shape) when the network is evaluated only at `nodes`
    values of A = C^2 evenly spaced from lo^2 to hi^2 (the network sees
    C_i = sqrt(A_i)) and interpolated linearly in A in between, clamped to the
    end nodes: the definition of the table mode.  With hi == lo every point
    takes the first node."""
    A = np.asarray(courant, np.float64) ** 2
    alo, ahi = lo * lo, hi * hi
    Ai = alo + (ahi - alo) * np.arange(nodes, dtype=np.float64) / (nodes - 1)
    X = np.stack([np.sqrt(Ai), np.full(nodes, h / 10.0), np.full(nodes, dt / 1.0),
                  np.full(nodes, f_hz / 10.0)], axis=1)
    T = coefficients(theta, X, c_taylor)                      # [nodes, 4]
    if ahi > alo:
        x = np.clip((A - alo) * ((nodes - 1) / (ahi - alo)), 0.0, nodes - 1)
    else:
        x = np.zeros_like(A)
    i = np.minimum(np.floor(x).astype(np.int64), nodes - 2)
    f = (x - i)[..., None]
    return T[i] + f * (T[i + 1] - T[i])
