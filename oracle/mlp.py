"""FP64 oracle of the learned far-field correction (test infrastructure).

Not in the paper: a small MLP predicts the residual between the exact force
of an accepted tree cell (direct sum over its particles, Eq. 1) and its
multipole force (monopole + quadrupole, Sect. 4.2), so the opening angle can
be widened.  Plain numpy, float64, no blocking or fusion:

  features(p, cell)  -- 12 numbers: r_hat (3), w/R, log10 N_c,
                        (com - centre)/w (3), and with Qh = Q / (M w^2):
                        r_hat.Qh.r_hat, |Qh r_hat|, tr(Qh^2), det(Qh)
                        (r = p - com, R = |r|)
  label(p, cell)     -- (a_exact - a_multipole) / (G M / R^2)
  forward/backward   -- 12 -> 64 -> 64 -> 64 -> 3, GELU (tanh form) on the
                        hidden layers, linear output, mean squared error
  adam               -- Adam update (Kingma & Ba 2015)

Parameters are one flat float64 vector in the order W1 (12x64, row-major:
input x output), b1 (64), W2 (64x64), b2, W3 (64x64), b3, W4 (64x3), b4 (3):
9347 values, the same order librb uses for its BF16 weights.
"""
from __future__ import annotations

import math

import numpy as np

SIZES = [12, 64, 64, 64, 3]
N_FEATURES = 12


def n_params() -> int:
    return sum(a * b + b for a, b in zip(SIZES[:-1], SIZES[1:]))


def unpack(theta):
    """Flat vector -> [(W, b), ...] (views)."""
    out, k = [], 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        W = theta[k: k + a * b].reshape(a, b)
        k += a * b
        bb = theta[k: k + b]
        k += b
        out.append((W, bb))
    return out


def init(seed: int) -> np.ndarray:
    """He-style initialisation from a seeded generator."""
    g = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        parts.append(g.normal(0.0, math.sqrt(2.0 / a), a * b))
        parts.append(np.zeros(b))
    return np.concatenate(parts)


_C = math.sqrt(2.0 / math.pi)


def gelu(z):
    """GELU, tanh form: z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))."""
    return 0.5 * z * (1.0 + np.tanh(_C * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    u = _C * (z + 0.044715 * z ** 3)
    t = np.tanh(u)
    du = _C * (1.0 + 3.0 * 0.044715 * z ** 2)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * du


def forward(theta, X):
    """Returns (Y, cache) for inputs X (n x 12)."""
    layers = unpack(theta)
    acts, pre = [X], []
    h = X
    for li, (W, b) in enumerate(layers):
        z = h @ W + b
        pre.append(z)
        h = gelu(z) if li < len(layers) - 1 else z
        acts.append(h)
    return h, (acts, pre)


def loss(theta, X, Y):
    """Mean squared error over all outputs."""
    P, _ = forward(theta, X)
    return float(np.mean((P - Y) ** 2))


def backward(theta, X, Y):
    """(loss, gradient of the mean squared error w.r.t. theta)."""
    layers = unpack(theta)
    P, (acts, pre) = forward(theta, X)
    n = X.shape[0]
    d = 2.0 * (P - Y) / (n * P.shape[1])
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        if li < len(layers) - 1:
            d = d * gelu_grad(pre[li])
        grads.append((acts[li].T @ d, d.sum(axis=0)))
        d = d @ W.T
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return float(np.mean((P - Y) ** 2)), flat


def adam(theta, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def quad_force(p, M, com, Q, G=1.0):
    """Monopole + quadrupole force of a cell at p (Sect. 4.2, reading R3)."""
    d = com - p
    r2 = d @ d
    inv = 1.0 / math.sqrt(r2)
    Qm = np.array([[Q[0], Q[3], Q[4]], [Q[3], Q[1], Q[5]], [Q[4], Q[5], Q[2]]])
    qd = Qm @ d
    dqd = d @ qd
    inv5 = inv ** 5
    return G * (M * inv ** 3 * d + 2.5 * dqd * inv5 * inv * inv * d - inv5 * qd)


def exact_force(p, xs, ms, G=1.0):
    """Eq. 1 over the cell's particles (no softening)."""
    d = xs - p
    r = np.sqrt(np.sum(d * d, axis=1))
    return G * np.sum((ms / r ** 3)[:, None] * d, axis=0)


def features(p, M, com, Q, centre, w, count):
    """The 12 inputs of the network for target point p and one cell."""
    r = p - com
    R = math.sqrt(r @ r)
    rh = r / R
    Qm = np.array([[Q[0], Q[3], Q[4]], [Q[3], Q[1], Q[5]], [Q[4], Q[5], Q[2]]]) / (M * w * w)
    Qr = Qm @ rh
    return np.array([rh[0], rh[1], rh[2], w / R, math.log10(count),
                     (com[0] - centre[0]) / w, (com[1] - centre[1]) / w, (com[2] - centre[2]) / w,
                     rh @ Qr, math.sqrt(Qr @ Qr), float(np.sum(Qm * Qm)), float(np.linalg.det(Qm))])


def label(p, M, com, Q, xs, ms, G=1.0):
    """(exact - multipole) cell force in units of G M / R^2."""
    r = p - com
    R2 = r @ r
    return (exact_force(p, xs, ms, G) - quad_force(p, M, com, Q, G)) / (G * M / R2)
