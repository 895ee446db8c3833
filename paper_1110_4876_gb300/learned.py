"""Training recipe of the learned far-field correction.

Residual samples are drawn with librb from two snapshots each of the small
(100 m, 2400 particles) and mid (650 m, 100 000 particles) shearing sheets:
every cell accepted at theta = 0.8 with w/R > 0.5 is a candidate, and a
counter-based hash keeps a fraction of them (about 10 million rows).  The network is then trained on the GPU by librb's own
kernels (Adam, standardised inputs/outputs, zero-initialised last layer).
Everything numeric runs in librb; this module only chooses the recipe.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I
from . import rb

THETA_WIDE = 0.8       # opening angle of the learned walk
THETA_FALLBACK = 0.5   # cells with w/R above this get the learned residual


def init_weights(seed: int) -> np.ndarray:
    """He-normal hidden layers, zero biases, zero last layer (9347 floats,
    standardised units for rb_mlp_train)."""
    g = np.random.Generator(np.random.PCG64(seed))
    sizes = [12, 64, 64, 64, 3]
    parts = []
    for li, (a, b) in enumerate(zip(sizes[:-1], sizes[1:])):
        last = li == len(sizes) - 2
        parts.append(np.zeros(a * b) if last else g.normal(0.0, np.sqrt(2.0 / a), a * b))
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


def sheet_config(walk: int, theta: float, L: float) -> dict:
    return dict(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
                integrator=rb.RB_INT_SEI, theta=theta, eps=0.5, dt=I.DT_SHEET, gravity=1,
                collisions=0, walk=walk)


# (box side, particles, seed, kept fraction, steps between snapshots): two
# snapshots of each sheet, the initial state and one after 50 steps of
# self-gravity, give ~10 million residuals
RECIPE = ((100.0, 2400, 1, 1.0), (650.0, 100_000, 2, 0.42))
SNAPSHOT_STEPS = (0, 50)


def samples(seed: int = 7):
    """(X, Y) residual samples from snapshots of the small and mid sheets."""
    Xs, Ys = [], []
    for L, N, s, prob in RECIPE:
        sim = rb.Sim(**sheet_config(rb.RB_WALK_FP32, THETA_WIDE, L))
        sim.set_particles(I.sheet(L, N, s))
        done = 0
        for k, steps in enumerate(SNAPSHOT_STEPS):
            sim.step(steps - done)
            done = steps
            X, Y, _ = rb.rb_mlp_samples(sim.h, THETA_WIDE, THETA_FALLBACK, prob, seed + k, 8_000_000,
                                        with_meta=False)
            Xs.append(X)
            Ys.append(Y)
    return np.concatenate(Xs), np.concatenate(Ys)


def train_default(seed: int = 3, epochs: int = 12):
    """Weights (raw units, for rb_load_mlp) and the per-epoch loss."""
    X, Y = samples()
    return rb.rb_mlp_train(X, Y, init_weights(seed), epochs=epochs, batch=2048, lr=1e-3, seed=1)
