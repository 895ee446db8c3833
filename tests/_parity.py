"""Shared step-by-step parity check of the GPU path against the oracle.

The GPU resolves Eq. 2 with the impulse written in a fused form (one
division, no square root) while the oracle follows the equation's steps
(n = r/|r|, v_n = u.n, Delta = -(1 + eps) v_n), so velocities agree to
rounding, not bit for bit.  Each step therefore starts the oracle from the
GPU's own state: drift and detection see identical positions, so positions
and the collision pair set must be identical, and the velocities after
resolution must agree to 1e-12 of each particle's speed (floored at 1e-3 of
the rms speed)."""
import numpy as np

FIELDS = ("x", "y", "z", "vx", "vy", "vz")


def arrays(d):
    return np.stack([d[k] for k in FIELDS], axis=1)


def state_arrays(st):
    return np.stack([getattr(st, k) for k in FIELDS], axis=1)


def vel_rel_err(v, v_ref):
    sp = np.linalg.norm(v_ref, axis=1)
    den = np.maximum(sp, 1e-3 * np.sqrt(np.mean(sp ** 2)))
    return float(np.max(np.linalg.norm(v - v_ref, axis=1) / den))


def stepwise(rb, orc, sim, p, nsteps, vtol=1e-12, xtol=None, brute_pairs=False):
    """Advance `sim` nsteps one at a time against the oracle started from the
    GPU state before each step; returns the total number of pairs found.
    xtol None: positions must be identical (no gravity: the drifts are
    FP64 in the oracle's operation order); else the largest position
    difference allowed.  brute_pairs: compare the pair set with the oracle's
    brute-force search on the GPU's own end-of-step positions (with gravity
    the kick differs in the last bits, so the two sides' positions may too)."""
    npairs = 0
    for k in range(nsteps):
        g0 = sim.particles()
        st = orc.State(p, *(g0[f] for f in FIELDS), g0["m"], g0["r"], ids=g0["id"])
        st.step_index = k
        st.step(1)
        sim.step(1)
        g = sim.particles()
        assert g["id"].tolist() == st.id.tolist(), k
        keys = rb.pair_keys(*sim.pairs(detect=False))
        if brute_pairs:
            ref_keys = orc.collide_brute(p, orc.time_at(p, 2 * (k + 1)), g["x"], g["y"], g["z"],
                                         g["r"], g["id"])
        else:
            ref_keys = st.last_pairs
        assert np.array_equal(keys, ref_keys), k
        npairs += len(keys)
        a, ref = arrays(g), state_arrays(st)
        if xtol is None:
            assert np.array_equal(a[:, :3], ref[:, :3]), k
        else:
            assert np.max(np.abs(a[:, :3] - ref[:, :3])) <= xtol, k
        assert vel_rel_err(a[:, 3:], ref[:, 3:]) <= vtol, k
    return npairs
