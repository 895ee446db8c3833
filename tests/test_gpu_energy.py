"""Energy and momentum diagnostics (Sect. 6.2) of the GPU path against the
oracle, term by term, on the GPU's own particles: the kinetic energy K, the
SEI tidal and vertical term U, the momentum P and the gravitational energy
W = (1/2) sum m phi (reading R11: phi from an FP64 tree walk at the step's
theta over the ghost images).

Tolerances: K, U and P are sums of n products, added in blocks on the GPU
and one by one in the oracle; each side is within about sqrt(n) u of the
exact sum of absolute terms for random rounding (n <= 1e5, u = 1.1e-16, so
~4e-14), bounded here by 1e-12 of the sum of absolute terms.  W: both walks
accept the same cells (tested with exact counts) and differ only in the order
of their ~1e3 terms per particle, all phi < 0, so 1e-12 relative."""
import numpy as np
import pytest

from paper_1110_4876_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    from paper_1110_4876_gb300 import build, rb as _rb

    build.build()
    _rb.load()
    return _rb


def _sheet(rb, orc, L, walk):
    cfg = dict(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
               integrator=rb.RB_INT_SEI, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1,
               walk=walk)
    p = orc.Params(G=I.G_SI, omega=I.OMEGA, L=(L, L, L), nghost=(1, 1, 0), boundary=2, integrator=1,
                   theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    return cfg, p


def _check_terms(orc, sim, p, t, box=0):
    g = sim.particles(box)
    K, U, W, P = sim.energy_terms(box)
    rK, rU, rW, rP = orc.energy_terms(p, t, g["x"], g["y"], g["z"], g["vx"], g["vy"], g["vz"], g["m"])
    m = g["m"]
    v2 = g["vx"] ** 2 + g["vy"] ** 2 + g["vz"] ** 2
    Oz = p.omega_z if p.omega_z > 0 else p.omega
    absU = np.sum(m * (0.5 * Oz * Oz * g["z"] ** 2 + 1.5 * p.omega ** 2 * g["x"] ** 2))
    assert abs(K - rK) <= 1e-12 * np.sum(0.5 * m * v2)
    assert abs(U - rU) <= 1e-12 * max(absU, 1e-300)
    for k, v in enumerate(("vx", "vy", "vz")):
        assert abs(P[k] - rP[k]) <= 1e-12 * np.sum(m * np.abs(g[v])), k
    assert rW < 0.0
    assert abs(W - rW) <= 1e-12 * abs(rW)
    E, PP = sim.energy(box)
    assert E == K + U + W
    np.testing.assert_array_equal(PP, P)
    return K, U, W


@pytest.mark.parametrize("L,N,seed,walk", [(100.0, 2400, 1, 0), (100.0, 2400, 1, 1),
                                            (650.0, 100_000, 2, 1)])
def test_sheet_energy_terms_match_oracle(rb, orc, L, N, seed, walk):
    """Small and mid shearing sheets (SEI, tree gravity, collisions): the
    terms agree with the oracle at t0 and after 3 steps; the potential walk
    is FP64 whatever the step's walk."""
    cfg, p = _sheet(rb, orc, L, walk)
    P = I.sheet(L, N, seed)
    sim = rb.Sim(**cfg)
    sim.set_particles(P)
    K0, U0, W0 = _check_terms(orc, sim, p, orc.time_at(p, 0))
    assert U0 < 0.0 < K0
    sim.step(3)
    _check_terms(orc, sim, p, orc.time_at(p, 6))


def test_open_leapfrog_energy_terms_match_oracle(rb, orc):
    """Plummer sphere, open boundaries, leap-frog, softening 1e-3 (U = 0)."""
    N = 4000
    P = I.plummer(N, 3)
    cfg = dict(G=1.0, box=(128.0,) * 3, boundary=rb.RB_BC_OPEN, integrator=rb.RB_INT_LEAPFROG,
               theta=0.5, softening=1e-3, dt=1e-3, gravity=1, collisions=0, walk=1)
    p = orc.Params(G=1.0, L=(128.0,) * 3, theta=0.5, soft=1e-3, dt=1e-3, gravity=1)
    sim = rb.Sim(**cfg)
    sim.set_particles(P)
    K, U, W = _check_terms(orc, sim, p, 0.0)
    assert U == 0.0
    # a Plummer sphere sampled from its distribution function is in virial
    # equilibrium: 2K + W ~ 0 within the sampling noise of 4000 particles
    assert abs(2 * K + W) < 0.1 * abs(W)


def test_batched_boxes_energy_terms_match_oracle(rb, orc):
    """Each box of a batched simulation (different sizes and particle
    counts) has the energy terms of that box alone, with its own ghost
    images and tree, after two steps."""
    boxes = [(60.0, 900, 41), (35.0, 300, 42), (80.0, 1500, 43)]
    cfg, _ = _sheet(rb, orc, 60.0, 1)
    ens = rb.Sim(nbox=len(boxes), **cfg)
    for b, (L, N, seed) in enumerate(boxes):
        ens.set_box(b, (L, L, L))
        ens.set_particles(I.sheet(L, N, seed), box=b)
    ens.step(2)
    for b, (L, N, seed) in enumerate(boxes):
        _, p = _sheet(rb, orc, L, 1)
        K, U, W = _check_terms(orc, ens, p, orc.time_at(p, 4), box=b)
        assert U < 0.0 < K
