"""Test particles (n_active) and the power-law restitution on the GPU
against the oracle: trajectories of a sheet whose second half are test
particles (FP64 walk) and FP32 forces at the same theta; collision-only
steps with the velocity-dependent coefficient."""
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


def _arrays(d):
    return np.stack([d[k] for k in ("x", "y", "z", "vx", "vy", "vz")], axis=1)


def test_test_particle_sheet_trajectory(rb, orc):
    """Small sheet, particles 1200..2399 are test particles: 5 DKD steps with
    tree gravity (FP64 walk) and collisions within 1e-9 of the oracle."""
    L, N, na = 100.0, 2400, 1200
    P = I.sheet(L, N, 1)
    sim = rb.Sim(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
                 integrator=rb.RB_INT_SEI, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1,
                 walk=rb.RB_WALK_FP64)
    rb.rb_set_n_active(sim.h, na)
    sim.set_particles(P)
    sim.step(5)
    got = sim.particles()
    p = orc.Params(G=I.G_SI, omega=I.OMEGA, L=(L, L, L), nghost=(1, 1, 0), boundary=2, integrator=1,
                   theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1, n_active=na)
    st = orc.State(p, *P.arrays())
    st.step(5)
    ref = np.stack([st.x, st.y, st.z, st.vx, st.vy, st.vz], axis=1)
    g = _arrays(got)
    assert np.max(np.abs(g[:, :3] - ref[:, :3])) <= 1e-9 * L
    assert np.max(np.abs(g[:, 3:] - ref[:, 3:])) <= 1e-9 * np.max(np.abs(ref[:, 3:]))


@pytest.mark.parametrize("walk", [0, 1])
def test_test_particle_forces(rb, orc, walk):
    """Forces with 40% test particles equal the oracle tree built on the
    source masses (FP64: 1e-12, FP32: 1e-5 relative, floored)."""
    L, N, na = 160.0, 6000, 3600
    P = I.sheet(L, N, 7)
    sim = rb.Sim(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
                 integrator=rb.RB_INT_SEI, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=0,
                 walk=walk)
    sim.set_particles(P)
    rb.rb_set_n_active(sim.h, na)
    a = sim.gravity()
    ms = np.where(np.arange(N) < na, P.m, 0.0)
    p = orc.Params(G=I.G_SI, omega=I.OMEGA, L=(L, L, L), nghost=(1, 1, 0), boundary=2, theta=0.5)
    ref = orc.Tree(P.x, P.y, P.z, ms, L).gravity(p, 0.0)
    e = orc.force_errors(a, ref)
    assert e[2] <= (1e-12 if walk == 0 else 1e-5), e
    rb.rb_set_n_active(sim.h, -1)   # back to all active
    a_all = sim.gravity()
    ref_all = orc.Tree(P.x, P.y, P.z, P.m, L).gravity(p, 0.0)
    assert orc.force_errors(a_all, ref_all)[2] <= (1e-12 if walk == 0 else 1e-5)


def test_power_law_restitution_steps(rb, orc):
    """Collision-only periodic box with eps = min(1, (|v_n|/v_c)^-0.234):
    4 steps agree with the oracle to rounding (pow may differ in the last
    bit), and the kinetic energy falls but less than with eps = 0.5."""
    g = np.random.default_rng(11)
    n, L = 3000, 40.0
    x, y, z = g.uniform(-L / 2, L / 2, (3, n))
    vx, vy, vz = g.normal(0, 0.5, (3, n))
    m = g.uniform(0.5, 2.0, n)
    r = np.full(n, 0.5)
    cfg = dict(box=(L, L, L), nghost=(1, 1, 1), boundary=rb.RB_BC_PERIODIC, z_periodic=1, eps=0.5,
               dt=0.02, gravity=0, collisions=1, integrator=rb.RB_INT_LEAPFROG)
    sim = rb.Sim(**cfg)
    rb.rb_set_restitution(sim.h, rb.RB_EPS_POWER, 0.3, 0.234)
    sim.set_particles((x, y, z, vx, vy, vz, m, r))
    E0, _ = sim.energy()
    sim.step(4)
    E1, _ = sim.energy()
    got = sim.particles()
    p = orc.Params(L=(L, L, L), nghost=(1, 1, 1), boundary=1, z_periodic=1, eps=0.5, dt=0.02, gravity=0,
                   collisions=1, integrator=0, eps_law=1, eps_vc=0.3, eps_p=0.234)
    st = orc.State(p, x, y, z, vx, vy, vz, m, r)
    st.step(4)
    ref = np.stack([st.x, st.y, st.z, st.vx, st.vy, st.vz], axis=1)
    gg = _arrays(got)
    assert np.max(np.abs(gg[:, :3] - ref[:, :3])) <= 1e-12 * L
    assert np.max(np.abs(gg[:, 3:] - ref[:, 3:])) <= 1e-12
    const = rb.Sim(**cfg)
    const.set_particles((x, y, z, vx, vy, vz, m, r))
    const.step(4)
    Ec, _ = const.energy()
    assert Ec < E1 < E0
    with pytest.raises(rb.RbError):
        rb.rb_set_restitution(sim.h, rb.RB_EPS_POWER, 0.0, 0.234)
