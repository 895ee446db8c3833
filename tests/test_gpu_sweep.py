"""Plane-sweep collision detection (Sect. 5.3) on the GPU against the oracle:
bit-identical pair sets (square and elongated boxes, every boundary, up to
the full-size elongated sheet), collision-only steps with identical positions
and pair sets and velocities to rounding,
FP64 trajectories with gravity, the zero-velocity limit equal to the tree
search, and the error reported for a degenerate input."""
import numpy as np
import pytest

from _parity import arrays, state_arrays, stepwise, vel_rel_err
from paper_1110_4876_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    from paper_1110_4876_gb300 import build, rb as _rb

    build.build()
    _rb.load()
    return _rb


def _moving(seed, n, L):
    g = np.random.default_rng(seed)
    x, y = g.uniform(-L / 2, L / 2, (2, n))
    z = g.normal(0, 1.0, n)
    vx, vy, vz = g.normal(0, 0.5, (3, n))
    r = g.uniform(0.3, 0.6, n)
    return x, y, z, vx, vy, vz, np.ones(n), r


@pytest.mark.parametrize("boundary,seed", [(0, 1), (1, 2), (2, 3)])
def test_sweep_pairs_bit_identical(rb, orc, boundary, seed):
    L, n, t0, dt = 30.0, 1500, 123.4, 0.8
    P = _moving(seed, n, L)
    sim = rb.Sim(G=1.0, omega=0.02, box=(L, L, L), nghost=(1, 1, 0), boundary=boundary,
                 integrator=rb.RB_INT_LEAPFROG, gravity=0, collisions=rb.RB_COLL_SWEEP, dt=dt, t0=t0)
    sim.set_particles(P)
    got = rb.pair_keys(*sim.pairs())
    p = orc.Params(omega=0.02, L=(L, L, L), nghost=(1, 1, 0), boundary=boundary, t0=t0, dt=dt)
    x, y, z, vx, vy, vz, _, r = P
    ref = orc.collide_line_brute(p, t0, x, y, z, vx, vy, vz, r, np.arange(n))
    assert len(ref) > 100
    assert np.array_equal(got, ref)


def _long_cfg(rb, Lx, Ly, **kw):
    c = dict(G=I.G_SI, omega=I.OMEGA, box=(Lx, Ly, Lx), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
             integrator=rb.RB_INT_SEI, eps=0.5, dt=I.DT_SHEET, gravity=0,
             collisions=rb.RB_COLL_SWEEP, walk=rb.RB_WALK_FP64)
    c.update(kw)
    return c


def _long_params(orc, Lx, Ly, **kw):
    p = orc.Params(G=I.G_SI, omega=I.OMEGA, L=(Lx, Ly, Lx), nghost=(1, 1, 0), boundary=2,
                   integrator=1, eps=0.5, dt=I.DT_SHEET, gravity=0, collisions=orc.COLL_SWEEP)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_sweep_elongated_box_pairs_bit_identical(rb, orc):
    """Elongated shearing box (azimuthal size 20 R): the sweep's own
    workload, including pairs across the sheared x boundary."""
    n, Ly = 20000, 20.0
    Lx = I.long_sheet_size(n, Ly)
    P = I.sheet_xy(Lx, Ly, n, 31)
    # a dispersion of 0.05 m/s makes the trajectories long enough to matter
    g = np.random.default_rng(32)
    P.vx += g.normal(0, 0.05, n)
    P.vy += g.normal(0, 0.05, n)
    sim = rb.Sim(**_long_cfg(rb, Lx, Ly))
    sim.set_particles(P)
    got = rb.pair_keys(*sim.pairs())
    p = _long_params(orc, Lx, Ly)
    ref = orc.collide_sweep(p, 0.0, P.x, P.y, P.z, P.vx, P.vy, P.vz, P.r, np.arange(n))
    assert len(ref) > 1000
    _, _, c = orc.decode_pairs(ref)
    assert np.any(c != orc.CENTRAL_CODE)
    assert np.array_equal(got, ref)


def test_sweep_collision_steps(rb, orc):
    """Collisions only (SEI, shear, elongated box): drift and sweep are FP64
    in the oracle's operation order, so every step from the same state gives
    identical positions and pair sets, and velocities within 1e-12 (Eq. 2's
    fused form on the GPU); 8 free-running steps stay within 1e-9."""
    n, Ly = 5000, 20.0
    Lx = I.long_sheet_size(n, Ly)
    P = I.sheet_xy(Lx, Ly, n, 33)
    g = np.random.default_rng(34)
    P.vx += g.normal(0, 0.02, n)
    sim = rb.Sim(**_long_cfg(rb, Lx, Ly))
    sim.set_particles(P)
    p = _long_params(orc, Lx, Ly)
    assert stepwise(rb, orc, sim, p, 8) > 100
    got = sim.particles()
    st = orc.State(p, *P.arrays())
    st.step(8)
    ref = state_arrays(st)
    assert got["id"].tolist() == st.id.tolist()
    assert np.max(np.abs(arrays(got)[:, :3] - ref[:, :3])) <= 1e-9 * Lx
    assert vel_rel_err(arrays(got)[:, 3:], ref[:, 3:]) <= 1e-9


def test_sweep_with_tree_gravity_fp64_steps(rb, orc):
    """Small sheet with FP64 tree gravity and the sweep detector: 5 steps
    within 1e-9 relative of the oracle."""
    L, N = 100.0, 2400
    P = I.sheet(L, N, 1)
    sim = rb.Sim(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
                 integrator=rb.RB_INT_SEI, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1,
                 collisions=rb.RB_COLL_SWEEP, walk=rb.RB_WALK_FP64)
    sim.set_particles(P)
    sim.step(5)
    got = sim.particles()
    p = orc.Params(G=I.G_SI, omega=I.OMEGA, L=(L, L, L), nghost=(1, 1, 0), boundary=2, integrator=1,
                   theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=orc.COLL_SWEEP)
    st = orc.State(p, *P.arrays())
    st.step(5)
    ref = np.stack([st.x, st.y, st.z, st.vx, st.vy, st.vz], axis=1)
    g = arrays(got)
    assert got["id"].tolist() == st.id.tolist()
    assert np.max(np.abs(g[:, :3] - ref[:, :3])) <= 1e-9 * L
    assert np.max(np.abs(g[:, 3:] - ref[:, 3:])) <= 1e-9 * np.max(np.abs(ref[:, 3:]))


def test_sweep_without_motion_equals_the_tree_search(rb):
    """Periodic box, v = 0: the straight-line criterion is the overlap test,
    so the GPU sweep and the GPU tree search give the same pairs."""
    L, n = 30.0, 2000
    x, y, z, _, _, _, m, r = _moving(5, n, L)
    zero = np.zeros(n)
    keys = []
    for det in (rb.RB_COLL_TREE, rb.RB_COLL_SWEEP):
        sim = rb.Sim(G=1.0, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_PERIODIC,
                     integrator=rb.RB_INT_LEAPFROG, gravity=0, collisions=det, dt=1.0)
        sim.set_particles((x, y, z, zero, zero, zero, m, r))
        keys.append(rb.pair_keys(*sim.pairs()))
    assert len(keys[0]) > 100
    assert np.array_equal(keys[0], keys[1])


def test_sweep_full_size_elongated_sheet(rb, orc):
    """1,000,000 particles in the elongated box after 2 steps: the pair set
    of a detection on the GPU state equals the oracle sweep's on the same
    state."""
    n, Ly = 1_000_000, 20.0
    Lx = I.long_sheet_size(n, Ly)
    P = I.sheet_xy(Lx, Ly, n, 35)
    sim = rb.Sim(**_long_cfg(rb, Lx, Ly))
    sim.set_particles(P)
    sim.step(2)
    assert sim.stats()["pairs_found"] > 10000
    got = rb.pair_keys(*sim.pairs())
    d = sim.particles()
    p = _long_params(orc, Lx, Ly)
    t = 2 * I.DT_SHEET
    ref = orc.collide_sweep(p, t, d["x"], d["y"], d["z"], d["vx"], d["vy"], d["vz"], d["r"], d["id"])
    assert len(ref) > 10000
    assert np.array_equal(got, ref)


def test_degenerate_sweep_is_reported(rb):
    """More than 65536 trajectories overlapping in x: the step returns
    RB_ERR_CAPACITY instead of scanning quadratically."""
    n, L = 70000, 1000.0
    g = np.random.default_rng(6)
    x = g.uniform(-0.01, 0.01, n)
    y = g.uniform(-L / 2, L / 2, n)
    z = g.uniform(-1, 1, n)
    zero = np.zeros(n)
    sim = rb.Sim(G=1.0, box=(L, L, L), boundary=rb.RB_BC_OPEN, integrator=rb.RB_INT_LEAPFROG,
                 gravity=0, collisions=rb.RB_COLL_SWEEP, dt=1.0)
    sim.set_particles((x, y, z, zero, zero, zero, np.ones(n), np.full(n, 0.05)))
    with pytest.raises(rb.RbError) as e:
        sim.step(1)
    assert e.value.code == rb.RB_ERR_CAPACITY


def test_batched_sweep_boxes_equal_single_boxes(rb):
    """The plane sweep in a batched simulation: elongated boxes of different
    lengths and particle counts (the sweep's items sorted by box, then by
    lower end) advance exactly as each box does alone."""
    Ly = 20.0
    boxes = []
    for n, seed in ((1500, 51), (600, 52), (2500, 53)):
        Lx = I.long_sheet_size(n, Ly)
        P = I.sheet_xy(Lx, Ly, n, seed)
        P.vx += np.random.default_rng(seed + 100).normal(0, 0.02, n)
        boxes.append((Lx, P))
    Lmax = max(Lx for Lx, _ in boxes)
    ens = rb.Sim(nbox=len(boxes), **_long_cfg(rb, Lmax, Ly))
    for b, (Lx, P) in enumerate(boxes):
        ens.set_box(b, (Lx, Ly, Lx))
        ens.set_particles(P, box=b)
    ens.step(5)
    for b, (Lx, P) in enumerate(boxes):
        one = rb.Sim(**_long_cfg(rb, Lx, Ly))
        one.set_particles(P)
        one.step(5)
        ge, go = ens.particles(b), one.particles()
        assert ge["id"].tolist() == go["id"].tolist()
        np.testing.assert_array_equal(arrays(ge), arrays(go))
