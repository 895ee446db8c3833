"""Edge sizes through the C ABI: a single particle, one ragged warp tile and
a few tiles, where the walks' per-SM tile queues hold fewer tiles than there
are SMs.  Forces against the oracle's tree (FP64 walk 1e-12, FP32 walk 1e-5)
and the step's pair set on the gravity tree against brute force on the GPU's
positions (bit-identical)."""
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


def _dense(n, seed, L=12.0):
    """n particles of radius 1 m packed into an L x L sheet (many overlaps)."""
    g = np.random.default_rng(seed)
    x, y = g.uniform(-L / 2, L / 2, (2, n))
    z = g.normal(0.0, 0.5, n)
    vx, vz = g.normal(0.0, 2e-4, (2, n))
    vy = -1.5 * I.OMEGA * x + g.normal(0.0, 2e-4, n)
    m = np.full(n, 1675.516)
    return (x, y, z, vx, vy, vz, m, np.ones(n))


def _cfg(rb, L, walk):
    return dict(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
                integrator=rb.RB_INT_SEI, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1,
                walk=walk)


def _params(orc, L):
    return orc.Params(G=I.G_SI, omega=I.OMEGA, L=(L, L, L), nghost=(1, 1, 0), boundary=2, integrator=1,
                      theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)


@pytest.mark.parametrize("n", [1, 2, 31, 33, 97])
@pytest.mark.parametrize("walk", [0, 1])
def test_forces_at_edge_sizes(rb, orc, n, walk):
    L = 12.0
    P = _dense(n, 100 + n)
    sim = rb.Sim(**_cfg(rb, L, walk))
    sim.set_particles(P)
    a = sim.gravity()
    ref = orc.tree_gravity(_params(orc, L), 0.0, P[0], P[1], P[2], P[6])
    if n == 1:
        # a lone particle feels only its own images, whose pulls cancel: the
        # net force is rounding noise on the scale of one image's pull
        scale = I.G_SI * P[6][0] / L**2
        assert np.max(np.abs(ref)) <= 1e-14 * scale
        assert np.max(np.abs(a)) <= (1e-12 if walk == 0 else 1e-6) * scale
        return
    e = orc.force_errors(a, ref)
    assert e[2] <= (1e-12 if walk == 0 else 1e-5), e


@pytest.mark.parametrize("n", [2, 31, 33, 97])
def test_step_pairs_at_edge_sizes(rb, orc, n):
    L = 12.0
    P = _dense(n, 200 + n)
    sim = rb.Sim(**_cfg(rb, L, 1))
    sim.set_particles(P)
    p = _params(orc, L)
    found = 0
    for k in range(2):
        sim.step(1)
        got = sim.particles()
        keys = rb.pair_keys(*sim.pairs(detect=False))
        ref = orc.collide_brute(p, orc.time_at(p, 2 * (k + 1)), got["x"], got["y"], got["z"], got["r"],
                                got["id"])
        assert np.array_equal(keys, ref), k
        found += len(ref)
    if n > 2:
        assert found > 0


@pytest.mark.parametrize("boundary", [0, 1, 2])
def test_positions_on_the_box_faces(rb, orc, boundary):
    """Particles at rest exactly on the box faces, one ulp inside and outside
    them, and on Morton grid lines: one drift-only step (open, periodic and
    shear-periodic boxes) keeps, wraps or removes each of them exactly as the
    oracle does, bit for bit."""
    L = 16.0
    h = L / 2
    edge = np.array([-h, h, np.nextafter(-h, 0.0), np.nextafter(h, 0.0), np.nextafter(-h, -np.inf),
                     np.nextafter(h, np.inf), 0.0, -0.0, L / 2 ** 21 - h, np.nextafter(L / 2 ** 21 - h, 0.0)])
    g = np.random.default_rng(31)
    k = len(edge)
    x = np.concatenate([edge, g.choice(edge, 3 * k), g.uniform(-h, h, 40)])
    n = len(x)
    y = np.concatenate([g.uniform(-h, h, k), g.choice(edge, 3 * k), g.choice(edge, 40)])
    z = np.concatenate([g.uniform(-1, 1, k + 3 * k), g.choice(edge[[0, 2, 3, 6, 7, 8, 9]], 40)])
    zero = np.zeros(n)
    bc = (rb.RB_BC_OPEN, rb.RB_BC_PERIODIC, rb.RB_BC_SHEAR)[boundary]
    sim = rb.Sim(G=1.0, omega=1e-3, box=(L, L, L), nghost=(1, 1, 0), boundary=bc,
                 integrator=rb.RB_INT_LEAPFROG, dt=0.01, gravity=0, collisions=0)
    sim.set_particles((x, y, z, zero, zero, zero, np.ones(n), zero))
    sim.step(1)
    got = sim.particles()
    p = orc.Params(omega=1e-3, L=(L, L, L), nghost=(1, 1, 0), boundary=boundary, integrator=0, dt=0.01,
                   gravity=0, collisions=0)
    st = orc.State(p, x, y, z, zero, zero, zero, np.ones(n), zero)
    st.step(1)
    assert got["id"].tolist() == st.id.tolist()
    for key in ("x", "y", "z", "vy"):
        assert np.array_equal(got[key], getattr(st, key)), key
    if boundary:
        assert np.any(got["x"] == -h) and not np.any(got["x"] >= h)


@pytest.mark.parametrize("boundary", [1, 2])
def test_fast_particles_wrap_several_boxes(rb, orc, boundary):
    """Particles whose drift half carries them up to 7.3 box lengths in x and
    y, either way, over three drift-only steps: the periodic and the
    shear-periodic wrap of Sect. 2.3 (an x crossing shifts y by the shear
    offset and v_y by 1.5 Omega Lx) give the oracle's positions and
    velocities bit for bit.  By reading R6 x is wrapped once per drift half
    and y one box length at a time until it is inside, so y always ends in
    the box and x need not."""
    L = 16.0
    g = np.random.default_rng(41)
    n = 200
    x, y = g.uniform(-L / 2, L / 2, (2, n))
    z = g.uniform(-1, 1, n)
    dt = 0.5
    # |v| dt / 2 up to 7.3 L, both signs, in x and in y
    vx = g.uniform(-7.3, 7.3, n) * L / (dt / 2)
    vy = g.uniform(-7.3, 7.3, n) * L / (dt / 2)
    vz = np.zeros(n)
    zero = np.zeros(n)
    bc = (rb.RB_BC_OPEN, rb.RB_BC_PERIODIC, rb.RB_BC_SHEAR)[boundary]
    sim = rb.Sim(G=1.0, omega=1e-2, box=(L, L, L), nghost=(1, 1, 0), boundary=bc,
                 integrator=rb.RB_INT_LEAPFROG, dt=dt, gravity=0, collisions=0)
    sim.set_particles((x, y, z, vx, vy, vz, np.ones(n), zero))
    p = orc.Params(omega=1e-2, L=(L, L, L), nghost=(1, 1, 0), boundary=boundary, integrator=0, dt=dt,
                   gravity=0, collisions=0)
    st = orc.State(p, x, y, z, vx, vy, vz, np.ones(n), zero)
    for k in range(3):
        sim.step(1)
        st.step(1)
        got = sim.particles()
        assert got["id"].tolist() == st.id.tolist(), k
        for key in ("x", "y", "z", "vx", "vy"):
            assert np.array_equal(got[key], getattr(st, key)), (k, key)
        assert np.all(np.abs(got["y"]) <= L / 2)


def _leaving(n, seed):
    """_dense particles of radius 0.3 m (a few hundred pairs) of which 40 sit
    at z = +-5.9 m moving outward at 3 mm/s: inside the 12 m box after the
    first drift half of a step, outside it after the second."""
    x, y, z, vx, vy, vz, m, r = (np.array(a) for a in _dense(n, seed))
    r[:] = 0.3
    g = np.random.default_rng(seed + 1)
    k = g.choice(n, 40, replace=False)
    side = np.where(np.arange(40) % 2 == 0, 1.0, -1.0)
    z[k] = side * 5.9
    vz[k] = side * 3e-3
    return (x, y, z, vx, vy, vz, m, r)


@pytest.mark.parametrize("walk", [0, 1])
def test_particles_leaving_in_the_second_drift(rb, orc, walk):
    """Particles that leave through the open z faces in a step's second drift
    half: they still sit in that step's gravity tree when its cells get the
    boxes of the end-of-step positions and the collision search runs.  The
    pair set of every step equals brute force on the positions the GPU
    returns, the removed ids equal the oracle's, and reads skip them."""
    L, n = 12.0, 300
    P = _leaving(n, 5)
    sim = rb.Sim(**_cfg(rb, L, walk))
    sim.set_particles(P)
    p = _params(orc, L)
    st = orc.State(p, *P)
    for s in range(2):
        sim.step(1)
        st.step(1)
        got = sim.particles()
        keys = rb.pair_keys(*sim.pairs(detect=False))
        ref = orc.collide_brute(p, orc.time_at(p, 2 * (s + 1)), got["x"], got["y"], got["z"], got["r"],
                                got["id"])
        assert np.array_equal(keys, ref), s
        assert len(ref) > 0
        assert got["id"].tolist() == st.id.tolist(), s
        assert np.all(np.abs(got["z"]) < L / 2)
    assert len(got["id"]) <= n - 40
    if walk == 0:
        assert np.max(np.abs(got["x"] - st.x)) <= 1e-9 * L


@pytest.mark.parametrize("walk", [0, 1])
def test_ensemble_with_particles_leaving(rb, orc, walk):
    """The same in a batched simulation of three boxes: each box advances as
    it does alone, and each box's pairs equal brute force on its positions."""
    L, n = 12.0, 300
    seeds = (5, 15, 25)
    ens = rb.Sim(nbox=len(seeds), **_cfg(rb, L, walk))
    for b, seed in enumerate(seeds):
        ens.set_particles(_leaving(n, seed), box=b)
    ens.step(2)
    p = _params(orc, L)
    tol = 1e-12 if walk == 0 else 1e-9
    for b, seed in enumerate(seeds):
        one = rb.Sim(**_cfg(rb, L, walk))
        one.set_particles(_leaving(n, seed))
        one.step(2)
        ge, go = ens.particles(b), one.particles()
        assert len(ge["id"]) <= n - 40
        assert ge["id"].tolist() == go["id"].tolist()
        for f in ("x", "y", "z", "vx", "vy", "vz"):
            assert np.max(np.abs(ge[f] - go[f])) <= tol * max(L, np.max(np.abs(go[f]))), (b, f)
        keys = rb.pair_keys(*ens.pairs(box=b, detect=False))
        ref = orc.collide_brute(p, orc.time_at(p, 4), ge["x"], ge["y"], ge["z"], ge["r"], ge["id"])
        assert np.array_equal(keys, ref), b


@pytest.mark.parametrize("walk", [0, 1])
def test_boxes_that_empty_and_empty_simulations(rb, orc, walk):
    """Every particle of a box leaves through the open z faces in the first
    step: the following steps run on an empty box (alone, and beside a box
    that keeps its particles), and a simulation with no particles steps."""
    L, n = 12.0, 64
    g = np.random.default_rng(9)
    x, y = g.uniform(-L / 2, L / 2, (2, n))
    side = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    z = side * 5.9
    vz = side * 3e-3
    zero = np.zeros(n)
    P = (x, y, z, zero, -1.5 * I.OMEGA * x, vz, np.full(n, 1675.516), np.full(n, 0.3))
    sim = rb.Sim(**_cfg(rb, L, walk))
    sim.set_particles(P)
    sim.step(3)
    assert len(sim.particles()["id"]) == 0
    ens = rb.Sim(nbox=2, **_cfg(rb, L, walk))
    ens.set_particles(P, box=0)
    Q = _leaving(200, 41)
    ens.set_particles(Q, box=1)
    ens.step(3)
    one = rb.Sim(**_cfg(rb, L, walk))
    one.set_particles(Q)
    one.step(3)
    assert len(ens.particles(0)["id"]) == 0
    ge, go = ens.particles(1), one.particles()
    assert ge["id"].tolist() == go["id"].tolist()
    tol = 1e-12 if walk == 0 else 1e-9
    assert np.max(np.abs(ge["x"] - go["x"])) <= tol * L
    empty = rb.Sim(**_cfg(rb, L, walk))
    empty.set_particles(tuple(np.zeros(0) for _ in range(8)))
    empty.step(2)
    assert len(empty.particles()["id"]) == 0


def test_sweep_detector_with_particles_leaving(rb, orc):
    """The plane sweep with FP64 tree gravity while particles leave through
    the open z faces in the second drift half: the same ids as the oracle and
    its trajectory within 1e-9 after 3 steps."""
    L, n = 12.0, 300
    P = _leaving(n, 51)
    cfg = _cfg(rb, L, rb.RB_WALK_FP64)
    cfg["collisions"] = rb.RB_COLL_SWEEP
    sim = rb.Sim(**cfg)
    sim.set_particles(P)
    sim.step(3)
    got = sim.particles()
    p = orc.Params(G=I.G_SI, omega=I.OMEGA, L=(L, L, L), nghost=(1, 1, 0), boundary=2, integrator=1,
                   theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=orc.COLL_SWEEP)
    st = orc.State(p, *P)
    st.step(3)
    assert st.n <= n - 40
    assert got["id"].tolist() == st.id.tolist()
    for f in ("x", "y", "z"):
        assert np.max(np.abs(got[f] - getattr(st, f))) <= 1e-9 * L, f
    for f in ("vx", "vy", "vz"):
        ref = getattr(st, f)
        assert np.max(np.abs(got[f] - ref)) <= 1e-9 * np.max(np.abs(ref)), f


def test_set_box_after_particles_left(rb, orc):
    """rb_set_box after some ids left through the open z faces keeps the live
    particles, renumbered 0 .. n_live - 1 in id order, and the simulation
    then steps exactly as a fresh one given those particles."""
    L, n = 12.0, 300
    P = _leaving(n, 61)
    fields = ("x", "y", "z", "vx", "vy", "vz", "m", "r")
    sim = rb.Sim(**_cfg(rb, L, rb.RB_WALK_FP64))
    sim.set_particles(P)
    sim.step(1)
    a = sim.particles()
    assert len(a["id"]) <= n - 40
    sim.set_box(0, (L, L, L))
    b = sim.particles()
    assert b["id"].tolist() == list(range(len(a["id"])))
    for f in fields:
        assert np.array_equal(b[f], a[f]), f
    sim.step(2)
    fresh = rb.Sim(**_cfg(rb, L, rb.RB_WALK_FP64))
    fresh.set_particles(tuple(a[f] for f in fields))
    fresh.step(2)
    c, d = sim.particles(), fresh.particles()
    assert c["id"].tolist() == d["id"].tolist()
    for f in fields:
        assert np.max(np.abs(c[f] - d[f])) <= 1e-12 * max(L, np.max(np.abs(d[f]))), f


@pytest.mark.parametrize("walk", [0, 1])
def test_setting_fewer_then_more_particles(rb, orc, walk):
    """rb_set_particles on a simulation already on the device with fewer
    particles than before (copied into the existing buffers), then with more
    than its capacity (new buffers): each time the simulation steps exactly
    as a fresh one given the same particles."""
    L = 12.0
    fields = ("x", "y", "z", "vx", "vy", "vz", "m", "r")
    sim = rb.Sim(**_cfg(rb, L, walk))
    for n, seed in ((200, 71), (90, 72), (350, 73)):
        P = _dense(n, seed)
        P = P[:7] + (np.full(n, 0.3),)
        sim.set_particles(P)
        sim.step(2)
        fresh = rb.Sim(**_cfg(rb, L, walk))
        fresh.set_particles(P)
        fresh.step(2)
        c, d = sim.particles(), fresh.particles()
        assert c["id"].tolist() == d["id"].tolist() == list(range(n))
        for f in fields:
            assert np.max(np.abs(c[f] - d[f])) <= 1e-12 * max(L, np.max(np.abs(d[f]))), (n, f)
        assert np.array_equal(rb.pair_keys(*sim.pairs(detect=False)), rb.pair_keys(*fresh.pairs(detect=False)))


def test_ensemble_box_replaced_after_others_lost_particles(rb, orc):
    """In a batched simulation, replacing one box's particles keeps the other
    box's live particles (renumbered over the ids that left through the open
    z faces); both boxes then step as fresh single boxes with those states.
    FP64 walk: the FP32 walk groups a box's terms by the warps that hold its
    targets, and in these dense boxes the collisions carry that rounding
    into the trajectories."""
    L, walk = 12.0, 0
    fields = ("x", "y", "z", "vx", "vy", "vz", "m", "r")
    A, B, Cp = _leaving(300, 81), _leaving(200, 82), _leaving(250, 83)
    ens = rb.Sim(nbox=2, **_cfg(rb, L, walk))
    ens.set_particles(A, box=0)
    ens.set_particles(B, box=1)
    ens.step(2)
    a0 = ens.particles(0)
    assert len(a0["id"]) <= 300 - 40
    ens.set_particles(Cp, box=1)
    b0 = ens.particles(0)
    assert b0["id"].tolist() == list(range(len(a0["id"])))
    for f in fields:
        assert np.array_equal(b0[f], a0[f]), f
    ens.step(2)
    tol = 1e-12
    for box, state in ((0, tuple(a0[f] for f in fields)), (1, Cp)):
        one = rb.Sim(**_cfg(rb, L, walk))
        one.set_particles(state)
        one.step(2)
        ge, go = ens.particles(box), one.particles()
        assert ge["id"].tolist() == go["id"].tolist(), box
        for f in fields:
            assert np.max(np.abs(ge[f] - go[f])) <= tol * max(L, np.max(np.abs(go[f]))), (box, f)
