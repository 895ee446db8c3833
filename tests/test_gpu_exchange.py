"""Host <-> device exchange through the C ABI: the direct copy into a
single-box simulation already on the device equals a fresh upload, reads
into caller-provided arrays equal ordinary reads, ids stay in order with gaps
closed after open-boundary removals, and rb_set_box keeps the particles."""
import numpy as np
import pytest

from paper_1110_4876_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "r")


@pytest.fixture(scope="module")
def rb():
    from paper_1110_4876_gb300 import build, rb as _rb

    build.build()
    _rb.load()
    return _rb


def _cfg(rb, L):
    return dict(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
                integrator=rb.RB_INT_SEI, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in FIELDS) and np.array_equal(a["id"], b["id"])


def test_direct_copy_equals_fresh_upload(rb):
    L, N = 160.0, 6000
    P1, P2 = I.sheet(L, N, 3), I.sheet(L, N, 4)
    reused = rb.Sim(**_cfg(rb, L))
    reused.set_particles(P1)
    reused.step(2)
    reused.set_particles(P2)          # single box, already on the device: direct copy
    reused.step(3)
    fresh = rb.Sim(**_cfg(rb, L))
    fresh.set_particles(P2)
    fresh.step(3)
    assert _same(reused.particles(), fresh.particles())
    assert reused.stats()["steps"] == 3


def test_read_into_caller_arrays(rb):
    L, N = 160.0, 6000
    sim = rb.Sim(**_cfg(rb, L))
    sim.set_particles(I.sheet(L, N, 5))
    sim.step(2)
    ref = sim.particles()
    out = {k: np.full(N + 7, np.nan) for k in FIELDS}
    out["id"] = np.full(N + 7, -1, dtype=np.int64)
    got = sim.particles(out=out)
    assert _same(got, ref)
    assert np.array_equal(ref["id"], np.arange(N))


def test_removed_particles_leave_gaps_in_ids(rb, orc):
    g = np.random.default_rng(8)
    n, L = 4000, 10.0
    x, y, z = g.uniform(-L / 2, L / 2, (3, n))
    vx, vy, vz = g.normal(0, 20.0, (3, n))
    zero = np.zeros(n)
    sim = rb.Sim(G=1.0, box=(L, L, L), boundary=rb.RB_BC_OPEN, dt=0.01, gravity=0, collisions=0,
                 integrator=rb.RB_INT_LEAPFROG)
    sim.set_particles((x, y, z, vx, vy, vz, np.ones(n), zero))
    sim.step(3)
    # the second upload goes straight to the device; the removals still work
    sim.set_particles((x, y, z, vx, vy, vz, np.ones(n), zero))
    sim.step(3)
    got = sim.particles()
    p = orc.Params(L=(L, L, L), boundary=0, dt=0.01, gravity=0, collisions=0)
    st = orc.State(p, x, y, z, vx, vy, vz, np.ones(n), zero)
    st.step(3)
    assert 0 < st.n < n
    assert got["id"].tolist() == st.id.tolist()
    for k, ref in zip(("x", "y", "z", "vx", "vy", "vz"), (st.x, st.y, st.z, st.vx, st.vy, st.vz)):
        assert np.array_equal(got[k], ref), k


def test_set_box_keeps_the_particles(rb):
    L, N = 160.0, 6000
    sim = rb.Sim(**_cfg(rb, L))
    sim.set_particles(I.sheet(L, N, 6))
    sim.step(2)
    sim.set_particles(I.sheet(L, N, 7))   # direct copy: the host copy is now stale
    sim.step(1)
    before = sim.particles()
    sim.set_box(0, (L, L, L))
    assert _same(sim.particles(), before)


def test_rejected_direct_copy_keeps_the_state(rb):
    """The direct copy is checked on the device before the simulation
    switches to it: a non-finite or negative entry is refused and the
    previous particles stay in place."""
    L, N = 160.0, 6000
    sim = rb.Sim(**_cfg(rb, L))
    sim.set_particles(I.sheet(L, N, 8))
    sim.step(2)
    before = sim.particles()
    for field, value, code in ((0, np.nan, rb.RB_ERR_NONFINITE), (4, np.inf, rb.RB_ERR_NONFINITE),
                               (6, -1.0, rb.RB_ERR_ARG), (7, -0.5, rb.RB_ERR_ARG)):
        bad = [a.copy() for a in I.sheet(L, N, 9).arrays()]
        bad[field][1234] = value
        with pytest.raises(rb.RbError) as e:
            sim.set_particles(tuple(bad))
        assert e.value.code == code
        assert _same(sim.particles(), before)
    sim.step(1)
    assert sim.stats()["steps"] == 3
