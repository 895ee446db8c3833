"""Error handling through the C ABI without any GPU fault: the pair buffer
overflow is repaired inside the step, bad inputs and states return their
codes, a position that overflows to infinity is reported, and the bounded
wait of the resolution queue gives up with RB_ERR_TIMEOUT."""
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


def sheet(rb, L, **kw):
    c = dict(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
             integrator=rb.RB_INT_SEI, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    c.update(kw)
    return c


def test_pair_overflow_is_repaired_inside_the_step(rb):
    L, N = 100.0, 2400
    P = I.sheet(L, N, 1)
    a = rb.Sim(**sheet(rb, L))
    b = rb.Sim(**sheet(rb, L))
    a.set_particles(P)
    b.set_particles(P)
    rb.rb_set_pair_capacity(b.h, 16)
    a.step(3)
    b.step(3)
    assert b.stats()["pair_capacity"] > 16
    pa, pb = a.particles(), b.particles()
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(pa[k], pb[k]), k
    assert [x.tolist() for x in a.pairs(detect=False)] == [x.tolist() for x in b.pairs(detect=False)]


def test_bad_inputs_and_states(rb):
    L, N = 100.0, 100
    P = I.sheet(L, N, 3)
    s = rb.Sim(**sheet(rb, L))
    bad = [a.copy() for a in P.arrays()]
    bad[0][5] = np.nan
    with pytest.raises(rb.RbError) as e:
        s.set_particles(tuple(bad))
    assert e.value.code == rb.RB_ERR_NONFINITE
    with pytest.raises(rb.RbError) as e:
        rb.rb_set_particles(s.h, 3, *P.arrays())
    assert e.value.code == rb.RB_ERR_ARG
    learned = rb.Sim(**sheet(rb, L, walk=rb.RB_WALK_FP32_LEARNED))
    learned.set_particles(P)
    with pytest.raises(rb.RbError) as e:
        learned.step(1)
    assert e.value.code == rb.RB_ERR_STATE
    with pytest.raises(rb.RbError) as e:
        rb.rb_load_mlp(learned.h, np.zeros(10, np.float32), 0.5)
    assert e.value.code == rb.RB_ERR_ARG


def test_overflowing_position_is_reported(rb):
    n, L = 64, 10.0
    g = np.random.default_rng(1)
    x, y, z = g.uniform(-4, 4, (3, n))
    vx = np.zeros(n)
    vx[7] = 1e306
    zero = np.zeros(n)
    s = rb.Sim(box=(L, L, L), boundary=rb.RB_BC_OPEN, dt=1e3, gravity=0, collisions=0)
    s.set_particles((x, y, z, vx, zero, zero, np.ones(n), zero))
    with pytest.raises(rb.RbError) as e:
        s.step(1)
    assert e.value.code == rb.RB_ERR_NONFINITE


def test_resolution_wait_is_bounded(rb):
    """A pair held back from the resolution's ready queue (test hook) makes
    the threads' bounded wait for its slot run out: the step reports
    RB_ERR_TIMEOUT after about half a second, and the context stays usable
    (a fresh upload steps normally, equal to an untouched simulation)."""
    import time

    L, N = 100.0, 2400
    P = I.sheet(L, N, 1)
    s = rb.Sim(**sheet(rb, L))
    s.set_particles(P)
    rb.rb_debug_hold_pair(s.h, True)
    t0 = time.perf_counter()
    with pytest.raises(rb.RbError) as e:
        s.step(1)
    assert e.value.code == rb.RB_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 20.0
    rb.rb_debug_hold_pair(s.h, False)
    s.set_particles(P)
    s.step(2)
    ref = rb.Sim(**sheet(rb, L))
    ref.set_particles(P)
    ref.step(2)
    a, b = s.particles(), ref.particles()
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(a[k], b[k]), k
