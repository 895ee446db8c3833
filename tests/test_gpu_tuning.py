"""The autotuner picks walk/search launch shapes by timing them, and the
shape does not change any result: every lane runs its own walk."""
import numpy as np
import pytest

from paper_1110_4876_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_autotune_keeps_results_bit_identical():
    from paper_1110_4876_gb300 import build, rb

    build.build()
    L, N = 650.0, 100_000
    P = I.sheet(L, N, 2)
    cfg = dict(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
               integrator=rb.RB_INT_SEI, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    a = rb.Sim(**cfg)
    a.set_particles(P)
    acc0 = a.gravity()
    pairs0 = a.pairs()
    wb, sb = rb.rb_autotune(a.h, use_cache=False)
    assert wb in (64, 128, 256) and sb in (64, 128, 256)
    assert np.array_equal(a.gravity(), acc0)
    assert all(np.array_equal(x, y) for x, y in zip(a.pairs(), pairs0))
    # a second simulation of the same kind takes the cached choice
    b = rb.Sim(**cfg)
    b.set_particles(P)
    assert rb.rb_autotune(b.h, use_cache=True) == (wb, sb)
    a.step(2)
    b.step(2)
    pa, pb = a.particles(), b.particles()
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(pa[k], pb[k])


def test_every_launch_shape_gives_the_same_forces_and_pairs():
    """Every block size of the walk and of the search."""
    from paper_1110_4876_gb300 import build, rb

    build.build()
    L, N = 160.0, 6000
    P = I.sheet(L, N, 7)
    cfg = dict(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
               integrator=rb.RB_INT_SEI, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    sim = rb.Sim(**cfg)
    sim.set_particles(P)
    ref_a, ref_p = None, None
    for wb in (64, 128, 256):
        for sb in (64, 128, 256):
            rb.rb_set_launch_shape(sim.h, wb, sb)
            acc = sim.gravity()
            pairs = rb.pair_keys(*sim.pairs())
            if ref_a is None:
                ref_a, ref_p = acc, pairs
            assert np.array_equal(acc, ref_a), (wb, sb)
            assert np.array_equal(pairs, ref_p), (wb, sb)
    with pytest.raises(rb.RbError):
        rb.rb_set_launch_shape(sim.h, 96, 128)
