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
