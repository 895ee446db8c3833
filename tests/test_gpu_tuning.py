"""The autotuner picks the walk/search launch shapes by timing them.  The
block sizes do not change any result; the FP32 walk's warp shape (union walk
or group walk with 4-lane subgroups) and the tile order of the targets
(Morton, 2D or 3D Hilbert) change only the order in which each target's
FP32 terms are summed: its accepted cells and particle terms
are the same (counts equal), and forces agree to FP32 rounding: each shape is
within 1e-5 of the FP64 tree (the parity tests), so two shapes are within
2e-5 of each other (per-particle denominator floored at 1e-3 of the rms)."""
import numpy as np
import pytest

from paper_1110_4876_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    n = np.linalg.norm(b, axis=1)
    den = np.maximum(n, 1e-3 * np.sqrt(np.mean(n ** 2)))
    return float(np.max(np.linalg.norm(a - b, axis=1) / den))


def test_autotune_keeps_results():
    from paper_1110_4876_gb300 import build, rb

    build.build()
    L, N = 650.0, 100_000
    P = I.sheet(L, N, 2)
    cfg = dict(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
               integrator=rb.RB_INT_SEI, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    a = rb.Sim(**cfg)
    a.set_particles(P)
    acc0, cnt0 = a.gravity(counts=True)
    pairs0 = a.pairs()
    wb, sb, wg, to = rb.rb_autotune(a.h, use_cache=False)
    assert wb in (64, 128, 256) and sb in (64, 128, 256) and wg in (0, 4) and to in (0, 1, 2)
    acc1, cnt1 = a.gravity(counts=True)
    assert _rel(acc1, acc0) <= 2e-5
    for c0, c1 in zip(cnt0[:2], cnt1[:2]):
        np.testing.assert_array_equal(c0, c1)
    assert all(np.array_equal(x, y) for x, y in zip(a.pairs(), pairs0))
    # a second simulation of the same kind takes the cached choice
    b = rb.Sim(**cfg)
    b.set_particles(P)
    assert rb.rb_autotune(b.h, use_cache=True) == (wb, sb, wg, to)
    a.step(2)
    b.step(2)
    pa, pb = a.particles(), b.particles()
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.array_equal(pa[k], pb[k])


@pytest.mark.parametrize("theta", [0.5, 0.7])
def test_every_launch_shape_gives_the_same_forces_and_pairs(theta):
    """Every block size of the walk and of the search, every warp shape of
    the FP32 walk (theta = 0.7 also exercises the inside rule)."""
    from paper_1110_4876_gb300 import build, rb

    build.build()
    L, N = 160.0, 6000
    P = I.sheet(L, N, 7)
    cfg = dict(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
               integrator=rb.RB_INT_SEI, theta=theta, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    sim = rb.Sim(**cfg)
    sim.set_particles(P)
    rb.rb_set_profiling(sim.h, 2)   # the counting search
    ref_a, ref_c, ref_p, ref_v = None, None, None, None
    for to in (rb.RB_TILE_MORTON, rb.RB_TILE_HILBERT_XY, rb.RB_TILE_HILBERT_XYZ):
        for wg in (0, 4):
            shape_a = None
            for wb in (64, 128, 256):
                for sb in (64, 128, 256):
                    rb.rb_set_launch_shape(sim.h, wb, sb, wg, to)
                    acc, cnt = sim.gravity(counts=True)
                    pairs = rb.pair_keys(*sim.pairs())
                    st = sim.stats()
                    visits, iters = st["search_visits"], st["search_iterations"]
                    if ref_a is None:
                        ref_a, ref_c, ref_p, ref_v = acc, cnt, pairs, visits
                    if shape_a is None:
                        shape_a = acc
                    # block sizes: bit for bit; warp shapes and tile orders:
                    # the same terms summed in another FP32 order
                    assert np.array_equal(acc, shape_a), (to, wg, wb, sb)
                    assert _rel(acc, ref_a) <= 2e-5, (to, wg, wb, sb)
                    for c, r in zip(cnt, ref_c):
                        np.testing.assert_array_equal(c, r)
                    assert np.array_equal(pairs, ref_p), (to, wg, wb, sb)
                    # each target's search is its own walk, whichever warp
                    # carries it: the entries it tests do not depend on the
                    # shape; every target tests the root of each of the 9
                    # images, and a warp iteration serves at most 32 lanes
                    assert visits == ref_v, (to, wg, wb, sb)
                    assert 9 * N <= visits <= 32 * iters
    with pytest.raises(rb.RbError):
        rb.rb_set_launch_shape(sim.h, 96, 128, 0)
    with pytest.raises(rb.RbError):
        rb.rb_set_launch_shape(sim.h, 128, 128, 8)
    with pytest.raises(rb.RbError):
        rb.rb_set_launch_shape(sim.h, 128, 128, 0, 3)


def test_search_visits_of_a_step_do_not_depend_on_the_search_block():
    """The step's search (cell boxes on the gravity tree) counts the entries
    its targets test; block sizes give bit-identical steps, so equal counts."""
    from paper_1110_4876_gb300 import build, rb

    build.build()
    L, N = 160.0, 6000
    P = I.sheet(L, N, 8)
    cfg = dict(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
               integrator=rb.RB_INT_SEI, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    sim = rb.Sim(**cfg)
    got = []
    sim.set_particles(P)
    sim.step(1)
    assert sim.stats()["search_visits"] == 0   # not counted below level 2
    rb.rb_set_profiling(sim.h, 2)
    for sb in (64, 128, 256):
        sim.set_particles(P)
        rb.rb_set_launch_shape(sim.h, 128, sb, 0, rb.RB_TILE_HILBERT_XY)
        sim.step(1)
        st = sim.stats()
        assert st["pairs_found"] > 0
        assert 9 * N <= st["search_visits"] <= 32 * st["search_iterations"]
        got.append((st["search_visits"], st["pairs_found"]))
    assert got[0] == got[1] == got[2]
    with pytest.raises(rb.RbError):
        rb.rb_set_profiling(sim.h, 3)
