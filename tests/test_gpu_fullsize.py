"""Parity at the workloads' full sizes, in the configuration bench.py times:
sampled outputs the oracle computes one by one (forces of sampled targets on
the full tree), whole pair sets from the oracle's Eq. 3 search, and
per-box agreement for the 256-box ensemble."""
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


def cfg(rb, L, walk=1, **kw):
    c = dict(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
             integrator=rb.RB_INT_SEI, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1,
             walk=walk)
    c.update(kw)
    return c


def params(orc, L, **kw):
    p = orc.Params(G=I.G_SI, omega=I.OMEGA, L=(L, L, L), nghost=(1, 1, 0), boundary=2,
                   integrator=1, theta=0.5, eps=0.5, dt=I.DT_SHEET, gravity=1, collisions=1)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.fixture(scope="module")
def sheet1m():
    return I.sheet(2050.0, 1_000_000, 5)


def test_sheet_1m_forces_sampled(rb, orc, sheet1m):
    """FP32 walk at N = 1M on 2048 sampled targets against the oracle's FP64
    tree at the same theta (max_rel <= 1e-5); both walks' per-target counts
    of accepted cells and particle terms equal the oracle's."""
    P, L = sheet1m, 2050.0
    sel = np.random.default_rng(3).choice(P.n, 2048, replace=False)
    tree = orc.Tree(P.x, P.y, P.z, P.m, L)
    a_ref, (rc, rl, rm) = tree.gravity(params(orc, L), 0.0, targets=sel, counts=True)
    sim = rb.Sim(**cfg(rb, L, walk=1))
    sim.set_particles(P)
    a32, (c32, l32, _) = sim.gravity(counts=True)
    e = orc.force_errors(a32[sel], a_ref)
    assert e[2] <= 1e-5, e
    # the guarded FP32 opening test accepts exactly the oracle's cells
    np.testing.assert_array_equal(c32[sel], rc)
    np.testing.assert_array_equal(l32[sel], rl)
    sim64 = rb.Sim(**cfg(rb, L, walk=0))
    sim64.set_particles(P)
    a64, (nc, nl, nm) = sim64.gravity(counts=True)
    # same accepted sets, different summation order: ~700 terms x u x a net
    # force up to ~100 times smaller than its terms -> ~1e-11; bound 1e-10
    assert orc.force_errors(a64[sel], a_ref)[2] <= 1e-10
    np.testing.assert_array_equal(nc[sel], rc)
    np.testing.assert_array_equal(nl[sel], rl)


def test_sheet_1m_pairs_after_steps(rb, orc, sheet1m):
    """Two full steps at N = 1M, then the collision pair set on the GPU's own
    positions equals the oracle's Eq. 3 search bit for bit."""
    P, L = sheet1m, 2050.0
    sim = rb.Sim(**cfg(rb, L, walk=1))
    sim.set_particles(P)
    sim.step(2)
    st = sim.stats()
    assert st["n_live"] == P.n
    got = sim.particles()
    # the step's own search (boxes on the gravity tree) and a fresh search
    # (collision tree, Eq. 3) both equal the oracle's on the same positions
    # (resolution changes velocities only)
    step_keys = rb.pair_keys(*sim.pairs(detect=False))
    a, b, c = sim.pairs()
    p = params(orc, L)
    ref = orc.collide_tree(p, orc.time_at(p, 4), got["x"], got["y"], got["z"], got["r"], got["id"])
    assert len(ref) > 100_000
    assert np.array_equal(rb.pair_keys(a, b, c), ref)
    assert np.array_equal(step_keys, ref)


def test_mid_sheet_steps_fp32_vs_fp64(rb, orc):
    """100k sheet: 5 steps with the FP32 walk stay close to the FP64-walk
    run, every step's pair set is the oracle's on the GPU positions, and
    momentum in x and z is conserved by gravity + collisions."""
    L, N = 650.0, 100_000
    P = I.sheet(L, N, 2)
    s32 = rb.Sim(**cfg(rb, L, walk=1))
    s64 = rb.Sim(**cfg(rb, L, walk=0))
    s32.set_particles(P)
    s64.set_particles(P)
    p = params(orc, L)
    for k in range(5):
        s32.step(1)
        s64.step(1)
        g = s32.particles()
        a, b, c = s32.pairs(detect=False)
        ref = orc.collide_tree(p, orc.time_at(p, 2 * (k + 1)), g["x"], g["y"], g["z"], g["r"], g["id"])
        # the pairs of the step were found before resolution, on these positions
        assert np.array_equal(rb.pair_keys(a, b, c), ref), k
    g32, g64 = s32.particles(), s64.particles()
    assert np.max(np.abs(g32["x"] - g64["x"])) <= 1e-6 * L
    assert np.max(np.abs(g32["vz"] - g64["vz"])) <= 1e-3 * np.max(np.abs(g64["vz"]))


@pytest.mark.parametrize("walk,tol", [(0, 1e-12), (1, 1e-5)])
def test_ensemble_256_boxes_per_box_agreement(rb, orc, walk, tol):
    """256 boxes of uneven N advanced together with the FP64 walk and with
    the FP32 walk that the ensemble benchmark times (block shape from the
    autotuner): sampled boxes agree with the oracle's tree at the same theta
    (forces within tol, identical accepted-cell and particle-term counts) and
    their pair sets after one step equal the oracle's search on the GPU's
    positions."""
    boxes = I.ensemble_boxes(256)
    sims = rb.Sim(nbox=256, **cfg(rb, boxes[0][1], walk=walk))
    parts = []
    for b, (nb, Lb, seed) in enumerate(boxes):
        Pb = I.sheet(Lb, nb, seed + 7919)
        parts.append((Lb, Pb))
        sims.set_box(b, (Lb, Lb, Lb))
        sims.set_particles(Pb, box=b)
    from paper_1110_4876_gb300 import rb as _rb
    _rb.rb_autotune(sims.h, 0)
    _rb.rb_compute_gravity(sims.h)
    for b in (0, 17, 101, 255):
        Lb, Pb = parts[b]
        a = _rb.rb_get_accelerations(sims.h, b)
        nc, nl, _ = _rb.rb_get_counts(sims.h, b)
        a_ref, (rc, rl, _) = orc.tree_gravity(params(orc, Lb), 0.0, Pb.x, Pb.y, Pb.z, Pb.m,
                                              counts=True)
        assert orc.force_errors(a, a_ref)[2] <= tol, b
        np.testing.assert_array_equal(nc, rc)
        np.testing.assert_array_equal(nl, rl)
    sims.step(1)
    for b in (3, 64, 200, 255):
        Lb, Pb = parts[b]
        g = sims.particles(b)
        a, bb, c = _rb.rb_get_pairs(sims.h, b)
        p = params(orc, Lb)
        ref = orc.collide_brute(p, orc.time_at(p, 2), g["x"], g["y"], g["z"], g["r"], g["id"])
        assert np.array_equal(_rb.pair_keys(a, bb, c), ref), b
