"""Learned far-field correction on the GPU against the FP64 oracle
(oracle/mlp.py): gradients of the tensor-core training kernels, the
residual samples (features and labels of every band cell of sampled
targets), training progress, and the accuracy gain over the plain tree at
the same wide opening angle, judged by the direct sum."""
import math

import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1110_4876_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    from paper_1110_4876_gb300 import build, rb as _rb

    build.build()
    _rb.load()
    return _rb


def sheet_cfg(rb, L, walk, theta, **kw):
    c = dict(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0), boundary=rb.RB_BC_SHEAR,
             integrator=rb.RB_INT_SEI, theta=theta, eps=0.5, dt=I.DT_SHEET, gravity=1,
             collisions=0, walk=walk)
    c.update(kw)
    return c


def test_gradients_match_oracle_backward(rb):
    """BF16 operands with FP32 accumulation: gradients within 1e-2 relative
    (per layer, in norm) of the FP64 backward pass."""
    g = np.random.default_rng(5)
    theta = omlp.init(11)
    X = g.normal(0, 1, (256, 12))
    Y = g.normal(0, 0.3, (256, 3))
    L_ref, grad_ref = omlp.backward(theta, X, Y)
    grad, L = rb.rb_mlp_grad(theta, X, Y)
    assert L == pytest.approx(L_ref, rel=1e-2)
    k = 0
    for a, b in zip(omlp.SIZES[:-1], omlp.SIZES[1:]):
        for size in (a * b, b):
            ref = grad_ref[k: k + size]
            got = grad[k: k + size]
            assert np.linalg.norm(got - ref) <= 1e-2 * np.linalg.norm(ref) + 1e-12, (k, size)
            k += size


def _abs_envelope(theta, X, Y):
    """Per gradient element, the sum over rows of the absolute values of the
    terms the element adds up (|a|^T |d| for weights, sum |d| for biases),
    from the FP64 forward and backward of oracle/mlp.py.  An FP32 evaluation
    of an element is accurate relative to this sum, not to the net value,
    which can nearly cancel."""
    layers = omlp.unpack(theta)
    P, (acts, pre) = omlp.forward(theta, X)
    d = 2.0 * (P - Y) / (X.shape[0] * P.shape[1])
    env = []
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        if li < len(layers) - 1:
            d = d * omlp.gelu_grad(pre[li])
        env.append((np.abs(acts[li]).T @ np.abs(d), np.abs(d).sum(axis=0)))
        d = d @ W.T
    env.reverse()
    return np.concatenate([np.concatenate([eW.ravel(), eb]) for eW, eb in env])


def test_fp32_debug_gradients_match_oracle_elementwise(rb):
    """FP32 debug mode of the backward pass against the FP64 backward,
    element by element.  Every FP32 operation rounds to within u = 6e-8; an
    element's error is then a few u times the sum of the absolute values of
    the row terms it adds up (256 rows, each a product of an activation and
    an output gradient that went through 64-term sums and tanhf), so the
    bound is 1e-6 of that sum (about 16 u, the random-walk size of 256
    roundings), element by element.  The losses agree to 1e-6."""
    g = np.random.default_rng(5)
    theta = omlp.init(11)
    X = g.normal(0, 1, (256, 12))
    Y = g.normal(0, 0.3, (256, 3))
    # the FP64 reference on the same FP32-rounded inputs and weights
    t32, X32, Y32 = (a.astype(np.float32).astype(np.float64) for a in (theta, X, Y))
    L_ref, grad_ref = omlp.backward(t32, X32, Y32)
    env = _abs_envelope(t32, X32, Y32)
    grad, L = rb.rb_mlp_grad_fp32(theta, X, Y)
    assert L == pytest.approx(L_ref, rel=1e-6)
    rel = np.abs(grad.astype(np.float64) - grad_ref) / env
    print("worst error / absolute sum", float(np.max(rel)))
    assert float(np.max(rel)) <= 1e-6
    with pytest.raises(rb.RbError):
        rb.rb_mlp_grad_fp32(theta, np.zeros((4097, 12)), np.zeros((4097, 3)))


def _canonical_tree(orc, P, L):
    """Oracle canonical cells with parent/child links and direct members."""
    cells = sorted(orc.Tree(P.x, P.y, P.z, P.m, L).cells(), key=lambda c: c[0])
    owner, parent = {}, []
    for k, (d, mem, *_r) in enumerate(cells):
        parent.append(owner.get(int(mem[0]), -1))
        for q in mem:
            owner[int(q)] = k
    children = [[] for _ in cells]
    roots = []
    for k, p in enumerate(parent):
        (children[p] if p >= 0 else roots).append(k)
    direct = [set(c[1].tolist()) for c in cells]
    for k, p in enumerate(parent):
        if p >= 0:
            direct[p] -= set(cells[k][1].tolist())
    return cells, children, roots


def _oracle_band_samples(orc, P, L, targets, theta_hi, theta_lo):
    """Band cells (accepted at theta_hi with w/R > theta_lo) of the targets,
    by a plain walk over the oracle's canonical cells; features and labels
    from oracle/mlp.py."""
    cells, children, roots = _canonical_tree(orc, P, L)
    p = orc.Params(omega=I.OMEGA, L=(L,) * 3, nghost=(1, 1, 0), boundary=2)
    off, _, codes = orc.images(p, 0.0)
    pos = np.stack([P.x, P.y, P.z], axis=1)
    lo = -0.5 * L
    out = {}
    for i in targets:
        for gi in range(len(codes)):
            t = pos[i] - off[gi]
            stack = list(roots)
            while stack:
                k = stack.pop()
                d, mem, M, com, Q = cells[k]
                w = L / 2 ** d
                dd = com - t
                r2 = dd @ dd
                corner = lo + np.floor(((pos[mem[0]] - lo) / L) * 2 ** 21) // 2 ** (21 - d) * w
                inside = np.all(corner <= t) and np.all(t <= corner + w)
                if d < 21 and w * w < theta_hi ** 2 * r2 and not inside:
                    if w * w > theta_lo ** 2 * r2:
                        centre = corner + 0.5 * w
                        f = omlp.features(t, M, com, Q, centre, w, len(mem))
                        y = omlp.label(t, M, com, Q, pos[mem], P.m[mem], G=1.0)
                        out[(i, int(codes[gi]), d, int(mem.min()), len(mem))] = (
                            f, y, math.sqrt(w * w / r2), M / r2)
                    continue
                stack.extend(children[k])
    return out


def test_samples_match_oracle(rb, orc):
    L, N = 100.0, 2400
    P = I.sheet(L, N, 1)
    sim = rb.Sim(**sheet_cfg(rb, L, rb.RB_WALK_FP32, 0.8))
    sim.set_particles(P)
    X, Y, meta = rb.rb_mlp_samples(sim.h, 0.8, 0.5, 1.0, 0, 4_000_000)
    targets = list(range(0, N, 150))
    ref = _oracle_band_samples(orc, P, L, targets, 0.8, 0.5)
    got = {tuple(int(v) for v in m): (x, y) for x, y, m in zip(X, Y, meta) if int(m[0]) in targets}
    assert len(ref) > 200
    missing = set(ref) - set(got)
    extra = set(got) - set(ref)
    # only band-edge ties (w/R within 1e-5 of theta_lo) may differ
    assert all(abs(ref[k][2] - 0.5) < 1e-5 for k in missing), missing
    assert len(extra) <= max(2, len(ref) // 1000), extra
    for k in set(ref) & set(got):
        f_ref, y_ref, _, _ = ref[k]
        x, y = got[k]
        np.testing.assert_allclose(x, f_ref, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(y, y_ref, rtol=1e-4, atol=1e-6 * max(1e-3, np.abs(y_ref).max()))


def _bf16(a):
    """Round float32 values to bfloat16 (nearest even), back as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_correction_equals_oracle_sum_over_band_cells(rb, orc):
    """With any weights, learned-minus-plain force at theta = 0.8 is the sum
    over the target's band cells (w/R > 0.5) of G M / R^2 times the network
    output (oracle forward with the same BF16-rounded weights and inputs)."""
    L, N = 100.0, 2400
    P = I.sheet(L, N, 1)
    w = omlp.init(5) * 0.3
    plain = rb.Sim(**sheet_cfg(rb, L, rb.RB_WALK_FP32, 0.8))
    plain.set_particles(P)
    a0 = plain.gravity()
    learned = rb.Sim(**sheet_cfg(rb, L, rb.RB_WALK_FP32_LEARNED, 0.8))
    learned.set_particles(P)
    rb.rb_load_mlp(learned.h, w, 0.5)
    a1 = learned.gravity()
    targets = list(range(7, N, 300))
    ref = _oracle_band_samples(orc, P, L, targets, 0.8, 0.5)
    wb = _bf16(w)
    for i in targets:
        rows = [v for k, v in ref.items() if k[0] == i]
        X = _bf16(np.array([r[0] for r in rows]))
        unit = np.array([r[3] for r in rows]) * I.G_SI
        Yp, _ = omlp.forward(wb, X)
        expect = (unit[:, None] * Yp).sum(axis=0)
        got = a1[i] - a0[i]
        assert np.linalg.norm(got - expect) <= 2e-2 * np.linalg.norm(expect) + 1e-3 * np.linalg.norm(a0[i])


def test_zero_network_is_the_plain_walk(rb):
    """With every weight zero the network outputs zero, so the learned walk
    (band cells queued through the network inside the walk) gives the plain
    FP32 walk's forces bit for bit, with the same accepted sets."""
    L, N = 100.0, 2400
    P = I.sheet(L, N, 1)
    plain = rb.Sim(**sheet_cfg(rb, L, rb.RB_WALK_FP32, 0.8))
    plain.set_particles(P)
    a0, c0 = plain.gravity(counts=True)
    learned = rb.Sim(**sheet_cfg(rb, L, rb.RB_WALK_FP32_LEARNED, 0.8))
    learned.set_particles(P)
    rb.rb_load_mlp(learned.h, np.zeros(rb.RB_MLP_PARAMS, np.float32), 0.5)
    a1, c1 = learned.gravity(counts=True)
    assert learned.stats()["corrections"] > 0
    np.testing.assert_array_equal(a1, a0)
    for x, y in zip(c0, c1):
        np.testing.assert_array_equal(x, y)


@pytest.fixture(scope="module")
def trained(rb):
    """Weights trained on residuals of the small and mid sheets."""
    Xs, Ys = [], []
    for L, N, seed, prob in ((100.0, 2400, 1, 1.0), (650.0, 100_000, 2, 0.05)):
        sim = rb.Sim(**sheet_cfg(rb, L, rb.RB_WALK_FP32, 0.8))
        sim.set_particles(I.sheet(L, N, seed))
        X, Y, _ = rb.rb_mlp_samples(sim.h, 0.8, 0.5, prob, 7, 2_000_000)
        Xs.append(X)
        Ys.append(Y)
    X = np.concatenate(Xs)
    Y = np.concatenate(Ys)
    w0 = omlp.init(3)
    w0[-3 - 64 * 3:] = 0.0   # zero last layer: training starts from the mean residual
    w, hist = rb.rb_mlp_train(X, Y, w0, epochs=12, batch=2048, lr=1e-3, seed=1)
    return w, hist, X, Y


def test_training_reduces_the_loss(rb, trained):
    w, hist, X, Y = trained
    assert len(X) > 100_000
    Yd = Y.astype(np.float64)
    base = float(np.mean((Yd - Yd.mean(axis=0)) ** 2))   # predicting the mean residual
    print("loss per epoch", hist, "mean-predictor loss", base)
    assert hist[-1] < hist[0]
    assert hist[-1] < base
    # the trained weights evaluated by the FP64 oracle agree with the GPU loss
    sub = np.random.default_rng(0).choice(len(X), 4096, replace=False)
    l_ref = omlp.loss(w.astype(np.float64), X[sub].astype(np.float64), Y[sub].astype(np.float64))
    _, l_gpu = rb.rb_mlp_grad(w, X[sub], Y[sub])
    assert l_gpu == pytest.approx(l_ref, rel=5e-2)


def test_learned_walk_beats_plain_wide_walk(rb, orc, trained):
    """At theta = 0.8 the corrected forces are closer to the direct sum than
    the plain tree's (a 650 m sheet, 100k particles, 512 targets)."""
    w = trained[0]
    L, N = 650.0, 100_000
    P = I.sheet(L, N, 4)
    sel = np.random.default_rng(2).choice(N, 512, replace=False)
    p = orc.Params(G=I.G_SI, omega=I.OMEGA, L=(L,) * 3, nghost=(1, 1, 0), boundary=2)
    a_dir = orc.direct_gravity(p, 0.0, P.x, P.y, P.z, P.m, targets=sel)
    err = {}
    for name, walk, theta in (("plain 0.8", rb.RB_WALK_FP32, 0.8),
                              ("learned 0.8", rb.RB_WALK_FP32_LEARNED, 0.8),
                              ("plain 0.5", rb.RB_WALK_FP32, 0.5)):
        sim = rb.Sim(**sheet_cfg(rb, L, walk, theta))
        sim.set_particles(P)
        if walk == rb.RB_WALK_FP32_LEARNED:
            rb.rb_load_mlp(sim.h, w, 0.5)
        a = sim.gravity()
        err[name] = orc.e_sum(a[sel], a_dir)
    print(err)
    assert err["learned 0.8"] < err["plain 0.8"]
