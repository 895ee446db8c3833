"""rb_energy_sums_noalloc: the energy and momentum sums for callers that
cannot allocate device memory (their device memory belongs to another
runtime's pool, or they must not trigger an allocation's implicit device
synchronisation).  The test owns the device buffers (through torch); the entry
point itself uses only its fixed in-library scratch.  Its output must equal
rb_energy's on the same particles, on two calls in a row, and a size beyond
its fixed maximum must be refused.  The file name makes pytest collect it
last."""
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


def test_noalloc_energy_matches_rb_energy(rb):
    torch = pytest.importorskip("torch")
    L, N = 650.0, 100_000
    P = I.sheet(L, N, 2)
    sim = rb.Sim(G=I.G_SI, omega=I.OMEGA, box=(L, L, L), nghost=(1, 1, 0),
                 boundary=rb.RB_BC_SHEAR, integrator=rb.RB_INT_SEI, dt=I.DT_SHEET, gravity=0,
                 collisions=0)
    sim.set_particles(P)
    E_ref, P_ref = sim.energy()

    dev = torch.device("cuda:0")
    arr = {k: torch.tensor(getattr(P, k), dtype=torch.float64, device=dev)
           for k in ("m", "x", "z", "vx", "vy", "vz")}
    out = torch.full((7,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    results = []
    for _ in range(2):
        rb.rb_energy_sums_noalloc(N, arr["m"].data_ptr(), arr["x"].data_ptr(), arr["z"].data_ptr(),
                                  arr["vx"].data_ptr(), arr["vy"].data_ptr(), arr["vz"].data_ptr(),
                                  None, rb.RB_INT_SEI, I.OMEGA, 0.0, out.data_ptr(),
                                  stream.cuda_stream)
        torch.cuda.synchronize(dev)
        results.append(out.cpu().numpy().copy())
        out.fill_(float("nan"))
    for r in results:
        assert r[6] == N
        E = r[0] + r[1] + r[2]
        assert abs(E - E_ref) <= 1e-12 * (abs(r[0]) + abs(r[1]))
        scale = np.sum(P.m * np.abs(P.vy))
        np.testing.assert_allclose(r[3:6], P_ref, rtol=0, atol=1e-12 * scale)
    np.testing.assert_array_equal(results[0], results[1])


def test_noalloc_leapfrog_and_potential_terms(rb):
    """Leap-frog without x and z (the tidal term is 0) and a device array phi:
    the kinetic and momentum sums equal rb_energy's on a leap-frog box, and
    the W slot equals (1/2) sum m phi summed on the host, on two calls."""
    torch = pytest.importorskip("torch")
    L, N = 650.0, 70_001
    P = I.sheet(L, N, 4)
    sim = rb.Sim(G=1.0, box=(L, L, L), boundary=rb.RB_BC_PERIODIC, integrator=rb.RB_INT_LEAPFROG,
                 dt=1e-3, gravity=0, collisions=0)
    sim.set_particles(P)
    E_ref, P_ref = sim.energy()
    phi = -np.random.default_rng(5).uniform(0.5, 2.0, N)
    W_ref = float(np.sum(0.5 * P.m * phi))
    dev = torch.device("cuda:0")
    arr = {k: torch.tensor(getattr(P, k), dtype=torch.float64, device=dev)
           for k in ("m", "vx", "vy", "vz")}
    dphi = torch.tensor(phi, dtype=torch.float64, device=dev)
    out = torch.full((7,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        out.fill_(float("nan"))
        rb.rb_energy_sums_noalloc(N, arr["m"].data_ptr(), None, None, arr["vx"].data_ptr(),
                                  arr["vy"].data_ptr(), arr["vz"].data_ptr(), dphi.data_ptr(),
                                  rb.RB_INT_LEAPFROG, 0.0, 0.0, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize(dev)
        r = out.cpu().numpy()
        assert r[6] == N and r[1] == 0.0
        assert abs(r[0] - E_ref) <= 1e-12 * abs(E_ref)
        assert abs(r[2] - W_ref) <= 1e-12 * abs(W_ref)
        scale = np.sum(P.m * np.abs(P.vy))
        np.testing.assert_allclose(r[3:6], P_ref, rtol=0, atol=1e-12 * scale)


def test_noalloc_rejects_sizes_beyond_its_scratch(rb):
    with pytest.raises(rb.RbError) as ei:
        rb.rb_energy_sums_noalloc(16_777_217, None, None, None, None, None, None, None,
                                  rb.RB_INT_LEAPFROG, 0.0, 0.0, None, None)
    assert ei.value.code == rb.RB_ERR_ARG
    assert "16777216" in str(ei.value)
