"""Pins for the oracle's Cayley (BCOCB) free ring-polymer flow (no GPU)."""
import numpy as np
import pytest

from oracle import rpmd


@pytest.mark.parametrize("m,w,h", [(1.008, 500.0, 2.5e-4), (15.999, 3000.0, 1e-3), (1.008, 4e4, 2.5e-4)])
def test_cayley_flow_is_the_cayley_transform(m, w, h):
    A = np.array([[0.0, 1.0 / m], [-m * w * w, 0.0]])
    I = np.eye(2)
    C = np.linalg.solve(I - 0.5 * h * A, I + 0.5 * h * A)
    z = np.array([0.3, -1.7])
    q, p = rpmd.cayley_flow(z[0], z[1], m, w, h)
    np.testing.assert_allclose([q, p], C @ z, rtol=1e-13, atol=1e-15)


def test_cayley_flow_conserves_the_mode_energy_and_is_stable():
    """Cayley maps of S-skew matrices are S-orthogonal: 1/2 p^2/m + 1/2 m w^2 q^2 is conserved
    for any h w, however large (the strong stability BCOCB is used for)."""
    m, q, p = 1.008, 0.02, 3.0
    for w, h in [(100.0, 1e-3), (1e5, 1e-3), (3e6, 5e-4)]:
        E0 = 0.5 * p * p / m + 0.5 * m * w * w * q * q
        qq, pp = q, p
        for _ in range(1000):
            qq, pp = rpmd.cayley_flow(qq, pp, m, w, h)
        E = 0.5 * pp * pp / m + 0.5 * m * w * w * qq * qq
        assert abs(E - E0) < 1e-12 * E0


def test_cayley_flow_is_third_order_close_to_the_exact_flow():
    """Both maps are rotations in (m w q, p); the Cayley angle 2 atan(w h/2) falls short of
    w h by (w h)^3/12, so the distance between the two images shrinks 8-fold per halving."""
    m, w, q, p = 1.008, 2000.0, 0.01, 2.0
    errs = []
    for h in (2e-4, 1e-4, 5e-5):
        th = w * h
        qe = q * np.cos(th) + p / (m * w) * np.sin(th)
        pe = p * np.cos(th) - m * w * q * np.sin(th)
        qc, pc = rpmd.cayley_flow(q, p, m, w, h)
        errs.append(np.hypot(m * w * (qc - qe), pc - pe))
    R = np.hypot(m * w * q, p)
    assert abs(errs[-1] / R - (w * 5e-5) ** 3 / 12) < 1e-3 * (w * 5e-5) ** 3
    assert 7.5 < errs[0] / errs[1] < 8.5 and 7.5 < errs[1] / errs[2] < 8.5


def test_bcocb_free_ring_polymer_conserves_mode_energies():
    P, N = 32, 3
    prm = rpmd.Params(P=P, temperature=300.0, dt=0.001, gamma0=0.0, seed=4, integrator="bcocb")
    masses = np.array([15.999, 1.008, 1.008])
    st = rpmd.init_state(np.zeros((N, 3)), masses, prm)
    w = prm.omegas()
    m = masses[:, None, None]

    def mode_energy(s):
        return 0.5 * s.Pm[:, :, 1:] ** 2 / m + 0.5 * m * w[None, None, 1:] ** 2 * s.Q[:, :, 1:] ** 2
    E0 = mode_energy(st)
    for _ in range(200):
        rpmd.free_flow(st, prm, masses, 0.5 * prm.dt)
        rpmd.free_flow(st, prm, masses, 0.5 * prm.dt)
    np.testing.assert_allclose(mode_energy(st), E0, rtol=1e-12)
