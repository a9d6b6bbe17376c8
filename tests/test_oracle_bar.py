"""Pins for the oracle's (PI-)BAR estimator (no GPU)."""
import numpy as np

from oracle import bar, normal_modes


def _ring_samples(rng, n, P, w0, wn):
    """n exact samples of one harmonic dof (m = kT = hbar = 1) as a P-bead ring polymer:
    independent Gaussian modes of variance 1 / (w0^2 + w_n^2); returns beads [n, P]."""
    Q = rng.standard_normal((n, P)) / np.sqrt(w0 ** 2 + wn ** 2)
    T = normal_modes.transfer_matrix(P)
    return np.sqrt(P) * Q @ T.T


def test_identical_states_give_zero():
    dF, _, _ = bar.pibar(np.zeros(50), np.zeros(80), beta=1.7)
    assert abs(dF) < 1e-15


def test_fixed_point_is_solved():
    rng = np.random.default_rng(0)
    dA, dB = rng.normal(0.3, 0.5, 4000), rng.normal(0.1, 0.5, 3000)
    beta = 1.3
    dF, C, _ = bar.pibar(dA, dB, beta)
    lhs = C + np.log(np.mean(bar.fermi(-dB + C, beta)) / np.mean(bar.fermi(dA - C, beta))) / beta
    assert abs(lhs - dF) < 1e-11 and abs(C - (dF + np.log(3000 / 4000) / beta)) < 1e-12


def test_classical_harmonic_states():
    """P = 1: Dlt F = (kT/2) ln(k_B / k_A) for U = k x^2 / 2, from exact samples of each state."""
    rng = np.random.default_rng(1)
    kA, kB, n = 1.0, 1.44, 400000
    xA = rng.standard_normal(n) / np.sqrt(kA)
    xB = rng.standard_normal(n) / np.sqrt(kB)
    dF, _, _ = bar.pibar(0.5 * (kB - kA) * xA ** 2, 0.5 * (kB - kA) * xB ** 2, beta=1.0)
    assert abs(dF - 0.5 * np.log(kB / kA)) < 3e-3


def test_path_integral_harmonic_states_and_single_bead_estimator():
    """P = 8 ring polymers of harmonic states w_A = 1, w_B = 1.2 (m = kT = hbar = 1): PI-BAR with the
    bead-averaged potentials recovers the exact discrete Dlt F_P; the single-bead estimator
    (one bead's potential) agrees to within the second-order bias of the appendix."""
    rng = np.random.default_rng(2)
    P, n, wA, wB = 8, 300000, 1.0, 1.2
    wn = 2.0 * P * np.sin(np.pi * np.arange(P) / P)
    exact = bar.harmonic_ring_polymer_free_energy_difference(P, 1.0, 1.0, wA, wB)
    xA = _ring_samples(rng, n, P, wA, wn)
    xB = _ring_samples(rng, n, P, wB, wn)
    UP = lambda x: 0.5 * np.mean(x ** 2, axis=1)            # (1/P) sum_b x_b^2 / 2, per unit w^2
    dF, _, _ = bar.pibar((wB ** 2 - wA ** 2) * UP(xA), (wB ** 2 - wA ** 2) * UP(xB), beta=1.0)
    assert abs(dF - exact) < 3e-3
    d1, _, _ = bar.pibar((wB ** 2 - wA ** 2) * 0.5 * xA[:, 0] ** 2, (wB ** 2 - wA ** 2) * 0.5 * xB[:, 0] ** 2, 1.0)
    assert abs(d1 - exact) < 2e-2
    # the classical (P = 1) value differs: the quantum correction is resolved
    assert abs(exact - np.log(wB / wA)) > 5 * 3e-3
