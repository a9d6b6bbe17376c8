"""Pins for the oracle's random numbers and normal-mode algebra (no GPU)."""
import math
import os

import numpy as np
import pytest

from oracle import normal_modes as nm
from oracle import philox
from oracle.units import HBAR, KB

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    got = philox.philox4x32_10(np.array(ctr), np.array(key))
    assert [int(x) for x in got] == out


def test_uniform53_range_and_exact_values():
    z = np.array([0], dtype=np.uint32)
    f = np.array([0xFFFFFFFF], dtype=np.uint32)
    assert philox.uniform53(z, z)[0] == 0.5 * 2.0 ** -53
    u_max = philox.uniform53(f, f)[0]
    assert 0.0 < u_max <= 1.0
    # k = 2^26 * (hi >> 5) + (lo >> 6) is an exact 53-bit integer
    hi = np.array([0x80000000], dtype=np.uint32)
    assert philox.uniform53(hi, z)[0] == (2 ** 52 + 0.5) * 2.0 ** -53


def test_box_muller_pair_identity_and_moments():
    e = np.arange(200_000, dtype=np.uint64)
    z0 = philox.normals(99, e, 5, philox.TAG_OSTEP, 0)
    z1 = philox.normals(99, e, 5, philox.TAG_OSTEP, 1)
    # Box-Muller: z0^2 + z1^2 = -2 ln u1 for the same draw
    ctr = np.stack([e, np.full_like(e, 5), np.zeros_like(e), np.full_like(e, philox.TAG_OSTEP)], -1)
    x = philox.philox4x32_10(ctr, np.array([99, 0]))
    u1 = philox.uniform53(x[:, 0], x[:, 1])
    np.testing.assert_allclose(z0 ** 2 + z1 ** 2, -2.0 * np.log(u1), rtol=1e-12)
    for z in (z0, z1):
        assert abs(z.mean()) < 5.0 / math.sqrt(z.size)
        assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / z.size)
    # distinct streams are uncorrelated
    assert abs(np.corrcoef(z0, z1)[0, 1]) < 5.0 / math.sqrt(z0.size)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 7, 8, 16, 32, 64])
def test_transfer_matrix_orthonormal(P):
    T = nm.transfer_matrix(P)
    np.testing.assert_allclose(T.T @ T, np.eye(P), atol=1e-15)
    np.testing.assert_allclose(T[:, 0], 1.0 / math.sqrt(P), atol=1e-16)


@pytest.mark.parametrize("P", [2, 3, 4, 6, 8, 16, 32, 64])
def test_columns_are_eigenvectors_of_free_ring_matrix(P):
    """Eq. (2): columns of T are eigenvectors of circ(2,-1,..,-1); frequencies are the
    square roots of the eigenvalues of Omega_P^2 (checked against LAPACK)."""
    C = 2.0 * np.eye(P) - np.roll(np.eye(P), 1, axis=1) - np.roll(np.eye(P), -1, axis=1)
    if P == 2:
        C = np.array([[2.0, -2.0], [-2.0, 2.0]])
    T = nm.transfer_matrix(P)
    lam = np.array([T[:, n] @ C @ T[:, n] for n in range(P)])
    np.testing.assert_allclose(C @ T, T * lam[None, :], atol=1e-12)
    kT = KB * 300.0
    w = nm.mode_frequencies(P, kT, HBAR)
    omega2 = (P * kT / HBAR) ** 2 * C
    ev = np.sort(np.linalg.eigvalsh(omega2))
    np.testing.assert_allclose(np.sort(w ** 2), ev, rtol=1e-12, atol=1e-9 * ev.max())
    assert w[0] == 0.0


def test_centroid_is_mode_zero():
    rng = np.random.default_rng(0)
    P = 8
    Q = rng.standard_normal((5, 3, P))
    x = nm.modes_to_beads(Q, nm.transfer_matrix(P))
    np.testing.assert_allclose(x.mean(axis=-1), Q[..., 0], atol=1e-14)
    np.testing.assert_allclose(nm.beads_to_modes(x, nm.transfer_matrix(P)), Q, atol=1e-13)


@pytest.mark.parametrize("P", [1, 4, 6, 8])
def test_projection_is_minus_gradient_of_UP(P):
    """Eqs. (10)-(11): f_n equals -dU_P/dQ_n, U_P = (1/P) sum_i V(x_i) (Eq. (3)), by central FD."""
    rng = np.random.default_rng(1)
    T = nm.transfer_matrix(P)

    def V(x):            # anharmonic 1D potential per coordinate
        return 0.3 * x ** 4 - x ** 2 + 0.5 * np.sin(3 * x)

    def dV(x):
        return 1.2 * x ** 3 - 2 * x + 1.5 * np.cos(3 * x)

    Q = rng.standard_normal(P) * 0.4
    x = nm.modes_to_beads(Q, T)
    f = nm.project_forces(-dV(x), T)
    h = 1e-6
    for n in range(P):
        e = np.zeros(P)
        e[n] = h
        up = V(nm.modes_to_beads(Q + e, T)).mean()
        um = V(nm.modes_to_beads(Q - e, T)).mean()
        assert abs(-(up - um) / (2 * h) - f[n]) < 1e-8


def test_cyclic_bead_permutation_invariance():
    """Sec. App. A: U_P and the spring energy are invariant under a cyclic shift of the beads."""
    rng = np.random.default_rng(2)
    P = 8
    T = nm.transfer_matrix(P)
    w = nm.mode_frequencies(P, KB * 300.0, HBAR)
    x = rng.standard_normal((4, 3, P))
    for s in range(1, P):
        xs = np.roll(x, s, axis=-1)
        Q, Qs = nm.beads_to_modes(x, T), nm.beads_to_modes(xs, T)
        np.testing.assert_allclose(np.sum(w ** 2 * Q ** 2), np.sum(w ** 2 * Qs ** 2), rtol=1e-12)
        np.testing.assert_allclose(np.sum(np.cos(xs)), np.sum(np.cos(x)), rtol=1e-12)
