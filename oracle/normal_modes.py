"""Free ring-polymer normal modes (Sec. II.A).

* Eq. (2): Omega_P^2 = (P/(hbar*beta))^2 * circ(2, -1, 0, ..., 0, -1); the mode
  frequencies omega_n are the square roots of its eigenvalues.
* Eq. (4): x_i = Q_0 + sqrt(P) sum_{n>=1} T_in Q_n, T orthonormal with the
  eigenvectors of Eq. (2) as columns.
* Eqs. (10)-(11): f_0 = -(1/P) sum_i grad V(x_i), f_n = -(1/sqrt P) sum_i T_in grad V(x_i).

Reading: eigenvectors of the degenerate pairs (n, P-n) are not unique, so T is
fixed to the real DFT basis (cosines for 1 <= n < P/2, the alternating vector
for n = P/2, sines for P/2 < n < P).
"""
from __future__ import annotations

import numpy as np


def transfer_matrix(P: int) -> np.ndarray:
    """T[i, n] (bead i, mode n), real orthonormal DFT basis."""
    T = np.empty((P, P))
    i = np.arange(P)
    for n in range(P):
        phase = 2.0 * np.pi * ((i * n) % P) / P      # argument reduced exactly in integers
        if n == 0:
            T[:, n] = 1.0 / np.sqrt(P)
        elif 2 * n < P:
            T[:, n] = np.sqrt(2.0 / P) * np.cos(phase)
        elif 2 * n == P:
            T[:, n] = (-1.0) ** i / np.sqrt(P)
        else:
            T[:, n] = np.sqrt(2.0 / P) * np.sin(phase)
    return T


def mode_frequencies(P: int, kT: float, hbar: float) -> np.ndarray:
    """omega_n = 2 (P/(beta*hbar)) sin(pi n / P), the square roots of the eigenvalues of Eq. (2)."""
    n = np.arange(P)
    return 2.0 * P * kT / hbar * np.sin(np.pi * n / P)


def modes_to_beads(Q: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Eq. (4).  Q[..., n] -> x[..., i] = sqrt(P) * sum_n T[i, n] Q[..., n]."""
    P = T.shape[0]
    return np.sqrt(P) * np.einsum("in,...n->...i", T, Q)


def beads_to_modes(x: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Inverse of Eq. (4): Q[..., n] = (1/sqrt P) sum_i T[i, n] x[..., i]."""
    P = T.shape[0]
    return np.einsum("in,...i->...n", T, x) / np.sqrt(P)


def project_forces(F: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Eqs. (10)-(11).  F[..., i] = -grad V(x_i) -> f[..., n] = (1/sqrt P) sum_i T[i, n] F[..., i].

    For n = 0, T[i, 0] = 1/sqrt(P) gives f_0 = (1/P) sum_i F_i as in Eq. (10).
    """
    P = T.shape[0]
    return np.einsum("in,...i->...n", T, F) / np.sqrt(P)
