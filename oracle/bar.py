"""Path-integral Bennett acceptance ratio (Sec. V, Perspective 2, Eqs. (27)-(28); Appendix A), FP64.

Two thermodynamic states A and B of the same system (here: two force-field parameter
sets).  From configurations sampled in each state, dU = U_{B,P} - U_{A,P} with U_P the
bead-averaged potential of Eq. (3).  The estimator of Dlt F_AB = beta^-1 ln(Z_A / Z_B)
(= F_B - F_A) is the self-consistent solution of

    Dlt F = C + beta^-1 ln( <f(-dU + C)>_B / <f(dU - C)>_A ),     f(x) = 1 / (1 + exp(beta x)),
    C     = Dlt F + beta^-1 ln(n_B / n_A),

solved here by iterating the two equations in that order from C = beta^-1 ln(n_B/n_A)
until C changes by less than tol.  The single-bead estimator of the appendix is the same
expression with dU taken on one bead, V_B(x_0) - V_A(x_0).

Exact references for the pins: for harmonic states U = 1/2 m w^2 x^2 of one degree of
freedom, the P-bead ring polymer has independent Gaussian normal modes (variance
kT / (m (w^2 + w_n^2)) for mode n), so Dlt F_P = (kT/2) sum_n ln((w_B^2 + w_n^2) / (w_A^2 + w_n^2)).
"""
from __future__ import annotations

import numpy as np
from scipy.special import expit


def fermi(x, beta: float):
    """f_beta(x) = 1 / (1 + exp(beta x)), evaluated without overflow."""
    return expit(-beta * np.asarray(x, dtype=float))


def pibar(dU_A: np.ndarray, dU_B: np.ndarray, beta: float, tol: float = 1e-12, max_iter: int = 10000):
    """(Dlt F_AB, C, iterations) from dU = U_B - U_A sampled in state A (dU_A) and in B (dU_B)."""
    dU_A = np.asarray(dU_A, dtype=float)
    dU_B = np.asarray(dU_B, dtype=float)
    nA, nB = len(dU_A), len(dU_B)
    shift = np.log(nB / nA) / beta
    C = shift
    for it in range(1, max_iter + 1):
        num = np.mean(fermi(-dU_B + C, beta))
        den = np.mean(fermi(dU_A - C, beta))
        dF = C + np.log(num / den) / beta
        C_new = dF + shift
        if abs(C_new - C) < tol:
            return dF, C_new, it
        C = C_new
    raise RuntimeError("BAR iteration did not converge")


def harmonic_ring_polymer_free_energy_difference(P: int, kT: float, hbar: float, wA: float, wB: float) -> float:
    """Exact Dlt F_P = F_B - F_A of one harmonic degree of freedom as a P-bead ring polymer."""
    wn = 2.0 * P * kT / hbar * np.sin(np.pi * np.arange(P) / P)
    return 0.5 * kT * float(np.sum(np.log((wB ** 2 + wn ** 2) / (wA ** 2 + wn ** 2))))
