"""BAOAB-RESPA multiple time stepping with ring-polymer contraction (Sec. III.A.2), FP64.

* Eq. (18): V = V_s + V_f.  Here V_f is the bonded part (two O-H bonds and the angle of
  every molecule) and V_s the nonbonded part (DSF Coulomb, LJ, the DSF self term).
* RESPA (the Trotter break-up of Sec. III.A.2): one outer step is
  B_s(n dt/2) [B_f(dt/2) A(dt/2) O(dt) A(dt/2) B_f(dt/2)]^n B_s(n dt/2),
  with dt the inner time step and n = n_alt.
* Ring-polymer contraction (Eq. (20)): V_s is evaluated on Pc <= P beads whose positions
  are the ring polymer's Fourier interpolant restricted to its Pc lowest-frequency normal
  modes, evaluated at Pc equally spaced imaginary times:
      xc_b = sum_{n in K} sqrt(P) T[b P/Pc, n] Q_n,   b = 0 .. Pc-1,
  with T the P-point transform of Eq. (4) and K the Pc lowest-frequency modes (the
  centroid, the cos and sin modes of frequencies 1 .. Pc/2 - 1, and the cos mode of
  frequency Pc/2, whose sin partner vanishes at the contracted beads).  The slow part of
  U_P is (1/Pc) sum_b V_s(xc_b), so its force on mode n is (1/Pc) sum_b C[b, n] F_s(xc_b).
  Pc = P recovers the full ring polymer; Pc = 1 evaluates V_s at the centroid.

Noise: inner step k of the trajectory draws the O-step normals of step counter k, the
same counter a plain BAOAB step k uses.
"""
from __future__ import annotations

import numpy as np

from . import rpmd
from .normal_modes import project_forces, transfer_matrix
from .units import ACC
from .water import ForceField, bonded, dsf_self_energy, nonbonded


def kept_modes(P: int, Pc: int) -> np.ndarray:
    """Indices n (of the P-point basis) of the Pc lowest-frequency modes kept by the contraction."""
    if Pc < 1 or P % Pc:
        raise ValueError("Pc must divide P")
    if Pc == P:
        return np.arange(P)
    keep = [0]
    for k in range(1, Pc // 2):
        keep += [k, P - k]
    if Pc >= 2:
        keep.append(Pc // 2)
    return np.array(sorted(keep))


def contraction_matrix(P: int, Pc: int) -> np.ndarray:
    """C[b, n] = sqrt(P) T[b P/Pc, n] for n in K, 0 otherwise ([Pc, P])."""
    T = transfer_matrix(P)
    C = np.zeros((Pc, P))
    K = kept_modes(P, Pc)
    for b in range(Pc):
        C[b, K] = np.sqrt(P) * T[b * (P // Pc), K]
    return C


def contract(Q: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Contracted bead positions [Pc, N, 3] from modes Q [N, 3, P]."""
    return np.einsum("bn,adn->bad", C, Q)


def project_contracted(Fs: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Mode forces [N, 3, P] of (1/Pc) sum_b V_s(xc_b): (1/Pc) sum_b C[b, n] F_s,b."""
    return np.einsum("bn,bad->adn", C, Fs) / C.shape[0]


def split_force_fns(types, mol, L: float, ff: ForceField):
    """fast_fn(xb) -> (V_f [B], F_f [B, N, 3]) bonded; slow_fn(xb) -> (V_s, F_s) nonbonded + self."""
    e_self = dsf_self_energy(ff.charges(types), ff)

    def fast_fn(xb):
        V = np.zeros(xb.shape[0])
        F = np.zeros_like(xb)
        for b in range(xb.shape[0]):
            V[b], F[b] = bonded(xb[b], L, ff)
        return V, F

    def slow_fn(xb):
        V = np.zeros(xb.shape[0])
        F = np.zeros_like(xb)
        for b in range(xb.shape[0]):
            E, F[b] = nonbonded(xb[b], types, mol, L, ff)
            V[b] = E + e_self
        return V, F
    return fast_fn, slow_fn


def forces(state: rpmd.State, prm: rpmd.Params, fast_fn, slow_fn, C: np.ndarray):
    """(f_f, f_s) mode forces: f_f from the bonded forces on all P beads (Eqs. (10)-(11)),
    f_s from the nonbonded forces on the contracted beads."""
    xb = rpmd.beads(state, prm.P)
    _, Ff = fast_fn(xb)
    f_f = project_forces(np.transpose(Ff, (1, 2, 0)), transfer_matrix(prm.P))
    _, Fs = slow_fn(contract(state.Q, C))
    return f_f, project_contracted(Fs, C)


def respa_step(state: rpmd.State, prm: rpmd.Params, masses: np.ndarray, fast_fn, slow_fn, n_alt: int,
               C: np.ndarray) -> None:
    """One outer step: B_s(n dt/2), n inner B_f A O A B_f steps of dt = prm.dt, B_s(n dt/2)."""
    if "f_f" not in state.extra:
        state.extra["f_f"], state.extra["f_s"] = forces(state, prm, fast_fn, slow_fn, C)
    dt = prm.dt
    state.Pm = state.Pm + 0.5 * n_alt * dt * ACC * state.extra["f_s"]
    for _ in range(n_alt):
        state.Pm = state.Pm + 0.5 * dt * ACC * state.extra["f_f"]
        rpmd.free_flow(state, prm, masses, 0.5 * dt)
        rpmd.ou(state, prm, masses, dt)
        rpmd.free_flow(state, prm, masses, 0.5 * dt)
        xb = rpmd.beads(state, prm.P)
        _, Ff = fast_fn(xb)
        state.extra["f_f"] = project_forces(np.transpose(Ff, (1, 2, 0)), transfer_matrix(prm.P))
        state.Pm = state.Pm + 0.5 * dt * ACC * state.extra["f_f"]
        state.step += 1
    _, Fs = slow_fn(contract(state.Q, C))
    state.extra["f_s"] = project_contracted(Fs, C)
    state.Pm = state.Pm + 0.5 * n_alt * dt * ACC * state.extra["f_s"]


def contracted_potential(Q: np.ndarray, slow_fn, C: np.ndarray) -> float:
    """(1/Pc) sum_b V_s(xc_b): the slow part of U_P under contraction (Eq. (20))."""
    V, _ = slow_fn(contract(Q, C))
    return float(np.mean(V))

