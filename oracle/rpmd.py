"""Thermostatted RPMD in normal modes: BAOAB with exact free ring-polymer A (Sec. III.A.1).

* Eq. (9): dQ_n/dt = P_n/m, dP_n/dt = f_n - omega_n^2 m Q_n, the physical mass for every mode.
* Eq. (16): a Langevin thermostat on every mode with gamma_n = max(gamma_0, omega_n)
  for n > 0 (critically damped, TRPMD) and gamma_0 on the centroid.
* Eq. (17): one step is B(dt/2) A(dt/2) O(dt) A(dt/2) B(dt/2); A is the exact harmonic
  (n > 0) or free (n = 0) flow, O the exact Ornstein-Uhlenbeck update, B the force kick.
* Eq. (7): momenta are Gaussian with variance m kT for every mode.

Units: Q in A, momenta in amu*A/ps, forces in kcal/mol/A, energies in kcal/mol;
``ACC`` converts kcal/mol to amu*A^2/ps^2.  State arrays are [N, 3, P] (atom,
dimension, mode).  Reading: the initial fluctuation modes are drawn from the
free ring-polymer Gaussian, Q_n ~ N(0, kT/(m omega_n^2)), with Q_0 the input
positions.  O-step normals use Philox counter (element, step, tag 3) with
element = (3*atom + dim)*P + n.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import philox
from .normal_modes import beads_to_modes, mode_frequencies, modes_to_beads, project_forces, transfer_matrix
from .units import ACC, HBAR, KB


@dataclass
class Params:
    P: int
    temperature: float
    dt: float              # ps
    gamma0: float          # ps^-1
    seed: int
    hbar: float = HBAR
    integrator: str = "baoab"   # "baoab" (exact A) or "bcocb" (Cayley A, Sec. III.A.1)
    thermostat: str = "pile"    # "pile" (Eq. (16)) or "nve": no O step, the flow of Eq. (9) alone

    @property
    def kT(self) -> float:
        return KB * self.temperature

    def omegas(self) -> np.ndarray:
        return mode_frequencies(self.P, self.kT, self.hbar)

    def gammas(self) -> np.ndarray:
        """Eq. (16): gamma_0 on the centroid, max(gamma_0, omega_n) on the other modes."""
        w = self.omegas()
        g = np.maximum(self.gamma0, w)
        g[0] = self.gamma0
        return g


@dataclass
class State:
    Q: np.ndarray          # [N, 3, P]
    Pm: np.ndarray         # [N, 3, P]
    f: np.ndarray | None = None   # projected mode forces [N, 3, P]
    step: int = 0
    V: np.ndarray | None = None   # bead energies of the last force call [P]
    F: np.ndarray | None = None   # bead forces [P, N, 3]
    extra: dict = field(default_factory=dict)


def element_index(N: int, P: int) -> np.ndarray:
    """Philox element index (3*atom + dim)*P + n laid out as [N, 3, P]."""
    return np.arange(N * 3 * P, dtype=np.uint64).reshape(N, 3, P)


def init_state(x0: np.ndarray, masses: np.ndarray, prm: Params) -> State:
    N, P = x0.shape[0], prm.P
    kT = prm.kT * ACC
    w = prm.omegas()
    e = element_index(N, P)
    m = masses[:, None, None]
    zq = philox.normals(prm.seed, e, 0, philox.TAG_INIT_Q)
    zp = philox.normals(prm.seed, e, 0, philox.TAG_INIT_P)
    Q = np.zeros((N, 3, P))
    Q[:, :, 0] = x0
    if P > 1:
        Q[:, :, 1:] = np.sqrt(kT / (m * w[None, None, 1:] ** 2)) * zq[:, :, 1:]
    Pm = np.sqrt(m * kT) * zp
    return State(Q=Q, Pm=Pm)


def beads(state: State, P: int) -> np.ndarray:
    """Bead positions [P, N, 3] from Eq. (4)."""
    T = transfer_matrix(P)
    x = modes_to_beads(state.Q, T)            # [N, 3, P]
    return np.transpose(x, (2, 0, 1)).copy()


def evaluate_forces(state: State, prm: Params, force_fn) -> None:
    """Bead forces at the current modes and their projection (Eqs. (10)-(11))."""
    xb = beads(state, prm.P)
    V, F = force_fn(xb)                        # V [P], F [P, N, 3]
    state.V, state.F = np.asarray(V, dtype=float), F
    state.f = project_forces(np.transpose(F, (1, 2, 0)), transfer_matrix(prm.P))


def kick(state: State, tau: float) -> None:
    """B: P_n += tau * f_n."""
    state.Pm = state.Pm + tau * ACC * state.f


def free_flow(state: State, prm: Params, masses: np.ndarray, tau: float) -> None:
    """A: exact flow of Eq. (9) without f_n for a time tau.

    n = 0 is a free drift.  For n > 0 the flow is the rotation by theta = omega_n tau in
    (m omega_n Q_n, P_n); it is applied as three shears,
    Q += tan(theta/2) P/(m w); P -= sin(theta) m w Q; Q += tan(theta/2) P/(m w),
    whose product equals the rotation by the half-angle identities.  Each shear has
    determinant exactly one for any rounded coefficient, so rounding does not make the
    mode energy drift step after step."""
    m = masses[:, None]
    w = prm.omegas()
    Q, Pm = state.Q.copy(), state.Pm.copy()
    Q[:, :, 0] = state.Q[:, :, 0] + state.Pm[:, :, 0] * tau / m
    if prm.integrator == "bcocb":
        for n in range(1, prm.P):
            Q[:, :, n], Pm[:, :, n] = cayley_flow(state.Q[:, :, n], state.Pm[:, :, n], m, w[n], tau)
        state.Q, state.Pm = Q, Pm
        return
    for n in range(1, prm.P):
        th = w[n] * tau
        a = np.tan(0.5 * th) / (m * w[n])
        b = np.sin(th) * m * w[n]
        q = state.Q[:, :, n] + a * state.Pm[:, :, n]
        p = state.Pm[:, :, n] - b * q
        Q[:, :, n] = q + a * p
        Pm[:, :, n] = p
    state.Q, state.Pm = Q, Pm


def cayley_flow(q, p, m, w: float, h: float):
    """C: the Cayley transform of the free ring-polymer flow of one mode over h (the BCOCB
    scheme of Sec. III.A.1, after Korol et al.): with A = [[0, 1/m], [-m w^2, 0]],
    cay(hA) = (I - hA/2)^{-1} (I + hA/2), written out:
        q' = ((1 - u) q + (h/m) p) / (1 + u),  p' = (-h m w^2 q + (1 - u) p) / (1 + u),  u = (h w/2)^2."""
    u = (0.5 * h * w) ** 2
    d = 1.0 + u
    return ((1.0 - u) * q + (h / m) * p) / d, (-h * m * w * w * q + (1.0 - u) * p) / d


def ou(state: State, prm: Params, masses: np.ndarray, dt: float, noise: np.ndarray | None = None) -> None:
    """O: exact Ornstein-Uhlenbeck update with friction gamma_n (Eq. (16)) over dt.  With the
    "nve" thermostat there is no friction and no noise, so O is the identity."""
    if prm.thermostat == "nve":
        return
    N, P = state.Q.shape[0], prm.P
    c1 = np.exp(-prm.gammas() * dt)                               # [P]
    if noise is None:
        noise = philox.normals(prm.seed, element_index(N, P), state.step, philox.TAG_OSTEP)
    amp = np.sqrt((1.0 - c1[None, None, :] ** 2) * masses[:, None, None] * prm.kT * ACC)
    state.Pm = c1[None, None, :] * state.Pm + amp * noise


def step(state: State, prm: Params, masses: np.ndarray, force_fn) -> None:
    """One BAOAB step (Eq. (17)); forces are evaluated once, at the end."""
    if state.f is None:
        evaluate_forces(state, prm, force_fn)
    dt = prm.dt
    kick(state, 0.5 * dt)
    free_flow(state, prm, masses, 0.5 * dt)
    ou(state, prm, masses, dt)
    free_flow(state, prm, masses, 0.5 * dt)
    evaluate_forces(state, prm, force_fn)
    kick(state, 0.5 * dt)
    state.step += 1


# ---------------------------------------------------------------- estimators

def potential_estimator(state: State) -> float:
    """Eq. (3): U_P = (1/P) sum_i V(x_i)."""
    return float(np.mean(state.V))


def spring_energy(state: State, prm: Params, masses: np.ndarray) -> float:
    """sum_{n>0} 1/2 m omega_n^2 Q_n^2 (the ring-polymer term of Eq. (1)), kcal/mol."""
    w = prm.omegas()
    return float(np.sum(0.5 * masses[:, None, None] * w[None, None, :] ** 2 * state.Q ** 2)) / ACC


def kinetic_energy(state: State, masses: np.ndarray) -> float:
    """sum_n P_n^2 / (2m) (Eq. (7)), kcal/mol."""
    return float(np.sum(state.Pm ** 2 / (2.0 * masses[:, None, None]))) / ACC


def centroid_virial_kinetic(state: State, prm: Params) -> float:
    """3N kT/2 - (1/2P) sum_i (x_i - Q_0) . F(x_i): the centroid-virial estimator built
    from Eq. (6) applied to the kinetic energy."""
    N, P = state.Q.shape[0], prm.P
    xb = beads(state, P)                                      # [P, N, 3]
    dev = xb - state.Q[None, :, :, 0]
    return 1.5 * N * prm.kT - float(np.sum(dev * state.F)) / (2.0 * P)


def harmonic_forces(omega0: float, masses: np.ndarray):
    """force_fn for independent 1D-per-dof oscillators V = 1/2 m omega0^2 x^2 (kcal/mol)."""
    def fn(xb):
        k = masses[None, :, None] * omega0 ** 2 / ACC
        V = np.sum(0.5 * k * xb ** 2, axis=(1, 2))
        return V, -k * xb
    return fn


def modes_from_beads(xb: np.ndarray, P: int) -> np.ndarray:
    """[P, N, 3] bead positions -> [N, 3, P] modes (inverse of Eq. (4))."""
    return beads_to_modes(np.transpose(xb, (1, 2, 0)), transfer_matrix(P))
