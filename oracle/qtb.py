"""Adaptive quantum thermal bath (Secs. II.B and III.B), single bead.

* Eq. (12): dp/dt = -grad V - gamma_0 p + F(t).
* Eqs. (13)-(14): C_FF(omega) = 2 m gamma(omega) Theta(omega, beta),
  Theta = (hbar omega / 2) / tanh(beta hbar omega / 2).
* Sec. III.B.1: the noise is generated per segment of N_seg steps by convolving
  white noise with the Fourier transform of sqrt(C_FF); 3 N_seg white numbers per
  degree of freedom keep the memory consistent between segments.
* Eqs. (21)-(22): Delta_FDT,i(omega) = m_i C_vv(omega) gamma_i(omega) - Re C_vF(omega)
  with C_vv ~ |v~|^2 and C_vF ~ v~ F~*, the DFTs of the last segment.
* Sec. III.B.2: gamma is shared by all dofs of one atom type; Delta is averaged
  over them; SIMPLE (Eq. (23)) gamma <- gamma - A_gamma Delta_bar; RATIO
  (Eqs. (24)-(26)) gamma <- Re<C_vF>_tau / (m <C_vv>_tau) with exponential running
  averages; finally gamma <- max(gamma_min, gamma).

Readings where the paper is silent (it defers the discretisation to other work):
* frequency grid of N_f = 2 N_seg points, omega_j = 2 pi min(j, N_f - j) / (N_f dt);
  gamma_z is stored on the N_seg + 1 bins j = 0..N_seg;
* noise power S_z(omega_j) = Theta(omega_j) gamma_z(omega_j) / gamma_0 for
  omega_j <= omega_cut, 0 above (hard cutoff), Theta(0) = kT; no extra
  finite-dt / finite-gamma corrections;
* filter h = IDFT_{N_f}(sqrt(S)) (real, even), u_n = sum_{l=-N_seg}^{N_seg-1} h_l xi_{n-l};
  the O step is p <- c1 p + sqrt((1 - c1^2) m) u_n with c1 = exp(-gamma_0 dt), which
  is classical BAOAB when S = kT at every frequency;
* v_n = (p_before_O + p_after_O) / (2m), F_n = sqrt((1 - c1^2) m) u_n / dt;
* C_vv = (dt / N_seg) |v~|^2, C_vF = (dt / N_seg) v~ F~*, DFT of the segment zero-padded to N_f;
* Delta is converted to kcal/mol before SIMPLE, so A_gamma is in ps^-1 per kcal/mol;
* white noise xi for dof i at global index g (g >= -N_seg) is Box-Muller output
  (g + N_seg) & 1 of Philox counter (i, (g + N_seg) >> 1, tag 4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import philox
from .units import ACC, HBAR, KB


@dataclass
class QTBParams:
    n_seg: int
    dt: float                 # ps
    gamma0: float             # ps^-1
    temperature: float
    omega_cut: float          # rad/ps (np.inf for none)
    a_gamma: float = 10.0     # ps^-1 per kcal/mol
    gamma_min_frac: float = 0.01
    seed: int = 1234
    hbar: float = HBAR
    tau_ratio: float = 1.0    # ps, RATIO running-average time

    @property
    def kT(self) -> float:
        return KB * self.temperature

    @property
    def n_f(self) -> int:
        return 2 * self.n_seg


def theta(omega: np.ndarray, kT: float, hbar: float) -> np.ndarray:
    """Eq. (14), with its omega -> 0 limit kT."""
    omega = np.asarray(omega, dtype=float)
    out = np.full(omega.shape, kT)
    nz = omega > 0
    x = hbar * omega[nz]
    out[nz] = 0.5 * x / np.tanh(0.5 * x / kT)
    return out


def omega_bins(prm: QTBParams) -> np.ndarray:
    """omega of bins j = 0..N_seg."""
    j = np.arange(prm.n_seg + 1)
    return 2.0 * np.pi * j / (prm.n_f * prm.dt)


def noise_power(gamma_z: np.ndarray, prm: QTBParams) -> np.ndarray:
    """S_z(omega_j) on the N_seg + 1 bins (noise power in kcal/mol, per the reading above)."""
    w = omega_bins(prm)
    S = theta(w, prm.kT, prm.hbar) * gamma_z / prm.gamma0
    return np.where(w <= prm.omega_cut, S, 0.0)


def filter_taps(S_bins: np.ndarray, prm: QTBParams) -> np.ndarray:
    """h_l for l in [-N_seg, N_seg), returned as an array indexed by l + N_seg."""
    n_f = prm.n_f
    j = np.arange(n_f)
    full = S_bins[np.minimum(j, n_f - j)]
    h = np.fft.ifft(np.sqrt(full)).real            # (1/N_f) sum_j sqrt(S_j) e^{+2 pi i j l / N_f}
    l = np.arange(-prm.n_seg, prm.n_seg)
    return h[l % n_f]


def white(prm: QTBParams, dofs: np.ndarray, g: np.ndarray) -> np.ndarray:
    """xi[g, dof] for global white-noise indices g >= -N_seg."""
    gs = np.asarray(g, dtype=np.int64)[:, None] + prm.n_seg
    return philox.normals(prm.seed, np.asarray(dofs, dtype=np.uint64)[None, :], (gs >> 1).astype(np.uint64),
                          philox.TAG_QTB_WHITE, which=(gs & 1))


def colored_segment_direct(k: int, taps: np.ndarray, dofs: np.ndarray, prm: QTBParams) -> np.ndarray:
    """u[m, dof] for steps n = k N_seg + m by the time-domain sum (tiny cases).

    taps: [n_dof, 2 N_seg] filter per dof (index l + N_seg)."""
    N = prm.n_seg
    g = np.arange(k * N - N, k * N + 2 * N)
    xi = white(prm, dofs, g)                                # [3N, n_dof]
    u = np.zeros((N, len(dofs)))
    for m in range(N):
        n = k * N + m
        for li, l in enumerate(range(-N, N)):
            u[m] += taps[:, li] * xi[n - l - (k * N - N)]
    return u


def colored_segment_fft(k: int, taps: np.ndarray, dofs: np.ndarray, prm: QTBParams) -> np.ndarray:
    """Same as ``colored_segment_direct`` through a 4 N_seg-point FFT (linear convolution)."""
    N = prm.n_seg
    L4 = 4 * N
    g = np.arange(k * N - N, k * N + 2 * N)
    xi = white(prm, dofs, g)                                # [3N, n_dof]
    x = np.zeros((L4, len(dofs)))
    x[:3 * N] = xi
    hc = np.zeros((L4, len(dofs)))
    l = np.arange(-N, N)
    hc[l % L4] = taps.T
    y = np.fft.ifft(np.fft.fft(x, axis=0) * np.fft.fft(hc, axis=0), axis=0).real
    return y[N:2 * N]


def spectra(v: np.ndarray, F: np.ndarray, prm: QTBParams):
    """C_vv and C_vF on bins 0..N_seg from one segment of v[m, dof], F[m, dof] (Eq. (22))."""
    vt = np.fft.rfft(v, n=prm.n_f, axis=0)
    Ft = np.fft.rfft(F, n=prm.n_f, axis=0)
    norm = prm.dt / prm.n_seg
    return norm * np.abs(vt) ** 2, norm * vt * np.conj(Ft)


def delta_fdt(Cvv, CvF, m_dof, gamma_dof):
    """Eq. (21) in kcal/mol: (m C_vv gamma - Re C_vF) / ACC, per bin and dof."""
    return (m_dof[None, :] * Cvv * gamma_dof - CvF.real) / ACC


def type_mean(x: np.ndarray, dof_type: np.ndarray, n_types: int) -> np.ndarray:
    """Average over the dofs of each type (Sec. III.B.2) -> [n_types, bins]."""
    out = np.zeros((n_types, x.shape[0]))
    for z in range(n_types):
        out[z] = x[:, dof_type == z].mean(axis=1)
    return out


def adapt_simple(gamma: np.ndarray, delta_bar: np.ndarray, prm: QTBParams) -> np.ndarray:
    """Eq. (23) followed by the lower bound gamma_min = gamma_min_frac * gamma_0."""
    return np.maximum(prm.gamma_min_frac * prm.gamma0, gamma - prm.a_gamma * delta_bar)


def adapt_ratio(avg_vv: np.ndarray, avg_vf: np.ndarray, Cvv_bar: np.ndarray, CvF_bar: np.ndarray,
                m_type: np.ndarray, prm: QTBParams, first: bool):
    """Eqs. (24)-(26): exponential running averages of the type-mean spectra, then the ratio."""
    w = math.exp(-prm.n_seg * prm.dt / prm.tau_ratio)
    if first:
        avg_vv, avg_vf = Cvv_bar.copy(), CvF_bar.real.copy()
    else:
        avg_vv = avg_vv * w + Cvv_bar * (1.0 - w)
        avg_vf = avg_vf * w + CvF_bar.real * (1.0 - w)
    gamma = avg_vf / (m_type[:, None] * avg_vv)
    return np.maximum(prm.gamma_min_frac * prm.gamma0, gamma), avg_vv, avg_vf


class QTB:
    """adQTB thermostat state for ``n_dof`` degrees of freedom (dof = 3*atom + dim)."""

    def __init__(self, prm: QTBParams, m_dof: np.ndarray, dof_type: np.ndarray, n_types: int,
                 adapt: str = "simple", direct: bool = False):
        self.prm = prm
        self.m = np.asarray(m_dof, dtype=float)
        self.dof_type = np.asarray(dof_type)
        self.n_types = n_types
        self.gamma = np.full((n_types, prm.n_seg + 1), prm.gamma0)
        self.adapt = adapt
        self.direct = direct
        self.k = -1
        self.u = None
        self.v = np.zeros((prm.n_seg, len(self.m)))
        self.F = np.zeros((prm.n_seg, len(self.m)))
        self.avg_vv = None
        self.avg_vf = None
        self.last_delta_bar = None
        self.c1 = math.exp(-prm.gamma0 * prm.dt)
        self.amp = np.sqrt((1.0 - self.c1 ** 2) * self.m * ACC)

    def taps(self) -> np.ndarray:
        h = np.stack([filter_taps(noise_power(self.gamma[z], self.prm), self.prm) for z in range(self.n_types)])
        return h[self.dof_type]

    def generate(self, k: int) -> None:
        dofs = np.arange(len(self.m))
        gen = colored_segment_direct if self.direct else colored_segment_fft
        self.u = gen(k, self.taps(), dofs, self.prm)
        self.k = k

    def end_segment(self) -> None:
        Cvv, CvF = spectra(self.v, self.F, self.prm)
        if self.adapt == "ratio":
            Cvv_bar = type_mean(Cvv, self.dof_type, self.n_types)
            CvF_bar = type_mean(CvF.real, self.dof_type, self.n_types)
            m_type = np.array([self.m[self.dof_type == z][0] for z in range(self.n_types)])
            self.gamma, self.avg_vv, self.avg_vf = adapt_ratio(self.avg_vv, self.avg_vf, Cvv_bar, CvF_bar,
                                                              m_type, self.prm, self.avg_vv is None)
        else:
            gam_dof = self.gamma[self.dof_type].T                 # [bins, dof]
            d = delta_fdt(Cvv, CvF, self.m, gam_dof)
            self.last_delta_bar = type_mean(d, self.dof_type, self.n_types)
            if self.adapt == "simple":
                self.gamma = adapt_simple(self.gamma, self.last_delta_bar, self.prm)

    def ostep(self, p: np.ndarray, step: int) -> np.ndarray:
        """O step of global step ``step`` on flat momenta p[dof]; records v and F."""
        N = self.prm.n_seg
        k, m = divmod(step, N)
        if self.u is None or self.k != k:
            self.generate(k)
        noise = self.amp * self.u[m]
        p_new = self.c1 * p + noise
        self.v[m] = (p + p_new) / (2.0 * self.m)
        self.F[m] = noise / self.prm.dt
        if m == N - 1:
            self.end_segment()
            self.generate(k + 1)
        return p_new


def qtb_step(state, masses: np.ndarray, bath: QTB, force_fn) -> None:
    """One classical BAOAB step (P = 1) with the adQTB O step (Sec. III.B)."""
    from .rpmd import State  # noqa: F401  (state is an rpmd.State with P = 1)
    dt = bath.prm.dt
    m = masses[:, None]
    if state.f is None:
        V, F = force_fn(state.Q[None, :, :, 0])
        state.V, state.F, state.f = V, F, F[0][:, :, None]
    state.Pm = state.Pm + 0.5 * dt * ACC * state.f
    state.Q[:, :, 0] += state.Pm[:, :, 0] * (0.5 * dt) / m
    p = bath.ostep(state.Pm[:, :, 0].reshape(-1), state.step)
    state.Pm[:, :, 0] = p.reshape(-1, 3)
    state.Q[:, :, 0] += state.Pm[:, :, 0] * (0.5 * dt) / m
    V, F = force_fn(state.Q[None, :, :, 0])
    state.V, state.F, state.f = V, F, F[0][:, :, None]
    state.Pm = state.Pm + 0.5 * dt * ACC * state.f
    state.step += 1
