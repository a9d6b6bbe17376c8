"""Derivatives of the potential and of short trajectories with respect to the
force-field parameters theta = (eps, sigma, q_O, k_b, k_theta), FP64.

The paper has no gradient machinery; what is differentiated is its own
quantities:

* the bead-averaged potential U_P = (1/P) sum_b V(x_b) of Eq. (3), with respect
  to the bead positions (dU_P/dx_b = -F_b / P) and to theta (analytic: every
  term of V is written out and differentiated by hand below);
* the time average J = (1/K) sum_{k=1..K} a(state_k) of an observable a along a
  K-step BAOAB trajectory (Eq. (17), the thermostat noise held fixed, i.e. the
  same Philox counters), computed by central finite differences of whole
  oracle trajectories (dJ/dtheta_k = (J(theta_k(1+h)) - J(theta_k(1-h))) /
  (2 h theta_k), h = 1e-4).

Observables: 0 = the potential energy at the centroid, V(Q_0); 1 = the mean O-H
bond length over all beads and both bonds of every molecule.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.special import erfc

from . import rpmd
from .units import ACC, COULOMB
from .water import ForceField, make_force_fn, min_image, potential

PARAM_NAMES = ("eps", "sigma", "q_O", "k_b", "k_theta")
OBS_CENTROID_ENERGY = 0
OBS_MEAN_OH = 1


def param_vector(ff: ForceField) -> np.ndarray:
    return np.array([getattr(ff, n) for n in PARAM_NAMES], dtype=float)


def with_params(ff: ForceField, theta) -> ForceField:
    return dataclasses.replace(ff, **{n: float(v) for n, v in zip(PARAM_NAMES, theta)})


def param_gradient(x: np.ndarray, types: np.ndarray, mol: np.ndarray, L: float, ff: ForceField) -> np.ndarray:
    """dV/dtheta for one configuration x [N, 3] (V including the DSF self term).

    LJ (O-O, r < rc):  dV/deps = 4 (s^12 - s^6) - 4 (s_c^12 - s_c^6), s = sigma/r, s_c = sigma/rc;
                       dV/dsigma = (4 eps / sigma) [(12 s^12 - 6 s^6) - (12 s_c^12 - 6 s_c^6)].
    DSF Coulomb: q_i = q_O c_i with c_O = 1, c_H = -1/2, so each pair term is q_O^2 times
    k_e c_i c_j [erfc(a r)/r - erfc(a rc)/rc + S_c (r - rc)] and its q_O derivative is 2 q_O times
    that bracket; the self term -(erfc(a rc)/(2 rc) + a/sqrt(pi)) k_e q_O^2 sum_i c_i^2 likewise.
    Bonds and angle: dV/dk_b = sum 1/2 (r - r0)^2, dV/dk_theta = sum 1/2 (theta - theta0)^2.
    """
    N = x.shape[0]
    c = np.where(types == 0, 1.0, -0.5)
    a, rc = ff.alpha, ff.rc
    sc = erfc(a * rc) / rc ** 2 + 2.0 * a / math.sqrt(math.pi) * math.exp(-(a * rc) ** 2) / rc
    g = np.zeros(5)
    for i in range(N - 1):
        d = min_image(x[i + 1:] - x[i], L)
        r = np.sqrt(np.einsum("jk,jk->j", d, d))
        j = np.arange(i + 1, N)
        m = (mol[j] != mol[i]) & (r < rc)
        rr, jj = r[m], j[m]
        bracket = erfc(a * rr) / rr - erfc(a * rc) / rc + sc * (rr - rc)
        g[2] += float(np.sum(2.0 * ff.q_O * COULOMB * c[i] * c[jj] * bracket))
        if types[i] == 0:
            ro = rr[types[jj] == 0]
            s6, sc6 = (ff.sigma / ro) ** 6, (ff.sigma / rc) ** 6
            g[0] += float(np.sum(4.0 * (s6 * s6 - s6) - 4.0 * (sc6 * sc6 - sc6)))
            g[1] += float(np.sum(4.0 * ff.eps / ff.sigma * ((12.0 * s6 * s6 - 6.0 * s6)
                                                            - (12.0 * sc6 * sc6 - 6.0 * sc6))))
    g[2] += -(erfc(a * rc) / (2.0 * rc) + a / math.sqrt(math.pi)) * COULOMB * 2.0 * ff.q_O * float(np.sum(c * c))
    xm = x.reshape(-1, 3, 3)
    d1 = min_image(xm[:, 1] - xm[:, 0], L)
    d2 = min_image(xm[:, 2] - xm[:, 0], L)
    r1 = np.linalg.norm(d1, axis=1)
    r2 = np.linalg.norm(d2, axis=1)
    th = np.arccos(np.einsum("ij,ij->i", d1, d2) / (r1 * r2))
    g[3] = 0.5 * float(np.sum((r1 - ff.r0) ** 2 + (r2 - ff.r0) ** 2))
    g[4] = 0.5 * float(np.sum((th - ff.theta0) ** 2))
    return g


def bead_energy_gradients(xb: np.ndarray, types: np.ndarray, mol: np.ndarray, L: float, ff: ForceField):
    """U_P = (1/P) sum_b V(x_b) (Eq. (3)), dU_P/dx [P, N, 3] = -F_b / P and dU_P/dtheta [5]."""
    P = xb.shape[0]
    U, dx, dth = 0.0, np.zeros_like(xb), np.zeros(5)
    for b in range(P):
        V, F = potential(xb[b], types, mol, L, ff)
        U += V / P
        dx[b] = -F / P
        dth += param_gradient(xb[b], types, mol, L, ff) / P
    return U, dx, dth


def mean_oh_length(xb: np.ndarray, L: float) -> float:
    """Mean |x_H - x_O| (minimum image) over beads [P, N, 3] and the two bonds of every molecule."""
    xm = xb.reshape(xb.shape[0], -1, 3, 3)
    d1 = min_image(xm[:, :, 1] - xm[:, :, 0], L)
    d2 = min_image(xm[:, :, 2] - xm[:, :, 0], L)
    return 0.5 * float(np.mean(np.linalg.norm(d1, axis=-1) + np.linalg.norm(d2, axis=-1)))


def observable(state: rpmd.State, P: int, types, mol, L: float, ff: ForceField, which: int) -> float:
    if which == OBS_CENTROID_ENERGY:
        return potential(state.Q[:, :, 0], types, mol, L, ff)[0]
    if which == OBS_MEAN_OH:
        return mean_oh_length(rpmd.beads(state, P), L)
    raise ValueError("observable must be 0 (centroid energy) or 1 (mean O-H length)")


def segment_objective(state0: rpmd.State, prm: rpmd.Params, types, mol, L: float, ff: ForceField, K: int,
                      which: int) -> float:
    """J = (1/K) sum_{k=1..K} a(state_k) along K BAOAB steps (Eq. (17)) from state0 (not modified)."""
    masses = ff.masses(types)
    st = rpmd.State(Q=state0.Q.copy(), Pm=state0.Pm.copy(), step=state0.step)
    fn = make_force_fn(types, mol, L, ff)
    J = 0.0
    for _ in range(K):
        rpmd.step(st, prm, masses, fn)
        J += observable(st, prm.P, types, mol, L, ff, which)
    return J / K


def segment_gradient_fd(state0: rpmd.State, prm: rpmd.Params, types, mol, L: float, ff: ForceField, K: int,
                        which: int, h: float = 1e-4) -> np.ndarray:
    """Central finite differences of segment_objective in each theta_k with relative step h."""
    th = param_vector(ff)
    g = np.zeros(5)
    for k in range(5):
        tp, tm = th.copy(), th.copy()
        tp[k] = th[k] * (1.0 + h)
        tm[k] = th[k] * (1.0 - h)
        Jp = segment_objective(state0, prm, types, mol, L, with_params(ff, tp), K, which)
        Jm = segment_objective(state0, prm, types, mol, L, with_params(ff, tm), K, which)
        g[k] = (Jp - Jm) / (tp[k] - tm[k])
    return g


def one_step_from_rest_gradient(x0: np.ndarray, types, mol, L: float, ff: ForceField, dt: float,
                                which: int) -> np.ndarray:
    """Closed form for the pin: one NVE step of one bead from rest moves the atoms to
    x1 = x0 + (dt^2 / 2m) ACC F(x0), so dJ/dtheta = da/dtheta(x1) + grad a(x1) . (dt^2/2m) ACC dF(x0)/dtheta.
    F is linear in eps, k_b, k_theta and in q_O^2, so dF/dtheta comes from force evaluations
    with the other terms switched off; sigma (not linear) is left out (returned as NaN)."""
    masses = ff.masses(types)[:, None]
    F0 = potential(x0, types, mol, L, ff)[1]
    x1 = x0 + 0.5 * dt * dt * ACC * F0 / masses
    off = dict(eps=0.0, q_O=0.0, k_b=0.0, k_theta=0.0)

    def part(**on):
        f = dataclasses.replace(ff, **{**off, **on})
        return potential(x0, types, mol, L, f)[1]
    dF = [part(eps=1.0), None, 2.0 * part(q_O=ff.q_O) / ff.q_O, part(k_b=1.0), part(k_theta=1.0)]
    if which == OBS_CENTROID_ENERGY:
        V1, F1 = potential(x1, types, mol, L, ff)
        grad_a, direct = -F1, param_gradient(x1, types, mol, L, ff)
    else:
        n_mol = x1.shape[0] // 3
        grad_a = np.zeros_like(x1)
        for m in range(n_mol):
            for hh in (1, 2):
                d = min_image(x1[3 * m + hh] - x1[3 * m], L)
                u = d / np.linalg.norm(d) / (2.0 * n_mol)
                grad_a[3 * m + hh] += u
                grad_a[3 * m] -= u
        direct = np.zeros(5)
    out = np.full(5, np.nan)
    for k in (0, 2, 3, 4):
        out[k] = direct[k] + float(np.sum(grad_a * 0.5 * dt * dt * ACC * dF[k] / masses))
    return out
