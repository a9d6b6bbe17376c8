"""Interatomic potential V(x) of one bead configuration, FP64.

The paper's method is independent of V (Eqs. (3), (9), (12) only need V and
grad V); its own force fields (AMOEBA family) are not reproduced.  V here is a
flexible q-SPC/Fw-style water:

* LJ 12-6 between O atoms only, energy-shifted to zero at the cutoff rc;
* damped-shifted-force (DSF) Coulomb between all atoms (Fennell & Gezelter,
  J. Chem. Phys. 124, 234104 (2006)): energy and force both vanish at rc, plus
  the constant self term -(erfc(a rc)/(2 rc) + a/sqrt(pi)) k_e sum_i q_i^2;
* harmonic bonds 1/2 k_b (r_OH - r0)^2 (two per molecule) and a harmonic angle
  1/2 k_theta (theta - theta0)^2;
* the three intramolecular pairs carry no nonbonded term;
* cutoffs are atom-atom with the minimum-image convention in a cubic box.

Pair convention: d = x_j - x_i (minimum image), r = |d|, g = -V'(r)/r, so the
force on j is +g d and on i is -g d.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import erfc

from .units import COULOMB


@dataclass
class ForceField:
    eps: float = 0.1554
    sigma: float = 3.1655
    q_O: float = -0.84
    k_b: float = 1059.162
    r0: float = 1.0
    k_theta: float = 75.90
    theta0: float = math.radians(112.0)
    alpha: float = 0.2
    rc: float = 9.0
    m_O: float = 15.999
    m_H: float = 1.008

    @property
    def q_H(self) -> float:
        return -self.q_O / 2.0

    def charges(self, types: np.ndarray) -> np.ndarray:
        return np.where(types == 0, self.q_O, self.q_H)

    def masses(self, types: np.ndarray) -> np.ndarray:
        return np.where(types == 0, self.m_O, self.m_H)


def min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.rint(d / L)


def dsf_shift_slope(ff: ForceField) -> float:
    """S_c = erfc(a rc)/rc^2 + (2a/sqrt(pi)) exp(-a^2 rc^2)/rc, the force value at rc."""
    a, rc = ff.alpha, ff.rc
    return erfc(a * rc) / rc ** 2 + 2.0 * a / math.sqrt(math.pi) * math.exp(-(a * rc) ** 2) / rc


def coulomb_dsf(r: np.ndarray, qq: np.ndarray, ff: ForceField):
    """DSF pair energy and g = -V'(r)/r for r < rc (caller masks r >= rc)."""
    a, rc = ff.alpha, ff.rc
    sc = dsf_shift_slope(ff)
    e = erfc(a * r)
    energy = COULOMB * qq * (e / r - erfc(a * rc) / rc + sc * (r - rc))
    minus_dv = COULOMB * qq * (e / r ** 2 + 2.0 * a / math.sqrt(math.pi) * np.exp(-(a * r) ** 2) / r - sc)
    return energy, minus_dv / r


def lj_shifted(r: np.ndarray, ff: ForceField):
    """Energy-shifted 12-6 LJ energy and g = -V'(r)/r for r < rc."""
    sr6 = (ff.sigma / r) ** 6
    src6 = (ff.sigma / ff.rc) ** 6
    energy = 4.0 * ff.eps * (sr6 * sr6 - sr6) - 4.0 * ff.eps * (src6 * src6 - src6)
    g = 24.0 * ff.eps * (2.0 * sr6 * sr6 - sr6) / r ** 2
    return energy, g


def dsf_self_energy(q: np.ndarray, ff: ForceField) -> float:
    a, rc = ff.alpha, ff.rc
    return -(erfc(a * rc) / (2.0 * rc) + a / math.sqrt(math.pi)) * COULOMB * float(np.sum(q * q))


def nonbonded(x: np.ndarray, types: np.ndarray, mol: np.ndarray, L: float, ff: ForceField, block: int = 512):
    """O(N^2) brute force over all pairs i < j of different molecules with r < rc.

    Returns (energy without the self term, forces [N,3]).
    """
    N = x.shape[0]
    q = ff.charges(types)
    isO = types == 0
    F = np.zeros_like(x)
    E = 0.0
    for s in range(0, N, block):
        e = min(N, s + block)
        xi = x[s:e]
        d = min_image(x[None, :, :] - xi[:, None, :], L)           # [b, N, 3]
        r2 = np.einsum("ijk,ijk->ij", d, d)
        idx_i = np.arange(s, e)[:, None]
        idx_j = np.arange(N)[None, :]
        mask = (idx_j > idx_i) & (mol[None, :] != mol[s:e, None]) & (r2 < ff.rc ** 2)
        ii, jj = np.nonzero(mask)
        if ii.size == 0:
            continue
        dd = d[ii, jj]
        r = np.sqrt(r2[ii, jj])
        gi = ii + s
        ec, gc = coulomb_dsf(r, q[gi] * q[jj], ff)
        oo = isO[gi] & isO[jj]
        el = np.zeros_like(r)
        gl = np.zeros_like(r)
        if np.any(oo):
            el[oo], gl[oo] = lj_shifted(r[oo], ff)
        g = gc + gl
        E += float(np.sum(ec) + np.sum(el))
        fij = g[:, None] * dd
        np.add.at(F, jj, fij)
        np.add.at(F, gi, -fij)
    return E, F


def nonbonded_on_atoms(x: np.ndarray, atoms: np.ndarray, types: np.ndarray, mol: np.ndarray, L: float,
                       ff: ForceField) -> np.ndarray:
    """Force on each listed atom from all partners, one atom at a time (sampling helper)."""
    q = ff.charges(types)
    isO = types == 0
    out = np.zeros((len(atoms), 3))
    for k, i in enumerate(atoms):
        d = min_image(x - x[i], L)
        r2 = np.einsum("jk,jk->j", d, d)
        m = (mol != mol[i]) & (r2 < ff.rc ** 2)
        m[i] = False
        r = np.sqrt(r2[m])
        _, gc = coulomb_dsf(r, q[i] * q[m], ff)
        g = gc
        if isO[i]:
            oo = isO[m]
            gl = np.zeros_like(r)
            if np.any(oo):
                _, gl[oo] = lj_shifted(r[oo], ff)
            g = g + gl
        out[k] = -np.sum(g[:, None] * d[m], axis=0)
    return out


def bonded(x: np.ndarray, L: float, ff: ForceField):
    """Harmonic O-H bonds and H-O-H angle for molecules stored as (O, H, H) triples."""
    xm = x.reshape(-1, 3, 3)
    d1 = min_image(xm[:, 1] - xm[:, 0], L)
    d2 = min_image(xm[:, 2] - xm[:, 0], L)
    r1 = np.linalg.norm(d1, axis=1)
    r2 = np.linalg.norm(d2, axis=1)
    E = 0.5 * ff.k_b * float(np.sum((r1 - ff.r0) ** 2 + (r2 - ff.r0) ** 2))
    cos_t = np.einsum("ij,ij->i", d1, d2) / (r1 * r2)
    theta = np.arccos(cos_t)
    E += 0.5 * ff.k_theta * float(np.sum((theta - ff.theta0) ** 2))
    F = np.zeros_like(xm)
    # bonds: F_H = -k_b (r - r0) d / r
    fb1 = -ff.k_b * ((r1 - ff.r0) / r1)[:, None] * d1
    fb2 = -ff.k_b * ((r2 - ff.r0) / r2)[:, None] * d2
    # angle: F_H1 = k_theta (theta - theta0)/sin(theta) * d(cos theta)/d d1
    sin_t = np.sqrt(1.0 - cos_t ** 2)
    pref = (ff.k_theta * (theta - ff.theta0) / sin_t)[:, None]
    dc_d1 = d2 / (r1 * r2)[:, None] - cos_t[:, None] * d1 / (r1 ** 2)[:, None]
    dc_d2 = d1 / (r1 * r2)[:, None] - cos_t[:, None] * d2 / (r2 ** 2)[:, None]
    fa1 = pref * dc_d1
    fa2 = pref * dc_d2
    F[:, 1] = fb1 + fa1
    F[:, 2] = fb2 + fa2
    F[:, 0] = -(fb1 + fa1 + fb2 + fa2)
    return E, F.reshape(-1, 3)


def potential(x: np.ndarray, types: np.ndarray, mol: np.ndarray, L: float, ff: ForceField):
    """V(x) and -grad V(x) for one bead configuration."""
    En, Fn = nonbonded(x, types, mol, L, ff)
    Eb, Fb = bonded(x, L, ff)
    return En + Eb + dsf_self_energy(ff.charges(types), ff), Fn + Fb


def potential_energy_only(x, types, mol, L, ff) -> float:
    """Energy by direct pair summation, written without any force expression (used by FD pins)."""
    N = x.shape[0]
    q = ff.charges(types)
    E = 0.0
    for i in range(N - 1):
        d = min_image(x[i + 1:] - x[i], L)
        r = np.sqrt(np.einsum("jk,jk->j", d, d))
        j = np.arange(i + 1, N)
        m = (mol[j] != mol[i]) & (r < ff.rc)
        rr = r[m]
        a, rc = ff.alpha, ff.rc
        sc = erfc(a * rc) / rc ** 2 + 2.0 * a / math.sqrt(math.pi) * math.exp(-(a * rc) ** 2) / rc
        E += float(np.sum(COULOMB * q[i] * q[j[m]] * (erfc(a * rr) / rr - erfc(a * rc) / rc + sc * (rr - rc))))
        if types[i] == 0:
            oo = types[j[m]] == 0
            ro = rr[oo]
            E += float(np.sum(4 * ff.eps * ((ff.sigma / ro) ** 12 - (ff.sigma / ro) ** 6)
                              - 4 * ff.eps * ((ff.sigma / rc) ** 12 - (ff.sigma / rc) ** 6)))
    xm = x.reshape(-1, 3, 3)
    for m_ in range(xm.shape[0]):
        o, h1, h2 = xm[m_]
        a1 = min_image(h1 - o, L)
        a2 = min_image(h2 - o, L)
        l1, l2 = np.linalg.norm(a1), np.linalg.norm(a2)
        th = math.acos(float(np.dot(a1, a2) / (l1 * l2)))
        E += 0.5 * ff.k_b * ((l1 - ff.r0) ** 2 + (l2 - ff.r0) ** 2) + 0.5 * ff.k_theta * (th - ff.theta0) ** 2
    return E + dsf_self_energy(q, ff)


def nonbonded_cells(x: np.ndarray, types: np.ndarray, mol: np.ndarray, L: float, ff: ForceField):
    """Same pair set as ``nonbonded`` found through a cell grid (cells >= rc wide, 27-cell
    stencil, full neighbourhood with the energy halved).  Needs at least 3 cells per edge."""
    n_c = int(math.floor(L / ff.rc))
    if n_c < 3:
        return nonbonded(x, types, mol, L, ff)
    N = x.shape[0]
    q = ff.charges(types)
    isO = types == 0
    t = x / L
    frac = t - np.floor(t)
    frac = np.where(frac == 1.0, 0.0, frac)
    c3 = np.minimum(np.floor(frac * n_c), n_c - 1).astype(np.int64)
    cid = (c3[:, 2] * n_c + c3[:, 1]) * n_c + c3[:, 0]
    order = np.argsort(cid, kind="stable")
    starts = np.searchsorted(cid[order], np.arange(n_c ** 3 + 1))
    F = np.zeros_like(x)
    E = 0.0
    for cz in range(n_c):
        for cy in range(n_c):
            for cx in range(n_c):
                c = (cz * n_c + cy) * n_c + cx
                ia = order[starts[c]:starts[c + 1]]
                if ia.size == 0:
                    continue
                nb = []
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            cc = (((cz + dz) % n_c) * n_c + (cy + dy) % n_c) * n_c + (cx + dx) % n_c
                            nb.append(order[starts[cc]:starts[cc + 1]])
                ja = np.concatenate(nb)
                d = min_image(x[None, ja, :] - x[ia, None, :], L)
                r2 = np.einsum("ijk,ijk->ij", d, d)
                m = (ja[None, :] != ia[:, None]) & (mol[ja][None, :] != mol[ia][:, None]) & (r2 < ff.rc ** 2)
                a, b = np.nonzero(m)
                gi, gj = ia[a], ja[b]
                r = np.sqrt(r2[a, b])
                ec, g = coulomb_dsf(r, q[gi] * q[gj], ff)
                oo = isO[gi] & isO[gj]
                el = np.zeros_like(r)
                if np.any(oo):
                    el_oo, gl_oo = lj_shifted(r[oo], ff)
                    el[oo] = el_oo
                    g = g.copy()
                    g[oo] += gl_oo
                E += 0.5 * float(np.sum(ec) + np.sum(el))
                np.add.at(F, gi, -g[:, None] * d[a, b])
    return E, F


def make_force_fn(types: np.ndarray, mol: np.ndarray, L: float, ff: ForceField, cells: bool = False):
    """force_fn(xb[P, N, 3]) -> (V[P], F[P, N, 3]) for the water potential."""
    q = ff.charges(types)
    e_self = dsf_self_energy(q, ff)

    def fn(xb):
        P = xb.shape[0]
        V = np.zeros(P)
        F = np.zeros_like(xb)
        for b in range(P):
            En, Fn = (nonbonded_cells if cells else nonbonded)(xb[b], types, mol, L, ff)
            Eb, Fb = bonded(xb[b], L, ff)
            V[b] = En + Eb + e_self
            F[b] = Fn + Fb
        return V, F
    return fn
