"""Centroid cell assignment and Verlet list (Sec. III.A.3).

The paper computes neighbour lists on ring-polymer centroids: when two
centroids are neighbours, every pair of their beads is treated as neighbours,
so one list serves all P beads.  The paper does not define the cells or the
list radius; the readings used here are:

* list radius r_list = rc + skin;
* cell grid n_c = floor(2 L / r_list) per dimension (cells at least r_list / 2 wide, so
  every partner of an atom lies within two cells of it: a 5 x 5 x 5 stencil);
* cell of a centroid C: t = C/L, frac = t - floor(t) (set to 0 when it rounds
  to 1), cell index per dimension min(floor(frac * n_c), n_c - 1), linear id
  (cz * n_c + cy) * n_c + cx;
* atoms are ordered by cell id, ties by ascending atom index;
* (i, j) is a list pair iff the atoms belong to different molecules and the
  minimum-image centroid distance satisfies d^2 < r_list^2 (strict), with
  d = C_j - C_i - L*rint((C_j - C_i)/L) and d^2 = (dx*dx + dy*dy) + dz*dz, every
  operation rounded separately (no fused multiply-add).

The list is defined by brute force over all pairs; the cell grid only orders
atoms.  Both sides must produce the identical pair set and order of cells.
"""
from __future__ import annotations

import math

import numpy as np


def cell_grid(L: float, r_list: float) -> int:
    return int(math.floor(2.0 * L / r_list))


def assign_cells(C: np.ndarray, L: float, n_c: int) -> np.ndarray:
    """Linear cell id for every centroid C[N,3]."""
    t = C / L
    frac = t - np.floor(t)
    frac = np.where(frac == 1.0, 0.0, frac)
    c = np.minimum(np.floor(frac * n_c), n_c - 1).astype(np.int64)
    return (c[:, 2] * n_c + c[:, 1]) * n_c + c[:, 0]


def sort_by_cell(cell: np.ndarray) -> np.ndarray:
    """Sorted order (position -> atom index): by cell id, ties by atom index."""
    return np.argsort(cell, kind="stable")


def pair_distance2(Ci: np.ndarray, Cj: np.ndarray, L: float) -> np.ndarray:
    """Minimum-image squared centroid distance with the fixed operation order above."""
    d = Cj - Ci
    d = d - L * np.rint(d / L)
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def verlet_pairs(C: np.ndarray, mol: np.ndarray, L: float, r_list: float, block: int = 1024) -> np.ndarray:
    """All unordered pairs (i < j) within r_list, as an int64 array [n_pairs, 2]."""
    N = C.shape[0]
    r2max = r_list * r_list
    out = []
    for s in range(0, N, block):
        e = min(N, s + block)
        d2 = pair_distance2(C[s:e, None, :], C[None, :, :], L)
        ii = np.arange(s, e)[:, None]
        jj = np.arange(N)[None, :]
        m = (jj > ii) & (mol[None, :] != mol[s:e, None]) & (d2 < r2max)
        a, b = np.nonzero(m)
        out.append(np.stack([a + s, b], axis=1))
    return np.concatenate(out, axis=0) if out else np.zeros((0, 2), dtype=np.int64)


def neighbours_of(i: int, C: np.ndarray, mol: np.ndarray, L: float, r_list: float) -> np.ndarray:
    """Sorted partner list of one atom (sampling helper for large boxes)."""
    d2 = pair_distance2(C[i][None, :], C, L)
    m = (d2 < r_list * r_list) & (mol != mol[i])
    m[i] = False
    return np.nonzero(m)[0]


def use_centroid_list(L: float, rc: float, skin: float) -> bool:
    """Reading for small boxes: the cell grid is used only when it is at least 5 wide
    (125 distinct stencil cells) and r_list < L/2.  Otherwise the same list (pairs of
    different molecules with minimum-image centroid distance below r_list) is found by
    brute force, and the pair sum applies a per-bead minimum image."""
    r_list = rc + skin
    return cell_grid(L, r_list) >= 5 and r_list < 0.5 * L
