"""Pins for the oracle's potential and centroid neighbour list (no GPU)."""
import math

import numpy as np
import pytest

from oracle import neighbor, water
from oracle.units import COULOMB
from paper_2212_03137_b300.workloads import water_box


def _small_box(n_mol=27, seed=11):
    return water_box(n_mol, seed)


def test_dsf_energy_and_force_vanish_at_cutoff():
    ff = water.ForceField(rc=7.0)
    r = np.array([ff.rc])
    e, g = water.coulomb_dsf(r, np.array([0.84 * 0.42]), ff)
    assert abs(e[0]) < 1e-13 and abs(g[0]) < 1e-13
    el, _ = water.lj_shifted(r, ff)
    assert abs(el[0]) < 1e-15


def test_dsf_reduces_to_coulomb_law():
    """alpha = 0 and a far cutoff: the DSF pair energy approaches k_e q_i q_j / r."""
    ff = water.ForceField(alpha=0.0, rc=1e7)
    r = np.array([2.5, 3.0, 4.5])
    e, g = water.coulomb_dsf(r, np.full(3, -0.84 * 0.42), ff)
    np.testing.assert_allclose(e, COULOMB * (-0.84 * 0.42) / r, rtol=1e-6)
    np.testing.assert_allclose(g * r, COULOMB * (-0.84 * 0.42) / r ** 2, rtol=1e-6)


def test_dsf_with_self_term_gives_the_madelung_energy():
    """Rock salt (+-1 charges, nearest-neighbour distance a): the DSF pair sum plus the DSF
    self term approximates the Ewald sum, -M k_e/a per ion pair with the Madelung constant
    M = 1.747565 (Fennell & Gezelter 2006).  Without the self term it misses by > 5 %."""
    n, a = 6, 2.82
    idx = np.stack(np.meshgrid(*(np.arange(2 * n),) * 3, indexing="ij"), -1).reshape(-1, 3)
    x = idx * a
    q = np.where(idx.sum(1) % 2 == 0, 1.0, -1.0)
    L = 2 * n * a
    ff = water.ForceField(alpha=0.25, rc=12.0)
    assert 2 * ff.rc < L
    pairs = 0.0
    for i in range(len(x) - 1):
        d = water.min_image(x[i + 1:] - x[i], L)
        r = np.sqrt((d * d).sum(1))
        m = r < ff.rc
        e, _ = water.coulomb_dsf(r[m], q[i] * q[i + 1:][m], ff)
        pairs += e.sum()
    madelung = -1.747565 * COULOMB / a
    per_pair = (pairs + water.dsf_self_energy(q, ff)) / (len(x) / 2)
    assert abs(per_pair / madelung - 1.0) < 2e-4, per_pair / madelung
    assert abs(pairs / (len(x) / 2) / madelung - 1.0) > 0.05


def test_lj_minimum_at_two_to_one_sixth_sigma():
    ff = water.ForceField(rc=1e6)
    r = np.array([2 ** (1 / 6) * ff.sigma])
    e, g = water.lj_shifted(r, ff)
    assert abs(g[0]) < 1e-14
    np.testing.assert_allclose(e[0], -ff.eps, rtol=1e-9)


def test_bonded_zero_at_equilibrium_geometry():
    ff = water.ForceField()
    h = ff.theta0 / 2
    x = np.array([[1.0, 1.0, 1.0], [1 + math.sin(h), 1.0, 1 + math.cos(h)], [1 - math.sin(h), 1.0, 1 + math.cos(h)]])
    E, F = water.bonded(x, 30.0, ff)
    assert abs(E) < 1e-24 and np.abs(F).max() < 1e-12


def test_forces_match_finite_differences():
    """-grad V by central differences of an energy written without any force term."""
    w = _small_box(8, 5)
    ff = water.ForceField(rc=3.5)
    E, F = water.potential(w.pos, w.types, w.molecule, w.box, ff)
    # no pair within the FD step of the cutoff
    d = water.min_image(w.pos[None] - w.pos[:, None], w.box)
    r = np.linalg.norm(d, axis=-1)
    assert np.min(np.abs(r - ff.rc)) > 1e-3
    E2 = water.potential_energy_only(w.pos, w.types, w.molecule, w.box, ff)
    np.testing.assert_allclose(E, E2, rtol=1e-12)
    h = 1e-5
    rng = np.random.default_rng(0)
    for a in rng.choice(w.n_atoms, 6, replace=False):
        for k in range(3):
            xp, xm = w.pos.copy(), w.pos.copy()
            xp[a, k] += h
            xm[a, k] -= h
            fd = -(water.potential_energy_only(xp, w.types, w.molecule, w.box, ff)
                   - water.potential_energy_only(xm, w.types, w.molecule, w.box, ff)) / (2 * h)
            assert abs(fd - F[a, k]) < 2e-6 * max(1.0, abs(F[a, k]))


def test_total_force_vanishes():
    w = _small_box(27, 3)
    ff = water.ForceField(rc=4.0)
    _, F = water.potential(w.pos, w.types, w.molecule, w.box, ff)
    assert np.abs(F.sum(axis=0)).max() < 1e-10


def test_cell_list_forces_equal_brute_force():
    w = water_box(512, 3)
    ff = water.ForceField(rc=7.5)
    E1, F1 = water.nonbonded(w.pos, w.types, w.molecule, w.box, ff)
    E2, F2 = water.nonbonded_cells(w.pos, w.types, w.molecule, w.box, ff)
    np.testing.assert_allclose(E1, E2, rtol=1e-12)
    np.testing.assert_allclose(F1, F2, atol=1e-11)
    Fs = water.nonbonded_on_atoms(w.pos, np.arange(0, w.n_atoms, 97), w.types, w.molecule, w.box, ff)
    np.testing.assert_allclose(Fs, F1[::97], atol=1e-11)


def test_cell_assignment_edge_cases():
    L, n_c = 10.0, 4
    C = np.array([[0.0, 0.0, 0.0], [10.0, 0, 0], [-1e-20, 0, 0], [-10.0, 0, 0], [9.999999999999998, 0, 0],
                  [2.5, 5.0, 7.5], [25.0, -2.5, 0]])
    cell = neighbor.assign_cells(C, L, n_c)
    cx = cell % n_c
    assert list(cx) == [0, 0, 0, 0, 3, 1, 2]
    assert cell[5] == (3 * n_c + 2) * n_c + 1


def test_sort_is_by_cell_then_index():
    rng = np.random.default_rng(4)
    cell = rng.integers(0, 20, 500)
    order = neighbor.sort_by_cell(cell)
    key = cell[order] * 1000 + order
    assert np.all(np.diff(key) > 0)


def test_list_complete_through_cell_stencil():
    """Every brute-force list pair is found among the 5 x 5 x 5 stencil cells of the grid."""
    w = water_box(512, 9)
    r_list = 8.0
    n_c = neighbor.cell_grid(w.box, r_list)
    assert n_c >= 5
    pairs = neighbor.verlet_pairs(w.pos, w.molecule, w.box, r_list)
    cell = neighbor.assign_cells(w.pos, w.box, n_c)
    cz, cy, cx = cell // (n_c * n_c), (cell // n_c) % n_c, cell % n_c
    i, j = pairs[:, 0], pairs[:, 1]

    def cdist(a, b):
        d = np.abs(a - b)
        return np.minimum(d, n_c - d)
    assert np.all(cdist(cx[i], cx[j]) <= 2) and np.all(cdist(cy[i], cy[j]) <= 2) and np.all(cdist(cz[i], cz[j]) <= 2)
    # brute-force count from an independent per-atom enumeration
    cnt = sum(len(neighbor.neighbours_of(a, w.pos, w.molecule, w.box, r_list)) for a in range(0, w.n_atoms, 37))
    ref = sum(np.sum((i == a) | (j == a)) for a in range(0, w.n_atoms, 37))
    assert cnt == ref


def test_list_uses_strict_inequality():
    L = 20.0
    C = np.array([[0.0, 0.0, 0.0], [4.0, 0.0, 0.0], [3.0, 0.0, 0.0]])
    mol = np.array([0, 1, 2])
    pairs = neighbor.verlet_pairs(C, mol, L, 4.0)
    assert sorted(map(tuple, pairs.tolist())) == [(0, 2), (1, 2)]


def test_same_molecule_excluded_and_small_box_rule():
    w = water_box(64, 1, box=12.42)
    pairs = neighbor.verlet_pairs(w.pos, w.molecule, w.box, 8.0)
    assert np.all(w.molecule[pairs[:, 0]] != w.molecule[pairs[:, 1]])
    assert not neighbor.use_centroid_list(12.42, 6.0, 2.0)
    assert not neighbor.use_centroid_list(18.6, 9.0, 2.0)
    assert neighbor.use_centroid_list(49.7, 9.0, 2.0)
