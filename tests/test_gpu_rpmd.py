"""CUDA path vs the FP64 oracle: initial modes, bead transform, centroid list, forces,
estimators and short trajectories (RPMD with the PILE thermostat).

Tolerances: FP64 path 1e-12 RMS relative force error and 1e-10 A on 10-step
centroids; mixed path 1e-5 RMS relative force error and 1e-6 A on 10-step centroids.
"""
import dataclasses

import numpy as np
import pytest

from oracle import neighbor, normal_modes, rpmd
from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import CONFIGS, small_mixed_config

from oracle_bridge import force_fn, list_pairs_oracle, oracle_ff, oracle_params, rms_rel

pytestmark = pytest.mark.gpu

C1 = CONFIGS["rpmd_fp64_64w"]
C2 = CONFIGS["rpmd_mixed_4096w"]
SMALL = small_mixed_config(512, P=8)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


def _sys(cfg, precision=None, **kw):
    return qhp.System.from_config(cfg, precision=precision, **kw)


def _oracle_state(cfg, seed=None):
    box = cfg.system()
    ff = oracle_ff(cfg.rc)
    prm = oracle_params(cfg, seed)
    st = rpmd.init_state(box.pos, ff.masses(box.types), prm)
    return box, ff, prm, st


@pytest.mark.parametrize("cfg", [C1, SMALL], ids=["fp64_64w", "mixed_512w"])
def test_initial_modes_and_beads(cfg):
    box, ff, prm, st = _oracle_state(cfg)
    with _sys(cfg) as s:
        Q, Pm = qhp.qhp_get_modes(s.h)
        np.testing.assert_allclose(Q, st.Q, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(Pm, st.Pm, rtol=1e-13, atol=1e-12)
        xb = qhp.qhp_get_beads(s.h)
        np.testing.assert_allclose(xb, rpmd.beads(st, cfg.P), rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("cfg", [SMALL, C2], ids=["512w", "4096w"])
def test_cells_and_centroid_list_bit_exact(cfg):
    with _sys(cfg) as s:
        qhp.qhp_build_list(s.h)
        info = qhp.qhp_get_info(s.h)
        assert info.list_mode == 1
        Q, _ = qhp.qhp_get_modes(s.h)
        C = Q[:, :, 0]
        box = cfg.system()
        r_list = cfg.rc + cfg.skin
        n_c = neighbor.cell_grid(box.box, r_list)
        assert info.n_cells_per_edge == n_c
        cell, order = qhp.qhp_get_cells(s.h)
        ocell = neighbor.assign_cells(C, box.box, n_c)
        np.testing.assert_array_equal(cell, ocell)
        np.testing.assert_array_equal(order, neighbor.sort_by_cell(ocell))
        got = qhp.qhp_get_list_pairs(s.h)
        assert len(got) == len(set(map(tuple, got.tolist())))
        assert set(map(tuple, got.tolist())) == list_pairs_oracle(C, box.molecule, box.box, r_list)


def test_list_with_crowded_cells():
    """A 10 A skin makes the cells 9.9 A wide (5 per edge), about 98 atoms each. The list fill
    then takes a cell's atoms in more than one pass, and an atom's ~12,000 candidates span many
    staged chunks."""
    cfg = dataclasses.replace(C2, skin=10.0, P=1)
    with _sys(cfg) as s:
        qhp.qhp_step_rpmd(s.h, 5)
        qhp.qhp_build_list(s.h)
        info = qhp.qhp_get_info(s.h)
        assert info.list_mode == 1 and info.n_cells_per_edge == 5
        Q, _ = qhp.qhp_get_modes(s.h)
        box = cfg.system()
        cell, _ = qhp.qhp_get_cells(s.h)
        assert np.bincount(cell).max() > 64
        got = qhp.qhp_get_list_pairs(s.h).astype(np.int64)
    ref = neighbor.verlet_pairs(Q[:, :, 0], box.molecule, box.box, cfg.rc + cfg.skin).astype(np.int64)
    n = np.int64(3 * cfg.n_mol)
    g = np.sort(got[:, 0] * n + got[:, 1])
    assert np.all(np.diff(g) > 0)   # no duplicates
    np.testing.assert_array_equal(g, np.sort(ref[:, 0] * n + ref[:, 1]))


@pytest.mark.parametrize("cfg", [C1, CONFIGS["grad_216w"]], ids=["64w_L12.42", "216w_L18.6"])
def test_small_box_list_bit_exact(cfg):
    """Boxes with r_list >= L/2 have no cell grid: the rows still hold exactly the pairs of
    different molecules whose minimum-image centroid distance is below r_list."""
    with _sys(cfg) as s:
        for n in (0, 15):
            qhp.qhp_step_rpmd(s.h, n)
            qhp.qhp_build_list(s.h)
            assert qhp.qhp_get_info(s.h).list_mode == 0
            Q, _ = qhp.qhp_get_modes(s.h)
            box = cfg.system()
            got = set(map(tuple, qhp.qhp_get_list_pairs(s.h).tolist()))
            ref = list_pairs_oracle(Q[:, :, 0], box.molecule, box.box, cfg.rc + cfg.skin)
            assert got == ref
            n_mol_pairs = cfg.n_mol * (cfg.n_mol - 1) // 2 * 9
            assert len(ref) < n_mol_pairs   # the distance filter removes pairs


def test_list_after_dynamics_and_edge_positions():
    """Centroids moved by dynamics and pushed onto cell/box boundaries: still bit-exact."""
    cfg = SMALL
    with _sys(cfg) as s:
        qhp.qhp_step_rpmd(s.h, 15)
        Q, Pm = qhp.qhp_get_modes(s.h)
        box = cfg.system()
        L = box.box
        Q[0, 0, 0] = 0.0
        Q[3, 1, 0] = L
        Q[6, 2, 0] = -1e-17
        Q[9, 0, 0] = L * 2 / 3
        Q[12, 0, 0] = -L + 1e-9
        qhp.qhp_set_modes(s.h, Q, Pm)
        qhp.qhp_build_list(s.h)
        r_list = cfg.rc + cfg.skin
        n_c = neighbor.cell_grid(L, r_list)
        cell, order = qhp.qhp_get_cells(s.h)
        ocell = neighbor.assign_cells(Q[:, :, 0], L, n_c)
        np.testing.assert_array_equal(cell, ocell)
        np.testing.assert_array_equal(order, neighbor.sort_by_cell(ocell))
        got = set(map(tuple, qhp.qhp_get_list_pairs(s.h).tolist()))
        assert got == list_pairs_oracle(Q[:, :, 0], box.molecule, L, r_list)


def test_forces_fp64_allpairs():
    cfg = C1
    with _sys(cfg) as s:
        assert qhp.qhp_get_info(s.h).list_mode == 0
        qhp.qhp_compute_forces(s.h)
        xb = qhp.qhp_get_beads(s.h)
        F = qhp.qhp_get_forces(s.h)
    _, Fo = force_fn(cfg.system(), cfg.rc)(xb)
    assert rms_rel(F, Fo) < 1e-12


def test_forces_mixed_list_small_box():
    cfg = SMALL
    with _sys(cfg) as s:
        qhp.qhp_compute_forces(s.h)
        xb = qhp.qhp_get_beads(s.h)
        F = qhp.qhp_get_forces(s.h)
    _, Fo = force_fn(cfg.system(), cfg.rc)(xb)
    err = rms_rel(F, Fo)
    assert err < 1e-5, err


def test_forces_fp64_list_small_box():
    cfg = SMALL
    with _sys(cfg, precision="fp64") as s:
        qhp.qhp_compute_forces(s.h)
        xb = qhp.qhp_get_beads(s.h)
        F = qhp.qhp_get_forces(s.h)
    _, Fo = force_fn(cfg.system(), cfg.rc)(xb)
    assert rms_rel(F, Fo) < 1e-12


def test_forces_fp64_bead_lanes():
    """1,000 waters (3,000 atoms): the FP64 pair kernel runs with bead lanes (a warp per atom);
    the smaller boxes above run with row lanes (a warp per atom and bead)."""
    cfg = small_mixed_config(1000, P=4)
    with _sys(cfg, precision="fp64") as s:
        assert qhp.qhp_get_info(s.h).list_mode == 1
        qhp.qhp_step_rpmd(s.h, 2)
        qhp.qhp_compute_forces(s.h)
        xb = qhp.qhp_get_beads(s.h)
        F = qhp.qhp_get_forces(s.h)
    _, Fo = force_fn(cfg.system(), cfg.rc, cells=True)(xb[[0, 3]])
    assert rms_rel(F[[0, 3]], Fo) < 1e-12


def test_forces_mixed_full_size_sampled_beads():
    """4,096 waters, P = 32: two beads compared over every atom (oracle cell-list sum)."""
    cfg = C2
    with _sys(cfg) as s:
        qhp.qhp_step_rpmd(s.h, 3)
        qhp.qhp_compute_forces(s.h)
        xb = qhp.qhp_get_beads(s.h)
        F = qhp.qhp_get_forces(s.h)
    fn = force_fn(cfg.system(), cfg.rc, cells=True)
    for b in (0, 17):
        _, Fo = fn(xb[b:b + 1])
        err = rms_rel(F[b], Fo[0])
        assert err < 1e-5, (b, err)


@pytest.mark.parametrize("cfg,prec,tol", [(C1, "fp64", 1e-11), (SMALL, "mixed", 2e-6)], ids=["fp64", "mixed"])
def test_estimators(cfg, prec, tol):
    box, ff, prm, st = _oracle_state(cfg)
    with _sys(cfg, precision=prec) as s:
        e = qhp.qhp_get_energy(s.h)
    rpmd.evaluate_forces(st, prm, force_fn(box, cfg.rc))
    m = ff.masses(box.types)
    UP = rpmd.potential_estimator(st)
    scale = np.mean(np.abs(st.V)) + 1.0
    assert abs(e.potential - UP) < tol * scale * 10, (e.potential, UP)
    np.testing.assert_allclose(e.spring, rpmd.spring_energy(st, prm, m), rtol=1e-12)
    np.testing.assert_allclose(e.kinetic_nm, rpmd.kinetic_energy(st, m), rtol=1e-12)
    kcv = rpmd.centroid_virial_kinetic(st, prm)
    assert abs(e.kinetic_cv - kcv) < tol * 100 * abs(kcv), (e.kinetic_cv, kcv)


@pytest.mark.parametrize("cfg,prec,tol", [(C1, "fp64", 1e-10), (SMALL, "mixed", 1e-6)], ids=["fp64", "mixed"])
def test_ten_step_trajectory(cfg, prec, tol):
    box, ff, prm, st = _oracle_state(cfg)
    m = ff.masses(box.types)
    fn = force_fn(box, cfg.rc)
    for _ in range(10):
        rpmd.step(st, prm, m, fn)
    with _sys(cfg, precision=prec) as s:
        qhp.qhp_step_rpmd(s.h, 10)
        Q, Pm = qhp.qhp_get_modes(s.h)
        xb = qhp.qhp_get_beads(s.h)
    dC = np.abs(Q[:, :, 0] - st.Q[:, :, 0]).max()
    assert dC < tol, dC
    assert np.abs(xb - rpmd.beads(st, cfg.P)).max() < 10 * tol


def test_free_ring_polymer_energy_conservation():
    """V = 0 and no thermostat: every mode energy is conserved (exact A flow)."""
    cfg = C1
    box = cfg.system()
    ff = qhp.make_ff(cfg.rc, eps=0.0, q_O=0.0, k_b=0.0, k_theta=0.0)
    th = qhp.make_thermo(kind=qhp.QHP_THERMO_NVE, dt_fs=0.25)
    s = qhp.System(box.box, box.types, box.molecule, box.pos, qhp.QHP_FP64, ff, cfg.P, 300.0, 5, th)
    try:
        P = cfg.P
        prm = oracle_params(cfg)
        w = prm.omegas()
        mass = oracle_ff(cfg.rc).masses(box.types)[:, None, None]
        Q0, P0 = qhp.qhp_get_modes(s.h)
        e0 = P0 ** 2 / (2 * mass) + 0.5 * mass * w ** 2 * Q0 ** 2
        nsteps = 200_000
        qhp.qhp_step_rpmd(s.h, nsteps)
        Q1, P1 = qhp.qhp_get_modes(s.h)
        e1 = P1 ** 2 / (2 * mass) + 0.5 * mass * w ** 2 * Q1 ** 2
        rel = np.abs(e1[..., 1:] - e0[..., 1:]).max() / e0[..., 1:].max()
        assert rel < 1e-12, rel
        t = nsteps * 0.25e-3
        Qe = Q0[..., 1:] * np.cos(w[1:] * t) + P0[..., 1:] / (mass * w[1:]) * np.sin(w[1:] * t)
        assert np.abs(Q1[..., 1:] - Qe).max() < 1e-8
        # free centroid drift: two FP64 additions per step, each rounded within 2^-53 relative
        drift_rtol = 2 * nsteps * 2.0 ** -53
        np.testing.assert_allclose(Q1[..., 0], Q0[..., 0] + P0[..., 0] * t / mass[..., 0], rtol=drift_rtol,
                                   atol=1e-10)
    finally:
        s.close()


def test_runs_are_bitwise_reproducible_and_checkpoint_resumes():
    cfg = SMALL
    with _sys(cfg) as a, _sys(cfg) as b:
        qhp.qhp_step_rpmd(a.h, 12)
        qhp.qhp_step_rpmd(b.h, 12)
        Qa, Pa = qhp.qhp_get_modes(a.h)
        Qb, Pb = qhp.qhp_get_modes(b.h)
        assert np.array_equal(Qa, Qb) and np.array_equal(Pa, Pb)
        blob = qhp.qhp_get_state(a.h)
        qhp.qhp_step_rpmd(a.h, 9)
        Q1, P1 = qhp.qhp_get_modes(a.h)
        qhp.qhp_set_state(a.h, blob)
        qhp.qhp_step_rpmd(a.h, 4)
        qhp.qhp_step_rpmd(a.h, 5)
        Q2, P2 = qhp.qhp_get_modes(a.h)
        assert np.array_equal(Q1, Q2) and np.array_equal(P1, P2)
        assert qhp.qhp_get_info(a.h).step == 21


def test_direct_launches_match_step_graphs():
    """Kernel-by-kernel launches give the same trajectory, bit for bit, as the step graphs."""
    cfg = SMALL
    with _sys(cfg) as a, _sys(cfg) as b:
        qhp.qhp_set_graph_mode(b.h, False)
        qhp.qhp_step_rpmd(a.h, 30)                 # crosses list rebuilds
        for _ in range(3):
            qhp.qhp_step_rpmd(b.h, 10)
        Qa, Pa = qhp.qhp_get_modes(a.h)
        Qb, Pb = qhp.qhp_get_modes(b.h)
        assert np.array_equal(Qa, Qb) and np.array_equal(Pa, Pb)
        assert qhp.qhp_get_info(a.h).rebuilds == qhp.qhp_get_info(b.h).rebuilds > 1
        for h in (a.h, b.h):                       # stage timestamps in both modes
            qhp.qhp_set_profiling(h, True)
            qhp.qhp_step_rpmd(h, 1)
            pr = qhp.qhp_get_profile(h)
            assert pr.pair_ms > 0 and pr.step_ms >= pr.pair_ms
        with pytest.raises(qhp.QHPError):
            qhp._check(qhp.lib().qhp_set_graph_mode(a.h, 2))


def test_mode_equipartition_under_pile():
    """PILE samples <P_n^2> = m kT on every mode (Eq. (7))."""
    cfg = C1
    with _sys(cfg) as s:
        acc = np.zeros(cfg.P)
        n = 0
        qhp.qhp_step_rpmd(s.h, 200)
        for _ in range(40):
            qhp.qhp_step_rpmd(s.h, 25)
            _, Pm = qhp.qhp_get_modes(s.h)
            m = oracle_ff(cfg.rc).masses(cfg.system().types)[:, None, None]
            acc += np.mean(Pm ** 2 / m, axis=(0, 1))
            n += 1
        kT = oracle_params(cfg).kT * 418.4
        np.testing.assert_allclose(acc[1:] / n, kT, rtol=0.08)


def test_argument_and_state_errors():
    cfg = C1
    box = cfg.system()
    h = qhp.qhp_create_system(box.types, box.molecule, box.pos, box.box, qhp.QHP_MIXED)
    try:
        with pytest.raises(qhp.QHPError) as e:
            qhp.qhp_step_rpmd(h, 1)
        assert e.value.code == -6
        with pytest.raises(qhp.QHPError) as e:
            qhp.qhp_set_forcefield(h, qhp.make_ff(7.0))       # rc >= L/2
        assert e.value.code == -1
        with pytest.raises(qhp.QHPError):
            qhp.qhp_set_beads(h, 8, 300.0, 1)                 # before the force field
        qhp.qhp_set_forcefield(h, qhp.make_ff(6.0))
        for bad in (0, 3, 12, 128):
            with pytest.raises(qhp.QHPError) as e:
                qhp.qhp_set_beads(h, bad, 300.0, 1)
            assert e.value.code == -1
        qhp.qhp_set_beads(h, 4, 300.0, 1)
        with pytest.raises(qhp.QHPError) as e:
            qhp.qhp_set_thermostat(h, qhp.make_thermo(kind=qhp.QHP_THERMO_ADQTB, gamma0=20.0, n_seg=64))
        assert e.value.code == -6                              # adQTB needs P = 1
        with pytest.raises(qhp.QHPError) as e:
            qhp.qhp_step_rpmd(h, -1)
        assert e.value.code == -1
        qhp.qhp_step_rpmd(h, 0)
        qhp.qhp_step_rpmd(h, 1)
    finally:
        qhp.qhp_destroy_system(h)
