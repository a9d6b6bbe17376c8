"""Full-size cases in the launch configuration the bench times, checked on sampled outputs
the oracle computes one by one.

* 72,000 waters (216,000 atoms, 129 A box), single bead, adQTB: list rows of sampled atoms
  (bit-exact), forces of sampled atoms, colored noise of sampled degrees of freedom;
* 4,096 waters x 32 beads after dynamics: list rows and rebuild bookkeeping.
"""
import numpy as np
import pytest

from oracle import neighbor, qtb, water
from oracle.units import CM1_TO_RAD_PS
from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import CONFIGS

from oracle_bridge import oracle_ff

pytestmark = pytest.mark.gpu

C3 = CONFIGS["adqtb_mixed_72000w"]
C2 = CONFIGS["rpmd_mixed_4096w"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


@pytest.fixture(scope="module")
def c3_system():
    s = qhp.System.from_config(C3)
    yield s
    s.close()


def _row(h, a):
    r = qhp.qhp_get_list_row(h, int(a))
    assert len(r) == len(set(r.tolist()))          # no duplicate partners
    return set(r.tolist())


def test_adqtb_fullsize_list_rows_bit_exact(c3_system):
    s = c3_system
    qhp.qhp_build_list(s.h)
    info = qhp.qhp_get_info(s.h)
    assert info.list_mode == 1 and info.n_atoms == 216000
    box = C3.system()
    Q, _ = qhp.qhp_get_modes(s.h)
    C = Q[:, :, 0]
    r_list = C3.rc + C3.skin
    rng = np.random.default_rng(3)
    atoms = rng.choice(box.n_atoms, 48, replace=False)
    for a in atoms:
        want = set(neighbor.neighbours_of(int(a), C, box.molecule, box.box, r_list).tolist())
        assert _row(s.h, a) == want
    cell, order = qhp.qhp_get_cells(s.h)
    n_c = neighbor.cell_grid(box.box, r_list)
    np.testing.assert_array_equal(cell, neighbor.assign_cells(C, box.box, n_c))
    np.testing.assert_array_equal(order, neighbor.sort_by_cell(cell))


def test_adqtb_fullsize_sampled_forces(c3_system):
    s = c3_system
    qhp.qhp_compute_forces(s.h)
    F = qhp.qhp_get_forces(s.h)[0]
    x = qhp.qhp_get_beads(s.h)[0]
    box = C3.system()
    ff = oracle_ff(C3.rc)
    rng = np.random.default_rng(5)
    mols = rng.choice(box.n_mol, 40, replace=False)
    atoms = np.sort(np.concatenate([3 * mols, 3 * mols + 1, 3 * mols + 2]))
    Fn = water.nonbonded_on_atoms(x, atoms, box.types, box.molecule, box.box, ff)
    sel = np.concatenate([np.arange(3 * m, 3 * m + 3) for m in np.sort(mols)])
    _, Fb = water.bonded(x[sel], box.box, ff)
    Fo = Fn + Fb
    err = float(np.sqrt(np.sum((F[atoms] - Fo) ** 2) / np.sum(Fo ** 2)))
    assert err < 1e-5, err


def test_adqtb_fullsize_sampled_noise(c3_system):
    s = c3_system
    u = qhp.qhp_get_qtb_noise(s.h, C3.n_seg)
    box = C3.system()
    ff = oracle_ff(C3.rc)
    prm = qtb.QTBParams(n_seg=C3.n_seg, dt=C3.dt_fs * 1e-3, gamma0=C3.gamma0, temperature=C3.temperature,
                        omega_cut=C3.omega_cut_cm * CM1_TO_RAD_PS, a_gamma=C3.a_gamma, seed=C3.seed)
    rng = np.random.default_rng(9)
    dofs = np.sort(rng.choice(3 * box.n_atoms, 24, replace=False))
    dtype = box.types[dofs // 3]
    gam = np.full(prm.n_seg + 1, prm.gamma0)
    taps = np.stack([qtb.filter_taps(qtb.noise_power(gam, prm), prm) for _ in dofs])
    uo = qtb.colored_segment_fft(0, taps, dofs, prm)
    scale = np.sqrt(np.mean(uo ** 2))
    assert np.abs(u[:, dofs] - uo).max() < 2e-5 * scale
    del dtype, ff


def test_rpmd_fullsize_list_rows_after_dynamics():
    with qhp.System.from_config(C2) as s:
        qhp.qhp_step_rpmd(s.h, 40)
        info = qhp.qhp_get_info(s.h)
        assert info.rebuilds >= 1
        Q, _ = qhp.qhp_get_modes(s.h)
        qhp.qhp_build_list(s.h)
        box = C2.system()
        atoms = np.random.default_rng(1).choice(box.n_atoms, 64, replace=False)
        for a in atoms:
            want = set(neighbor.neighbours_of(int(a), Q[:, :, 0], box.molecule, box.box, C2.rc + C2.skin).tolist())
            assert _row(s.h, a) == want
