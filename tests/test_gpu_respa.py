"""RESPA with ring-polymer contraction on the CUDA path against the FP64 oracle.

Mixed precision: centroid trajectories agree with the oracle to 1e-6 A (the FP32 pair
forces' error, ~1e-6 relative, integrated over a few tens of femtoseconds)."""
import numpy as np
import pytest

from oracle import respa, rpmd
from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import small_mixed_config

from oracle_bridge import oracle_ff, oracle_params

pytestmark = pytest.mark.gpu

SMALL = small_mixed_config(512, P=8)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


def _oracle_run(cfg, n_alt, Pc, n_outer):
    box = cfg.system()
    ff = oracle_ff(cfg.rc)
    prm = oracle_params(cfg)
    m = ff.masses(box.types)
    st = rpmd.init_state(box.pos, m, prm)
    fast, slow = respa.split_force_fns(box.types, box.molecule, box.box, ff)
    C = respa.contraction_matrix(cfg.P, Pc)
    for _ in range(n_outer):
        respa.respa_step(st, prm, m, fast, slow, n_alt, C)
    return st


@pytest.mark.parametrize("P,n_alt,Pc", [(8, 4, 4), (8, 2, 1), (8, 3, 8), (64, 2, 16), (4, 2, 2)],
                         ids=["P8_n4_Pc4", "P8_n2_centroid", "P8_n3_full", "P64_n2_Pc16", "P4_n2_Pc2"])
def test_respa_contraction_trajectory_matches_oracle(P, n_alt, Pc):
    cfg = small_mixed_config(512, P=P)
    n_outer = 4 if P <= 8 else 2
    st = _oracle_run(cfg, n_alt, Pc, n_outer)
    with qhp.System.from_config(cfg) as s:
        qhp.qhp_set_respa(s.h, n_alt, Pc)
        qhp.qhp_step_rpmd(s.h, n_outer)
        Q, _ = qhp.qhp_get_modes(s.h)
        assert qhp.qhp_get_info(s.h).step == n_outer * n_alt
    dC = np.abs(Q[:, :, 0] - st.Q[:, :, 0]).max()
    assert dC < 1e-6, dC
    assert np.abs(Q - st.Q).max() < 1e-5


def test_single_inner_step_full_ring_is_plain_baoab():
    """n_alt = 1 with no contraction takes the plain step, up to FP32 rounding: the slow forces
    act on contracted-bead positions formed by their own FP32 transform and are summed
    apart from the bonded ones (~1e-8 A after 10 steps; the oracle tolerance is 1e-6 A)."""
    cfg = SMALL
    with qhp.System.from_config(cfg) as a, qhp.System.from_config(cfg) as b:
        qhp.qhp_set_respa(b.h, 1, 0)
        qhp.qhp_step_rpmd(a.h, 10)
        qhp.qhp_step_rpmd(b.h, 10)
        Qa, Pa = qhp.qhp_get_modes(a.h)
        Qb, Pb = qhp.qhp_get_modes(b.h)
    assert np.abs(Qa - Qb).max() < 2e-7
    assert np.abs(Pa - Pb).max() < 1e-5 * np.abs(Pa).max()


def test_respa_graph_direct_and_checkpoint_bitwise():
    cfg = SMALL
    with qhp.System.from_config(cfg) as a, qhp.System.from_config(cfg) as b:
        for s in (a, b):
            qhp.qhp_set_respa(s.h, 4, 2)
        qhp.qhp_set_graph_mode(b.h, False)
        qhp.qhp_step_rpmd(a.h, 6)
        qhp.qhp_step_rpmd(b.h, 6)
        assert np.array_equal(qhp.qhp_get_modes(a.h)[0], qhp.qhp_get_modes(b.h)[0])
        blob = qhp.qhp_get_state(a.h)
        qhp.qhp_step_rpmd(a.h, 3)
        Q1 = qhp.qhp_get_modes(a.h)[0]
        qhp.qhp_set_state(a.h, blob)
        qhp.qhp_set_respa(a.h, 4, 2)
        qhp.qhp_step_rpmd(a.h, 3)
        assert np.array_equal(Q1, qhp.qhp_get_modes(a.h)[0])
        # energies keep the full-ring-polymer definition and leave the trajectory intact
        e = qhp.qhp_get_energy(b.h)
        assert np.isfinite(e.potential)
        qhp.qhp_step_rpmd(b.h, 3)
        assert np.array_equal(Q1, qhp.qhp_get_modes(b.h)[0])


def test_respa_argument_errors():
    cfg = SMALL
    with qhp.System.from_config(cfg) as s:
        for bad in [(2, 3), (2, 16), (-1, 0)]:
            with pytest.raises(qhp.QHPError):
                qhp.qhp_set_respa(s.h, *bad)
        qhp.qhp_set_respa(s.h, 2, 4)
        qhp.qhp_set_respa(s.h, 0, 0)          # back to plain BAOAB
        qhp.qhp_step_rpmd(s.h, 1)
        assert qhp.qhp_get_info(s.h).step == 1
    with qhp.System.from_config(cfg, precision="fp64") as s:
        with pytest.raises(qhp.QHPError):
            qhp.qhp_set_respa(s.h, 2, 4)
