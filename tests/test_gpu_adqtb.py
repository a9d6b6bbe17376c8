"""adQTB on the CUDA path vs the FP64 oracle: colored-noise segments, FDT spectra,
SIMPLE / RATIO adaptation and short trajectories (single bead, mixed precision).

Tolerances come from the arithmetic: the noise, records and FFTs are FP32
(relative rounding ~6e-8 per operation, ~1e-6 after an FFT of a few hundred
points), so colored noise is compared at 2e-5 of its RMS and the per-type FDT
deviation at 1e-4 of the scale m*gamma*C_vv of the spectra it is a difference of.
"""
import math

import numpy as np
import pytest

from oracle import qtb, rpmd
from oracle.units import ACC, CM1_TO_RAD_PS
from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import RunConfig

from oracle_bridge import force_fn, oracle_ff

pytestmark = pytest.mark.gpu

CFG = RunConfig(name="adqtb_64w", n_mol=64, box=12.42, rc=6.0, P=1, dt_fs=0.5, gamma0=20.0,
                thermostat="adqtb", precision="mixed", n_seg=64, omega_cut_cm=15000.0, a_gamma=10.0, seed=99)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


def _gpu(cfg, adapt=qhp.QHP_ADAPT_SIMPLE):
    box = cfg.system()
    th = qhp.make_thermo(kind=qhp.QHP_THERMO_ADQTB, gamma0=cfg.gamma0, dt_fs=cfg.dt_fs, n_seg=cfg.n_seg,
                         omega_cut_cm=cfg.omega_cut_cm, a_gamma=cfg.a_gamma, adapt=adapt, tau_ratio_ps=0.5)
    return qhp.System(box.box, box.types, box.molecule, box.pos, qhp.QHP_MIXED, qhp.make_ff(cfg.rc, cfg.skin),
                      1, cfg.temperature, cfg.seed, th)


def _oracle(cfg, adapt="simple"):
    box = cfg.system()
    ff = oracle_ff(cfg.rc)
    m = ff.masses(box.types)
    prm = qtb.QTBParams(n_seg=cfg.n_seg, dt=cfg.dt_fs * 1e-3, gamma0=cfg.gamma0, temperature=cfg.temperature,
                        omega_cut=cfg.omega_cut_cm * CM1_TO_RAD_PS, a_gamma=cfg.a_gamma, seed=cfg.seed,
                        tau_ratio=0.5)
    bath = qtb.QTB(prm, np.repeat(m, 3), np.repeat(box.types, 3), 2, adapt=adapt)
    st = rpmd.init_state(box.pos, m, rpmd.Params(P=1, temperature=cfg.temperature, dt=prm.dt, gamma0=cfg.gamma0,
                                                 seed=cfg.seed))
    return box, m, prm, bath, st


def test_first_noise_segment():
    box, m, prm, bath, st = _oracle(CFG)
    bath.generate(0)
    with _gpu(CFG) as s:
        u = qhp.qhp_get_qtb_noise(s.h, CFG.n_seg)
    scale = np.sqrt(np.mean(bath.u ** 2))
    assert np.abs(u - bath.u).max() < 2e-5 * scale
    # the noise is far from white: quantum power at high frequency
    assert scale > 1.5 * math.sqrt(prm.kT)


@pytest.mark.parametrize("adapt", ["simple", "ratio"])
def test_segment_adaptation_and_trajectory(adapt):
    code = {"simple": qhp.QHP_ADAPT_SIMPLE, "ratio": qhp.QHP_ADAPT_RATIO}[adapt]
    box, m, prm, bath, st = _oracle(CFG, adapt)
    fn = force_fn(box, CFG.rc)
    n = CFG.n_seg
    for _ in range(n - 1):
        qtb.qtb_step(st, m, bath, fn)
    v_o, F_o = bath.v.copy(), bath.F.copy()
    with _gpu(CFG, code) as s:
        qhp.qhp_step_adqtb(s.h, n - 1)
        v_g, F_g = qhp.qhp_get_qtb_records(s.h, n)
        # records of the segment so far (last row not yet written)
        np.testing.assert_allclose(v_g[: n - 1], v_o[: n - 1], rtol=0, atol=2e-5 * np.abs(v_o).max())
        np.testing.assert_allclose(F_g[: n - 1], F_o[: n - 1], rtol=0, atol=2e-5 * np.abs(F_o).max())
        qhp.qhp_step_adqtb(s.h, 1)                 # completes segment 0: adapt + new noise
        qtb.qtb_step(st, m, bath, fn)
        g = qhp.qhp_get_gamma(s.h, n)
        u1 = qhp.qhp_get_qtb_noise(s.h, n)
        qhp.qhp_step_adqtb(s.h, 6)
        for _ in range(6):
            qtb.qtb_step(st, m, bath, fn)
        C = qhp.qhp_get_centroid(s.h)
    Cvv, _ = qtb.spectra(v_o, F_o, prm)
    scale = np.max(np.repeat(m, 3)[None, :] * prm.gamma0 * Cvv) / ACC
    if adapt == "simple":
        assert np.abs(g - bath.gamma).max() < prm.a_gamma * 1e-4 * scale + 1e-9
    else:
        assert np.abs(g - bath.gamma).max() < 1e-3 * prm.gamma0
    assert not np.allclose(bath.gamma, prm.gamma0)         # adaptation did act
    np.testing.assert_allclose(u1, bath.u, rtol=0, atol=1e-3 * np.sqrt(np.mean(bath.u ** 2)))
    assert np.abs(C - st.Q[:, :, 0]).max() < 1e-5


def test_adqtb_checkpoint_resume_mid_segment():
    with _gpu(CFG) as s:
        qhp.qhp_step_adqtb(s.h, 40)
        blob = qhp.qhp_get_state(s.h)
        qhp.qhp_step_adqtb(s.h, 50)                # crosses a segment end
        Q1, P1 = qhp.qhp_get_modes(s.h)
        g1 = qhp.qhp_get_gamma(s.h, CFG.n_seg)
        qhp.qhp_set_state(s.h, blob)
        qhp.qhp_step_adqtb(s.h, 20)
        qhp.qhp_step_adqtb(s.h, 30)
        Q2, P2 = qhp.qhp_get_modes(s.h)
        g2 = qhp.qhp_get_gamma(s.h, CFG.n_seg)
    assert np.array_equal(Q1, Q2) and np.array_equal(P1, P2) and np.array_equal(g1, g2)


def test_adqtb_direct_launches_match_step_graphs():
    with _gpu(CFG) as a, _gpu(CFG) as b:
        qhp.qhp_set_graph_mode(b.h, False)
        qhp.qhp_step_adqtb(a.h, 70)                # crosses a segment end
        qhp.qhp_step_adqtb(b.h, 70)
        Qa, Pa = qhp.qhp_get_modes(a.h)
        Qb, Pb = qhp.qhp_get_modes(b.h)
        assert np.array_equal(Qa, Qb) and np.array_equal(Pa, Pb)
        assert np.array_equal(qhp.qhp_get_gamma(a.h, CFG.n_seg), qhp.qhp_get_gamma(b.h, CFG.n_seg))


def test_adqtb_rejects_bad_segments():
    box = CFG.system()
    h = qhp.qhp_create_system(box.types, box.molecule, box.pos, box.box, qhp.QHP_MIXED)
    try:
        qhp.qhp_set_forcefield(h, qhp.make_ff(6.0))
        qhp.qhp_set_beads(h, 1, 300.0, 3)
        for bad in (3, 100, 8192):
            with pytest.raises(qhp.QHPError) as e:
                qhp.qhp_set_thermostat(h, qhp.make_thermo(kind=qhp.QHP_THERMO_ADQTB, gamma0=20.0, n_seg=bad))
            assert e.value.code == -1
        with pytest.raises(qhp.QHPError) as e:
            qhp.qhp_step_adqtb(h, 1)                # thermostat is still PILE
        assert e.value.code == -6
    finally:
        qhp.qhp_destroy_system(h)
