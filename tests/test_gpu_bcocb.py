"""BCOCB (Cayley free ring-polymer flow, Sec. III.A.1) on the CUDA path against the oracle."""
import numpy as np
import pytest

from oracle import rpmd
from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import CONFIGS, small_mixed_config

from oracle_bridge import force_fn, oracle_ff

pytestmark = pytest.mark.gpu

C1 = CONFIGS["rpmd_fp64_64w"].with_(extra={"integrator": "bcocb"})
SMALL32 = small_mixed_config(512, P=32).with_(extra={"integrator": "bcocb"})


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


def _oracle(cfg):
    box = cfg.system()
    ff = oracle_ff(cfg.rc)
    prm = rpmd.Params(P=cfg.P, temperature=cfg.temperature, dt=cfg.dt_fs * 1e-3, gamma0=cfg.gamma0, seed=cfg.seed,
                      integrator="bcocb")
    m = ff.masses(box.types)
    return box, ff, prm, m, rpmd.init_state(box.pos, m, prm)


@pytest.mark.parametrize("cfg,prec,tol", [(C1, "fp64", 1e-10), (SMALL32, "mixed", 1e-6)], ids=["fp64_P8", "mixed_P32"])
def test_bcocb_ten_steps_match_oracle(cfg, prec, tol):
    box, ff, prm, m, st = _oracle(cfg)
    fn = force_fn(box, cfg.rc)
    for _ in range(10):
        rpmd.step(st, prm, m, fn)
    with qhp.System.from_config(cfg, precision=prec) as s:
        qhp.qhp_step_rpmd(s.h, 10)
        Q, _ = qhp.qhp_get_modes(s.h)
    assert np.abs(Q[:, :, 0] - st.Q[:, :, 0]).max() < tol
    assert np.abs(Q - st.Q).max() < 10 * tol


def test_bcocb_differs_from_exact_flow():
    """The two integrators are different maps: after a few steps the fluctuation modes differ."""
    cfg = C1
    with qhp.System.from_config(cfg) as a, qhp.System.from_config(cfg.with_(extra={})) as b:
        qhp.qhp_step_rpmd(a.h, 5)
        qhp.qhp_step_rpmd(b.h, 5)
        Qa, _ = qhp.qhp_get_modes(a.h)
        Qb, _ = qhp.qhp_get_modes(b.h)
    assert np.abs(Qa[:, :, 1:] - Qb[:, :, 1:]).max() > 1e-6


def test_bcocb_free_ring_polymer_conserves_mode_energies():
    cfg = C1
    box = cfg.system()
    ff = qhp.make_ff(cfg.rc, eps=0.0, q_O=0.0, k_b=0.0, k_theta=0.0)
    th = qhp.make_thermo(kind=qhp.QHP_THERMO_NVE, gamma0=0.0, dt_fs=1.0, integrator=qhp.QHP_INTEGRATOR_BCOCB)
    with qhp.System(box.box, box.types, box.molecule, box.pos, qhp.QHP_FP64, ff, 32, 300.0, 5, th) as s:
        def energies():
            Q, Pm = qhp.qhp_get_modes(s.h)
            prm = rpmd.Params(P=32, temperature=300.0, dt=1e-3, gamma0=0.0, seed=5)
            w = prm.omegas()
            m = oracle_ff(cfg.rc).masses(box.types)[:, None, None]
            return 0.5 * Pm[:, :, 1:] ** 2 / m + 0.5 * m * w[None, None, 1:] ** 2 * Q[:, :, 1:] ** 2
        E0 = energies()
        qhp.qhp_step_rpmd(s.h, 2000)
        np.testing.assert_allclose(energies(), E0, rtol=1e-11)
