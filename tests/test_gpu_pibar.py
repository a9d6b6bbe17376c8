"""PI-BAR (Sec. V, Perspective 2, Eqs. (27)-(28); Appendix A) on the CUDA path against the oracle."""
import math

import numpy as np
import pytest

from oracle import bar, gradients, water
from oracle.units import KB
from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import CONFIGS, small_mixed_config

from oracle_bridge import oracle_ff

pytestmark = pytest.mark.gpu

C1 = CONFIGS["rpmd_fp64_64w"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


def _oracle_state_energies(cfg, xb, theta):
    box = cfg.system()
    ff = gradients.with_params(oracle_ff(cfg.rc), theta)
    U, _, _ = gradients.bead_energy_gradients(xb, box.types, box.molecule, box.box, ff)
    V0, _ = water.potential(xb[0], box.types, box.molecule, box.box, ff)
    return U, V0


@pytest.mark.parametrize("cfg,prec", [(C1, "fp64"), (small_mixed_config(512, P=4), "mixed")], ids=["64w", "512w"])
def test_state_energies_match_oracle(cfg, prec):
    with qhp.System.from_config(cfg, precision=prec) as s:
        qhp.qhp_step_rpmd(s.h, 4)
        thA = qhp.ff_params(s.ff)
        thB = thA * np.array([0.9, 1.01, 0.95, 1.0, 1.1])
        got = qhp.qhp_state_energies(s.h, thA, thB)
        xb = qhp.qhp_get_beads(s.h)
    UA, VA = _oracle_state_energies(cfg, xb, thA)
    UB, VB = _oracle_state_energies(cfg, xb, thB)
    np.testing.assert_allclose(got, [UA, UB, VA, VB], rtol=1e-11)


@pytest.mark.parametrize("nA,nB,beta", [(1000, 1000, 1.68), (37, 5000, 0.5), (20000, 300, 3.0)])
def test_bar_solver_matches_oracle(nA, nB, beta):
    rng = np.random.default_rng(nA + nB)
    dA = rng.normal(0.4, 0.6, nA)
    dB = rng.normal(0.1, 0.6, nB)
    dF, it = qhp.qhp_bar(dA, dB, beta)
    ref, _, _ = bar.pibar(dA, dB, beta)
    assert abs(dF - ref) < 1e-10 and it >= 1


def test_two_state_pibar_from_trajectories():
    """Two parameter sets of the 64-water box (charges x 0.97, LJ eps x 0.9 in state B) sampled
    by their own RPMD trajectories; dU taken on the sampled beads, PI-BAR and single-bead BAR
    on the GPU equal the oracle's on the same samples, and the energies on the samples equal
    the oracle's."""
    cfg = C1
    beta = 1.0 / (KB * cfg.temperature)
    with qhp.System.from_config(cfg) as a, qhp.System.from_config(cfg, seed=cfg.seed + 1) as b:
        thA = qhp.ff_params(a.ff)
        thB = thA * np.array([0.9, 1.0, 0.97, 1.0, 1.0])
        b.set_params(thB)
        dPI = {"A": [], "B": []}
        d1 = {"A": [], "B": []}
        kept = None
        for name, s in (("A", a), ("B", b)):
            qhp.qhp_step_rpmd(s.h, 20)
            for _ in range(12):
                qhp.qhp_step_rpmd(s.h, 5)
                e = qhp.qhp_state_energies(s.h, thA, thB)
                dPI[name].append(e[1] - e[0])
                d1[name].append(e[3] - e[2])
                if kept is None:
                    kept = (qhp.qhp_get_beads(s.h), e)
    F_gpu, _ = qhp.qhp_bar(dPI["A"], dPI["B"], beta)
    F_ref, _, _ = bar.pibar(dPI["A"], dPI["B"], beta)
    assert abs(F_gpu - F_ref) < 1e-10
    F1_gpu, _ = qhp.qhp_bar(d1["A"], d1["B"], beta)
    F1_ref, _, _ = bar.pibar(d1["A"], d1["B"], beta)
    assert abs(F1_gpu - F1_ref) < 1e-10
    assert math.isfinite(F_gpu) and abs(F_gpu - F1_gpu) < 5.0   # same quantity, two estimators
    xb, e = kept
    UA, VA = _oracle_state_energies(cfg, xb, thA)
    UB, VB = _oracle_state_energies(cfg, xb, thB)
    np.testing.assert_allclose(e, [UA, UB, VA, VB], rtol=1e-11)
