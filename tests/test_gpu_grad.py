"""Differentiation: the gradient kernels and the segment adjoint against the FP64 oracle
and against central differences of the CUDA path itself.

Tolerances: energy 1e-11 relative, dU/dx 1e-11 RMS relative, dU/dtheta 1e-10
relative (FP64 against FP64, different summation orders); trajectory gradients
against central differences with h = 1e-4 relative: 2e-6 relative to the largest
component (the differences' own truncation error is ~h^2).
"""
import numpy as np
import pytest
import torch

from oracle import gradients as OG
from oracle import rpmd
from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.autograd import bead_energy, segment_average
from paper_2212_03137_b300.workloads import CONFIGS, small_mixed_config

from oracle_bridge import oracle_ff, oracle_params, rms_rel

pytestmark = pytest.mark.gpu

C1 = CONFIGS["rpmd_fp64_64w"]
C5 = CONFIGS["grad_216w"]
LISTBOX = small_mixed_config(512, P=4)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


def _oracle_energy(cfg, xb):
    box = cfg.system()
    return OG.bead_energy_gradients(xb, box.types, box.molecule, box.box, oracle_ff(cfg.rc))


@pytest.mark.parametrize("cfg,prec", [(C5, "fp64"), (LISTBOX, "mixed")], ids=["allpairs_216w_P16", "list_512w_P4"])
def test_energy_gradients_match_oracle(cfg, prec):
    with qhp.System.from_config(cfg, precision=prec) as s:
        qhp.qhp_step_rpmd(s.h, 3)
        E, gx, gt = qhp.qhp_energy_grad(s.h)
        xb = qhp.qhp_get_beads(s.h)
        assert qhp.qhp_get_info(s.h).list_mode == (1 if cfg is LISTBOX else 0)
    Eo, gxo, gto = _oracle_energy(cfg, xb)
    assert abs(E - Eo) < 1e-11 * abs(Eo)
    assert rms_rel(gx, gxo) < 1e-11
    np.testing.assert_allclose(gt, gto, rtol=1e-10)


def test_energy_grad_device_takes_positions():
    cfg = C5
    rng = np.random.default_rng(3)
    with qhp.System.from_config(cfg) as s:
        xb = qhp.qhp_get_beads(s.h) + 0.02 * rng.standard_normal((cfg.P, 3 * cfg.n_mol, 3))
        x = torch.tensor(xb, dtype=torch.float64, device="cuda")
        gx = torch.empty_like(x)
        qhp.qhp_set_stream(s.h, torch.cuda.current_stream().cuda_stream)
        E, gt = qhp.qhp_energy_grad_device(s.h, x.data_ptr(), gx.data_ptr())
        np.testing.assert_allclose(qhp.qhp_get_beads(s.h), xb, atol=1e-12)
    Eo, gxo, gto = _oracle_energy(cfg, xb)
    assert abs(E - Eo) < 1e-11 * abs(Eo)
    assert rms_rel(gx.cpu().numpy(), gxo) < 1e-11
    np.testing.assert_allclose(gt, gto, rtol=1e-10)


def test_autograd_backward_matches_central_differences():
    cfg = C5
    with qhp.System.from_config(cfg) as s:
        x0 = torch.tensor(qhp.qhp_get_beads(s.h), dtype=torch.float64, device="cuda")
        th0 = torch.tensor(qhp.ff_params(s.ff), dtype=torch.float64)
        x = x0.clone().requires_grad_(True)
        th = th0.clone().requires_grad_(True)
        E = bead_energy(s, x, th)
        E.backward()
        u = torch.randn(x0.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
        h = 1e-5
        fd = (bead_energy(s, x0 + h * u, th0) - bead_energy(s, x0 - h * u, th0)).item() / (2 * h)
        an = float(torch.sum(x.grad * u))
        assert abs(fd - an) < 1e-7 * abs(an)
        for k in range(5):
            hk = 1e-6 * abs(float(th0[k]))
            tp, tm = th0.clone(), th0.clone()
            tp[k] += hk
            tm[k] -= hk
            fdk = (bead_energy(s, x0, tp) - bead_energy(s, x0, tm)).item() / (2 * hk)
            assert abs(fdk - float(th.grad[k])) < 1e-6 * abs(fdk) + 1e-9, (k, fdk, float(th.grad[k]))


@pytest.mark.parametrize("which", [OG.OBS_CENTROID_ENERGY, OG.OBS_MEAN_OH], ids=["centroid_V", "mean_OH"])
def test_segment_gradient_matches_oracle(which):
    """64 waters, P = 8, 12 PILE steps: the adjoint against central differences of oracle trajectories."""
    cfg, K = C1, 12
    with qhp.System.from_config(cfg) as s:
        J, g = qhp.qhp_segment_grad(s.h, K, 5, which)
        Q, P = qhp.qhp_get_modes(s.h)
        assert qhp.qhp_get_info(s.h).step == 0            # the system is left as it was
    box = cfg.system()
    ff = oracle_ff(cfg.rc)
    prm = oracle_params(cfg)
    st0 = rpmd.init_state(box.pos, ff.masses(box.types), prm)
    np.testing.assert_allclose(Q, st0.Q, atol=1e-12)
    Jo = OG.segment_objective(st0, prm, box.types, box.molecule, box.box, ff, K, which)
    go = OG.segment_gradient_fd(st0, prm, box.types, box.molecule, box.box, ff, K, which)
    assert abs(J - Jo) < 1e-9 * abs(Jo)
    assert np.max(np.abs(g - go)) < 2e-6 * np.max(np.abs(go)), (g, go)


@pytest.mark.parametrize("which", [0, 1], ids=["centroid_V", "mean_OH"])
def test_segment_gradient_full_size_against_gpu_differences(which):
    """216 waters, P = 16, K = 200: the adjoint against central differences (h = 1e-4
    relative) of the CUDA trajectory itself; checkpoint spacing does not change a bit."""
    cfg, K = C5, 200
    with qhp.System.from_config(cfg) as s:
        th0 = qhp.ff_params(s.ff)
        J, g = qhp.qhp_segment_grad(s.h, K, 15, which)
        J1, g1 = qhp.qhp_segment_grad(s.h, K, K, which)
        assert J == J1 and np.array_equal(g, g1)
        fd = np.zeros(5)
        for k in range(5):
            tp, tm = th0.copy(), th0.copy()
            tp[k] *= 1 + 1e-4
            tm[k] *= 1 - 1e-4
            s.set_params(tp)
            Jp, _ = qhp.qhp_segment_grad(s.h, K, K, which)
            s.set_params(tm)
            Jm, _ = qhp.qhp_segment_grad(s.h, K, K, which)
            fd[k] = (Jp - Jm) / (tp[k] - tm[k])
        s.set_params(th0)
    assert np.max(np.abs(g - fd)) < 2e-5 * np.max(np.abs(fd)), (g, fd)


def test_segment_average_autograd_and_errors():
    cfg = C1
    with qhp.System.from_config(cfg) as s:
        th = torch.tensor(qhp.ff_params(s.ff), dtype=torch.float64, requires_grad=True)
        J = segment_average(s, th, 6, 1)
        J.backward()
        J2, g2 = qhp.qhp_segment_grad(s.h, 6, 3, 1)
        assert float(J.detach()) == J2 and np.array_equal(th.grad.numpy(), g2)
        with pytest.raises(qhp.QHPError):
            qhp.qhp_segment_grad(s.h, 0, 1, 0)
        with pytest.raises(qhp.QHPError):
            qhp.qhp_segment_grad(s.h, 4, 1, 2)
    with qhp.System.from_config(LISTBOX) as s:   # mixed precision: no segment adjoint
        with pytest.raises(qhp.QHPError):
            qhp.qhp_segment_grad(s.h, 4, 2, 0)
        bad = qhp.ff_with_params(s.ff, qhp.ff_params(s.ff))
        bad.rc = bad.rc - 0.5
        with pytest.raises(qhp.QHPError):
            qhp.qhp_set_forcefield(s.h, bad)
