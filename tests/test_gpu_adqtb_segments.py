"""adQTB segment ends on the CUDA path at every spectra specialisation, against the oracle.

At the end of a segment the GPU forms the spectra of the segment's records (Eq. (22)), the
per-type FDT deviation (Eq. (21), averaged over the type's dofs, Sec. III.B.2), adapts gamma
(SIMPLE, Eq. (23), or RATIO, Eqs. (24)-(26)) and generates the next colored-noise segment
(Sec. III.B.1).  Here the oracle recomputes each of those from the GPU's own records of the
segment, which isolates the end-of-segment kernels from the trajectory:
- the spectra kernel is specialised on n_seg (bins per thread 1, 2, 3 and 5 for n_seg = 256,
  512, 1024 and 2048), so each of those runs once on a 64-water box;
- the 8,000-water box runs the 72,000-water workload's segment length (1024) with all 72,000 dofs
  averaged.

Tolerances: the records and FFTs are FP32 (~1e-6 relative after an FFT of a few thousand
points) and the per-type sums FP64.  Delta_bar is a difference of two spectra of scale
m gamma C_vv, so gamma after SIMPLE is compared at a_gamma * 1e-4 of that scale, gamma after
RATIO at 1e-4 relative plus the FFT noise floor of weak bins (see the test), fdt_delta at 1e-4
relative, and the next noise segment at 1e-3 of its RMS (its filter is built from the gamma,
which carries the differences above).
"""
import numpy as np
import pytest

from oracle import qtb
from oracle.units import ACC, CM1_TO_RAD_PS
from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import RunConfig

from oracle_bridge import oracle_ff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


def _cfg(n_mol, box, n_seg):
    return RunConfig(name=f"adqtb_{n_mol}w_seg{n_seg}", n_mol=n_mol, box=box, rc=6.0 if box < 20 else 9.0, P=1,
                     dt_fs=0.5, gamma0=20.0, thermostat="adqtb", precision="mixed", n_seg=n_seg,
                     omega_cut_cm=15000.0, a_gamma=10.0, seed=321)


def _gpu(cfg, adapt):
    box = cfg.system()
    th = qhp.make_thermo(kind=qhp.QHP_THERMO_ADQTB, gamma0=cfg.gamma0, dt_fs=cfg.dt_fs, n_seg=cfg.n_seg,
                         omega_cut_cm=cfg.omega_cut_cm, a_gamma=cfg.a_gamma, adapt=adapt, tau_ratio_ps=0.5)
    return qhp.System(box.box, box.types, box.molecule, box.pos, qhp.QHP_MIXED, qhp.make_ff(cfg.rc, cfg.skin), 1,
                      cfg.temperature, cfg.seed, th)


def _prm(cfg):
    return qtb.QTBParams(n_seg=cfg.n_seg, dt=cfg.dt_fs * 1e-3, gamma0=cfg.gamma0, temperature=cfg.temperature,
                         omega_cut=cfg.omega_cut_cm * CM1_TO_RAD_PS, a_gamma=cfg.a_gamma, seed=cfg.seed,
                         tau_ratio=0.5)


def _type_mean_spectra(v, F, dof_type, prm, chunk=6000):
    """Type means of C_vv and Re C_vF (Eq. (22); the average of Sec. III.B.2), in dof chunks."""
    nb = prm.n_seg + 1
    svv, svf, cnt = np.zeros((2, nb)), np.zeros((2, nb)), np.zeros(2)
    for a in range(0, v.shape[1], chunk):
        Cvv, CvF = qtb.spectra(v[:, a:a + chunk].astype(np.float64), F[:, a:a + chunk].astype(np.float64), prm)
        for z in (0, 1):
            sel = dof_type[a:a + chunk] == z
            svv[z] += Cvv[:, sel].sum(axis=1)
            svf[z] += CvF.real[:, sel].sum(axis=1)
            cnt[z] += sel.sum()
    return svv / cnt[:, None], svf / cnt[:, None]


def _segment_end(cfg, adapt, n_sample_dofs=24):
    code = {"simple": qhp.QHP_ADAPT_SIMPLE, "ratio": qhp.QHP_ADAPT_RATIO}[adapt]
    prm = _prm(cfg)
    box = cfg.system()
    m = oracle_ff(cfg.rc).masses(box.types)
    m_type = np.array([m[box.types == 0][0], m[box.types == 1][0]])
    dof_type = np.repeat(box.types, 3)
    n = cfg.n_seg
    with _gpu(cfg, code) as s:
        qhp.qhp_step_adqtb(s.h, n)                      # segment 0, its end: spectra, adaptation, noise 1
        v, F = qhp.qhp_get_qtb_records(s.h, n)          # the records of segment 0
        g_gpu = qhp.qhp_get_gamma(s.h, n)
        u1 = qhp.qhp_get_qtb_noise(s.h, n)
        e = qhp.qhp_get_energy(s.h)
    Cvv, CvF = _type_mean_spectra(v, F, dof_type, prm)
    g0 = np.full((2, n + 1), prm.gamma0)
    dbar = (m_type[:, None] * g0 * Cvv - CvF) / ACC       # Eq. (21), type means
    scale = float(np.max(m_type[:, None] * prm.gamma0 * Cvv)) / ACC
    if adapt == "simple":
        g_want = qtb.adapt_simple(g0, dbar, prm)
        assert np.abs(g_gpu - g_want).max() < prm.a_gamma * 1e-4 * scale + 1e-9
    else:
        g_want, _, _ = qtb.adapt_ratio(None, None, Cvv, CvF, m_type, prm, True)
        # RATIO divides two spectra: where C_vv lies far below its peak the FP32 FFT's absolute
        # noise floor (about 1e-6 of the peak) dominates the bin, so each bin is allowed
        # 1e-4 + 2e-6 C_vv,max / C_vv relative; the bulk of the bins must agree to 1e-5
        rel = np.abs(g_gpu - g_want) / np.abs(g_want)
        bound = 1e-4 + 2e-6 * Cvv.max(axis=1, keepdims=True) / np.maximum(Cvv, 1e-300)
        worst = np.unravel_index(np.argmax(rel / bound), rel.shape)
        assert np.all(rel <= bound), (worst, rel[worst], bound[worst])
        assert np.median(rel) < 1e-5, np.median(rel)
    assert not np.allclose(g_want, prm.gamma0)           # the adaptation did act
    # fdt_delta: mean |Delta_bar| over both types and all bins of the segment just ended
    want = float(np.mean(np.abs(dbar)))
    assert abs(e.fdt_delta - want) < 1e-4 * want + 1e-12 * scale, (e.fdt_delta, want)
    # the next segment's noise on sampled dofs, filtered with the adapted gamma
    rng = np.random.default_rng(cfg.n_seg)
    dofs = np.sort(rng.choice(len(dof_type), size=min(n_sample_dofs, len(dof_type)), replace=False))
    taps = np.stack([qtb.filter_taps(qtb.noise_power(g_want[z], prm), prm) for z in (0, 1)])[dof_type[dofs]]
    u_want = qtb.colored_segment_fft(1, taps, dofs, prm)
    rms = np.sqrt(np.mean(u_want ** 2))
    np.testing.assert_allclose(u1[:, dofs], u_want, rtol=0, atol=1e-3 * rms)


@pytest.mark.parametrize("n_seg", [256, 512, 1024, 2048])
@pytest.mark.parametrize("adapt", ["simple", "ratio"])
def test_segment_end_every_spectra_specialisation(n_seg, adapt):
    _segment_end(_cfg(64, 12.42, n_seg), adapt)


@pytest.mark.slow
def test_segment_end_8000_waters_config_segment_length():
    _segment_end(_cfg(8000, 62.1, 1024), "simple", n_sample_dofs=32)
