"""Long runs compared by ensemble averages (Eq. (6)) within their statistical errors.

Trajectories of chaotic dynamics part after a few hundred steps, so beyond the 10-step
trajectory parity the paths are compared by what they sample:
- RPMD (Sec. II.A): <U_P> (Eq. (3)), <KE_cv> (the centroid-virial estimator) and the mean O-H
  bead distance on the 64-water box, P = 8, from the FP64 path and the mixed path.  The FP64
  path equals the oracle step for step (10-step parity at 1e-10 A); the mixed path keeps its
  bead positions, pair arithmetic and the fluctuation-mode projection in FP32, so this is the
  check that those departures from FP64 do not bias the ensemble.
- adQTB (Sec. II.B): the kinetic energy per atom of each species, <p^2/2m>, from the mixed CUDA
  path and from the FP64 oracle, single bead, fixed gamma = gamma_0 (the adaptation has its own
  parity tests; here the stationary colored-noise sampling is compared).
- NVE (no thermostat): the ring-polymer Hamiltonian H_P = sum P^2/2m + springs + U_P drifts
  no more on the mixed path than on the FP64 path.

Errors: block averages over 20 blocks give sigma for each run; two runs agree when
|a - b| < 3 sqrt(sigma_a^2 + sigma_b^2).  Runs with one seed share their early noise, which
only makes that bound looser.
"""
import math

import numpy as np
import pytest

from oracle import qtb, rpmd
from oracle.units import CM1_TO_RAD_PS
from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import CONFIGS, RunConfig

from oracle_bridge import force_fn, oracle_ff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


def _block(x, nb=20):
    x = np.asarray(x, dtype=float)
    b = x[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(nb))


def _agree(a, b, name):
    (ma, sa), (mb, sb) = a, b
    assert abs(ma - mb) < 3.0 * math.hypot(sa, sb), (name, ma, sa, mb, sb)


def _r_oh(xb, L):
    """Mean O-H distance over beads and the two bonds of every molecule (minimum image)."""
    o = xb[:, 0::3, :]
    out = []
    for k in (1, 2):
        d = xb[:, k::3, :] - o
        d -= L * np.rint(d / L)
        out.append(np.linalg.norm(d, axis=-1))
    return float(np.mean(out))


def _rpmd_run(precision, steps, burn, every):
    cfg = CONFIGS["rpmd_fp64_64w"]
    box = cfg.system()
    th = qhp.make_thermo(kind=qhp.QHP_THERMO_PILE, gamma0=10.0, dt_fs=0.5)
    prec = qhp.QHP_FP64 if precision == "fp64" else qhp.QHP_MIXED
    up, kcv, roh = [], [], []
    with qhp.System(box.box, box.types, box.molecule, box.pos, prec, qhp.make_ff(cfg.rc, cfg.skin), 8, 300.0, 2024,
                    th) as s:
        qhp.qhp_step_rpmd(s.h, burn)
        for _ in range(steps // every):
            qhp.qhp_step_rpmd(s.h, every)
            e = qhp.qhp_get_energy(s.h)
            up.append(e.potential / box.n_mol)
            kcv.append(e.kinetic_cv / box.n_mol)
            roh.append(_r_oh(qhp.qhp_get_beads(s.h), box.box))
    return _block(up), _block(kcv), _block(roh)


def test_rpmd_ensemble_averages_fp64_and_mixed_paths_agree():
    """20 ps per path (40,000 steps of 0.5 fs after 1 ps), PILE with gamma_0 = 10 ps^-1."""
    f = _rpmd_run("fp64", 40000, 2000, 20)
    m = _rpmd_run("mixed", 40000, 2000, 20)
    for k, name in enumerate(("U_P per molecule", "KE_cv per molecule", "r_OH")):
        _agree(f[k], m[k], name)
    # the comparison resolves something: errors well below the quantities' thermal scale
    assert f[0][1] < 0.05 and f[1][1] < 0.05 and f[2][1] < 2e-4, f


@pytest.mark.slow
def test_adqtb_kinetic_energy_per_species_gpu_and_oracle_agree():
    """8 ps (16,000 steps) on each side after 1 ps, gamma fixed at gamma_0 = 20 ps^-1."""
    cfg = RunConfig(name="adqtb_64w", n_mol=64, box=12.42, rc=6.0, P=1, dt_fs=0.5, gamma0=20.0, thermostat="adqtb",
                    precision="mixed", n_seg=64, omega_cut_cm=15000.0, a_gamma=10.0, seed=808)
    box = cfg.system()
    m = oracle_ff(cfg.rc).masses(box.types)
    steps, burn, every = 16000, 2000, 10
    # oracle
    prm = qtb.QTBParams(n_seg=cfg.n_seg, dt=cfg.dt_fs * 1e-3, gamma0=cfg.gamma0, temperature=cfg.temperature,
                        omega_cut=cfg.omega_cut_cm * CM1_TO_RAD_PS, a_gamma=cfg.a_gamma, seed=cfg.seed)
    bath = qtb.QTB(prm, np.repeat(m, 3), np.repeat(box.types, 3), 2, adapt="none")
    st = rpmd.init_state(box.pos, m, rpmd.Params(P=1, temperature=cfg.temperature, dt=prm.dt, gamma0=cfg.gamma0,
                                                 seed=cfg.seed))
    fn = force_fn(box, cfg.rc)
    ko, kh = [], []
    ke_atom = lambda p: np.sum(p ** 2, axis=-1) / (2.0 * m) / 418.4
    for k in range(burn + steps):
        qtb.qtb_step(st, m, bath, fn)
        if k >= burn and (k - burn) % every == every - 1:
            e = ke_atom(st.Pm[:, :, 0])
            ko.append(e[box.types == 0].mean())
            kh.append(e[box.types == 1].mean())
    # GPU
    th = qhp.make_thermo(kind=qhp.QHP_THERMO_ADQTB, gamma0=cfg.gamma0, dt_fs=cfg.dt_fs, n_seg=cfg.n_seg,
                         omega_cut_cm=cfg.omega_cut_cm, a_gamma=cfg.a_gamma, adapt=qhp.QHP_ADAPT_NONE)
    go, gh = [], []
    with qhp.System(box.box, box.types, box.molecule, box.pos, qhp.QHP_MIXED, qhp.make_ff(cfg.rc, cfg.skin), 1,
                    cfg.temperature, cfg.seed, th) as s:
        qhp.qhp_step_adqtb(s.h, burn)
        for _ in range(steps // every):
            qhp.qhp_step_adqtb(s.h, every)
            _, Pm = qhp.qhp_get_modes(s.h)
            e = ke_atom(Pm[:, :, 0])
            go.append(e[box.types == 0].mean())
            gh.append(e[box.types == 1].mean())
    _agree(_block(ko), _block(go), "KE per O atom")
    _agree(_block(kh), _block(gh), "KE per H atom")
    # quantum kinetic energy of H well above the classical 3kT/2 (the bath does its job)
    assert _block(gh)[0] > 2.0 * 1.5 * 0.0019872041 * cfg.temperature


def _nve_drift(precision, steps, every):
    cfg = CONFIGS["rpmd_fp64_64w"]
    box = cfg.system()
    th = qhp.make_thermo(kind=qhp.QHP_THERMO_NVE, gamma0=0.0, dt_fs=0.25)
    prec = qhp.QHP_FP64 if precision == "fp64" else qhp.QHP_MIXED
    t, h = [], []
    with qhp.System(box.box, box.types, box.molecule, box.pos, prec, qhp.make_ff(cfg.rc, cfg.skin), 8, 300.0, 77,
                    th) as s:
        for k in range(steps // every + 1):
            if k:
                qhp.qhp_step_rpmd(s.h, every)
            e = qhp.qhp_get_energy(s.h)
            t.append(k * every * 0.25e-3)
            h.append(e.potential + e.spring + e.kinetic_nm)
    t, h = np.array(t), np.array(h)
    slope = np.polyfit(t, h, 1)[0]                    # kcal/mol per ps
    return slope, float(np.max(np.abs(h - h[0]))), float(np.std(h))


def test_nve_ring_polymer_energy_drift_mixed_path_not_above_fp64_path():
    """100,000 steps of 0.25 fs (25 ps) of Eq. (9) without thermostat, P = 8, 64 waters."""
    sf, mf, stdf = _nve_drift("fp64", 100000, 2000)
    sm, mm, stdm = _nve_drift("mixed", 100000, 2000)
    print(f"NVE H_P drift: fp64 {sf:.3e} kcal/mol/ps (max dev {mf:.3e}, std {stdf:.3e}); "
          f"mixed {sm:.3e} (max dev {mm:.3e}, std {stdm:.3e})")
    # 192 atoms: a drift of 0.05 kcal/mol/ps is 2.6e-4 kcal/mol per atom per ps
    assert abs(sf) < 0.05 and abs(sm) < 0.05, (sf, sm)
    assert mm < 3.0 * mf + 0.05, (mf, mm)
