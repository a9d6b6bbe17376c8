"""Pins for the oracle's RPMD integrator and adQTB thermostat (no GPU).

Closed forms used:
* RPMD on V = 1/2 m w0^2 x^2 at finite P (Eqs. (1), (3)): the modes decouple and
  <x^2>_P = sum_n kT / (m (w0^2 + w_n^2)), which tends to hbar/(2 m w0) coth(beta hbar w0/2);
  momenta have <P_n^2> = m kT for every mode (Eq. (7)).
* Free ring polymer (V = 0, no friction): the exact A flow of Eq. (9) is a rotation in
  (Q_n, P_n/(m w_n)) and conserves every mode's energy.
* adQTB on a harmonic oscillator with gamma = gamma_0 (Sec. II.B):
  m<v^2> = (1/pi) int_0^wcut 2 gamma_0 Theta(w) w^2 / ((w0^2 - w^2)^2 + gamma_0^2 w^2) dw,
  and the FDT deviation of Eq. (21) vanishes (gamma_0 is the fixed point of Eq. (25)).
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import normal_modes as nm
from oracle import philox, qtb, rpmd
from oracle.units import ACC, HBAR, KB


def _ho_run(P, n_atoms=500, steps=4000, burn=400, dt=0.0005, gamma0=50.0, omega0=100.0, mass=1.008, seed=5):
    prm = rpmd.Params(P=P, temperature=300.0, dt=dt, gamma0=gamma0, seed=seed)
    masses = np.full(n_atoms, mass)
    st = rpmd.init_state(np.zeros((n_atoms, 3)), masses, prm)
    fn = rpmd.harmonic_forces(omega0, masses)
    x2, p2 = [], []
    for s in range(steps):
        rpmd.step(st, prm, masses, fn)
        if s >= burn:
            x2.append(np.mean(np.sum(st.Q ** 2, axis=-1)))
            p2.append(np.mean(st.Pm ** 2, axis=(0, 1)))
    return prm, np.array(x2), np.array(p2)


def _block_err(a, nb=20):
    b = a[: len(a) // nb * nb].reshape(nb, -1).mean(axis=1)
    return b.std(ddof=1) / math.sqrt(nb)


def test_rpmd_harmonic_finite_P_closed_form():
    P, omega0, mass = 8, 100.0, 1.008
    prm, x2, p2 = _ho_run(P, omega0=omega0, mass=mass)
    kT = prm.kT * ACC
    w = prm.omegas()
    exact_P = np.sum(kT / (mass * (omega0 ** 2 + w ** 2)))
    err = _block_err(x2)
    assert abs(x2.mean() - exact_P) < 4 * err + 0.003 * exact_P, (x2.mean(), exact_P, err)
    classical = kT / (mass * omega0 ** 2)
    assert exact_P > 1.3 * classical          # the test resolves the quantum effect
    pm = p2.mean(axis=0)
    np.testing.assert_allclose(pm, mass * kT, rtol=0.02)


def test_finite_P_sum_converges_to_quantum_result():
    kT, omega0, m = KB * 300.0 * ACC, 100.0, 1.008
    hb = HBAR * ACC
    exact = hb / (2 * m * omega0) / math.tanh(HBAR * omega0 / (2 * KB * 300.0))
    prev = None
    for P in (8, 32, 128, 1024):
        w = nm.mode_frequencies(P, KB * 300.0, HBAR)
        s = np.sum(kT / (m * (omega0 ** 2 + w ** 2)))
        if prev is not None:
            assert abs(s - exact) < abs(prev - exact)
        prev = s
    assert abs(prev - exact) / exact < 1e-5


def test_free_ring_polymer_conserves_mode_energy():
    P, n = 16, 50
    prm = rpmd.Params(P=P, temperature=300.0, dt=0.0005, gamma0=0.0, seed=3)
    masses = np.linspace(1.0, 16.0, n)
    st = rpmd.init_state(np.zeros((n, 3)), masses, prm)
    w = prm.omegas()
    m = masses[:, None, None]

    def emode(s):
        return s.Pm ** 2 / (2 * m) + 0.5 * m * w ** 2 * s.Q ** 2

    e0 = emode(st)
    Q0, P0 = st.Q.copy(), st.Pm.copy()
    k = 20000
    for _ in range(k):
        rpmd.free_flow(st, prm, masses, 0.5 * prm.dt)
    e1 = emode(st)
    assert np.max(np.abs(e1[..., 1:] - e0[..., 1:]) / e0[..., 1:].max()) < 1e-13
    t = k * 0.5 * prm.dt
    Qexact = Q0[..., 1:] * np.cos(w[1:] * t) + P0[..., 1:] / (m * w[1:]) * np.sin(w[1:] * t)
    np.testing.assert_allclose(st.Q[..., 1:], Qexact, atol=1e-11)
    np.testing.assert_allclose(st.Q[..., 0], Q0[..., 0] + P0[..., 0] * t / m[..., 0], rtol=1e-12)


def _nve_energy_error(cfg, P, dt, t_total):
    """Max |H_P(t) - H_P(0)| of velocity Verlet in normal modes (B A A B, exact free flow, no
    thermostat) on the interacting water box, H_P = sum_n P_n^2/2m + sum_n m w_n^2 Q_n^2/2 + U_P."""
    from oracle import water
    from oracle_bridge import oracle_ff
    box = cfg.system()
    ff = oracle_ff(cfg.rc)
    m = ff.masses(box.types)
    prm = rpmd.Params(P=P, temperature=300.0, dt=dt, gamma0=0.0, seed=11)
    st = rpmd.init_state(box.pos, m, prm)
    fn = water.make_force_fn(box.types, box.molecule, box.box, ff)
    rpmd.evaluate_forces(st, prm, fn)

    def H():
        return rpmd.kinetic_energy(st, m) + rpmd.spring_energy(st, prm, m) + rpmd.potential_estimator(st)

    h0, err = H(), 0.0
    for _ in range(int(round(t_total / dt))):
        rpmd.kick(st, 0.5 * dt)
        rpmd.free_flow(st, prm, m, dt)
        rpmd.evaluate_forces(st, prm, fn)
        rpmd.kick(st, 0.5 * dt)
        err = max(err, abs(H() - h0))
    return err, rpmd.kinetic_energy(st, m)


def test_ring_polymer_hamiltonian_is_conserved_to_second_order():
    """With interactions on and no thermostat, the flow of Eq. (9) conserves
    H_P = sum_n P_n^2/2m + sum_n m w_n^2 Q_n^2/2 + U_P: the projected forces f_n (Eqs. (10)-(11))
    must be exactly -dU_P/dQ_n and U_P must carry its 1/P (Eq. (3)).  Velocity Verlet with the
    exact free flow then keeps H_P to O(dt^2): halving dt quarters the error."""
    from paper_2212_03137_b300.workloads import CONFIGS
    cfg = CONFIGS["rpmd_fp64_64w"]
    e1, ke = _nve_energy_error(cfg, 4, 0.0002, 0.004)
    e2, _ = _nve_energy_error(cfg, 4, 0.0001, 0.004)
    # the error is the integrator's (O-H stretch period ~9 fs, omega dt ~ 0.14 at 0.2 fs), not a
    # drift: a wrong factor in f_n would leave an error that does not scale with dt^2
    assert e1 < 1e-2 * ke, (e1, ke)
    assert 0.2 < e2 / e1 < 0.3, (e1, e2)


def _langevin_momentum_acf(t, w, g):
    """<p(t) p(0)> / (m kT) of a stationary Langevin oscillator dq = p/m dt,
    dp = -m w^2 q dt - g p dt + sqrt(2 g m kT) dW (textbook result; w = 0 is the free particle)."""
    if w == 0.0:
        return np.exp(-g * t)
    d = w * w - 0.25 * g * g
    if abs(d) < 1e-12 * w * w:
        return np.exp(-w * t) * (1.0 - w * t)
    if d > 0:
        w1 = math.sqrt(d)
        return np.exp(-0.5 * g * t) * (np.cos(w1 * t) - 0.5 * g / w1 * np.sin(w1 * t))
    k = math.sqrt(-d)
    return np.exp(-0.5 * g * t) * (np.cosh(k * t) - 0.5 * g / k * np.sinh(k * t))


def test_pile_friction_per_mode_from_momentum_autocorrelation():
    """Eq. (16): gamma_n = max(gamma_0, omega_n) on the fluctuation modes, gamma_0 on the centroid.
    With V = 0 every mode is a Langevin oscillator of frequency omega_n (omega_0 = 0), so the
    stationary momentum autocorrelation of mode n is fixed by (omega_n, gamma_n) alone.  hbar is
    scaled so that omega_P = 20 ps^-1 (omega_n dt <= 0.02: the splitting error is negligible) and
    gamma_0 = 10 ps^-1 < omega_1 = 15.3 ps^-1, so the two branches of the max differ.  The states
    start in the stationary distribution (Eq. (7) momenta, free ring-polymer modes).  The other
    plausible readings (gamma_0 everywhere, 2 omega_n, no centroid friction) miss by > 0.14."""
    P, n_atoms, steps, lags = 8, 64, 6000, 600
    T, gamma0, mass = 300.0, 10.0, 4.0
    prm = rpmd.Params(P=P, temperature=T, dt=0.0005, gamma0=gamma0, seed=9, hbar=P * KB * T / 20.0)
    masses = np.full(n_atoms, mass)
    st = rpmd.init_state(np.zeros((n_atoms, 3)), masses, prm)

    def free(xb):
        return np.zeros(xb.shape[0]), np.zeros_like(xb)

    rec = np.empty((steps, n_atoms * 3, P))
    for s in range(steps):
        rpmd.step(st, prm, masses, free)
        rec[s] = st.Pm.reshape(-1, P)
    f = np.fft.rfft(rec, n=2 * steps, axis=0)
    ac = np.fft.irfft(f * np.conj(f), axis=0)[:lags] / (steps - np.arange(lags))[:, None, None]
    acf = ac.mean(axis=1) / (mass * prm.kT * ACC)          # normalised by the exact <p^2> = m kT
    t = np.arange(lags) * prm.dt
    w = prm.omegas()
    readings = {
        "paper": np.r_[gamma0, np.maximum(gamma0, w[1:])],
        "gamma0 everywhere": np.full(P, gamma0),
        "2 omega_n": np.r_[gamma0, 2.0 * w[1:]],
        "no centroid friction": np.r_[0.0, np.maximum(gamma0, w[1:])],
    }
    dev = {k: np.array([np.max(np.abs(acf[:, n] - _langevin_momentum_acf(t, w[n], g[n]))) for n in range(P)])
           for k, g in readings.items()}
    assert np.all(dev["paper"] < 0.07), dev["paper"]
    for k in ("gamma0 everywhere", "2 omega_n"):
        assert np.all(dev[k][1:] > 0.14), (k, dev[k])
    assert dev["no centroid friction"][0] > 0.5, dev["no centroid friction"]


def test_centroid_virial_estimator_harmonic_identity():
    """For V = 1/2 k x^2 per dof, -(1/2P) sum_b (x_b - Q_0).F_b = (k/2) sum_{n>0} Q_n^2 exactly
    (x_b - Q_0 = sqrt(P) sum_{n>0} T_bn Q_n and sum_b (x_b - Q_0).Q_0 = 0), so the
    centroid-virial kinetic estimator of any mode state is 3N kT/2 + (k/2) sum_{n>0} Q_n^2."""
    P, n, omega0 = 8, 5, 40.0
    prm = rpmd.Params(P=P, temperature=300.0, dt=0.0005, gamma0=1.0, seed=2)
    masses = np.linspace(1.0, 16.0, n)
    rng = np.random.default_rng(4)
    st = rpmd.init_state(rng.standard_normal((n, 3)), masses, prm)
    st.Q[..., 1:] = 0.3 * rng.standard_normal(st.Q[..., 1:].shape)
    rpmd.evaluate_forces(st, prm, rpmd.harmonic_forces(omega0, masses))
    k = masses[:, None] * omega0 ** 2 / ACC
    expect = 1.5 * n * prm.kT + 0.5 * float(np.sum(k * np.sum(st.Q[..., 1:] ** 2, axis=-1)))
    assert abs(rpmd.centroid_virial_kinetic(st, prm) - expect) < 1e-12 * abs(expect)


def test_single_bead_step_is_classical_baoab():
    """P = 1: one step equals textbook BAOAB (Leimkuhler-Matthews) with the same normals."""
    n = 20
    prm = rpmd.Params(P=1, temperature=300.0, dt=0.001, gamma0=5.0, seed=17)
    masses = np.full(n, 15.999)
    rng = np.random.default_rng(0)
    x0 = rng.standard_normal((n, 3))
    fn = rpmd.harmonic_forces(30.0, masses)
    st = rpmd.init_state(x0, masses, prm)
    x, p = x0.copy(), st.Pm[..., 0].copy()
    rpmd.step(st, prm, masses, fn)
    k = masses[:, None] * 900.0 / ACC
    m = masses[:, None]
    h = prm.dt
    p = p + 0.5 * h * ACC * (-k * x)
    x = x + 0.5 * h * p / m
    c1 = math.exp(-prm.gamma0 * h)
    R = philox.normals(prm.seed, np.arange(3 * n, dtype=np.uint64).reshape(n, 3), 0, philox.TAG_OSTEP)
    p = c1 * p + np.sqrt((1 - c1 ** 2) * m * KB * 300.0 * ACC) * R
    x = x + 0.5 * h * p / m
    p = p + 0.5 * h * ACC * (-k * x)
    np.testing.assert_allclose(st.Q[..., 0], x, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(st.Pm[..., 0], p, rtol=1e-13, atol=1e-14)


def test_initial_modes_follow_free_ring_polymer_gaussian():
    P, n = 8, 4000
    prm = rpmd.Params(P=P, temperature=300.0, dt=0.0005, gamma0=1.0, seed=21)
    masses = np.full(n, 1.008)
    st = rpmd.init_state(np.zeros((n, 3)), masses, prm)
    kT = prm.kT * ACC
    w = prm.omegas()
    var_q = st.Q[..., 1:].reshape(-1, P - 1).var(axis=0)
    np.testing.assert_allclose(var_q, kT / (1.008 * w[1:] ** 2), rtol=0.06)
    np.testing.assert_allclose(st.Pm.reshape(-1, P).var(axis=0), 1.008 * kT, rtol=0.06)


# ------------------------------------------------------------------- adQTB

def _qtb_prm(**kw):
    base = dict(n_seg=64, dt=0.0005, gamma0=20.0, temperature=300.0, omega_cut=np.inf, seed=77)
    base.update(kw)
    return qtb.QTBParams(**base)


def test_colored_noise_fft_equals_direct_convolution():
    prm = _qtb_prm(n_seg=16, omega_cut=2000.0)
    gam = np.full(prm.n_seg + 1, prm.gamma0) * (1 + 0.3 * np.sin(np.arange(prm.n_seg + 1)))
    taps = np.stack([qtb.filter_taps(qtb.noise_power(gam, prm), prm)] * 5)
    dofs = np.arange(5)
    for k in (0, 3):
        np.testing.assert_allclose(qtb.colored_segment_fft(k, taps, dofs, prm),
                                   qtb.colored_segment_direct(k, taps, dofs, prm), atol=1e-13)


def test_filter_is_even_and_obeys_parseval():
    prm = _qtb_prm(n_seg=128, omega_cut=1500.0)
    S = qtb.noise_power(np.full(prm.n_seg + 1, prm.gamma0), prm)
    h = qtb.filter_taps(S, prm)
    l = np.arange(-prm.n_seg, prm.n_seg)
    hl = dict(zip(l, h))
    assert max(abs(hl[k] - hl[-k]) for k in range(1, prm.n_seg)) < 1e-15
    j = np.arange(prm.n_f)
    full = S[np.minimum(j, prm.n_f - j)]
    np.testing.assert_allclose(np.sum(h ** 2), full.mean(), rtol=1e-12)


def test_classical_limit_gives_white_noise():
    """hbar -> 0, no frequency cutoff, gamma = gamma_0: S = kT, h = sqrt(kT) delta, u = sqrt(kT) xi."""
    prm = _qtb_prm(n_seg=32, hbar=1e-12)
    h = qtb.filter_taps(qtb.noise_power(np.full(prm.n_seg + 1, prm.gamma0), prm), prm)
    taps = np.stack([h] * 3)
    u = qtb.colored_segment_fft(2, taps, np.arange(3), prm)
    xi = qtb.white(prm, np.arange(3), np.arange(2 * prm.n_seg, 3 * prm.n_seg))
    np.testing.assert_allclose(u, math.sqrt(prm.kT) * xi, atol=1e-13)


def test_theta_limits():
    kT = KB * 300.0
    assert qtb.theta(np.array([0.0]), kT, HBAR)[0] == kT
    w = np.array([1e-6, 5000.0])
    t = qtb.theta(w, kT, HBAR)
    np.testing.assert_allclose(t[0], kT, rtol=1e-9)
    np.testing.assert_allclose(t[1], HBAR * 5000.0 / 2, rtol=1e-9)


def test_spectrum_normalisation_white_velocity():
    """For white v of variance s^2, E C_vv = dt s^2 at every bin."""
    prm = _qtb_prm(n_seg=256)
    rng = np.random.default_rng(1)
    v = rng.standard_normal((prm.n_seg, 4000)) * 2.0
    Cvv, CvF = qtb.spectra(v, v, prm)
    np.testing.assert_allclose(Cvv.mean(axis=1)[5:-5].mean(), prm.dt * 4.0, rtol=0.01)
    np.testing.assert_allclose(CvF.real, Cvv, rtol=1e-12)


def test_gamma_min_clamp_and_ratio_fixed_point():
    prm = _qtb_prm()
    g = np.full((2, prm.n_seg + 1), prm.gamma0)
    out = qtb.adapt_simple(g, np.full_like(g, 1e9), prm)
    assert np.all(out == prm.gamma_min_frac * prm.gamma0)
    m = np.array([15.999, 1.008])
    Cvv = np.abs(np.random.default_rng(0).standard_normal((2, prm.n_seg + 1))) + 0.1
    CvF = m[:, None] * prm.gamma0 * Cvv
    gam, _, _ = qtb.adapt_ratio(None, None, Cvv, CvF, m, prm, True)
    np.testing.assert_allclose(gam, prm.gamma0, rtol=1e-14)


def _qtb_ho(omega0, n_atoms, n_segments, prm, adapt="none"):
    masses = np.full(n_atoms, 1.008)
    st = rpmd.init_state(np.zeros((n_atoms, 3)), masses, rpmd.Params(P=1, temperature=prm.temperature,
                                                                       dt=prm.dt, gamma0=prm.gamma0, seed=prm.seed))
    bath = qtb.QTB(prm, np.repeat(masses, 3), np.zeros(3 * n_atoms, dtype=int), 1, adapt=adapt)
    fn = rpmd.harmonic_forces(omega0, masses)
    ke, deltas, ratios = [], [], []
    w = qtb.omega_bins(prm)
    band = (w > omega0 - 2 * prm.gamma0) & (w < omega0 + 2 * prm.gamma0)
    for s in range(n_segments * prm.n_seg):
        qtb.qtb_step(st, masses, bath, fn)
        if s >= prm.n_seg:
            ke.append(np.mean(st.Pm ** 2 / (2 * masses[:, None, None])) / ACC)
        if (s + 1) % prm.n_seg == 0 and s >= prm.n_seg:
            Cvv, CvF = qtb.spectra(bath.v, bath.F, prm)
            deltas.append(bath.last_delta_bar[0][band])
            ratios.append(CvF.real.mean(axis=1)[band].sum() / (1.008 * Cvv.mean(axis=1)[band].sum()))
    return np.array(ke), np.array(deltas), np.array(ratios), bath


def test_adqtb_harmonic_kinetic_energy_matches_quadrature():
    omega0 = 200.0
    prm = _qtb_prm(n_seg=256, omega_cut=2825.0)
    ke, deltas, ratios, _ = _qtb_ho(omega0, 1000, 6, prm)
    g0 = prm.gamma0
    kT = prm.kT

    def integrand(w):
        return 2 * g0 * qtb.theta(np.array([w]), kT, HBAR)[0] * w ** 2 / ((omega0 ** 2 - w ** 2) ** 2 + g0 ** 2 * w ** 2)
    mv2 = quad(integrand, 0, prm.omega_cut, points=[omega0], limit=400)[0] / math.pi
    expect = 0.5 * mv2                      # per dof, kcal/mol
    err = _block_err(ke, 10)
    assert abs(ke.mean() - expect) < 4 * err + 0.01 * expect, (ke.mean(), expect, err)
    quantum = HBAR * omega0 / 4 / math.tanh(HBAR * omega0 / (2 * kT))
    assert expect > 2 * (kT / 2) and abs(expect - quantum) / quantum < 0.15
    # FDT (Eq. (21)) holds on a harmonic system at gamma = gamma_0: the band-summed ratio of
    # Eq. (24) sits at gamma_0.
    np.testing.assert_allclose(ratios.mean(), g0, rtol=0.05)


def test_adqtb_simple_adaptation_stays_near_gamma0_on_harmonic_system():
    prm = _qtb_prm(n_seg=128, omega_cut=2825.0, a_gamma=2.0)
    _, _, _, bath = _qtb_ho(200.0, 1000, 5, prm, adapt="simple")
    w = qtb.omega_bins(prm)
    band = (w > 150) & (w < 250)
    assert abs(bath.gamma[0][band].mean() - prm.gamma0) / prm.gamma0 < 0.1


def test_simple_adaptation_contracts_at_the_linear_fdt_rate():
    """Sign and scale of SIMPLE (Eqs. (21)-(23)).  A harmonic oscillator (omega_0) driven by the
    colored noise of power 2 m gamma(omega) Theta(omega) (Eq. (13)) under the friction gamma_0 has
    C_vv = 2 gamma Theta w^2 / (m |D|^2) and Re C_vF = 2 gamma gamma_0 Theta w^2 / |D|^2 with
    D = omega_0^2 - w^2 + i gamma_0 w, so Delta_FDT = 2 gamma Theta w^2 (gamma - gamma_0) / |D|^2:
    gamma = gamma_0 is the fixed point, and near it one SIMPLE update multiplies gamma - gamma_0
    by 1 - A_gamma 2 gamma_0 Theta w^2 / |D|^2 (Theta in kcal/mol, A_gamma in ps^-1 per kcal/mol).
    Starting from gamma = 1.2 gamma_0 (one segment held fixed to reach the stationary state), the
    measured factor in each resonance bin must match that value and be below one: a flipped sign
    gives factors above one, a Delta left in amu A^2/ps^2 (no kcal/mol conversion) or a wrong
    spectrum normalisation moves them far from it."""
    omega0, n_atoms = 200.0, 300
    prm = _qtb_prm(n_seg=1024, omega_cut=2825.0, a_gamma=2.0)
    g0 = prm.gamma0
    masses = np.full(n_atoms, 1.008)
    st = rpmd.init_state(np.zeros((n_atoms, 3)), masses, rpmd.Params(P=1, temperature=prm.temperature, dt=prm.dt,
                                                                       gamma0=g0, seed=prm.seed))
    bath = qtb.QTB(prm, np.repeat(masses, 3), np.zeros(3 * n_atoms, dtype=int), 1, adapt="none")
    bath.gamma[:] = 1.2 * g0
    fn = rpmd.harmonic_forces(omega0, masses)
    gs = []
    for s in range(3 * prm.n_seg):
        qtb.qtb_step(st, masses, bath, fn)
        if (s + 1) % prm.n_seg == 0:
            gs.append(bath.gamma[0].copy())
            bath.adapt = "simple"
    w = qtb.omega_bins(prm)
    th = qtb.theta(w, prm.kT, prm.hbar)
    pred = 1.0 - prm.a_gamma * 2.0 * g0 * th * w ** 2 / ((omega0 ** 2 - w ** 2) ** 2 + g0 ** 2 * w ** 2)
    band = (w > omega0 - g0) & (w < omega0 + g0)
    for k in (1, 2):
        r = (gs[k][band] - g0) / (gs[k - 1][band] - g0)
        assert np.all(r < 1.0), r
        np.testing.assert_allclose(r, pred[band], atol=0.07)

