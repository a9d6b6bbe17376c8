"""Pins for the oracle's ring-polymer contraction and RESPA step (no GPU)."""
import numpy as np
import pytest

from oracle import normal_modes, respa, rpmd, water
from paper_2212_03137_b300.workloads import water_box


@pytest.mark.parametrize("P,Pc", [(8, 1), (8, 2), (8, 4), (16, 4), (32, 8), (8, 8)])
def test_kept_modes_are_the_lowest_frequencies(P, Pc):
    w = normal_modes.mode_frequencies(P, 0.6, 0.0152)
    K = respa.kept_modes(P, Pc)
    assert len(K) == Pc
    assert np.max(w[K]) <= np.sort(w)[Pc - 1] + 1e-12 * np.max(w)


@pytest.mark.parametrize("P,Pc", [(8, 2), (8, 4), (32, 8), (64, 4)])
def test_contraction_interpolates_band_limited_ring_polymers_exactly(P, Pc):
    """A ring polymer excited only in the kept modes is reproduced at the contracted beads
    (imaginary times b P/Pc), including the cos mode of frequency Pc/2."""
    rng = np.random.default_rng(P + Pc)
    Q = np.zeros((5, 3, P))
    K = respa.kept_modes(P, Pc)
    Q[:, :, K] = rng.standard_normal((5, 3, len(K)))
    x = normal_modes.modes_to_beads(Q, normal_modes.transfer_matrix(P))       # [N, 3, P]
    xc = respa.contract(Q, respa.contraction_matrix(P, Pc))                  # [Pc, N, 3]
    for b in range(Pc):
        np.testing.assert_allclose(xc[b], x[:, :, b * P // Pc], atol=1e-12)


def test_full_and_centroid_limits():
    rng = np.random.default_rng(3)
    P = 8
    Q = rng.standard_normal((4, 3, P))
    T = normal_modes.transfer_matrix(P)
    C = respa.contraction_matrix(P, P)
    np.testing.assert_allclose(respa.contract(Q, C), np.transpose(normal_modes.modes_to_beads(Q, T), (2, 0, 1)),
                               atol=1e-12)
    F = rng.standard_normal((P, 4, 3))
    np.testing.assert_allclose(respa.project_contracted(F, C),
                               normal_modes.project_forces(np.transpose(F, (1, 2, 0)), T), atol=1e-12)
    np.testing.assert_allclose(respa.contract(Q, respa.contraction_matrix(P, 1))[0], Q[:, :, 0], atol=1e-14)


def test_contracted_forces_are_minus_gradient():
    """(1/Pc) C^T F_s = -d/dQ of (1/Pc) sum_b V_s(xc_b), by central differences."""
    w = water_box(8, 4)
    ff = water.ForceField(rc=3.5)
    _, slow = respa.split_force_fns(w.types, w.molecule, w.box, ff)
    P, Pc = 8, 4
    rng = np.random.default_rng(5)
    Q = np.zeros((w.n_atoms, 3, P))
    Q[:, :, 0] = w.pos
    Q[:, :, 1:] = 0.03 * rng.standard_normal((w.n_atoms, 3, P - 1))
    C = respa.contraction_matrix(P, Pc)
    _, Fs = slow(respa.contract(Q, C))
    f = respa.project_contracted(Fs, C)
    h = 1e-6
    for (a, d, n) in [(0, 0, 0), (5, 2, 1), (9, 1, P - 1), (3, 0, 2), (14, 1, 5)]:
        Qp, Qm = Q.copy(), Q.copy()
        Qp[a, d, n] += h
        Qm[a, d, n] -= h
        fd = -(respa.contracted_potential(Qp, slow, C) - respa.contracted_potential(Qm, slow, C)) / (2 * h)
        assert abs(fd - f[a, d, n]) < 1e-6 * max(1.0, abs(f[a, d, n])), (a, d, n, fd, f[a, d, n])


def test_one_inner_step_full_contraction_is_baoab():
    """n_alt = 1 and Pc = P: the RESPA step is the BAOAB step of Eq. (17) with V = V_f + V_s."""
    w = water_box(8, 2)
    ff = water.ForceField(rc=3.5)
    prm = rpmd.Params(P=4, temperature=300.0, dt=0.0005, gamma0=1.0, seed=9)
    m = ff.masses(w.types)
    a = rpmd.init_state(w.pos, m, prm)
    b = rpmd.init_state(w.pos, m, prm)
    fast, slow = respa.split_force_fns(w.types, w.molecule, w.box, ff)
    fn = water.make_force_fn(w.types, w.molecule, w.box, ff)
    C = respa.contraction_matrix(4, 4)
    for _ in range(3):
        respa.respa_step(a, prm, m, fast, slow, 1, C)
        rpmd.step(b, prm, m, fn)
    np.testing.assert_allclose(a.Q, b.Q, atol=1e-12)
    np.testing.assert_allclose(a.Pm, b.Pm, atol=1e-10)
    assert a.step == b.step == 3


def _respa_nve_error(n_alt, dt, t_total, P=4):
    """Max |H_P(t) - H_P(0)| over outer steps of NVE RESPA (no O step) with Pc = P on the
    64-water box; H_P = sum_n P_n^2/2m + sum_n m w_n^2 Q_n^2/2 + U_P with the full V."""
    from oracle_bridge import oracle_ff
    from paper_2212_03137_b300.workloads import CONFIGS
    cfg = CONFIGS["rpmd_fp64_64w"]
    box = cfg.system()
    ff = oracle_ff(cfg.rc)
    m = ff.masses(box.types)
    prm = rpmd.Params(P=P, temperature=300.0, dt=dt, gamma0=0.0, seed=11, thermostat="nve")
    st = rpmd.init_state(box.pos, m, prm)
    fast, slow = respa.split_force_fns(box.types, box.molecule, box.box, ff)
    full = water.make_force_fn(box.types, box.molecule, box.box, ff)
    C = respa.contraction_matrix(P, P)

    def H():
        V, _ = full(rpmd.beads(st, P))
        return rpmd.kinetic_energy(st, m) + rpmd.spring_energy(st, prm, m) + float(np.mean(V))

    h0, err = H(), 0.0
    for _ in range(int(round(t_total / (n_alt * dt)))):
        respa.respa_step(st, prm, m, fast, slow, n_alt, C)
        err = max(err, abs(H() - h0))
    return err, rpmd.kinetic_energy(st, m)


@pytest.mark.parametrize("n_alt", [2, 4])
def test_respa_outer_kick_conserves_ring_polymer_hamiltonian_to_second_order(n_alt):
    """Eq. (19) with n_alt > 1: B_s(n dt/2) [B_f(dt/2) A A B_f(dt/2)]^n B_s(n dt/2) without the
    thermostat is a symplectic splitting of the flow of Eq. (9) with V = V_f + V_s, so H_P is
    conserved to second order: halving the inner (and so the outer) step quarters the error.  An
    outer kick weighted dt/2 instead of n dt/2 integrates V_f + V_s/n instead and leaves an
    error that does not shrink with dt (measured: ratio 0.97-0.99, ten times larger errors)."""
    e1, ke = _respa_nve_error(n_alt, 0.0001, 0.004)
    e2, _ = _respa_nve_error(n_alt, 0.00005, 0.004)
    assert e1 < 5e-3 * ke, (e1, ke)
    assert 0.2 < e2 / e1 < 0.3, (e1, e2)

