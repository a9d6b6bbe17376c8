"""Pins for the oracle's parameter gradients and trajectory-gradient machinery (no GPU)."""
import numpy as np
import pytest

from oracle import gradients as G
from oracle import rpmd, water
from paper_2212_03137_b300.workloads import water_box


def _box(n_mol=8, seed=5):
    return water_box(n_mol, seed)


def test_param_gradient_matches_finite_differences_of_the_energy():
    """dV/dtheta against central differences of an energy written without any derivative."""
    w = _box()
    ff = water.ForceField(rc=3.5)
    g = G.param_gradient(w.pos, w.types, w.molecule, w.box, ff)
    th = G.param_vector(ff)
    for k in range(5):
        h = 1e-5 * abs(th[k])
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        Ep = water.potential_energy_only(w.pos, w.types, w.molecule, w.box, G.with_params(ff, tp))
        Em = water.potential_energy_only(w.pos, w.types, w.molecule, w.box, G.with_params(ff, tm))
        fd = (Ep - Em) / (2 * h)
        assert abs(fd - g[k]) < 1e-7 * max(1.0, abs(g[k])), (G.PARAM_NAMES[k], fd, g[k])


def test_param_gradient_is_zero_where_the_term_vanishes():
    """At the bonded equilibrium the k_b and k_theta derivatives vanish; with no O-O pair
    inside rc the LJ derivatives vanish."""
    ff = water.ForceField(rc=2.0)
    h = ff.theta0 / 2
    x = np.array([[1.0, 1.0, 1.0], [1 + np.sin(h), 1.0, 1 + np.cos(h)], [1 - np.sin(h), 1.0, 1 + np.cos(h)],
                  [6.0, 6.0, 6.0], [6 + np.sin(h), 6.0, 6 + np.cos(h)], [6 - np.sin(h), 6.0, 6 + np.cos(h)]])
    types = np.array([0, 1, 1, 0, 1, 1])
    mol = np.array([0, 0, 0, 1, 1, 1])
    g = G.param_gradient(x, types, mol, 30.0, ff)
    assert abs(g[3]) < 1e-28 and abs(g[4]) < 1e-24 and g[0] == 0.0 and g[1] == 0.0


def test_bead_energy_gradient_scales_by_one_over_P():
    w = _box(8, 2)
    ff = water.ForceField(rc=3.5)
    rng = np.random.default_rng(1)
    P = 4
    xb = w.pos[None] + 0.05 * rng.standard_normal((P,) + w.pos.shape)
    U, dx, dth = G.bead_energy_gradients(xb, w.types, w.molecule, w.box, ff)
    V = [water.potential_energy_only(xb[b], w.types, w.molecule, w.box, ff) for b in range(P)]
    np.testing.assert_allclose(U, np.mean(V), rtol=1e-12)
    h = 1e-6
    for (b, a, k) in [(0, 3, 1), (3, 10, 2), (2, 0, 0)]:
        xp, xm = xb.copy(), xb.copy()
        xp[b, a, k] += h
        xm[b, a, k] -= h
        Up = np.mean([water.potential_energy_only(xp[c], w.types, w.molecule, w.box, ff) for c in range(P)])
        Um = np.mean([water.potential_energy_only(xm[c], w.types, w.molecule, w.box, ff) for c in range(P)])
        assert abs((Up - Um) / (2 * h) - dx[b, a, k]) < 1e-6 * max(1.0, abs(dx[b, a, k]))


@pytest.mark.parametrize("which", [G.OBS_CENTROID_ENERGY, G.OBS_MEAN_OH])
def test_segment_gradient_one_step_from_rest_closed_form(which):
    """One NVE step of one bead from rest: the finite-difference trajectory gradient equals
    the closed form built from force evaluations with single terms switched on."""
    w = _box(8, 6)
    ff = water.ForceField(rc=3.5)
    prm = rpmd.Params(P=1, temperature=300.0, dt=0.0005, gamma0=0.0, seed=3)
    st = rpmd.State(Q=w.pos[:, :, None].copy(), Pm=np.zeros((w.n_atoms, 3, 1)))
    fd = G.segment_gradient_fd(st, prm, w.types, w.molecule, w.box, ff, K=1, which=which)
    ref = G.one_step_from_rest_gradient(w.pos, w.types, w.molecule, w.box, ff, prm.dt, which)
    for k in (0, 2, 3, 4):
        assert abs(fd[k] - ref[k]) < 2e-6 * max(abs(ref[k]), 1e-3 * np.nanmax(np.abs(ref))), (k, fd[k], ref[k])
