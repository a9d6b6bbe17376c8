"""Batched systems: many uneven boxes stepped by the batched launches give, bit for bit,
the trajectories of the same boxes stepped one at a time (one cooperative launch per step
adds every system's pair and bonded terms as int64 atomics; integer sums do not depend on
their order; a system whose list check fires finishes its step in a conditional node with
the single-system kernels), and those match the FP64 oracle at the mixed-precision
tolerance."""
import numpy as np
import pytest

from oracle import rpmd
from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import RunConfig, batch_configs, box_edge_for

from oracle_bridge import force_fn, oracle_ff, oracle_params

pytestmark = pytest.mark.gpu


def _cfg(n_mol, P, seed):
    L = box_edge_for(n_mol)
    return RunConfig(name=f"b{n_mol}_{P}", n_mol=n_mol, box=L, rc=min(9.0, 0.48 * L), P=P, dt_fs=0.5, gamma0=1.0,
                     precision="mixed", seed=seed)


# all-pairs boxes (64, 100, 216, 300 waters) and centroid-list boxes (700, 1000 waters)
MIX = [_cfg(64, 4, 11), _cfg(100, 64, 12), _cfg(300, 8, 13), _cfg(700, 32, 14), _cfg(216, 16, 15), _cfg(1000, 4, 16)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


def _systems(cfgs):
    return [qhp.System.from_config(c) for c in cfgs]


def test_batch_equals_single_systems_bitwise():
    singles = _systems(MIX)
    for s in singles:
        qhp.qhp_step_rpmd(s.h, 25)
    members = _systems(MIX)
    with qhp.Batch(members) as b:
        b.step(10)
        b.step(15)
        b.sync()
        info = qhp.qhp_batch_get_info(b.h)
        # one cooperative launch whatever the mix (integrate + checks, forces, projection)
        assert info.n_sys == len(MIX) and info.steps == 25 and info.kernels_per_step == 1
        assert info.grid_bonded == 0 and info.items_pair > 0 and info.grid_pair == 2 * info.grid_integrate
        assert info.atom_beads == sum(3 * c.n_mol * c.P for c in MIX)
        for s, m in zip(singles, members):
            Qa, Pa = qhp.qhp_get_modes(s.h)
            Qb, Pb = qhp.qhp_get_modes(m.h)
            assert np.array_equal(Qa, Qb) and np.array_equal(Pa, Pb)
            assert qhp.qhp_get_info(s.h).rebuilds == qhp.qhp_get_info(m.h).rebuilds
            assert qhp.qhp_get_info(m.h).step == 25
        assert info.rebuilds > len(MIX)
        pr = qhp.qhp_batch_get_profile(b.h)
        assert pr.pair_ms > 0 and pr.step_ms > pr.pair_ms
    # the members work on their own again after the batch is gone
    qhp.qhp_step_rpmd(members[0].h, 2)
    qhp.qhp_step_rpmd(singles[0].h, 2)
    assert np.array_equal(qhp.qhp_get_modes(members[0].h)[0], qhp.qhp_get_modes(singles[0].h)[0])
    for s in singles + members:
        s.close()


def test_batch_member_matches_oracle():
    """The 64-water P = 4 member after 10 batched steps against the FP64 oracle (1e-6 A)."""
    cfg = MIX[0]
    members = _systems(MIX[:3])
    with qhp.Batch(members) as b:
        b.step(10)
        b.sync()
        Q, _ = qhp.qhp_get_modes(members[0].h)
    box = cfg.system()
    ff = oracle_ff(cfg.rc)
    prm = oracle_params(cfg)
    st = rpmd.init_state(box.pos, ff.masses(box.types), prm)
    fn = force_fn(box, cfg.rc)
    for _ in range(10):
        rpmd.step(st, prm, ff.masses(box.types), fn)
    assert np.max(np.abs(Q[:, :, 0] - st.Q[:, :, 0])) < 1e-6
    for s in members:
        s.close()


def test_autotune_and_fixed_warps_reproduce():
    members = _systems(MIX)
    with qhp.Batch(members) as b:
        tuned = qhp.qhp_batch_autotune(b.h, 3)
        assert set(tuned) == {c.P for c in MIX} and set(tuned.values()) <= {1, 2, 4}
        b.step(12)
        b.sync()
        singles = _systems(MIX)
        for s, c in zip(singles, MIX):
            qhp.qhp_set_pair_warps(s.h, tuned[c.P])
            qhp.qhp_step_rpmd(s.h, 12)
        for s, m in zip(singles, members):
            assert np.array_equal(qhp.qhp_get_modes(s.h)[0], qhp.qhp_get_modes(m.h)[0])
    w = qhp.qhp_autotune(singles[3].h, 3)
    assert w in (1, 2, 4)
    with pytest.raises(qhp.QHPError):
        qhp.qhp_set_pair_warps(singles[0].h, 3)
    for s in singles + members:
        s.close()


def test_batch_rejects_unsupported_members():
    fp64 = qhp.System.from_config(MIX[0], precision="fp64")
    ok = qhp.System.from_config(MIX[1])
    with pytest.raises(qhp.QHPError):
        qhp.Batch([ok, fp64])
    with pytest.raises(qhp.QHPError):
        qhp.Batch([ok, ok])
    fp64.close()
    ok.close()


@pytest.mark.slow
def test_full_batch_of_256_boxes():
    """The 256-box workload (64-2,048 waters, P in {4..64}): 20 batched steps; one member of
    each bead count equals the same box stepped alone."""
    cfgs = batch_configs()
    members = _systems(cfgs)
    with qhp.Batch(members) as b:
        tuned = qhp.qhp_batch_autotune(b.h, 2)
        b.step(20)
        b.sync()
        info = qhp.qhp_batch_get_info(b.h)
        assert info.n_sys == 256 and info.atom_beads == sum(3 * c.n_mol * c.P for c in cfgs)
        picks = {}
        for k, c in enumerate(cfgs):
            picks.setdefault(c.P, k)
        for P, k in picks.items():
            single = qhp.System.from_config(cfgs[k])
            qhp.qhp_set_pair_warps(single.h, tuned[P])
            qhp.qhp_step_rpmd(single.h, 20)
            assert np.array_equal(qhp.qhp_get_modes(single.h)[0], qhp.qhp_get_modes(members[k].h)[0])
            single.close()
    for s in members:
        s.close()
