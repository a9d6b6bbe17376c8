"""Every specialisation of the mixed-precision pair kernel against the FP64 oracle.

The nonbonded sum of Sec. III.A.3 (one centroid list shared by all beads) is compiled
per bead count and per warps-per-atom split:
- P >= 2: a lane carries two beads of one list entry (packed FP32x2 arithmetic), so a warp
  takes 64/P entries at a time; P = 1: a lane takes one entry.
- W = 1, 2 or 4 warps share one atom's row, by blocks of 32 entries.

Each is compared with the oracle on sampled beads of a 343-water box (1,029 atoms, a
multiple of no block's atom count). The small-box path (per-bead minimum image over a
brute-force row) is compared on the 64-water box. The energy variant of the kernel is
checked through the bead-averaged potential.

The forces must not depend on W (every block of 32 entries is summed in FP32 and converted
to int64 once, and the integers are added), nor on skipping the entries that lie beyond
reach of every bead: both are checked bit for bit.
"""
import dataclasses

import numpy as np
import pytest

from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import CONFIGS, small_mixed_config

from oracle_bridge import force_fn, rms_rel

pytestmark = pytest.mark.gpu

SAMPLE = {1: (0,), 2: (0, 1), 4: (0, 3), 8: (0, 5), 16: (0, 9, 15), 32: (0, 17, 31), 64: (0, 37, 63)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


def _check_all_splits(cfg, list_mode):
    P = cfg.P
    sel = list(SAMPLE[P])
    with qhp.System.from_config(cfg, precision="mixed") as s:
        assert qhp.qhp_get_info(s.h).list_mode == list_mode
        qhp.qhp_step_rpmd(s.h, 3)
        xb = qhp.qhp_get_beads(s.h)
        V, Fo = force_fn(cfg.system(), cfg.rc)(xb[sel])
        forces = {}
        for W in (1, 2, 4):
            qhp.qhp_set_pair_warps(s.h, W)
            qhp.qhp_compute_forces(s.h)
            F = qhp.qhp_get_forces(s.h)
            for k, b in enumerate(sel):
                err = rms_rel(F[b], Fo[k])
                assert err < 1e-5, (P, W, b, err)
            forces[W] = F
        # block sums are converted to integers before the splits combine them: same bits
        for W in (2, 4):
            assert np.array_equal(forces[W], forces[1]), W
        # entries beyond reach of every bead add exactly nothing: skipping them keeps the bits
        qhp.qhp_set_pair_skip(s.h, False)
        qhp.qhp_compute_forces(s.h)
        assert np.array_equal(qhp.qhp_get_forces(s.h), forces[4])
        qhp.qhp_set_pair_skip(s.h, True)
        qhp.qhp_set_pair_warps(s.h, 0)
        e = qhp.qhp_get_energy(s.h)
    if P <= 8:   # bead-averaged potential from every bead (Eq. (3))
        V_all, _ = force_fn(cfg.system(), cfg.rc)(xb)
        UP = float(np.mean(V_all))
        assert abs(e.potential - UP) < 2e-5 * (np.mean(np.abs(V_all)) + 1.0), (e.potential, UP)


@pytest.mark.parametrize("P", [1, 2, 4, 8, 16, 32, 64])
def test_list_path_every_bead_count_and_split(P):
    _check_all_splits(small_mixed_config(343, P=P), list_mode=1)


@pytest.mark.parametrize("P", [1, 4, 32])
def test_small_box_path_every_split(P):
    _check_all_splits(dataclasses.replace(CONFIGS["rpmd_fp64_64w"], P=P), list_mode=0)
