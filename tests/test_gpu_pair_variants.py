"""Every specialisation of the mixed-precision pair kernel against the FP64 oracle.

The nonbonded sum of Sec. III.A.3 (one centroid list shared by all beads) is compiled
per bead count and per warps-per-atom split:
- P < 32: a warp takes 32/P entries at a time; with P = 2 and 4, four entries per lane
  are in flight.
- P = 16 and 32: the lanes are the beads.
- P = 64: two beads per lane.
- W = 1, 2 or 4 warps share one atom's row.

Each is compared with the oracle on sampled beads of a 343-water box (1,029 atoms, a
multiple of no block's atom count). The small-box path (per-bead minimum image over a
brute-force row) is compared on the 64-water box. The energy variant of the kernel is
checked through the bead-averaged potential.
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
        # the splits differ only in the FP32 summation order of each atom's row
        for W in (2, 4):
            assert rms_rel(forces[W], forces[1]) < 1e-6, W
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
