"""Degenerate inputs on the CUDA path against the FP64 oracle: empty neighbour rows.

One water molecule in a 20 A box, and two molecules 10 A apart (beyond r_list = rc + skin =
8 A). Both boxes use the cell grid (5 cells per edge). Every row of the centroid list is
empty: the intramolecular pairs are excluded and no other atom is near. The pair kernels then
walk zero-length rows, and the forces and U_P (Eq. (3)) are the bonded terms and the DSF self
term alone.
"""
import dataclasses

import numpy as np
import pytest

from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import CONFIGS

from oracle_bridge import force_fn, rms_rel

pytestmark = pytest.mark.gpu

C1 = CONFIGS["rpmd_fp64_64w"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


@pytest.mark.parametrize("n_mol", [1, 2])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_empty_neighbour_rows(n_mol, prec):
    cfg = dataclasses.replace(C1, n_mol=n_mol, box=20.0, rc=6.0, P=8)
    with qhp.System.from_config(cfg, precision=prec) as s:
        qhp.qhp_step_rpmd(s.h, 5)
        qhp.qhp_compute_forces(s.h)
        info = qhp.qhp_get_info(s.h)
        assert info.list_mode == 1 and info.n_cells_per_edge == 5
        assert info.list_entries == 0
        xb = qhp.qhp_get_beads(s.h)
        F = qhp.qhp_get_forces(s.h)
        e = qhp.qhp_get_energy(s.h)
    V, Fo = force_fn(cfg.system(), cfg.rc)(xb)
    tol = 1e-5 if prec == "mixed" else 1e-12
    assert rms_rel(F, Fo) < tol
    UP = float(np.mean(V))
    assert abs(e.potential - UP) < tol * (abs(UP) + 1.0), (e.potential, UP)
