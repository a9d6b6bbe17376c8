"""Failure detection, injected from the host (no GPU fault, no hang).

The step kernels keep status words: non-finite momenta (QHP_ERR_NONFINITE) and a bead
farther than skin/2 from its anchor right after a list rebuild (QHP_ERR_LIST_OVERFLOW: the
list would no longer be complete).  The error surfaces at the next synchronising call, and
the CUDA context stays usable: a fresh system steps normally afterwards.  The failures are
made by the caller's inputs: a NaN in a normal mode, a bead pushed outside the skin, and a
time step far beyond the O-H stretch's stability limit.  The 64-water box runs without a cell
grid, and no index is ever formed from a position.

The batched step's grid barriers wait with a time limit: the self-test runs the barrier with
one arrival that never comes (a count that nothing completes), every wait gives up after the
limit with ST_TIMEOUT, and the context stays usable.
"""
import math

import numpy as np
import pytest

from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import CONFIGS

pytestmark = pytest.mark.gpu

C1 = CONFIGS["rpmd_fp64_64w"]
REPORTED = (-4, -5)   # QHP_ERR_NONFINITE, QHP_ERR_LIST_OVERFLOW


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_03137_b300 import build
    build.build()


def _healthy(prec):
    with qhp.System.from_config(C1, precision=prec) as s:
        qhp.qhp_step_rpmd(s.h, 3)
        qhp.qhp_sync(s.h)
        assert math.isfinite(qhp.qhp_get_energy(s.h).potential)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_nan_in_a_mode_is_reported(prec):
    with qhp.System.from_config(C1, precision=prec) as s:
        qhp.qhp_step_rpmd(s.h, 2)
        Q, Pm = qhp.qhp_get_modes(s.h)
        Q[5, 1, 3] = np.nan
        qhp.qhp_set_modes(s.h, Q, Pm)
        with pytest.raises(qhp.QHPError) as e:
            qhp.qhp_step_rpmd(s.h, 2)
            qhp.qhp_sync(s.h)
        assert e.value.code in REPORTED
    _healthy(prec)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_bead_outside_the_skin_is_reported(prec):
    """Mode 1 of one atom moved by 2 A puts some of its beads up to 2.8 A from the centroid,
    beyond skin/2 = 1 A: the cover check after the rebuild reports it."""
    with qhp.System.from_config(C1, precision=prec) as s:
        qhp.qhp_step_rpmd(s.h, 2)
        Q, Pm = qhp.qhp_get_modes(s.h)
        Q[7, 0, 1] += 2.0
        qhp.qhp_set_modes(s.h, Q, Pm)
        with pytest.raises(qhp.QHPError) as e:
            qhp.qhp_step_rpmd(s.h, 1)
            qhp.qhp_sync(s.h)
        assert e.value.code == -5
    _healthy(prec)


def test_absurd_time_step_is_reported():
    """25 fs without friction: the O-H stretch (period ~9 fs) is far past the Verlet stability
    limit, and the blow-up is reported within a few hundred steps."""
    with qhp.System.from_config(C1, precision="mixed") as s:
        qhp.qhp_set_thermostat(s.h, qhp.make_thermo(kind=qhp.QHP_THERMO_NVE, dt_fs=25.0))
        with pytest.raises(qhp.QHPError) as e:
            for _ in range(20):
                qhp.qhp_step_rpmd(s.h, 20)
                qhp.qhp_sync(s.h)
        assert e.value.code in REPORTED
    _healthy("mixed")


def test_grid_barrier_wait_runs_out_and_reports_timeout():
    """20 ms limit, one missing arrival: QHP_ERR_TIMEOUT with ST_TIMEOUT, in well under a second."""
    import time
    t0 = time.perf_counter()
    rc, status = qhp.qhp_selftest_grid_barrier(20_000_000)
    elapsed = time.perf_counter() - t0
    assert rc == -3 and status & 4, (rc, status)
    assert elapsed < 5.0
    _healthy("mixed")


def test_batch_wait_limit_is_validated_and_steps_run_under_it():
    from paper_2212_03137_b300.workloads import small_mixed_config
    systems = [qhp.System.from_config(small_mixed_config(n, P=p, seed=n)) for n, p in ((64, 4), (216, 8))]
    with qhp.Batch(systems) as b:
        with pytest.raises(qhp.QHPError):
            qhp.qhp_batch_set_wait_limit(b.h, 10)
        qhp.qhp_batch_set_wait_limit(b.h, 500_000_000)
        b.step(5)
        b.sync()
    for s in systems:
        s.close()
