"""The C-ABI library loads and exports every entry point of include/qhp.h (no GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qhp.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(qhp_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_03137_b300 import build, qhp
    build.build()
    return qhp.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("qhp_create_system", "qhp_set_forcefield", "qhp_set_beads", "qhp_set_thermostat",
                 "qhp_step_rpmd", "qhp_step_adqtb", "qhp_get_energy", "qhp_get_forces", "qhp_get_centroid"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2212_03137_b300 import qhp
    names = set(_declared()) - {"qhp_last_error"}
    assert names <= set(qhp._SIGS), names - set(qhp._SIGS)


def test_argument_errors_need_no_device(lib):
    from paper_2212_03137_b300 import qhp
    pos = np.zeros((4, 3))
    with pytest.raises(qhp.QHPError) as e:          # not a multiple of 3 atoms
        qhp.qhp_create_system([0, 1, 1, 0], [0, 0, 0, 1], pos, 10.0, qhp.QHP_MIXED)
    assert e.value.code == -1
    with pytest.raises(qhp.QHPError) as e:          # H first: not an (O, H, H) layout
        qhp.qhp_create_system([1, 0, 1], [0, 0, 0], pos[:3], 10.0, qhp.QHP_MIXED)
    assert e.value.code == -1
    with pytest.raises(qhp.QHPError) as e:          # bad precision flag
        qhp.qhp_create_system([0, 1, 1], [0, 0, 0], pos[:3], 10.0, 7)
    assert e.value.code == -1
    with pytest.raises(qhp.QHPError) as e:          # non-positive box
        qhp.qhp_create_system([0, 1, 1], [0, 0, 0], pos[:3], -1.0, qhp.QHP_MIXED)
    assert e.value.code == -1
    assert "box_L" in lib.qhp_last_error().decode()


def test_null_handles_are_rejected(lib):
    assert lib.qhp_step_rpmd(None, 1) == -1
    assert lib.qhp_sync(None) == -1
    assert lib.qhp_destroy_system(None) == 0
