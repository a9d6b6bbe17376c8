"""The bounds-checked build (-DQHP_CHECK, build(check=True)) on the step paths.

compute-sanitizer is closed on this machine; this build stands in for its memory checker on
the indices the kernels read from device data (list partners and row lengths, the atom
permutations of the cell sort, cell and row positions of the list build): each is tested
before use, and one out of range would set a status bit that the next synchronising call
reports as QHP_ERR_BOUNDS.  The same workloads run once through the checked library and
once through the plain one, each in its own process (QHP_LIBRARY picks the library): the
checked runs must finish without QHP_ERR_BOUNDS and give the same bits, since the checks
read indices and change no arithmetic.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import dataclasses, sys
import numpy as np
from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import CONFIGS, RunConfig, small_mixed_config
out = {}
runs = [("list_P8", small_mixed_config(343, P=8)), ("list_P32", small_mixed_config(343, P=32)),
        ("small_box", dataclasses.replace(CONFIGS["rpmd_fp64_64w"], P=4, precision="mixed")),
        ("fp64", CONFIGS["rpmd_fp64_64w"]), ("list_P1", small_mixed_config(512, P=1))]
for name, cfg in runs:
    with qhp.System.from_config(cfg) as s:
        qhp.qhp_step_rpmd(s.h, 40)
        qhp.qhp_sync(s.h)
        out[name + "_Q"], out[name + "_P"] = qhp.qhp_get_modes(s.h)
qcfg = RunConfig(name="adqtb_64w", n_mol=64, box=12.42, rc=6.0, P=1, dt_fs=0.5, gamma0=20.0, thermostat="adqtb",
                 precision="mixed", n_seg=64, omega_cut_cm=15000.0, a_gamma=10.0, seed=5)
with qhp.System.from_config(qcfg) as s:
    qhp.qhp_step_adqtb(s.h, 80)
    qhp.qhp_sync(s.h)
    out["adqtb_Q"], out["adqtb_P"] = qhp.qhp_get_modes(s.h)
systems = [qhp.System.from_config(small_mixed_config(n, P=p, seed=n)) for n, p in ((64, 4), (216, 16), (343, 8))]
with qhp.Batch(systems) as b:
    b.step(20)
    b.sync()
for k, s in enumerate(systems):
    out[f"batch{k}_Q"], out[f"batch{k}_P"] = qhp.qhp_get_modes(s.h)
    s.close()
np.savez(sys.argv[1], **out)
"""


def _run(lib, path):
    env = dict(os.environ)
    env.pop("QHP_LIBRARY", None)
    if lib:
        env["QHP_LIBRARY"] = lib
    r = subprocess.run([sys.executable, "-c", SCRIPT, str(path)], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(path)


def test_bounds_checked_build_is_clean_and_changes_nothing(tmp_path):
    from paper_2212_03137_b300 import build
    build.build()
    checked = build.build(check=True)
    a = _run(checked, tmp_path / "checked.npz")
    b = _run(None, tmp_path / "plain.npz")
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
