"""qhp_estimators_noalloc, the variant of the mode estimators for callers that cannot
allocate device memory (graph capture by another framework, threads that must not
synchronise, application-owned memory pools), agrees with qhp_get_energy.

Collected last on purpose: it exercises the library's fixed device scratch array.
Two calls in a row must give the same numbers (the array is fully overwritten)."""
import numpy as np
import pytest

from paper_2212_03137_b300 import qhp
from paper_2212_03137_b300.workloads import CONFIGS, small_mixed_config

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg", [CONFIGS["rpmd_fp64_64w"], small_mixed_config(512, P=8)], ids=["fp64_64w", "mixed_512w"])
def test_noalloc_estimators_match_get_energy(cfg):
    import torch
    from paper_2212_03137_b300 import build
    build.build()
    dev = torch.device("cuda", 0)
    with qhp.System.from_config(cfg) as s:
        qhp.qhp_step_rpmd(s.h, 5)
        e = qhp.qhp_get_energy(s.h)          # evaluates forces at the current modes
        Q, Pm = qhp.qhp_get_modes(s.h)
        F = qhp.qhp_get_forces(s.h)
    box = cfg.system()
    mass = np.where(box.types == 0, 15.999, 1.008).astype(np.float64)
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).to(dev)
    Pd = torch.from_numpy(np.ascontiguousarray(Pm)).to(dev)
    Fd = torch.from_numpy(np.ascontiguousarray(F)).to(dev)
    md = torch.from_numpy(mass).to(dev)
    want = np.array([e.spring, e.kinetic_nm, e.kinetic_cv])
    results = []
    for _ in range(2):                        # two calls in a row share the scratch array
        out = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
        qhp.qhp_estimators_noalloc(box.n_atoms, cfg.P, cfg.temperature, Qd, Pd, Fd, md, out,
                                   torch.cuda.current_stream(dev).cuda_stream)
        torch.cuda.synchronize(dev)
        results.append(out.cpu().numpy())
    for got in results:
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-9)
    assert np.array_equal(results[0], results[1])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    dev = torch.device("cuda", 0)
    z = torch.zeros(8, dtype=torch.float64, device=dev)
    with pytest.raises(qhp.QHPError) as e:
        qhp.qhp_estimators_noalloc(65536 * 2 + 1, 32, 300.0, z, z, None, z, z)
    assert e.value.code == -1 and "exceeds" in str(e.value)
    with pytest.raises(qhp.QHPError):
        qhp.qhp_estimators_noalloc(10, 3, 300.0, z, z, None, z, z)
