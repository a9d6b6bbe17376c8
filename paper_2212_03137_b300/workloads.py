"""Seeded synthetic water boxes and the run configurations they are used in.

This module only *generates inputs*: lattice sites, random molecular
orientations, Gaussian jitter and the parameter sets.  It holds none of the
method's arithmetic, so both the CUDA path and the FP64 oracle consume it.

Input recipe (stands in for the paper's water boxes of Sec. III.D and the
216/1000-molecule boxes of Sec. IV, which are not available here):

* ``n_mol`` rigid q-SPC/Fw-geometry molecules (r_OH = 1.0 A, HOH = 112 deg)
  are centred on the sites of the smallest cubic lattice n^3 >= n_mol; when
  the lattice has more sites than molecules a seeded random subset is used.
* each molecule gets a uniformly random orientation (unit quaternion from four
  standard normals) and every atom a 0.05 A isotropic Gaussian jitter;
* atoms are ordered O, H, H per molecule; ``type`` is 0 for O, 1 for H and
  ``molecule`` is the molecule index.
* the cubic box edge is the stated value of each configuration, or
  (29.915 * n_mol)^(1/3) A (liquid water at 1.0 g/cm^3) when none is stated.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

# q-SPC/Fw-style water parameters (kcal/mol, Angstrom, degrees, e).
WATER_FF = dict(
    eps=0.1554, sigma=3.1655, q_O=-0.84,
    k_b=1059.162, r0=1.0, k_theta=75.90, theta0_deg=112.0,
    alpha=0.2, m_O=15.999, m_H=1.008,
)

MOLAR_VOLUME_A3 = 29.915  # A^3 per molecule at 1.0 g/cm^3


@dataclass
class WaterBox:
    pos: np.ndarray          # [n_atoms, 3] float64, Angstrom
    types: np.ndarray        # [n_atoms] int32, 0 = O, 1 = H
    molecule: np.ndarray     # [n_atoms] int32
    box: float               # cubic edge, Angstrom

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_mol(self) -> int:
        return self.n_atoms // 3


def box_edge_for(n_mol: int) -> float:
    return (MOLAR_VOLUME_A3 * n_mol) ** (1.0 / 3.0)


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def water_box(n_mol: int, seed: int, box: float | None = None, jitter: float = 0.05) -> WaterBox:
    """Seeded lattice of randomly oriented water molecules (recipe above)."""
    if box is None:
        box = box_edge_for(n_mol)
    rng = np.random.default_rng(seed)
    n = int(math.ceil(round(n_mol ** (1.0 / 3.0), 9)))
    while n ** 3 < n_mol:
        n += 1
    sites = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    if sites.shape[0] > n_mol:
        keep = np.sort(rng.choice(sites.shape[0], size=n_mol, replace=False))
        sites = sites[keep]
    centres = (sites + 0.5) * (box / n)
    r0 = WATER_FF["r0"]
    half = math.radians(WATER_FF["theta0_deg"]) / 2
    body = np.array([[0.0, 0.0, 0.0],
                     [r0 * math.sin(half), 0.0, r0 * math.cos(half)],
                     [-r0 * math.sin(half), 0.0, r0 * math.cos(half)]])
    R = _random_rotations(rng, n_mol)
    atoms = centres[:, None, :] + np.einsum("mij,aj->mai", R, body)
    atoms = atoms + jitter * rng.standard_normal(atoms.shape)
    pos = atoms.reshape(-1, 3).astype(np.float64)
    types = np.tile(np.array([0, 1, 1], dtype=np.int32), n_mol)
    molecule = np.repeat(np.arange(n_mol, dtype=np.int32), 3)
    return WaterBox(pos=pos, types=types, molecule=molecule, box=float(box))


@dataclass
class RunConfig:
    """One workload: box, force-field cutoff, beads and thermostat."""
    name: str
    n_mol: int
    box: float
    rc: float
    P: int
    temperature: float = 300.0
    dt_fs: float = 0.5
    gamma0: float = 1.0           # ps^-1
    thermostat: str = "pile"      # "pile" (RPMD/TRPMD) or "adqtb"
    precision: str = "mixed"      # "fp64" or "mixed"
    steps: int = 100
    seed: int = 1234
    skin: float = 2.0
    n_seg: int = 1024
    omega_cut_cm: float = 15000.0
    a_gamma: float = 10.0
    gamma_min_frac: float = 0.01
    extra: dict = field(default_factory=dict)

    def with_(self, **kw) -> "RunConfig":
        return replace(self, **kw)

    def system(self) -> WaterBox:
        return water_box(self.n_mol, self.seed, self.box)


def _rc_for(box: float) -> float:
    return min(9.0, 0.48 * box)


# The five workloads: plain FP64 RPMD on 64 waters, mixed-precision RPMD on
# 4,096 waters, single-bead adQTB on 72,000 waters, a batch of 256 uneven boxes
# and the differentiation box of 216 waters.
CONFIGS = {
    "rpmd_fp64_64w": RunConfig(name="rpmd_fp64_64w", n_mol=64, box=12.42, rc=6.0, P=8,
                               dt_fs=0.25, gamma0=1.0, precision="fp64", steps=100),
    "rpmd_mixed_4096w": RunConfig(name="rpmd_mixed_4096w", n_mol=4096, box=49.7, rc=9.0, P=32,
                                  dt_fs=0.5, gamma0=1.0, precision="mixed", steps=1000),
    "adqtb_mixed_72000w": RunConfig(name="adqtb_mixed_72000w", n_mol=72000, box=129.0, rc=9.0, P=1,
                                    dt_fs=0.5, gamma0=20.0, thermostat="adqtb", precision="mixed",
                                    steps=10240, n_seg=1024, omega_cut_cm=15000.0, a_gamma=10.0),
    # the 4,096-water RPMD box with BAOAB-RESPA (4 inner steps of 0.5 fs per 2 fs outer step)
    # and the nonbonded forces on 8 contracted beads (Sec. III.A.2)
    "rpmd_respa_rpc_4096w": RunConfig(name="rpmd_respa_rpc_4096w", n_mol=4096, box=49.7, rc=9.0, P=32,
                                      dt_fs=0.5, gamma0=1.0, precision="mixed", steps=1000,
                                      extra={"respa": 4, "contracted_beads": 8}),
    # a smaller adQTB box of the same density and settings (profiling and parity sizes)
    "adqtb_mixed_8000w": RunConfig(name="adqtb_mixed_8000w", n_mol=8000, box=box_edge_for(8000), rc=9.0, P=1,
                                   dt_fs=0.5, gamma0=20.0, thermostat="adqtb", precision="mixed",
                                   steps=2048, n_seg=1024, omega_cut_cm=15000.0, a_gamma=10.0),
    "grad_216w": RunConfig(name="grad_216w", n_mol=216, box=18.6, rc=9.0, P=16,
                           dt_fs=0.5, gamma0=1.0, precision="fp64", steps=200),
}


def batch_configs(seed: int = 1234, n_sys: int = 256) -> list[RunConfig]:
    """256 independent boxes: n_mol log-uniform in [64, 2048], P from {4..64}."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_sys):
        n_mol = int(round(math.exp(rng.uniform(math.log(64), math.log(2048)))))
        P = int(rng.choice([4, 8, 16, 32, 64]))
        box = box_edge_for(n_mol)
        out.append(RunConfig(name=f"batch_{k}", n_mol=n_mol, box=box, rc=_rc_for(box), P=P,
                             dt_fs=0.5, gamma0=1.0, precision="mixed", steps=500, seed=seed + 1 + k))
    return out


def small_mixed_config(n_mol: int = 512, P: int = 8, seed: int = 7) -> RunConfig:
    """A box large enough for the centroid Verlet list yet quick for the oracle."""
    box = box_edge_for(n_mol)
    return RunConfig(name=f"rpmd_mixed_{n_mol}w", n_mol=n_mol, box=box, rc=min(9.0, box / 3.0 - 2.2),
                     P=P, dt_fs=0.5, gamma0=1.0, precision="mixed", steps=10, seed=seed)
