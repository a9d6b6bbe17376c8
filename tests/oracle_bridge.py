"""Builds the oracle counterpart of a workload (test helper; imports only oracle/ and workloads)."""
from __future__ import annotations

import math

import numpy as np

from oracle import neighbor, rpmd, water
from paper_2212_03137_b300.workloads import WATER_FF


def oracle_ff(rc: float) -> water.ForceField:
    W = WATER_FF
    return water.ForceField(eps=W["eps"], sigma=W["sigma"], q_O=W["q_O"], k_b=W["k_b"], r0=W["r0"],
                            k_theta=W["k_theta"], theta0=math.radians(W["theta0_deg"]), alpha=W["alpha"], rc=rc,
                            m_O=W["m_O"], m_H=W["m_H"])


def oracle_params(cfg, seed=None) -> rpmd.Params:
    return rpmd.Params(P=cfg.P, temperature=cfg.temperature, dt=cfg.dt_fs * 1e-3, gamma0=cfg.gamma0,
                       seed=cfg.seed if seed is None else seed)


def masses(box, ff: water.ForceField) -> np.ndarray:
    return ff.masses(box.types)


def force_fn(box, rc: float, cells: bool = False):
    return water.make_force_fn(box.types, box.molecule, box.box, oracle_ff(rc), cells=cells)


def rms_rel(a: np.ndarray, ref: np.ndarray) -> float:
    return float(np.sqrt(np.sum((a - ref) ** 2) / np.sum(ref ** 2)))


def list_pairs_oracle(C: np.ndarray, mol: np.ndarray, L: float, r_list: float) -> set:
    p = neighbor.verlet_pairs(C, mol, L, r_list)
    return set(map(tuple, p.tolist()))
