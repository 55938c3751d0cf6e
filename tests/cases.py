"""Shared helpers for the tests: oracle runs on the seeded workloads, cached per
process, and the error measures the parity tests use."""
from __future__ import annotations

import functools

import numpy as np

from oracle import fem, mor
from paper_2411_12690_gb300 import workloads as W


@functools.lru_cache(maxsize=None)
def oracle_block(spec: W.BlockSpec) -> mor.ReducedBlock:
    mesh = fem.tsv_block_mesh(spec.lx, spec.ly, spec.lz, spec.ex, spec.ey, spec.ez, spec.r_cu, spec.t_liner)
    n = spec.order + 1
    return mor.local_stage(mesh, (n, n, n))


def oracle_pair(spec: W.BlockSpec):
    return [oracle_block(spec), oracle_block(spec.dummy())]


def oracle_solve(spec, site_type, dT, clamp_bottom=True, clamp_top=False, prescribed=None):
    blocks = oracle_pair(spec)
    sol = mor.global_stage(blocks, np.asarray(site_type, dtype=int), dT, clamp_bottom, clamp_top, prescribed)
    return blocks, sol


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def rel_max(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


SMALL_MESH = W.BlockSpec(10.0, 10.0, 30.0, 6, 6, 4, 2.5, 0.5, 2)   # quick block for edge cases
