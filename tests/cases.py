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


# Operand rounding unit of each reduced-precision mode (TF32 10-bit mantissa;
# BF16 7-bit; split BF16 hi + lo: the dropped lo*lo term and the lo rounding).
U_IN = {1: 2.0 ** -11, 2: 2.0 ** -8, 3: 3 * 2.0 ** -16}
_ABS_SMEAN = {}


def abs_smean(block):
    """|S_mean| (n_el, 6, m+1) of an oracle block: the Gauss mean of its stress
    modes, taken elementwise in absolute value (cached per block object)."""
    k = id(block)
    if k not in _ABS_SMEAN:
        m1 = block.m + 1
        _ABS_SMEAN[k] = (block, np.abs(block.S.reshape(block.n_el, 8, 6, m1).mean(axis=1)))
    return _ABS_SMEAN[k][1]


def vm_bound_rows(blocks, types, coeffs, dT, mode):
    """Per-element bound on |vm_gpu - vm_exact| for the blocks whose oracle
    types and element DOFs are given (one row each): each Gauss-mean stress
    component obeys |err| <= (2 u_in + (m+17) 2^-24) (|S_mean| |[c; dT]|)
    (operand rounding, FP32 accumulation over m+1 terms, FP32 epilogue), and
    von Mises is sqrt(3/2)-Lipschitz in the stress's Frobenius norm (shears
    counted twice)."""
    m1 = blocks[0].m + 1
    u = 2 * U_IN[mode] + (m1 + 16) * 2.0 ** -24
    out = []
    for t, c in zip(types, coeffs):
        Sm = abs_smean(blocks[int(t)])
        cc = np.abs(np.concatenate([c, [dT]]))
        ab = u * (Sm @ cc)
        fro = np.sqrt((ab[:, :3] ** 2).sum(1) + 2 * (ab[:, 3:] ** 2).sum(1))
        out.append(np.sqrt(1.5) * fro)
    return np.stack(out)


def oracle_vm_rows(blocks, types, coeffs, dT):
    """Per-element von Mises of the Gauss-mean stress S [c; dT] for the given
    blocks (oracle recovery, one row per block)."""
    out = []
    for t, c in zip(types, coeffs):
        b = blocks[int(t)]
        sig = (b.S @ np.concatenate([c, [dT]])).reshape(b.n_el, 8, 6)
        out.append(fem.element_von_mises(sig))
    return np.stack(out)
