"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and names geometry; it holds none of the
method's arithmetic, so both the CUDA path and the CPU oracle tests may use it.
All draws use numpy's counter-based Philox bit generator, so a (seed, stream)
pair gives the same layout to every consumer in a process.

Workloads (geometry from section 5.2 of the paper and the benchmark configs):

* ``BLOCK_SMALL``: unit block 10x10x50 um, Cu TSV radius 2.5 um, 0.5 um SiO2
  liner, 12x12x10 Q1 hex mesh (1,440 elements), degree-2 face basis (m = 78);
* ``BLOCK_P15`` / ``BLOCK_P20``: 15x15x50 and 20x20x50 um blocks, same TSV,
  24x24x20 mesh (11,520 elements), degree-4 face basis (m = 294);
* site types: 0 = TSV block, 1 = dummy (pure Si) block of the same geometry
  (section 4.4), occupancy Bernoulli(rho);
* the 256-array batch: side log-uniform in [4, 64] (square arrays), occupancy
  U[0.5, 1], pitch 15 or 20 um, dT U[-300, -150] K;
* the request stream: Poisson arrivals, side log-uniform in [2, 128].
"""
from __future__ import annotations

import dataclasses

import numpy as np

# material table order used everywhere: 0 = Si, 1 = Cu, 2 = SiO2 (E MPa, nu, alpha 1/K)
MATERIALS = ((130e3, 0.28, 2.8e-6), (110e3, 0.35, 17e-6), (71e3, 0.16, 0.5e-6))
DT_DEFAULT = -250.0


@dataclasses.dataclass(frozen=True)
class BlockSpec:
    lx: float
    ly: float
    lz: float
    ex: int
    ey: int
    ez: int
    r_cu: float
    t_liner: float
    order: int

    def dummy(self) -> "BlockSpec":
        return dataclasses.replace(self, r_cu=0.0, t_liner=0.0)


BLOCK_SMALL = BlockSpec(10.0, 10.0, 50.0, 12, 12, 10, 2.5, 0.5, 2)
BLOCK_P15 = BlockSpec(15.0, 15.0, 50.0, 24, 24, 20, 2.5, 0.5, 4)
BLOCK_P20 = BlockSpec(20.0, 20.0, 50.0, 24, 24, 20, 2.5, 0.5, 4)


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed, stream]))


def site_types(nx: int, ny: int, occupancy: float = 1.0, seed: int = 0, stream: int = 0) -> np.ndarray:
    """(ny, nx) uint8 site map: 0 = TSV block, 1 = dummy; x index fastest in memory."""
    if occupancy >= 1.0:
        return np.zeros((ny, nx), dtype=np.uint8)
    occ = rng(seed, stream).random((ny, nx)) < occupancy
    return np.where(occ, 0, 1).astype(np.uint8)


@dataclasses.dataclass
class ArrayJob:
    nx: int
    ny: int
    site_type: np.ndarray   # (ny, nx) uint8, 0 = TSV, 1 = dummy
    pitch: int              # index into the block-variant list
    dT: float


def batch_arrays(n: int = 256, seed: int = 0, smin: int = 4, smax: int = 64,
                 n_pitch: int = 2) -> list[ArrayJob]:
    """Independent arrays: side log-uniform in [smin, smax], occupancy
    U[0.5, 1] then Bernoulli per site, pitch variant uniform, dT U[-300, -150]."""
    g = rng(seed, 1)
    jobs = []
    for k in range(n):
        s = int(round(float(np.exp(g.uniform(np.log(smin), np.log(smax))))))
        rho = g.uniform(0.5, 1.0)
        occ = g.random((s, s)) < rho
        pitch = int(g.integers(0, n_pitch))
        dT = float(g.uniform(-300.0, -150.0))
        jobs.append(ArrayJob(s, s, np.where(occ, 0, 1).astype(np.uint8), pitch, dT))
    return jobs


@dataclasses.dataclass
class Request:
    t_arrival: float        # seconds from stream start
    job: ArrayJob


def request_stream(rate: float, n: int, seed: int = 0, smin: int = 2, smax: int = 128,
                   n_pitch: int = 2) -> list[Request]:
    """Poisson arrivals at ``rate`` per second, arrays as in ``batch_arrays``
    but with side log-uniform in [smin, smax]."""
    g = rng(seed, 2)
    gaps = g.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    jobs = batch_arrays(n, seed=seed + 7919, smin=smin, smax=smax, n_pitch=n_pitch)
    return [Request(float(t[k]), jobs[k]) for k in range(n)]
