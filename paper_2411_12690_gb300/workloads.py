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


# Blocks of the paper's scenarios with its default (4,4,4) interpolation nodes
# (degree 3, m = 168): pitch 15 um on the 24x24x20 mesh, pitch 10 um on a
# 16x16x20 mesh of the same element size.
BLOCK_P15_O3 = BlockSpec(15.0, 15.0, 50.0, 24, 24, 20, 2.5, 0.5, 3)
BLOCK_P10_O3 = BlockSpec(10.0, 10.0, 50.0, 16, 16, 20, 2.5, 0.5, 3)


def submodel_sites(n_tsv: int = 15, rings: int = 2) -> np.ndarray:
    """Site map of a sub-model (section 4.4, scenario 2 of section 5.1): an
    n_tsv x n_tsv TSV array (type 0) inside `rings` rings of dummy blocks
    (type 1)."""
    s = n_tsv + 2 * rings
    st = np.ones((s, s), dtype=np.uint8)
    st[rings:rings + n_tsv, rings:rings + n_tsv] = 0
    return st


def submodel_boundary(nx: int, ny: int, spec: BlockSpec, seed: int = 0, dT: float = DT_DEFAULT):
    """A synthetic coarse-model displacement field on the boundary of a
    sub-model (it stands in for the package-level coarse solution that the
    paper takes from ANSYS): a smooth warpage-like field, sampled at every
    Lagrange-lattice point on the six outer faces of an nx x ny array of
    `spec` blocks. With (xc, yc, zc) the centre of the sub-model,
        u_x = e_x X + g_x X^2 + t Y - k_x X Z,
        u_y = e_y Y + g_y Y^2 - t X - k_y Y Z,
        u_z = e_z Z + (k_x X^2 + k_y Y^2) / 2 + w X Y,
    X = x - xc, Y = y - yc, Z = z - zc: an in-plane mismatch strain of the
    order of alpha_Si |dT| (e_x, e_y, e_z), curvatures k_x, k_y of a warping
    package, a twist w, an in-plane rotation t and a gradient g of the
    background strain across the sub-model. Coefficients are drawn from the
    seed. Returns (dof, value): lattice DOF indices 3 ((z Y + y) X + x) + comp
    (the prescribed-DOF convention of the C ABI) and displacements in um."""
    g = rng(seed, 3)
    n = spec.order + 1
    X, Y, Z = nx * (n - 1) + 1, ny * (n - 1) + 1, n
    Lx, Ly, Lz = nx * spec.lx, ny * spec.ly, spec.lz
    eps = 2.8e-6 * abs(dT)
    ex, ey, ez = eps * g.uniform(0.5, 1.5, 3)
    kx, ky = eps / max(Lx, Ly) * g.uniform(-2.0, 2.0, 2)
    w = eps / (Lx * Ly) ** 0.5 * g.uniform(-1.0, 1.0)
    t = eps * g.uniform(-0.2, 0.2)
    gx_, gy_ = eps / max(Lx, Ly) * g.uniform(-1.0, 1.0, 2)
    iz, iy, ix = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    on = (ix == 0) | (ix == X - 1) | (iy == 0) | (iy == Y - 1) | (iz == 0) | (iz == Z - 1)
    ix, iy, iz = ix[on], iy[on], iz[on]
    xs = ix * (spec.lx / (n - 1)) - Lx / 2
    ys = iy * (spec.ly / (n - 1)) - Ly / 2
    zs = iz * (spec.lz / (n - 1)) - Lz / 2
    ux = ex * xs + gx_ * xs ** 2 + t * ys - kx * xs * zs
    uy = ey * ys + gy_ * ys ** 2 - t * xs - ky * ys * zs
    uz = ez * zs + 0.5 * (kx * xs ** 2 + ky * ys ** 2) + w * xs * ys
    node = (iz * Y + iy) * X + ix
    dof = (3 * node[:, None] + np.arange(3)[None, :]).ravel().astype(np.int64)
    val = np.stack([ux, uy, uz], axis=1).ravel()
    return dof, val
