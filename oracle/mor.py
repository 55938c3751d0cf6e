"""Model-order-reduced (MORE-Stress) reference implementation, plain FP64 CPU.

TEST INFRASTRUCTURE: part of the oracle; only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may use it.

Follows MORE-Stress (arXiv 2411.12690), section 4, in the paper's order:

* local stage (section 4.2): equally spaced Lagrange nodes on the surface of the
  unit block (Eqs. 8-10, count by Eq. 16), the Dirichlet block problem split into
  free and boundary DOFs (Eqs. 11-12), lifting (Eq. 13), the reduced local problems
  (Eq. 14) solved with ONE factorisation of A_ff reused for every right-hand side,
  giving the local basis f_i, f_T (Eq. 15);
* reduced element (section 4.3): A_element = F^T A_local F (Eq. 18) and
  b_element = F^T b_local per unit dT (Eq. 19);
* global stage (section 4.3): blocks as abstract elements, standard assembly of
  A_global, b_global over shared boundary nodes, solve of Eq. 20 (here a sparse
  direct factorisation, so there is no tolerance question), and recovery of the
  fine fields by the linear combination of Eq. 15 and the stress of Eq. 1;
* sub-modeling (section 4.4) reuses the lifting of Eq. 13 for prescribed
  boundary displacements of the array.

Element-DOF order (documented contract with the CUDA path): Lagrange node
(i, j, k) at (x_i, y_j, z_k), surface nodes only, i fastest then j then k; DOF
3*q + component for the q-th surface node (this matches the listing order
u_(0,0,0),x, u_(0,0,0),y, u_(0,0,0),z, ... of Eqs. 14-15).

Reading of the paper where it is silent (see the design notes): the basis is
taken as n_x = n_y = n_z = order + 1 unless given explicitly; eq. 19's
phi_{local,i} is read as phi_{local,p}; the global solve uses a direct method
instead of GMRES (same solution); the per-element von Mises is that of the
Gauss-mean stress.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


# ------------------------------------------------------- Lagrange (Eqs. 8-10)
def lagrange_nodes_1d(n: int, length: float) -> np.ndarray:
    """n equally spaced interpolation points on [0, length], corners included."""
    if n < 2:
        raise ValueError("need at least the two corner nodes per axis")
    return np.array([length * i / (n - 1) for i in range(n)])


def lagrange_1d(x, nodes: np.ndarray, i: int):
    """Eq. 9: the 1D Lagrange polynomial of node i evaluated at x."""
    num = np.ones_like(np.asarray(x, dtype=float))
    den = 1.0
    for j, xj in enumerate(nodes):
        if j == i:
            continue
        num = num * (x - xj)
        den *= nodes[i] - xj
    return num / den


def surface_nodes(nx: int, ny: int, nz: int) -> list[tuple[int, int, int]]:
    """Surface Lagrange nodes (i, j, k), i fastest; their number times 3 is Eq. 16."""
    out = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if i in (0, nx - 1) or j in (0, ny - 1) or k in (0, nz - 1):
                    out.append((i, j, k))
    return out


def mode_count(nx: int, ny: int, nz: int) -> int:
    """Eq. 16: n = 3 (nx ny nz - (nx-2)(ny-2)(nz-2))."""
    return 3 * (nx * ny * nz - (nx - 2) * (ny - 2) * (nz - 2))


def trace_matrix(coords: np.ndarray, lengths, nxyz) -> np.ndarray:
    """The matrix L of Eq. 14: row 3*b + c is the fine boundary DOF (node b at
    coords[b], component c); column 3*q + c is the q-th surface Lagrange node's
    component c. Entry = L_3D(r_b; i, j, k) (Eq. 8), per component (Eq. 10)."""
    nx, ny, nz = nxyz
    ax = [lagrange_nodes_1d(n, l) for n, l in zip(nxyz, lengths)]
    nodes = surface_nodes(nx, ny, nz)
    nb = coords.shape[0]
    L = np.zeros((3 * nb, 3 * len(nodes)))
    for q, (i, j, k) in enumerate(nodes):
        v = (lagrange_1d(coords[:, 0], ax[0], i) * lagrange_1d(coords[:, 1], ax[1], j)
             * lagrange_1d(coords[:, 2], ax[2], k))
        for c in range(3):
            L[c::3, 3 * q + c] = v
    return L


# --------------------------------------------------------- local stage
@dataclasses.dataclass
class ReducedBlock:
    """Reduced model of one unit block (the output of the local stage)."""
    mesh: fem.BoxMesh
    nxyz: tuple[int, int, int]
    m: int
    F: np.ndarray        # (n_dof, m+1): columns f_0..f_{m-1}, f_T (Eq. 15)
    K_r: np.ndarray      # (m, m)   A_element (Eq. 18)
    b_r: np.ndarray      # (m,)     b_element per unit dT (Eq. 19)
    S: np.ndarray        # (n_el*8*6, m+1) stress modes at Gauss points; row (e*8+g)*6+comp
    A_local: sp.csr_matrix
    b_local: np.ndarray

    @property
    def n_el(self):
        return self.mesh.n_el


def local_stage(mesh: fem.BoxMesh, nxyz, materials=fem.DEFAULT_MATERIALS) -> ReducedBlock:
    """Section 4.2 for one unit block, then Eqs. 18-19 and the stress modes."""
    nxyz = tuple(int(v) for v in nxyz)
    A, b = fem.assemble(mesh, materials)                 # Eq. 11 per unit dT
    ndof = A.shape[0]
    coords = mesh.node_coords()
    bmask = mesh.boundary_node_mask()
    bnodes = np.flatnonzero(bmask)
    fnodes = np.flatnonzero(~bmask)
    bc = (3 * bnodes[:, None] + np.arange(3)).ravel()    # Eq. 12 partition
    fr = (3 * fnodes[:, None] + np.arange(3)).ravel()
    L = trace_matrix(coords[bnodes], (mesh.lx, mesh.ly, mesh.lz), nxyz)
    m = L.shape[1]
    assert m == mode_count(*nxyz)
    A_ff = A[fr][:, fr].tocsc()
    A_fbc = A[fr][:, bc]
    lu = spla.splu(A_ff)                                  # factorise once (section 4.2, last paragraph)
    rhs = np.zeros((fr.size, m + 1))
    rhs[:, :m] = -(A_fbc @ L)                             # Eq. 14 with dT = 0, unit nodal value
    rhs[:, m] = b[fr]                                     # dT = 1, zero nodal values
    X = lu.solve(rhs)
    F = np.zeros((ndof, m + 1))                           # Eq. 15 basis, fine-mesh coefficients
    F[bc, :m] = L
    F[fr, :] = X
    Fm = F[:, :m]
    K_r = Fm.T @ (A @ Fm)                                 # Eq. 18
    b_r = Fm.T @ b                                        # Eq. 19 per unit dT
    S = stress_modes(mesh, F, materials)
    return ReducedBlock(mesh, nxyz, m, F, K_r, b_r, S, A, b)


def stress_modes(mesh: fem.BoxMesh, F: np.ndarray, materials=fem.DEFAULT_MATERIALS) -> np.ndarray:
    """Stress of each basis column at each Gauss point by Eq. 1: column i < m
    is sigma(f_i) with dT = 0; column m is sigma(f_T) with dT = 1, i.e. it holds
    the thermal term -alpha (3 lam + 2 mu) 1 as well."""
    Bg = fem.element_strain_matrices(mesh.h)              # (8, 6, 24)
    dofs = mesh.element_dofs()                            # (n_el, 24)
    m1 = F.shape[1]
    S = np.zeros((mesh.n_el, 8, 6, m1))
    for k in np.unique(mesh.mat_id):
        sel = np.flatnonzero(mesh.mat_id == k)
        mat = materials[int(k)]
        D = fem.elasticity_matrix(mat)
        Fe = F[dofs[sel]]                                 # (ne, 24, m1)
        eps = np.einsum("gij,ejc->egic", Bg, Fe)          # (ne, 8, 6, m1)
        sig = np.einsum("ij,egjc->egic", D, eps)
        sig[:, :, :, m1 - 1] -= fem.thermal_modulus(mat) * fem.VOIGT_ONE
        S[sel] = sig
    return S.reshape(mesh.n_el * 48, m1)


def stiffness_by_condensation(block: ReducedBlock) -> np.ndarray:
    """K_r computed a second way, as L^T (A_bb - A_bf A_ff^-1 A_fb) L (the Schur
    complement on the boundary DOFs restricted to the Lagrange trace)."""
    mesh = block.mesh
    A = block.A_local
    bmask = mesh.boundary_node_mask()
    bnodes = np.flatnonzero(bmask)
    fnodes = np.flatnonzero(~bmask)
    bc = (3 * bnodes[:, None] + np.arange(3)).ravel()
    fr = (3 * fnodes[:, None] + np.arange(3)).ravel()
    L = trace_matrix(mesh.node_coords()[bnodes], (mesh.lx, mesh.ly, mesh.lz), block.nxyz)
    A_bb = A[bc][:, bc]
    A_bf = A[bc][:, fr]
    lu = spla.splu(A[fr][:, fr].tocsc())
    AbbL = A_bb @ L
    W = lu.solve(np.asarray((A_bf.T @ L)))
    return L.T @ AbbL - L.T @ (A_bf @ W)


# --------------------------------------------------------- global stage
@dataclasses.dataclass
class GlobalSolution:
    nxyz: tuple[int, int, int]
    site_type: np.ndarray      # (Ny, Nx)
    dT: float
    lattice_shape: tuple[int, int, int]   # (X, Y, Z) Lagrange lattice points
    gdof: np.ndarray           # (N_blocks, m) global DOF index of each element DOF
    u: np.ndarray              # (n_global_dof,) nodal displacements (Eq. 20)
    coeffs: np.ndarray         # (N_blocks, m) element DOFs, blocks ordered j*Nx + i
    A_global: sp.csr_matrix
    b_global: np.ndarray
    fixed: np.ndarray          # bool mask of constrained global DOFs
    lattice_of_dof: np.ndarray # (n_global_dof,) lattice point id (gz*Y + gy)*X + gx


def element_dof_map(nxyz, site_type: np.ndarray):
    """Standard assembly bookkeeping (section 4.3): block (i, j) local Lagrange
    node (a, b, c) sits on global lattice point (i (nx-1) + a, j (ny-1) + b, c).
    Returns (gdof (N_blocks, m), lattice id per global DOF, lattice shape)."""
    nx, ny, nz = nxyz
    Ny, Nx = site_type.shape
    X, Y, Z = Nx * (nx - 1) + 1, Ny * (ny - 1) + 1, nz
    snodes = surface_nodes(nx, ny, nz)
    m = 3 * len(snodes)
    lat = np.zeros((Ny * Nx, len(snodes)), dtype=np.int64)
    for j in range(Ny):
        for i in range(Nx):
            for q, (a, b, c) in enumerate(snodes):
                gx, gy = i * (nx - 1) + a, j * (ny - 1) + b
                lat[j * Nx + i, q] = (c * Y + gy) * X + gx
    used, inv = np.unique(lat.ravel(), return_inverse=True)
    gnode = inv.reshape(lat.shape)
    gdof = (3 * gnode[:, :, None] + np.arange(3)).reshape(Ny * Nx, m)
    lattice_of_dof = np.repeat(used, 3)
    return gdof, lattice_of_dof, (X, Y, Z)


def assemble_global(blocks: list[ReducedBlock], site_type: np.ndarray, dT: float):
    nxyz = blocks[0].nxyz
    gdof, lattice_of_dof, shape = element_dof_map(nxyz, site_type)
    n = lattice_of_dof.size
    m = blocks[0].m
    st = site_type.ravel()
    Kall = np.stack([blocks[int(t)].K_r for t in st])    # (N, m, m)
    rows = np.broadcast_to(gdof[:, :, None], Kall.shape).ravel()
    cols = np.broadcast_to(gdof[:, None, :], Kall.shape).ravel()
    A = sp.coo_matrix((Kall.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    b = np.zeros(n)
    np.add.at(b, gdof.ravel(), dT * np.stack([blocks[int(t)].b_r for t in st]).ravel())
    assert all(blk.m == m and blk.nxyz == nxyz for blk in blocks)
    return A, b, gdof, lattice_of_dof, shape


def fixed_mask(lattice_of_dof, shape, clamp_bottom=True, clamp_top=False):
    X, Y, Z = shape
    gz = lattice_of_dof // (X * Y)
    fixed = np.zeros(lattice_of_dof.size, dtype=bool)
    if clamp_bottom:
        fixed |= gz == 0
    if clamp_top:
        fixed |= gz == Z - 1
    return fixed


def global_stage(blocks: list[ReducedBlock], site_type: np.ndarray, dT: float,
                 clamp_bottom=True, clamp_top=False, prescribed=None) -> GlobalSolution:
    """Assemble and solve Eq. 20. A clamped face fixes every global DOF on it
    (the interpolant of a face depends only on that face's nodes, so the whole
    face is clamped exactly). ``prescribed`` optionally maps global DOF index ->
    value for sub-modeling (section 4.4), imposed by lifting (Eq. 13)."""
    site_type = np.asarray(site_type)
    A, b, gdof, lat, shape = assemble_global(blocks, site_type, dT)
    fixed = fixed_mask(lat, shape, clamp_bottom, clamp_top)
    vals = np.zeros(lat.size)
    if prescribed is not None:
        idx = np.asarray(list(prescribed.keys()), dtype=np.int64)
        fixed[idx] = True
        vals[idx] = np.asarray(list(prescribed.values()))
    fixed_dofs = np.flatnonzero(fixed)
    u = fem.solve_dirichlet(A, b, fixed_dofs, vals[fixed_dofs])
    return GlobalSolution(blocks[0].nxyz, site_type, dT, shape, gdof, u, u[gdof], A, b, fixed, lat)


# ------------------------------------------------------------- recovery
def block_displacement(block: ReducedBlock, c: np.ndarray, dT: float) -> np.ndarray:
    """Eq. 15: u_local = dT f_T + sum_i c_i f_i (fine-mesh nodal vector)."""
    return block.F @ np.concatenate([c, [dT]])


def block_gauss_stress(block: ReducedBlock, c: np.ndarray, dT: float) -> np.ndarray:
    """(n_el, 8, 6) Gauss-point stress: Eq. 1 applied to the Eq. 15 field, done
    straight from the fine displacement (not through the stored modes S)."""
    u = block_displacement(block, c, dT)
    return fem.gauss_stresses(block.mesh, u, dT)


def recover_vm(blocks: list[ReducedBlock], sol: GlobalSolution, via_modes=True) -> np.ndarray:
    """(N_blocks, n_el) per-element von Mises of the Gauss-mean stress."""
    st = sol.site_type.ravel()
    out = []
    for e, t in enumerate(st):
        blk = blocks[int(t)]
        if via_modes:
            sig = (blk.S @ np.concatenate([sol.coeffs[e], [sol.dT]])).reshape(blk.n_el, 8, 6)
        else:
            sig = block_gauss_stress(blk, sol.coeffs[e], sol.dT)
        out.append(fem.element_von_mises(sig))
    return np.stack(out)


def recover_vm_grid(blocks: list[ReducedBlock], sol: GlobalSolution, side: int) -> np.ndarray:
    """(N_blocks, side^2) gridded von Mises on the half-height cut plane of
    every block (section 5.1): the fine field of Eq. 15, u_e = F [c_e; dT],
    evaluated point by point with Eq. 1 (fem.point_stresses on the block's
    own mesh)."""
    out = []
    grids = {}
    for e, t in enumerate(sol.site_type.ravel()):
        blk = blocks[int(t)]
        m = blk.mesh
        key = (m.lx, m.ly, m.lz)
        if key not in grids:
            grids[key] = fem.midplane_grid(m.lx, m.ly, m.lz, side)
        u = block_displacement(blk, sol.coeffs[e], sol.dT)
        out.append(fem.von_mises(fem.point_stresses(m, u, sol.dT, grids[key])))
    return np.stack(out)


def grid_stress_modes(block: ReducedBlock, side: int) -> np.ndarray:
    """(side^2, 6, m+1) stress of every basis column of Eq. 15 at the
    half-height grid points (Eq. 1; column m is f_T with dT = 1, so it holds
    the thermal term): sigma at point p = modes[p] @ [c; dT]."""
    m = block.mesh
    loads = np.zeros(block.m + 1)
    loads[-1] = 1.0
    return fem.point_stresses(m, block.F, loads, fem.midplane_grid(m.lx, m.ly, m.lz, side))
