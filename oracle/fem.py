"""Fine-mesh finite-element model of linear thermoelasticity (plain FP64 CPU).

TEST INFRASTRUCTURE: this package is the oracle. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it; the product (``paper_2411_12690_gb300``) never does.

What is computed follows MORE-Stress (arXiv 2411.12690), section 3:

* Eq. 1  constitutive law  sigma = lam tr(eps) 1 + 2 mu eps - alpha (3 lam + 2 mu) dT 1
* Eq. 2  Lame parameters from (E, nu)
* Eq. 4  bilinear form a(u, v) = int (lam tr eps(u) 1 + 2 mu eps(u)) : eps(v)
* Eq. 5  thermal load L(v) = int alpha (3 lam + 2 mu) dT 1 : eps(v)
* Eqs. 6-7  assembly A alpha = b, u = sum phi_i alpha_i

Discretisation (the paper meshes with Gmsh and leaves the element type open;
this oracle uses the structured voxel reading): 8-node trilinear (Q1) hexahedra
on a structured box mesh, 2x2x2 Gauss quadrature, one isotropic material per
element. Dirichlet conditions are imposed by elimination (symmetric), the linear
system is solved with a sparse direct factorisation (scipy SuperLU).

Conventions (shared *by documentation only* with the CUDA path):
* units um and MPa, so u is in um and sigma in MPa;
* node (ix, iy, iz) of an ex*ey*ez mesh has id ix + (ex+1)*(iy + (ey+1)*iz);
* DOF = 3*node + component (x, y, z);
* element (kx, ky, kz) has id kx + ex*(ky + ey*kz); its local node
  l = lx + 2 ly + 4 lz sits at mesh node (kx+lx, ky+ly, kz+lz);
* Gauss point g = gx + 2 gy + 4 gz at xi = (2 gx - 1)/sqrt(3) etc.;
* Voigt order (xx, yy, zz, xy, yz, zx) with engineering shear strains.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

VOIGT_ONE = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])


# ----------------------------------------------------------------- materials
@dataclasses.dataclass(frozen=True)
class Material:
    E: float      # Young modulus, MPa
    nu: float     # Poisson ratio
    alpha: float  # thermal expansion coefficient, 1/K


SI = Material(130e3, 0.28, 2.8e-6)
CU = Material(110e3, 0.35, 17e-6)
SIO2 = Material(71e3, 0.16, 0.5e-6)
# material ids used by the voxeliser: 0 = Si, 1 = Cu, 2 = SiO2 liner
DEFAULT_MATERIALS = (SI, CU, SIO2)


def lame(mat: Material) -> tuple[float, float]:
    """Eq. 2: lam = E nu / (1+nu) / (1-2nu), mu = E / 2 / (1+nu)."""
    lam = mat.E * mat.nu / (1.0 + mat.nu) / (1.0 - 2.0 * mat.nu)
    mu = mat.E / 2.0 / (1.0 + mat.nu)
    return lam, mu


def elasticity_matrix(mat: Material) -> np.ndarray:
    """Eq. 1 (second line) without the thermal term, as a 6x6 Voigt matrix
    acting on engineering strains: sigma = D eps."""
    lam, mu = lame(mat)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    for i in range(3):
        D[i, i] = lam + 2.0 * mu
        D[3 + i, 3 + i] = mu
    return D


def thermal_modulus(mat: Material) -> float:
    """alpha (3 lam + 2 mu): the thermal stress per unit dT (Eqs. 1, 5)."""
    lam, mu = lame(mat)
    return mat.alpha * (3.0 * lam + 2.0 * mu)


# ------------------------------------------------------------ Q1 hex element
GAUSS_1D = np.array([-1.0, 1.0]) / np.sqrt(3.0)


def _local_node_signs() -> np.ndarray:
    s = np.zeros((8, 3))
    for l in range(8):
        s[l] = [2 * (l & 1) - 1, 2 * ((l >> 1) & 1) - 1, 2 * ((l >> 2) & 1) - 1]
    return s


def gauss_points() -> np.ndarray:
    """(8, 3) reference coordinates, g = gx + 2 gy + 4 gz."""
    g = np.zeros((8, 3))
    for k in range(8):
        g[k] = [GAUSS_1D[k & 1], GAUSS_1D[(k >> 1) & 1], GAUSS_1D[(k >> 2) & 1]]
    return g


def shape_gradients(xi: np.ndarray, h: tuple[float, float, float]) -> np.ndarray:
    """Physical gradients dN_l/dx_d (8, 3) of the trilinear shape functions
    N_l = prod_d (1 + s_ld xi_d)/2 for a box element of edge lengths h."""
    s = _local_node_signs()
    grad = np.zeros((8, 3))
    for l in range(8):
        f = [(1.0 + s[l, d] * xi[d]) / 2.0 for d in range(3)]
        for d in range(3):
            df = s[l, d] / 2.0
            prod = df
            for e in range(3):
                if e != d:
                    prod *= f[e]
            grad[l, d] = prod * (2.0 / h[d])  # d xi / d x = 2 / h
    return grad


def strain_matrix(grad: np.ndarray) -> np.ndarray:
    """B (6, 24) with eps_voigt = B u_e, u_e ordered (node, component)."""
    B = np.zeros((6, 24))
    for l in range(8):
        gx, gy, gz = grad[l]
        c = 3 * l
        B[0, c + 0] = gx
        B[1, c + 1] = gy
        B[2, c + 2] = gz
        B[3, c + 0] = gy
        B[3, c + 1] = gx
        B[4, c + 1] = gz
        B[4, c + 2] = gy
        B[5, c + 0] = gz
        B[5, c + 2] = gx
    return B


def element_strain_matrices(h) -> np.ndarray:
    """(8, 6, 24): B at each Gauss point of a box element."""
    return np.stack([strain_matrix(shape_gradients(xi, h)) for xi in gauss_points()])


def element_matrices(h, mat: Material) -> tuple[np.ndarray, np.ndarray]:
    """Element stiffness Ke (24, 24) from Eq. 4 and thermal load fe (24,) per
    unit dT from Eq. 5, both by 2x2x2 Gauss quadrature (unit weights)."""
    detJ = h[0] * h[1] * h[2] / 8.0
    D = elasticity_matrix(mat)
    tm = thermal_modulus(mat)
    Ke = np.zeros((24, 24))
    fe = np.zeros(24)
    for B in element_strain_matrices(h):
        Ke += B.T @ D @ B * detJ
        fe += B.T @ (tm * VOIGT_ONE) * detJ
    return Ke, fe


# ---------------------------------------------------------------- the mesh
@dataclasses.dataclass
class BoxMesh:
    """Structured ex*ey*ez Q1 mesh of the box [0,lx]x[0,ly]x[0,lz]."""
    lx: float
    ly: float
    lz: float
    ex: int
    ey: int
    ez: int
    mat_id: np.ndarray  # (n_el,) int, element order kx fastest

    @property
    def h(self):
        return (self.lx / self.ex, self.ly / self.ey, self.lz / self.ez)

    @property
    def n_nodes(self):
        return (self.ex + 1) * (self.ey + 1) * (self.ez + 1)

    @property
    def n_el(self):
        return self.ex * self.ey * self.ez

    def node_coords(self) -> np.ndarray:
        ix, iy, iz = np.meshgrid(np.arange(self.ex + 1), np.arange(self.ey + 1),
                                 np.arange(self.ez + 1), indexing="ij")
        hx, hy, hz = self.h
        # node id = ix + (ex+1)*(iy + (ey+1)*iz)  -> order by iz, iy, ix
        c = np.stack([ix * hx, iy * hy, iz * hz], axis=-1)  # [ix, iy, iz, 3]
        return c.transpose(2, 1, 0, 3).reshape(-1, 3)

    def node_index(self) -> np.ndarray:
        """(ex+1, ey+1, ez+1) array of node ids."""
        ix, iy, iz = np.meshgrid(np.arange(self.ex + 1), np.arange(self.ey + 1),
                                 np.arange(self.ez + 1), indexing="ij")
        return ix + (self.ex + 1) * (iy + (self.ey + 1) * iz)

    def element_nodes(self) -> np.ndarray:
        """(n_el, 8) node ids, local node l = lx + 2 ly + 4 lz."""
        nid = self.node_index()
        kx, ky, kz = np.meshgrid(np.arange(self.ex), np.arange(self.ey),
                                 np.arange(self.ez), indexing="ij")
        kx, ky, kz = (a.transpose(2, 1, 0).ravel() for a in (kx, ky, kz))
        out = np.zeros((kx.size, 8), dtype=np.int64)
        for l in range(8):
            out[:, l] = nid[kx + (l & 1), ky + ((l >> 1) & 1), kz + ((l >> 2) & 1)]
        return out

    def element_dofs(self) -> np.ndarray:
        en = self.element_nodes()
        return (3 * en[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)

    def element_centroids(self) -> np.ndarray:
        hx, hy, hz = self.h
        kx, ky, kz = np.meshgrid(np.arange(self.ex), np.arange(self.ey),
                                 np.arange(self.ez), indexing="ij")
        c = np.stack([(kx + 0.5) * hx, (ky + 0.5) * hy, (kz + 0.5) * hz], axis=-1)
        return c.transpose(2, 1, 0, 3).reshape(-1, 3)

    def boundary_node_mask(self) -> np.ndarray:
        ix, iy, iz = np.meshgrid(np.arange(self.ex + 1), np.arange(self.ey + 1),
                                 np.arange(self.ez + 1), indexing="ij")
        m = ((ix == 0) | (ix == self.ex) | (iy == 0) | (iy == self.ey)
             | (iz == 0) | (iz == self.ez))
        return m.transpose(2, 1, 0).ravel()


def tsv_material_ids(lx, ly, lz, ex, ey, ez, r_cu, t_liner) -> np.ndarray:
    """Voxelised TSV unit block (section 4.2, Fig. 2): a Cu cylinder of radius
    r_cu along z through the block centre, a SiO2 liner annulus of thickness
    t_liner around it, Si elsewhere. An element takes the material of its
    centroid: Cu if r <= r_cu, SiO2 if r <= r_cu + t_liner, else Si
    (ties inclusive). r_cu <= 0 gives a pure-Si ("dummy") block (section 4.4)."""
    m = BoxMesh(lx, ly, lz, ex, ey, ez, np.zeros(ex * ey * ez, dtype=np.int64))
    c = m.element_centroids()
    r = np.hypot(c[:, 0] - lx / 2.0, c[:, 1] - ly / 2.0)
    ids = np.zeros(c.shape[0], dtype=np.int64)
    if r_cu > 0:
        ids[r <= r_cu + t_liner] = 2
        ids[r <= r_cu] = 1
    return ids


def tsv_block_mesh(lx, ly, lz, ex, ey, ez, r_cu, t_liner) -> BoxMesh:
    return BoxMesh(lx, ly, lz, ex, ey, ez,
                   tsv_material_ids(lx, ly, lz, ex, ey, ez, r_cu, t_liner))


# ---------------------------------------------------------------- assembly
def assemble(mesh: BoxMesh, materials=DEFAULT_MATERIALS):
    """Global stiffness A (CSR) and load vector b per unit dT (Eqs. 4-6)."""
    mats = np.unique(mesh.mat_id)
    Ke_tab = {}
    fe_tab = {}
    for k in mats:
        Ke_tab[int(k)], fe_tab[int(k)] = element_matrices(mesh.h, materials[int(k)])
    dofs = mesh.element_dofs()
    Ke_all = np.stack([Ke_tab[int(k)] for k in mesh.mat_id])
    fe_all = np.stack([fe_tab[int(k)] for k in mesh.mat_id])
    rows = np.broadcast_to(dofs[:, :, None], Ke_all.shape).ravel()
    cols = np.broadcast_to(dofs[:, None, :], Ke_all.shape).ravel()
    ndof = 3 * mesh.n_nodes
    A = sp.coo_matrix((Ke_all.ravel(), (rows, cols)), shape=(ndof, ndof)).tocsr()
    b = np.zeros(ndof)
    np.add.at(b, dofs.ravel(), fe_all.ravel())
    return A, b


def solve_dirichlet(A, rhs, fixed_dofs, fixed_values):
    """Solve A u = rhs with u[fixed] = values by elimination (the symmetric
    equivalent of the paper's row 'lifting', Eq. 13)."""
    ndof = A.shape[0]
    fixed = np.zeros(ndof, dtype=bool)
    fixed[fixed_dofs] = True
    free = np.flatnonzero(~fixed)
    u = np.zeros(ndof)
    u[fixed_dofs] = fixed_values
    Aff = A[free][:, free].tocsc()
    r = rhs[free] - A[free] @ u
    u[free] = spla.splu(Aff).solve(r)
    return u


# ---------------------------------------------------------------- stresses
def gauss_stresses(mesh: BoxMesh, u: np.ndarray, dT: float,
                   materials=DEFAULT_MATERIALS) -> np.ndarray:
    """(n_el, 8, 6) stress at every Gauss point by Eq. 1."""
    Bg = element_strain_matrices(mesh.h)                     # (8, 6, 24)
    ue = u[mesh.element_dofs()]                              # (n_el, 24)
    eps = np.einsum("gij,ej->egi", Bg, ue)                   # (n_el, 8, 6)
    out = np.zeros_like(eps)
    for k in np.unique(mesh.mat_id):
        sel = mesh.mat_id == k
        mat = materials[int(k)]
        D = elasticity_matrix(mat)
        out[sel] = eps[sel] @ D.T - thermal_modulus(mat) * dT * VOIGT_ONE
    return out


def von_mises(s: np.ndarray) -> np.ndarray:
    """von Mises equivalent stress of Voigt stress vectors (..., 6)."""
    sxx, syy, szz, sxy, syz, szx = (s[..., i] for i in range(6))
    return np.sqrt(0.5 * ((sxx - syy) ** 2 + (syy - szz) ** 2 + (szz - sxx) ** 2)
                   + 3.0 * (sxy ** 2 + syz ** 2 + szx ** 2))


def element_von_mises(sig_gp: np.ndarray) -> np.ndarray:
    """Per-element von Mises of the Gauss-mean stress (the mean of the eight
    Gauss-point stresses, i.e. the element-volume average for a box element)."""
    return von_mises(sig_gp.mean(axis=1))


# ------------------------------------------------ whole-array fine model
def array_mesh(block: BoxMesh, site_mat_ids: list[np.ndarray], site_type: np.ndarray) -> BoxMesh:
    """Tile one block geometry over an Ny x Nx site array. site_type[j, i]
    selects the per-element material map of the block at column i, row j."""
    Ny, Nx = site_type.shape
    ex, ey, ez = block.ex, block.ey, block.ez
    mat = np.zeros((ez, Ny * ey, Nx * ex), dtype=np.int64)
    for j in range(Ny):
        for i in range(Nx):
            mb = site_mat_ids[int(site_type[j, i])].reshape(ez, ey, ex)
            mat[:, j * ey:(j + 1) * ey, i * ex:(i + 1) * ex] = mb
    return BoxMesh(Nx * block.lx, Ny * block.ly, block.lz, Nx * ex, Ny * ey, ez, mat.ravel())


def solve_array_fem(block: BoxMesh, site_mat_ids, site_type, dT,
                    clamp_bottom=True, clamp_top=False, materials=DEFAULT_MATERIALS):
    """O-FEM: the full fine-mesh thermoelastic solve of a whole TSV array
    (Eqs. 3-7) with the bottom (and optionally top) face clamped and all other
    faces traction free. Returns (mesh, u, sigma_gp)."""
    mesh = array_mesh(block, site_mat_ids, site_type)
    A, b = assemble(mesh, materials)
    nid = mesh.node_index()
    fixed_nodes = []
    if clamp_bottom:
        fixed_nodes.append(nid[:, :, 0].ravel())
    if clamp_top:
        fixed_nodes.append(nid[:, :, -1].ravel())
    fixed_nodes = np.unique(np.concatenate(fixed_nodes)) if fixed_nodes else np.zeros(0, int)
    fixed_dofs = (3 * fixed_nodes[:, None] + np.arange(3)).ravel()
    u = solve_dirichlet(A, dT * b, fixed_dofs, np.zeros(fixed_dofs.size))
    return mesh, u, gauss_stresses(mesh, u, dT, materials)


# ------------------------------------- point evaluation (the section 5.1 metric)
def axis_locate(x: float, length: float, n: int):
    """Elements of one axis that hold coordinate x of [0, length] cut into n
    equal elements: [(element, local coordinate in [-1, 1], weight)]. An
    interior point lies in one element (weight 1); a point on the face shared
    by two elements takes both, at xi = +1 and -1, weight 1/2 each, so that a
    field that jumps across the face is read as the mean of its two one-sided
    limits; the outer faces belong to their one element."""
    h = length / n
    t = x / h
    k = int(round(t))
    if abs(t - k) <= 1e-9 * max(1.0, abs(t)):
        sides = [(k - 1, 1.0)] if k - 1 >= 0 else []
        if k <= n - 1:
            sides.append((k, -1.0))
        return [(e, xi, 1.0 / len(sides)) for e, xi in sides]
    k = min(max(int(np.floor(t)), 0), n - 1)
    return [(k, 2.0 * (t - k) - 1.0, 1.0)]


def point_stresses(mesh: BoxMesh, u: np.ndarray, dT, points: np.ndarray,
                   materials=DEFAULT_MATERIALS) -> np.ndarray:
    """Stress by Eq. 1 at arbitrary points of the mesh, from the nodal
    displacement u: in the element holding the point, sigma = D B(xi) u_e -
    alpha (3 lam + 2 mu) dT 1, with B of the trilinear shape functions at the
    point's local coordinates; on element faces, edges and corners the
    weighted mean over the elements that meet there (axis_locate per axis).
    u (n_dof,) with a scalar dT gives (n_pts, 6); u (n_dof, k) with dT of
    length k (one load per column) gives (n_pts, 6, k)."""
    en = mesh.element_nodes()
    h = mesh.h
    single = u.ndim == 1
    U = u.reshape(-1, 3, 1) if single else u.reshape(-1, 3, u.shape[1])
    dTs = np.atleast_1d(np.asarray(dT, dtype=np.float64))
    out = np.zeros((points.shape[0], 6, U.shape[2]))
    for p, (x, y, z) in enumerate(points):
        for kx, xi, wx in axis_locate(x, mesh.lx, mesh.ex):
            for ky, eta, wy in axis_locate(y, mesh.ly, mesh.ey):
                for kz, zeta, wz in axis_locate(z, mesh.lz, mesh.ez):
                    e = kx + mesh.ex * (ky + mesh.ey * kz)
                    B = strain_matrix(shape_gradients(np.array([xi, eta, zeta]), h))
                    ue = U[en[e]].reshape(24, -1)
                    mat = materials[int(mesh.mat_id[e])]
                    sig = elasticity_matrix(mat) @ (B @ ue) - thermal_modulus(mat) * np.outer(VOIGT_ONE, dTs)
                    out[p] += wx * wy * wz * sig
    return out[:, :, 0] if single else out


def midplane_grid(lx: float, ly: float, lz: float, side: int) -> np.ndarray:
    """(side^2, 3) points of the gridded cut plane of section 5.1 in one unit
    block: side x side cell-centred points ((i+1/2) lx/side, (j+1/2) ly/side)
    on the half-height plane z = lz/2, i fastest."""
    j, i = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    return np.stack([(i.ravel() + 0.5) * lx / side, (j.ravel() + 0.5) * ly / side,
                     np.full(side * side, lz / 2.0)], axis=1)


def normalized_mae(vm: np.ndarray, vm_ref: np.ndarray) -> float:
    """The error measure of section 5.1: mean absolute error of the gridded
    von Mises stress against the ground truth, divided by the largest ground
    truth von Mises stress."""
    vm = np.asarray(vm, dtype=np.float64).ravel()
    vm_ref = np.asarray(vm_ref, dtype=np.float64).ravel()
    return float(np.abs(vm - vm_ref).mean() / np.abs(vm_ref).max())


def array_grid_vm(amesh: BoxMesh, u: np.ndarray, dT: float, nx: int, ny: int, block_lx: float,
                  block_ly: float, side: int, materials=DEFAULT_MATERIALS) -> np.ndarray:
    """(nx*ny, side^2) gridded mid-plane von Mises of a whole-array fine
    solution (O-FEM), block by block in site order j*nx + i."""
    g = midplane_grid(block_lx, block_ly, amesh.lz, side)
    out = []
    for j in range(ny):
        for i in range(nx):
            pts = g + np.array([i * block_lx, j * block_ly, 0.0])
            out.append(von_mises(point_stresses(amesh, u, dT, pts, materials)))
    return np.stack(out)
