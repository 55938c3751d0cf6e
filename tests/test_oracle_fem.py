"""Pins for the fine-mesh oracle (O-FEM) against closed forms and invariants.

Each test checks the oracle against something other than itself: the algebra of
a rigid motion, the exactness of Q1 elements for linear fields (patch test),
free thermal expansion, and the Lame solution for a Cu cylinder in Si.
"""
import numpy as np
import pytest

from oracle import fem

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def rigid_modes(coords):
    """Six rigid-body motions evaluated at the given node coordinates, (3N, 6)."""
    n = coords.shape[0]
    R = np.zeros((3 * n, 6))
    for c in range(3):
        R[c::3, c] = 1.0
    x, y, z = coords.T
    # rotations about x, y, z: omega x r
    R[1::3, 3], R[2::3, 3] = -z, y
    R[0::3, 4], R[2::3, 4] = z, -x
    R[0::3, 5], R[1::3, 5] = -y, x
    return R


def test_von_mises_special_cases():
    s = 123.0
    assert fem.von_mises(np.array([s, 0, 0, 0, 0, 0])) == pytest.approx(s)          # uniaxial
    assert fem.von_mises(np.array([0, 0, 0, s, 0, 0])) == pytest.approx(np.sqrt(3) * s)  # pure shear
    assert fem.von_mises(np.array([s, s, s, 0, 0, 0])) == pytest.approx(0.0, abs=1e-12)  # hydrostatic
    # biaxial equal tension: sigma_vm = s
    assert fem.von_mises(np.array([s, s, 0, 0, 0, 0])) == pytest.approx(s)


def test_lame_parameters_closed_form():
    # E = 2 mu (1 + nu) and the bulk modulus K = lam + 2 mu / 3 = E / (3 (1 - 2 nu))
    for mat in fem.DEFAULT_MATERIALS:
        lam, mu = fem.lame(mat)
        assert 2 * mu * (1 + mat.nu) == pytest.approx(mat.E, rel=1e-14)
        assert lam + 2 * mu / 3 == pytest.approx(mat.E / (3 * (1 - 2 * mat.nu)), rel=1e-14)


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (0.8, 0.5, 2.5)])
def test_element_stiffness_invariants(h):
    Ke, fe = fem.element_matrices(h, fem.CU)
    assert np.abs(Ke - Ke.T).max() <= 1e-12 * np.abs(Ke).max()
    w = np.linalg.eigvalsh(Ke)
    assert w[:6].max() <= 1e-10 * w[-1]          # exactly six zero modes
    assert w[6] > 1e-3 * w[-1]                    # and no spurious seventh
    corners = np.array([[(l & 1) * h[0], ((l >> 1) & 1) * h[1], ((l >> 2) & 1) * h[2]] for l in range(8)])
    R = rigid_modes(corners)
    assert np.abs(Ke @ R).max() <= 1e-10 * np.abs(Ke).max()
    # a uniform dT on a free element is self-equilibrated: the load does no work on rigid motions
    assert np.abs(R.T @ fe).max() <= 1e-9 * np.abs(fe).max()


def _linear_field(coords, G, t):
    return (coords @ G.T + t).ravel()


@pytest.mark.parametrize("dT", [0.0, -250.0])
def test_patch_test_linear_field_is_exact(dT):
    """Prescribing a linear displacement on the boundary of a homogeneous
    block must reproduce it exactly inside, with constant stress D eps - tm dT 1."""
    mesh = fem.BoxMesh(3.0, 2.0, 4.0, 3, 4, 3, np.zeros(36, dtype=np.int64))
    A, b = fem.assemble(mesh)
    coords = mesh.node_coords()
    G = np.array([[1e-3, 2e-3, -1e-3], [0.5e-3, -2e-3, 1e-3], [3e-3, 0.0, 1e-3]])
    t = np.array([0.1, -0.2, 0.3])
    u_exact = _linear_field(coords, G, t)
    bnd = np.flatnonzero(mesh.boundary_node_mask())
    fixed = (3 * bnd[:, None] + np.arange(3)).ravel()
    u = fem.solve_dirichlet(A, dT * b, fixed, u_exact[fixed])
    assert np.abs(u - u_exact).max() <= 1e-12 * np.abs(u_exact).max()
    sig = fem.gauss_stresses(mesh, u, dT)
    eps = np.array([G[0, 0], G[1, 1], G[2, 2], G[0, 1] + G[1, 0], G[1, 2] + G[2, 1], G[2, 0] + G[0, 2]])
    expect = fem.elasticity_matrix(fem.SI) @ eps - fem.thermal_modulus(fem.SI) * dT * fem.VOIGT_ONE
    assert np.abs(sig - expect).max() <= 1e-9 * np.abs(expect).max()


def test_free_thermal_expansion_is_stress_free():
    """Homogeneous body, uniform dT, statically determinate (3-2-1) supports:
    u = alpha dT (x - x0) exactly and sigma = 0 (thermal load of Eq. 5)."""
    mesh = fem.BoxMesh(4.0, 3.0, 5.0, 4, 3, 5, np.zeros(60, dtype=np.int64))
    A, b = fem.assemble(mesh)
    nid = mesh.node_index()
    n0, n1, n2 = nid[0, 0, 0], nid[-1, 0, 0], nid[0, -1, 0]
    fixed = np.array([3 * n0, 3 * n0 + 1, 3 * n0 + 2, 3 * n1 + 1, 3 * n1 + 2, 3 * n2 + 2])
    dT = -250.0
    u = fem.solve_dirichlet(A, dT * b, fixed, np.zeros(6))
    u_exact = (fem.SI.alpha * dT * mesh.node_coords()).ravel()
    assert np.abs(u - u_exact).max() <= 1e-10 * np.abs(u_exact).max()
    sig = fem.gauss_stresses(mesh, u, dT)
    assert np.abs(sig).max() <= 1e-8 * fem.thermal_modulus(fem.SI) * abs(dT)


def lame_cylinder(a, cu, si, dT):
    """Closed-form plane-strain thermal misfit of a cylinder (radius a, material
    cu) in an infinite matrix (si) whose far field expands freely in plane.
    u_r = A1 r inside, u_r = A2 r + B/r outside with A2 = (1 + nu_si) alpha_si dT."""
    lam1, mu1 = fem.lame(cu)
    lam2, mu2 = fem.lame(si)
    k1 = lam1 + mu1
    A2 = (1 + si.nu) * si.alpha * dT
    B = a * a * k1 * ((1 + cu.nu) * cu.alpha - (1 + si.nu) * si.alpha) * dT / (k1 + mu2)
    return A2, B, mu2


def _lame_case(N):
    a = 2.5
    Lh = 8.0 * a
    dT = -250.0
    mesh = fem.BoxMesh(2 * Lh, 2 * Lh, 1.0, N, N, 1, np.zeros(N * N, dtype=np.int64))
    c = mesh.element_centroids() - np.array([Lh, Lh, 0.0])
    mesh.mat_id = np.where(np.hypot(c[:, 0], c[:, 1]) <= a, 1, 0)
    A, b = fem.assemble(mesh)
    A2, B, mu2 = lame_cylinder(a, fem.CU, fem.SI, dT)
    X = mesh.node_coords() - np.array([Lh, Lh, 0.0])
    r = np.maximum(np.hypot(X[:, 0], X[:, 1]), 1e-30)   # only boundary nodes (r >= 8a) are used
    ur = A2 * r + B / r
    u_ex = np.zeros_like(X)
    u_ex[:, 0] = ur * X[:, 0] / r
    u_ex[:, 1] = ur * X[:, 1] / r
    u_ex = u_ex.ravel()
    nodes = np.arange(mesh.n_nodes)
    lateral = np.flatnonzero((np.abs(X[:, 0]) > Lh - 1e-9) | (np.abs(X[:, 1]) > Lh - 1e-9))
    fixed = np.concatenate([3 * nodes + 2, 3 * lateral, 3 * lateral + 1])   # plane strain u_z = 0
    u = fem.solve_dirichlet(A, dT * b, fixed, u_ex[fixed])
    sig = fem.gauss_stresses(mesh, u, dT).mean(axis=1)
    rc = np.hypot(c[:, 0], c[:, 1])
    sel = (rc >= 1.5 * a) & (rc <= 3.0 * a)
    ct, st = c[sel, 0] / rc[sel], c[sel, 1] / rc[sel]
    s = sig[sel]
    srr = s[:, 0] * ct ** 2 + s[:, 1] * st ** 2 + 2 * s[:, 3] * ct * st
    stt = s[:, 0] * st ** 2 + s[:, 1] * ct ** 2 - 2 * s[:, 3] * ct * st
    ref = 2 * mu2 * B / a ** 2                       # |sigma| at the interface
    err = max(np.abs(srr + 2 * mu2 * B / rc[sel] ** 2).max(), np.abs(stt - 2 * mu2 * B / rc[sel] ** 2).max()) / abs(ref)
    szz_err = np.abs(s[:, 2] + fem.SI.E * fem.SI.alpha * dT).max() / abs(fem.SI.E * fem.SI.alpha * dT)
    return err, szz_err


def test_lame_cylinder_closed_form():
    """Eq. 1 physics against the Lame plane-strain solution: the error near the
    via (r in [1.5a, 3a]) falls under refinement and ends within a few percent
    (the voxel staircase makes it first order)."""
    errs = [_lame_case(N) for N in (40, 80, 160)]
    e = [x[0] for x in errs]
    assert e[0] > e[1] > e[2]
    assert e[2] < 0.05
    assert errs[2][1] < 0.02      # sigma_zz = -E alpha dT in the matrix (plane strain)


# ------------------------------------------- voxelised TSV block: census
# Hand-derived element census of the voxeliser (section 4.2, Fig. 2: Cu core of
# radius d/2 = 2.5 um, SiO2 liner of t = 0.5 um outside it, Si elsewhere; an
# element takes the material at its centroid). In a block of side p meshed by
# c x c cells (h = p / c, c even), the centroids of one quarter of a layer sit
# at offsets (a h, b h) from the axis with a, b in {1/2, 3/2, ...}. So an
# element is Cu iff a^2 + b^2 <= (2.5 / h)^2 and SiO2 iff it is not Cu and
# a^2 + b^2 <= (3.0 / h)^2; no centroid lies on either circle for these sizes
# (a^2 + b^2 = (odd^2 + odd^2) / 4 is never 9, 12.96, 16 or 23.04).
#   p = 10, c = 12 (h = 5/6): (2.5/h)^2 = 9, (3/h)^2 = 12.96.
#     Cu per quarter: (1/2,1/2) (1/2,3/2)x2 (1/2,5/2)x2 (3/2,3/2) (3/2,5/2)x2 = 8;
#     SiO2 per quarter: (5/2,5/2) [12.5] and (1/2,7/2)x2 [12.5] = 3;
#     per layer Cu 32, SiO2 12, Si 144 - 44 = 100.
#   p = 15, c = 24 (h = 5/8): (2.5/h)^2 = 16, (3/h)^2 = 23.04.
#     b-counts per a = 1/2, 3/2, 5/2, 7/2: Cu 4 + 4 + 3 + 2 = 13 per quarter;
#     within 23.04 per a = 1/2 .. 9/2: 5 + 5 + 4 + 3 + 2 = 19, so SiO2 6 per
#     quarter; per layer Cu 52, SiO2 24, Si 576 - 76 = 500.
#   p = 20, c = 24 (h = 5/6): the same radii in cells as p = 10, c = 12, so Cu
#     32, SiO2 12 and Si 576 - 44 = 532 per layer.
CENSUS = [  # (lx, cells, ez, Cu, SiO2, Si per layer)
    (10.0, 12, 10, 32, 12, 100),
    (15.0, 24, 20, 52, 24, 500),
    (20.0, 24, 20, 32, 12, 532),
]


@pytest.mark.parametrize("lx,c,ez,n_cu,n_ox,n_si", CENSUS)
def test_voxelised_tsv_census(lx, c, ez, n_cu, n_ox, n_si):
    ids = fem.tsv_material_ids(lx, lx, 50.0, c, c, ez, 2.5, 0.5).reshape(ez, c, c)   # [kz, ky, kx]
    for kz in range(ez):   # every layer identical (a straight through-via)
        assert np.array_equal(ids[kz], ids[0])
    cnt = np.bincount(ids[0].ravel(), minlength=3)
    assert tuple(cnt) == (n_si, n_cu, n_ox)
    # the axis is the block centre: the layer map has the square's eight symmetries
    lay = ids[0]
    for t in (lay[::-1, :], lay[:, ::-1], lay.T):
        assert np.array_equal(t, lay)
    # Cu at the four cells around the axis; Si in the corners
    h = c // 2
    assert np.all(lay[h - 1:h + 1, h - 1:h + 1] == 1)
    assert lay[0, 0] == lay[-1, -1] == 0
    # dummy block: all Si
    assert np.all(fem.tsv_material_ids(lx, lx, 50.0, c, c, ez, 0.0, 0.0) == 0)


def test_voxelised_liner_cells_p10():
    """The SiO2 cells of the p = 10 um, 12-cell block are exactly those with
    centroid offsets (5/2, 5/2) h (r = 2.946 um) and (1/2, 7/2) h, (7/2, 1/2) h
    (r = 2.946 um) in each quarter: the liner sits outside the Cu radius."""
    lay = fem.tsv_material_ids(10.0, 10.0, 50.0, 12, 12, 10, 2.5, 0.5).reshape(10, 12, 12)[0]
    want = set()
    for a, b in ((2.5, 2.5), (0.5, 3.5), (3.5, 0.5)):
        for sa in (-1, 1):
            for sb in (-1, 1):
                want.add((int(5.5 + sb * b + 0.5), int(5.5 + sa * a + 0.5)))   # (ky, kx)
    got = {(int(ky), int(kx)) for ky, kx in zip(*np.nonzero(lay == 2))}
    assert got == want


# ------------------------------------------------ point stresses (section 5.1)
def _trilinear_field(coords, a):
    """u = (a0 xyz + a3 x, a1 xyz + a4 y, a2 xyz + a5 z + a6 x): trilinear in
    x, y, z, so reproduced exactly by Q1 elements on a box mesh."""
    x, y, z = coords.T
    return np.stack([a[0] * x * y * z + a[3] * x, a[1] * x * y * z + a[4] * y,
                     a[2] * x * y * z + a[5] * z + a[6] * x], 1).ravel()


def _trilinear_strain(p, a):
    x, y, z = p
    return np.array([a[0] * y * z + a[3], a[1] * x * z + a[4], a[2] * x * y + a[5],
                     a[0] * x * z + a[1] * y * z, a[1] * x * y + a[2] * x * z, a[0] * x * y + a[2] * y * z + a[6]])


def test_point_stress_exact_for_trilinear_fields():
    """Inside each element the stress of a trilinear field is D eps(x) - alpha
    (3 lam + 2 mu) dT 1 with the exact strain at the point (which varies
    linearly inside the element), in the element's own material."""
    rng = np.random.default_rng(3)
    mesh = fem.BoxMesh(4.0, 3.0, 5.0, 4, 3, 5, rng.integers(0, 3, 60))
    a = rng.standard_normal(7)
    u = _trilinear_field(mesh.node_coords(), a)
    pts = rng.uniform([0, 0, 0], [4.0, 3.0, 5.0], size=(40, 3))
    sig = fem.point_stresses(mesh, u, -250.0, pts)
    for p, s in zip(pts, sig):
        e = int(p[0] // 1.0) + 4 * (int(p[1] // 1.0) + 3 * int(p[2] // 1.0))
        mat = fem.DEFAULT_MATERIALS[int(mesh.mat_id[e])]
        ref = fem.elasticity_matrix(mat) @ _trilinear_strain(p, a) + 250.0 * fem.thermal_modulus(mat) * fem.VOIGT_ONE
        assert np.abs(s - ref).max() <= 1e-10 * np.abs(ref).max()


def test_point_stress_on_faces_edges_corners_is_the_mean():
    """On a face between elements of different materials the stress jumps;
    the point value is the mean over the elements meeting there (2 on a face,
    4 on an edge, 8 at a corner), each in its own material."""
    rng = np.random.default_rng(4)
    mat = rng.integers(0, 3, 8)
    mesh = fem.BoxMesh(2.0, 2.0, 2.0, 2, 2, 2, mat)
    a = rng.standard_normal(7)
    u = _trilinear_field(mesh.node_coords(), a)
    cases = [((1.0, 0.5, 0.5), [(0, 0, 0), (1, 0, 0)]),
             ((1.0, 1.0, 0.5), [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0)]),
             ((1.0, 1.0, 1.0), [(i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1)]),
             ((0.0, 0.5, 0.5), [(0, 0, 0)]),                       # outer face: its one element
             ((2.0, 2.0, 2.0), [(1, 1, 1)])]
    for p, els in cases:
        s = fem.point_stresses(mesh, u, 100.0, np.array([p]))[0]
        eps = _trilinear_strain(np.array(p), a)
        ref = np.mean([fem.elasticity_matrix(fem.DEFAULT_MATERIALS[int(mat[i + 2 * (j + 2 * k)])]) @ eps
                       - 100.0 * fem.thermal_modulus(fem.DEFAULT_MATERIALS[int(mat[i + 2 * (j + 2 * k)])])
                       * fem.VOIGT_ONE for i, j, k in els], axis=0)
        assert np.abs(s - ref).max() <= 1e-10 * np.abs(ref).max(), p


def test_midplane_grid_and_normalized_mae():
    g = fem.midplane_grid(10.0, 20.0, 50.0, 4)
    assert g.shape == (16, 3)
    assert np.allclose(g[:4, 0], [1.25, 3.75, 6.25, 8.75]) and np.allclose(g[::4, 1], [2.5, 7.5, 12.5, 17.5])
    assert np.all(g[:, 2] == 25.0)
    ref = np.array([1.0, 4.0, 2.0, 3.0])
    assert fem.normalized_mae(ref, ref) == 0.0
    assert fem.normalized_mae(ref + 0.5, ref) == pytest.approx(0.5 / 4.0)
    assert fem.normalized_mae([0, 4, 2, 3], ref) == pytest.approx(0.25 / 4.0)
