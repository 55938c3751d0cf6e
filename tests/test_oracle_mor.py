"""Pins for the reduced-model oracle (O-MOR).

The strongest pin is exact static condensation: with a Lagrange node on every
fine boundary node the trace is the identity, so the reduced global solve must
reproduce the full fine-mesh FEM (O-FEM) to round-off. The others: the mode
count printed in Table 3 (Eq. 16), rigid-body null space and symmetry of
A_element (Eq. 18), self-equilibrated b_element (Eq. 19), orthogonality of f_T to
the f_i, reproduction of free thermal expansion, linearity in dT, the Galerkin
energy ordering for nested bases, and convergence of von Mises to O-FEM as the
basis order rises (the trend of Table 3).
"""
import os

import numpy as np
import pytest

from oracle import fem, mor

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_mode_count_table3():
    for nx, ny, nz, n in read_golden("table3_mode_counts.txt"):
        nx, ny, nz, n = int(nx), int(ny), int(nz), int(n)
        assert mor.mode_count(nx, ny, nz) == n
        assert 3 * len(mor.surface_nodes(nx, ny, nz)) == n


def test_lagrange_is_cardinal_and_reproduces_polynomials():
    nodes = mor.lagrange_nodes_1d(5, 10.0)
    for i in range(5):
        v = np.array([mor.lagrange_1d(x, nodes, i) for x in nodes])
        assert np.allclose(v, np.eye(5)[i], atol=0, rtol=0)
    x = np.linspace(0, 10, 17)
    poly = 0.3 * x ** 4 - x ** 2 + 2.0
    interp = sum(mor.lagrange_1d(x, nodes, i) * (0.3 * nodes[i] ** 4 - nodes[i] ** 2 + 2.0) for i in range(5))
    assert np.abs(interp - poly).max() < 1e-9 * np.abs(poly).max()


@pytest.fixture(scope="module")
def small_block():
    mesh = fem.tsv_block_mesh(10.0, 10.0, 50.0, 12, 12, 10, 2.5, 0.5)
    return mor.local_stage(mesh, (3, 3, 3))


def _lagrange_coords(blk):
    mesh = blk.mesh
    ax = [mor.lagrange_nodes_1d(n, l) for n, l in zip(blk.nxyz, (mesh.lx, mesh.ly, mesh.lz))]
    return np.array([[ax[0][i], ax[1][j], ax[2][k]] for (i, j, k) in mor.surface_nodes(*blk.nxyz)])


def _rigid(coords):
    n = coords.shape[0]
    R = np.zeros((3 * n, 6))
    for c in range(3):
        R[c::3, c] = 1.0
    x, y, z = coords.T
    R[1::3, 3], R[2::3, 3] = -z, y
    R[0::3, 4], R[2::3, 4] = z, -x
    R[0::3, 5], R[1::3, 5] = -y, x
    return R


def test_reduced_element_invariants(small_block):
    blk = small_block
    K = blk.K_r
    assert K.shape == (78, 78)
    assert np.abs(K - K.T).max() <= 1e-13 * np.abs(K).max()
    R = _rigid(_lagrange_coords(blk))
    assert np.abs(K @ R).max() <= 1e-10 * np.abs(K).max()           # 6 reduced rigid motions
    w = np.linalg.eigvalsh(0.5 * (K + K.T))
    assert w[:6].max() <= 1e-12 * w[-1] and w[6] > 1e-6 * w[-1]
    assert np.abs(R.T @ blk.b_r).max() <= 1e-10 * np.abs(blk.b_r).max()   # self-equilibrated load
    # A_element two ways: F^T A F (Eq. 18) and the boundary Schur complement
    K2 = mor.stiffness_by_condensation(blk)
    assert np.abs(K - K2).max() <= 1e-10 * np.abs(K).max()
    # f_T is A-orthogonal to every f_i (f_T vanishes on the boundary, f_i is discrete-harmonic)
    AF = blk.A_local @ blk.F
    cross = blk.F[:, :78].T @ AF[:, 78]
    assert np.abs(cross).max() <= 1e-9 * np.abs(K).max() * np.abs(blk.F[:, 78]).max()


def test_basis_reproduces_free_expansion():
    """A homogeneous block under uniform dT with the linear boundary trace
    alpha dT x is stress-free; the Eq. 15 combination must reproduce it."""
    mesh = fem.tsv_block_mesh(10.0, 10.0, 50.0, 6, 6, 5, 0.0, 0.0)
    blk = mor.local_stage(mesh, (3, 3, 3))
    dT = -250.0
    c = (fem.SI.alpha * dT * _lagrange_coords(blk)).ravel()
    u = mor.block_displacement(blk, c, dT)
    u_ex = (fem.SI.alpha * dT * mesh.node_coords()).ravel()
    assert np.abs(u - u_ex).max() <= 1e-10 * np.abs(u_ex).max()
    sig = blk.S @ np.concatenate([c, [dT]])
    assert np.abs(sig).max() <= 1e-7 * fem.thermal_modulus(fem.SI) * abs(dT)


def _site_mats(mesh_tsv, mesh_dummy):
    return [mesh_tsv.mat_id, mesh_dummy.mat_id]


def test_exact_static_condensation_equals_fem():
    """Lagrange nodes on every fine boundary node: L = identity on the boundary
    DOFs, the reduced solve is static condensation, and O-MOR must equal O-FEM."""
    ex, ey, ez = 4, 4, 3
    tsv = fem.tsv_block_mesh(10.0, 10.0, 20.0, ex, ey, ez, 2.5, 0.5)
    dum = fem.tsv_block_mesh(10.0, 10.0, 20.0, ex, ey, ez, 0.0, 0.0)
    nxyz = (ex + 1, ey + 1, ez + 1)
    blocks = [mor.local_stage(tsv, nxyz), mor.local_stage(dum, nxyz)]
    st = np.array([[0, 1], [0, 0]])
    dT = -250.0
    sol = mor.global_stage(blocks, st, dT)
    amesh, u_fem, sig_fem = fem.solve_array_fem(tsv, _site_mats(tsv, dum), st, dT)
    nid = amesh.node_index()
    worst = 0.0
    for j in range(2):
        for i in range(2):
            blk = blocks[st[j, i]]
            ub = mor.block_displacement(blk, sol.coeffs[j * 2 + i], dT).reshape(-1, 3)
            sub = nid[i * ex:(i + 1) * ex + 1, j * ey:(j + 1) * ey + 1, :]     # [ix, iy, iz]
            ids = sub.transpose(2, 1, 0).ravel()
            uf = u_fem.reshape(-1, 3)[ids]
            worst = max(worst, np.abs(ub - uf).max() / np.abs(u_fem).max())
    assert worst <= 1e-10
    vm_mor = mor.recover_vm(blocks, sol)
    vm_fem = fem.element_von_mises(sig_fem).reshape(ez, 2 * ey, 2 * ex)
    for j in range(2):
        for i in range(2):
            ref = vm_fem[:, j * ey:(j + 1) * ey, i * ex:(i + 1) * ex].ravel()
            assert np.abs(vm_mor[j * 2 + i] - ref).max() <= 1e-9 * vm_fem.max()


def _energy_fine_blocks(blocks, sol):
    """Total potential energy 1/2 a(u,u) - dT L1(u) summed over the blocks' fine fields."""
    e = 0.0
    for k, t in enumerate(sol.site_type.ravel()):
        blk = blocks[int(t)]
        u = mor.block_displacement(blk, sol.coeffs[k], sol.dT)
        e += 0.5 * u @ (blk.A_local @ u) - sol.dT * (u @ blk.b_local)
    return e


def test_galerkin_energy_ordering_and_vm_convergence():
    """Nested face spaces Q1 c Q2 c Q4 give nested reduced spaces inside the
    fine FE space, so Pi_FEM <= Pi_MOR(4) <= Pi_MOR(2) <= Pi_MOR(1); the
    von Mises error to O-FEM falls as the order rises (cf. Table 3)."""
    spec = dict(lx=10.0, ly=10.0, lz=50.0, ex=12, ey=12, ez=10)
    tsv = fem.tsv_block_mesh(**spec, r_cu=2.5, t_liner=0.5)
    dum = fem.tsv_block_mesh(**spec, r_cu=0.0, t_liner=0.0)
    st = np.array([[0, 0], [1, 0]])
    dT = -250.0
    amesh, u_fem, sig_fem = fem.solve_array_fem(tsv, _site_mats(tsv, dum), st, dT)
    A, b = fem.assemble(amesh)
    pi_fem = 0.5 * u_fem @ (A @ u_fem) - dT * (u_fem @ b)
    vm_fem = fem.element_von_mises(sig_fem).reshape(10, 24, 24)
    pis, errs = [], []
    for order in (1, 2, 4):
        n = order + 1
        blocks = [mor.local_stage(tsv, (n, n, n)), mor.local_stage(dum, (n, n, n))]
        sol = mor.global_stage(blocks, st, dT)
        pis.append(_energy_fine_blocks(blocks, sol))
        # reduced energy equals the fine one (consistency of K_r, b_r with F)
        Af, bf = sol.A_global, sol.b_global
        red = 0.5 * sol.u @ (Af @ sol.u) - sol.u @ bf
        bubble = sum(0.5 * dT * dT * (blocks[int(t)].F[:, -1] @ (blocks[int(t)].A_local @ blocks[int(t)].F[:, -1]))
                     - dT * dT * (blocks[int(t)].F[:, -1] @ blocks[int(t)].b_local) for t in st.ravel())
        assert red + bubble == pytest.approx(pis[-1], rel=1e-10)
        vm = mor.recover_vm(blocks, sol)
        err = 0.0
        for j in range(2):
            for i in range(2):
                ref = vm_fem[:, j * 12:(j + 1) * 12, i * 12:(i + 1) * 12].ravel()
                err += np.abs(vm[j * 2 + i] - ref).sum()
        errs.append(err / (4 * 1440) / vm_fem.max())
    assert pi_fem < pis[2]
    assert pis[2] < pis[1] < pis[0]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.02


def test_linearity_in_dT(small_block):
    st = np.zeros((2, 3), dtype=int)
    s1 = mor.global_stage([small_block], st, 1.0)
    s2 = mor.global_stage([small_block], st, -250.0)
    assert np.abs(s2.u + 250.0 * s1.u).max() <= 1e-12 * np.abs(s2.u).max()


def test_recovery_by_modes_equals_direct_stress(small_block):
    st = np.zeros((2, 2), dtype=int)
    sol = mor.global_stage([small_block], st, -250.0)
    a = mor.recover_vm([small_block], sol, via_modes=True)
    b = mor.recover_vm([small_block], sol, via_modes=False)
    assert np.abs(a - b).max() <= 1e-11 * a.max()


def test_clamped_face_is_clamped_in_the_fine_field(small_block):
    st = np.zeros((1, 2), dtype=int)
    sol = mor.global_stage([small_block], st, -250.0)
    mesh = small_block.mesh
    bottom = mesh.node_index()[:, :, 0].ravel()
    for k in range(2):
        u = mor.block_displacement(small_block, sol.coeffs[k], -250.0).reshape(-1, 3)
        assert np.abs(u[bottom]).max() == 0.0


def _mirror_checks(u3, tol):
    """u3[z, y, x, comp] on a grid symmetric about its mid-planes, of a
    homogeneous body under a uniform dT with both z faces clamped: reflection
    about z = h/2 keeps u_x, u_y and flips u_z; reflection about x = L/2 flips
    u_x and keeps u_y, u_z (and likewise in y)."""
    zr = u3[::-1]
    assert np.abs(zr[..., :2] - u3[..., :2]).max() <= tol
    assert np.abs(zr[..., 2] + u3[..., 2]).max() <= tol
    xr = u3[:, :, ::-1]
    assert np.abs(xr[..., 0] + u3[..., 0]).max() <= tol
    assert np.abs(xr[..., 1:] - u3[..., 1:]).max() <= tol
    yr = u3[:, ::-1]
    assert np.abs(yr[..., 1] + u3[..., 1]).max() <= tol
    assert np.abs(yr[..., [0, 2]] - u3[..., [0, 2]]).max() <= tol


def test_top_and_bottom_clamp_symmetry():
    """Scenario 1 of section 5.2 clamps the top and the bottom face. For a
    homogeneous (pure-Si) array under uniform dT the clamped slab is symmetric
    about its mid-plane: both z faces stay fixed, u_z vanishes on the
    mid-plane, u_x, u_y are even and u_z odd in z - h/2 (O-FEM and O-MOR);
    with the bottom clamp alone the free top face rises and the symmetry is
    lost. Clamping the wrong layer, or not clamping the top, breaks these."""
    dT = -250.0
    ex, ey, ez = 4, 4, 6
    dum = fem.tsv_block_mesh(10.0, 10.0, 20.0, ex, ey, ez, 0.0, 0.0)
    st = np.zeros((2, 3), dtype=int)
    amesh, u, _ = fem.solve_array_fem(dum, [dum.mat_id], st, dT, clamp_bottom=True, clamp_top=True)
    u3 = u.reshape(ez + 1, 2 * ey + 1, 3 * ex + 1, 3)
    scale = np.abs(u3).max()
    assert scale > 0
    assert np.abs(u3[0]).max() == 0.0 and np.abs(u3[-1]).max() == 0.0
    assert np.abs(u3[ez // 2, :, :, 2]).max() <= 1e-12 * scale
    _mirror_checks(u3, 1e-11 * scale)
    _, ub, _ = fem.solve_array_fem(dum, [dum.mat_id], st, dT, clamp_bottom=True, clamp_top=False)
    assert np.abs(ub.reshape(u3.shape)[-1, :, :, 2]).max() > 0.1 * scale   # free top face moves

    blk = mor.local_stage(dum, (3, 3, 3))
    sol = mor.global_stage([blk], st, dT, clamp_bottom=True, clamp_top=True)
    X, Y, Z = sol.lattice_shape
    lat = np.zeros((Z, Y, X, 3))
    idx = sol.lattice_of_dof.reshape(-1, 3)[:, 0]
    lat.reshape(-1, 3)[idx] = sol.u.reshape(-1, 3)
    s2 = np.abs(lat).max()
    assert s2 > 0
    assert np.abs(lat[0]).max() == 0.0 and np.abs(lat[-1]).max() == 0.0
    assert np.abs(lat[Z // 2, :, :, 2]).max() <= 1e-12 * s2
    _mirror_checks(lat, 1e-11 * s2)
    fixed = sol.fixed.reshape(-1, 3)
    gz = idx // (X * Y)
    assert np.array_equal(fixed.all(axis=1), (gz == 0) | (gz == Z - 1))


def test_exact_static_condensation_top_clamped():
    """The exact static-condensation pin (every fine boundary node a Lagrange
    node) with the top face clamped as well: O-MOR's clamp of the top lattice
    layer equals O-FEM's clamp of the top mesh face."""
    ex, ey, ez = 4, 4, 3
    tsv = fem.tsv_block_mesh(10.0, 10.0, 20.0, ex, ey, ez, 2.5, 0.5)
    dum = fem.tsv_block_mesh(10.0, 10.0, 20.0, ex, ey, ez, 0.0, 0.0)
    nxyz = (ex + 1, ey + 1, ez + 1)
    blocks = [mor.local_stage(tsv, nxyz), mor.local_stage(dum, nxyz)]
    st = np.array([[0, 1, 0]])
    dT = -250.0
    sol = mor.global_stage(blocks, st, dT, clamp_bottom=True, clamp_top=True)
    amesh, u_fem, _ = fem.solve_array_fem(tsv, _site_mats(tsv, dum), st, dT, clamp_bottom=True, clamp_top=True)
    nid = amesh.node_index()
    for i in range(3):
        blk = blocks[st[0, i]]
        ub = mor.block_displacement(blk, sol.coeffs[i], dT).reshape(-1, 3)
        ids = nid[i * ex:(i + 1) * ex + 1, 0:ey + 1, :].transpose(2, 1, 0).ravel()
        assert np.abs(ub - u_fem.reshape(-1, 3)[ids]).max() <= 1e-10 * np.abs(u_fem).max()


def test_exact_condensation_gridded_von_mises_equals_fem():
    """The gridded mid-plane von Mises of section 5.1 (point values of the
    fine field of Eq. 15) equals O-FEM's at the same points when the reduced
    basis holds every fine boundary node; the mesh has an even number of
    layers, so the plane runs along element faces (two-sided means)."""
    ex, ey, ez = 4, 4, 4
    tsv = fem.tsv_block_mesh(10.0, 10.0, 20.0, ex, ey, ez, 2.5, 0.5)
    dum = fem.tsv_block_mesh(10.0, 10.0, 20.0, ex, ey, ez, 0.0, 0.0)
    nxyz = (ex + 1, ey + 1, ez + 1)
    blocks = [mor.local_stage(tsv, nxyz), mor.local_stage(dum, nxyz)]
    st = np.array([[0, 1], [0, 0]])
    dT = -250.0
    sol = mor.global_stage(blocks, st, dT)
    amesh, u_fem, _ = fem.solve_array_fem(tsv, _site_mats(tsv, dum), st, dT)
    g_mor = mor.recover_vm_grid(blocks, sol, 6)
    g_fem = fem.array_grid_vm(amesh, u_fem, dT, 2, 2, 10.0, 10.0, 6)
    assert np.abs(g_mor - g_fem).max() <= 1e-9 * g_fem.max()


def test_gridded_error_falls_with_the_basis_order():
    """The normalised MAE of the gridded von Mises against O-FEM (the error
    measure of section 5.1 and Table 3) falls as the face order rises."""
    spec = dict(lx=10.0, ly=10.0, lz=50.0, ex=12, ey=12, ez=10)
    tsv = fem.tsv_block_mesh(**spec, r_cu=2.5, t_liner=0.5)
    dum = fem.tsv_block_mesh(**spec, r_cu=0.0, t_liner=0.0)
    st = np.array([[0, 0], [1, 0]])
    dT = -250.0
    amesh, u_fem, _ = fem.solve_array_fem(tsv, _site_mats(tsv, dum), st, dT)
    ref = fem.array_grid_vm(amesh, u_fem, dT, 2, 2, 10.0, 10.0, 20)
    errs = []
    for order in (1, 2, 4):
        n = order + 1
        blocks = [mor.local_stage(tsv, (n, n, n)), mor.local_stage(dum, (n, n, n))]
        sol = mor.global_stage(blocks, st, dT)
        errs.append(fem.normalized_mae(mor.recover_vm_grid(blocks, sol, 20), ref))
    print("normalised MAE by order 1, 2, 4:", errs)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.02


def test_grid_stress_modes_are_the_pointwise_stress_of_each_basis_column(small_block):
    """Linearity of Eqs. 15 and 1: the grid modes times [c; dT] give the
    point stresses of the fine field F [c; dT] under dT."""
    rng = np.random.default_rng(9)
    c = rng.standard_normal(small_block.m) * 1e-3
    modes = mor.grid_stress_modes(small_block, 7)
    u = mor.block_displacement(small_block, c, -250.0)
    m = small_block.mesh
    ref = fem.point_stresses(m, u, -250.0, fem.midplane_grid(m.lx, m.ly, m.lz, 7))
    got = modes @ np.concatenate([c, [-250.0]])
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
