"""GPU parity of the FP64 path against the CPU oracle, through the C ABI.

Tolerance: relative L2 <= 1e-9 in displacement (element DOFs and fine nodal
field) and in per-element von Mises stress, for the plain FP64 method. The
local stage is checked array by array (A_element, b_element, stress modes,
basis) at the same bound.
"""
import numpy as np
import pytest

from cases import SMALL_MESH, oracle_block, oracle_pair, oracle_solve, rel_l2, rel_max
from oracle import fem, mor
from paper_2411_12690_gb300 import _lib as L
from paper_2411_12690_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]
TOL = 1e-9


@pytest.fixture(scope="module")
def ctx():
    from paper_2411_12690_gb300 import api, build
    build.build()
    return api.Context()


@pytest.fixture(scope="module")
def small_blocks(ctx):
    return [ctx.build_block(W.BLOCK_SMALL), ctx.build_block(W.BLOCK_SMALL.dummy())]


def _check_block(gpu_blk, ob):
    Kr = gpu_blk.export(L.MSTRESS_BLOCK_KR)
    assert rel_max(Kr, ob.K_r) <= TOL
    assert np.abs(Kr - Kr.T).max() == 0.0
    assert rel_max(gpu_blk.export(L.MSTRESS_BLOCK_BR), ob.b_r) <= TOL
    assert rel_max(gpu_blk.export(L.MSTRESS_BLOCK_S), ob.S) <= TOL
    Sm = ob.S.reshape(ob.n_el, 8, 6, -1).mean(axis=1).reshape(ob.n_el * 6, -1)
    assert rel_max(gpu_blk.export(L.MSTRESS_BLOCK_SMEAN), Sm) <= TOL
    assert rel_max(gpu_blk.export(L.MSTRESS_BLOCK_F), ob.F) <= TOL


def test_local_stage_matches_oracle(small_blocks):
    for blk, ob in zip(small_blocks, oracle_pair(W.BLOCK_SMALL)):
        info = blk.info()
        assert info["m"] == 78 and info["n_el"] == 1440 and info["n_dof"] == 5577
        assert 0 < info["cg_iters"] < 2000
        _check_block(blk, ob)


@pytest.mark.parametrize("order", [1, 3, 4, 5])
def test_local_stage_other_orders(ctx, order):
    spec = W.BlockSpec(10.0, 10.0, 30.0, 8, 8, 6, 2.5, 0.5, order)
    _check_block(ctx.build_block(spec), oracle_block(spec))


def _gpu_vs_oracle(sol, blocks, osol, spec_n_el):
    nb = osol.coeffs.shape[0]
    c = sol.recover(L.MSTRESS_COEFF).reshape(nb, -1)
    assert rel_l2(c, osol.coeffs) <= TOL
    vm = sol.recover(L.MSTRESS_VM_ELEM).reshape(nb, spec_n_el)
    ovm = mor.recover_vm(blocks, osol)
    assert rel_l2(vm, ovm) <= TOL
    return c, vm


def test_solve_2x2_imported_blocks(ctx):
    """The global stage alone: the oracle's reduced models imported, same inputs."""
    ob = oracle_pair(W.BLOCK_SMALL)
    blks = [ctx.import_block(W.BLOCK_SMALL, b.K_r, b.b_r, b.S, b.F) for b in ob]
    st = np.zeros((2, 2), dtype=np.uint8)
    sol = ctx.solve(st, blks, -250.0)
    info = sol.info()
    assert info["status"] == 0 and info["rel_res"] <= 1e-12
    _, osol = oracle_solve(W.BLOCK_SMALL, st, -250.0)
    _gpu_vs_oracle(sol, ob, osol, 1440)
    u = sol.recover(L.MSTRESS_U_NODE).reshape(4, -1)
    ou = np.stack([mor.block_displacement(ob[0], osol.coeffs[k], -250.0) for k in range(4)])
    assert rel_l2(u, ou) <= TOL


def test_solve_2x2_end_to_end(ctx, small_blocks):
    """Both stages on the GPU (blocks built by the GPU local stage) vs the oracle."""
    st = np.array([[0, 1], [0, 0]], dtype=np.uint8)
    sol = ctx.solve(st, small_blocks, -250.0)
    ob, osol = oracle_solve(W.BLOCK_SMALL, st, -250.0)
    _gpu_vs_oracle(sol, ob, osol, 1440)
    sig = sol.recover(L.MSTRESS_SIGMA_GP).reshape(4, -1)
    osig = np.stack([ob[int(t)].S @ np.concatenate([osol.coeffs[k], [-250.0]])
                     for k, t in enumerate(st.ravel())])
    assert rel_l2(sig, osig) <= TOL


@pytest.mark.parametrize("shape,occ,top", [((1, 1), 1.0, False), ((1, 7), 0.5, False), ((5, 3), 0.6, True),
                                           ((4, 9), 0.8, False)])
def test_ragged_arrays(ctx, shape, occ, top):
    spec = SMALL_MESH
    blks = [ctx.build_block(spec), ctx.build_block(spec.dummy())]
    st = W.site_types(shape[1], shape[0], occ, seed=3)
    sol = ctx.solve(st, blks, -180.0, clamp_top=top)
    ob, osol = oracle_solve(spec, st, -180.0, clamp_top=top)
    _gpu_vs_oracle(sol, ob, osol, spec.ex * spec.ey * spec.ez)


def test_operator_apply_matches_assembled_matrix(ctx, small_blocks):
    import torch
    st = W.site_types(5, 4, 0.7, seed=1)
    ob, osol = oracle_solve(W.BLOCK_SMALL, st, -250.0)
    X, Y, Z = osol.lattice_shape
    rng = np.random.default_rng(0)
    x = rng.standard_normal(3 * X * Y * Z)
    lat = 3 * osol.lattice_of_dof + np.tile(np.arange(3), osol.lattice_of_dof.size // 3)
    xd = torch.tensor(x, device="cuda")
    yd = torch.zeros_like(xd)
    ctx.apply(st, small_blocks, xd.data_ptr(), yd.data_ptr())
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ref = osol.A_global @ x[lat]
    assert rel_l2(y[lat], ref) <= 1e-12
    holes = np.ones(x.size, dtype=bool)
    holes[lat] = False
    assert np.all(y[holes] == 0.0)


def test_bitwise_reproducible(ctx, small_blocks):
    st = W.site_types(6, 6, 0.8, seed=2)
    a = ctx.solve(st, small_blocks, -250.0).recover(L.MSTRESS_LATTICE)
    b = ctx.solve(st, small_blocks, -250.0).recover(L.MSTRESS_LATTICE)
    assert np.array_equal(a, b)


def test_linear_in_dT(ctx, small_blocks):
    st = W.site_types(3, 3, 0.7, seed=5)
    a = ctx.solve(st, small_blocks, -250.0).recover(L.MSTRESS_COEFF)
    b = ctx.solve(st, small_blocks, -125.0).recover(L.MSTRESS_COEFF)
    assert rel_l2(a, 2 * b) <= 1e-11


def test_argument_errors(ctx, small_blocks):
    from paper_2411_12690_gb300.api import Context, MstressError
    st = np.zeros((2, 2), dtype=np.uint8)
    with pytest.raises(MstressError) as e:
        ctx.solve(st, small_blocks, -250.0, clamp_bottom=False)
    assert e.value.code == L.MSTRESS_EINVAL
    with pytest.raises(MstressError) as e:
        ctx.solve(np.full((2, 2), 5, dtype=np.uint8), small_blocks, -250.0)
    assert e.value.code == L.MSTRESS_EINVAL
    with pytest.raises(MstressError) as e:
        ctx.solve(st, small_blocks, float("nan"))
    assert e.value.code == L.MSTRESS_EINVAL
    tiny = Context(hbm_budget=1 << 20)
    with pytest.raises(MstressError) as e:
        tiny.build_block(W.BLOCK_SMALL)
    assert e.value.code == L.MSTRESS_ENOMEM
    limited = Context(max_iter=3)
    b2 = [limited.build_block(W.BLOCK_SMALL)]
    sol = limited.solve(np.zeros((3, 3), dtype=np.uint8), b2, -250.0)
    assert sol.rc == L.MSTRESS_ENOT_CONVERGED and sol.info()["status"] == L.MSTRESS_ENOT_CONVERGED


def test_prescribed_boundary_lifting(ctx, small_blocks):
    """Sub-modeling (section 4.4): prescribed lateral displacements by lifting."""
    st = W.site_types(4, 3, 0.75, seed=4)
    _, o0 = oracle_solve(W.BLOCK_SMALL, st, -250.0)
    X, Y, Z = o0.lattice_shape
    lat = o0.lattice_of_dof
    gx = lat % X
    gy = (lat // X) % Y
    gz = lat // (X * Y)
    comp = np.tile(np.arange(3), lat.size // 3)
    side = np.flatnonzero(((gx == 0) | (gx == X - 1) | (gy == 0) | (gy == Y - 1)) & (gz > 0))
    val = 1e-3 * (0.5 + gx[side] / X) * (1 + comp[side]) * (gz[side] + 1)
    presc_or = dict(zip(side.tolist(), val.tolist()))
    presc_gpu = dict(zip((3 * lat[side] + comp[side]).tolist(), val.tolist()))
    ob, osol = oracle_solve(W.BLOCK_SMALL, st, -250.0, prescribed=presc_or)
    sol = ctx.solve(st, small_blocks, -250.0, prescribed=presc_gpu)
    _gpu_vs_oracle(sol, ob, osol, 1440)


def test_config_20x20_m294(ctx):
    """The 20x20 array of 15x15x50 um blocks, 24x24x20 mesh, degree-4 basis,
    Bernoulli(0.8) occupancy."""
    spec = W.BLOCK_P15
    blks = [ctx.build_block(spec), ctx.build_block(spec.dummy())]
    ob = oracle_pair(spec)
    for b, o in zip(blks, ob):
        assert rel_max(b.export(L.MSTRESS_BLOCK_KR), o.K_r) <= TOL
    st = W.site_types(20, 20, 0.8, seed=0)
    sol = ctx.solve(st, blks, -250.0)
    assert sol.info()["status"] == 0
    _, osol = oracle_solve(spec, st, -250.0)
    _gpu_vs_oracle(sol, ob, osol, spec.ex * spec.ey * spec.ez)


def test_config_100x100_full_size(ctx, small_blocks):
    """The 100x100 array in the bench's configuration, against a full direct
    oracle solve (element DOFs everywhere) and the oracle's recovery of a
    sample of blocks."""
    st = W.site_types(100, 100, 1.0)
    sol = ctx.solve(st, small_blocks, -250.0)
    info = sol.info()
    assert info["status"] == 0 and info["rel_res"] <= 1e-12
    ob, osol = oracle_solve(W.BLOCK_SMALL, st, -250.0)
    c = sol.recover(L.MSTRESS_COEFF).reshape(10000, -1)
    assert rel_l2(c, osol.coeffs) <= TOL
    vm = sol.recover(L.MSTRESS_VM_ELEM).reshape(10000, 1440)
    rng = np.random.default_rng(7)
    sample = np.concatenate([[0, 99, 9900, 9999, 5050], rng.choice(10000, 60, replace=False)])
    for e in sample:
        sig = (ob[0].S @ np.concatenate([osol.coeffs[e], [-250.0]])).reshape(1440, 8, 6)
        assert rel_l2(vm[e], fem.element_von_mises(sig)) <= TOL
