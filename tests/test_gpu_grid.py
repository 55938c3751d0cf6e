"""Gridded cut-plane output (section 5.1): the von Mises stress on the plane
through the half height of every block, at side x side points per block
(100 x 100 in the paper), recovered on the GPU from the block's grid modes
(mstress_block_grid, MSTRESS_VM_GRID), and the paper's error measure on it.

* grid modes: the exported mode matrix equals the oracle's point stresses of
  every basis column (rel. max 1e-9);
* FP64: gridded von Mises at rel. L2 1e-9 against the oracle's evaluation of
  the fine field (oracle.mor.recover_vm_grid) on the 2x2 array of the plain
  configuration, and the normalised MAE against O-FEM equals the oracle's to
  1e-9 relative (and is printed);
* mixed modes (tensor-core recovery): every sampled grid value within its
  rounding bound (the per-output bound of test_gpu_mixed with the grid modes
  in place of the Gauss-mean modes), at m = 78 over several 128-block
  recovery tiles and at m = 294 (the streamed recovery).
"""
import numpy as np
import pytest

from cases import SMALL_MESH, oracle_block, oracle_solve, rel_l2, rel_max, U_IN
from oracle import fem, mor
from paper_2411_12690_gb300 import _lib as L
from paper_2411_12690_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]
DT = W.DT_DEFAULT
_MODES = {}


def grid_modes(spec, dummy, side):
    key = (spec, dummy, side)
    if key not in _MODES:
        _MODES[key] = mor.grid_stress_modes(oracle_block(spec.dummy() if dummy else spec), side)
    return _MODES[key]


def grid_bound(spec, types, coeffs, side, mode):
    """Per-point bound on |vm_gpu - vm_exact|: (2 u_in + (m+17) 2^-24)
    |modes| |[c; dT]| per stress component, times sqrt(3/2) on the
    Frobenius norm (shears counted twice)."""
    out = []
    for t, c in zip(types, coeffs):
        Mabs = np.abs(grid_modes(spec, int(t) == 1, side))
        m1 = Mabs.shape[2]
        u = 2 * U_IN[mode] + (m1 + 16) * 2.0 ** -24
        ab = u * (Mabs @ np.abs(np.concatenate([c, [DT]])))
        out.append(np.sqrt(1.5) * np.sqrt((ab[:, :3] ** 2).sum(1) + 2 * (ab[:, 3:] ** 2).sum(1)))
    return np.stack(out)


def grid_vm_rows(spec, types, coeffs, side):
    return np.stack([fem.von_mises(grid_modes(spec, int(t) == 1, side) @ np.concatenate([c, [DT]]))
                     for t, c in zip(types, coeffs)])


@pytest.fixture(scope="module")
def api():
    from paper_2411_12690_gb300 import api, build
    build.build()
    return api


def test_grid_modes_match_oracle(api):
    ctx = api.Context()
    for spec in (W.BLOCK_SMALL, SMALL_MESH):
        for dummy in (False, True):
            blk = ctx.build_block(spec.dummy() if dummy else spec).grid(12)
            got = blk.export(L.MSTRESS_BLOCK_SGRID).reshape(144, 6, -1)
            assert rel_max(got, grid_modes(spec, dummy, 12)) <= 1e-9


def test_grid_fp64_and_error_measure_plain_config(api):
    """The 2x2 array of the plain configuration, 100 x 100 points per block."""
    spec = W.BLOCK_SMALL
    ctx = api.Context()
    blks = [ctx.build_block(spec).grid(100), ctx.build_block(spec.dummy()).grid(100)]
    st = np.array([[0, 1], [0, 0]], dtype=np.uint8)
    sol = ctx.solve(st, blks, DT)
    vm = sol.recover(L.MSTRESS_VM_GRID).reshape(4, 10000)
    ob, osol = oracle_solve(spec, st, DT)
    ovm = mor.recover_vm_grid(ob, osol, 100)
    assert rel_l2(vm, ovm) <= 1e-9
    # the error measure of section 5.1 against the full fine-mesh model
    t_mesh = fem.tsv_block_mesh(spec.lx, spec.ly, spec.lz, spec.ex, spec.ey, spec.ez, spec.r_cu, spec.t_liner)
    d_mesh = fem.tsv_block_mesh(spec.lx, spec.ly, spec.lz, spec.ex, spec.ey, spec.ez, 0.0, 0.0)
    amesh, u_fem, _ = fem.solve_array_fem(t_mesh, [t_mesh.mat_id, d_mesh.mat_id], st, DT)
    ref = fem.array_grid_vm(amesh, u_fem, DT, 2, 2, spec.lx, spec.ly, 100)
    mae_gpu = fem.normalized_mae(vm, ref)
    mae_oracle = fem.normalized_mae(ovm, ref)
    print(f"2x2, degree-2 basis: normalised MAE of the gridded von Mises vs O-FEM: {mae_gpu:.4%}")
    assert abs(mae_gpu - mae_oracle) <= 1e-9 * mae_oracle
    assert mae_gpu < 0.05


@pytest.mark.parametrize("spec,n,mode", [(W.BLOCK_SMALL, 18, L.MSTRESS_BF16X3), (W.BLOCK_SMALL, 18, L.MSTRESS_TF32),
                                         (W.BLOCK_P15, 3, L.MSTRESS_BF16X3)])
def test_grid_mixed_within_bound(api, spec, n, mode):
    side = 40
    ctx = api.Context(precision=mode)
    blks = [ctx.build_block(spec).grid(side), ctx.build_block(spec.dummy()).grid(side)]
    st = W.site_types(n, n, 0.7, seed=12)
    sol = ctx.solve(st, blks, DT)
    vm = sol.recover(L.MSTRESS_VM_GRID).reshape(st.size, side * side).astype(np.float64)
    _, osol = oracle_solve(spec, st, DT)
    rng = np.random.default_rng(2)
    pick = np.unique(np.concatenate([[0, st.size - 1], rng.choice(st.size, min(10, st.size), replace=False)]))
    types = st.ravel()[pick]
    ovm = grid_vm_rows(spec, types, osol.coeffs[pick], side)
    bound = grid_bound(spec, types, osol.coeffs[pick], side, mode)
    err = np.abs(vm[pick] - ovm)
    print(f"m={oracle_block(spec).m} mode {mode}: grid vm rel L2 {rel_l2(vm[pick], ovm):.2e}, "
          f"max err/bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound + 1e-12 * ovm.max())
