"""The reduced-precision operator of the inner PCG (Eq. 18 applied matrix-free,
with the interface sum of section 4.3) at every basis size the tensor cores
take: m = 78 (operator resident in shared memory), m = 168, m = 294 and
m = 456 (operator streamed along K, the last two split into two MMA column
groups).

Bound, per lattice DOF g of y = A_global x with x rounded to FP32: each element
product entry is a K-term dot product of operands rounded to the mode's format
(relative error u_in each) accumulated in FP32, and the interface sum adds at
most four FP32 terms, so
    |y_mode[g] - y[g]| <= (2 u_in + (m + 16) 2^-24) * (sum_e G_e^T |K_e| G_e |x|)[g]
with u_in = 2^-11 (TF32), 2^-8 (BF16), 3 * 2^-16 (BF16X3). The right-hand side
is assembled by the oracle from |K_r|.
"""
import dataclasses

import numpy as np
import pytest

from cases import oracle_block, oracle_solve, rel_l2
from oracle import mor
from paper_2411_12690_gb300 import _lib as L
from paper_2411_12690_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

U_IN = {L.MSTRESS_TF32: 2.0 ** -11, L.MSTRESS_BF16: 2.0 ** -8, L.MSTRESS_BF16X3: 3 * 2.0 ** -16}
MODES = [L.MSTRESS_TF32, L.MSTRESS_BF16, L.MSTRESS_BF16X3]
SPECS = {2: W.BlockSpec(10.0, 10.0, 30.0, 8, 8, 6, 2.5, 0.5, 2),    # m = 78
         3: W.BlockSpec(10.0, 10.0, 30.0, 8, 8, 6, 2.5, 0.5, 3),    # m = 168
         4: W.BlockSpec(10.0, 10.0, 30.0, 8, 8, 6, 2.5, 0.5, 4),    # m = 294
         5: W.BlockSpec(10.0, 10.0, 30.0, 8, 8, 6, 2.5, 0.5, 5)}    # m = 456


@pytest.fixture(scope="module")
def api():
    from paper_2411_12690_gb300 import api, build
    build.build()
    return api


def _abs_operator(blocks, site_type):
    absb = [dataclasses.replace(b, K_r=np.abs(b.K_r)) for b in blocks]
    A, _, _, lat, shape = mor.assemble_global(absb, site_type, 0.0)
    return A, lat, shape


@pytest.mark.parametrize("order", [2, 3, 4, 5])
@pytest.mark.parametrize("mode", MODES)
def test_reduced_operator_within_rounding_bound(api, order, mode):
    import torch
    spec = SPECS[order]
    ctx = api.Context(precision=mode)
    blks = [ctx.build_block(spec), ctx.build_block(spec.dummy())]
    st = W.site_types(19, 17, 0.7, seed=order)          # 323 sites: several tiles and a ragged tail
    ob = [oracle_block(spec), oracle_block(spec.dummy())]
    A, _, gdof, lat_of_dof, shape = mor.assemble_global(ob, st, 0.0)
    Aabs, _, _ = _abs_operator(ob, st)
    X, Y, Z = shape
    rng = np.random.default_rng(order * 10 + mode)
    x = rng.standard_normal(3 * X * Y * Z).astype(np.float32).astype(np.float64)
    lat = 3 * lat_of_dof + np.tile(np.arange(3), lat_of_dof.size // 3)
    xd = torch.tensor(x, device="cuda")
    yd = torch.zeros_like(xd)
    ctx.apply(st, blks, xd.data_ptr(), yd.data_ptr(), precision=mode)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ref = A @ x[lat]
    m = ob[0].m
    bound = (2 * U_IN[mode] + (m + 16) * 2.0 ** -24) * (Aabs @ np.abs(x[lat]))
    err = np.abs(y[lat] - ref)
    print(f"order {order} m {m} mode {mode}: relL2 {rel_l2(y[lat], ref):.2e} max err/bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)
    holes = np.ones(x.size, dtype=bool)
    holes[lat] = False
    assert np.all(y[holes] == 0.0)


@pytest.mark.parametrize("order,mode", [(4, m) for m in MODES] + [(5, L.MSTRESS_BF16X3), (5, L.MSTRESS_TF32)])
def test_refinement_streamed_reaches_fp64_accuracy(api, order, mode):
    """Iterative refinement around the streamed tensor-core operator reaches
    the FP64 path's accuracy on the element DOFs (m = 294 and 456)."""
    spec = SPECS[order]
    ctx = api.Context(precision=mode)
    blks = [ctx.build_block(spec), ctx.build_block(spec.dummy())]
    st = W.site_types(9, 8, 0.8, seed=5)
    sol = ctx.solve(st, blks, -220.0)
    info = sol.info()
    ob, osol = oracle_solve(spec, st, -220.0)
    c = sol.recover(L.MSTRESS_COEFF).reshape(osol.coeffs.shape)
    print(f"mode {mode}: iters {info['iters']} outer {info['outer']} rel_res {info['rel_res']:.2e} "
          f"coeff relL2 {rel_l2(c, osol.coeffs):.2e}")
    assert info["status"] == 0 and info["rel_res"] <= 1e-12
    assert rel_l2(c, osol.coeffs) <= 1e-9
    # per-element von Mises through the tensor-core recovery with K streamed
    # (m + 1 = 295 or 457), within its rounding bound
    from test_gpu_mixed import vm_bound
    vm = sol.recover(L.MSTRESS_VM_ELEM).reshape(-1, spec.ex * spec.ey * spec.ez)
    ovm = mor.recover_vm(ob, osol)
    err = np.abs(vm.astype(np.float64) - ovm)
    bound = vm_bound(ob, osol, mode)
    print(f"mode {mode}: vm relL2 {rel_l2(vm, ovm):.2e} max err/bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound + 1e-12 * ovm.max())
    if mode == L.MSTRESS_BF16X3:
        assert rel_l2(vm, ovm) <= 1e-4



@pytest.mark.parametrize("mode", MODES)
def test_recovery_m168_within_rounding_bound(api, mode):
    """Per-element von Mises at m = 168 (a larger tensor-core recovery tile:
    one S_mean stage next to the coefficients in the split modes) against the
    oracle, within the per-element rounding bound of the recovery."""
    from test_gpu_mixed import vm_bound
    spec = SPECS[3]
    ctx = api.Context(precision=mode)
    blks = [ctx.build_block(spec), ctx.build_block(spec.dummy())]
    st = W.site_types(13, 11, 0.75, seed=9)       # 143 blocks: two 128-block recovery tiles
    sol = ctx.solve(st, blks, -200.0)
    assert sol.info()["status"] == 0
    ob, osol = oracle_solve(spec, st, -200.0)
    n_el = spec.ex * spec.ey * spec.ez
    vm = sol.recover(L.MSTRESS_VM_ELEM).reshape(-1, n_el)
    ovm = mor.recover_vm(ob, osol)
    bound = vm_bound(ob, osol, mode)
    err = np.abs(vm.astype(np.float64) - ovm)
    print(f"mode {mode}: vm relL2 {rel_l2(vm, ovm):.2e} max err/bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound + 1e-12 * ovm.max())
