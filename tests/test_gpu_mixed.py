"""Reduced-precision modes: FP64-residual iterative refinement around an inner
PCG whose operator runs in TF32, BF16 or split BF16 (BF16X3).

Stated accuracy, per output:
* element DOFs (reduced displacements): the refinement stops on the FP64
  residual at the context's rtol, so they meet the FP64 path's 1e-9 bound;
* per-element von Mises: the recovery contraction runs in the mode's operand
  format with FP32 accumulation, so each Gauss-mean stress component obeys
  |err| <= (2 u_in + (m+1) u_acc) (|S_mean| |[c; dT]|) elementwise, with
  u_in = 2^-11 (TF32), 2^-8 (BF16), 3 * 2^-16 (BF16X3) and u_acc = 2^-24;
  von Mises is sqrt(3/2)-Lipschitz in the stress (Frobenius norm), which turns
  that into a per-element bound checked here, alongside the observed error.
"""
import numpy as np
import pytest

from cases import oracle_pair, oracle_solve, rel_l2, vm_bound_rows
from oracle import fem, mor
from paper_2411_12690_gb300 import _lib as L
from paper_2411_12690_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

MODES = [L.MSTRESS_TF32, L.MSTRESS_BF16, L.MSTRESS_BF16X3]


def vm_bound(blocks, osol, mode):
    """Per-element bound on |vm_gpu - vm_exact| from the recovery rounding."""
    return vm_bound_rows(blocks, osol.site_type.ravel(), osol.coeffs, osol.dT, mode)


@pytest.fixture(scope="module")
def blocks_fp64():
    from paper_2411_12690_gb300 import api, build
    build.build()
    return api


@pytest.mark.parametrize("mode", MODES)
def test_refinement_reaches_fp64_accuracy(blocks_fp64, mode):
    api = blocks_fp64
    ctx = api.Context(precision=mode)
    blks = [ctx.build_block(W.BLOCK_SMALL), ctx.build_block(W.BLOCK_SMALL.dummy())]
    st = W.site_types(12, 10, 0.8, seed=11)
    sol = ctx.solve(st, blks, -250.0)
    info = sol.info()
    ob, osol = oracle_solve(W.BLOCK_SMALL, st, -250.0)
    c = sol.recover(L.MSTRESS_COEFF).reshape(osol.coeffs.shape)
    vm = sol.recover(L.MSTRESS_VM_ELEM).reshape(-1, 1440)
    ovm = mor.recover_vm(ob, osol)
    bound = vm_bound(ob, osol, mode)
    err = np.abs(vm.astype(np.float64) - ovm)
    print(f"mode {mode}: iters {info['iters']} outer {info['outer']} rel_res {info['rel_res']:.2e} "
          f"coeff relL2 {rel_l2(c, osol.coeffs):.2e} vm relL2 {rel_l2(vm, ovm):.2e} "
          f"vm max err/bound {np.max(err / bound):.3f}")
    assert info["status"] == 0 and info["rel_res"] <= 1e-12
    assert rel_l2(c, osol.coeffs) <= 1e-9
    assert np.all(err <= bound + 1e-12 * ovm.max())
    if mode == L.MSTRESS_BF16X3:      # the mixed-path accuracy target for von Mises
        assert rel_l2(vm, ovm) <= 1e-4
