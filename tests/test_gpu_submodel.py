"""Sub-modeling (section 4.4; scenario 2 of section 5.1): a 15x15 TSV array
inside two rings of dummy (pure-Si) blocks, every outer face of the
sub-model driven by a coarse-model displacement field imposed by lifting
(Eq. 13), no clamped face. The coarse field is the synthetic warpage-like
field of workloads.submodel_boundary (the paper's ANSYS chiplet model is not
available).

Against the oracle's lifting (oracle.mor.global_stage with the same
prescribed values): FP64 at rel. L2 1e-9 in element DOFs and per-element von
Mises; BF16X3 with element DOFs at 1e-9 and every von Mises value within its
per-element rounding bound (test_gpu_mixed).
"""
import numpy as np
import pytest

from cases import oracle_pair, oracle_vm_rows, rel_l2, vm_bound_rows
from oracle import mor
from paper_2411_12690_gb300 import _lib as L
from paper_2411_12690_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]
DT = W.DT_DEFAULT


def oracle_submodel(spec, st, dof, val):
    """The oracle's solve of the same sub-model: lattice DOFs mapped to the
    oracle's global DOF numbering, imposed by its lifting."""
    blocks = oracle_pair(spec)
    _, _, gdof, lat, _ = mor.assemble_global(blocks, st.astype(int), DT)
    key = 3 * lat + np.tile(np.arange(3), lat.size // 3)       # lattice DOF of each oracle DOF
    index = {int(k): i for i, k in enumerate(key)}
    presc = {index[int(d)]: float(v) for d, v in zip(dof, val)}
    sol = mor.global_stage(blocks, st.astype(int), DT, clamp_bottom=False, clamp_top=False, prescribed=presc)
    return blocks, sol


@pytest.mark.parametrize("spec,n_tsv,prec", [(W.BLOCK_SMALL, 15, L.MSTRESS_FP64),
                                             (W.BLOCK_SMALL, 15, L.MSTRESS_BF16X3),
                                             (W.BLOCK_P15_O3, 3, L.MSTRESS_BF16X3)])
def test_submodel_matches_oracle(spec, n_tsv, prec):
    from paper_2411_12690_gb300 import api, build
    build.build()
    st = W.submodel_sites(n_tsv, 2)
    ny, nx = st.shape
    dof, val = W.submodel_boundary(nx, ny, spec, seed=5)
    ctx = api.Context(precision=prec)
    blks = [ctx.build_block(spec), ctx.build_block(spec.dummy())]
    sol = ctx.solve(st, blks, DT, clamp_bottom=False, prescribed=dict(zip(dof.tolist(), val.tolist())))
    info = sol.info()
    ob, osol = oracle_submodel(spec, st, dof, val)
    nb = st.size
    n_el = spec.ex * spec.ey * spec.ez
    c = sol.recover(L.MSTRESS_COEFF).reshape(nb, -1)
    vm = sol.recover(L.MSTRESS_VM_ELEM).reshape(nb, n_el).astype(np.float64)
    lat = sol.recover(L.MSTRESS_LATTICE)
    print(f"{nx}x{ny} m={ob[0].m} prec {prec}: iters {info['iters']} outer {info['outer']} rel_res "
          f"{info['rel_res']:.2e} coeff relL2 {rel_l2(c, osol.coeffs):.2e}")
    assert info["status"] == 0 and info["rel_res"] <= 1e-12
    # the prescribed values are in the returned solution exactly
    assert np.array_equal(lat[dof], val)
    assert rel_l2(c, osol.coeffs) <= 1e-9
    ovm = oracle_vm_rows(ob, osol.site_type.ravel(), osol.coeffs, DT)
    if prec == L.MSTRESS_FP64:
        assert rel_l2(vm, ovm) <= 1e-9
    else:
        bound = vm_bound_rows(ob, osol.site_type.ravel(), osol.coeffs, DT, prec)
        assert np.all(np.abs(vm - ovm) <= bound + 1e-12 * ovm.max())
