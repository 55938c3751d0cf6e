"""Batched solves of uneven arrays (mstress_solve_batch): every array's result
is the same alone and inside the batch (bitwise: an array's arithmetic never
depends on the other arrays), and every array matches the oracle: FP64 at
rel. L2 1e-9; the mixed modes with element DOFs at 1e-9 and every von Mises
value within its per-element rounding bound (test_gpu_mixed)."""
import numpy as np
import pytest

from cases import SMALL_MESH, oracle_solve, oracle_vm_rows, rel_l2, vm_bound_rows
from oracle import mor
from paper_2411_12690_gb300 import _lib as L
from paper_2411_12690_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]


@pytest.fixture(scope="module")
def api():
    from paper_2411_12690_gb300 import api, build
    build.build()
    return api


def _per_array(sol, sizes, what, width):
    out = sol.recover(what)
    res, off = [], 0
    for s in sizes:
        res.append(out[off:off + s * width].copy())
        off += s * width
    return res


@pytest.mark.parametrize("prec", [L.MSTRESS_FP64, L.MSTRESS_BF16X3, L.MSTRESS_TF32])
def test_batch_equals_alone(api, prec):
    ctx = api.Context(precision=prec)
    blks = [ctx.build_block(SMALL_MESH), ctx.build_block(SMALL_MESH.dummy())]
    rng = np.random.default_rng(5)
    jobs = []
    for k, (nx, ny) in enumerate([(1, 1), (3, 2), (7, 5), (2, 9), (12, 12), (4, 4)]):
        st = W.site_types(nx, ny, 0.7, seed=10 + k)
        jobs.append(dict(site_type=st, blocks=blks, dT=float(rng.uniform(-300, -150)), clamp_top=(k == 3)))
    batch = ctx.solve_batch(jobs)
    n_el = SMALL_MESH.ex * SMALL_MESH.ey * SMALL_MESH.ez
    m = 78
    sizes = [j["site_type"].size for j in jobs]
    bc = _per_array(batch, sizes, L.MSTRESS_COEFF, m)
    bv = _per_array(batch, sizes, L.MSTRESS_VM_ELEM, n_el)
    for k, j in enumerate(jobs):
        alone = ctx.solve(j["site_type"], blks, j["dT"], clamp_top=j["clamp_top"])
        assert alone.info()["status"] == 0 and batch.info(k)["status"] == 0
        assert batch.info(k)["iters"] == alone.info()["iters"]
        assert np.array_equal(alone.recover(L.MSTRESS_COEFF), bc[k])
        assert np.array_equal(alone.recover(L.MSTRESS_VM_ELEM), bv[k])
        ob, osol = oracle_solve(SMALL_MESH, j["site_type"], j["dT"], clamp_top=j["clamp_top"])
        assert rel_l2(bc[k].reshape(-1, m), osol.coeffs) <= 1e-9
        ovm = mor.recover_vm(ob, osol)
        if prec == L.MSTRESS_FP64:
            assert rel_l2(bv[k].reshape(-1, n_el), ovm) <= 1e-9
        else:
            bound = vm_bound_rows(ob, osol.site_type.ravel(), osol.coeffs, j["dT"], prec)
            err = np.abs(bv[k].reshape(-1, n_el).astype(np.float64) - ovm)
            assert np.all(err <= bound + 1e-12 * ovm.max())


def test_batch_two_block_variants_m294(api):
    """Degree-4 basis (m = 294), 24x24x20 meshes, two pitch variants, each
    with its dummy block, in one batch; results equal the single-array solves
    bitwise and the oracle (element DOFs at 1e-9; the von Mises of a sample of
    blocks of every array within the per-element rounding bound)."""
    ctx = api.Context(precision=L.MSTRESS_BF16X3)
    variants = [W.BLOCK_P15, W.BLOCK_P20]
    models = [[ctx.build_block(v), ctx.build_block(v.dummy())] for v in variants]
    jobs = W.batch_arrays(5, seed=3, smin=2, smax=6)
    spec = [dict(site_type=j.site_type, blocks=models[j.pitch], dT=j.dT) for j in jobs]
    batch = ctx.solve_batch(spec)
    sizes = [j.site_type.size for j in jobs]
    n_el = W.BLOCK_P15.ex * W.BLOCK_P15.ey * W.BLOCK_P15.ez
    bc = _per_array(batch, sizes, L.MSTRESS_COEFF, 294)
    bv = _per_array(batch, sizes, L.MSTRESS_VM_ELEM, n_el)
    rng = np.random.default_rng(4)
    for k, (j, job) in enumerate(zip(spec, jobs)):
        alone = ctx.solve(j["site_type"], j["blocks"], j["dT"])
        assert np.array_equal(alone.recover(L.MSTRESS_COEFF), bc[k])
        assert np.array_equal(alone.recover(L.MSTRESS_VM_ELEM), bv[k])
        assert batch.info(k)["rel_res"] <= 1e-12
        ob, osol = oracle_solve(variants[job.pitch], j["site_type"], j["dT"])
        c = bc[k].reshape(-1, 294)
        assert rel_l2(c, osol.coeffs) <= 1e-9
        pick = rng.choice(sizes[k], min(4, sizes[k]), replace=False)
        types = osol.site_type.ravel()[pick]
        ovm = oracle_vm_rows(ob, types, osol.coeffs[pick], j["dT"])
        bound = vm_bound_rows(ob, types, osol.coeffs[pick], j["dT"], L.MSTRESS_BF16X3)
        err = np.abs(bv[k].reshape(-1, n_el)[pick].astype(np.float64) - ovm)
        assert np.all(err <= bound + 1e-12 * ovm.max())


@pytest.mark.parametrize("prec", [L.MSTRESS_BF16X3, L.MSTRESS_TF32])
def test_large_streamed_batch_per_phase_equals_alone(api, prec):
    """A batch of 4 113 blocks of the degree-4 basis (m = 294) runs the
    per-phase iteration (launches of its own per phase: at least 4 096 blocks
    on the streamed apply), while each of its arrays alone (3 969, 144 and 35
    blocks) runs the persistent solver: the two paths give bitwise the same
    element DOFs, von Mises values and iteration counts, and the small arrays
    match the oracle (element DOFs at 1e-9, sampled von Mises within the
    per-element rounding bound)."""
    spec = W.BlockSpec(10.0, 10.0, 30.0, 8, 8, 6, 2.5, 0.5, 4)
    ctx = api.Context(precision=prec)
    blks = [ctx.build_block(spec), ctx.build_block(spec.dummy())]
    jobs = [dict(site_type=W.site_types(63, 63, 0.8, seed=31), blocks=blks, dT=-260.0),
            dict(site_type=W.site_types(12, 12, 0.7, seed=32), blocks=blks, dT=-180.0),
            dict(site_type=W.site_types(5, 7, 0.6, seed=33), blocks=blks, dT=-220.0, clamp_top=True)]
    sizes = [j["site_type"].size for j in jobs]
    assert sum(sizes) >= 4096 and max(sizes) < 4096
    batch = ctx.solve_batch(jobs)
    n_el = spec.ex * spec.ey * spec.ez
    bc = _per_array(batch, sizes, L.MSTRESS_COEFF, 294)
    bv = _per_array(batch, sizes, L.MSTRESS_VM_ELEM, n_el)
    rng = np.random.default_rng(6)
    for k, j in enumerate(jobs):
        alone = ctx.solve(j["site_type"], blks, j["dT"], clamp_top=j.get("clamp_top", False))
        assert alone.info()["status"] == 0 and batch.info(k)["status"] == 0
        assert batch.info(k)["rel_res"] <= 1e-12
        assert batch.info(k)["iters"] == alone.info()["iters"]
        assert np.array_equal(alone.recover(L.MSTRESS_COEFF), bc[k])
        assert np.array_equal(alone.recover(L.MSTRESS_VM_ELEM), bv[k])
        if k == 0:
            continue   # the 63 x 63 array: the oracle's sparse direct solve is too large for a test
        ob, osol = oracle_solve(spec, j["site_type"], j["dT"], clamp_top=j.get("clamp_top", False))
        c = bc[k].reshape(-1, 294)
        assert rel_l2(c, osol.coeffs) <= 1e-9
        pick = rng.choice(sizes[k], min(6, sizes[k]), replace=False)
        types = osol.site_type.ravel()[pick]
        ovm = oracle_vm_rows(ob, types, osol.coeffs[pick], j["dT"])
        bound = vm_bound_rows(ob, types, osol.coeffs[pick], j["dT"], prec)
        err = np.abs(bv[k].reshape(-1, n_el)[pick].astype(np.float64) - ovm)
        assert np.all(err <= bound + 1e-12 * ovm.max())
