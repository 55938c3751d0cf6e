"""Failure detection on the device, in forms that fault, trap or hang no GPU.

* A bounded wait that runs out: the next persistent solver launch has one
  CTA skip its first grid-barrier arrival (mstress_set_wait_limit's test
  hook) under a 20 ms wait limit. Every other CTA's wait expires, the kernel
  records the failure and returns, the solve reports MSTRESS_EDEVICE_TIMEOUT,
  and the same context then solves correctly (checked against the oracle).
* A NaN in a block model (injected on the host into an imported A_element):
  the PCG detects the non-finite curvature and stops with MSTRESS_ENUMERIC,
  in FP64 and in the mixed mode, without hanging.
"""
import numpy as np
import pytest

from cases import SMALL_MESH, oracle_pair, oracle_solve, rel_l2
from paper_2411_12690_gb300 import _lib as L
from paper_2411_12690_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]


@pytest.fixture(scope="module")
def api():
    from paper_2411_12690_gb300 import api, build
    build.build()
    return api


@pytest.mark.parametrize("prec", [L.MSTRESS_FP64, L.MSTRESS_BF16X3])
def test_barrier_timeout_is_reported_and_the_context_recovers(api, prec):
    from paper_2411_12690_gb300.api import MstressError
    ctx = api.Context(precision=prec)
    blks = [ctx.build_block(SMALL_MESH), ctx.build_block(SMALL_MESH.dummy())]
    st = W.site_types(6, 6, 0.8, seed=21)          # below the tile autotuner's size: no trial launches
    ctx.set_wait_limit(20_000_000, withhold_next=True)
    with pytest.raises(MstressError) as e:
        ctx.solve(st, blks, -250.0)
    assert e.value.code == L.MSTRESS_EDEVICE_TIMEOUT
    ctx.set_wait_limit()                            # default limit, nothing withheld
    sol = ctx.solve(st, blks, -250.0)
    info = sol.info()
    assert info["status"] == 0 and info["rel_res"] <= 1e-12
    _, osol = oracle_solve(SMALL_MESH, st, -250.0)
    assert rel_l2(sol.recover(L.MSTRESS_COEFF).reshape(osol.coeffs.shape), osol.coeffs) <= 1e-9


@pytest.mark.parametrize("prec", [L.MSTRESS_FP64, L.MSTRESS_BF16X3])
def test_nan_in_a_block_model_gives_enumeric(api, prec):
    ob = oracle_pair(SMALL_MESH)
    K = ob[0].K_r.copy()
    K[3, 40] = K[40, 3] = np.nan
    ctx = api.Context(precision=prec, max_outer=6)
    blks = [ctx.import_block(SMALL_MESH, K, ob[0].b_r, ob[0].S), ctx.import_block(SMALL_MESH.dummy(), ob[1].K_r,
                                                                                    ob[1].b_r, ob[1].S)]
    st = W.site_types(4, 5, 0.8, seed=22)
    sol = ctx.solve(st, blks, -250.0, allow=(L.MSTRESS_ENUMERIC, L.MSTRESS_ENOT_CONVERGED))
    assert sol.rc == L.MSTRESS_ENUMERIC and sol.info()["status"] == L.MSTRESS_ENUMERIC
    # the context still serves a clean model
    good = [ctx.import_block(SMALL_MESH, ob[0].K_r, ob[0].b_r, ob[0].S), blks[1]]
    assert ctx.solve(st, good, -250.0).info()["status"] == 0
