"""Continuous-batching server (mstress_server_*).

Requests that arrive while others are running join the batch at the next
refinement step, and each result is the same alone and in the mix: the same
requests served one at a time and served together (arriving at different
steps, sharing the batch) give bitwise-identical von Mises fields, which also
match the oracle within the mode's stated accuracy (FP64: rel. L2 1e-9;
BF16X3: every von Mises value within its per-element rounding bound and rel.
L2 1e-4). Admission respects
the slot count and the HBM budget.
"""
import numpy as np
import pytest

from cases import SMALL_MESH, oracle_solve, rel_l2, vm_bound_rows
from oracle import mor
from paper_2411_12690_gb300 import _lib as L
from paper_2411_12690_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

N_EL = SMALL_MESH.ex * SMALL_MESH.ey * SMALL_MESH.ez


def _jobs():
    g = np.random.default_rng(8)
    jobs = []
    for k, s in enumerate([3, 7, 2, 11, 5, 9, 4]):
        jobs.append((W.site_types(s, s, float(g.uniform(0.5, 1.0)), seed=40 + k), float(g.uniform(-300, -150))))
    return jobs


def _run_server(api, ctx, blocks, jobs, arrival_steps, max_slots=64, budget=0):
    srv = api.Server(ctx, max_slots=max_slots, hbm_budget=budget)
    ids, out, pending = {}, {}, list(range(len(jobs)))
    step = 0
    max_running = 0
    while len(out) < len(jobs):
        for k in [k for k in pending if arrival_steps[k] <= step]:
            ids[srv.submit(jobs[k][0], blocks, jobs[k][1])] = k
            pending.remove(k)
        _, running, _ = srv.step()
        max_running = max(max_running, running)
        while True:
            rid = srv.poll()
            if not rid:
                break
            info = srv.info(rid)
            assert info["status"] == 0 and info["state"] == L.MSTRESS_RQ_DONE, info
            k = ids[rid]
            vm = np.empty(jobs[k][0].size * N_EL, dtype=np.float32 if ctx.opts.precision else np.float64)
            out[k] = (srv.result(rid, vm), info)
            srv.release(rid)
        step += 1
        assert step < 500
    srv.close()
    return out, max_running


@pytest.mark.parametrize("prec", [L.MSTRESS_BF16X3, L.MSTRESS_FP64])
def test_served_alone_equals_in_the_mix(prec):
    from paper_2411_12690_gb300 import api, build
    build.build()
    ctx = api.Context(precision=prec)
    blocks = [ctx.build_block(SMALL_MESH), ctx.build_block(SMALL_MESH.dummy())]
    jobs = _jobs()
    alone = {}
    for k, job in enumerate(jobs):
        res, _ = _run_server(api, ctx, blocks, [job], [0])
        alone[k] = res[0]
    mixed, max_running = _run_server(api, ctx, blocks, jobs, [0, 0, 1, 2, 2, 4, 7])
    assert max_running >= 3        # requests overlapped on the device
    for k, job in enumerate(jobs):
        assert np.array_equal(alone[k][0], mixed[k][0]), f"request {k} differs alone vs in the mix"
        assert alone[k][1]["iters"] == mixed[k][1]["iters"]
        assert mixed[k][1]["rel_res"] <= 1e-12
        ob, osol = oracle_solve(SMALL_MESH, job[0], job[1])
        ovm = mor.recover_vm(ob, osol)
        got = mixed[k][0].reshape(-1, N_EL).astype(np.float64)
        if prec == L.MSTRESS_FP64:
            assert rel_l2(got, ovm) <= 1e-9
        else:
            bound = vm_bound_rows(ob, osol.site_type.ravel(), osol.coeffs, job[1], prec)
            assert np.all(np.abs(got - ovm) <= bound + 1e-12 * ovm.max())
            assert rel_l2(got, ovm) <= 1e-4


def test_admission_by_slots_and_budget():
    from paper_2411_12690_gb300 import api, build
    build.build()
    ctx = api.Context(precision=L.MSTRESS_BF16X3)
    blocks = [ctx.build_block(SMALL_MESH), ctx.build_block(SMALL_MESH.dummy())]
    jobs = _jobs()
    _, max_running = _run_server(api, ctx, blocks, jobs, [0] * len(jobs), max_slots=2)
    assert max_running <= 2
    # a budget that fits about one mid-size request at a time still serves everything
    _, max_running = _run_server(api, ctx, blocks, jobs, [0] * len(jobs), budget=64 << 20)
    assert max_running >= 1
    srv = api.Server(ctx, hbm_budget=1 << 20)   # nothing fits: the request fails cleanly
    rid = srv.submit(jobs[3][0], blocks, jobs[3][1])
    srv.step()
    assert srv.poll() == rid
    assert srv.info(rid)["status"] == L.MSTRESS_ENOMEM and srv.info(rid)["state"] == L.MSTRESS_RQ_FAILED
    srv.close()
