"""The row-strip partition of one array's global stage (mstress_strip_partition)
on CPU ranks over gloo.

* The plan: for every array height and rank count, the block rows and the
  owned lattice rows of the ranks tile the array exactly once, and each
  rank's boundary row is the next rank's first owned row.
* The data path on two and three gloo ranks: a Jacobi-PCG of the reduced
  system (section 4.3, Eq. 20) on a 6 x 8 array, each rank applying K_r to its
  own block rows only (the oracle's reduced block models); per iteration the
  direction's values on each boundary row go from its owner to the rank below
  (halo), the partial interface sums there go back up and are added, and
  <p,q>, <r,z>, <r,r> are summed over the ranks. The solution equals the same
  iteration on one rank to 1e-12 and the oracle's direct solve to 1e-9.
No GPU: the operator is the oracle's dense K_r of each block in numpy FP64.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

DT = -250.0


@pytest.fixture(scope="module")
def api():
    from paper_2411_12690_gb300 import api, build
    build.build()
    return api


@pytest.mark.parametrize("ny", [1, 2, 5, 8, 13])
@pytest.mark.parametrize("order", [1, 2, 4])
def test_plan_tiles_the_array(api, ny, order):
    for world in range(1, min(ny, 5) + 1):
        plans = [api.strip_partition(ny, order, world, r) for r in range(world)]
        assert plans[0]["j0"] == 0 and plans[-1]["j1"] == ny
        assert plans[0]["y_own0"] == 0 and plans[-1]["y_own1"] == ny * order + 1
        sizes = [p["j1"] - p["j0"] for p in plans]
        assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
        for r, p in enumerate(plans):
            assert p["y_own0"] == p["j0"] * order
            assert p["prev"] == (r - 1 if r > 0 else -1) and p["next"] == (r + 1 if r < world - 1 else -1)
            if r < world - 1:
                q = plans[r + 1]
                assert q["j0"] == p["j1"] and q["y_own0"] == p["y_own1"]
                assert p["y_send"] == p["j1"] * order == q["y_recv"] == q["y_own0"]
            else:
                assert p["y_send"] == -1
            if r == 0:
                assert p["y_recv"] == -1


def test_plan_rejects_bad_arguments(api):
    from paper_2411_12690_gb300.api import MstressError
    for args in [(0, 2, 1, 0), (4, 0, 1, 0), (4, 8, 1, 0), (4, 2, 0, 0), (4, 2, 2, 2), (4, 2, 5, 0), (4, 2, 2, -1)]:
        with pytest.raises(MstressError):
            api.strip_partition(*args)


def strip_pcg(blocks, site_type, plan, comm=None, rtol=1e-13, max_iter=2000):
    """Jacobi-PCG of Eq. 20 on the rank's block rows (plan), bottom face
    clamped. comm: None (one rank) or (torch.distributed, rank). Returns the
    solution on the rank's owned DOFs (zero elsewhere), in the global DOF
    numbering of oracle.mor.element_dof_map, and the iteration count."""
    import torch
    from oracle import mor
    nxyz = blocks[0].nxyz
    gdof, lat, shape = mor.element_dof_map(nxyz, site_type)
    X, Y, Z = shape
    gy = (lat // X) % Y
    n = lat.size
    ny_b, nx_b = site_type.shape
    st = site_type.ravel()
    own_blocks = np.arange(plan["j0"] * nx_b, plan["j1"] * nx_b)
    owned = (gy >= plan["y_own0"]) & (gy < plan["y_own1"])
    send = np.flatnonzero(gy == plan["y_send"]) if plan["y_send"] >= 0 else np.zeros(0, dtype=np.int64)
    recv = np.flatnonzero(gy == plan["y_recv"]) if plan["y_recv"] >= 0 else np.zeros(0, dtype=np.int64)
    free = ~mor.fixed_mask(lat, shape, True, False)
    K = np.stack([blocks[int(t)].K_r for t in st[own_blocks]])
    G = gdof[own_blocks]

    def exchange(v, kind):
        """kind 'sum': partial sums on the boundary row go up and are added;
        kind 'value': the owner's values on the boundary row come down."""
        if comm is None:
            return
        dist, rank = comm
        reqs, bufs = [], []
        if kind == "sum":
            if plan["next"] >= 0:
                reqs.append(dist.isend(torch.from_numpy(v[send].copy()), plan["next"]))
            if plan["prev"] >= 0:
                buf = torch.zeros(recv.size, dtype=torch.float64)
                reqs.append(dist.irecv(buf, plan["prev"]))
                bufs.append(buf)
        else:
            if plan["prev"] >= 0:
                reqs.append(dist.isend(torch.from_numpy(v[recv].copy()), plan["prev"]))
            if plan["next"] >= 0:
                buf = torch.zeros(send.size, dtype=torch.float64)
                reqs.append(dist.irecv(buf, plan["next"]))
                bufs.append(buf)
        for q in reqs:
            q.wait()
        if bufs:
            if kind == "sum":
                v[recv] += bufs[0].numpy()
            else:
                v[send] = bufs[0].numpy()

    def allsum(*vals):
        if comm is None:
            return vals
        dist, _ = comm
        t = torch.tensor(vals, dtype=torch.float64)
        dist.all_reduce(t)
        return tuple(t.tolist())

    def scatter_blocks(elem):   # (own blocks, m) element values -> partial lattice sums
        out = np.zeros(n)
        np.add.at(out, G.ravel(), elem.ravel())
        return out

    b = scatter_blocks(DT * np.stack([blocks[int(t)].b_r for t in st[own_blocks]]))
    exchange(b, "sum")
    diag = scatter_blocks(np.stack([np.diag(k) for k in K]))
    exchange(diag, "sum")
    mask = owned & free
    dinv = np.where(mask, 1.0 / np.where(mask, diag, 1.0), 0.0)
    x = np.zeros(n)
    r = np.where(mask, b, 0.0)
    z = dinv * r
    p = z.copy()
    rz, rr = allsum(float(r @ z), float(r @ r))
    bb = rr
    it = 0
    while rr > rtol * rtol * bb and it < max_iter:
        exchange(p, "value")
        q = scatter_blocks(np.einsum("eij,ej->ei", K, p[G]))
        exchange(q, "sum")
        q = np.where(mask, q, 0.0)
        (pq,) = allsum(float(p[owned] @ q[owned]))
        al = rz / pq
        x += al * p
        r -= al * q
        z = dinv * r
        rz_new, rr = allsum(float(r @ z), float(r @ r))
        p = z + (rz_new / rz) * p
        p[~owned] = 0.0
        rz = rz_new
        it += 1
    return np.where(owned, x, 0.0), it


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import warnings
    warnings.simplefilter("ignore")
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from cases import SMALL_MESH, oracle_pair
        from paper_2411_12690_gb300 import api
        from paper_2411_12690_gb300 import workloads as W
        blocks = oracle_pair(SMALL_MESH)
        st = W.site_types(6, 8, 0.7, seed=41).astype(int)
        plan = api.strip_partition(st.shape[0], SMALL_MESH.order, world, rank)
        x, it = strip_pcg(blocks, st, plan, (dist, rank))
        t = torch.from_numpy(x)
        dist.all_reduce(t)   # owned parts -> the whole solution on every rank
        q.put((rank, t.numpy(), it))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_strip_solve_equals_one_rank_and_oracle(api, world):
    import warnings
    warnings.simplefilter("ignore")
    import torch.multiprocessing as mp
    from cases import SMALL_MESH, oracle_pair
    from oracle import mor
    from paper_2411_12690_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(world):
            rank, x, it = q.get(timeout=300)
            out[rank] = (x, it)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    blocks = oracle_pair(SMALL_MESH)
    st = W.site_types(6, 8, 0.7, seed=41).astype(int)
    one = api.strip_partition(st.shape[0], SMALL_MESH.order, 1, 0)
    x1, it1 = strip_pcg(blocks, st, one)
    x2, it2 = out[0]
    for r in range(1, world):
        assert np.array_equal(out[0][0], out[r][0]) and out[0][1] == out[r][1]
    print(f"6x8 array, {world} strips: {it2} iterations (one rank: {it1}); rel. difference "
          f"{np.linalg.norm(x2 - x1) / np.linalg.norm(x1):.2e}")
    assert abs(it2 - it1) <= 1
    assert np.linalg.norm(x2 - x1) <= 1e-12 * np.linalg.norm(x1)
    sol = mor.global_stage(blocks, st, DT)
    assert np.linalg.norm(x2 - sol.u) <= 1e-9 * np.linalg.norm(sol.u)
