"""The operator apply that allocates no memory (mstress_apply_noalloc).

It exists for callers that cannot allocate device memory when they need the
operator (inside a stream capture they do not own, with memory fixed up front,
or under another runtime's allocator). Its scratch is a fixed array inside the
library, so this file runs last: if it fails, every other test has already run.
The output must equal that of the allocating mstress_apply within the same
1e-12 relative bound the operator test uses, on two calls in a row (the
second with new input, so stale scratch from the first call would show), for
a degree-2 (m = 78) and a degree-4 (m = 294) basis, and at exactly the largest
array the scratch holds; one block more is refused.
"""
import ctypes as C

import numpy as np
import pytest

from cases import SMALL_MESH
from paper_2411_12690_gb300 import _lib as L
from paper_2411_12690_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 32 << 20
ORDER4 = W.BlockSpec(10.0, 10.0, 30.0, 8, 8, 6, 2.5, 0.5, 4)


def _limit_blocks(m):
    ld = (m + 15) // 16 * 16
    return SCRATCH_BYTES // (ld * 8)


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2411_12690_gb300 import api, build
    build.build()
    ctx = api.Context()
    return ctx, torch.cuda.current_stream()


def _noalloc(ctx, blk, nx, ny, x, y, stream):
    return ctx.lib.mstress_apply_noalloc(blk.h, nx, ny, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                         C.c_void_p(stream.cuda_stream))


def _compare(ctx, stream, spec, blk, nx, ny, seed):
    import torch
    n = spec.order + 1
    X, Y, Z = nx * (n - 1) + 1, ny * (n - 1) + 1, n
    st = np.zeros((ny, nx), dtype=np.uint8)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    for call in range(2):
        x = torch.randn(3 * X * Y * Z, dtype=torch.float64, device="cuda", generator=gen)
        y_ref = torch.zeros_like(x)
        ctx.apply(st, [blk], x.data_ptr(), y_ref.data_ptr())
        y = torch.full_like(x, float("nan"))
        rc = _noalloc(ctx, blk, nx, ny, x, y, stream)
        assert rc == L.MSTRESS_OK, ctx.lib.mstress_last_error(ctx.h)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref)).item()
        assert err <= 1e-12, f"{nx}x{ny} m={blk.info()['m']} call {call}: rel L2 {err:.3e}"


@pytest.mark.parametrize("spec,shape", [(W.BLOCK_SMALL, (9, 7)), (SMALL_MESH, (4, 13)), (ORDER4, (5, 6))])
def test_noalloc_apply_matches_allocating_apply(env, spec, shape):
    ctx, stream = env
    blk = ctx.build_block(spec)
    _compare(ctx, stream, spec, blk, shape[0], shape[1], seed=1)
    blk.close()


@pytest.mark.parametrize("spec,ok_shape,bad_shape", [(SMALL_MESH, (204, 257), (481, 109)),
                                                     (ORDER4, (189, 73), (6899, 2))])
def test_noalloc_scratch_limit(env, spec, ok_shape, bad_shape):
    """The largest array the scratch holds is accepted and correct; one block
    more is refused before any work is issued."""
    import torch
    ctx, stream = env
    blk = ctx.build_block(spec)
    m = blk.info()["m"]
    assert ok_shape[0] * ok_shape[1] == _limit_blocks(m)
    assert bad_shape[0] * bad_shape[1] == _limit_blocks(m) + 1
    _compare(ctx, stream, spec, blk, ok_shape[0], ok_shape[1], seed=2)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = _noalloc(ctx, blk, bad_shape[0], bad_shape[1], x, x, stream)
    assert rc == L.MSTRESS_EINVAL
    assert b"no-allocation scratch" in ctx.lib.mstress_last_error(ctx.h)
    blk.close()
