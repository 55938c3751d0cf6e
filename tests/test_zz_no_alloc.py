"""The operator apply that allocates no memory (mstress_apply_noalloc).

It exists for callers that cannot allocate device memory when they need the
operator (inside a stream capture they do not own, with memory fixed up front,
or under another runtime's allocator). Its scratch is a fixed array inside the
library, so this file runs last: if it fails, every other test has already run.
The output must equal that of the allocating mstress_apply within the same
1e-12 relative bound the operator test uses, on two calls in a row (the
second with new input, so stale scratch from the first call would show).
"""
import ctypes as C

import numpy as np
import pytest

from cases import SMALL_MESH
from paper_2411_12690_gb300 import _lib as L
from paper_2411_12690_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_apply_matches_allocating_apply():
    import torch

    from paper_2411_12690_gb300 import api, build
    build.build()
    ctx = api.Context()
    stream = torch.cuda.current_stream()
    for spec, (nx, ny) in ((W.BLOCK_SMALL, (9, 7)), (SMALL_MESH, (4, 13))):
        blk = ctx.build_block(spec)
        n = spec.order + 1
        X, Y, Z = nx * (n - 1) + 1, ny * (n - 1) + 1, n
        st = np.zeros((ny, nx), dtype=np.uint8)
        gen = torch.Generator(device="cuda").manual_seed(1)
        for call in range(2):
            x = torch.randn(3 * X * Y * Z, dtype=torch.float64, device="cuda", generator=gen)
            y_ref = torch.zeros_like(x)
            ctx.apply(st, [blk], x.data_ptr(), y_ref.data_ptr())
            y = torch.full_like(x, float("nan"))
            rc = ctx.lib.mstress_apply_noalloc(blk.h, nx, ny, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                               C.c_void_p(stream.cuda_stream))
            assert rc == L.MSTRESS_OK, ctx.lib.mstress_last_error(ctx.h)
            torch.cuda.synchronize()
            err = (torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref)).item()
            assert err <= 1e-12, f"call {call}: rel L2 {err:.3e}"


def test_noalloc_rejects_arrays_beyond_the_scratch():
    import torch

    from paper_2411_12690_gb300 import api, build
    build.build()
    ctx = api.Context()
    blk = ctx.build_block(SMALL_MESH)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = ctx.lib.mstress_apply_noalloc(blk.h, 400, 400, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), None)
    assert rc == L.MSTRESS_EINVAL
    assert b"no-allocation scratch" in ctx.lib.mstress_last_error(ctx.h)
