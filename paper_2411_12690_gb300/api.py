"""Thin Python layer over the libmstress C ABI.

Each method marshals its arguments and calls the function of the same name in
include/mstress.h; no step of the method runs in Python. Device buffers and
streams come from PyTorch (``torch.Tensor.data_ptr()``,
``torch.cuda.Stream.cuda_stream``) or from any other CUDA allocator.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from .workloads import MATERIALS, BlockSpec


class MstressError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{L.STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _u8(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _f64(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Context:
    """A libmstress context (device memory budget, CUDA stream, options)."""

    def __init__(self, stream: int | None = None, precision: int = L.MSTRESS_FP64, **opts):
        self.lib = L.load()
        o = L.mstress_opts()
        self._check(self.lib.mstress_opts_default(C.byref(o)), None)
        o.precision = precision
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        if stream is None:
            # Run on torch's current stream. The legacy default stream cannot be
            # captured into a CUDA graph, so if it is current a new stream is
            # created and made current for this thread.
            try:
                import torch
                if torch.cuda.is_available():
                    cur = torch.cuda.current_stream()
                    if cur.cuda_stream == 0:
                        self._torch_stream = torch.cuda.Stream()
                        torch.cuda.set_stream(self._torch_stream)
                        cur = self._torch_stream
                    stream = cur.cuda_stream
            except ImportError:
                stream = None
        self._stream = stream
        h = C.c_void_p()
        rc = self.lib.mstress_create(C.byref(h), C.c_void_p(stream or 0), C.byref(o))
        if rc != 0:
            raise MstressError(rc, "mstress_create failed")
        self.h = h

    # ------------------------------------------------------------ plumbing
    def _check(self, rc, h=-1, allow=()):
        if rc == 0 or rc in allow:
            return rc
        hh = self.h if h == -1 else h
        msg = self.lib.mstress_last_error(hh).decode() if hh else ""
        raise MstressError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.mstress_free_ctx(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def opts(self) -> L.mstress_opts:
        o = L.mstress_opts()
        self._check(self.lib.mstress_get_opts(self.h, C.byref(o)))
        return o

    def set_opts(self, **kw):
        o = self.opts
        for k, v in kw.items():
            setattr(o, k, v)
        self._check(self.lib.mstress_set_opts(self.h, C.byref(o)))

    def mem_info(self):
        a, b = C.c_size_t(), C.c_size_t()
        self._check(self.lib.mstress_mem_info(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def sync(self):
        self._check(self.lib.mstress_sync(self.h))

    def set_wait_limit(self, limit_ns: int = 2_000_000_000, withhold_next: bool = False):
        """Device-time limit of the solver's grid-barrier waits; withhold_next
        makes the next persistent launch's wait run out (testing the timeout
        path)."""
        self._check(self.lib.mstress_set_wait_limit(self.h, int(limit_ns), int(withhold_next)))

    # ------------------------------------------------------- local stage
    def build_block(self, spec: BlockSpec, materials=MATERIALS, mat_id: np.ndarray | None = None,
                    allow_not_converged=False) -> "Block":
        mesh = L.mstress_block_mesh(spec.lx, spec.ly, spec.lz, spec.ex, spec.ey, spec.ez, None)
        keep = None
        if mat_id is not None:
            keep = np.ascontiguousarray(mat_id, dtype=np.uint8)
            mesh.mat_id = _u8(keep)
        tsv = L.mstress_tsv_geom(spec.r_cu, spec.t_liner)
        mats = (L.mstress_material * len(materials))(*[L.mstress_material(*m) for m in materials])
        h = C.c_void_p()
        rc = self.lib.mstress_build_block(self.h, C.byref(mesh), C.byref(tsv), mats, len(materials), spec.order,
                                          C.byref(h))
        self._check(rc, allow=(L.MSTRESS_ENOT_CONVERGED,) if allow_not_converged else ())
        return Block(self, h, spec)

    def import_block(self, spec: BlockSpec, K_r, b_r, S, F=None) -> "Block":
        mesh = L.mstress_block_mesh(spec.lx, spec.ly, spec.lz, spec.ex, spec.ey, spec.ez, None)
        K_r = np.ascontiguousarray(K_r, dtype=np.float64)
        b_r = np.ascontiguousarray(b_r, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.float64)
        Fp = None
        if F is not None:
            F = np.ascontiguousarray(F, dtype=np.float64)
            Fp = _f64(F)
        h = C.c_void_p()
        self._check(self.lib.mstress_block_import(self.h, C.byref(mesh), spec.order, _f64(K_r), _f64(b_r), _f64(S),
                                                  Fp, C.byref(h)))
        return Block(self, h, spec)

    # ------------------------------------------------------ global stage
    @staticmethod
    def _layout(site_type: np.ndarray, blocks: list["Block"]):
        st = np.ascontiguousarray(site_type, dtype=np.uint8)
        ny, nx = st.shape
        arr = (C.c_void_p * len(blocks))(*[b.h.value for b in blocks])
        lay = L.mstress_layout(nx, ny, _u8(st), C.cast(arr, C.POINTER(C.c_void_p)), len(blocks))
        return lay, (st, arr)

    @staticmethod
    def _bc(clamp_bottom=True, clamp_top=False, prescribed: dict | None = None):
        bc = L.mstress_bc(int(clamp_bottom), int(clamp_top), None, None, 0)
        keep = ()
        if prescribed:
            d = np.ascontiguousarray(list(prescribed.keys()), dtype=np.int64)
            v = np.ascontiguousarray(list(prescribed.values()), dtype=np.float64)
            bc.prescribed_dof = d.ctypes.data_as(C.POINTER(C.c_int64))
            bc.prescribed_val = _f64(v)
            bc.n_prescribed = d.size
            keep = (d, v)
        return bc, keep

    def solve(self, site_type, blocks, dT, clamp_bottom=True, clamp_top=False, prescribed=None,
              allow=(L.MSTRESS_ENOT_CONVERGED,)) -> "Solution":
        lay, keep1 = self._layout(site_type, blocks)
        bc, keep2 = self._bc(clamp_bottom, clamp_top, prescribed)
        h = C.c_void_p()
        rc = self.lib.mstress_solve(self.h, C.byref(lay), float(dT), C.byref(bc), C.byref(h))
        if not h.value:
            self._check(rc)
        sol = Solution(self, h, rc)
        self._check(rc, allow=allow)
        return sol

    def solve_batch(self, jobs, allow=(L.MSTRESS_ENOT_CONVERGED,)) -> "Solution":
        """jobs: list of dicts with site_type, blocks, dT and optional clamp_bottom, clamp_top, prescribed."""
        n = len(jobs)
        lays = (L.mstress_layout * n)()
        bcs = (L.mstress_bc * n)()
        dts = np.ascontiguousarray([float(j["dT"]) for j in jobs], dtype=np.float64)
        keep = []
        for k, j in enumerate(jobs):
            lay, kp = self._layout(j["site_type"], j["blocks"])
            bc, kp2 = self._bc(j.get("clamp_bottom", True), j.get("clamp_top", False), j.get("prescribed"))
            lays[k] = lay
            bcs[k] = bc
            keep.append((kp, kp2))
        h = C.c_void_p()
        rc = self.lib.mstress_solve_batch(self.h, lays, _f64(dts), bcs, n, C.byref(h))
        if not h.value:
            self._check(rc)
        sol = Solution(self, h, rc)
        self._check(rc, allow=allow)
        return sol

    def apply(self, site_type, blocks, x_ptr: int, y_ptr: int, precision=L.MSTRESS_FP64):
        lay, keep = self._layout(site_type, blocks)
        self._check(self.lib.mstress_apply(self.h, C.byref(lay), C.c_void_p(x_ptr), C.c_void_p(y_ptr), precision))


class Block:
    def __init__(self, ctx: Context, h, spec: BlockSpec):
        self.ctx, self.h, self.spec = ctx, h, spec

    def info(self):
        vals = [C.c_int() for _ in range(4)]
        self.ctx._check(self.ctx.lib.mstress_block_info(self.h, *[C.byref(v) for v in vals]))
        return dict(zip(("m", "n_el", "n_dof", "cg_iters"), [v.value for v in vals]))

    def grid(self, side: int = 100) -> "Block":
        """Build the grid modes of the half-height cut plane (side x side points)."""
        self.ctx._check(self.ctx.lib.mstress_block_grid(self.h, side))
        self.grid_side = side
        return self

    def export(self, what: int) -> np.ndarray:
        inf = self.info()
        m, n_el, n_dof = inf["m"], inf["n_el"], inf["n_dof"]
        ng = getattr(self, "grid_side", 0) ** 2
        shape = {L.MSTRESS_BLOCK_KR: (m, m), L.MSTRESS_BLOCK_BR: (m,), L.MSTRESS_BLOCK_S: (48 * n_el, m + 1),
                 L.MSTRESS_BLOCK_F: (n_dof, m + 1), L.MSTRESS_BLOCK_SMEAN: (6 * n_el, m + 1),
                 L.MSTRESS_BLOCK_SGRID: (6 * ng, m + 1)}[what]
        out = np.empty(shape, dtype=np.float64)
        self.ctx._check(self.ctx.lib.mstress_block_export(self.h, what, _f64(out), out.size))
        return out

    def close(self):
        if getattr(self, "h", None) and self.ctx.h:
            self.ctx.lib.mstress_free_block(self.h)
        self.h = None


class Solution:
    def __init__(self, ctx: Context, h, rc: int):
        self.ctx, self.h, self.rc = ctx, h, rc

    def count(self):
        n, b = C.c_int(), C.c_int64()
        self.ctx._check(self.ctx.lib.mstress_sol_count(self.h, C.byref(n), C.byref(b)))
        return n.value, b.value

    def info(self, array: int = 0):
        it, outer, st = C.c_int(), C.c_int(), C.c_int()
        rr = C.c_double()
        self.ctx._check(self.ctx.lib.mstress_sol_info(self.h, array, C.byref(it), C.byref(outer), C.byref(rr),
                                                      C.byref(st)))
        return dict(iters=it.value, outer=outer.value, rel_res=rr.value, status=st.value)

    def tiling(self):
        """Whether the reduced-precision operator ran on the tensor cores, the
        blocks per tensor-core tile the solve used, and whether the autotuner
        picked that tile."""
        u, t, a = C.c_int(), C.c_int(), C.c_int()
        self.ctx._check(self.ctx.lib.mstress_sol_tiling(self.h, C.byref(u), C.byref(t), C.byref(a)))
        return dict(use_tc=bool(u.value), tc_tile=t.value, tuned=bool(a.value))

    def phase_ms(self):
        """Device time in the persistent solver's phases (element products,
        interface sum, vector update), summed over iterations, and the count."""
        v = (C.c_double * 4)()
        self.ctx._check(self.ctx.lib.mstress_sol_phase_ms(self.h, v))
        return dict(apply=v[0], isum=v[1], update=v[2], iterations=int(v[3]))

    def recover_size(self, what: int) -> int:
        n = C.c_size_t()
        self.ctx._check(self.ctx.lib.mstress_recover_size(self.h, what, C.byref(n)))
        return n.value

    def recover(self, what: int, out=None):
        """Write output ``what`` into ``out`` (a numpy array or a CUDA torch
        tensor); with out=None returns a new numpy array (FP64, or FP32 for
        reduced-precision VM_ELEM / SIGMA_GP)."""
        nbytes = self.recover_size(what)
        if out is None:
            fp32 = (what in (L.MSTRESS_VM_ELEM, L.MSTRESS_SIGMA_GP, L.MSTRESS_VM_GRID)
                    and self.ctx.opts.precision != L.MSTRESS_FP64)
            out = np.empty(nbytes // (4 if fp32 else 8), dtype=np.float32 if fp32 else np.float64)
        if isinstance(out, np.ndarray):
            ptr, dev, have = out.ctypes.data, 0, out.nbytes
        else:
            ptr, dev, have = out.data_ptr(), int(out.is_cuda), out.numel() * out.element_size()
        self.ctx._check(self.ctx.lib.mstress_recover(self.ctx.h, self.h, what, C.c_void_p(ptr), have, dev))
        return out

    def close(self):
        if getattr(self, "h", None) and self.ctx.h:
            self.ctx.lib.mstress_free_sol(self.h)
        self.h = None


class Server:
    """Continuous-batching server over one context (mstress_server_*)."""

    def __init__(self, ctx: Context, max_slots: int = 64, hbm_budget: int = 0):
        self.ctx = ctx
        h = C.c_void_p()
        ctx._check(ctx.lib.mstress_server_create(ctx.h, max_slots, hbm_budget, C.byref(h)))
        self.h = h

    def submit(self, site_type, blocks, dT, clamp_bottom=True, clamp_top=False) -> int:
        lay, keep = Context._layout(site_type, blocks)
        bc, _ = Context._bc(clamp_bottom, clamp_top)
        rid = C.c_int64()
        self.ctx._check(self.ctx.lib.mstress_server_submit(self.h, C.byref(lay), float(dT), C.byref(bc),
                                                           C.byref(rid)))
        return rid.value

    def step(self):
        q, r, f = C.c_int(), C.c_int(), C.c_int()
        self.ctx._check(self.ctx.lib.mstress_server_step(self.h, C.byref(q), C.byref(r), C.byref(f)))
        return q.value, r.value, f.value

    def poll(self) -> int:
        rid = C.c_int64()
        self.ctx._check(self.ctx.lib.mstress_server_poll(self.h, C.byref(rid)))
        return rid.value

    def info(self, rid: int):
        st, it, outer = C.c_int(), C.c_int(), C.c_int()
        rr, lat = C.c_double(), C.c_double()
        rc = self.ctx.lib.mstress_server_info(self.h, rid, C.byref(st), C.byref(it), C.byref(outer), C.byref(rr),
                                              C.byref(lat))
        return dict(status=rc, state=st.value, iters=it.value, outer=outer.value, rel_res=rr.value,
                    latency_ms=lat.value)

    def result(self, rid: int, out):
        if isinstance(out, np.ndarray):
            ptr, dev, have = out.ctypes.data, 0, out.nbytes
        else:
            ptr, dev, have = out.data_ptr(), int(out.is_cuda), out.numel() * out.element_size()
        self.ctx._check(self.ctx.lib.mstress_server_result(self.h, rid, C.c_void_p(ptr), have, dev))
        return out

    def release(self, rid: int):
        self.ctx._check(self.ctx.lib.mstress_server_release(self.h, rid))

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.mstress_free_server(self.h)
            self.h = None


def launch_count() -> int:
    """Kernels launched by libmstress in this process so far."""
    lib = L.load()
    n = C.c_int64()
    lib.mstress_launch_count(C.byref(n))
    return n.value


def strip_partition(ny: int, order: int, world: int, rank: int) -> dict:
    """Row-strip plan of one array's global stage for `rank` of `world`
    (mstress_strip_partition): block rows [j0, j1), owned lattice rows
    [y_own0, y_own1), the boundary rows sent (y_send) and received (y_recv),
    and the neighbouring ranks (-1 where none)."""
    lib = L.load()
    out = L.mstress_strip()
    rc = lib.mstress_strip_partition(ny, order, world, rank, C.byref(out))
    if rc != L.MSTRESS_OK:
        raise MstressError(rc, "invalid strip partition arguments")
    return {name: getattr(out, name) for name, _ in L.mstress_strip._fields_}


def profile(ctx: Context, sol: Solution, phase: int, reps: int = 20) -> float:
    """Mean duration (ms) of one launch of a solve phase kernel (see mstress_profile)."""
    ms = C.c_double()
    ctx._check(ctx.lib.mstress_profile(ctx.h, sol.h, phase, reps, C.byref(ms)))
    return ms.value
