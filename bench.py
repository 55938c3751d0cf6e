#!/usr/bin/env python3
"""Benchmark of the MORE-Stress global stage on one GB300.

Workload: the 100x100 TSV array of 10x10x50 um blocks (Cu TSV radius 2.5 um,
0.5 um SiO2 liner, 12x12x10 Q1 hex mesh, degree-2 face basis, m = 78), every
site occupied, dT = -250 K, bottom clamped. One step = one global-stage solve
(mstress_solve) plus the per-element von Mises recovery of every block
(mstress_recover, VM_ELEM) through the C ABI; the reduced block models are
built once beforehand on the GPU (the one-shot local stage, not timed).

Metric: TSV blocks solved+recovered per second. With --gpus N (torchrun) every
rank runs its own replica of the workload (weak scaling, no collective on the
data path); the value is all ranks' blocks over the slowest rank's time.

``--impl reference`` times the CPU oracle (plain FP64 reduced model with a
sparse direct solve) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TSV blocks solved+recovered/s (100x100 array)"
PREC = {"fp64": 0, "tf32": 1, "bf16": 2, "bf16x3": 3}
DTYPE = {"fp64": "f64", "tf32": "tf32+f32+f64", "bf16": "bf16+f32+f64", "bf16x3": "bf16x3+f32+f64"}
ORACLE_SIDE = 40          # bounded CPU sample: a 40x40 array of the same block
# ncu dram__bytes_read.sum + dram__bytes_write.sum of the k_pcg launches of one
# 100x100 solve divided by its PCG iterations (bytes per iteration), by
# precision mode; a mode is absent until it has been measured on the current
# kernel (the figure is then reported as null).
# BF16X3 (mode 3): 31.76 MB read + written by the 4 launches of one solve over
# its 304 iterations.
PCG_TRAFFIC: dict[int, float] = {3: 104500.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=list(PREC))
    ap.add_argument("--nx", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the sub-records (FP64 array, 256-array batch and served stream in both forms)")
    ap.add_argument("--workload", default="array100", choices=["array100", "batch256", "serve"],
                    help="array100: the headline 100x100 array; batch256: 256 uneven arrays in one batched "
                         "solve; serve: a Poisson request stream through the continuous-batching server")
    ap.add_argument("--n-arrays", type=int, default=256)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--load", type=float, default=0.8, help="serve: arrival rate as a fraction of capacity")
    return ap.parse_args()


# ------------------------------------------------------------ CPU oracle
ORACLE_CODE = r"""
import json, sys, time, os
sys.path.insert(0, {root!r})
import numpy as np, warnings
warnings.simplefilter("ignore")
from oracle import fem, mor
from paper_2411_12690_gb300 import workloads as W
spec = W.BLOCK_SMALL
mesh = fem.tsv_block_mesh(spec.lx, spec.ly, spec.lz, spec.ex, spec.ey, spec.ez, spec.r_cu, spec.t_liner)
blk = mor.local_stage(mesh, (3, 3, 3))                 # local stage: not part of the timed sample
st = W.site_types({side}, {side}, 1.0)
start = float({start})
while time.time() < start:                             # concurrent runs start their timed work together
    time.sleep(0.01)
times = []
w0 = time.time()
for k in range({reps}):
    t0 = time.perf_counter()
    sol = mor.global_stage([blk], st, W.DT_DEFAULT)
    vm = mor.recover_vm([blk], sol)
    times.append(time.perf_counter() - t0)
print(json.dumps(dict(times=times, blocks=int(st.size), wall=[w0, time.time()])))
"""


def _oracle_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    return env


def run_oracle(side: int, reps: int) -> dict:
    """Time the oracle's online part (assembly + direct solve + recovery) in a
    fresh single-threaded interpreter."""
    code = ORACLE_CODE.format(root=ROOT, side=side, reps=reps, start=0.0)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=_oracle_env(), timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_all_cores(side: int, reps: int) -> dict:
    """The same sample on every host core at once: one single-threaded oracle
    process per core (the direct solver is sequential, so a core per
    independent array is how the oracle uses a many-core host), all starting
    their timed work together; throughput = all processes' blocks over the
    span from the first start to the last finish."""
    n = os.cpu_count() or 1
    start = time.time() + 20.0 + 0.5 * n        # after every process has built its block model
    code = ORACLE_CODE.format(root=ROOT, side=side, reps=reps, start=start)
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True, env=_oracle_env()) for _ in range(n)]
    res = []
    for p in procs:
        out, err = p.communicate(timeout=1800)
        if p.returncode != 0:
            raise RuntimeError("oracle run failed: " + err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    w0 = min(r["wall"][0] for r in res)
    w1 = max(r["wall"][1] for r in res)
    return dict(blocks=sum(r["blocks"] * len(r["times"]) for r in res), seconds=w1 - w0, procs=n,
                late_start=max(r["wall"][0] for r in res) - start)


def cpu_baseline_entry(one: dict, allc: dict | None = None) -> dict:
    t = statistics.median(one["times"])
    single = {"value": one["blocks"] / t, "unit": "blocks/s", "cores": 1, "kind": "oracle",
              "sample": f"{ORACLE_SIDE}x{ORACLE_SIDE} array of the same block (assembly + sparse direct solve + "
                        f"von Mises recovery of every block, FP64), median of {len(one['times'])} runs in one "
                        f"single-threaded process; the direct solve grows faster than linearly, so this "
                        f"overstates the oracle at 100x100"}
    if not allc:
        return single
    return {"value": allc["blocks"] / allc["seconds"], "unit": "blocks/s", "cores": allc["procs"], "kind": "oracle",
            "sample": f"{allc['procs']} concurrent single-threaded oracle processes (one per host core), each "
                      f"solving and recovering a {ORACLE_SIDE}x{ORACLE_SIDE} array of the same block; blocks of all "
                      f"processes over the span from the first start to the last finish "
                      f"({allc['seconds']:.1f} s)",
            "nproc": os.cpu_count(), "single_core": single}


def whole_job_rate(dist, world: int, units_per_rank: float, rank_seconds: float, device="cuda"):
    """Whole-job throughput of `world` replicas: every rank's units over the
    slowest rank's time (barrier, then the max of the ranks' times). Returns
    (units per second, slowest rank's seconds). dist is torch.distributed or
    None for a single process."""
    import torch
    t = torch.tensor([rank_seconds], dtype=torch.float64, device=device)
    if dist is not None:
        dist.barrier()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    slowest = float(t.item())
    return world * units_per_rank / slowest, slowest


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    res = run_oracle(ORACLE_SIDE, args.warmup + args.steps)
    times = res["times"][args.warmup:]
    blocks = res["blocks"]
    total = sum(times)
    value = blocks * len(times) / total
    cb = cpu_baseline_entry(dict(times=times, blocks=blocks))
    cb["value"] = value
    cb["nproc"] = os.cpu_count()
    line = {"metric": METRIC, "value": value, "unit": "blocks/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"oracle sample: {ORACLE_SIDE}x{ORACLE_SIDE} array of the 10x10x50 um TSV block "
                                   f"(12x12x10 hex mesh, degree-2 basis, m=78), dT=-250 K, bottom clamped",
                       "sample_of": "100x100 array", "l2": "n/a (CPU)"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "blocks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ GPU arm
def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def array_roofline(prec, nx, ny, ph, t_rec, sm_mhz, it_mode):
    """Roofline of the 100x100 step's kernels. The PCG runs as one persistent
    kernel (k_pcg) whose phases are timed on the device (globaltimer at its
    grid barriers); the recovery kernel is timed with CUDA events on the
    context stream. Algorithmic work per PCG iteration (N blocks, m = 78,
    n_glob global DOFs = lattice points on block surfaces x 3, w vector bytes):
      two-phase iteration (tensor-core apply): phase A reads p, z and writes
        Y (m N w), phase B reads dinv, p, z, x, r and Y and writes p, x, r, z:
        bytes = 11 n_glob w + 2 m N w
      three-phase iteration (FP64 / CUDA-core apply): A reads p, z, writes Y;
        B reads dinv, p, z, Y, writes p, q; C reads p, q, x, r, dinv, writes
        x, r, z: bytes = 15 n_glob w + 2 m N w
      a3 flops = 2 m^2 N per operand product (3 products issued in bf16x3);
      a6 recovery flops = 2 (6 N_el) (m+1) N, the method's contraction of the
        Gauss-mean stress modes (one product); von Mises out N_el N w bytes."""
    m, n_el = 78, 1440
    n_blocks = nx * ny
    n_glob = 3 * ((2 * nx + 1) * (2 * ny + 1) * 3 - n_blocks)   # n = 3: one interior lattice point per block
    w = 8 if prec == 0 else 4
    products = 3 if prec == 3 else 1
    passes = 11 if it_mode == 2 else 15
    it_bytes = passes * n_glob * w + 2 * m * n_blocks * w
    a3_bytes = 2 * n_glob * w + m * n_blocks * w
    a3_flops = 2.0 * m * m * n_blocks
    rec_flops = 2.0 * 6 * n_el * (m + 1) * n_blocks
    rec_bytes = n_el * n_blocks * w
    pk = _peaks()
    hbm = pk.get("hbm_gbs") or 6800.0
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (measured)" if pk.get("hbm_gbs") else "fallback 6800 GB/s"
    bf16 = pk.get("bf16_tflops") or 1900.0
    # tensor peak of the mode's operand type: bf16 measured; tf32 = bf16 x nominal 1.1 / 2.25
    tensor_peak = {1: bf16 * 1.1 / 2.25, 2: bf16, 3: bf16}.get(prec)
    fp64_peak = 152 * 4 * sm_mhz * 1e6 / 1e12     # 152 SMs x 2 DFMA/clk at the sampled SM clock
    n_iter = max(1, ph["iterations"])
    t_apply = ph["apply"] / n_iter
    t_pcg = (ph["apply"] + ph["isum"] + ph["update"]) / n_iter        # ms per iteration
    if prec == 0:
        roof = {"bound": "alu", "achieved": a3_flops / (t_apply * 1e-3) / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s", "traffic": None,
                "kernel": "k_pcg<FP64> phase A (element products on the FP64 pipe)",
                "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x sampled SM clock (probe measured 1.257 TFLOP/s)"}
    else:
        roof = {"bound": "hbm", "achieved": it_bytes / (t_pcg * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "traffic": PCG_TRAFFIC.get(prec), "peak_source": hbm_src,
                "kernel": "k_pcg (persistent PCG: tensor-core apply, fused interface sum + vector update)",
                "note": "the vectors are L2-resident at this size, so the iteration is latency-bound (two grid "
                        "barriers and folds per iteration), not HBM-bound; traffic = ncu DRAM bytes of the k_pcg "
                        "launches of one solve divided by its iterations (bytes per iteration), null when not "
                        "measured on the current kernel"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["algorithmic_bytes_per_iteration"] = it_bytes
    roof["global_dofs"] = n_glob
    roof["per_iteration_ms"] = {"apply": t_apply, "vector": (ph["isum"] + ph["update"]) / n_iter, "total": t_pcg}
    roof["a3_apply"] = {"bytes": a3_bytes, "flops": a3_flops, "ms": t_apply,
                        "gbs": a3_bytes / (t_apply * 1e-3) / 1e9,
                        "frac_hbm": a3_bytes / (t_apply * 1e-3) / 1e9 / hbm,
                        "tflops": a3_flops / (t_apply * 1e-3) / 1e12}
    roof["a6_recover"] = {"flops": rec_flops, "ms": t_rec, "tflops": rec_flops / (t_rec * 1e-3) / 1e12,
                          "out_bytes": rec_bytes, "gbs": rec_bytes / (t_rec * 1e-3) / 1e9,
                          "frac_hbm": rec_bytes / (t_rec * 1e-3) / 1e9 / hbm}
    if tensor_peak:
        roof["a3_apply"]["frac_tensor"] = roof["a3_apply"]["tflops"] / tensor_peak
        roof["a6_recover"]["frac_tensor"] = roof["a6_recover"]["tflops"] / tensor_peak
        roof["a6_recover"]["products_issued"] = products
        roof["a6_recover"]["frac_tensor_issued"] = roof["a6_recover"]["frac_tensor"] * products
        roof["a6_recover"]["tensor_peak_tflops"] = tensor_peak
    else:
        roof["a6_recover"]["frac_fp64"] = roof["a6_recover"]["tflops"] / fp64_peak
    roof["recover_ms"] = t_rec
    share = {"pcg": ph["apply"] + ph["isum"] + ph["update"], "recover": t_rec}
    roof["time_share"] = {k: v / sum(share.values()) for k, v in share.items()}
    return roof


def array_run(prec_name, nx, steps, warmup, local, dist=None, world=1, e2e=True):
    """The nx x nx array workload in one precision: warm-up, timed steps (L2
    flushed before each, CUDA events on the context stream, clocks sampled),
    the end-to-end pass through the C ABI with host buffers, and the
    roofline figures of the last solve. Returns a dict."""
    import torch

    from paper_2411_12690_gb300 import _lib as L
    from paper_2411_12690_gb300 import api
    from paper_2411_12690_gb300 import workloads as W

    prec = PREC[prec_name]
    stream = torch.cuda.current_stream()
    ctx = api.Context(stream=stream.cuda_stream, precision=prec)
    spec = W.BLOCK_SMALL
    blks = [ctx.build_block(spec), ctx.build_block(spec.dummy())]
    n_el = spec.ex * spec.ey * spec.ez
    st = W.site_types(nx, nx, 1.0)
    n_blocks = nx * nx
    vm_dtype = torch.float64 if prec == 0 else torch.float32
    vm_dev = torch.empty(n_blocks * n_el, dtype=vm_dtype, device="cuda")
    vm_host = torch.empty(n_blocks * n_el, dtype=vm_dtype).pin_memory()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")    # > 129 MB L2

    def step(out):
        sol = ctx.solve(st, blks, W.DT_DEFAULT)
        sol.recover(L.MSTRESS_VM_ELEM, out=out)
        return sol

    for _ in range(warmup):
        step(vm_dev).close()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = api.launch_count()
    total_ms = 0.0
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sol = step(vm_dev)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        sol.close()
    launches = api.launch_count() - l0
    clk = clocks.stop()
    value, slowest = whole_job_rate(dist, world, n_blocks * steps, total_ms / 1e3)
    out = {"value": value, "ms_per_step": 1e3 * slowest / steps, "steps": steps, "warmup": warmup,
           "gpu_launches": int(launches), "clocks": clk}
    if e2e:
        # end to end: host inputs (site map, dT) in, von Mises to pinned host memory, every step
        e2e_t = 0.0
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = ctx.solve(st, blks, W.DT_DEFAULT)
            s2.recover(L.MSTRESS_VM_ELEM, out=vm_host)
            e2e_t += time.perf_counter() - t0
            s2.close()
        e2e_value, _ = whole_job_rate(dist, world, n_blocks * steps, e2e_t)
        out["e2e"] = {"value": e2e_value, "unit": "blocks/s", "h2d_bytes_per_step": int(st.size + 8),
                      "d2h_bytes_per_step": int(vm_host.numel() * vm_host.element_size())}
    sol = step(vm_dev)
    info = sol.info()
    ph = sol.phase_ms()
    t_rec = api.profile(ctx, sol, 3, 5)
    tiling = sol.tiling()
    two_phase = tiling["use_tc"]
    out["roofline"] = array_roofline(prec, nx, nx, ph, t_rec, clk.get("sm_mhz") or 1900.0, 2 if two_phase else 3)
    out["config"] = {"precision": prec_name, "blocks": n_blocks, "pcg_iters": info["iters"],
                     "refinement_steps": info["outer"], "rel_res": info["rel_res"],
                     "tc_tile": tiling["tc_tile"], "tile_autotuned": tiling["tuned"],
                     "l2": "flushed before every timed step (512 MB write)"}
    sol.close()
    ctx.close()
    del flush
    torch.cuda.empty_cache()
    return out


def ours(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # before any GPU work in this process: one thread, then every core
        cpu = cpu_baseline_entry(run_oracle(ORACLE_SIDE, 3), run_oracle_all_cores(ORACLE_SIDE, 2))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    r = array_run(args.precision, args.nx, args.steps, args.warmup, local, dist, world)
    if rank == 0:
        nx = ny = args.nx
        line = {"metric": METRIC, "value": r["value"], "unit": "blocks/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
                "config": dict({"workload": f"{nx}x{ny} TSV array, 10x10x50 um blocks, Cu r=2.5 um + 0.5 um SiO2 "
                                            f"liner, 12x12x10 Q1 hex mesh, degree-2 face basis (m=78), all sites "
                                            f"occupied, dT=-250 K, bottom clamped; solve + per-element von Mises",
                                "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
                               **r["config"]),
                "roofline": r["roofline"], "e2e": r["e2e"], "gpu_launches": r["gpu_launches"],
                "clocks": r["clocks"]}
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if world == 1 and not args.no_extras:
            line["sub_records"] = extra_records(args, local)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def extra_records(args, local):
    """Further configurations measured in the same run, each with its own
    timing, roofline and clock record: the plain FP64 path on the same
    100x100 array, the 256-array batch and the served request stream, each in
    the mixed (BF16X3) and in the plain FP64 form."""
    recs = {}
    t0 = time.perf_counter()
    r = array_run("fp64", args.nx, 5, 3, local, e2e=False)
    recs["array100_fp64"] = dict(r, metric=METRIC, unit="blocks/s", dtype=DTYPE["fp64"], wall_s=time.perf_counter() - t0)
    for prec_name, steps, warm in (("bf16x3", 2, 1), ("fp64", 1, 0)):
        t0 = time.perf_counter()
        recs[f"batch256_{prec_name}"] = dict(batch_run(prec_name, args.n_arrays, steps, warm, local),
                                             wall_s=time.perf_counter() - t0)
    for prec_name, nreq in (("bf16x3", args.requests), ("fp64", max(24, args.requests // 4))):
        t0 = time.perf_counter()
        recs[f"serve_{prec_name}"] = dict(serve_run(prec_name, nreq, args.load, local),
                                          wall_s=time.perf_counter() - t0)
    t0 = time.perf_counter()
    recs["scenario1_sweep_bf16x3"] = dict(scenario1_run("bf16x3", local), wall_s=time.perf_counter() - t0)
    t0 = time.perf_counter()
    recs["submodel_bf16x3"] = dict(submodel_run("bf16x3", local), wall_s=time.perf_counter() - t0)
    return recs


# the paper's global-stage times (seconds) for scenario 1 (Table 1) and the
# sub-model of scenario 2 (Table 2), on its CPU (context for the GPU times)
PAPER_S1_SECONDS = {15: {10: 2.5, 20: 4.4, 30: 9.5, 40: 13.1, 50: 17.1},
                    10: {10: 2.3, 20: 4.5, 30: 11.4, 40: 13.9, 50: 18.5}}
PAPER_S2_SECONDS = (3.5, 3.7)


def _timed_steps(stream, step, steps, warmup):
    """Device time (CUDA events on the context stream) of `steps` calls of
    step() after `warmup` untimed ones; returns seconds per step."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1) / 1e3
    return tot / steps


def scenario1_run(prec_name, local, sizes=(10, 20, 30, 40, 50), steps=3, warmup=1):
    """Scenario 1 of section 5.1: stand-alone arrays of 10x10 .. 50x50 TSV
    blocks, pitch 15 and 10 um, (4,4,4) interpolation nodes (m = 168), top and
    bottom clamped, dT = -250 K; a step is the solve plus the per-element von
    Mises and the gridded half-height von Mises (100 x 100 points per block,
    the paper's error-measure output)."""
    import torch

    from paper_2411_12690_gb300 import _lib as L
    from paper_2411_12690_gb300 import api
    from paper_2411_12690_gb300 import workloads as W

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = api.Context(stream=stream.cuda_stream, precision=PREC[prec_name])
    out = {"metric": "TSV blocks solved+recovered/s per array size (scenario 1)", "unit": "blocks/s",
           "dtype": DTYPE[prec_name], "steps": steps, "warmup": warmup, "by_pitch": {}}
    clocks = ClockSampler(local)
    clocks.start()
    for pitch, spec in ((15, W.BLOCK_P15_O3), (10, W.BLOCK_P10_O3)):
        blks = [ctx.build_block(spec).grid(100), ctx.build_block(spec.dummy()).grid(100)]
        n_el = spec.ex * spec.ey * spec.ez
        rows = {}
        for n in sizes:
            st = W.site_types(n, n, 1.0)
            vm = torch.empty(n * n * n_el, dtype=torch.float32, device="cuda")
            vg = torch.empty(n * n * 10000, dtype=torch.float32, device="cuda")
            info = {}

            def step():
                sol = ctx.solve(st, blks, W.DT_DEFAULT, clamp_top=True)
                sol.recover(L.MSTRESS_VM_ELEM, out=vm)
                sol.recover(L.MSTRESS_VM_GRID, out=vg)
                info.update(sol.info())
                sol.close()

            sec = _timed_steps(stream, step, steps, warmup)
            rows[f"{n}x{n}"] = {"blocks": n * n, "ms_per_step": 1e3 * sec, "value": n * n / sec,
                                "pcg_iters": info["iters"], "refinement_steps": info["outer"],
                                "rel_res": info["rel_res"],
                                "paper_global_stage_s": PAPER_S1_SECONDS[pitch][n],
                                "paper_over_this": PAPER_S1_SECONDS[pitch][n] / sec}
            del vm, vg
        out["by_pitch"][f"p{pitch}"] = rows
        for b in blks:
            b.close()
    out["clocks"] = clocks.stop()
    out["config"] = {"workload": "stand-alone TSV arrays, p = 15 um (24x24x20 mesh) and 10 um (16x16x20 mesh) "
                                 "blocks, (4,4,4) nodes (m=168), top+bottom clamped, dT=-250 K; solve + per-element "
                                 "and gridded (100x100 per block) von Mises",
                     "paper_times": "the paper's global-stage seconds on its CPU (8 threads), context only"}
    ctx.close()
    torch.cuda.empty_cache()
    return out


def submodel_run(prec_name, local, steps=5, warmup=2):
    """Scenario 2 (sections 4.4, 5.1): a 15x15 TSV array of pitch-15 um
    blocks ((4,4,4) nodes) inside two rings of dummy blocks, every outer face
    of the sub-model driven by the synthetic coarse-model boundary field
    (lifting), no clamped face; solve + gridded von Mises (100 x 100 per
    block)."""
    import torch

    from paper_2411_12690_gb300 import _lib as L
    from paper_2411_12690_gb300 import api
    from paper_2411_12690_gb300 import workloads as W

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = api.Context(stream=stream.cuda_stream, precision=PREC[prec_name])
    spec = W.BLOCK_P15_O3
    blks = [ctx.build_block(spec).grid(100), ctx.build_block(spec.dummy()).grid(100)]
    st = W.submodel_sites(15, 2)
    ny, nx = st.shape
    dof, val = W.submodel_boundary(nx, ny, spec, seed=0)
    presc = dict(zip(dof.tolist(), val.tolist()))
    vg = torch.empty(st.size * 10000, dtype=torch.float32, device="cuda")
    info = {}

    def step():
        sol = ctx.solve(st, blks, W.DT_DEFAULT, clamp_bottom=False, prescribed=presc)
        sol.recover(L.MSTRESS_VM_GRID, out=vg)
        info.update(sol.info())
        sol.close()

    clocks = ClockSampler(local)
    clocks.start()
    sec = _timed_steps(stream, step, steps, warmup)
    clk = clocks.stop()
    ctx.close()
    torch.cuda.empty_cache()
    return {"metric": "sub-model blocks solved+recovered/s (15x15 TSV array + 2 dummy rings)", "unit": "blocks/s",
            "value": st.size / sec, "ms_per_step": 1e3 * sec, "steps": steps, "warmup": warmup,
            "dtype": DTYPE[prec_name], "pcg_iters": info["iters"], "refinement_steps": info["outer"],
            "rel_res": info["rel_res"], "paper_global_stage_s": list(PAPER_S2_SECONDS),
            "config": {"workload": "19x19 sites (15x15 TSV + 2 dummy rings), p = 15 um, (4,4,4) nodes (m=168), "
                                   "synthetic warpage-like boundary field on all six faces by lifting, dT=-250 K; "
                                   "solve + gridded von Mises (100x100 per block)",
                       "prescribed_dofs": int(dof.size)},
            "clocks": clk}


def _variant_models(ctx, W):
    """Both pitch variants (15 and 20 um, 24x24x20 mesh, degree 4) with their dummy blocks."""
    return [[ctx.build_block(v), ctx.build_block(v.dummy())] for v in (W.BLOCK_P15, W.BLOCK_P20)]


def batch_run(prec_name, n_arrays, steps, warmup, local):
    """256 independent arrays (side log-uniform 4..64, occupancy U[0.5,1],
    pitch 15/20 um, dT U[-300,-150] K) solved and recovered in one batch,
    timed with CUDA events on the context stream. With no warm-up steps of the
    full batch, a 4-array batch warms the same code paths first."""
    import torch

    from paper_2411_12690_gb300 import _lib as L
    from paper_2411_12690_gb300 import api
    from paper_2411_12690_gb300 import workloads as W

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    prec = PREC[prec_name]
    ctx = api.Context(stream=stream.cuda_stream, precision=prec)
    models = _variant_models(ctx, W)
    jobs = W.batch_arrays(n_arrays, seed=0)
    spec = [dict(site_type=j.site_type, blocks=models[j.pitch], dT=j.dT) for j in jobs]
    n_blocks = sum(j.site_type.size for j in jobs)
    n_el = W.BLOCK_P15.ex * W.BLOCK_P15.ey * W.BLOCK_P15.ez
    vm = torch.empty(n_blocks * n_el, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    if warmup == 0:
        small = spec[:4]
        nb = sum(j["site_type"].size for j in small)
        s0 = ctx.solve_batch(small)
        s0.recover(L.MSTRESS_VM_ELEM, out=vm[:nb * n_el])
        s0.close()
    times, split = [], []
    clocks = None
    for k in range(warmup + steps):
        if k == warmup:
            clocks = ClockSampler(local)
            clocks.start()
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        sol = ctx.solve_batch(spec)
        e1.record(stream)
        sol.recover(L.MSTRESS_VM_ELEM, out=vm)
        e2.record(stream)
        torch.cuda.synchronize()
        if k >= warmup:
            times.append(e0.elapsed_time(e2) / 1e3)
            split.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
        infos = [sol.info(a) for a in range(len(jobs))]
        phases = sol.phase_ms()
        tiling = sol.tiling()
        if k == warmup + steps - 1 and not phases["iterations"]:
            # per-phase iteration: its apply kernel timed alone (CUDA events, context stream)
            phases["apply_kernel_ms"] = api.profile(ctx, sol, 0, 5)
        sol.close()
    clk = clocks.stop()
    total = sum(times)
    rec_ms = sum(b for _, b in split) / len(split)
    out = {"metric": "TSV blocks solved+recovered/s (256-array batch)", "value": n_blocks * len(times) / total,
           "unit": "blocks/s", "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * total / len(times),
           "higher_is_better": True, "dtype": DTYPE[prec_name],
           "config": {"workload": f"{len(jobs)} arrays, side log-uniform 4..64, occupancy U[0.5,1], pitch 15/20 um "
                                  f"(24x24x20 mesh, degree-4 basis, m=294), dT U[-300,-150] K, one batched solve",
                      "blocks": n_blocks, "max_pcg_iters": max(i["iters"] for i in infos),
                      "max_refinement_steps": max(i["outer"] for i in infos),
                      "max_rel_res": max(i["rel_res"] for i in infos),
                      "solve_ms": sum(a for a, _ in split) / len(split), "recover_ms": rec_ms,
                      "iteration": ("persistent cooperative kernel" if phases["iterations"] else
                                    "per-phase launches in a CUDA graph (k_apply_tcs, k_w_isum, k_w_alpha, "
                                    "k_w_vec, k_w_beta)"),
                      "persistent_phase_ms": phases,
                      "tc_tile": tiling.get("tc_tile"), "tile_autotuned": tiling.get("tuned"),
                      "l2": "inputs larger than L2 (the batch's vectors and element products exceed 129 MB)"},
           "roofline": batch_roofline(prec, jobs, n_blocks, n_el, phases, rec_ms, clk.get("sm_mhz") or 1900.0),
           "clocks": clk}
    ctx.close()
    del vm
    torch.cuda.empty_cache()
    return out


def batch_roofline(prec, jobs, n_blocks, n_el, ph, rec_ms, sm_mhz):
    """a3 (element products, per PCG iteration) against the measured HBM peak
    (bytes = gathered coefficients m N w_in + Y written m N w + p, z read
    2 n_vec w) and a6 (the recovery) against the tensor peak (the method's
    flops 2 (6 n_el) (m+1) N, one product) and HBM (the von Mises written,
    N n_el w bytes); FP64: the element products against the FP64 pipe."""
    m = 294
    n_vec = sum(3 * (j.site_type.shape[1] * 4 + 1) * (j.site_type.shape[0] * 4 + 1) * 5 for j in jobs)
    w = 8 if prec == 0 else 4
    w_in = {0: 8, 1: 4, 2: 2, 3: 4}[prec]
    pk = _peaks()
    hbm = pk.get("hbm_gbs") or 6800.0
    bf16 = pk.get("bf16_tflops") or 1900.0
    it = max(1, ph["iterations"])
    t_apply = ph["apply"] / it if ph["iterations"] else ph["apply_kernel_ms"]
    a3_bytes = m * n_blocks * w_in + m * n_blocks * w + 2 * n_vec * w
    a3_flops = 2.0 * m * m * n_blocks
    rec_bytes = n_blocks * n_el * w
    a3 = {"bytes": a3_bytes, "flops": a3_flops, "ms": t_apply, "gbs": a3_bytes / (t_apply * 1e-3) / 1e9,
          "tflops": a3_flops / (t_apply * 1e-3) / 1e12}
    a3["frac_hbm"] = a3["gbs"] / hbm
    a6 = {"bytes": rec_bytes, "ms": rec_ms, "gbs": rec_bytes / (rec_ms * 1e-3) / 1e9}
    a6["frac_hbm"] = a6["gbs"] / hbm
    a6["flops"] = 2.0 * 6 * n_el * (m + 1) * n_blocks
    a6["tflops"] = a6["flops"] / (rec_ms * 1e-3) / 1e12
    tensor_peak = {1: bf16 * 1.1 / 2.25, 2: bf16, 3: bf16}.get(prec)
    if tensor_peak:
        a6["frac_tensor"] = a6["tflops"] / tensor_peak
        a6["products_issued"] = 3 if prec == 3 else 1
        return {"bound": "hbm", "achieved": a3["gbs"], "peak": hbm, "unit": "GB/s", "frac": a3["frac_hbm"],
                "traffic": None,
                "kernel": ("k_pcg phase A (streamed tensor-core element products, per iteration)" if ph["iterations"]
                           else "k_apply_tcs (streamed tensor-core element products, one launch per iteration)"),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)", "a3_apply": a3, "a6_recover": a6,
                "lattice_dofs": n_vec}
    fp64_peak = 152 * 4 * sm_mhz * 1e6 / 1e12
    return {"bound": "alu", "achieved": a3["tflops"], "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": a3["tflops"] / fp64_peak, "traffic": None,
            "kernel": "k_pcg<FP64> phase A (element products on the FP64 pipe, per iteration)",
            "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x sampled SM clock", "a3_apply": a3, "a6_recover": a6,
            "lattice_dofs": n_vec}


def serve_run(prec_name, n_requests, load, local):
    """Poisson request stream through the continuous-batching server: arrays
    log-uniform 2..128, occupancy U[0.5,1], pitch 15/20 um, dT U[-300,-150] K;
    arrival rate = load x the capacity measured by a closed-loop pass."""
    import torch

    from paper_2411_12690_gb300 import api
    from paper_2411_12690_gb300 import workloads as W

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = api.Context(stream=stream.cuda_stream, precision=PREC[prec_name])
    models = _variant_models(ctx, W)

    def run(reqs, rate_scale):
        srv = api.Server(ctx, max_slots=64)
        t0 = time.perf_counter()
        pending = list(reqs)
        done, lat, blocks = 0, [], 0
        ids = {}
        while done < len(reqs):
            now = time.perf_counter() - t0
            while pending and pending[0].t_arrival * rate_scale <= now:
                r = pending.pop(0)
                ids[srv.submit(r.job.site_type, models[r.job.pitch], r.job.dT)] = r
            q, running, _ = srv.step()
            while True:
                rid = srv.poll()
                if not rid:
                    break
                inf = srv.info(rid)
                lat.append(inf["latency_ms"])
                blocks += ids[rid].job.site_type.size
                srv.release(rid)
                done += 1
            if not running and not q and pending:
                time.sleep(max(0.0, min(0.01, pending[0].t_arrival * rate_scale - (time.perf_counter() - t0))))
        elapsed = time.perf_counter() - t0
        srv.close()
        return blocks / elapsed, lat, elapsed

    warm = W.request_stream(1.0, 8, seed=1)
    run([W.Request(0.0, r.job) for r in warm], 0.0)                       # warm-up
    probe = W.request_stream(1.0, max(16, n_requests // 4), seed=2)
    cap_blocks, _, cap_t = run([W.Request(0.0, r.job) for r in probe], 0.0)  # closed loop: capacity
    cap_rps = len(probe) / cap_t
    reqs = W.request_stream(load * cap_rps, n_requests, seed=0)
    clocks = ClockSampler(local)
    clocks.start()
    thr, lat, elapsed = run(reqs, 1.0)
    clk = clocks.stop()
    lat = sorted(lat)
    ctx.close()
    torch.cuda.empty_cache()
    return {"metric": "served TSV blocks/s with p50/p99 request latency", "value": thr, "unit": "blocks/s",
            "higher_is_better": True, "dtype": DTYPE[prec_name],
            "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "requests": len(lat), "elapsed_s": elapsed,
            "config": {"workload": "Poisson stream, arrays log-uniform 2..128, occupancy U[0.5,1], pitch "
                                   "15/20 um (m=294), dT U[-300,-150] K, max 64 slots",
                       "arrival_rate_per_s": load * cap_rps, "load": load,
                       "closed_loop_capacity_blocks_per_s": cap_blocks},
            "clocks": clk}


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "batch256":
        print(json.dumps(dict(batch_run(args.precision, args.n_arrays, args.steps, args.warmup,
                                        int(os.environ.get("LOCAL_RANK", "0"))), n_gpus=1, data="synthetic")),
              flush=True)
    elif args.workload == "serve":
        print(json.dumps(dict(serve_run(args.precision, args.requests, args.load,
                                        int(os.environ.get("LOCAL_RANK", "0"))), n_gpus=1, data="synthetic")),
              flush=True)
    else:
        ours(args)


if __name__ == "__main__":
    main()
