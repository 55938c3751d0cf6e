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
# 100x100 solve divided by its PCG iterations, per precision (bytes per
# iteration: 30.85 MB over the 4 launches of a solve, nearly the same for every
# launch whatever its length, over the solve's 315 iterations); absent for a
# precision not measured with the current kernel.
PCG_TRAFFIC = {"bf16x3": 97940}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=list(PREC))
    ap.add_argument("--nx", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
times = []
for k in range({reps}):
    t0 = time.perf_counter()
    sol = mor.global_stage([blk], st, W.DT_DEFAULT)
    vm = mor.recover_vm([blk], sol)
    times.append(time.perf_counter() - t0)
print(json.dumps(dict(times=times, blocks=int(st.size))))
"""


def run_oracle(side: int, reps: int) -> dict:
    """Time the oracle's online part (assembly + direct solve + recovery) in a
    fresh single-threaded interpreter."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ORACLE_CODE.format(root=ROOT, side=side, reps=reps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline_entry(res: dict) -> dict:
    t = statistics.median(res["times"])
    return {"value": res["blocks"] / t, "unit": "blocks/s", "cores": 1, "kind": "oracle",
            "sample": f"{ORACLE_SIDE}x{ORACLE_SIDE} array of the same block (assembly + sparse direct solve + "
                      f"von Mises recovery of every block, FP64), median of {len(res['times'])} runs; the "
                      f"direct solve grows faster than linearly, so this overstates the oracle at 100x100"}


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
def ours(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu_res = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu_res = run_oracle(ORACLE_SIDE, 3)      # before any GPU work in this process
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2411_12690_gb300 import _lib as L
    from paper_2411_12690_gb300 import api
    from paper_2411_12690_gb300 import workloads as W

    prec = PREC[args.precision]
    stream = torch.cuda.current_stream()
    ctx = api.Context(stream=stream.cuda_stream, precision=prec)
    spec = W.BLOCK_SMALL
    blks = [ctx.build_block(spec), ctx.build_block(spec.dummy())]
    n_el = spec.ex * spec.ey * spec.ez
    nx = ny = args.nx
    st = W.site_types(nx, ny, 1.0)
    n_blocks = nx * ny
    vm_dtype = torch.float64 if prec == 0 else torch.float32
    vm_dev = torch.empty(n_blocks * n_el, dtype=vm_dtype, device="cuda")
    vm_host = torch.empty(n_blocks * n_el, dtype=vm_dtype).pin_memory()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")    # > 129 MB L2

    def step(out):
        sol = ctx.solve(st, blks, W.DT_DEFAULT)
        sol.recover(L.MSTRESS_VM_ELEM, out=out)
        return sol

    for _ in range(args.warmup):
        step(vm_dev).close()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = api.launch_count()
    total_ms = 0.0
    infos = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sol = step(vm_dev)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        infos.append(sol.info())
        sol.close()
    launches = api.launch_count() - l0
    clk = clocks.stop()
    value, slowest = whole_job_rate(dist, world, n_blocks * args.steps, total_ms / 1e3)
    total_ms = 1e3 * slowest

    # end to end: host inputs (site map, dT) in, von Mises to pinned host memory, every step
    e2e_t = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = ctx.solve(st, blks, W.DT_DEFAULT)
        s2.recover(L.MSTRESS_VM_ELEM, out=vm_host)
        e2e_t += time.perf_counter() - t0
        s2.close()
    e2e_value, _ = whole_job_rate(dist, world, n_blocks * args.steps, e2e_t)

    # roofline of the dominant kernel. The PCG runs as one persistent kernel
    # (k_pcg) whose phases are timed on the device (globaltimer at its grid
    # barriers); the recovery kernel is timed with CUDA events on the context
    # stream. Algorithmic work per PCG iteration (N blocks, m = 78, n_vec
    # lattice DOFs, w vector bytes, w_in operand bytes per coefficient):
    #   a3 apply   bytes = C read m N w_in + Y write m N w + vectors 2 n_vec w,
    #              flops = 2 m^2 N per operand product (3 products in bf16x3)
    #   a4 vectors bytes = 10 vector passes of n_vec w
    #   a6 recovery flops = 2 (6 N_el) (m+1) N (Gauss-mean stress modes: 8x
    #              fewer than the 48 N_el Gauss-point rows), VM out N_el N 4 B
    sol = step(vm_dev)
    info = sol.info()
    ph = sol.phase_ms()
    t_rec = api.profile(ctx, sol, 3, 5)
    n_iter = max(1, ph["iterations"])
    m = 78
    n_vec = 3 * (2 * nx + 1) * (2 * ny + 1) * 3          # lattice DOFs of the array (n = 3)
    w = 8 if prec == 0 else 4
    w_in = {0: 8, 1: 4, 2: 2, 3: 4}[prec]
    products = 3 if prec == 3 else 1
    a3_bytes = m * n_blocks * w_in + m * n_blocks * w + 2 * n_vec * w
    a4_bytes = 10 * n_vec * w
    it_bytes = a3_bytes + a4_bytes
    a3_flops = 2.0 * m * m * n_blocks * products
    rec_flops = 2.0 * 6 * n_el * (m + 1) * n_blocks * products
    rec_bytes = n_el * n_blocks * (8 if prec == 0 else 4)
    sm_mhz = clk.get("sm_mhz") or 1900.0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs") or 6800.0
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks.get("hbm_gbs") else "fallback 6800 GB/s"
    bf16 = peaks.get("bf16_tflops") or 1900.0
    # tensor peak of the mode's operand type: bf16 measured; tf32 = bf16 x nominal 1.1 / 2.25
    tensor_peak = {1: bf16 * 1.1 / 2.25, 2: bf16, 3: bf16}.get(prec)
    fp64_peak = 152 * 4 * sm_mhz * 1e6 / 1e12     # 152 SMs x 2 DFMA/clk at the sampled SM clock
    t_apply = ph["apply"] / n_iter
    t_pcg = (ph["apply"] + ph["isum"] + ph["update"]) / n_iter        # ms per iteration
    share = {"pcg": ph["apply"] + ph["isum"] + ph["update"], "recover": t_rec}
    if prec == 0:
        roof = {"bound": "alu", "achieved": a3_flops / (t_apply * 1e-3) / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s", "traffic": None,
                "kernel": "k_pcg<FP64> phase A (element products on the FP64 pipe)",
                "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x sampled SM clock (probe measured 1.257 TFLOP/s)"}
    else:
        tr = PCG_TRAFFIC.get(args.precision)
        roof = {"bound": "hbm", "achieved": it_bytes / (t_pcg * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "traffic": tr,
                "kernel": "k_pcg (persistent PCG: tensor-core apply + interface sum + vector update)",
                "peak_source": hbm_src,
                "note": "vectors are L2-resident at this size, so the iteration is latency-bound (three grid "
                        "barriers and folds per iteration), not HBM-bound; traffic = ncu dram bytes of the "
                        "k_pcg launches of one solve divided by its iterations, bytes per iteration"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["algorithmic_bytes_per_iteration"] = it_bytes
    roof["per_iteration_ms"] = {"apply": t_apply, "isum": ph["isum"] / n_iter, "update": ph["update"] / n_iter}
    roof["a3_apply"] = {"bytes": a3_bytes, "flops": a3_flops, "ms": t_apply,
                        "gbs": a3_bytes / (t_apply * 1e-3) / 1e9, "frac_hbm": a3_bytes / (t_apply * 1e-3) / 1e9 / hbm,
                        "tflops": a3_flops / (t_apply * 1e-3) / 1e12}
    roof["a6_recover"] = {"flops": rec_flops, "ms": t_rec, "tflops": rec_flops / (t_rec * 1e-3) / 1e12,
                          "out_bytes": rec_bytes, "gbs": rec_bytes / (t_rec * 1e-3) / 1e9,
                          "frac_hbm": rec_bytes / (t_rec * 1e-3) / 1e9 / hbm}
    if tensor_peak:
        roof["a3_apply"]["frac_tensor"] = roof["a3_apply"]["tflops"] / tensor_peak
        roof["a6_recover"]["frac_tensor"] = roof["a6_recover"]["tflops"] / tensor_peak
        roof["a6_recover"]["tensor_peak_tflops"] = tensor_peak
    else:
        roof["a6_recover"]["frac_fp64"] = roof["a6_recover"]["tflops"] / fp64_peak
    roof["recover_ms"] = t_rec
    roof["time_share"] = {k: v / sum(share.values()) for k, v in share.items()}
    sol.close()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "blocks/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
                "config": {"workload": f"{nx}x{ny} TSV array, 10x10x50 um blocks, Cu r=2.5 um + 0.5 um SiO2 liner, "
                                       f"12x12x10 Q1 hex mesh, degree-2 face basis (m=78), all sites occupied, "
                                       f"dT=-250 K, bottom clamped; solve + per-element von Mises",
                           "precision": args.precision, "blocks": n_blocks, "pcg_iters": info["iters"],
                           "refinement_steps": info["outer"], "rel_res": info["rel_res"],
                           "l2": "flushed before every timed step (512 MB write)",
                           "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
                "roofline": roof,
                "e2e": {"value": e2e_value, "unit": "blocks/s", "h2d_bytes_per_step": int(st.size + 8),
                        "d2h_bytes_per_step": int(vm_host.numel() * vm_host.element_size())},
                "gpu_launches": int(launches),
                "clocks": clk}
        if cpu_res is not None:
            line["cpu_baseline"] = cpu_baseline_entry(cpu_res)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _variant_models(ctx, W):
    """Both pitch variants (15 and 20 um, 24x24x20 mesh, degree 4) with their dummy blocks."""
    return [[ctx.build_block(v), ctx.build_block(v.dummy())] for v in (W.BLOCK_P15, W.BLOCK_P20)]


def batch_bench(args):
    """256 independent arrays (side log-uniform 4..64, occupancy U[0.5,1],
    pitch 15/20 um, dT U[-300,-150] K) solved and recovered in one batch."""
    import torch

    from paper_2411_12690_gb300 import _lib as L
    from paper_2411_12690_gb300 import api
    from paper_2411_12690_gb300 import workloads as W

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    ctx = api.Context(stream=stream.cuda_stream, precision=PREC[args.precision])
    models = _variant_models(ctx, W)
    jobs = W.batch_arrays(args.n_arrays, seed=0)
    spec = [dict(site_type=j.site_type, blocks=models[j.pitch], dT=j.dT) for j in jobs]
    n_blocks = sum(j.site_type.size for j in jobs)
    n_el = W.BLOCK_P15.ex * W.BLOCK_P15.ey * W.BLOCK_P15.ez
    vm = torch.empty(n_blocks * n_el, dtype=torch.float64 if PREC[args.precision] == 0 else torch.float32,
                     device="cuda")
    times, split = [], []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sol = ctx.solve_batch(spec)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sol.recover(L.MSTRESS_VM_ELEM, out=vm)
        torch.cuda.synchronize()
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
            split.append((t1 - t0, time.perf_counter() - t1))
        infos = [sol.info(a) for a in range(len(jobs))]
        phases = sol.phase_ms()
        sol.close()
    total = sum(times)
    print(json.dumps({"metric": "TSV blocks solved+recovered/s (256-array batch)", "value": n_blocks * len(times) / total,
                      "unit": "blocks/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "dtype": DTYPE[args.precision],
                      "data": "synthetic", "config": {
                          "workload": f"{len(jobs)} arrays, side log-uniform 4..64, occupancy U[0.5,1], pitch 15/20 um "
                                      f"(24x24x20 mesh, degree-4 basis, m=294), dT U[-300,-150] K, one batched solve",
                          "blocks": n_blocks, "max_pcg_iters": max(i["iters"] for i in infos),
                          "max_refinement_steps": max(i["outer"] for i in infos),
                          "max_rel_res": max(i["rel_res"] for i in infos),
                          "solve_ms": 1e3 * sum(a for a, _ in split) / len(split),
                          "recover_ms": 1e3 * sum(b for _, b in split) / len(split),
                          "persistent_phase_ms": phases},
                      "roofline": batch_roofline(args, jobs, n_blocks, n_el, phases,
                                                 1e3 * sum(b for _, b in split) / len(split))}), flush=True)


def batch_roofline(args, jobs, n_blocks, n_el, ph, rec_ms):
    """a3 (element products, per PCG iteration) against the measured HBM peak
    (bytes = C read m N w_in + Y write m N 4 + vectors 2 n_vec 4) and a6 (the
    recovery) against the tensor peak (flops 2 (6 n_el) (m+1) N per operand
    product) and HBM (the von Mises written, N n_el 4 bytes)."""
    m, prec = 294, PREC[args.precision]
    n_vec = sum(3 * (j.site_type.shape[1] * 4 + 1) * (j.site_type.shape[0] * 4 + 1) * 5 for j in jobs)
    w = 8 if prec == 0 else 4
    w_in = {0: 8, 1: 4, 2: 2, 3: 4}[prec]
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs") or 6800.0
    except OSError:
        hbm = 6800.0
    it = max(1, ph["iterations"])
    t_apply = ph["apply"] / it
    a3_bytes = m * n_blocks * w_in + m * n_blocks * w + 2 * n_vec * w
    rec_bytes = n_blocks * n_el * w
    a3 = {"bytes": a3_bytes, "ms": t_apply, "gbs": a3_bytes / (t_apply * 1e-3) / 1e9}
    a3["frac"] = a3["gbs"] / hbm
    a6 = {"bytes": rec_bytes, "ms": rec_ms, "gbs": rec_bytes / (rec_ms * 1e-3) / 1e9}
    a6["frac_hbm"] = a6["gbs"] / hbm
    # flops of the Gauss-mean contraction (x3 operand products in bf16x3)
    a6["flops"] = 2.0 * 6 * n_el * (m + 1) * n_blocks * (3 if prec == 3 else 1)
    a6["tflops"] = a6["flops"] / (rec_ms * 1e-3) / 1e12
    try:
        bf16 = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("bf16_tflops") or 1900.0
    except OSError:
        bf16 = 1900.0
    tensor_peak = {1: bf16 * 1.1 / 2.25, 2: bf16, 3: bf16}.get(prec)
    if tensor_peak:
        a6["frac_tensor"] = a6["tflops"] / tensor_peak
    return {"bound": "hbm", "achieved": a3["gbs"], "peak": hbm, "unit": "GB/s", "frac": a3["frac"],
            "traffic": None, "kernel": "k_pcg phase A (streamed tensor-core element products, per iteration)",
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)", "a3_apply": a3, "a6_recover": a6,
            "lattice_dofs": n_vec}


def serve_bench(args):
    """Poisson request stream through the continuous-batching server: arrays
    log-uniform 2..128, occupancy U[0.5,1], pitch 15/20 um, dT U[-300,-150] K;
    arrival rate = load x the capacity measured by a closed-loop pass."""
    import torch

    from paper_2411_12690_gb300 import api
    from paper_2411_12690_gb300 import workloads as W

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    ctx = api.Context(stream=stream.cuda_stream, precision=PREC[args.precision])
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
    probe = W.request_stream(1.0, max(16, args.requests // 4), seed=2)
    cap_blocks, _, cap_t = run([W.Request(0.0, r.job) for r in probe], 0.0)  # closed loop: capacity
    cap_rps = len(probe) / cap_t
    reqs = W.request_stream(args.load * cap_rps, args.requests, seed=0)
    thr, lat, elapsed = run(reqs, 1.0)
    lat = sorted(lat)
    print(json.dumps({"metric": "served TSV blocks/s with p50/p99 request latency", "value": thr, "unit": "blocks/s",
                      "n_gpus": 1, "higher_is_better": True, "dtype": DTYPE[args.precision], "data": "synthetic",
                      "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                      "requests": len(lat), "elapsed_s": elapsed,
                      "config": {"workload": "Poisson stream, arrays log-uniform 2..128, occupancy U[0.5,1], pitch "
                                             "15/20 um (m=294), dT U[-300,-150] K, max 64 slots",
                                 "arrival_rate_per_s": args.load * cap_rps, "load": args.load,
                                 "closed_loop_capacity_blocks_per_s": cap_blocks}}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "batch256":
        batch_bench(args)
    elif args.workload == "serve":
        serve_bench(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
