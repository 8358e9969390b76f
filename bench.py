"""Benchmark: DOFs/s of PHIF factorization + PCG to relres 1e-10 on one GB300.

Workload (one step = the whole hot path over one problem): the 2D 5-point
finite-difference problem on a 1023 x 1023 interior grid (N = 1,046,529),
per-pixel coefficient log10 a ~ U[-4, 4] (seeded), b = 0, f ~ N(0,1), leaf
16, ID tolerance 1e-3; assembly of A from the per-pixel field, the PHIF
factorization and PCG to a relative residual of 1e-10, all on the GPU.
The headline `value` uses the FP32 factor (FP64 PCG); the plain-FP64 factor
is measured beside it under "fp64".

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs its own independent replica (the path does not
shard); `value` sums the DOFs of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOFs/s factor+PCG to relres 1e-10, mixed vs plain FP64 on GPU; % roofline"
WORKLOAD = "2d-fd5-1023sq-logunif1e-4..1e4-leaf16-tol1e-3"
RTOL = 1e-10
CPU_SAMPLE_SIDE = 511       # bounded oracle sample for cpu_baseline (same recipe, smaller grid)
REF_STEP_SIDE = 255         # bounded oracle sample per step of --impl reference


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--fp64-steps", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--side", type=int, default=1023)
    return p.parse_args()


# ---------------------------------------------------------------------------
# the oracle on host cores (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

_ORACLE_SNIPPET = r"""
import sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import fd, phif
side = {side}
p = W.make_problem((side, side), 1e-4, 1e4, 0.0, 16, 1e-3, W.SEED_BASE + 1)
t0 = time.perf_counter()
A = fd.assemble(p.ns, p.a, p.b)
F = phif.factor(A, p.ns, p.leaf, p.tol)
u, it, rr = phif.pcg(A, p.f, M=lambda r: phif.solve(F, r), rtol={rtol})
t = time.perf_counter() - t0
print(json.dumps({{"seconds": t, "n": p.n, "iters": it, "relres": rr}}))
"""


def run_oracle(side: int) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = _ORACLE_SNIPPET.format(root=ROOT, side=side, rtol=RTOL)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        run_oracle(REF_STEP_SIDE)
    secs, n = [], 0
    for _ in range(args.steps):
        r = run_oracle(REF_STEP_SIDE)
        secs.append(r["seconds"])
        n = r["n"]
    tot = sum(secs)
    val = n * len(secs) / tot
    sample = (f"FP64 numpy/scipy oracle, {REF_STEP_SIDE}^2 grid of the same recipe per step "
              f"(N={n}), factor+PCG to relres {RTOL}, 1 thread")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "DOFs/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * tot / len(secs), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample_side": REF_STEP_SIDE},
           "cpu_baseline": {"value": val, "unit": "DOFs/s", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": "DOFs/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"rhif_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def alu_peaks(torch):
    """FP32 and FP64 throughput of cuBLAS GEMM on this GPU (no TF32), TFLOP/s."""
    out = {}
    torch.backends.cuda.matmul.allow_tf32 = False
    for name, dt, n in (("fp64", torch.float64, 4096), ("fp32", torch.float32, 8192)):
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        for _ in range(2):
            torch.matmul(a, b)
        torch.cuda.synchronize()
        best = 1e9
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[name] = 2.0 * n ** 3 / best / 1e12
        del a, b
    torch.cuda.empty_cache()
    return out


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1808_01364_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(kernel: str, precision: str):
    """Per-launch DRAM traffic recorded by an ncu capture, if the kernel sources
    are unchanged since; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = source_hash()
    for line in open(path):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel and f[1] == precision:
            return float(f[2]) if f[3] == want else None
    return None


def gpu_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1808_01364_gb300 as rhif
    import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    rhif.load()

    side = args.side
    ns = (side, side)
    seed = W.SEED_BASE + 1
    p = W.make_problem(ns, 1e-4, 1e4, 0.0, 16, 1e-3, seed)
    N = p.n
    dev = torch.device("cuda", local)
    a_d = torch.as_tensor(p.a, device=dev)
    f_d = torch.as_tensor(p.f, device=dev)
    nnz = rhif.rhif_fd_nnz(ns)
    stream = torch.cuda.current_stream()

    def step(precision):
        csr = rhif.rhif_assemble_fd(ns, a_d, 0.0)
        F = rhif.rhif_factor(csr, ns, p.leaf, p.tol, precision=precision)
        u, its, rr = F.pcg(f_d, rtol=RTOL, maxit=500)
        F.free()
        return u, its, rr

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(precision, steps, warmup, timing=False):
        for _ in range(warmup):
            step(precision)
        barrier()
        rhif.rhif_reset_kernel_stats()
        rhif.rhif_set_timing(timing)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = None
        for _ in range(steps):
            info = step(precision)
        e1.record(stream)
        barrier()
        rhif.rhif_set_timing(False)
        ks = rhif.rhif_kernel_stats()
        sec = e0.elapsed_time(e1) / 1e3
        if world > 1:
            t = torch.tensor([sec], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            sec = float(t.item())
        return sec, info, ks

    clocks = ClockSampler(local)
    # headline: FP32 factor, FP64 PCG, no instrumentation in the timed region
    clocks.start()
    sec, (u, its, rr), ks_count = timed("fp32", args.steps, args.warmup, timing=False)
    clk = clocks.stop()
    value = world * N * args.steps / sec
    gpu_launches = int(sum(v["launches"] for v in ks_count.values()))
    # the same steps again with CUDA events around every library launch (per-kernel durations)
    _, _, ks = timed("fp32", args.steps, 0, timing=True)
    # plain FP64 factor
    sec64, (u64, its64, rr64), ks64 = timed("fp64", args.fp64_steps, 1, timing=False)
    value64 = world * N * args.fp64_steps / sec64
    du = float(torch.linalg.norm(u - u64) / torch.linalg.norm(u64))

    # end to end through the C-ABI with host buffers (pinned), copies inside the timed region
    a_h = torch.as_tensor(p.a).pin_memory()
    f_h = torch.as_tensor(p.f).pin_memory()
    u_h = torch.empty(N, dtype=torch.float64).pin_memory()

    def e2e_step():
        a_dev = a_h.to(dev, non_blocking=True)
        f_dev = f_h.to(dev, non_blocking=True)
        csr = rhif.rhif_assemble_fd(ns, a_dev, 0.0)
        F = rhif.rhif_factor(csr, ns, p.leaf, p.tol, precision="fp32")
        uu, _, _ = F.pcg(f_dev, rtol=RTOL, maxit=500)
        u_h.copy_(uu, non_blocking=True)
        F.free()

    for _ in range(args.warmup):
        e2e_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    barrier()
    sec_e2e = e0.elapsed_time(e1) / 1e3
    if world > 1:
        t = torch.tensor([sec_e2e], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        sec_e2e = float(t.item())
    e2e_val = world * N * args.steps / sec_e2e

    # roofline of the dominant kernel of the headline path
    peaks = alu_peaks(torch)
    hbm, hbm_kind = measured_peaks()
    top = max(ks.items(), key=lambda kv: kv[1]["total_ms"])
    name, st = top
    per_launch_ms = st["total_ms"] / max(st["launches"], 1)
    if name.startswith("apply") or name in ("spmv", "pcg_vector", "extend_add", "expand_gids"):
        achieved = st["bytes"] / max(st["launches"], 1) / (per_launch_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "peak_kind": hbm_kind}
    else:
        achieved = st["flops"] / max(st["launches"], 1) / (per_launch_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peaks["fp32"], "unit": "TFLOP/s",
                "peak_kind": "measured cuBLAS SGEMM (no TF32) on this GPU"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = name
    roof["launch_ms"] = per_launch_ms
    roof["traffic"] = profile_traffic(name, "fp32")

    result = {
        "metric": METRIC, "value": value, "unit": "DOFs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 factor + f64 PCG", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "leaf": p.leaf, "tol": p.tol, "rtol": RTOL,
                   "parallelism": f"replicas{world}",
                   "l2": "working set (fronts >1 GB) larger than L2; no flush"},
        "pcg_iters": its[0], "relres": rr[0],
        "fp64": {"value": value64, "ms_per_step": 1e3 * sec64 / args.fp64_steps,
                 "pcg_iters": its64[0], "relres": rr64[0], "rel_diff_u_vs_fp32_path": du},
        "mixed_over_fp64": value / value64,
        "roofline": roof,
        "alu_peaks_tflops": peaks,
        "kernels": {k: {"launches": v["launches"], "ms": round(v["total_ms"], 3)}
                    for k, v in ks.items() if v["launches"]},
        "gpu_launches": gpu_launches,
        "clocks": clk,
        "e2e": {"value": e2e_val, "unit": "DOFs/s",
                "h2d_bytes_per_step": int(a_h.numel() * 8 + f_h.numel() * 8),
                "d2h_bytes_per_step": int(u_h.numel() * 8)},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = run_oracle(CPU_SAMPLE_SIDE)
        result["cpu_baseline"] = {
            "value": r["n"] / r["seconds"], "unit": "DOFs/s", "cores": 1, "kind": "oracle",
            "sample": (f"FP64 oracle factor+PCG on a {CPU_SAMPLE_SIDE}^2 grid of the same recipe "
                       f"(N={r['n']}, {r['seconds']:.1f} s, {r['iters']} PCG its), 1 thread")}
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = _args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
