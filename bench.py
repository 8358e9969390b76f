"""Benchmark: DOFs/s of PHIF factorization + PCG to relres 1e-10 on one GB300.

Default workload (one step = the whole hot path over one problem): the 2D
5-point finite-difference problem on a 1023 x 1023 interior grid
(N = 1,046,529), per-pixel coefficient log10 a ~ U[-4, 4] (seeded), b = 0,
f ~ N(0,1), leaf 16, ID tolerance 1e-3; assembly of A from the per-pixel
field, the PHIF factorization and PCG to a relative residual of 1e-10, all on
the GPU.  The headline `value` uses the FP32 factor (FP64 PCG); the plain-FP64
factor is measured beside it under "fp64".

--workload selects the other synthetic workloads (same JSON line):
  c1  2D 127^2, log10 a ~ U[-2,2], leaf 8, tol 1e-3, FP64 factor, PCG to 1e-12
  c2  the default above
  c3  3D 7-point 63^3, log10 a ~ U[-3,3], b = 1e-2, leaf 8, faces + edges
      skeletonized, tol 1e-3, FP32 factor
  c4  64 independent 2D problems (sides uniform in 127..511, log10 a ~ U[-3,3],
      leaf 8, tol 1e-3) with 32 right-hand sides each, FP32 factors, one merged
      factorization (one launch per level step for all problems) and PCG of
      every (problem, rhs) pair with the same launches; DOFs count each
      problem once
  c5  differentiable solve on 511^2: log a from a smooth seeded field, forward
      PHIF solve, loss 0.5 ||u - u_obs||^2, backward (adjoint PCG with the same
      factor + gradient kernel); leaf 16, tol 1e-6, FP32 factor, PCG to 1e-12

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload c1|c2|c3|c4|c5] [--tol T]
       python bench.py --paper-tables | --skeleton-growth   (studies, one JSON line)
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
RTOL = 1e-10

WORKLOADS = {
    "c1": "2d-fd5-127sq-logunif1e-2..1e2-leaf8-tol1e-3-fp64-rtol1e-12",
    "c2": "2d-fd5-1023sq-logunif1e-4..1e4-leaf16-tol1e-3",
    "c3": "3d-fd7-63cube-logunif1e-3..1e3-b1e-2-leaf8-tol1e-3-faces+edges",
    "c4": "batched-64x2d-fd5-sides127..511-logunif1e-3..1e3-leaf8-tol1e-3-32rhs",
    "c5": "grad-2d-fd5-511sq-smooth-log-a-leaf16-tol1e-6-adjoint-rtol1e-12",
}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="timed steps (default: about half a second of GPU work per workload; "
                        "5 for --impl reference)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    p.add_argument("--fp64-steps", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--tol", type=float, default=None,
                   help="ID tolerance of the single-problem workloads (default: the workload's)")
    p.add_argument("--tc-kernel", action="store_true",
                   help="throughput of the tensor-core tile product per operand kind (4096 x 4096 x 1024)")
    p.add_argument("--skeleton-growth", action="store_true",
                   help="3D root-size study with and without edge skeletonization (Remark 3.1)")
    p.add_argument("--paper-tables", action="store_true",
                   help="HIF vs PHIF study on the paper's quantized field (Sec. 4 tables)")
    return p.parse_args()


# ---------------------------------------------------------------------------
# the oracle on host cores (cpu_baseline and --impl reference): a bounded
# sample of each workload, the same recipe at a smaller size
# ---------------------------------------------------------------------------

_ORACLE_HEAD = r"""
import sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import fd, phif
"""

_ORACLE_BODY = {
    "2d": r"""
p = W.make_problem(({side}, {side}), {lo}, {hi}, 0.0, {leaf}, 1e-3, {seed})
t0 = time.perf_counter()
A = fd.assemble(p.ns, p.a, p.b)
F = phif.factor(A, p.ns, p.leaf, p.tol)
u, it, rr = phif.pcg(A, p.f, M=lambda r: phif.solve(F, r), rtol={rtol})
t = time.perf_counter() - t0
if {save!r}:
    try:
        np.save({save!r}, u)
    except OSError:
        pass
print(json.dumps({{"seconds": t, "dofs": p.n, "iters": it}}))
""",
    "3d": r"""
p = W.make_problem(({side}, {side}, {side}), 1e-3, 1e3, 1e-2, 8, 1e-3, {seed})
t0 = time.perf_counter()
A = fd.assemble(p.ns, p.a, p.b)
F = phif.factor(A, p.ns, p.leaf, p.tol, edge_skel=True)
u, it, rr = phif.pcg(A, p.f, M=lambda r: phif.solve(F, r), rtol={rtol})
t = time.perf_counter() - t0
print(json.dumps({{"seconds": t, "dofs": p.n, "iters": it}}))
""",
    "batch": r"""
p = W.batched_problems(1, 32, sides=[{side}])[0]
t0 = time.perf_counter()
A = fd.assemble(p.ns, p.a, p.b)
F = phif.factor(A, p.ns, p.leaf, p.tol)
its = []
for r in range(p.f.shape[0]):
    u, it, rr = phif.pcg(A, p.f[r], M=lambda x: phif.solve(F, x), rtol={rtol})
    its.append(it)
t = time.perf_counter() - t0
print(json.dumps({{"seconds": t, "dofs": p.n, "iters": max(its)}}))
""",
    "grad": r"""
import scipy.sparse.linalg as spla
ns = ({side}, {side})
log_star, f = W.inverse_problem(ns)
u_obs = spla.spsolve(fd.assemble(ns, np.exp(log_star), 0.0).tocsc(), f)
log_a = 0.3 * W.gaussian_bump_log_field(ns, {seed})
t0 = time.perf_counter()
a = np.exp(log_a)
A = fd.assemble(ns, a, 0.0)
F = phif.factor(A, ns, 16, 1e-6)
u, it, rr = phif.pcg(A, f, M=lambda r: phif.solve(F, r), rtol={rtol})
lam, it2, rr2 = phif.pcg(A, u - u_obs, M=lambda r: phif.solve(F, r), rtol={rtol})
g = fd.dA_dlog_a(ns, a, u, lam)
t = time.perf_counter() - t0
print(json.dumps({{"seconds": t, "dofs": int(np.prod(ns)), "iters": max(it, it2)}}))
""",
}

# (body, side, format fields, description) of the bounded cpu_baseline sample
_SAMPLES = {
    "c1": ("2d", 127, dict(lo=1e-2, hi=1e2, leaf=8, rtol=1e-12), "the full 127^2 workload"),
    "c2": ("2d", 511, dict(lo=1e-4, hi=1e4, leaf=16, rtol=RTOL), "a 511^2 grid of the same recipe"),
    "c3": ("3d", 31, dict(rtol=RTOL), "a 31^3 grid of the same recipe"),
    "c4": ("batch", 127, dict(rtol=RTOL), "one 127^2 problem of the batch recipe, all 32 RHS"),
    "c5": ("grad", 255, dict(rtol=1e-12), "the forward+adjoint+gradient step on 255^2"),
}
_REF_SIDE = {"c1": 127, "c2": 255, "c3": 23, "c4": 127, "c5": 127}


def oracle_seed(workload: str) -> int:
    """Seed of the oracle's sample: the 127^2 sample is the c1 workload itself."""
    return 180800 + (0 if workload == "c1" else 1)


def run_oracle(workload: str, side: int, save: str = "") -> dict:
    """Times the oracle on a sample of the workload in a one-thread
    subprocess; with `save`, the 2D samples also write their PCG solution
    there (.npy, outside the timed part)."""
    body, _, extra, _ = _SAMPLES[workload]
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    fields = dict(side=side, seed=oracle_seed(workload), rtol=extra.get("rtol", RTOL),
                  lo=extra.get("lo", 1e-4), hi=extra.get("hi", 1e4), leaf=extra.get("leaf", 16),
                  save=save)
    code = _ORACLE_HEAD.format(root=ROOT) + _ORACLE_BODY[body].format(**fields)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    side = _REF_SIDE[args.workload]
    for _ in range(args.warmup):
        run_oracle(args.workload, side)
    secs, n, its = [], 0, 0
    for _ in range(args.steps):
        r = run_oracle(args.workload, side)
        secs.append(r["seconds"])
        n, its = r["dofs"], r["iters"]
    tot = sum(secs)
    val = n * len(secs) / tot
    sample = (f"FP64 numpy/scipy oracle, side {side} of the {args.workload} recipe per step "
              f"(DOFs={n}, {its} PCG its), 1 thread")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "DOFs/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * tot / len(secs), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "sample_side": side},
           "cpu_baseline": {"value": val, "unit": "DOFs/s", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": "DOFs/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# replicas: the path does not shard, so N ranks run N independent problems
# ---------------------------------------------------------------------------

def max_over_ranks(sec: float, device=None) -> float:
    """The job's time is its slowest replica's: all-reduce MAX over the ranks
    of the initialized process group (NCCL between GPUs, gloo in the CPU
    tests); the local time when there is no group or one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return sec
    t = torch.tensor([sec], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: float, steps: int, sec_max: float, world: int) -> float:
    """Units processed by all ranks over the slowest rank's time."""
    return world * units_per_rank * steps / sec_max


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

_CLOCK_REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def _smi_time(text: str):
    """Seconds since the epoch of an nvidia-smi timestamp (local time), or None."""
    import datetime
    for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
        try:
            return datetime.datetime.strptime(text.strip(), fmt).timestamp()
        except ValueError:
            pass
    return None


def parse_clock_samples(lines, t0=None, t1=None) -> dict:
    """Clock record of the timed region from nvidia-smi CSV lines (fields:
    timestamp, index, clocks.sm, clocks.max.sm, power.draw, reasons bitmask,
    then the four reasons of _CLOCK_REASONS as Active / Not Active).

    With the region's host times t0..t1, the samples taken inside it are used;
    when the region is shorter than the sampling period, the last sample
    before it and the first after it stand for it.  Without times (or with
    unreadable timestamps) every sample is used."""
    rows = []
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 10:
            continue
        try:
            sm, mx = float(f[2]), float(f[3])
        except ValueError:
            continue
        active = {nm for nm, v in zip(_CLOCK_REASONS, f[6:10]) if v.lower().startswith("active")}
        rows.append((_smi_time(f[0]), sm, mx, active))
    use, where = rows, "all samples"
    if t0 is not None and t1 is not None and rows and all(r[0] is not None for r in rows):
        inside = [r for r in rows if t0 <= r[0] <= t1]
        if inside:
            use, where = inside, "inside the timed region"
        else:
            before = [r for r in rows if r[0] < t0]
            after = [r for r in rows if r[0] > t1]
            use = before[-1:] + after[:1]
            where = "adjacent to the timed region (shorter than the sampling period)"
    if not use:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
    reasons = set().union(*(r[3] for r in use))
    return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": use[-1][2],
            "reasons": sorted(reasons), "samples": len(use), "sampled": where}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons around the timed region."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"rhif_clocks_rank{index}.csv")

    def start(self):
        """Starts the sampler and waits (up to 1 s) for its first sample, so that
        it is running when the timed region begins."""
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t = time.time()
        while time.time() - t < 1.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self, t0=None, t1=None) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            return parse_clock_samples(fh.readlines(), t0, t1)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def hbm_bound(kernel: str) -> bool:
    """Kernel categories bounded by memory traffic (the F^-1 sweeps, SpMV,
    vector updates, assembly, extend-add); the others count flops."""
    return kernel.startswith("apply") or kernel in (
        "spmv", "pcg_vector", "extend_add", "expand_gids", "assemble_fd", "stencil_from_csr",
        "band_inverse")


def alu_peak_nominal(precision: str, torch=None, sm_max_mhz=None):
    """Plain-ALU peak from the unit counts and clock (TFLOP/s): FP32 = SMs (read
    from the device) x 128 FMA lanes x 2 flops x the maximum SM clock (sampled
    by nvidia-smi during the run, else 2070 MHz); FP64 = GB300's nominal 1.25
    TFLOP/s.  The cuBLAS GEMM rates measured live are reported beside it."""
    if precision == "fp32":
        sms = torch.cuda.get_device_properties(0).multi_processor_count if torch is not None else 152
        mhz = float(sm_max_mhz) if sm_max_mhz else 2070.0
        return (sms * 128 * 2 * mhz * 1e6 / 1e12,
                f"derived: {sms} SMs (device) x 128 FP32 lanes x 2 flops x {mhz:.0f} MHz (max SM clock)")
    return 1.25, "nominal GB300 FP64 rate"


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


# device code of each kernel category: its .cu file plus the shared headers
_APPLY_CATS = ("apply_cell_up", "apply_cell_down", "apply_group_up", "apply_group_down",
               "apply_leaf_up", "apply_leaf_down", "spmv", "pcg_vector", "assemble_fd", "grad_logcoef")
_SHARED_SRC = ("common.cuh", "tables.h")


def source_files(kernel: str):
    main = "apply_kernels.cu" if kernel in _APPLY_CATS else "factor_kernels.cu"
    return (main,) + _SHARED_SRC


def source_hash(kernel: str) -> str:
    """Hash of the sources that hold the device code of a kernel category, so
    that a recorded DRAM traffic figure is used only while that code is
    unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1808_01364_gb300", "csrc")
    for fn in source_files(kernel):
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(kernel: str, precision: str, workload: str):
    """Per-launch DRAM traffic recorded by an ncu capture of this workload, if
    the kernel sources are unchanged since; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = source_hash(kernel)
    for line in open(path):
        f = line.split()
        if line.startswith("#") or len(f) < 4 or f[0] != kernel or f[1] != precision:
            continue
        if (f[4] if len(f) >= 5 else "c2") == workload:
            return float(f[2]) if f[3] == want else None
    return None


class Workload:
    """One step of the hot path with inputs resident on the device (`step`),
    and end to end from pinned host buffers (`e2e_step`)."""

    def __init__(self, key, rhif, W, torch, dev, tol=None):
        self.key, self.rhif, self.W, self.torch, self.dev = key, rhif, W, torch, dev
        self.headline = "fp64" if key == "c1" else "fp32"
        self.rtol = 1e-12 if key in ("c1", "c5") else RTOL
        t = torch
        if key in ("c1", "c2", "c3"):
            p = W.config_problem({"c1": 0, "c2": 1, "c3": 2}[key])
            if tol is not None:
                p.tol = float(tol)
            self.p = p
            self.dofs = p.n
            self.edge = key == "c3"
            self.a_d = t.as_tensor(p.a, device=dev)
            self.f_d = t.as_tensor(p.f, device=dev)
            self.a_h = t.as_tensor(p.a).pin_memory()
            self.f_h = t.as_tensor(p.f).pin_memory()
            self.u_h = t.empty(p.n, dtype=t.float64).pin_memory()
            self.h2d = (p.a.size + p.f.size) * 8
            self.d2h = p.n * 8
        elif key == "c4":
            self.ps = W.batched_problems(64, 32)
            self.dofs = sum(q.n for q in self.ps)
            self.a_d = [t.as_tensor(q.a, device=dev) for q in self.ps]
            self.f_d = [t.as_tensor(q.f, device=dev) for q in self.ps]
            self.a_h = [t.as_tensor(q.a).pin_memory() for q in self.ps]
            self.f_h = [t.as_tensor(q.f).pin_memory() for q in self.ps]
            self.u_h = [t.empty(q.f.shape, dtype=t.float64).pin_memory() for q in self.ps]
            self.h2d = sum((q.a.size + q.f.size) * 8 for q in self.ps)
            self.d2h = sum(q.f.size * 8 for q in self.ps)
        else:   # c5
            self.ns = (511, 511)
            log_star, f = W.inverse_problem(self.ns)
            log_a = 0.3 * W.gaussian_bump_log_field(self.ns, W.SEED_BASE + 1)
            self.dofs = int(f.size)
            self.la_d = t.as_tensor(log_a, device=dev)
            self.f_d = t.as_tensor(f, device=dev)
            # observations of the true field: an FP64 solve on the device (setup only)
            csr, _ = rhif.rhif_assemble_fd_log(self.ns, t.as_tensor(log_star, device=dev))
            F = rhif.rhif_factor(csr, self.ns, 16, 1e-6, precision="fp64")
            self.uo_d, _, _ = F.pcg(self.f_d, rtol=1e-13, maxit=1000)
            F.free()
            self.la_h = t.as_tensor(log_a).pin_memory()
            self.f_h = t.as_tensor(f).pin_memory()
            self.uo_h = self.uo_d.cpu().pin_memory()
            self.g_h = t.empty(log_a.shape, dtype=t.float64).pin_memory()
            self.h2d = (log_a.size + 2 * f.size) * 8
            self.d2h = log_a.size * 8

    def _solve_one(self, a, f, precision, precond=True):
        r, p = self.rhif, self.p
        csr = r.rhif_assemble_fd(p.ns, a, p.b)
        F = r.rhif_factor(csr, p.ns, p.leaf, p.tol, precision=precision, edge_skel_3d=self.edge,
                          precondition=precond)
        u, its, rr = F.pcg(f, rtol=self.rtol, maxit=1000)
        F.free()
        return u, its, rr

    def _batch(self, a_list, f_list, precision):
        # one merged factorization of all problems (one launch per level step)
        # and PCG of every (problem, rhs) pair with the same launches
        r = self.rhif
        csrs = [r.rhif_assemble_fd(q.ns, a, q.b) for q, a in zip(self.ps, a_list)]
        FB = r.rhif_factor_batch(csrs, [q.ns for q in self.ps], 8, 1e-3, precision=precision)
        us, its, rr = FB.pcg_batch(f_list, rtol=self.rtol)
        FB.free()
        return us, [max(i) for i in its], [max(x) for x in rr]

    def _grad(self, la, f, uo, precision):
        t, r = self.torch, self.rhif
        la = la.detach().requires_grad_(True)
        u = r.rhif_solve(la, f, self.ns, leaf=16, tol=1e-6, precision=precision, rtol=self.rtol)
        loss = 0.5 * t.sum((u - uo) ** 2)
        loss.backward()
        return la.grad, [0], [float(loss.detach())]

    def step(self, precision):
        if self.key == "c4":
            return self._batch(self.a_d, self.f_d, precision)
        if self.key == "c5":
            return self._grad(self.la_d, self.f_d, self.uo_d, precision)
        return self._solve_one(self.a_d, self.f_d, precision)

    def e2e_step(self):
        dev = self.dev
        if self.key == "c4":
            a = [x.to(dev, non_blocking=True) for x in self.a_h]
            f = [x.to(dev, non_blocking=True) for x in self.f_h]
            us, _, _ = self._batch(a, f, self.headline)
            for h, u in zip(self.u_h, us):
                h.copy_(u, non_blocking=True)
            return
        if self.key == "c5":
            la = self.la_h.to(dev, non_blocking=True)
            f = self.f_h.to(dev, non_blocking=True)
            uo = self.uo_h.to(dev, non_blocking=True)
            g, _, _ = self._grad(la, f, uo, self.headline)
            self.g_h.copy_(g, non_blocking=True)
            return
        a = self.a_h.to(dev, non_blocking=True)
        f = self.f_h.to(dev, non_blocking=True)
        u, _, _ = self._solve_one(a, f, self.headline)
        self.u_h.copy_(u, non_blocking=True)

    def config(self):
        name = WORKLOADS[self.key]
        if self.key in ("c1", "c2", "c3") and self.p.tol != 1e-3:
            name = name.replace("tol1e-3", f"tol{self.p.tol:g}")
        c = {"workload": name, "dofs_per_step": self.dofs, "rtol": self.rtol}
        if self.key in ("c1", "c2", "c3"):
            c.update(N=self.p.n, leaf=self.p.leaf, tol=self.p.tol)
        elif self.key == "c4":
            c.update(problems=len(self.ps), rhs_per_problem=32, leaf=8, tol=1e-3,
                     batching="merged levels: one launch per level step for all problems")
        else:
            c.update(N=self.dofs, leaf=16, tol=1e-6, step="forward PCG + adjoint PCG + gradient")
        return c


def local_precond_compare(wl, timed) -> dict:
    """The headline step with each local preconditioner of the separator
    groups (none = HIF, diagonal, block Jacobi = PHIF) and factor precision,
    outside the headline's timed region: DOFs/s and PCG iterations.  A factor
    that breaks down (not SPD, as HIF does on high-contrast fields, Sec. 4) is
    reported, not raised."""
    out = {}
    for prec in ("fp32", "fp64"):
        for mode in ("none", "diag", "block"):
            key = f"{mode}_{prec}"
            try:
                sec, (u, its, rr), _ = timed(lambda: wl._solve_one(wl.a_d, wl.f_d, prec, mode), 3, 1)
                out[key] = {"value": wl.dofs * 3 / sec, "ms_per_step": 1e3 * sec / 3,
                            "pcg_iters": its[0], "relres": rr[0]}
            except Exception as e:   # noqa: BLE001 - reported in the line
                out[key] = {"error": str(e).split(":")[0] + ": " + str(e).split(":")[-1][:120]}
    return out


def tensor_core_kinds(wl, timed, torch) -> dict:
    """The headline step with each operand kind of the tensor-core Schur tiles
    (TF32 split = FP32-accurate, one TF32 product, BF16) and with the FP64
    factor, outside the headline's timed region: DOFs/s, PCG iterations, the
    apply error ||F^{-1} A x - x|| / ||x|| on a seeded x, and the solution's
    difference from the FP64 factor's.  Errors are reported, not raised."""
    out = {}
    p, r = wl.p, wl.rhif
    x = torch.as_tensor(wl.W.normal_rhs(p.ns, 4242), device=wl.dev)
    u_ref = None
    for prec in ("fp64", "fp32", "tf32", "bf16"):
        try:
            sec, (u, its, rr), _ = timed(lambda: wl._solve_one(wl.a_d, wl.f_d, prec), 2, 1)
            csr = r.rhif_assemble_fd(p.ns, wl.a_d, p.b)
            F = r.rhif_factor(csr, p.ns, p.leaf, p.tol, precision=prec, edge_skel_3d=wl.edge)
            ea = float(torch.linalg.norm(F.apply(F.spmv(x)) - x) / torch.linalg.norm(x))
            F.free()
            if prec == "fp64":
                u_ref = u
            out[prec] = {"value": wl.dofs * 2 / sec, "ms_per_step": 1e3 * sec / 2,
                         "pcg_iters": its[0], "relres": rr[0], "apply_error": ea,
                         "rel_diff_u_vs_fp64": float(torch.linalg.norm(u - u_ref) /
                                                     torch.linalg.norm(u_ref))}
        except Exception as e:   # noqa: BLE001 - reported in the line
            out[prec] = {"error": str(e)[:200]}
    return out


def step_breakdown(wl, torch) -> dict:
    """Device time of each part of one headline step of a single-problem
    workload (assembly, factorization, one application of F^{-1}, PCG),
    with CUDA events on the current stream, outside every timed region.
    An error is reported in the result instead of ending the run."""
    try:
        r, p = wl.rhif, wl.p
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        torch.cuda.synchronize()
        ev[0].record()
        csr = r.rhif_assemble_fd(p.ns, wl.a_d, p.b)
        ev[1].record()
        F = r.rhif_factor(csr, p.ns, p.leaf, p.tol, precision=wl.headline, edge_skel_3d=wl.edge)
        ev[2].record()
        F.apply(wl.f_d)
        ev[3].record()
        _, its, _ = F.pcg(wl.f_d, rtol=wl.rtol, maxit=1000)
        ev[4].record()
        torch.cuda.synchronize()
        F.free()
        names = ("assemble_ms", "factor_ms", "apply_ms", "pcg_ms")
        out = {n: ev[i].elapsed_time(ev[i + 1]) for i, n in enumerate(names)}
        out["pcg_iters"] = int(its[0])
        return out
    except Exception as e:   # reported, not fatal: the headline line stands
        return {"error": str(e)[:300]}


def compare_with_oracle(rhif, W, torch, dev, workload, side, extra, path, oracle_iters, rtol):
    """The GPU path (both factor precisions, PCG to the workload's rtol) on
    the oracle's 2D sample: relative 2-norm difference of the PCG solutions
    and the iteration counts.  Outside every timed region; an error is
    reported in the result instead of ending the run."""
    import numpy as np
    out = {"sample": f"{side}^2 grid of the {workload} recipe (the cpu_baseline problem)"}
    try:
        u_o = np.load(path)
        p = W.make_problem((side, side), extra.get("lo", 1e-4), extra.get("hi", 1e4), 0.0,
                           extra.get("leaf", 16), 1e-3, oracle_seed(workload))
        a = torch.as_tensor(p.a, device=dev)
        f = torch.as_tensor(p.f, device=dev)
        uo = torch.as_tensor(u_o, device=dev)
        diff, its = {}, {"oracle": oracle_iters}
        for prec in ("fp32", "fp64"):
            csr = rhif.rhif_assemble_fd(p.ns, a, 0.0)
            F = rhif.rhif_factor(csr, p.ns, p.leaf, p.tol, precision=prec)
            u, it, _ = F.pcg(f, rtol=rtol, maxit=1000)
            F.free()
            diff[prec] = float(torch.linalg.norm(u - uo) / torch.linalg.norm(uo))
            its[prec] = int(it[0])
        out.update(rel_diff_u=diff, pcg_iters=its, rtol=rtol)
    except Exception as e:   # reported, not fatal: the headline line stands
        out["error"] = str(e)[:300]
    finally:
        try:
            os.remove(path)
        except OSError:
            pass
    return out


def gpu_arm(args):
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
    dev = torch.device("cuda", local)
    wl = Workload(args.workload, rhif, W, torch, dev, args.tol)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def reduce_max(sec):
        return max_over_ranks(sec, dev)

    region = {}   # host times bracketing the last timed region (for the clock record)

    def timed(fn, steps, warmup, timing=False):
        for _ in range(warmup):
            fn()
        barrier()
        rhif.rhif_reset_kernel_stats()
        rhif.rhif_set_timing(timing)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        region["t0"] = time.time()
        e0.record(stream)
        info = None
        for _ in range(steps):
            info = fn()
        e1.record(stream)
        barrier()
        region["t1"] = time.time()
        rhif.rhif_set_timing(False)
        ks = rhif.rhif_kernel_stats()
        return reduce_max(e0.elapsed_time(e1) / 1e3), info, ks

    clocks = ClockSampler(local)
    # headline precision, no instrumentation in the timed region
    clocks.start()
    sec, (u, its, rr), ks_count = timed(lambda: wl.step(wl.headline), args.steps, args.warmup)
    clk = clocks.stop(region.get("t0"), region.get("t1"))
    value = whole_job_value(wl.dofs, args.steps, sec, world)
    gpu_launches = int(sum(v["launches"] for v in ks_count.values()))
    # the same steps again with CUDA events around every library launch (per-kernel durations)
    _, _, ks = timed(lambda: wl.step(wl.headline), args.steps, 0, timing=True)
    # the other precision beside it
    other = "fp32" if wl.headline == "fp64" else "fp64"
    sec_o, (u_o, its_o, rr_o), _ = timed(lambda: wl.step(other), args.fp64_steps, 1)
    value_o = whole_job_value(wl.dofs, args.fp64_steps, sec_o, world)

    def rel(a, b):
        if isinstance(a, list):
            return max(float(torch.linalg.norm(x - y) / torch.linalg.norm(y)) for x, y in zip(a, b))
        return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))

    du = rel(u, u_o)

    # end to end from pinned host buffers, copies inside the timed region
    for _ in range(args.warmup):
        wl.e2e_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        wl.e2e_step()
    e1.record(stream)
    barrier()
    sec_e2e = reduce_max(e0.elapsed_time(e1) / 1e3)
    e2e_val = whole_job_value(wl.dofs, args.steps, sec_e2e, world)

    # roofline of the dominant kernel category of the headline path
    peaks = alu_peaks(torch)
    hbm, hbm_kind = measured_peaks()
    name, st = max(ks.items(), key=lambda kv: kv[1]["total_ms"])
    per_launch_ms = st["total_ms"] / max(st["launches"], 1)
    if hbm_bound(name):
        achieved = st["bytes"] / max(st["launches"], 1) / (per_launch_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "peak_kind": hbm_kind}
    else:
        achieved = st["flops"] / max(st["launches"], 1) / (per_launch_ms / 1e3) / 1e12
        peak, kind = alu_peak_nominal(wl.headline, torch, (clk or {}).get("sm_max_mhz"))
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_kind": kind}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = name
    # every kernel category against its roofline: counted work over its
    # CUDA-event time in the instrumented steps
    alu_pk, _ = alu_peak_nominal(wl.headline, torch, (clk or {}).get("sm_max_mhz"))
    gemm_pk = peaks.get(wl.headline, peaks.get("fp32"))
    by_kernel = {}
    for k, v in sorted(ks.items(), key=lambda kv: -kv[1]["total_ms"]):
        if not v["launches"] or v["total_ms"] <= 0:
            continue
        t = v["total_ms"] / 1e3
        row = {"ms_per_step": round(v["total_ms"] / args.steps, 4),
               "launches_per_step": round(v["launches"] / args.steps, 2)}
        if hbm_bound(k) and v["bytes"] > 0:
            a = v["bytes"] / t / 1e9
            row.update(bound="hbm", achieved=round(a, 2), unit="GB/s", frac=round(a / hbm, 5))
        elif v["flops"] > 0:
            a = v["flops"] / t / 1e12
            row.update(bound="alu", achieved=round(a, 5), unit="TFLOP/s", frac=round(a / alu_pk, 6),
                       frac_of_gemm=round(a / gemm_pk, 6))
        else:
            row.update(bound="latency", note="no counted work (condition estimate, FP64 re-elimination)")
        by_kernel[k] = row
    roof["launch_ms"] = per_launch_ms
    roof["traffic"] = profile_traffic(name, wl.headline, args.workload)

    dtype = "f64" if wl.headline == "fp64" else "f32 factor + f64 PCG"
    result = {
        "metric": METRIC, "value": value, "unit": "DOFs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype, "data": "synthetic",
        "config": dict(wl.config(), parallelism=f"replicas{world}",
                       l2="working set larger than L2 (fronts, frames); no flush"),
        "pcg_iters": its[0], "relres": rr[0],
        other: {"value": value_o, "ms_per_step": 1e3 * sec_o / args.fp64_steps,
                "pcg_iters": its_o[0], "relres": rr_o[0], "rel_diff_vs_headline": du},
        "roofline": roof,
        "roofline_by_kernel": by_kernel,
        "alu_peaks_tflops": peaks,
        "kernels": {k: {"launches": v["launches"], "ms": round(v["total_ms"], 3)}
                    for k, v in ks.items() if v["launches"]},
        "gpu_launches": gpu_launches,
        "clocks": clk,
        "e2e": {"value": e2e_val, "unit": "DOFs/s", "h2d_bytes_per_step": int(wl.h2d),
                "d2h_bytes_per_step": int(wl.d2h)},
    }
    if wl.headline == "fp32":
        result["mixed_over_fp64"] = value / value_o
    if args.workload in ("c1", "c2", "c3"):
        result["breakdown"] = step_breakdown(wl, torch)
    if args.workload == "c2":
        result["local_precond"] = local_precond_compare(wl, timed)
    if args.workload == "c3":
        result["tensor_core_kinds"] = tensor_core_kinds(wl, timed, torch)
    if args.workload == "c4":
        result["rhs_dofs_per_s"] = value * 32
    if args.workload == "c5":
        result["loss"] = rr[0]
        result.pop("relres")
        result.pop("pcg_iters")
        result[other]["loss"] = result[other].pop("relres")
        result[other].pop("pcg_iters")
        result[other]["grad_rel_diff_vs_headline"] = result[other].pop("rel_diff_vs_headline")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        body, side, extra, desc = _SAMPLES[args.workload]
        save = os.path.join(tempfile.gettempdir(), f"rhif_oracle_u_{os.getpid()}.npy") \
            if body == "2d" else ""
        r = run_oracle(args.workload, side, save)
        result["cpu_baseline"] = {
            "value": r["dofs"] / r["seconds"], "unit": "DOFs/s", "cores": 1, "kind": "oracle",
            "sample": (f"FP64 oracle on {desc} (DOFs={r['dofs']}, {r['seconds']:.1f} s, "
                       f"{r['iters']} PCG its), 1 thread")}
        if save:
            result["vs_oracle"] = compare_with_oracle(rhif, W, torch, dev, args.workload, side,
                                                      extra, save, r["iters"], wl.rtol)
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()


def paper_tables(args):
    """The structure of the paper's Tables 1-2 on this GPU: for the quantized
    high-contrast field (Sec. 4) at 1023^2 (leaf 16; tol 1e-3, 1e-4, 1e-6,
    1e-8 as in Table 1) and 31^3 / 63^3 (leaf 8, faces + edges; tol 1e-3,
    1e-6), HIF, PHIF with the diagonal local preconditioner and PHIF (FP64
    factors): factor time, root size, e_a and e_s (power iterations, 1e-2
    relative change) and PCG iterations to relres 1e-12.  One JSON line."""
    import numpy as np
    import torch

    import paper_1808_01364_gb300 as rhif
    import workloads as W
    rhif.load()
    rows = []
    tols = {2: (1e-3, 1e-4, 1e-6, 1e-8), 3: (1e-3, 1e-6)}
    for ns, leaf in (((1023, 1023), 16), ((31, 31, 31), 8), ((63, 63, 63), 8)):
        a = torch.as_tensor(W.paper_quantized_field(ns, seed=W.SEED_BASE + 5), device="cuda")
        n = int(np.prod(ns))
        f = torch.as_tensor(W.normal_rhs(ns, W.SEED_BASE + 6), device="cuda")
        x0 = torch.as_tensor(np.random.Generator(np.random.PCG64(7)).standard_normal(n),
                             device="cuda")
        x1 = torch.as_tensor(np.random.Generator(np.random.PCG64(8)).standard_normal(n),
                             device="cuda")
        csr = rhif.rhif_assemble_fd(ns, a, 0.0)
        for tol in tols[len(ns)]:
            for pre in ("none", "diag", "block"):
                row = {"grid": "x".join(map(str, ns)), "N": n, "leaf": leaf, "tol": tol,
                       "method": {"none": "HIF", "diag": "PHIF-diag", "block": "PHIF"}[pre]}
                try:
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    F = rhif.rhif_factor(csr, ns, leaf, tol, precision="fp64", precondition=pre,
                                         edge_skel_3d=len(ns) == 3)
                    e1.record()
                    e1.synchronize()
                    st = F.stats()
                    es, _ = F.estimate_es(x0)
                    ea, _ = F.estimate_ea(x0, x1)
                    _, its, rr = F.pcg(f, rtol=1e-12, maxit=1000, check=False)
                    row.update(factor_ms=e0.elapsed_time(e1), root=st["root_size"], e_a=ea, e_s=es,
                               pcg_iters=its[0], relres=rr[0],
                               factor_gb=st["factor_bytes"] / 1e9)
                    F.free()
                except rhif.RhifError as e:
                    row["failed"] = str(e).split(":")[0]
                rows.append(row)
    print(json.dumps({"paper_tables": rows}))


def tc_kernel(args):
    """C -= A B^T through rhif_tc_gemm_check on 4096 x 4096 x 1024 FP32 data,
    each operand kind: CUDA-event time per call (2 warm-up, 5 timed calls)
    and the useful rate 2MNK / t.  One JSON line."""
    import torch

    import paper_1808_01364_gb300 as rhif
    rhif.load()
    M = N = 4096
    K = 1024
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn(K, M, device="cuda", generator=g).t()
    B = torch.randn(K, N, device="cuda", generator=g).t()
    out = {}
    for kind in ("tf32x3", "tf32", "bf16"):
        C = torch.zeros(N, M, device="cuda").t()
        for _ in range(2):
            rhif.rhif_tc_gemm_check(A, B, C, kind=kind)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            rhif.rhif_tc_gemm_check(A, B, C, kind=kind)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        out[kind] = {"ms": ms, "useful_tflops": 2 * M * N * K / ms / 1e9,
                     "products": 3 if kind == "tf32x3" else 1}
    print(json.dumps({"tc_kernel": out, "M": M, "N": N, "K": K}))


def skeleton_growth(args):
    """Root size |S_L| of 3D factors with and without edge skeletonization
    (Remark 3.1) as the grid grows: i.i.d. log-uniform [1e-3, 1e3] field,
    b = 1e-2, leaf 8, tol 1e-3, FP64 PHIF; per-level active DOF counts, factor
    time and memory, PCG iterations to relres 1e-10.  One JSON line."""
    import numpy as np
    import torch

    import paper_1808_01364_gb300 as rhif
    import workloads as W
    rhif.load()
    rows = []
    for side in (15, 31, 63, 127):
        ns = (side,) * 3
        a = torch.as_tensor(W.log_uniform_pixels(ns, 1e-3, 1e3, W.SEED_BASE + 2), device="cuda")
        f = torch.as_tensor(W.normal_rhs(ns, W.SEED_BASE + 7), device="cuda")
        csr = rhif.rhif_assemble_fd(ns, a, 1e-2)
        for edge in (False, True):
            row = {"grid": f"{side}^3", "N": side ** 3, "edge_skel": edge}
            try:
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                F = rhif.rhif_factor(csr, ns, 8, 1e-3, precision="fp64", edge_skel_3d=edge)
                e1.record()
                e1.synchronize()
                st = F.stats()
                _, its, rr = F.pcg(f, rtol=1e-10, maxit=1000, check=False)
                row.update(factor_ms=e0.elapsed_time(e1), root=st["root_size"],
                           active=[int(x) for x in st["active"][:st["levels"]]],
                           pcg_iters=its[0], relres=rr[0], factor_gb=st["factor_bytes"] / 1e9)
                F.free()
            except rhif.RhifError as e:
                row["failed"] = str(e)[:120]
            rows.append(row)
            torch.cuda.empty_cache()
    print(json.dumps({"skeleton_growth": rows}))


# default timed steps of the GPU arm: about half a second of work, so that
# several clock samples (100 ms period) fall inside the timed region
DEFAULT_STEPS = {"c1": 100, "c2": 40, "c3": 5, "c4": 3, "c5": 40}


def main():
    args = _args()
    if args.steps is None:
        args.steps = 5 if args.impl == "reference" else DEFAULT_STEPS[args.workload]
    if args.tc_kernel:
        tc_kernel(args)
        return
    if args.skeleton_growth:
        skeleton_growth(args)
        return
    if args.paper_tables:
        paper_tables(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
