"""Benchmark of the GB300 compressed-Taylor FMM.

Workload (one "step" = one full evaluation: tree build, M2L derivative
tables, P2M, M2M, M2L, L2L, L2P + P2P): 3D Laplace G = 1/(4 pi r),
compressed Taylor p = 10, uniform octree of 5 levels, N = 1,000,000 sources =
targets uniform in [0,1]^3, weights uniform[-1,1] (seeded synthetic data).

Prints ONE JSON line.  value = targets/s of the whole job (all ranks);
inputs are resident in HBM when the timed region starts; L2 is flushed
between timed steps (each step is timed alone with CUDA events on the
launching stream).  `e2e` repeats the measurement through the public API
with host buffers (pinned), the host<->device copies inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "laplace3d_p10_L5_n1m"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default=os.environ.get("FMM_BENCH_PRECISION", "tf32x3"))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m2l", default="dense", choices=["dense", "fft"],
                    help="M2L form: dense products or the FFT convolution form")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison line")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--cpu-leaves", type=int, default=48)
    ap.add_argument("--points", type=int, default=0,
                    help="override the point count (profiling captures: the same L=5 tree and "
                         "the identical M2L launch on less memory)")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            # start timing only once the sampler is producing rows
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def m2l_count(d: int, L: int) -> int:
    """Number of M2L translations of a full uniform tree (interaction lists)."""
    tot = 0
    for l in range(2, L + 1):
        n = 1 << l
        # per dimension: for target t, sources s with parent(s) adjacent to
        # parent(t), s not adjacent to t (count by brute force on 1D factors
        # is not separable because of the 'not adjacent' condition) -> count
        # pairs directly with numpy on the box grid.
        t = np.arange(n)
        pt = t >> 1
        par_adj = np.abs(pt[:, None] - pt[None, :]) <= 1
        adj = np.abs(t[:, None] - t[None, :]) <= 1
        A = par_adj.astype(np.int64)
        B = (par_adj & adj).astype(np.int64)
        # pairs with all dims parent-adjacent minus those adjacent in all dims
        tot += int(A.sum() ** d - B.sum() ** d)
    return tot


M2L_SOURCES = ["paper_2305_17867_gb300/csrc/m2l_tc.cu", "paper_2305_17867_gb300/csrc/tc_ptx.cuh",
               "paper_2305_17867_gb300/csrc/m2l_simt.cu"]


def m2l_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in M2L_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(prec: str):
    """DRAM bytes per launch of the M2L contraction from the committed ncu summary.

    The summary carries one line per precision,
    ``traffic: <precision> <bytes per launch> sources <hash>``; the figure is
    reported only while the kernel sources still hash to the captured value.
    """
    path = os.path.join(ROOT, "profiles", "m2l_tc_laplace3d_p10_L5.md")
    if not os.path.exists(path):
        return None, "no capture"
    want = m2l_source_hash()
    with open(path) as fh:
        for line in fh:
            f = line.strip().strip("`").split()
            if len(f) == 5 and f[0] == "traffic:" and f[1] == prec and f[3] == "sources":
                if f[4] != want:
                    return None, "kernel changed since the capture"
                return int(f[2]), ("ncu dram__bytes.sum.per_second x gpu__time_duration.sum of one "
                                   "launch, " + path[len(ROOT) + 1:])
    return None, "no capture for this precision"


def leaf_of(x, L):
    n = 1 << L
    b = np.minimum(np.floor(x / (1.0 / n)).astype(np.int64), n - 1)
    return (b[:, 2] * n + b[:, 1]) * n + b[:, 0]


def run_cpu_oracle(src, w, L, p, nleaves, seed=12345):
    """Oracle on a bounded sample: every target of `nleaves` random leaves."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import fmm_oracle

    fmm_oracle.lib()
    leaves = leaf_of(src, L)
    rng = np.random.default_rng(seed)
    pick = rng.choice(1 << (3 * L), nleaves, replace=False)
    idx = np.nonzero(np.isin(leaves, pick))[0]
    t0 = time.perf_counter()
    ref = fmm_oracle.fmm_uniform("laplace", 3, p, L, src, w, src, sample=idx)
    dt = time.perf_counter() - t0
    return idx, ref, dt, fmm_oracle.num_threads()


def main():
    args = parse()
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2305_17867_gb300 import workloads as Wk

    wl = Wk.WORKLOADS[WORKLOAD]
    if args.impl == "reference":
        return run_reference(args, wl, rank)

    from paper_2305_17867_gb300.fmm import FMM

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    # every rank runs an independent replica of the workload (weak scaling)
    src, w, _ = Wk.make_inputs(wl, n_src=args.points or None,
                               seed=wl.seed + 1000 * rank if rank else None)
    n = src.shape[0]
    t_plan = time.perf_counter()
    plan = FMM("laplace", d=3, p=wl.p, levels=wl.levels, precision=args.precision, device=dev,
               m2l=args.m2l)
    t_plan = (time.perf_counter() - t_plan) * 1e3
    s = torch.tensor(src, device=dev)
    wt = torch.tensor(w, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        return plan.eval(s, wt)

    for _ in range(max(args.warmup, 3)):
        phi = step()
    torch.cuda.synchronize()
    launches = plan.last_launch_count()
    # the plan's own phase events and the events around the M2L contraction are
    # recorded on the launching stream inside every timed step
    plan.set_timing(True)

    times, ph_steps, k_steps = [], [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            phi = step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            ph_steps.append(plan.phase_times())
            k_steps.append(plan.m2l_kernel_time())
    torch.cuda.synchronize()
    plan.set_timing(False)
    if dist:
        dist.barrier()
    ms = sum(times) / len(times)
    phases = {k: sum(p[k] for p in ph_steps) / len(ph_steps) for k in ph_steps[0]}
    m2l_kernel_ms = sum(k_steps) / len(k_steps)
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = n * world / (ms * 1e-3)

    # end to end through the public API from pinned host buffers
    hs = torch.tensor(src).pin_memory()
    hw = torch.tensor(w).pin_memory()
    e2e_times = []
    for _ in range(0 if args.no_e2e else max(2, min(args.steps, 5))):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = plan.eval(hs, hw)
        e2e_times.append((time.perf_counter() - t0) * 1e3)
        assert out.device.type == "cpu"
    e2e_ms = statistics.median(e2e_times) if e2e_times else float("nan")

    # M2L work and roofline
    nm2l = m2l_count(3, wl.levels)
    flops_m2l = 2.0 * plan.nj * plan.nj * nm2l
    # FFT form: one complex multiply-add (8 flop) per kept frequency and translation
    kf = (wl.p + 1) * (2 * wl.p + 1) * (2 * min(plan.c, wl.p + 1) - 1)
    algo = f"2*|j|^2 = {2 * plan.nj ** 2} FLOP/translation x {nm2l} translations"
    if args.m2l == "fft":
        flops_m2l = 8.0 * kf * nm2l
        algo = (f"8 * {kf} (complex multiply-add per kept frequency) FLOP/translation x "
                f"{nm2l} translations")
    m2l_ms = m2l_kernel_ms
    peaks, peak_src = load_peaks()
    prec = args.precision
    tf32_dense = peaks["bf16_tflops"] * 1.1 / 2.25
    if prec == "tf32":
        peak = tf32_dense
        bound, unit, pname = "tensor", "TFLOP/s", f"tf32 dense = bf16 {peak_src} x 1.1/2.25"
    elif prec == "tf32x3":
        # the split contraction issues three tf32 products per algorithmic multiply-add
        peak = tf32_dense / 3.0
        bound, unit, pname = ("tensor", "TFLOP/s",
                              f"tf32x3 = (bf16 {peak_src} x 1.1/2.25) / 3 passes")
    elif prec == "bf16x3":
        peak = peaks["bf16_tflops"] / 3.0
        bound, unit, pname = "tensor", "TFLOP/s", f"bf16x3 = bf16 dense {peak_src} / 3 passes"
    elif prec == "fp32":
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        bound, unit, pname = "alu", "TFLOP/s", "fp32 FMA: 152 SMs x 128 lanes x 2 x max clock"
    else:
        peak = 152 * 2 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        bound, unit, pname = ("alu", "TFLOP/s",
                              "fp64 FMA: 152 SMs x 2 lanes x 2 x max clock (nominal 1.25 TFLOP/s)")
    achieved = flops_m2l / (m2l_ms * 1e-3) / 1e12
    traffic, traffic_src = profiled_traffic(prec) if args.m2l == "dense" else (None, "no capture")
    roof = {"kernel": "m2l contraction" if args.m2l == "dense" else "m2l fft stencil", "bound": bound, "achieved": achieved, "peak": peak,
            "unit": unit, "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
            "kernel_ms": m2l_ms, "peak_source": pname,
            "frac_vs_tf32_dense": achieved / tf32_dense,
            "algorithmic": algo}

    wname = WORKLOAD if not args.points else f"{WORKLOAD} with n={args.points} (profiling case)"
    result = {
        "metric": "full-FMM targets/sec (3D Laplace, compressed Taylor p=10, uniform octree L=5, "
                  "N=1e6) with M2L translations/sec",
        "value": value, "unit": "targets/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": wname, "n_src": n, "n_tgt": n, "p": wl.p, "levels": wl.levels,
                   "precision": prec, "m2l": args.m2l, "l2": "flushed (256 MiB write) between timed steps",
                   "parallelism": "replicas" if world > 1 else "single"},
        "m2l_translations_per_s": nm2l * world / (ms * 1e-3),
        "m2l_translations": nm2l,
        "phases_ms": phases,
        "plan_create_ms": t_plan,
        "roofline": roof,
        "gpu_launches": launches * args.steps,
        "clocks": clk.summary(),
        "e2e": {"value": n * world / (e2e_ms * 1e-3), "unit": "targets/s",
                "ms_per_step": e2e_ms, "h2d_bytes_per_step": int(src.nbytes + w.nbytes),
                "d2h_bytes_per_step": int(n * 8)},
    }
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    phi_np = phi.cpu().numpy()
    if not args.no_fp64 and prec != "fp64":
        plan64 = FMM("laplace", d=3, p=wl.p, levels=wl.levels, precision="fp64", device=dev)
        for _ in range(2):
            phi64 = plan64.eval(s, wt)
        torch.cuda.synchronize()
        t64 = []
        for _ in range(2):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            phi64 = plan64.eval(s, wt)
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
        plan64.set_timing(True)
        plan64.eval(s, wt)
        ph64 = plan64.phase_times()
        p64 = phi64.cpu().numpy()
        result["fp64"] = {"value": n / (statistics.median(t64) * 1e-3), "unit": "targets/s",
                          "ms_per_step": statistics.median(t64), "phases_ms": ph64,
                          "m2l_tflops": flops_m2l / (ph64["m2l"] * 1e-3) / 1e12}
        result["rel_err_vs_fp64_gpu"] = float(np.linalg.norm(phi_np - p64) / np.linalg.norm(p64))

    if not args.no_cpu:
        idx, ref, dt, cores = run_cpu_oracle(src, w, wl.levels, wl.p, args.cpu_leaves)
        result["rel_err_vs_oracle"] = float(np.linalg.norm(phi_np[idx] - ref) / np.linalg.norm(ref))
        result["cpu_baseline"] = {
            "value": len(idx) / dt, "unit": "targets/s", "cores": cores, "kind": "oracle",
            "sample": f"every target of {args.cpu_leaves} random leaves ({len(idx)} targets) of the "
                      f"same 1e6-point tree; upward pass over all sources included; {dt:.1f} s"}
        sys.path.insert(0, os.path.join(ROOT, "oracle"))
        import fmm_oracle

        dref = fmm_oracle.direct("laplace", 3, src, w, src[idx[:200]])
        result["rel_err_vs_direct"] = float(np.linalg.norm(phi_np[idx[:200]] - dref) /
                                            np.linalg.norm(dref))
    print(json.dumps(result))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args, wl, rank):
    """The reference arm: the CPU oracle, timed on the host cores."""
    if rank != 0:
        return
    src, w, _ = __import__("paper_2305_17867_gb300.workloads", fromlist=["x"]).make_inputs(wl)
    times, n_t, cores = [], 0, 1
    for k in range(max(args.warmup, 0) + args.steps):
        idx, ref, dt, cores = run_cpu_oracle(src, w, wl.levels, wl.p, max(4, args.cpu_leaves // 4),
                                             seed=777 + k)
        if k >= args.warmup:
            times.append(dt)
            n_t += len(idx)
    value = n_t / sum(times)
    line = {
        "impl": "reference", "metric": "full-FMM targets/sec (3D Laplace, compressed Taylor p=10, "
        "uniform octree L=5, N=1e6) with M2L translations/sec",
        "value": value, "unit": "targets/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n_src": len(w), "p": wl.p,
                                        "levels": wl.levels},
        "cpu_baseline": {"value": value, "unit": "targets/s", "cores": cores, "kind": "oracle",
                         "sample": "per step: every target of a few random leaves of the 1e6-point "
                                   "tree (upward pass over all sources included)"},
        "e2e": {"value": value, "unit": "targets/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
