"""Benchmark of the GB300 compressed-Taylor FMM.

Default workload (one "step" = one full evaluation: tree build, M2L
derivative tables, P2M, M2M, M2L, L2L, L2P + P2P): 3D biharmonic G = |x - y|,
compressed Taylor p = 8, uniform octree of 6 levels, N = 4,000,000 sources =
targets uniform in [0,1]^3, weights uniform[-1,1] (seeded synthetic data) --
the largest single-GPU workload of the set; M2L as dense contractions on the
tensor cores (TF32x3), beside the FP64 form (FFT M2L, the fastest FP64 form)
on the same GPU and the other split form (BF16x3).  `--workload` selects the
other particle sets of paper_2305_17867_gb300/workloads.py (2D Laplace, 3D
Laplace p = 10 with 10^6 points, adaptive Yukawa/Plummer, the backward step).

Prints ONE JSON line.  value = targets/s of the whole job (all ranks);
inputs are resident in HBM when the timed region starts; L2 is flushed
between timed steps (each step is timed alone with CUDA events on the
launching stream).  `e2e` repeats the measurement through the public API
with host buffers (pinned), the host<->device copies inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--p P]
                  [--precision P] [--m2l dense|fft] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "biharmonic3d_p8_L6_n4m"
METRIC = "full-FMM targets/sec and M2L translations/sec at stated rel. error, % of roofline"
ADAPTIVE_DEPTH = 10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--p", type=int, default=0, help="override the expansion order")
    ap.add_argument("--precision", default=os.environ.get("FMM_BENCH_PRECISION", "auto"),
                    help="fp64|fp32|tf32|tf32x3|bf16x3|f16x3; auto = f16x3 on uniform 3D trees, "
                         "else fp64")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m2l", default="dense", choices=["dense", "fft"],
                    help="M2L form: dense products or the FFT convolution form")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison arm")
    ap.add_argument("--alt-precision", default="auto",
                    help="second tensor-core form reported in the same line (none to skip); "
                         "auto = tf32x3 beside f16x3 and bf16x3, f16x3 beside tf32x3")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--cpu-level", type=int, default=3,
                    help="level of the subtree whose targets the CPU oracle evaluates")
    ap.add_argument("--cpu-targets", type=int, default=16,
                    help="adaptive workloads: targets the CPU oracle evaluates")
    ap.add_argument("--points", type=int, default=0,
                    help="override the point count (profiling captures: the same tree depth and, "
                         "for uniform trees, the identical M2L launch on less memory)")
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
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")

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
        t = np.arange(n)
        pt = t >> 1
        par_adj = np.abs(pt[:, None] - pt[None, :]) <= 1
        adj = np.abs(t[:, None] - t[None, :]) <= 1
        A = par_adj.astype(np.int64)
        B = (par_adj & adj).astype(np.int64)
        # pairs with all axes parent-adjacent minus those adjacent on all axes
        tot += int(A.sum() ** d - B.sum() ** d)
    return tot


# The tensor-core contraction's device code: m2l_tc.cu above its host-side
# section, and the PTX wrappers it uses.  The traffic figure of a capture stays
# valid while this code is unchanged (host-side launch code may change).
M2L_SOURCES = [("paper_2305_17867_gb300/csrc/m2l_tc.cu", "// ---- host side"),
               ("paper_2305_17867_gb300/csrc/tc_ptx.cuh", None)]


def device_part(text: str, marker) -> str:
    return text if marker is None else text.split(marker, 1)[0]


def code_digest(texts) -> str:
    """Hash of source texts with // comments, trailing blanks and empty lines
    removed, so that editing a comment does not void a capture of the code."""
    import hashlib

    h = hashlib.sha256()
    for text in texts:
        for line in text.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def m2l_source_hash() -> str:
    texts = []
    for f, marker in M2L_SOURCES:
        with open(os.path.join(ROOT, f)) as fh:
            texts.append(device_part(fh.read(), marker))
    return code_digest(texts)


def profiled_traffic(prec: str, workload: str, profiles=None):
    """DRAM bytes per launch of the M2L contraction from a committed ncu summary.

    A summary under profiles/ carries one line per captured (precision,
    workload):
    ``traffic: <precision> <bytes per launch> sources <hash> workload <name>``;
    the figure is reported only while the kernel's device code still hashes to
    the captured value.
    """
    folder = profiles or os.path.join(ROOT, "profiles")
    if not os.path.isdir(folder):
        return None, "no capture"
    want = m2l_source_hash()
    stale = False
    for fn in sorted(os.listdir(folder)):
        if not fn.endswith(".md"):
            continue
        path = os.path.join(folder, fn)
        with open(path) as fh:
            for line in fh:
                f = line.strip().strip("`").split()
                if (len(f) == 7 and f[0] == "traffic:" and f[1] == prec and f[3] == "sources"
                        and f[5] == "workload" and f[6] == workload):
                    if f[4] != want:
                        stale = True
                        continue
                    return int(f[2]), ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                       "launch, profiles/" + fn)
    return None, ("kernel changed since the capture" if stale else "no capture for this "
                  "precision and workload")


def leaf_of(x, L):
    n = 1 << L
    d = x.shape[1]
    b = np.minimum(np.floor(x / (1.0 / n)).astype(np.int64), n - 1)
    key = np.zeros(len(x), dtype=np.int64)
    for k in range(d - 1, -1, -1):
        key = key * n + b[:, k]
    return key


def max_over_ranks(ms: float, dist, device) -> float:
    """Step time of the job: the slowest rank's (replicas run concurrently)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_per_rank: int, world: int, ms: float) -> float:
    """Targets per second of the whole job: every rank's targets in the job's step time."""
    return n_per_rank * world / (ms * 1e-3)


def precision_of(args, wl):
    if args.precision != "auto":
        return args.precision
    return "f16x3" if (wl.d == 3 and wl.levels > 0) else "fp64"


def make_plan(wl, p, prec, m2l, dev):
    from paper_2305_17867_gb300.fmm import FMM

    levels = wl.levels if wl.levels > 0 else -ADAPTIVE_DEPTH
    return FMM(wl.kernel, d=wl.d, p=p, levels=levels, lam=wl.lam, precision=prec, device=dev,
               m2l=m2l, max_leaf=wl.max_leaf or 64)


def subtree_targets(tgt, level, rng):
    """Indices of the targets inside one seeded random box of `level` of the
    unit root box (the targets of a whole subtree), and the box."""
    n = 1 << level
    d = tgt.shape[1]
    cell = np.minimum(np.floor(tgt * n).astype(np.int64), n - 1)
    while True:
        pick = rng.integers(0, n, size=d)
        idx = np.nonzero(np.all(cell == pick, axis=1))[0]
        if len(idx):
            return idx, pick


def run_cpu_oracle(wl, p, src, w, tgt, args, seed=12345, t_up=None):
    """The oracle's throughput on the whole workload, modelled from two bounded runs.

    t_up: the oracle evaluated at ONE target -- the tree, the upward pass over
    every source (P2M, M2M), the M2L derivative tables and one leaf's downward
    chain.  t_sub: every target of one seeded random box of level `cpu_level`
    (uniform trees: a whole subtree, whose boxes share their ancestors as in a
    full run) or `cpu_targets` random targets (adaptive trees).  The
    per-target downward cost is (t_sub - t_up) / n_sub, so a whole evaluation
    takes t_up + N (t_sub - t_up) / n_sub; the value is N over that time.
    Returns (idx, phi at idx, modelled seconds, t_up, t_sub, cores, text).
    """
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import fmm_oracle

    fmm_oracle.lib()
    rng = np.random.default_rng(seed)
    if wl.levels > 0:
        lev = min(args.cpu_level, wl.levels - 1)
        idx, box = subtree_targets(tgt, lev, rng)
        run = lambda sample: fmm_oracle.fmm_uniform(wl.kernel, wl.d, p, wl.levels, src, w, tgt,
                                                    lam=wl.lam, sample=sample)
        what = f"every target of the level-{lev} box {box.tolist()} ({len(idx)} targets)"
    else:
        idx = np.sort(rng.choice(len(tgt), args.cpu_targets, replace=False))
        run = lambda sample: fmm_oracle.fmm_adaptive(wl.kernel, wl.d, p, src, w, tgt,
                                                     max_leaf=wl.max_leaf,
                                                     max_depth=ADAPTIVE_DEPTH, lam=wl.lam,
                                                     sample=sample)
        what = f"{len(idx)} random targets"
    if t_up is None:
        t0 = time.perf_counter()
        run(idx[:1])
        t_up = time.perf_counter() - t0
    t0 = time.perf_counter()
    ref = run(idx)
    t_sub = time.perf_counter() - t0
    n_t = tgt.shape[0]
    t_full = t_up + n_t * max(t_sub - t_up, 0.0) / len(idx)
    text = (f"oracle at one target (tree, upward pass over all {len(src)} sources, tables, one "
            f"leaf chain) t_up = {t_up:.2f} s; at {what} t_sub = {t_sub:.2f} s; whole "
            f"evaluation modelled as t_up + N (t_sub - t_up) / n_sub = {t_full:.1f} s")
    return idx, ref, t_full, t_up, t_sub, fmm_oracle.num_threads(), text


def peak_of(prec, m2l, d, peaks, peak_src):
    """(peak TFLOP/s, bound, text) of the M2L contraction in this arithmetic."""
    tf32_dense = peaks["bf16_tflops"] * 1.1 / 2.25
    clock = peaks.get("sm_max_mhz", 2070.0) * 1e6
    tensor = m2l == "dense" and d == 3 and prec in ("tf32", "tf32x3", "bf16x3", "f16x3")
    if tensor and prec == "tf32":
        return tf32_dense, "tensor", f"tf32 dense = bf16 {peak_src} x 1.1/2.25"
    if tensor and prec == "tf32x3":
        # the split contraction issues three tf32 products per algorithmic multiply-add
        return tf32_dense / 3.0, "tensor", f"tf32x3 = (bf16 {peak_src} x 1.1/2.25) / 3 passes"
    if tensor and prec == "bf16x3":
        return peaks["bf16_tflops"] / 3.0, "tensor", f"bf16x3 = bf16 dense {peak_src} / 3 passes"
    if tensor and prec == "f16x3":  # fp16 and bf16 share the 16-bit tensor rate
        return peaks["bf16_tflops"] / 3.0, "tensor", f"f16x3 = bf16 dense {peak_src} / 3 passes"
    if prec == "fp64":
        return (152 * 2 * 2 * clock / 1e12, "alu",
                "fp64 FMA: 152 SMs x 2 lanes x 2 x max clock (nominal 1.25 TFLOP/s)")
    return 152 * 128 * 2 * clock / 1e12, "alu", "fp32 FMA: 152 SMs x 128 lanes x 2 x max clock"


def m2l_flops(m2l, nj, nm2l, p, c, d):
    if m2l == "fft":
        kf = (p + 1) * (2 * p + 1) ** (d - 2) * (2 * min(c, p + 1) - 1)
        return 8.0 * kf * nm2l, (f"8 * {kf} (complex multiply-add per kept frequency) "
                                 f"FLOP/translation x {nm2l} translations")
    return 2.0 * nj * nj * nm2l, f"2*|j|^2 = {2 * nj ** 2} FLOP/translation x {nm2l} translations"


def roofline(plan, prec, m2l, m2l_ms, nm2l, p, c, workload):
    peaks, peak_src = load_peaks()
    flops, algo = m2l_flops(m2l, plan.nj, nm2l, p, c, plan.d)
    peak, bound, pname = peak_of(prec, m2l, plan.d, peaks, peak_src)
    tensor = bound == "tensor"
    achieved = flops / (m2l_ms * 1e-3) / 1e12
    traffic, traffic_src = (profiled_traffic(prec, workload) if tensor else (None, "no capture"))
    kname = {"dense": "m2l tensor-core contraction" if tensor else "m2l simt contraction",
             "fft": "m2l fft stencil"}[m2l]
    return {"kernel": kname, "bound": bound, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "traffic_source": traffic_src, "kernel_ms": m2l_ms,
            "peak_source": pname + (" (of measured)" if peak_src == "measured" else
                                    " (of fallback)"),
            "algorithmic": algo}


def near_pairs(src, tgt, L):
    """Source-target pairs of the near field of a uniform tree (3^d adjacent
    leaves, the leaf itself included; coinciding points excluded when the
    targets are the sources)."""
    d = src.shape[1]
    n = 1 << L
    shape = (n,) * d

    def hist(x):
        cell = np.minimum(np.floor(x * n).astype(np.int64), n - 1)
        key = np.ravel_multi_index(tuple(cell[:, k] for k in range(d - 1, -1, -1)), shape)
        return np.bincount(key, minlength=n ** d).reshape(shape).astype(np.float64)

    hs = hist(src)
    ht = hs if tgt is src else hist(tgt)
    pad = np.pad(hs, 1)
    acc = np.zeros(shape)
    for off in np.ndindex(*(3,) * d):
        acc += pad[tuple(slice(o, o + n) for o in off)]
    pairs = float((ht * acc).sum())
    return pairs - (len(src) if tgt is src else 0)


def phase_floors(wl, plan, prec, m2l, nm2l, p, n_src, n_tgt, same, pairs):
    """Lower bounds (ms) of each phase of one evaluation on this GPU, from the
    phase's algorithmic work and the unit that bounds it:
      tree  HBM: 32 B in + 32 B out per point (positions and weight, float64),
            + 16 B per point for the float box-relative copy;
      p2m   FP32: 4 N(p) FLOP per source (monomials, weighted sums);
      m2m   HBM: every child's multipole read once and each parent's written,
            float64, levels 2..L-1;
      m2l   the contraction's own roofline (tensor pipe, or FMA units);
      l2l   HBM: parents read, children's locals read and written, float64;
      leaf  L2P 2 N(p) FLOP per target, P2P 8 FP32 instructions and one
            reciprocal square root (MUFU, 16 per SM per clock) per pair.
    """
    peaks, peak_src = load_peaks()
    hbm = peaks["hbm_gbs"] * 1e9
    clock = peaks.get("sm_max_mhz", 2070.0) * 1e6
    fp32 = 152 * 128 * 2 * clock
    mufu = 152 * 16 * clock
    d, L, nj, nf = wl.d, wl.levels, plan.nj, plan.nfull
    npts = n_src + (0 if same else n_tgt)
    nb = [1 << (d * l) for l in range(L + 1)]
    f = {}
    f["tree"] = (64 + 16) * npts / hbm
    f["p2m"] = 4.0 * nf * n_src / fp32
    f["m2m"] = sum(nb[l + 1] + nb[l] for l in range(2, L)) * nj * 8 / hbm
    flops, _ = m2l_flops(m2l, nj, nm2l, p, plan.c, d)
    peak, _, _ = peak_of(prec, m2l, d, peaks, peak_src)
    f["m2l"] = flops / (peak * 1e12)
    f["l2l"] = sum(nb[l - 1] + 2 * nb[l] for l in range(3, L + 1)) * nj * 8 / hbm
    f["leaf"] = 2.0 * nf * n_tgt / fp32 + max(8.0 * pairs / (fp32 / 2), pairs / mufu)
    return {k: v * 1e3 for k, v in f.items()}


def time_steps(fn, n, flush, stream):
    """CUDA-event times (ms) of n calls of fn, L2 flushed before each."""
    import torch

    out = []
    for _ in range(n):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def side_arm(wl, p, prec, m2l, dev, s, wt, t, flush, stream, nm2l, steps):
    """Another arithmetic on the same inputs: throughput, phases, M2L roofline and phi."""
    plan = make_plan(wl, p, prec, m2l, dev)
    resolved = plan.m2l if plan.m2l != "auto" else ("fft" if prec in ("fp64", "fp32") and
                                                     wl.levels > 0 else "dense")
    for _ in range(2):
        phi = plan.eval(s, wt, t)
    torch_sync()
    ms = time_steps(lambda: plan.eval(s, wt, t), steps, flush, stream)
    plan.set_timing(True)
    phi = plan.eval(s, wt, t)
    ph = plan.phase_times()
    k = plan.m2l_kernel_time()
    plan.set_timing(False)
    n_t = len(phi)
    roof = roofline(plan, prec, resolved, k, nm2l, p, plan.c, wl.name)
    med = statistics.median(ms)
    out = {"precision": prec, "m2l": resolved, "value": n_t / (med * 1e-3), "unit": "targets/s",
           "ms_per_step": med, "steps": steps, "phases_ms": ph,
           "m2l_translations_per_s": nm2l / (med * 1e-3),
           "roofline": {kk: roof[kk] for kk in ("kernel", "bound", "achieved", "peak", "unit",
                                                "frac", "kernel_ms", "peak_source")}}
    phi_np = phi.cpu().numpy()
    plan.close()
    return out, phi_np


def torch_sync():
    import torch

    torch.cuda.synchronize()


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

    wl = Wk.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl, rank)

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    p = args.p or wl.p
    prec = precision_of(args, wl)
    backward = "bwd" in wl.name
    # every rank runs an independent replica of the workload (weak scaling)
    src, w, tgt = Wk.make_inputs(wl, n_src=args.points or None,
                                 n_tgt=(args.points or None) if wl.n_tgt else None,
                                 seed=wl.seed + 1000 * rank if rank else None)
    same = tgt is src
    u = Wk.cotangent(len(tgt), wl.seed) if backward else None
    n_t = tgt.shape[0]
    t_plan = time.perf_counter()
    plan = make_plan(wl, p, prec, args.m2l, dev)
    t_plan = (time.perf_counter() - t_plan) * 1e3
    s = torch.tensor(src, device=dev)
    wt = torch.tensor(w, device=dev)
    t = None if same else torch.tensor(tgt, device=dev)
    ut = torch.tensor(u, device=dev) if backward else None
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        if backward:  # training step: phi and grad phi, then the transposed FMM
            phi, gphi = plan.eval(s, wt, t, grad=True)
            plan.backward(s, wt, s if t is None else t, ut, grad_phi=gphi)
            return phi
        return plan.eval(s, wt, t)

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
            if not backward:
                ph_steps.append(plan.phase_times())
                k_steps.append(plan.m2l_kernel_time())
    torch.cuda.synchronize()
    plan.set_timing(False)
    if dist:
        dist.barrier()
    ms = max_over_ranks(sum(times) / len(times), dist, dev)
    value = job_throughput(n_t, world, ms)
    if backward:  # phases of a forward evaluation alone
        plan.set_timing(True)
        plan.eval(s, wt, t)
        ph_steps = [plan.phase_times()]
        k_steps = [plan.m2l_kernel_time()]
        plan.set_timing(False)
    phases = {k: sum(q[k] for q in ph_steps) / len(ph_steps) for k in ph_steps[0]}
    m2l_kernel_ms = sum(k_steps) / len(k_steps)
    nm2l = plan.last_m2l_count()
    boxes, depth = plan.last_tree()

    # end to end through the public API from pinned host buffers
    hs = torch.tensor(src).pin_memory()
    hw = torch.tensor(w).pin_memory()
    ht = None if same else torch.tensor(tgt).pin_memory()
    hu = torch.tensor(u).pin_memory() if backward else None
    e2e_times = []
    d2h = n_t * 8
    for _ in range(0 if args.no_e2e else max(2, min(args.steps, 5))):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if backward:
            out, gphi = plan.eval(hs, hw, ht, grad=True)
            gw, gs, gt = plan.backward(hs, hw, hs if ht is None else ht, hu,
                                       grad_phi=gphi.to(dev))
            gw, gs, gt = gw.cpu(), gs.cpu(), gt.cpu()
        else:
            out = plan.eval(hs, hw, ht)
        e2e_times.append((time.perf_counter() - t0) * 1e3)
        assert out.device.type == "cpu"
    if backward:  # grad phi comes back with phi and returns to the device; three gradients
        d2h += (n_t * wl.d + len(w) + len(w) * wl.d + n_t * wl.d) * 8
    e2e_ms = statistics.median(e2e_times) if e2e_times else float("nan")
    h2d = int(src.nbytes + w.nbytes + (0 if same else tgt.nbytes) +
              ((u.nbytes + n_t * wl.d * 8) if backward else 0))

    roof = roofline(plan, prec, args.m2l, m2l_kernel_ms, nm2l, p, plan.c, wl.name)
    wname = wl.name if p == wl.p else f"{wl.name} with p={p}"
    if args.points:
        wname += f" with n={args.points} (profiling case)"
    config = {"workload": wname, "kernel": wl.kernel, "d": wl.d, "n_src": len(w), "n_tgt": n_t,
              "p": p, "tree": (f"uniform, {wl.levels} levels" if wl.levels > 0 else
                               f"adaptive, <= {wl.max_leaf} points per leaf, depth <= "
                               f"{ADAPTIVE_DEPTH}"),
              "boxes": boxes, "depth": depth, "precision": prec, "m2l": args.m2l,
              "step": ("forward (phi and grad phi) + backward (transposed FMM)" if backward
                       else "forward"),
              "l2": "flushed (256 MiB write) between timed steps",
              "parallelism": "replicas" if world > 1 else "single"}
    result = {
        "metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec,
        "data": "synthetic", "config": config,
        "m2l_translations_per_s": nm2l * world / (ms * 1e-3), "m2l_translations": nm2l,
        "phases_ms": phases, "plan_create_ms": t_plan, "roofline": roof,
        "gpu_launches": launches * args.steps, "clocks": clk.summary(),
        "e2e": {"value": n_t * world / (e2e_ms * 1e-3), "unit": "targets/s",
                "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
    }
    if wl.levels > 0 and not backward and wl.d == 3:
        pairs = near_pairs(src, tgt, wl.levels)
        floors = phase_floors(wl, plan, prec, args.m2l, nm2l, p, len(w), n_t, same, pairs)
        result["full_fmm_roofline"] = {
            "frac": sum(floors.values()) / ms, "floor_ms": floors,
            "floor_sum_ms": sum(floors.values()), "near_field_pairs": pairs,
            "definition": "sum over phases of the phase's algorithmic floor time / measured step"}
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    phi_np = phi.cpu().numpy()
    arms = {}
    if not backward and wl.levels > 0:
        alt = args.alt_precision
        if alt == "auto":
            alt = {"f16x3": "tf32x3", "tf32x3": "f16x3", "bf16x3": "tf32x3"}.get(prec, "none")
        if alt != "none" and alt != prec:
            arms["alt"] = side_arm(wl, p, alt, "dense", dev, s, wt, t, flush, stream, nm2l,
                                   max(2, min(args.steps, 10)))
        if not args.no_fp64 and prec != "fp64":
            # the fastest FP64 form: what FMM_M2L_AUTO picks (the FFT form)
            arms["fp64"] = side_arm(wl, p, "fp64", "auto", dev, s, wt, t, flush, stream, nm2l, 2)
    for k, (info, ph) in arms.items():
        result[k] = info
        if k == "fp64":
            result["rel_err_vs_fp64_gpu"] = float(np.linalg.norm(phi_np - ph) /
                                                  np.linalg.norm(ph))

    if not args.no_cpu:
        idx, ref, t_full, t_up, t_sub, cores, what = run_cpu_oracle(wl, p, src, w, tgt, args)
        nrm = np.linalg.norm(ref)
        result["rel_err_vs_oracle"] = float(np.linalg.norm(phi_np[idx] - ref) / nrm)
        for k, (info, ph) in arms.items():
            info["rel_err_vs_oracle"] = float(np.linalg.norm(ph[idx] - ref) / nrm)
        result["cpu_baseline"] = {"value": n_t / t_full, "unit": "targets/s", "cores": cores,
                                  "kind": "oracle", "sample": what,
                                  "oracle_targets_compared": int(len(idx))}
        import fmm_oracle

        k = idx[:200]
        dref = fmm_oracle.direct(wl.kernel, wl.d, src, w, tgt[k], lam=wl.lam)
        result["rel_err_vs_direct"] = float(np.linalg.norm(phi_np[k] - dref) /
                                            np.linalg.norm(dref))
    print(json.dumps(result))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args, wl, rank):
    """The reference arm: the CPU oracle as it stands, timed on the host cores.

    Each step evaluates the oracle on a bounded sample of the workload (every
    target of one random level-3 subtree, or a few random targets of an
    adaptive tree); the step's value is the whole-workload throughput modelled
    from it (t_up, the oracle's cost at one target, is measured once during
    the warm-up).  Timed steps stop after a time budget."""
    if rank != 0:
        return
    from paper_2305_17867_gb300 import workloads as Wk

    src, w, tgt = Wk.make_inputs(wl)
    p = args.p or wl.p
    budget_s, spent = 120.0, 0.0
    warm = max(args.warmup, 0)
    t_up = None
    fulls, what, cores = [], "", 1
    for k in range(warm + args.steps):
        t0 = time.perf_counter()
        idx, ref, t_full, t_up, t_sub, cores, what = run_cpu_oracle(wl, p, src, w, tgt, args,
                                                                   seed=777 + k, t_up=t_up)
        if k >= warm:
            spent += time.perf_counter() - t0
            fulls.append(t_full)
            if spent > budget_s:
                break
    value = tgt.shape[0] / statistics.mean(fulls)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "targets/s",
        "n_gpus": args.gpus, "steps": len(fulls), "steps_requested": args.steps,
        "warmup": warm, "time_budget_s": budget_s,
        "ms_per_step": 1e3 * statistics.mean(fulls), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "n_src": len(w), "n_tgt": len(tgt), "p": p},
        "cpu_baseline": {"value": value, "unit": "targets/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step: {what}"},
        "e2e": {"value": value, "unit": "targets/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
