"""Benchmark of the permute-scale-add hot path (TTC, arXiv 1607.01249, Eq. 1).

Default workload (`sweep`): one step = every case of the 2D..6D sweep of
single transposes with 2^26 elements per tensor (N = 2..6, 8 seeded perms per
N, FP32 and FP64, alpha = 1.7, beta in {0, 0.4}) = 160 transposes through the
C ABI, inputs resident in HBM.  Metric: effective HBM bandwidth (decimal GB/s)
counting n*(s_A + s_B) bytes for beta = 0 and n*(s_A + 2 s_B) otherwise.

With the default workload on one GPU the line also carries `batch` (4096
uneven transposes in one graph-launched persistent kernel against one launch
per transpose) and `serving` (a Poisson request trace through the
continuous-batching server against one launch per request, in arrival order,
on one stream) summaries; --no-batch / --no-serving skip them.

Other workloads (`--workload`): single4d, packing, batch, serving.

--impl reference times the CPU oracle (plain C, FP64 arithmetic) on the host
cores on a bounded sample of the same workload.

Multi-GPU (torchrun): every rank runs the same workload on its own GPU
(replicas, no data exchange); the step time is the max over ranks and the
value is the bytes of all ranks over that time.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1607_01249_gb300 import inputs  # noqa: E402

METRIC = "effective HBM GB/s (frac of ~8 TB/s); served transposes/s + p99 vs per-call"
# sources of each workload's kernels: a committed traffic figure counts only
# while their hash is the one it was measured with
KERNEL_SOURCES = {
    "batch": ["paper_1607_01249_gb300/csrc/batch.cu", "paper_1607_01249_gb300/csrc/kernels_impl.cuh",
              "paper_1607_01249_gb300/csrc/kernels.cuh", "paper_1607_01249_gb300/csrc/fpint.h"],
    None: ["paper_1607_01249_gb300/csrc/kernels_impl.cuh", "paper_1607_01249_gb300/csrc/kernels.cuh",
           "paper_1607_01249_gb300/csrc/fpint.h"],
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest of every rank's x (each rank's step time): the job is as
    slow as its slowest replica."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as tdist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (replicas: each rank processes the same units)."""
    return world * units_per_rank / (ms_max * 1e-3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash(workload=None):
    h = hashlib.sha256()
    for src in KERNEL_SOURCES.get(workload, KERNEL_SOURCES[None]):
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{workload}:{kernel}")
    if not e or e.get("kernel_hash") != kernel_hash(workload):
        return None
    return e


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for i, nm in enumerate(names):
                if s[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ------------------------------------------------------------- workloads --

def sweep_problems():
    return inputs.sweep_cases()


def workload_problems(name: str, target: int = 1 << 26, only: str = ""):
    if name == "sweep":
        probs = inputs.sweep_cases(target=target)
        if only:
            keep = set(only.split(","))
            probs = [p for p in probs if p.tag in keep or f"{p.tag}/{p.dtype_in}/b{p.beta}" in keep]
        return probs
    if name == "single4d":
        return [inputs.single_4d()]
    if name == "packing":
        return inputs.packing_cases()
    if name == "pow2":
        return inputs.pow2_cases()
    if name == "complex":
        probs = inputs.complex_cases(target=target // 2)
        if only:
            keep = set(only.split(","))
            probs = [p for p in probs if p.tag in keep or f"{p.tag}/{p.dtype_in}>{p.dtype_out}" in keep]
        return probs
    if name == "batch":
        return inputs.batch_problems(4096)
    if name == "serving":
        return [p for _, p in inputs.serving_requests(1500, seed=4)]
    raise ValueError(name)


def storage_torch(dt):
    import torch
    return {"f32": torch.float32, "f64": torch.float64, "bf16": torch.int16, "e4m3": torch.uint8,
            "c64": torch.complex64, "c128": torch.complex128}[dt]


class DeviceSet:
    """Device buffers for a list of problems: two alternating A/B sets per
    dtype pair so that consecutive transposes never re-read the same input."""

    def __init__(self, probs, seed=0, dist="uniform"):
        import torch
        self.dist = dist
        self.bufs = {}
        need = {}
        for p in probs:
            key = (p.dtype_in, p.dtype_out)
            a, b = need.get(key, (0, 0))
            need[key] = (max(a, p.vol_a), max(b, p.vol_b))
        g = torch.Generator(device="cuda")
        g.manual_seed(seed)
        for (di, do), (va, vb) in need.items():
            sets = []
            for j in range(2):
                A = self._rand(di, va, g, dist)
                B = self._rand(do, vb, g, dist)
                sets.append((A, B))
            self.bufs[(di, do)] = sets

    @staticmethod
    def _rand(dt, n, g, dist="uniform"):
        import torch
        if dt in ("f32", "f64"):
            t = torch.empty(n, dtype=storage_torch(dt), device="cuda")
            if dist == "normal":
                t.normal_(0.0, 1.0, generator=g)
            else:
                t.uniform_(-1.0, 1.0, generator=g)
            return t
        if dt in ("c64", "c128"):
            # both parts uniform[-1, 1]
            t = torch.empty(2 * n, dtype=torch.float32 if dt == "c64" else torch.float64, device="cuda")
            t.uniform_(-1.0, 1.0, generator=g)
            return t.view(storage_torch(dt))
        x = torch.empty(n, dtype=torch.float32, device="cuda").uniform_(-1.0, 1.0, generator=g)
        if dt == "bf16":
            return (x.view(torch.int32) >> 16).to(torch.int16)
        return torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda", generator=g)

    def get(self, p, i):
        return self.bufs[(p.dtype_in, p.dtype_out)][i % 2]


def run_ours(args, rank, world):
    import torch
    from paper_1607_01249_gb300 import build as ttc_build
    from paper_1607_01249_gb300 import ttc

    ttc_build.build()
    ttc.lib()
    dev = rank % max(torch.cuda.device_count(), 1)
    torch.cuda.set_device(dev)
    probs = workload_problems(args.workload, args.target, args.only)
    plans = [ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta, p.outer_a, p.outer_b)
             for p in probs]
    # the packing workload's A is normal(0, 1) (its configuration); the
    # transposes' tensors are uniform[-1, 1]
    bufs = DeviceSet(probs, dist="normal" if args.workload == "packing" else "uniform")
    stream = torch.cuda.current_stream()
    bytes_step = sum(p.algorithmic_bytes() for p in probs)

    def step(events=None):
        for i, (p, pl) in enumerate(zip(probs, plans)):
            A, B = bufs.get(p, i)
            if events is not None:
                events[i][0].record(stream)
            pl.execute(A, B, stream)
            if events is not None:
                events[i][1].record(stream)

    def event_pass():
        # per-launch durations (CUDA events on the launching stream); the
        # device is kept busy while the host enqueues the first launches, so
        # that no event interval includes host time
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in probs]
        torch.cuda._sleep(20_000_000)
        step(ev)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    for _ in range(max(args.warmup, 3) if args.warmup >= 0 else 3):
        step()
    torch.cuda.synchronize()
    cost_model_ms = None
    if args.autotune:
        # the cost model's schedules, then the autotuner's (timed per plan on
        # scratch buffers of the same size)
        cost_model_ms = event_pass()
        t_tune = time.perf_counter()
        for pl in plans:
            pl.autotune(max_candidates=args.autotune)
        t_tune = time.perf_counter() - t_tune
        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize()
    per_case_ms = event_pass()

    # FP8 outputs with the scale supplied by the caller (no amax pre-pass):
    # the same plans, timed once more with a device scale set
    fp8_supplied = None
    if any(p.dtype_out == "e4m3" for p in probs):
        scale = torch.ones(1, dtype=torch.float32, device="cuda")
        for p, pl in zip(probs, plans):
            if p.dtype_out == "e4m3":
                pl.set_fp8_scale(scale)
        step()
        sup = event_pass()
        for p, pl in zip(probs, plans):
            if p.dtype_out == "e4m3":
                pl.set_fp8_scale(None)
        fp8_supplied = {f"{p.tag}/{p.dtype_in}>{p.dtype_out}": {
            "computed_scale_GBs": round(p.algorithmic_bytes() / (a * 1e-3) / 1e9, 1),
            "supplied_scale_GBs": round(p.algorithmic_bytes() / (b * 1e-3) / 1e9, 1)}
            for p, a, b in zip(probs, per_case_ms, sup) if p.dtype_out == "e4m3"}

    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(dev) if rank == 0 else None
    if clk:
        clk.start()
    l0 = ttc.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.profile_timed:
        torch.cuda.cudart().cudaProfilerStart()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if args.profile_timed:
        torch.cuda.cudart().cudaProfilerStop()
    launches = ttc.launch_count() - l0
    clocks = clk.stop() if clk else None
    ms_total = max_over_ranks(e0.elapsed_time(e1), world)
    if dist:
        tdist.barrier()
    ms_step = ms_total / args.steps
    value = job_rate(bytes_step, world, ms_step) / 1e9

    # dominant kernel: group launches by variant
    by_var = {}
    for p, pl, ms in zip(probs, plans, per_case_ms):
        v = pl.info()["kernel"]
        d = by_var.setdefault(v, {"ms": 0.0, "bytes": 0, "launches": 0})
        d["ms"] += ms
        d["bytes"] += p.algorithmic_bytes()
        d["launches"] += 1
    dom = max(by_var, key=lambda k: by_var[k]["ms"])
    peak, peak_kind = measured_peaks()
    kname = dom
    achieved = by_var[dom]["bytes"] / (by_var[dom]["ms"] * 1e-3) / 1e9
    tr = ncu_traffic(kname, args.workload)
    case_gbs = [p.algorithmic_bytes() / (ms * 1e-3) / 1e9 for p, ms in zip(probs, per_case_ms)]
    big = [g for p, g in zip(probs, case_gbs) if p.n * inputs.DTYPE_BYTES[p.dtype_in] >= (256 << 20)]

    if args.cases_out:
        with open(args.cases_out, "w") as f:
            json.dump([{"case": f"{p.tag}/{p.dtype_in}/b{p.beta}", "sizes": p.sizes, "perm": p.perm,
                        "canon": pl.info()["sizes"], "cperm": pl.info()["perm"], "kernel": pl.info()["kernel"],
                        "tile": pl.info()["tile"], "GBs": round(g, 1)}
                       for p, pl, g in zip(probs, plans, case_gbs)], f, indent=0)

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, probs, plans, bufs, stream, world)

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "value_GiB_per_s": round(value * 1e9 / 2 ** 30, 2),   # the unit of the paper's Eq. 2
        "dtype": "f32+f64" if args.workload == "sweep" else "+".join(sorted({p.dtype_in for p in probs})),
        "data": "synthetic (seeded uniform[-1,1], torch Philox on the device)",
        "config": {"workload": workload_desc(args.workload, probs), "transposes_per_step": len(probs),
                   "algorithmic_bytes_per_step": bytes_step, "l2": "inputs > L2 (256-512 MiB per tensor), "
                   "two alternating buffer sets" if args.workload == "sweep" else "see workload",
                   "parallelism": f"replicas x{world}", "autotune": bool(args.autotune)},
        "schedule": ({"autotuned_case_sum_GB/s": round(bytes_step / (sum(per_case_ms) * 1e-3) / 1e9, 1),
                      "cost_model_case_sum_GB/s": round(bytes_step / (sum(cost_model_ms) * 1e-3) / 1e9, 1),
                      "candidates_timed_per_plan": args.autotune, "tuning_wall_s": round(t_tune, 1)}
                     if cost_model_ms else None),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "kernel": kname, "launches": by_var[dom]["launches"],
                     "traffic": (tr["bytes_per_launch"] if tr else None),
                     "traffic_note": (tr.get("note") if tr else "no ncu capture of the current kernel source")},
        "per_variant": {k: {"GB/s": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1), "launches": v["launches"],
                            "ms": round(v["ms"], 3)} for k, v in by_var.items()},
        "cases": {"min_GBs": round(min(case_gbs), 1), "median_GBs": round(float(np.median(case_gbs)), 1),
                  "max_GBs": round(max(case_gbs), 1),
                  "frac_ge_256MiB_at_80pct_of_8TBs": (round(sum(g >= 6400 for g in big) / len(big), 3)
                                                      if big else None),
                  "frac_ge_256MiB_at_80pct_of_measured": (round(sum(g >= 0.8 * peak for g in big) / len(big), 3)
                                                          if big else None)},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
    }
    if args.workload in ("packing", "single4d"):
        out["per_case"] = [{"case": f"{p.tag}/{p.dtype_in}>{p.dtype_out}", "us": round(ms * 1e3, 2),
                            "GB/s": round(g, 1), "frac_of_peak": round(g / peak, 4), "kernel": pl.info()["kernel"]}
                           for p, pl, ms, g in zip(probs, plans, per_case_ms, case_gbs)]
    if args.workload == "packing":
        out["fp8_error"] = {f"{p.tag}/{p.dtype_in}>{p.dtype_out}": fp8_error_stats(p, pl, bufs.get(p, i), stream)
                            for i, (p, pl) in enumerate(zip(probs, plans)) if p.dtype_out == "e4m3"}
    if args.workload == "complex":
        out["fp64_pipe"] = fp64_roofline(probs, per_case_ms)
    if fp8_supplied:
        out["fp8"] = {"note": "algorithmic bytes n (s_A + s_B) in both columns; the computed scale also reads A "
                              "once more (amax pre-pass)", "cases": fp8_supplied}
    return out


def colmajor_view(flat, sizes, outer):
    """The (sub-)tensor of column-major sizes inside outer extents, as a
    strided torch view indexed [i0, i1, ...]."""
    st, acc = [], 1
    for s, o in zip(sizes, outer):
        st.append(acc)
        acc *= o
    return flat.as_strided(tuple(sizes), tuple(st))


def fp8_error_stats(p, pl, bufs, stream):
    """Error of one FP8 result (the scale computed on the device) against the
    exact value alpha*a: the product of two binary32 numbers is exact in
    binary64, so the reference is alpha_f * a in float64.  The plan runs once
    on the case's A; its E4M3 codes, dequantised with the scale it used, are
    compared element by element through the permutation (torch views of A's
    sub-tensor and of B)."""
    import torch
    A, B = bufs
    pl.execute(A, B, stream)
    scale_t = torch.zeros(1, dtype=torch.float32, device="cuda")
    pl.get_fp8_scale(scale_t, stream)
    torch.cuda.synchronize()
    scale = float(scale_t.item())
    outer_a = p.outer_a or p.sizes
    sizes_b = [p.sizes[k] for k in p.perm]
    outer_b = p.outer_b or sizes_b
    a = colmajor_view(A.view(torch.float32), p.sizes, outer_a).permute(*p.perm).to(torch.float64)
    ref = float(torch.tensor(p.alpha, dtype=torch.float32).item()) * a
    codes = colmajor_view(B.view(torch.uint8), sizes_b, outer_b)
    deq = codes.view(torch.float8_e4m3fn).to(torch.float64) * scale
    err = (deq - ref).abs()
    mag = ref.abs()
    rel = torch.where(mag > 0, err / torch.where(mag > 0, mag, torch.ones_like(mag)), torch.zeros_like(err))
    return {"scale": scale, "max_abs": float(err.max()), "max_rel": float(rel.max()),
            "rms": float(err.pow(2).mean().sqrt()), "max_abs_ref": float(mag.max()),
            "bound_ok": bool((err <= 2.0 ** -4 * mag + scale * 2.0 ** -10 + 1e-30).all())}


# FP64 pipe: nominal 1.25 TFLOP/s dense FP64 on GB300 = 0.625 T fused
# multiply-adds per second; a dependent-free FMA loop measured 505 G/s
FP64_FMA_PEAK_G = 625.0
FP64_FMA_MEASURED_G = 505.0


def fp64_fmas_per_element(p) -> int:
    """FP64-pipe instructions of the double-complex update per element: the
    products alpha_re * a run as integer code, the cross term of alpha_im and
    both beta terms are fused multiply-adds (two parts each)."""
    if "c128" not in (p.dtype_in, p.dtype_out):
        return 0
    a, b = complex(p.alpha), complex(p.beta)
    return 2 * (a.imag != 0) + 2 * (b != 0) + 2 * (b.imag != 0)


def fp64_roofline(probs, per_case_ms):
    """ALU roofline of the cases computed in double-complex: FP64-pipe fused
    multiply-adds per second against the pipe's peak."""
    ops = sum(p.n * fp64_fmas_per_element(p) for p in probs)
    ms = sum(t for p, t in zip(probs, per_case_ms) if fp64_fmas_per_element(p))
    if not ops or not ms:
        return None
    achieved = ops / (ms * 1e-3) / 1e9
    return {"bound": "alu", "unit": "G FP64 FMA/s", "achieved": round(achieved, 1), "peak": FP64_FMA_PEAK_G,
            "frac": round(achieved / FP64_FMA_PEAK_G, 4), "frac_of_measured_fma_loop": round(
                achieved / FP64_FMA_MEASURED_G, 4),
            "peak_source": "nominal 1.25 TFLOP/s FP64 / 2 per FMA; measured FMA loop 505 G/s",
            "cases": sum(1 for p in probs if fp64_fmas_per_element(p))}


def workload_desc(name, probs):
    if name == "sweep":
        return ("single transposes, N=2..6 x 8 seeded perms, 2^26 elems/tensor (+-1%), f32+f64, "
                "alpha=1.7, beta in {0,0.4}")
    if name == "single4d":
        return "4D f32 (32,40,24,36) perm (2,0,3,1) alpha=1 beta=0"
    if name == "pow2":
        return ("single transposes, N=2..6, power-of-two sizes, 2^26 elems/tensor, 1-2 seeded perms per N, "
                "f32+f64, alpha=1.7, beta=0")
    if name == "complex":
        return ("complex transposes c, z, cz, zc, N=2..6 x 2 seeded perms, 2^25 elems/tensor (+-1%: 256 MiB "
                "single-, 512 MiB double-complex), alpha=1.7-0.6i, beta in {0, 0.4+0.25i}")
    if name == "packing":
        return "GEMM packing 4096x2048 of 8192^2 f32 -> 256x128 panels, and (48,64,40,56) in (64,80,48,64) perm (1,3,0,2); -> bf16 / e4m3+scale"
    return name


def pack_buffers(probs, seed=0):
    """One device arena for all A's and one for all B's (256-byte aligned
    slices), filled with seeded uniform data."""
    import torch
    offs_a, offs_b, ta, tb = [], [], 0, 0
    for p in probs:
        offs_a.append(ta)
        offs_b.append(tb)
        ta += (p.vol_a * inputs.DTYPE_BYTES[p.dtype_in] + 255) // 256 * 256
        tb += (p.vol_b * inputs.DTYPE_BYTES[p.dtype_out] + 255) // 256 * 256
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    A = torch.empty(ta // 4, dtype=torch.float32, device="cuda").uniform_(-1, 1, generator=g)
    B = torch.empty(tb // 4, dtype=torch.float32, device="cuda").uniform_(-1, 1, generator=g)
    pa = [A.data_ptr() + o for o in offs_a]
    pb = [B.data_ptr() + o for o in offs_b]
    return A, B, pa, pb


def run_batch(args, rank, world):
    """Thousands of uneven transposes: one graph-launched persistent batch vs
    one ttc_execute call per transpose on the same stream."""
    import torch
    from paper_1607_01249_gb300 import build as ttc_build
    from paper_1607_01249_gb300 import ttc

    ttc_build.build()
    ttc.lib()
    torch.cuda.set_device(rank % max(torch.cuda.device_count(), 1))
    probs = inputs.batch_problems(args.batch_count)
    plans = [ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta) for p in probs]
    A, B, pa, pb = pack_buffers(probs)
    direct_min = ttc.Batch.DIRECT_MIN_DEFAULT
    batch = ttc.Batch().set_direct_threshold(direct_min)
    for pl, a, b in zip(plans, pa, pb):
        batch.add(pl, a, b)
    stream = torch.cuda.current_stream()
    bytes_step = sum(p.algorithmic_bytes() for p in probs)

    def timed(fn, steps, profile=False):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ttc.launch_count()
        if profile:
            torch.cuda.cudart().cudaProfilerStart()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if profile:
            torch.cuda.cudart().cudaProfilerStop()
        ms = e0.elapsed_time(e1) / steps
        return max_over_ranks(ms, world), (ttc.launch_count() - l0) // steps

    def per_call():
        for pl, a, b in zip(plans, pa, pb):
            pl.execute(a, b, stream)

    # the cost model's batch-body schedules, then (unless --autotune 0) the
    # timed choice among each plan's best few (ttc_batch_autotune, outside
    # the timed region), which the reported step uses
    tune = None
    if args.autotune > 0:
        ms_cm, _ = timed(lambda: batch.graph_launch(stream), max(1, args.steps // 2))
        ncand = min(args.autotune, 4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        retuned = batch.autotune(ncand, stream)
        torch.cuda.synchronize()
        tune = {"candidates_timed_per_plan": ncand, "plans": len(plans), "plans_retuned": retuned,
                "tuning_wall_s": round(time.perf_counter() - t0, 2),
                "cost_model_GB/s": round(job_rate(bytes_step, world, ms_cm) / 1e9, 2)}
    clk = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clk:
        clk.start()
    ms_b, launches_b = timed(lambda: batch.graph_launch(stream), args.steps, args.profile_timed)
    clocks = clk.stop() if clk else None
    ms_c, launches_c = timed(per_call, max(1, args.steps // 2))
    info = batch.info()
    value = job_rate(bytes_step, world, ms_b) / 1e9
    peak, peak_kind = measured_peaks()
    return {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_b, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic (seeded sizes/perms; uniform data)",
        "config": {"workload": f"batch of {len(probs)} transposes, N 2..5, 2^10..2^22 elements log-uniform, "
                               "f32/bf16 50/50, alpha=1, beta in {0,0.5}; one CUDA-graph launch per step",
                   "tiles": info["tiles"],
                   "direct_problems": sum(p.n >= direct_min for p in probs) if direct_min > 0 else 0,
                   "direct_threshold_elements": direct_min, "algorithmic_bytes_per_step": bytes_step,
                   "parallelism": f"replicas x{world}"},
        "batch": {"transposes_per_s": round(job_rate(len(probs), world, ms_b), 1), "ms": round(ms_b, 4),
                  "kernel_launches_per_step": launches_b},
        "per_call": {"transposes_per_s": round(job_rate(len(probs), world, ms_c), 1), "ms": round(ms_c, 4),
                     "GB/s": round(job_rate(bytes_step, world, ms_c) / 1e9, 2),
                     "kernel_launches_per_step": launches_c},
        "speedup_vs_per_call": round(ms_c / ms_b, 3),
        "schedule": tune if tune else "cost model (--autotune 0)",
        "roofline": {"bound": "hbm", "achieved": round(bytes_step / (ms_b * 1e-3) / 1e9, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(bytes_step / (ms_b * 1e-3) / 1e9 / peak, 4),
                     "kernel": "one graph launch: the batch_kernel launches (one per class)"
                               + (" + the side stream's single-plan kernels" if direct_min > 0 else ""),
                     "traffic": (ncu_traffic("step", "batch") or {}).get("bytes_per_launch")
                     if args.batch_count == 4096 and direct_min == ttc.Batch.DIRECT_MIN_DEFAULT else None},
        "gpu_launches": launches_b * args.steps,
        "clocks": clocks,
    }


def serve_trace(srv, ttc, trace, plans, pa, pb, paced: bool):
    """Submit the trace's requests at their arrival times (paced) or all at
    once, wait for every one, and return per-request latency from arrival
    (microseconds), the served wall time and the largest submission lag."""
    t0 = time.perf_counter() + 2e-3
    tickets, lag, sub_perf = [], 0.0, []
    for (ta, _), pl, a, b in zip(trace, plans, pa, pb):
        if paced:
            target = t0 + ta
            while time.perf_counter() < target:
                pass
        else:
            target = t0
        now = time.perf_counter()
        tickets.append(srv.submit(pl, a, b))
        sub_perf.append(now)
        lag = max(lag, now - target)
    srv.drain(600_000_000)
    lat, first, last, detail = [], None, None, []
    for (ta, _), t, sp in zip(trace, tickets, sub_perf):
        s_sub, s_admit, s_launch, s_done = srv.times(t)
        arrival = (t0 + ta) if paced else t0
        lat.append(((s_done - s_sub) + (sp - arrival)) * 1e6)
        detail.append(((s_admit - s_sub) * 1e6, (s_launch - s_admit) * 1e6, (s_done - s_launch) * 1e6))
        first = s_sub if first is None else min(first, s_sub)
        last = s_done if last is None else max(last, s_done)
    serve_trace.detail = detail
    return np.array(lat), last - first, lag


def run_serving(args, rank, world):
    """Requests arriving over time (Poisson), served by the continuous-batching
    server (ttc_server_*) and, for comparison, one launch per request in
    arrival order on one stream.  Plans and buffers stay on the device."""
    import torch
    from paper_1607_01249_gb300 import build as ttc_build
    from paper_1607_01249_gb300 import ttc

    ttc_build.build()
    ttc.lib()
    dev = rank % max(torch.cuda.device_count(), 1)
    torch.cuda.set_device(dev)
    trace = inputs.serving_requests(args.serve_count, seed=4, rate_per_s=args.serve_rate)
    probs = [p for _, p in trace]
    plans = [ttc.Plan(p.perm, p.sizes, p.dtype_in, p.dtype_out, p.alpha, p.beta, p.outer_a, p.outer_b)
             for p in probs]
    # A: one shared read-only region, each request reading a slice of it;
    # B: a buffer of its own per request (the results of concurrent requests
    # never share bytes)
    span_a = [p.vol_a * inputs.DTYPE_BYTES[p.dtype_in] for p in probs]
    span_b = [(p.vol_b * inputs.DTYPE_BYTES[p.dtype_out] + 255) // 256 * 256 for p in probs]
    region_a = max(max(span_a) + (64 << 20), 1 << 30)
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    A = torch.empty(region_a // 4, dtype=torch.float32, device="cuda").uniform_(-1, 1, generator=g)
    B = torch.zeros(sum(span_b) // 4, dtype=torch.float32, device="cuda")
    h = inputs.rng(12)
    pa = [A.data_ptr() + int(h.integers(0, (region_a - sa) // 256 + 1)) * 256 for sa in span_a]
    offs = np.concatenate([[0], np.cumsum(span_b)[:-1]]).astype(np.int64)
    pb = [B.data_ptr() + int(o) for o in offs]
    torch.cuda.synchronize()
    bytes_trace = sum(p.algorithmic_bytes() for p in probs)
    budget = int(args.serve_budget_gb * 1e9)
    arms = {"continuous": (args.serve_streams, args.serve_small_tiles), "per_call": (1, 0)}
    res = {}
    clk = ClockSampler(dev) if rank == 0 else None
    for name, (ns, small) in arms.items():
        warm = ttc.Server(budget, ns, small)         # plans' device resources, batch descriptions
        serve_trace(warm, ttc, trace, plans, pa, pb, paced=False)
        warm.close()
        srv = ttc.Server(budget, ns, small)
        l0 = ttc.launch_count()
        if clk and name == "continuous":
            clk.start()
        lat_all, lags, walls = [], [], []
        for _ in range(args.steps):
            lat, wall, lag = serve_trace(srv, ttc, trace, plans, pa, pb, paced=True)
            if args.serve_dump:
                with open(f"{args.serve_dump}.{name}.json", "w") as f:
                    json.dump([{"perm": p.perm, "sizes": p.sizes, "din": p.dtype_in, "dout": p.dtype_out,
                                "outer": p.outer_a is not None, "bytes": p.algorithmic_bytes(),
                                "kernel": pl.info()["kernel"], "lat_us": round(float(l), 1),
                                "queue_us": round(d[0], 1), "launch_us": round(d[1], 1), "run_us": round(d[2], 1)}
                               for p, pl, l, d in zip(probs, plans, lat, serve_trace.detail)], f)
            lat_all.append(lat)
            lags.append(lag)
            walls.append(wall)
        clocks = clk.stop() if (clk and name == "continuous") else None
        st = srv.stats()
        launches = ttc.launch_count() - l0
        srv.close()
        sat = ttc.Server(budget, ns, small)
        _, sat_wall, _ = serve_trace(sat, ttc, trace, plans, pa, pb, paced=False)
        sat.close()
        lat = np.concatenate(lat_all)
        res[name] = {
            "offered_req_per_s": args.serve_rate,
            "served_transposes_per_s": round(len(probs) / float(np.mean(walls)), 1),
            "served_GB/s": round(bytes_trace / float(np.mean(walls)) / 1e9, 1),
            "p50_us": round(float(np.percentile(lat, 50)), 1), "p90_us": round(float(np.percentile(lat, 90)), 1),
            "p99_us": round(float(np.percentile(lat, 99)), 1), "max_us": round(float(lat.max()), 1),
            "max_submit_lag_us": round(max(lags) * 1e6, 1),
            "saturated_transposes_per_s": round(len(probs) / sat_wall, 1),
            "saturated_GB/s": round(bytes_trace / sat_wall / 1e9, 1),
            "epochs": st["epochs"], "kernel_launches": launches, "peak_inflight_GB": round(st["peak_inflight_bytes"] / 1e9, 2),
            "streams": ns, "small_tiles": small, "clocks": clocks,
        }
        log(name, json.dumps(res[name]))
    c, q = res["continuous"], res["per_call"]
    return {
        "workload": (f"serving: {len(probs)} requests, Poisson {args.serve_rate:g} req/s, A 4 KiB..512 MiB "
                     "log-uniform, N 2..6, f32/f64/bf16 50/20/30, 10% packing f32->bf16 with outer sizes, "
                     f"admission budget {args.serve_budget_gb:g} GB; {args.steps} paced passes of the trace "
                     "per arm, host steady clock from arrival to detected completion"),
        "algorithmic_bytes_per_trace": bytes_trace,
        "continuous": c, "per_call": q,
        "p99_ratio_per_call_over_continuous": round(q["p99_us"] / c["p99_us"], 3),
        "saturated_speedup_vs_per_call": round(c["saturated_transposes_per_s"] / q["saturated_transposes_per_s"], 3),
    }


# FP32 SIMT peak from the unit counts and clock: 152 SMs x 128 FP32 lanes x
# 2 FLOP per FMA x 2.07 GHz
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def run_contraction(args, rank, world):
    """TTGT contractions (ttc_contraction_*): each case once with an exact
    FP32 GEMM and once with BF16 operands packed by the transposes (FP32
    accumulation); against a cuBLAS GEMM of the same m, n, k on operands that
    are already matrices (torch.mm), which is what TTGT adds its transposes
    to."""
    import torch
    from paper_1607_01249_gb300 import build as ttc_build
    from paper_1607_01249_gb300 import ttc

    ttc_build.build()
    ttc.lib()
    torch.cuda.set_device(rank % max(torch.cuda.device_count(), 1))
    torch.backends.cuda.matmul.allow_tf32 = False
    stream = torch.cuda.current_stream()
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    peak_bf16 = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            peak_bf16 = float(json.load(f)["bf16_tflops"])
    steps = max(args.steps, 1)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / steps, world)

    cases, tot_flop, tot_ms, launches = [], 0.0, 0.0, 0
    for c in inputs.contraction_cases():
        ext = c["extents"]
        sa, sb, sc = (tuple(ext[m] for m in c[k]) for k in ("modes_a", "modes_b", "modes_c"))
        A = torch.empty(int(np.prod(sa)), device="cuda").uniform_(-1, 1, generator=g)
        B = torch.empty(int(np.prod(sb)), device="cuda").uniform_(-1, 1, generator=g)
        C = torch.zeros(int(np.prod(sc)), device="cuda")
        row = {"case": c["tag"]}
        for gd in ("f32", "bf16"):
            con = ttc.Contraction(c["modes_a"], sa, c["modes_b"], sb, c["modes_c"], sc, "f32", gd, 1.0, 0.0)
            if args.autotune > 0:
                con.autotune(args.autotune, stream)     # the permute plans, before the first execution
            inf = con.info()
            flop = 2.0 * inf["m"] * inf["n"] * inf["k"]
            l0 = ttc.launch_count()
            ms = timed(lambda: con.execute(A, B, C, stream))
            launches += (ttc.launch_count() - l0) // (steps + max(args.warmup, 3))
            ms_cublas = None
            if gd == "bf16":
                # the timed comparison: the same K-major BF16 operands on cuBLAS
                con.use_cublas(True)
                ms_cublas = timed(lambda: con.execute(A, B, C, stream))
                con.use_cublas(False)
            mt = torch.float32 if gd == "f32" else torch.bfloat16
            X = torch.empty(inf["m"], inf["k"], device="cuda", dtype=mt).uniform_(-1, 1, generator=g)
            Y = torch.empty(inf["k"], inf["n"], device="cuda", dtype=mt).uniform_(-1, 1, generator=g)
            ms_gemm = timed(lambda: torch.mm(X, Y))
            del X, Y
            tf = world * flop / (ms * 1e-3) / 1e12
            peak = FP32_SIMT_PEAK_TFLOPS if gd == "f32" else peak_bf16
            row[gd] = {"m": inf["m"], "n": inf["n"], "k": inf["k"], "permuted": inf["permuted"],
                       "ms": round(ms, 4), "TFLOP/s": round(tf, 1), "gemm_only_ms": round(ms_gemm, 4),
                       "transpose_share": round(max(ms - ms_gemm, 0.0) / ms, 3),
                       "frac_of_peak": round(tf / world / peak, 3) if peak else None,
                       "gemm": "tcgen05 (this library)" if gd == "bf16" else "cuBLAS SIMT FP32 (pedantic)"}
            if gd == "bf16":
                row[gd]["gemm_tile"] = ttc.Contraction.GEMM_VARIANTS.get(con.gemm_variant(), "?")
            if ms_cublas:
                row[gd]["with_cublas_gemm_ms"] = round(ms_cublas, 4)
                row[gd]["speedup_vs_cublas_gemm"] = round(ms_cublas / ms, 3)
            tot_flop += flop
            tot_ms += ms
            con.close()
        cases.append(row)
        del A, B, C
    value = world * tot_flop / (tot_ms * 1e-3) / 1e12
    return {
        "metric": "TTGT tensor contraction TFLOP/s (2 m n k per contraction)", "value": round(value, 2),
        "unit": "TFLOP/s", "n_gpus": world, "steps": steps, "warmup": args.warmup,
        "ms_per_step": round(tot_ms, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (exact FP32 GEMM) + f32 packed to bf16 (FP32 accumulation)",
        "data": "synthetic (uniform[-1,1], torch Philox on the device)",
        "config": {"workload": "contractions " + ", ".join(c["tag"] for c in inputs.contraction_cases()),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "fp32 SIMT / bf16 tensor", "fp32_peak_tflops": round(FP32_SIMT_PEAK_TFLOPS, 1),
                     "fp32_peak_source": "152 SMs x 128 lanes x 2 x 2.07 GHz",
                     "bf16_peak_tflops": peak_bf16, "bf16_peak_source": "MEASURED_PEAKS.json bf16_tflops"},
        "cases": cases, "gpu_launches": launches,
    }


def run_packed_gemm(args, rank, world):
    """The GEMM that consumes the packing routine (ttc_packed_gemm_*: gather,
    BF16 rounding and tcgen05.mma in one kernel) against the unfused path:
    the permute plan writes the BF16 panel to memory, then a cuBLAS BF16
    GEMM (torch.mm) reads it."""
    import torch
    from paper_1607_01249_gb300 import build as ttc_build
    from paper_1607_01249_gb300 import ttc

    ttc_build.build()
    ttc.lib()
    torch.cuda.set_device(rank % max(torch.cuda.device_count(), 1))
    stream = torch.cuda.current_stream()
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    peak = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            peak = float(json.load(f)["bf16_tflops"])
    steps = max(args.steps, 1)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / steps, world)

    cases, tot_flop, tot_ms, launches = [], 0.0, 0.0, 0
    for c in inputs.packed_gemm_cases():
        oa = c["outer"] or c["sizes"]
        A = torch.empty(int(np.prod(oa)), device="cuda").uniform_(-1, 1, generator=g)
        gemm = ttc.PackedGemm(c["perm"], c["sizes"], c["rank_m"], c["n"], 1.0, c["outer"])
        inf = gemm.info()
        M, N, K = inf["m"], inf["n"], inf["k"]
        B = torch.empty(K * N, device="cuda").uniform_(-1, 1, generator=g).to(torch.bfloat16)
        C = torch.empty(M * N, device="cuda")
        l0 = ttc.launch_count()
        ms = timed(lambda: gemm.execute(A, B, C, stream))
        launches += (ttc.launch_count() - l0) // (steps + max(args.warmup, 3))
        gemm.check()
        plan = ttc.Plan(c["perm"], c["sizes"], "f32", "bf16", outer_a=c["outer"])
        P = torch.empty(M * K, device="cuda", dtype=torch.bfloat16)
        Bt, Pt = B.view(N, K), P.view(K, M)
        # cuBLAS with an FP32 result where this torch has it, else a BF16 result
        # (half the result bytes: favours the unfused path)
        try:
            torch.mm(Bt, Pt, out_dtype=torch.float32)
            mm_out = "f32"
        except (TypeError, RuntimeError):
            mm_out = "bf16"

        def unfused():
            plan.execute(A, P, stream)
            if mm_out == "f32":
                torch.mm(Bt, Pt, out_dtype=torch.float32)
            else:
                torch.mm(Bt, Pt)

        ms_unfused = timed(unfused)
        ms_pack = timed(lambda: plan.execute(A, P, stream))
        flop = 2.0 * M * N * K
        tf = world * flop / (ms * 1e-3) / 1e12
        row = {"case": c["tag"], "m": M, "n": N, "k": K, "fused_ms": round(ms, 4),
               "fused_TFLOP/s": round(tf, 1), "unfused_ms": round(ms_unfused, 4),
               "unfused_pack_ms": round(ms_pack, 4), "unfused_gemm_result": mm_out,
               "unfused_TFLOP/s": round(world * flop / (ms_unfused * 1e-3) / 1e12, 1),
               "speedup_vs_unfused": round(ms_unfused / ms, 3),
               "frac_of_bf16_peak": round(tf / world / peak, 3) if peak else None}
        if K % 16 == 0:
            # E4M3 operands (P packed as codes with a per-tensor scale, Bm as
            # codes): kind::f8f6f4; its peak is the measured BF16 one times the
            # nominal FP8/BF16 ratio (4.5 / 2.25)
            B8 = torch.full((K * N,), 0x38, dtype=torch.uint8, device="cuda")
            sp = torch.full((1,), 0.01, device="cuda")
            sb = torch.full((1,), 0.5, device="cuda")
            gemm.set_fp8(sp, sb)
            ms8 = timed(lambda: gemm.execute(A, B8, C, stream))
            gemm.check()
            gemm.set_fp8(None, None)
            tf8 = world * flop / (ms8 * 1e-3) / 1e12
            row["fp8"] = {"fused_ms": round(ms8, 4), "fused_TFLOP/s": round(tf8, 1),
                          "frac_of_fp8_peak": round(tf8 / world / (2 * peak), 3) if peak else None,
                          "fp8_peak_source": "2 x MEASURED_PEAKS.json bf16_tflops (nominal 4.5 / 2.25)"}
            del B8
        cases.append(row)
        tot_flop += flop
        tot_ms += ms
        del A, B, C, P
        gemm.close()
    value = world * tot_flop / (tot_ms * 1e-3) / 1e12
    return {"metric": "packed-operand GEMM TFLOP/s (2 m n k)", "value": round(value, 2), "unit": "TFLOP/s",
            "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": round(tot_ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 operands (f32 A packed on the fly), f32 accumulation",
            "data": "synthetic (uniform[-1,1], torch Philox on the device)",
            "config": {"workload": "packed GEMM " + ", ".join(c["tag"] for c in inputs.packed_gemm_cases()),
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "tensor", "peak": peak, "unit": "TFLOP/s",
                         "achieved": round(value / world, 1), "frac": round(value / world / peak, 4) if peak else None,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)"},
            "cases": cases, "gpu_launches": launches}


def run_serving_line(args, rank, world):
    s = run_serving(args, rank, world)
    c = s["continuous"]
    peak, _ = measured_peaks()
    return {
        "metric": METRIC, "value": c["saturated_GB/s"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": 1, "ms_per_step": round(1e3 * args.serve_count / c["served_transposes_per_s"], 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64+bf16",
        "data": "synthetic (seeded trace; uniform data)",
        "config": {"workload": s["workload"], "parallelism": f"replicas x{world}",
                   "timing": "host steady clock (served throughput and latency are host-observed)"},
        "serving": s,
        "roofline": {"bound": "hbm", "achieved": c["saturated_GB/s"], "peak": peak, "unit": "GB/s",
                     "frac": round(c["saturated_GB/s"] / peak, 4), "kernel": "whole served trace",
                     "traffic": None},
        "gpu_launches": c["kernel_launches"],
        "clocks": c["clocks"],
    }


def run_e2e(args, probs, plans, bufs, stream, world):
    """Same metric with host (pinned) inputs: every step copies A (and B when
    beta != 0) host->device, runs the plan, and copies B back, for every
    transpose of the workload.  The transposes are independent, so the copies
    of one overlap the kernel of the next and the read-back of the previous
    one (three streams; the two alternating device and host buffer sets are
    reused only after their previous read-back has finished)."""
    import torch
    host = {}
    for key, sets in bufs.bufs.items():
        for j in range(2):
            A, B = sets[j]
            hA = torch.empty(A.numel(), dtype=A.dtype, pin_memory=True)
            hB = torch.empty(B.numel(), dtype=B.dtype, pin_memory=True)
            hA.copy_(A.cpu())
            hB.copy_(B.cpu())
            host[(key, j)] = (hA, hB)
    h2d = d2h = 0
    for p in probs:
        ea, eb = torch.empty(0, dtype=storage_torch(p.dtype_in)).element_size(), \
            torch.empty(0, dtype=storage_torch(p.dtype_out)).element_size()
        h2d += p.vol_a * ea + (p.vol_b * eb if p.beta != 0 else 0)
        d2h += p.vol_b * eb
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    last_out = {}

    def step():
        for i, (p, pl) in enumerate(zip(probs, plans)):
            key = (p.dtype_in, p.dtype_out)
            A, B = bufs.get(p, i)
            hA, hB = host[(key, i % 2)]
            ev = last_out.get((key, i % 2))
            if ev is not None:
                s_in.wait_event(ev)          # this set's previous read-back is done
            with torch.cuda.stream(s_in):
                A[:p.vol_a].copy_(hA[:p.vol_a], non_blocking=True)
                if p.beta != 0:
                    B[:p.vol_b].copy_(hB[:p.vol_b], non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(s_in)
            stream.wait_event(ready)
            pl.execute(A, B, stream)
            done = torch.cuda.Event()
            done.record(stream)
            s_out.wait_event(done)
            with torch.cuda.stream(s_out):
                hB[:p.vol_b].copy_(B[:p.vol_b], non_blocking=True)
            back = torch.cuda.Event()
            back.record(s_out)
            last_out[(key, i % 2)] = back

    step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for _ in range(steps):
        step()
    s_in.wait_stream(s_out)
    s_in.wait_stream(stream)
    e1.record(s_in)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1) / steps
    ms = max_over_ranks(ms, world)
    bytes_step = sum(p.algorithmic_bytes() for p in probs)
    return {"value": round(job_rate(bytes_step, world, ms) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": round(ms, 3),
            "wall_s": round(wall, 3), "steps": steps,
            "copies": "pinned host buffers; H2D, kernel and D2H of consecutive transposes overlap on three streams"}


# ------------------------------------------------------ CPU oracle timing --

def oracle_slabs(p, A, B, threads):
    """Run the oracle on `threads` slabs of the problem (split along A's last
    index; each slab is itself a valid sub-tensor problem) in parallel threads
    (ctypes releases the GIL)."""
    import oracle
    N = len(p.sizes)
    last = p.sizes[-1]
    oA = list(p.outer_a or p.sizes)
    sB = p.sizes_b
    oB = list(p.outer_b or sB)
    strideA = int(np.prod(oA[:-1], dtype=np.int64))
    posB = p.perm.index(N - 1)
    strideB = int(np.prod(oB[:posB], dtype=np.int64))
    ODT = {"f32": oracle.F32, "f64": oracle.F64, "bf16": oracle.BF16, "e4m3": oracle.E4M3, "c64": oracle.C64,
           "c128": oracle.C128}
    chunks = np.array_split(np.arange(last), min(threads, last))

    def work(ch):
        if len(ch) == 0:
            return
        s0 = int(ch[0])
        sizes = list(p.sizes[:-1]) + [len(ch)]
        subA = A[s0 * strideA:]
        subB = B[s0 * strideB:]
        if p.dtype_in in ("c64", "c128"):
            oracle.permute_complex(p.perm, sizes, subA, subB, p.alpha, p.beta, ODT[p.dtype_in], ODT[p.dtype_out],
                                   oA, oB)
        else:
            oracle.permute(p.perm, sizes, subA, subB, p.alpha, p.beta, ODT[p.dtype_in], ODT[p.dtype_out],
                           oA, oB)

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(work, chunks))


def cpu_baseline(budget_s: float, probs, threads: int):
    """Time the oracle as it stands on a bounded sample of the workload: its
    cases at full size, taken in an order that spreads over N, perm and dtype,
    until budget_s seconds of oracle time are spent (the input buffers are
    generated once per dtype and sliced per case)."""
    import oracle
    oracle.build()
    pool = {}
    for p in probs:
        for dt, v in ((p.dtype_in, p.vol_a), (p.dtype_out, p.vol_b)):
            pool[dt] = max(pool.get(dt, 0), v)
    bufs = {dt: inputs.tensor_for(dt, v, 1) for dt, v in pool.items()}
    done_bytes, t_total, names = 0, 0.0, []
    stride = 7 if len(probs) % 7 else 11
    for i in range(4 * len(probs)):
        p = probs[(i * stride) % len(probs)]
        A = bufs[p.dtype_in][:p.vol_a]
        B = bufs[p.dtype_out][:p.vol_b].copy()
        t0 = time.perf_counter()
        oracle_slabs(p, A, B, threads)
        t_total += time.perf_counter() - t0
        done_bytes += p.algorithmic_bytes()
        names.append(f"{p.tag}/{p.dtype_in}/b{p.beta}")
        if t_total > budget_s:
            break
    shown = ", ".join(names[:6]) + (", ..." if len(names) > 6 else "")
    return {"value": round(done_bytes / t_total / 1e9, 3), "unit": "GB/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(names)} runs over the workload's {len(probs)} cases at full size ({shown}), "
                      f"{t_total:.1f} s of oracle time on {threads} threads (slabs along the last index)"}


def run_reference(args, rank, world):
    if args.workload in ("contraction", "packgemm"):
        return {"impl": "reference", "unavailable": "the GEMM workloads have no timed CPU arm (their oracles are "
                                                    "numpy contractions in float64, test references only)"}
    probs = workload_problems(args.workload, args.target, args.only)
    threads = os.cpu_count() or 1
    import oracle
    oracle.build()
    # warm-up steps: small
    per_step = []
    for s in range(args.warmup + args.steps):
        p = probs[(s * 7) % len(probs)]
        A = inputs.tensor_for(p.dtype_in, p.vol_a, 1)
        B = inputs.tensor_for(p.dtype_out, p.vol_b, 2)
        t0 = time.perf_counter()
        oracle_slabs(p, A, B, threads)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            per_step.append((p.algorithmic_bytes(), dt))
    tot_b = sum(b for b, _ in per_step)
    tot_t = sum(t for _, t in per_step)
    value = tot_b / tot_t / 1e9
    sample = (f"each step = one full-size case of the workload (rotating), oracle on {threads} host threads")
    return {"metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * tot_t / len(per_step), 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (oracle arithmetic)",
            "data": "synthetic (seeded uniform[-1,1])", "impl": "reference",
            "config": {"workload": workload_desc(args.workload, probs), "parallelism": "host threads"},
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "pow2", "complex", "single4d", "packing", "batch", "serving", "contraction",
                             "packgemm"])
    ap.add_argument("--serve-count", type=int, default=1500)
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-budget-gb", type=float, default=40.0)
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--serve-small-tiles", type=int, default=1024)
    ap.add_argument("--serve-dump", default="", help="write per-request latencies (JSON) to <path>.<arm>.json")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--autotune", type=int, default=24,
                    help="time up to this many candidates per plan before the timed steps (0: cost model only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="default workload: skip the batched-launch summary")
    ap.add_argument("--no-pow2", action="store_true", help="default workload: skip the power-of-two-sizes row")
    ap.add_argument("--no-serving", action="store_true", help="default workload: skip the serving summary")
    ap.add_argument("--no-complex", action="store_true", help="default workload: skip the complex-types row")
    ap.add_argument("--no-contraction", action="store_true", help="default workload: skip the TTGT contraction row")
    ap.add_argument("--no-packing", action="store_true",
                    help="default workload: skip the single-4D and GEMM-packing rows")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--target", type=int, default=1 << 26,
                    help="elements per tensor of the sweep (the complex workload takes half)")
    ap.add_argument("--only", default="", help="comma-separated case tags of the sweep or the complex workload "
                                               "(e.g. N5p3, C2p0/c128>c128)")
    ap.add_argument("--cases-out", default="", help="write per-case timings (JSON) to this file")
    ap.add_argument("--profile-timed", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
        tdist.init_process_group("nccl")
    if args.workload == "batch":
        out = run_batch(args, rank, world)
    elif args.workload == "contraction":
        out = run_contraction(args, rank, world)
    elif args.workload == "packgemm":
        out = run_packed_gemm(args, rank, world)
    elif args.workload == "serving":
        out = run_serving_line(args, rank, world)
    else:
        out = run_ours(args, rank, world)
        if args.workload == "sweep" and world == 1:
            # the other two headline patterns, summarised in the same line:
            # the batched launch and the server, each against one launch per
            # transpose on the same GPU
            import copy
            sub = copy.copy(args)
            sub.steps, sub.warmup = min(args.steps, 5), max(args.warmup, 3)
            if not args.no_pow2:
                # the same shapes with power-of-two sizes (a separate row, not
                # part of the headline value)
                pw = copy.copy(sub)
                pw.workload, pw.no_e2e, pw.cases_out, pw.only = "pow2", True, "", ""
                r = run_ours(pw, rank, world)
                out["pow2"] = {"workload": r["config"]["workload"], "GB/s": r["value"], "cases": r["cases"],
                               "per_variant": r["per_variant"], "timing": "CUDA events"}
            if not args.no_complex:
                # the paper's complex types (a separate row)
                cx = copy.copy(sub)
                cx.workload, cx.no_e2e, cx.cases_out, cx.only = "complex", True, "", ""
                r = run_ours(cx, rank, world)
                out["complex"] = {"workload": r["config"]["workload"], "GB/s": r["value"], "cases": r["cases"],
                                  "per_variant": r["per_variant"], "roofline_frac": r["roofline"]["frac"],
                                  "fp64_pipe": r.get("fp64_pipe"), "timing": "CUDA events"}
            if not args.no_packing:
                # the single 4D transpose and the GEMM-packing downcasts
                # (BF16, FP8 with the scale computed and supplied), each case
                # with its roofline fraction; FP8 results with their error
                # against the exact alpha*a
                s4 = copy.copy(sub)
                s4.workload, s4.no_e2e, s4.cases_out, s4.only = "single4d", True, "", ""
                r = run_ours(s4, rank, world)
                # (GB/s from the kernel's event time; the per-call loop's rate,
                # with the host's launch of each call, beside it)
                out["single4d"] = {"workload": r["config"]["workload"], "us": r["per_case"][0]["us"],
                                   "GB/s": r["per_case"][0]["GB/s"], "frac_of_peak": r["per_case"][0]["frac_of_peak"],
                                   "per_call_loop_GB/s": r["value"], "kernel": r["per_case"][0]["kernel"],
                                   "timing": "CUDA events"}
                pk = copy.copy(sub)
                pk.workload, pk.no_e2e, pk.cases_out, pk.only = "packing", True, "", ""
                r = run_ours(pk, rank, world)
                out["packing"] = {"workload": r["config"]["workload"], "GB/s": r["value"],
                                  "cases": r["per_case"], "fp8_supplied_scale": (r.get("fp8") or {}).get("cases"),
                                  "fp8_error": r.get("fp8_error"), "timing": "CUDA events"}
            if not args.no_contraction:
                pg = run_packed_gemm(sub, rank, world)
                out["packed_gemm"] = {"workload": pg["config"]["workload"], "TFLOP/s": pg["value"],
                                      "roofline": pg["roofline"], "cases": pg["cases"], "timing": "CUDA events"}
                ct = run_contraction(sub, rank, world)
                out["contraction"] = {"workload": ct["config"]["workload"], "TFLOP/s": ct["value"],
                                      "cases": ct["cases"], "timing": "CUDA events"}
            if not args.no_batch:
                b = run_batch(sub, rank, world)
                out["batch"] = {"workload": b["config"]["workload"], "GB/s": b["value"],
                                "transposes_per_s": b["batch"]["transposes_per_s"],
                                "per_call_transposes_per_s": b["per_call"]["transposes_per_s"],
                                "speedup_vs_per_call": b["speedup_vs_per_call"], "ms_per_step": b["ms_per_step"],
                                "roofline_frac": b["roofline"]["frac"], "schedule": b["schedule"],
                                "timing": "CUDA events"}
            if not args.no_serving:
                sub.steps = min(args.steps, 3)
                sv = run_serving(sub, rank, world)
                c, q = sv["continuous"], sv["per_call"]
                keys = ("served_transposes_per_s", "p50_us", "p90_us", "p99_us", "saturated_transposes_per_s",
                        "saturated_GB/s")
                out["serving"] = {"workload": sv["workload"], "continuous": {k: c[k] for k in keys},
                                  "per_call": {k: q[k] for k in keys},
                                  "p99_ratio_per_call_over_continuous": sv["p99_ratio_per_call_over_continuous"],
                                  "saturated_speedup_vs_per_call": sv["saturated_speedup_vs_per_call"],
                                  "timing": "host steady clock, arrival to detected completion"}
    if rank == 0:
        if not args.no_cpu and world == 1 and args.workload not in ("batch", "serving", "contraction", "packgemm"):
            out["cpu_baseline"] = cpu_baseline(args.cpu_budget,
                                               workload_problems(args.workload, args.target, args.only),
                                               os.cpu_count() or 1)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
