"""Benchmark: 10-phase 4DCT slices reconstructed per second (TNLM, Sec. 2.2).

Default workload (--workload large): one step reconstructs the four dose
scenarios of the 512 x 512 slice (0.8 mm pixels, 10 phases, 888 bins of
1 mm, source-isocentre 1000 mm, source-detector 1500 mm; d = 7, W = 15,
K = 100 outer iterations, M1 = 3 CGLS steps, M2 = 5 Gauss-Jacobi sweeps):
  (a) 360 views per phase at I0 = 5e3, (b) 90 views at I0 = 1e5,
  (c) 360 views at I0 = 1e5, (d) 90 views at I0 = 5e3
i.e. four tnlm_reconstruct calls, so value = 4 * steps * ranks / time.
--workload mid times the three 256 x 256 scenarios (d = 5, W = 11, K = 50)
instead; --workload batch the batched many-slice workload.

Each reconstruction is the whole TNLM algorithm box: the initial image by
FBP of all views (tnlm_fbp, step 1) followed by the K outer iterations
(tnlm_reconstruct: the first one launch by launch with the dominant kernel
class timed by CUDA events, the other K - 1 as graph replays).  Inputs are
synthetic (seeded phantom, analytic line integrals, Poisson noise).  After
the timed steps the last timed result of every scenario with a stored FP64
oracle result (tests/golden/large_<s>_k100.txt, same start and K) is
compared with it at the stored pixel positions (relative L2).  --impl
reference times the FP64 CPU oracle instead, on a bounded sample of the same
step.

Multi-GPU: slices are independent, so each rank reconstructs its own
slices (weak scaling); ranks only meet for the barrier and the max-time
reduction.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1009_1351_gb300 import synth  # noqa: E402

METRIC = "10-phase slices reconstructed/s at fixed accuracy; TNLM+projector % HBM roofline"
UNIT = "slices/s"
WORKLOADS = {
    "large": (("large_a", "large_b", "large_c", "large_d"),
              "512x512 px @0.8 mm, 10 phases, 888 bins @1 mm, SID 1000 / SDD 1500 mm; "
              "scenarios (a) 360 views I0=5e3, (b) 90 views I0=1e5, (c) 360 views I0=1e5, "
              "(d) 90 views I0=5e3; d=7, W=15, K=100, M1=3, M2=5, mu_hat=0.5, h=0.014"),
    "mid": (("mid_a", "mid_b", "mid_c"),
            "256x256 px @1.5 mm, 10 phases, 512 bins @1 mm, SID 1000 / SDD 1500 mm; "
            "scenarios (a) 360 views I0=1e4, (b) 60 views I0=1e6, (c) 60 views I0=1e4; "
            "d=5, W=11, K=50, M1=3, M2=5, mu_hat=0.5, h=0.01"),
}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"tnlm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work of the kernels (for the roofline)
# ---------------------------------------------------------------------------
def system_nnz(g) -> int:
    """Number of non-zero system-matrix entries (pixels crossed by each ray),
    counted from the ray geometry: a segment inside the image square crosses
    1 + (# vertical grid lines) + (# horizontal grid lines) pixels."""
    src, d = synth.ray_endpoints(g)
    sx, sy, ux, uy = src[..., 0] / g.pixel_mm, src[..., 1] / g.pixel_mm, d[..., 0], d[..., 1]
    hx, hy = g.nx / 2.0, g.ny / 2.0
    lo = np.full(sx.shape, -np.inf)
    hi = np.full(sx.shape, np.inf)
    for s, u, h in ((sx, ux, hx), (sy, uy, hy)):
        with np.errstate(divide="ignore", invalid="ignore"):
            t0, t1 = (-h - s) / u, (h - s) / u
        lo = np.maximum(lo, np.where(u == 0, -np.inf, np.minimum(t0, t1)))
        hi = np.minimum(hi, np.where(u == 0, np.inf, np.maximum(t0, t1)))
    hit = hi > lo
    xa, xb = sx + lo * ux + hx, sx + hi * ux + hx
    ya, yb = sy + lo * uy + hy, sy + hi * uy + hy
    cx = np.abs(np.floor(np.clip(xb, 0, g.nx - 1e-9)) - np.floor(np.clip(xa, 0, g.nx - 1e-9)))
    cy = np.abs(np.floor(np.clip(yb, 0, g.ny - 1e-9)) - np.floor(np.clip(ya, 0, g.ny - 1e-9)))
    return int(np.where(hit, 1 + cx + cy, 0).sum())


def roofline_units(case, cls: str):
    """(algorithmic amount per launch, unit, bound) of a kernel class."""
    g, p = case.geom, case.params
    N, L2 = g.n_phases, g.nx * g.ny
    W2 = p.window * p.window
    if cls == "gj":
        # one Gauss-Jacobi sweep reads each stored distance once (pair-centric
        # storage, second direction served by L2) plus g, u, minima and writes u
        b = 4 * N * L2 * W2 + 4 * N * L2 * (1 + 2 + 2 + 1)
        return b, "GB/s", "hbm"
    if cls == "weights":
        b = 4 * N * L2 * W2 + 4 * N * L2 * (2 + 2 + 1)
        return b, "GB/s", "hbm"
    if cls in ("project", "backproject"):
        # per non-zero of A (one segment update): 1 FMA + 6 ALU operations to form
        # the entry (position, floor, fraction, row index, bounds), i.e. 7 lane
        # operations of the FP32 pipe
        return 7.0 * system_nnz(g), "Tops/s", "alu"
    return None, None, None


def measured_traffic(cls: str, case_names):
    """Mean DRAM bytes per launch of a kernel class over the given cases, from
    the ncu captures listed in profiles/traffic.txt, or None when a case is
    missing or a source file the capture depends on has changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    rows = {}
    for line in open(path):
        f = line.split()
        if len(f) != 6 or line.startswith("#"):
            continue
        rows[(f[0], f[1])] = (int(f[2]) + int(f[3]), f[4], f[5])
    vals = []
    for c in case_names:
        r = rows.get((cls, c))
        if r is None:
            return None
        # the source column lists the files the counters depend on, joined
        # by '+'; the hash is over their contents in that order
        h = hashlib.sha1()
        for part in r[1].split("+"):
            src = os.path.join(ROOT, part)
            if not os.path.exists(src):
                return None
            h.update(open(src, "rb").read())
        if h.hexdigest()[:12] != r[2]:
            return None
        vals.append(r[0])
    return float(np.mean(vals))


def traffic_class(cls: str, mixed: bool) -> str:
    """Row name of a kernel class in profiles/traffic.txt: with mixed precision
    the weights class is the tensor-core kernel, which has rows of its own."""
    return "weights_tc" if mixed and cls == "weights" else cls


_ALU_PEAK = {}


def alu_peak_tops(device: int = 0):
    """FP32-pipe peak in T lane operations/s (an FMA counts as one operation,
    as in the per-nnz count): measured by the library's FMA microbenchmark
    (tnlm_measure_peaks) on the device, once per process.  Returns (peak,
    source)."""
    if device not in _ALU_PEAK:
        try:
            import paper_1009_1351_gb300 as tn
            _ALU_PEAK[device] = (tn.tnlm_measure_peaks(device)["fp32_ops"] / 1e12,
                                 "measured: FP32 FMA microbenchmark (tnlm_measure_peaks)")
        except Exception as exc:     # no GPU: the derived figure, said so
            import torch
            sms = torch.cuda.get_device_properties(device).multi_processor_count if torch.cuda.is_available() else 152
            mhz = _peaks().get("sm_max_mhz", 2070.0)
            _ALU_PEAK[device] = (sms * 128 * mhz * 1e6 / 1e12,
                                 f"derived: SMs x 128 FP32 lanes x max SM clock ({exc})")
    return _ALU_PEAK[device]


# ---------------------------------------------------------------------------
# multi-rank aggregation (replicas: every rank reconstructs its own slices)
# ---------------------------------------------------------------------------
def max_over_ranks(vals, dev, world: int):
    """Element-wise maximum over all ranks (the slowest rank sets the time)."""
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def job_throughput(slices_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job slices per second: all ranks' slices over the slowest rank's time."""
    return slices_per_rank * steps * world / (max_ms / 1e3)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_1009_1351_gb300 as tn

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    scenarios, workload = WORKLOADS[args.workload]
    cases = [synth.case(s) for s in scenarios]
    mixed = args.precision == "mixed" and args.precision_set
    if mixed:
        cases = [dataclasses.replace(c, params=dataclasses.replace(c.params, precision=tn.PREC_MIXED))
                 for c in cases]
        workload += "; patch-distance cross terms as split-FP16 tensor-core products (mixed precision)"
    slices = []
    for c in cases:
        d = synth.make_inputs(c)
        geo = tn.tnlm_create_geometry(c.geom, device=local)
        y = torch.tensor(d["y"], dtype=torch.float32, device=dev)
        w = torch.tensor(d["w"], dtype=torch.float32, device=dev)
        f0 = torch.full((10, c.geom.ny, c.geom.nx), 0.01, dtype=torch.float32, device=dev)
        slices.append(dict(case=c, geo=geo, y=y, w=w, f0=f0, f=f0.clone(),
                           hy=torch.tensor(d["y"], dtype=torch.float32).pin_memory(),
                           hw=torch.tensor(d["w"], dtype=torch.float32).pin_memory(),
                           hf0=f0.cpu().pin_memory(), hout=torch.empty_like(f0, device="cpu").pin_memory()))
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(int(256 * 2 ** 20 / 4), dtype=torch.float32, device=dev)

    # Each reconstruction runs its first outer iteration launch by launch,
    # with the timed kernel classes bracketed by CUDA events, and the other
    # K - 1 as replays of the captured one-iteration graph.  The split is
    # exact: a reconstruction resumes bitwise where the previous call ended,
    # and eager launches and graph replays give bitwise the same result.
    for s in slices:
        k = s["case"].params.k_outer
        s["p_first"] = synth.Params(**{**s["case"].params.__dict__, "k_outer": 1})
        s["p_rest"] = synth.Params(**{**s["case"].params.__dict__, "k_outer": k - 1})
    timed_classes = [tn.KCLASSES]

    def step():
        for s in slices:
            tn.tnlm_fbp(s["geo"], s["y"], s["f"], stream=stream)
            tn.tnlm_profile_enable(s["geo"], timed_classes[0])
            tn.tnlm_reconstruct(s["geo"], s["p_first"], s["y"], s["w"], s["f"], report=False,
                                stream=stream)
            tn.tnlm_profile_enable(s["geo"], ())
            tn.tnlm_reconstruct(s["geo"], s["p_rest"], s["y"], s["w"], s["f"], report=False,
                                stream=stream)

    # warm-up, with every kernel class timed to find the dominant one
    for _ in range(max(args.warmup, 3)):
        step()
    # launch counters cover every outer iteration, the event times only the
    # first one: the timed launches are the counts divided by K
    prof, prof_n = {}, {}
    for s in slices:
        kk = s["case"].params.k_outer
        for k, v in tn.tnlm_profile_read(s["geo"]).items():
            prof[k] = prof.get(k, 0.0) + v["ms"]
            prof_n[k] = prof_n.get(k, 0) + v["launches"] / kk
    dominant = max(prof, key=prof.get)
    timed_classes[0] = (dominant,)
    for s in slices:
        tn.tnlm_profile_read(s["geo"])          # reset counters

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()                            # evict L2 between steps (not timed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    total_ms = float(sum(times))
    if world > 1:
        dist.barrier()
    kernel = {"ms": 0.0, "launches": 0}
    launches = 0
    for s in slices:
        r = tn.tnlm_profile_read(s["geo"])
        kernel["ms"] += r[dominant]["ms"]
        kernel["launches"] += r[dominant]["launches"] / s["case"].params.k_outer
        launches += sum(v["launches"] for v in r.values())
        tn.tnlm_profile_enable(s["geo"], ())

    # accuracy of the last timed result of every scenario with a stored FP64
    # oracle result (same FBP start, same K), at the stored pixel positions
    accuracy = []
    if rank == 0:
        from tests.golden import make_golden
        for s in slices:
            gold = make_golden.read_large(s["case"].name)
            if gold is None or s["case"].params.k_outer != make_golden.LARGE_K:
                continue
            pix = np.array([p[:3] for p in gold[1]], dtype=np.int64)
            want = np.array([p[3] for p in gold[1]])
            got = s["f"][pix[:, 0], pix[:, 1], pix[:, 2]].double().cpu().numpy()
            accuracy.append({"case": s["case"].name, "samples": int(len(want)),
                             "rel_l2_vs_fp64_oracle": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
                             "max_abs": float(np.max(np.abs(got - want))),
                             "tolerance": 1e-3 if mixed else 1e-4})

    # end-to-end through the C ABI with host buffers (pinned), copies timed
    for s in slices:
        tn.tnlm_profile_read(s["geo"])
    e2e_times = []
    h2d = d2h = 0
    for it in range(max(1, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for s in slices:
            s["y"].copy_(s["hy"], non_blocking=True)
            s["w"].copy_(s["hw"], non_blocking=True)
            tn.tnlm_fbp(s["geo"], s["y"], s["f"], stream=stream)
            tn.tnlm_reconstruct(s["geo"], s["case"].params, s["y"], s["w"], s["f"], report=False,
                                stream=stream)
            s["hout"].copy_(s["f"], non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_times.append(time.perf_counter() - t0)
    for s in slices:
        h2d += (s["hy"].numel() + s["hw"].numel()) * 4
        d2h += s["hout"].numel() * 4

    total_ms, e2e_s = max_over_ranks([total_ms, statistics.median(e2e_times)], dev, world)
    n_slices = len(slices)
    value = job_throughput(n_slices, args.steps, world, total_ms)
    e2e_value = job_throughput(n_slices, 1, world, e2e_s * 1e3)

    if rank == 0:
        amount, unit, bound = roofline_units(cases[0], dominant)
        per_launch_ms = kernel["ms"] / max(kernel["launches"], 1)
        peaks = _peaks()
        roof = None
        if amount is not None:
            # the dominant class's launches run over all three scenarios; report the
            # 360-view scenario's work divided by its launch time share
            if unit == "GB/s":
                amt = np.mean([roofline_units(c, dominant)[0] for c in cases])
                achieved = amt / (per_launch_ms / 1e3) / 1e9
                peak = peaks.get("hbm_gbs", 6800.0)
                src = "measured" if "hbm_gbs" in peaks else "fallback"
            else:
                amt = np.mean([roofline_units(c, dominant)[0] for c in cases])
                achieved = amt / (per_launch_ms / 1e3) / 1e12
                peak, src = alu_peak_tops(local)
            traffic = measured_traffic(traffic_class(dominant, mixed), scenarios)
            roof = {"bound": bound, "kernel": dominant, "achieved": round(achieved, 3),
                    "peak": round(peak, 1), "unit": unit, "frac": round(achieved / peak, 4),
                    "traffic": None if traffic is None else int(traffic),
                    "traffic_unit": "DRAM bytes per launch (ncu, profiles/traffic.txt)",
                    "peak_source": src, "launch_ms": round(per_launch_ms, 4)}
        # every kernel class, from the warm-up pass in which all classes were timed
        by_kernel = {}
        for cls in ("project", "backproject", "weights", "gj"):
            amt_c = np.mean([roofline_units(c, cls)[0] for c in cases])
            _, unit_c, bound_c = roofline_units(cases[0], cls)
            ms_c = prof.get(cls, 0.0) / max(prof_n.get(cls, 0), 1)
            if ms_c <= 0:
                continue
            if unit_c == "GB/s":
                ach, pk = amt_c / (ms_c / 1e3) / 1e9, peaks.get("hbm_gbs", 6800.0)
            else:
                ach, pk = amt_c / (ms_c / 1e3) / 1e12, alu_peak_tops(local)[0]
            tr = measured_traffic(traffic_class(cls, mixed), scenarios)
            by_kernel[cls] = {"bound": bound_c, "achieved": round(ach, 3), "peak": round(pk, 1),
                              "unit": unit_c, "frac": round(ach / pk, 4), "launch_ms": round(ms_c, 4),
                              "traffic": None if tr is None else int(tr)}
        out = {
            "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (patch cross terms f16x2 on tensor cores)" if mixed else "f32",
            "data": "synthetic (seeded ellipse phantom, analytic line integrals, Poisson noise)",
            "config": {"workload": workload, "slices_per_step": n_slices,
                       "l2": "flushed between steps (256 MiB write, untimed)",
                       "parity": ("GPU mixed precision vs FP64 oracle rel. L2 <= 1e-3 (tests/test_gpu_mixed.py)"
                                  if mixed else
                                  "GPU FP32 vs FP64 oracle rel. L2 <= 1e-4 (tests/test_gpu_full_k.py)"),
                       "parallelism": f"replicas x{world}"},
            "accuracy": accuracy,
            "clocks": clk, "gpu_launches": int(launches / args.steps),
            "e2e": {"value": round(e2e_value, 6), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": roof,
            "roofline_by_kernel": by_kernel,
            "kernel_ms_share": {k: round(v / max(sum(prof.values()), 1e-9), 4) for k, v in prof.items()},
        }
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.cpu_outer, scenarios, args.cpu_threads)
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# batched workload (not the default line): many uneven slices per step
# ---------------------------------------------------------------------------
def run_batch(args):
    import torch
    import paper_1009_1351_gb300 as tn

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    items = synth.batch_cases(args.batch_size, precision=1 if args.precision == "mixed" else 0)
    geos, params, ys, ws, fs, f0s = [], [], [], [], [], []
    for c, off in items:
        d = synth.make_inputs(c, off)
        geos.append(tn.tnlm_create_geometry(c.geom))
        params.append(c.params)
        ys.append(torch.tensor(d["y"], dtype=torch.float32, device=dev))
        ws.append(torch.tensor(d["w"], dtype=torch.float32, device=dev))
        fs.append(torch.zeros((c.geom.n_phases, c.geom.ny, c.geom.nx), dtype=torch.float32, device=dev))
    stream = torch.cuda.current_stream(dev)
    tuned = {}

    def step():
        for g, y, f in zip(geos, ys, fs):
            tn.tnlm_fbp(g, y, f, stream=stream)
        tn.tnlm_reconstruct_batch(geos, params, ys, ws, fs, autotune=True, stream=stream)

    for _ in range(max(args.warmup, 1)):
        step()
    for (c, _), g, y, w, f in zip(items, geos, ys, ws, fs):
        key = (c.geom.nx, c.geom.n_views)
        if key not in tuned:
            tuned[key] = tn.tnlm_autotune(g, c.params, y, w, f)    # cached: no timing
    clocks = ClockSampler(0)
    torch.cuda.synchronize(dev)
    clocks.start()
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    total_ms = float(sum(times))
    n = len(items)
    # the same batch as n separate tnlm_reconstruct calls (one captured graph
    # per slice, launched one after another), for the batching speed-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for g, p, y, w, f in zip(geos, params, ys, ws, fs):
        tn.tnlm_fbp(g, y, f, stream=stream)
        tn.tnlm_reconstruct(g, p, y, w, f, report=False, stream=stream)
    e1.record(stream)
    e1.synchronize()
    seq_ms = e0.elapsed_time(e1)
    sizes = {}
    for c, _ in items:
        sizes[f"{c.geom.nx}^2 x {c.geom.n_views} views"] = sizes.get(f"{c.geom.nx}^2 x {c.geom.n_views} views", 0) + 1
    out = {"metric": METRIC, "value": round(n * args.steps / (total_ms / 1e3), 4), "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(total_ms / args.steps, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if args.precision == "fp32" else "f32 (patch cross terms f16x2 on tensor cores)",
           "data": "synthetic (seeded ellipse phantom, analytic line integrals, Poisson noise)",
           "config": {"workload": (f"batch of {n} 10-phase slices per step, sides from 256/384/512 "
                                   "(384 mm field), 60/90/180/360 views, I0 log-uniform 5e3..1e6, "
                                   "d=5, W=11, K=50, FBP start, "
                                   + ("tensor-core (split-FP16) patch distances" if args.precision == "mixed"
                                      else "FP32 patch distances")
                                   + "; one graph per outer iteration for all slices "
                                   "(tnlm_reconstruct_batch), launch shapes autotuned"),
                      "slices": sizes, "autotuned": {f"{k[0]}^2/{k[1]}v": v for k, v in tuned.items()},
                      "l2": "inputs far larger than L2", "parallelism": "batch x1"},
           "clocks": clk, "e2e": None, "cpu_baseline": None,
           "sequential": {"value": round(n / (seq_ms / 1e3), 4), "unit": UNIT,
                          "note": "same slices, one tnlm_reconstruct call after another"}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# CPU oracle (reported baseline, and the reference arm)
# ---------------------------------------------------------------------------
def _oracle_time(name: str, k_outer: int):
    """Time the FP64 oracle on one scenario: its FBP start and k_outer outer
    iterations.  Returns (FBP seconds, seconds per outer iteration, K)."""
    import oracle
    c = synth.case(name)
    d = synth.make_inputs(c)
    G = oracle.Geom(c.geom)
    p = synth.Params(**{**c.params.__dict__, "k_outer": k_outer})
    y32, w32 = d["y"].astype(np.float32), d["w"].astype(np.float32)
    t0 = time.perf_counter()
    f0 = oracle.fbp(G, y32)
    t1 = time.perf_counter()
    oracle.reconstruct(G, y32, w32, f0, p)
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / k_outer, c.params.k_outer


def _oracle_threads(n: int = 0) -> int:
    import oracle
    oracle.build()
    return oracle.threads(n if n > 0 else (os.cpu_count() or 1))


def cpu_baseline(k_outer: int, scenarios, threads: int = 0):
    """The FP64 oracle on the host cores: the FBP and k_outer of the K outer
    iterations of every scenario slice, outer iterations extrapolated
    linearly to K (slices/s = slices / sum of the per-slice times)."""
    n = _oracle_threads(threads)
    spent, t_slices = 0.0, 0.0
    for s in scenarios:
        tf, ti, kk = _oracle_time(s, k_outer)
        spent += tf + ti * k_outer
        t_slices += tf + ti * kk
    kk = synth.case(scenarios[0]).params.k_outer
    return {"value": round(len(scenarios) / t_slices, 6), "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": (f"FBP plus {k_outer} of the K={kk} outer iterations of each of the "
                       f"{len(scenarios)} scenario slices ({spent:.1f} s of FP64 oracle time on {n} "
                       f"threads), outer iterations extrapolated linearly to K={kk}")}


def run_reference(args):
    """Reference arm: the FP64 oracle as it stands on the host cores.  Step j
    times scenario j mod S (its FBP and one outer iteration); the value is
    S slices over the sum of the mean extrapolated per-slice times of the
    scenarios measured.  Warm-up steps run one outer iteration of the tiny
    64^2 workload."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    scenarios, workload = WORKLOADS[args.workload if args.workload in WORKLOADS else "large"]
    n = _oracle_threads(args.cpu_threads)
    for _ in range(args.warmup):
        _oracle_time("tiny", 1)
    per = {}
    spent_total = 0.0
    for j in range(args.steps):
        name = scenarios[j % len(scenarios)]
        tf, ti, kk = _oracle_time(name, 1)
        spent_total += tf + ti
        per.setdefault(name, []).append(tf + ti * kk)
    t_sum = sum(statistics.mean(v) for v in per.values())
    value = len(per) / t_sum
    kk = synth.case(scenarios[0]).params.k_outer
    sample = (f"per step: the FBP and 1 of the K={kk} outer iterations of one scenario slice "
              f"(in turn: {', '.join(scenarios)}), extrapolated linearly to K={kk}; value = scenarios "
              f"measured / sum of their mean per-slice times")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * spent_total / max(args.steps, 1), 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload, "slices_per_step": 1},
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": n, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-outer", type=int, default=1,
                    help="outer iterations of the oracle per scenario for cpu_baseline")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="oracle threads for cpu_baseline and the reference arm (0: all host cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=("large", "mid", "batch"), default="large",
                    help="large: the four 512^2 scenarios (default line); mid: the three 256^2 "
                         "scenarios; batch: many uneven slices")
    ap.add_argument("--batch-size", type=int, default=64)
    ap.add_argument("--precision", choices=("mixed", "fp32"), default=None,
                    help="patch distances (batch workload: mixed by default; others: fp32 by default)")
    args = ap.parse_args()
    args.precision_set = args.precision is not None
    if args.precision is None:
        args.precision = "mixed" if args.workload == "batch" else "fp32"
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
