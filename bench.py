#!/usr/bin/env python
"""Benchmark: point-centre pairs/s of the mixed-precision assignment step.

One step = the whole hot path over the resident synthetic batch, through the
library's C-ABI: quantise X and C, tensor-core screening with the reliability
test, direct-formula refinement and certified argmin (labels, min_dist),
then the centre update (Eq. (center)).  Default workload: X uniform[0,1)
1e6 x 128 fp32, C = 1024 distinct rows of X, BF16 cross term, rho = 5.

Prints one JSON line (rank 0): the device-resident step rate (`value`), the
screening kernel against the measured BF16 roofline (`roofline`), the same
step end to end from pinned host buffers through km_lloyd_step_host (`e2e`),
the oracle on the host cores (`cpu_baseline`), the plain FP64 path on a row
sample (`fp64_path`), the served stream's latencies (`serving`), the
distance-matrix precision modes in the structure of the paper's Tables 6.1 /
6.2 (`table6`), clustering quality in the structure of Tables 6.3-6.7
(`quality`), the free-running config-3 SSE trajectories (`c3_trajectory`), SM clocks
sampled during the timed region (`clocks`) and the library's own launch count
(`gpu_launches`).  `--impl reference` times the CPU oracle instead (on a
bounded sample of the same workload).  Multi-GPU (torchrun): independent
replicas, one per GPU, no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (generator, n, d, k, description)
    "c2a": ("uniform_pairs", 1_000_000, 128, 1024,
            "dist+argmin, X uniform[0,1) 1e6 x 128 fp32, C = 1024 distinct rows of X"),
    "c2b": ("cancellation", 1_000_000, 128, 1024,
            "dist+argmin, X = 1e3 + N(0, 1e-2^2) 1e6 x 128 fp32, C = 1024 distinct rows of X"),
    "c3": ("gaussian_mixture", 4_000_000, 64, 256,
           "Lloyd iteration, Gaussian mixture 4e6 x 64 fp32, k = 256 (centre coordinates N(0, 25), cluster std "
           "log-uniform [0.1, 2]), C = 256 distinct rows of X"),
    "c4": ("voronoi_image", 4096 * 4096, 5, 16,
           "Lloyd iteration, 4096 x 4096 Voronoi image (16 regions, colour + N(0, 0.02^2)), features RGB + xy, "
           "d = 5, k = 16"),
}
METRIC = "point-center pairs/s (dist+argmin)"


def _direct_kernel_name(low: str, d: int, k: int) -> str:
    """The direct-formula kernel the library launches for this shape (the
    same choice as its launcher: small d with C in shared memory, the tiled
    FP32 kernel for 16 <= d <= 128 with d % 4 == 0, else one thread per row)."""
    if low == "fp64":
        return "k_direct_assign<double>"
    if d <= 8 and k * d * 4 <= 32 * 1024:
        return "k_direct_small<%d>" % d
    if d % 4 == 0 and 16 <= d <= 128:
        return "k_direct_tiled"
    return "k_direct_assign<float>"


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value of x over all ranks (the job's time is its slowest
    rank's); x itself when there is one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units processed by all ranks (weak scaling: the same work per rank) per second."""
    return units_per_rank * world / seconds


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def screen_source_hash() -> str:
    """First 16 hex digits of the SHA-256 of the screening kernel's sources."""
    csrc = os.path.join(ROOT, "paper_2407_12208_gb300", "csrc")
    hs = hashlib.sha256()
    for f in ("k_tc.cu", "common.cuh", "internal.h"):
        hs.update(open(os.path.join(csrc, f), "rb").read())
    return hs.hexdigest()[:16]


def _profile_traffic(n: int):
    """DRAM bytes per launch of the screening kernel from the committed ncu
    summary, scaled to n rows, if that summary was taken on the current
    kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "k_tc_screen_bf16_c2a.md")
    try:
        txt = open(path).read()
        h = screen_source_hash()
        mh = re.search(r"source_sha256_16:\s*([0-9a-f]+)", txt)
        mb = re.search(r"dram_bytes_per_row:\s*([0-9.eE+]+)", txt)
        if mh and mb and mh.group(1) == h:
            return float(mb.group(1)) * n
    except Exception:
        pass
    return None


def parse_clock_samples(path: str):
    """Median and largest SM clock and the throttle reasons seen in nvidia-smi
    samples (csv, no header: index, clocks.sm, clocks.max.sm, power.draw,
    active reasons, hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown,
    sw_power_cap); None without a usable sample."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() in ("active", "1"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


class ClockSampler:
    """nvidia-smi samples of SM clock / throttle reasons during the timed region."""

    def __init__(self, device_uuid: str | None, out_path: str | None = None):
        self.proc = None
        if out_path:
            self.out = out_path
        else:
            fd, self.out = tempfile.mkstemp(prefix="mpkm_clocks_", suffix=".csv")
            os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        cmd = ["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "100"]
        if device_uuid:
            cmd[1:1] = ["-i", device_uuid]
        try:
            os.makedirs(os.path.dirname(os.path.abspath(self.out)), exist_ok=True)
            self.f = open(self.out, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        return parse_clock_samples(self.out)


def run_ours(args):
    import numpy as np
    import torch

    import paper_2407_12208_gb300 as pkg
    from paper_2407_12208_gb300 import build as pbuild
    from paper_2407_12208_gb300 import workloads

    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world > 1:
        pbuild.build()
    gen, n, d, k, desc = WORKLOADS[args.workload]
    if args.n:
        n = args.n
        desc += " (first %d rows)" % n
    if gen == "voronoi_image":
        X, C = workloads.voronoi_image(4096, 4096, 16, k, seed=15 + rank)
        X = X[:n]
    else:
        X, C = getattr(workloads, gen)(n, d, k, seed=15 + rank)
    dev = torch.device("cuda", local)
    Xd = torch.from_numpy(X).to(dev)
    Cd = torch.from_numpy(C).to(dev)
    ctx = pkg.Context(local)
    p = pkg.params(args.low, "tc", rho=5.0)
    tensor_path = args.low in ("bf16", "fp16", "e4m3")
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    md = torch.empty(n, dtype=torch.float64, device=dev)
    Cn = torch.empty_like(Cd)
    counts = torch.empty(k, dtype=torch.int64, device=dev)
    ws = ctx.workspace(n, d, k, p)
    stream = torch.cuda.current_stream(dev)

    def step():
        # one iteration of Alg. 3: assignment then centre update (km_lloyd_step)
        ctx.lloyd_step(Xd, Cd, p, labels=labels, min_dist=md, C_new=Cn, counts=counts, ws=ws, stream=stream,
                       want_shift=False)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # the screening kernel's epilogue variant for this shape, timed on this data
    # (km_autotune: the fastest is kept for the shape class; results do not depend on it)
    tuned = None
    if tensor_path and not args.no_autotune:
        v, tms = ctx.autotune(Xd, Cd, p, ws=ws, stream=stream)
        tuned = {"variant": v, "ms_per_assign": dict(zip(("full", "half", "c32"), tms))}
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st0 = ctx.stats()
    # ---------------------------------------------------------- timed region
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clk = ClockSampler(uuid, args.clocks_csv)
    time.sleep(0.3)
    ctx.phase_times()
    ctx.set_profiling(True)
    l0 = ctx.launch_count()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = ctx.launch_count() - l0
    ctx.set_profiling(False)
    phases = ctx.phase_times()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_per_step = ms / args.steps
    pairs_per_step = float(n) * k
    value = whole_job_rate(pairs_per_step, world, ms_per_step / 1e3)

    # ------------------------------------------------ roofline of the screen kernel
    peaks = _measured_peaks()
    scr_ms, scr_cnt = phases["screen"]
    flops = 2.0 * n * k * d
    achieved = flops / (scr_ms / max(scr_cnt, 1) / 1e3) / 1e12 if scr_cnt else None
    # the timed region is well under a second: the burst figure applies
    if peaks and peaks.get("bf16_tflops"):
        peak = peaks["bf16_tflops"]
        peak_src = "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    else:
        peak, peak_src = 1900.0, "fallback"
    if args.low == "fp16":
        pass  # same nominal rate as bf16
    elif args.low == "e4m3":
        peak = peak * 2.0
        peak_src += " x2 (nominal fp8/bf16 ratio)"
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": _profile_traffic(n) if (args.workload == "c2a" and args.low == "bf16") else None,
            "kernel": "k_tc (tcgen05 screen)", "algorithmic_flops_per_launch": flops, "peak_source": peak_src}
    if not tensor_path:
        # direct-formula assignment (small d): bound by HBM, X read once, labels
        # and min_dist written
        dir_ms, dir_cnt = phases["direct"]
        nbytes = n * d * 4.0 + n * 12.0
        gbs = nbytes / (dir_ms / max(dir_cnt, 1) / 1e3) / 1e9 if dir_cnt else None
        hbm = (peaks or {}).get("hbm_gbs") or 6800.0
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": (gbs / hbm) if gbs else None,
                "traffic": None, "kernel": _direct_kernel_name(args.low, d, k),
                "algorithmic_bytes_per_launch": nbytes,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback"}

    # ------------------------------------------------------------- end to end
    e2e = None
    if args.only_step:
        args.no_fp64 = args.no_cpu_baseline = True
    Xh = torch.from_numpy(X).pin_memory() if not args.only_step else None
    Ch = torch.from_numpy(C).pin_memory()
    lab_h = torch.empty(n, dtype=torch.int32).pin_memory()
    md_h = torch.empty(n, dtype=torch.float64).pin_memory()
    Cn_h = torch.empty((k, d), dtype=torch.float32).pin_memory()
    cnt_h = torch.empty(k, dtype=torch.int64).pin_memory()
    e2e_steps = 0 if args.only_step else max(3, min(args.steps, 20))
    hws = ctx.host_workspace(n, d, k, p) if e2e_steps else None

    def e2e_step():
        # the public host-buffer call: X and C from pinned host memory, labels,
        # min_dist, the new centres and counts back to it (km_lloyd_step_host)
        ctx.lloyd_step_host(Xh, Ch, p, labels=lab_h, min_dist=md_h, C_new=Cn_h, counts=cnt_h, ws=hws, stream=stream,
                            want_shift=False)

    if e2e_steps:
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1) / max(e2e_steps, 1), world, dev)
    if e2e_steps:
        e2e = {"value": whole_job_rate(pairs_per_step, world, e2e_ms / 1e3), "unit": "pairs/s",
               "h2d_bytes_per_step": int(Xh.numel() * 4 + Ch.numel() * 4),
               "d2h_bytes_per_step": int(lab_h.numel() * 4 + md_h.numel() * 8 + Cn_h.numel() * 4 + cnt_h.numel() * 8),
               "ms_per_step": e2e_ms, "call": "km_lloyd_step_host"}

    stats = ctx.stats()
    # ------------------------------------------------- FP64 path, same GPU
    fp64 = None
    if not args.no_fp64:
        # the plain binary64 direct assignment on a row sample: one warm-up
        # call, then five timed calls (CUDA events each), the median reported
        rows = min(n, 65536)
        p64 = pkg.params("fp64")
        Xs = Xd[:rows]
        lab64 = torch.empty(rows, dtype=torch.int32, device=dev)
        md64 = torch.empty(rows, dtype=torch.float64, device=dev)
        ctx.assign(Xs, Cd, p64, labels=lab64, min_dist=md64, want_flagged=False)
        torch.cuda.synchronize()
        times = []
        for _ in range(5):
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            ctx.assign(Xs, Cd, p64, labels=lab64, min_dist=md64, stream=stream, want_flagged=False)
            g1.record(stream)
            torch.cuda.synchronize()
            times.append(g0.elapsed_time(g1) / 1e3)
        t64 = statistics.median(times)
        v64 = rows * float(k) / t64
        agree = bool(torch.equal(lab64, labels[:rows]))
        fp64 = {"value": v64, "unit": "pairs/s", "sample_rows": rows, "repeats": len(times),
                "ms_per_call": [t * 1e3 for t in times], "labels_equal_on_sample": agree,
                "mixed_over_fp64": value / world / v64}

    # ------------------------------------------------------- CPU oracle baseline
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        rows = args.cpu_rows
        t0 = time.perf_counter()
        olab, od1, _ = oracle.assign(X[:rows], C)
        oracle.update(X[:rows], olab, C, 1, od1)
        tc = time.perf_counter() - t0
        cpu = {"value": rows * float(k) / tc, "unit": "pairs/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "first %d of %d rows x %d centres (assign + centre update, binary64 direct)" % (rows, n, k),
               "seconds": tc}

    serving = None
    if rank == 0 and not args.only_step and not args.no_serving:
        serving = serving_leg(args, local)
    table6 = None
    if rank == 0 and not args.only_step and not args.no_table6:
        table6 = table6_leg(args, local)
    c3 = None
    if rank == 0 and not args.only_step and not args.no_c3:
        try:
            c3 = c3_trajectory_leg(args, local)
        except Exception as exc:
            c3 = {"error": "%s: %s" % (type(exc).__name__, exc)}
    quality = None
    if rank == 0 and not args.only_step and not args.no_quality:
        try:
            quality = quality_leg(args, local)
        except Exception as exc:  # a failing side leg must not lose the line
            quality = {"error": "%s: %s" % (type(exc).__name__, exc)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.low, "data": "synthetic",
            "config": {"workload": args.workload + ": " + desc, "n": n, "d": d, "k": k, "low": args.low,
                       "test": "tc", "rho": 5.0, "parallelism": "replicas" if world > 1 else "single",
                       "step": "km_lloyd_step: quantise X (+ max |x|), screen, refine, certified argmin, min_dist, exact centre update",
                       "l2": "inputs larger than L2 (X %d MB fp32, L2 126 MB)" % (n * d * 4 // 1000000)},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
            "fp64_path": fp64, "serving": serving, "table6": table6, "quality": quality, "c3_trajectory": c3, "autotune": tuned,
            "phases_ms_per_step": {k_: v[0] / max(args.steps, 1) for k_, v in phases.items()},
            "eta": stats["flagged"] / max(stats["pairs"], 1),
            "assign_stats": {kk: stats[kk] for kk in ("fp32_evals", "fp64_evals", "ambiguous_rows", "overflow_rows")},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


TABLE6_MODES = [
    # (label, low, test, fallback): the rows of Table 6.1 this library provides
    ("FP16->FP64", "fp16", "tc", "fp64"), ("FP16->FP32", "fp16", "tc", "fp32"), ("FP16->FP16", "fp16", "tc", "low"),
    ("BF16->FP64", "bf16", "tc", "fp64"), ("BF16->FP32", "bf16", "tc", "fp32"), ("BF16->BF16", "bf16", "tc", "low"),
    ("FP16->FP64 (Alg. 2 test)", "fp16", "paper", "fp64"), ("BF16->FP64 (Alg. 2 test)", "bf16", "paper", "fp64"),
    ("FP32->FP64 (Alg. 2)", "fp32x", "paper", "fp64"), ("FP32->FP32 (Alg. 2)", "fp32x", "paper", "fp32"),
    ("uniform FP16", "fp16", "off", "fp64"), ("uniform BF16", "bf16", "off", "fp64"),
    ("FP32 direct", "fp32", "tc", "fp64"), ("FP64 direct", "fp64", "tc", "fp64"),
]


# ------------------------------------------------------- clustering quality
# The measures of Section 6.2, written from their definitions: the adjusted
# Rand index, the adjusted mutual information (arithmetic normalisation, the
# expected mutual information under the hypergeometric model of Vinh, Epps
# and Bailey 2010), and Table 6.7's `Diff`: the share of labels that differ
# from a reference after the one-to-one matching of cluster ids that agrees
# most.
def contingency(a, b):
    import numpy as np
    ua, ia = np.unique(np.asarray(a), return_inverse=True)
    ub, ib = np.unique(np.asarray(b), return_inverse=True)
    m = np.bincount(ia.ravel() * len(ub) + ib.ravel(), minlength=len(ua) * len(ub))
    return m.reshape(len(ua), len(ub)).astype(np.int64)


def adjusted_rand_index(a, b) -> float:
    import numpy as np
    m = contingency(a, b)
    n = int(m.sum())
    c2 = lambda x: x * (x - 1) / 2.0
    sij = float(c2(m.astype(np.float64)).sum())
    sa = float(c2(m.sum(1).astype(np.float64)).sum())
    sb = float(c2(m.sum(0).astype(np.float64)).sum())
    expected = sa * sb / c2(float(n))
    top = 0.5 * (sa + sb)
    if top == expected:  # both partitions trivial in the same way
        return 1.0
    return (sij - expected) / (top - expected)


def _entropy(counts, n) -> float:
    import numpy as np
    p = counts[counts > 0] / float(n)
    return float(-(p * np.log(p)).sum())


def _expected_mutual_info(av, bv, n) -> float:
    """Sum over row sizes a, column sizes b and cell counts nij of
    nij/n log(n nij / (a b)) times the hypergeometric probability of nij;
    equal cluster sizes are summed once with their multiplicity."""
    import numpy as np
    from scipy.special import gammaln
    ua, wa = np.unique(np.asarray(av, dtype=np.int64), return_counts=True)
    ub, wb = np.unique(np.asarray(bv, dtype=np.int64), return_counts=True)
    lgb, lgnb, lgn = gammaln(ub + 1.0), gammaln(n - ub + 1.0), gammaln(n + 1.0)
    emi = 0.0
    for ai, wi in zip(ua, wa):
        lo = np.maximum(1, ai + ub - n)
        hi = np.minimum(ai, ub)
        cnt = np.maximum(hi - lo + 1, 0)
        tot = int(cnt.sum())
        if tot == 0:
            continue
        jj = np.repeat(np.arange(len(ub)), cnt)
        nij = (lo[jj] + np.arange(tot) - np.repeat(np.cumsum(cnt) - cnt, cnt)).astype(np.float64)
        b = ub[jj].astype(np.float64)
        lp = (gammaln(ai + 1.0) + lgb[jj] + gammaln(n - ai + 1.0) + lgnb[jj] - lgn - gammaln(nij + 1.0)
              - gammaln(ai - nij + 1.0) - gammaln(b - nij + 1.0) - gammaln(n - ai - b + nij + 1.0))
        emi += float(wi) * float((wb[jj] * nij / n * np.log(n * nij / (ai * b)) * np.exp(lp)).sum())
    return emi


def adjusted_mutual_info(a, b) -> float:
    import numpy as np
    m = contingency(a, b)
    n = int(m.sum())
    av, bv = m.sum(1), m.sum(0)
    if (len(av) == 1 and len(bv) == 1) or (len(av) == n and len(bv) == n):
        return 1.0
    nz = m > 0
    outer = np.outer(av, bv).astype(np.float64)
    mi = float((m[nz] / n * np.log(n * m[nz] / outer[nz])).sum())
    emi = _expected_mutual_info(av, bv, n)
    norm = 0.5 * (_entropy(av, n) + _entropy(bv, n))
    den = norm - emi
    den = min(den, -1e-15) if den < 0 else max(den, 1e-15)
    return (mi - emi) / den


def matched_label_diff(ref, lab) -> float:
    """Share of labels that differ from ref after the best one-to-one matching
    of cluster ids (Hungarian method on the contingency table)."""
    from scipy.optimize import linear_sum_assignment
    m = contingency(ref, lab)
    r, c = linear_sum_assignment(-m)
    return 1.0 - float(m[r, c].sum()) / float(m.sum())


def quality_leg(args, device: int) -> dict:
    """Clustering quality in the structure of Tables 6.3-6.6 (Gaussian blobs,
    n = 1e5, d in {10, 128}, k in {100, 500}) and Table 6.7 (image
    segmentation; a 1024 x 1024 Voronoi image with features (R, G, B, x, y)
    stands in for the ImageNet images, k in {8, 32}): Lloyd runs to
    tau = 1e-8 or 300 iterations from the same seeded initial centres, per
    method the time (CUDA events around km_lloyd_run, after one warm-up run),
    iterations, final SSE, ARI and AMI against the blobs' true labels, and
    Diff against the FP64 run's labels.  The mixed methods certify every
    argmin (labels equal the binary64 argmin wherever the margin exceeds the
    proved bounds), so they are expected to reproduce the FP64 run."""
    import numpy as np
    import torch
    import paper_2407_12208_gb300 as pkg
    from paper_2407_12208_gb300 import workloads
    ctx = pkg.Context(device)
    dev = torch.device("cuda", device)
    out = {"tau": 1e-8, "max_iter": 300, "blobs": {}, "image": {}}

    def run(Xd, C0d, low, rho):
        p = pkg.params(low, "tc", rho=rho, max_iter=300, tau=1e-8)
        n, d = Xd.shape
        ws = ctx.workspace(n, d, C0d.shape[0], p)
        ctx.lloyd_run(Xd, C0d, p, ws=ws)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        C, lab, sse, eta, it = ctx.lloyd_run(Xd, C0d, p, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, it, float(sse[-1]), lab.cpu().numpy(), float(np.mean(eta))

    def methods(d):
        m = [("FP64", "fp64", 5.0), ("FP32", "fp32", 5.0)]
        for low, name in (("bf16", "BF16->FP64"), ("fp16", "FP16->FP64")):
            for rho in (5.0, 10.0, 50.0):
                m.append(("%s rho=%g" % (name, rho), low, rho))
        if d >= 16:
            m.append(("E4M3->FP64 rho=5", "e4m3", 5.0))
        return m

    for d, k in ((10, 100), (10, 500), (128, 100), (128, 500)):
        X, C0, truth = workloads.blobs(100_000, d, k, seed=31 + d + k, with_labels=True)
        Xd, C0d = torch.from_numpy(X).to(dev), torch.from_numpy(C0).to(dev)
        rows, ref, cache = {}, None, {}
        for name, low, rho in methods(d):
            t, it, sse, lab, eta = run(Xd, C0d, low, rho)
            key = lab.tobytes()
            if key not in cache:
                cache[key] = (adjusted_mutual_info(truth, lab), adjusted_rand_index(truth, lab))
            ami, ari = cache[key]
            if ref is None:
                ref = lab
            rows[name] = {"time_s": t, "iters": it, "sse": sse, "ami": ami, "ari": ari,
                          "diff_vs_fp64": matched_label_diff(ref, lab), "eta": eta}
        t64 = rows["FP64"]["time_s"]
        for r in rows.values():
            r["speedup_vs_fp64"] = t64 / r["time_s"]
        out["blobs"]["n=100000 d=%d k=%d" % (d, k)] = rows
    X, _ = workloads.voronoi_image(1024, 1024, 16, 8, seed=47)
    Xd = torch.from_numpy(X).to(dev)
    for k in (8, 32):
        C0 = X[workloads.init_indices(X.shape[0], k, 48 + k)].copy()
        C0d = torch.from_numpy(C0).to(dev)
        rows, ref = {}, None
        for name, low, rho in (("FP64", "fp64", 5.0), ("FP32", "fp32", 5.0), ("BF16->FP64 rho=5", "bf16", 5.0),
                               ("FP16->FP64 rho=5", "fp16", 5.0)):
            t, it, sse, lab, eta = run(Xd, C0d, low, rho)
            if ref is None:
                ref = lab
            rows[name] = {"time_s": t, "iters": it, "sse": sse, "diff_vs_fp64": matched_label_diff(ref, lab),
                          "eta": eta}
        out["image"]["1024x1024 d=5 k=%d" % k] = rows
    ctx.close()
    return out


def c3_trajectory_leg(args, device: int) -> dict:
    """Config 3 free-running: Gaussian mixture n = 4e6, d = 64, k = 256 from
    the same seeded initial centres, 50 Lloyd iterations (km_lloyd_run) with
    the plain FP64 direct path, FP32 direct, and the mixed BF16 / FP16 / E4M3
    paths: the SSE of every iteration, the time of the run (CUDA events) and
    whether the final labels equal the FP64 run's."""
    import numpy as np
    import torch
    import paper_2407_12208_gb300 as pkg
    from paper_2407_12208_gb300 import workloads
    ctx = pkg.Context(device)
    X, C0 = workloads.gaussian_mixture(4_000_000, 64, 256, seed=15)
    Xd, C0d = torch.from_numpy(X).cuda(device), torch.from_numpy(C0).cuda(device)
    out, ref_lab, ref_sse = {}, None, None
    for low in ("fp64", "fp32", "bf16", "fp16", "e4m3"):
        p = pkg.params(low, "tc", rho=5.0, max_iter=50, tau=0.0)
        ws = ctx.workspace(X.shape[0], X.shape[1], C0.shape[0], p)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        C, lab, sse, eta, it = ctx.lloyd_run(Xd, C0d, p, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        lab = lab.cpu().numpy()
        if ref_lab is None:
            ref_lab, ref_sse = lab, sse
        out[low] = {"time_s": e0.elapsed_time(e1) / 1e3, "iters": it, "sse": [float(v) for v in sse],
                    "labels_equal_fp64": bool(np.array_equal(lab, ref_lab)),
                    "max_rel_sse_diff_vs_fp64": float(np.max(np.abs(sse - ref_sse) / ref_sse)),
                    "eta_mean": float(np.mean(eta))}
    ctx.close()
    return out


def table6_leg(args, device: int) -> dict:
    """Tables 6.1 / 6.2 of the paper, in structure: the 5000 x 5000 distance
    matrix of r = 128 points (Gaussian rows; a fraction of the centres are
    near-duplicates of the points, C = P + 1e-4 N(0, I), the rest fresh
    rows), every precision mode of km_distances: device time (mean of 3
    after one warm-up, CUDA events), the flagged share eta and the largest
    relative error against the binary64 direct values."""
    import torch
    import paper_2407_12208_gb300 as pkg
    from paper_2407_12208_gb300 import workloads
    ctx = pkg.Context(device)
    out = {}
    for frac in (0.0, 0.1, 0.5, 1.0):
        X, C = workloads.near_far(5000, 128, frac, seed=81)
        Xd, Cd = torch.from_numpy(X).cuda(device), torch.from_numpy(C).cuda(device)
        D64, _, _ = ctx.distances(Xd, Cd, pkg.params("fp64"))
        D64 = D64.double()
        rows = {}
        for label, low, test, fb in TABLE6_MODES:
            p = pkg.params(low, test, fallback=fb)
            ctx.distances(Xd, Cd, p)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                D, bits, nf = ctx.distances(Xd, Cd, p)
            e1.record()
            torch.cuda.synchronize()
            ref = D64.clamp_min(1e-300)
            rel = float(((D.double() - D64).abs() / ref).max())
            rows[label] = {"ms": e0.elapsed_time(e1) / 3, "eta": nf / 25e6, "max_rel_err": rel}
        out["near_%d%%" % round(100 * frac)] = rows
    ctx.close()
    return {"n": 5000, "k": 5000, "r": 128, "near_eps": 1e-4, "rho": 5.0, "c_A": 2.0, "modes": out}


def _job_data(sp, seed: int, device: int):
    """One served job's data, generated on the device (resident): a Gaussian
    mixture as in the Lloyd workload (centre coordinates N(0, 25), cluster
    std log-uniform [0.1, 2], uniform cluster choice), k initial centres =
    k distinct seeded rows."""
    import math
    import torch
    g = torch.Generator(device="cuda:%d" % device)
    g.manual_seed(seed)
    n, d, k = sp["n"], sp["d"], sp["k"]
    dev = torch.device("cuda", device)
    centres = torch.randn((k, d), generator=g, device=dev) * 5.0
    stds = torch.exp(torch.empty(k, device=dev).uniform_(math.log(0.1), math.log(2.0), generator=g))
    lab = torch.randint(0, k, (n,), generator=g, device=dev)
    X = centres[lab] + torch.randn((n, d), generator=g, device=dev) * stds[lab, None]
    C = X[torch.randperm(n, generator=g, device=dev)[:k]].contiguous()
    return X.contiguous(), C


def serving_leg(args, device: int) -> dict:
    """Served stream through km_submit / km_poll (continuous admission of
    Lloyd jobs of uneven n, d, k; 25 iterations each; the library's format
    rule (km_choose_low) for d > 8, FP32 direct below; 80 GB arena).  Job
    data are generated on the device just before their arrival and read in
    place (KM_JOB_DEVICE_DATA); at most 64 GB of job data is resident at once
    (a submitter that would exceed it waits for completions).  First the
    saturated stream (every job due at once), then Poisson arrivals at 0.5x
    and 0.8x its job rate.  Latency = submit -> result ready, measured by the
    library.  --serve-full: the stream of the served-batch workload (10,000
    jobs, n log-uniform [1e3, 1e6], d in {2, 8, 32, 128, 256}, k log-uniform
    [4, 1024]); by default a bounded stream of the same mix with n <= 1e5."""
    import numpy as np
    import torch
    import paper_2407_12208_gb300 as pkg
    from paper_2407_12208_gb300 import workloads
    full = args.serve_full
    njobs = 10_000 if full else args.serve_jobs
    specs = workloads.serving_jobs(njobs, seed=2024, n_lo=1e3, n_hi=1e6 if full else 1e5)
    ctx = pkg.Context(device, arena_bytes=80 << 30)
    budget = 64 << 30
    lows = {}

    def run(arrivals, tag):
        t0 = time.perf_counter()
        pending, lat, resident = {}, [], 0
        pairs = 0.0

        def reap(block):
            nonlocal resident
            while True:
                done = []
                for jid, (nb, keep) in pending.items():
                    r = ctx.poll(jid)
                    if r is not None:
                        assert r["status"] == 0, (r["status"], r["message"])
                        lat.append(r["latency_ms"])
                        done.append(jid)
                for jid in done:
                    ctx.release(jid)
                    resident -= pending.pop(jid)[0]
                if done or not block:
                    return
                time.sleep(0.0005)

        for i, (sp, ta) in enumerate(zip(specs, arrivals)):
            nb = sp["n"] * sp["d"] * 4
            while resident + nb > budget and pending:
                reap(True)
            while time.perf_counter() - t0 < ta:
                reap(False)
                time.sleep(0.0002)
            X, C = _job_data(sp, 5000 + i, device)
            key = i
            if key not in lows:
                lows[key] = "fp32" if sp["d"] <= 8 else ctx.choose_low(X, C)[0]
            torch.cuda.synchronize(device)
            jid = ctx.submit(X, C, pkg.params(lows[key], max_iter=25, tau=0.0), kind=0)
            pending[jid] = (nb, (X, C))
            resident += nb
            pairs += sp["n"] * float(sp["k"]) * 26  # 25 iterations + final assignment
            if i % 64 == 0:
                reap(False)
        while pending:
            reap(True)
        span = time.perf_counter() - t0
        pct = lambda q: float(np.percentile(np.asarray(lat), q))
        return {"p50_ms": pct(50), "p99_ms": pct(99), "pairs_per_s": pairs / span, "jobs_per_s": len(lat) / span,
                "makespan_s": span}

    warm = workloads.serving_jobs(8, seed=7, n_lo=1e3, n_hi=1e4)
    for i, sp in enumerate(warm):  # module loading, first launches
        X, C = _job_data(sp, 100 + i, device)
        jid = ctx.submit(X, C, pkg.params("fp32" if sp["d"] <= 8 else "bf16", max_iter=2), kind=0)
        while ctx.poll(jid) is None:
            time.sleep(0.001)
        ctx.release(jid)
    sat = run([0.0] * njobs, "saturated")
    out = {"jobs": njobs, "iterations_per_job": 25, "arena_gb": 80, "resident_budget_gb": 64,
           "saturated": sat,
           "sizes": "n log-uniform [1e3, %s], d in {2, 8, 32, 128, 256}, k log-uniform [4, 1024]" %
                    ("1e6" if full else "1e5 (bounded stand-in for [1e3, 1e6])"),
           "formats": {f: sum(1 for v in lows.values() if v == f) for f in set(lows.values())}}
    for load in (0.5, 0.8):
        rate = load * sat["jobs_per_s"]
        arr = workloads.poisson_arrivals(njobs, rate, seed=int(load * 10))
        res = run(list(arr), "poisson")
        res["rate_jobs_per_s"] = rate
        out["poisson_%d%%" % round(100 * load)] = res
    ctx.close()
    return out


def run_reference(args):
    """The CPU oracle, timed as the reference arm on a bounded sample."""
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2407_12208_gb300 import workloads
    oracle.build()
    gen, n, d, k, desc = WORKLOADS[args.workload]
    X, C = getattr(workloads, gen)(n, d, k, seed=15)
    rows = args.ref_rows
    Xs = X[:rows]

    def step():
        lab, d1, _ = oracle.assign(Xs, C)
        oracle.update(Xs, lab, C, 1, d1)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = rows * float(k) / dt
    sample = "first %d of %d rows x %d centres per step (assign + centre update, binary64 direct)" % (rows, n, k)
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload + ": " + desc, "n": n, "d": d, "k": k, "low": "fp64-direct (oracle)",
                       "step": "oracle assign + centre update on a row sample"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c2a")
    ap.add_argument("--low", choices=["bf16", "fp16", "e4m3", "fp32", "fp64"], default="bf16")
    ap.add_argument("--cpu-rows", type=int, default=100_000)
    ap.add_argument("--ref-rows", type=int, default=10_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="rows (profiling a smaller case of the same kernels)")
    ap.add_argument("--no-serving", action="store_true", help="skip the served-stream leg")
    ap.add_argument("--no-table6", action="store_true", help="skip the distance-matrix precision leg")
    ap.add_argument("--no-autotune", action="store_true", help="use the default screening variant (no km_autotune)")
    ap.add_argument("--no-quality", action="store_true", help="skip the clustering-quality leg (Tables 6.3-6.7)")
    ap.add_argument("--no-c3", action="store_true", help="skip the free-running config-3 trajectories")
    ap.add_argument("--clocks-csv", default=None, help="keep the nvidia-smi clock samples of the timed region here")
    ap.add_argument("--serve-jobs", type=int, default=200)
    ap.add_argument("--serve-full", action="store_true",
                    help="the served-batch workload at full size: 10,000 jobs, n up to 1e6 (minutes)")
    ap.add_argument("--only-step", action="store_true",
                    help="time the step only: no end-to-end, FP64 or CPU legs (for profiler runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.warmup < 1:
            args.warmup = 1
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
