"""Benchmark of the layered-media TE-FMM matrix-vector product.

One step = one full ``tefmm_eval`` (Morton sort, octrees, lists, P2M/M2M,
derivative tables, M2L, L2L, L2P and near field, all nine layer-pair
components) over the whole particle set, inputs resident in HBM.  The DCIM
fits are plan state: the same-layer ones are made at plan creation and the
cross-layer ones on the first evaluation for a root cube (warm-up), then
cached.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload NAME] [--precision fp64|mixed] [--no-fp64-form]
                  [--accuracy-samples S]

Besides the timed form (mixed by default) the line carries the FP64 form's
time on the same workload (one step), the relative L2 difference between the
two forms over all targets, and both forms' error against the oracle's FP64
direct sum at S sampled targets (the paper's Err_2 and Err_max of Sec. 5,
overall and per target layer).  The direct sums are read from tests/golden/
(written by the committed script beside it, from the oracle alone): 1000
targets of the 2M workload, 20 of the clustered 16M one; other workloads
report no direct-sum error.  The CPU
baseline is the oracle's TE-FMM (Python/numpy) timed on a bounded sample of
the same workload.  The roofline covers both dominant kernels: the
tensor-core M2L contraction (TF32 peak measured here through cuBLAS) and the
FP32 near field (FP32 FMA peak measured here).

Multi-GPU: the path does not shard (one matvec per GPU); N ranks run N
independent replicas of the same workload ("replicas only"); value sums the
ranks' interactions over the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("FMM matvec interactions/s (N_t*N_s per matvec time) at N=2M, mixed vs FP64 form, "
          "rel L2 err vs FP64 direct sum")
UNIT = "interactions/s"


def _wl(fn, *args, **kw):
    from paper_1902_05875_gb300 import workloads as W
    return getattr(W, fn)(*args, **kw)


WORKLOADS = {
    "three_layer_slabs_n2M_p10": lambda: _wl("cfg_mixed_2m"),
    "three_layer_slabs_n200k_p10": lambda: _wl("cfg_mixed_200k"),
    "three_layer_middle_n200k_p8": lambda: _wl("cfg_fp64_200k"),
    "three_layer_middle_n2000_p6": lambda: _wl("cfg_small"),
    # deep adaptive trees: 32 Gaussian clusters (sigma 0.05) in the middle layer, p = 8
    "clustered_n16M_p8": lambda: _wl("clustered", 16_000_000, 8, 64, seed=0, n_images=16,
                                     name="clustered_n16M_p8"),
}
# the paper's Example 2 (irregular domains, three layers), p = 6, for the time-vs-N check
for _n, _tag in ((250_000, "250k"), (500_000, "500k"), (1_000_000, "1M"), (2_000_000, "2M")):
    WORKLOADS[f"irregular_domains3_n{_tag}_p6"] = (
        lambda n=_n, tag=_tag: _wl("irregular_domains", n, 3, p=6, leaf_cap=64, seed=0, n_images=16,
                                   name=f"irregular_domains3_n{tag}_p6"))
DEFAULT_WORKLOAD = "three_layer_slabs_n2M_p10"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# algorithmic FP64 flops per evaluation of e^{ikR}/R with complex R (image
# term) and with real r (free-space term); counted from the formulas:
#   complex R^2 (rho^2 + w^2): 6; principal sqrt: 8; i k R: 6; exp(re)*(cos,sin)
#   of the imaginary part: 4; division by R: 11; times amplitude and
#   accumulate: 8  -> 43 per image term
#   real r = sqrt(dx^2+dy^2+dz^2): 6; e^{ikr}: 6; / r: 2; times q, accumulate: 8 -> 22
FLOPS_IMAGE = 43
FLOPS_FREE = 22

# mixed form: FP32 flops per pair evaluation in k_near_fp32, counted from its
# formulas (image term relative to the leaf-centre reference: D 5, complex sqrt
# 12, delta 10, e^{ik delta} - 1 from expm1/sin/cos 10, delta/R0 and the
# numerator 6, division by 1 + delta/R0 10, times E0 and accumulate 8;
# free-space term 20)
FLOPS32_IMAGE = 61
FLOPS32_FREE = 20


def measure_peaks(torch):
    """Arithmetic peaks of this GPU, measured now with CUDA events at default
    clocks: FP64 and FP32 FMA throughput (peaks/peaks.cu: every lane runs 8
    independent FMA chains) and the TF32 tensor rate of a cuBLAS FP32 GEMM
    with TF32 allowed (8192^3, best of 10; the same kind of measurement as the
    BF16 figure of MEASURED_PEAKS.json).  TFLOP/s."""
    import ctypes
    from paper_1902_05875_gb300 import _build
    lib = ctypes.CDLL(_build.build_peaks())
    for f in (lib.tefmm_peaks_fp64, lib.tefmm_peaks_fp32):
        f.restype = ctypes.c_double
        f.argtypes = [ctypes.c_int] * 4
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp64 = lib.tefmm_peaks_fp64(sms * 8, 256, 4096, 5) / 1e12
    fp32 = lib.tefmm_peaks_fp32(sms * 8, 256, 65536, 5) / 1e12
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    n = 8192
    a = torch.randn(n, n, device="cuda", dtype=torch.float32)
    b = torch.randn(n, n, device="cuda", dtype=torch.float32)
    c = a @ b
    best = 1e30
    for _ in range(10):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    torch.backends.cuda.matmul.allow_tf32 = prev
    del a, b, c
    torch.cuda.empty_cache()
    return {"fp64_fma_tflops": fp64, "fp32_fma_tflops": fp32, "tf32_tflops": 2.0 * n ** 3 / (best * 1e-3) / 1e12,
            "how": "CUDA events, default clocks: FMA chains (8 per lane, 152 x 8 CTAs of 256 threads), "
                   "cuBLAS FP32 GEMM 8192^3 with TF32 allowed, best of 10"}


# DRAM bytes (read + write) per launch from one ncu capture of the kernel as
# it stands (profiles/), keyed by (kernel, workload); None when not captured.
# 2M: one-pass metrics on the full workload; k_m2l_tc averaged over 39
# launches (430.4 GB read + 114.9 GB written), k_near_fp32 one launch.
TRAFFIC = {("k_m2l_tc", "three_layer_slabs_n2M_p10"): 13.98e9,
           ("k_near_fp32", "three_layer_slabs_n2M_p10"): 1.443e9}

# stored oracle direct sums (tests/golden/make_direct_reference.py)
REFERENCE = {"three_layer_slabs_n2M_p10": os.path.join(ROOT, "tests", "golden",
                                                      "direct_three_layer_slabs_n2M_1000.txt"),
             "clustered_n16M_p8": os.path.join(ROOT, "tests", "golden", "direct_clustered_n16M_p8_20.txt")}


def clocks_start():
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    try:
        p = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=f, stderr=subprocess.DEVNULL)
    except Exception:
        p = None
    return p, f.name


def clocks_stop(p, path, gpu_index):
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(gpu_index):
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    os.unlink(path)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def err_stats(phi, ref, layer=None):
    """The paper's error measures (Sec. 5): Err_2 = sqrt(sum |ref - phi|^2 / sum |ref|^2)
    and Err_max = max_i |ref_i - phi_i| / |ref_i|, over all sampled targets and,
    given each target's layer, per layer."""
    phi = np.asarray(phi)
    ref = np.asarray(ref)
    e = np.abs(phi - ref)

    def one(m):
        return {"rel_l2": float(np.sqrt(np.sum(e[m] ** 2) / np.sum(np.abs(ref[m]) ** 2))),
                "max_rel": float(np.max(e[m] / np.abs(ref[m])))}
    out = one(np.ones(len(ref), dtype=bool))
    if layer is not None:
        layer = np.asarray(layer)
        out["per_layer"] = {str(int(l)): one(layer == l) for l in np.unique(layer)}
    return out


def max_over_ranks(x, dist, device):
    """The largest of the ranks' values of x (the job's time is its slowest
    replica's); x itself when not distributed."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, interactions, ms):
    """Whole-job throughput of `world` independent replicas, each doing
    `interactions` pair interactions, over the slowest replica's time."""
    return world * float(interactions) / (ms * 1e-3)


def init_ranks(world, backend="nccl"):
    """Process group of a multi-rank run (None for one rank)."""
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend)
    return dist


def reference_at(w, n_samples):
    """The oracle's FP64 direct sum at up to n_samples targets, as stored by
    tests/golden/make_direct_reference.py (the first n_samples of its
    default_rng(1) sample).  Returns (indices, phi, source), or None when the
    workload has no stored reference."""
    path = REFERENCE.get(w.name)
    if not (path and os.path.exists(path)):
        return None
    d = np.loadtxt(path)[:n_samples]
    return d[:, 0].astype(np.int64), d[:, 1] + 1j * d[:, 2], os.path.relpath(path, ROOT)


def layer_of(interfaces, z):
    """Layer of each z (0 at the top): the number of interfaces above it."""
    d = np.asarray(interfaces, dtype=float).reshape(-1)
    return np.sum(np.asarray(z)[:, None] < d[None, :], axis=1)


CPU_SAMPLE_N = 2000


def oracle_fmm_sample(w, n_targets, warm=True):
    """The oracle's CPU TE-FMM (oracle/tefmm.py, Python/numpy) on a bounded
    sample of workload w: the same medium, particle distribution, p, leaf cap
    and images at CPU_SAMPLE_N points, potentials at n_targets sampled targets
    (setup, upward pass, tables and M2L of their boxes, downward pass, near
    field).  With warm, one untimed run first fits the cross-layer images
    (plan state, as on the GPU).  Returns (seconds, cores used = CPU time /
    wall time, description)."""
    from paper_1902_05875_gb300 import workloads as W
    from oracle.medium import Medium
    from oracle.dcim import ImageTable
    from oracle.tefmm import TEFMM
    if w.name.startswith("three_layer_slabs"):
        ws = W.three_layer_slabs(CPU_SAMPLE_N, w.p, w.leaf_cap, seed=0, n_images=w.n_images)
    else:
        ws = W.middle_layer_uniform(CPU_SAMPLE_N, w.p, w.leaf_cap, seed=0)
    med = Medium(ws.interfaces, ws.k)
    img = ImageTable(med, ws.zext, n_images=ws.n_images)
    f = TEFMM(med, img, ws.p, ws.leaf_cap, n_images=ws.n_images)
    idx = np.random.default_rng(1).choice(len(ws.src), n_targets, replace=False)
    if warm:
        f.setup(ws.src, ws.src).evaluate(ws.q, target_index=idx)
    c0, t0 = time.process_time(), time.perf_counter()
    f.setup(ws.src, ws.src).evaluate(ws.q, target_index=idx)
    dt = time.perf_counter() - t0
    cores = (time.process_time() - c0) / dt
    desc = (f"oracle TE-FMM (Python/numpy) on {CPU_SAMPLE_N} points of the {w.name} distribution "
            f"(p={ws.p}, leaf cap {ws.leaf_cap}, {ws.n_images} images), potentials at {n_targets} sampled "
            f"targets x {CPU_SAMPLE_N} sources, {dt:.1f} s, images fitted beforehand")
    return dt, cores, desc, n_targets * len(ws.src)


def cpu_baseline(w, n_targets=2):
    """The oracle's TE-FMM on a bounded sample (about 20-40 s of CPU work)."""
    dt, cores, desc, inter = oracle_fmm_sample(w, n_targets)
    return {"value": inter / dt, "unit": UNIT, "cores": round(cores, 2), "kind": "oracle", "sample": desc}


def run_reference(args, w):
    """--impl reference: the oracle's TE-FMM on the host cores, one bounded
    sample (potentials at one sampled target of a 2000-point sample of the
    workload) per step; ms_per_step is the measured time of that sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times, last = [], None
    for i in range(args.warmup + args.steps):
        dt, cores, desc, inter = oracle_fmm_sample(w, 1, warm=(i == 0))
        if i >= args.warmup:
            times.append(dt)
            last = (cores, desc, inter)
    ms = float(np.mean(times)) * 1e3
    v = last[2] / (ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": len(w.src), "p": w.p, "leaf_cap": w.leaf_cap,
                       "n_images": w.n_images, "layers": len(w.k), "precision": "fp64",
                       "sample": f"{CPU_SAMPLE_N} points, 1 target per step"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": round(last[0], 2), "kind": "oracle",
                             "sample": last[1]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BATCHED = "batched_256_instances_p6"


def run_batched(args):
    """The batched workload: 256 independent two- or three-layer instances
    (N log-uniform in [1k, 64k], about 3.8M points in all), mixed form, p = 6,
    leaf caps chosen by the library's autotuner, evaluated together by
    tefmm_eval_batched.  value = sum of N_i^2 per batch time."""
    import torch
    from paper_1902_05875_gb300 import tefmm
    from paper_1902_05875_gb300 import workloads as W
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            ws = W.batched_instances(256)
            cb = cpu_baseline(ws[0], n_targets=4)
            print(json.dumps({"impl": "reference", "metric": METRIC_BATCH, "value": cb["value"],
                              "unit": UNIT, "n_gpus": args.gpus, "steps": 1, "warmup": 0,
                              "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                              "config": {"workload": BATCHED, "sample": "instance 0"},
                              "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT,
                                                          "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    dist = init_ranks(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ws = W.batched_instances(256)
    t0 = time.perf_counter()
    plans = [tefmm.Plan(w.interfaces, w.k, p=w.p, leaf_cap=w.leaf_cap, n_images=w.n_images, zext=w.zext,
                        precision=tefmm.MIXED) for w in ws]
    plan_s = time.perf_counter() - t0
    inst = []
    for w in ws:
        x, y, z = [torch.tensor(np.ascontiguousarray(w.src[:, i]), device=dev) for i in range(3)]
        q = torch.tensor(w.q, device=dev)
        inst.append((x, y, z, q, torch.empty(len(w.src), dtype=torch.complex128, device=dev)))
    t0 = time.perf_counter()
    st = tefmm.eval_batched(plans, inst)            # first call: autotuner and cross-layer fits
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    assert all(v == 0 for v in st), st
    for _ in range(max(3, args.warmup) - 1):
        tefmm.eval_batched(plans, inst)
    torch.cuda.synchronize()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    cp, cpath = clocks_start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        tefmm.eval_batched(plans, inst)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    if dist is not None:
        dist.barrier()
    clocks = clocks_stop(cp, cpath, local)
    ms = max_over_ranks(float(np.mean(times)), dist, dev)
    inter = float(sum(len(w.src) ** 2 for w in ws))
    caps = [pl.stats()["leaf_cap_used"] for pl in plans]
    # the charge phases of all instances as one CUDA graph (geometry of the last
    # evaluation kept): one launch per batch
    outs = [o for (_, _, _, _, o) in inst]
    qs = [q for (_, _, _, q, _) in inst]
    t0 = time.perf_counter()
    g = tefmm.BatchGraph(plans, qs, outs)
    torch.cuda.synchronize()
    graph_build_s = time.perf_counter() - t0
    for _ in range(3):
        g.launch()
    torch.cuda.synchronize()
    gt = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.launch()
        e1.record()
        torch.cuda.synchronize()
        gt.append(e0.elapsed_time(e1))
    for pl in plans:
        pl.status()
    g.close()
    ms_graph = max_over_ranks(float(np.mean(gt)), dist, dev)
    line = {"metric": METRIC_BATCH, "value": replica_value(world, inter, ms), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+tf32x3/f64", "data": "synthetic",
            "config": {"workload": BATCHED, "instances": len(ws), "points": int(sum(len(w.src) for w in ws)),
                       "p": 6, "n_images": ws[0].n_images, "precision": "mixed",
                       "leaf_caps": {str(c): caps.count(c) for c in sorted(set(caps))},
                       "l2": "flushed (256 MB write) between timed steps"},
            "plan_s": plan_s, "first_batch_s_incl_autotune_and_fits": first_s,
            "graph_apply": {"ms_per_batch": ms_graph, "value": replica_value(world, inter, ms_graph),
                            "unit": UNIT, "build_s": graph_build_s,
                            "what": "tefmm_batch_graph: every instance's charge phases (P2M .. near field) "
                                    "on its fixed geometry, captured once into one CUDA graph, one launch per batch"},
            "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


METRIC_BATCH = "batched TE-FMM matvec interactions/s (sum of N_i^2 per batch time), 256 instances"


def timed_steps(plan, torch, x, y, z, q, out, flush, steps):
    """Per-step device time (CUDA events on the launching stream, L2 flushed
    before each step) and the plan's per-phase times."""
    times = []
    phase = {k: [] for k in ("ms_tree", "ms_upward", "ms_tables", "ms_m2l", "ms_downward", "ms_near",
                             "ms_cross_tables", "ms_cross_m2l")}
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.eval(x, y, z, q, out=out)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        st = plan.stats()
        for k in phase:
            phase[k].append(st[k])
    return times, {k: float(np.mean(v)) for k, v in phase.items()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + [BATCHED])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--algorithm", type=int, default=1, choices=[1, 2],
                    help="1: DCIM image recurrence; 2: Sommerfeld-integral tables (same-layer reaction M2L)")
    ap.add_argument("--table-n", type=int, default=0, help="Algorithm 2 grid points per direction (0: 64)")
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="skip the FP64-form step that the mixed form is compared with")
    ap.add_argument("--accuracy-samples", type=int, default=1000,
                    help="targets of the oracle direct sum for the accuracy check (0: none)")
    args = ap.parse_args()
    if args.workload == BATCHED:
        run_batched(args)
        return
    w = WORKLOADS[args.workload]()
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = init_ranks(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1902_05875_gb300 import tefmm
    mixed = args.precision == "mixed"

    def make(prec, algorithm=args.algorithm):
        return tefmm.Plan(w.interfaces, w.k, p=w.p, leaf_cap=w.leaf_cap, n_images=w.n_images,
                          zext=w.zext, precision=prec, algorithm=algorithm, table_n=args.table_n)
    plan = make(tefmm.MIXED if mixed else tefmm.FP64)
    x, y, z = [torch.tensor(np.ascontiguousarray(w.src[:, i]), device=dev) for i in range(3)]
    q = torch.tensor(w.q, device=dev)
    out = torch.empty(len(w.src), dtype=torch.complex128, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    for _ in range(max(3, args.warmup)):
        plan.eval(x, y, z, q, out=out)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    launches0 = plan.stats()["n_launches"]
    cp, cpath = clocks_start()
    barrier()
    times, ph = timed_steps(plan, torch, x, y, z, q, out, flush, args.steps)
    barrier()
    clocks = clocks_stop(cp, cpath, local)
    launches = plan.stats()["n_launches"] - launches0
    ms = max_over_ranks(float(np.mean(times)), dist, dev)
    N = len(w.src)
    value = replica_value(world, N * N, ms)
    st = plan.stats()
    phi = out.cpu().numpy()

    # e2e: host buffers through tefmm_eval_host, copies inside the timed region
    pin = {k: torch.tensor(np.ascontiguousarray(a)).pin_memory() for k, a in
           (("src", w.src), ("q", np.stack([w.q.real, w.q.imag], -1)))}
    src_h = pin["src"].numpy()
    q_h = pin["q"].numpy()
    qc = q_h[:, 0] + 1j * q_h[:, 1]
    plan.eval_host(src_h, qc)
    e2e_t = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.eval_host(src_h, qc)
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = float(np.mean(e2e_t)) * 1e3

    # repeated products on one geometry (an iterative solver's use): set_points
    # once, then only the charge-dependent phases (tefmm_apply) per step
    plan.set_points(x, y, z)
    plan.apply(q, out=out)
    app_t = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record()
        plan.apply(q, out=out)
        a1.record()
        torch.cuda.synchronize()
        app_t.append(a0.elapsed_time(a1))
    apply_ms = float(np.mean(app_t))

    # rooflines of the two dominant kernels, from their own device times
    pk_file, pk_src = peaks()
    pk = measure_peaks(torch)
    imgs = plan.images()
    np_ = plan.np
    flops_m2l = 8.0 * np_ * np_ * (st["n_m2l_items"] + st["n_m2l_items_cross"])
    img_layer = [sum(len(t["A"]) for t in imgs if t["layer"] == l) for l in range(len(w.k))]
    pairs_layer = st["n_p2p_pairs_layer"][:len(w.k)]
    n_pairs, n_img_terms = int(sum(pairs_layer)), int(st["n_near_img_terms"])
    if mixed:
        flops_near = FLOPS32_FREE * n_pairs + FLOPS32_IMAGE * n_img_terms
        ms_m2l_k = st["ms_m2l_kernel"]
        m2l_roof = {"kernel": "k_m2l_tc (tcgen05 kind::tf32, 3xTF32, key-grouped M2L, same- and cross-layer)",
                    "bound": "tensor", "achieved": flops_m2l / (ms_m2l_k * 1e-3) / 1e12,
                    "peak": pk["tf32_tflops"], "unit": "TFLOP/s",
                    "peak_source": "TF32 cuBLAS GEMM measured by this run",
                    "ms_per_step": ms_m2l_k, "launches_per_step": st["n_m2l_kernel_launches"],
                    "work": f"8 n_p^2 flops per translation item, {st['n_m2l_items']} same-layer + "
                            f"{st['n_m2l_items_cross']} cross-layer items"}
        near_roof = {"kernel": "k_near_fp32 (L2P + FP32 P2P, free space + DCIM images)", "bound": "alu",
                     "achieved": flops_near / (ph["ms_near"] * 1e-3) / 1e12, "peak": pk["fp32_fma_tflops"],
                     "unit": "TFLOP/s", "peak_source": "FP32 FMA throughput measured by this run",
                     "ms_per_step": ph["ms_near"],
                     "work": f"{FLOPS32_FREE} per particle pair + {FLOPS32_IMAGE} per (pair, image term) evaluated; "
                             f"{n_pairs} pairs, {n_img_terms} image terms after the far-of-near reading "
                             f"(images per layer {img_layer})"}
    else:
        flops_near = FLOPS_FREE * n_pairs + FLOPS_IMAGE * n_img_terms
        m2l_roof = {"kernel": "k_m2l_fp64 + k_m2l_x (key-grouped complex M2L, FP64)", "bound": "alu",
                    "achieved": flops_m2l / (ph["ms_m2l"] * 1e-3) / 1e12, "peak": pk["fp64_fma_tflops"],
                    "unit": "TFLOP/s", "peak_source": "FP64 FMA throughput measured by this run",
                    "ms_per_step": ph["ms_m2l"], "work": "8 n_p^2 flops per translation item"}
        near_roof = {"kernel": "k_near_fp64 (L2P + P2P, free space + DCIM images)", "bound": "alu",
                     "achieved": flops_near / (ph["ms_near"] * 1e-3) / 1e12, "peak": pk["fp64_fma_tflops"],
                     "unit": "TFLOP/s", "peak_source": "FP64 FMA throughput measured by this run",
                     "ms_per_step": ph["ms_near"]}
    for r in (m2l_roof, near_roof):
        r["frac"] = r["achieved"] / r["peak"]
        r["traffic"] = TRAFFIC.get((r["kernel"].split()[0], w.name))
    roof = dict(m2l_roof) if m2l_roof["ms_per_step"] >= near_roof["ms_per_step"] else dict(near_roof)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+tf32x3/f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": N, "p": w.p, "leaf_cap": w.leaf_cap, "n_images": w.n_images,
                   "layers": len(w.k), "precision": args.precision, "algorithm": args.algorithm,
                   "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": "replicas" if world > 1 else "single"},
        "phases_ms": ph,
        "counts": {"nodes": st["n_nodes"], "levels": st["n_levels"], "v_pairs": st["n_v_pairs"],
                   "p2p_pairs": st["n_p2p_pairs"], "tables": st["n_tables"], "tables_built": st["n_tables_built"],
                   "cross_tables": st["n_cross_tables"], "cross_fits": st["n_cross_fits"],
                   "images_total": st["n_images_total"]},
        "fits": {"same_layer_max_resid": st["fit_max_resid"],
                 "cross_layer_max_resid": st["fit_max_resid_cross"],
                 "cross_layer_fit_ms_first_eval": "see warm-up (cached afterwards)"},
        "roofline": roof,
        "rooflines": {"m2l": m2l_roof, "near": near_roof},
        "peaks_measured": pk,
        "e2e": {"value": world * N * N / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(N * 40), "d2h_bytes_per_step": int(N * 16),
                "ms_per_step": e2e_ms},
        "apply": {"ms_per_step": apply_ms, "value": N * N / (apply_ms * 1e-3), "unit": UNIT,
                  "what": "tefmm_apply on the geometry of one tefmm_set_points (trees, lists, tables "
                          "kept): the repeated products of an iterative solver"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "peaks_file": {"source": pk_src, "hbm_gbs": pk_file.get("hbm_gbs"), "bf16_tflops": pk_file.get("bf16_tflops")},
    }
    del plan
    torch.cuda.empty_cache()
    phi64 = None
    if rank == 0 and mixed and not args.no_fp64_form:
        p64 = make(tefmm.FP64)
        out64 = torch.empty_like(out)
        p64.eval(x, y, z, q, out=out64)
        torch.cuda.synchronize()
        t64, ph64 = timed_steps(p64, torch, x, y, z, q, out64, flush, 1)
        phi64 = out64.cpu().numpy()
        line["fp64_form"] = {"ms_per_step": float(np.mean(t64)), "value": N * N / (np.mean(t64) * 1e-3),
                             "unit": UNIT, "phases_ms": ph64, "steps": 1,
                             "speedup_mixed_over_fp64": float(np.mean(t64)) / ms}
        line["accuracy"] = {"mixed_vs_fp64_form_rel_l2": float(np.linalg.norm(phi - phi64) /
                                                                np.linalg.norm(phi64))}
        del p64
        torch.cuda.empty_cache()
    stored = reference_at(w, args.accuracy_samples) if rank == 0 and world == 1 and args.accuracy_samples > 0 else None
    if rank == 0 and world == 1 and args.accuracy_samples > 0 and stored is None:
        line.setdefault("accuracy", {})["direct_sum"] = "no stored oracle reference for this workload"
    if stored is not None:
        idx, ref, src_ref = stored
        acc = line.setdefault("accuracy", {})
        acc["samples"] = int(len(idx))
        acc["reference"] = f"oracle FP64 direct sum ({src_ref})"
        acc[f"{args.precision}_vs_direct_rel_l2"] = float(np.linalg.norm(phi[idx] - ref) / np.linalg.norm(ref))
        lay = layer_of(w.interfaces, w.src[idx, 2])
        acc[f"{args.precision}_vs_direct"] = err_stats(phi[idx], ref, lay)
        if phi64 is not None:
            acc["fp64_vs_direct_rel_l2"] = float(np.linalg.norm(phi64[idx] - ref) / np.linalg.norm(ref))
            acc["fp64_vs_direct"] = err_stats(phi64[idx], ref, lay)
        if args.algorithm == 2:
            # the same form with Algorithm 1's recurrence derivatives, at the same targets
            p1 = make(tefmm.MIXED if mixed else tefmm.FP64, algorithm=1)
            out1 = torch.empty_like(out)
            p1.eval(x, y, z, q, out=out1)
            phi1 = out1.cpu().numpy()
            del p1
            torch.cuda.empty_cache()
            acc["tables_vs_recurrence"] = {
                "tables_vs_direct": err_stats(phi[idx], ref, lay),
                "recurrence_vs_direct": err_stats(phi1[idx], ref, lay),
                "tables_vs_recurrence_rel_l2": float(np.linalg.norm(phi - phi1) / np.linalg.norm(phi1)),
                "table_n": args.table_n or 64, "alg2_tables": st["n_alg2_tables"],
                "ms_table_build": st["ms_alg2_build"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
