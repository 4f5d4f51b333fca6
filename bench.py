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
two forms over all targets, and both forms' relative L2 error against the
oracle's FP64 direct sum at S sampled targets (same-layer images plus the
cross-layer field by one DCIM fit per target); the time of that direct sum
is the CPU baseline.

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


def _wl(name):
    from paper_1902_05875_gb300 import workloads as W
    return getattr(W, name)()


WORKLOADS = {
    "three_layer_slabs_n2M_p10": lambda: _wl("cfg_mixed_2m"),
    "three_layer_slabs_n200k_p10": lambda: _wl("cfg_mixed_200k"),
    "three_layer_middle_n200k_p8": lambda: _wl("cfg_fp64_200k"),
    "three_layer_middle_n2000_p6": lambda: _wl("cfg_small"),
}
DEFAULT_WORKLOAD = "three_layer_slabs_n2M_p10"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 peak: the nominal dense FP64 rate of GB300 (no measured FP64 figure is
# provided); used for the FP64 SIMT kernels.
FP64_PEAK_TFLOPS = 1.25

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
# FP32 SIMT peak derived from the unit counts and the maximum clock:
# 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# TF32 dense peak: the measured BF16 figure x the nominal TF32/BF16 ratio (1.1/2.25)
TF32_OVER_BF16 = 1.1 / 2.25

# DRAM bytes (read + write) per launch from one ncu capture of the kernel as
# it stands (profiles/), keyed by (kernel, workload); None when not captured.
TRAFFIC = {
    ("k_m2l_fp64", "three_layer_middle_n200k_p8"): 4.659415e9 + 3.872982e9,
}


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


def direct_at(w, tgt_idx):
    """The oracle's FP64 direct sum at the given targets against every source:
    same-layer part (free space + DCIM images, C/OpenMP) plus the cross-layer
    part by reciprocity (one DCIM fit per target, C/OpenMP).  Returns
    (phi, seconds)."""
    from oracle.medium import Medium
    from oracle.dcim import ImageTable
    from oracle.direct import direct_sum, cross_sum
    med = Medium(w.interfaces, w.k)
    img = ImageTable(med, w.zext, n_images=w.n_images)
    tgt = w.src[tgt_idx]
    t0 = time.perf_counter()
    phi = direct_sum(med, img, w.src, w.q, tgt)
    if med.n_layers > 1:
        phi = phi + cross_sum(med, w.zext, w.src, w.q, tgt, n_images=w.n_images)
    return phi, time.perf_counter() - t0


def err_stats(phi, ref, layer=None):
    """The paper's error measures (Sec. 4): Err_2 = sqrt(sum |ref - phi|^2 / sum |ref|^2)
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


def cpu_baseline_from(n_t, n_s, seconds, name):
    return {"value": n_t * n_s / seconds, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 direct sum (C/OpenMP; cross-layer part by one DCIM fit per target) "
                      f"for {n_t} sampled targets x all {n_s} sources of {name}, {seconds:.1f} s"}


def cpu_baseline(w, seconds=12.0):
    """The oracle's direct sum on a bounded sample of targets (about `seconds`)."""
    rng = np.random.default_rng(123)
    n = 4
    _, dt = direct_at(w, rng.choice(len(w.src), n, replace=False))
    n = int(max(4, min(len(w.src), n * seconds / max(dt, 1e-3))))
    _, dt = direct_at(w, rng.choice(len(w.src), n, replace=False))
    return cpu_baseline_from(n, len(w.src), dt, w.name)


def run_reference(args, w):
    """--impl reference: the oracle on the host cores, one bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(w, seconds=2.0)
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(w, seconds=8.0)
        vals.append(last["value"])
    v = float(np.mean(vals))
    ms = len(w.src) * len(w.src) / v * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": len(w.src), "p": w.p, "leaf_cap": w.leaf_cap,
                       "n_images": w.n_images},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
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
            cb = cpu_baseline(ws[0], seconds=10.0)
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
    line = {"metric": METRIC_BATCH, "value": replica_value(world, inter, ms), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+tf32x3/f64", "data": "synthetic",
            "config": {"workload": BATCHED, "instances": len(ws), "points": int(sum(len(w.src) for w in ws)),
                       "p": 6, "n_images": ws[0].n_images, "precision": "mixed",
                       "leaf_caps": {str(c): caps.count(c) for c in sorted(set(caps))},
                       "l2": "flushed (256 MB write) between timed steps"},
            "plan_s": plan_s, "first_batch_s_incl_autotune_and_fits": first_s,
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
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="skip the FP64-form step that the mixed form is compared with")
    ap.add_argument("--accuracy-samples", type=int, default=100,
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

    def make(prec):
        return tefmm.Plan(w.interfaces, w.k, p=w.p, leaf_cap=w.leaf_cap, n_images=w.n_images,
                          zext=w.zext, precision=prec)
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

    # roofline of the dominant phase
    pk, pk_src = peaks()
    dom = max(("ms_near", "ms_m2l", "ms_tables", "ms_upward", "ms_downward"), key=lambda k: ph[k])
    imgs = plan.images()
    n_img_layer = max(sum(len(t["A"]) for t in imgs if t["layer"] == l) for l in range(len(w.k)))
    np_ = plan.np
    if dom == "ms_near":
        if mixed:
            flops = st["n_p2p_pairs"] * (FLOPS32_FREE + FLOPS32_IMAGE * n_img_layer)
            kern = "k_near_fp32 (L2P + FP32 P2P, free space + DCIM images)"
            peak, bound, psrc = FP32_PEAK_TFLOPS, "alu", "FP32 lanes x 2 x max clock (derived)"
        else:
            flops = st["n_p2p_pairs"] * (FLOPS_FREE + FLOPS_IMAGE * n_img_layer)
            kern = "k_near_fp64 (L2P + P2P, free space + DCIM images)"
            peak, bound, psrc = FP64_PEAK_TFLOPS, "alu", "nominal GB300 FP64 (no measured FP64 figure)"
    elif dom == "ms_m2l":
        flops = 2 * st["n_v_pairs"] * 8 * np_ * np_
        if mixed:
            kern = "k_m2l_tc (tcgen05 kind::tf32, 3xTF32 split, key-grouped M2L, same- and cross-layer)"
            peak = pk["bf16_tflops"] * TF32_OVER_BF16
            bound, psrc = "tensor", f"TF32 = {pk_src} BF16 burst x 1.1/2.25"
        else:
            kern = "k_m2l_fp64 (key-grouped complex M2L contraction)"
            peak, bound, psrc = FP64_PEAK_TFLOPS, "alu", "nominal GB300 FP64 (no measured FP64 figure)"
    elif dom == "ms_tables":
        np2 = (2 * w.p + 1) * (2 * w.p + 2) * (2 * w.p + 3) // 6
        flops = st["n_tables"] * (n_img_layer + 1) * np2 * 40
        kern = "k_tables + k_xtables (derivative recurrence, FP64)"
        peak, bound, psrc = FP64_PEAK_TFLOPS, "alu", "nominal GB300 FP64 (no measured FP64 figure)"
    else:
        # M2M / L2L: per child-parent pair, sum over k' <= k of the binomial shift (8 flops per
        # complex multiply-add), counted as 8 * n_p * n_p / 4 (the triangular fraction)
        flops = st["n_nodes"] * 8 * np_ * np_ / 4
        kern = "k_m2m / k_l2l (binomial shifts, FP64)"
        peak, bound, psrc = FP64_PEAK_TFLOPS, "alu", "nominal GB300 FP64 (no measured FP64 figure)"
    ach = flops / (ph[dom] * 1e-3) / 1e12
    roof = {"kernel": kern, "phase": dom, "bound": bound, "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak, "traffic": TRAFFIC.get((kern.split()[0], w.name)),
            "peak_source": psrc}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+tf32x3/f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": N, "p": w.p, "leaf_cap": w.leaf_cap, "n_images": w.n_images,
                   "layers": len(w.k), "precision": args.precision,
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
        "e2e": {"value": world * N * N / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(N * 40), "d2h_bytes_per_step": int(N * 16),
                "ms_per_step": e2e_ms},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "peaks_source": pk_src,
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
    if rank == 0 and world == 1 and args.accuracy_samples > 0:
        idx = np.random.default_rng(1).choice(N, min(N, args.accuracy_samples), replace=False)
        ref, dt = direct_at(w, idx)
        acc = line.setdefault("accuracy", {})
        acc["samples"] = int(len(idx))
        acc[f"{args.precision}_vs_direct_rel_l2"] = float(np.linalg.norm(phi[idx] - ref) / np.linalg.norm(ref))
        from oracle.medium import Medium
        lay = Medium(w.interfaces, w.k).layer_of(w.src[idx, 2])
        acc[f"{args.precision}_vs_direct"] = err_stats(phi[idx], ref, lay)
        if phi64 is not None:
            acc["fp64_vs_direct_rel_l2"] = float(np.linalg.norm(phi64[idx] - ref) / np.linalg.norm(ref))
            acc["fp64_vs_direct"] = err_stats(phi64[idx], ref, lay)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_from(len(idx), N, dt, w.name)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and "cpu_baseline" not in line:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
