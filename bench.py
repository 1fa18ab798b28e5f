#!/usr/bin/env python3
"""Benchmark of the generalized vec trick (GVT) path on one GB300 per rank.

Workload (the homogeneous drug-drug configuration): m = q = 2000 objects,
64-d N(0,1) features, Gaussian base kernel (gamma = 1/64), n = 200k ordered
pairs drawn uniformly without replacement, v ~ N(0,1), FP32 on the GPU.
One step applies all nine pairwise kernels of Table 4b (Kronecker, Gaussian,
linear, poly2d, Cartesian, symmetric, anti-symmetric, ranking, MLPK; 27
Kronecker terms of Corollary 1) to v over the training pairs: 9 calls of
gvt_pairwise_kernel_matvec through the C ABI.

value = pair-terms/s = sum over kernels of n * nhat * T_kernel / step time
(implicit kernel-matrix entries applied per second).  L2 is flushed (512 MB
write) before every timed step, outside the per-step CUDA events.

Also reported: the roofline of the dominant stage (live CUDA events around
each stage launch), the FP64 oracle on the host cores (cpu_baseline), an
end-to-end number through the same API with host buffers, SM clocks during
the timed region, and the KRR solve time (FP64 CG vs mixed-precision
refinement) on the Merget-shaped problem.

--impl reference times the FP64 oracle (plain C, OpenMP) on the host cores on
a bounded sample of the same workload.
"""
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

KINDS = ["kronecker", "gaussian", "linear", "poly2d", "cartesian", "symmetric",
         "antisymmetric", "ranking", "mlpk"]
TERMS = {"kronecker": 1, "gaussian": 1, "linear": 2, "poly2d": 3, "cartesian": 2,
         "symmetric": 2, "antisymmetric": 2, "ranking": 4, "mlpk": 10}
METRIC = "GVT pair-terms/s and KRR-CG solve time at rel. residual 1e-6 vs plain FP64 CG"
UNIT = "pair-terms/s"
WORKLOAD = ("homogeneous drug-drug: m=q=2000, 64-d features, Gaussian base kernel gamma=1/64, "
            "n=200k uniform ordered pairs, all 9 pairwise kernels (27 Kronecker terms), FP32")
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (max SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gvt", choices=["gvt", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--engine", default="auto", choices=["simt", "tc", "tc16", "auto"],
                    help="engine of the FP32 products: sparse SIMT stages; tc = stage 1 as a tcgen05 BF16x3 "
                         "GEMM; tc16 = both stages as tcgen05 FP16x3 GEMMs; auto = per-stage cost model")
    ap.add_argument("--streams", type=int, default=3,
                    help="streams (each with its own handle and plan) over which the nine independent "
                         "products of a step are spread")
    ap.add_argument("--tc-pairs", default="auto", choices=["auto", "off", "on"],
                    help="tile form of the tensor-core GEMM: auto = the library's choice (one SM per tile); "
                         "off = one SM per 128-row tile; on = SM pairs (256-row tiles, tcgen05 cta_group::2)")
    ap.add_argument("--solve-lambdas", default="1e-4,1e-2,1")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-problems", type=int, default=256)
    ap.add_argument("--batched-sample", type=int, default=8,
                    help="problems of the plain FP64 CG comparison run system by system (0: skip it)")
    return ap.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_rate(step_ms, units_per_step, ws, dist, device):
    """Whole-job rate of replicas: every rank processes units_per_step per step; the job's
    step time is the slowest rank's (max over ranks), so the rate is ws * units / max time."""
    import torch
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, ws * units_per_step / (ms / 1e3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def workload(seed):
    from paper_2009_01054_gb300 import synth
    return synth.homogeneous(seed)


def pair_terms_per_step(n):
    return float(n) * float(n) * sum(TERMS.values())


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
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
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# --------------------------------------------------------------------- oracle (CPU)
def cpu_oracle_rate(p, seconds, rows_per_call=64, seed=0, nthreads=0):
    """FP64 oracle pair-terms/s on sampled output rows (each row against all inputs); nthreads = 0
    uses every host core."""
    import numpy as np
    import oracle as orc
    M = orc.gaussian_kernel(p.Xd, gamma=p.gamma)
    rng = np.random.default_rng(seed)
    rows_done = 0
    t0 = time.perf_counter()
    while True:
        idx = rng.choice(p.n, rows_per_call, replace=False)
        for kind in KINDS:
            orc.pairwise_matvec(kind, M, M, p.d[idx], p.t[idx], p.d, p.t, p.v, nthreads=nthreads)
        rows_done += rows_per_call
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    rate = rows_done * float(p.n) * sum(TERMS.values()) / el
    return rate, el, rows_done, (orc.num_threads() if nthreads == 0 else nthreads)


def cpu_oracle_small_solve():
    """The oracle's plain FP64 CG (Eq. 1) on the small drug-target configuration (64 x 48 objects,
    1000 pairs, lambda = 1e-2) to relative residual 1e-6, every product the oracle's own."""
    import oracle as orc
    from paper_2009_01054_gb300 import synth
    p = synth.small(0)
    M, N = orc.gaussian_kernel(p.Xd, gamma=p.gamma), orc.gaussian_kernel(p.Xt, gamma=p.gamma)
    mv = lambda x: orc.pairwise_matvec("kronecker", M, N, p.d, p.t, p.d, p.t, x)
    t0 = time.perf_counter()
    a, it, rel = orc.cg_solve(mv, p.y, p.lambdas[0], tol=1e-6)
    return {"ms": (time.perf_counter() - t0) * 1e3, "iterations": it, "rel_residual": rel,
            "workload": "64 x 48 objects, 1000 pairs, Kronecker of Gaussians, lambda = 1e-2"}


# arithmetic of the products per engine: FP32 SIMT, or 16-bit hi/lo splits on the tensor cores
# with FP32 accumulation (the measured error against FP64 is reported beside it)
DTYPE_OF_ENGINE = {"simt": "f32", "tc": "bf16x3 stage 1 + f32 stage 2", "tc16": "f16x3 (f32 accumulate)",
                   "auto": "f16x3 (f32 accumulate) where dense, else f32"}

KERNEL_SOURCE = {"stage1_dense_kernel": "stages.cu", "stage2_dense_kernel": "stages.cu",
                 "gemv_rows_multi_vec_kernel": "stages.cu", "tc_gemm_kernel": "tc_gemm.cu"}


def kernel_text(kernel_name):
    """Source text of a __global__ kernel definition: from its template line (if any) to the brace
    that closes its body.  None if it is not found."""
    src = open(os.path.join(ROOT, "paper_2009_01054_gb300", "csrc", KERNEL_SOURCE[kernel_name])).read()
    pos = 0
    while True:
        i = src.find(kernel_name + "(", pos)
        if i < 0:
            return None
        g = src.rfind("__global__", 0, i)
        if g >= 0 and i - g < 200 and ";" not in src[g:i]:
            break
        pos = i + 1
    start = src.rfind("\ntemplate", 0, g)
    start = start + 1 if start >= 0 and g - start < 200 else src.rfind("\n", 0, g) + 1
    depth, k = 0, src.find("{", i)
    for j in range(k, len(src)):
        depth += {"{": 1, "}": -1}.get(src[j], 0)
        if depth == 0:
            return src[start:j + 1]
    return None


def traffic_for(kernel_name):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the kernel as its source
    reads now (the record keeps the sha256 of the kernel's definition)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get("kernels", {}).get(kernel_name)
        text = kernel_text(kernel_name)
        if not rec or text is None or rec.get("kernel_sha256") != hashlib.sha256(text.encode()).hexdigest():
            return None
        return rec.get("dram_bytes_per_launch")
    except Exception:
        return None


# --------------------------------------------------------------------- reference arm
def run_reference(args, ws, rank):
    if rank != 0:
        return
    import numpy as np
    import oracle as orc
    from oracle.build import build_oracle
    build_oracle()
    p = workload(0)
    M = orc.gaussian_kernel(p.Xd, gamma=p.gamma)
    rows = 256
    rng = np.random.default_rng(0)

    def step():
        idx = rng.choice(p.n, rows, replace=False)
        for kind in KINDS:
            orc.pairwise_matvec(kind, M, M, p.d[idx], p.t[idx], p.d, p.t, p.v)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    ms = el / max(args.steps, 1) * 1e3
    val = rows * float(p.n) * sum(TERMS.values()) / (ms / 1e3)
    sample = "%d sampled output pairs per step, each against all %d input pairs, 9 kernels" % (rows, p.n)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD + " (FP64 oracle, CPU)", "m": p.m, "n": p.n,
                      "kernels": KINDS, "sample": sample},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------- GPU arm
def run_gvt(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_2009_01054_gb300 import build as gbuild
    from paper_2009_01054_gb300 import gvt

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # one builder per node; the other ranks load what it built
    if local == 0:
        gbuild.build()
    if dist is not None:
        dist.barrier()
    if local != 0:
        gbuild.build()
    dev = torch.device("cuda", local)
    p = workload(rank)
    H = gvt.Handle()
    X = torch.as_tensor(p.Xd, device=dev)
    M = gvt.gaussian_kernel(H, X, gamma=p.gamma, dtype=torch.float32)
    plan = gvt.Plan(H, (p.m, p.m), (p.m, p.m), p.d, p.t)
    v = torch.as_tensor(p.v, dtype=torch.float32, device=dev)
    U = torch.empty((len(KINDS), p.n), dtype=torch.float32, device=dev)
    descs = [gvt.gvt_desc_make(k) for k in KINDS]
    Mm = gvt.matrix(M, symmetric=True)
    sp = gvt.stream_ptr()
    engine_code = {"simt": gvt.GVT_STAGE1_SIMT, "tc": gvt.GVT_STAGE1_TC_BF16X3, "tc16": gvt.GVT_STAGES_TC_F16X3,
                   "auto": gvt.GVT_STAGES_AUTO}[args.engine]
    stream = torch.cuda.current_stream()
    vp = gvt.ptr(v)
    up = [gvt.ptr(U[i]) for i in range(len(KINDS))]
    # the nine products are independent: with S streams, product i runs on stream i % S with a
    # handle and plan of its own, forked from and joined back into the main stream
    S = max(1, args.streams)
    extra_h = [gvt.Handle() for _ in range(S - 1)]
    handles = [H] + extra_h
    plans = [plan] + [gvt.Plan(h, (p.m, p.m), (p.m, p.m), p.d, p.t) for h in extra_h]
    streams = [stream] + [torch.cuda.Stream() for _ in range(S - 1)]
    sps = [sp] + [gvt.stream_ptr(st) for st in streams[1:]]
    fork = torch.cuda.Event()
    joins = [torch.cuda.Event() for _ in range(S)]

    def set_engine(code):
        for h in handles:
            gvt.gvt_set_stage1_engine(h.h, code)

    pair_code = {"auto": gvt.GVT_TC_PAIRS_AUTO, "off": gvt.GVT_TC_PAIRS_OFF, "on": gvt.GVT_TC_PAIRS_ON}
    for h in handles:
        gvt.gvt_set_tc_pairs(h.h, pair_code[args.tc_pairs])

    set_engine(engine_code)

    def step(nstreams=S, after=None):
        # the products of one step on one handle share the split copies of M: each handle splits
        # it once per step (the scope ends with the step, so the next step splits again)
        for h in handles:
            gvt.gvt_factor_cache_begin(h.h)
        if nstreams > 1:
            fork.record(stream)
            for st in streams[1:nstreams]:
                st.wait_event(fork)
        for i, d in enumerate(descs):
            j = i % nstreams
            gvt.gvt_pairwise_kernel_matvec(plans[j].p, d, Mm, Mm, vp, up[i], 1, gvt.GVT_F32, sps[j])
            if after is not None:
                after(i, streams[j])
        for j in range(1, nstreams):
            joins[j].record(streams[j])
            stream.wait_event(joins[j])
        for h in handles:
            gvt.gvt_factor_cache_end(h.h)

    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    l0 = gvt.gvt_launch_count()
    for k in range(K):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = gvt.gvt_launch_count() - l0
    barrier()
    clk = clocks.stop()
    # the same K steps again with the library's per-stage CUDA events on (kept out of the timed
    # steps above so that `value` carries no instrumentation): the roofline's launch durations
    # (one stream: each launch's event-bracketed duration is its own, not shared with another stream's)
    gvt.gvt_stats_enable(H.h, True)
    for k in range(K):
        flush.zero_()
        step(nstreams=1)
    torch.cuda.synchronize()
    stats = gvt.gvt_stats_read(H.h)
    gvt.gvt_stats_enable(H.h, False)
    step_ms = sum(a.elapsed_time(b) for a, b in ev) / K
    pts = pair_terms_per_step(p.n)
    step_ms_max, value = job_rate(step_ms, pts, ws, dist, dev)

    # ---- roofline of the dominant kernel
    peaks, peak_src = measured_peaks()
    dom = max(("stage1", "stage2", "one_sided"), key=lambda k: stats[k]["ms"])
    tg = stats["tc_gemm"]
    if tg["launches"] > 0 and tg["ms"] >= max(stats[k]["ms"] for k in ("stage1", "stage2", "one_sided")) / 2:
        # the dense engines: the split GEMM is the dominant kernel (its launches are a part of both
        # stages' time); FP16 and BF16 run at the same nominal tensor rate, so the measured BF16 peak
        # applies to the FP16 splits unchanged
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        per_launch_ms = tg["ms"] / tg["launches"]
        achieved = tg["flops"] / tg["ms"] / 1e9
        useful = (stats["stage1"]["flops"] + stats["stage2"]["flops"]) / max(tg["flops"], 1.0)
        roof = {"bound": "tensor", "achieved": achieved, "peak": bf16, "unit": "TFLOP/s",
                "frac": achieved / bf16, "peak_source": peak_src + " bf16 burst (fp16 nominal ratio 1)",
                "kernel": "tc_gemm_kernel", "traffic": traffic_for("tc_gemm_kernel"),
                "ms_per_launch": per_launch_ms, "launches_per_step": tg["launches"] // K,
                "algorithmic_flops_per_launch": tg["flops"] / tg["launches"],
                "algorithmic_bytes_per_launch": tg["bytes"] / tg["launches"],
                "note": "flops of the split GEMM C = A' B'^T (2 M N K, K = 3 x the 64-rounded inner length: "
                        "hi*hi + hi*lo + lo*hi); the stages' useful GVT flops are %.1f%% of them" % (100 * useful)}
        dom = None
    if dom is not None:
        st = stats[dom]
        per_launch_ms = st["ms"] / max(st["launches"], 1)
        flops_l = st["flops"] / max(st["launches"], 1)
        bytes_l = st["bytes"] / max(st["launches"], 1)
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        ridge = FP32_PEAK_TFLOPS * 1e12 / (hbm * 1e9)
        if flops_l / max(bytes_l, 1.0) > ridge:
            achieved = flops_l / (per_launch_ms / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_PEAK_TFLOPS,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}
        else:
            achieved = bytes_l / (per_launch_ms / 1e3) / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "peak_source": peak_src}
        kname = {"stage1": "stage1_dense_kernel", "stage2": "stage2_dense_kernel",
                 "one_sided": "gemv_rows_multi_vec_kernel"}[dom]
        roof.update({"kernel": kname, "traffic": traffic_for(kname), "ms_per_launch": per_launch_ms,
                     "algorithmic_flops_per_launch": flops_l, "algorithmic_bytes_per_launch": bytes_l,
                     "hbm_frac": (bytes_l / (per_launch_ms / 1e3) / 1e9) / hbm})
    stage_summary = {k: {"launches": stats[k]["launches"] // K,
                         "ms_per_step": stats[k]["ms"] / K,
                         "tflops": (stats[k]["flops"] / max(stats[k]["ms"], 1e-9)) / 1e9,
                         "gbs": (stats[k]["bytes"] / max(stats[k]["ms"], 1e-9)) / 1e6}
                     for k in stats}

    # ---- end to end through the same API with host buffers
    vh = torch.as_tensor(p.v, dtype=torch.float32).pin_memory()
    Uh = torch.empty((len(KINDS), p.n), dtype=torch.float32).pin_memory()
    Ke = max(10, K // 5)
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(Ke)]
    copy_stream = torch.cuda.Stream()
    done = [torch.cuda.Event() for _ in KINDS]

    def copy_back(i, st):
        done[i].record(st)
        copy_stream.wait_event(done[i])
        with torch.cuda.stream(copy_stream):
            Uh[i].copy_(U[i], non_blocking=True)

    def step_e2e():
        # v in from pinned memory; each kernel's result goes back on a copy stream while the
        # next products run; the step ends when the last copy has landed
        v.copy_(vh, non_blocking=True)
        step(after=copy_back)
        stream.wait_stream(copy_stream)

    barrier()
    torch.cuda.synchronize()
    for k in range(Ke):
        flush.zero_()
        ev2[k][0].record(stream)
        step_e2e()
        ev2[k][1].record(stream)
    torch.cuda.synchronize()
    assert torch.equal(Uh[-1], U[-1].cpu())
    e2e_ms = sum(a.elapsed_time(b) for a, b in ev2) / Ke
    e2e_ms_max, e2e_value = job_rate(e2e_ms, pts, ws, dist, dev)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": int(vh.numel() * 4), "d2h_bytes_per_step": int(Uh.numel() * 4),
           "ms_per_step": e2e_ms_max}

    # ---- the same steps on the FP32 SIMT engine, for comparison (device-timed like `value`)
    engines = None
    if args.engine != "simt":
        set_engine(gvt.GVT_STAGE1_SIMT)
        for _ in range(3):
            step()
        ev3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.synchronize()
        for k in range(K):
            flush.zero_()
            ev3[k][0].record(stream)
            step()
            ev3[k][1].record(stream)
        torch.cuda.synchronize()
        simt_ms = sum(a.elapsed_time(b) for a, b in ev3) / K
        engines = {"simt_f32": {"ms_per_step": simt_ms, "value": ws * pts / (simt_ms / 1e3), "unit": UNIT},
                   args.engine: {"ms_per_step": step_ms_max, "value": value, "unit": UNIT}}
        set_engine(engine_code)

    # ---- KRR solve: plain FP64 CG vs mixed-precision refinement
    accuracy = None
    if rank == 0:
        accuracy = sampled_error(p, M, plan, gvt, torch, dev)
        accuracy["fp32_tolerance"] = 1e-5
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    tc_gemm = bench_tc_gemm(H, gvt, torch, dev, peaks) if rank == 0 else None
    solve = None
    if not args.no_solve and rank == 0:
        solve = bench_solve(H, gvt, torch, dev, [float(x) for x in args.solve_lambdas.split(",")])
    batched = None
    if not args.no_batched and rank == 0:
        batched = bench_batched(H, gvt, torch, dev, args.batched_problems, args.batched_sample)

    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1:
        rate, el, rows, cores = cpu_oracle_rate(p, args.cpu_seconds)
        rate1, el1, rows1, _ = cpu_oracle_rate(p, min(3.0, args.cpu_seconds), nthreads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d sampled output pairs x all %d input pairs x 9 kernels, FP64, %.1f s"
                         % (rows, p.n, el),
               "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                               "sample": "%d sampled output pairs, %.1f s" % (rows1, el1)},
               "small_solve": cpu_oracle_small_solve()}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
               "warmup": args.warmup, "ms_per_step": step_ms_max, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_OF_ENGINE[args.engine], "data": "synthetic",
               "config": {"workload": WORKLOAD, "m": p.m, "q": p.m, "n": p.n, "nhat": p.n,
                          "kernels": KINDS, "kronecker_terms": sum(TERMS.values()),
                          "pair_terms_per_step": pts,
                          "l2": "flushed (512 MB write) before every timed step, outside the events",
                          "streams": S, "tc_pairs": args.tc_pairs,
                          "kernel_matrix_splits": "once per step per stream (gvt_factor_cache_begin/end "
                                                  "around each step)",
                          "roofline_timing": "per-stage CUDA events of the library, over a second pass of the same "
                                             "K steps (the timed pass runs without them)",
                          "parallelism": "replicas: independent problems per rank (seed = rank)"},
               "roofline": roof, "stages": stage_summary, "cpu_baseline": cpu, "e2e": e2e,
               "clocks": clk, "gpu_launches": launches,
               "engine": args.engine, "engines": engines,
               "error_vs_fp64_oracle": accuracy, "tensor_stage1_gemm": tc_gemm, "solve": solve,
               "batched": batched}
        print(json.dumps(out), flush=True)
    for pl in plans:
        pl.close()
    for h in handles:
        h.close()
    if dist is not None:
        dist.destroy_process_group()


def sampled_error(p, M, plan, gvt, torch, dev, rows=64):
    """Normwise error of the timed FP32 products vs the FP64 oracle on sampled output rows."""
    import numpy as np
    import oracle as orc
    Mo = orc.gaussian_kernel(p.Xd, gamma=p.gamma)
    idx = np.random.default_rng(1).choice(p.n, rows, replace=False)
    v = torch.as_tensor(p.v, dtype=torch.float32, device=dev)
    out = {}
    for kind in KINDS:
        u = gvt.pairwise_kernel_matvec(plan, kind, M, M, v).double().cpu().numpy()
        ref = orc.pairwise_matvec(kind, Mo, Mo, p.d[idx], p.t[idx], p.d, p.t, p.v.astype(np.float32))
        out[kind] = float(np.max(np.abs(u[idx] - ref)) / np.max(np.abs(ref)))
    out["max"] = max(out.values())
    out["sample"] = "%d output rows, normwise max|u - u*| / max|u*|" % rows
    return out


def bench_tc_gemm(H, gvt, torch, dev, peaks, reps=50):
    """The tcgen05 BF16 GEMM of the dense stage 1 on the Merget-shaped problem in ordering B:
    S' (2000 x 250) = [hi|hi|lo](M) [hi|lo|hi](W^T)^T, K' = 3 * 2048."""
    Y, X, K = 2000, 250, 3 * 2048
    g = torch.Generator(device=dev).manual_seed(0)
    A = torch.randn(Y, K, generator=g, device=dev).to(torch.bfloat16)
    B = torch.randn(X, K, generator=g, device=dev).to(torch.bfloat16)
    C = torch.empty(Y, X, device=dev)
    sp = gvt.stream_ptr()
    for _ in range(5):
        gvt.gvt_tc_gemm_bf16(H.h, gvt.ptr(A), K, gvt.ptr(B), K, gvt.ptr(C), X, Y, X, K, sp)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        gvt.gvt_tc_gemm_bf16(H.h, gvt.ptr(A), K, gvt.ptr(B), K, gvt.ptr(C), X, Y, X, K, sp)
    e1.record()
    torch.cuda.synchronize()
    gvt.gvt_check_device_errors(H.h, sp)
    ms = e0.elapsed_time(e1) / reps
    tf = 2.0 * Y * X * K / (ms / 1e3) / 1e12
    peak = float(peaks.get("bf16_tflops", 1900.0))
    return {"shape": "M=%d N=%d K=%d (bf16 in, fp32 out)" % (Y, X, K), "ms": ms, "bound": "tensor",
            "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
            "note": "includes launch and the split-K zeroing; small GEMM (16 x 1 output tiles x 10 K splits)"}


def bench_solve(H, gvt, torch, dev, lambdas):
    """Merget-shaped KRR (m=2000, q=250, n=120k, Kronecker kernel): wall time to FP64 rel.
    residual 1e-6 for plain FP64 CG, FP32-inner refinement, tensor-core-inner refinement, and
    the paper's FP64 MINRES."""
    from paper_2009_01054_gb300 import synth
    p = synth.merget(0)
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=dev), gamma=p.gamma)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=dev), gamma=p.gamma)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    y = torch.as_tensor(p.y, device=dev)
    res = {"workload": "merget-shaped: m=2000, q=250, 128-d, n=120k (24%), Kronecker of Gaussians, "
                       "target FP64 rel. residual 1e-6", "runs": {}}
    variants = (("fp64_cg", gvt.GVT_SOLVE_FP64_CG, gvt.GVT_F32, gvt.GVT_STAGE1_SIMT),
                ("mixed_ir_f32", gvt.GVT_SOLVE_MIXED_IR, gvt.GVT_F32, gvt.GVT_STAGE1_SIMT),
                ("mixed_ir_tc_bf16x3", gvt.GVT_SOLVE_MIXED_IR, gvt.GVT_BF16, gvt.GVT_STAGE1_SIMT),
                ("mixed_ir_tc_f16x3", gvt.GVT_SOLVE_MIXED_IR, gvt.GVT_F32, gvt.GVT_STAGES_TC_F16X3))
    for lam in lambdas:
        r = {}
        for name, mode, inner, engine in variants:
            gvt.gvt_set_stage1_engine(H.h, engine)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            a, st, info = gvt.krr_cg_solve(H, plan, "kronecker", M, N, y, lam, mode=mode, check_every=2,
                                           max_iter=20000, inner_dtype=inner)
            torch.cuda.synchronize()
            wall = (time.perf_counter() - t0) * 1e3
            gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
            r[name] = {"ms": wall, "status": gvt.STATUS_NAMES[st], "iterations": int(info.iterations),
                       "refinements": int(info.refinements), "rel_residual": info.rel_residual}
        # the paper's own solver (Sec. 6): FP64 MINRES to the same residual
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a, st, info, _ = gvt.krr_minres_solve(H, plan, "kronecker", M, N, y, lam, rel_tol=1e-6, max_iter=20000)
        torch.cuda.synchronize()
        r["fp64_minres"] = {"ms": (time.perf_counter() - t0) * 1e3, "status": gvt.STATUS_NAMES[st],
                            "iterations": int(info.iterations), "rel_residual": info.rel_residual}
        for name in ("mixed_ir_f32", "mixed_ir_tc_bf16x3", "mixed_ir_tc_f16x3"):
            if r[name]["status"] == "GVT_OK" and r["fp64_cg"]["status"] == "GVT_OK":
                r[name]["speedup_vs_fp64_cg"] = r["fp64_cg"]["ms"] / r[name]["ms"]
        res["runs"]["lambda=%g" % lam] = r
    # the whole sweep from one Krylov space: multi-shift FP64 CG against the separate FP64 CG solves
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    A, st, info, rr = gvt.krr_cg_solve_multishift(H, plan, "kronecker", M, N, y, lambdas, rel_tol=1e-6,
                                                  max_iter=20000)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    sep = sum(res["runs"]["lambda=%g" % lam]["fp64_cg"]["ms"] for lam in lambdas)
    res["fp64_cg_multishift_sweep"] = {"ms": ms, "status": gvt.STATUS_NAMES[st], "iterations": int(info.iterations),
                                       "rel_residuals": rr, "fp64_cg_separate_ms": sep,
                                       "speedup_vs_separate_fp64_cg": sep / ms if st == 0 else None}
    plan.close()
    return res


def bench_batched(H, gvt, torch, dev, n_probs, sample=8):
    """Batched uneven problems: n_probs KRR problems (m, q ~ U{32..512}, density ~ U[5%, 60%],
    32-d features, Kronecker of Gaussians) x 16 lambdas (logspace 1e-4..1) in one batched solve to
    FP64 rel. residual 1e-6, against plain FP64 CG run system by system on a sample of problems."""
    from paper_2009_01054_gb300 import synth
    t0 = time.perf_counter()
    ps = synth.batched(n_probs)
    gen_s = time.perf_counter() - t0
    lambdas = list(ps[0].lambdas)
    probs = []
    for p in ps:
        M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=dev), gamma=p.gamma)
        N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=dev), gamma=p.gamma)
        probs.append(dict(M=M, N=N, d=torch.as_tensor(p.d, device=dev), t=torch.as_tensor(p.t, device=dev),
                          y=torch.as_tensor(p.y, device=dev)))
    total_pairs = sum(p.n for p in ps)
    # first call includes the autotuner; time the second (tuned, cached) call
    gvt.krr_solve_batched(H, probs, lambdas, rel_tol=1e-6)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    A, st, info, rr = gvt.krr_solve_batched(H, probs, lambdas, rel_tol=1e-6)
    torch.cuda.synchronize()
    batched_ms = (time.perf_counter() - t0) * 1e3
    worst = max(max(r) for r in rr)
    # plain FP64 CG, one system at a time, on the first `sample` problems
    t0 = time.perf_counter()
    fp_iters, fp_worst, sample_pairs = 0, 0.0, 0
    sample = max(0, sample)
    for b in range(min(sample, len(ps))):
        p = probs[b]
        plan = gvt.Plan(H, tuple(p["M"].shape), tuple(p["N"].shape), p["d"], p["t"])
        for lam in lambdas:
            a, st2, inf2 = gvt.krr_cg_solve(H, plan, "kronecker", p["M"], p["N"], p["y"], lam, max_iter=50000,
                                            check_every=2)
            fp_iters += inf2.iterations
            fp_worst = max(fp_worst, inf2.rel_residual)
        sample_pairs += ps[b].n
        plan.close()
    torch.cuda.synchronize()
    fp_ms = (time.perf_counter() - t0) * 1e3
    est_full = fp_ms * total_pairs / max(sample_pairs, 1)
    return {"workload": "%d problems, m,q ~ U{32..512}, density ~ U[5%%,60%%], 32-d, %d lambdas logspace(-4,0), "
                        "%d pairs total, %d systems" % (len(ps), len(lambdas), total_pairs, len(ps) * len(lambdas)),
            "batched_ms": batched_ms, "status": gvt.STATUS_NAMES[st], "inner_iterations": int(info.iterations),
            "refinements": int(info.refinements), "max_rel_residual": worst,
            "plain_fp64_cg_sample": {"problems": min(sample, len(ps)), "systems": min(sample, len(ps)) * len(lambdas),
                                     "ms": fp_ms, "iterations": fp_iters, "max_rel_residual": fp_worst,
                                     "pairs": sample_pairs},
            "plain_fp64_cg_estimate_ms": est_full if sample_pairs else None,
            "estimate_note": "plain FP64 CG time for all systems scaled from the sample by pair count",
            "speedup_vs_plain_fp64_cg_estimate": est_full / batched_ms if sample_pairs else None,
            "data_generation_s": gen_s}


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    run_gvt(args, ws, rank, local)


if __name__ == "__main__":
    main()
