#!/usr/bin/env python3
"""Benchmark of the generalized vec trick (GVT) path on one GB300 per rank.

Headline workload (the kernel-filling scale, the largest configuration): m = q = 20000 objects
on each side, 256-d N(0,1) features, Gaussian base kernels M and N (gamma = 1/256), n = 10M
training pairs with power-law degrees (Zipf 1.1 weights on drug and target ids), v ~ N(0,1),
FP32 on the GPU.  One step is one product u = R (M kron N) R^T v of the Gaussian pairwise
kernel of Table 4b (one Kronecker term of Corollary 1) over the training pairs: one call of
gvt_pairwise_kernel_matvec through the C ABI.

value = pair-terms/s = n * nhat * T / step time (T Kronecker terms; implicit kernel-matrix
entries applied per second).  The kernel matrices (1.6 GB each in FP32) exceed L2, and L2 is
also flushed (512 MB write) before every timed step, outside the per-step CUDA events.

roofline: the dominant kernel's algorithmic work per launch (2 qbar n flops for stage 1 and
2 m nhat for stage 2 per Kronecker term, counting only the pairs the launch serves) over its
CUDA-event duration, against the measured peak of its arithmetic.  The dense tensor-core GEMM's
executed flops are reported apart as `tensor_pipe`.

Other sections of the JSON line: all nine kernels of Table 4b on the homogeneous 2000-object
configuration (`all_kernels`), the FP64 oracle on the host cores (`cpu_baseline`), an
end-to-end number through the same API with host buffers (`e2e`), SM clocks during the timed
region, KRR solves on the Merget-shaped problem (`solve`), solves at the kernel-filling scale
(`c5_solve`), the batched solve (`batched`) and the tcgen05 GEMM alone (`tensor_stage1_gemm`).

--impl reference times the FP64 oracle (plain C, OpenMP) on the host cores on a bounded sample
of the same workload (sampled output rows, each against all input pairs).
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
WORKLOADS = {
    "c5": ("kernel-filling scale: m=q=20000, 256-d features, Gaussian base kernels gamma=1/256, "
           "n=10M pairs with Zipf(1.1) degrees, Gaussian pairwise kernel (1 Kronecker term), FP32"),
    "c2": ("homogeneous drug-drug: m=q=2000, 64-d features, Gaussian base kernel gamma=1/64, "
           "n=200k uniform ordered pairs, all 9 pairwise kernels (27 Kronecker terms), FP32"),
}
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (max SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# FP64: the nominal GB300 rate (no measured figure exists for it)
FP64_PEAK_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gvt", choices=["gvt", "reference"])
    ap.add_argument("--headline", default="c5", choices=["c5", "c2"],
                    help="workload of `value`: c5 = kernel-filling scale (10M Zipf pairs, Gaussian kernel); "
                         "c2 = homogeneous 2000 objects, all nine kernels")
    ap.add_argument("--c5-m", type=int, default=20000,
                    help="objects per side of the kernel-filling workload (a smaller instance of the same "
                         "recipe serves profiler captures that must stay small)")
    ap.add_argument("--c5-n", type=int, default=10_000_000, help="pairs of the kernel-filling workload")
    ap.add_argument("--no-all-kernels", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-c5-solve", action="store_true")
    ap.add_argument("--c5-fp64-cg", action="store_true",
                    help="also run plain FP64 CG at the kernel-filling scale (lambda = 1); minutes of GPU time")
    ap.add_argument("--c5-precond", action="store_true",
                    help="train the learned preconditioner at the kernel-filling scale on 2000 residual -> "
                         "correction pairs and compare flexible CG with it against the solves without it; "
                         "minutes of GPU time")
    ap.add_argument("--c5-bounded-iters", type=int, default=240,
                    help="inner-iteration cap of the bounded lambda = 1e-2 attempt at the kernel-filling scale "
                         "(0: skip it)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--engine", default="auto", choices=["simt", "tc", "tc16", "auto", "f16x1"],
                    help="engine of the FP32 products: sparse SIMT stages; tc = stage 1 as a tcgen05 BF16x3 "
                         "GEMM; tc16 = both stages as tcgen05 FP16x3 GEMMs; auto = per-stage cost model; "
                         "f16x1 = auto with single-pass FP16 dense stages (the mixed solves' inner operator, "
                         "2^-11 relative errors)")
    ap.add_argument("--streams", type=int, default=3,
                    help="streams (each with its own handle and plan) over which the nine independent "
                         "products of an all-kernels step are spread")
    ap.add_argument("--tc-pairs", default="auto", choices=["auto", "off", "on"],
                    help="tile form of the tensor-core GEMM: auto = the library's choice (one SM per tile); "
                         "off = one SM per 128-row tile; on = SM pairs (256-row tiles, tcgen05 cta_group::2)")
    ap.add_argument("--solve-lambdas", default="1e-4,1e-2,1")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-sparse-hbm", action="store_true")
    ap.add_argument("--no-headline", action="store_true",
                    help="skip the headline product (profiling runs of the other sections); the line then "
                         "carries no value")
    ap.add_argument("--batched-problems", type=int, default=256)
    ap.add_argument("--batched-sample", type=int, default=32,
                    help="problems (every k-th of the set) solved both batched and by plain FP64 CG system by "
                         "system, for the measured speed-up (0: skip the comparison)")
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


def workload(name, seed, c5_m=20000, c5_n=10_000_000):
    from paper_2009_01054_gb300 import synth
    return synth.zipf(seed, m=c5_m, n=c5_n, labels=True) if name == "c5" else synth.homogeneous(seed)


def kinds_of(name):
    return ["gaussian"] if name == "c5" else KINDS


def pair_terms_per_step(n, kinds):
    return float(n) * float(n) * sum(TERMS[k] for k in kinds)


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
def oracle_rows(p, kinds, idx, v, nthreads=0):
    """The FP64 oracle's products at output rows idx (each against all input pairs).  The
    heterogeneous problem evaluates only the kernel rows those outputs need; the homogeneous
    one (2000 objects) evaluates its whole kernel matrix."""
    import numpy as np
    import oracle as orc
    out = {}
    if p.homogeneous:
        M = orc.gaussian_kernel(p.Xd, gamma=p.gamma)
        for kind in kinds:
            out[kind] = orc.pairwise_matvec(kind, M, M, p.d[idx], p.t[idx], p.d, p.t, v, nthreads=nthreads)
        return out
    ud, id_ = np.unique(p.d[idx], return_inverse=True)
    ut, it_ = np.unique(p.t[idx], return_inverse=True)
    Mo = orc.gaussian_kernel(p.Xd[ud], p.Xd, gamma=p.gamma, nthreads=nthreads)
    No = orc.gaussian_kernel(p.Xt[ut], p.Xt, gamma=p.gamma, nthreads=nthreads)
    for kind in kinds:
        out[kind] = orc.pairwise_matvec(kind, Mo, No, id_.astype(np.int32), it_.astype(np.int32), p.d, p.t, v,
                                        nthreads=nthreads)
    return out


def cpu_oracle_rate(p, kinds, seconds, rows_per_call=64, seed=0, nthreads=0):
    """FP64 oracle pair-terms/s on sampled output rows (each row against all inputs); nthreads = 0
    uses every host core."""
    import numpy as np
    import oracle as orc
    rng = np.random.default_rng(seed)
    rows_done = 0
    t0 = time.perf_counter()
    while True:
        idx = rng.choice(p.n, rows_per_call, replace=False)
        oracle_rows(p, kinds, idx, p.v, nthreads=nthreads)
        rows_done += rows_per_call
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    rate = rows_done * float(p.n) * sum(TERMS[k] for k in kinds) / el
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
                   "auto": "f16x3 (f32 accumulate) where dense, else f32",
                   "f16x1": "f16 single pass (f32 accumulate) where dense, else f32"}

KERNEL_SOURCE = {"stage1_sparse_kernel": "stages.cu", "stage2_gather_kernel": "stages.cu",
                 "gemv_rows_multi_vec_kernel": "stages.cu", "tc_gemm_kernel": "tc_gemm.cu"}
KERNEL_OF_STAT = {"sparse_stage1": "stage1_sparse_kernel", "sparse_stage2": "stage2_gather_kernel",
                  "one_sided": "gemv_rows_multi_vec_kernel", "tc_gemm": "tc_gemm_kernel"}


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


def traffic_for(kernel_name, workload_name):
    """DRAM bytes per launch from a committed ncu summary of this workload, if it was taken on the
    kernel as its source reads now (the record keeps the sha256 of the kernel's definition)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get("kernels", {}).get(kernel_name)
        text = kernel_text(kernel_name)
        if not rec or text is None or rec.get("kernel_sha256") != hashlib.sha256(text.encode()).hexdigest():
            return None
        per = rec.get("dram_bytes_per_launch")
        return per.get(workload_name) if isinstance(per, dict) else None
    except Exception:
        return None


def roofline(stats, K, peaks, peak_src, elem_bytes, workload_name):
    """Roofline of the dominant kernel (largest summed device time among the tensor-core GEMM,
    the sparse stage-1 kernel, the sampled gather-dot kernel and the one-sided pass) from the
    library's per-launch CUDA events.  achieved = the method's algorithmic work per launch
    (`useful_flops`, SURVEY-defined units: 2 qbar n per stage-1 term, 2 m nhat per stage-2 term)
    / the launch's average duration."""
    cand = [k for k in ("tc_gemm", "sparse_stage1", "sparse_stage2", "one_sided") if stats[k]["launches"] > 0]
    if not cand:
        return None, None
    dom = max(cand, key=lambda k: stats[k]["ms"])
    st = stats[dom]
    L = st["launches"]
    ms_l = st["ms"] / L
    useful_l = st["useful_flops"] / L
    bytes_l = st["bytes"] / L
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    kname = KERNEL_OF_STAT[dom]
    roof = {"kernel": kname, "launches_per_step": L / K, "ms_per_launch": ms_l,
            "algorithmic_flops_per_launch": useful_l, "algorithmic_bytes_per_launch": bytes_l,
            "traffic": traffic_for(kname, workload_name)}
    tensor_pipe = None
    if dom == "tc_gemm":
        # the GEMM is timed inside the multi-step product loop, under the power cap: the sustained
        # BF16 peak (the burst one where no sustained figure was measured); FP16 at the nominal ratio 1
        sustained = "bf16_tflops_sustained" in peaks
        bf16 = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0)))
        ach = useful_l / (ms_l / 1e3) / 1e12
        roof.update({"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
                     "peak_source": peak_src + (" bf16 sustained" if sustained else " bf16 burst") +
                                    " (fp16 at the nominal ratio 1; the GEMM is timed inside a long loop)",
                     "note": "achieved counts the GVT flops of the pairs the GEMM serves (2 qbar n or 2 m nhat "
                             "per term), not the GEMM's own"})
        exe = st["flops"] / L / (ms_l / 1e3) / 1e12
        tensor_pipe = {"kernel": kname, "executed_tflops": exe, "peak": bf16, "frac": exe / bf16,
                       "useful_share": st["useful_flops"] / max(st["flops"], 1.0),
                       "note": "executed flops of the split GEMM per launch (2 M N K, K = the split's parts x the "
                               "64-rounded inner length: 3 parts hi*hi + hi*lo + lo*hi, 1 on the single pass)"}
    else:
        peak_alu = FP32_PEAK_TFLOPS if elem_bytes == 4 else FP64_PEAK_TFLOPS
        ridge = peak_alu * 1e12 / (hbm * 1e9)
        if useful_l / max(bytes_l, 1.0) > ridge:
            ach = useful_l / (ms_l / 1e3) / 1e12
            roof.update({"bound": "alu", "achieved": ach, "peak": peak_alu, "unit": "TFLOP/s",
                         "frac": ach / peak_alu,
                         "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz" if elem_bytes == 4
                                         else "nominal GB300 FP64 rate")})
        else:
            ach = bytes_l / (ms_l / 1e3) / 1e9
            roof.update({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "peak_source": peak_src})
        roof["hbm_frac"] = (bytes_l / (ms_l / 1e3) / 1e9) / hbm
    return roof, tensor_pipe


def stage_summary(stats, K):
    out = {}
    for k, st in stats.items():
        if st["launches"] == 0:
            continue
        out[k] = {"launches_per_step": st["launches"] / K, "ms_per_step": st["ms"] / K,
                  "useful_tflops": st["useful_flops"] / max(st["ms"], 1e-9) / 1e9,
                  "algorithmic_gbs": st["bytes"] / max(st["ms"], 1e-9) / 1e6}
        if st["flops"] != st["useful_flops"]:
            out[k]["executed_tflops"] = st["flops"] / max(st["ms"], 1e-9) / 1e9
    return out


# --------------------------------------------------------------------- reference arm
def run_reference(args, ws, rank):
    if rank != 0:
        return
    import numpy as np
    import oracle as orc
    from oracle.build import build_oracle
    build_oracle()
    p = workload(args.headline, 0, args.c5_m, args.c5_n)
    kinds = kinds_of(args.headline)
    rows = 64
    rng = np.random.default_rng(0)

    def step():
        idx = rng.choice(p.n, rows, replace=False)
        oracle_rows(p, kinds, idx, p.v)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    ms = el / max(args.steps, 1) * 1e3
    val = rows * float(p.n) * sum(TERMS[k] for k in kinds) / (ms / 1e3)
    sample = ("%d sampled output pairs per step, each against all %d input pairs, %d kernel(s), the kernel "
              "rows they need evaluated per step" % (rows, p.n, len(kinds)))
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.headline] + " (FP64 oracle, CPU)", "m": p.m, "q": p.q,
                      "n": p.n, "kernels": kinds, "sample": sample},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------- GPU arm
class Products:
    """The products of one workload: `kinds` applied to v over the training pairs, spread over
    `nstreams` streams (each with a handle and plan of its own)."""

    def __init__(self, gvt, torch, dev, p, kinds, nstreams, engine_code, pair_code):
        self.gvt, self.torch, self.p, self.kinds = gvt, torch, p, kinds
        S = max(1, min(nstreams, len(kinds)))
        self.handles = [gvt.Handle() for _ in range(S)]
        H = self.handles[0]
        Xd = torch.as_tensor(p.Xd, device=dev)
        self.M = gvt.gaussian_kernel(H, Xd, gamma=p.gamma, dtype=torch.float32)
        self.N = self.M if p.homogeneous else gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=dev), gamma=p.gamma,
                                                                  dtype=torch.float32)
        del Xd
        self.plans = [gvt.Plan(h, (p.m, p.m), (p.q, p.q), p.d, p.t) for h in self.handles]
        self.v = torch.as_tensor(p.v, dtype=torch.float32, device=dev)
        self.U = torch.empty((len(kinds), p.n), dtype=torch.float32, device=dev)
        self.descs = [gvt.gvt_desc_make(k) for k in kinds]
        self.Mm = gvt.matrix(self.M, symmetric=True)
        self.Nm = gvt.matrix(self.N, symmetric=True)
        self.stream = torch.cuda.current_stream()
        self.streams = [self.stream] + [torch.cuda.Stream() for _ in range(S - 1)]
        self.sps = [gvt.stream_ptr(st) for st in self.streams]
        self.vp = gvt.ptr(self.v)
        self.up = [gvt.ptr(self.U[i]) for i in range(len(kinds))]
        self.fork = torch.cuda.Event()
        self.joins = [torch.cuda.Event() for _ in range(S)]
        self.S = S
        for h in self.handles:
            gvt.gvt_set_tc_pairs(h.h, pair_code)
        self.set_engine(engine_code)

    def set_engine(self, code):
        for h in self.handles:
            self.gvt.gvt_set_stage1_engine(h.h, code)

    def set_tiles(self, mode):
        for h in self.handles:
            self.gvt.gvt_set_stage_tiles(h.h, mode)

    def step(self, nstreams=None, after=None):
        gvt = self.gvt
        ns = self.S if nstreams is None else nstreams
        # the products of one step on one handle share the split copies of the kernel matrices:
        # each handle splits them once per step (the scope ends with the step)
        for h in self.handles:
            gvt.gvt_factor_cache_begin(h.h)
        if ns > 1:
            self.fork.record(self.stream)
            for st in self.streams[1:ns]:
                st.wait_event(self.fork)
        for i, d in enumerate(self.descs):
            j = i % ns
            gvt.gvt_pairwise_kernel_matvec(self.plans[j].p, d, self.Mm, self.Nm, self.vp, self.up[i], 1,
                                           gvt.GVT_F32, self.sps[j])
            if after is not None:
                after(i, self.streams[j])
        for j in range(1, ns):
            self.joins[j].record(self.streams[j])
            self.stream.wait_event(self.joins[j])
        for h in self.handles:
            gvt.gvt_factor_cache_end(h.h)

    def close(self):
        for pl in self.plans:
            pl.close()
        for h in self.handles:
            h.close()


def time_steps(torch, step, K, flush, stream):
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / K


def bench_products(args, gvt, torch, dev, name, p, K, W, ws, dist, local, flush, peaks, peak_src, with_e2e):
    """Timed steps of one workload: value, roofline, stage summary, clocks, e2e, engines."""
    engine_code = {"simt": gvt.GVT_STAGE1_SIMT, "tc": gvt.GVT_STAGE1_TC_BF16X3, "tc16": gvt.GVT_STAGES_TC_F16X3,
                   "auto": gvt.GVT_STAGES_AUTO, "f16x1": gvt.GVT_STAGES_TC_F16X1}[args.engine]
    pair_code = {"auto": gvt.GVT_TC_PAIRS_AUTO, "off": gvt.GVT_TC_PAIRS_OFF, "on": gvt.GVT_TC_PAIRS_ON}[args.tc_pairs]
    kinds = kinds_of(name)
    pr = Products(gvt, torch, dev, p, kinds, args.streams, engine_code, pair_code)
    for _ in range(max(W, 3)):
        pr.step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    l0 = gvt.gvt_launch_count()
    step_ms = time_steps(torch, pr.step, K, flush, pr.stream)
    launches = gvt.gvt_launch_count() - l0
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    # the same K steps again on one stream with the library's per-launch CUDA events on (kept out
    # of the timed steps above so that `value` carries no instrumentation): the roofline's launch
    # durations are each launch's own, not shared with another stream's
    H = pr.handles[0]
    gvt.gvt_stats_enable(H.h, True)
    for _ in range(K):
        flush.zero_()
        pr.step(nstreams=1)
    torch.cuda.synchronize()
    stats = gvt.gvt_stats_read(H.h)
    gvt.gvt_stats_enable(H.h, False)
    pts = pair_terms_per_step(p.n, kinds)
    step_ms_max, value = job_rate(step_ms, pts, ws, dist, dev)
    # committed DRAM traffic is recorded per workload at its full size, and per engine other than the
    # default (a reduced instance has no record)
    tkey = name if args.engine == "auto" else name + "_" + args.engine
    if name == "c5" and (p.m != 20000 or p.n != 10_000_000):
        tkey += "_reduced"
    roof, tpipe = roofline(stats, K, peaks, peak_src, 4, tkey)
    wl = WORKLOADS[name]
    if name == "c5" and (p.m != 20000 or p.n != 10_000_000):
        wl += " -- reduced instance of the same recipe: m=q=%d, n=%d" % (p.m, p.n)
    res = {"workload": wl, "m": p.m, "q": p.q, "n": p.n, "nhat": p.n, "kernels": kinds,
           "kronecker_terms": sum(TERMS[k] for k in kinds), "pair_terms_per_step": pts,
           "ms_per_step": step_ms_max, "value": value, "unit": UNIT, "streams": pr.S,
           "gpu_launches": launches, "clocks": clk, "roofline": roof, "tensor_pipe": tpipe,
           "stages": stage_summary(stats, K)}
    if with_e2e:
        # end to end through the same API with host buffers: v in from pinned memory, each kernel's
        # result back to pinned memory on a copy stream while the next products run
        vh = torch.as_tensor(p.v, dtype=torch.float32).pin_memory()
        Uh = torch.empty((len(kinds), p.n), dtype=torch.float32).pin_memory()
        copy_stream = torch.cuda.Stream()
        done = [torch.cuda.Event() for _ in kinds]

        def copy_back(i, st):
            done[i].record(st)
            copy_stream.wait_event(done[i])
            with torch.cuda.stream(copy_stream):
                Uh[i].copy_(pr.U[i], non_blocking=True)

        def step_e2e():
            pr.v.copy_(vh, non_blocking=True)
            pr.step(after=copy_back)
            pr.stream.wait_stream(copy_stream)

        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        Ke = max(10, K // 2)
        e2e_ms = time_steps(torch, step_e2e, Ke, flush, pr.stream)
        assert torch.equal(Uh[-1], pr.U[-1].cpu())
        e2e_ms_max, e2e_value = job_rate(e2e_ms, pts, ws, dist, dev)
        res["e2e"] = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(vh.numel() * 4),
                      "d2h_bytes_per_step": int(Uh.numel() * 4), "ms_per_step": e2e_ms_max}
    # the same steps on the FP32 SIMT engine, for comparison (device-timed like `value`)
    if args.engine != "simt":
        pr.set_engine(gvt.GVT_STAGE1_SIMT)
        for _ in range(2):
            pr.step()
        torch.cuda.synchronize()
        simt_ms = time_steps(torch, pr.step, max(3, min(K, 10)), flush, pr.stream)
        res["engines"] = {"simt_f32": {"ms_per_step": simt_ms, "value": ws * pts / (simt_ms / 1e3), "unit": UNIT},
                          args.engine: {"ms_per_step": step_ms_max, "value": value, "unit": UNIT}}
        pr.set_engine(engine_code)
        if args.engine in ("auto", "tc16", "f16x1"):
            # the same engine with the per-tile stages off: every stage wholly dense or wholly SIMT
            pr.set_tiles(gvt.GVT_TILES_OFF)
            for _ in range(2):
                pr.step()
            torch.cuda.synchronize()
            off_ms = time_steps(torch, pr.step, max(3, min(K, 10)), flush, pr.stream)
            res["engines"][args.engine + "_without_tiles"] = {"ms_per_step": off_ms,
                                                              "value": ws * pts / (off_ms / 1e3), "unit": UNIT}
            pr.set_tiles(gvt.GVT_TILES_AUTO)
        if args.engine == "auto":
            # the single-pass FP16 stages: the inner operator of the mixed-precision solves (its
            # products carry 2^-11 relative errors, which the FP64 refinement removes)
            pr.set_engine(gvt.GVT_STAGES_TC_F16X1)
            for _ in range(2):
                pr.step()
            torch.cuda.synchronize()
            k1 = max(3, min(K, 10))
            f1_ms = time_steps(torch, pr.step, k1, flush, pr.stream)
            gvt.gvt_stats_enable(H.h, True)
            for _ in range(k1):
                flush.zero_()
                pr.step(nstreams=1)
            torch.cuda.synchronize()
            st1 = gvt.gvt_stats_read(H.h)
            gvt.gvt_stats_enable(H.h, False)
            res["engines"]["f16x1"] = {"ms_per_step": f1_ms, "value": ws * pts / (f1_ms / 1e3), "unit": UNIT,
                                       "stages": stage_summary(st1, k1)}
            pr.set_engine(engine_code)
    return pr, res


def error_vs_fp64(gvt, torch, dev, pr, p, kinds, args_engine="auto"):
    """Normwise error max|u - u64| / max|u64| over all outputs of the FP32 products against the
    library's FP64 products of the same kernels (FP64 kernel matrices, SIMT stages), which the
    parity tests hold to the FP64 oracle within 1e-10."""
    pr.step(nstreams=1)
    torch.cuda.synchronize()
    H = pr.handles[0]
    M64 = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=dev), gamma=p.gamma)
    N64 = M64 if p.homogeneous else gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=dev), gamma=p.gamma)
    v64 = pr.v.double()
    out = {}
    for i, kind in enumerate(kinds):
        u64 = gvt.pairwise_kernel_matvec(pr.plans[0], kind, M64, N64, v64)
        out[kind] = float((pr.U[i].double() - u64).abs().max() / u64.abs().max())
    out["max"] = max(out.values())
    out["sample"] = ("all %d outputs, normwise max|u - u64| / max|u64| against the library's FP64 product "
                     "(held to the FP64 oracle within 1e-10 by the parity tests)" % p.n)
    out["fp32_tolerance"] = 1e-5
    if args_engine == "f16x1":
        out["note"] = "single-pass FP16 dense stages: errors of order 2^-11 of the term magnitudes, not FP32-accurate"
    del M64, N64
    torch.cuda.empty_cache()
    return out


def run_gvt(args, ws, rank, local):
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
    peaks, peak_src = measured_peaks()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    K, W = args.steps, args.warmup

    head = args.headline
    p, res, accuracy = None, None, None
    if not args.no_headline:
        p = workload(head, rank, args.c5_m, args.c5_n)
        pr, res = bench_products(args, gvt, torch, dev, head, p, K, W, ws, dist, local, flush, peaks, peak_src,
                                 True)
        accuracy = error_vs_fp64(gvt, torch, dev, pr, p, kinds_of(head), args.engine) if rank == 0 else None
        pr.close()
        del pr
        torch.cuda.empty_cache()

    others = {}
    if not args.no_all_kernels and head != "c2":
        p2 = workload("c2", rank)
        pr2, r2 = bench_products(args, gvt, torch, dev, "c2", p2, K, W, ws, dist, local, flush, peaks, peak_src,
                                 False)
        if rank == 0:
            r2["error_vs_fp64"] = error_vs_fp64(gvt, torch, dev, pr2, p2, KINDS, args.engine)
        pr2.close()
        del pr2
        torch.cuda.empty_cache()
        others["all_kernels"] = r2

    H = gvt.Handle()
    tc_gemm = bench_tc_gemm(H, gvt, torch, dev, peaks) if rank == 0 else None
    solve = None
    if not args.no_solve and rank == 0:
        solve = bench_solve(H, gvt, torch, dev, [float(x) for x in args.solve_lambdas.split(",")])
    c5_solve = None
    if not args.no_c5_solve and rank == 0:
        c5_solve = bench_c5_solve(H, gvt, torch, dev,
                                  p if head == "c5" and p is not None else workload("c5", 0, args.c5_m, args.c5_n),
                                  args)
    c5_precond = None
    if args.c5_precond and rank == 0:
        c5_precond = bench_c5_precond(H, gvt, torch, dev,
                                      p if head == "c5" and p is not None else
                                      workload("c5", 0, args.c5_m, args.c5_n))
    sparse_hbm = bench_sparse_hbm(gvt, torch, dev, peaks) if rank == 0 and not args.no_sparse_hbm else None
    batched = None
    if not args.no_batched and rank == 0:
        batched = bench_batched(H, gvt, torch, dev, args.batched_problems, args.batched_sample)
    H.close()

    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1 and p is not None:
        kinds = kinds_of(head)
        rate, el, rows, cores = cpu_oracle_rate(p, kinds, args.cpu_seconds)
        rate1, el1, rows1, _ = cpu_oracle_rate(p, kinds, min(3.0, args.cpu_seconds), rows_per_call=8, nthreads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d sampled output pairs x all %d input pairs x %d kernel(s), FP64, %.1f s"
                         % (rows, p.n, len(kinds), el),
               "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                               "sample": "%d sampled output pairs, %.1f s" % (rows1, el1)},
               "small_solve": cpu_oracle_small_solve()}

    if rank == 0 and res is None:
        out = {"metric": METRIC, "value": None, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
               "note": "headline skipped (--no-headline): a profiling run of the other sections",
               "tensor_stage1_gemm": tc_gemm, "solve": solve, "c5_solve": c5_solve, "c5_precond": c5_precond,
               "sparse_hbm": sparse_hbm, "batched": batched}
        out.update(others)
        print(json.dumps(out), flush=True)
    elif rank == 0:
        cfg = {k: res[k] for k in ("workload", "m", "q", "n", "nhat", "kernels", "kronecker_terms",
                                   "pair_terms_per_step", "streams")}
        cfg.update({"l2": "inputs larger than L2 (the kernel matrices are 1.6 GB each in FP32) and L2 flushed "
                          "(512 MB write) before every timed step, outside the events"
                          if head == "c5" else
                          "flushed (512 MB write) before every timed step, outside the events",
                    "tc_pairs": args.tc_pairs,
                    "roofline_timing": "per-launch CUDA events of the library, over a second pass of the same K "
                                       "steps on one stream (the timed pass runs without them)",
                    "parallelism": "replicas: independent problems per rank (seed = rank)"})
        out = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": ws, "steps": K,
               "warmup": W, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_OF_ENGINE[args.engine], "data": "synthetic",
               "config": cfg, "roofline": res["roofline"], "tensor_pipe": res["tensor_pipe"],
               "stages": res["stages"], "cpu_baseline": cpu, "e2e": res.get("e2e"),
               "clocks": res["clocks"], "gpu_launches": res["gpu_launches"],
               "engine": args.engine, "engines": res.get("engines"),
               "error_vs_fp64": accuracy, "tensor_stage1_gemm": tc_gemm, "solve": solve,
               "c5_solve": c5_solve, "c5_precond": c5_precond, "sparse_hbm": sparse_hbm, "batched": batched}
        out.update(others)
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


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


def timed_solve(torch, fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, (time.perf_counter() - t0) * 1e3


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
                ("mixed_ir_tc_f16x3", gvt.GVT_SOLVE_MIXED_IR, gvt.GVT_F32, gvt.GVT_STAGES_TC_F16X3),
                ("mixed_ir_tc_f16x1", gvt.GVT_SOLVE_MIXED_IR, gvt.GVT_F16, gvt.GVT_STAGE1_SIMT))
    for lam in lambdas:
        r = {}
        for name, mode, inner, engine in variants:
            gvt.gvt_set_stage1_engine(H.h, engine)
            (a, st, info), wall = timed_solve(torch, lambda: gvt.krr_cg_solve(
                H, plan, "kronecker", M, N, y, lam, mode=mode, check_every=2, max_iter=20000, inner_dtype=inner))
            gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
            r[name] = {"ms": wall, "status": gvt.STATUS_NAMES[st], "iterations": int(info.iterations),
                       "refinements": int(info.refinements), "rel_residual": info.rel_residual}
        # the paper's own solver (Sec. 6): FP64 MINRES to the same residual
        (a, st, info, _), wall = timed_solve(torch, lambda: gvt.krr_minres_solve(
            H, plan, "kronecker", M, N, y, lam, rel_tol=1e-6, max_iter=20000))
        r["fp64_minres"] = {"ms": wall, "status": gvt.STATUS_NAMES[st], "iterations": int(info.iterations),
                            "rel_residual": info.rel_residual}
        for name in r:
            if name != "fp64_cg" and r[name]["status"] == "GVT_OK" and r["fp64_cg"]["status"] == "GVT_OK":
                r[name]["speedup_vs_fp64_cg"] = r["fp64_cg"]["ms"] / r[name]["ms"]
        res["runs"]["lambda=%g" % lam] = r
    # the whole sweep from one Krylov space: multi-shift FP64 CG against the separate FP64 CG solves
    (A, st, info, rr), ms = timed_solve(torch, lambda: gvt.krr_cg_solve_multishift(
        H, plan, "kronecker", M, N, y, lambdas, rel_tol=1e-6, max_iter=20000))
    sep = sum(res["runs"]["lambda=%g" % lam]["fp64_cg"]["ms"] for lam in lambdas)
    res["fp64_cg_multishift_sweep"] = {"ms": ms, "status": gvt.STATUS_NAMES[st], "iterations": int(info.iterations),
                                       "rel_residuals": rr, "fp64_cg_separate_ms": sep,
                                       "speedup_vs_separate_fp64_cg": sep / ms if st == 0 else None}
    plan.close()
    return res


def bench_c5_solve(H, gvt, torch, dev, p, args):
    """Kernel ridge solves at the kernel-filling scale (m=q=20000, 10M Zipf pairs, Gaussian
    kernel, FP64 M and N): at lambda = 1, mixed-precision refinement to FP64 rel. residual 1e-6 with
    two inner operators (single-pass FP16 tensor-core stages; FP16x3 stages on the automatic engine)
    and (--c5-fp64-cg) plain FP64 CG; every residual is the solver's own FP64 recomputation (the
    oracle re-checks one such solve on sampled rows in the scale tests); at
    lambda = 1e-2 a bounded attempt whose residual history is reported."""
    import numpy as np
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=dev), gamma=p.gamma)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=dev), gamma=p.gamma)
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    y = torch.as_tensor(p.y, device=dev)
    res = {"workload": "kernel-filling scale: m=q=20000, 256-d, n=10M Zipf(1.1) pairs, Gaussian kernel, "
                       "y = bilinear signal + N(0, 0.1^2)", "runs": {}}
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGES_AUTO)
    try:
        runs1 = {}
        for name, inner, itol, note in (
                ("mixed_ir_f16x1", gvt.GVT_F16, 1e-3, "FP32 CG on single-pass FP16 tensor-core stages where dense"),
                ("mixed_ir_f16x1_inner_tol_1e-2", gvt.GVT_F16, 1e-2,
                 "the same, each inner solve stopped at 1e-2 (the single-pass operator's own error limits "
                 "what one refinement can gain)"),
                ("mixed_ir_f16x3", gvt.GVT_F32, 1e-3,
                 "FP32 CG, automatic engine (FP16x3 tensor-core stages where dense)")):
            (a, st_, info, hist), wall = timed_solve(torch, lambda: gvt.krr_cg_solve(
                H, plan, "kronecker", M, N, y, 1.0, mode=gvt.GVT_SOLVE_MIXED_IR, check_every=2, max_iter=1500,
                history=64, inner_dtype=inner, inner_tol=itol))
            rr = {"ms": wall, "status": gvt.STATUS_NAMES[st_], "iterations": int(info.iterations),
                  "refinements": int(info.refinements), "rel_residual": info.rel_residual, "history": hist,
                  "inner": note, "inner_tol": itol}
            runs1[name] = rr
        res["runs"]["lambda=1"] = runs1
        if args.c5_fp64_cg:
            gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
            (a2, st2, info2, hist2), wall2 = timed_solve(torch, lambda: gvt.krr_cg_solve(
                H, plan, "kronecker", M, N, y, 1.0, check_every=5, max_iter=5000, history=256))
            r2 = {"ms": wall2, "status": gvt.STATUS_NAMES[st2], "iterations": int(info2.iterations),
                  "rel_residual": info2.rel_residual, "history": hist2[::4]}
            res["runs"]["lambda=1"]["fp64_cg"] = r2
            for rr in runs1.values():
                if rr["status"] == "GVT_OK" and st2 == 0:
                    rr["speedup_vs_fp64_cg"] = wall2 / rr["ms"]
            gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGES_AUTO)
        if args.c5_bounded_iters > 0:
            (a3, st3, info3, hist3), wall3 = timed_solve(torch, lambda: gvt.krr_cg_solve(
                H, plan, "kronecker", M, N, y, 1e-2, mode=gvt.GVT_SOLVE_MIXED_IR, check_every=2,
                max_iter=args.c5_bounded_iters, history=64, inner_dtype=gvt.GVT_F16))
            res["runs"]["lambda=0.01"] = {"mixed_ir_bounded": {
                "ms": wall3, "status": gvt.STATUS_NAMES[st3], "iterations": int(info3.iterations),
                "refinements": int(info3.refinements), "rel_residual": info3.rel_residual, "history": hist3,
                "note": "bounded attempt: at most %d inner iterations on the single-pass FP16 inner operator"
                        % args.c5_bounded_iters}}
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    plan.close()
    del M, N
    torch.cuda.empty_cache()
    return res


def bench_c5_precond(H, gvt, torch, dev, p, n_rhs=4, per_rhs=500, steps=400, lam=1.0):
    """The learned preconditioner at the kernel-filling scale (lambda = 1): 2000 residual -> correction
    pairs (n_rhs right-hand sides x the first per_rhs iterations of exact CG on the FP32 operator of
    the automatic engine, stored in BF16), the BF16 network trained on them on the tensor cores, then
    mixed-precision refinement whose inner CG is flexible CG with the learned P, against the same
    refinement with plain inner CG (the plain FP64 CG time is in c5_solve)."""
    import numpy as np
    from paper_2009_01054_gb300 import synth
    res = {"workload": "kernel-filling scale, lambda = %g, %d pairs from %d right-hand sides" % (lam, n_rhs * per_rhs, n_rhs)}
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=dev), gamma=p.gamma)
    N = gvt.gaussian_kernel(H, torch.as_tensor(p.Xt, device=dev), gamma=p.gamma)
    M32, N32 = M.float(), N.float()
    plan = gvt.Plan(H, (p.m, p.m), (p.q, p.q), p.d, p.t)
    rng = np.random.default_rng(11)
    ys = [torch.as_tensor(p.y, device=dev)] + [torch.as_tensor(rng.standard_normal(p.n), device=dev)
                                               for _ in range(n_rhs - 1)]
    # the pairs, column-major n x (n_rhs * per_rhs) in BF16: one buffer each, filled in place
    Rrows = torch.empty((n_rhs * per_rhs, p.n), dtype=torch.bfloat16, device=dev)
    Erows = torch.empty_like(Rrows)
    t0 = time.perf_counter()
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGES_AUTO)
    try:
        for k, y in enumerate(ys):
            a_star, st, info = gvt.krr_cg_solve(H, plan, "kronecker", M, N, y, lam, mode=gvt.GVT_SOLVE_MIXED_IR,
                                                rel_tol=1e-8, check_every=2, max_iter=4000, inner_dtype=gvt.GVT_F16)
            gvt.cg_record_pairs(H, plan, "kronecker", M32, N32, y, lam, a_star, list(range(per_rhs)),
                                store=torch.bfloat16,
                                out=(Rrows[k * per_rhs:(k + 1) * per_rhs], Erows[k * per_rhs:(k + 1) * per_rhs]))
        torch.cuda.synchronize()
        res["record_s"] = time.perf_counter() - t0
        res["pairs_gb_bf16"] = 2 * Rrows.numel() * 2 / 1e9
        R, E = Rrows.t(), Erows.t()
        t0 = time.perf_counter()
        pc = gvt.Precond(H, plan, "kronecker", M, N, synth.mlp_init_params(0, out_scale=0.01))
        hist = pc.train(R, E, steps=steps, batch=16, lr=3e-3)
        torch.cuda.synchronize()
        res["train_s"] = time.perf_counter() - t0
        res["loss_first5"] = float(np.mean(hist[:5]))
        res["loss_last20"] = float(np.mean(hist[-20:]))
        res["scale"] = pc.scale()
        del R, E, Rrows, Erows
        torch.cuda.empty_cache()
        y = ys[0]
        runs = {}
        for name, prec in (("mixed_ir_plain_inner", None), ("mixed_ir_learned_fcg_inner", pc)):
            (a, st, info), wall = timed_solve(torch, lambda: gvt.krr_cg_solve(
                H, plan, "kronecker", M, N, y, lam, mode=gvt.GVT_SOLVE_MIXED_IR, check_every=2, max_iter=3000,
                precond=prec, precond_budget=1500))
            runs[name] = {"ms": wall, "status": gvt.STATUS_NAMES[st], "iterations": int(info.iterations),
                          "refinements": int(info.refinements), "rel_residual": info.rel_residual,
                          "precond_fallback": int(info.precond_fallback)}
        runs["gain_in_inner_iterations"] = (runs["mixed_ir_plain_inner"]["iterations"] /
                                            max(runs["mixed_ir_learned_fcg_inner"]["iterations"], 1))
        runs["gain_in_time"] = runs["mixed_ir_plain_inner"]["ms"] / runs["mixed_ir_learned_fcg_inner"]["ms"]
        res["runs"] = runs
        pc.close()
    finally:
        gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    plan.close()
    del M, N, M32, N32
    torch.cuda.empty_cache()
    return res


def bench_sparse_hbm(gvt, torch, dev, peaks, reps=10):
    """The sparse SIMT stages where HBM binds: a heterodimer-like density (0.2 %) on a
    kernel-filling-sized id space, homogeneous m = q = 20000, 64-d, 800k ordered pairs, the
    Kronecker kernel in FP32 on the SIMT engine.  Per stage kernel: the algorithmic bytes of
    SURVEY-defined minimum traffic (factor and S once, the entries once) per launch over the
    launch's time, against the measured HBM bandwidth (`hbm_frac`), and the bytes the kernel
    streams (one factor row per entry, 4 Y bytes; two rows per sampled dot) at that time."""
    from paper_2009_01054_gb300 import synth
    p = synth.homogeneous(0, m=20000, dim=64, n=800_000)
    H = gvt.Handle()
    M = gvt.gaussian_kernel(H, torch.as_tensor(p.Xd, device=dev), gamma=p.gamma, dtype=torch.float32)
    plan = gvt.Plan(H, (p.m, p.m), (p.m, p.m), p.d, p.t)
    v = torch.as_tensor(p.v, dtype=torch.float32, device=dev)
    gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)
    for _ in range(2):
        gvt.pairwise_kernel_matvec(plan, "kronecker", M, M, v)
    torch.cuda.synchronize()
    gvt.gvt_stats_enable(H.h, True)
    for _ in range(reps):
        gvt.pairwise_kernel_matvec(plan, "kronecker", M, M, v)
    torch.cuda.synchronize()
    st = gvt.gvt_stats_read(H.h)
    gvt.gvt_stats_enable(H.h, False)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {"workload": "homogeneous m=q=20000, 64-d, 800k uniform ordered pairs (0.2 %, heterodimer-like), "
                       "Kronecker kernel, FP32 SIMT stages", "hbm_peak_gbs": hbm}
    for k, stream_bytes in (("sparse_stage1", 4.0 * p.m * p.n), ("sparse_stage2", 2 * 4.0 * p.m * p.n)):
        r = st[k]
        ms = r["ms"] / max(r["launches"], 1)
        ab = r["bytes"] / max(r["launches"], 1)
        out[k] = {"ms_per_launch": ms, "algorithmic_gbs": ab / (ms / 1e3) / 1e9,
                  "hbm_frac": ab / (ms / 1e3) / 1e9 / hbm,
                  "useful_tflops": r["useful_flops"] / max(r["launches"], 1) / (ms / 1e3) / 1e12,
                  "streamed_gbs": stream_bytes / (ms / 1e3) / 1e9}
    plan.close()
    H.close()
    return out


def bench_batched(H, gvt, torch, dev, n_probs, sample=32):
    """Batched uneven problems: n_probs KRR problems (m, q ~ U{32..512}, density ~ U[5%, 60%],
    32-d features, Kronecker of Gaussians) x 16 lambdas (logspace 1e-4..1) in one batched solve to
    FP64 rel. residual 1e-6.  The speed-up over plain FP64 CG is measured on a stratified sample
    (every k-th problem): the sample is solved batched, and by plain FP64 CG system by system."""
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

    def solve_on(engine, problems):
        gvt.gvt_set_stage1_engine(H.h, engine)
        try:
            # first call includes the autotuner; time the second (tuned, cached) call
            gvt.krr_solve_batched(H, problems, lambdas, rel_tol=1e-6)
            return timed_solve(torch, lambda: gvt.krr_solve_batched(H, problems, lambdas, rel_tol=1e-6))
        finally:
            gvt.gvt_set_stage1_engine(H.h, gvt.GVT_STAGE1_SIMT)

    (A, st, info, rr), batched_ms = solve_on(gvt.GVT_STAGES_AUTO, probs)
    (_, st_s, info_s, rr_s), simt_ms = solve_on(gvt.GVT_STAGE1_SIMT, probs)
    worst = max(max(r) for r in rr)
    out = {"workload": "%d problems, m,q ~ U{32..512}, density ~ U[5%%,60%%], 32-d, %d lambdas logspace(-4,0), "
                       "%d pairs total, %d systems" % (len(ps), len(lambdas), total_pairs, len(ps) * len(lambdas)),
           "engine": "auto: tensor-core stages (FP16x3, grouped GEMMs) for the problems the cost model picks, "
                     "SIMT stages for the others",
           "batched_ms": batched_ms, "status": gvt.STATUS_NAMES[st], "inner_iterations": int(info.iterations),
           "refinements": int(info.refinements), "max_rel_residual": worst, "data_generation_s": gen_s,
           "simt_engine": {"batched_ms": simt_ms, "status": gvt.STATUS_NAMES[st_s],
                           "inner_iterations": int(info_s.iterations), "refinements": int(info_s.refinements),
                           "max_rel_residual": max(max(r) for r in rr_s)}}
    if sample > 0:
        step = max(1, len(ps) // sample)
        sel = list(range(0, len(ps), step))[:sample]
        sub = [probs[b] for b in sel]
        (A2, st2, info2, rr2), sub_ms = solve_on(gvt.GVT_STAGES_AUTO, sub)
        per = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fp_worst = 0.0
        for b in sel:
            p = probs[b]
            plan = gvt.Plan(H, tuple(p["M"].shape), tuple(p["N"].shape), p["d"], p["t"])
            its = []
            for lam in lambdas:
                a, st3, inf3 = gvt.krr_cg_solve(H, plan, "kronecker", p["M"], p["N"], p["y"], lam, max_iter=50000,
                                                check_every=2)
                its.append(int(inf3.iterations))
                fp_worst = max(fp_worst, inf3.rel_residual)
            plan.close()
            per.append({"problem": b, "m": ps[b].m, "q": ps[b].q, "n": ps[b].n, "fp64_cg_iterations": its})
        torch.cuda.synchronize()
        fp_ms = (time.perf_counter() - t0) * 1e3
        out["sample"] = {"problems": len(sel), "systems": len(sel) * len(lambdas),
                         "pairs": sum(ps[b].n for b in sel), "batched_ms": sub_ms,
                         "batched_status": gvt.STATUS_NAMES[st2], "batched_max_rel_residual": max(max(r) for r in rr2),
                         "plain_fp64_cg_ms": fp_ms, "plain_fp64_cg_max_rel_residual": fp_worst,
                         "speedup_vs_plain_fp64_cg": fp_ms / sub_ms, "per_problem": per,
                         "note": "measured on the same problems: batched solve vs plain FP64 CG system by system"}
    return out


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    run_gvt(args, ws, rank, local)


if __name__ == "__main__":
    main()
