"""Benchmark: time to the k dominant POD modes with the GB300 ISMA library.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Headline workload (the largest single-GPU configuration of the method's
benchmark set): planted-1000000x4000-f32, a planted spectrum
sigma_i = exp(-i/15) over 200 modes (Haar factors) plus N(0, 1e-4^2) noise,
rows centred, stored FP32 (16 GB); k = 50 modes, c = 100 columns per
iteration, uniform sampling after the column-norm round, subspace tolerance
1e-8 (the loop runs until every column is merged), closing refinement
QR(A^T U), SVD(R).  The FP32 flow workload (316 x 316 grid x 2000
snapshots, k = 20, c = 40) is timed beside it under "flow_316".

One step = one whole problem: pod_reset (column norms, state) + every ISMA
round + pod_modes (refinement, sign fix, copy-out).  `value` is the device
time of a step with A resident in HBM (16 GB, far larger than the 129 MB L2,
so no flush between steps); `e2e` is the same step through the C ABI with
the host->device copy of A from pinned memory and the device->host copy of
U and sigma inside the timed region.

N > 1 (torchrun): independent replicas, one problem per GPU, no collective
on the data path; the timed region is bracketed by a barrier and the max
over ranks is reported.

--impl reference times the FP64 CPU oracle (oracle/isma.py) on the host
cores.  Each step runs the next few units of the problem (column norms, one
ISMA round each, the refinement), resuming where the previous step stopped
and starting over after the refinement, so that the timed steps cover the
whole problem; `value` adds up the measured units of one complete problem.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-k-POD-modes (s)"
SEED_SAMPLING = 0x5107
HEAD = dict(workload="planted-1000000x4000-f32", k=50, c=100, tol=1e-8)
FLOW = dict(workload="flow-316x316x2000-f32", k=20, c=40, tol=1e-8)

# FP32 SIMT peak of a GB300 from its unit counts and clock: 152 SMs x 128
# FP32 lanes x 2 flop (FMA) x 2.07 GHz; and the same for one SM.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP32_SM_PEAK_GFLOPS = 128 * 2 * 2.07e9 / 1e9
# nominal dense TF32 / BF16 tensor rate ratio (1.1 / 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25

# DRAM bytes per launch from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the kernel as it was when captured; the hash of
# its sources at that time guards against reporting stale counters.
NCU_TRAFFIC = {
    # one k_core launch (n_c = 150, the headline's core size; its traffic does
    # not depend on m) of bench.py --only-head --m 262144 --n 2048
    "core_svd": {"bytes": 592128, "src_sha": "6dcad455dd784916"},
}
KERNEL_SOURCES = {
    "core_svd": ["paper_1905_05107_gb300/csrc/small.cu", "paper_1905_05107_gb300/csrc/common.cuh",
                 "paper_1905_05107_gb300/csrc/pod_internal.h"],
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # profiling runs: the headline workload alone (no flow, precision,
    # differentiable or CPU legs), optionally at reduced m x n; the timed
    # steps sit inside the NVTX range "timed" (ncu --nvtx --nvtx-include timed/)
    ap.add_argument("--only-head", action="store_true")
    ap.add_argument("--m", type=int, default=0)
    ap.add_argument("--n", type=int, default=0)
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(value, world, device):
    """The largest of every rank's value (the slowest replica sets the time);
    `device` is where the collective's buffer lives (cuda for NCCL, cpu for
    gloo)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def sources_sha(kernel):
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    rec = NCU_TRAFFIC.get(kernel)
    if not rec or rec["src_sha"] != sources_sha(kernel):
        return None
    return rec["bytes"]


def load_peaks():
    """(HBM GB/s, BF16 dense TFLOP/s burst, BF16 sustained, source)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return (float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1902.8)),
                float(d.get("bf16_tflops_sustained", d.get("bf16_tflops", 1710.0))), "measured")
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def make_head(m=0, n=0):
    from paper_1905_05107_gb300 import synth
    if m or n:
        return synth.make_precision_c3(m=m or 1_000_000, n=n or 4000)
    return synth.make_precision_c3()      # (m, n) Fortran-ordered float32


def shared_head(m, n, local, world):
    """The headline matrix for N > 1 replicas: local rank 0 generates it once
    into /dev/shm and every rank maps that file (one host copy instead of one
    per rank, whose FP64 generation buffers alone would not fit N = 8 on one
    host).  Returns (A as an (m, n) Fortran-ordered view, path) or (None,
    None) when /dev/shm is missing or too small (each rank then generates its
    own)."""
    import shutil
    import torch.distributed as dist
    mm = m or 1_000_000
    nn = n or 4000
    path = "/dev/shm/pod_bench_head_%dx%d.f32" % (mm, nn)
    nbytes = mm * nn * 4
    try:
        ok = shutil.disk_usage("/dev/shm").free > nbytes + (1 << 30) or os.path.exists(path)
    except OSError:
        ok = False
    flag = [1 if ok else 0]
    if world > 1:
        import torch
        t = torch.tensor(flag, dtype=torch.int32, device="cuda" if dist.get_backend() == "nccl" else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        flag = [int(t.item())]
    if not flag[0]:
        return None, None
    if local == 0:
        A = make_head(m, n)
        tmp = path + ".tmp"
        np.ascontiguousarray(A.T).tofile(tmp)   # (n, m) rows = the columns of A
        del A
        os.replace(tmp, path)
    barrier(world)
    At = np.memmap(path, dtype=np.float32, mode="r+", shape=(nn, mm))
    return At.T, path


def make_flow():
    from paper_1905_05107_gb300 import synth
    return synth.make_flow_316()


def cpu_cores():
    return os.cpu_count() or 1


def floor_u(sig_E_like, k, u):
    """Predicted accuracy floor u sigma_1 / (sigma_k - sigma_{k+1})."""
    s = np.asarray(sig_E_like)
    if s.size <= k:
        return None
    return float(u * s[0] / max(s[k - 1] - s[k], 1e-300))


# ---------------------------------------------------------------- CPU oracle
def oracle_params(w):
    from oracle import isma as O
    return O.Params(k=w["k"], c=w["c"], tol=w["tol"], refine=True, seed=SEED_SAMPLING)


def oracle_full(A, w):
    """One whole FP64 oracle run on the host cores: (seconds, Result)."""
    from oracle import isma as O
    A64 = np.asarray(A, dtype=np.float64)
    t0 = time.perf_counter()
    res = O.isma(A64, oracle_params(w))
    return time.perf_counter() - t0, res


def run_reference(args):
    """The FP64 oracle as it stands, on the host cores, in bounded steps that
    together cover the whole problem (see the module docstring)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import isma as O
    A = make_head()
    A64 = np.asarray(A, dtype=np.float64)
    del A
    m, n = A64.shape
    # units of one problem: column norms, T rounds, refinement; T from the
    # draws alone (UNF after round 0 until S is empty; identical on every
    # implementation)
    in_S = np.ones(n, dtype=bool)
    s = O.column_sq_norms(A64)
    rounds = 0
    while in_S.any():
        vals = s if rounds == 0 else np.ones(n)
        idx, _ = O.sample_columns(vals, in_S, HEAD["c"], SEED_SAMPLING, rounds)
        in_S[idx] = False
        rounds += 1
    units_total = rounds + 2
    per_step = max(1, math.ceil(units_total / max(args.steps, 1)))
    gen = [None]
    pos = [0]

    def next_unit():
        if gen[0] is None:
            gen[0] = O.isma_steps(A64, oracle_params(HEAD))
            pos[0] = 0
        t0 = time.perf_counter()
        kind, _ = next(gen[0])
        dt = time.perf_counter() - t0
        u = pos[0]
        pos[0] += 1
        if kind == "done":
            gen[0] = None
        return u, dt

    for _ in range(args.warmup):
        for _ in range(per_step):
            next_unit()
    measured = {}
    step_s = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step):
            u, dt = next_unit()
            measured.setdefault(u, dt)
        step_s.append(time.perf_counter() - t0)
    covered = len(measured)
    if covered >= units_total:
        value = float(sum(measured[u] for u in range(units_total)))
        how = "every unit measured"
    else:
        rmean = np.mean([measured[u] for u in measured if 0 < u < units_total - 1] or [0.0])
        value = float(sum(measured.values()) + rmean * (units_total - covered))
        how = "%d of %d units measured, the rest at the measured mean round time" % (covered, units_total)
    sample = ("FP64 NumPy/LAPACK oracle (Algorithm 1 with its QR and SVD steps from LAPACK) on %d host "
              "cores; the problem is cut into %d units (column norms, %d rounds, refinement), each step runs "
              "the next %d, resuming the previous step's state; value = one whole problem's units (%s)"
              % (cpu_cores(), units_total, rounds, per_step, how))
    ms = 1e3 * float(np.mean(step_s))
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": HEAD["workload"], "m": int(m), "n": int(n), "k": HEAD["k"], "c": HEAD["c"],
                       "tol": HEAD["tol"], "rounds": rounds, "strategy": "L2N round 0, UNF after"},
            "cpu_baseline": {"value": value, "unit": "s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
def kernel_model(m, es, r, g):
    """Algorithmic bytes and flops per launch of the round's streaming passes
    (what the method must move)."""
    return {
        "proj": (m * (r + g) * es, 2.0 * m * r * g),
        # CGS: read U, C; write Z = C - U P.  Z = C - U P, P2 = U^T Z, Z^T Z
        "cgs_gram": (m * (r + g) * es + m * g * es, 4.0 * m * r * g + 1.0 * m * g * g),
        # QR2: read U, Z; write W over Z.  Z - U P2, W = (.) M1 (triangular), W^T W
        "qr2_gram": (m * (r + g) * es + m * g * es, 2.0 * m * r * g + 2.0 * m * g * g),
        "update": (m * (r + g) * es + m * r * es, 2.0 * m * (r + g) * r),
    }


def time_problem(torch, pod, A_np, w, steps, warmup, dev, world, detail, register=False):
    """Device-timed and end-to-end steps of one workload; with `detail`, also
    per-kernel timings, core statistics and the refinement's A^T U.  With
    `register`, the host matrix (a shared mapping) is page-locked in place
    instead of copied into pinned memory."""
    m, n = A_np.shape
    k = w["k"]
    A_t = torch.from_numpy(np.ascontiguousarray(A_np.T))   # (n, m) = column-major A
    if register:
        cudart = torch.cuda.cudart()
        rc = cudart.cudaHostRegister(A_t.data_ptr(), A_t.numel() * A_t.element_size(), 0)
        if rc != cudart.cudaError.success:
            raise RuntimeError("cudaHostRegister failed (%s)" % rc)
        A_host = A_t
    else:
        A_host = A_t.pin_memory()
    A_dev_t = A_host.to(dev)
    A = A_dev_t.t()
    stream = torch.cuda.Stream(dev)
    out = {}
    with torch.cuda.stream(stream):
        ctx = pod.Context(A, k, w["c"], tol=w["tol"], stream=stream)

        def step():
            ctx.reset()
            ctx.iterate()
            return ctx.modes()

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        rounds = ctx.counters()[1]
        barrier(world)
        torch.cuda.synchronize()
        clocks = ClockSampler(dev.index) if detail else None
        if clocks:
            clocks.start()
        l0, _ = ctx.counters()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for _ in range(steps):
            U, sigma, _ = step()
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        l1, _ = ctx.counters()
        out["clocks"] = clocks.stop() if clocks else None
        ms = e0.elapsed_time(e1) / steps
        out["ms"] = max_over_ranks(ms, world, dev)
        out["launches"] = (l1 - l0) // steps
        out["rounds"] = rounds
        out["U"] = U.double().cpu().numpy()
        out["sigma"] = sigma.cpu().numpy()
        barrier(world)
        # ------------------------------------------------ end-to-end steps
        U_host = torch.empty((k, m), dtype=torch.float32).pin_memory()
        s_host = torch.empty(k, dtype=torch.float64).pin_memory()

        def step_e2e():
            A_dev_t.copy_(A_host, non_blocking=True)
            U, sigma, _ = step()
            U_host.copy_(U.t(), non_blocking=True)
            s_host.copy_(sigma, non_blocking=True)

        step_e2e()
        torch.cuda.synchronize()
        barrier(world)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(steps):
            step_e2e()
        f1.record(stream)
        torch.cuda.synchronize()
        out["ms_e2e"] = max_over_ranks(f0.elapsed_time(f1) / steps, world, dev)
        out["h2d"] = int(m * n * 4)
        out["d2h"] = int(m * k * 4 + k * 8)
        if detail:
            # one more run, round by round, with CUDA events between kernels
            ctx.reset()
            per, rg, sweeps, core_cyc = {}, [], [], []
            for t in range(rounds):
                for kname, v in ctx.round_timings().items():
                    per.setdefault(kname, []).append(v)
                rg.append(len(ctx.trace(t)[0]))
                sw, cyc = ctx.core_stats()
                sweeps.append(sw)
                core_cyc.append(cyc)
            ref = ctx.refine_timings()
            ctx.modes()
            per["refine_atu"] = [ref["atu"]]
            per["refine_rest"] = [sum(v for kk, v in ref.items() if kk != "atu")]
            cn = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            torch.cuda.synchronize()
            cn[0].record(stream)
            reps = 3
            for _ in range(reps):
                pod.colnorms(A, stream=stream)
            cn[1].record(stream)
            torch.cuda.synchronize()
            per["colnorms"] = [cn[0].elapsed_time(cn[1]) / reps]
            out.update(per=per, rg=rg, sweeps=sweeps, core_cyc=core_cyc)
        ctx.close()
    del A_dev_t
    if register:
        torch.cuda.cudart().cudaHostUnregister(A_host.data_ptr())
    del A_host
    torch.cuda.empty_cache()
    return out


def roofline_of(t, m, n, k, hbm, bf16, tc_proj):
    """The dominant kernel's roofline plus every kernel's fractions, from the
    per-kernel timings of one run.  The round's FP32 SIMT passes are bound by
    whichever of HBM bytes and FP32 flops they are closer to; the tensor-core
    contractions by HBM bytes (their split products keep the tensor pipe far
    from busy), with the tensor-pipe fraction beside it."""
    per, rg, sweeps = t["per"], t["rg"], t["sweeps"]
    es = 4
    totals = {kname: float(np.sum(v)) for kname, v in per.items()}
    dominant = max(totals, key=totals.get)
    moved, flops = {}, {}
    for i, g in enumerate(rg):
        mdl = kernel_model(m, es, 0 if i == 0 else k, g)
        for kname in ("proj", "cgs_gram", "qr2_gram", "update"):
            moved[kname] = moved.get(kname, 0.0) + mdl[kname][0]
            flops[kname] = flops.get(kname, 0.0) + mdl[kname][1] * (3 if (kname == "proj" and tc_proj) else 1)
    moved["colnorms"] = float(m * n * es + n * 8)
    flops["colnorms"] = 2.0 * m * n
    moved["refine_atu"] = float(m * n * es + m * k * es)
    flops["refine_atu"] = 3 * 2.0 * m * n * k
    tf32_peak = bf16 * TF32_PER_BF16
    tensor = {"proj"} if tc_proj else set()
    tensor.add("refine_atu")
    kernels = {}
    for kname in moved:
        if kname not in totals or totals[kname] <= 0:
            continue
        sec = totals[kname] * 1e-3
        gbs = moved[kname] / sec / 1e9
        tfs = flops[kname] / sec / 1e12
        peak_f = tf32_peak if kname in tensor else FP32_PEAK_TFLOPS
        kernels[kname] = {"GB/s": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4), "TFLOP/s": round(tfs, 2),
                          "flop_frac": round(tfs / peak_f, 4),
                          "flop_peak": "TF32 tensor" if kname in tensor else "FP32 SIMT"}
    core_flops = 0.0
    for i, g in enumerate(rg):
        nc = (0 if i == 0 else k) + g
        core_flops += 6.0 * nc ** 3 * (sweeps[i] if i < len(sweeps) else 0)
    if dominant == "core_svd":
        launches_k = len(per["core_svd"])
        avg_ms = totals["core_svd"] / launches_k
        achieved = core_flops / launches_k / (avg_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "core_svd", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": ncu_traffic("core_svd"),
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (FP32 FMA)",
                "algorithmic_flops_per_launch": core_flops / launches_k, "avg_launch_ms": avg_ms,
                "note": "one CTA on one of 152 SMs, latency-bound Jacobi rounds; frac of that SM's "
                        "FP32 peak: %.4f" % (achieved * 1e3 / FP32_SM_PEAK_GFLOPS)}
    else:
        kk = dominant if dominant in kernels else max((x for x in totals if x in kernels), key=totals.get)
        launches_k = len(per[kk])
        avg_ms = totals[kk] / launches_k
        kr = kernels[kk]
        if kk not in tensor and kr["flop_frac"] > kr["hbm_frac"]:
            roof = {"bound": "alu", "kernel": kk, "achieved": flops[kk] / launches_k / (avg_ms * 1e-3) / 1e12,
                    "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "traffic": ncu_traffic(kk),
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (FP32 FMA)",
                    "algorithmic_flops_per_launch": flops[kk] / launches_k, "avg_launch_ms": avg_ms,
                    "hbm_frac": kr["hbm_frac"]}
        else:
            roof = {"bound": "hbm", "kernel": kk, "achieved": moved[kk] / launches_k / (avg_ms * 1e-3) / 1e9,
                    "peak": hbm, "unit": "GB/s", "traffic": ncu_traffic(kk),
                    "algorithmic_bytes_per_launch": moved[kk] / launches_k, "avg_launch_ms": avg_ms}
        roof["frac"] = roof["achieved"] / roof["peak"]
    roof["time_share"] = {x: round(totals[x] / sum(totals.values()), 4) for x in totals}
    roof["dominant_kernel"] = dominant
    roof["kernels"] = kernels
    return roof


def sin_max(U, W):
    """Largest sine of the principal angles between span(U) and span(W)
    (orthonormal columns): |(I - U U^T) W|_2."""
    return float(np.linalg.norm(W - U @ (U.T @ W), 2))


def accuracy(U, sigma, ref, k):
    """sigma relative errors and sin(theta) of the top-j subspaces against the
    oracle's result, with the FP32 floor u sigma_1 / gap_j of the oracle's
    spectrum."""
    u32 = 5.96e-8
    rel = np.abs(sigma - ref.sigma) / ref.sigma
    sall = ref.sigma_all if ref.sigma_all is not None else ref.sigma
    out = {"sigma_rel_max": float(rel.max())}
    for j in sorted({10, 20, 30, 40, k}):
        if j > k:
            continue
        out["sin_top%d" % j] = sin_max(ref.U[:, :j], U[:, :j])
        out["floor_top%d" % j] = floor_u(sall, j, u32)
    out["sigma_rel_top20"] = float(rel[:20].max())
    return out


def precision_forms(torch, pod, A_np, w, dev, steps=3):
    """The same workload with U^T C and A^T U in split BF16 and in BF16 on
    the tensor cores (and split TF32, the headline's form, for the same-run
    comparison): device time per problem and the modes for the accuracy
    report."""
    A = torch.from_numpy(np.ascontiguousarray(A_np.T)).to(dev).t()
    stream = torch.cuda.Stream(dev)
    out = {}
    with torch.cuda.stream(stream):
        for prec in ("tf32x3", "bf16x3", "bf16"):
            ctx = pod.Context(A, w["k"], w["c"], tol=w["tol"], stream=stream, precision=prec)

            def step():
                ctx.reset()
                ctx.iterate()
                return ctx.modes()

            step()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                U, sigma, _ = step()
            e1.record(stream)
            torch.cuda.synchronize()
            out[prec] = {"ms_per_step": e0.elapsed_time(e1) / steps, "rounds": ctx.counters()[1],
                         "U": U.double().cpu().numpy(), "sigma": sigma.cpu().numpy()}
            ctx.close()
    del A
    torch.cuda.empty_cache()
    return out


def differentiable_form(torch, pod, dev, reps=3):
    """The differentiation workload (planted 200000 x 1000 FP32, k = 16,
    c = 32; loss sum_i w_i (u_i^T g)^2): the plain forward, the forward that
    records the tape, and pod_backward, device times; the taped forward's
    modes against the plain forward's (equal subspace accuracy)."""
    from paper_1905_05107_gb300 import synth
    A_np = synth.make_diff_c4()
    A = torch.from_numpy(np.ascontiguousarray(A_np.T)).to(dev).t()
    wv, gv = synth.diff_loss_weights(16, A_np.shape[0])
    stream = torch.cuda.Stream(dev)
    res = {"workload": "planted-200000x1000-f32-diff", "k": 16, "c": 32}
    with torch.cuda.stream(stream):
        def timed(fn):
            fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps, out

        plain = pod.Context(A, 16, 32, tol=1e-8, stream=stream)

        def fwd_plain():
            plain.reset()
            plain.iterate()
            return plain.modes()

        res["forward_ms"], (U0, s0, _) = timed(fwd_plain)
        plain.close()
        gt = torch.as_tensor(gv, dtype=torch.float32, device=dev)
        wt = torch.as_tensor(wv, dtype=torch.float64, device=dev)

        def fwd_tape():
            ctx = pod.Context(A, 16, 32, tol=1e-8, stream=stream, keep_tape=True)
            ctx.iterate()
            U, s, _ = ctx.modes()
            return ctx, U, s

        ms, (ctx, U1, s1) = timed(lambda: fwd_tape())
        res["forward_tape_ms"] = ms
        proj = U1.t().double() @ gt.double()
        dU = (gt.double()[:, None] * (2.0 * wt * proj)[None, :]).float()
        res["backward_ms"], _ = timed(lambda: ctx.backward(dU))
        ctx.close()
        u0, u1 = U0.double().cpu().numpy(), U1.double().cpu().numpy()
        res["sin_tape_vs_plain"] = sin_max(u0, u1)
    del A
    torch.cuda.empty_cache()
    return res


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1905_05107_gb300 import build, pod
    build.build()
    shm_path = None
    if world > 1:
        A_np, shm_path = shared_head(args.m, args.n, local, world)
    if shm_path is None:
        A_np = make_head(args.m, args.n)
    m, n = A_np.shape
    k = HEAD["k"]
    head = dict(HEAD)
    if (m, n) != (1_000_000, 4000):
        head["workload"] = "planted-%dx%d-f32" % (m, n)
    t = time_problem(torch, pod, A_np, head, args.steps, args.warmup, dev, world, detail=True,
                     register=shm_path is not None)
    hbm, bf16, bf16_sus, peak_kind = load_peaks()
    roof = roofline_of(t, m, n, k, hbm, bf16, tc_proj=True)
    roof["peak_source"] = roof.get("peak_source", "%s: MEASURED_PEAKS.json hbm_gbs" % peak_kind)
    roof["tensor_peak_source"] = ("%s: MEASURED_PEAKS.json bf16_tflops x nominal TF32/BF16 ratio (1.1 / 2.25)"
                                  % peak_kind)
    core_phase = np.mean(np.array(t["core_cyc"], dtype=np.float64), axis=0).tolist()
    flow, forms, diff = None, None, None
    if not args.only_head:
        # the FP32 flow workload beside it
        F_np = make_flow()
        tf = time_problem(torch, pod, F_np, FLOW, args.steps, args.warmup, dev, world, detail=False)
        flow = {"workload": FLOW["workload"], "m": int(F_np.shape[0]), "n": int(F_np.shape[1]), "k": FLOW["k"],
                "c": FLOW["c"], "rounds": tf["rounds"], "ms_per_step": tf["ms"], "e2e_ms": tf["ms_e2e"],
                "gpu_launches": int(tf["launches"])}
        del F_np
        forms = precision_forms(torch, pod, A_np, head, dev) if world == 1 else None
        diff = differentiable_form(torch, pod, dev) if world == 1 else None
    cpu, acc = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.only_head:
        secs, ref = oracle_full(A_np, head)
        cpu = {"value": secs, "unit": "s", "cores": cpu_cores(), "kind": "oracle",
               "sample": "the whole problem once: FP64 NumPy/LAPACK oracle (Algorithm 1, %d rounds, refinement) "
                         "on the host cores" % len(ref.trace)}
        acc = accuracy(t["U"], t["sigma"], ref, k)
        acc["rounds_equal"] = int(len(ref.trace) == t["rounds"])
        if forms:
            for name, f in forms.items():
                f["accuracy_vs_oracle"] = accuracy(f.pop("U"), f.pop("sigma"), ref, k)
    if forms:
        for f in forms.values():
            f.pop("U", None)
            f.pop("sigma", None)
    if rank == 0:
        line = {"metric": METRIC, "value": t["ms"] / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t["ms"], "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": head["workload"], "m": int(m), "n": int(n), "k": k, "c": HEAD["c"],
                           "tol": HEAD["tol"], "rounds": t["rounds"], "strategy": "L2N round 0, UNF after",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "contractions": "A^T U on tcgen05 tensor cores, split-TF32 (3 products)",
                           "l2": "A is 16 GB, larger than the 129 MB L2: no flush between steps"},
                "e2e": {"value": t["ms_e2e"] / 1e3, "unit": "s", "h2d_bytes_per_step": t["h2d"],
                        "d2h_bytes_per_step": t["d2h"]},
                "gpu_launches": int(t["launches"]),
                "accuracy_vs_oracle": acc,
                "core_svd": {"jacobi_sweeps_mean": float(np.mean(t["sweeps"])),
                             "jacobi_sweeps_max": int(np.max(t["sweeps"])),
                             "phase_cycles_mean": {kk: round(v) for kk, v in zip(
                                 ["chol2_and_E", "jacobi", "finish", "convergence", "coefficients", "total"],
                                 core_phase)}},
                "roofline": roof,
                "flow_316": flow,
                "precision_forms": forms,
                "differentiable_form": diff,
                "clocks": t["clocks"],
                "cpu_baseline": cpu}
        print(json.dumps(line))
    if world > 1:
        if shm_path is not None:
            del A_np
            barrier(world)   # every rank is done with the shared matrix
            if local == 0:
                try:
                    os.remove(shm_path)
                except OSError:
                    pass
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
