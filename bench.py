"""Benchmark: time to the k dominant POD modes with the GB300 ISMA library.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (the FP32 configuration of the method's benchmark): synthetic
flow-like snapshots on a 316 x 316 grid (m = 99856) x n = 2000 time steps,
60 separable travelling waves with amplitudes j^-1.5 plus N(0, 1e-3^2)
noise, rows centred; k = 20 modes, c = 40 columns per iteration, uniform
sampling after the column-norm round, subspace tolerance 1e-8 (the loop runs
until every column is merged), closing refinement QR(A^T U), SVD(R).

One step = one whole problem: pod_reset (column norms, state) + every ISMA
round + pod_modes (refinement, sign fix, copy-out).  `value` is the device
time of a step with A resident in HBM (0.8 GB, larger than the 129 MB L2, so
no flush between steps); `e2e` is the same step through the C ABI with the
host->device copy of A from pinned memory and the device->host copy of U and
sigma inside the timed region.

N > 1 (torchrun): independent replicas, one problem per GPU, no collective
on the data path; the timed region is bracketed by a barrier and the max
over ranks is reported.

--impl reference times the FP64 CPU oracle (oracle/isma.py) on the host
cores on a bounded sample of the same problem (see `cpu_baseline.sample`).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

K_MODES, C_DRAWS, TOL = 20, 40, 1e-8
METRIC = "time-to-k-POD-modes (s)"
WORKLOAD = "flow-316x316x2000-f32"

# FP32 SIMT peak of a GB300 from its unit counts and clock: 152 SMs x 128
# FP32 lanes x 2 flop (FMA) x 2.07 GHz; and the same for one SM.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP32_SM_PEAK_GFLOPS = 128 * 2 * 2.07e9 / 1e9

# DRAM bytes per launch from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the kernel as it was when captured; the hash of
# its sources at that time guards against reporting stale counters.
NCU_TRAFFIC = {
    # profiles/k_core_flow316x316x2000_f32.md: 281.6 KB read, 0 written
    "core_svd": {"bytes": 281600, "src_sha": "e1e94b5850f01494"},
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
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1902.8)), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


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


def make_input():
    from paper_1905_05107_gb300 import synth
    return synth.make_flow_316()          # (m, n) Fortran-ordered float32


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(A, rounds_total, sample_rounds=3):
    """The FP64 oracle on a bounded sample of the problem: column norms and
    the refinement are timed in full; `sample_rounds` ISMA rounds are timed
    and scaled to the rounds the whole problem needs."""
    from oracle import isma as O
    A64 = A.astype(np.float64)
    t0 = time.perf_counter()
    O.column_sq_norms(A64)
    t_norms = time.perf_counter() - t0
    p = O.Params(k=K_MODES, c=C_DRAWS, tol=TOL, refine=False, max_iter=sample_rounds - 1, seed=0x5107)
    t0 = time.perf_counter()
    res = O.isma(A64, p)
    t_isma = time.perf_counter() - t0
    t_round = max(t_isma - t_norms, 0.0) / max(len(res.trace), 1)
    t0 = time.perf_counter()
    O.refine(A64, res.U)
    t_ref = time.perf_counter() - t0
    value = t_norms + rounds_total * t_round + t_ref
    return value, dict(t_norms=t_norms, t_round=t_round, t_refine=t_ref, rounds=len(res.trace))


def cpu_cores():
    return os.cpu_count() or 1


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    A = make_input()
    # rounds of the whole problem: UNF draws until S is empty (identical on
    # every implementation); counted with the oracle's sampler alone
    from oracle import isma as O
    n = A.shape[1]
    in_S = np.ones(n, dtype=bool)
    s = O.column_sq_norms(A.astype(np.float64))
    rounds = 0
    while in_S.any():
        vals = s if rounds == 0 else np.ones(n)
        idx, _ = O.sample_columns(vals, in_S, C_DRAWS, 0x5107, rounds)
        in_S[idx] = False
        rounds += 1
    times = []
    for i in range(args.warmup + args.steps):
        v, parts = oracle_sample(A, rounds)
        if i >= args.warmup:
            times.append(v)
    value = float(np.mean(times))
    sample = ("FP64 NumPy/LAPACK oracle on the host: column norms and refinement in full, %d of %d "
              "ISMA rounds timed and scaled; mean of %d steps" % (parts["rounds"], rounds, args.steps))
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "m": int(A.shape[0]), "n": int(A.shape[1]), "k": K_MODES,
                       "c": C_DRAWS, "rounds": rounds},
            "cpu_baseline": {"value": value, "unit": "s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
def kernel_model(m, n, es, r, g):
    """Algorithmic bytes and flops per launch (what the method must move)."""
    return {
        "colnorms": (m * n * es + n * 8, 2.0 * m * n),
        "proj": (m * (r + g) * es, 2.0 * m * r * g),
        "cgs_gram": (m * (r + g) * es, 4.0 * m * r * g + 1.0 * m * g * g),
        "qr2_gram": (m * (r + g) * es, 4.0 * m * r * g + 2.0 * m * g * g),
        "update": (m * (r + g) * es + m * r * es, 2.0 * m * (r + g) * r),
    }


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
    A_np = make_input()
    m, n = A_np.shape
    es = 4
    A_host = torch.from_numpy(np.ascontiguousarray(A_np.T)).pin_memory()   # (n, m) = column-major A
    A_dev_t = A_host.to(dev)
    A = A_dev_t.t()
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        ctx = pod.Context(A, K_MODES, C_DRAWS, tol=TOL, stream=stream)

        def step():
            ctx.reset()
            ctx.iterate()
            return ctx.modes()

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        rounds = ctx.counters()[1]
        # ------------------------------------------------ device-timed steps
        barrier(world)
        torch.cuda.synchronize()
        clocks = ClockSampler(dev.index)
        clocks.start()
        l0, _ = ctx.counters()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            U, sigma, _ = step()
        e1.record(stream)
        torch.cuda.synchronize()
        l1, _ = ctx.counters()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1) / args.steps
        ms = max_over_ranks(ms, world, dev)
        barrier(world)
        launches = (l1 - l0) // args.steps
        # ------------------------------------------------ end-to-end steps
        U_host = torch.empty((K_MODES, m), dtype=torch.float32).pin_memory()
        s_host = torch.empty(K_MODES, dtype=torch.float64).pin_memory()

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
        for _ in range(args.steps):
            step_e2e()
        f1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = f0.elapsed_time(f1) / args.steps
        ms_e2e = max_over_ranks(ms_e2e, world, dev)
        # ------------------------------------------------ per-kernel timings
        # one more run, round by round, with CUDA events between kernels
        ctx.reset()
        per = {}
        rg = []
        sweeps, core_cyc = [], []
        for t in range(rounds):
            for kname, v in ctx.round_timings().items():
                per.setdefault(kname, []).append(v)
            rg.append(len(ctx.trace(t)[0]))
            sw, cyc = ctx.core_stats()
            sweeps.append(sw)
            core_cyc.append(cyc)
        ctx.modes()
        cn = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        cn[0].record(stream)
        reps = 5
        for _ in range(reps):
            pod.colnorms(A, stream=stream)
        cn[1].record(stream)
        torch.cuda.synchronize()
        per["colnorms"] = [cn[0].elapsed_time(cn[1]) / reps]
        # refinement + copy-out, once
        ctx.reset()
        ctx.iterate()
        mm = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        mm[0].record(stream)
        ctx.modes()
        mm[1].record(stream)
        torch.cuda.synchronize()
        per["modes_refine"] = [mm[0].elapsed_time(mm[1])]
        ctx.close()

    totals = {kname: float(np.sum(v)) for kname, v in per.items()}
    dominant = max(totals, key=totals.get)
    hbm, bf16, peak_kind = load_peaks()
    # algorithmic bytes of every launch of each streaming kernel (round t has
    # r_t = 0 modes in round 0 and K_MODES after, g_t distinct columns)
    moved = {}
    for t, g in enumerate(rg):
        mdl = kernel_model(m, n, es, 0 if t == 0 else K_MODES, g)
        for kname in ("proj", "cgs_gram", "qr2_gram", "update"):
            moved[kname] = moved.get(kname, 0.0) + mdl[kname][0]
    moved["colnorms"] = kernel_model(m, n, es, K_MODES, C_DRAWS)["colnorms"][0] * len(per["colnorms"])
    hbm_kernels = {}
    for kname, b in moved.items():
        gbs = b / (totals[kname] * 1e-3) / 1e9
        hbm_kernels[kname] = {"GB/s": round(gbs, 1), "frac": round(gbs / hbm, 4)}
    # the core SVD: one CTA, one-sided Jacobi on the (r + g)-wide core;
    # algorithmic flops 6 n_c^3 per sweep (n_c = r_t + g_t)
    core_flops = 0.0
    for t, g in enumerate(rg):
        nc = (0 if t == 0 else K_MODES) + g
        core_flops += 6.0 * nc ** 3 * (sweeps[t] if t < len(sweeps) else 0)
    if dominant == "core_svd":
        launches_k = len(per["core_svd"])
        avg_ms = totals["core_svd"] / launches_k
        achieved = core_flops / launches_k / (avg_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": "core_svd", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": ncu_traffic("core_svd"),
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (FP32 FMA)",
                    "algorithmic_flops_per_launch": core_flops / launches_k, "avg_launch_ms": avg_ms,
                    "note": "one CTA on one of 152 SMs, latency-bound Jacobi rounds; frac of that SM's "
                            "FP32 peak: %.4f" % (achieved * 1e3 / FP32_SM_PEAK_GFLOPS)}
    else:
        roof_kernel = dominant if dominant in moved else max((k for k in totals if k in moved), key=totals.get)
        launches_k = len(per[roof_kernel])
        avg_ms = totals[roof_kernel] / launches_k
        bytes_ = moved[roof_kernel] / launches_k
        achieved = bytes_ / (avg_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": roof_kernel, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "traffic": ncu_traffic(roof_kernel),
                    "peak_source": "%s: MEASURED_PEAKS.json hbm_gbs" % peak_kind,
                    "algorithmic_bytes_per_launch": bytes_, "avg_launch_ms": avg_ms}
    roofline["time_share"] = {k: round(totals[k] / sum(totals.values()), 4) for k in totals}
    roofline["dominant_kernel"] = dominant
    roofline["hbm_kernels"] = hbm_kernels
    core_phase = np.mean(np.array(core_cyc, dtype=np.float64), axis=0).tolist() if core_cyc else []

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, parts = oracle_sample(A_np, rounds)
        cpu = {"value": v, "unit": "s", "cores": cpu_cores(), "kind": "oracle",
               "sample": "FP64 NumPy/LAPACK oracle, column norms and refinement in full, %d of %d ISMA "
                         "rounds timed and scaled to the whole problem" % (parts["rounds"], rounds)}
    if rank == 0:
        line = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "m": int(m), "n": int(n), "k": K_MODES, "c": C_DRAWS,
                           "tol": TOL, "rounds": rounds, "strategy": "L2N round 0, UNF after",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "contractions": "A^T U on tcgen05 tensor cores, split-TF32 (3 products)",
                           "l2": "A is 0.80 GB, larger than the 129 MB L2: no flush between steps"},
                "e2e": {"value": ms_e2e / 1e3, "unit": "s", "h2d_bytes_per_step": int(m * n * es),
                        "d2h_bytes_per_step": int(m * K_MODES * 4 + K_MODES * 8)},
                "gpu_launches": int(launches),
                "core_svd": {"jacobi_sweeps_mean": float(np.mean(sweeps)) if sweeps else None,
                             "jacobi_sweeps_max": int(np.max(sweeps)) if sweeps else None,
                             "phase_cycles_mean": {k: round(v) for k, v in zip(
                                 ["chol2_and_E", "jacobi", "finish", "convergence", "coefficients", "total"],
                                 core_phase)}},
                "roofline": roofline,
                "clocks": clk,
                "cpu_baseline": cpu}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
