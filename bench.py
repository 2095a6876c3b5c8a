#!/usr/bin/env python
"""Benchmark of the batched OMP / CLOMP hot path on GB300.

Workload (one step): n=1024, m=256, one shared Gaussian A with unit columns,
4096 signals, each 32-sparse with values +-(1+|N(0,1)|), 40 dB noise; CLOMP
with 50 Adam steps per iteration at lr 1e-2, k = 32 iterations.  Inputs are
synthetic (seeded), resident in HBM when the timed region starts; L2 is
flushed (256 MiB write, untimed) before every timed step.

Headline: CLOMP signals/s (bf16 tensor-core correlation, Gram-form CL fit),
with plain float32 OMP and the other forms timed on the same GPU, the
per-phase kernel times and the roofline of the dominant kernel, a live parity
check of a sample against the FP64 oracle, the oracle's own throughput on the
host cores (cpu_baseline) and an end-to-end run through the host-buffer C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun), each rank solves its own 4096-signal batch (signals are
independent problems, Eq. 3): weak scaling, no collective on the data path;
the timing barrier and max over ranks use torch.distributed.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "signals/s at rel-err≤1e-5 vs FP64 oracle; CLOMP vs plain OMP, same GB300"
UNIT = "signals/s"
CL = dict(steps=50, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["bf16", "fp32"], default="bf16")
    ap.add_argument("--form", choices=["gram", "gather"], default="gram")
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--cpu-sample", type=int, default=12288,
                    help="signals the FP64 oracle solves for cpu_baseline (the workload's signals, cycled)")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--profile-case", default=None,
                    help="run one small named workload once (for an ncu capture of its kernels) and exit: "
                         + ", ".join(PROFILE_CASES))
    return ap.parse_args()


PROFILE_CASES = ("omp_fp32", "omp_fp8", "clomp_bf16_per_iteration", "clomp_gather", "threshold", "single",
                 "clfit_pair", "columnwise_image", "large_small", "large_small_clomp", "large_mid", "large_1d",
                 "large_group", "iht", "persist")


def profile_case(name):
    """One solve of a named workload, for ncu: no timing, no oracle."""
    import torch
    import paper_2501_11592_gb300 as cs
    import workloads
    cs.load()
    dev = lambda x: torch.from_numpy(np.asfortranarray(x, dtype=np.float32)).cuda()
    if name in ("omp_fp32", "omp_fp8", "clomp_bf16_per_iteration", "clomp_gather", "threshold", "persist"):
        p = workloads.config_batched()
        A, Y = dev(p.A), dev(p.Y)
        plan = cs.Plan(p.m, p.n, p.B, p.k)
        if name == "omp_fp32":
            cs.omp_solve_batched(A, Y, p.k, prec="fp32", plan=plan)
        elif name == "omp_fp8":
            cs.omp_solve_batched(A, Y, p.k, prec="fp8", plan=plan)
        else:
            plan.set_option(cs.OPT_PERSIST, 1 if name == "persist" else 0)
            plan.set_option(cs.OPT_FUSE_UPDATE, 0 if name == "clomp_gather" else 1)
            cs.clomp_solve_batched(A, Y, p.k, prec="fp32" if name == "threshold" else "bf16",
                                   form="gather" if name == "clomp_gather" else "gram", plan=plan,
                                   th=0.7 if name == "threshold" else 0.0, **CL)
    elif name == "single":
        p = workloads.config_single_fp64()
        cs.omp_solve_batched(dev(p.A), dev(p.Y), p.k, tol=p.tol, plan=cs.Plan(64, 256, 1, 8))
    elif name == "clfit_pair":
        # the gradient sub-configuration of the long 1-D workload: n = 4096, m = 1024, t = 128, 1024 signals
        rng = np.random.default_rng(11)
        A = dev(workloads.gaussian_matrix(rng, 1024, 4096))
        S = torch.from_numpy(np.stack([rng.choice(4096, 128, replace=False) for _ in range(1024)]).astype(np.int32)).cuda()
        Sv = torch.randn(1024, 128, device="cuda")
        Y = torch.randn(1024, 1024, device="cuda").t().contiguous().t()
        R, _ = cs.clfit_forward(A, S, Sv, Y)
        mom, vel = torch.zeros_like(Sv), torch.zeros_like(Sv)
        cs.clfit_adam_step(A, S, Sv, R, mom, vel, 1)
    elif name == "columnwise_image":
        pc = workloads.config_columnwise_2d(0.3, n_images=8)
        D = dev(pc.meta["D"])
        cs.reconstruct_columnwise(dev(pc.A), D, dev(pc.Y), pc.k, 256, ref=dev(pc.meta["X_img"]), algo="clomp",
                                  prec="bf16", plan=cs.Plan(pc.m, pc.n, pc.B, pc.k), tv_weight=32.0, image_prior=True,
                                  **CL)
    elif name == "large_1d":
        # the full-size long signal (for a launch list of a few iterations only)
        pl = workloads.config_large_1d()
        cs.omp_solve_batched(dev(pl.A), dev(pl.Y), pl.k, prec="bf16", plan=cs.Plan(pl.m, pl.n, 1, pl.k))
    elif name == "iht":
        # IHT on the batched workload, 20 iterations, t = 1 / sigma_max(A)^2
        p = workloads.config_batched()
        step = float(np.float32(1.0 / np.linalg.norm(p.A, 2) ** 2))
        cs.iht_solve_batched(dev(p.A), dev(p.Y), p.k, step, max_iter=20)
    elif name == "large_group":
        # one large class of the uneven batch: 72 signals sharing A (the GEMM correlation)
        p = workloads.random_problem(4336, 15360, 72, 40, seed=7, snr_db=30.0, values="pm")
        cs.omp_solve_batched(dev(p.A), dev(p.Y), p.k, prec="bf16", plan=cs.Plan(4336, 15360, 72, 40))
    elif name == "large_mid":
        pl = workloads.config_large_1d(n=16384, m=4915, k=600)
        cs.omp_solve_batched(dev(pl.A), dev(pl.Y), pl.k, prec="bf16", plan=cs.Plan(pl.m, pl.n, 1, pl.k))
    elif name in ("large_small", "large_small_clomp"):
        pl = workloads.config_large_1d(n=16384, m=4915, k=100)
        fn = cs.omp_solve_batched if name == "large_small" else cs.clomp_solve_batched
        kw = {} if name == "large_small" else dict(form="gram", **CL)
        fn(dev(pl.A), dev(pl.Y), pl.k, prec="bf16", plan=cs.Plan(pl.m, pl.n, 1, pl.k), **kw)
    else:
        raise SystemExit(f"unknown profile case {name}")
    torch.cuda.synchronize()
    print(f"profile case {name}: done", flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(args, p):
    return {"workload": f"batched OMP/CLOMP, n={p.n}, m={p.m}, {p.B} signals per GPU, k={p.k}, "
                        f"Gaussian A (unit columns), 32-sparse +-(1+|N(0,1)|), 40 dB SNR",
            "n": p.n, "m": p.m, "signals_per_gpu": p.B, "k": p.k, "algo": "clomp",
            "correlation": args.prec, "cl_form": args.form, "adam_steps_per_iter": CL["steps"],
            "lr": CL["lr"], "l2": "flushed before every timed step (256 MiB write, untimed)",
            "parallelism": "signals sharded across GPUs, A replicated (no collective)"}


# ------------------------------------------------------------ reference arm
def run_reference(args):
    """The reference arm is the FP64 CPU oracle, run as it stands on the host
    cores: each step solves a bounded sample of the same workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import workloads
    p = workloads.config_batched(B=args.batch)
    sample = min(256, p.B)
    A32 = np.asfortranarray(p.A, dtype=np.float32).astype(np.float64, order="F")
    Y32 = np.asfortranarray(p.Y[:, :sample], dtype=np.float32).astype(np.float64, order="F")
    f = lambda x: float(np.float32(x))
    kw = dict(steps=CL["steps"], lr=f(CL["lr"]), beta1=f(CL["beta1"]), beta2=f(CL["beta2"]), eps=f(CL["eps"]))
    for _ in range(args.warmup):
        oracle.clomp(A32, Y32[:, :32], p.k, **kw)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.clomp(A32, Y32, p.k, **kw)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = sample / (ms / 1e3)
    cores = oracle.max_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, p),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample} of the {p.B} signals per step (CLOMP, FP64 oracle, OpenMP)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", str(self.idx)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    pass
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        loaded = [c for c, _, _ in rows if c > 300] or [c for c, _, _ in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(m for _, m, _ in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ our arm
def kernel_sha(rel):
    h = hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()
    return h[:16]


def recorded_traffic(kernel, sha):
    """dram bytes per launch from a committed ncu summary, if it was taken on
    this exact kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == kernel and f[1] == sha:
            return float(f[2])
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


def peaks_and_src():
    return measured_peaks()


def events_ms(torch, stream, fn, reps):
    """Mean device time of fn over reps runs (CUDA events on `stream`)."""
    out = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b))
    return float(np.mean(out))


def bench_large_1d(cs, torch, stream, barrier, rank, peaks_src):
    """The long 1-D signal (n = 65536, m = 19661, k = 2000; A 5.2 GB float32):
    one plain-OMP solve on the large-instance path per correlation precision,
    the correlation's achieved HBM bandwidth, exact recovery of the noiseless
    signal, and parity of the first 200 iterations with the FP64 oracle."""
    import workloads
    peaks, src = peaks_src
    pl = workloads.config_large_1d()
    m, n, k = pl.m, pl.n, pl.k
    A = torch.from_numpy(pl.A).cuda()
    y = torch.from_numpy(np.float32(pl.Y)).cuda()
    plan = cs.Plan(m, n, 1, k)
    res = {"workload": f"n={n}, m={m}, k={k}, one signal, Gaussian A (unit columns, float32, "
                       f"{m * n * 4 / 1e9:.2f} GB), x k-sparse N(0,1), noiseless"}
    truth = np.nonzero(pl.X_true[:, 0])[0]
    for prec in ("bf16", "fp32"):
        fn = lambda: cs.omp_solve_batched(A, y, k, prec=prec, plan=plan)
        fn()
        barrier()
        ms = events_ms(torch, stream, fn, 2)
        plan.set_profiling(True)
        plan.profile(reset=True)
        r = fn()
        torch.cuda.synchronize()
        ph = plan.profile(reset=True)
        plan.set_profiling(False)
        sup = r.support.cpu().numpy()[0]
        coef = r.coef.cpu().numpy()[0].astype(np.float64)
        xr = np.zeros(n)
        xr[sup[sup >= 0]] = coef[sup >= 0]
        n_c, t_c = ph["correlation"]
        mp = (m + 7) // 8 * 8
        a_bytes = n * mp * 2 if prec == "bf16" else n * m * 4
        per_launch = a_bytes + mp * 4 + n * 4          # A once, r, the |c| written
        gbs = per_launch * n_c / (t_c / 1e3) / 1e9 if n_c else None
        res[prec] = {"ms_per_solve": ms, "signals_per_s": 1e3 / ms,
                     "support_is_the_true_support": bool(sorted(sup.tolist()) == sorted(truth.tolist())),
                     "coef_rel_err_vs_x_true": float(np.linalg.norm(xr - pl.X_true[:, 0]) /
                                                     np.linalg.norm(pl.X_true[:, 0])),
                     "status": int(r.status.cpu()[0]), "n_iter": int(r.n_iter.cpu()[0]),
                     "phase_ms": {q: round(v[1], 3) for q, v in ph.items() if v[0]},
                     "roofline_correlation": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"],
                                              "unit": "GB/s", "frac": (gbs / peaks["hbm_gbs"]) if gbs else None,
                                              "bytes_per_launch": per_launch, "launches": n_c,
                                              "peak_source": f"hbm_gbs ({src})"}}
    # CLOMP (Gram form, 50 Adam steps per iteration at lr 1e-2), bf16 correlation:
    # the configuration the long 1-D CLOMP workload is stated for
    fn = lambda: cs.clomp_solve_batched(A, y, k, prec="bf16", form="gram", plan=plan, **CL)
    fn()
    barrier()
    ms = events_ms(torch, stream, fn, 1)
    plan.set_profiling(True)
    plan.profile(reset=True)
    r = fn()
    torch.cuda.synchronize()
    ph = plan.profile(reset=True)
    plan.set_profiling(False)
    sup = r.support.cpu().numpy()[0]
    res["clomp_bf16"] = {"ms_per_solve": ms, "signals_per_s": 1e3 / ms,
                         "true_atoms_selected": int(len(set(sup.tolist()) & set(truth.tolist()))), "k": k,
                         "status": int(r.status.cpu()[0]), "n_iter": int(r.n_iter.cpu()[0]),
                         "res_norm_over_norm_y": float(r.res_norm.cpu()[0]) / float(np.linalg.norm(pl.Y)),
                         "phase_ms": {q: round(v[1], 3) for q, v in ph.items() if v[0]},
                         "note": "Adam steps: one grid-wide launch each (2000 x 50); parity of this path is "
                                 "tested at n = 8192, m = 2048, k = 150 (tests/test_gpu_large.py)"}
    if rank == 0:
        # the first 200 iterations against the FP64 oracle (incremental QR, atoms over the host's threads)
        import oracle
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        import parity as prules
        it = 200
        r = cs.omp_solve_batched(A, y, k, prec="bf16", plan=plan, max_iter=it)
        torch.cuda.synchronize()
        g = prules.to_numpy(r)
        t0 = time.perf_counter()
        o = oracle.omp(pl.A.astype(np.float64, order="F"), np.float32(pl.Y).astype(np.float64), k, max_iter=it)
        to = time.perf_counter() - t0
        g = {q: v[:, :it] if v.ndim == 2 else v for q, v in g.items()}
        o = {q: v[:, :it] if v.ndim == 2 else v for q, v in o.items()}
        summ, fails = prules.summarize(g, o)
        res["parity_first_200_iterations_bf16"] = {
            "supports_identical": bool(np.array_equal(g["support"], o["support"])),
            "ambiguous_ties": summ["ambiguous"], "non_ambiguous_mismatches": summ["failures"],
            "max_coef_rel_err": summ["max_coef_rel_err"], "oracle_s": to, "oracle_cores": oracle.max_threads()}
        # CLOMP: the first 50 iterations (the Adam step counter does not depend on k)
        it = 50
        r = cs.clomp_solve_batched(A, y, k, prec="bf16", form="gram", plan=plan, max_iter=it, **CL)
        torch.cuda.synchronize()
        g = prules.to_numpy(r)
        t0 = time.perf_counter()
        o = oracle.clomp(pl.A.astype(np.float64, order="F"), np.float32(pl.Y).astype(np.float64), k,
                         max_iter=it, steps=CL["steps"],
                         **{q: float(np.float32(v)) for q, v in CL.items() if q != "steps"})
        to = time.perf_counter() - t0
        g = {q: v[:, :it] if v.ndim == 2 else v for q, v in g.items()}
        o = {q: v[:, :it] if v.ndim == 2 else v for q, v in o.items()}
        summ, fails = prules.summarize(g, o)
        res["parity_first_50_iterations_clomp_bf16"] = {
            "supports_identical": bool(np.array_equal(g["support"], o["support"])),
            "ambiguous_ties": summ["ambiguous"], "non_ambiguous_mismatches": summ["failures"],
            "max_coef_rel_err": summ["max_coef_rel_err"], "oracle_s": to, "oracle_cores": oracle.max_threads()}
    res["autotune"] = plan.autotune_report()
    del A, plan
    torch.cuda.empty_cache()
    return res


def uneven_class_roofline(m, n, kss, seconds, tc_tflops, hbm_gbs):
    """Roofline of one size class of the uneven batch solved on its own: its
    correlation flops (2 m n k per instance) against min(tensor peak, AI x
    HBM), AI = those flops over the algorithmic bytes -- A's bf16 copy read
    once per iteration, k_max iterations."""
    flops = sum(2.0 * m * n * k for k in kss)
    bytes_a = 2.0 * m * n * max(kss)
    ai = flops / bytes_a
    roof = min(tc_tflops, ai * hbm_gbs / 1e3)
    ach = flops / seconds / 1e12
    return {"m": m, "n": n, "instances": len(kss), "k_max": max(kss), "ms": 1e3 * seconds,
            "tflops": ach, "ai_flop_per_byte": ai, "bound": "hbm" if roof < tc_tflops else "tensor",
            "roof_tflops": roof, "frac": ach / roof, "a_stream_gbs": bytes_a / seconds / 1e9}


def bench_uneven(cs, torch, stream, barrier):
    """The uneven batch (2000 instances in 32 size classes, n in [512, 16384],
    m/n in [0.1, 0.5], k = 1-10 % of n) through omp_solve_varlen: instances
    within the on-chip kernels run batched per (A, m, n, k) group, the others
    on the large-instance path per (A, m, n) group."""
    import workloads
    classes, assign, ks = workloads.config_uneven()
    keep, items = [], [None] * len(assign)
    work = 0.0
    for c in range(len(classes)):
        A, inst = workloads.uneven_class_data(classes, assign, ks, c, dtype=np.float32)
        At = torch.from_numpy(A).cuda()
        keep.append(At)
        for i, yv, _ in inst:
            items[i] = (At, torch.from_numpy(np.float32(yv)).cuda(), ks[i])
            work += 2.0 * A.shape[0] * A.shape[1] * ks[i]
    m_max = max(cl["m"] for cl in classes)
    n_max = max(cl["n"] for cl in classes)
    plan = cs.Plan(m_max, n_max, 128, max(ks))
    res = {"workload": "2000 instances, 32 classes, n log-uniform in [512, 16384], m/n in [0.1, 0.5], "
                       "k uniform in [0.01 n, 0.1 n], Gaussian/Bernoulli A, 30 dB",
           "correlation_flops": work}
    for prec in ("fp32", "bf16"):
        fn = lambda: cs.omp_solve_varlen(items, prec=prec, plan=plan)
        outs = fn()
        barrier()
        t0 = time.perf_counter()
        outs = fn()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        st = np.array([int(o.status[0]) for o in outs])
        res["omp_" + prec] = {"s_per_batch": wall, "instances_per_s": len(items) / wall,
                              "solved": int(np.sum(st != cs.SIG_UNSUPPORTED)), "refused": int(np.sum(st == cs.SIG_UNSUPPORTED)),
                              "note": "wall clock of one call (on-chip groups one after another; plain-OMP large groups up to four at once on their own streams, each synchronising every 64 iterations)"}
    # bf16 OMP one size class per call (the plan is tuned by the calls above):
    # each class's roofline, and the aggregate of the one-call time above
    peaks, src = measured_peaks()
    per_class = []
    for c, cl in enumerate(classes):
        idx = [i for i in range(len(assign)) if assign[i] == c]
        if not idx:
            continue
        sub = [items[i] for i in idx]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cs.omp_solve_varlen(sub, prec="bf16", plan=plan)
        torch.cuda.synchronize()
        per_class.append(uneven_class_roofline(cl["m"], cl["n"], [ks[i] for i in idx], time.perf_counter() - t0,
                                               peaks["bf16_tflops"], peaks["hbm_gbs"]))
    agg_s = res["omp_bf16"]["s_per_batch"]
    res["roofline_omp_bf16"] = {
        "per_class": per_class,
        "sum_of_class_seconds": sum(q["ms"] for q in per_class) / 1e3,
        "aggregate": {"tflops": work / agg_s / 1e12, "unit": "TFLOP/s",
                      "frac_of_tensor_peak": work / agg_s / 1e12 / peaks["bf16_tflops"],
                      "a_stream_gbs": sum(2.0 * q["m"] * q["n"] * q["k_max"] for q in per_class) / agg_s / 1e9},
        "peak_source": f"bf16_tflops burst, hbm_gbs ({src})",
        "note": "wall clock per class (host-timed, one call each); AI = correlation flops over A's bf16 copy read once per iteration"}
    fn = lambda: cs.clomp_solve_varlen(items, prec="bf16", plan=plan, **CL)
    outs = fn()
    barrier()
    t0 = time.perf_counter()
    outs = fn()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = np.array([int(o.status[0]) for o in outs])
    res["clomp_bf16"] = {"s_per_batch": wall, "instances_per_s": len(items) / wall,
                         "solved": int(np.sum(st != cs.SIG_UNSUPPORTED)), "refused": int(np.sum(st == cs.SIG_UNSUPPORTED))}
    res["autotune"] = plan.autotune_report()
    del keep, plan
    torch.cuda.empty_cache()
    return res


def main():
    args = parse()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args)
    ws, rank, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2501_11592_gb300 as cs
    import workloads
    cs.load()

    p = workloads.config_batched(B=args.batch)
    A32 = np.asfortranarray(p.A, dtype=np.float32)
    Y32 = np.asfortranarray(p.Y, dtype=np.float32)
    A = torch.from_numpy(A32).cuda()
    Y = torch.from_numpy(Y32).cuda()
    plan = cs.Plan(p.m, p.n, p.B, p.k)
    out = cs._outputs(p.B, p.k, A.device)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def make_step(algo, prec, form="gram", th=0.0):
        if algo == "omp":
            return lambda: cs.omp_solve_batched(A, Y, p.k, prec=prec, plan=plan, out=out)
        return lambda: cs.clomp_solve_batched(A, Y, p.k, prec=prec, form=form, plan=plan, out=out, th=th, **CL)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        plan.profile(reset=True)
        t0 = time.perf_counter()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        barrier()
        wall = time.perf_counter() - t0
        ms = sum(a.elapsed_time(b) for a, b in ev)
        launches = sum(n for n, _ in plan.profile(reset=True).values())
        if dist is not None:
            t = torch.tensor([ms], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms / steps, wall, launches

    # --- headline: CLOMP, bf16 correlation, Gram-form fit
    head = make_step("clomp", args.prec, args.form)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").replace(",", "").isdigit() else local
    clk = ClockSampler(gpu_index)
    clk.start()
    ms, wall, launches = timed(head, args.steps, args.warmup)
    clocks = clk.stop()
    plan.counters(reset=True)
    value = ws * p.B / (ms / 1e3)

    # --- per-phase kernel times (separate pass with events around every launch)
    plan.set_profiling(True)
    for _ in range(args.warmup):
        head()
    plan.profile(reset=True)
    nprof = max(3, min(args.steps, 20))
    for _ in range(nprof):
        flush.zero_()
        head()
    phases = plan.profile(reset=True)
    plan.set_profiling(False)
    fallbacks, errflags = plan.counters(reset=True)

    # --- live parity of every signal against the FP64 oracle: the headline
    # solve, plain fp32 OMP and bf16 OMP, under the rules of tests/parity.py
    parity = None
    if rank == 0:
        import oracle
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        import parity as prules
        f = lambda x: float(np.float32(x))
        A64, Y64 = A32.astype(np.float64), Y32.astype(np.float64)
        ora = {"clomp": oracle.clomp(A64, Y64, p.k, steps=CL["steps"], lr=f(CL["lr"]), beta1=f(CL["beta1"]),
                                     beta2=f(CL["beta2"]), eps=f(CL["eps"])),
               "omp": oracle.omp(A64, Y64, p.k)}
        parity = {"tolerance": prules.COEF_RTOL, "ambiguous_margin": prules.AMBIGUOUS_MARGIN}
        for name, fn, algo in (("headline_" + "clomp_" + args.prec, head, "clomp"),
                               ("omp_fp32", make_step("omp", "fp32"), "omp"),
                               ("omp_bf16", make_step("omp", "bf16"), "omp")):
            fn()
            torch.cuda.synchronize()
            g = prules.to_numpy(out)
            summ, fails = prules.summarize(g, ora[algo])
            parity[name] = {"signals": summ["signals"], "ambiguous_ties": summ["ambiguous"],
                            "non_ambiguous_mismatches": summ["failures"],
                            "supports_identical": int(np.sum(np.all(g["support"] == ora[algo]["support"], axis=1))),
                            "max_coef_rel_err": summ["max_coef_rel_err"]}

    # --- the other forms on the same GPU
    compare = {}
    if not args.no_extras:
        ksteps = max(3, min(args.steps, 10))
        for name, algo, prec, form in [("omp_fp32", "omp", "fp32", "gram"), ("omp_bf16", "omp", "bf16", "gram"),
                                       ("omp_fp8", "omp", "fp8", "gram"), ("clomp_fp8_gram", "clomp", "fp8", "gram"),
                                       ("clomp_fp32_gram", "clomp", "fp32", "gram"),
                                       ("clomp_bf16_gather", "clomp", "bf16", "gather"),
                                       ("clomp_bf16_gram_per_iteration", "clomp", "bf16", "gram"),
                                       ("clomp_bf16_gram_unfused", "clomp", "bf16", "gram"),
                                       ("clomp_fp32_gram_threshold_0.7", "clomp", "fp32", "gram")]:
            th = 0.7 if "threshold" in name else 0.0
            fn = make_step(algo, prec, form, th)
            plan.set_option(cs.OPT_FUSE_UPDATE, 0 if name.endswith("unfused") else 1)
            # the per-iteration kernels instead of the persistent solve
            plan.set_option(cs.OPT_PERSIST, 0 if name.startswith("clomp_bf16_gram_") else 1)
            m_, _, _ = timed(fn, ksteps, 3)
            plan.set_profiling(True)
            plan.profile(reset=True)
            for _ in range(3):
                flush.zero_()
                fn()
            ph = plan.profile(reset=True)
            plan.set_profiling(False)
            compare[name] = {"ms_per_step": m_, "signals_per_s": ws * p.B / (m_ / 1e3),
                             "phase_ms_per_step": {k: round(v[1] / 3, 4) for k, v in ph.items()}}
            if th:
                # a different selection rule: its supports are not the argmax rule's
                torch.cuda.synchronize()
                compare[name]["mean_support_size"] = float(out.n_iter.float().mean().item())
                compare[name]["note"] = ("threshold rule Th = 0.7 (several atoms per iteration); "
                                         "not the headline metric's selection rule")
        plan.set_option(cs.OPT_FUSE_UPDATE, 1)
        plan.set_option(cs.OPT_PERSIST, 1)
        # IHT, the paper's comparison method, on the same workload: k = 32, R = 200
        # iterations, step 1 / sigma_max(A)^2 (a configuration input, from numpy)
        step = float(np.float32(1.0 / np.linalg.norm(A32.astype(np.float64), 2) ** 2))
        fi = lambda: cs.iht_solve_batched(A, Y, p.k, step, max_iter=200, plan=plan, out=out)
        mi, _, _ = timed(fi, ksteps, 3)
        compare["iht_fp32_r200"] = {"ms_per_step": mi, "signals_per_s": ws * p.B / (mi / 1e3), "step": step,
                                    "note": "IHT s <- H_k(s + t A^T r), 200 iterations, float32 correlation"}
        # column-wise 2D output path: 64 images of 256 x 256 at Sr = 0.3 (m = 77,
        # k = 25): CLOMP solve of the 16384 columns, x = D s, PSNR and SSIM
        pc = workloads.config_columnwise_2d(0.3, n_images=64)
        Ac = torch.from_numpy(np.asfortranarray(pc.A, dtype=np.float32)).cuda()
        Yc = torch.from_numpy(np.asfortranarray(pc.Y, dtype=np.float32)).cuda()
        Dc = torch.from_numpy(np.asfortranarray(pc.meta["D"], dtype=np.float32)).cuda()
        Rc = torch.from_numpy(np.asfortranarray(pc.meta["X_img"], dtype=np.float32)).cuda()
        planc = cs.Plan(pc.A.shape[0], pc.A.shape[1], pc.Y.shape[1], pc.k)
        # (the TV prior's weight, 0: none; its image form, Eq. 6; the LV prior's
        # weight, Eq. 7)
        for tvw, img, lvw in ((0.0, False, 0.0), (32.0, False, 0.0), (32.0, True, 0.0), (0.0, True, 40.0)):
            fnc = lambda: cs.reconstruct_columnwise(Ac, Dc, Yc, pc.k, 256, ref=Rc, algo="clomp", prec="bf16",
                                                    plan=planc, tv_weight=tvw, image_prior=img, lv_weight=lvw,
                                                    **CL)
            for _ in range(3):
                rc = fnc()
            barrier()
            tc_ms = []
            for _ in range(ksteps):
                flush.zero_()
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record(stream)
                rc = fnc()
                b_.record(stream)
                barrier()
                tc_ms.append(a_.elapsed_time(b_))
            mc = float(np.mean(tc_ms))
            key = ("columnwise_2d_sr0.3" + ("" if tvw == 0.0 else "_tv%g" % tvw)
                   + ("_image" if img and tvw else "") + ("" if lvw == 0.0 else "_lv%g" % lvw))
            compare[key] = {
                "ms_per_step": mc, "images_per_s": ws * 64 / (mc / 1e3),
                "columns_per_s": ws * pc.Y.shape[1] / (mc / 1e3),
                "mean_psnr_db": float(rc["psnr"].mean().item()), "mean_ssim": float(rc["ssim"].mean().item()),
                "note": ("64 images 256x256, m=77, k=25: CLOMP (bf16) + x = D s + PSNR/SSIM per image"
                         + ("" if tvw == 0.0 or img else "; total-variation prior (Eq. 5) on x = D s, w = %g" % tvw)
                         + ("; image total-variation prior (Eq. 6), w = %g: per-iteration kernels, the fit one "
                            "cluster per image" % tvw if img and tvw else "")
                         + ("; local-variation prior (Eq. 7, 3x3 windows), w = %g: per-iteration kernels, the "
                            "fit one cluster per image synthesising D s every Adam step" % lvw if lvw else ""))}
        del planc
        # the column-wise workload at the other sampling rates (Sr = 0.5: k = 42
        # runs on the per-iteration kernels)
        for sr in (0.1, 0.5):
            pq = workloads.config_columnwise_2d(sr, n_images=64)
            Aq = torch.from_numpy(np.asfortranarray(pq.A, dtype=np.float32)).cuda()
            Yq = torch.from_numpy(np.asfortranarray(pq.Y, dtype=np.float32)).cuda()
            Rq = torch.from_numpy(np.asfortranarray(pq.meta["X_img"], dtype=np.float32)).cuda()
            planq = cs.Plan(pq.A.shape[0], pq.A.shape[1], pq.Y.shape[1], pq.k)
            fnq = lambda: cs.reconstruct_columnwise(Aq, Dc, Yq, pq.k, 256, ref=Rq, algo="clomp", prec="bf16",
                                                    plan=planq, **CL)
            for _ in range(3):
                rq = fnq()
            barrier()
            tq = []
            for _ in range(ksteps):
                flush.zero_()
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record(stream)
                rq = fnq()
                b_.record(stream)
                barrier()
                tq.append(a_.elapsed_time(b_))
            mq = float(np.mean(tq))
            compare["columnwise_2d_sr%g" % sr] = {
                "ms_per_step": mq, "images_per_s": ws * 64 / (mq / 1e3),
                "columns_per_s": ws * pq.Y.shape[1] / (mq / 1e3), "m": pq.A.shape[0], "k": pq.k,
                "mean_psnr_db": float(rq["psnr"].mean().item()), "mean_ssim": float(rq["ssim"].mean().item())}
            del planq
        # single signal (n = 256, m = 64, k = 8, noiseless, tol 1e-10): latency of
        # one plain-OMP solve (graph replay), and the oracle on one host core
        p1 = workloads.config_single_fp64()
        A1 = torch.from_numpy(np.asfortranarray(p1.A, dtype=np.float32)).cuda()
        y1 = torch.from_numpy(np.asfortranarray(p1.Y, dtype=np.float32)).cuda()
        plan1 = cs.Plan(64, 256, 1, 8)
        out1 = cs._outputs(1, p1.k, A1.device)     # output buffers made once, as a caller would
        f1 = lambda: cs.omp_solve_batched(A1, y1, p1.k, tol=p1.tol, plan=plan1, out=out1)
        for _ in range(5):
            f1()
        barrier()
        t1 = []
        for _ in range(50):
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            f1()
            b_.record(stream)
            barrier()
            t1.append(a_.elapsed_time(b_))
        plan1.set_profiling(True)
        plan1.profile(reset=True)
        for _ in range(20):
            f1()
        barrier()
        ph1 = plan1.profile(reset=True)
        plan1.set_profiling(False)
        n1, ms1 = ph1["persist"]
        single = {"gpu_ms_median": float(np.median(t1)), "algo": "omp fp32 (fp64 Cholesky)",
                  "kernel_ms": ms1 / max(n1, 1),
                  "note": "gpu_ms: CUDA events around the C-ABI call (output buffers allocated once); "
                          "kernel_ms: the one fused launch of the solve"}
        if rank == 0:
            import oracle
            A1h = np.asfortranarray(p1.A, dtype=np.float32).astype(np.float64, order="F")
            y1h = np.asfortranarray(p1.Y, dtype=np.float32).astype(np.float64, order="F")
            n0 = oracle.max_threads()
            tt = []
            for _ in range(20):
                t0_ = time.perf_counter()
                oracle.omp(A1h, y1h, p1.k, tol=p1.tol, nthreads=1)
                tt.append(time.perf_counter() - t0_)
            oracle.omp(A1h, y1h, p1.k, tol=p1.tol, nthreads=n0)   # back to all host cores
            single["oracle_ms_median_1_core"] = 1e3 * float(np.median(tt))
        compare["single_signal_n256_m64_k8"] = single
        del plan1
        compare["large_1d_n65536_m19661_k2000"] = bench_large_1d(cs, torch, stream, barrier, rank, peaks_and_src())
        compare["uneven_batch_2000"] = bench_uneven(cs, torch, stream, barrier)
        compare["clomp_headline"] = {"ms_per_step": ms, "signals_per_s": value}
        compare["clomp_over_omp_fp32"] = value / compare["omp_fp32"]["signals_per_s"]

    # --- end to end through the host-buffer C ABI (copies inside the timed region)
    Ah = torch.from_numpy(A32.T.copy()).pin_memory().numpy().T          # Fortran-order pinned views
    Yh = torch.from_numpy(Y32.T.copy()).pin_memory().numpy().T
    hout = dict(support=torch.empty((p.B, p.k), dtype=torch.int32).pin_memory().numpy(),
                coef=torch.empty((p.B, p.k), dtype=torch.float32).pin_memory().numpy(),
                n_iter=torch.empty(p.B, dtype=torch.int32).pin_memory().numpy(),
                res_norm=torch.empty(p.B, dtype=torch.float32).pin_memory().numpy(),
                status=torch.empty(p.B, dtype=torch.int32).pin_memory().numpy())
    hstep = lambda: cs.clomp_solve_batched_host(Ah, Yh, p.k, prec=args.prec, form=args.form, plan=plan,
                                                out=hout, **CL)
    for _ in range(3):
        hstep()
    barrier()
    esteps = max(3, min(args.steps, 20))
    te = 0.0
    for _ in range(esteps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hstep()            # returns after the outputs are back on the host
        te += time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([te], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        te = float(t.item())
    e2e_value = ws * p.B * esteps / te
    h2d = (p.m * p.n + p.m * p.B) * 4
    d2h = p.B * p.k * 8 + p.B * 12

    # --- CPU baseline: the FP64 oracle on the host cores, bounded sample
    cpu = None
    if rank == 0 and ws == 1:
        import oracle
        S = max(1, args.cpu_sample)
        f = lambda x: float(np.float32(x))
        A64 = A32.astype(np.float64, order="F")
        Y64 = np.asfortranarray(Y32[:, np.arange(S) % p.B], dtype=np.float64)
        t0 = time.perf_counter()
        oracle.clomp(A64, Y64, p.k, steps=CL["steps"], lr=f(CL["lr"]), beta1=f(CL["beta1"]),
                     beta2=f(CL["beta2"]), eps=f(CL["eps"]))
        tc = time.perf_counter() - t0
        cpu = {"value": S / tc, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
               "sample": (f"{S} signals (" + (f"the first {S} of the workload's {p.B}" if S <= p.B
                                             else f"the workload's {p.B}, cycled")
                          + f"; CLOMP, FP64 oracle, OpenMP over signals), {tc:.1f} s")}

    # --- roofline of the dominant kernel
    peaks, src = measured_peaks()
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    per = {ph: {"launches": n, "ms_total": t, "ms_avg": (t / n if n else None)} for ph, (n, t) in phases.items()}
    dom = max((ph for ph in phases if ph != "setup"), key=lambda ph: phases[ph][1])
    iters = p.k
    B = p.B
    roof_corr = None
    n_corr, t_corr = phases["correlation"]
    corr_src = "headline"
    if not n_corr and "clomp_bf16_gram_per_iteration" in compare:
        # the persistent solve has no separate correlation launch: take the
        # tensor-core correlation kernel of the per-iteration form
        n_corr = iters
        t_corr = compare["clomp_bf16_gram_per_iteration"]["phase_ms_per_step"]["correlation"]
        corr_src = "per-iteration bf16 CLOMP (k_corr_tc)"
    fp32_peak = n_sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    fp32_src = f"nominal: {n_sms} SMs (device) x 128 FP32 FMA/clk x 2 x sm_max_mhz (not measured)"
    if n_corr:
        flops = 2.0 * p.m * p.n * B                    # per launch: every signal is live for all k iterations
        avg_s = t_corr / n_corr / 1e3
        ach = flops / avg_s / 1e12
        if args.prec == "bf16":
            pk = peaks["bf16_tflops"]
            roof_corr = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                         "peak_source": f"bf16_tflops, burst ({src})", "kernel": corr_src}
        else:
            roof_corr = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": ach / fp32_peak, "peak_source": fp32_src}
        sha = kernel_sha("paper_2501_11592_gb300/csrc/" + ("k_corr_tc.cu" if args.prec == "bf16" else "k_corr_fp32.cu"))
        tr = recorded_traffic("corr_" + args.prec, sha)
        roof_corr["traffic"] = tr
    # algorithmic work of the other phases (per solve, summed over the k iterations)
    sum_t = iters * (iters + 1) / 2.0
    sum_t2 = iters * (iters + 1) * (2 * iters + 1) / 6.0
    fit_flops = B * CL["steps"] * (2 * sum_t2 + 10 * sum_t)
    resid_flops = B * 2.0 * p.m * sum_t
    work = {
        # Gram form: g = G s - b per Adam step (2 t^2 flops) + Adam update (~10 t flops)
        "fit": ("alu", fit_flops, fp32_peak, "TFLOP/s"),
        # persistent solve: its CUDA-core arithmetic (fit + residual); the
        # correlation's tensor work is reported separately below
        "persist": ("alu", fit_flops + resid_flops, fp32_peak, "TFLOP/s"),
        # fused selection + fit + residual: its arithmetic is the fit's
        "update": ("alu", fit_flops, fp32_peak, "TFLOP/s"),
        # residual: read t columns of A (4m bytes each), y, write r (fp32 + bf16)
        "residual": ("hbm", B * (4.0 * p.m * sum_t + iters * p.m * (4 + 4 + 2)), peaks["hbm_gbs"], "GB/s"),
        # select: read topc*nch candidate pairs and re-score 8 columns + the new column and y
        "select": ("hbm", B * iters * (8.0 * 8 * 4 + 10 * 4.0 * p.m), peaks["hbm_gbs"], "GB/s"),
    }
    roofs = {"correlation": roof_corr}
    for ph, (bound, amount, pk, unit) in work.items():
        n_, t_ = phases[ph]
        if not n_ or t_ <= 0:
            continue
        nsolves = n_ if ph == "persist" else n_ / iters   # one persistent launch per solve
        ach = amount * nsolves / (t_ / 1e3) / (1e12 if unit == "TFLOP/s" else 1e9)
        roofs[ph] = {"bound": bound, "achieved": ach, "peak": pk, "unit": unit, "frac": ach / pk,
                     "traffic": None}
        if unit == "TFLOP/s":
            roofs[ph]["peak_source"] = fp32_src
    if dom == "persist":
        # The dominant kernel is the whole solve; its roofline is that of the
        # correlation it carries: 2 m n B k flops per launch (every signal is
        # live for all k iterations) over the launch's event time, against the
        # measured bf16 peak.  Its CUDA-core work (fit + residual) is reported
        # beside it against the nominal fp32 rate.
        n_, t_ = phases["persist"]
        tflops = 2.0 * p.m * p.n * B * iters * n_ / (t_ / 1e3) / 1e12
        pk = peaks["bf16_tflops"]
        roofline = {"bound": "tensor", "achieved": tflops, "peak": pk, "unit": "TFLOP/s", "frac": tflops / pk,
                    "traffic": recorded_traffic("persist_bf16",
                                                kernel_sha("paper_2501_11592_gb300/csrc/k_persist.cu")),
                    "kernel": "k_clomp_persist", "kernel_phase": dom,
                    "work_per_launch": f"2*m*n*B*k = {2.0 * p.m * p.n * B * iters:.4g} flop",
                    "ms_per_launch": t_ / n_, "peak_source": f"bf16_tflops, burst ({src})"}
        roofs["persist"]["note"] = "CUDA-core work (Adam fit + residual) of the persistent kernel"
    else:
        roofline = dict(roofs[dom]) if roofs.get(dom) else roof_corr
        roofline["kernel_phase"] = dom

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": workload_config(args, p),
            "roofline": roofline,
            "roofline_correlation": roof_corr,
            "roofline_cuda_core": roofs.get("persist"),
            "roofline_phases": roofs,
            "phases": per,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "clomp_solve_batched_host (pinned host buffers, outputs copied back)"},
            "clocks": clocks,
            "gpu_launches": int(launches),
            "parity": parity,
            "autotune": plan.autotune_report(),
            "bf16_certificate_fallbacks": fallbacks,
            "device_error_flags": errflags,
            "compare": compare,
            "wall_s_timed_region": wall}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
