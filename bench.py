#!/usr/bin/env python3
"""Benchmark: ME-GRBK iterations per second on one GB300 (and N independent
replicas under torchrun), with the HBM roofline of the persistent iteration
kernel, the end-to-end number through the C ABI with host buffers, and the
FP64 CPU oracle as the baseline.

Workload (default, "precision"): A 20000x2000 and B 2000x20000 with N(0, 1/cols)
entries, X* N(0,1), C = A X* B; FP32 residual pass with the R refresh every 64
iterations as split-BF16 tensor-core products ("chosen" form), next to the
plain FP64 form (no refresh) on the same system.  One step = 64 iterations of
the whole hot path (select, W/U, V, fused residual pass) plus one refresh of
R = C - A X B and the stop check.  R (1.6 GB) is far larger than L2, so no
flush is needed between steps.

--impl reference times the FP64 CPU oracle (its OpenMP timing build, on every
host core) on the same system: each step is a few ME-GRBK iterations of the
selected workload itself, so the line needs no scaling.

The default run also measures, at N = 1, time to a solution-error target
("ttt"): the 20000x2000 / 2000x20000 system to RSE <= 1e-4 in the chosen form,
the row-space form and the plain FP64 form, and the 200x100 / 80x150 system to
RSE <= 1e-6 in FP64 (about four minutes in all; --no-ttt skips it).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "ME-GRBK iters/s & time-to-RSE<=1e-6 (HBM GB/s vs peak), chosen vs plain form"
UNIT = "iters/s"

WORKLOADS = {
    # name: (m, p, q, n, generator kwargs)
    "precision": dict(m=20000, p=2000, q=2000, n=20000),
    "precision_slice": dict(m=2000, p=200, q=200, n=2000),
    # same recipe at 8000x800 / 800x8000: R is 256 MB (larger than L2), about
    # 2 GB on the device in all; used for ncu captures
    "precision_8k": dict(m=8000, p=800, q=800, n=8000),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="precision", choices=sorted(WORKLOADS))
    ap.add_argument("--iters-per-step", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-rowspace", action="store_true")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-target legs of the default run")
    ap.add_argument("--cpu-iters", type=int, default=20,
                    help="oracle iterations of the full system timed for cpu_baseline")
    ap.add_argument("--mode", default="rate", choices=["rate", "ttt", "warmstart", "batch", "unet", "sparse", "colour", "fp64pipe"],
                    help="rate: iterations per second (the bench line); ttt: time to a solution error target")
    ap.add_argument("--split-terms", type=int, default=2)
    ap.add_argument("--train-images", type=int, default=20000)
    ap.add_argument("--train-side", type=int, default=128)
    ap.add_argument("--eval-images", type=int, default=64)
    ap.add_argument("--eval-side", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--batch-maxit", type=int, default=5_000_000)
    ap.add_argument("--batch-images", type=int, default=64)
    ap.add_argument("--unet-channels", type=int, default=16, help="--mode unet: channels of 512^2 per forward")
    ap.add_argument("--colour-iters", type=int, default=150_000, help="--mode colour: iterations per variant")
    ap.add_argument("--sparse-iters", type=int, default=100_000, help="--mode sparse: iterations per system and variant")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gen_inputs(wl):
    d = WORKLOADS[wl]
    A, B, C, Xs = workloads.config_precision(d["m"], d["p"], d["q"], d["n"])
    return A, B, C, Xs


def workload_label(wl, T):
    """config.workload of both arms: the timed system and the form the native arm runs."""
    d = WORKLOADS[wl]
    return (f"{wl}: A {d['m']}x{d['p']}, B {d['q']}x{d['n']} N(0,1/cols), X* N(0,1), C = A X* B; "
            f"chosen form FP32 + split-BF16 refresh every {T}")


def recorded_traffic(kernel, algorithmic_bytes):
    """DRAM bytes per launch of `kernel` from profiles/traffic.json, scaled to a
    launch of `algorithmic_bytes` by the ratio of algorithmic bytes when the
    counters were taken on a smaller case, or None when the kernel's sources
    changed since the counters were taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() != rec["sources_sha256"]:
            return None
        measured = rec["dram_bytes_read"] + rec["dram_bytes_write"]
        return int(round(measured * algorithmic_bytes / rec["algorithmic_bytes"]))
    except Exception:
        return None


def iter_bytes(m, p, q, n, esz, gram=False, kpath=False, deferred=False, T=64):
    """Algorithmic bytes of one iteration: R read + written, B read twice
    (w = R_i B^T and v = w B), A read once for u = A A_i^T (or one row of the
    precomputed A A^T), the vectors u, v, w and the row norms.  kpath: the
    row-space form, whose update vector is R_i K with K = Lt^T Lt (n x n, read
    once) instead of two passes over B (then n is the kept rank).  deferred:
    R is read once and not written (the chunk's updates are applied by the
    refresh or a write-back after it); an iteration also reads, on average over
    a chunk of T, (T - 1) / 2 of the kept U' columns (m) and v rows (n)."""
    u_bytes = m * esz if gram else m * p * esz
    b_bytes = n * n * esz if kpath else 2 * q * n * esz
    r_bytes = (1 if deferred else 2) * m * n * esz
    extra = (T - 1) / 2 * (m + n) * esz if deferred else 0
    return r_bytes + b_bytes + u_bytes + (m + n + q) * esz + 3 * m * 8 + extra


def _alpha_estimate(B, iters=30):
    """1/||B||_2^2 from a few power iterations (the oracle's timing does not
    depend on the step's last digits)."""
    x = np.ones(B.shape[0]) / np.sqrt(B.shape[0])
    lam = 1.0
    for _ in range(iters):
        y = B @ (B.T @ x)
        lam = float(x @ y)
        x = y / np.linalg.norm(y)
    return 1.0 / lam


def _oracle_rate(A, B, C, alpha, n_it, omp):
    """Iterations per second of the FP64 oracle (FACTORED mode: the rank-1
    update with A A_i^T and (R_i B^T) B formed per iteration) on this system,
    from the oracle's own clock around its iteration loop (set-up excluded)."""
    import oracle
    r = oracle.solve(A, B, C, "grbk", alpha=alpha, maxit=n_it, seed=1, mode=oracle.MODE_FACTORED, trace=False,
                     omp=omp)
    el = max(r["loop_seconds"], 1e-9)
    return r["iters"] / el, el


def cpu_baseline_oracle(A, B, C, wl, n_it):
    """The FP64 oracle on the benchmark's own system (no slice, no scaling):
    n_it ME-GRBK iterations on every host core (OpenMP timing build, the
    reported value) and single-threaded (the tests' build)."""
    import oracle
    d = WORKLOADS[wl]
    alpha = _alpha_estimate(B)
    nproc = os.cpu_count() or 1
    rate_all, el_all = _oracle_rate(A, B, C, alpha, n_it, True)
    rate_one, el_one = _oracle_rate(A, B, C, alpha, n_it, False)
    thr = oracle.threads(True)
    return {"value": rate_all, "unit": UNIT, "cores": thr, "kind": "oracle", "nproc": nproc,
            "single_thread": {"value": rate_one, "unit": UNIT, "cores": 1, "seconds": el_one},
            "sample": f"FP64 oracle (FACTORED mode), {n_it} ME-GRBK iterations of the full {d['m']}x{d['p']} / "
                      f"{d['q']}x{d['n']} system from X0 = 0: {el_all:.2f} s on {thr} threads (OpenMP build over "
                      f"rows; host nproc {nproc}), {el_one:.2f} s on one thread; the oracle's set-up (R^0 = C, "
                      f"||A_i||^2, ||C||_F) is outside its timed loop"}


def reference_arm(args):
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    A, B, C, Xs = gen_inputs(args.workload)
    alpha = _alpha_estimate(B)
    d = WORKLOADS[args.workload]
    # iterations per step: about 0.3 s of the oracle's loop on every core at the full size
    n_it = max(4, int(4 * 20000 * 20000 / (d["m"] * d["n"])))
    run = lambda s: oracle.solve(A, B, C, "grbk", alpha=alpha, maxit=n_it, seed=s, mode=oracle.MODE_FACTORED,
                                 trace=False, omp=True)
    for _ in range(args.warmup):
        run(0)
    times = [max(run(s)["loop_seconds"], 1e-9) for s in range(args.steps)]
    tot = sum(times)
    value = args.steps * n_it / tot
    thr = oracle.threads(True)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_label(args.workload, args.iters_per_step),
                                            "iters_per_step": n_it, "variant": "ME-GRBK",
                                            "sample": f"{n_it} iterations per step of the full system"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "nproc": os.cpu_count(),
                             "sample": f"FP64 oracle (OpenMP timing build, {thr} threads, FACTORED mode), {n_it} "
                                       f"ME-GRBK iterations per step of the {d['m']}x{d['p']} / {d['q']}x{d['n']} "
                                       f"system itself, timed by the oracle's clock around its iteration loop "
                                       f"(its set-up excluded)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def native_arm(args):
    import torch
    import torch.distributed as dist
    import paper_2408_05444_gb300 as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    T = args.iters_per_step
    wl = args.workload
    dm = WORKLOADS[wl]
    m, p, q, n = dm["m"], dm["p"], dm["q"], dm["n"]

    A, B, C, Xs = gen_inputs(wl)
    Ah, Bh, Ch = (torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).pin_memory() for x in (A, B, C))
    Ad, Bd, Cd = (x.to(dev) for x in (Ah, Bh, Ch))
    keep_host = rank == 0 and world == 1 and not args.no_cpu_baseline
    if not keep_host:
        del A, B, C
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---------------- chosen form: FP32 bulk + split-BF16 refresh every T ----
    # each step: T iterations and one refresh R = C - A X B; the solve starts
    # from the current iterate, so its initial residual is the first refresh
    ctx = g.grbk_create(Ad, Bd, Cd, precision="f32", refresh_T=T, check_every=T, stream=stream,
                        split_terms=args.split_terms)
    Xd = torch.zeros(p, q, dtype=torch.float64, device=dev)
    g.grbk_solve(ctx, "grbk", X0=Xd, maxit=args.warmup * T, seed=1, X_out=Xd)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        st, res = g.grbk_solve(ctx, "grbk", X0=Xd, maxit=args.steps * T, seed=2, X_out=Xd)
        ev1.record(stream)
        barrier()
    el_ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([el_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el_ms = float(t.item())
    iters = args.steps * T
    value = world * iters / (el_ms / 1e3)
    kern_ms = res["iter_kernel_ms"] / max(res["iter_kernel_launches"], 1)
    deferred = bool(res["deferred"])
    bytes_per_launch = iter_bytes(m, p, q, n, 4, gram=bool(res["gram"]), deferred=deferred, T=T) * T
    hbm_peak, bf16_peak, peak_src = peaks()
    achieved = bytes_per_launch / (kern_ms / 1e3) / 1e9

    # ---------------- plain form: FP64, X0 = 0, no refresh ------------------
    plain = None
    if not args.no_plain:
        ctx64 = g.grbk_create(Ad, Bd, Cd, precision="f64", check_every=T, stream=stream, use_gram=1)
        X64 = torch.zeros(p, q, dtype=torch.float64, device=dev)
        g.grbk_solve(ctx64, "grbk", maxit=T, seed=1, X_out=X64)
        barrier()
        k64 = max(2, args.steps // 2)
        ev0.record(stream)
        st64, r64 = g.grbk_solve(ctx64, "grbk", maxit=k64 * T, seed=2, X_out=X64)
        ev1.record(stream)
        barrier()
        ms64 = ev0.elapsed_time(ev1)
        km64 = r64["iter_kernel_ms"] / max(r64["iter_kernel_launches"], 1)
        gbs64 = iter_bytes(m, p, q, n, 8, gram=bool(r64["gram"])) * T / (km64 / 1e3) / 1e9
        # FP64 roof: two FMAs per element of R per iteration (the update and the square)
        dfma_peak, probe_ms = g.grbk_fp64_probe(stream=stream)
        dfma64 = 2.0 * m * n * T / (km64 / 1e3)
        plain = {"precision": "f64", "value": k64 * T / (ms64 / 1e3), "unit": UNIT,
                 "kernel_GBs": gbs64, "kernel_frac_of_hbm": gbs64 / hbm_peak,
                 "kernel_fp64_fma_per_s": dfma64,
                 "fp64_fma_peak_measured": dfma_peak, "kernel_frac_of_fp64": dfma64 / dfma_peak,
                 "fp64_probe": f"grbk_fp64_probe: 8 independent FMA chains per thread, 8 x 256-thread blocks per "
                               f"SM, {probe_ms:.2f} ms timed launch",
                 "note": "FP64 residual pass, X0 = 0, no refresh (R^0 = C); A A^T formed at set-up (outside the timed region)"}
        g.grbk_destroy(ctx64)
        del X64

    # ---------------- row-space form: keeps Z = R Bt^T (m x rank B) ---------
    # same iterates as the chosen form (FP32 + split-BF16 refresh every T), with
    # the residual kept in an orthonormal basis of the row space of B
    rowspace = None
    if not args.no_rowspace:
        barrier()
        t0 = time.perf_counter()
        ctxz = g.grbk_create(Ad, Bd, Cd, precision="f32", refresh_T=T, check_every=T, stream=stream,
                             split_terms=args.split_terms, form="rowspace")
        torch.cuda.synchronize(dev)
        setup_s = time.perf_counter() - t0
        r_cols = g.grbk_form_info(ctxz)[1]
        Xz = torch.zeros(p, q, dtype=torch.float64, device=dev)
        g.grbk_solve(ctxz, "grbk", X0=Xz, maxit=args.warmup * T, seed=1, X_out=Xz)
        barrier()
        kz = 4 * args.steps
        ev0.record(stream)
        stz, rz = g.grbk_solve(ctxz, "grbk", X0=Xz, maxit=kz * T, seed=2, X_out=Xz)
        ev1.record(stream)
        barrier()
        msz = ev0.elapsed_time(ev1)
        if world > 1:
            t = torch.tensor([msz], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            msz = float(t.item())
        kmz = rz["iter_kernel_ms"] / max(rz["iter_kernel_launches"], 1)
        bz = iter_bytes(m, p, q, r_cols, 4, gram=bool(rz["gram"]), kpath=True, deferred=bool(rz["deferred"]),
                        T=T) * T
        rowspace = {"precision": "f32", "value": world * kz * T / (msz / 1e3), "unit": UNIT,
                    "ms_per_step": msz / kz, "steps": kz, "kept_columns": r_cols, "setup_s": setup_s,
                    "kernel_ms_per_launch": kmz, "kernel_GBs": bz / (kmz / 1e3) / 1e9,
                    "kernel_frac_of_hbm": bz / (kmz / 1e3) / 1e9 / hbm_peak,
                    "algorithmic_bytes_per_launch": bz,
                    "traffic": (recorded_traffic("iterate_kernel<float>/rowspace", bz)
                                if T == 64 else None),
                    "note": "residual kept as Z = R Bt^T (m x rank B) plus fixed row offsets; same iterates as "
                            "the chosen form; set-up (pivoted Cholesky of B B^T, Z^0, offsets) outside the timed "
                            "region"}
        g.grbk_destroy(ctxz)
        del Xz

    # ---------------- end to end through the C ABI with host buffers --------
    e2e = None
    if not args.no_e2e:
        Xh = torch.zeros(p, q, dtype=torch.float64).pin_memory()
        k_e2e = min(args.steps, 3)
        # one untimed step first: the library's block cache then holds blocks of this context's sizes
        c2 = g.grbk_create(Ah, Bh, Ch, precision="f32", refresh_T=T, check_every=T, stream=stream,
                           split_terms=args.split_terms)
        g.grbk_solve(c2, "grbk", X0=Xh, maxit=T, seed=99, X_out=Xh)
        g.grbk_destroy(c2)
        Xh.zero_()
        barrier()
        t0 = time.perf_counter()
        step_s = []
        for s in range(k_e2e):
            ts = time.perf_counter()
            c2 = g.grbk_create(Ah, Bh, Ch, precision="f32", refresh_T=T, check_every=T, stream=stream,
                               split_terms=args.split_terms)
            g.grbk_solve(c2, "grbk", X0=Xh, maxit=T, seed=s, X_out=Xh)
            g.grbk_destroy(c2)
            step_s.append(time.perf_counter() - ts)
        barrier()
        e2e_s = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": world * k_e2e * T / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(Ah.numel() * 4 + Bh.numel() * 4 + Ch.numel() * 4),
               "d2h_bytes_per_step": int(p * q * 8), "step_seconds": step_s,
               "note": "per step: grbk_create from pinned host A, B, C (FP32), X0 from pinned host memory, "
                       "one refresh and 64 iterations, X copied back to pinned host memory, grbk_destroy; one "
                       "untimed step before the timed ones"}

    clocks = clk.summary()
    ttt = None
    if rank == 0 and world == 1 and not args.no_ttt:
        ttt = ttt_legs(args, g, torch, dev, stream, Ad, Bd, Cd, Xs)

    cpu = None
    if keep_host:
        cpu = cpu_baseline_oracle(A, B, C, wl, args.cpu_iters)
        del A, B, C

    # solution error reached by the timed run (context for the metric)
    rse = float(torch.linalg.norm(Xd.cpu() - torch.from_numpy(Xs)) / np.linalg.norm(Xs))
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_label(wl, T),
                       "iters_per_step": T, "variant": "ME-GRBK", "parallelism": f"replicas{world}",
                       "split_terms": args.split_terms, "gram": bool(res["gram"]),
                       "update": "deferred (R read once per iteration, applied by the refresh)" if deferred
                                 else "in place (R read and written every iteration)",
                       "l2": "inputs larger than L2 (R is %.2f GB)" % (m * n * 4 / 1e9)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak,
                         "traffic": (recorded_traffic("iterate_kernel<float>", bytes_per_launch)
                                     if T == 64 else None),
                         "algorithmic_bytes_per_launch": bytes_per_launch,
                         "kernel": "iterate_kernel<float> (persistent, %d iterations per launch)" % T,
                         "kernel_ms_per_launch": kern_ms, "peak_source": peak_src},
            "plain": plain,
            "rowspace_form": rowspace,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "ttt": ttt,
            "rse_after_timed_run": rse,
            "clocks": clocks,
            "gpu_launches": int(res["launches"]),
        }
        print(json.dumps(line), flush=True)
    g.grbk_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


def _ttt_run(g, torch, dev, stream, A, B, C, Xs, precision, tol, maxit, refresh_T, check, split_terms,
             form="full"):
    """One solve from X0 = 0 to ||X - X*|| <= tol ||X*||: set-up wall time
    (grbk_create from device buffers) and the solve's device time (CUDA events
    on the launch stream around grbk_solve)."""
    t0 = time.perf_counter()
    ctx = g.grbk_create(A, B, C, precision=precision, refresh_T=refresh_T, check_every=check, stop_kind="rse",
                        x_ref=Xs, stream=stream, split_terms=split_terms, use_gram=1, form=form)
    torch.cuda.synchronize(dev)
    setup_s = time.perf_counter() - t0
    X = torch.zeros(Xs.shape, dtype=torch.float64, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    st, res = g.grbk_solve(ctx, "grbk", tol=tol, maxit=maxit, seed=1, X_out=X)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    g.grbk_destroy(ctx)
    return {"precision": precision, "form": form, "tol": tol, "status": g.grbk_strerror(st),
            "iters": res["iters"], "seconds": ev0.elapsed_time(ev1) / 1e3, "setup_s": setup_s,
            "rse": res["rse"], "refresh_T": refresh_T}


def ttt_legs(args, g, torch, dev, stream, Ad, Bd, Cd, Xs):
    """Time to target in the default run: the selected system to RSE <= 1e-4
    (chosen FP32 + split-BF16 refresh, row-space FP32, plain FP64), and the
    200x100 / 80x150 system to RSE <= 1e-6 in FP64 (the metric's target)."""
    Xsd = torch.from_numpy(Xs).to(dev)
    T = args.iters_per_step
    out = {"variant": "ME-GRBK", "stop": "||X - X*||_F <= tol ||X*||_F, tested every check_every iterations"}
    out["chosen_f32_rse1e-4"] = _ttt_run(g, torch, dev, stream, Ad, Bd, Cd, Xsd, "f32", 1e-4, 2_000_000, T, T,
                                         args.split_terms)
    out["rowspace_f32_rse1e-4"] = _ttt_run(g, torch, dev, stream, Ad, Bd, Cd, Xsd, "f32", 1e-4, 2_000_000, T, T,
                                           args.split_terms, form="rowspace")
    Ad64, Bd64, Cd64 = Ad.double(), Bd.double(), Cd.double()
    out["plain_f64_rse1e-4"] = _ttt_run(g, torch, dev, stream, Ad64, Bd64, Cd64, Xsd, "f64", 1e-4, 2_000_000, 0,
                                        256, args.split_terms)
    del Ad64, Bd64, Cd64
    A1, B1, C1, X1 = workloads.config_small()
    out["small_f64_rse1e-6"] = _ttt_run(g, torch, dev, stream, A1, B1, C1, torch.from_numpy(X1).to(dev), "f64",
                                        1e-6, 5_000_000, 0, 4096, args.split_terms)
    ch, pl, rs = out["chosen_f32_rse1e-4"], out["plain_f64_rse1e-4"], out["rowspace_f32_rse1e-4"]
    out["chosen_over_plain_speedup"] = pl["seconds"] / ch["seconds"] if ch["seconds"] > 0 else None
    out["rowspace_over_plain_speedup"] = pl["seconds"] / rs["seconds"] if rs["seconds"] > 0 else None
    out["chosen_faster_than_plain"] = bool(ch["status"] == "ok" and pl["status"] == "ok"
                                           and ch["seconds"] < pl["seconds"])
    return out


def time_to_target(args):
    """--mode ttt: the time-to-target legs alone, plus the row-space FP64 form
    and (with --steps >= 2) the plain FP64 form to RSE <= 1e-6."""
    import torch
    import paper_2408_05444_gb300 as g
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    A, B, C, Xs = gen_inputs(args.workload)
    Ad, Bd, Cd = (torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev) for x in (A, B, C))
    del A, B, C
    out = {"mode": "time_to_target", "workload": args.workload}
    out.update(ttt_legs(args, g, torch, dev, stream, Ad, Bd, Cd, Xs))
    Xsd = torch.from_numpy(Xs).to(dev)
    Ad64, Bd64, Cd64 = Ad.double(), Bd.double(), Cd.double()
    out["rowspace_f64_rse1e-4"] = _ttt_run(g, torch, dev, stream, Ad64, Bd64, Cd64, Xsd, "f64", 1e-4, 2_000_000, 0,
                                           256, args.split_terms, form="rowspace")
    if args.steps >= 2:
        out["plain_f64_rse1e-6"] = _ttt_run(g, torch, dev, stream, Ad64, Bd64, Cd64, Xsd, "f64", 1e-6, 4_000_000, 0,
                                            256, args.split_terms)
    out["split_terms"] = args.split_terms
    print(json.dumps(out), flush=True)


def warmstart_bench(args):
    """Learned warm start on batched colour-image restoration: generate
    train-images seeded images (train-side^2, 3 channels each), restore every
    channel with ME-GRBK (theta fixed at 1/2) to the discrepancy stop, train the U-Net
    (width 20) on (blurred channel, restoration) pairs, then restore
    eval-images held-out eval-side^2 RGB images (seeds disjoint from training)
    from X0 = 0 and from X0 = U-Net(C): iterations, device time, PSNR."""
    import torch
    import paper_2408_05444_gb300 as g
    from paper_2408_05444_gb300 import warmstart as ws
    dev = torch.device("cuda", 0)
    t_all = time.perf_counter()
    import os as _os
    procs = max(1, min(16, (_os.cpu_count() or 2) - 1))
    Cs_t, Ts_t = [], []
    chunk = 1024
    gen_s = solve_s = 0.0
    n_iters_train = 0
    for c0 in range(0, args.train_images, chunk):
        nimg = min(chunk, args.train_images - c0)
        t0 = time.perf_counter()
        sy = workloads.blur_systems(n_images=nimg, min_side=args.train_side, max_side=args.train_side, seed=11,
                                    first=c0, processes=procs)
        gen_s += time.perf_counter() - t0
        t0 = time.perf_counter()
        Xr, res = ws.restore([q["A"] for q in sy], [q["B"] for q in sy], [q["C"] for q in sy],
                             [np.linalg.norm(q["E"]) for q in sy], seed=c0)
        solve_s += time.perf_counter() - t0
        n_iters_train += sum(r["iters"] for r in res)
        Cs_t.append(torch.tensor(np.stack([q["C"] for q in sy]), dtype=torch.float32, device=dev))
        Ts_t.append(torch.tensor(np.stack(Xr), dtype=torch.float32, device=dev))
    C_t, T_t = torch.cat(Cs_t), torch.cat(Ts_t)
    del Cs_t, Ts_t
    net = ws.make_net(20, seed=0)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    losses = ws.train(net, C_t, T_t, epochs=args.epochs, batch=64, lr=2e-3)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    del C_t, T_t

    ev = workloads.blur_systems(n_images=args.eval_images, min_side=args.eval_side, max_side=args.eval_side,
                                seed=12, processes=procs)
    As, Bs, Cs = [q["A"] for q in ev], [q["B"] for q in ev], [q["C"] for q in ev]
    nn_ = [np.linalg.norm(q["E"]) for q in ev]
    clean = [q["X"] for q in ev]

    def psnr(X, ref):
        return 10 * np.log10(1.0 / np.mean((np.clip(X, 0, 1) - ref) ** 2))

    def timed_restore(X0s):
        b = g.grbk_batch_create(As, Bs, Cs)
        # written (not just allocated) before timing: the first copy into fresh pages would time the
        # host's page faults, not the solve
        X = [np.full((A.shape[1], B.shape[0]), 0.0) for A, B in zip(As, Bs)]
        targets = ws.DISCREPANCY_TAU * np.asarray(nn_)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        st, res = g.grbk_batch_solve(b, "grbk", X0s=X0s, targets=targets, maxit=5_000_000, seed=7,
                                     X_outs=X)
        el = time.perf_counter() - t0
        return X, res, el

    X0z, r0, t0s = timed_restore(None)
    torch.cuda.synchronize(dev)
    tw = time.perf_counter()
    X0n = ws.warm_starts(net, Cs, on_device=True)   # C to the device, U-Net forward; X0 stays there
    torch.cuda.synchronize(dev)
    t_net = time.perf_counter() - tw
    Xw, rw, tws = timed_restore(X0n)
    it0 = np.array([r["iters"] for r in r0])
    itw = np.array([r["iters"] for r in rw])
    out = {"mode": "warmstart", "train_images": args.train_images, "train_side": args.train_side,
           "train_systems": 3 * args.train_images, "train_target_iters": int(n_iters_train),
           "data_gen_s": gen_s, "target_solve_s": solve_s, "train_s": train_s, "epochs": args.epochs,
           "final_loss": float(np.mean(losses[-20:])) if losses else None,
           "eval_images": args.eval_images, "eval_side": args.eval_side, "eval_systems": len(ev),
           "x0_zero": {"iters_mean": float(it0.mean()), "iters_max": int(it0.max()), "solve_s": t0s,
                       "psnr_db": float(np.mean([psnr(x, c) for x, c in zip(X0z, clean)]))},
           "x0_unet": {"iters_mean": float(itw.mean()), "iters_max": int(itw.max()), "solve_s": tws,
                       "unet_forward_s": t_net, "rejected": int(sum(r["x0_rejected"] for r in rw)),
                       "psnr_db": float(np.mean([psnr(x, c) for x, c in zip(Xw, clean)]))},
           "blurred_psnr_db": float(np.mean([psnr(C, c) for C, c in zip(Cs, clean)])),
           "total_s": time.perf_counter() - t_all}
    print(json.dumps(out), flush=True)


def batch_bench(args):
    """Batched colour-image restoration: batch-images seeded RGB images of uneven
    sides in [128, 512] (3 systems each), all solved in one persistent launch
    with ME-GRBK (theta fixed at 1/2) to the discrepancy stop ||R_s|| <= 1.05 ||E_s||
    (or batch-maxit iterations).  Reports aggregate iterations per second."""
    import torch
    import paper_2408_05444_gb300 as g
    from paper_2408_05444_gb300 import warmstart as ws
    procs = max(1, min(16, (os.cpu_count() or 2) - 1))
    sy = workloads.blur_systems(n_images=args.batch_images, min_side=128, max_side=512, seed=13, processes=procs)
    As, Bs, Cs = [q["A"] for q in sy], [q["B"] for q in sy], [q["C"] for q in sy]
    targets = ws.DISCREPANCY_TAU * np.array([np.linalg.norm(q["E"]) for q in sy])
    work = np.array([A.shape[0] * B.shape[1] for A, B in zip(As, Bs)])

    def timed(tune):
        t0 = time.perf_counter()
        b = g.grbk_batch_create(As, Bs, Cs, tune=tune)
        create_s = time.perf_counter() - t0
        X = [np.zeros((A.shape[1], B.shape[0])) for A, B in zip(As, Bs)]
        g.grbk_batch_solve(b, "grbk", targets=targets, maxit=min(args.batch_maxit, 64), seed=1, X_outs=X)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, res = g.grbk_batch_solve(b, "grbk", targets=targets, maxit=args.batch_maxit, seed=1, X_outs=X)
        el = time.perf_counter() - t0
        its = np.array([r["iters"] for r in res])
        psnr = np.mean([10 * np.log10(1.0 / np.mean((np.clip(x, 0, 1) - q["X"]) ** 2)) for x, q in zip(X, sy)])
        variants = [g.grbk_batch_variant(b, s)[0] for s in range(len(sy))]
        tune_s = g.grbk_batch_variant(b, 0)[1]
        g.grbk_batch_destroy(b)
        return {"status": g.grbk_strerror(st), "seconds": el, "create_s": create_s, "tune_s": tune_s,
                "iters_total": int(its.sum()), "iters_mean": float(its.mean()), "iters_max": int(its.max()),
                "system_iters_per_s": float(its.sum() / el), "residual_elements_per_s": float((its * work).sum() / el),
                "stopped_by_rule": int(sum(1 for r in res if r["status"] == 0)), "psnr_db": float(psnr),
                "variants_used": {str(v): variants.count(v) for v in sorted(set(variants))}}

    g.grbk_tune_clear()
    default = timed(False)
    tuned = timed(True)
    out = {"mode": "batch", "systems": len(sy), "variants": g.grbk_tune_variants(), "default": default,
           "autotuned": tuned, "speedup": default["seconds"] / tuned["seconds"]}
    print(json.dumps(out), flush=True)


def sparse_bench(args):
    """Sparse A and B (CSR, FP64): the paper's four sprandn-shaped sets (Tables 3
    and 5, sets 3 and 6) in one launch, every variant for a fixed number of
    iterations per system (--sparse-iters, default 1e5), timed with CUDA events;
    the FP64 oracle's single-thread rate on the same dense systems for comparison."""
    import torch
    import oracle
    import paper_2408_05444_gb300 as g
    names = sorted(workloads.SPARSE_SETS)
    sets = [workloads.sparse_set(nm) for nm in names]
    K = args.sparse_iters
    out = {"mode": "sparse", "systems": names, "iters_per_system": K, "dtype": "f64", "variants": {}}
    sp = g.grbk_sparse_create([s_[0] for s_ in sets], [s_[1] for s_ in sets], [s_[2] for s_ in sets])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for variant, theta in [("rbk", 0.5), ("grbk", 0.5), ("rgrbk", 0.8), ("mwrbk", 1.0)]:
        X = [np.zeros((s_[0].shape[1], s_[1].shape[0])) for s_ in sets]
        g.grbk_sparse_solve(sp, variant, theta=theta, maxit=100, seed=1, X_outs=X)
        torch.cuda.synchronize()
        ev0.record()
        st, res = g.grbk_sparse_solve(sp, variant, theta=theta, maxit=K, seed=1)
        ev1.record()
        torch.cuda.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3
        out["variants"][f"{variant}_theta{theta}"] = {
            "seconds": sec, "system_iters_per_s": len(sets) * K / sec,
            "us_per_iteration_longest": 1e6 * sec / K,
            "relres": [r["relres"] for r in res]}
    out["ctas_per_system"] = g.grbk_sparse_cluster(sp)
    for nm, (A, B, C, Xs) in zip(names, sets):
        gn, al = g.grbk_sparse_info(sp, names.index(nm))
        out.setdefault("gram_nnz", {})[nm] = gn
    # oracle rate on the largest set (dense FACTORED, single thread)
    A, B, C, Xs = sets[names.index("table5_set6")]
    r = oracle.solve(A, B, C, "grbk", alpha=1.0 / np.linalg.norm(B, 2) ** 2, maxit=2000, mode=oracle.MODE_FACTORED,
                     trace=False)
    out["oracle_table5_set6_iters_per_s"] = r["iters"] / max(r["loop_seconds"], 1e-9)
    g.grbk_sparse_destroy(sp)
    print(json.dumps(out), flush=True)


def colour_bench(args):
    """Section 6's colour model B = A X A_c^T + E on synthetic images of the
    paper's four sizes (92x92, 96x96, 125x120, 240x192; 5 x 5 Gaussian blur with
    sigma 6, zero boundary, A_c of Section 6, noise N(0, 1e-3^2)), one system
    per image, all four in one launch; ME-RBK, ME-GRBK, ME-RGRBK (theta 0.8) and
    ME-MWRBK for 1.5e5 iterations (the largest count of Section 6) from X^0 = 0:
    device time, PSNR and SSIM as in Table 9."""
    import torch
    import scipy.sparse as sps
    import paper_2408_05444_gb300 as g
    from paper_2408_05444_gb300 import quality as Q
    names = list(workloads.COLOUR_SIZES)
    ds = [workloads.colour_model(h, w, seed=5, index=i, noise=1e-3)
          for i, (h, w) in enumerate(workloads.COLOUR_SIZES.values())]
    As = [sps.csr_matrix((d["A"][2], d["A"][1], d["A"][0]), shape=(d["h"] * d["w"],) * 2) for d in ds]
    sp = g.grbk_sparse_create(As, [d["B"] for d in ds], [d["C"] for d in ds])
    K = args.colour_iters
    out = {"mode": "colour", "images": names, "iterations": K, "dtype": "f64", "blurred": {}, "variants": {}}
    for nm, d in zip(names, ds):
        bl = workloads.unvec_image(d["C"], d["h"], d["w"])
        out["blurred"][nm] = {"psnr": Q.psnr(bl, d["image"]), "ssim": Q.ssim(bl, d["image"])}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for variant, theta in [("rbk", 0.5), ("grbk", 0.5), ("rgrbk", 0.8), ("mwrbk", 1.0)]:
        X = [np.zeros((d["h"] * d["w"], 3)) for d in ds]
        torch.cuda.synchronize()
        ev0.record()
        st, res = g.grbk_sparse_solve(sp, variant, theta=theta, maxit=K, seed=3, X_outs=X)
        ev1.record()
        torch.cuda.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3
        per = {}
        for nm, d, x in zip(names, ds, X):
            img = workloads.unvec_image(x, d["h"], d["w"])
            per[nm] = {"psnr": Q.psnr(img, d["image"]), "ssim": Q.ssim(img, d["image"])}
        out["variants"][f"{variant}_theta{theta}"] = {"seconds_incl_copies": sec,
                                                       "us_per_iteration_longest": 1e6 * sec / K, "images": per}
    g.grbk_sparse_destroy(sp)
    print(json.dumps(out), flush=True)


def unet_bench(args):
    """Warm-start network inference: the U-Net (width 20, random weights) on a batch
    of 16 channels of 512 x 512 already on the device; three untimed forwards,
    then one timed with CUDA events."""
    import torch
    import paper_2408_05444_gb300 as g
    from paper_2408_05444_gb300 import warmstart as ws
    net = ws.make_net(width=20, seed=0)
    nch = args.unet_channels
    C = torch.rand(nch, 512, 512, dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    out = {"mode": "unet", "channels": nch, "side": 512, "width": 20}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    X = {}
    names = {1: "forward_ms_tensor_cores", 2: "forward_ms_tensor_cores_one_load_per_tap", 0: "forward_ms_simt"}
    for mode in (1, 2, 0):
        g.grbk_unet_use_tensor_cores(net, mode)
        X[mode] = torch.empty_like(C)
        for _ in range(3):
            g.grbk_unet_forward(net, C, X[mode])
        torch.cuda.synchronize()
        ev0.record()
        g.grbk_unet_forward(net, C, X[mode])
        ev1.record()
        torch.cuda.synchronize()
        out[names[mode]] = ev0.elapsed_time(ev1)
    out["speedup"] = out["forward_ms_simt"] / out["forward_ms_tensor_cores"]
    out["max_rel_diff"] = float((X[1] - X[0]).abs().max() / (X[0] - C).abs().max())
    # 192 channels of 512^2 (64 RGB images, the warm start's evaluation) in batches of 16
    g.grbk_unet_use_tensor_cores(net, 1)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(192 // nch):
        g.grbk_unet_forward(net, C, X[1])
    ev1.record()
    torch.cuda.synchronize()
    out["forward_ms_192_channels_tensor_cores"] = ev0.elapsed_time(ev1)
    # one training step (forward, loss, backward, Adam) on a batch of 64 channels of 128^2,
    # the warm start's training shape: input gradients on the tensor cores vs all SIMT
    Ct = torch.rand(64, 128, 128, dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    Tt = torch.rand_like(Ct)
    for mode, name in ((1, "train_step_ms_tensor_cores"), (0, "train_step_ms_simt")):
        g.grbk_unet_use_tensor_cores(net, mode)
        for _ in range(3):
            g.grbk_unet_train_step(net, Ct, Tt, 1e-6)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(10):
            g.grbk_unet_train_step(net, Ct, Tt, 1e-6)
        torch.cuda.synchronize()
        out[name] = (time.perf_counter() - t0) * 100.0
    print(json.dumps(out), flush=True)


def fp64pipe_bench(args):
    """FP64 issue costs on one SM (grbk_fp64_issue_probe): SM cycles per operation
    per warp for dependent chains, 1 / 4 / 16 warps, 32 or 1 active lanes."""
    import paper_2408_05444_gb300 as g
    table = {}
    for op in ("add", "fma", "mul", "div", "cvt"):
        for warps in (1, 4, 16):
            for act in (32, 1):
                table[f"{op} warps={warps} lanes={act}"] = round(g.grbk_fp64_issue_probe(op, warps, act, 2048), 1)
    print(json.dumps({"mode": "fp64pipe", "unit": "SM cycles per operation per warp", "table": table}), flush=True)


def main():
    args = parse()
    if args.mode == "fp64pipe":
        fp64pipe_bench(args)
        return
    if args.mode == "unet":
        unet_bench(args)
        return
    if args.mode == "sparse":
        sparse_bench(args)
        return
    if args.mode == "colour":
        colour_bench(args)
        return
    if args.mode == "batch":
        batch_bench(args)
        return
    if args.mode == "warmstart":
        warmstart_bench(args)
        return
    if args.mode == "ttt":
        time_to_target(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        native_arm(args)


if __name__ == "__main__":
    main()
