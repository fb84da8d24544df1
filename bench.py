#!/usr/bin/env python
"""Throughput of the TDB compressor step on GB300.

One step = one tdb_push_snapshot: snapshot difference, fused projection
(Eqs. 2.15/2.16), pseudo-inverse and complement projection, Euler update,
re-orthonormalisation, error (Eq. 2.20) and the Sec. 2.5 rank control, on one
streamed snapshot.  Default workload: the 256 x 128 x 512 stochastic-flow-like
stream (FP32 snapshots, 512 samples, r <= 20, eps_th = 1e-3, gamma_th = 99.999 %),
BF16 tensor-core projection, the learned error estimator gating the exact error
(trained first, untimed, on a separate stream of the same workload).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tdb|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) each rank compresses its own
independent stream (replicas; the method has no exchange step on one tensor per
GPU), barrier + max-over-ranks timing, value = all ranks' snapshots / time.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "snapshots/s and HBM GB/s of TDB step vs plain FP32 GPU path at equal error"
UNIT = "snapshots/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps; default: the workload's stream length (stochastic 500, reactive "
                         "1000, channel 300, analytic 200, runge 400, batch 200)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="tdb", choices=["tdb", "reference"])
    ap.add_argument("--workload", default="stochastic",
                    choices=["reactive", "stochastic", "channel", "analytic", "runge", "reactive_dbo", "reactive_tdb2", "batch"])
    ap.add_argument("--precision", default="auto", choices=["auto", "bf16", "fp32", "fp64"])
    ap.add_argument("--error-mode", default="auto", choices=["auto", "exact", "mlp", "every_k"])
    ap.add_argument("--integrator", default="euler", choices=["euler", "heun", "rk2_central"],
                    help="heun / rk2_central: two projection passes per snapshot (second-order schemes; "
                         "rk2_central uses central differences of the data and tdb_push_snapshot)")
    ap.add_argument("--train-steps", type=int, default=300,
                    help="steps of the separate training stream for the error estimator")
    ap.add_argument("--api", default="pointer", choices=["slots", "pointer"],
                    help="pointer: tdb_push_snapshot on the resident snapshots (default); slots: each "
                         "snapshot copied into an input slot, recorded step graphs")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain FP32 comparison run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the timed steps of the main run with cudaProfilerStart/Stop (for "
                         "ncu --profile-from-start off)")
    ap.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    ap.add_argument("--scaling-sweep", action="store_true",
                    help="TDB step vs on-GPU HOSVD over N^3 grids of the Runge function (one JSON line)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (torchrun); barrier + max over ranks only
# ---------------------------------------------------------------------------
def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(workload: str, rank: int):
    """Each replica compresses its own stream: rank 0 keeps the workload's default
    seed (so one GPU measures the named configuration), rank k > 0 uses that seed + 10 k."""
    from paper_2201_06958_gb300 import synth as S
    if rank == 0:
        return None
    return S.default_seed(workload) + 10 * rank


def replica_value(world: int, steps: int, ms_local: float, host_s_local: float):
    """Whole-job snapshots/s: the steps of every rank over the slowest rank's time (the
    longer of its device-event and host-clock measurements).  Returns (value, ms)."""
    ms_total = max_over_ranks(max(ms_local, host_s_local * 1e3), world)
    return world * steps / (ms_total * 1e-3), ms_total


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline inputs
# ---------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2201_06958_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key: str, sha: str):
    """DRAM bytes per launch from a committed ncu summary, if the kernel source still matches."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(kernel_key)
    if not e or e.get("source_sha") != sha:
        return None
    return e.get("dram_bytes_per_launch")


def projection_flops(dims, ranks):
    """Algorithmic flops of one projection pass (Eqs. 2.15, 2.16) at the given ranks.
    'first_contractions': what the fused kernel does on S-sized data, the mode-1 and mode-2
    contractions of the difference (2 r_1 + 2 r_2 per element; the rest is rank-sized).
    'paper_2rd': the paper's O(r d S) count for projecting onto every mode, 2 sum_n r_n per
    element (Sec. 2.6)."""
    S = 1
    for d in dims:
        S *= int(d)
    r = [float(x) for x in ranks]
    return {"first_contractions": 2.0 * (r[0] + r[1]) * S, "paper_2rd": 2.0 * sum(r) * S}


def flops_fields(dims, acts, kernel_ms):
    """projection_flops at the mean ranks of a timed run (acts: (action, ranks) per step),
    with the rate of the first contractions over the projection kernel's duration.  The
    path is bound by HBM, not by these flops."""
    p = len(dims)
    mean_ranks = [sum(a[1][n] for a in acts) / max(len(acts), 1) for n in range(p)]
    fl = projection_flops(dims, mean_ranks)
    return dict(fl, mean_ranks=[round(x, 2) for x in mean_ranks],
                tflops_first_contractions=fl["first_contractions"] / (kernel_ms * 1e-3) / 1e12)


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands on a bounded sample (spawned process)
# ---------------------------------------------------------------------------
CPU_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np, torch
import oracle as O
from paper_2201_06958_gb300 import synth as S
wl = S.make_workload({wl!r})
w = wl.weights
budget = {budget}
ctrl = O.ControllerConfig(wl.eps_th, wl.gamma_th, 10, wl.rank_max) if wl.eps_th > 0 else None
# only the compressor is timed; snapshot generation is outside the clock
V_prev = S.to_logical(wl.snapshot(0))
V_pp = None
spec = O.hosvd_spectrum(V_prev, w)
caps = O.rank_caps(wl.dims, wl.rank_max)
r = [min(caps[n], O.rank_from_spectrum(spec[n][0], wl.gamma_th)) if wl.rank[n] == 0 else wl.rank[n] for n in range(wl.ndim)]
r = O.clamp_product_bound(r)
T, U, _ = O.hosvd(V_prev, w, r, spectrum=spec)
st = O.TDBState(T, U)
controller = O.Controller(ctrl, wl.dims, w) if ctrl else None
elapsed, steps = 0.0, 0
k = 0
while elapsed < budget and steps < {max_steps}:
    k += 1
    V = S.to_logical(wl.snapshot(k))
    t0 = time.perf_counter()
    if {heun}:
        T1, U1 = O.step_heun(st.T, st.U, w, V_prev, V)
    elif {rk2c}:
        T1, U1 = O.step_rk2_central(st.T, st.U, w, V_pp, V_prev, V)
    else:
        T1, U1, _, _ = O.step_euler(st.T, st.U, w, V_prev, V)
    st = O.TDBState(T1, U1)
    eps = O.error_exact(V, st.T, st.U, w)
    if controller is not None:
        st, eps, _, _ = controller.act(V, st, eps)
    elapsed += time.perf_counter() - t0
    steps += 1
    V_pp, V_prev = V_prev, V
print(json.dumps({{"steps": steps, "seconds": elapsed}}))
"""


def _oracle_sample(workload: str, budget_s: float, max_steps: int, integrator: str, threads: int):
    """Run the oracle on the first steps of the stream in a child process with ``threads``
    BLAS/OpenMP threads; returns (steps, seconds) or an error string."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = CPU_SNIPPET.format(root=ROOT, wl=workload, budget=budget_s, max_steps=max_steps,
                              heun=integrator == "heun", rk2c=integrator == "rk2_central")
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if p.returncode != 0:
        return p.stderr[-400:]
    d = json.loads(p.stdout.strip().splitlines()[-1])
    return d["steps"], d["seconds"]


def cpu_baseline(workload: str, budget_s: float, max_steps: int, integrator: str = "euler"):
    """The oracle as it stands on the host cores (all of them), plus a shorter
    single-threaded sample of the same stream."""
    cores = os.cpu_count() or 1
    r = _oracle_sample(workload, budget_s, max_steps, integrator, cores)
    if isinstance(r, str):
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle", "error": r}
    steps, secs = r
    out = {"value": steps / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"first {steps} steps of the same stream (FP64 numpy oracle, {integrator} step, exact "
                     f"error and rank control every step), {secs:.1f} s of CPU time"}
    r1 = _oracle_sample(workload, max(budget_s / 3.0, 1.0), max_steps, integrator, 1)
    if not isinstance(r1, str):
        out["single_thread"] = {"value": r1[0] / r1[1], "unit": UNIT, "cores": 1,
                                "sample": f"first {r1[0]} steps, {r1[1]:.1f} s"}
    return out


# ---------------------------------------------------------------------------
# reference arm: the oracle, as it stands, on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, world, rank):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    wl_name = args.workload
    total = args.warmup + args.steps
    code = CPU_SNIPPET.format(root=ROOT, wl=wl_name, budget=1e9, max_steps=total, heun=args.integrator == "heun",
                              rk2c=args.integrator == "rk2_central")
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    env["CUDA_VISIBLE_DEVICES"] = ""
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3600)
    if p.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + p.stderr[-200:]}))
        return
    d = json.loads(p.stdout.strip().splitlines()[-1])
    per_step = d["seconds"] / max(d["steps"], 1)
    value = 1.0 / per_step
    wl = dict(workload_desc(wl_name), integrator=args.integrator)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": wl,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{d['steps']} full steps (warm-up included in the mean) of the FP64 numpy oracle, "
                                   f"{args.integrator} step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def workload_desc(name):
    from paper_2201_06958_gb300 import synth as S
    wl = S.make_workload(name)
    dims = "x".join(str(d) for d in wl.dims)
    return {"workload": f"{name} {dims} {wl.dtype}, rank<= {wl.rank_max}, eps_th={wl.eps_th:g}, "
                        f"gamma_th={wl.gamma_th}%, {wl.steps}-step stream",
            "dims": wl.dims, "rank_max": wl.rank_max, "eps_th": wl.eps_th, "gamma_th": wl.gamma_th,
            "seed": S.default_seed(name)}


# ---------------------------------------------------------------------------
# main arm
# ---------------------------------------------------------------------------
def run_tdb(args, world, rank, local):
    import ctypes as C

    import torch

    from paper_2201_06958_gb300 import build_lib, synth as S, tdb

    build_lib.build()
    lib = tdb.load()
    lib.tdb_set_profiling.argtypes = [C.c_void_p, C.c_int]
    lib.tdb_get_profile.argtypes = [C.c_void_p, C.c_void_p]
    lib.tdb_kernel_launches.restype = C.c_int64

    tdb_profile = tdb.tdb_profile

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = S.make_workload(args.workload, seed=replica_seed(args.workload, rank))
    precision = args.precision
    if precision == "auto":
        precision = "fp64" if wl.dtype == "f64" else "bf16"
    err_mode = args.error_mode
    if err_mode == "auto":
        # float contexts: the learned estimator gates the exact error (the G_n refresh runs
        # beside it); FP64 contexts evaluate the exact error every step
        err_mode = "exact" if precision == "fp64" else "mlp"
    K, W = args.steps, args.warmup
    est_params, est_info = None, None
    if err_mode == "mlp":
        est_params, est_info = train_estimator(args, wl, precision, dev, tdb, S)
    nsnap = W + K + 1
    snaps = torch.empty((nsnap,) + tuple(reversed(wl.dims)), dtype=wl.torch_dtype, device=dev)
    for k in range(nsnap):
        snaps[k] = wl.snapshot(k, device=dev)
    torch.cuda.synchronize()

    def make(prec, mode):
        c = tdb.TDB(wl.dims, wl.rank, rank_max=wl.rank_max, weights=wl.weights, eps_th=wl.eps_th,
                    gamma_th=wl.gamma_th, precision=prec, error_mode=mode, error_every=20,
                    integrator=args.integrator, device=dev)
        return c

    def run(prec, timed_profile=True, mode=None, api=None):
        """api 'slots': each snapshot is copied from the resident stream into the context's
        input slot inside the timed region and the recorded step replayed (one graph launch
        per step); 'pointer': tdb_push_snapshot on the resident snapshot."""
        mode = mode or err_mode
        api = api or args.api
        c = make(prec, mode)
        slots = None
        if api == "slots":
            slots = [torch.empty_like(snaps[0]), torch.empty_like(snaps[0])]
            slots[1].copy_(snaps[0])
        try:
            c.init(slots[1] if slots else snaps[0])
        except tdb.TDBError as e:
            if prec == "bf16" and e.status == 11:
                return None
            raise
        if slots:
            c.set_input_slots(slots[0], slots[1])
        if mode == "mlp":
            c.estimator_params(est_params, gate=0.9)
        info = tdb.tdb_step_info()

        def step(k):
            if slots is None:
                return c.push_raw(snaps[k].data_ptr(), info)
            par = (k - 1) % 2
            slots[par].copy_(snaps[k])
            return lib.tdb_push_slot(c.ctx, par, C.byref(info))

        for k in range(1, W + 1):
            st = step(k)
            assert st in (0, 9), (st, lib.tdb_last_error(c.ctx))
        eps, acts = [], []
        barrier(world)
        torch.cuda.synchronize()
        if timed_profile:
            lib.tdb_set_profiling(c.ctx, 1)
        l0 = lib.tdb_kernel_launches()
        sampler = ClockSampler(dev.index)
        sampler.start()
        time.sleep(0.3)
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        region = args.profile_region and not timed_profile and mode == err_mode and prec == precision
        if region:
            torch.cuda.cudart().cudaProfilerStart()
        t_host0 = time.perf_counter()
        e0.record(stream)
        for k in range(W + 1, W + K + 1):
            st = step(k)
            if st not in (0, 9):
                raise tdb.TDBError(st, lib.tdb_last_error(c.ctx).decode())
            eps.append(info.eps if info.eps_exact else float("nan"))
            acts.append((info.action, tuple(info.ranks[: wl.ndim])))
        e1.record(stream)
        torch.cuda.synchronize()
        t_host = time.perf_counter() - t_host0
        if region:
            torch.cuda.cudart().cudaProfilerStop()
        clocks = sampler.stop()
        launches = lib.tdb_kernel_launches() - l0
        barrier(world)
        ms = e0.elapsed_time(e1)
        prof = tdb_profile()
        lib.tdb_get_profile(c.ctx, C.byref(prof))
        lib.tdb_set_profiling(c.ctx, 0)
        counters = c.counters()
        try:
            tuning = c.tuning() if prec == "bf16" else None
        except tdb.TDBError:
            tuning = None
        c.close()
        return {"ms": ms, "host_s": t_host, "eps": eps, "prof": prof, "clocks": clocks, "launches": launches,
                "counters": counters, "acts": acts, "tuning": tuning}

    # timed run: recorded steps, no instrumentation; then a profiled run of the same stream
    # (CUDA events around each phase and the projection kernel, recorded into the step's graph
    # as external event nodes)
    res = run(precision, timed_profile=False)
    resp = run(precision, timed_profile=True) if res is not None else None
    if res is None:
        precision = "fp32"
        res = run(precision, timed_profile=False)
        resp = run(precision, timed_profile=True)
    value, ms_total = replica_value(world, K, res["ms"], res["host_s"])

    # roofline of the dominant kernel (the projection pass)
    prof = resp["prof"]
    S_el = 1
    for d in wl.dims:
        S_el *= d
    esz = 8 if wl.dtype == "f64" else 4
    alg_bytes = 2 * esz * S_el                      # V_{k+1} and V_k read once
    kernel_ms = prof.ms_project_main / max(prof.launches_main, 1)
    if precision == "bf16":
        kname, kfiles = "tc_project", ["tc_project.cu"]
    else:
        kname, kfiles = "mode-1 product", ["k_basic.cu"]
        alg_bytes = esz * S_el                      # the mode-1 product reads the materialised difference once
    achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    sha = kernel_source_sha(kfiles)
    traffic = recorded_traffic(f"{kname}|{args.workload}|{precision}", sha)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kname, "kernel_ms": kernel_ms,
                "algorithmic_bytes_per_launch": alg_bytes, "peak_source": peak_kind,
                "phase_ms_per_step": {"project": prof.ms_project / max(prof.steps, 1),
                                      "update": prof.ms_update / max(prof.steps, 1),
                                      "error": prof.ms_error / max(prof.steps, 1),
                                      "control_host": prof.ms_control / max(prof.steps, 1)},
                "update_phase_us_per_step": [round(prof.us_update_phase[k] / max(prof.steps, 1), 2)
                                             for k in range(prof.update_phases)]}
    roofline["flops_per_launch"] = flops_fields(wl.dims, res["acts"], kernel_ms)
    # where the kernel's CUDA events ran: inside the recorded step (external event-record
    # nodes of the replayed graph, as in the timed run) or in eager steps
    roofline["kernel_events_in"] = ("recorded step (graph replay)" if resp["counters"]["graph_replays"] > 0
                                    else "eager steps")
    if prof.spans > 0:
        # the kernel's own duration (first CTA start to last CTA end, device global timer), for
        # comparison with the event time above, which adds the launch and the event nodes
        span_ms = prof.us_project_span / prof.spans * 1e-3
        roofline["kernel_span_ms"] = span_ms
        roofline["span_frac"] = alg_bytes / (span_ms * 1e-3) / 1e9 / peak

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_total / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16": "bf16", "fp32": "f32", "fp64": "f64"}[precision], "data": "synthetic",
        "config": dict(workload_desc(args.workload), precision=precision, error_mode=err_mode, api=args.api,
                       integrator=args.integrator,
                       l2=("streamed inputs larger than L2: every step reads a new snapshot "
                           f"({esz * S_el / 1e6:.1f} MB) from a {nsnap * esz * S_el / 1e9:.2f} GB device-resident "
                           "stream; the previous snapshot is the one read in the step before"),
                       parallelism=f"replicas x{world}"),
        "roofline": roofline, "clocks": res["clocks"], "gpu_launches": int(res["launches"]),
        "reinits": res["counters"]["reinits"], "exact_evals": res["counters"]["exact_evals"],
        "graph": {"replays": res["counters"]["graph_replays"], "records": res["counters"]["graph_records"]},
        "tc_shape": res.get("tuning"),
    }
    if est_info is not None:
        line["estimator"] = dict(est_info, exact_eval_fraction=res["counters"]["exact_evals"] / max(K + W, 1))

    # the plain FP32 GPU path on the same stream, for the "at equal error" comparison
    if not args.no_compare and precision != "fp32" and wl.dtype == "f32":
        ref = run("fp32", timed_profile=False, mode="exact")
        _, ms_ref = replica_value(world, K, ref["ms"], ref["host_s"])
        pairs = [(a, b) for a, b in zip(res["eps"], ref["eps"]) if a == a and b == b]
        rel = max(abs(a - b) / b for a, b in pairs) if pairs else None
        line["plain_fp32"] = {"value": world * K / (ms_ref * 1e-3), "unit": UNIT, "ms_per_step": ms_ref / K,
                              "eps_max_rel_diff_at_exact_steps": rel, "reinits": ref["counters"]["reinits"],
                              "same_decisions": res["acts"] == ref["acts"],
                              "exact_evals": ref["counters"]["exact_evals"]}
        div = next((i for i, (a, b) in enumerate(zip(res["acts"], ref["acts"])) if a != b), None)
        if div is not None:
            # the first timed step whose action or ranks differ (actions: 0 none, 1 re-init,
            # 2 increase, 3 decrease, 4 revert, 5 cap); whether this path evaluated it exactly
            line["plain_fp32"]["first_divergence"] = {
                "step": W + 1 + div, "this": list(res["acts"][div]), "plain": list(ref["acts"][div]),
                "this_exact": res["eps"][div] == res["eps"][div]}

    # what the learned estimator gains: the same path with the exact error on every step
    if not args.no_compare and err_mode == "mlp":
        ex = run(precision, timed_profile=False, mode="exact")
        if ex is not None:
            _, ms_ex = replica_value(world, K, ex["ms"], ex["host_s"])
            v_ex = world * K / (ms_ex * 1e-3)
            line["estimator_gain"] = {"exact_every_step": v_ex, "unit": UNIT, "ratio": value / v_ex,
                                      "same_decisions": res["acts"] == ex["acts"],
                                      "exact_evals": [res["counters"]["exact_evals"], ex["counters"]["exact_evals"]]}

    # end to end through the C ABI from pinned host buffers, two ways a producer can feed
    # it: the snapshot's copy overlapped with the previous step (a ring of device buffers,
    # tdb_push_snapshot), and copy then step one after the other through the input slots.
    # The line carries the faster (a large snapshot's copy hides the step; a small one's
    # does not pay for the second stream), the other beside it.
    if not args.no_e2e:
        e2e_serial = run_e2e(wl, precision, err_mode, dev, snaps, W, K, world, lib, tdb, est_params,
                             "pointer" if args.integrator == "rk2_central" else "slots", args.integrator)
        e2e_serial["how"] = "each step's copy, then the step"
        e2e_pipe = run_e2e_pipelined(wl, precision, err_mode, dev, snaps, W, K, world, tdb, est_params,
                                     args.integrator)
        best, other = (e2e_pipe, e2e_serial) if e2e_pipe["value"] >= e2e_serial["value"] else (e2e_serial, e2e_pipe)
        best["other"] = {k: other[k] for k in ("value", "api", "how") if k in other}
        line["e2e"] = best

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_sample_seconds, K, args.integrator)
    if rank == 0:
        print(json.dumps(line))


def train_estimator(args, wl, precision, dev, tdb, S):
    """Fit the error estimator on a separate stream of the same workload (another seed),
    evaluated exactly every step; returns (parameters, report).  Not timed."""
    import torch
    tseed = 7000 + S.default_seed(args.workload)
    wt = S.make_workload(args.workload, seed=tseed)
    c = tdb.TDB(wt.dims, wt.rank, rank_max=wt.rank_max, weights=wt.weights, eps_th=wt.eps_th,
                gamma_th=wt.gamma_th, precision=precision, error_mode="exact", device=dev)
    bufs = [wt.snapshot(0, device=dev), None]
    c.init(bufs[0])
    for k in range(1, args.train_steps + 1):
        bufs[k % 2] = wt.snapshot(k, device=dev)
        c.push(bufs[k % 2])
    t0 = time.perf_counter()
    loss = c.estimator_fit(iters=2000, lr=3e-3, seed=11, gate=0.9)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    params = c.estimator_params()
    c.close()
    return params, {"train_stream": f"{args.workload} stream with seed {tseed}, {args.train_steps} exact steps",
                    "fit_seconds": fit_s, "fit_loss": loss,
                    "gate": 0.9, "max_skip": 20}


def run_e2e(wl, precision, err_mode, dev, snaps, W, K, world, lib, tdb, est_params=None, api="slots",
            integrator="euler"):
    import ctypes as C
    import torch
    host = torch.empty_like(snaps, device="cpu").pin_memory()
    host.copy_(snaps)
    c = tdb.TDB(wl.dims, wl.rank, rank_max=wl.rank_max, weights=wl.weights, eps_th=wl.eps_th,
                gamma_th=wl.gamma_th, precision=precision, error_mode=err_mode, error_every=20,
                integrator=integrator, device=dev)
    # the library borrows the last pushed snapshot (the last two under central differences)
    nring = 3 if integrator == "rk2_central" else 2
    ring = [torch.empty_like(snaps[0]) for _ in range(nring)]
    stream = torch.cuda.current_stream(dev)
    ring[0].copy_(host[0], non_blocking=True)
    c.init(ring[0])
    slots = api == "slots"
    if slots:
        c.set_input_slots(ring[1], ring[0])       # step k reads V_{k+1} from ring[k % 2]
    if err_mode == "mlp":
        c.estimator_params(est_params, gate=0.9)
    info = tdb.tdb_step_info()

    def step(k):
        buf = ring[k % nring]
        buf.copy_(host[k], non_blocking=True)          # H2D of this step's snapshot (pinned)
        if slots:                                      # the step; it reads the result back to the host
            return lib.tdb_push_slot(c.ctx, 1 - k % 2, C.byref(info))
        return c.push_raw(buf.data_ptr(), info)

    for k in range(1, W + 1):
        step(k)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(W + 1, W + K + 1):
        st = step(k)
        if st not in (0, 9):
            raise tdb.TDBError(st, lib.tdb_last_error(c.ctx).decode())
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, world)
    cnt = c.counters()
    c.close()
    h2d = snaps[0].numel() * snaps.element_size()
    return {"value": world * K / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": 1056,        # the per-step status block read back by the step
            "api": "input slots (tdb_push_slot)" if slots else "pointer (tdb_push_snapshot)",
            "graph": {"replays": cnt["graph_replays"], "records": cnt["graph_records"]},
            "exact_evals": cnt["exact_evals"]}


def run_e2e_pipelined(wl, precision, err_mode, dev, snaps, W, K, world, tdb, est_params=None,
                      integrator="euler"):
    """End to end through tdb_push_snapshot from pinned host buffers, the way a producer
    streams snapshots: three device buffers (four for central differences, which borrow two
    previous snapshots), the host-to-device copy of snapshot k+1 issued on a copy stream
    before step k, and step k waiting for its own snapshot's copy.  Every step's copy and
    its step-record readback are inside the timed region."""
    import torch
    host = torch.empty_like(snaps, device="cpu").pin_memory()
    host.copy_(snaps)
    c = tdb.TDB(wl.dims, wl.rank, rank_max=wl.rank_max, weights=wl.weights, eps_th=wl.eps_th,
                gamma_th=wl.gamma_th, precision=precision, error_mode=err_mode, error_every=20,
                integrator=integrator, device=dev)
    nbuf = 4 if integrator == "rk2_central" else 3
    ring = [torch.empty_like(snaps[0]) for _ in range(nbuf)]
    main = torch.cuda.current_stream(dev)
    copy = torch.cuda.Stream(dev)
    ready = [torch.cuda.Event() for _ in range(nbuf)]
    ring[0].copy_(host[0])
    c.init(ring[0])
    if err_mode == "mlp":
        c.estimator_params(est_params, gate=0.9)
    info = tdb.tdb_step_info()

    def fetch(k):
        with torch.cuda.stream(copy):
            ring[k % nbuf].copy_(host[k], non_blocking=True)
            ready[k % nbuf].record(copy)

    fetch(1)

    def step(k):
        if k + 1 < host.shape[0]:
            fetch(k + 1)                   # its buffer held V_{k+1-nbuf}, no longer borrowed
        main.wait_event(ready[k % nbuf])
        return c.push_raw(ring[k % nbuf].data_ptr(), info)

    for k in range(1, W + 1):
        step(k)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(W + 1, W + K + 1):
        st = step(k)
        if st not in (0, 9):
            raise tdb.TDBError(st, c.lib.tdb_last_error(c.ctx).decode())
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, world)
    cnt = c.counters()
    c.close()
    h2d = snaps[0].numel() * snaps.element_size()
    return {"value": world * K / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": 1056, "api": "pointer (tdb_push_snapshot)",
            "how": "copy of the next snapshot overlapped with the step",
            "graph": {"replays": cnt["graph_replays"], "records": cnt["graph_records"]},
            "exact_evals": cnt["exact_evals"]}


def train_estimator_on_configs(dev, tdb, S, steps=120):
    """Fit the error estimator on traces of the analytic, reactive and stochastic streams
    (the single-tensor workloads), each run in BF16 with the exact error every step; returns
    (parameters, report).  Not timed."""
    import torch
    Xs, ts, used = [], [], []
    for name, kw in (("analytic", {"n": 64}), ("reactive", {}), ("stochastic", {})):
        wl = S.make_workload(name, seed=7000 + S.default_seed(name), **kw)
        c = tdb.TDB(wl.dims, wl.rank or [4] * wl.ndim, rank_max=wl.rank_max, weights=wl.weights,
                    eps_th=wl.eps_th, gamma_th=wl.gamma_th, precision="bf16", error_mode="exact", device=dev)
        bufs = [wl.snapshot(0, device=dev, dtype=torch.float32), None]
        c.init(bufs[0])
        for k in range(1, steps + 1):
            bufs[k % 2] = wl.snapshot(k, device=dev, dtype=torch.float32)
            c.push(bufs[k % 2])
        X, t = c.estimator_trace()
        Xs.append(X)
        ts.append(t)
        used.append(f"{name} ({len(t)} rows)")
        c.close()
    import numpy as np
    X, t = np.concatenate(Xs), np.concatenate(ts)
    wl = S.make_workload("reactive", nx=64, ny=48, ns=6)
    c = tdb.TDB(wl.dims, [4, 4, 3], weights=wl.weights, precision="bf16", error_mode="exact", device=dev)
    c.init(wl.snapshot(0, device=dev))
    c.estimator_load_trace(X, t)
    t0 = time.perf_counter()
    loss = c.estimator_fit(iters=2000, lr=3e-3, seed=11, gate=0.9)
    torch.cuda.synchronize()
    params = c.estimator_params()
    c.close()
    return params, {"train_streams": ", ".join(used), "rows": int(len(t)), "fit_loss": loss,
                    "fit_seconds": time.perf_counter() - t0, "gate": 0.9, "max_skip": 20}


def run_batch(args, world, rank, local):
    """The batched configuration: 64 independent 3-mode tensors (N_n ~ U{32..128}, ranks
    U{4..24}), one BF16 tensor-core context each (members whose N_1 is not a multiple of 4
    stream zero-padded copies), launch shapes picked by the projection's tuner on each
    member's first step, the learned error estimator trained on traces of the
    single-tensor streams (configs 1-3) gating each member's exact error (eps_th = 5e-3,
    above the members' 1e-3 noise floor; ranks fixed at their initial values), every
    member's step recorded into one graph over 8 streams.  value = member snapshots per
    second.  Each batch step first moves the 64 resident snapshots into the members'
    input slots (torch._foreach_copy_, inside the timed region)."""
    import ctypes as C
    import torch
    from paper_2201_06958_gb300 import build_lib, tdb, synth as S
    build_lib.build()
    lib = tdb.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    est_params, est_info = train_estimator_on_configs(dev, tdb, S)
    members = S.make_batch(seed=1005 + 10 * rank, count=64)
    K, W = min(args.steps, 200), args.warmup
    nsnap = W + K + 1
    streams, ctxs, slots = [], [], []
    total = 0
    for wl in members:
        n = 1
        for d in wl.dims:
            n *= d
        total += n
        st = torch.empty((nsnap,) + tuple(reversed(wl.dims)), dtype=torch.float32, device=dev)
        for k in range(nsnap):
            st[k] = wl.snapshot(k, device=dev)
        streams.append(st)
        c = tdb.TDB(wl.dims, wl.rank, rank_max=wl.rank_max, weights=wl.weights, eps_th=5e-3, gamma_th=wl.gamma_th,
                    precision="bf16", error_mode="mlp", error_every=20, device=dev)
        sl = [torch.empty_like(st[0]), torch.empty_like(st[0])]
        sl[1].copy_(st[0])
        c.init(sl[1]).set_input_slots(sl[0], sl[1])
        c.estimator_params(est_params, gate=0.9)
        ctxs.append(c)
        slots.append(sl)
    batch = tdb.Batch(ctxs, nstreams=8)
    infos = (tdb.tdb_step_info * len(ctxs))()

    def step(k):
        par = (k - 1) % 2
        torch._foreach_copy_([sl[par] for sl in slots], [st[k] for st in streams])
        return lib.tdb_batch_push(batch.b, par, C.cast(infos, C.c_void_p))

    for k in range(1, W + 1):
        assert step(k) in (0, 9), lib.tdb_batch_last_error(batch.b)
    barrier(world)
    torch.cuda.synchronize()
    l0 = lib.tdb_kernel_launches()
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.profile_region:
        torch.cuda.cudart().cudaProfilerStart()
    t0 = time.perf_counter()
    e0.record(stream)
    for k in range(W + 1, W + K + 1):
        st = step(k)
        if st not in (0, 9):
            raise tdb.TDBError(st, lib.tdb_batch_last_error(batch.b).decode())
    e1.record(stream)
    torch.cuda.synchronize()
    host_s = time.perf_counter() - t0
    if args.profile_region:
        torch.cuda.cudart().cudaProfilerStop()
    clocks = sampler.stop()
    launches = lib.tdb_kernel_launches() - l0
    ms = e0.elapsed_time(e1)
    value, ms_total = replica_value(world, K * len(ctxs), ms, host_s)
    counters = batch.counters()
    nbf16 = sum(1 for c in ctxs if c.precision == "bf16")
    tun = [c.tuning() for c in ctxs]
    exact = sum(c.counters()["exact_evals"] for c in ctxs)
    alg = 2 * 4 * total
    gbs = alg / (ms_total / K * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_total / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"batch of {len(ctxs)} 3-mode tensors, N_n ~ U{{32..128}}, r ~ U{{4..24}}, "
                               f"{total / 1e6:.1f}M elements per batch step, ranks fixed at their initial values, "
                               "exact error gated by the learned estimator (eps_th = 5e-3)",
                   "members": len(ctxs), "members_bf16": nbf16,
                   "members_padded": sum(1 for wl in members if wl.dims[0] % 4 != 0),
                   "elements_per_step": total, "api": "batch graph",
                   "ingest": "torch._foreach_copy_ of the resident snapshots into the slots, timed",
                   "parallelism": f"replicas x{world}"},
        "estimator": dict(est_info, exact_eval_fraction=exact / max(len(ctxs) * (K + W), 1)),
        "tuner": {"members_below_full_grid": sum(1 for t in tun
                                                 if t["candidates"] and t["ctas_per_position"] < max(t["candidates"])),
                  "members_timed": sum(1 for t in tun if t["timed"]),
                  "choices": [t["ctas_per_position"] for t in tun],
                  "finish_split_targets": [t["finish_split_target"] for t in tun]},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                     "traffic": None, "kernel": "whole batch step (graph)", "algorithmic_bytes_per_launch": alg,
                     "peak_source": peak_kind},
        "clocks": clocks, "gpu_launches": int(launches), "batch_steps_per_s": K / (ms_total * 1e-3),
        "graph": counters,
    }
    batch.close()
    for c in ctxs:
        c.close()
    if rank == 0:
        print(json.dumps(line))


def run_scaling_sweep(args):
    """Cost of one TDB step against one HOSVD re-initialisation over N^3 grids (the paper's
    Sec. 2.6 claim: the step grows like S = N^3, the HOSVD like N^4 = S^(4/3) through its
    mode Grams).  Runge function of Sec. 3.1 at t = 1, FP32 snapshots, BF16 projection,
    fixed ranks (6, 6, 6); CUDA-event times averaged over `steps` pushes and 5 HOSVDs."""
    import torch

    from paper_2201_06958_gb300 import build_lib, synth as S, tdb
    build_lib.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rows = []
    for n in (32, 64, 96, 128, 192, 256, 384, 512):
        K = 50 if n <= 192 else 10            # snapshots held on the device: <= 0.6 GB each at N = 512
        wl = S.make_workload("runge", n=n)
        snaps = [wl.snapshot(200 + k, device=dev, dtype=torch.float32) for k in range(K + 2)]
        c = tdb.TDB(wl.dims, [6, 6, 6], rank_max=[8, 8, 8], weights=wl.weights, eps_th=0.0, precision="bf16",
                    error_mode="exact", device=dev).init(snaps[0])
        for k in range(1, 3):
            c.push(snaps[k])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(2, K + 2):
            c.push(snaps[k])
        e1.record()
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / K
        e0.record()
        for _ in range(5):
            c.reinit(snaps[K + 1])
        e1.record()
        torch.cuda.synchronize()
        hosvd_ms = e0.elapsed_time(e1) / 5
        c.close()
        rows.append({"N": n, "S": n ** 3, "step_ms": step_ms, "hosvd_ms": hosvd_ms})
    lg = lambda v: [math.log(x) for x in v]
    big = [r for r in rows if r["N"] >= 192]
    def slope(key):
        xs, ys = lg([r["S"] for r in big]), lg([r[key] for r in big])
        mx, my = sum(xs) / len(xs), sum(ys) / len(ys)
        return sum((x - mx) * (y - my) for x, y in zip(xs, ys)) / sum((x - mx) ** 2 for x in xs)
    print(json.dumps({"metric": "TDB step vs HOSVD re-initialisation time over N^3 (Runge function, BF16 projection)",
                      "unit": "ms", "rows": rows,
                      "exponent_in_S_for_N_ge_192": {"step": slope("step_ms"), "hosvd": slope("hosvd_ms")},
                      "data": "synthetic", "config": {"workload": "runge N^3, t = 1, ranks (6, 6, 6) fixed"}}))


# the configured stream length of each workload (its synthetic stream's step count)
DEFAULT_STEPS = {"stochastic": 500, "reactive": 1000, "channel": 300, "analytic": 200, "runge": 400,
                 "reactive_dbo": 1000, "reactive_tdb2": 1000, "batch": 200}


def main():
    args = parse_args()
    if args.steps is None:
        args.steps = DEFAULT_STEPS.get(args.workload, 100)
    if args.integrator == "rk2_central":
        args.api = "pointer"          # its central differences need three snapshots; slots hold two
    if args.scaling_sweep:
        run_scaling_sweep(args)
        return
    world, rank, local = dist_setup() if args.impl == "tdb" else (
        int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batch":
        run_batch(args, world, rank, local)
    else:
        run_tdb(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
