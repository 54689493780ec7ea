"""Benchmark of the Dichotomy solve on GB300 (one JSON line on stdout, rank 0).

Default workload (N = 1 GPU): the single large non-symmetric Toeplitz system
tridiag{-1.2, 2.5, -0.8}, N = 2^26, F ~ N(0, 1) from seed 0.  A "step" is one solve of that
system (the local sweeps, the dichotomy tree and the basis correction -- Stage 2 of the
paper, Table 1) with the plan (Stage 1, the Toeplitz preliminary step) built before the
timed region; Stage 1's host time is reported beside it as `plan_us`.  `value` is the
precision form chosen by the library's AUTO policy (compensated-FP32 sweeps, float-float
block quantities and tree) which meets the 1e-12 bar on this system; the plain FP64 solve is timed the same way and
reported under `fp64_plain`.  Both errors against the CPU oracle are measured every run.

Inputs (512 MB each for F and x) are larger than the 129 MB L2, so no flush is needed.
Under torchrun (N > 1) every rank solves its own system of the same size: the solve does
not shard, so the GPUs run replicas ("scaling": "weak"), timed with a barrier and the max
over ranks.

`--impl reference` times the CPU oracle (the sequential FP64 Thomas algorithm, one core)
on the same workload as the reference arm.

The CPU leg: the oracle (test infrastructure under oracle/) is called only for the reference
solutions of the error columns and for the cpu_baseline / reference timings, always after the
GPU work it checks; no timed GPU region and no library call goes through it.
"""
from __future__ import annotations

import argparse
import hashlib
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

WORKLOAD = "single Toeplitz system tridiag{-1.2, 2.5, -0.8}, N=2^26, F~N(0,1) seed 0"
METRIC = "Gunknowns/s & HBM GB/s (% of 8 TB/s) vs plain FP64 solve, at <=1e-12 rel err"
N_DEFAULT = 1 << 26
T = (-1.2, 2.5, -0.8)
BYTES_PER_UNKNOWN = 16.0   # read F, write x (algorithmic)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _src_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1002_2469_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def _profiled(kernel_key: str):
    """The committed ncu record of a kernel (DRAM bytes per launch, what binds it), if it was
    taken on the current source; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            d = json.load(fh)
        ent = d.get(kernel_key)
        if ent and ent.get("src_hash") == _src_hash():
            return ent
    except Exception:
        pass
    return None


def _traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current source."""
    ent = _profiled(kernel_key)
    return ent.get("dram_bytes_per_launch") if ent else None


def _bound(kernel_key: str, default: str):
    """What binds the kernel according to its committed profile (current source only)."""
    ent = _profiled(kernel_key)
    return ent.get("bound", default) if ent else default


def batched_cpu_baseline(tm1, t0, tp1, N, off, F, budget_s=4.0, adjoint_w=None):
    """The oracle's per-system Thomas (and, with adjoint_w, its adjoint) over all visible host
    cores, on the whole batch or on its first systems up to about budget_s seconds of work.
    Returns the cpu_baseline record (Gunknowns/s, cores, what the sample was)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    cores = len(os.sched_getaffinity(0))
    N = np.asarray(N, dtype=np.int64)
    off = np.asarray(off, dtype=np.int64)
    # a first pass on a small prefix estimates the rate, which sizes the timed sample
    k0 = int(min(N.size, max(1, np.searchsorted(np.cumsum(N), 1 << 22) + 1)))

    def run(k):
        if adjoint_w is None:
            oracle.thomas_batched(tm1[:k], t0[:k], tp1[:k], N[:k], off[:k] - off[0], F[off[0]:off[k - 1] + N[k - 1]])
            return
        def one(s):
            sl = slice(int(off[s]), int(off[s] + N[s]))
            tt = (tm1[s], t0[s], tp1[s])
            oracle.adjoint(tt, adjoint_w[sl], oracle.thomas(tt, F[sl]))
        with ThreadPoolExecutor(cores) as ex:
            list(ex.map(one, range(k)))

    t_ = time.perf_counter()
    run(k0)
    rate = int(N[:k0].sum()) / max(time.perf_counter() - t_, 1e-6)
    k = int(min(N.size, max(k0, np.searchsorted(np.cumsum(N), rate * budget_s) + 1)))
    reps, t_ = 0, time.perf_counter()
    while True:
        run(k)
        reps += 1
        el = time.perf_counter() - t_
        if el > 0.5 * budget_s or reps >= 20:
            break
    unk = int(N[:k].sum())
    what = "forward Thomas + adjoint (transposed Thomas, three sums)" if adjoint_w is not None else "Thomas"
    return {"value": round(reps * unk / el / 1e9, 4), "unit": "Gunknowns/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} pass(es) over the first {k} of {N.size} systems ({unk} unknowns): the oracle's FP64 "
                      f"{what} per system over a pool of {cores} host threads"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
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
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    """The largest v over the ranks (NCCL on device tensors, gloo on host tensors)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: int, ms_per_rank: float, world: int) -> float:
    """Gunknowns/s of the whole job: every rank's units over the slowest rank's time."""
    ms = max_over_ranks(ms_per_rank, world)
    return world * units_per_rank / (ms * 1e-3) / 1e9


def time_solves(plan, F, x, steps, warmup, world, events_stream):
    """Device time of `steps` back-to-back solves (two CUDA events on the launching stream around
    them, barrier + sync on both sides, max over ranks).  Returns (total ms, [average ms per
    launch]): a solve of this plan is one kernel launch, and no event sits between two launches
    (an event between them would keep each launch from starting while the previous one drains)."""
    import torch
    for _ in range(warmup):
        plan.solve(F, out=x)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(events_stream)
    for k in range(steps):
        plan.solve(F, out=x)
    e1.record(events_stream)
    torch.cuda.synchronize()
    barrier(world)
    total = e0.elapsed_time(e1)
    return max_over_ranks(total, world), [total / steps]


def run_gpu(args):
    import torch
    import paper_1002_2469_gb300 as D
    import oracle
    import workloads as W

    world, rank, local = dist_setup()
    dev = torch.device("cuda", torch.cuda.current_device())
    N = args.n
    # inputs: generated on the host with numpy (seed 0) so the oracle sees the same bytes
    t, F_h = W.single_c2(N=N)
    F = torch.from_numpy(F_h).to(dev)
    x = torch.empty_like(F)
    stream = torch.cuda.current_stream()

    results = {}
    # the window geometry of the headline form: the project's autotuner times (threads, block size)
    # candidates with the library's own solve on this GPU before anything is timed
    from paper_1002_2469_gb300 import autotune as AT
    if args.geometry:
        # a fixed (threads, block size), e.g. to profile one geometry without the tuner's launches
        th, bs = (int(v) for v in args.geometry.split(","))
        tuned_kw = {"threads": th, "block_size": bs}
        geometry = "fixed: " + json.dumps(tuned_kw)
    else:
        tuned = AT.tune(t, N, precision=D.PREC_AUTO, candidates=[(128, 16), (64, 16), (256, 16), (128, 24)])
        tuned_kw = {"threads": tuned["threads"], "block_size": tuned["block_size"]} if tuned else {}
        geometry = "autotuned: " + json.dumps(tuned_kw)
    # the FP64 comparator first: its ~50 ms of solves also bring the GPU out of idle before the
    # headline form's timed steps
    for name, prec in (("fp64_plain", D.PREC_F64), ("auto", D.PREC_AUTO)):
        t0 = time.perf_counter()
        plan = D.Plan(*t, N, precision=prec, **(tuned_kw if prec == D.PREC_AUTO else {}))
        plan_us = (time.perf_counter() - t0) * 1e6
        total_ms, per = time_solves(plan, F, x, args.steps, args.warmup, world, stream)
        st = plan.status()
        x_h = x.cpu().numpy()
        results[name] = dict(plan=plan, plan_us=plan_us, total_ms=total_ms, per=per, status=st,
                             x=x_h, info=plan.info)

    # accuracy against the CPU oracle (the whole vector)
    x_ref = oracle.thomas(t, F_h)
    for r in results.values():
        r["rel_err"] = float(np.max(np.abs(r["x"] - x_ref)) / np.max(np.abs(x_ref)))
        r["backward_err"] = backward_error(t, F_h, r["x"])

    # clocks during a separate timed pass of the headline form, long enough (~1.5 s) for the
    # 200 ms nvidia-smi samples; its per-step time is reported beside the main one
    head = results["auto"]
    f64 = results["fp64_plain"]
    clock_steps = max(args.steps, int(1500.0 / max(head["total_ms"] / args.steps, 1e-3)))
    with ClockSampler(torch.cuda.current_device()) as cs:
        total_ms2, per2 = time_solves(head["plan"], F, x, clock_steps, 2, world, stream)
    clocks = cs.summary()
    clocks["ms_per_step_in_pass"] = round(total_ms2 / clock_steps, 5)
    clocks["steps_in_pass"] = clock_steps

    # end to end through the public API: host F (pinned) -> plan + solve_host -> host x, every
    # step (dichotomy_solve_host: the kernels read and write the pinned host buffers directly)
    F_pin = torch.from_numpy(F_h).pin_memory()
    x_pin = torch.empty_like(F_pin).pin_memory()
    for _ in range(2):
        D.Plan(*t, N, precision=D.PREC_AUTO).solve_host(F_pin, out=x_pin)
    torch.cuda.synchronize()
    barrier(world)
    e0 = time.perf_counter()
    esteps = max(3, min(args.steps, 10))
    for _ in range(esteps):
        D.Plan(*t, N, precision=D.PREC_AUTO).solve_host(F_pin, out=x_pin)
    torch.cuda.synchronize()
    e_ms = max_over_ranks((time.perf_counter() - e0) * 1e3 / esteps, world)
    e_err = float(np.max(np.abs(x_pin.numpy() - x_ref)) / np.max(np.abs(x_ref)))
    e_same = bool(np.array_equal(x_pin.numpy(), results["auto"]["x"]))
    e_diff = float(np.max(np.abs(x_pin.numpy() - results["auto"]["x"])) / np.max(np.abs(results["auto"]["x"])))

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(F_h, t, budget_s=args.cpu_seconds)

    # the batched configurations, timed the same way (device events, inputs resident)
    others = {}
    if not args.no_other_configs:
        del F, x, results, F_pin, x_pin
        head.pop("x", None)
        f64.pop("x", None)
        torch.cuda.empty_cache()
        only = None if args.only is None else set(args.only.split(","))
        others = other_configs(D, W, oracle, stream, world, steps=max(5, min(args.steps, 20)), only=only,
                               cpu_leg=(rank == 0 and not args.no_cpu_baseline), c4_systems=args.c4_systems)

    if rank != 0:
        return
    peak, peak_kind = _peaks()
    ms = head["total_ms"] / args.steps
    value = world * N / (ms * 1e-3) / 1e9
    per_launch = statistics.median(head["per"])
    achieved = BYTES_PER_UNKNOWN * N / (per_launch * 1e-3) / 1e9
    f64_ms = f64["total_ms"] / args.steps
    form = "mixed" if head["info"]["precision"] == 1 else "f64"
    kernel_key = f"k_window_{form}_NT{head['info']['threads']}_N{N}"
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "Gunknowns/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "ff32+f64" if form == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "t": list(t), "precision_form": form,
                   "block_size": head["info"]["n"], "blocks": head["info"]["P"],
                   "threads_per_window": head["info"]["threads"], "halo": [head["info"]["halo_l"],
                                                                          head["info"]["halo_r"]],
                   "path": ["single", "halo", "general"][head["info"]["path"]], "l2": "inputs > L2 (no flush)",
                   "geometry": geometry,
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "hbm_gbs": round(achieved, 1),
        "hbm_pct_of_8tbs": round(100.0 * achieved / 8000.0, 1),
        "rel_err_vs_oracle": head["rel_err"],
        "backward_err": head["backward_err"],
        "plan_us": round(head["plan_us"], 1),
        "device_status": head["status"],
        "fp64_plain": {"value": round(world * N / (f64_ms * 1e-3) / 1e9, 3), "unit": "Gunknowns/s",
                       "ms_per_step": round(f64_ms, 5), "rel_err_vs_oracle": f64["rel_err"],
                       "backward_err": f64["backward_err"],
                       "bound": "alu (FP64 pipe)", "block_size": f64["info"]["n"],
                       "threads_per_window": f64["info"]["threads"], "device_status": f64["status"]},
        "roofline": {"bound": _bound(kernel_key, "unprofiled"), "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": _traffic(kernel_key),
                     "peak_kind": peak_kind, "kernel": kernel_key,
                     "algorithmic_bytes_per_launch": BYTES_PER_UNKNOWN * N},
        "e2e": {"value": round(world * N / (e_ms * 1e-3) / 1e9, 3), "unit": "Gunknowns/s",
                "ms_per_step": round(e_ms, 3), "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N,
                "includes": "plan + dichotomy_solve_host (pinned F, x: the window kernels read F from and write x to "
                            "host memory over the host link)",
                "rel_err_vs_oracle": e_err, "bitwise_equal_to_device_solve": e_same,
                "rel_diff_vs_device_solve": e_diff},
        "gpu_launches": args.steps * (3 if head["info"]["path"] == 2 else 1),
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if others:
        line["other_configs"] = others
    print(json.dumps(line), flush=True)


def _time_batch(solve, steps, world, stream, label=None):
    """Device time per call of solve() over `steps` calls after 3 warm-up calls.  label: the name of
    an NVTX range around the timed calls (a profiler can select their kernels by it)."""
    import torch
    for _ in range(3):
        solve()
    torch.cuda.synchronize()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if label:
        torch.cuda.nvtx.range_push(label)
    e0.record(stream)
    for _ in range(steps):
        solve()
    e1.record(stream)
    if label:
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return max_over_ranks(e0.elapsed_time(e1), world) / steps


def backward_error(t, F, x):
    """Norm-wise backward error ||F - T x||_inf / (||T||_inf ||x||_inf + ||F||_inf)."""
    tm1, t0, tp1 = t
    r = F - t0 * x
    r[1:] -= tm1 * x[:-1]
    r[:-1] -= tp1 * x[1:]
    normT = abs(tm1) + abs(t0) + abs(tp1)
    return float(np.max(np.abs(r)) / (normT * np.max(np.abs(x)) + np.max(np.abs(F))))


def cusparse_comparator(W, oracle, stream, steps):
    """The vendor library beside the Dichotomy kernels: cuSPARSE's gtsv2_nopivot (general
    tridiagonal, no pivoting: the fair choice for a diagonally dominant matrix) on the headline
    system tridiag{-1.2, 2.5, -0.8}, N = 2^26.  It overwrites its right-hand side, so every step
    copies F into it first; the copy's own time is reported beside it."""
    import ctypes
    import torch
    lib = None
    for name in ("libcusparse.so.12", os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64",
                                                   "libcusparse.so.12")):
        try:
            lib = ctypes.CDLL(name)
            break
        except OSError:
            pass
    if lib is None:
        return {"unavailable": "libcusparse.so.12 not found"}
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.cusparseCreate.argtypes = [ctypes.POINTER(P)]
    lib.cusparseSetStream.argtypes = [P, P]
    lib.cusparseDestroy.argtypes = [P]
    lib.cusparseDgtsv2_nopivot_bufferSizeExt.argtypes = [P, I, I, P, P, P, P, I, ctypes.POINTER(ctypes.c_size_t)]
    lib.cusparseDgtsv2_nopivot.argtypes = [P, I, I, P, P, P, P, I, P]
    t, F_h = W.single_c2()
    N = F_h.size
    F = torch.from_numpy(F_h).cuda()
    dl = torch.full((N,), t[0], dtype=torch.float64, device="cuda")
    d = torch.full((N,), t[1], dtype=torch.float64, device="cuda")
    du = torch.full((N,), t[2], dtype=torch.float64, device="cuda")
    dl[0] = 0.0
    du[-1] = 0.0
    B = torch.empty_like(F)
    h = P()
    if lib.cusparseCreate(ctypes.byref(h)) != 0:
        return {"unavailable": "cusparseCreate failed"}
    try:
        lib.cusparseSetStream(h, P(stream.cuda_stream))
        nbuf = ctypes.c_size_t()
        ptr = lambda x: P(x.data_ptr())
        rc = lib.cusparseDgtsv2_nopivot_bufferSizeExt(h, N, 1, ptr(dl), ptr(d), ptr(du), ptr(B), N, ctypes.byref(nbuf))
        if rc != 0:
            return {"unavailable": f"gtsv2_nopivot_bufferSizeExt status {rc}"}
        buf = torch.empty(max(1, nbuf.value), dtype=torch.uint8, device="cuda")
        status = []

        def step():
            B.copy_(F)
            status.append(lib.cusparseDgtsv2_nopivot(h, N, 1, ptr(dl), ptr(d), ptr(du), ptr(B), N, ptr(buf)))

        ms = _time_batch(step, steps, 1, stream)
        ms_copy = _time_batch(lambda: B.copy_(F), steps, 1, stream)
        if any(status):
            return {"unavailable": f"gtsv2_nopivot status {max(status)}"}
        step()
        x_ref = oracle.thomas(t, F_h)
        err = float(np.max(np.abs(B.cpu().numpy() - x_ref)) / np.max(np.abs(x_ref)))
        return {"routine": "cusparseDgtsv2_nopivot", "unknowns": N, "ms": round(ms, 4), "ms_copy_of_F": round(ms_copy, 4),
                "Gunknowns_s": round(N / ms / 1e6, 2), "Gunknowns_s_without_copy": round(N / (ms - ms_copy) / 1e6, 2),
                "workspace_bytes": int(nbuf.value), "rel_err": err}
    finally:
        lib.cusparseDestroy(h)


OTHER_CONFIGS = ("cusparse", "c1", "c2w", "c3", "c4", "c5", "f3", "f3n", "f4", "table1")


def other_configs(D, W, oracle, stream, world, steps=10, only=None, cpu_leg=True, c4_systems=0):
    """C1 (latency), the weakly dominant C2 variant, C3 (2-D Poisson modes), C4 (uneven series),
    C5 (adjoint), the rows beyond the hot path and the paper's Table 1 run: time and Gunknowns/s
    per form, with the error against the oracle (on a sample of systems for the batches).
    only: the names (OTHER_CONFIGS) to run; None runs all.  cpu_leg: time the oracle beside the
    batched configurations (C3, C4, C5) on all host cores."""
    import torch
    out = {}

    def want(name):
        return only is None or name in only

    rng = np.random.default_rng(0)

    def sample_err(xd, Fd, N, off, tm1, t0, tp1, k=24, exact=False):
        """Largest norm-wise relative error over k sampled systems, against the oracle's FP64
        Thomas, or (exact=True) against its binary128 Thomas, for systems so ill-conditioned
        that the FP64 oracle's own error approaches the tolerance."""
        errs = []
        solve = oracle.thomas_q if exact else oracle.thomas
        for s_ in rng.choice(N.size, min(k, N.size), replace=False):
            o, n = int(off[s_]), int(N[s_])
            ref = solve((tm1[s_], t0[s_], tp1[s_]), Fd[o:o + n].cpu().numpy())
            errs.append(float(np.max(np.abs(xd[o:o + n].cpu().numpy() - ref)) / max(np.max(np.abs(ref)), 1e-300)))
        return max(errs)

    if want("cusparse"):
        out["cusparse_gtsv2_nopivot_c2"] = cusparse_comparator(W, oracle, stream, steps)
        torch.cuda.empty_cache()

    if want("c1"):
        # C1: tridiag{-1, 4, -1}, N = 65536 (1 MB in, 1 MB out): latency of one solve, three
        # buffer sets in rotation, back-to-back solves between two events (replays of a CUDA graph;
        # the loop of Python calls is reported beside it)
        t1, F1 = W.single_c1()
        sets = [(torch.from_numpy(F1 * (1.0 + 0.1 * k)).cuda(), torch.empty(F1.size, dtype=torch.float64, device="cuda"))
                for k in range(3)]
        c1 = {"unknowns": int(F1.size)}
        for name, prec in (("auto", D.PREC_AUTO), ("fp64_plain", D.PREC_F64)):
            plan = D.Plan(*t1, F1.size, precision=prec)
            reps = 300
            us_host = 1e3 * _time_batch(lambda: [plan.solve(Fk, out=xk) for Fk, xk in sets], reps, world, stream) / 3
            # device latency: 90 solves captured in one CUDA graph, replayed between two events (the
            # Python call overhead of each solve is then off the timeline)
            graph = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for Fk, xk in sets:
                    plan.solve(Fk, out=xk)
            torch.cuda.current_stream().wait_stream(side)
            with torch.cuda.graph(graph):
                for _ in range(30):
                    for Fk, xk in sets:
                        plan.solve(Fk, out=xk)
            us = 1e3 * _time_batch(graph.replay, 10, world, stream) / 90
            err = max(float(np.max(np.abs(xk.cpu().numpy() - oracle.thomas(t1, Fk.cpu().numpy())))
                            / np.max(np.abs(oracle.thomas(t1, Fk.cpu().numpy())))) for Fk, xk in sets)
            c1[name] = {"us_per_solve": round(us, 2), "us_per_solve_python_loop": round(us_host, 2),
                        "Gunknowns_s": round(F1.size / us / 1e3, 2), "windows": plan.info["tiles"], "rel_err": err}
            del graph
        out["c1_latency_65536"] = c1
        del sets

    if want("c2w"):
        # C2 variant: the weakly dominant tridiag{-1, 2.001, -1} at N = 2^26 (decay length ~1400
        # rows; the AUTO policy takes the FP64 form here, gain 64 > 24)
        t2w, F2w = W.single_c2(weak=True)
        Fd = torch.from_numpy(F2w).cuda()
        xd = torch.empty_like(Fd)
        ref2w = oracle.thomas(t2w, F2w)
        c2w = {"unknowns": int(F2w.size)}
        for name, prec in (("auto", D.PREC_AUTO), ("mixed", D.PREC_MIXED), ("fp64_plain", D.PREC_F64)):
            plan = D.Plan(*t2w, F2w.size, precision=prec)
            ms = _time_batch(lambda: plan.solve(Fd, out=xd), steps, world, stream)
            xh = xd.cpu().numpy()
            c2w[name] = {"ms": round(ms, 4), "Gunknowns_s": round(F2w.size / ms / 1e6, 2),
                         "form": ["f64", "mixed"][plan.info["precision"]], "path": ["single", "halo", "general"][plan.info["path"]],
                         "block_size": plan.info["n"], "halo": [plan.info["halo_l"], plan.info["halo_r"]],
                         "rel_err": float(np.max(np.abs(xh - ref2w)) / np.max(np.abs(ref2w))),
                         "backward_err": backward_error(t2w, F2w, xh)}
        out["c2_weak_2e26"] = c2w
        del Fd, xd, ref2w

    if want("c3"):
        # C3: 4096 Poisson modes of N = 4096 (DST of a seeded smooth source)
        tm1, t0, tp1, N, rhs = W.poisson_c3()
        off = W.offsets(N)
        Fd = torch.from_numpy(rhs.reshape(-1)).cuda()
        xd = torch.empty_like(Fd)
        c3 = {"unknowns": int(N.sum())}
        from paper_1002_2469_gb300 import autotune as AT
        tb = AT.tune_batch(N, tm1, t0, tp1, precision=D.PREC_AUTO, F=Fd)
        c3["autotuned"] = tb
        for name, prec in (("auto", D.PREC_AUTO), ("fp64_plain", D.PREC_F64)):
            kw = {k: tb[k] for k in ("threads", "block_size", "flags")} if (tb and prec == D.PREC_AUTO) else {}
            b = D.Batch(N, tm1, t0, tp1, precision=prec, **kw)
            ms = _time_batch(lambda: b.solve(Fd, out=xd), steps, world, stream, label=f"c3_{name}")
            forms = b.info["form"]
            c3[name] = {"ms": round(ms, 4), "Gunknowns_s": round(N.sum() / ms / 1e6, 2),
                        "hbm_GBs": round(16 * N.sum() / ms / 1e6, 1), "mixed_systems": int(forms.sum()),
                        "max_rel_err_sampled_vs_binary128": sample_err(xd, Fd, N, off, tm1, t0, tp1, exact=True)}
        if cpu_leg:
            c3["cpu_baseline"] = batched_cpu_baseline(tm1, t0, tp1, N, off, rhs.reshape(-1))
        out["c3_poisson_4096x4096"] = c3
        del Fd, xd

    if want("c4"):
        # C4: 10000 systems, N log-uniform in [256, 2^20]
        N, off_tight, tm1, t0, tp1, _ = W.uneven_c4(with_rhs=False)
        if c4_systems:   # the first systems only (a smaller case of the same series, for profiling)
            N, off_tight, tm1, t0, tp1 = N[:c4_systems], off_tight[:c4_systems], tm1[:c4_systems], \
                t0[:c4_systems], tp1[:c4_systems]
        # layout: every system at a 16-byte aligned offset (even row), where the register path's bulk
        # copies can start; the tightly packed layout (odd offsets after odd sizes) is timed beside it
        off = W.offsets(N + (N & 1))
        Fd = W.device_uniform(int(off[-1] + N[-1]), W.SEED_RHS, "cuda")
        xd = torch.empty_like(Fd)
        c4 = {"unknowns": int(N.sum()), "layout": "systems at 16-byte aligned (even-row) offsets"}
        from paper_1002_2469_gb300 import autotune as AT
        tb = AT.tune_batch(N, tm1, t0, tp1, precision=D.PREC_AUTO, F=Fd, offset=off,
                           candidates=[(0, 0, 0), (0, 0, D.FLAG_SMEM_PATH), (64, 16, 0), (256, 16, 0)])
        c4["autotuned"] = tb
        for name, prec in (("auto", D.PREC_AUTO), ("fp64_plain", D.PREC_F64)):
            kw = {k: tb[k] for k in ("threads", "block_size", "flags")} if (tb and prec == D.PREC_AUTO) else {}
            b = D.Batch(N, tm1, t0, tp1, offset=off, precision=prec, **kw)
            ms = _time_batch(lambda: b.solve(Fd, out=xd), max(3, steps // 2), world, stream, label=f"c4_{name}")
            c4[name] = {"ms": round(ms, 3), "Gunknowns_s": round(N.sum() / ms / 1e6, 2),
                        "hbm_GBs": round(16 * N.sum() / ms / 1e6, 1), "windows": int(b.info["windows"]),
                        "max_rel_err_sampled": sample_err(xd, Fd, N, off, tm1, t0, tp1)}
            if prec == D.PREC_AUTO:
                bt = D.Batch(N, tm1, t0, tp1, offset=off_tight, precision=prec, **kw)
                mst = _time_batch(lambda: bt.solve(Fd, out=xd), max(3, steps // 2), world, stream)
                c4["auto_tight_layout"] = {"ms": round(mst, 3), "Gunknowns_s": round(N.sum() / mst / 1e6, 2),
                                           "odd_offsets": int((off_tight & 1).sum()),
                                           "note": "systems at odd offsets take the shared-memory path"}
                del bt
        if cpu_leg:
            nh = int(np.searchsorted(np.cumsum(N), 1 << 28) + 1)      # the first ~2 GB of systems
            c4["cpu_baseline"] = batched_cpu_baseline(tm1[:nh], t0[:nh], tp1[:nh], N[:nh], off[:nh],
                                                      Fd[:int(off[nh - 1] + N[nh - 1])].cpu().numpy())
        out["c4_uneven_10000"] = c4
        del Fd, xd
        torch.cuda.empty_cache()

    if want("c5"):
        # C5: forward + adjoint over 1024 systems of N = 65536
        Ns, off, tm1, t0, tp1, _, _ = W.adjoint_c5(with_data=False)
        Fd = W.device_uniform(int(Ns.sum()), W.SEED_RHS, "cuda")
        wd = W.device_uniform(int(Ns.sum()), W.SEED_W, "cuda")
        xd = torch.empty_like(Fd)
        c5 = {"unknowns": int(Ns.sum())}
        for name, prec in (("auto", D.PREC_AUTO), ("fp64_plain", D.PREC_F64)):
            b = D.Batch(Ns, tm1, t0, tp1, precision=prec)
            gF = torch.empty_like(Fd)
            gt = torch.empty((Ns.size, 3), dtype=torch.float64, device="cuda")

            def step():
                b.solve(Fd, out=xd)
                D.dichotomy_adjoint_batched(b.handle, wd, xd, gF, gt)
            ms = _time_batch(step, steps, world, stream, label=f"c5_{name}")
            s_ = 7
            o, n = int(off[s_]), int(Ns[s_])
            tt = (tm1[s_], t0[s_], tp1[s_])
            lam, g = oracle.adjoint(tt, wd[o:o + n].cpu().numpy(), oracle.thomas(tt, Fd[o:o + n].cpu().numpy()))
            c5[name] = {"ms_forward_plus_adjoint": round(ms, 4), "Gunknowns_s": round(Ns.sum() / ms / 1e6, 2),
                        "rel_err_gF_sys7": float(np.max(np.abs(gF[o:o + n].cpu().numpy() - lam)) / np.max(np.abs(lam))),
                        "rel_err_gt_sys7": float(np.max(np.abs(gt[s_].cpu().numpy() - g)) / np.max(np.abs(g)))}
        if cpu_leg:
            c5["cpu_baseline"] = batched_cpu_baseline(tm1, t0, tp1, Ns, off, Fd.cpu().numpy(),
                                                      adjoint_w=wd.cpu().numpy())
        out["c5_adjoint_1024x65536"] = c5
        del Fd, wd, xd
        torch.cuda.empty_cache()

    if want("f3"):
        # f3: 2-D Dirichlet Poisson by separation of variables on a 4096 x 4096-interval grid
        # (M = 4095 interior points per direction): DST-I along x, the 4095 mode systems through the
        # batched Dichotomy solve, inverse DST-I; manufactured solution u* ~ U[-1, 1]
        from paper_1002_2469_gb300 import poisson as PS
        from oracle import poisson as OP
        M = 4095
        us = np.random.default_rng(0).uniform(-1.0, 1.0, (M, M))
        fd = torch.from_numpy(OP.laplacian5(us)).cuda()
        solver = PS.Poisson2D(M)
        ms_total = _time_batch(lambda: solver.solve(fd), steps, world, stream)
        rhs = torch.empty(M * M, dtype=torch.float64, device="cuda")
        v = torch.empty_like(rhs)
        ms_solve = _time_batch(lambda: solver.batch.solve(rhs, out=v), steps, world, stream)
        u = solver.solve(fd).cpu().numpy()
        out["f3_poisson2d_4095"] = {"unknowns": M * M, "ms_total": round(ms_total, 4), "ms_dichotomy": round(ms_solve, 4),
                                    "Gunknowns_s": round(M * M / ms_total / 1e6, 2),
                                    "form": "AUTO per mode", "transform": "DST-I via torch.fft (cuFFT)",
                                    "rel_err_vs_manufactured": float(np.max(np.abs(u - us)) / np.max(np.abs(us)))}
        del fd, rhs, v, solver
        torch.cuda.empty_cache()

    if want("f3n"):
        # f2 + f3: the same driver with Neumann conditions in y (4096 cell centres): every mode is a
        # quasi-Toeplitz system of eq. 21 (psi = chi = -1), solved in one batch with the corner step
        My = 4096
        us = np.random.default_rng(0).uniform(-1.0, 1.0, (M, My))
        fd = torch.from_numpy(OP.laplacian5_neumann_y(us)).cuda()
        solver = PS.Poisson2D(M, My=My, bc_y="neumann")
        ms_total = _time_batch(lambda: solver.solve(fd), steps, world, stream)
        rhs = torch.empty(M * My, dtype=torch.float64, device="cuda")
        v = torch.empty_like(rhs)
        ms_solve = _time_batch(lambda: solver.batch.solve(rhs, out=v), steps, world, stream)
        u = solver.solve(fd).cpu().numpy()
        out["f3_poisson2d_neumann_y_4095x4096"] = {
            "unknowns": M * My, "ms_total": round(ms_total, 4), "ms_dichotomy": round(ms_solve, 4),
            "Gunknowns_s": round(M * My / ms_total / 1e6, 2), "form": "AUTO per mode, quasi-Toeplitz corners",
            "rel_err_vs_manufactured": float(np.max(np.abs(u - us)) / np.max(np.abs(us)))}
        del fd, rhs, v, solver
        torch.cuda.empty_cache()

    if want("f4"):
        # f4: a general tridiagonal matrix, N = 2^24: |a_i|, |c_i| <= 1 random, b_i = +-(|a_i| + |c_i| + U[0.3, 1.5]),
        # F ~ N(0, 1); the O(N) preliminary step (plan and bind: on the device by default, plan_s; on
        # the host, plan_s_host_prelim), then solves on the device in the AUTO form (float-float here)
        # and in the plain FP64 form
        Ng = 1 << 24
        rng = np.random.default_rng(1)
        ga, gc = rng.uniform(-1, 1, Ng), rng.uniform(-1, 1, Ng)
        gb = (np.abs(ga) + np.abs(gc) + rng.uniform(0.3, 1.5, Ng)) * rng.choice([-1.0, 1.0], Ng)
        gF = np.random.default_rng(2).standard_normal(Ng)
        t0_ = time.perf_counter()
        D.GenPlan(ga, gb, gc, flags=D.FLAG_HOST_PRELIM)
        plan_s_host = time.perf_counter() - t0_
        torch.cuda.empty_cache()
        gFd = torch.from_numpy(gF).cuda()
        gxd = torch.empty_like(gFd)
        gref = oracle.thomas_tridiag(ga, gb, gc, gF)
        f4 = {"unknowns": Ng, "bytes_per_unknown": 56, "plan_s_host_prelim": round(plan_s_host, 3)}
        for name, prec in (("auto", D.PREC_AUTO), ("fp64_plain", D.PREC_F64)):
            t0_ = time.perf_counter()
            gplan = D.GenPlan(ga, gb, gc, precision=prec)
            plan_s = time.perf_counter() - t0_
            ms_g = _time_batch(lambda: gplan.solve(gFd, out=gxd), steps, world, stream)
            gx = gxd.cpu().numpy()
            f4[name] = {"ms": round(ms_g, 4), "Gunknowns_s": round(Ng / ms_g / 1e6, 2),
                        "hbm_GBs": round(56 * Ng / ms_g / 1e6, 1), "plan_s": round(plan_s, 3),
                        "path": ["single", "halo", "general"][gplan.info["path"]], "block_size": gplan.info["n"],
                        "threads": gplan.info["threads"], "form": "mixed" if gplan.info["precision"] == 1 else "f64",
                        "rel_err": float(np.max(np.abs(gx - gref)) / np.max(np.abs(gref)))}
            del gplan
        out["f4_general_2e24"] = f4
        del gFd, gxd
        torch.cuda.empty_cache()

    if want("table1"):
        # the paper's largest 2-D Poisson run (Table 1: 65536 x 65536, Stage 2 = the dichotomy process):
        # the 65536 mode systems of N = 65536 (4.3e9 unknowns, 34 GB per vector) as one batch; the
        # right-hand sides are synthetic (U[-1, 1] drawn on the device) in place of the DST of a source.
        # Stage 1 here is the batch plan on the host.  The paper's times are context only (4096 MPI
        # processes on Xeon X5570 nodes).
        Mp = 65536
        t0p = PS.mode_t0(Mp)
        onesp = np.ones(Mp)
        t1_ = time.perf_counter()
        bp = D.Batch(np.full(Mp, Mp, dtype=np.int64), -onesp, t0p, -onesp, precision=D.PREC_AUTO)
        stage1_s = time.perf_counter() - t1_
        Fp = W.device_uniform(Mp * Mp, W.SEED_RHS, "cuda")
        xp = torch.empty_like(Fp)
        ms_p = _time_batch(lambda: bp.solve(Fp, out=xp), max(3, steps // 4), world, stream)
        errs, oerrs = [], []
        for k in (1, 2, 100, 30000, 65535):      # sampled modes against the binary128 oracle
            row = slice((k - 1) * Mp, k * Mp)
            tk = (-1.0, float(t0p[k - 1]), -1.0)
            Fk = Fp[row].cpu().numpy()
            ref = oracle.thomas_q(tk, Fk)
            errs.append(float(np.max(np.abs(xp[row].cpu().numpy() - ref)) / np.max(np.abs(ref))))
            oerrs.append(float(np.max(np.abs(oracle.thomas(tk, Fk) - ref)) / np.max(np.abs(ref))))
        out["paper_table1_poisson_65536"] = {
            "unknowns": Mp * Mp, "stage2_ms": round(ms_p, 3), "Gunknowns_s": round(Mp * Mp / ms_p / 1e6, 2),
            "hbm_GBs": round(16 * Mp * Mp / ms_p / 1e6, 1), "stage1_host_s": round(stage1_s, 3),
            "mixed_systems": int(bp.info["form"].sum()), "sampled_modes": [1, 2, 100, 30000, 65535],
            "rel_err_vs_binary128": errs, "fp64_oracle_rel_err_vs_binary128": oerrs,
            "paper_context": {"stage2_s": {"p=256": 3.83, "p=4096": 0.35}, "stage1_toeplitz_s": {"p=4096": 0.30},
                              "hardware": "Lomonosov cluster, Xeon X5570 nodes, MPI (Table 1)"}}
        del bp, Fp, xp
        torch.cuda.empty_cache()
    return out


def cpu_baseline(F_h, t, budget_s=15.0):
    """The oracle's sequential FP64 Thomas (one core) on the same system, repeated for about
    budget_s seconds; reported in Gunknowns/s."""
    import oracle
    N = F_h.size
    oracle.thomas(t, F_h[: 1 << 16])
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.thomas(t, F_h)
        done += 1
        el = time.perf_counter() - t0
        if el > budget_s or done >= 64:
            break
    return {"value": round(done * N / el / 1e9, 4), "unit": "Gunknowns/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} full solves of the N={N} system (sequential Thomas, FP64)"}


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores for the same workload."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import workloads as W
    N = args.n
    t, F_h = W.single_c2(N=N)
    for _ in range(args.warmup):
        oracle.thomas(t, F_h)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.thomas(t, F_h)
    el = time.perf_counter() - t0
    ms = el * 1e3 / args.steps
    value = N / (ms * 1e-3) / 1e9
    line = {
        "impl": "reference",
        "metric": METRIC, "value": round(value, 4), "unit": "Gunknowns/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "t": list(T), "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": round(value, 4), "unit": "Gunknowns/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} full solves of the N={N} system (sequential Thomas, FP64)"},
        "e2e": {"value": round(value, 4), "unit": "Gunknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true")
    ap.add_argument("--c4-systems", type=int, default=0,
                    help="time only the first K systems of the uneven series (a smaller case for profiling)")
    ap.add_argument("--geometry", default=None,
                    help="threads,block_size of the headline solve instead of the autotuner's choice")
    ap.add_argument("--only", default=None,
                    help="comma-separated subset of the other configurations: " + ",".join(OTHER_CONFIGS))
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
