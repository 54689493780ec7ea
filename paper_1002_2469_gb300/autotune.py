"""Autotuner for the window width (threads) and the block size n (hence P = ceil(N / n)).

The best (threads, n) depends on the GPU, on the precision form, on N (one window or many)
and on how fast the coupling between blocks decays (|rs|, |ib|: the halo blocks and the spike
corrections grow with the decay length).  `tune()` times every candidate with the library's
own solve on synthetic data of the requested shape and keeps the fastest; results are cached
per (GPU name, form, log2 N bucket, decay-length bucket) in a JSON file so that later plans
reuse them (`tuned_opts()`).  Timing: CUDA events on the current stream after warm-up, median
of several repetitions, inputs larger than L2 when N allows.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import torch

from . import dichotomy as D

CACHE = os.environ.get("DICH_AUTOTUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json"))

CANDIDATES = {
    D.PREC_MIXED: [(64, 12), (64, 16), (64, 24), (64, 32), (128, 12), (128, 16), (128, 24), (128, 32), (256, 16)],
    D.PREC_F64: [(64, 32), (64, 48), (64, 64), (64, 96), (128, 48), (128, 64)],
}


def _roots(t):
    tm1, t0, tp1 = t
    disc = t0 * t0 - 4.0 * tm1 * tp1
    q = -0.5 * (t0 + math.copysign(math.sqrt(max(disc, 0.0)), t0))
    return abs(tm1 / q), abs(tp1 / q)


def key_of(t, N: int, form: int, device_name: str | None = None) -> str:
    """Cache key: GPU name, precision form, log2 N bucket and log2 decay-length bucket."""
    rs, ib = _roots(t)
    r = max(rs, ib)
    L = 1e9 if r >= 1.0 else (1 if r == 0.0 else math.log(2.0 ** -64) / math.log(r))
    dev = device_name if device_name is not None else torch.cuda.get_device_name()
    return f"{dev}|form{form}|logN{int(math.log2(max(N, 2)))}|logL{int(math.log2(max(L, 1.0)))}"


def _load():
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _save(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp%d" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _time(plan, F, x, reps=7, inner=10):
    """Median over `reps` of the mean device time (ms) of `inner` solves of a Plan or Batch."""
    for _ in range(3):
        plan.solve(F, out=x)
    torch.cuda.synchronize()
    out = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(inner):
            plan.solve(F, out=x)
        e1.record()
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1) / inner)
    return statistics.median(out)


def tune(t, N: int, precision: int = D.PREC_AUTO, candidates=None, verbose: bool = False) -> dict:
    """Time the candidates for (t, N, precision) and cache the fastest.  Returns the entry
    {"threads", "block_size", "ms", "form"}."""
    probe = D.Plan(*t, N, precision=precision)
    form = probe.info["precision"]
    cands = candidates or CANDIDATES[D.PREC_MIXED if form == 1 else D.PREC_F64]
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    F = torch.randn(N, dtype=torch.float64, device="cuda", generator=g)
    x = torch.empty_like(F)
    best = None
    for nt, bs in cands:
        try:
            p = D.Plan(*t, N, precision=form, threads=nt, block_size=bs)
        except D.DichotomyError:
            continue
        ms = _time(p, F, x)
        if verbose:
            print(f"threads={nt} n={bs} path={p.info['path']} -> {ms:.4f} ms")
        if best is None or ms < best["ms"]:
            best = {"threads": nt, "block_size": bs, "ms": ms, "form": form}
    if best is not None:
        d = _load()
        d[key_of(t, N, form)] = best
        _save(d)
    return best


def tuned_opts(t, N: int, precision: int = D.PREC_AUTO) -> dict:
    """Keyword arguments for Plan/Batch from the cache ({} when nothing was tuned)."""
    probe = D.dichotomy_plan(t[0], t[1], t[2], N, D.make_opts(precision=precision))
    try:
        form = D.dichotomy_plan_info(probe)["precision"]
    finally:
        D.dichotomy_destroy(probe)
    ent = _load().get(key_of(t, N, form))
    if not ent:
        return {}
    return {"threads": ent["threads"], "block_size": ent["block_size"], "precision": form}


def plan(t, N: int, precision: int = D.PREC_AUTO, tune_if_missing: bool = False) -> "D.Plan":
    """A Plan using the tuned (threads, block size) when cached (tuning first if asked)."""
    kw = tuned_opts(t, N, precision)
    if not kw and tune_if_missing:
        tune(t, N, precision)
        kw = tuned_opts(t, N, precision)
    if not kw:
        kw = {"precision": precision}
    return D.Plan(*t, N, **kw)


# (threads, block size, flags): 0 = the library's choice; the flags pick the MIXED window kernel's
# register path or shared-memory path (by default a per-batch heuristic)
BATCH_CANDIDATES = [(0, 0, 0), (0, 0, D.FLAG_REG_PATH), (0, 0, D.FLAG_SMEM_PATH), (64, 16, 0), (128, 24, 0),
                    (64, 32, 0), (256, 16, 0)]


def tune_batch(N, t_m1, t_0, t_1, precision: int = D.PREC_AUTO, candidates=None, verbose: bool = False,
               F: "torch.Tensor | None" = None, offset=None) -> dict:
    """Time (threads, block size, flags) candidates for one batch of systems (sizes N, coefficient
    arrays, row offsets: packed back to back when None) with the library's batched solve and return
    the fastest as {"threads", "block_size", "flags", "ms"}; (0, 0, 0) is the library's default
    choice.  F: the right-hand sides to time with (their exponent ranges decide which conversions a
    window takes), else seeded normal values.  Not cached: a batch's composition is its own key."""
    import numpy as np
    N = np.asarray(N, dtype=np.int64)
    if F is None:
        total = int(N.sum()) if offset is None else int((np.asarray(offset) + N).max())
        g = torch.Generator(device="cuda")
        g.manual_seed(0)
        F = torch.randn(total, dtype=torch.float64, device="cuda", generator=g)
    x = torch.empty_like(F)
    best = None
    for cand in (candidates or BATCH_CANDIDATES):
        nt, bs, fl = (tuple(cand) + (0,))[:3]
        try:
            b = D.Batch(N, t_m1, t_0, t_1, offset=offset, precision=precision, threads=nt, block_size=bs,
                        flags=fl)
        except D.DichotomyError:
            continue
        ms = _time(b, F, x)
        if verbose:
            print(f"threads={nt} n={bs} flags={fl} -> {ms:.4f} ms")
        if best is None or ms < best["ms"]:
            best = {"threads": nt, "block_size": bs, "flags": fl, "ms": ms}
        del b
    return best
