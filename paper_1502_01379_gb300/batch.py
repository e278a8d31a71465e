"""Batches of independent butterfly operators, and the autotuner that picks
their launch configuration.

A batch applies many factorizations of uneven size, rank and vector count
together (bf_batch_* in libbfly.so): one grouped launch runs every
operator's down half, a second every up half, and the pair is captured once
into a CUDA graph.  What the grouped kernels can vary is the RHS tile per
thread block (T = 1, 2, 4, 8) and the factor ring (slot size, slots): bigger
tiles reuse each factor entry more, smaller rings let more thread blocks
share an SM.  `autotune` times each candidate on the actual batch (CUDA
events, the graph mode), keeps the fastest, and caches the choice on disk,
keyed by the batch's shapes, vector counts and GPU.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile

from . import capi

# (T, slot_kb, stages)
CANDIDATES = [(T, kb, st) for T in (1, 2, 4, 8) for (kb, st) in ((8, 2), (16, 2), (32, 2), (64, 2), (16, 3))] + \
    [(4, 48, 3), (8, 32, 3), (8, 48, 2)]


def default_cache_path() -> str:
    return os.environ.get("BF_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                           "paper_1502_01379_gb300", "batch_tuning.json")


def signature(factors_list, nrhs) -> str:
    import torch
    desc = ";".join(f"{F.L},{F.n0},{F.r},{n}" for F, n in zip(factors_list, nrhs))
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return hashlib.sha256(f"{dev}|{desc}".encode()).hexdigest()[:24]


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path) or ".", suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1)
    os.replace(tmp, path)


def time_batch(batch, reps: int = 5, mode: int = capi.BF_BATCH_GRAPH, adjoint: bool = False) -> float:
    """Mean milliseconds of one batch apply (CUDA events on the current stream)."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(2):
        capi.bf_batch_apply(batch, adjoint, mode, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        capi.bf_batch_apply(batch, adjoint, mode, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    capi.bf_batch_check(batch)
    return e0.elapsed_time(e1) / reps


def autotune(factors_list, ins, outs, nrhs, candidates=CANDIDATES, cache_path: str | None = None,
             reps: int = 5) -> dict:
    """Best (T, slot_kb, stages) for this batch: from the cache if present,
    else by timing every candidate that fits; the result is cached."""
    path = cache_path or default_cache_path()
    key = signature(factors_list, nrhs)
    cache = _load(path)
    if key in cache:
        return dict(cache[key], cached=True)
    tried = []
    for T, kb, st in candidates:
        try:
            b = capi.bf_batch_create(factors_list, ins, outs, nrhs, T=T, slot_kb=kb, stages=st)
        except capi.BfError as e:
            if e.status == capi.BF_ERR_UNSUPPORTED:
                continue
            raise
        ms = time_batch(b, reps)
        b.destroy()
        tried.append({"T": T, "slot_kb": kb, "stages": st, "ms": ms})
    if not tried:
        raise RuntimeError("no batch configuration fits these operators")
    best = min(tried, key=lambda d: d["ms"])
    entry = {"T": best["T"], "slot_kb": best["slot_kb"], "stages": best["stages"], "ms": best["ms"],
             "tried": tried}
    cache = _load(path)
    cache[key] = entry
    _store(path, cache)
    return dict(entry, cached=False)


def create_tuned(factors_list, ins, outs, nrhs, cache_path: str | None = None) -> tuple:
    """(batch, config): the batch built with its autotuned configuration."""
    cfg = autotune(factors_list, ins, outs, nrhs, cache_path=cache_path)
    b = capi.bf_batch_create(factors_list, ins, outs, nrhs, T=cfg["T"], slot_kb=cfg["slot_kb"],
                             stages=cfg["stages"])
    return b, cfg
