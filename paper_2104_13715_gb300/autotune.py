"""Autotuner of the fused kernel's tile shape per (kernel side, image size),
and of the batched evaluation's work-item size per kernel-side group.

tune(): times every tile variant of the fused loss+gradient kernel
(dia_loss_grad, CUDA events on the caller's stream) on the caller's own pair
and selects the fastest for that kernel side.  tune_batch(): for each
kernel-side group present in a batch, times a fixed number of batched
optimiser iterations of that group's own pairs under every work-item variant
(dia_select_batch_variant) and selects the fastest.  Results are cached in a
JSON file keyed by GPU name and the shape of the problem, so later runs skip
the timing."""
from __future__ import annotations

import hashlib
import json
import os
import threading

import torch

from . import native as nat

def _default_cache():
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "dia_gb300", "tuning.json")


# the cache lives outside the package (a user cache directory, or DIA_TUNING_CACHE)
CACHE = os.environ.get("DIA_TUNING_CACHE") or _default_cache()
_lock = threading.Lock()


def _key(m, H, W, dev):
    # the variant table's shapes are part of the key: a rebuilt library with a
    # different table must not reuse indices tuned for the old one
    table = [tuple(nat.kernel_variant_desc(m, v).values()) for v in range(nat.kernel_variants(m))]
    sig = hashlib.sha256(repr(table).encode()).hexdigest()[:12]
    return f"{torch.cuda.get_device_name(dev)}|m={m}|{H}x{W}|{sig}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d, path):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(R, I, m, spec, mask=None, var=None, flat=None, reps=5, use_cache=True, stream=None,
         cache_path=None):
    """Select (and return) the fastest tile variant for this pair's shape.
    ``cache_path``: the JSON cache file (default: CACHE)."""
    path = cache_path or CACHE
    H, W = R.shape
    dev = R.device
    key = _key(m, H, W, dev)
    nvar = nat.kernel_variants(m)
    with _lock:
        cache = _load(path) if use_cache else {}
        if key in cache and cache[key]["variant"] < nvar:
            nat.select_kernel_variant(m, cache[key]["variant"])
            return cache[key]
    if nvar <= 1:
        nat.select_kernel_variant(m, 0)
        return {"variant": 0, "times_ms": None}
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    ws = nat.workspace(H, W, m, ld=R.stride(0), device=dev)
    th = torch.full((m * m + 1,), 1.0 / (m * m), dtype=torch.float64, device=dev)
    th[-1] = float(I.float().median())
    times = []
    for v in range(nvar):
        nat.select_kernel_variant(m, v)
        for _ in range(2):
            nat.loss_grad(R, I, m, th, spec, mask, var, flat, ws=ws, stream=s)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            nat.loss_grad(R, I, m, th, spec, mask, var, flat, ws=ws, stream=s)
        e1.record(s)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / reps)
    best = min(range(nvar), key=lambda v: times[v])
    nat.select_kernel_variant(m, best)
    rec = {"variant": best, "times_ms": times, "desc": nat.kernel_variant_desc(m, best)}
    with _lock:
        cache = _load(path)
        cache[key] = rec
        _save(cache, path)
    return rec


def _batch_group(m):
    return 0 if m <= 7 else 1 if m <= 15 else 2 if m <= 23 else 3


def _batch_key(g, sub, dev):
    sig = hashlib.sha256(repr(sorted((int(it["R"].shape[0]), int(it["R"].shape[1]), int(it["m"]))
                                     for it in sub)).encode()).hexdigest()[:12]
    table = [nat.lib.dia_batch_chunk_tiles(m, v) for m in range(1, 32, 2) for v in range(4)]
    tsig = hashlib.sha256(repr(table).encode()).hexdigest()[:8]
    return f"{torch.cuda.get_device_name(dev)}|batch-group={g}|{sig}|{tsig}"


def tune_batch(items, spec, iters=24, reps=1, use_cache=True, stream=None, cache_path=None):
    """Select (and return, per group) the fastest work-item variant of the
    batched evaluation for these pairs: for every kernel-side group present,
    `iters` batched optimiser iterations (Adam steps, one evaluation each) of
    that group's pairs are timed under each variant."""
    path = cache_path or CACHE
    dev = items[0]["R"].device
    groups = {}
    for it in items:
        groups.setdefault(_batch_group(it["m"]), []).append(it)
    out = {}
    for g, sub in sorted(groups.items()):
        key = _batch_key(g, sub, dev)
        with _lock:
            cache = _load(path) if use_cache else {}
        if key in cache and 0 <= cache[key]["variant"] < 4:
            nat.select_batch_variant(g, cache[key]["variant"])
            out[g] = cache[key]
            continue
        opts = nat.default_opts(max_evals=iters, max_adam_iters=iters, timeout_s=600.0)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        times = []
        for v in range(4):
            nat.select_batch_variant(g, v)
            nat.fit_batch(sub, spec, opts, stream=s)   # graph capture, workspace
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                nat.fit_batch(sub, spec, opts, stream=s)
            e1.record(s)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / reps)
        best = min(range(4), key=lambda v: times[v])
        nat.select_batch_variant(g, best)
        rec = {"variant": best, "times_ms": times, "pairs": len(sub),
               "tiles_per_item_at_m": {str(m): nat.lib.dia_batch_chunk_tiles(m, best)
                                       for m in sorted({it["m"] for it in sub})}}
        with _lock:
            cache = _load(path)
            cache[key] = rec
            _save(cache, path)
        out[g] = rec
    return out
