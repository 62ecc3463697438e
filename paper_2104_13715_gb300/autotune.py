"""Autotuner of the fused kernel's tile shape per (kernel side, image size).

Times every tile variant of the fused loss+gradient kernel (dia_loss_grad,
CUDA events on the caller's stream) on the caller's own pair and selects the
fastest for that kernel side; results are cached in a JSON file keyed by GPU
name, kernel side and image size, so later runs skip the timing."""
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
