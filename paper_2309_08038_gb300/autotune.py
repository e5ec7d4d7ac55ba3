"""Autotuner for librosar's launch-shape choices.

* choose_azimuth(n_rng, n_az, K): the gather-MAC filter (rosar_sparse_azimuth) or its exact
  frequency-domain form (rosar_sparse_azimuth_fft), timed on synthetic data of that shape.
* tune_batch(scans): the batched kernel's azimuth tile width, persistent CTAs per SM and tile
  order (rosar_batch_tuning), timed on the caller's own scans.

Winners are cached in a JSON file keyed by GPU name and shape class
($ROSAR_AUTOTUNE_CACHE, default ~/.cache/rosar_gb300/autotune.json), so a later run on the
same GPU reuses them without timing.  Every candidate produces the same image (the
choices only change tiling and summation order), so tuning never changes results beyond
float32 rounding of the azimuth path.
"""

from __future__ import annotations

import hashlib
import json
import os
import threading

import torch

from . import ops
from .batch import Batch, Tuning

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("ROSAR_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "rosar_gb300", "autotune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value) -> None:
    with _lock:
        d = _load()
        d[key] = value
        path = cache_path()
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(d, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
        except OSError:
            pass            # a read-only home only loses the cache, not the choice


def _gpu() -> str:
    return torch.cuda.get_device_name().replace(" ", "_")


def _time_ms(fn, reps: int, warmup: int = 2) -> float:
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def choose_azimuth(n_rng: int, n_az: int, K: int, per_row: bool = False, reps: int = 20,
                   use_cache: bool = True) -> dict:
    """{'path': 'fft' | 'gather', 'us': {...}} for an n_rng x n_az image with K taps."""
    key = f"azimuth/{_gpu()}/{n_rng}x{n_az}/K{K}/{'rows' if per_row else 'shared'}"
    if use_cache:
        hit = _load().get(key)
        if hit is not None:
            return hit
    dev = torch.device("cuda")
    g = torch.Generator(device=dev).manual_seed(0)
    S = torch.randn((n_rng, n_az), dtype=torch.complex64, device=dev, generator=g)
    w = torch.randn((n_rng, K), dtype=torch.complex64, device=dev, generator=g)
    span = min(n_az, max(2 * K, n_az // 6))
    if per_row:
        o = torch.stack([torch.randperm(span, device=dev, generator=g)[:K].sort().values for _ in range(n_rng)])
    else:
        o = torch.randperm(span, device=dev, generator=g)[:K].sort().values
    o = (o - span // 2).to(torch.int32).contiguous()
    out = torch.empty_like(S)
    us = {"gather": 1e3 * _time_ms(lambda: ops.sparse_azimuth(S, w, o, out=out), reps)}
    if ops.azimuth_fft_supported(n_az):
        H = ops.azimuth_plan(w, o, n_az)
        us["fft"] = 1e3 * _time_ms(lambda: ops.sparse_azimuth_fft(S, H, out=out), reps)
    res = {"path": min(us, key=us.get), "us": us}
    _store(key, res)
    return res


def batch_candidates(fft_tiles: bool = True):
    """The tuning space.  Whole-row FFT tiles: tile order (all range tiles first; range tiles 1 or 2 scans ahead of
    the azimuth tiles, in one block or alternating in 8 chunks per scan) x dropping S from L2 once read.  Gather
    tiles: azimuth tile width x persistent CTAs per SM x tile order."""
    from .batch import DISCARD_S
    out = []
    if fft_tiles:
        for flags in (0, DISCARD_S):
            out.append(Tuning(interleave=0, flags=flags))
            for interleave, mix in ((2, 1), (3, 1), (3, 8)):
                out.append(Tuning(interleave=interleave, mix=mix, flags=flags))
        return out
    for az_tile in (512, 1024, 2048):
        for ctas in (0, 2):
            for interleave in (0, 1, 2, 3):
                out.append(Tuning(az_tile=az_tile, ctas_per_sm=ctas, interleave=interleave))
    return out


def _batch_key(scans) -> str:
    shapes = sorted((tuple(s["raw"].shape), s["w"].shape[1], s["o"].dim(), s.get("H") is not None) for s in scans)
    h = hashlib.sha1(repr(shapes).encode()).hexdigest()[:16]
    return f"batch2/{_gpu()}/{len(scans)}scans/{h}"


def tune_batch(scans, candidates=None, reps: int = 3, use_cache: bool = True) -> dict:
    """Times each candidate tuning on these scans; returns {'tuning': Tuning, 'ms': {...}}."""
    key = _batch_key(scans)
    if use_cache and candidates is None:
        hit = _load().get(key)
        if hit is not None:
            return {"tuning": Tuning(**hit["tuning"]), "ms": hit["ms"], "cached": True}
    cands = candidates or batch_candidates(all(s.get("H") is not None for s in scans))
    ms = {}
    best, best_ms = None, float("inf")
    for t in cands:
        b = Batch(scans, t)
        m = _time_ms(b.launch, reps, warmup=1)
        b.status()
        b.close()
        name = f"az{t.az_tile}_cta{t.ctas_per_sm}_il{t.interleave}_mix{t.mix}_f{t.flags}"
        ms[name] = m
        if m < best_ms:
            best, best_ms = t, m
    _store(key, {"tuning": vars(best), "ms": ms})
    return {"tuning": best, "ms": ms, "cached": False}
