"""Autotuning of the column sweep (tile width and radix order), with a JSON
cache on disk.

``autotune(sizes)`` runs rt_autotune on the current GPU for each grid side
(the library keeps the winners for this process) and writes them to the
cache file under the GPU's name; ``load()`` feeds cached winners for this
GPU back to the library through rt_tune_set, so later processes skip the
measurement.
"""
from __future__ import annotations

import ctypes
import json
import os

from . import rt

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune.json")


def _sig():
    L = rt.lib()
    L.rt_autotune.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.rt_tune_set.argtypes = [ctypes.c_int, ctypes.c_int]
    L.rt_tune_get.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.rt_tune_set_order.argtypes = [ctypes.c_int, ctypes.c_int]
    L.rt_tune_get_order.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.rt_tune_set_order.restype = L.rt_tune_get_order.restype = ctypes.c_int
    L.rt_tune_set_batch_mixed.argtypes = [ctypes.c_int]
    L.rt_tune_get_batch_mixed.argtypes = [ctypes.POINTER(ctypes.c_int)]
    L.rt_tune_set_batch_split.argtypes = [ctypes.c_int]
    L.rt_tune_get_batch_split.argtypes = [ctypes.POINTER(ctypes.c_int)]
    for f in (L.rt_autotune, L.rt_tune_set, L.rt_tune_get, L.rt_tune_set_batch_mixed, L.rt_tune_get_batch_mixed,
              L.rt_tune_set_batch_split, L.rt_tune_get_batch_split):
        f.restype = ctypes.c_int
    return L


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def rt_autotune(n: int, reps: int = 50):
    best, us = ctypes.c_int(), ctypes.c_double()
    rt._check(_sig().rt_autotune(n, reps, ctypes.byref(best), ctypes.byref(us)), "rt_autotune")
    return best.value, us.value


def rt_autotune_concurrent(n: int, resonators: int = 2, bounces: int = 100, reps: int = 3):
    """Tile width and radix order for `resonators` n x n resonators stepped
    together, one stream each (rt_autotune_concurrent); recorded for this
    process.  Returns (col_tile, order, round trips/s)."""
    L = _sig()
    L.rt_autotune_concurrent.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                                              ctypes.POINTER(ctypes.c_double)]
    L.rt_autotune_concurrent.restype = ctypes.c_int
    tile, order, rate = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    rt._check(L.rt_autotune_concurrent(n, resonators, bounces, reps, ctypes.byref(tile), ctypes.byref(order),
                                       ctypes.byref(rate)), "rt_autotune_concurrent")
    return tile.value, order.value, rate.value


def rt_tune_set(n: int, col_tile: int):
    rt._check(_sig().rt_tune_set(n, col_tile), "rt_tune_set")


def rt_tune_get(n: int):
    c, tuned = ctypes.c_int(), ctypes.c_int()
    rt._check(_sig().rt_tune_get(n, ctypes.byref(c), ctypes.byref(tuned)), "rt_tune_get")
    return c.value, bool(tuned.value)


def rt_tune_set_order(n: int, order: int):
    rt._check(_sig().rt_tune_set_order(n, order), "rt_tune_set_order")


def rt_tune_get_order(n: int):
    """(radix order in use for side n, number of orders n offers)."""
    o, k = ctypes.c_int(), ctypes.c_int()
    rt._check(_sig().rt_tune_get_order(n, ctypes.byref(o), ctypes.byref(k)), "rt_tune_get_order")
    return o.value, k.value


def rt_tune_set_batch_mixed(mixed: bool):
    rt._check(_sig().rt_tune_set_batch_mixed(1 if mixed else 0), "rt_tune_set_batch_mixed")


def rt_tune_get_batch_mixed() -> bool:
    m = ctypes.c_int()
    rt._check(_sig().rt_tune_get_batch_mixed(ctypes.byref(m)), "rt_tune_get_batch_mixed")
    return bool(m.value)


def rt_tune_set_batch_split(parts: int):
    """Chains per size class of batch graphs captured from now on (0: about
    three chains in all; 1..8: that many per class)."""
    rt._check(_sig().rt_tune_set_batch_split(int(parts)), "rt_tune_set_batch_split")


def rt_tune_get_batch_split() -> int:
    m = ctypes.c_int()
    rt._check(_sig().rt_tune_get_batch_split(ctypes.byref(m)), "rt_tune_get_batch_split")
    return m.value


def autotune_batch(jobs, bounces: int = 100, splits=(1, 2, 3, 4), **batch_opts) -> dict:
    """Time `bounces` bounces of a batch of `jobs` in each launch form (one
    launch per sweep across sizes, or one per size class) with each number
    of graph chains per class in `splits` (all give the same fields), and
    keep the fastest pair for batches and servers created afterwards.
    Returns the pair chosen and every rate in round trips per second."""
    import time
    rates = {}
    for mixed in (False, True):
        rt_tune_set_batch_mixed(mixed)
        for parts in splits:
            rt_tune_set_batch_split(parts)
            with rt.Batch(jobs, chunk=bounces, **batch_opts) as b:
                b.step(bounces)
                b.sync()
                t0 = time.perf_counter()
                b.step(bounces)
                b.sync()
                rates[(mixed, parts)] = len(jobs) * bounces / (time.perf_counter() - t0)
    best = max(rates, key=rates.get)
    rt_tune_set_batch_mixed(best[0])
    rt_tune_set_batch_split(best[1])
    return {"mixed": best[0], "split": best[1],
            "round_trips_per_s": {("mixed" if m else "per_class") + f"_split{k}": r for (m, k), r in rates.items()}}


def autotune(sizes=(256, 512, 1024, 2048), reps: int = 50, cache: str | None = CACHE) -> dict:
    found = {}
    for n in sizes:
        tile, us = rt_autotune(n, reps)
        found[str(n)] = {"col_tile": tile, "col_order": rt_tune_get_order(n)[0], "us": us}
    if cache:
        data = {}
        if os.path.exists(cache):
            with open(cache) as f:
                data = json.load(f)
        data.setdefault(gpu_name(), {}).update(found)
        with open(cache, "w") as f:
            json.dump(data, f, indent=1)
    return found


def load(cache: str = CACHE) -> dict:
    if not os.path.exists(cache):
        return {}
    with open(cache) as f:
        entries = json.load(f).get(gpu_name(), {})
    for n, e in entries.items():
        rt_tune_set(int(n), int(e["col_tile"]))
        rt_tune_set_order(int(n), int(e.get("col_order", 0)))
    return entries
