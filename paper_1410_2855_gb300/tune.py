"""Autotuning of the column-sweep tile width, with a JSON cache on disk.

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
    for f in (L.rt_autotune, L.rt_tune_set, L.rt_tune_get):
        f.restype = ctypes.c_int
    return L


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def rt_autotune(n: int, reps: int = 50):
    best, us = ctypes.c_int(), ctypes.c_double()
    rt._check(_sig().rt_autotune(n, reps, ctypes.byref(best), ctypes.byref(us)), "rt_autotune")
    return best.value, us.value


def rt_tune_set(n: int, col_tile: int):
    rt._check(_sig().rt_tune_set(n, col_tile), "rt_tune_set")


def rt_tune_get(n: int):
    c, tuned = ctypes.c_int(), ctypes.c_int()
    rt._check(_sig().rt_tune_get(n, ctypes.byref(c), ctypes.byref(tuned)), "rt_tune_get")
    return c.value, bool(tuned.value)


def autotune(sizes=(256, 512, 1024, 2048), reps: int = 50, cache: str | None = CACHE) -> dict:
    found = {str(n): dict(zip(("col_tile", "us"), rt_autotune(n, reps))) for n in sizes}
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
    return entries
