"""Autotuning of the column-sweep tile width: rt_autotune picks a width that
fits and records it for later handles; results do not depend on the width
(each column's transform is the same arithmetic), and a cache round-trips."""
import json

import numpy as np
import pytest

from paper_1410_2855_gb300 import build, rt, tune, workloads as wl

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_valid_width_and_results_do_not_depend_on_it(tmp_path):
    build.build()
    best, us = tune.rt_autotune(512, reps=20)
    assert best in (2, 4, 8, 16) and us > 0
    assert tune.rt_tune_get(512) == (best, True)
    p = wl.Resonator(n=1024, fresnel=300.0, g0=0.25, T1=1000.0, R=0.95, seed=3)
    fields = []
    for c in (4, 8, 16):
        with rt.Resonator.from_params(p, col_tile=c, chunk=0) as r:
            r.set_field(wl.smooth_field(1024, 2, 1.0, dtype=np.complex64))
            r.step(5)
            fields.append(r.field())
    assert all(np.array_equal(f, fields[0]) for f in fields[1:])
    cache = tmp_path / "tune.json"
    found = tune.autotune(sizes=(256,), reps=10, cache=str(cache))
    data = json.loads(cache.read_text())
    assert data[tune.gpu_name()]["256"]["col_tile"] == found["256"]["col_tile"]
    tune.rt_tune_set(256, 0)
    assert tune.rt_tune_get(256)[1] is False
    assert tune.load(str(cache))["256"]["col_tile"] == found["256"]["col_tile"]
    assert tune.rt_tune_get(256) == (found["256"]["col_tile"], True)
    for n in (256, 512):
        tune.rt_tune_set(n, 0)
