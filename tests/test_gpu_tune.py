"""Autotuning of the column sweep: rt_autotune picks a tile width and a radix
order that fit and records them for later handles.  Every choice it can make
is a correct transform: for each radix order (and tile width) the bounce map
matches the FP64 oracle at the parity tolerances after 1 and 20 bounces, the
tile width does not change a single bit for a given order, and the tuned
choices round-trip through the JSON cache.  The batch launch form (one launch
per sweep across sizes, or one per size class) does not change the fields
either."""
import json

import numpy as np
import pytest

import oracle as orc
from paper_1410_2855_gb300 import build, rt, tune, workloads as wl

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


@pytest.fixture(autouse=True)
def _clean():
    build.build()
    orc.build()
    yield
    for n in (128, 256, 512, 1024, 2048):
        tune.rt_tune_set(n, 0)
        tune.rt_tune_set_order(n, 0)
    tune.rt_tune_set_batch_mixed(False)


def test_autotune_picks_a_width_and_order_that_fit():
    best, us = tune.rt_autotune(512, reps=20)
    assert best in (2, 4, 8, 16) and us > 0
    assert tune.rt_tune_get(512) == (best, True)
    order, orders = tune.rt_tune_get_order(512)
    assert orders == 3 and 0 <= order < orders


def test_concurrent_autotune_records_a_pair_that_matches_the_oracle():
    n = 512
    tile, order, rate = tune.rt_autotune_concurrent(n, resonators=2, bounces=10, reps=1)
    assert tile in (2, 4, 8, 16) and 0 <= order < tune.rt_tune_get_order(n)[1] and rate > 0
    assert tune.rt_tune_get(n) == (tile, True) and tune.rt_tune_get_order(n)[0] == order
    # a handle created now runs the recorded pair and stays within the one-bounce bar
    p = wl.Resonator(n=n, fresnel=150.0, g0=0.25, T1=1000.0, R=0.95, seed=4)
    E0 = wl.smooth_field(n, 2, 1.0, dtype=np.complex64)
    q = orc.make_params(n, orc.alpha_from_fresnel(p.fresnel, p.d_over_w), p.g0, p.T1, p.R)
    o1, _, _ = orc.run(q, E0.astype(np.complex128), orc.pump(q), 1, nthreads=4, history=False)
    with rt.Resonator.from_params(p, chunk=0) as r:
        r.set_field(E0)
        r.step(1)
        assert rel(r.field(), o1) <= 1e-5


@pytest.mark.parametrize("n", [128, 512, 1024, 2048])
def test_every_radix_order_matches_the_oracle(n):
    p = wl.Resonator(n=n, fresnel=300.0 * n / 1024, g0=0.25, T1=1000.0, R=0.95, seed=3)
    E0 = wl.smooth_field(n, 2, 1.0, dtype=np.complex64)
    q = orc.make_params(n, orc.alpha_from_fresnel(p.fresnel, p.d_over_w), p.g0, p.T1, p.R)
    o1, _, _ = orc.run(q, E0.astype(np.complex128), orc.pump(q), 1, nthreads=4, history=False)
    o20, _, _ = orc.run(q, E0.astype(np.complex128), orc.pump(q), 20, nthreads=4, history=False)
    _, orders = tune.rt_tune_get_order(n)
    assert orders == (3 if n >= 512 else 2)
    runs = {}
    for order in range(orders):
        tune.rt_tune_set_order(n, order)
        for tile in (2, 4):
            tune.rt_tune_set(n, tile)
            with rt.Resonator.from_params(p, chunk=0) as r:
                r.set_field(E0)
                r.step(1)
                e1 = r.field()
                r.step(19)
                runs[(order, tile)] = (e1, r.field())
        assert np.array_equal(runs[(order, 2)][0], runs[(order, 4)][0])
        assert np.array_equal(runs[(order, 2)][1], runs[(order, 4)][1])
        assert rel(runs[(order, 4)][0], o1) <= 1e-5, (order, rel(runs[(order, 4)][0], o1))
        assert rel(runs[(order, 4)][1], o20) <= 1e-3, (order, rel(runs[(order, 4)][1], o20))


def test_a_tuned_order_gives_the_same_bits_in_handles_batch_slots_and_served_requests():
    p = wl.Resonator(n=1024, fresnel=400.0, g0=0.25, T1=900.0, R=0.93, seed=12)
    tune.rt_tune_set_order(1024, 2)
    with rt.Resonator.from_params(p, chunk=0) as r:
        r.step(9)
        ref = r.field()
    with rt.Batch([p, wl.Resonator(n=512, fresnel=200.0, g0=0.2, T1=500.0, R=0.95, seed=13)], chunk=4) as b:
        b.step(9)
        slot = b.field(0)
    out = np.zeros((1024, 1024), np.complex64)
    with rt.Server(chunk=4, budget_bytes=1 << 30) as srv:
        srv.submit(p, 9, out)
        srv.drain(120)
        assert srv.poll()[0].status == 0
    assert np.array_equal(slot, ref) and np.array_equal(out, ref)
    tune.rt_tune_set_order(1024, 0)
    with rt.Resonator.from_params(p, chunk=0) as r:
        r.step(9)
        assert not np.array_equal(r.field(), ref)     # a different order rounds differently
        assert rel(r.field(), ref.astype(np.complex128)) <= 1e-5


def test_tuned_choices_round_trip_through_the_cache(tmp_path):
    cache = tmp_path / "tune.json"
    found = tune.autotune(sizes=(256, 1024), reps=10, cache=str(cache))
    data = json.loads(cache.read_text())
    for n in ("256", "1024"):
        assert data[tune.gpu_name()][n]["col_tile"] == found[n]["col_tile"]
        assert data[tune.gpu_name()][n]["col_order"] == found[n]["col_order"]
    tune.rt_tune_set(256, 0)
    tune.rt_tune_set_order(1024, 0)
    assert tune.rt_tune_get(256)[1] is False
    loaded = tune.load(str(cache))
    assert tune.rt_tune_get(256) == (loaded["256"]["col_tile"], True)
    assert tune.rt_tune_get_order(1024)[0] == loaded["1024"]["col_order"]


def test_batch_launch_form_does_not_change_the_fields():
    # chunk 5 of 12 bounces: two chunks (graphs) and two bounces outside one
    jobs = [wl.Resonator(n=s, fresnel=150.0, g0=0.25, T1=800.0, R=0.93, seed=90 + j)
            for j, s in enumerate((128, 256, 512, 1024, 256, 2048, 64))]
    fields, means = {}, {}
    try:
        for mixed, parts in ((True, 0), (False, 0), (False, 1), (True, 4)):
            tune.rt_tune_set_batch_mixed(mixed)
            tune.rt_tune_set_batch_split(parts)
            assert tune.rt_tune_get_batch_mixed() is mixed and tune.rt_tune_get_batch_split() == parts
            with rt.Batch(jobs, chunk=5) as b:
                b.step(12)
                fields[(mixed, parts)] = [b.field(i) for i in range(len(jobs))]
                means[(mixed, parts)] = [b.stats(i).mean_intensity for i in range(len(jobs))]
                assert all(b.stats(i).bounces == 12 for i in range(len(jobs)))
    finally:
        tune.rt_tune_set_batch_split(0)
    ref = (False, 0)
    for key in fields:
        for a, c in zip(fields[key], fields[ref]):
            assert np.array_equal(a, c), key
        for a, c in zip(means[key], means[ref]):
            assert abs(a - c) <= 1e-12 * abs(c), key
