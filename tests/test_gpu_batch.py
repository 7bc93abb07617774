"""Batched resonators (C ABI rt_batch_*): each slot of a mixed-size batch
evolves exactly as the same resonator on its own handle (same per-element
arithmetic, so bit-identical fields and inversions), bounce budgets stop
slots independently, and a slot matches the FP64 oracle."""
import numpy as np
import pytest

import oracle as orc
from paper_1410_2855_gb300 import build, rt, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    rt.lib()


MIX = [wl.Resonator(n=64, fresnel=30.0, g0=0.25, T1=500.0, R=0.95, seed=11),
       wl.Resonator(n=128, fresnel=50.0, g0=0.2, T1=800.0, R=0.9, seed=12),
       wl.Resonator(n=256, fresnel=200.0, g0=0.3, T1=1000.0, R=0.95, seed=13),
       wl.Resonator(n=128, fresnel=80.0, g0=0.15, T1=2000.0, R=0.95, seed=14),
       wl.Resonator(n=2048, fresnel=1000.0, g0=0.3, T1=1e4, R=0.9, seed=15)]


def test_batch_slots_match_single_handles_bit_for_bit():
    with rt.Batch(MIX, chunk=7, history_cap=64) as b:
        for i in range(len(MIX)):
            b.write_field(i, wl.smooth_field(MIX[i].n, 100 + i, 1.0, dtype=np.complex64))
        b.step(23)
        for i, p in enumerate(MIX):
            with rt.Resonator.from_params(p, chunk=0) as r:
                r.set_field(wl.smooth_field(p.n, 100 + i, 1.0, dtype=np.complex64))
                r.step(23)
                assert np.array_equal(b.field(i), r.field()), i
                assert np.array_equal(b.inversion(i), r.inversion()), i
                s, rs = b.stats(i), r.stats()
                assert s.bounces == 23
                assert abs(s.mean_intensity - rs.mean_intensity) <= 1e-12 * rs.mean_intensity
                assert np.allclose(b.history(i, 23), r.history(23), rtol=1e-12)


def test_class_split_across_graph_branches_keeps_every_slot_bit_identical():
    # Five resonators of one size: a captured batch graph runs them as three
    # branches of 2, 2 and 1 consecutive slots; with a second size class and
    # a remainder of direct launches (10 = 2 x 4 + 2 bounces).
    jobs = [wl.Resonator(n=128, fresnel=40.0 + 10 * k, g0=0.15 + 0.03 * k, T1=600.0 + 100 * k, R=0.9, seed=60 + k)
            for k in range(5)] + [wl.Resonator(n=64, fresnel=25.0, g0=0.2, T1=700.0, R=0.95, seed=66)]
    with rt.Batch(jobs, chunk=4, history_cap=16) as b:
        for i, p in enumerate(jobs):
            b.write_field(i, wl.smooth_field(p.n, 200 + i, 1.0, dtype=np.complex64))
        b.step(10)
        for i, p in enumerate(jobs):
            with rt.Resonator.from_params(p, chunk=0) as r:
                r.set_field(wl.smooth_field(p.n, 200 + i, 1.0, dtype=np.complex64))
                r.step(10)
                assert np.array_equal(b.field(i), r.field()), i
                assert np.array_equal(b.inversion(i), r.inversion()), i
                assert b.stats(i).bounces == 10
                assert np.allclose(b.history(i, 10), r.history(10), rtol=1e-12)


def test_bounce_budget_stops_a_slot_while_others_continue():
    with rt.Batch(MIX[:3], chunk=5) as b:
        b.step(4)
        job = wl.Resonator(n=128, fresnel=60.0, g0=0.28, T1=300.0, R=0.92, seed=99)
        b.set_job(1, job, 10)
        b.step(25)
        assert list(b.bounces()) == [29, 10, 29]
        with rt.Resonator.from_params(job, chunk=0) as r:
            r.step(10)
            assert np.array_equal(b.field(1), r.field())
        b.set_job(1, job, 0)          # idle slot
        b.step(3)
        assert list(b.bounces()) == [32, 0, 32]


def test_batch_slot_matches_oracle():
    p = wl.Resonator(n=256, fresnel=150.0, g0=0.25, T1=700.0, R=0.93, seed=5)
    E0 = wl.smooth_field(256, 8, 1.0, dtype=np.complex64)
    with rt.Batch([MIX[0], p, MIX[1]], chunk=0) as b:
        b.write_field(1, E0)
        b.step(20)
        E, N = b.field(1), b.inversion(1)
    op = orc.make_params(256, orc.alpha_from_fresnel(p.fresnel, p.d_over_w), p.g0, p.T1, p.R)
    oE, oN, _ = orc.run(op, E0.astype(np.complex128), orc.pump(op), 20, nthreads=4)
    assert np.linalg.norm(E - oE) / np.linalg.norm(oE) <= 1e-3
    assert np.linalg.norm(N - oN) / np.linalg.norm(oN) <= 1e-3


def test_parameter_sweep_batch_runs_and_stays_finite():
    jobs = wl.batch_sweep(count=24, sides=(256, 512, 1024))
    with rt.Batch(jobs, chunk=10, history_cap=16) as b:
        b.step(20)
        b.sync()
        assert all(x == 20 for x in b.bounces())
        assert b.footprint() > sum(12 * j.n * j.n for j in jobs)
        i = max(range(len(jobs)), key=lambda k: jobs[k].n)
        with rt.Resonator.from_params(jobs[i], chunk=0) as r:
            r.step(20)
            assert np.array_equal(b.field(i), r.field())
