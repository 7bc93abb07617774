"""Serving loop (C ABI rt_serve_*): continuous batching gives every request
the result it would get alone on its own handle (bit-identical final field:
the batched kernels do the same per-element arithmetic), requests of
different sizes and lengths share rounds and stop exactly at their own
bounce counts, and the device-memory budget bounds what is resident."""
import time

import numpy as np
import pytest

from paper_1410_2855_gb300 import build, rt, tune, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    rt.lib()


def alone(p, nb):
    with rt.Resonator.from_params(p, chunk=0) as h:
        h.step(nb)
        return h.field(), h.stats().mean_intensity


@pytest.fixture(params=[False, True], ids=["per_class", "mixed"])
def launch_form(request):
    tune.rt_tune_set_batch_mixed(request.param)
    yield request.param
    tune.rt_tune_set_batch_mixed(False)


def test_each_request_matches_its_run_alone(launch_form):
    # in every launch form (the classes are set up while the form is in force)
    reqs = [(wl.Resonator(n=64, fresnel=30.0, g0=0.25, T1=500.0, R=0.95, seed=21), 37),
            (wl.Resonator(n=128, fresnel=50.0, g0=0.2, T1=800.0, R=0.9, seed=22), 120),
            (wl.Resonator(n=256, fresnel=300.0, g0=0.3, T1=1000.0, R=0.95, seed=23), 75),
            (wl.Resonator(n=128, fresnel=90.0, g0=0.15, T1=2000.0, R=0.95, seed=24), 9),
            (wl.Resonator(n=512, fresnel=200.0, g0=0.22, T1=3000.0, R=0.93, seed=25), 51),
            (wl.Resonator(n=2048, fresnel=1000.0, g0=0.3, T1=1e4, R=0.9, seed=26), 23)]
    outs = [np.zeros((p.n, p.n), np.complex64) for p, _ in reqs]
    with rt.Server(chunk=16, budget_bytes=1 << 30) as srv:
        ids = [srv.submit(p, nb, o) for (p, nb), o in zip(reqs, outs)]
        srv.drain(300)
        got = {r.id: r for r in srv.poll()}
        st = srv.stats()
    assert st.done == len(reqs) and st.queued == 0 and st.running == 0
    for (p, nb), o, i in zip(reqs, outs, ids):
        r = got[i]
        assert r.status == 0 and r.bounces == nb and r.n == p.n
        assert r.submit_s <= r.admit_s <= r.finish_s
        ref, ref_mean = alone(p, nb)
        assert np.array_equal(o, ref), p.n
        assert abs(r.mean_intensity - ref_mean) <= 1e-12 * ref_mean


def test_budget_bounds_residency_and_queued_requests_finish():
    p = wl.Resonator(n=512, fresnel=200.0, g0=0.25, T1=1000.0, R=0.95, seed=7)
    slot = 512 * 512 * 12
    budget = int(2.6 * slot)             # two requests of this size at a time
    outs = [np.zeros((512, 512), np.complex64) for _ in range(6)]
    with rt.Server(chunk=10, budget_bytes=budget) as srv:
        ids = [srv.submit(p, 40, o) for o in outs]
        srv.drain(300)
        res = sorted(srv.poll(), key=lambda r: r.id)
        st = srv.stats()
    assert [r.id for r in res] == ids and all(r.status == 0 and r.bounces == 40 for r in res)
    # the server's own high-water mark of resident bytes, kept at every admission
    assert slot <= st.peak_resident_bytes <= budget
    assert 0 <= st.resident_bytes <= st.peak_resident_bytes
    # at most two requests are resident at any moment (checked at every admission)
    for r in res:
        live = sum(1 for q in res if q.admit_s <= r.admit_s < q.finish_s)
        assert live <= 2
    ref, _ = alone(p, 40)
    assert all(np.array_equal(o, ref) for o in outs)


def test_invalid_requests_are_rejected():
    with rt.Server(chunk=8, budget_bytes=1 << 24) as srv:     # 16 MiB: a 2048^2 request needs ~48 MiB
        ok = wl.Resonator(n=64, fresnel=30.0, g0=0.2, T1=100.0, R=0.95)
        for job, nb in [(wl.Resonator(n=4096, fresnel=30.0, g0=0.2, T1=100.0, R=0.95), 5),  # too large a grid
                        (ok, 0),                                                              # no bounces
                        (wl.Resonator(n=2048, fresnel=30.0, g0=0.2, T1=100.0, R=0.95), 5)]:  # over budget
            with pytest.raises(rt.RtError) as ei:
                srv.submit(job, nb)
            assert ei.value.status == rt.RT_EINVAL
        j = rt.job_from_params(ok)
        j.pump.order = 8.0                    # needs an N0 table: not served
        with pytest.raises(rt.RtError):
            srv.submit(j, 5)


def test_cancellation_of_queued_and_running_requests():
    # A long request is stopped after a round; a request still waiting for
    # room is dropped without running; the other request is unaffected.
    long = wl.Resonator(n=256, fresnel=150.0, g0=0.25, T1=900.0, R=0.93, seed=31)
    short = wl.Resonator(n=256, fresnel=150.0, g0=0.25, T1=900.0, R=0.93, seed=32)
    slot = 256 * 256 * 12
    out = np.zeros((256, 256), np.complex64)
    with rt.Server(chunk=20, budget_bytes=int(1.5 * slot)) as srv:   # one request resident at a time
        a = srv.submit(long, 10_000_000)
        b = srv.submit(short, 40, out)
        c = srv.submit(short, 40)
        t0 = time.time()
        while srv.stats().running == 0 and time.time() - t0 < 60:
            time.sleep(0.002)
        srv.cancel(c)                       # still queued behind a
        srv.cancel(a)                       # running
        with pytest.raises(rt.RtError):
            srv.cancel(987654)
        srv.drain(120)
        res = {r.id: r for r in srv.poll()}
        with pytest.raises(rt.RtError):
            srv.cancel(a)                   # already posted
    assert res[a].status == rt.RT_ECANCELED and 0 < res[a].bounces < 10_000_000
    assert res[c].status == rt.RT_ECANCELED and res[c].bounces == 0 and res[c].admit_s < 0
    assert res[b].status == 0 and res[b].bounces == 40
    ref, _ = alone(short, 40)
    assert np.array_equal(out, ref)


def test_shortest_first_policy_runs_short_requests_first_with_identical_results():
    # With a round budget of one 256^2 grid, only the request with the least
    # work left advances each round: the short request submitted after the
    # long one finishes first, and both results equal their runs alone.
    long = wl.Resonator(n=512, fresnel=150.0, g0=0.25, T1=900.0, R=0.93, seed=41)
    short = wl.Resonator(n=128, fresnel=60.0, g0=0.2, T1=500.0, R=0.95, seed=42)
    outs = [np.zeros((512, 512), np.complex64), np.zeros((128, 128), np.complex64)]
    with rt.Server(chunk=100, budget_bytes=1 << 28, policy=rt.RT_SERVE_SHORTEST_FIRST,
                   round_points=256 * 256) as srv:
        a = srv.submit(long, 60_000, outs[0])          # about a second of rounds
        t0 = time.time()
        while srv.stats().running == 0 and time.time() - t0 < 60:
            time.sleep(0.002)
        b = srv.submit(short, 300, outs[1])
        srv.drain(300)
        res = {r.id: r for r in srv.poll()}
    assert res[a].status == 0 and res[b].status == 0
    assert res[b].finish_s < res[a].finish_s
    for p, nb, o in ((long, 60_000, outs[0]), (short, 300, outs[1])):
        ref, _ = alone(p, nb)
        assert np.array_equal(o, ref)
