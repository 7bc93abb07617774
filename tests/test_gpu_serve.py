"""Serving loop (C ABI rt_serve_*): continuous batching gives every request
the result it would get alone on its own handle (bit-identical final field:
the batched kernels do the same per-element arithmetic), requests of
different sizes and lengths share rounds and stop exactly at their own
bounce counts, and the device-memory budget bounds what is resident."""
import time

import numpy as np
import pytest

from paper_1410_2855_gb300 import build, rt, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    rt.lib()


def alone(p, nb):
    with rt.Resonator.from_params(p, chunk=0) as h:
        h.step(nb)
        return h.field(), h.stats().mean_intensity


def test_each_request_matches_its_run_alone():
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
    peak = 0
    with rt.Server(chunk=10, budget_bytes=budget) as srv:
        ids = [srv.submit(p, 40, o) for o in outs]
        t0 = time.time()
        while srv.stats().done < 6 and time.time() - t0 < 300:
            peak = max(peak, srv.stats().resident_bytes)
            time.sleep(0.002)
        srv.drain(300)
        res = sorted(srv.poll(), key=lambda r: r.id)
    assert [r.id for r in res] == ids and all(r.status == 0 and r.bounces == 40 for r in res)
    assert 0 < peak <= budget
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
