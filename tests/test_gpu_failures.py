"""Failure paths on the GPU, provoked on the host (nothing faults, traps or
hangs the device): an injected allocation failure at every allocation of a
handle's and a batch's set-up returns RT_ENOMEM and releases what was
allocated; a resonator whose gain diverges reports RT_ENUMERIC from its
device error word and stays usable for reads; the serving loop admits a
request once a failed allocation is retried, and posts RT_ENOMEM for a
request that cannot be placed even with nothing else resident; the sweeps'
bounded copy waits give up on a copy that never completes and report
RT_ETIMEOUT, and the context stays usable."""
import time

import numpy as np
import pytest
import torch

from paper_1410_2855_gb300 import build, rt, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    rt.lib()
    yield
    rt.rt_debug_fail_alloc(-1)


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_injected_allocation_failures_return_enomem_and_release_everything():
    p = wl.Resonator(n=512, fresnel=100.0, g0=0.2, T1=500.0, R=0.95, z_over_F=0.2, roughness_rms=0.1, seed=5)
    with rt.Resonator.from_params(p) as warm:      # first use: context and module set-up
        warm.step(1)
    base = free_bytes()
    failures = 0
    for k in range(64):
        rt.rt_debug_fail_alloc(k)
        try:
            r = rt.Resonator.from_params(p, slices=2)
        except rt.RtError as e:
            assert e.status == rt.RT_ENOMEM
            failures += 1
            continue
        rt.rt_debug_fail_alloc(-1)
        r.step(3)
        r.sync()
        r.close()
        break
    else:
        pytest.fail("creation never succeeded")
    assert failures >= 10                           # every allocation of the set-up was hit once
    assert abs(free_bytes() - base) < (8 << 20)    # nothing leaked (allocator granularity aside)


def test_injected_allocation_failure_in_batch_creation():
    jobs = [wl.Resonator(n=128, fresnel=50.0, g0=0.2, T1=800.0, R=0.9, seed=s) for s in range(4)]
    for k in (0, 3, 6):
        rt.rt_debug_fail_alloc(k)
        with pytest.raises(rt.RtError) as ei:
            rt.Batch(jobs)
        assert ei.value.status == rt.RT_ENOMEM
    rt.rt_debug_fail_alloc(-1)
    with rt.Batch(jobs, chunk=0) as b:
        b.step(2)
        assert list(b.bounces()) == [2, 2, 2, 2]


def test_served_request_is_admitted_after_a_failed_allocation():
    p = wl.Resonator(n=128, fresnel=50.0, g0=0.2, T1=800.0, R=0.9, seed=9)
    out = np.zeros((128, 128), np.complex64)
    with rt.Server(chunk=8, budget_bytes=1 << 26) as srv:
        rt.rt_debug_fail_alloc(0)              # the slot allocation of the first admission fails
        i = srv.submit(p, 12, out)
        srv.drain(120)
        r = {x.id: x for x in srv.poll()}[i]
        assert r.status == 0 and r.bounces == 12
    rt.rt_debug_fail_alloc(-1)
    with rt.Resonator.from_params(p, chunk=0) as h:
        h.step(12)
        assert np.array_equal(out, h.field())


def test_served_request_that_cannot_be_placed_fails_instead_of_waiting():
    # Every allocation fails: with nothing else resident no later round could
    # make room, so the request's result is posted at once with RT_ENOMEM
    # (and drain returns) instead of the request waiting for ever.  The server
    # keeps working once allocations succeed again.
    p = wl.Resonator(n=128, fresnel=50.0, g0=0.2, T1=800.0, R=0.9, seed=10)
    out = np.zeros((128, 128), np.complex64)
    with rt.Server(chunk=8, budget_bytes=1 << 26) as srv:
        rt.rt_debug_fail_alloc_n(0, -1)
        try:
            i = srv.submit(p, 12, out)
            srv.drain(60)
            r = {x.id: x for x in srv.poll()}[i]
        finally:
            rt.rt_debug_fail_alloc_n(-1, 0)
        assert r.status == rt.RT_ENOMEM and r.bounces == 0 and r.admit_s < 0
        assert not out.any()
        j = srv.submit(p, 12, out)
        srv.drain(120)
        r = {x.id: x for x in srv.poll()}[j]
        assert r.status == 0 and r.bounces == 12
    with rt.Resonator.from_params(p, chunk=0) as h:
        h.step(12)
        assert np.array_equal(out, h.field())


def test_divergent_gain_reports_a_numeric_error():
    # g0 = 60 per pass with no saturation to speak of: |E|^2 grows by e^60
    # per bounce and overflows FP32 within a few bounces.
    with rt.Resonator(64, 20.0, 60.0, 1e6, 1.0, Isat=1e30, edge_px=0, noise_amp=1.0, chunk=0) as r:
        r.step(6)
        with pytest.raises(rt.RtError) as ei:
            r.sync()
        assert ei.value.status == rt.RT_ENUMERIC
        assert r.stats().last_error == rt.RT_ENUMERIC


@pytest.mark.parametrize("drain", [False, True])
def test_copy_waits_are_bounded_and_the_context_survives(drain):
    # a stage barrier armed for bytes that no copy delivers: the sweeps' own
    # wait gives up after its limit (and, with drain, so does the wait for
    # the next stage) and records RT_ETIMEOUT; nothing faults or hangs
    t0 = time.perf_counter()
    assert rt.rt_debug_wait_probe(drain) == rt.RT_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    p = wl.Resonator(n=128, fresnel=60.0, g0=0.2, T1=500.0, R=0.9, seed=5)
    with rt.Resonator.from_params(p, chunk=0) as h:
        h.step(3)
        assert h.stats().bounces == 3 and np.isfinite(h.stats().mean_intensity)
