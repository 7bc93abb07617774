"""The 2048^2 benchmark workload in the launch configuration bench.py times
(two resonators on two concurrent streams, one CUDA graph per 500 bounces,
the autotuned column tile): its fields after 500 bounces are bit-identical to
the same resonators stepped by direct launches on one stream, and they keep
the properties the map guarantees at any size: a zero absorbing band, an
inversion between 0 and the pump peak g0, finite values, and the mean
intensity the library reports equal to the field's own."""
import numpy as np
import pytest
import torch

from paper_1410_2855_gb300 import build, rt, tune, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    rt.lib()


def test_bench_configuration_matches_direct_launches_and_keeps_invariants():
    B = 500
    tune.rt_autotune(2048, reps=10)
    streams = [torch.cuda.Stream() for _ in wl.C3]
    res = [rt.Resonator.from_params(p, chunk=B, cuda_stream=s.cuda_stream) for p, s in zip(wl.C3, streams)]
    for r in res:
        rt.rt_step(r.h, B)                       # both graphs in flight at once
    torch.cuda.synchronize()
    fields = [r.field() for r in res]
    invs = [r.inversion() for r in res]
    means = [r.stats().mean_intensity for r in res]
    for r in res:
        r.close()
    for p, E, N, mean in zip(wl.C3, fields, invs, means):
        with rt.Resonator.from_params(p, chunk=0) as d:
            d.step(B)
            assert np.array_equal(d.field(), E)
            assert np.array_equal(d.inversion(), N)
        e = p.edge
        assert np.all(E[:e] == 0) and np.all(E[-e:] == 0) and np.all(E[:, :e] == 0) and np.all(E[:, -e:] == 0)
        assert np.all(np.isfinite(E)) and np.all(np.isfinite(N))
        assert N.min() >= 0.0 and N.max() <= p.g0 * (1 + 1e-6)
        own = float(np.mean(np.abs(E.astype(np.complex128)) ** 2))
        assert abs(mean - own) <= 1e-6 * own


def test_largest_handle_grid_one_bounce_matches_oracle():
    # n = 4096, the largest grid a handle takes, one bounce from a lasing-scale field.
    import oracle as orc

    p = wl.Resonator(n=4096, fresnel=4000.0, g0=0.3, T1=1e4, R=0.9, seed=77)
    E0 = wl.smooth_field(4096, 5, 1.0, dtype=np.complex64)
    op = orc.make_params(4096, orc.alpha_from_fresnel(p.fresnel, p.d_over_w), p.g0, p.T1, p.R, edge=p.edge)
    with rt.Resonator.from_params(p, chunk=0) as r:
        r.set_field(E0)
        r.step(1)
        E1, N1 = r.field(), r.inversion()
    oE, oN, _ = orc.run(op, E0.astype(np.complex128), orc.pump(op), 1, nthreads=16)
    assert np.linalg.norm(E1 - oE) / np.linalg.norm(oE) <= 1e-5
    assert np.linalg.norm(N1 - oN) / np.linalg.norm(oN) <= 1e-5


@pytest.mark.parametrize("start", ["smooth", "noise"])
@pytest.mark.parametrize("precision, tol", [(rt.RT_FP32, 1e-5), (rt.RT_FP64, 1e-12)])
def test_passive_cavity_conserves_power_at_full_size(precision, tol, start):
    # No gain, R = 1, no absorbing edge, flat pump at zero: the map is the
    # unitary propagator alone, so the mean intensity after 200 bounces equals
    # the starting one up to rounding.  A property that holds at any size.
    # In FP32 the radix-16 rotation constants and the twiddle and propagator
    # tables lie within about 1e-8 of the unit circle, so the power may drift
    # by a few 1e-8 per bounce (1e-5 over 200 bounces allows 5e-8); with the
    # rounded (cos, sin) constants it lost about 2.7e-7 per bounce.
    n = 2048
    p = wl.Resonator(n=n, fresnel=1000.0, g0=0.0, T1=1e4, R=1.0, edge=0, seed=78)
    dt = np.complex128 if precision == rt.RT_FP64 else np.complex64
    with rt.Resonator.from_params(p, precision=precision, chunk=100) as r:
        if start == "smooth":
            r.set_field(wl.smooth_field(n, 6, 1.0, dtype=dt))
        E0 = r.field()
        p0 = float(np.mean(np.abs(E0.astype(np.complex128)) ** 2))
        r.step(0)                                  # a no-op
        assert r.stats().bounces == 0 and np.array_equal(r.field(), E0)
        r.step(200)
        hist = r.history(200)
    assert np.max(np.abs(hist / p0 - 1.0)) <= tol
