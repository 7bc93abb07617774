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
