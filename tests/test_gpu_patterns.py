"""Structured starting fields (rt_set_field_pattern) on the GPU: the
library's generator against the oracle's, element by element, for every kind
(including the neighbourhood search the library uses for fine lattices), and
a Talbot-matched beam array as the start of a lasing run against the oracle."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1410_2855_gb300 import build, rt, workloads as wl

pytestmark = pytest.mark.gpu

FP32, FP64 = rt.RT_FP32, rt.RT_FP64


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    rt.lib()


PATTERNS = [  # (n, kwargs)
    (128, dict(kind=rt.RT_PATTERN_GAUSSIAN, width=0.15, envelope=0.4, curvature=7.5, amplitude=2.0)),
    (128, dict(kind=rt.RT_PATTERN_BEAM_ARRAY, width=0.04, periods=8)),
    (128, dict(kind=rt.RT_PATTERN_BEAM_ARRAY, width=0.05, periods=8, out_of_phase=True, envelope=0.6)),
    (128, dict(kind=rt.RT_PATTERN_VORTEX_ARRAY, width=0.06, periods=8, curvature=-3.0)),
    (128, dict(kind=rt.RT_PATTERN_VORTEX_ARRAY, width=0.06, periods=8, out_of_phase=True)),
    (256, dict(kind=rt.RT_PATTERN_BEAM_ARRAY, width=0.01, periods=32, out_of_phase=True)),   # neighbourhood path
    (256, dict(kind=rt.RT_PATTERN_VORTEX_ARRAY, width=0.012, periods=32)),
]


@pytest.mark.parametrize("precision", [FP32, FP64])
@pytest.mark.parametrize("case", PATTERNS, ids=lambda c: f"n{c[0]}-k{c[1]['kind']}-q{c[1].get('periods', 1)}")
def test_pattern_matches_oracle(precision, case):
    n, kw = case
    want = orc.pattern(n, kw["kind"], kw["width"], periods=kw.get("periods", 1),
                       out_of_phase=kw.get("out_of_phase", False), envelope=kw.get("envelope", 0.0),
                       curvature=kw.get("curvature", 0.0), amplitude=kw.get("amplitude", 1.0))
    with rt.Resonator(n, 50.0, 0.2, 500.0, 0.95, precision=precision, chunk=0) as r:
        r.set_pattern(**kw)
        got = r.field()
        assert r.stats().bounces == 0
    tol = 1e-13 if precision == FP64 else 2e-7
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


def test_talbot_matched_beam_array_lasing_run_matches_oracle():
    # Out-of-phase beam array whose period meets the Talbot condition:
    # alpha q^2 = 1 (half a Talbot length per bounce), D/W = 1.
    n, q = 256, 16
    fresnel = float(q * q)
    p = wl.Resonator(n=n, fresnel=fresnel, g0=0.3, T1=200.0, R=0.9, d_over_w=1.0, seed=91)
    with rt.Resonator.from_params(p, chunk=0) as r:
        r.set_pattern(rt.RT_PATTERN_BEAM_ARRAY, 0.02, periods=q, out_of_phase=True, envelope=0.5, amplitude=0.5)
        E0 = r.field()
        r.step(20)
        E20 = r.field()
    op = orc.make_params(n, 1.0 / fresnel, p.g0, p.T1, p.R, edge=p.edge)
    oE, _, _ = orc.run(op, E0.astype(np.complex128), orc.pump(op), 20, nthreads=4)
    assert np.linalg.norm(E20 - oE) / np.linalg.norm(oE) <= 1e-3


def test_invalid_patterns_are_rejected():
    with rt.Resonator(64, 50.0, 0.2, 500.0, 0.95, chunk=0) as r:
        for kw in (dict(kind=7, width=0.1), dict(kind=rt.RT_PATTERN_GAUSSIAN, width=0.0),
                   dict(kind=rt.RT_PATTERN_BEAM_ARRAY, width=0.1, periods=0),
                   dict(kind=rt.RT_PATTERN_VORTEX_ARRAY, width=0.1, periods=5, out_of_phase=True),
                   dict(kind=rt.RT_PATTERN_GAUSSIAN, width=0.1, envelope=-1.0)):
            with pytest.raises(rt.RtError):
                r.set_pattern(**kw)
