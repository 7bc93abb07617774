"""Smooth aperture taper and the exact (exponential) inversion update on the
GPU: parity with the FP64 oracle element by element (FP32 <= 1e-5 after one
bounce and <= 1e-3 after 20; FP64 <= 1e-12), alone and combined with a curved
mirror and a sliced gain medium, and batch slots bit-identical to single
handles."""
import numpy as np
import pytest

import oracle as orc
from paper_1410_2855_gb300 import build, rt, workloads as wl

pytestmark = pytest.mark.gpu

FP32, FP64 = rt.RT_FP32, rt.RT_FP64
TOL1 = {FP32: 1e-5, FP64: 1e-12}
TOL20 = {FP32: 1e-3, FP64: 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    rt.lib()


def rel(a, b):
    a = np.asarray(a, np.complex128 if np.iscomplexobj(a) else np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [  # (resonator, slices)
    (wl.Resonator(n=128, fresnel=30.0, g0=0.3, T1=60.0, R=0.9, taper_px=6, seed=81), 1),
    (wl.Resonator(n=256, fresnel=150.0, g0=0.25, T1=40.0, R=0.93, relax=1, seed=82), 1),
    (wl.Resonator(n=256, fresnel=150.0, g0=0.25, T1=50.0, R=0.93, taper_px=10, relax=1, z_over_F=0.2,
                  seed=83), 1),
    (wl.Resonator(n=128, fresnel=40.0, g0=0.3, T1=30.0, R=0.9, taper_px=4, relax=1, seed=84), 3),
]


@pytest.mark.parametrize("precision", [FP32, FP64])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0].n}-w{c[0].taper_px}-x{c[0].relax}-m{c[1]}")
def test_bounces_match_oracle(precision, case):
    p, m = case
    dt = np.complex128 if precision == FP64 else np.complex64
    E0 = wl.smooth_field(p.n, p.seed, 1.0, dtype=dt)
    op = orc.make_params(p.n, orc.alpha_from_fresnel(p.fresnel, p.d_over_w), p.g0, p.T1, p.R, edge=p.edge,
                         z_over_F=p.z_over_F, slices=m, taper=p.taper_px, relax=p.relax)
    with rt.Resonator.from_params(p, precision=precision, chunk=0, slices=m) as r:
        r.set_field(E0)
        r.step(1)
        E1, N1 = r.field(), r.inversion()
        r.step(19)
        E20, N20 = r.field(), r.inversion()
    oE1, oN1, _ = orc.run(op, E0.astype(np.complex128), orc.initial_inversion(op), 1, nthreads=4)
    oE20, oN20, _ = orc.run(op, oE1, oN1, 19, nthreads=4)
    assert rel(E1, oE1) <= TOL1[precision]
    assert rel(N1, oN1) <= TOL1[precision]
    assert rel(E20, oE20) <= TOL20[precision]
    assert rel(N20, oN20) <= TOL20[precision]


def test_batch_slots_with_taper_and_exact_relaxation_match_handles():
    mix = [CASES[0][0], CASES[1][0], CASES[2][0],
           wl.Resonator(n=64, fresnel=25.0, g0=0.2, T1=400.0, R=0.95, seed=85)]
    with rt.Batch(mix, chunk=3, history_cap=8) as b:
        for i, p in enumerate(mix):
            b.write_field(i, wl.smooth_field(p.n, 300 + i, 1.0, dtype=np.complex64))
        b.step(7)
        for i, p in enumerate(mix):
            with rt.Resonator.from_params(p, chunk=0) as r:
                r.set_field(wl.smooth_field(p.n, 300 + i, 1.0, dtype=np.complex64))
                r.step(7)
                assert np.array_equal(b.field(i), r.field()), i
                assert np.array_equal(b.inversion(i), r.inversion()), i
