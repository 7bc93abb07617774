"""Multi-slice gain medium (opts.slices = m): a bounce is m steps of
diffraction over z/m, each followed by a thin gain slice with its own
inversion and a pump of N0/m; the mirror acts after the last slice.  Parity
with the FP64 oracle element by element (FP32 <= 1e-5 after one bounce and
<= 1e-3 after 20; FP64 <= 1e-12), graphs vs direct launches bit-identical,
and the slice-major inversion layout of the readout."""
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
    (wl.Resonator(n=128, fresnel=30.0, g0=0.3, T1=500.0, R=0.9, seed=71), 3),
    (wl.Resonator(n=256, fresnel=150.0, g0=0.25, T1=800.0, R=0.93, z_over_F=0.2, seed=72), 4),
    (wl.Resonator(n=512, fresnel=300.0, g0=0.2, T1=2000.0, R=0.95, seed=73), 2),
]


@pytest.mark.parametrize("precision", [FP32, FP64])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0].n}-m{c[1]}")
def test_sliced_bounces_match_oracle(precision, case):
    p, m = case
    dt = np.complex128 if precision == FP64 else np.complex64
    E0 = wl.smooth_field(p.n, p.seed, 1.0, dtype=dt)
    op = orc.make_params(p.n, orc.alpha_from_fresnel(p.fresnel, p.d_over_w), p.g0, p.T1, p.R, edge=p.edge,
                         z_over_F=p.z_over_F, slices=m)
    with rt.Resonator.from_params(p, precision=precision, chunk=0, slices=m) as r:
        N0 = r.inversion()
        assert N0.shape == (m, p.n, p.n)
        assert rel(N0, orc.initial_inversion(op)) <= TOL1[precision]
        r.set_field(E0)
        r.step(1)
        E1, N1 = r.field(), r.inversion()
        r.step(19)
        E20, N20 = r.field(), r.inversion()
        assert r.stats().bounces == 20
    oE1, oN1, _ = orc.run(op, E0.astype(np.complex128), orc.initial_inversion(op), 1, nthreads=4)
    oE20, oN20, _ = orc.run(op, oE1, oN1, 19, nthreads=4)
    assert rel(E1, oE1) <= TOL1[precision]
    assert rel(N1, oN1) <= TOL1[precision]
    assert rel(E20, oE20) <= TOL20[precision]
    assert rel(N20, oN20) <= TOL20[precision]


def test_sliced_graphs_match_direct_launches_and_inversion_round_trips():
    p, m = CASES[0]
    with rt.Resonator.from_params(p, chunk=4, slices=m) as g, rt.Resonator.from_params(p, chunk=0, slices=m) as d:
        g.step(11)
        d.step(11)
        assert np.array_equal(g.field(), d.field())
        assert np.array_equal(g.inversion(), d.inversion())
        N = d.inversion()
        N[1] *= 0.5
        d.set_inversion(N)
        assert np.array_equal(d.inversion(), N)
        with pytest.raises(rt.RtError):
            rt.rt_sweep(d.h, rt.RT_SWEEP_ROWS)          # sweeps are per single-slice bounce
        with pytest.raises(rt.RtError):
            rt.rt_read_inversion(d.h, np.empty((p.n, p.n), np.float32))


def test_one_slice_is_the_default_map():
    p = CASES[0][0]
    with rt.Resonator.from_params(p, chunk=0, slices=1) as a, rt.Resonator.from_params(p, chunk=0) as b:
        a.step(5)
        b.step(5)
        assert np.array_equal(a.field(), b.field())
        assert np.array_equal(a.inversion(), b.inversion())
