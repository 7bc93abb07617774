"""Intracavity-plane readout (rt_read_field_at): the field diffracted a
further zeta * z from the mirror plane, element by element against the
oracle's diffraction, and the fractional Talbot images between the mirrors
(z_T/4 closed form, z_T/2 half-period shift, z_T self-image) through the CUDA
path.  The handle's own state is left unchanged."""
import numpy as np
import pytest

import oracle as orc
from paper_1410_2855_gb300 import build, rt, workloads as wl

pytestmark = pytest.mark.gpu

FP32, FP64 = rt.RT_FP32, rt.RT_FP64
TOL = {FP32: 1e-5, FP64: 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    rt.lib()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", [FP32, FP64])
@pytest.mark.parametrize("n, fresnel", [(64, 20.0), (256, 200.0), (1024, 500.0)])
def test_field_at_matches_oracle_diffraction(precision, n, fresnel):
    p = wl.Resonator(n=n, fresnel=fresnel, g0=0.25, T1=800.0, R=0.93, seed=61)
    dt = np.complex128 if precision == FP64 else np.complex64
    with rt.Resonator.from_params(p, precision=precision, chunk=0) as r:
        r.set_field(wl.smooth_field(n, 62, 1.0, dtype=dt))
        r.step(3)
        E = r.field()
        alpha = orc.alpha_from_fresnel(fresnel, p.d_over_w)
        for zeta in (0.25, 1.0, -0.5, 3.7):
            got = r.field_at(zeta)
            assert rel_l2(got, orc.diffract(E.astype(np.complex128), alpha * zeta)) <= TOL[precision], zeta
        assert np.array_equal(r.field(), E)          # state untouched
        assert r.stats().bounces == 3


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_fractional_talbot_planes(precision):
    q, n = 8, 256
    rng = np.random.default_rng(9)
    pp = n // q
    block = rng.standard_normal((pp, pp)) + 1j * rng.standard_normal((pp, pp))
    E = np.tile(block, (q, q))
    h = pp // 2
    a, b = (1 - 1j) / 2, (1 + 1j) / 2
    quarter = (a * a * E + a * b * (np.roll(E, h, axis=1) + np.roll(E, h, axis=0))
               + b * b * np.roll(E, (h, h), axis=(0, 1)))
    # D/W = 1 and N_F = q^2: alpha = 1/q^2, one bounce is half a Talbot length.
    with rt.Resonator(n, float(q * q), 0.0, 10.0, 1.0, precision=precision, edge_px=0, pump_diam_over_window=1.0,
                      chunk=0) as r:
        r.set_field(E)
        assert rel_l2(r.field_at(0.5), quarter) <= TOL[precision]
        assert rel_l2(r.field_at(1.0), np.roll(E, (h, h), axis=(0, 1))) <= TOL[precision]
        assert rel_l2(r.field_at(2.0), E) <= TOL[precision]
        assert rel_l2(r.field_at(0.0), E) <= TOL[precision]


def test_field_at_rejects_bad_arguments():
    with rt.Resonator(64, 20.0, 0.2, 100.0, 0.95, chunk=0) as r:
        with pytest.raises(rt.RtError):
            rt.rt_read_field_at(r.h, float("nan"), np.empty((64, 64), np.complex64))
        with pytest.raises(rt.RtError):
            rt.rt_read_field_at(r.h, 0.5, np.empty((64, 32), np.complex64))
