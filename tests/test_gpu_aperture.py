"""Curved and rough mirror (the phase of the complex aperture, eq.
complex_aperture2) on the GPU: parity with the FP64 oracle element by element,
the oracle's closed-form lens-guide pin run through the CUDA path, batch slots
and served requests bit-identical to single handles, and the 2048^2 bench
resonators (flat and curved) against the oracle at full size.

Tolerances as for the flat mirror: FP32 relative L2 <= 1e-5 after one bounce
and <= 1e-3 after 20; FP64 <= 1e-12.
"""
import math

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


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


def oparams(p: wl.Resonator):
    return orc.make_params(p.n, orc.alpha_from_fresnel(p.fresnel, p.d_over_w), p.g0, p.T1, p.R, Isat=p.Isat,
                           edge=p.edge, pump_order=p.pump_order, pump_radius=p.pump_radius, z_over_F=p.z_over_F,
                           roughness=p.roughness())


# (resonator, what it exercises)
CASES = [
    wl.Resonator(n=64, fresnel=20.0, g0=0.2, T1=500.0, R=0.95, z_over_F=0.5, seed=31),            # lens
    wl.Resonator(n=128, fresnel=50.0, g0=0.25, T1=800.0, R=0.9, z_over_F=0.16, roughness_rms=0.3,
                 seed=32),                                                                          # lens + roughness
    wl.Resonator(n=256, fresnel=200.0, g0=0.3, T1=1000.0, R=0.95, z_over_F=-0.2, seed=33),         # diverging
    wl.Resonator(n=512, fresnel=300.0, g0=0.2, T1=3000.0, R=0.93, roughness_rms=1.0,
                 roughness_corr=0.02, seed=34),                                                     # roughness only
]


@pytest.mark.parametrize("precision", [FP32, FP64])
@pytest.mark.parametrize("p", CASES, ids=lambda p: f"n{p.n}")
def test_one_and_twenty_bounces_match_oracle(precision, p):
    dt = np.complex128 if precision == FP64 else np.complex64
    E0 = wl.smooth_field(p.n, p.seed, 1.0, dtype=dt)
    op = oparams(p)
    with rt.Resonator.from_params(p, precision=precision, chunk=0) as r:
        r.set_field(E0)
        r.step(1)
        E1, N1 = r.field(), r.inversion()
        r.step(19)
        E20, N20 = r.field(), r.inversion()
    oE1, oN1, _ = orc.run(op, E0.astype(np.complex128), orc.pump(op), 1, nthreads=4)
    oE20, oN20, _ = orc.run(op, oE1, oN1, 19, nthreads=4)
    assert rel_l2(E1, oE1) <= TOL1[precision]
    assert float(np.linalg.norm(N1 - oN1) / np.linalg.norm(oN1)) <= TOL1[precision]
    assert rel_l2(E20, oE20) <= TOL20[precision]
    assert float(np.linalg.norm(N20 - oN20) / np.linalg.norm(oN20)) <= TOL20[precision]


@pytest.mark.parametrize("precision", [FP32, FP64])
@pytest.mark.parametrize("u", [0.16, 1.0, 3.0])
def test_lens_guide_eigenmode_returns_with_the_gouy_phase(precision, u):
    # The oracle pin run through the library: the Gaussian eigenmode of the
    # flat/curved-mirror cavity comes back each bounce times
    # exp(-i arccos(1 - z/2F)) (Kogelnik & Li).
    n, beta = 128, min(0.008, 0.01 * u * math.sqrt(4.0 / u - 1.0) / 2.0)
    alpha = math.pi * beta / 2.0
    s = 1j * beta * complex(-0.5, -math.sqrt(4.0 / u - 1.0) / 2.0)
    x = (np.arange(n) - n // 2) / (n // 2)
    E0 = np.exp(-(x[None, :] ** 2 + x[:, None] ** 2) / (2.0 * s))
    theta = math.acos(1.0 - u / 2.0)
    # fresnel from alpha with D/W = 0.8: alpha = 0.64 / N_F
    with rt.Resonator(n, 0.64 / alpha, 0.0, 1e9, 1.0, precision=precision, edge_px=0, pump_kind=rt.RT_PUMP_UNIFORM,
                      z_over_F=u, chunk=0) as r:
        r.set_field(E0)
        r.step(5)
        E5 = r.field()
    tol = 1e-11 if precision == FP64 else 2e-5
    assert np.max(np.abs(E5 - np.exp(-5j * theta) * E0)) < tol


def test_batch_slots_with_mirrors_match_single_handles_bit_for_bit():
    mix = [CASES[0], wl.Resonator(n=64, fresnel=25.0, g0=0.2, T1=400.0, R=0.95, seed=40), CASES[1], CASES[2],
           wl.Resonator(n=2048, fresnel=1000.0, g0=0.3, T1=1e4, R=0.9, z_over_F=0.16, roughness_rms=0.05,
                        seed=41)]
    with rt.Batch(mix, chunk=4, history_cap=16) as b:
        for i, p in enumerate(mix):
            b.write_field(i, wl.smooth_field(p.n, 200 + i, 1.0, dtype=np.complex64))
        b.step(9)
        for i, p in enumerate(mix):
            with rt.Resonator.from_params(p, chunk=0) as r:
                r.set_field(wl.smooth_field(p.n, 200 + i, 1.0, dtype=np.complex64))
                r.step(9)
                assert np.array_equal(b.field(i), r.field()), i
                assert np.array_equal(b.inversion(i), r.inversion()), i
        # A rough job needs a slot created with a roughness table.
        with pytest.raises(rt.RtError):
            b.set_job(1, wl.Resonator(n=64, fresnel=25.0, g0=0.2, T1=400.0, R=0.95, roughness_rms=0.1), 3)
        b.set_job(1, CASES[0], 3)     # a lens needs nothing extra
        b.step(3)
        with rt.Resonator.from_params(CASES[0], chunk=0) as r:
            r.step(3)
            assert np.array_equal(b.field(1), r.field())


def test_served_curved_mirror_request_matches_its_run_alone():
    p = wl.Resonator(n=256, fresnel=150.0, g0=0.25, T1=900.0, R=0.93, z_over_F=0.3, seed=51)
    out = np.zeros((p.n, p.n), np.complex64)
    with rt.Server(chunk=8, budget_bytes=1 << 28) as srv:
        i = srv.submit(p, 21, out)
        srv.drain(120)
        r = {x.id: x for x in srv.poll()}[i]
        assert r.status == 0 and r.bounces == 21
        with pytest.raises(rt.RtError):
            srv.submit(wl.Resonator(n=256, fresnel=150.0, g0=0.25, T1=900.0, R=0.93, roughness_rms=0.1), 5)
    with rt.Resonator.from_params(p, chunk=0) as h:
        h.step(21)
        assert np.array_equal(out, h.field())


@pytest.mark.parametrize("p", [wl.C3[0], wl.C3[1], wl.CURVED], ids=["2048-g0.1", "2048-g0.3", "2048-curved"])
def test_full_size_2048_bounce_matches_oracle(p):
    # The bench resonators at full size, in the bench's launch configuration
    # (library noise start, graph chunk of 500, autotuned-or-built-in column
    # tile), one bounce from a lasing-scale field and from the library noise.
    op = oparams(p)
    E0 = wl.smooth_field(p.n, p.seed, 1.0, dtype=np.complex64)
    with rt.Resonator.from_params(p, chunk=500) as r:
        noise = r.field()
        r.step(1)
        En = r.field()
        r.set_field(E0)
        r.set_inversion(orc.pump(op).astype(np.float32))
        r.step(1)
        E1, N1 = r.field(), r.inversion()
    oE, oN, _ = orc.run(op, E0.astype(np.complex128), orc.pump(op), 1, nthreads=16)
    assert rel_l2(E1, oE) <= TOL1[FP32]
    assert float(np.linalg.norm(N1 - oN) / np.linalg.norm(oN)) <= TOL1[FP32]
    oEn, _, _ = orc.run(op, noise.astype(np.complex128), orc.pump(op), 1, nthreads=16)
    assert rel_l2(En, oEn) <= TOL1[FP32]
