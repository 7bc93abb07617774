"""Parity of the CUDA bounce map (through the C ABI) with the FP64 oracle,
element by element on seeded inputs, plus the oracle's closed-form pins run
through the GPU path.

Tolerances (relative L2 over the grid): FP32 fused path <= 1e-5 after one
bounce and <= 1e-3 after 20; FP64 plain path <= 1e-12 after one and 20
bounces.
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


def oparams(n, fresnel, g0, T1, R, edge=8, Isat=1.0, d_over_w=0.8, pump_kind=orc.PUMP_SUPERGAUSS,
            order=10.0, radius=0.8):
    return orc.make_params(n, orc.alpha_from_fresnel(fresnel, d_over_w), g0, T1, R, Isat=Isat, edge=edge,
                           pump_kind=pump_kind, pump_order=order, pump_radius=radius)


def gpu(n, fresnel, g0, T1, R, precision, edge=8, d_over_w=0.8, **kw):
    return rt.Resonator(n, fresnel, g0, T1, R, precision=precision, edge_px=edge,
                        pump_diam_over_window=d_over_w, **kw)


def start_field(kind, n, precision, seed):
    dt = np.complex128 if precision == FP64 else np.complex64
    if kind == "noise":
        return wl.noise_field(n, seed, 1e-6, dt)
    return wl.smooth_field(n, seed, 1.0, dtype=dt)


CASES = [  # (n, fresnel, g0, T1, R)
    (32, 20.0, 0.2, 2000.0, 0.95),
    (64, 20.0, 0.2, 2000.0, 0.95),
    (128, 20.0, 0.2, 2000.0, 0.95),
    (256, 100.0, 0.3, 1000.0, 0.9),
    (512, 100.0, 0.15, 5000.0, 0.95),
    (1024, 300.0, 0.25, 3000.0, 0.95),
]


@pytest.mark.parametrize("precision", [FP32, FP64])
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("kind", ["noise", "lasing"])
def test_one_bounce_matches_oracle(precision, case, kind):
    n, fres, g0, T1, R = case
    E0 = start_field(kind, n, precision, 7 + n)
    with gpu(n, fres, g0, T1, R, precision) as r:
        r.set_field(E0)
        r.step(1)
        E1, N1 = r.field(), r.inversion()
    p = oparams(n, fres, g0, T1, R)
    oE, oN, _ = orc.run(p, E0.astype(np.complex128), orc.pump(p), 1)
    assert rel_l2(E1, oE) <= TOL1[precision]
    assert float(np.linalg.norm(N1 - oN) / np.linalg.norm(oN)) <= TOL1[precision]


EXTREMES = [  # (label, n, fresnel, g0, T1, R, edge, Isat, bounces)
    ("T1=1", 64, 20.0, 0.3, 1.0, 0.9, 8, 1.0, 2),                 # the inversion follows the intensity at once
    ("edge=n/2", 64, 20.0, 0.3, 500.0, 0.9, 32, 1.0, 2),          # every pixel absorbed
    ("edge=0", 64, 20.0, 0.3, 500.0, 0.9, 0, 1.0, 3),
    ("Isat=1e-6", 64, 20.0, 0.3, 1000.0, 0.9, 8, 1e-6, 1),        # deep saturation: N is driven far negative
    ("Isat=1e30", 64, 20.0, 0.5, 1000.0, 0.95, 8, 1e30, 3),       # no saturation
    ("NF=0.5", 128, 0.5, 0.2, 1000.0, 0.95, 8, 1.0, 3),           # alpha m^2 up to 5e3: phase wraps thousands of times
    ("NF=1e5", 128, 1e5, 0.2, 1000.0, 0.95, 8, 1.0, 3),           # almost no diffraction
    ("R=1e-6", 64, 20.0, 0.2, 1000.0, 1e-6, 8, 1.0, 2),           # the mirror takes 1e-3 of the amplitude
]


@pytest.mark.parametrize("precision", [FP32, FP64])
@pytest.mark.parametrize("case", EXTREMES, ids=[c[0] for c in EXTREMES])
def test_parameter_extremes_match_oracle(precision, case):
    # The ends of the ranges the library accepts (T1 >= 1, 0 < R <= 1,
    # 0 <= edge <= n/2, any Isat and Fresnel number > 0), a lasing-scale
    # start, a few bounces: same bars as one bounce, scaled by the bounces.
    _, n, fres, g0, T1, R, edge, Isat, nb = case
    E0 = start_field("lasing", n, precision, 31 + n)
    with gpu(n, fres, g0, T1, R, precision, edge=edge, Isat=Isat) as r:
        r.set_field(E0)
        r.step(nb)
        E1, N1 = r.field(), r.inversion()
    p = oparams(n, fres, g0, T1, R, edge=edge, Isat=Isat)
    oE, oN, _ = orc.run(p, E0.astype(np.complex128), orc.pump(p), nb)
    if edge == n // 2:
        assert not np.any(E1) and not np.any(oE)        # exactly zero, as the oracle
    else:
        assert rel_l2(E1, oE) <= TOL1[precision] * nb
    assert float(np.linalg.norm(N1 - oN) / np.linalg.norm(oN)) <= TOL1[precision] * nb


@pytest.mark.parametrize("precision", [FP32, FP64])
@pytest.mark.parametrize("pump", ["array", "order4", "uniform"])
def test_pump_forms_match_oracle(precision, pump):
    # The N0-table path (an array pump, a super-Gaussian of order other than
    # 10) and the uniform pump, after 1 and 20 bounces.
    n, fres, g0, T1, R = 128, 50.0, 0.3, 500.0, 0.9
    prof = np.random.default_rng(17).uniform(0.0, 1.0, size=(n, n))
    kw = {"array": dict(pump_kind=rt.RT_PUMP_ARRAY, pump_profile=prof),
          "order4": dict(pump_order=4.0, pump_radius=0.6),
          "uniform": dict(pump_kind=rt.RT_PUMP_UNIFORM)}[pump]
    okw = {"array": dict(pump_kind=orc.PUMP_ARRAY, pump_profile=prof),
           "order4": dict(pump_order=4.0, pump_radius=0.6),
           "uniform": dict(pump_kind=orc.PUMP_UNIFORM)}[pump]
    op = orc.make_params(n, orc.alpha_from_fresnel(fres, 0.8), g0, T1, R, **okw)
    E0 = start_field("lasing", n, precision, 41)
    with gpu(n, fres, g0, T1, R, precision, **kw) as r:
        assert np.allclose(r.inversion(), orc.pump(op), rtol=1e-6, atol=1e-12)   # N starts at N0
        r.set_field(E0)
        r.step(20)
        E20, N20 = r.field(), r.inversion()
    E1o, N1o, _ = orc.run(op, E0.astype(np.complex128), orc.pump(op), 1)
    E20o, N20o, _ = orc.run(op, E1o, N1o, 19)
    assert rel_l2(E20, E20o) <= TOL20[precision]
    assert float(np.linalg.norm(N20 - N20o) / np.linalg.norm(N20o)) <= TOL20[precision]
    with gpu(n, fres, g0, T1, R, precision, **kw) as r:
        r.set_field(E0)
        r.step(1)
        assert rel_l2(r.field(), E1o) <= TOL1[precision]
        assert float(np.linalg.norm(r.inversion() - N1o) / np.linalg.norm(N1o)) <= TOL1[precision]


@pytest.mark.parametrize("precision", [FP32, FP64])
@pytest.mark.parametrize("case", CASES[1:5])
def test_twenty_bounces_match_oracle(precision, case):
    n, fres, g0, T1, R = case
    E0 = start_field("lasing", n, precision, 11 + n)
    with gpu(n, fres, g0, T1, R, precision, chunk=7) as r:
        r.set_field(E0)
        r.step(20)
        E20, N20, hist = r.field(), r.inversion(), r.history(20)
    p = oparams(n, fres, g0, T1, R)
    oE, oN, oh = orc.run(p, E0.astype(np.complex128), orc.pump(p), 20, nthreads=4)
    assert rel_l2(E20, oE) <= TOL20[precision]
    assert float(np.linalg.norm(N20 - oN) / np.linalg.norm(oN)) <= TOL20[precision]
    assert np.max(np.abs(hist - oh) / oh) <= TOL20[precision]


def test_plain_fp64_config_500_bounces_from_library_noise():
    # Plain FP64 map, 128^2, N_F = 20, 500 round trips from the seeded noise
    # start that both sides draw from the same counter-based generator.
    c = wl.C1
    with rt.Resonator.from_params(c, precision=FP64) as r:
        E0 = r.field()
        r.step(wl.C1_BOUNCES)
        E, N, hist = r.field(), r.inversion(), r.history(wl.C1_BOUNCES)
    p = oparams(c.n, c.fresnel, c.g0, c.T1, c.R)
    oE0, oN0 = orc.init_state(p, c.seed, c.noise_amp)
    assert rel_l2(E0, oE0) <= 1e-14
    oE, oN, oh = orc.run(p, oE0, oN0, wl.C1_BOUNCES, nthreads=4)
    assert rel_l2(E, oE) <= 1e-9
    assert np.max(np.abs(hist - oh) / oh) <= 1e-9


def test_library_noise_matches_oracle_generator():
    for precision in (FP32, FP64):
        with gpu(64, 50.0, 0.2, 100.0, 0.9, precision, seed=123, noise_amp=2e-3) as r:
            E = r.field()
        ref = orc.noise(64, 123, 2e-3)
        if precision == FP64:
            assert rel_l2(E, ref) <= 1e-15
        else:
            assert np.max(np.abs(E - ref.astype(np.complex64))) <= 1e-7 * 2e-3


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("precision", [FP32, FP64])
def test_talbot_self_imaging_and_half_period_shift(precision):
    q, n = 8, 256
    rng = np.random.default_rng(3)
    p_px = n // q
    block = rng.standard_normal((p_px, p_px)) + 1j * rng.standard_normal((p_px, p_px))
    E = np.tile(block, (q, q))
    tol = 1e-5 if precision == FP32 else 1e-12
    # alpha = 1/fresnel with D/W = 1: z_T (alpha q^2 = 2) and z_T/2 (alpha q^2 = 1)
    for fres, expect in [(q * q / 2.0, E), (q * q, np.roll(E, (p_px // 2, p_px // 2), axis=(0, 1)))]:
        with gpu(n, fres, 0.0, 10.0, 1.0, precision, edge=0, d_over_w=1.0) as r:
            r.set_field(E)
            r.step(1)
            assert rel_l2(r.field(), expect) <= tol


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_gaussian_beam_spreading(precision):
    n, a, zeta = 256, 0.1, 0.5
    fres = 1.0 / (zeta * math.pi * a * a / 2.0)
    alpha = 1.0 / fres
    zeta = 2 * alpha / (math.pi * a * a)
    x = (np.arange(n) - n // 2) / (n // 2)
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    q = 1 + 1j * zeta
    with gpu(n, fres, 0.0, 10.0, 1.0, precision, edge=0, d_over_w=1.0) as r:
        r.set_field(np.exp(-r2 / (2 * a * a)))
        r.step(1)
        out = r.field()
    assert np.max(np.abs(out - np.exp(-r2 / (2 * a * a * q)) / q)) <= (1e-5 if precision == FP32 else 1e-12)


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_uniform_field_reaches_saturation_fixed_point(precision):
    g0, R, n = 0.2, 0.95, 64
    with gpu(n, 100.0, g0, 10.0, R, precision, edge=0, pump_kind=rt.RT_PUMP_UNIFORM) as r:
        r.set_field(np.full((n, n), 0.3 + 0.1j))
        r.step(3000)
        E, N = r.field(), r.inversion()
    Nstar = -math.log(R)
    Istar = g0 / Nstar - 1.0
    tol = 1e-5 if precision == FP32 else 1e-10
    assert np.max(np.abs(N - Nstar)) <= tol * Nstar * 10
    assert np.max(np.abs(np.abs(E) ** 2 - Istar)) <= tol * Istar * 10


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_absorbing_edge_is_exactly_zero(precision):
    n, edge = 128, 8
    with gpu(n, 50.0, 0.2, 100.0, 0.95, precision, edge=edge) as r:
        r.set_field(start_field("lasing", n, precision, 5))
        r.step(3)
        E = r.field()
    mask = np.zeros((n, n), bool)
    mask[edge:n - edge, edge:n - edge] = True
    assert np.all(E[~mask] == 0) and np.all(np.abs(E[mask]) > 0)


# ------------------------------------------------------------ engine behaviour

@pytest.mark.parametrize("precision", [FP32, FP64])
def test_graph_chunks_direct_launches_and_checkpoint_are_bit_identical(precision):
    n = 128
    E0 = start_field("lasing", n, precision, 9)
    outs = []
    for chunk in (0, 5, 64):
        with gpu(n, 20.0, 0.2, 200.0, 0.95, precision, chunk=chunk) as r:
            r.set_field(E0)
            r.step(37)
            outs.append((r.field(), r.inversion(), r.stats().bounces))
    for E, N, b in outs[1:]:
        assert np.array_equal(E, outs[0][0]) and np.array_equal(N, outs[0][1]) and b == 37
    # checkpoint after 20 bounces, restore into a fresh handle, continue 17
    with gpu(n, 20.0, 0.2, 200.0, 0.95, precision, chunk=5) as r:
        r.set_field(E0)
        r.step(20)
        cE, cN = r.field(), r.inversion()
    with gpu(n, 20.0, 0.2, 200.0, 0.95, precision, chunk=5) as r:
        r.set_field(cE)
        r.set_inversion(cN)
        rt.rt_set_bounces(r.h, 20)
        r.step(17)
        assert np.array_equal(r.field(), outs[0][0]) and np.array_equal(r.inversion(), outs[0][1])
        assert r.stats().bounces == 37


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_spectrum_and_peak_match_oracle(precision):
    n = 256
    y, x = np.mgrid[0:n, 0:n]
    E = 0.3 * np.exp(2j * np.pi * (5 * x - 9 * y) / n) + start_field("lasing", n, precision, 4) * 0.1
    with gpu(n, 50.0, 0.2, 100.0, 0.95, precision) as r:
        r.set_field(E)
        S = r.spectrum()
        pk0, pk4 = r.peak(0), r.peak(4)
    Eo = E.astype(np.complex64 if precision == FP32 else np.complex128).astype(np.complex128)
    So = orc.spectrum(Eo)
    assert float(np.linalg.norm(S - So) / np.linalg.norm(So)) <= TOL1[precision]
    for ring, got in ((0, pk0), (4, pk4)):
        mx, my, pw, ru = orc.spectrum_peak(So, ring)
        assert (got[0], got[1]) == (mx, my)
        assert abs(got[2] - pw) <= 1e-5 * pw


def test_non_finite_field_is_reported():
    n = 64
    with gpu(n, 50.0, 0.2, 100.0, 0.95, FP32, edge=0) as r:
        E = np.zeros((n, n), np.complex64)
        E[10, 10] = np.inf
        r.set_field(E)
        r.step(1)
        with pytest.raises(rt.RtError) as ei:
            r.sync()
        assert ei.value.status == rt.RT_ENUMERIC


def test_history_ring_keeps_the_most_recent_bounces():
    n = 64
    with gpu(n, 50.0, 0.2, 100.0, 0.95, FP32, history_cap=16, chunk=0) as r:
        r.set_field(start_field("lasing", n, FP32, 2))
        r.step(10)
        first = r.history(10)
        r.step(30)
        st = r.stats()
        last = r.history(100)
    assert st.bounces == 40 and st.history_len == 16 and len(last) == 16
    assert len(first) == 10 and abs(last[-1] - st.mean_intensity) == 0
