"""The seeded synthetic inputs (paper_1410_2855_gb300/workloads.py) against the
recipe they state: the fixed resonator configurations, the batched parameter
sweep and the Poisson request stream (ranges and distributions), the noise
and low-frequency start fields, and the rough-mirror phase screen (rms and
Gaussian correlation).  Statistical checks use bounds several standard
errors wide; every generator is deterministic for a given seed."""
import math

import numpy as np

from paper_1410_2855_gb300 import workloads as wl


def test_fixed_configurations():
    assert (wl.C1.n, wl.C1.fresnel, wl.C1.g0, wl.C1.T1, wl.C1.R, wl.C1_BOUNCES) == (128, 20.0, 0.2, 2000.0, 0.95, 500)
    assert (wl.C2.n, wl.C2.fresnel, wl.C2.g0, wl.C2.T1, wl.C2.R, wl.C2_BOUNCES) == (512, 100.0, 0.15, 5000.0, 0.95,
                                                                                    10_000)
    assert [r.g0 for r in wl.C3] == [0.1, 0.3] and wl.C3_BOUNCES == 10_000
    for r in wl.C3:
        assert (r.n, r.fresnel, r.T1, r.R) == (2048, 1000.0, 1e4, 0.9)
    assert len({r.seed for r in wl.C3}) == len(wl.C3)
    assert wl.CURVED.z_over_F == 0.16 and wl.C2_CURVED.z_over_F == 0.16


def test_batch_sweep_follows_its_recipe():
    jobs = wl.batch_sweep(count=3000)
    assert jobs == wl.batch_sweep(count=3000)                      # deterministic
    assert [j.seed for j in jobs] == [wl.BASE_SEED + i for i in range(3000)]
    sides = np.array([j.n for j in jobs])
    for s in (256, 512, 1024):
        assert abs(np.mean(sides == s) - 1 / 3) < 0.03            # uniform over the three sides
    assert set(sides) == {256, 512, 1024}
    lf = np.log10([j.fresnel for j in jobs])
    assert lf.min() >= 2.0 and lf.max() <= 3.0
    assert abs(lf.mean() - 2.5) < 0.02 and abs(lf.std() - 1 / math.sqrt(12)) < 0.02   # log-uniform
    g0 = np.array([j.g0 for j in jobs])
    T1 = np.array([j.T1 for j in jobs])
    assert g0.min() >= 0.1 and g0.max() <= 0.3 and abs(g0.mean() - 0.2) < 0.005
    assert T1.min() >= 1e3 and T1.max() <= 1e4 and abs(T1.mean() - 5.5e3) < 150
    assert all(j.R == 0.95 and j.edge == 8 for j in jobs)


def test_serve_trace_is_a_poisson_stream_with_log_uniform_work():
    tr = wl.serve_trace(count=2000, rate_hz=50.0)
    t = np.array([q.arrival_s for q in tr])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0.0)
    assert abs(gaps.mean() - 0.02) < 0.02 * 0.1                     # mean 1/rate (std error 2.2%)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1                # exponential: cv = 1
    assert {q.job.n for q in tr} == {128, 256, 512, 1024, 2048}
    lb = np.log10([q.bounces for q in tr])
    assert lb.min() >= 3.0 - 1e-9 and lb.max() <= 5.0 + 1e-9 and abs(lb.mean() - 4.0) < 0.05


def test_noise_and_smooth_fields():
    n, amp = 256, 1e-6
    E = wl.noise_field(n, 3, amp)
    assert np.array_equal(E, wl.noise_field(n, 3, amp))
    for part in (E.real, E.imag):
        assert abs(part.mean()) < 5 * amp / math.sqrt(2 * n * n)
        assert abs(part.var() / (amp * amp / 2) - 1.0) < 0.02
    assert wl.noise_field(n, 3, amp, dtype=np.complex64).dtype == np.complex64
    S = wl.smooth_field(64, 5, 2.0, modes=6)
    assert abs(np.mean(np.abs(S) ** 2) - 4.0) < 1e-12               # normalised to amp^2
    F = np.fft.fft2(S)
    m = np.fft.fftfreq(64) * 64
    band = (np.abs(m)[:, None] < 6) & (np.abs(m)[None, :] < 6)
    assert np.all(np.abs(F[~band]) < 1e-9 * np.abs(F).max())         # only |m| < modes


def test_roughness_screen_rms_and_correlation():
    n, rms, corr = 256, 0.05, 0.05
    psi = wl.roughness_field(n, 11, rms, corr)
    assert np.array_equal(psi, wl.roughness_field(n, 11, rms, corr)) and psi.dtype == np.float64
    assert abs(psi.mean()) < 1e-15 and abs(psi.std() - rms) < 1e-15
    # Gaussian filter of width sigma = corr n / 2 pixels on white noise: the
    # autocorrelation is exp(-d^2 / (4 sigma^2)) (periodic window).
    sigma = corr * n / 2.0
    P = np.abs(np.fft.fft2(psi)) ** 2
    acf = np.fft.ifft2(P).real
    acf /= acf[0, 0]
    for d in (0.5 * sigma, sigma, 2 * sigma):
        k = int(round(d))
        want = math.exp(-k * k / (4 * sigma * sigma))
        got = 0.5 * (acf[0, k] + acf[k, 0])
        assert abs(got - want) < 0.08, (k, got, want)
