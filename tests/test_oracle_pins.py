"""Pins of the FP64 oracle to things other than itself: library FFTs, brute
force, closed forms of paraxial optics (Talbot self-imaging, Gaussian-beam
spreading), fixed points and linearisations of the gain/inversion recursion,
published generator test vectors, and the paper's printed parameters.

A plausible slip in the oracle (a dropped 1/n^2, a flipped propagator sign, an
exp(N) for exp(N/2), the updated inversion used in the gain, an off-by-one in
the absorbing edge) fails at least one test here.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def crandn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ----------------------------------------------------------------- transforms

@pytest.mark.parametrize("n", [8, 16, 32])
@pytest.mark.parametrize("sign", [-1, +1])
def test_bruteforce_dft_matches_numpy(n, sign):
    x = crandn(np.random.default_rng(n), n)
    ref = np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * n
    assert np.max(np.abs(orc.dft(x, sign) - ref)) < 1e-12 * n


@pytest.mark.parametrize("n", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("sign", [-1, +1])
def test_fft_matches_bruteforce_dft(n, sign):
    x = crandn(np.random.default_rng(100 + n), n)
    assert rel_l2(orc.fft(x, sign), orc.dft(x, sign)) < 1e-13


@pytest.mark.parametrize("n", [8, 32, 64])
def test_fft2_matches_numpy(n):
    a = crandn(np.random.default_rng(7), (n, n))
    assert rel_l2(orc.fft2(a, -1), np.fft.fft2(a)) < 1e-14
    assert rel_l2(orc.fft2(a, +1), np.fft.ifft2(a) * n * n) < 1e-14


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        orc.fft(np.ones(12), -1)


def test_parseval_and_inverse():
    a = crandn(np.random.default_rng(3), (64, 64))
    A = orc.fft2(a, -1)
    assert abs(np.sum(np.abs(A) ** 2) / a.size - np.sum(np.abs(a) ** 2)) < 1e-10 * np.sum(np.abs(a) ** 2)
    assert rel_l2(orc.fft2(A, +1) / a.size, a) < 1e-14


# --------------------------------------------------------------- diffraction

def test_phase_table_unit_modulus_and_symmetry():
    n, alpha = 64, 0.0173
    H = orc.phase_2d(n, alpha)
    assert np.max(np.abs(np.abs(H) - 1.0)) < 1e-15
    assert H[0, 0] == 1.0
    k = np.arange(1, n)
    # H depends on mx^2 + my^2 only: even in each index and symmetric in (mx, my).
    assert np.max(np.abs(H[:, k] - H[:, n - k])) < 1e-13
    assert np.max(np.abs(H - H.T)) < 1e-13


def test_phase_table_large_argument_range_reduction():
    # At 2048^2 and N_F = 1000 the phase pi*alpha*m^2 reaches ~2.1e3 rad; a
    # value of alpha with a short binary expansion lets the exact phase be
    # written down: alpha = 2^-10, m = 1024 -> pi * 1024 = 512 turns -> 1.
    n = 2048
    H = orc.phase_2d(n, 2.0 ** -10)
    assert abs(H[0, n // 2] - 1.0) < 1e-15            # m = -1024: alpha m^2 = 1024
    assert abs(H[0, 1000] - np.exp(-1j * np.pi * (1000 ** 2 % 2048) / 1024.0)) < 1e-14


def test_diffraction_is_unitary():
    a = crandn(np.random.default_rng(11), (64, 64))
    out = orc.diffract(a, 0.0123)
    assert abs(np.linalg.norm(out) / np.linalg.norm(a) - 1.0) < 1e-13


def _talbot_setup(q=8, n=64, seed=5):
    """Field with q periods across the window: period p = n/q pixels."""
    rng = np.random.default_rng(seed)
    p = n // q
    return np.tile(crandn(rng, (p, p)), (q, q)), p


def _alpha_for_distance(lam, z, W):
    return lam * z / W ** 2


def test_talbot_self_imaging():
    # Talbot length z_T = 2 p^2 / lambda (introduction, point 3, and the
    # Talbot condition L = m p^2 / lambda of the exact-solutions section).
    q, n = 8, 64
    E, p_px = _talbot_setup(q, n)
    lam, p = 1.064e-6, 50e-6
    alpha = _alpha_for_distance(lam, 2 * p * p / lam, q * p)
    assert abs(alpha - 2.0 / q ** 2) < 1e-15
    assert rel_l2(orc.diffract(E, 2.0 / q ** 2), E) < 1e-13
    # A field that is not periodic with p does not self-image.
    F = crandn(np.random.default_rng(6), (n, n))
    assert rel_l2(orc.diffract(F, 2.0 / q ** 2), F) > 0.5


def test_half_talbot_shifts_by_half_period():
    # At z_T / 2 = p^2 / lambda the pattern returns shifted by p/2 in x and y
    # (the in-phase / anti-phase Talbot locking of the multiscale section).
    q, n = 8, 64
    E, p = _talbot_setup(q, n)
    out = orc.diffract(E, 1.0 / q ** 2)
    assert rel_l2(out, np.roll(E, (p // 2, p // 2), axis=(0, 1))) < 1e-13


def test_quarter_talbot_closed_form():
    # At z_T / 4 each spectral line m = q s picks up exp(-i pi s^2 / 2), i.e.
    # 1 for even s and -i for odd s: per axis a + b * (half-period shift)
    # with a = (1 - i)/2, b = (1 + i)/2.
    q, n = 8, 64
    E, p = _talbot_setup(q, n)
    a, b = (1 - 1j) / 2, (1 + 1j) / 2
    h = p // 2
    sx = np.roll(E, h, axis=1)
    sy = np.roll(E, h, axis=0)
    sxy = np.roll(E, (h, h), axis=(0, 1))
    expect = a * a * E + a * b * (sx + sy) + b * b * sxy
    assert rel_l2(orc.diffract(E, 0.5 / q ** 2), expect) < 1e-13


def test_gaussian_beam_spreading_matches_paraxial_closed_form():
    # A Gaussian of width a (window half-width 1) after distance z:
    # (1 + i zeta)^-1 exp(-r^2 / (2 a^2 (1 + i zeta))), zeta = z / (k a^2),
    # i.e. the prefactor (1 + i N_f^-1)^-1 and envelope of the exact solution
    # of the exact-solutions section with N_f = k a^2 / z and F = infinity.
    # With W = 2: alpha = lambda z / W^2 gives zeta = 2 alpha / (pi a^2).
    n, a, zeta = 128, 0.1, 0.5
    alpha = zeta * math.pi * a * a / 2.0
    x = (np.arange(n) - n // 2) / (n // 2)
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    E0 = np.exp(-r2 / (2 * a * a)).astype(np.complex128)
    q = 1 + 1j * zeta
    expect = np.exp(-r2 / (2 * a * a * q)) / q
    out = orc.diffract(E0, alpha)
    assert np.max(np.abs(out - expect)) < 1e-12
    # The opposite propagator sign gives the conjugate solution: far off.
    assert np.max(np.abs(out - np.conj(expect))) > 0.1


# ----------------------------------------------------- gain and inversion map

def uniform_params(n=8, g0=0.2, T1=10.0, R=0.95, Isat=1.0, alpha=0.01):
    return orc.make_params(n, alpha, g0, T1, R, Isat=Isat, edge=0, pump_kind=orc.PUMP_UNIFORM)


def test_uniform_field_converges_to_saturation_fixed_point():
    # Uniform field, uniform pump: the fixed point of the map has the round-trip
    # gain R exp(N*) = 1 and the saturated inversion N* (1 + I*/Isat) = g0
    # (steady state of dN/dt = (N0 - N)/T1 - sigma |E|^2 N).
    for g0, R, Isat in [(0.2, 0.95, 1.0), (0.3, 0.9, 2.0)]:
        p = uniform_params(g0=g0, R=R, Isat=Isat)
        E0 = np.full((8, 8), 0.3 + 0.1j)
        N0 = np.full((8, 8), g0)
        E, N, hist = orc.run(p, E0, N0, 3000)
        Nstar = -math.log(R)
        Istar = Isat * (g0 / Nstar - 1.0)
        assert np.max(np.abs(N - Nstar)) < 1e-12
        assert np.max(np.abs(np.abs(E) ** 2 - Istar)) < 1e-10
        assert abs(hist[-1] - Istar) < 1e-10


def test_relaxation_oscillation_matches_linearised_map():
    # Near the fixed point the (I, N) recursion is linear with Jacobian
    #   [[1, I*], [-N*/(Isat T1), 1 - (1 + I*/Isat)/T1]]
    # (the round-trip gain R e^N = 1, gain acting with the frozen N_n and the
    # depletion driven by the arriving intensity).  Its complex eigenvalues
    # give the relaxation-oscillation frequency ~ sqrt(N* I*/T1) per bounce,
    # cf. tau_rel = sqrt(T1 tau_c)/sqrt(sigma N0 c tau_c - 1).
    g0, R, T1, Isat = 0.2, 0.95, 2000.0, 1.0
    Nstar = -math.log(R)
    Istar = Isat * (g0 / Nstar - 1.0)
    p = uniform_params(g0=g0, T1=T1, R=R, Isat=Isat)
    E0 = np.full((8, 8), math.sqrt(Istar * (1 + 1e-6)) + 0j)
    N0 = np.full((8, 8), Nstar)
    _, _, hist = orc.run(p, E0, N0, 2500)
    d = hist - Istar
    A = np.stack([d[1:-1], d[:-2]], axis=1)
    a1, a0 = np.linalg.lstsq(A, d[2:], rcond=None)[0]
    fit = np.sort_complex(np.roots([1.0, -a1, -a0]))
    J = np.array([[1.0, Istar], [-Nstar / (Isat * T1), 1.0 - (1.0 + Istar / Isat) / T1]])
    lam = np.sort_complex(np.linalg.eigvals(J))
    assert np.max(np.abs(fit - lam)) < 1e-7
    period = 2 * math.pi / abs(np.angle(lam[0]))
    assert abs(period / (2 * math.pi / math.sqrt(Nstar * Istar / T1)) - 1.0) < 0.05
    # The other plausible reading (depletion by the amplified intensity) moves
    # the damping by a few per cent, far outside the fit's error.
    J2 = J.copy()
    J2[1, 1] -= Nstar * Istar / T1
    assert np.max(np.abs(fit - np.sort_complex(np.linalg.eigvals(J2)))) > 1e-6


def test_inversion_relaxes_exponentially_without_field():
    # No field: N_{n+1} = N_n + (N0 - N_n)/T1, so
    # N_b = N0 + (N_init - N0) (1 - 1/T1)^b at every pixel.
    n, T1, nb = 32, 37.0, 50
    p = orc.make_params(n, 0.02, 0.25, T1, 0.9, edge=3)
    N0 = orc.pump(p)
    Ninit = np.random.default_rng(1).uniform(0, 0.4, (n, n))
    E, N, hist = orc.run(p, np.zeros((n, n), complex), Ninit, nb)
    assert np.all(E == 0) and np.all(hist == 0)
    assert np.max(np.abs(N - (N0 + (Ninit - N0) * (1 - 1 / T1) ** nb))) < 1e-14


def test_one_bounce_with_identity_diffraction():
    # alpha = 2 makes exp(-i pi alpha m^2) = 1 for every integer m (the Talbot
    # distance of a one-period window), leaving the local map alone:
    # E1 = sqrt(R) A e^{N0/2} E0 and N1 = N0 - N0 |E0|^2 / (Isat T1).
    n, g0, T1, R, Isat, edge = 32, 0.3, 50.0, 0.9, 1.5, 4
    p = orc.make_params(n, 2.0, g0, T1, R, Isat=Isat, edge=edge)
    N0 = orc.pump(p)
    E0 = crandn(np.random.default_rng(2), (n, n))
    E1, N1, _ = orc.run(p, E0, N0, 1)
    A = np.zeros(n)
    A[edge:n - edge] = 1.0
    assert np.max(np.abs(E1 - math.sqrt(R) * np.outer(A, A) * np.exp(N0 / 2) * E0)) < 1e-13
    assert np.max(np.abs(N1 - (N0 - N0 * np.abs(E0) ** 2 / (Isat * T1)))) < 1e-14


def test_absorbing_edge_zeroes_exactly_the_outer_band():
    n, edge = 64, 8
    p = orc.make_params(n, 0.03, 0.2, 100.0, 0.95, edge=edge)
    E0 = crandn(np.random.default_rng(4), (n, n))
    E1, _, _ = orc.run(p, E0, orc.pump(p), 1)
    mask = np.zeros((n, n), bool)
    mask[edge:n - edge, edge:n - edge] = True
    assert np.all(E1[~mask] == 0)
    assert np.all(np.abs(E1[mask]) > 0)


def test_map_without_gain_is_pure_diffraction():
    # g0 = 0, N = 0, R = 1, no edge: the map is the diffraction operator alone,
    # so the Talbot pin holds for the whole bounce.
    q, n = 8, 64
    E, p_px = _talbot_setup(q, n)
    p = orc.make_params(n, 2.0 / q ** 2, 0.0, 10.0, 1.0, edge=0)
    E1, N1, _ = orc.run(p, E, np.zeros((n, n)), 3)
    assert rel_l2(E1, E) < 1e-13


def test_super_gaussian_pump_profile():
    n, g0 = 16, 0.25
    p = orc.make_params(n, 0.01, g0, 10.0, 0.9, pump_order=10.0, pump_radius=0.5)
    N0 = orc.pump(p)
    c = n // 2
    assert N0[c, c] == g0                                    # pixel n/2 is the origin
    assert abs(N0[c, c + 4] - g0 / math.e) < 1e-15           # x = 0.5 = r_p
    for d, e in [(1, 2), (3, 5), (2, 7)]:
        assert N0[c + d, c + e] == N0[c - d, c - e] == N0[c + e, c + d]
    assert np.all(np.diff(N0[c, c:]) < 0)


def test_super_gaussian_of_order_two_is_the_gaussian():
    # order and radius are the caller's: order 2, radius 0.3 is g0 exp(-(r/0.3)^2)
    n, g0 = 32, 0.2
    N0 = orc.pump(orc.make_params(n, 0.01, g0, 10.0, 0.9, pump_order=2.0, pump_radius=0.3))
    x = (np.arange(n) - n // 2) / (n // 2)
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    assert np.max(np.abs(N0 - g0 * np.exp(-r2 / 0.09))) <= 1e-15


def test_uniform_and_array_pumps():
    n, g0 = 16, 0.3
    assert np.all(orc.pump(orc.make_params(n, 0.01, g0, 10.0, 0.9, pump_kind=orc.PUMP_UNIFORM)) == g0)
    prof = np.zeros((n, n))
    prof[2, 11] = 1.0                                        # row 2, column 11: y = 2, x = 11
    prof[5, :] = 0.5
    N0 = orc.pump(orc.make_params(n, 0.01, g0, 10.0, 0.9, pump_kind=orc.PUMP_ARRAY, pump_profile=prof))
    assert np.array_equal(N0, g0 * prof) and N0[2, 11] == g0 and N0[11, 2] == 0.0


# --------------------------------------------------------------------- noise

def test_splitmix64_published_vectors():
    # First three outputs of splitmix64 from state 0 (Steele, Lea & Flood 2014;
    # the reference generator's widely reproduced test vector).
    assert orc.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert orc.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert orc.splitmix64(0, 2) == 0x06C45D188009454F


def test_noise_statistics():
    n, amp = 256, 1e-6
    E = orc.noise(n, 14102855, amp)
    assert abs(np.mean(np.abs(E) ** 2) / amp ** 2 - 1.0) < 0.02
    assert abs(np.mean(E)) < 0.02 * amp
    re = E.real.ravel() / (amp / math.sqrt(2))
    assert abs(np.var(re) - 1.0) < 0.02
    assert abs(np.mean(re ** 4) - 3.0) < 0.1                # Gaussian kurtosis
    assert abs(np.mean(E.real * E.imag)) < 0.02 * amp ** 2  # Re, Im uncorrelated
    assert not np.array_equal(E, orc.noise(n, 14102856, amp))


# ---------------------------------------------------------------- spectrum peak

def test_spectrum_peak_folding_and_ring():
    n = 32
    y, x = np.mgrid[0:n, 0:n]
    wave = np.exp(2j * np.pi * (3 * x - 5 * y) / n)
    S = orc.spectrum(wave)
    assert abs(S[n - 5, 3] - n ** 4) < 1e-6 * n ** 4
    mx, my, pk, ru = orc.spectrum_peak(S)
    # (3, -5) and (-3, 5) are one peak; it is filed under the smaller flat index.
    assert (mx, my) == (-3, 5) and abs(pk - n ** 4) < 1e-6 * n ** 4 and ru < 1e-12 * pk
    S2 = orc.spectrum(2.0 + wave)
    assert orc.spectrum_peak(S2)[:2] == (0, 0)
    assert orc.spectrum_peak(S2, ring=4)[:2] == (-3, 5)


def test_spectrum_parseval_and_history_is_the_mean_intensity():
    # sum_m S(m) = n^2 sum_j |E_j|^2 for the unnormalised transform; the
    # reported mean intensity of a bounce is <|E|^2> of the field it returns.
    n = 32
    rng = np.random.default_rng(5)
    E = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    S = orc.spectrum(E)
    assert np.all(S >= 0.0)
    assert abs(S.sum() - n * n * np.sum(np.abs(E) ** 2)) <= 1e-12 * S.sum()
    p = orc.make_params(n, 0.05, 0.3, 200.0, 0.9)
    for nb in (1, 4):
        E1, _, hist = orc.run(p, E, orc.pump(p), nb)
        assert len(hist) == nb and abs(hist[-1] - np.mean(np.abs(E1) ** 2)) <= 1e-14 * hist[-1]


def test_thread_count_reported_for_the_host_baseline():
    # The host baseline states how many threads the oracle used: all that
    # were asked for with OpenMP, one without it.
    assert orc.lib().orc_openmp() in (0, 1)
    assert orc.threads_available(6) == (6 if orc.lib().orc_openmp() else 1)
    assert orc.threads_available(0) == 1


def test_threaded_oracle_is_bit_identical_to_one_thread():
    # The host baseline runs the oracle on all cores; threads split rows and
    # columns of the transforms and rows of the local map, so every value is
    # computed by the same operations whatever the thread count.
    n = 64
    p = orc.make_params(n, 0.05, 0.3, 300.0, 0.9, z_over_F=0.2, taper=3, relax=1)
    E0 = orc.noise(n, 9, 1.0)
    N0 = orc.initial_inversion(p)
    one = orc.run(p, E0, N0, 3, nthreads=1)
    for t in (2, 5):
        many = orc.run(p, E0, N0, 3, nthreads=t)
        assert all(np.array_equal(a, b) for a, b in zip(one, many)), t
    assert np.array_equal(orc.fft2(E0, nthreads=1), orc.fft2(E0, nthreads=3))


# ----------------------------------------------------- the paper's own numbers

def test_paper_parameters_give_the_quoted_fresnel_range_and_period():
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as f:
        g = json.load(f)
    lam, L = g["wavelength_m"], g["cavity_length_m"]
    lo, hi = (D * D / (lam * L) for D in g["gain_region_diameter_m"])
    # "global" Fresnel number D^2/(lambda L) of the quoted geometry: 100..1000.
    assert g["fresnel_quoted"][0] * 0.9 < lo < g["fresnel_quoted"][0] * 1.5
    assert g["fresnel_quoted"][1] * 0.9 < hi < g["fresnel_quoted"][1] * 1.1
    # Lattice period p ~ sqrt(L lambda), quoted as roughly 50-60 um.
    p = math.sqrt(L * lam)
    assert 0.8 * g["period_quoted_m"][0] < p < g["period_quoted_m"][1]
    # alpha = lambda z / W^2 from the Fresnel number and D/W agree.
    for D in g["gain_region_diameter_m"]:
        W = D / 0.8
        assert abs(orc.alpha_from_fresnel(D * D / (lam * L), 0.8) - lam * L / W ** 2) < 1e-15


# ------------------------------------------- complex aperture: curved mirror, roughness

def _lens_guide_eigenmode(u, beta):
    """Self-reproducing Gaussian exp(-r^2 / (2 s)) of the unfolded cavity
    "propagate one bounce, then the mirror lens" with z/F = u (0 < u < 4),
    in window units.  Paraxial Gaussian algebra: free propagation adds
    i beta to s (beta = 2 alpha / pi, the 1/k of the window units), the
    thin lens exp(-i c r^2) adds 2 i c to 1/s, and c = (pi / (4 alpha)) u =
    u / (2 beta).  The fixed point s = i beta sigma solves
    sigma^2 + sigma + 1/u = 0 with Re s > 0."""
    w = math.sqrt(4.0 / u - 1.0) / 2.0
    return 1j * beta * complex(-0.5, -w)


@pytest.mark.parametrize("u", [0.16, 1.0, 2.0, 3.0])
def test_curved_mirror_eigenmode_advances_by_the_gouy_phase(u):
    # A flat/curved-mirror cavity is a periodic lens guide (lens spacing z,
    # focal length F).  Its Gaussian eigenmode returns each period with the
    # same profile and the on-axis phase advance -theta, cos theta =
    # (A + D)/2 = 1 - z/(2F) in two transverse dimensions (Kogelnik & Li,
    # 1966).  theta depends on z/F only, so it pins the lens strength
    # relative to the propagator as well as the focusing sign.
    n = 128
    beta = min(0.008, 0.01 * u * math.sqrt(4.0 / u - 1.0) / 2.0)
    alpha = math.pi * beta / 2.0
    s = _lens_guide_eigenmode(u, beta)
    x = (np.arange(n) - n // 2) / (n // 2)
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    E0 = np.exp(-r2 / (2.0 * s))
    p = orc.make_params(n, alpha, 0.0, 1e9, 1.0, edge=0, pump_kind=orc.PUMP_UNIFORM, z_over_F=u)
    theta = math.acos(1.0 - u / 2.0)
    E = E0
    for b in range(1, 6):
        E, N, _ = orc.run(p, E, np.zeros((n, n)), 1)
        assert np.max(np.abs(E - np.exp(-1j * b * theta) * E0)) < 1e-11
    # The opposite lens sign (a diverging mirror) has no such mode.
    q = orc.make_params(n, alpha, 0.0, 1e9, 1.0, edge=0, pump_kind=orc.PUMP_UNIFORM, z_over_F=-u)
    E, _, _ = orc.run(q, E0, np.zeros((n, n)), 5)
    assert np.max(np.abs(E - np.exp(-5j * theta) * E0)) > 0.05


def test_curved_mirror_focuses_a_gaussian_beam_to_the_closed_form_waist():
    # A Gaussian of waist a reaches the mirror with a flat front; the lens
    # then curves it: 1/s -> 1/a^2 + 2 i c, c = (pi/(4 alpha)) z/F.  It comes
    # to a focus (s real) after d_w = F / (1 + (F/Z)^2) bounces, Z = a^2/beta
    # the Rayleigh range in bounces and F = 1/(z/F), with the second moment
    # <r^2> = Re s there.  One oracle bounce diffracts first, so start from
    # the field one bounce before the waist: s0 = a^2 - i beta.
    n, a, u, beta = 256, 0.12, 0.25, 0.004
    alpha = math.pi * beta / 2.0
    c = u / (2.0 * beta)
    x = (np.arange(n) - n // 2) / (n // 2)
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    s0 = complex(a * a, -beta)
    E0 = np.exp(-r2 / (2.0 * s0))
    p = orc.make_params(n, alpha, 0.0, 1e9, 1.0, edge=0, pump_kind=orc.PUMP_UNIFORM, z_over_F=u)
    E1, _, _ = orc.run(p, E0, np.zeros((n, n)), 1)
    s_lens = 1.0 / (1.0 / (a * a) + 2j * c)
    expect = (s0 / (a * a)) * np.exp(-r2 / (2.0 * s_lens))
    assert np.max(np.abs(E1 - expect)) < 1e-11
    F, Z = 1.0 / u, a * a / beta
    d_w = F / (1.0 + (F / Z) ** 2)

    def second_moment(d):
        I = np.abs(orc.diffract(E1, alpha * d)) ** 2
        return float(np.sum(I * r2) / np.sum(I))

    w = second_moment(d_w)
    assert abs(w - s_lens.real) < 1e-9 * s_lens.real
    assert w < second_moment(0.9 * d_w) and w < second_moment(1.1 * d_w)
    # A diverging mirror (z/F < 0) has no focus ahead: the beam only grows.
    q = orc.make_params(n, alpha, 0.0, 1e9, 1.0, edge=0, pump_kind=orc.PUMP_UNIFORM, z_over_F=-u)
    E1d, _, _ = orc.run(q, E0, np.zeros((n, n)), 1)
    I0 = np.abs(E1d) ** 2
    I1 = np.abs(orc.diffract(E1d, alpha * d_w)) ** 2
    assert np.sum(I1 * r2) / np.sum(I1) > np.sum(I0 * r2) / np.sum(I0)


def test_roughness_phase_tilt_closed_form():
    # A linear roughness phase psi = pi (mx0 x + my0 y) is a tilted mirror:
    # on a uniform field it imprints the plane wave of frequency -(mx0, my0),
    # the next bounce propagates that wave (phase -pi alpha |m|^2) and tilts
    # it again.  After b bounces:
    #   E_b = exp(-i pi alpha |m0|^2 sum_{k<b} k^2) exp(-i b psi).
    # Distinct mx0, my0 pin the table's orientation (psi[y n + x]).
    n, alpha, mx0, my0 = 64, 0.013, 3, -2
    x = (np.arange(n) - n // 2) / (n // 2)
    psi = math.pi * (mx0 * x[None, :] + my0 * x[:, None])
    p = orc.make_params(n, alpha, 0.0, 1e9, 1.0, edge=0, pump_kind=orc.PUMP_UNIFORM, roughness=psi)
    E = np.ones((n, n), np.complex128)
    m2 = mx0 * mx0 + my0 * my0
    for b in range(1, 7):
        E, _, _ = orc.run(p, E, np.zeros((n, n)), 1)
        k2 = sum(k * k for k in range(1, b))
        expect = np.exp(-1j * math.pi * alpha * m2 * k2) * np.exp(-1j * b * psi)
        assert np.max(np.abs(E - expect)) < 1e-11
    # Transposing psi gives a different field.
    q = orc.make_params(n, alpha, 0.0, 1e9, 1.0, edge=0, pump_kind=orc.PUMP_UNIFORM, roughness=psi.T.copy())
    Et, _, _ = orc.run(q, np.ones((n, n), np.complex128), np.zeros((n, n)), 2)
    E2, _, _ = orc.run(p, np.ones((n, n), np.complex128), np.zeros((n, n)), 2)
    assert np.max(np.abs(Et - E2)) > 0.5


def test_aperture_phase_leaves_intensity_and_gain_untouched():
    # The aperture argument is a pure phase: with diffraction switched off
    # (alpha = 2, an identity bounce) the intensities, the inversion and the
    # mean intensity equal those of the flat, smooth mirror exactly.
    n = 32
    rng = np.random.default_rng(3)
    E0 = crandn(rng, (n, n))
    N0 = rng.uniform(0.0, 0.3, (n, n))
    psi = rng.normal(0.0, 1.0, (n, n))
    flat = orc.make_params(n, 2.0, 0.2, 50.0, 0.9, edge=2)
    rough = orc.make_params(n, 2.0, 0.2, 50.0, 0.9, edge=2, z_over_F=0.7, roughness=psi)
    Ef, Nf, hf = orc.run(flat, E0, N0, 1)
    Er, Nr, hr = orc.run(rough, E0, N0, 1)
    assert np.max(np.abs(np.abs(Er) - np.abs(Ef))) < 1e-14
    assert np.array_equal(Nf, Nr)
    assert abs(hf[0] - hr[0]) < 1e-15 * hf[0]
    x = (np.arange(n) - n // 2) / (n // 2)
    theta = math.pi / (4 * 2.0) * 0.7 * (x[None, :] ** 2 + x[:, None] ** 2) + psi
    inside = np.abs(Ef) > 0
    assert np.max(np.abs(Er[inside] - Ef[inside] * np.exp(-1j * theta[inside]))) < 1e-13


def test_paper_cavity_mirror_is_a_stable_lens_guide():
    # Flat facet + concave mirror of radius Rc at distance L, unfolded: one
    # bounce propagates z = 2L and passes one lens of focal length Rc/2, so
    # z/F = 4 L / Rc.  For the quoted geometry that is 0.16: inside the
    # stability range 0 < z/F < 4 (|cos theta| < 1), which the eigenmode test
    # above exercises at this value.
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as f:
        g = json.load(f)
    u = 4.0 * g["cavity_length_m"] / g["mirror_radius_of_curvature_m"]
    assert abs(u - 0.16) < 1e-12
    assert abs(1.0 - u / 2.0) < 1.0


# ----------------------------------------------------- multi-slice gain medium

def test_slices_without_gain_compose_to_one_bounce():
    # With no gain the m sub-steps of z/m compose to the diffraction over z
    # (the propagator is a one-parameter group), and the mirror acts once:
    # the m-slice map then equals the single-slice map.  Using z instead of
    # z/m per slice, or the mirror in every slice, breaks this.
    n = 64
    rng = np.random.default_rng(4)
    E0 = crandn(rng, (n, n))
    psi = rng.normal(0.0, 0.5, (n, n))
    kw = dict(edge=3, pump_kind=orc.PUMP_UNIFORM, z_over_F=0.3, roughness=psi)
    one = orc.make_params(n, 0.03, 0.0, 50.0, 0.9, **kw)
    four = orc.make_params(n, 0.03, 0.0, 50.0, 0.9, slices=4, **kw)
    E1, _, h1 = orc.run(one, E0, np.zeros((n, n)), 3)
    E4, N4, h4 = orc.run(four, E0, np.zeros((4, n, n)), 3)
    assert rel_l2(E4, E1) < 1e-13
    assert np.allclose(h4, h1, rtol=1e-13)
    assert not np.any(N4)


def test_slices_small_signal_gain_per_pass_is_g0():
    # Each slice is pumped to N0/m, so a weak field gains exp(g0) in
    # intensity per bounce whatever m (alpha = 2m makes every z/m step the
    # identity on the grid; R = 1, no edge).
    n, g0 = 16, 0.3
    for m in (1, 2, 5):
        p = orc.make_params(n, 2.0 * m, g0, 1e12, 1.0, edge=0, pump_kind=orc.PUMP_UNIFORM, slices=m)
        E0 = np.full((n, n), 1e-6 + 0j)
        E, N, _ = orc.run(p, E0, orc.initial_inversion(p), 1)
        assert np.max(np.abs(E - math.exp(g0 / 2) * E0)) < 1e-20
        assert np.max(np.abs(N - g0 / m)) < 1e-15


@pytest.mark.parametrize("m", [2, 3])
def test_slices_reach_the_saturated_amplifier_fixed_point(m):
    # Uniform field and pump, identity diffraction: in steady state slice s
    # holds N_s = (g0/m) / (1 + I_s/Isat) for the intensity I_s arriving at
    # it, I_{s+1} = I_s exp(N_s), and the round trip closes with
    # R exp(sum_s N_s) = 1.  The arriving intensity I_1 solves that scalar
    # equation (bracketed root); the iterated map must converge to it.
    from scipy.optimize import brentq

    n, g0, R, Isat, T1 = 8, 0.3, 0.9, 1.5, 10.0

    def chain(I1):
        I, Ns = I1, []
        for _ in range(m):
            Ns.append((g0 / m) / (1.0 + I / Isat))
            I *= math.exp(Ns[-1])
        return Ns

    I1 = brentq(lambda I: math.log(R) + sum(chain(I)), 1e-9, 100.0, xtol=1e-15)
    p = orc.make_params(n, 2.0 * m, g0, T1, R, Isat=Isat, edge=0, pump_kind=orc.PUMP_UNIFORM, slices=m)
    E, N, hist = orc.run(p, np.full((n, n), 0.5 + 0.2j), orc.initial_inversion(p), 4000)
    assert abs(hist[-1] - I1) < 1e-10 * I1
    for s, Ns in enumerate(chain(I1)):
        assert np.max(np.abs(N[s] - Ns)) < 1e-10
    # ... which is not the single-slice fixed point I* = Isat (g0 / N* - 1).
    assert abs(I1 - Isat * (g0 / -math.log(R) - 1.0)) > 1e-3


# -------------------------------------------- smooth aperture, exact relaxation

def _aperture_after_one_bounce(n, edge, taper):
    # alpha = 2: every diffraction phase is a multiple of 2 pi, so one bounce
    # of a uniform field with no gain and R = 1 leaves exactly A(x) A(y).
    p = orc.make_params(n, 2.0, 0.0, 1e9, 1.0, edge=edge, pump_kind=orc.PUMP_UNIFORM, taper=taper)
    E, _, _ = orc.run(p, np.ones((n, n), np.complex128), np.zeros((n, n)), 1)
    return E


def test_taper_zero_is_the_hard_edge_and_the_ramp_is_a_sin2_profile():
    n, edge = 64, 4
    hard = _aperture_after_one_bounce(n, edge, 0)
    band = np.zeros(n, bool)
    band[:edge] = band[n - edge:] = True
    assert np.all(hard[band, :] == 0) and np.all(hard[:, band] == 0) and np.all(hard[~band][:, ~band] == 1)
    for w in (1, 3, 6):
        E = _aperture_after_one_bounce(n, edge, w)
        assert np.max(np.abs(E.imag)) == 0.0
        A = E.real[n // 2]                        # the row through the centre: A(x) A(y_c), A(y_c) = 1
        ramp = A[edge:edge + w]
        assert np.all(A[band] == 0) and np.all(A[edge + w:n - edge - w] == 1)
        assert np.allclose(A, A[::-1], atol=0, rtol=0)         # symmetric
        assert np.all(np.diff(ramp) > 0) and ramp[-1] < 1.0     # rising, below 1
        assert np.allclose(ramp + ramp[::-1], 1.0, atol=1e-15)  # sin^2 t + sin^2(pi/2 - t) = 1
        assert abs(ramp[0] - math.sin(math.pi / (2 * (w + 1))) ** 2) < 1e-15
        assert np.allclose(E.real, np.outer(A, A), atol=1e-15)  # separable
    assert abs(_aperture_after_one_bounce(n, edge, 1).real[n // 2, edge] - 0.5) < 1e-15


def test_exact_relaxation_field_free_closed_form():
    # No field: dN/dt = (N0 - N)/T1 has N_b = N0 + (N_init - N0) exp(-b/T1),
    # where the Euler step gives (1 - 1/T1)^b instead.
    n, g0, T1, b = 8, 0.25, 7.0, 30
    p = orc.make_params(n, 0.02, g0, T1, 0.9, edge=0, pump_kind=orc.PUMP_UNIFORM, relax=1)
    _, N, _ = orc.run(p, np.zeros((n, n), np.complex128), np.full((n, n), 0.05), b)
    assert np.max(np.abs(N - (g0 + (0.05 - g0) * math.exp(-b / T1)))) < 1e-15
    q = orc.make_params(n, 0.02, g0, T1, 0.9, edge=0, pump_kind=orc.PUMP_UNIFORM, relax=0)
    _, Ne, _ = orc.run(q, np.zeros((n, n), np.complex128), np.full((n, n), 0.05), b)
    assert np.max(np.abs(Ne - (g0 + (0.05 - g0) * (1 - 1 / T1) ** b))) < 1e-15


def test_exact_relaxation_differs_from_euler_by_the_second_order_term():
    # One step with intensity I: exact minus Euler is
    # (N - Nss) (exp(-h) - 1 + h), h = (1 + I/Isat)/T1, i.e. between
    # (N - Nss) h^2/2 (1 - h/3) and (N - Nss) h^2/2.
    n, g0, T1, Isat = 16, 0.3, 40.0, 1.3
    rng = np.random.default_rng(8)
    E0 = crandn(rng, (n, n))
    N0 = rng.uniform(0.0, 0.5, (n, n))
    kw = dict(Isat=Isat, edge=0, pump_kind=orc.PUMP_UNIFORM)
    _, Nx, _ = orc.run(orc.make_params(n, 2.0, g0, T1, 0.9, relax=1, **kw), E0, N0, 1)
    _, Ne, _ = orc.run(orc.make_params(n, 2.0, g0, T1, 0.9, relax=0, **kw), E0, N0, 1)
    I = np.abs(E0) ** 2                        # alpha = 2: the field arriving at the gain is E0
    h = (1 + I / Isat) / T1
    dev = (N0 - g0 / (1 + I / Isat)) * h * h / 2
    d = Nx - Ne
    lo, hi = np.minimum(dev * (1 - h / 3), dev), np.maximum(dev * (1 - h / 3), dev)
    assert np.all(d >= lo - 1e-16) and np.all(d <= hi + 1e-16)


def test_exact_relaxation_keeps_the_saturation_fixed_point():
    g0, R, Isat = 0.2, 0.95, 1.0
    p = orc.make_params(8, 0.01, g0, 10.0, R, Isat=Isat, edge=0, pump_kind=orc.PUMP_UNIFORM, relax=1)
    E, N, hist = orc.run(p, np.full((8, 8), 0.3 + 0.1j), np.full((8, 8), g0), 3000)
    Nstar = -math.log(R)
    assert np.max(np.abs(N - Nstar)) < 1e-12
    assert abs(hist[-1] - Isat * (g0 / Nstar - 1.0)) < 1e-10


# ------------------------------------------------------ structured starting fields

def _winding(E, j, i):
    # total phase change, in turns, around the 8 pixels surrounding (row j, column i)
    ring = [(-1, -1), (-1, 0), (-1, 1), (0, 1), (1, 1), (1, 0), (1, -1), (0, -1), (-1, -1)]
    ph = [np.angle(E[j + dj, i + di]) for dj, di in ring]
    d = np.diff(ph)
    d = (d + np.pi) % (2 * np.pi) - np.pi
    return d.sum() / (2 * np.pi)


@pytest.mark.parametrize("out_of_phase", [False, True])
def test_vortex_array_has_unit_charges_on_the_lattice(out_of_phase):
    # A lattice of first-order vortices (the vortex-array solution): the
    # phase winds once around every lattice point, with alternating sign for
    # the out-of-phase array (antiparallel charges) and the same sign for the
    # in-phase one; the intensity vanishes there.
    n, q, w = 128, 8, 0.06
    E = orc.pattern(n, orc.PATTERN_VORTEX_ARRAY, w, periods=q, out_of_phase=out_of_phase)
    step = n // q                                  # lattice points fall on pixel centres
    for b in range(q):
        for a in range(q):
            j, i = (n // 2 + b * step) % n, (n // 2 + a * step) % n
            want = (-1) ** (a + b) if out_of_phase else 1
            assert abs(_winding(E, j, i) - want) < 1e-9, (a, b)
            assert abs(E[j, i]) < 1e-12


def test_beam_array_is_periodic_and_self_images_at_the_talbot_length():
    # The array of Gaussian beams is periodic with p = 2/q on the window, so
    # (with no envelope) it returns after the Talbot length, alpha q^2 = 2,
    # and is shifted by half a period at half of it.
    n, q, w = 128, 8, 0.04
    E = orc.pattern(n, orc.PATTERN_BEAM_ARRAY, w, periods=q)
    step = n // q
    assert rel_l2(np.roll(E, (step, step), axis=(0, 1)), E) < 1e-15
    assert rel_l2(orc.diffract(E, 2.0 / q ** 2), E) < 1e-12
    assert rel_l2(orc.diffract(E, 1.0 / q ** 2), np.roll(E, (step // 2, step // 2), axis=(0, 1))) < 1e-12
    # out of phase: the sign alternates between neighbours, period 2p
    F = orc.pattern(n, orc.PATTERN_BEAM_ARRAY, w, periods=q, out_of_phase=True)
    assert rel_l2(np.roll(F, step, axis=1), -F) < 1e-15
    tail = 4 * math.exp(-(2.0 / q) ** 2 / (2 * w * w))    # the four nearest neighbours' tails
    assert abs(F[n // 2, n // 2] - 1.0) < 1.01 * tail and abs(F[n // 2, n // 2 + step] + 1.0) < 1.01 * tail


def test_gaussian_envelope_multiplies_like_a_narrower_gaussian():
    # exp(-r^2/(2w^2)) exp(-r^2/(2D^2)) = exp(-r^2/(2 w'^2)), 1/w'^2 = 1/w^2 + 1/D^2
    n, w, D = 64, 0.2, 0.3
    a = orc.pattern(n, orc.PATTERN_GAUSSIAN, w, envelope=D, amplitude=2.5)
    b = orc.pattern(n, orc.PATTERN_GAUSSIAN, 1.0 / math.sqrt(1 / w ** 2 + 1 / D ** 2), amplitude=2.5)
    assert np.max(np.abs(a - b)) < 1e-14


def test_gaussian_pattern_with_curvature_is_the_lens_guide_eigenmode():
    # exp(-r^2/(2 w^2) - i c r^2) = exp(-r^2/(2 s)) with 1/s = 1/w^2 + 2 i c:
    # built from the eigenmode s of the flat/curved-mirror cavity it returns
    # each bounce with the Gouy phase exp(-i arccos(1 - z/2F)).
    n, u, beta = 128, 1.0, 0.008
    alpha = math.pi * beta / 2.0
    s = _lens_guide_eigenmode(u, beta)
    w, c = 1.0 / math.sqrt((1 / s).real), (1 / s).imag / 2.0
    E0 = orc.pattern(n, orc.PATTERN_GAUSSIAN, w, curvature=c)
    p = orc.make_params(n, alpha, 0.0, 1e9, 1.0, edge=0, pump_kind=orc.PUMP_UNIFORM, z_over_F=u)
    E3, _, _ = orc.run(p, E0, np.zeros((n, n)), 3)
    assert np.max(np.abs(E3 - np.exp(-3j * math.acos(1 - u / 2)) * E0)) < 1e-11


def test_pattern_rejects_bad_input():
    with pytest.raises(ValueError):
        orc.pattern(64, orc.PATTERN_BEAM_ARRAY, 0.05, periods=7, out_of_phase=True)   # odd q cannot alternate
    with pytest.raises(ValueError):
        orc.pattern(64, orc.PATTERN_GAUSSIAN, 0.0)
