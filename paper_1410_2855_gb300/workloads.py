"""Seeded synthetic workloads for the bounce-map library.

This module holds parameter sets and seeded random inputs only; it contains
none of the map's arithmetic.  The tests and the benchmark draw the inputs
that both the CUDA path and the FP64 oracle consume from here.

The paper (Okulov, microchip laser resonator) reports no dataset; its regime
is a high-Fresnel-number (100-1000) microchip cavity started from noise.  The
workloads below have that shape: power-of-two square grids, Fresnel numbers
20-1000, a super-Gaussian pump of order 10 and radius 0.8 of the window
half-width, an 8-pixel absorbing edge and a complex Gaussian noise start of
amplitude 1e-6.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 14102855
D_OVER_W = 0.8      # gain-region diameter over window width (pump radius 0.8)
NOISE_AMP = 1e-6


@dataclasses.dataclass(frozen=True)
class Resonator:
    """Parameters of one resonator, in the units of the C ABI."""
    n: int
    fresnel: float
    g0: float
    T1: float
    R: float
    Isat: float = 1.0
    edge: int = 8
    pump_order: float = 10.0
    pump_radius: float = 0.8
    d_over_w: float = D_OVER_W
    seed: int = BASE_SEED
    noise_amp: float = NOISE_AMP
    z_over_F: float = 0.0        # curved mirror: distance per bounce over focal length (0 = flat)
    roughness_rms: float = 0.0   # mirror roughness phase, rms radians (0 = smooth)
    roughness_corr: float = 0.05  # its correlation length, fraction of the window half-width
    taper_px: int = 0             # smooth aperture ramp inside the absorbing edge (0 = hard edge)
    relax: int = 0                # inversion update: 0 explicit Euler step, 1 exact over the bounce

    def roughness(self):
        """The mirror's roughness phase psi (n x n float64), or None."""
        if self.roughness_rms == 0.0:
            return None
        return roughness_field(self.n, self.seed, self.roughness_rms, self.roughness_corr)


# Plain FP64 map on a 128^2 complex128 grid, N_F = 20, 500 round trips.
C1 = Resonator(n=128, fresnel=20.0, g0=0.2, T1=2000.0, R=0.95)
C1_BOUNCES = 500
# Single 512^2 complex64 resonator, N_F = 100, 1e4 round trips.
C2 = Resonator(n=512, fresnel=100.0, g0=0.15, T1=5000.0, R=0.95)
C2_BOUNCES = 10_000
# The same resonator with the paper's curved mirror (z/F = 0.16) and a rough
# surface (0.05 rad rms).
C2_CURVED = Resonator(n=512, fresnel=100.0, g0=0.15, T1=5000.0, R=0.95, z_over_F=0.16, roughness_rms=0.05)
# Single 2048^2 complex64 resonator, N_F = 1000, g0 in {0.1, 0.3}, 1e4 round trips.
C3 = tuple(Resonator(n=2048, fresnel=1000.0, g0=g, T1=1e4, R=0.9, seed=BASE_SEED + i)
           for i, g in enumerate((0.1, 0.3)))
C3_BOUNCES = 10_000
# The 2048^2 resonator with the paper's curved mirror (radius 50 mm at
# L = 2 mm: z/F = 4L/Rc = 0.16) and a weakly rough surface (0.05 rad rms).
CURVED = Resonator(n=2048, fresnel=1000.0, g0=0.3, T1=1e4, R=0.9, seed=BASE_SEED + 7, z_over_F=0.16,
                   roughness_rms=0.05)


def batch_sweep(count: int = 256, seed: int = BASE_SEED, sides=(256, 512, 1024)) -> list[Resonator]:
    """Batched parameter sweep: sides uniform over `sides`, N_F log-uniform in
    [100, 1000], g0 uniform in [0.1, 0.3], T1 uniform in [1e3, 1e4], R = 0.95,
    super-Gaussian pump, 8-pixel edge; resonator i is seeded with seed + i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sides))
        fres = float(math.exp(rng.uniform(math.log(100.0), math.log(1000.0))))
        g0 = float(rng.uniform(0.1, 0.3))
        T1 = float(rng.uniform(1e3, 1e4))
        out.append(Resonator(n=n, fresnel=fres, g0=g0, T1=T1, R=0.95, seed=seed + i))
    return out


@dataclasses.dataclass(frozen=True)
class Request:
    arrival_s: float
    job: Resonator
    bounces: int


def serve_trace(count: int = 1000, rate_hz: float = 50.0, seed: int = BASE_SEED,
                sides=(128, 256, 512, 1024, 2048), min_bounces: int = 1_000,
                max_bounces: int = 100_000) -> list[Request]:
    """Poisson stream of simulation requests: exponential inter-arrival times
    of mean 1/rate_hz, side uniform over `sides`, bounce count log-uniform in
    [min_bounces, max_bounces] rounded to an integer, other parameters drawn
    as in `batch_sweep`."""
    rng = np.random.default_rng(seed + 1)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        n = int(rng.choice(sides))
        fres = float(math.exp(rng.uniform(math.log(100.0), math.log(1000.0))))
        g0 = float(rng.uniform(0.1, 0.3))
        T1 = float(rng.uniform(1e3, 1e4))
        nb = int(round(math.exp(rng.uniform(math.log(min_bounces), math.log(max_bounces)))))
        out.append(Request(t, Resonator(n=n, fresnel=fres, g0=g0, T1=T1, R=0.95, seed=seed + i), nb))
    return out


def noise_field(n: int, seed: int, amp: float = NOISE_AMP, dtype=np.complex128) -> np.ndarray:
    """Seeded complex Gaussian field (numpy PCG64), Re and Im each with
    variance amp^2/2.  For complex64 the values are rounded to float32."""
    rng = np.random.default_rng(seed)
    s = amp / math.sqrt(2.0)
    f = rng.normal(0.0, s, (n, n)) + 1j * rng.normal(0.0, s, (n, n))
    return f.astype(dtype)


def smooth_field(n: int, seed: int, amp: float = 1.0, modes: int = 6, dtype=np.complex128) -> np.ndarray:
    """Seeded field made of a few low spatial frequencies (|m| < modes) with
    random complex amplitudes: a lasing-scale field with O(1) intensity."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:n, 0:n]
    f = np.zeros((n, n), np.complex128)
    for _ in range(3 * modes):
        mx, my = rng.integers(-modes + 1, modes, size=2)
        c = rng.normal() + 1j * rng.normal()
        f += c * np.exp(2j * np.pi * (mx * x + my * y) / n)
    f *= amp / math.sqrt(np.mean(np.abs(f) ** 2))
    return f.astype(dtype)


def random_inversion(n: int, seed: int, lo: float = 0.0, hi: float = 0.3, dtype=np.float64) -> np.ndarray:
    """Seeded inversion field, uniform in [lo, hi)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (n, n)).astype(dtype)


def roughness_field(n: int, seed: int, rms: float, corr: float) -> np.ndarray:
    """Seeded random phase screen: white Gaussian noise (PCG64, stream
    seed ^ 0x5eed) smoothed periodically by a Gaussian of width `corr`
    window half-widths and scaled to `rms` radians."""
    rng = np.random.default_rng(seed ^ 0x5EED)
    w = rng.standard_normal((n, n))
    k = np.fft.fftfreq(n) * n                        # cycles per window
    sigma = corr * n / 2.0                           # pixels
    g = np.exp(-0.5 * (2.0 * np.pi * k / n * sigma) ** 2)
    psi = np.fft.ifft2(np.fft.fft2(w) * g[:, None] * g[None, :]).real
    psi -= psi.mean()
    return psi * (rms / psi.std())

