"""Bounce-map oracle: ctypes wrapper around ``bouncemap_oracle.c``.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only importers.  The CUDA library and
its Python binding never import this package, and it imports nothing from
them.

The C file restates the paper's bounce map (eqs. conv_map, complex_8F,
complex_aperture2, limit_of_operators_renorm_final) in plain FP64; this module
only marshals numpy arrays.  Arrays are complex128 / float64, n x n,
row-major (E[y, x]).
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bouncemap_oracle.c")
_LIB_NAME = f"liboracle_{platform.machine()}.so"
_LIB_PATH = os.path.join(_HERE, _LIB_NAME)
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source (gcc, -O2;
    OpenMP over rows when the compiler supports it).  Returns the path."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    """Field-for-field mirror of ``orc_params`` in bouncemap_oracle.c."""

    _fields_ = [
        ("n", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("g0", ctypes.c_double),
        ("T1", ctypes.c_double),
        ("R", ctypes.c_double),
        ("Isat", ctypes.c_double),
        ("edge", ctypes.c_int),
        ("pump_kind", ctypes.c_int),
        ("pump_order", ctypes.c_double),
        ("pump_radius", ctypes.c_double),
        ("pump_profile", ctypes.c_void_p),
        ("z_over_F", ctypes.c_double),
        ("roughness", ctypes.c_void_p),
        ("slices", ctypes.c_int),
        ("taper", ctypes.c_int),
        ("relax", ctypes.c_int),
    ]


PUMP_SUPERGAUSS, PUMP_UNIFORM, PUMP_ARRAY = 0, 1, 2
PATTERN_GAUSSIAN, PATTERN_BEAM_ARRAY, PATTERN_VORTEX_ARRAY = 0, 1, 2


class Pattern(ctypes.Structure):
    """Field-for-field mirror of ``orc_pattern_t`` in bouncemap_oracle.c."""

    _fields_ = [
        ("kind", ctypes.c_int),
        ("periods", ctypes.c_int),
        ("out_of_phase", ctypes.c_int),
        ("width", ctypes.c_double),
        ("envelope", ctypes.c_double),
        ("curvature", ctypes.c_double),
        ("amplitude", ctypes.c_double),
    ]

_dp = ctypes.POINTER(ctypes.c_double)


def threads_available(requested: int) -> int:
    """Threads a call with nthreads=requested really uses: `requested` when
    the library was compiled with OpenMP, else 1."""
    return max(1, int(requested)) if lib().orc_openmp() else 1


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            L.orc_version.restype = i
            L.orc_openmp.restype = i
            L.orc_dft.argtypes = [vp, vp, i, i]
            L.orc_fft.argtypes = [vp, i, i]
            L.orc_fft.restype = i
            L.orc_fft2.argtypes = [vp, i, i, i]
            L.orc_fft2.restype = i
            L.orc_phase_2d.argtypes = [i, d, vp]
            L.orc_diffract.argtypes = [vp, i, d, i]
            L.orc_diffract.restype = i
            L.orc_pump.argtypes = [ctypes.POINTER(Params), vp]
            L.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.orc_splitmix64.restype = ctypes.c_uint64
            L.orc_noise.argtypes = [i, ctypes.c_uint64, d, vp]
            L.orc_pattern.argtypes = [i, ctypes.POINTER(Pattern), vp]
            L.orc_pattern.restype = i
            L.orc_run.argtypes = [ctypes.POINTER(Params), vp, vp, ctypes.c_longlong, vp, i]
            L.orc_run.restype = i
            L.orc_spectrum.argtypes = [vp, i, vp, i]
            L.orc_spectrum.restype = i
            L.orc_spectrum_peak.argtypes = [vp, i, i, ctypes.POINTER(i), ctypes.POINTER(i), _dp, _dp]
            _lib = L
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def alpha_from_fresnel(fresnel: float, d_over_w: float) -> float:
    """alpha = lambda z / W^2 with the cavity Fresnel number N_F = D^2 / (lambda z)
    and D/W the gain-region diameter over the window width (the "global" Fresnel
    number of the comparison-with-experiment section)."""
    return d_over_w * d_over_w / fresnel


def make_params(n, alpha, g0, T1, R, Isat=1.0, edge=8, pump_kind=PUMP_SUPERGAUSS,
                pump_order=10.0, pump_radius=0.8, pump_profile=None, z_over_F=0.0, roughness=None, slices=1,
                taper=0, relax=0):
    p = Params(n=n, alpha=alpha, g0=g0, T1=T1, R=R, Isat=Isat, edge=edge, pump_kind=pump_kind,
               pump_order=pump_order, pump_radius=pump_radius, pump_profile=None, z_over_F=z_over_F,
               roughness=None, slices=slices, taper=taper, relax=relax)
    keep = []
    if pump_kind == PUMP_ARRAY:
        prof = _f64(pump_profile).reshape(n, n)
        p.pump_profile = prof.ctypes.data
        keep.append(prof)
    if roughness is not None:
        psi = _f64(roughness).reshape(n, n)
        p.roughness = psi.ctypes.data
        keep.append(psi)
    p._keep = keep  # keeps the arrays alive as long as the params
    return p


def dft(x, sign=-1) -> np.ndarray:
    x = _c128(x)
    y = np.empty_like(x)
    lib().orc_dft(x.ctypes.data, y.ctypes.data, x.size, sign)
    return y


def fft(x, sign=-1) -> np.ndarray:
    x = _c128(x).copy()
    if lib().orc_fft(x.ctypes.data, x.size, sign) != 0:
        raise ValueError("length must be a power of two")
    return x


def fft2(a, sign=-1, nthreads=1) -> np.ndarray:
    a = _c128(a).copy()
    if lib().orc_fft2(a.ctypes.data, a.shape[0], sign, nthreads) != 0:
        raise ValueError("side must be a power of two")
    return a


def phase_2d(n, alpha) -> np.ndarray:
    H = np.empty((n, n), np.complex128)
    lib().orc_phase_2d(n, alpha, H.ctypes.data)
    return H


def diffract(E, alpha, nthreads=1) -> np.ndarray:
    E = _c128(E).copy()
    if lib().orc_diffract(E.ctypes.data, E.shape[0], alpha, nthreads) != 0:
        raise ValueError("side must be a power of two")
    return E


def pump(params: Params) -> np.ndarray:
    N0 = np.empty((params.n, params.n), np.float64)
    lib().orc_pump(ctypes.byref(params), N0.ctypes.data)
    return N0


def initial_inversion(params: Params) -> np.ndarray:
    """The fully pumped start: N = N0 (one slice), or N0/m in each of m
    slices (m x n x n)."""
    N0 = pump(params)
    m = max(params.slices, 1)
    return N0 if m == 1 else np.repeat((N0 / m)[None], m, axis=0)


def splitmix64(seed: int, c: int) -> int:
    return int(lib().orc_splitmix64(seed, c))


def pattern(n, kind, width, periods=1, out_of_phase=False, envelope=0.0, curvature=0.0,
            amplitude=1.0) -> np.ndarray:
    """Structured starting field (Gaussian beam, beam array, vortex array)."""
    pt = Pattern(kind=kind, periods=periods, out_of_phase=int(bool(out_of_phase)), width=width, envelope=envelope,
                 curvature=curvature, amplitude=amplitude)
    E = np.empty((n, n), np.complex128)
    if lib().orc_pattern(n, ctypes.byref(pt), E.ctypes.data) != 0:
        raise ValueError("invalid pattern")
    return E


def noise(n, seed, amp) -> np.ndarray:
    E = np.empty((n, n), np.complex128)
    lib().orc_noise(n, seed, amp, E.ctypes.data)
    return E


def run(params: Params, E, N, nb, nthreads=1, history=True):
    """Run nb bounces from (E, N).  Returns (E, N, hist) with fresh arrays;
    hist[b] is the mean intensity after bounce b (None if history=False).
    With m > 1 slices N holds m inversions (m x n x n)."""
    E = _c128(E).copy()
    N = _f64(N).copy()
    m = max(params.slices, 1)
    if E.size != params.n ** 2 or N.size != m * params.n ** 2:
        raise ValueError("field must be n x n and the inversion slices x n x n")
    hist = np.empty(max(int(nb), 0), np.float64) if history else None
    rc = lib().orc_run(ctypes.byref(params), E.ctypes.data, N.ctypes.data, int(nb),
                       hist.ctypes.data if history else None, nthreads)
    if rc != 0:
        raise ValueError(f"orc_run failed with {rc}")
    return E, N, hist


def spectrum(E, nthreads=1) -> np.ndarray:
    E = _c128(E)
    S = np.empty(E.shape, np.float64)
    if lib().orc_spectrum(E.ctypes.data, E.shape[0], S.ctypes.data, nthreads) != 0:
        raise ValueError("side must be a power of two")
    return S


def spectrum_peak(S, ring=0):
    """(mx, my, folded_peak_power, runner_up_power) of the dominant spatial
    frequency with m and -m folded together; ring > 0 restricts the search to
    max(|mx|, |my|) >= ring."""
    S = _f64(S)
    mx, my = ctypes.c_int(), ctypes.c_int()
    pk, ru = ctypes.c_double(), ctypes.c_double()
    lib().orc_spectrum_peak(S.ctypes.data, S.shape[0], ring, ctypes.byref(mx), ctypes.byref(my),
                            ctypes.byref(pk), ctypes.byref(ru))
    return mx.value, my.value, pk.value, ru.value


def init_state(params: Params, seed: int, amp: float):
    """Initial state of a run: seeded complex Gaussian noise field and the
    fully pumped inversion N = N0."""
    return noise(params.n, seed, amp), pump(params)
