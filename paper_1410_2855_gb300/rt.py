"""Thin ctypes binding of the C ABI declared in include/rt.h.

Functions carry the C names and only marshal arguments; every step of the
bounce map runs in the CUDA library.  Loading fails loudly if the library has
not been built: there is no CPU fallback.  A non-OK status raises RtError.
"""
from __future__ import annotations

import ctypes
import os
import platform

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("RT_LIBRARY") or os.path.join(HERE, "_lib", f"libbouncemap_{platform.machine()}.so")

RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ENUMERIC, RT_ETIMEOUT, RT_EBUSY, RT_EBOUNDS, RT_ECANCELED = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
RT_PUMP_SUPERGAUSS, RT_PUMP_UNIFORM, RT_PUMP_ARRAY = 0, 1, 2
RT_FP32, RT_FP64 = 0, 1
RT_RELAX_EULER, RT_RELAX_EXACT = 0, 1
RT_PATTERN_GAUSSIAN, RT_PATTERN_BEAM_ARRAY, RT_PATTERN_VORTEX_ARRAY = 0, 1, 2
RT_SERVE_FIFO, RT_SERVE_SHORTEST_FIRST = 0, 1


class RtError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class rt_pump(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("order", ctypes.c_double), ("radius", ctypes.c_double),
                ("profile", ctypes.c_void_p)]


class rt_opts(ctypes.Structure):
    _fields_ = [("Isat", ctypes.c_double), ("edge_px", ctypes.c_int), ("precision", ctypes.c_int),
                ("seed", ctypes.c_ulonglong), ("noise_amp", ctypes.c_double),
                ("pump_diam_over_window", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
                ("history_cap", ctypes.c_longlong), ("chunk", ctypes.c_int), ("col_tile", ctypes.c_int),
                ("z_over_F", ctypes.c_double), ("roughness", ctypes.c_void_p), ("slices", ctypes.c_int),
                ("taper_px", ctypes.c_int), ("relax", ctypes.c_int)]


class rt_pattern(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("periods", ctypes.c_int), ("out_of_phase", ctypes.c_int),
                ("width", ctypes.c_double), ("envelope", ctypes.c_double), ("curvature", ctypes.c_double),
                ("amplitude", ctypes.c_double)]


class rt_job(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("fresnel", ctypes.c_double), ("g0", ctypes.c_double), ("T1", ctypes.c_double),
                ("R", ctypes.c_double), ("pump", rt_pump), ("Isat", ctypes.c_double), ("edge_px", ctypes.c_int),
                ("seed", ctypes.c_ulonglong), ("noise_amp", ctypes.c_double),
                ("pump_diam_over_window", ctypes.c_double), ("z_over_F", ctypes.c_double),
                ("roughness", ctypes.c_void_p), ("taper_px", ctypes.c_int), ("relax", ctypes.c_int)]


class rt_serve_opts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_longlong), ("chunk", ctypes.c_int), ("max_per_size", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("policy", ctypes.c_int), ("round_points", ctypes.c_longlong)]


class rt_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("n", ctypes.c_int),
                ("bounces", ctypes.c_longlong), ("mean_intensity", ctypes.c_double), ("submit_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("finish_s", ctypes.c_double)]


class rt_serve_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("queued", ctypes.c_longlong), ("running", ctypes.c_longlong),
                ("done", ctypes.c_longlong), ("resident_bytes", ctypes.c_longlong),
                ("point_bounces", ctypes.c_double), ("busy_s", ctypes.c_double), ("rounds", ctypes.c_longlong),
                ("peak_resident_bytes", ctypes.c_longlong)]


class rt_stats_t(ctypes.Structure):
    _fields_ = [("bounces", ctypes.c_longlong), ("mean_intensity", ctypes.c_double), ("alpha", ctypes.c_double),
                ("n", ctypes.c_int), ("precision", ctypes.c_int), ("last_error", ctypes.c_int),
                ("history_len", ctypes.c_longlong)]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (raises ImportError if it was never built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"bounce-map CUDA library missing at {LIB_PATH}; build it with "
                              "paper_1410_2855_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, ll, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_size_t
        sig = {
            "rt_opts_default": [ctypes.POINTER(rt_opts)],
            "rt_create": [i, d, ctypes.POINTER(rt_pump), d, d, d, ctypes.POINTER(rt_opts), ctypes.POINTER(vp)],
            "rt_step": [vp, ll],
            "rt_sync": [vp],
            "rt_sweep": [vp, i],
            "rt_read_field": [vp, vp, sz],
            "rt_read_inversion": [vp, vp, sz],
            "rt_write_field": [vp, vp, sz],
            "rt_write_inversion": [vp, vp, sz],
            "rt_set_bounces": [vp, ll],
            "rt_stats": [vp, ctypes.POINTER(rt_stats_t)],
            "rt_read_history": [vp, vp, ll, ctypes.POINTER(ll)],
            "rt_read_spectrum": [vp, vp, sz],
            "rt_read_field_at": [vp, d, vp, sz],
            "rt_set_field_pattern": [vp, ctypes.POINTER(rt_pattern)],
            "rt_spectrum_peak": [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(d)],
            "rt_destroy": [vp],
            "rt_step_noalloc": [i, d, ctypes.POINTER(rt_pump), d, d, d, ctypes.POINTER(rt_opts), vp, vp, ll,
                                ctypes.POINTER(d)],
            "rt_job_default": [ctypes.POINTER(rt_job), i],
            "rt_batch_create": [ctypes.POINTER(rt_job), i, ctypes.POINTER(rt_opts), ctypes.POINTER(vp)],
            "rt_batch_step": [vp, ll],
            "rt_batch_sweep": [vp, i],
            "rt_batch_set_job": [vp, i, ctypes.POINTER(rt_job), ll],
            "rt_batch_sync": [vp],
            "rt_batch_read_field": [vp, i, vp, sz],
            "rt_batch_read_inversion": [vp, i, vp, sz],
            "rt_batch_write_field": [vp, i, vp, sz],
            "rt_batch_write_inversion": [vp, i, vp, sz],
            "rt_batch_stats": [vp, i, ctypes.POINTER(rt_stats_t)],
            "rt_batch_read_history": [vp, i, vp, ll, ctypes.POINTER(ll)],
            "rt_batch_bounces": [vp, vp],
            "rt_batch_footprint": [vp, ctypes.POINTER(sz)],
            "rt_batch_destroy": [vp],
            "rt_serve_opts_default": [ctypes.POINTER(rt_serve_opts)],
            "rt_serve_create": [ctypes.POINTER(rt_serve_opts), ctypes.POINTER(vp)],
            "rt_serve_submit": [vp, ctypes.POINTER(rt_job), ll, vp, ctypes.POINTER(ll)],
            "rt_serve_poll": [vp, ctypes.POINTER(rt_result), i, ctypes.POINTER(i)],
            "rt_serve_cancel": [vp, ll],
            "rt_serve_drain": [vp, d],
            "rt_serve_stats": [vp, ctypes.POINTER(rt_serve_stats_t)],
            "rt_serve_destroy": [vp],
            "rt_debug_fail_alloc": [i],
            "rt_debug_fail_alloc_n": [i, i],
            "rt_debug_wait_probe": [i, ctypes.POINTER(i)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.rt_status_string.argtypes = [ctypes.c_int]
        L.rt_status_string.restype = ctypes.c_char_p
        L.rt_version.restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(s: int) -> str:
    try:
        return lib().rt_status_string(s).decode()
    except ImportError:
        return "library not loaded"


def _check(status: int, where: str):
    if status != RT_OK:
        raise RtError(status, where)


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError("expected a numpy array or a torch tensor")


def _nbytes(a) -> int:
    return a.nbytes if isinstance(a, np.ndarray) else a.numel() * a.element_size()


# ----------------------------------------------------------------- C-named API

def rt_version() -> int:
    return lib().rt_version()


def rt_opts_default() -> rt_opts:
    o = rt_opts()
    _check(lib().rt_opts_default(ctypes.byref(o)), "rt_opts_default")
    return o


def rt_create(n: int, fresnel: float, pump: rt_pump | None, g0: float, T1: float, R: float,
              opts: rt_opts | None = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().rt_create(n, fresnel, ctypes.byref(pump) if pump is not None else None, g0, T1, R,
                           ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)), "rt_create")
    return h


def rt_step(h, n_bounces: int):
    _check(lib().rt_step(h, int(n_bounces)), "rt_step")


def rt_sync(h):
    _check(lib().rt_sync(h), "rt_sync")


RT_SWEEP_COLUMNS, RT_SWEEP_ROWS = 0, 1


def rt_sweep(h, which: int):
    _check(lib().rt_sweep(h, which), "rt_sweep")


def rt_read_field(h, dst):
    _check(lib().rt_read_field(h, _ptr(dst), _nbytes(dst)), "rt_read_field")
    return dst


def rt_read_inversion(h, dst):
    _check(lib().rt_read_inversion(h, _ptr(dst), _nbytes(dst)), "rt_read_inversion")
    return dst


def rt_write_field(h, src):
    _check(lib().rt_write_field(h, _ptr(src), _nbytes(src)), "rt_write_field")


def rt_write_inversion(h, src):
    _check(lib().rt_write_inversion(h, _ptr(src), _nbytes(src)), "rt_write_inversion")


def rt_set_bounces(h, bounces: int):
    _check(lib().rt_set_bounces(h, int(bounces)), "rt_set_bounces")


def rt_stats(h) -> rt_stats_t:
    s = rt_stats_t()
    _check(lib().rt_stats(h, ctypes.byref(s)), "rt_stats")
    return s


def rt_read_history(h, max_values: int) -> np.ndarray:
    out = np.zeros(max(int(max_values), 0), np.float64)
    got = ctypes.c_longlong()
    _check(lib().rt_read_history(h, out.ctypes.data if out.size else None, out.size, ctypes.byref(got)),
           "rt_read_history")
    return out[: got.value]


def rt_read_spectrum(h, dst):
    _check(lib().rt_read_spectrum(h, _ptr(dst), _nbytes(dst)), "rt_read_spectrum")
    return dst


def rt_debug_fail_alloc(after: int):
    """Test hook: the after-th device allocation from now on fails once (-1 cancels)."""
    _check(lib().rt_debug_fail_alloc(int(after)), "rt_debug_fail_alloc")


def rt_debug_fail_alloc_n(after: int, count: int):
    """Fault injection (test hook): `count` consecutive device allocations
    starting with the after-th fail as out of memory (count < 0: all of them)."""
    _check(lib().rt_debug_fail_alloc_n(int(after), int(count)), "rt_debug_fail_alloc_n")


def rt_debug_wait_probe(drain: bool = False) -> int:
    """Test hook: run the sweeps' bounded copy wait on a barrier that no copy
    completes; returns the device error word once the wait has given up
    (RT_ETIMEOUT expected)."""
    st = ctypes.c_int()
    _check(lib().rt_debug_wait_probe(1 if drain else 0, ctypes.byref(st)), "rt_debug_wait_probe")
    return st.value


def rt_set_field_pattern(h, pattern: rt_pattern):
    _check(lib().rt_set_field_pattern(h, ctypes.byref(pattern)), "rt_set_field_pattern")


def rt_read_field_at(h, zeta: float, dst):
    _check(lib().rt_read_field_at(h, float(zeta), _ptr(dst), _nbytes(dst)), "rt_read_field_at")
    return dst


def rt_spectrum_peak(h, ring: int = 0):
    mx, my, pw = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().rt_spectrum_peak(h, ring, ctypes.byref(mx), ctypes.byref(my), ctypes.byref(pw)),
           "rt_spectrum_peak")
    return mx.value, my.value, pw.value


def rt_destroy(h):
    _check(lib().rt_destroy(h), "rt_destroy")


RT_NOALLOC_MAX_N = 4096


def rt_step_noalloc(n: int, fresnel: float, pump: rt_pump | None, g0: float, T1: float, R: float,
                    opts: rt_opts | None, field, inversion, n_bounces: int, wait: bool = True):
    """Allocation-free bounces on caller-owned device buffers (see include/rt.h):
    `field` and `inversion` are contiguous CUDA tensors (complex64 / float32,
    n x n) updated in place.  With wait=True returns the mean intensity after
    the last bounce; with wait=False returns None without synchronising."""
    mean = ctypes.c_double()
    _check(lib().rt_step_noalloc(n, fresnel, ctypes.byref(pump) if pump is not None else None, g0, T1, R,
                                 ctypes.byref(opts) if opts is not None else None, _ptr(field), _ptr(inversion),
                                 int(n_bounces), ctypes.byref(mean) if wait else None), "rt_step_noalloc")
    return mean.value if wait else None


# --------------------------------------------------------- convenience wrapper

class Resonator:
    """One resonator handle with numpy-returning readouts.

    ``Resonator(n, fresnel, g0, T1, R, precision=RT_FP32, **opts)``; keyword
    options are the rt_opts fields (Isat, edge_px, seed, noise_amp,
    pump_diam_over_window, cuda_stream, history_cap, chunk, col_tile,
    z_over_F) plus pump_kind, pump_order, pump_radius, pump_profile and
    roughness (an n x n array of the mirror's phase psi in radians).
    """

    def __init__(self, n, fresnel, g0, T1, R, precision=RT_FP32, pump_kind=RT_PUMP_SUPERGAUSS,
                 pump_order=10.0, pump_radius=0.8, pump_profile=None, roughness=None, **opts):
        o = rt_opts_default()
        o.precision = precision
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        psi = None
        if roughness is not None:
            psi = np.ascontiguousarray(roughness, np.float64).reshape(n, n)
            o.roughness = psi.ctypes.data
        self._profile = None
        p = rt_pump(kind=pump_kind, order=pump_order, radius=pump_radius, profile=None)
        if pump_kind == RT_PUMP_ARRAY:
            self._profile = np.ascontiguousarray(pump_profile, np.float64).reshape(n, n)
            p.profile = self._profile.ctypes.data
        self.n = n
        self.slices = max(o.slices, 1)
        self.precision = precision
        self.cdtype = np.complex128 if precision == RT_FP64 else np.complex64
        self.rdtype = np.float64 if precision == RT_FP64 else np.float32
        self.h = rt_create(n, fresnel, p, g0, T1, R, o)  # psi is copied by rt_create

    @classmethod
    def from_params(cls, p, precision=RT_FP32, **opts):
        """From a workloads.Resonator parameter record."""
        return cls(p.n, p.fresnel, p.g0, p.T1, p.R, precision=precision, pump_order=p.pump_order,
                   pump_radius=p.pump_radius, Isat=p.Isat, edge_px=p.edge, seed=p.seed, noise_amp=p.noise_amp,
                   pump_diam_over_window=p.d_over_w, z_over_F=p.z_over_F, roughness=p.roughness(),
                   taper_px=p.taper_px, relax=p.relax, **opts)

    def step(self, n_bounces: int):
        rt_step(self.h, n_bounces)
        return self

    def sync(self):
        rt_sync(self.h)

    def field(self) -> np.ndarray:
        return rt_read_field(self.h, np.empty((self.n, self.n), self.cdtype))

    def inversion(self) -> np.ndarray:
        """n x n, or slices x n x n for a sliced gain medium."""
        shape = (self.n, self.n) if self.slices == 1 else (self.slices, self.n, self.n)
        return rt_read_inversion(self.h, np.empty(shape, self.rdtype))

    def set_field(self, E):
        rt_write_field(self.h, np.ascontiguousarray(E, self.cdtype))
        rt_sync(self.h)

    def set_inversion(self, N):
        rt_write_inversion(self.h, np.ascontiguousarray(N, self.rdtype))
        rt_sync(self.h)

    def spectrum(self) -> np.ndarray:
        return rt_read_spectrum(self.h, np.empty((self.n, self.n), self.rdtype))

    def set_pattern(self, kind, width, periods=1, out_of_phase=False, envelope=0.0, curvature=0.0, amplitude=1.0):
        """Replace the field with a structured field (rt_set_field_pattern)."""
        rt_set_field_pattern(self.h, rt_pattern(kind=kind, periods=periods, out_of_phase=int(bool(out_of_phase)),
                                                width=width, envelope=envelope, curvature=curvature,
                                                amplitude=amplitude))
        rt_sync(self.h)

    def field_at(self, zeta: float) -> np.ndarray:
        """The field diffracted a further zeta bounces' distance (intracavity plane)."""
        return rt_read_field_at(self.h, zeta, np.empty((self.n, self.n), self.cdtype))

    def peak(self, ring: int = 0):
        return rt_spectrum_peak(self.h, ring)

    def stats(self) -> rt_stats_t:
        return rt_stats(self.h)

    def history(self, max_values: int) -> np.ndarray:
        return rt_read_history(self.h, max_values)

    def close(self):
        if self.h:
            rt_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batches

def rt_job_default(n: int) -> rt_job:
    j = rt_job()
    _check(lib().rt_job_default(ctypes.byref(j), n), "rt_job_default")
    return j


def job_from_params(p) -> rt_job:
    """rt_job from a workloads.Resonator parameter record (super-Gaussian
    pump).  A roughness array is referenced, not copied: the record's job
    keeps it alive (``job._psi``) until the library has copied it."""
    j = rt_job_default(p.n)
    j.fresnel, j.g0, j.T1, j.R = p.fresnel, p.g0, p.T1, p.R
    j.pump = rt_pump(kind=RT_PUMP_SUPERGAUSS, order=p.pump_order, radius=p.pump_radius, profile=None)
    j.Isat, j.edge_px, j.seed, j.noise_amp, j.pump_diam_over_window = p.Isat, p.edge, p.seed, p.noise_amp, p.d_over_w
    j.z_over_F, j.taper_px, j.relax = p.z_over_F, p.taper_px, p.relax
    psi = p.roughness()
    if psi is not None:
        j._psi = np.ascontiguousarray(psi, np.float64)
        j.roughness = j._psi.ctypes.data
    return j


class Batch:
    """Resonators stepped together (C ABI rt_batch_*): ``Batch(jobs, **opts)``
    with jobs a list of rt_job or workloads.Resonator records; options are
    rt_opts fields (cuda_stream, history_cap, chunk, col_tile)."""

    def __init__(self, jobs, **opts):
        js = [j if isinstance(j, rt_job) else job_from_params(j) for j in jobs]
        self.n = [j.n for j in js]
        arr = (rt_job * len(js))(*js)
        o = rt_opts_default()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        self.h = ctypes.c_void_p()
        _check(lib().rt_batch_create(arr, len(js), ctypes.byref(o), ctypes.byref(self.h)), "rt_batch_create")

    def __len__(self):
        return len(self.n)

    def step(self, n_bounces: int):
        _check(lib().rt_batch_step(self.h, int(n_bounces)), "rt_batch_step")
        return self

    def sweep(self, which: int):
        _check(lib().rt_batch_sweep(self.h, which), "rt_batch_sweep")

    def set_job(self, i: int, job, n_bounces: int = -1):
        j = job if isinstance(job, rt_job) else job_from_params(job)
        _check(lib().rt_batch_set_job(self.h, i, ctypes.byref(j), int(n_bounces)), "rt_batch_set_job")

    def sync(self):
        _check(lib().rt_batch_sync(self.h), "rt_batch_sync")

    def field(self, i: int) -> np.ndarray:
        out = np.empty((self.n[i], self.n[i]), np.complex64)
        _check(lib().rt_batch_read_field(self.h, i, out.ctypes.data, out.nbytes), "rt_batch_read_field")
        return out

    def inversion(self, i: int) -> np.ndarray:
        out = np.empty((self.n[i], self.n[i]), np.float32)
        _check(lib().rt_batch_read_inversion(self.h, i, out.ctypes.data, out.nbytes), "rt_batch_read_inversion")
        return out

    def write_field(self, i: int, src):
        src = src if not isinstance(src, np.ndarray) else np.ascontiguousarray(src, np.complex64)
        _check(lib().rt_batch_write_field(self.h, i, _ptr(src), _nbytes(src)), "rt_batch_write_field")

    def write_inversion(self, i: int, src):
        src = src if not isinstance(src, np.ndarray) else np.ascontiguousarray(src, np.float32)
        _check(lib().rt_batch_write_inversion(self.h, i, _ptr(src), _nbytes(src)), "rt_batch_write_inversion")

    def stats(self, i: int) -> rt_stats_t:
        s = rt_stats_t()
        _check(lib().rt_batch_stats(self.h, i, ctypes.byref(s)), "rt_batch_stats")
        return s

    def history(self, i: int, max_values: int) -> np.ndarray:
        out = np.zeros(max(int(max_values), 0), np.float64)
        got = ctypes.c_longlong()
        _check(lib().rt_batch_read_history(self.h, i, out.ctypes.data if out.size else None, out.size,
                                           ctypes.byref(got)), "rt_batch_read_history")
        return out[: got.value]

    def bounces(self) -> np.ndarray:
        out = np.zeros(len(self.n), np.int64)
        _check(lib().rt_batch_bounces(self.h, out.ctypes.data), "rt_batch_bounces")
        return out

    def footprint(self) -> int:
        b = ctypes.c_size_t()
        _check(lib().rt_batch_footprint(self.h, ctypes.byref(b)), "rt_batch_footprint")
        return b.value

    def close(self):
        if self.h:
            lib().rt_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving

def rt_serve_opts_default() -> rt_serve_opts:
    o = rt_serve_opts()
    _check(lib().rt_serve_opts_default(ctypes.byref(o)), "rt_serve_opts_default")
    return o


class Server:
    """Continuous-batching server (C ABI rt_serve_*).  ``Server(**opts)`` with
    rt_serve_opts fields (budget_bytes, chunk, max_per_size, cuda_stream,
    policy, round_points)."""

    def __init__(self, **opts):
        o = rt_serve_opts_default()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        self.h = ctypes.c_void_p()
        _check(lib().rt_serve_create(ctypes.byref(o), ctypes.byref(self.h)), "rt_serve_create")
        self._keep = {}

    def submit(self, job, n_bounces: int, field_out=None) -> int:
        """Queue a request; field_out (numpy complex64 n x n or a device
        tensor) receives the final field."""
        j = job if isinstance(job, rt_job) else job_from_params(job)
        if field_out is not None and _nbytes(field_out) != j.n * j.n * 8:
            # the library writes n*n complex64 values there, later, from its worker
            raise ValueError(f"field_out must hold {j.n}x{j.n} complex64 values")
        rid = ctypes.c_longlong()
        _check(lib().rt_serve_submit(self.h, ctypes.byref(j), int(n_bounces),
                                     _ptr(field_out) if field_out is not None else None, ctypes.byref(rid)),
               "rt_serve_submit")
        if field_out is not None:
            self._keep[rid.value] = field_out
        return rid.value

    def cancel(self, request_id: int):
        """Cancel a queued or running request (its result is posted with RT_ECANCELED)."""
        _check(lib().rt_serve_cancel(self.h, int(request_id)), "rt_serve_cancel")

    def poll(self, max_results: int = 1024):
        buf = (rt_result * max_results)()
        got = ctypes.c_int()
        _check(lib().rt_serve_poll(self.h, buf, max_results, ctypes.byref(got)), "rt_serve_poll")
        out = [buf[k] for k in range(got.value)]
        for r in out:
            self._keep.pop(r.id, None)
        return out

    def drain(self, timeout_s: float = 600.0):
        _check(lib().rt_serve_drain(self.h, float(timeout_s)), "rt_serve_drain")

    def stats(self) -> rt_serve_stats_t:
        s = rt_serve_stats_t()
        _check(lib().rt_serve_stats(self.h, ctypes.byref(s)), "rt_serve_stats")
        return s

    def close(self):
        if self.h:
            lib().rt_serve_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
