"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
function include/rt.h declares, and its structures have the layout the
Python binding assumes.  Only host-side logic is exercised (no compute)."""
import ctypes
import os
import re
import subprocess
import textwrap

import pytest

from paper_1410_2855_gb300 import build, rt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rt.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return rt.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["rt_create", "rt_step", "rt_read_field", "rt_read_inversion", "rt_destroy",
                     "rt_write_field", "rt_write_inversion", "rt_stats", "rt_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(lib):
    assert rt.status_string(0) == "ok"
    assert rt.status_string(-1) == "invalid argument"
    assert rt.status_string(-4) == "non-finite field intensity"
    assert rt.rt_version() >= 100


def test_default_options(lib):
    o = rt.rt_opts_default()
    assert (o.Isat, o.edge_px, o.precision, o.seed, o.noise_amp) == (1.0, 8, 0, 14102855, 1e-6)
    assert o.pump_diam_over_window == 0.8 and o.history_cap == 65536 and o.chunk == 500
    assert o.z_over_F == 0.0 and not o.roughness


@pytest.mark.parametrize("args", [
    dict(n=100), dict(n=16), dict(n=8192), dict(fresnel=0.0), dict(fresnel=float("nan")),
    dict(g0=-0.1), dict(T1=0.5), dict(R=0.0), dict(R=1.5),
    # just past each end of the accepted ranges, and non-finite values
    dict(n=2 ** 13), dict(fresnel=-1.0), dict(fresnel=float("inf")), dict(g0=float("nan")), dict(g0=float("inf")),
    dict(T1=0.999999), dict(T1=float("inf")), dict(R=1.0 + 1e-12), dict(R=-0.5), dict(R=float("nan")),
])
def test_create_rejects_bad_arguments_before_touching_the_device(lib, args):
    p = dict(n=64, fresnel=100.0, g0=0.2, T1=1000.0, R=0.95)
    p.update(args)
    h = ctypes.c_void_p()
    st = lib.rt_create(p["n"], p["fresnel"], None, p["g0"], p["T1"], p["R"], None, ctypes.byref(h))
    assert st == rt.RT_EINVAL and not h.value


def test_create_rejects_bad_options(lib):
    h = ctypes.c_void_p()
    for field, value in [("precision", 3), ("edge_px", -1), ("edge_px", 33), ("Isat", 0.0), ("Isat", float("nan")),
                         ("Isat", float("inf")), ("noise_amp", -1e-6), ("noise_amp", float("nan")),
                         ("pump_diam_over_window", 0.0), ("history_cap", -5), ("chunk", -1),
                         ("z_over_F", float("inf")), ("z_over_F", float("nan")), ("slices", -1), ("slices", 65),
                         ("taper_px", -1), ("taper_px", 33), ("relax", 2)]:
        o = rt.rt_opts_default()
        setattr(o, field, value)
        assert lib.rt_create(64, 100.0, None, 0.2, 1000.0, 0.95, ctypes.byref(o), ctypes.byref(h)) == rt.RT_EINVAL
    p = rt.rt_pump(kind=rt.RT_PUMP_ARRAY, order=10.0, radius=0.8, profile=None)
    assert lib.rt_create(64, 100.0, ctypes.byref(p), 0.2, 1000.0, 0.95, None, ctypes.byref(h)) == rt.RT_EINVAL


def test_noalloc_rejects_oversize_and_unsupported_requests_on_the_host(lib):
    big = ctypes.c_void_p(16)
    assert lib.rt_step_noalloc(8192, 100.0, None, 0.2, 1000.0, 0.95, None, big, big, 1, None) == rt.RT_EINVAL
    o = rt.rt_opts_default()
    o.precision = rt.RT_FP64
    assert lib.rt_step_noalloc(64, 100.0, None, 0.2, 1000.0, 0.95, ctypes.byref(o), big, big, 1, None) == rt.RT_EINVAL
    assert lib.rt_step_noalloc(64, 100.0, None, 0.2, 1000.0, 0.95, None, None, big, 1, None) == rt.RT_EINVAL
    # A rough mirror needs an n x n table: not available without allocating.
    o = rt.rt_opts_default()
    psi = (ctypes.c_double * (64 * 64))()
    o.roughness = ctypes.cast(psi, ctypes.c_void_p)
    assert lib.rt_step_noalloc(64, 100.0, None, 0.2, 1000.0, 0.95, ctypes.byref(o), big, big, 1, None) == rt.RT_EINVAL


def test_concurrent_autotune_rejects_arguments_out_of_range(lib):
    t, o, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    f = lib.rt_autotune_concurrent
    f.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p] * 3
    args = (ctypes.byref(t), ctypes.byref(o), ctypes.byref(r))
    assert f(33, 2, 10, 1, *args) == rt.RT_EINVAL        # not a power of two
    assert f(8192, 2, 10, 1, *args) == rt.RT_EINVAL      # too large
    assert f(512, 0, 10, 1, *args) == rt.RT_EINVAL       # no resonators
    assert f(512, 17, 10, 1, *args) == rt.RT_EINVAL      # too many
    assert f(512, 2, 0, 1, *args) == rt.RT_EINVAL        # no bounces
    assert f(512, 2, 10, 0, *args) == rt.RT_EINVAL       # no timings
    assert f(512, 2, 10, 1, None, args[1], args[2]) == rt.RT_EINVAL


def test_batch_split_setting_is_checked(lib):
    assert lib.rt_tune_set_batch_split(9) == rt.RT_EINVAL
    assert lib.rt_tune_set_batch_split(-1) == rt.RT_EINVAL
    assert lib.rt_tune_get_batch_split(None) == rt.RT_EINVAL
    p = ctypes.c_int(-1)
    assert lib.rt_tune_set_batch_split(2) == rt.RT_OK
    assert lib.rt_tune_get_batch_split(ctypes.byref(p)) == rt.RT_OK and p.value == 2
    assert lib.rt_tune_set_batch_split(0) == rt.RT_OK


def test_null_handles_are_rejected(lib):
    assert lib.rt_step(None, 1) == rt.RT_EINVAL
    assert lib.rt_read_field_at(None, 0.5, None, 0) == rt.RT_EINVAL
    assert lib.rt_set_field_pattern(None, None) == rt.RT_EINVAL
    assert lib.rt_sync(None) == rt.RT_EINVAL
    assert lib.rt_read_field(None, None, 0) == rt.RT_EINVAL
    assert lib.rt_destroy(None) == rt.RT_OK


def test_struct_layouts_match_the_header(tmp_path, lib):
    src = tmp_path / "sizes.c"
    src.write_text(textwrap.dedent("""
        #include <stdio.h>
        #include <stddef.h>
        #include "rt.h"
        int main(void) {
            printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(rt_opts), sizeof(rt_pump), sizeof(rt_stats_t),
                   offsetof(rt_opts, chunk), offsetof(rt_stats_t, history_len), offsetof(rt_opts, cuda_stream));
            printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", offsetof(rt_opts, z_over_F), offsetof(rt_opts, roughness),
                   sizeof(rt_job), offsetof(rt_job, pump), offsetof(rt_job, z_over_F), offsetof(rt_job, roughness),
                   sizeof(rt_serve_opts), sizeof(rt_result));
            printf("%zu %zu\\n", sizeof(rt_serve_stats_t), offsetof(rt_serve_stats_t, peak_resident_bytes));
            return 0;
        }
    """))
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    want = [ctypes.sizeof(rt.rt_opts), ctypes.sizeof(rt.rt_pump), ctypes.sizeof(rt.rt_stats_t),
            rt.rt_opts.chunk.offset, rt.rt_stats_t.history_len.offset, rt.rt_opts.cuda_stream.offset,
            rt.rt_opts.z_over_F.offset, rt.rt_opts.roughness.offset, ctypes.sizeof(rt.rt_job), rt.rt_job.pump.offset,
            rt.rt_job.z_over_F.offset, rt.rt_job.roughness.offset, ctypes.sizeof(rt.rt_serve_opts),
            ctypes.sizeof(rt.rt_result), ctypes.sizeof(rt.rt_serve_stats_t),
            rt.rt_serve_stats_t.peak_resident_bytes.offset]
    assert got == want


def test_sliced_gain_medium_is_refused_where_unsupported(lib):
    # Batches, serving and the allocation-free entry run single-slice bounces.
    o = rt.rt_opts_default()
    o.slices = 2
    big = ctypes.c_void_p(16)
    assert lib.rt_step_noalloc(64, 100.0, None, 0.2, 1000.0, 0.95, ctypes.byref(o), big, big, 1, None) == rt.RT_EINVAL
    jobs = (rt.rt_job * 1)(rt.rt_job_default(64))
    h = ctypes.c_void_p()
    assert lib.rt_batch_create(jobs, 1, ctypes.byref(o), ctypes.byref(h)) == rt.RT_EINVAL and not h.value


def test_server_rejects_bad_options_before_touching_the_device(lib):
    h = ctypes.c_void_p()
    for field, value in [("policy", 7), ("round_points", -1), ("chunk", 0)]:
        o = rt.rt_serve_opts_default()
        setattr(o, field, value)
        assert lib.rt_serve_create(ctypes.byref(o), ctypes.byref(h)) == rt.RT_EINVAL and not h.value


def test_server_refuses_a_wrong_sized_output_buffer_before_calling_the_library():
    # The server writes n*n complex64 values into field_out from its worker
    # thread; the binding checks the size first (no device is touched).
    import numpy as np

    from paper_1410_2855_gb300 import workloads as wl
    srv = rt.Server.__new__(rt.Server)
    srv.h, srv._keep = None, {}
    n = wl.C2.n
    for bad in (np.zeros((n // 2, n), np.complex64), np.zeros((n, n), np.complex128), np.zeros((n, n), np.float32)):
        with pytest.raises(ValueError):
            srv.submit(wl.C2, 10, bad)
    assert srv._keep == {}


def test_job_from_params_carries_every_field(lib):
    # A workloads record with a distinct value in every field reaches the
    # C struct field for field; a rough mirror's phase array is referenced.
    import numpy as np

    from paper_1410_2855_gb300 import workloads as wl
    p = wl.Resonator(n=256, fresnel=123.0, g0=0.21, T1=4321.0, R=0.87, Isat=2.5, edge=5, pump_order=6.0,
                     pump_radius=0.55, d_over_w=0.7, seed=99, noise_amp=3e-6, z_over_F=0.12, roughness_rms=0.07,
                     roughness_corr=0.1, taper_px=4, relax=1)
    j = rt.job_from_params(p)
    assert (j.n, j.fresnel, j.g0, j.T1, j.R) == (256, 123.0, 0.21, 4321.0, 0.87)
    assert (j.pump.kind, j.pump.order, j.pump.radius) == (rt.RT_PUMP_SUPERGAUSS, 6.0, 0.55) and not j.pump.profile
    assert (j.Isat, j.edge_px, j.seed, j.noise_amp, j.pump_diam_over_window) == (2.5, 5, 99, 3e-6, 0.7)
    assert (j.z_over_F, j.taper_px, j.relax) == (0.12, 4, 1)
    assert j.roughness == j._psi.ctypes.data and np.array_equal(j._psi, p.roughness())
    smooth = rt.job_from_params(wl.Resonator(n=64, fresnel=10.0, g0=0.2, T1=100.0, R=0.9))
    assert not smooth.roughness


def test_resonator_from_params_passes_every_field():
    # The same record through Resonator.from_params: the constructor's
    # arguments are recorded (no device is touched) and must carry every field.
    import numpy as np

    from paper_1410_2855_gb300 import workloads as wl

    class Probe(rt.Resonator):
        def __init__(self, *args, **kw):
            self.args, self.kw, self.h = args, kw, None

    p = wl.Resonator(n=256, fresnel=123.0, g0=0.21, T1=4321.0, R=0.87, Isat=2.5, edge=5, pump_order=6.0,
                     pump_radius=0.55, d_over_w=0.7, seed=99, noise_amp=3e-6, z_over_F=0.12, roughness_rms=0.07,
                     roughness_corr=0.1, taper_px=4, relax=1)
    r = Probe.from_params(p, precision=rt.RT_FP64, chunk=7)
    assert r.args == (256, 123.0, 0.21, 4321.0, 0.87)
    kw = dict(r.kw)
    assert np.array_equal(kw.pop("roughness"), p.roughness())
    assert kw == dict(precision=rt.RT_FP64, pump_order=6.0, pump_radius=0.55, Isat=2.5, edge_px=5, seed=99,
                      noise_amp=3e-6, pump_diam_over_window=0.7, z_over_F=0.12, taper_px=4, relax=1, chunk=7)
