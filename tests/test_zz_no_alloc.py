"""rt_step_noalloc gives the same bounces as the handle path.

Some callers cannot call cudaMalloc: a plugin whose host framework owns all
device memory and hands out buffers from its own pool, or a latency-critical
loop where an allocation could synchronise the device.  rt_step_noalloc
serves them: it runs on buffers the caller already owns and keeps its
scratch in a fixed device array inside the library.  This test drives it
through the C ABI and checks two calls in a row against rt_step on a
resonator handle started from the same state, within the FP32 parity
tolerance used by the other GPU tests.
"""
import numpy as np
import pytest

from paper_1410_2855_gb300 import build, rt, workloads as wl

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n, fresnel, g0, T1, R, z_over_F, taper_px, relax",
                         [(256, 100.0, 0.3, 1000.0, 0.9, 0.0, 0, 0),
                          (256, 100.0, 0.3, 1000.0, 0.9, 0.3, 5, 1),
                          (2048, 1000.0, 0.3, 1e4, 0.9, 0.0, 0, 0),
                          (4096, 4000.0, 0.3, 1e4, 0.9, 0.0, 0, 0)])      # RT_NOALLOC_MAX_N
def test_noalloc_matches_handle_path_on_two_calls(n, fresnel, g0, T1, R, z_over_F, taper_px, relax):
    import torch

    build.build()
    E0 = wl.smooth_field(n, 21, 1.0, dtype=np.complex64)
    with rt.Resonator(n, fresnel, g0, T1, R, chunk=0, z_over_F=z_over_F, taper_px=taper_px, relax=relax) as ref:
        N0 = ref.inversion()
        ref.set_field(E0)
        # Buffers owned by the caller (here allocated by the test, not by the entry point).
        E_dev = torch.from_numpy(E0.view(np.float32).copy()).cuda()
        N_dev = torch.from_numpy(N0.copy()).cuda()
        opts = rt.rt_opts_default()
        opts.cuda_stream = torch.cuda.current_stream().cuda_stream
        # a curved mirror and a taper need only per-axis factors: no allocation
        opts.z_over_F, opts.taper_px, opts.relax = z_over_F, taper_px, relax
        for nb in (7, 5):
            ref.step(nb)
            mean = rt.rt_step_noalloc(n, fresnel, None, g0, T1, R, opts, E_dev, N_dev, nb)
            E_ref, N_ref = ref.field(), ref.inversion()
            E = E_dev.cpu().numpy().view(np.complex64).reshape(n, n)
            N = N_dev.cpu().numpy()
            assert rel(E, E_ref) <= TOL
            assert float(np.linalg.norm(N - N_ref) / np.linalg.norm(N_ref)) <= TOL
            ref_mean = ref.stats().mean_intensity
            assert abs(mean - ref_mean) <= TOL * ref_mean


def test_error_of_an_asynchronous_call_reaches_the_next_synchronous_call():
    # An Inf in the caller's field makes the mean intensity non-finite.  The
    # asynchronous call (no host pointer for the mean) cannot report it; the
    # next synchronous call does, once, and the call after that is clean.
    import torch

    build.build()
    n = 64
    E = np.ones((n, n), np.complex64)
    E[n // 2, n // 2] = np.inf
    E_dev = torch.from_numpy(E.view(np.float32).copy()).cuda()
    N_dev = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    opts = rt.rt_opts_default()
    opts.cuda_stream = torch.cuda.current_stream().cuda_stream
    rt.rt_step_noalloc(n, 50.0, None, 0.2, 100.0, 0.95, opts, E_dev, N_dev, 1, wait=False)
    with pytest.raises(rt.RtError) as ei:
        rt.rt_step_noalloc(n, 50.0, None, 0.2, 100.0, 0.95, opts, E_dev, N_dev, 0)
    assert ei.value.status == rt.RT_ENUMERIC
    E_dev.copy_(torch.from_numpy(np.ones((n, n), np.complex64).view(np.float32)))
    N_dev.zero_()
    mean = rt.rt_step_noalloc(n, 50.0, None, 0.2, 100.0, 0.95, opts, E_dev, N_dev, 1)
    assert np.isfinite(mean) and mean > 0
