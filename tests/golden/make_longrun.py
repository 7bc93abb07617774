"""Write tests/golden/longrun_512.json (flat mirror) or
tests/golden/longrun_512_curved.json (curved, rough mirror): the FP64
oracle's long run of the 512^2 resonator (N_F = 100, g0 = 0.15, T1 = 5000,
R = 0.95, super-Gaussian pump of order 10 and radius 0.8, 8-pixel edge,
splitmix64 noise start of amplitude 1e-6, 1e4 bounces; the curved case adds
z/F = 0.16 and the seeded 0.05 rad rms roughness of workloads.C2_CURVED).

Beyond a few tens of bounces the map is chaotic, so the stored values are
statistics that a faithful FP32 run must reproduce rather than the field
itself: the mean intensity averaged over the last 1000 bounces, the mean
intensity every 100 bounces, the dominant spatial frequency of the final
field (all bins, and bins with max(|mx|, |my|) >= 2), with m and -m folded,
and the spectrum's ring fractions: the share of the power |DFT2(E)|^2 in
each Chebyshev ring max(|mx|, |my|) = 0, [1, 2), [2, 4), ... of doubling
radius, at each of the ten snapshots 100 bounces apart that end the run, with
their mean over the snapshots and the largest distance of one snapshot from
that mean (the spread of a single sample of the attractor).

Calls only the oracle:  python tests/golden/make_longrun.py [flat|curved] [threads]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as orc  # noqa: E402
from paper_1410_2855_gb300 import workloads as wl  # noqa: E402


def ring_fractions(S):
    """Share of the spectral power in each Chebyshev ring of doubling radius
    (signed frequencies: ring 0 is the DC bin, ring k >= 1 holds
    2^(k-1) <= max(|mx|, |my|) < 2^k, the last ring includes n/2)."""
    n = S.shape[0]
    m = np.abs(np.fft.fftfreq(n, 1.0 / n)).astype(np.int64)
    rho = np.maximum(m[:, None], m[None, :])
    k = np.zeros_like(rho)
    nz = rho > 0
    k[nz] = np.floor(np.log2(rho[nz])).astype(np.int64) + 1
    k = np.minimum(k, int(np.log2(n // 2)))
    tot = float(S.sum())
    return [float(S[k == r].sum()) / tot for r in range(int(np.log2(n // 2)) + 1)]


def main():
    case = sys.argv[1] if len(sys.argv) > 1 else "flat"
    threads = int(sys.argv[2]) if len(sys.argv) > 2 else (os.cpu_count() or 1)
    c, nb = (wl.C2 if case == "flat" else wl.C2_CURVED), wl.C2_BOUNCES
    p = orc.make_params(c.n, orc.alpha_from_fresnel(c.fresnel, c.d_over_w), c.g0, c.T1, c.R, Isat=c.Isat,
                        edge=c.edge, pump_order=c.pump_order, pump_radius=c.pump_radius, z_over_F=c.z_over_F,
                        roughness=c.roughness())
    E, N = orc.init_state(p, c.seed, c.noise_amp)
    t0 = time.time()
    snaps, every = 10, 100
    E, N, hist = orc.run(p, E, N, nb - snaps * every, nthreads=threads)
    hists, fracs = [hist], []
    for _ in range(snaps):
        E, N, h = orc.run(p, E, N, every, nthreads=threads)
        hists.append(h)
        fracs.append(ring_fractions(orc.spectrum(E, nthreads=threads)))
    hist = np.concatenate(hists)
    fracs = np.array(fracs)
    S = orc.spectrum(E, nthreads=threads)
    peaks = {}
    for ring in (0, 2):
        mx, my, pw, ru = orc.spectrum_peak(S, ring)
        peaks[str(ring)] = {"mx": mx, "my": my, "power": pw, "runner_up": ru}
    out = {
        "_source": "FP64 oracle (oracle/bouncemap_oracle.c), written by tests/golden/make_longrun.py",
        "resonator": {"n": c.n, "fresnel": c.fresnel, "g0": c.g0, "T1": c.T1, "R": c.R, "Isat": c.Isat,
                      "edge": c.edge, "pump_order": c.pump_order, "pump_radius": c.pump_radius,
                      "d_over_w": c.d_over_w, "seed": c.seed, "noise_amp": c.noise_amp, "z_over_F": c.z_over_F,
                      "roughness_rms": c.roughness_rms, "roughness_corr": c.roughness_corr},
        "bounces": nb,
        "mean_intensity_last_1000": float(np.mean(hist[-1000:])),
        "mean_intensity_every_100": [float(v) for v in hist[99::100]],
        "final_mean_intensity": float(hist[-1]),
        "final_mean_inversion": float(np.mean(N)),
        "peaks": peaks,
        "ring_fractions": {"rings": "max(|mx|,|my|) = 0, [1,2), [2,4), ..., [n/4, n/2]",
                           "snapshot_bounces": [nb - snaps * every + every * (k + 1) for k in range(snaps)],
                           "snapshots": fracs.tolist(), "mean": fracs.mean(axis=0).tolist(),
                           "spread": np.abs(fracs - fracs.mean(axis=0)).max(axis=0).tolist()},
        "oracle_seconds": round(time.time() - t0, 1),
        "threads": threads,
    }
    name = "longrun_512.json" if case == "flat" else "longrun_512_curved.json"
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["mean_intensity_last_1000"], out["peaks"])


if __name__ == "__main__":
    main()
