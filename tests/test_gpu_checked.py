"""Bounds-checked build: the library compiled with RTK_CHECKED=1 checks every
shared-memory access of the line FFT inside the bounce sweeps and records
RT_EBOUNDS in the sticky error word instead of touching memory outside the
line.  Running every sweep form through it (all grid sizes, column tiles,
radix orders, pump forms, aperture forms, slices, batches) must report no
violation and give the same fields as the normal build."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1410_2855_gb300 import build, rt, workloads as wl

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [  # (n, col_tile, kwargs); "order": the column transforms' radix order (tile from the tuner's record)
    (32, 16, {}), (64, 8, dict(z_over_F=0.3)), (128, 4, dict(taper_px=5, relax=1)), (256, 8, dict(roughness_rms=0.2)),
    (512, 16, dict(slices=2)), (1024, 4, {}), (2048, 4, dict(relax=1)), (2048, 2, {}), (4096, 2, {}),
    (64, 0, dict(order=1)), (512, 0, dict(order=1)), (512, 0, dict(order=2)), (1024, 0, dict(order=2)),
    (2048, 0, dict(order=1)), (2048, 0, dict(order=2)),
]

SCRIPT = r'''
import json, sys, dataclasses
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1410_2855_gb300 import rt, tune, workloads as wl
cases = json.loads(sys.argv[2])
out = {}
for i, (n, C, kw) in enumerate(cases):
    tune.rt_tune_set_order(n, kw.get("order", 0))
    opts = {k: v for k, v in kw.items() if k in ("slices",)}
    rec = {k: v for k, v in kw.items() if k not in ("slices", "order")}
    p = dataclasses.replace(wl.Resonator(n=n, fresnel=100.0 * n / 256, g0=0.3, T1=300.0, R=0.93, seed=40 + i), **rec)
    with rt.Resonator.from_params(p, chunk=0, col_tile=C, **opts) as r:
        r.set_field(wl.smooth_field(n, i, 1.0, dtype=np.complex64))
        r.step(3)
        r.sync()
        np.save(sys.argv[3] + f"/{i}.npy", r.field())
jobs = [wl.Resonator(n=s, fresnel=80.0, g0=0.25, T1=400.0, R=0.9, seed=70 + j, z_over_F=0.1 * (j % 2),
                     relax=j % 3 == 0) for j, s in enumerate((64, 128, 256, 128, 512))]
with rt.Batch(jobs, chunk=0) as b:
    b.step(3)
    b.sync()
    for j in range(len(jobs)):
        np.save(sys.argv[3] + f"/b{j}.npy", b.field(j))
print("ok")
'''


def test_checked_build_reports_no_violation_and_matches_the_normal_build(tmp_path):
    checked = build.build(extra_flags=["-DRTK_CHECKED=1"], tag="checked")
    script = tmp_path / "run.py"
    script.write_text(SCRIPT)
    outs = {}
    for name, lib in (("normal", build.build()), ("checked", checked)):
        d = tmp_path / name
        d.mkdir()
        env = dict(os.environ, RT_LIBRARY=lib)
        r = subprocess.run([sys.executable, str(script), ROOT, json.dumps(CASES), str(d)], env=env,
                           capture_output=True, text=True, timeout=900)
        assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr[-3000:]
        outs[name] = d
    for f in sorted(os.listdir(outs["normal"])):
        a, b = np.load(outs["normal"] / f), np.load(outs["checked"] / f)
        assert np.allclose(a, b, rtol=1e-6, atol=1e-6 * np.abs(a).max()), f
