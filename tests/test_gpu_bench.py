"""bench.py's roofline sweep on the GPU at small sizes: one line per scheme,
storage and size, with throughput and HBM fraction that agree with the step
time."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_roofline_sweep_lines():
    r = subprocess.run([sys.executable, "bench.py", "--roofline-sweep", "256,512"], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [json.loads(l) for l in r.stdout.strip().splitlines()]
    rows, tail = lines[:-1], lines[-1]
    assert "clocks" in tail
    assert [(x["sweep"], x["n"]) for x in rows] == [(s, n) for n in (256, 512)
                                                    for s in ("st_f32", "st_bf16dev", "st_f16dev", "fv_f32")]
    for x in rows:
        assert x["cells"] == x["n"] ** 2 and x["bytes_per_cell"] == {"st_f32": 72, "fv_f32": 72}.get(x["sweep"], 36)
        assert x["mlups"] == pytest.approx(x["cells"] / (x["ms_per_step"] * 1e-3) / 1e6, rel=5e-3)
        frac = x["bytes_per_cell"] * x["mlups"] * 1e6 / 1e9 / x["peak"]
        assert x["frac_hbm"] == pytest.approx(frac, rel=1e-3, abs=2e-4) and 0 < x["frac_hbm"] < 1.2
