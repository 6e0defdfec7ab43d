"""The bench's reference arm (CPU: the FP64 oracle on the line's workload)
prints one JSON line with the keys of the bench contract and honours
--steps and --warmup; and the input recipes have the sizes and order
fractions they state."""
import json
import os
import subprocess
import sys

import numpy as np

from paper_2311_11348_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "32",
                          "--steps", "3", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["impl"] == "reference" and line["unit"] == "DOF-stage/s" and line["value"] > 0
    assert line["steps"] == 3 and line["warmup"] == 3 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and 1 <= cb["cores"] <= cb["nproc"] == (os.cpu_count() or 1)
    assert cb["cpu_model"] and cb["value"] == line["value"]
    assert set(line["config"]) == {"workload", "triangles", "dof_stage_per_step", "l2", "replicas"}
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["triangles"] == 2 * 32 * 32


def test_dam_break_recipe_fractions():
    for nth, frac in ((0, 0.0), (64, 1 / 64), (32, 1 / 32), (1, 1.0)):
        w = inputs.dam_break_p12(64, nth)
        assert len(w["tri"]) == 2 * 64 * 64
        assert set(np.unique(w["orders"])) <= {1, 2}
        assert abs(np.mean(w["orders"] == 2) - frac) < 1e-3
    xi = inputs.dam_break_p12(16, 0)["ic"](np.array([5e3, 0.0]), np.array([5e3, 0.0]))[0]
    assert abs(xi[0] - 1.0) < 1e-12 and abs(xi[1]) < 1e-12  # the dam holds 1 m inside, nothing outside
