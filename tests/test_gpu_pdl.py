"""Programmatic dependent launch changes when the library's kernels start, not
what they compute.  Each kernel begins with griddepcontrol.wait, so a step
launched with programmatic stream serialization (the default) and one launched
without it (NS_PDL=0, read once per process, hence the subprocesses) give the
same records and image bit for bit; the gradients are sums of atomic additions
whose order varies from run to run, so they agree within that rounding."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import scenes
from gpu_util import run_step
sc = scenes.small_closed(351, n_curves=4, size=64, filled="alternate", h=1.0).with_raster(tile=8, fill_layers=1)
out = run_step(sc)
G = out["G"]
np.savez({out!r}, image=out["image"], rec=out["sp"].rec[:G].cpu().numpy(), dkey=out["dkey"],
         dtau=out["dtau"], dcolor=out["dcolor"], loss=np.array([out["loss"]]))
"""


def _step(tmp_path, pdl):
    out = str(tmp_path / f"step_pdl{pdl}.npz")
    env = dict(os.environ, NS_PDL=str(pdl))
    code = SCRIPT.format(root=ROOT, tests=os.path.join(ROOT, "tests"), out=out)
    subprocess.run([sys.executable, "-c", code], env=env, check=True, timeout=600)
    return np.load(out)


def _rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_step_same_with_and_without_pdl(tmp_path):
    on = _step(tmp_path, 1)
    off = _step(tmp_path, 0)
    assert np.array_equal(on["rec"], off["rec"])
    assert np.array_equal(on["image"], off["image"])
    assert abs(float(on["loss"][0]) - float(off["loss"][0])) <= 1e-6 * abs(float(off["loss"][0]))
    for nm in ("dkey", "dtau", "dcolor"):
        assert _rel(on[nm], off[nm]) <= 1e-5, nm
