"""The debug build (-DDPSR_DEBUG_CHECKS): its index checks fire on an
out-of-range index without touching memory outside the allocation (the
self-test), raise no false alarm on valid solves on either plane path, and
leave the results equal to the oracle's; the release build has the checks
compiled away."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, "tests")
import oracle
from paper_2106_03452_gb300 import synth, libdpsr as L
from gpu_util import gpu_fwd_bwd, relmax
out = {"enabled": L.dpsr_debug_checks(), "selftest": L.dpsr_debug_check_selftest()}
rng = synth.Rng(77)
pts = (rng.uniform(700, 3) * 1.4 - 0.2).astype(np.float32)
nrm = rng.normal(700, 3).astype(np.float32)
w = synth.workload_ellipsoids_r128()
cases = [(32, 2.0, pts, nrm), (64, 1.5, pts, nrm), (128, 2.0, w["points"], w["normals"])]
res = []
for r, sigma, p, n in cases:
    g = gpu_fwd_bwd(r, sigma, p, n, synth.Rng(r).normal(r, r, r).astype(np.float32))
    ref = oracle.forward(r, sigma, p.astype(np.float64), n.astype(np.float64))
    res.append({"r": r, "status": g["status"], "bstatus": g["bstatus"], "chi": relmax(g["chi"], ref)})
out["cases"] = res
print(json.dumps(out))
"""


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_03452_gb300 import build
    build.build()
    build.build(debug=True)


@pytest.mark.parametrize("path", ["0", "1", "split"])
def test_debug_build_checks(path):
    env = dict(os.environ, DPSR_DEBUG_CHECKS="1", DPSR_PLANE_PATH="1" if path == "split" else path,
               PYTHONPATH=ROOT)
    if path == "split":  # one-CTA planes, the adjoint kind split by channel where it exists
        env.update(DPSR_PLANE_PATHS_64="1,1,1,3", DPSR_PLANE_PATHS_128="1,1,1,3")
    res = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    from paper_2106_03452_gb300 import libdpsr as L
    assert out["enabled"] == 1
    assert out["selftest"] == L.DPSR_EBOUNDS
    for c in out["cases"]:
        assert c["status"] == 0 and c["bstatus"] == 0, c     # no false alarm
        assert c["chi"] <= 1e-5, c


def test_release_build_has_no_checks():
    from paper_2106_03452_gb300 import libdpsr as L
    if L._DEBUG:
        pytest.skip("this process loaded the debug build")
    assert L.dpsr_debug_checks() is False
    assert L.dpsr_debug_check_selftest() == L.DPSR_OK
