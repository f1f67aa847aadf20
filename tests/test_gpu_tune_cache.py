"""The persisted autotuner cache (DPSR_TUNE_CACHE): a first process records
its plane-path choices as JSON Lines, a second process on the same device
uses the recorded choices without timing, and lines it does not own (other
devices, text it cannot parse) survive a rewrite. Each process is a fresh
interpreter so that nothing is cached in memory between them."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SOLO = r"""
import json, sys, torch
from paper_2106_03452_gb300 import synth, libdpsr as L
from paper_2106_03452_gb300.dpsr import Plan
w = synth.workload_sphere_r32()
r = 64
plan = Plan(r, 2.0)
P = torch.from_numpy(w["points"]).cuda(); N = torch.from_numpy(w["normals"]).cuda()
plan.forward(P, N)
plan.backward(torch.ones((r, r, r), device="cuda"))
assert plan.sync() == 0
print(json.dumps(L.dpsr_plan_clusters(plan.handle)))
"""

BATCH = r"""
import json, torch
from paper_2106_03452_gb300 import synth
from paper_2106_03452_gb300.dpsr import Batch
w = synth.workload_sphere_r32()
r, n = 64, 3
b = Batch([r] * n, [2.0] * n, [len(w["points"])] * n)
keep = []
for i in range(n):
    P = torch.from_numpy(w["points"]).cuda(); N = torch.from_numpy(w["normals"]).cuda()
    chi = torch.empty((r, r, r), device="cuda"); d = torch.ones((r, r, r), device="cuda")
    dp = torch.empty_like(P); dn = torch.empty_like(P)
    b.bind(i, P, N, chi, d, dp, dn); keep.append((P, N, chi, d, dp, dn))
b.run(with_bwd=True, graph=False)
torch.cuda.synchronize()
print(json.dumps(b.paths(r)))
"""


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_03452_gb300 import build
    build.build()


def _run(code, cache):
    env = dict(os.environ, DPSR_TUNE_CACHE=str(cache), PYTHONPATH=ROOT)
    env.pop("DPSR_PLANE_PATH", None)
    env.pop("DPSR_TUNE", None)
    res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-3000:]
    return json.loads(res.stdout.strip().splitlines()[-1])


def _lines(cache):
    with open(cache) as f:
        return [l.rstrip("\n") for l in f if l.strip()]


def test_solo_choices_persist_and_are_reused(tmp_path):
    cache = tmp_path / "tune.jsonl"
    first = _run(SOLO, cache)
    ent = [json.loads(l) for l in _lines(cache)]
    mine = {e["kind"]: e for e in ent if e["r"] == 64 and e["batch"] == 0}
    assert sorted(mine) == [0, 1, 2, 3]
    assert [mine[k]["path"] for k in range(4)] == first
    key = {k: ent[0][k] for k in ("cc", "sms", "driver")}
    assert key["sms"] > 0 and key["cc"] >= 100
    # Keep three of the four choices, rewritten to the pencil passes (valid at
    # every r), and add a line of another device and a line that does not
    # parse. The second process reads the three back and tunes the fourth,
    # which rewrites the file.
    other = dict(ent[0], sms=key["sms"] + 1, path=8)
    with open(cache, "w") as f:
        for k in range(3):
            f.write(json.dumps(dict(mine[k], path=0, ms=0.0)) + "\n")
        f.write(json.dumps(other) + "\n")
        f.write("not json at all\n")
    second = _run(SOLO, cache)
    assert second[:3] == [0, 0, 0]           # read back, not re-timed
    lines = _lines(cache)
    assert "not json at all" in lines
    parsed = [json.loads(l) for l in lines if l != "not json at all"]
    keys = ("cc", "sms", "driver", "r", "kind", "batch", "path")
    assert any(all(e[k] == other[k] for k in keys) for e in parsed)
    now = {e["kind"]: e["path"] for e in parsed if e["sms"] == key["sms"] and e["r"] == 64 and e["batch"] == 0}
    assert [now[k] for k in range(4)] == second


def test_batch_choices_are_keyed_by_class_size(tmp_path):
    cache = tmp_path / "tune.jsonl"
    first = _run(BATCH, cache)
    ent = [json.loads(l) for l in _lines(cache)]
    mine = {e["kind"]: e["path"] for e in ent if e["r"] == 64 and e["batch"] == 3}
    assert sorted(mine) == [0, 1, 2, 3] and [mine[k] for k in range(4)] == first
    with open(cache, "w") as f:
        for e in ent:
            if e["batch"] == 3:
                e = dict(e, path=0)
            f.write(json.dumps(e) + "\n")
    assert _run(BATCH, cache) == [0, 0, 0, 0]
