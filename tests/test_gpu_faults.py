"""Failure paths, injected on the host: with MF_FAULT_INJECT=alloc every
device allocation of the library fails, and each entry point that needs one
must return MF_ERR_ALLOC with a message, leave the device usable, and work
again once the injection is lifted.  Runs in a child process so the
injection never leaks into other tests."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, os, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_2507_19926_gb300 as mf
from paper_2507_19926_gb300 import synth
mf.load_library()
res = {}
x = torch.from_numpy(synth.uniform((64, 80), "u8", 1)).cuda()
y = torch.empty_like(x)
d = mf.ImageDesc(x.data_ptr(), y.data_ptr(), 64, 80, 80, 1, mf.MF_U8, 5)
def status(f):
    try:
        f(); return "ok"
    except mf.MedianFilterError as e:
        return str(e)
os.environ["MF_FAULT_INJECT"] = "alloc"
res["batch"] = status(lambda: mf.mf_batch_plan_create([d]))
h = np.zeros((64, 80), np.uint8)
h2 = np.zeros((64, 80), np.uint8)
res["host"] = status(lambda: mf.mf_median_filter_host(h.ctypes.data, h2.ctypes.data, 64, 80, 80, 1, 0, 5))
res["data_aware"] = status(lambda: mf.median_filter(x, 41, variant="data_aware"))
res["device_ok_during"] = status(lambda: mf.median_filter(x, 5, variant="oblivious"))
del os.environ["MF_FAULT_INJECT"]
res["batch_after"] = status(lambda: mf.mf_batch_plan_destroy(mf.mf_batch_plan_create([d])))
res["data_aware_after"] = status(lambda: mf.median_filter(x, 41, variant="data_aware"))
torch.cuda.synchronize()
print(json.dumps(res))
'''


def test_injected_allocation_failures():
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["batch"].startswith("allocation failed"), res
    assert res["host"].startswith("allocation failed"), res
    assert res["data_aware"].startswith("allocation failed"), res
    assert res["device_ok_during"] == "ok"
    assert res["batch_after"] == "ok" and res["data_aware_after"] == "ok"


def test_autotune_cache_roundtrip(tmp_path):
    """mf_autotune records the fastest candidate in the JSON cache named by
    MF_TUNE_CACHE; a new process reads it back and dispatches to it."""
    cache = tmp_path / "tune.jsonl"
    code = r'''
import sys; sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_2507_19926_gb300 as mf
from paper_2507_19926_gb300 import synth
x = torch.from_numpy(synth.uniform((512, 512), "u8", 2)).cuda(); y = torch.empty_like(x)
if sys.argv[2] == "tune":
    mf.mf_autotune(x.data_ptr(), y.data_ptr(), 512, 512, 512, 1, mf.MF_U8, 27)
print(mf.mf_describe(512, 512, 1, mf.MF_U8, 27))
'''
    env = dict(os.environ, MF_TUNE_CACHE=str(cache))
    a = subprocess.run([sys.executable, "-c", code, ROOT, "tune"], capture_output=True, text=True, env=env, timeout=300)
    assert a.returncode == 0, a.stderr[-2000:]
    lines = cache.read_text().strip().splitlines()
    assert lines and json.loads(lines[-1])["k"] == 27
    assert json.loads(lines[-1])["bucket"] == 9  # 512 x 512: floor(log2(2^18) / 2)
    b = subprocess.run([sys.executable, "-c", code, ROOT, "read"], capture_output=True, text=True, env=env, timeout=300)
    assert b.returncode == 0 and b.stdout.strip().splitlines()[-1] == a.stdout.strip().splitlines()[-1]
