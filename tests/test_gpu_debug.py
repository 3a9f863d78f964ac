"""The bounds-checked build (FIRERT_DEBUG, libfirert_debug.so) on the fit
paths: every launch shape and the ragged, small-table and five-endmember
cases run with all index checks on; no check may fail (device error word 0)
and the outputs must equal the release build's. The debug library runs in a
child process (a process loads one of the two builds)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
import numpy as np
sys.path.insert(0, os.environ["FR_ROOT"]); sys.path.insert(0, os.path.join(os.environ["FR_ROOT"], "tests"))
import torch
from paper_2608_07580_b300 import firert as fr
from cases import debug_cases
out = {"flags": fr.build_flags(), "words": {}}
arrs = {}
for name, t, L, wv, variant in debug_cases():
    ctx = fr.Context(t)
    ctx.set_tuning(variant, 1)
    o = ctx.retrieve(torch.from_numpy(L).cuda(), torch.from_numpy(wv.astype(np.int16)).cuda())
    out["words"][name] = ctx.debug_word()
    for k, v in o.items():
        arrs[f"{name}/{k}"] = v.cpu().numpy()
np.savez(os.environ["FR_OUT"], **arrs)
print(json.dumps(out))
"""


@pytest.mark.gpu
def test_bounds_checked_build_runs_clean_and_matches_release(tmp_path):
    from paper_2608_07580_b300 import build
    build.build(debug=True)
    env = dict(os.environ, FIRERT_DEBUG="1", FR_ROOT=ROOT, FR_OUT=str(tmp_path / "dbg.npz"))
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    info = json.loads(r.stdout.strip().splitlines()[-1])
    assert info["flags"] & 1 == 1, "the child did not load the bounds-checked build"
    assert all(w == 0 for w in info["words"].values()), info["words"]
    dbg = np.load(tmp_path / "dbg.npz")

    import torch
    from paper_2608_07580_b300 import firert as fr
    from cases import debug_cases
    assert fr.build_flags() & 1 == 0
    n_cases = 0
    for name, t, L, wv, variant in debug_cases():
        ctx = fr.Context(t)
        ctx.set_tuning(variant, 1)
        o = ctx.retrieve(torch.from_numpy(L).cuda(), torch.from_numpy(wv.astype(np.int16)).cuda())
        for k, v in o.items():
            a, b = v.cpu().numpy(), dbg[f"{name}/{k}"]
            # the checks add branches, not arithmetic: the same results bit for bit
            assert np.array_equal(a, b, equal_nan=True), (name, k)
        n_cases += 1
    assert n_cases == len(info["words"])
