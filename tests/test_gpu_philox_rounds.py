"""Round-count study of the pair noise (Philox-4x32-R, Sec. 2.1 noise): a
library built with R = 7 gives, bit for bit, the oracle's R = 7 words and
its forces within the contract tolerance.  R = 10 stays the library default.

The R = 7 library is built beside the default one and exercised in a child
process (one library per process in the binding)."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, math, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle as O
import paper_1911_04712_gb300.dpd as dpd
from paper_1911_04712_gb300.workloads import uniform_box_state
R = dpd.philox_rounds()
rng = np.random.default_rng(3)
lo = rng.integers(0, 2**32, 1 << 14, dtype=np.uint64).astype(np.uint32)
hi = rng.integers(0, 2**32, 1 << 14, dtype=np.uint64).astype(np.uint32)
words, xi = dpd.debug_rng(lo, hi, 77, 0x1234567890ABCDEF)
ref_w, _ = O.pair_rng(lo, hi, 77, 0x1234567890ABCDEF, rounds=R)
ref10, _ = O.pair_rng(lo, hi, 77, 0x1234567890ABCDEF, rounds=10)
L = 8.0
x, v = uniform_box_state(L, rho=3, seed=4)
p = O.Params(L=(L, L, L), a=25.0, gamma=4.5, kT=1.0, dt=0.005, seed=9, rounds=R)
box = dpd.Box(L, a=25.0, gamma=4.5, kT=1.0, rc=1.0, dt=0.005, seed=9)
box.set_state(x, v)
f_ref, _ = O.forces(p, x, v, 0)
fg = box.get_forces().astype(np.float64)
rms = math.sqrt((f_ref ** 2).sum(1).mean())
print(json.dumps({"rounds": R, "version": dpd.version(),
                  "words_equal": bool(np.array_equal(words, ref_w)),
                  "differs_from_r10": int((words != ref10).sum()),
                  "force_err_rel": float(np.abs(fg - f_ref).max() / rms)}))
"""


def test_philox_r7_library_matches_oracle_r7():
    from paper_1911_04712_gb300 import build
    build.build()
    path = build.build(philox_rounds=7)
    env = dict(os.environ, DPD_LIBRARY=path)
    out = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res["rounds"] == 7 and "Philox-4x32-7" in res["version"]
    assert res["words_equal"]
    assert res["differs_from_r10"] > (1 << 14) - 10   # a different generator
    assert res["force_err_rel"] <= 1e-5
