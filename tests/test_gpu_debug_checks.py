"""The debug library (libsp2_debug.so, device-side bounds checks compiled in) through the C ABI.

Each case runs in a child process with SP2_LIB=debug, since a process loads one library.
- A check made to fail reports SP2_ERR_BOUNDS. It fails on an operand slot beyond the arena,
  which only addresses tensor-map loads, and those read zeros outside the map.
- The parity cases of the release library pass unchanged with every check compiled in: FP64,
  the fp16x3 tensor-core path on both tile kinds, and the block-sparse tensor-core path.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

CHILD = r'''
import json, sys
sys.path.insert(0, ROOT)
import numpy as np, torch
from oracle import sp2_oracle as o, bsr_oracle as bo
from paper_1507_02087_gb300 import inputs, sp2
L = sp2.lib()
out = {"checks": int(L.sp2_build_device_checks())}
ld = 256
arena = torch.zeros(2, 3, ld, ld, dtype=torch.bfloat16, device="cuda")
C = torch.zeros(ld, ld, dtype=torch.float32, device="cuda")
out["bounds_status"] = int(L.sp2_test_tc_bounds(arena.data_ptr(), ld, 2, 5, C.data_ptr(),
                                                torch.cuda.current_stream().cuda_stream))
case = inputs.dense_gapped(200, 90, gap=0.05, seed=12)
ref = o.sp2(case.F.numpy(), 90)
with sp2.Purifier(200, 90, "fp64") as P:
    D = P.run(case.F.cuda()).cpu().numpy(); i = P.info()
out["fp64"] = [i["status"], i["n_iter"], ref.n, o.rel_error(D, ref.D, 90)]
case = inputs.dense_gapped(512, 250, gap=0.05, seed=13)
ref = o.sp2(case.F.numpy(), 250)
ref32 = o.sp2(case.F.numpy(), 250, storage="fp32", trace="fro")
for tile in ("pair", "128"):
    with sp2.Purifier(512, 250, "fp16x3", tile=tile) as P:
        D = P.run(case.F.cuda()).cpu().numpy(); i = P.info()
    out["fp16x3_" + tile] = [i["status"], i["n_iter"], ref32.n, ref.n, o.rel_error(D, ref.D, 250)]
tb = inputs.tight_binding(dims=(32, 8, 4))
rp, ci, vals = (torch.from_numpy(x).cuda() for x in tb.bsr(32))
F = tb.dense().numpy()
with sp2.BsrPurifier(tb.N, tb.nocc, 1e-4, rule="error") as P:
    D = P.run(rp, ci, vals).cpu().numpy(); i = P.info()
ref32 = bo.sp2_bsr(F, tb.nocc, 32, 1e-4, rule="error", storage="fp32")
out["bsr"] = [i["status"], i["n_iter"], ref32.n, o.rel_error(D, ref32.D, tb.nocc)]
print("RESULT " + json.dumps(out))
'''


@pytest.fixture(scope="module")
def child_result():
    from paper_1507_02087_gb300 import build
    if not os.path.exists(build.LIB_DEBUG):
        build.build(debug=True)
    env = dict(os.environ, SP2_LIB="debug")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_debug_library_is_loaded_and_a_failed_check_is_reported(child_result):
    assert child_result["checks"] == 1
    assert child_result["bounds_status"] == 8          # SP2_ERR_BOUNDS, no fault


def test_parity_cases_pass_with_every_check_compiled_in(child_result):
    st, n, nref, err = child_result["fp64"]
    assert st == 0 and abs(n - nref) <= 2 and err <= 1e-10
    for tile in ("pair", "128"):
        st, n, n32, n64, err = child_result["fp16x3_" + tile]
        assert st == 0 and n32 - 3 <= n <= n32 + 2 and n <= n64 and err <= 1e-6
    st, n, n32, err = child_result["bsr"]
    assert st == 0 and abs(n - n32) <= 1 and np.isfinite(err) and err <= 1e-5
