"""The checked build (-DPILOT_CHECKED, libpilot_checked.so): every graph index
is range-tested before it addresses a row.  On a valid index it must give the
oracle's results and count no skipped index.  Run in a child process because
the binding loads one library per process (PILOT_LIBRARY selects it)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import oracle
from paper_2503_21206_b300 import index_build, pilot, synth
assert pilot.LIB_PATH.endswith("libpilot_checked.so"), pilot.LIB_PATH
w = synth.WORKLOADS["c1_mixture_20k_d96"]
out = {}
for dtype in ("f32", "fp8"):
    idx, Q, _, _ = index_build.build_workload(w, n=4000, nq=48, reduced_dtype=dtype)
    g = pilot.load_index_data(idx)
    o = pilot.pilot_search_options_default()
    status = np.zeros(8, np.int32)
    o.status_words = status.ctypes.data
    cnt = np.empty((len(Q), 8), np.int32)
    ids, dists = pilot.pilot_search_ex(g, Q, 10, 64, options=o, counters=cnt)
    oi = oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced,
                            {"f32": 0, "bf16": 1, "fp8": 2}[dtype], idx.reduced_scales, idx.full, idx.entry_ids, 0)
    ref = oracle.search(oi, Q, 10, 64)
    # the entry point that allocates nothing reports skipped indices the same way
    qd = torch.from_numpy(Q).cuda()
    ids_d = torch.empty((len(Q), 10), dtype=torch.int32, device="cuda")
    d_d = torch.empty((len(Q), 10), dtype=torch.float32, device="cuda")
    pilot.pilot_search_noalloc(g, qd, 10, 64, ids_d, d_d)
    torch.cuda.synchronize()
    out[dtype] = dict(same=bool(np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
                                and np.array_equal(cnt, ref["counters"])), skipped=int(status[6]),
                      noalloc_same=bool(np.array_equal(ids_d.cpu().numpy(), ref["ids"])
                                        and np.array_equal(d_d.cpu().numpy(), ref["dists"])))
print(json.dumps(out))
"""


def test_checked_build_matches_the_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_21206_b300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, PILOT_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for dtype, v in res.items():
        assert v["same"], dtype
        assert v["noalloc_same"], dtype
        assert v["skipped"] == 0, dtype
