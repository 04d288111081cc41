"""The checked build (-DGN_CHECKS): the search kernels verify the indices they compute from
data (occurrence quads, hit buckets, bank positions, query and sequence ids) before using
them, and a failed check fails the search with GN_EINTERNAL.  On valid inputs no check may
fail and the results must equal the oracle's, on every hit-grouping path."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import os, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle, synth
import paper_1507_02987_gb300 as gn
from paper_1507_02987_gb300 import _build
lib = gn.load()
assert lib._name == _build.CHECKS_LIB, lib._name
bank = synth.make_bank("mid", n_seqs=4000)
qs = synth.make_queries("mid", bank, n=40)
ref = oracle.Index(bank).search(qs, oracle.Params(), threads=os.cpu_count() or 1)
ix = gn.Index.from_bank(bank)
envs = [{}, {"GN_BUCKET_CAP": "64", "GN_SPILL_ROOM": "16"}, {"GN_TILE_FILTER": "0"}, {"GN_HIT_GROUPING": "sort"},
        {"GN_SW_LANES": "32"}]
for env in envs:
    for k in ("GN_BUCKET_CAP", "GN_SPILL_ROOM", "GN_TILE_FILTER", "GN_HIT_GROUPING", "GN_SW_LANES"):
        os.environ.pop(k, None)
    os.environ.update(env)
    res = gn.search(ix, qs.start, qs.bases)
    for i in range(qs.n):
        got, exp = res.query(i), ref[i].ranked
        assert len(got) == len(exp), (env, i)
        for a, b in (("seq", "seq"), ("q_start", "qs"), ("q_end", "qe"), ("db_start", "ds"), ("db_end", "de"),
                     ("score", "score"), ("rank", "rank")):
            assert np.array_equal(got[a].astype(np.int64), exp[b].astype(np.int64)), (env, i, a)
    res.close()
print("checked build ok")
"""


def test_checked_build_passes_its_checks_and_matches_the_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02987_gb300 import _build
    _build.build(checks=True)
    env = dict(os.environ, GN_LIBRARY="checks")
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "checked build ok" in r.stdout
