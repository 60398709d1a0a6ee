"""The stored full-size orderings (tests/golden/*_order.txt) against the generators and
the oracle, on the CPU: each record's surfel keys are re-derived with the oracle's
sampling of the seeded mesh (Sec. 3.1), its start index with the oracle's Philox start
(Sec. 3.2), and its rad2 at index 0 is the INT64_MAX of an empty prefix.  The ordering
digests themselves are compared with the GPU's full output in the -m gpu tests."""
import os

import numpy as np
import pytest

import oracle
from paper_1904_08225_gb300 import workloads as W

import golden_order as G

I64MAX = np.iinfo(np.int64).max


def test_batch_golden_inputs_match_the_generator():
    recs = G.read("batch4096_largest_order.txt")
    assert len(recs) == 3
    specs = W.batch_parts(4096, seed=0)
    for r in recs:
        sp = specs[r["id"]]
        sv, mn, s = oracle.sample_mesh(sp.mesh(), W.AXIS_DIRS, sp.res)
        assert len(sv["key"]) == r["n"] and G.sha(sv["key"]) == r["key"]
        assert s == r["scale"]
        assert r["start"] == oracle.start_index(r["n"], seed=0, part_id=r["id"])
        assert r["at"][0] == (r["start"], I64MAX) and r["at"][r["n"] - 1][1] >= 0


@pytest.mark.skipif(not os.path.exists(os.path.join(G.HERE, "cad_part_seed0_order.txt")),
                    reason="the CAD-part golden has not been written")
def test_cad_golden_input_matches_the_generator():
    (r,) = G.read("cad_part_seed0_order.txt")
    sv, mn, s = oracle.sample_mesh(W.cad_part(seed=0), np.concatenate([W.AXIS_DIRS, W.DIAG_DIRS]), 1024)
    assert len(sv["key"]) == r["n"] == 5_423_479 and G.sha(sv["key"]) == r["key"]
    assert r["start"] == oracle.start_index(r["n"], seed=0) and r["at"][0] == (r["start"], I64MAX)
