"""The stored full-size oracle values (tests/golden/*_fullsize.json, written by
tests/golden/make_fullsize.py) still describe today's inputs and today's oracle: the seeded
inputs hash to the stored digests, and a sample of the stored fields recomputes exactly."""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2506_23246_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("name", ["c3", "c4"])
def test_fullsize_golden_current(oracle, name):
    with open(os.path.join(GOLDEN, "%s_fullsize.json" % name)) as fh:
        g = json.load(fh)
    circ, prob, params, sets = W.c3_workload(0) if name == "c3" else W.c4_workload(0)
    assert g["circuit"] == circ and g["problem"] == prob
    dig = lambda a: hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()
    assert g["sha256"]["params"] == dig(params)
    for k, v in sets.items():
        assert g["sha256"][k] == dig(v), k
        assert g["n_points"][k] == v.shape[0]
    assert len(g["loss"]) == 9 + prob["energy_nt"]
    assert len(g["grad_idx"]) == len(g["grad"]) >= 16
    lay = oracle.param_layout(circ)
    idx = np.asarray(g["grad_idx"])
    for lo, hi in ((lay["fixed"], lay["circuit"]), (lay["circuit"], lay["head"]),
                   (lay["head"], lay["total"])):
        assert np.any((idx >= lo) & (idx < hi))
    fsel = np.asarray(g["field_idx"])[::32]
    f, df = oracle.forward(circ, params, sets["colloc"][fsel])
    assert np.array_equal(f, np.asarray(g["fields"])[::32])
    assert np.array_equal(df.reshape(-1, 9), np.asarray(g["dfields"])[::32])
