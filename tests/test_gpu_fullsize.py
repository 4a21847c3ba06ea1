"""Full-size parity of the default (tensor-core) path against the FP64 oracle.

The benchmark step itself -- 8 qubits, 6 strongly entangling layers, RFF(64) + tanh MLP(32),
dielectric disk, 64x64x16 collocation grid + 64x64 initial-condition plane, 16 energy slices,
path AUTO -- and the 10-qubit, 8-layer step on the 64^3 grid, each in the launch configuration
the benchmark uses. At these sizes every weight-gradient CTA accumulates thousands of rows
(accumulator flushes, partial slots, the compensated slot sum), which the small parity cases
never reach. The oracle's values come from tests/golden/make_fullsize.py (the oracle alone,
minutes to hours of CPU time); the inputs are regenerated here from their seeds and checked
against the digests stored with those values.

Bars (fp32 arithmetic against FP64): every loss term within 1e-5 of the larger of itself and
the total loss and within 1e-4 of itself, every energy slice within 1e-5 of itself;
every gradient entry within 1e-5 of its block's largest oracle entry plus 1e-4 of its own
value; fields and input derivatives at 256 sampled points within 1e-5 of their group's largest
value, each channel within 1e-4 of its own.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2506_23246_b300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = 1e-5
CHAN_TOL = 1e-4


def _golden(name):
    path = os.path.join(GOLDEN, "%s_fullsize.json" % name)
    with open(path) as fh:
        g = json.load(fh)
    circ, prob, params, sets = W.c3_workload(0) if name == "c3" else W.c4_workload(0)
    dig = lambda a: hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()
    assert g["sha256"]["params"] == dig(params)
    for k, v in sets.items():
        assert g["sha256"][k] == dig(v), k
    return g, circ, prob, params, sets


def _blocks(lay):
    return [("mlp", lay["fixed"], lay["circuit"]), ("circuit", lay["circuit"], lay["head"]),
            ("head", lay["head"], lay["total"])]


@pytest.mark.parametrize("name", ["c3", "c4"])
def test_fullsize_loss_grad_fields_vs_oracle(name):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_23246_b300 import build, qp
    build.build()
    g, circ, prob, params, sets = _golden(name)
    plan = qp.Plan(circ, prob, path="auto")
    assert plan.path == "gemm_split"
    dp = torch.tensor(params, device="cuda")
    dsets = {k: torch.tensor(v, device="cuda") for k, v in sets.items()}
    loss, grad = plan.loss_grad(dp, dsets)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    loss = loss.cpu().numpy()
    grad = grad.cpu().numpy()

    lo = np.asarray(g["loss"])
    assert loss.shape == lo.shape
    for i in range(lo.shape[0]):
        err = abs(loss[i] - lo[i])
        if err < 1e-10:
            continue
        scale = max(abs(lo[i]), abs(lo[0])) if i < 9 else abs(lo[i])
        assert err <= TOL * scale, ("loss term", i, loss[i], lo[i])
        assert err <= CHAN_TOL * abs(lo[i]), ("loss term (own value)", i, loss[i], lo[i])

    idx = np.asarray(g["grad_idx"])
    go = np.asarray(g["grad"])
    gg = grad[idx].astype(np.float64)
    lay = plan.layout
    for bname, lo_, hi_ in _blocks(lay):
        sel = (idx >= lo_) & (idx < hi_)
        assert sel.any(), bname
        scale = float(np.max(np.abs(go[sel])))
        err = np.abs(gg[sel] - go[sel])
        assert np.all(err <= TOL * scale + CHAN_TOL * np.abs(go[sel])), \
            (bname, float(np.max(err / scale)), idx[sel][np.argmax(err)])

    fsel = np.asarray(g["field_idx"])
    f, df = plan.forward(dp, dsets["colloc"])
    torch.cuda.synchronize()
    f = f.cpu().numpy()[fsel].astype(np.float64)
    df = df.cpu().numpy()[fsel].reshape(-1, 9).astype(np.float64)
    fo = np.asarray(g["fields"])
    dfo = np.asarray(g["dfields"])
    for got, want, what in ((f, fo, "fields"), (df, dfo, "dfields")):
        scale = float(np.max(np.abs(want)))
        assert float(np.max(np.abs(got - want))) <= TOL * scale, what
        for c in range(want.shape[1]):
            cs = float(np.max(np.abs(want[:, c])))
            assert float(np.max(np.abs(got[:, c] - want[:, c]))) <= CHAN_TOL * cs, (what, c)
