"""Write the FP64 oracle's values for the full-size workloads to tests/golden/*_fullsize.json.

The GPU parity tests at full size (the 8-qubit, 6-layer benchmark step: 64x64x16 collocation
grid + 64x64 initial-condition plane, dielectric, 16 energy slices; and the 10-qubit, 8-layer
step on the 64^3 grid) compare the library with these stored values, because the oracle needs
minutes to hours of CPU time at these sizes. This script calls only the oracle and the seeded
input generators; the inputs are regenerated from their seeds by the tests and checked against
the SHA-256 digests stored here.

  python tests/golden/make_fullsize.py [c3|c4 ...] [--threads N]

Stored per workload: every loss term (Eqs. 11-24 and the energy slices of Eq. 31), the
gradient of the total loss at a fixed spread of parameter indices (first-layer weights and
biases, output layer, every circuit layer, head), and fields + input derivatives at 256
collocation points drawn with a fixed seed.
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import api as oracle  # noqa: E402
from paper_2506_23246_b300 import workloads as W  # noqa: E402

N_FIELD_SAMPLES = 256


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def workload(name):
    if name == "c3":
        return W.c3_workload(0)
    if name == "c4":
        return W.c4_workload(0)
    raise ValueError(name)


def grad_indices(circ, n_mlp, n_circ, n_head):
    """A fixed spread of parameter indices over the MLP blocks (first layer W and b, output
    layer W and b), the circuit block (first to last layer) and the head."""
    off = W.param_offsets(circ)
    rng = np.random.default_rng(7)
    idx = []
    w0, s0 = off["W0"]
    b0, _ = off["b0"]
    wo, so = off["W_out"]
    bo, _ = off["b_out"]
    per = [(w0, int(np.prod(s0)), max(n_mlp // 2, 1)), (b0, s0[0], max(n_mlp // 4, 1)),
           (wo, int(np.prod(so)), max(n_mlp // 8, 1)), (bo, so[0], 1)]
    for start, size, k in per:
        idx.extend(int(start + j) for j in np.sort(rng.choice(size, k, replace=False)))
    c0, cs = off["circuit"]
    ncirc = int(np.prod(cs))
    idx.extend(int(c0 + j) for j in np.linspace(0, ncirc - 1, n_circ).round().astype(int))
    h0, _ = off["head_W"]
    nh = off["total"][0] - h0
    idx.extend(int(h0 + j) for j in np.linspace(0, nh - 1, n_head).round().astype(int))
    return sorted(set(idx))


def main(argv):
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*", default=["c3", "c4"])
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args(argv)
    names, nt = args.names, args.threads
    for name in names:
        circ, prob, params, sets = workload(name)
        sizes = (8, 10, 6) if name == "c3" else (6, 6, 4)
        idx = grad_indices(circ, *sizes)
        rng = np.random.default_rng(1)
        fsel = np.sort(rng.choice(sets["colloc"].shape[0], N_FIELD_SAMPLES, replace=False))
        t0 = time.time()
        f, df = oracle.forward(circ, params, sets["colloc"][fsel], nthreads=nt)
        lo = oracle.loss(circ, prob, params, sets, nthreads=nt)
        t1 = time.time()
        print("%s: loss in %.0f s" % (name, t1 - t0), flush=True)
        g = oracle.grad(circ, prob, params, sets, idx, nthreads=nt)
        print("%s: %d gradient entries in %.0f s" % (name, len(idx), time.time() - t1), flush=True)
        out = {
            "what": "FP64 oracle values of the full-size %s workload (tests/golden/make_fullsize.py)" % name,
            "workload": name, "circuit": circ, "problem": prob,
            "sha256": {"params": digest(params), **{k: digest(v) for k, v in sets.items()}},
            "n_points": {k: int(v.shape[0]) for k, v in sets.items()},
            "loss": [float(x) for x in lo],
            "grad_idx": idx, "grad": [float(x) for x in g],
            "field_idx": [int(x) for x in fsel],
            "fields": np.asarray(f).tolist(),
            "dfields": np.asarray(df).reshape(-1, 9).tolist(),
        }
        path = os.path.join(HERE, "%s_fullsize.json" % name)
        with open(path, "w") as fh:
            json.dump(out, fh, indent=0)
        print("wrote", path, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
