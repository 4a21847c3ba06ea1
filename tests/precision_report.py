"""Error of every compute path against the FP64 oracle, per output group, on the 10-qubit,
8-layer configuration (RFF(64) + tanh MLP(32) premap, strongly entangling layers, 64^3 grid).

For each path -- FP32 SIMT gate by gate, the fused-unitary tensor-core path with FP16 operand
pairs, and the same with 3xTF32 operands -- it prints max and RMS of |gpu - oracle| divided by
the group's max |oracle|: the three fields, d/dx, d/dy and d/dt of the fields (over a seeded
sample of the grid), every loss term, and the MLP, circuit and head blocks of the gradient
(on a small grid with its IC plane; all circuit and head parameters and a seeded MLP sample).

Run on a GPU:  python tests/precision_report.py [--points 1024] [--json out.json]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

PATHS = (("simt", "fp16_pairs", "FP32 SIMT"),
         ("gemm_split", "fp16_pairs", "tensor cores, FP16 pairs"),
         ("gemm_split", "tf32_pairs", "tensor cores, 3xTF32"))


def _err(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    scale = max(float(np.max(np.abs(ref))), 1e-30)
    d = np.abs(gpu - ref) / scale
    return float(d.max()), float(np.sqrt(np.mean(d * d)))


def run(n_qubits=10, n_layers=8, points=1024, seed=0):
    import torch
    from oracle import api as O
    from paper_2506_23246_b300 import qp
    from paper_2506_23246_b300 import workloads as W

    circ = W.c3_circuit(n_qubits, n_layers)
    params = W.init_params(circ, seed)
    grid = W.grid_points(64, 64, 64, 1.0)
    rng = np.random.default_rng(seed)
    pts = grid[np.sort(rng.choice(grid.shape[0], points, replace=False))]
    t0 = time.time()
    fo, dfo = O.forward(circ, params, pts)
    t_fwd = time.time() - t0

    prob = W.c3_problem("vacuum", 4, 4, 3)
    sets = {"colloc": W.grid_points(4, 4, 3, 1.0), "ic": W.ic_grid(4, 2)}
    lay = O.param_layout(circ)
    mlp = np.sort(rng.choice(np.arange(lay["fixed"], lay["circuit"]), 48, replace=False))
    idx = np.concatenate([mlp, np.arange(lay["circuit"], lay["total"])])
    t0 = time.time()
    lo = O.loss(circ, prob, params, sets)
    go = O.grad(circ, prob, params, sets, idx)
    t_grad = time.time() - t0
    blocks = {"gradient, MLP": idx < lay["circuit"],
              "gradient, circuit": (idx >= lay["circuit"]) & (idx < lay["head"]),
              "gradient, head": idx >= lay["head"]}

    dp = torch.tensor(params, device="cuda")
    dx = torch.tensor(pts, device="cuda")
    dsets = {k: torch.tensor(v, device="cuda") for k, v in sets.items()}
    rows = []
    for path, ops, label in PATHS:
        plan = qp.Plan(circ, prob, path=path, operands=ops)
        f, df = plan.forward(dp, dx, want_df=True)
        loss, grad = plan.loss_grad(dp, dsets)
        torch.cuda.synchronize()
        if plan.last_device_error() != 0:
            raise RuntimeError("device status %d on %s" % (plan.last_device_error(), label))
        f = f.cpu().numpy()
        df = df.cpu().numpy()
        loss = loss.cpu().numpy()
        grad = grad.cpu().numpy()[idx]
        r = {"path": label, "fields": _err(f, fo)}
        for d, name in enumerate(("d/dx", "d/dy", "d/dt")):
            r[name] = _err(df[:, :, d], dfo[:, :, d])
        terms = [abs(loss[i] - lo[i]) / max(abs(lo[i]), 1e-12) for i in range(lo.shape[0])]
        r["loss terms"] = (float(max(terms)), float(np.sqrt(np.mean(np.square(terms)))))
        for name, m in blocks.items():
            r[name] = _err(grad[m], go[m])
        rows.append(r)
    meta = {"circuit": "%d qubits x %d layers, RFF(64) + tanh MLP(32)" % (n_qubits, n_layers),
            "forward_points": points, "grad_params": int(idx.size),
            "grad_sets": {k: int(v.shape[0]) for k, v in sets.items()},
            "oracle_s": {"forward": round(t_fwd, 2), "loss_grad": round(t_grad, 2)},
            "device": torch.cuda.get_device_name(0)}
    return meta, rows


def table(rows):
    cols = [k for k in rows[0] if k != "path"]
    out = ["| output group | " + " | ".join(r["path"] for r in rows) + " |",
           "|---|" + "---|" * len(rows)]
    for c in cols:
        out.append("| %s | " % c + " | ".join("%.1e / %.1e" % r[c] for r in rows) + " |")
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--qubits", type=int, default=10)
    ap.add_argument("--layers", type=int, default=8)
    ap.add_argument("--points", type=int, default=1024)
    ap.add_argument("--json", default=None)
    a = ap.parse_args()
    meta, rows = run(a.qubits, a.layers, a.points)
    print(json.dumps(meta))
    print("max / RMS of |gpu - oracle| / max |oracle| per group")
    print(table(rows))
    if a.json:
        with open(a.json, "w") as fh:
            json.dump({"meta": meta, "rows": rows}, fh, indent=1)


if __name__ == "__main__":
    main()
