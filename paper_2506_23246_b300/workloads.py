"""Seeded synthetic workloads: circuit/problem presets, collocation sets, parameters.

This module only draws numbers and lays them out; it holds none of the method's
arithmetic. Both the CUDA path (tests, bench) and the FP64 oracle (tests) consume
what it produces. Everything is float32, the dtype the C-ABI takes; the oracle
receives exact float64 copies.

Shapes follow the paper's workloads: collocation points on [-1,1]^2 x [0,T]
(Sec. 2.1 domain), equispaced grids (64 per coordinate, Sec. 2.2) or uniform
draws, a 64^2 initial-condition plane at t = 0 (Eq. 17), and PEC edge points.
"""
import math

import numpy as np

# ----------------------------------------------------------------------------- presets

def circuit(n_qubits, n_layers, n_readout=None, ansatz="strong_rot", enc="rx", scale="acos",
            premap="rff_mlp", n_direct=3, rff_freqs=64, mlp_width=32, mlp_depth=1, periodic=False):
    """periodic: the periodic input map of Eqs. 25-26 in front of the RFF layer (a learned time
    period T becomes the first trainable premap parameter)."""
    c = {"n_qubits": n_qubits, "n_layers": n_layers,
         "n_readout": n_qubits if n_readout is None else n_readout, "ansatz": ansatz,
         "enc": enc, "scale": scale, "premap": premap, "n_direct": n_direct,
         "rff_freqs": rff_freqs if premap == "rff_mlp" else 0,
         "mlp_width": mlp_width if premap == "rff_mlp" else 0,
         "mlp_depth": mlp_depth if premap == "rff_mlp" else 0}
    if periodic and premap == "rff_mlp":
        c["periodic"] = True
    return c


# Initial value of the learned time period of the periodic map (Eqs. 25-26): longer than every
# time range of the paper's problems (t <= 1.5), as the paper notes the simulated time does not
# complete a period.
PERIOD_INIT = 4.0


def problem(medium="vacuum", eps_r=4.0, disk_r=0.25, disk_x0=0.5, disk_y0=0.0, sigmoid_w=0.02,
            ic_sigma=math.sqrt(1.0 / 50.0), ic_x0=0.0, ic_y0=0.0, w_ic=10.0, w_bc=10.0,
            w_energy=10.0, energy_slice=0, energy_nt=0, phys_loss="split", w_sym=0.0):
    """phys_loss: "split" (Eq. 13: separate MSEs of res1 over the vacuum and dielectric sets) or
    "intuitive" (Eqs. 34-35); w_sym: weight of the symmetry penalty L_sym (Eq. 18), 0 = off."""
    p = {"medium": medium, "eps_r": eps_r, "disk_r": disk_r, "disk_x0": disk_x0,
         "disk_y0": disk_y0, "sigmoid_w": sigmoid_w, "ic_sigma": ic_sigma, "ic_x0": ic_x0,
         "ic_y0": ic_y0, "w_ic": w_ic, "w_bc": w_bc, "w_energy": w_energy,
         "energy_slice": energy_slice, "energy_nt": energy_nt}
    if phys_loss != "split":
        p["phys_loss"] = phys_loss
    if w_sym:
        p["w_sym"] = w_sym
    return p


def c1_circuit():
    """4 qubits, 2 layers of RY,RZ + CNOT ring, RY(pi v) on qubits 0-2, readout Z0..Z2."""
    return circuit(4, 2, 3, ansatz="basic_ryrz", enc="ry", scale="pi", premap="direct")


def c2_circuit():
    return circuit(6, 4, 3, ansatz="basic_ryrz", enc="ry", scale="pi", premap="direct")


def c2_problem():
    # Gaussian IC with sigma = 0.1, PEC edges, no energy term.
    return problem("vacuum", ic_sigma=0.1, w_ic=10.0, w_bc=10.0, w_energy=0.0)


def c3_circuit(n_qubits=8, n_layers=6):
    return circuit(n_qubits, n_layers, ansatz="strong_rot", enc="rx", scale="acos",
                   premap="rff_mlp", rff_freqs=64, mlp_width=32, mlp_depth=1)


def c3_problem(medium="dielectric", nx=64, ny=64, nt=16):
    return problem(medium, w_energy=10.0, energy_slice=nx * ny, energy_nt=nt)


def c3_tmax(medium):
    # Sec. 2.1: t in [0, 1.5] (vacuum), [0, 0.7] (dielectric).
    return 1.5 if medium == "vacuum" else 0.7


# ----------------------------------------------------------------------------- points

def uniform_points(n, seed, tmax=1.0):
    rng = np.random.default_rng(seed)
    p = np.empty((n, 3), dtype=np.float32)
    p[:, 0] = rng.uniform(-1.0, 1.0, n)
    p[:, 1] = rng.uniform(-1.0, 1.0, n)
    p[:, 2] = rng.uniform(0.0, tmax, n)
    return p


def grid_points(nx, ny, nt, tmax):
    """Equispaced periodic grid: x_i = -1 + 2i/nx (no endpoint), t_k = tmax k/(nt-1).

    Point order is t-major: index = (k*ny + iy)*nx + ix, so slice k of the energy
    sums holds nx*ny consecutive points.
    """
    x = (-1.0 + 2.0 * np.arange(nx) / nx).astype(np.float32)
    y = (-1.0 + 2.0 * np.arange(ny) / ny).astype(np.float32)
    t = (tmax * np.arange(nt) / max(nt - 1, 1)).astype(np.float32) if nt > 1 else np.zeros(1, np.float32)
    T, Y, X = np.meshgrid(t, y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), T.ravel()], axis=1).astype(np.float32)


def ic_points_uniform(n, seed):
    p = uniform_points(n, seed)
    p[:, 2] = 0.0
    return p


def ic_grid(nx=64, ny=64):
    return grid_points(nx, ny, 1, 0.0)


def bc_points(n, seed, tmax=1.0):
    """Points on the four edges of [-1,1]^2: edge ~ U{4}, position ~ U, t ~ U[0,tmax]."""
    rng = np.random.default_rng(seed)
    edge = rng.integers(0, 4, n)
    s = rng.uniform(-1.0, 1.0, n)
    t = rng.uniform(0.0, tmax, n)
    p = np.empty((n, 3), dtype=np.float32)
    p[:, 0] = np.where(edge == 0, -1.0, np.where(edge == 1, 1.0, s))
    p[:, 1] = np.where(edge == 2, -1.0, np.where(edge == 3, 1.0, s))
    p[:, 2] = t
    return p


# ----------------------------------------------------------------------------- params

CRZ_ANSATZE = ("cross_mesh", "cross_mesh_2rot")


def single_qubit_params(ansatz):
    """Angles of the single-qubit gate per qubit and layer: RY, RZ (basic_ryrz); RX
    (cross_mesh); RX, RZ (cross_mesh_2rot); Rot(a, b, g) otherwise (Sec. 2.3, Eq. 28)."""
    return {"basic_ryrz": 2, "cross_mesh": 1, "cross_mesh_2rot": 2}.get(ansatz, 3)


def param_blocks(circ):
    """Sizes of the parameter blocks in the flat layout, in order."""
    n, L, m = circ["n_qubits"], circ["n_layers"], circ["n_readout"]
    k = single_qubit_params(circ["ansatz"])
    blocks = []
    if circ["premap"] == "rff_mlp":
        F, H, depth = circ["rff_freqs"], circ["mlp_width"], circ["mlp_depth"]
        blocks.append(("omega", (F, 6 if circ.get("periodic") else 3)))
        if circ.get("periodic"):
            blocks.append(("period", (1,)))
        fan = 2 * F
        for li in range(depth):
            blocks.append(("W%d" % li, (H, fan)))
            blocks.append(("b%d" % li, (H,)))
            fan = H
        blocks.append(("W_out", (n, fan)))
        blocks.append(("b_out", (n,)))
    if circ["ansatz"] in CRZ_ANSATZE:
        # per layer: n x k single-qubit angles, then the n (n - 1) CRZ angles [i][j != i]
        blocks.append(("circuit", (L, n * k + n * (n - 1))))
    else:
        blocks.append(("circuit", (L, n, k)))
    blocks.append(("head_W", (3, m)))
    blocks.append(("head_b", (3,)))
    return blocks


def param_offsets(circ):
    off = {}
    o = 0
    for name, shape in param_blocks(circ):
        size = int(np.prod(shape))
        off[name] = (o, shape)
        o += size
    off["total"] = (o, ())
    return off


def init_params(circ, seed=0):
    """Draw parameters: circuit ~ U(-pi, pi); head W, b ~ U(+-1/sqrt(m)); MLP layers with
    the usual Linear init U(+-1/sqrt(fan_in)); Omega ~ N(0, 1). Draw order is fixed so a
    seed always gives the same tensors.
    """
    rng = np.random.default_rng(seed)
    blocks = dict(param_blocks(circ))
    vals = {}
    vals["circuit"] = rng.uniform(-math.pi, math.pi, blocks["circuit"])
    m = circ["n_readout"]
    vals["head_W"] = rng.uniform(-1 / math.sqrt(m), 1 / math.sqrt(m), blocks["head_W"])
    vals["head_b"] = rng.uniform(-1 / math.sqrt(m), 1 / math.sqrt(m), blocks["head_b"])
    if circ["premap"] == "rff_mlp":
        for name, shape in param_blocks(circ):
            if name.startswith("W"):
                fan = shape[1]
                vals[name] = rng.uniform(-1 / math.sqrt(fan), 1 / math.sqrt(fan), shape)
                bname = "b" + name[1:]
                vals[bname] = rng.uniform(-1 / math.sqrt(fan), 1 / math.sqrt(fan), blocks[bname])
        vals["omega"] = rng.standard_normal(blocks["omega"])
        if circ.get("periodic"):
            vals["period"] = np.full(1, PERIOD_INIT)
    flat = [np.asarray(vals[name], dtype=np.float64).ravel() for name, _ in param_blocks(circ)]
    return np.concatenate(flat).astype(np.float32)


# ----------------------------------------------------------------------------- bundles

def c1_workload(seed=0, n=1024):
    circ = c1_circuit()
    return circ, init_params(circ, seed), uniform_points(n, seed)


def c2_workload(seed=0, n_colloc=16384, n_ic=2048, n_bc=2048):
    circ = c2_circuit()
    sets = {"colloc": uniform_points(n_colloc, seed + 1), "ic": ic_points_uniform(n_ic, seed + 2),
            "bc": bc_points(n_bc, seed + 3)}
    return circ, c2_problem(), init_params(circ, seed), sets


def c3_workload(seed=0, medium="dielectric", nx=64, ny=64, nt=16, n_qubits=8, n_layers=6):
    circ = c3_circuit(n_qubits, n_layers)
    prob = c3_problem(medium, nx, ny, nt)
    sets = {"colloc": grid_points(nx, ny, nt, c3_tmax(medium)), "ic": ic_grid(nx, ny)}
    return circ, prob, init_params(circ, seed), sets


def c4_workload(seed=0, medium="vacuum", n=64):
    circ = c3_circuit(10, 8)
    prob = c3_problem(medium, n, n, n)
    sets = {"colloc": grid_points(n, n, n, 1.0), "ic": ic_grid(n, n)}
    return circ, prob, init_params(circ, seed), sets


def c5_instances(count=32, seed=0, bmin=1024, bmax=65536):
    """Uneven instances: n ~ U{4..10}, L ~ U{2..8}, B = floor(2^U(log2 bmin, log2 bmax))."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(1000 + seed * 7919 + i)
        n = int(rng.integers(4, 11))
        L = int(rng.integers(2, 9))
        B = int(math.floor(2.0 ** rng.uniform(math.log2(bmin), math.log2(bmax))))
        circ = c3_circuit(n, L)
        prob = problem("vacuum", w_energy=10.0)
        sets = {"colloc": uniform_points(B, 5000 + i, 1.5), "ic": ic_points_uniform(max(B // 16, 1), 9000 + i)}
        out.append((circ, prob, init_params(circ, i), sets))
    return out
