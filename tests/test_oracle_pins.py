"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test reaches the expected value by a route that does not reuse the oracle's
code: values printed in the paper (tests/golden), closed forms (Bloch rotations,
Clifford Z-propagation, plane waves), matrix exponentials and Kronecker products,
finite differences, and the exact general parameter-shift rule.
"""
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm

from paper_2506_23246_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)


def _rot_exp(P, t):
    # exp(-i t P / 2), the half-angle rotation convention pinned by Fig. 3 (<Z> = cos t).
    return expm(-0.5j * t * P)


def _set_head(circ, params, rows):
    off = W.param_offsets(circ)
    o, shape = off["head_W"]
    Wh = np.zeros(shape)
    for r, i in enumerate(rows):
        Wh[r, i] = 1.0
    params = params.astype(np.float64).copy()
    params[o:o + Wh.size] = Wh.ravel()
    ob, sb = off["head_b"]
    params[ob:ob + 3] = 0.0
    return params


def _z_from_state(psi, n):
    p = np.abs(psi) ** 2
    k = np.arange(psi.shape[0])
    return np.array([np.sum(p * (1 - 2 * ((k >> (n - 1 - i)) & 1))) for i in range(n)])


# ----------------------------------------------------------------------------- Fig. 3

def _read_fig3():
    rows = []
    with open(os.path.join(GOLDEN, "fig3_scalings.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                s, a, z = line.split()
                rows.append((s, float(a), float(z)))
    return rows


@pytest.mark.parametrize("row", _read_fig3())
def test_fig3_scaling_identities(oracle, row):
    scale, a, z_expected = row
    circ = W.circuit(1, 0, 1, ansatz="basic_rot", enc="rx", scale=scale, premap="direct",
                     n_direct=1)
    params = _set_head(circ, np.zeros(W.param_offsets(circ)["total"][0]), [0, 0, 0])
    f, df = oracle.forward(circ, params, np.array([[a, 0.0, 0.0]]))
    assert abs(f[0, 0] - z_expected) < 1e-13
    if abs(a) < 0.95:  # d<Z>/da = +1 (acos) or -1 (asin) away from the endpoints
        assert abs(df[0, 0, 0] - (1.0 if scale == "acos" else -1.0)) < 1e-12


@pytest.mark.parametrize("scale", ["none", "pi", "bias"])
def test_single_qubit_cos_theta(oracle, scale):
    circ = W.circuit(1, 0, 1, ansatz="basic_rot", enc="rx", scale=scale, premap="direct",
                     n_direct=1)
    params = _set_head(circ, np.zeros(W.param_offsets(circ)["total"][0]), [0, 0, 0])
    for a in np.linspace(-1, 1, 7):
        theta = {"none": a, "pi": math.pi * a, "bias": (a + 1) * math.pi / 2}[scale]
        f, _ = oracle.forward(circ, params, np.array([[a, 0.0, 0.0]]))
        assert abs(f[0, 0] - math.cos(theta)) < 1e-13


# ----------------------------------------------------------------------------- Table 1

def test_table1_param_counts(oracle):
    rows = {}
    with open(os.path.join(GOLDEN, "table1_param_counts.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                parts = line.split()
                rows[tuple(parts[:-1])] = int(parts[-1])
    for ans in ("basic_rot", "strong_rot", "noent_rot", "cross_mesh", "cross_mesh_2rot",
                "cross_mesh_cnot"):
        circ = W.circuit(7, 4, 7, ansatz=ans, enc="rx", scale="acos", premap="direct")
        lay = oracle.param_layout(circ)
        assert lay["head"] - lay["circuit"] == rows[("quantum", ans)]
    circ = W.circuit(7, 4, 7, ansatz="strong_rot", premap="rff_mlp", rff_freqs=128,
                     mlp_width=128, mlp_depth=3)
    lay = oracle.param_layout(circ)
    quantum = lay["head"] - lay["circuit"]
    classical = lay["total"] - lay["fixed"] - quantum
    assert classical + rows[("learned_period",)] == rows[("classical_qpinn",)]
    assert lay["total"] == W.param_offsets(circ)["total"][0]
    # with the periodic input map (Eqs. 25-26) the learned period is a parameter of the layout
    circ = dict(circ, periodic=True)
    lay = oracle.param_layout(circ)
    assert lay["total"] - lay["fixed"] - (lay["head"] - lay["circuit"]) == rows[("classical_qpinn",)]
    assert lay["total"] == W.param_offsets(circ)["total"][0]


# ----------------------------------------------------------------------------- closed forms

def _Rz3(p):
    return np.array([[math.cos(p), -math.sin(p), 0], [math.sin(p), math.cos(p), 0], [0, 0, 1]])


def _Ry3(p):
    return np.array([[math.cos(p), 0, math.sin(p)], [0, 1, 0], [-math.sin(p), 0, math.cos(p)]])


@pytest.mark.parametrize("n,L,enc", [(3, 2, "rx"), (5, 3, "ry"), (10, 4, "rx")])
def test_noent_bloch_closed_form(oracle, n, L, enc):
    """No-entanglement ansatz: each qubit's Bloch vector is rotated independently."""
    circ = W.circuit(n, L, n, ansatz="noent_rot", enc=enc, scale="pi", premap="direct")
    rng = np.random.default_rng(n)
    params = W.init_params(circ, n).astype(np.float64)
    off = W.param_offsets(circ)
    o, shape = off["circuit"]
    cp = params[o:o + int(np.prod(shape))].reshape(shape)
    pts = np.array([[rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0, 1)]])
    theta = [math.pi * pts[0, j] if j < 3 else 0.0 for j in range(n)]
    expect = []
    for q in range(n):
        t = theta[q]
        v = np.array([0.0, -math.sin(t), math.cos(t)]) if enc == "rx" else np.array(
            [math.sin(t), 0.0, math.cos(t)])
        for l in range(L):
            a, b, g = cp[l, q]
            v = _Rz3(g) @ _Ry3(b) @ _Rz3(a) @ v
        expect.append(v[2])
    for start in range(0, n, 3):
        rows = [min(start + r, n - 1) for r in range(3)]
        p2 = _set_head(circ, params, rows)
        f, _ = oracle.forward(circ, p2, pts)
        for r in range(3):
            assert abs(f[0, r] - expect[rows[r]]) < 1e-12


def _cnot_ring(n, L, ansatz):
    gates = []
    for l in range(L):
        r = 1 + (l % (n - 1)) if ansatz == "strong_rot" else 1
        gates.append([(i, (i + r) % n) for i in range(n)])
    return gates


@pytest.mark.parametrize("n,L,ansatz", [(4, 2, "basic_ryrz"), (6, 4, "basic_ryrz"),
                                        (8, 6, "strong_rot"), (10, 8, "strong_rot")])
def test_clifford_z_propagation(oracle, n, L, ansatz):
    """With every RY angle zero the layers are diagonal phases times CNOT permutations,
    so <Z_i> = prod_{j in S_i} cos(theta_j) with S_i the Z-string of Z_i pulled back
    through the CNOTs over GF(2) (CNOT^dag Z_t CNOT = Z_c Z_t)."""
    circ = W.circuit(n, L, n, ansatz=ansatz, enc="rx", scale="pi", premap="direct")
    params = W.init_params(circ, 7).astype(np.float64)
    off = W.param_offsets(circ)
    o, shape = off["circuit"]
    cp = params[o:o + int(np.prod(shape))].reshape(shape)
    if ansatz == "basic_ryrz":
        cp[:, :, 0] = 0.0          # RY angles
    else:
        cp[:, :, 1] = 0.0          # Rot beta (the RY inside RZ RY RZ)
    params[o:o + cp.size] = cp.ravel()
    rng = np.random.default_rng(3)
    theta = rng.uniform(-math.pi, math.pi, n)
    psi = oracle.state(circ, params, theta)
    z = _z_from_state(psi, n)
    rings = _cnot_ring(n, L, ansatz)
    for i in range(n):
        s = np.zeros(n, dtype=bool)
        s[i] = True
        for ring in reversed(rings):
            for c, t in reversed(ring):
                if s[t]:
                    s[c] = not s[c]
        assert abs(z[i] - np.prod(np.cos(theta[s]))) < 1e-12


@pytest.mark.parametrize("n,ansatz", [(1, "basic_rot"), (3, "basic_ryrz"), (6, "strong_rot"),
                                      (8, "strong_rot"), (5, "cross_mesh"), (6, "cross_mesh_2rot"),
                                      (5, "cross_mesh_cnot")])
def test_norm_and_layer_unitarity(oracle, n, ansatz):
    L = 3
    circ = W.circuit(n, L, 1, ansatz=ansatz, enc="rx", scale="pi", premap="direct",
                     n_direct=min(3, n))
    params = W.init_params(circ, 11)
    rng = np.random.default_rng(5)
    psi = oracle.state(circ, params, rng.uniform(-3, 3, n))
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-13
    for l in range(L):
        U = oracle.layer_unitary(circ, params, l)
        assert np.max(np.abs(U.conj().T @ U - np.eye(1 << n))) < 1e-13


def _kron_gate(n, q, g):
    mats = [np.eye(2, dtype=complex)] * n
    mats = list(mats)
    mats[q] = g
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def _kron_cnot(n, c, t):
    P0 = np.array([[1, 0], [0, 0]], dtype=complex)
    P1 = np.array([[0, 0], [0, 1]], dtype=complex)
    a = [np.eye(2, dtype=complex)] * n
    a = list(a)
    a[c] = P0
    b = [np.eye(2, dtype=complex)] * n
    b = list(b)
    b[c] = P1
    b[t] = X
    ka, kb = a[0], b[0]
    for i in range(1, n):
        ka = np.kron(ka, a[i])
        kb = np.kron(kb, b[i])
    return ka + kb


def _kron_crz(n, c, t, theta):
    """Controlled RZ as the exponential of its generator |1><1|_c (x) Z_t (Kronecker)."""
    P1 = np.array([[0, 0], [0, 1]], dtype=complex)
    mats = [np.eye(2, dtype=complex)] * n
    mats = list(mats)
    mats[c] = P1
    mats[t] = Z
    gen = mats[0]
    for m in mats[1:]:
        gen = np.kron(gen, m)
    return expm(-0.5j * theta * gen)


@pytest.mark.parametrize("n,ansatz,enc", [(2, "basic_rot", "rx"), (3, "basic_ryrz", "ry"),
                                          (4, "strong_rot", "rx"), (4, "noent_rot", "ry"),
                                          (3, "cross_mesh", "rx"), (4, "cross_mesh_2rot", "ry"),
                                          (4, "cross_mesh_cnot", "rx")])
def test_bruteforce_dense_kronecker(oracle, n, ansatz, enc):
    """n <= 4: the dense product of Kronecker-expanded matrix exponentials equals the
    oracle's pair-loop state. The CRZ mesh (Eq. 29) is multiplied here in the reverse of the
    oracle's order: its gates are diagonal and commute."""
    L = 3
    circ = W.circuit(n, L, 1, ansatz=ansatz, enc=enc, scale="pi", premap="direct",
                     n_direct=min(3, n))
    params = W.init_params(circ, 2).astype(np.float64)
    off = W.param_offsets(circ)
    o, shape = off["circuit"]
    k = W.single_qubit_params(ansatz)
    cl = params[o:o + int(np.prod(shape))].reshape(L, -1)
    rng = np.random.default_rng(9)
    theta = rng.uniform(-3, 3, n)
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1.0
    for j in range(n):
        psi = _kron_gate(n, j, _rot_exp(X if enc == "rx" else Y, theta[j])) @ psi
    for l in range(L):
        for q in range(n):
            p = cl[l, q * k:(q + 1) * k]
            if ansatz == "basic_ryrz":
                g = _rot_exp(Z, p[1]) @ _rot_exp(Y, p[0])
            elif ansatz == "cross_mesh":
                g = _rot_exp(X, p[0])
            elif ansatz == "cross_mesh_2rot":
                g = _rot_exp(Z, p[1]) @ _rot_exp(X, p[0])
            else:
                a, b, gm = p
                g = _rot_exp(Z, gm) @ _rot_exp(Y, b) @ _rot_exp(Z, a)
            psi = _kron_gate(n, q, g) @ psi
        if ansatz in ("cross_mesh", "cross_mesh_2rot"):
            ang = cl[l, n * k:].reshape(n, n - 1)
            pairs = [(i, j) for i in range(n) for j in range(n) if j != i]
            for i, j in reversed(pairs):
                psi = _kron_crz(n, i, j, ang[i, j if j < i else j - 1]) @ psi
        elif ansatz == "cross_mesh_cnot":
            for i in range(n):
                for j in range(n):
                    if j != i:
                        psi = _kron_cnot(n, i, j) @ psi
        elif ansatz != "noent_rot" and n > 1:
            r = 1 + (l % (n - 1)) if ansatz == "strong_rot" else 1
            for i in range(n):
                psi = _kron_cnot(n, i, (i + r) % n) @ psi
    got = oracle.state(circ, params, theta)
    assert np.max(np.abs(got - psi)) < 1e-12


# ----------------------------------------------------------------------------- derivatives

SMALL_MLP = dict(rff_freqs=4, mlp_width=5, mlp_depth=1)


def _small_circuits():
    return [
        W.c1_circuit(),
        W.circuit(5, 3, 4, ansatz="strong_rot", enc="rx", scale="acos", premap="rff_mlp",
                  **SMALL_MLP),
        W.circuit(4, 2, 4, ansatz="basic_rot", enc="ry", scale="asin", premap="rff_mlp",
                  rff_freqs=3, mlp_width=4, mlp_depth=2),
    ]


@pytest.mark.parametrize("ci", range(3))
def test_input_derivatives_vs_central_fd(oracle, ci):
    circ = _small_circuits()[ci]
    params = W.init_params(circ, 4)
    pts = W.uniform_points(5, 8).astype(np.float64) * 0.9
    f, df = oracle.forward(circ, params, pts)
    h = 1e-5
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fp, _ = oracle.forward(circ, params, pts + e)
        fm, _ = oracle.forward(circ, params, pts - e)
        fd = (fp - fm) / (2 * h)
        assert np.max(np.abs(fd - df[:, :, d])) < 1e-7


def test_input_derivative_direct_shift_rule(oracle):
    """Direct RY(pi x) embedding: f is a first-harmonic trig polynomial in theta_x = pi x,
    so df/dx = pi (f(theta + pi/2) - f(theta - pi/2)) / 2 exactly."""
    circ = W.c1_circuit()
    params = W.init_params(circ, 1)
    pts = W.uniform_points(6, 2).astype(np.float64)
    _, df = oracle.forward(circ, params, pts)
    for d in range(3):
        e = np.zeros(3)
        e[d] = 0.5  # theta shift of pi/2 for theta = pi v
        fp, _ = oracle.forward(circ, params, pts + e)
        fm, _ = oracle.forward(circ, params, pts - e)
        assert np.max(np.abs(math.pi * (fp - fm) / 2 - df[:, :, d])) < 1e-12


def _shift_rule(fn, x0, R):
    """General parameter-shift rule, exact for trig polynomials of degree <= R:
    f'(x) = sum_{mu=1}^{2R} f(x + x_mu) (-1)^(mu-1) / (4 R sin^2(x_mu/2)),
    x_mu = (2 mu - 1) pi / (2R)."""
    tot = 0.0
    for mu in range(1, 2 * R + 1):
        xm = (2 * mu - 1) * math.pi / (2 * R)
        tot += fn(x0 + xm) * (-1) ** (mu - 1) / (4 * R * math.sin(xm / 2) ** 2)
    return tot


def test_shift_rule_self_check():
    rng = np.random.default_rng(0)
    c = rng.standard_normal(9)
    f = lambda x: c[0] + sum(c[2 * k - 1] * math.cos(k * x) + c[2 * k] * math.sin(k * x)
                             for k in range(1, 5))
    fp = lambda x: sum(-k * c[2 * k - 1] * math.sin(k * x) + k * c[2 * k] * math.cos(k * x)
                       for k in range(1, 5))
    for x in (0.0, 0.7, -2.1):
        assert abs(_shift_rule(f, x, 4) - fp(x)) < 1e-12


def _loss_setup(ci):
    circ = _small_circuits()[ci]
    prob = W.problem("dielectric" if ci == 1 else "vacuum", disk_x0=0.2, disk_r=0.5,
                     w_energy=10.0 if ci != 0 else 0.0, energy_slice=4, energy_nt=2)
    sets = {"colloc": W.uniform_points(8, 10 + ci), "ic": W.ic_points_uniform(3, 20 + ci),
            "bc": W.bc_points(3, 30 + ci)}
    params = W.init_params(circ, 6).astype(np.float64)
    return circ, prob, params, sets


@pytest.mark.parametrize("ci", range(3))
def test_param_gradient_vs_central_fd(oracle, ci):
    circ, prob, params, sets = _loss_setup(ci)
    lay = oracle.param_layout(circ)
    idx = np.arange(lay["fixed"], lay["total"])
    g = oracle.grad(circ, prob, params, sets, idx)
    h = 1e-5
    for j, i in enumerate(idx):
        pp = params.copy()
        pp[i] += h
        pm = params.copy()
        pm[i] -= h
        fd = (oracle.loss(circ, prob, pp, sets)[0] - oracle.loss(circ, prob, pm, sets)[0]) / (2 * h)
        assert abs(fd - g[j]) < 1e-6 * max(1.0, abs(g[j])), (i, fd, g[j])


@pytest.mark.parametrize("ci", range(3))
def test_param_gradient_exact_shift_rule(oracle, ci):
    """Circuit angles enter through one half-angle rotation each, so the fields and their
    input derivatives are first-harmonic in each angle and the loss (squares, and the
    squared Poynting residual) is a trig polynomial of degree <= 4: the R = 4 shift rule
    is exact."""
    circ, prob, params, sets = _loss_setup(ci)
    lay = oracle.param_layout(circ)
    idx = np.arange(lay["circuit"], lay["head"])
    g = oracle.grad(circ, prob, params, sets, idx)
    for j, i in enumerate(idx):
        def fn(x, i=i):
            pp = params.copy()
            pp[i] = x
            return oracle.loss(circ, prob, pp, sets)[0]
        assert abs(_shift_rule(fn, params[i], 4) - g[j]) < 1e-10 * max(1.0, abs(g[j]))


def test_omega_gradient_is_zero(oracle):
    circ, prob, params, sets = _loss_setup(1)
    lay = oracle.param_layout(circ)
    g = oracle.grad(circ, prob, params, sets, np.arange(lay["fixed"]))
    assert np.all(g == 0.0)


# ----------------------------------------------------------------------------- losses

def _vac():
    return W.problem("vacuum", w_ic=10.0, w_bc=10.0, w_energy=10.0)


def test_plane_wave_satisfies_residuals_and_poynting(oracle):
    """Ez = cos(kx - wt), Hy = -cos(kx - wt), Hx = 0 with w = k solves Eqs. 5/8-10 and the
    local Poynting balance, so every residual and the energy residual vanish."""
    k = 2.3
    pts = W.uniform_points(64, 1).astype(np.float64)
    x, t = pts[:, 0], pts[:, 2]
    ph = k * x - k * t
    f = np.stack([np.cos(ph), np.zeros_like(ph), -np.cos(ph)], axis=1)
    df = np.zeros((64, 3, 3))
    df[:, 0, 0] = -k * np.sin(ph)
    df[:, 0, 2] = k * np.sin(ph)
    df[:, 2, 0] = k * np.sin(ph)
    df[:, 2, 2] = -k * np.sin(ph)
    out = oracle.loss_from_fields(_vac(), pts, f, df)
    assert np.max(np.abs(out[:9])) < 1e-24 + 1e-13


def test_plane_wave_wrong_speed_closed_form(oracle):
    """With w != k: res1 = (w - k) sin, res3 = (k - w) sin, res2 = 0."""
    k, w = 2.0, 3.0
    pts = W.uniform_points(100, 2).astype(np.float64)
    ph = k * pts[:, 0] - w * pts[:, 2]
    f = np.stack([np.cos(ph), np.zeros_like(ph), -np.cos(ph)], axis=1)
    df = np.zeros((100, 3, 3))
    df[:, 0, 0] = -k * np.sin(ph)
    df[:, 0, 2] = w * np.sin(ph)
    df[:, 2, 0] = k * np.sin(ph)
    df[:, 2, 2] = -w * np.sin(ph)
    out = oracle.loss_from_fields(W.problem("vacuum", w_energy=0.0), pts, f, df)
    m = np.mean(((w - k) * np.sin(ph)) ** 2)
    assert abs(out[5] - m) < 1e-13 and abs(out[8] - m) < 1e-13 and abs(out[7]) < 1e-15
    assert abs(out[1] - 2 * m) < 1e-12


def test_ic_and_bc_terms(oracle):
    prob = W.problem("vacuum", ic_sigma=0.1, w_ic=10.0, w_bc=10.0, w_energy=0.0)
    ic = W.ic_points_uniform(50, 3).astype(np.float64)
    r2 = ic[:, 0] ** 2 + ic[:, 1] ** 2
    e0 = np.exp(-r2 / (2 * 0.01))
    fi = np.stack([e0, np.zeros(50), np.zeros(50)], axis=1)
    empty = np.zeros((0, 3))
    out = oracle.loss_from_fields(prob, empty, empty, np.zeros((0, 9)), ic, fi)
    assert abs(out[2]) < 1e-25
    fi0 = np.zeros((50, 3))
    fi0[:, 1] = 0.5
    out = oracle.loss_from_fields(prob, empty, empty, np.zeros((0, 9)), ic, fi0)
    assert abs(out[2] - 10.0 * np.mean(e0 ** 2 + 0.25)) < 1e-12
    bc = W.bc_points(40, 4).astype(np.float64)
    fb = np.zeros((40, 3))
    fb[:, 0] = 0.3
    out = oracle.loss_from_fields(prob, empty, empty, np.zeros((0, 9)), bc=bc, fb=fb)
    assert abs(out[3] - 10.0 * 0.09) < 1e-13


def test_dielectric_split_mse(oracle):
    """Eq. 12: separate means over the vacuum and dielectric sets."""
    prob = W.problem("dielectric", disk_x0=0.2, disk_y0=-0.1, disk_r=0.5, w_energy=0.0)
    pts = W.uniform_points(400, 5).astype(np.float64)
    inside = (pts[:, 0] - 0.2) ** 2 + (pts[:, 1] + 0.1) ** 2 < 0.25
    assert 10 < inside.sum() < 390
    df = np.zeros((400, 3, 3))
    df[:, 0, 2] = np.where(inside, 3.0, 1.0)  # dEz/dt only: res1 = dEz/dt
    out = oracle.loss_from_fields(prob, pts, np.zeros((400, 3)), df)
    assert abs(out[5] - 1.0) < 1e-14 and abs(out[6] - 9.0) < 1e-14


def test_energy_slice_sums(oracle):
    """U(t) of Eq. 31 on a full-period grid: sum cos^2 over 2 periods of 64 points = 32."""
    nx, ny, nt = 64, 8, 3
    pts = W.grid_points(nx, ny, nt, 1.0).astype(np.float64)
    prob = W.problem("vacuum", w_energy=0.0, energy_slice=nx * ny, energy_nt=nt)
    ph = 2 * math.pi * pts[:, 0] - 0.3 * pts[:, 2]
    f = np.stack([np.cos(ph), np.zeros_like(ph), np.cos(ph)], axis=1)
    out = oracle.loss_from_fields(prob, pts, f, np.zeros((pts.shape[0], 9)))
    for k in range(nt):
        assert abs(out[9 + k] - 0.5 * 2 * ny * nx / 2) < 1e-9


def test_plane_wave_along_y(oracle):
    """Ez = cos(ky - wt), Hx = cos(ky - wt), Hy = 0 with w = k: exercises the Hx terms of
    Eqs. 8 and 10a and of the Poynting residual (Eq. 23)."""
    k = 1.7
    pts = W.uniform_points(64, 6).astype(np.float64)
    ph = k * pts[:, 1] - k * pts[:, 2]
    f = np.stack([np.cos(ph), np.cos(ph), np.zeros_like(ph)], axis=1)
    df = np.zeros((64, 3, 3))
    df[:, 0, 1] = -k * np.sin(ph)
    df[:, 0, 2] = k * np.sin(ph)
    df[:, 1, 1] = -k * np.sin(ph)
    df[:, 1, 2] = k * np.sin(ph)
    out = oracle.loss_from_fields(_vac(), pts, f, df)
    assert np.max(np.abs(out[:9])) < 1e-13
    # flipping the wave direction breaks every residual
    df[:, 1, :] *= -1
    f[:, 1] *= -1
    out = oracle.loss_from_fields(_vac(), pts, f, df)
    assert out[7] > 0.1 and out[4] > 0.1


def test_dielectric_eps_limits(oracle):
    """eps -> eps_r at the disk centre and -> 1 far away: energy residual eps*Ez*dEz/dt."""
    prob = W.problem("dielectric", eps_r=4.0, disk_x0=0.5, disk_y0=0.0, disk_r=0.25,
                     sigmoid_w=0.02, w_energy=1.0)
    for (x, y), eps in (((0.5, 0.0), 4.0), ((-0.8, 0.7), 1.0)):
        pts = np.array([[x, y, 0.4]])
        f = np.array([[0.4, 0.0, 0.0]])
        df = np.zeros((1, 3, 3))
        df[0, 0, 2] = 1.0
        out = oracle.loss_from_fields(prob, pts, f, df)
        assert abs(out[4] - (eps * 0.4) ** 2) < 1e-4


# ----------------------------------------------------------------------------- BH indicator

def _bh_fields(amp, nx=16, ny=16, nt=6, tmax=1.5):
    """Energy slices of Ez = Hy = amp(t) cos(2 pi x) on a full-period grid: U(t) =
    amp(t)^2 * (nx ny / 2) exactly (sum of cos^2 over whole periods)."""
    pts = W.grid_points(nx, ny, nt, tmax).astype(np.float64)
    prob = W.problem("vacuum", w_energy=0.0, energy_slice=nx * ny, energy_nt=nt)
    a = amp(pts[:, 2])
    ph = 2 * math.pi * pts[:, 0]
    f = np.stack([a * np.cos(ph), np.zeros_like(ph), a * np.cos(ph)], axis=1)
    out = oracle_api().loss_from_fields(prob, pts, f, np.zeros((pts.shape[0], 9)))
    return out[9:9 + nt], tmax, nt


def oracle_api():
    from oracle import api
    return api


def test_bh_indicator_constant_energy(oracle):
    """A lossless field keeps U(t) = U(0): U~ = 1 at every slice and I_BH = 0."""
    u, tmax, nt = _bh_fields(lambda t: np.ones_like(t))
    ut, ibh = oracle.bh_indicator(u, tmax, 0.2)
    assert np.max(np.abs(ut - 1.0)) < 1e-12 and abs(ibh) < 1e-12


def test_bh_indicator_exponential_decay(oracle):
    """Amplitude exp(-lam t): U~(t) = exp(-2 lam t) in closed form, I_BH = 1 - exp(-2 lam T);
    delta = T leaves only the last slice."""
    lam = 0.8
    u, tmax, nt = _bh_fields(lambda t: np.exp(-lam * t))
    ut, ibh = oracle.bh_indicator(u, tmax, 0.1)
    t = tmax * np.arange(nt) / (nt - 1)
    assert np.max(np.abs(ut - np.exp(-2 * lam * t))) < 1e-6   # float32 grid times
    assert abs(ibh - (1 - math.exp(-2 * lam * tmax))) < 1e-6
    _, ibh_last = oracle.bh_indicator(u, tmax, tmax)
    assert abs(ibh_last - ibh) < 1e-12


def test_bh_indicator_collapse_and_window(oracle):
    """Collapse to the trivial solution (fields vanish after t = 0): I_BH = 1; a growing
    amplitude gives a negative I_BH; delta excludes earlier slices from the minimum."""
    u, tmax, nt = _bh_fields(lambda t: np.where(t > 0, 0.0, 1.0))
    assert abs(oracle.bh_indicator(u, tmax, 0.1)[1] - 1.0) < 1e-12
    u, tmax, nt = _bh_fields(lambda t: 1.0 + t)
    assert oracle.bh_indicator(u, tmax, 0.0)[1] == 0.0      # the minimum is U~(0) = 1
    assert oracle.bh_indicator(u, tmax, 0.5)[1] < 0.0       # every slice after 0.5 has grown
    with pytest.raises(ValueError):
        oracle.bh_indicator(u, tmax, tmax * 1.5)


# ----------------------------------------------------------------------------- RFF + MLP premap

def _premap_pin_params(circ, omega, layers, w_out, b_out, head_w, head_b):
    """Flat parameter vector in the documented layout: Omega[F][3], per hidden layer W and b,
    W_out, b_out, (no circuit parameters at L = 0), head W[3][1] and b[3]."""
    parts = [np.asarray(omega, dtype=np.float64).ravel()]
    for Wl, bl in layers:
        parts += [np.asarray(Wl, dtype=np.float64).ravel(), np.asarray(bl, dtype=np.float64).ravel()]
    parts += [np.asarray(w_out, dtype=np.float64).ravel(), np.asarray(b_out, dtype=np.float64).ravel(),
              np.asarray(head_w, dtype=np.float64).ravel(), np.asarray(head_b, dtype=np.float64).ravel()]
    p = np.concatenate(parts)
    assert p.shape[0] == W.param_offsets(circ)["total"][0]
    return p


# <Z> after RX(theta)|0> is cos(theta) (Fig. 3 caption); with the scalings of Eq. 27a-e applied
# to a = tanh(h) this is, as a function of h, and its derivative d<Z>/dh:
_Z_OF_H = {
    "acos": (lambda h: np.tanh(h), lambda h: 1 - np.tanh(h) ** 2),            # <Z> = a
    "asin": (lambda h: -np.tanh(h), lambda h: -(1 - np.tanh(h) ** 2)),        # <Z> = -a
    "pi": (lambda h: np.cos(np.pi * np.tanh(h)),
           lambda h: -np.pi * np.sin(np.pi * np.tanh(h)) * (1 - np.tanh(h) ** 2)),
    "bias": (lambda h: -np.sin(0.5 * np.pi * np.tanh(h)),                      # cos((a+1) pi/2)
             lambda h: -0.5 * np.pi * np.cos(0.5 * np.pi * np.tanh(h)) * (1 - np.tanh(h) ** 2)),
    "none": (lambda h: np.cos(np.tanh(h)), lambda h: -np.sin(np.tanh(h)) * (1 - np.tanh(h) ** 2)),
}


@pytest.mark.parametrize("scale", ["acos", "asin", "pi", "bias", "none"])
@pytest.mark.parametrize("enc", ["rx", "ry"])
def test_rff_premap_depth0_closed_form(oracle, scale, enc):
    """One qubit, no ansatz layer, one frequency per input axis: the RFF features of Sec. 2.2
    are (cos(omega v_d), sin(omega v_d)) and with no hidden layer the encoding angle is
    scale(tanh(w_c cos(omega v_d) + w_s sin(omega v_d) + b)). The head (W, b) maps <Z> to the
    three fields. Values and all three input derivatives against that closed form."""
    zf, dzf = _Z_OF_H[scale]
    head_w, head_b = np.array([1.0, -0.75, 2.5]), np.array([0.125, -0.5, 0.25])
    for d in range(3):
        omega = np.zeros((1, 3))
        omega[0, d] = 1.7
        wc, ws, b = 0.8, -0.45, 0.3
        circ = W.circuit(1, 0, 1, ansatz="basic_rot", enc=enc, scale=scale, premap="rff_mlp",
                         rff_freqs=1, mlp_width=4, mlp_depth=0)
        params = _premap_pin_params(circ, omega, [], [[wc, ws]], [b], head_w, head_b)
        pts = np.array([[0.3, -0.7, 0.55], [-0.9, 0.2, 0.05], [0.0, 0.6, 0.95]])
        f, df = oracle.forward(circ, params, pts)
        for i, v in enumerate(pts):
            s = 1.7 * v[d]
            h = wc * math.cos(s) + ws * math.sin(s) + b
            dh = 1.7 * (-wc * math.sin(s) + ws * math.cos(s))
            z, dz = zf(h), dzf(h) * dh
            assert np.max(np.abs(f[i] - (head_w * z + head_b))) < 1e-13
            for dd in range(3):
                want = head_w * dz if dd == d else np.zeros(3)
                assert np.max(np.abs(df[i, :, dd] - want)) < 1e-12, (scale, d, dd)


@pytest.mark.parametrize("scale", ["acos", "asin", "pi"])
def test_rff_premap_hidden_layers_closed_form(oracle, scale):
    """One qubit, no ansatz layer, two frequencies over all three axes and one or two tanh
    hidden layers: <Z> = z(h) with h = W_out tanh(... tanh(W_1 r + b_1) ...) + b_out and
    r = [cos(Omega v), sin(Omega v)] (all cosines first, Sec. 2.2). Input derivatives by the
    chain rule written out per layer."""
    zf, dzf = _Z_OF_H[scale]
    rng = np.random.default_rng(3)
    F, H = 2, 3
    omega = rng.normal(size=(F, 3))
    for depth in (1, 2):
        layers = []
        fan = 2 * F
        for _ in range(depth):
            layers.append((rng.uniform(-0.8, 0.8, size=(H, fan)), rng.uniform(-0.3, 0.3, size=H)))
            fan = H
        w_out, b_out = rng.uniform(-0.8, 0.8, size=(1, fan)), rng.uniform(-0.3, 0.3, size=1)
        circ = W.circuit(1, 0, 1, ansatz="noent_rot", enc="rx", scale=scale, premap="rff_mlp",
                         rff_freqs=F, mlp_width=H, mlp_depth=depth)
        head_w, head_b = np.array([1.0, 0.5, -2.0]), np.zeros(3)
        params = _premap_pin_params(circ, omega, layers, w_out, b_out, head_w, head_b)
        pts = W.uniform_points(4, 11).astype(np.float64)
        f, df = oracle.forward(circ, params, pts)
        for i, v in enumerate(pts):
            arg = omega @ v
            u = np.concatenate([np.cos(arg), np.sin(arg)])
            du = np.concatenate([-np.sin(arg)[:, None] * omega, np.cos(arg)[:, None] * omega])
            for Wl, bl in layers:
                y = np.tanh(Wl @ u + bl)
                du = (1 - y ** 2)[:, None] * (Wl @ du)
                u = y
            h = float((w_out @ u + b_out)[0])
            dh = (w_out @ du).ravel()
            z = zf(h)
            assert np.max(np.abs(f[i] - (head_w * z + head_b))) < 1e-13, (scale, depth)
            for d in range(3):
                assert np.max(np.abs(df[i, :, d] - head_w * dzf(h) * dh[d])) < 1e-12, (scale, depth, d)


def test_rff_premap_theta_and_jacobian(oracle):
    """The encoding angles themselves (qpo_premap) for every scaling of Eq. 27a-e at a = tanh(h)
    with h from one RFF frequency and no hidden layer, and their input Jacobian."""
    omega = np.array([[0.9, -1.3, 0.4]])
    wc, ws, b = -0.6, 1.1, 0.2
    pts = W.uniform_points(5, 12).astype(np.float64)
    theta_of_a = {"none": lambda a: a, "pi": lambda a: np.pi * a,
                  "bias": lambda a: (a + 1) * np.pi / 2,
                  "asin": lambda a: np.arcsin(a) + np.pi / 2, "acos": lambda a: np.arccos(a)}
    dtheta_da = {"none": lambda a: 1.0, "pi": lambda a: np.pi, "bias": lambda a: np.pi / 2,
                 "asin": lambda a: 1 / np.sqrt(1 - a * a), "acos": lambda a: -1 / np.sqrt(1 - a * a)}
    for scale in theta_of_a:
        circ = W.circuit(1, 0, 1, ansatz="noent_rot", enc="rx", scale=scale, premap="rff_mlp",
                         rff_freqs=1, mlp_width=2, mlp_depth=0)
        params = _premap_pin_params(circ, omega, [], [[wc, ws]], [b], np.ones(3), np.zeros(3))
        th, J = oracle.premap(circ, params, pts)
        for i, v in enumerate(pts):
            s = float(omega[0] @ v)
            h = wc * math.cos(s) + ws * math.sin(s) + b
            a = math.tanh(h)
            assert abs(th[i, 0] - theta_of_a[scale](a)) < 1e-13, scale
            dh = (-wc * math.sin(s) + ws * math.cos(s)) * omega[0]
            want = dtheta_da[scale](a) * (1 - a * a) * dh
            assert np.max(np.abs(J[i, 0] - want)) < 1e-12, scale


# ----------------------------------------------------------------------------- Cross-Mesh

@pytest.mark.parametrize("ansatz", ["cross_mesh", "cross_mesh_2rot"])
def test_cross_mesh_single_layer_readout(oracle, ansatz):
    """One Cross-Mesh layer: the CRZ mesh is diagonal, so it leaves every <Z_i> unchanged.
    RX(theta_i) then RX(a_i) (and RZ, which also commutes with Z) gives <Z_i> = cos(theta_i +
    a_i) whatever the CRZ angles, and the gradient of any loss w.r.t. a CRZ angle is 0."""
    n = 4
    circ = W.circuit(n, 1, n, ansatz=ansatz, enc="rx", scale="pi", premap="direct", n_direct=3)
    params = W.init_params(circ, 3).astype(np.float64)
    off = W.param_offsets(circ)
    o, _ = off["circuit"]
    k = W.single_qubit_params(ansatz)
    pts = W.uniform_points(5, 4).astype(np.float64)
    for rows in ([0, 1, 2], [3, 0, 1]):
        p = _set_head(circ, params, rows)
        f, _ = oracle.forward(circ, p, pts)
        for b, v in enumerate(pts):
            theta = [math.pi * v[0], math.pi * v[1], math.pi * v[2], 0.0]
            for c, i in enumerate(rows):
                assert abs(f[b, c] - math.cos(theta[i] + p[o + i * k])) < 1e-13
    prob = W.problem("vacuum", w_energy=10.0)
    sets = {"colloc": pts, "ic": W.ic_points_uniform(3, 5)}
    crz = np.arange(o + n * k, o + n * k + n * (n - 1))
    g = oracle.grad(circ, prob, params, sets, crz)
    assert np.max(np.abs(g)) < 1e-13


def test_crz_gradient_exact_shift_rule(oracle):
    """A CRZ angle theta enters through exp(-i theta P / 2) with P = |1><1|_c (x) Z_t, whose
    eigenvalues are 0 and +-1: the states carry frequencies 0 and 1/2 in theta, the fields
    and input derivatives are trig polynomials of degree 2 in u = theta / 2, the squared
    residuals degree 4 and the squared Poynting residual degree 8. The R = 8 shift rule in u
    is then exact: dL/dtheta = (1/2) dL/du."""
    circ = W.circuit(4, 2, 4, ansatz="cross_mesh_2rot", enc="rx", scale="acos", premap="rff_mlp",
                     **SMALL_MLP)
    prob = W.problem("dielectric", disk_x0=0.2, disk_r=0.5, w_energy=10.0, energy_slice=4,
                     energy_nt=2)
    sets = {"colloc": W.uniform_points(6, 40), "ic": W.ic_points_uniform(3, 41),
            "bc": W.bc_points(2, 42)}
    params = W.init_params(circ, 8).astype(np.float64)
    lay = oracle.param_layout(circ)
    per = (lay["head"] - lay["circuit"]) // 2
    idx = [lay["circuit"] + 8 + j for j in (0, 5, 11)] + [lay["circuit"] + per + 8 + 7, lay["circuit"] + 3]
    g = oracle.grad(circ, prob, params, sets, idx)
    for j, i in enumerate(idx):
        def fn(u, i=i):
            pp = params.copy()
            pp[i] = 2.0 * u
            return oracle.loss(circ, prob, pp, sets)[0]
        want = 0.5 * _shift_rule(fn, params[i] / 2.0, 8)
        assert abs(want - g[j]) < 1e-10 * max(1.0, abs(g[j])), (i, want, g[j])


# ----------------------------------------------------------------------------- intuitive loss

def _plane_wave_fields(pts, k, w):
    """Ez = cos(kx - w t), Hx = 0, Hy = -(k/w) cos(kx - w t) with w given per point: it solves
    the TM system (Eqs. 8-10) in a medium of permittivity k^2 / w^2."""
    ph = k * pts[:, 0] - w * pts[:, 2]
    a = -k / w
    f = np.stack([np.cos(ph), np.zeros_like(ph), a * np.cos(ph)], axis=1)
    df = np.zeros((pts.shape[0], 3, 3))
    df[:, 0, 0] = -k * np.sin(ph)
    df[:, 0, 2] = w * np.sin(ph)
    df[:, 2, 0] = -a * k * np.sin(ph)
    df[:, 2, 2] = a * w * np.sin(ph)
    return f, df, ph


def test_intuitive_dielectric_loss(oracle):
    """Eqs. 34-35: res1 with eps = eps_r on the dielectric set and 1 elsewhere, one MSE over all
    collocation points. A plane wave whose speed is 1/sqrt(eps) of each point's own region
    makes it vanish (and res2, res3), while Eq. 13's smooth eps(x, y) does not; with the
    vacuum speed everywhere, res1 = k (1 - 1/eps_r) sin(kx - wt) on the dielectric set only."""
    prob = W.problem("dielectric", disk_x0=0.2, disk_r=0.5, w_energy=0.0, phys_loss="intuitive")
    split = W.problem("dielectric", disk_x0=0.2, disk_r=0.5, w_energy=0.0)
    pts = W.uniform_points(400, 21).astype(np.float64)
    inside = ((pts[:, 0].astype(np.float32) - np.float32(0.2)) ** 2 +
              pts[:, 1].astype(np.float32) ** 2) < np.float32(0.5) ** 2
    assert 20 < inside.sum() < 380
    k, er = 2.0, prob["eps_r"]
    f, df, _ = _plane_wave_fields(pts, k, np.where(inside, k / math.sqrt(er), k))
    out = oracle.loss_from_fields(prob, pts, f, df)
    assert abs(out[5]) < 1e-13 and out[6] == 0.0 and abs(out[7]) < 1e-15 and abs(out[8]) < 1e-13
    assert abs(out[1]) < 1e-12
    assert oracle.loss_from_fields(split, pts, f, df)[1] > 1e-3
    f, df, ph = _plane_wave_fields(pts, k, np.full(pts.shape[0], k))
    out = oracle.loss_from_fields(prob, pts, f, df)
    m = np.mean(np.where(inside, (k * (1 - 1 / er) * np.sin(ph)) ** 2, 0.0))
    assert abs(out[5] - m) < 1e-13 and out[6] == 0.0 and abs(out[1] - m) < 1e-12


# ----------------------------------------------------------------------------- symmetry penalty

@pytest.mark.parametrize("medium", ["vacuum", "dielectric"])
def test_sym_penalty_closed_form(oracle, medium):
    """Eq. 18 on a circuit whose outputs have known parities: one qubit per input, RX(pi v_j),
    no ansatz layer, so z_0 = cos(pi x), z_1 = cos(pi y), z_2 = cos(pi t) are all even in x and
    y. Ez = z_0 + z_1 satisfies (i), so with Hx = Hy = 0 the penalty is 0. Hx = z_0 breaks the
    odd-in-y parity of (ii): (Hx + Hx(x,-y))^2 = 4 cos^2(pi x). Hy = z_1 breaks the odd-in-x
    parity of (iii): 4 cos^2(pi y), a term the dielectric case leaves out."""
    circ = W.circuit(3, 0, 3, ansatz="noent_rot", enc="rx", scale="pi", premap="direct", n_direct=3)
    prob = W.problem(medium, disk_x0=0.5, disk_r=0.25, w_ic=0.0, w_bc=0.0, w_energy=0.0, w_sym=10.0)
    pts = W.uniform_points(40, 6).astype(np.float64)
    off = W.param_offsets(circ)
    o, _ = off["head_W"]
    p = np.zeros(off["total"][0])
    p[o + 0] = p[o + 1] = 1.0                      # Ez = z_0 + z_1
    lo = oracle.loss(circ, prob, p, {"colloc": pts})
    assert abs(lo[-1]) < 1e-14
    p[o + 3] = 1.0                                  # Hx = z_0
    p[o + 7] = 1.0                                  # Hy = z_1
    lo = oracle.loss(circ, prob, p, {"colloc": pts})
    want = 4 * np.cos(np.pi * pts[:, 0]) ** 2
    if medium == "vacuum":
        want = want + 4 * np.cos(np.pi * pts[:, 1]) ** 2
    assert abs(lo[-1] - 10.0 * np.mean(want)) < 1e-12
    assert abs(lo[0] - (lo[1] + lo[4] + lo[-1])) < 1e-12


def test_sym_from_fields_parities(oracle):
    """Fields built with the parities (i)-(iii) give L_sym = 0; flipping a sign of one mirrored
    field gives 4 f^2 for that term."""
    prob = W.problem("vacuum", w_sym=1.0)
    rng = np.random.default_rng(2)
    pts = rng.uniform(-1, 1, (30, 3))
    x, y = pts[:, 0], pts[:, 1]
    def fields(x, y):
        return np.stack([np.cos(x) * np.cos(2 * y), np.cos(3 * x) * np.sin(y), np.sin(x) * np.cos(y)], axis=1)
    fc, fmx, fmy = fields(x, y), fields(-x, y), fields(x, -y)
    assert abs(oracle.sym_from_fields(prob, fc, fmx, fmy)) < 1e-15
    fmy_bad = fmy.copy()
    fmy_bad[:, 1] *= -1.0                           # Hx(x, -y) = +Hx(x, y): (ii) violated
    got = oracle.sym_from_fields(prob, fc, fmx, fmy_bad)
    assert abs(got - np.mean(4 * fc[:, 1] ** 2)) < 1e-14


def test_sym_penalty_gradient_exact_shift_rule(oracle):
    """With L_sym on, every loss term is still a trig polynomial of degree <= 4 in each circuit
    angle (squares of sums of first-harmonic fields): the R = 4 shift rule gives the exact
    gradient, also through the mirrored evaluations."""
    circ = W.circuit(4, 2, 4, ansatz="strong_rot", enc="rx", scale="acos", premap="rff_mlp", **SMALL_MLP)
    prob = W.problem("vacuum", w_energy=10.0, w_sym=10.0)
    sets = {"colloc": W.uniform_points(6, 50), "ic": W.ic_points_uniform(3, 51)}
    params = W.init_params(circ, 9).astype(np.float64)
    lay = oracle.param_layout(circ)
    idx = np.arange(lay["circuit"], lay["head"], 5)
    g = oracle.grad(circ, prob, params, sets, idx)
    for j, i in enumerate(idx):
        def fn(x, i=i):
            pp = params.copy()
            pp[i] = x
            return oracle.loss(circ, prob, pp, sets)[0]
        assert abs(_shift_rule(fn, params[i], 4) - g[j]) < 1e-10 * max(1.0, abs(g[j])), i


# ----------------------------------------------------------------------------- periodic input map

def _periodic_circ(**kw):
    return W.circuit(4, 2, 4, ansatz="strong_rot", enc="rx", scale="acos", premap="rff_mlp",
                     rff_freqs=5, mlp_width=6, mlp_depth=2, periodic=True, **kw)


def test_periodic_map_periodicity(oracle):
    """Eqs. 25-26 make the network periodic: f(x + 2, y, t) = f(x, y + 2, t) = f(x, y, t + T) =
    f(x, y, t) for the domain lengths 2 and the learned period T, fields and input derivatives."""
    circ = _periodic_circ()
    params = W.init_params(circ, 3).astype(np.float64)
    T = params[W.param_offsets(circ)["period"][0]]
    pts = W.uniform_points(12, 4).astype(np.float64)
    f, df = oracle.forward(circ, params, pts)
    for shift in (np.array([2.0, 0, 0]), np.array([0, -2.0, 0]), np.array([0, 0, T])):
        g, dg = oracle.forward(circ, params, pts + shift)
        assert np.max(np.abs(g - f)) < 1e-11 and np.max(np.abs(dg - df)) < 1e-10


def test_periodic_map_derivatives_vs_fd(oracle):
    """Input derivatives through the periodic map, and the gradient w.r.t. the learned period,
    against central differences."""
    circ = _periodic_circ()
    params = W.init_params(circ, 5).astype(np.float64)
    pts = W.uniform_points(6, 8).astype(np.float64)
    f, df = oracle.forward(circ, params, pts)
    h = 1e-5
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (oracle.forward(circ, params, pts + e)[0] - oracle.forward(circ, params, pts - e)[0]) / (2 * h)
        assert np.max(np.abs(fd - df[:, :, d])) < 1e-7
    prob = W.problem("vacuum", w_energy=10.0)
    sets = {"colloc": pts, "ic": W.ic_points_uniform(3, 9)}
    it = W.param_offsets(circ)["period"][0]
    g = oracle.grad(circ, prob, params, sets, [it])[0]
    pp, pm = params.copy(), params.copy()
    pp[it] += h
    pm[it] -= h
    fd = (oracle.loss(circ, prob, pp, sets)[0] - oracle.loss(circ, prob, pm, sets)[0]) / (2 * h)
    assert abs(fd - g) < 1e-6 * max(1.0, abs(g))
    assert abs(g) > 1e-6


def test_periodic_map_closed_form(oracle):
    """One qubit, no ansatz layer, one frequency selecting sin(2 pi x / 2) (Omega = e_1), no
    hidden layer, acos scaling: <Z> = tanh(w_c cos(sin(pi x)) + w_s sin(sin(pi x)) + b) (Fig. 3,
    Sec. 2.2 RFF and Eq. 25), and the time feature t / T enters only through the period."""
    circ = W.circuit(1, 0, 1, ansatz="noent_rot", enc="rx", scale="acos", premap="rff_mlp",
                     rff_freqs=1, mlp_width=2, mlp_depth=0, periodic=True)
    wc, ws, b = 0.7, -0.4, 0.1
    p = np.concatenate([[1.0, 0, 0, 0, 0, 0], [3.0], [wc, ws], [b], [1.0, 0, 0], [0, 0, 0]])
    assert p.shape[0] == W.param_offsets(circ)["total"][0]
    pts = W.uniform_points(7, 10).astype(np.float64)
    f, df = oracle.forward(circ, p, pts)
    for i, v in enumerate(pts):
        u = math.sin(math.pi * v[0])
        h = wc * math.cos(u) + ws * math.sin(u) + b
        assert abs(f[i, 0] - math.tanh(h)) < 1e-13
        dh = (-wc * math.sin(u) + ws * math.cos(u)) * math.pi * math.cos(math.pi * v[0])
        assert abs(df[i, 0, 0] - (1 - math.tanh(h) ** 2) * dh) < 1e-12
        assert abs(df[i, 0, 1]) < 1e-15 and abs(df[i, 0, 2]) < 1e-15
