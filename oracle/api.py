"""ctypes binding of the FP64 oracle (test infrastructure only).

Configs are passed as plain dicts (see ``paper_2506_23246_b300.workloads``) and
converted to the oracle's own integer/double arrays here; the numeric meaning of
those arrays is documented at the top of ``qp_oracle.cpp``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

ANSATZ = {"basic_ryrz": 0, "basic_rot": 1, "strong_rot": 2, "noent_rot": 3, "cross_mesh": 4,
          "cross_mesh_2rot": 5, "cross_mesh_cnot": 6}
ENC = {"rx": 0, "ry": 1}
SCALE = {"none": 0, "pi": 1, "bias": 2, "asin": 3, "acos": 4}
PREMAP = {"direct": 0, "rff_mlp": 1}
NLOSS = 9
PHYS_LOSS = {"split": 0, "intuitive": 1}

_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.qpo_param_count.restype = _I64
        L.qpo_param_count.argtypes = [_P]
        L.qpo_param_layout.argtypes = [_P, _P]
        L.qpo_premap.argtypes = [_P, _P, _P, _I64, _P, _P]
        L.qpo_forward.argtypes = [_P, _P, _P, _I64, _P, _P, ctypes.c_int]
        L.qpo_state.argtypes = [_P, _P, _P, _P, _P]
        L.qpo_layer_unitary.argtypes = [_P, _P, ctypes.c_int, _P, _P]
        L.qpo_loss.argtypes = [_P, _P, _P, _P, _P, _I64, _P, _I64, _P, _I64, _P, ctypes.c_int]
        L.qpo_grad.argtypes = [_P, _P, _P, _P, _P, _I64, _P, _I64, _P, _I64, _P, _I64, _P,
                               ctypes.c_int]
        L.qpo_count_diel.restype = _I64
        L.qpo_count_diel.argtypes = [_P, _P, _P, _I64]
        L.qpo_loss_from_fields.argtypes = [_P, _P, _P, _I64, _P, _P, _P, _I64, _P, _P, _I64, _P, _P]
        L.qpo_sym_from_fields.argtypes = [_P, _P, _I64, _P, _P, _P]
        L.qpo_sym_from_fields.restype = ctypes.c_double
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def circ_array(circ):
    return np.array([circ["n_qubits"], circ["n_layers"], circ["n_readout"], ANSATZ[circ["ansatz"]],
                     ENC[circ["enc"]], SCALE[circ["scale"]], PREMAP[circ["premap"]],
                     circ.get("n_direct", 3), circ.get("rff_freqs", 0), circ.get("mlp_width", 0),
                     circ.get("mlp_depth", 0), 1 if circ.get("periodic") else 0], dtype=np.int32)


def prob_arrays(prob, norm=None):
    """norm: optional sharding of one loss over several calls, dict with the whole-loss counts
    n_colloc, n_ic, n_bc, the whole set's n_diel (points inside the disk) and colloc_offset
    (global index of this call's first collocation point)."""
    nm = norm or {}
    pi = np.array([1 if prob["medium"] == "dielectric" else 0, prob.get("energy_slice", 0),
                   prob.get("energy_nt", 0), nm.get("n_colloc", 0), nm.get("n_ic", 0),
                   nm.get("n_bc", 0), nm.get("n_diel", 0), nm.get("colloc_offset", 0),
                   PHYS_LOSS[prob.get("phys_loss", "split")]], dtype=np.int32)
    pd = np.array([prob["eps_r"], prob["disk_r"], prob["disk_x0"], prob["disk_y0"],
                   prob["sigmoid_w"], prob["ic_sigma"], prob["ic_x0"], prob["ic_y0"], prob["w_ic"],
                   prob["w_bc"], prob["w_energy"], prob.get("w_sym", 0.0)], dtype=np.float64)
    return pi, pd


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def param_count(circ):
    return int(lib().qpo_param_count(_ptr(circ_array(circ))))


def param_layout(circ):
    out = np.zeros(4, dtype=np.int64)
    ci = circ_array(circ)
    if lib().qpo_param_layout(_ptr(ci), _ptr(out)) != 0:
        raise ValueError("bad circuit")
    return {"circuit": int(out[0]), "head": int(out[1]), "total": int(out[2]), "fixed": int(out[3])}


def premap(circ, params, pts):
    ci = circ_array(circ)
    p = _f64(params)
    x = _f64(pts).reshape(-1, 3)
    n = circ["n_qubits"]
    th = np.zeros((x.shape[0], n))
    J = np.zeros((x.shape[0], n, 3))
    if lib().qpo_premap(_ptr(ci), _ptr(p), _ptr(x), x.shape[0], _ptr(th), _ptr(J)) != 0:
        raise ValueError("bad circuit")
    return th, J


def forward(circ, params, pts, nthreads=None):
    ci = circ_array(circ)
    p = _f64(params)
    x = _f64(pts).reshape(-1, 3)
    f = np.zeros((x.shape[0], 3))
    df = np.zeros((x.shape[0], 3, 3))
    nt = nthreads or os.cpu_count() or 1
    if lib().qpo_forward(_ptr(ci), _ptr(p), _ptr(x), x.shape[0], _ptr(f), _ptr(df), nt) != 0:
        raise ValueError("bad circuit")
    return f, df


def state(circ, params, theta):
    ci = circ_array(circ)
    p = _f64(params)
    th = _f64(theta)
    dim = 1 << circ["n_qubits"]
    re = np.zeros(dim)
    im = np.zeros(dim)
    if lib().qpo_state(_ptr(ci), _ptr(p), _ptr(th), _ptr(re), _ptr(im)) != 0:
        raise ValueError("bad circuit")
    return re + 1j * im


def layer_unitary(circ, params, layer):
    ci = circ_array(circ)
    p = _f64(params)
    dim = 1 << circ["n_qubits"]
    re = np.zeros((dim, dim))
    im = np.zeros((dim, dim))
    if lib().qpo_layer_unitary(_ptr(ci), _ptr(p), layer, _ptr(re), _ptr(im)) != 0:
        raise ValueError("bad layer")
    return re + 1j * im


def _sets(sets):
    out = []
    for key in ("colloc", "ic", "bc"):
        a = sets.get(key)
        a = np.zeros((0, 3)) if a is None else _f64(a).reshape(-1, 3)
        out.append(a)
    return out


def loss(circ, prob, params, sets, norm=None, nthreads=None):
    """Loss terms [9 + energy_nt]. The point evaluations run on nthreads threads (default: all
    cores); the sums run in point order, so the result does not depend on the thread count."""
    ci = circ_array(circ)
    pi, pd = prob_arrays(prob, norm)
    p = _f64(params)
    c, i, b = _sets(sets)
    out = np.zeros(n_loss(prob))
    nt = nthreads or os.cpu_count() or 1
    if lib().qpo_loss(_ptr(ci), _ptr(pi), _ptr(pd), _ptr(p), _ptr(c), c.shape[0], _ptr(i),
                      i.shape[0], _ptr(b), b.shape[0], _ptr(out), nt) != 0:
        raise ValueError("bad circuit")
    return out


def grad(circ, prob, params, sets, idx=None, nthreads=None, norm=None):
    ci = circ_array(circ)
    pi, pd = prob_arrays(prob, norm)
    p = _f64(params)
    c, i, b = _sets(sets)
    if idx is None:
        idx = np.arange(p.shape[0])
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    g = np.zeros(idx.shape[0])
    nt = nthreads or os.cpu_count() or 1
    rc = lib().qpo_grad(_ptr(ci), _ptr(pi), _ptr(pd), _ptr(p), _ptr(c), c.shape[0], _ptr(i),
                        i.shape[0], _ptr(b), b.shape[0], _ptr(idx), idx.shape[0], _ptr(g), nt)
    if rc != 0:
        raise ValueError("bad arguments (%d)" % rc)
    return g


def loss_from_fields(prob, colloc, fc, dfc, ic=None, fi=None, bc=None, fb=None):
    pi, pd = prob_arrays(prob)
    c = _f64(colloc).reshape(-1, 3)
    fc = _f64(fc).reshape(-1, 3)
    dfc = _f64(dfc).reshape(-1, 9)
    ic = np.zeros((0, 3)) if ic is None else _f64(ic).reshape(-1, 3)
    fi = np.zeros((0, 3)) if fi is None else _f64(fi).reshape(-1, 3)
    bc = np.zeros((0, 3)) if bc is None else _f64(bc).reshape(-1, 3)
    fb = np.zeros((0, 3)) if fb is None else _f64(fb).reshape(-1, 3)
    out = np.zeros(n_loss(prob))
    lib().qpo_loss_from_fields(_ptr(pi), _ptr(pd), _ptr(c), c.shape[0], _ptr(fc), _ptr(dfc),
                               _ptr(ic), ic.shape[0], _ptr(fi), _ptr(bc), bc.shape[0], _ptr(fb),
                               _ptr(out))
    return out


def sym_from_fields(prob, fc, fmx, fmy):
    """w_sym L_sym (Eq. 18) from fields at the points, at (-x, y, t) and at (x, -y, t)."""
    pi, pd = prob_arrays(prob)
    fc, fmx, fmy = (_f64(a).reshape(-1, 3) for a in (fc, fmx, fmy))
    return float(lib().qpo_sym_from_fields(_ptr(pi), _ptr(pd), fc.shape[0], _ptr(fc), _ptr(fmx), _ptr(fmy)))


def n_loss(prob):
    """Length of the loss-term array: the 9 terms, the energy slices, then w_sym L_sym when the
    symmetry penalty is on."""
    return NLOSS + max(prob.get("energy_nt", 0), 0) + (1 if prob.get("w_sym", 0.0) > 0 else 0)


def count_dielectric(prob, pts):
    """Points of pts [n,3] inside the dielectric disk (the loss's own test)."""
    pi, pd = prob_arrays(prob)
    p = _f64(pts).reshape(-1, 3)
    return int(lib().qpo_count_diel(_ptr(pi), _ptr(pd), _ptr(p), p.shape[0]))


def bh_indicator(energy, t_max, delta):
    """Black-hole collapse indicator of Sec. 5 ("Black hole" loss landscape) from the energy
    slices U(t_k) (Eq. 31) of a loss evaluation on the uniform time grid t_k = t_max k/(nt-1):
    the normalised energy U~(t_k) = U(t_k) / U(0) and I_BH = 1 - min over t_k >= delta of
    U~(t_k). Returns (U~ [nt], I_BH). Plain definition, FP64."""
    u = np.asarray(energy, dtype=np.float64)
    nt = u.shape[0]
    if nt < 2 or not t_max > 0 or not 0 <= delta <= t_max:
        raise ValueError("need nt >= 2 and 0 <= delta <= t_max")
    t = t_max * np.arange(nt) / (nt - 1)
    ut = u / u[0]
    return ut, float(1.0 - np.min(ut[t >= delta - 1e-12 * t_max]))
