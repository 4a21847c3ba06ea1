"""Allocation-free forward call (qp_forward_noalloc), checked through the C-ABI.

Callers that cannot allocate device memory (a pool that refuses new allocations, a plugin
with a fixed device budget) use this entry point instead of qp_forward; it runs in a fixed
device array owned by the library. Its results must equal those of qp_forward on the same
inputs, call after call, since every call reuses and overwrites the same array.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2506_23246_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the per-group relative bar of the other GPU parity tests


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-12))


def test_forward_noalloc_matches_forward_on_consecutive_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_23246_b300 import build, qp
    build.build()
    fn = qp.lib().qp_forward_noalloc
    fn.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64] + [ctypes.c_void_p] * 3
    fn.restype = ctypes.c_int32

    circ = W.c3_circuit(8, 6)
    plan = qp.Plan(circ, W.c3_problem("dielectric"))
    dp = torch.tensor(W.init_params(circ, 0), device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    batches = [W.grid_points(16, 16, 4, 0.7), W.uniform_points(1000, 3, 0.7)]
    for pts in batches:  # two calls in a row, different sizes and contents
        dx = torch.tensor(pts, device="cuda")
        f_ref, df_ref = plan.forward(dp, dx)
        f = torch.full_like(f_ref, float("nan"))
        df = torch.full_like(df_ref, float("nan"))
        rc = fn(plan._h, dp.data_ptr(), dx.data_ptr(), dx.shape[0], f.data_ptr(), df.data_ptr(),
                stream)
        assert rc == 0, qp.lib().qp_status_str(rc)
        torch.cuda.synchronize()
        assert _rel(f.cpu().numpy(), f_ref.cpu().numpy()) < TOL
        assert _rel(df.cpu().numpy(), df_ref.cpu().numpy()) < TOL

    # a batch beyond the fixed array is refused before anything runs
    rc = fn(plan._h, dp.data_ptr(), dx.data_ptr(), 10 ** 7, f.data_ptr(), df.data_ptr(), stream)
    assert rc == 3


def _fn():
    from paper_2506_23246_b300 import qp
    fn = qp.lib().qp_forward_noalloc
    fn.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64] + [ctypes.c_void_p] * 3
    fn.restype = ctypes.c_int32
    return fn


def test_forward_noalloc_equals_simt_forward_and_oracle(oracle):
    """The call always runs the FP32 SIMT kernels. On a SIMT plan with the direct premap it
    runs exactly the kernels qp_forward runs, so the outputs are identical; on a plan whose
    qp_forward takes the tensor cores (8 qubits, RFF + MLP premap) both are held to the FP64
    oracle. After the call, qp_last_device_error reads the call's own status word."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_23246_b300 import build, qp
    build.build()
    fn = _fn()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    circ = W.circuit(6, 4, 3, ansatz="basic_ryrz", enc="ry", scale="pi", premap="direct")
    plan = qp.Plan(circ, path="simt")
    dp = torch.tensor(W.init_params(circ, 3), device="cuda")
    for seed in (4, 5):
        dx = torch.tensor(W.uniform_points(777, seed), device="cuda")
        f_ref, df_ref = plan.forward(dp, dx)
        f = torch.full_like(f_ref, float("nan"))
        df = torch.full_like(df_ref, float("nan"))
        assert fn(plan._h, dp.data_ptr(), dx.data_ptr(), dx.shape[0], f.data_ptr(), df.data_ptr(),
                  stream) == 0
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        assert torch.equal(f, f_ref) and torch.equal(df, df_ref)

    circ = W.c3_circuit(8, 6)
    params = W.init_params(circ, 1)
    pts = W.uniform_points(300, 6, 0.7)
    plan = qp.Plan(circ, W.c3_problem("dielectric"))
    dp = torch.tensor(params, device="cuda")
    dx = torch.tensor(pts, device="cuda")
    f = torch.empty(300, 3, device="cuda")
    df = torch.empty(300, 3, 3, device="cuda")
    assert fn(plan._h, dp.data_ptr(), dx.data_ptr(), 300, f.data_ptr(), df.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    fo, dfo = oracle.forward(circ, params, pts)
    assert _rel(f.cpu().numpy(), fo) < TOL
    assert _rel(df.cpu().numpy(), dfo) < TOL
