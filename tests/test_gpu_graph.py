"""GPU: the loss calls captured into a CUDA graph and replayed give the results of direct calls.

The library's calls allocate nothing and never synchronise; the tensor-core call forks a side
stream (unitary build, gate-gradient chain) and the batched call forks worker streams, all joined
back into the caller's stream. Capturing them into one graph and replaying it must reproduce the
direct calls, and a replay must read the buffers' current contents (new parameters in place)."""
import numpy as np
import pytest

from paper_2506_23246_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_23246_b300 import build
    build.build()
    return torch


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-30)


@pytest.mark.parametrize("n,L,path", [(8, 3, "gemm_split"), (9, 2, "gemm_split"), (6, 3, "simt")])
def test_loss_grad_graph_replay(torch_cuda, n, L, path):
    from paper_2506_23246_b300 import qp
    torch = torch_cuda
    circ = W.c3_circuit(n, L)
    prob = W.problem("dielectric", disk_x0=0.2, disk_r=0.6, w_energy=10.0, energy_slice=64, energy_nt=4)
    plan = qp.Plan(circ, prob, path=path)
    sets = {"colloc": torch.tensor(W.uniform_points(256, 3, 0.7), device="cuda"),
            "ic": torch.tensor(W.ic_points_uniform(40, 4), device="cuda")}
    p0 = W.init_params(circ, 1)
    p1 = W.init_params(circ, 2)
    dp = torch.tensor(p0, device="cuda")
    loss = torch.empty(9 + 4, dtype=torch.float64, device="cuda")
    grad = torch.empty(plan.n_params, dtype=torch.float32, device="cuda")
    plan.reserve(296, torch.device("cuda"))
    l_ref, g_ref = [x.clone() for x in plan.loss_grad(dp, sets)]
    dp.copy_(torch.tensor(p1, device="cuda"))
    l_ref1, g_ref1 = [x.clone() for x in plan.loss_grad(dp, sets)]
    dp.copy_(torch.tensor(p0, device="cuda"))
    plan.loss_grad(dp, sets, out=(loss, grad))   # warm-up on the output buffers
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.loss_grad(dp, sets, out=(loss, grad))
    g.replay()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    assert _rel(loss.cpu().numpy(), l_ref.cpu().numpy()) < 1e-6
    assert _rel(grad.cpu().numpy(), g_ref.cpu().numpy()) < 1e-6
    dp.copy_(torch.tensor(p1, device="cuda"))   # the replay reads the parameters in place
    g.replay()
    torch.cuda.synchronize()
    assert _rel(loss.cpu().numpy(), l_ref1.cpu().numpy()) < 1e-6
    assert _rel(grad.cpu().numpy(), g_ref1.cpu().numpy()) < 1e-6


def test_batch_step_graph_replay(torch_cuda):
    """The batched call (a multi-instance launch for the SIMT instances, worker streams for
    the tensor-core ones) captured and replayed equals the direct batched call."""
    from paper_2506_23246_b300 import qp
    torch = torch_cuda
    specs = [(4, 2, 300), (6, 3, 200), (7, 2, 150), (8, 2, 120), (5, 3, 90)]
    plans, params, sets, outs = [], [], [], []
    for i, (n, L, B) in enumerate(specs):
        circ = W.c3_circuit(n, L)
        prob = W.problem("vacuum", w_energy=10.0)
        pl = qp.Plan(circ, prob)
        plans.append(pl)
        params.append(torch.tensor(W.init_params(circ, 10 + i), device="cuda"))
        sets.append({"colloc": torch.tensor(W.uniform_points(B, 20 + i, 1.5), device="cuda"),
                     "ic": torch.tensor(W.ic_points_uniform(max(B // 16, 1), 40 + i), device="cuda")})
        pl.reserve(B + max(B // 16, 1), torch.device("cuda"))
        outs.append((torch.empty(9, dtype=torch.float64, device="cuda"),
                     torch.empty(pl.n_params, dtype=torch.float32, device="cuda")))
    ref = [(l.clone(), gr.clone()) for l, gr in qp.batch_step(plans, params, sets)]
    qp.batch_step(plans, params, sets, outs=outs)
    torch.cuda.synchronize()
    for o in outs:
        o[0].zero_()
        o[1].zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        qp.batch_step(plans, params, sets, outs=outs)
    g.replay()
    torch.cuda.synchronize()
    for (l, gr), (lr, grr), pl in zip(outs, ref, plans):
        assert pl.last_device_error() == 0
        assert _rel(l.cpu().numpy(), lr.cpu().numpy()) < 1e-6
        assert _rel(gr.cpu().numpy(), grr.cpu().numpy()) < 2e-6


@pytest.mark.parametrize("n,path", [(5, "simt"), (8, "gemm_split")])
def test_deep_premap_graph_replay(torch_cuda, n, path):
    """A layer-by-layer premap (periodic map, three tanh layers; its contractions are library
    GEMMs bound to the call's stream and the plan's workspace) captured and replayed equals the
    direct call, and a replay reads new parameters in place."""
    from paper_2506_23246_b300 import qp
    torch = torch_cuda
    circ = W.circuit(n, 2, n, ansatz="strong_rot", enc="rx", scale="acos", premap="rff_mlp",
                     rff_freqs=24, mlp_width=40, mlp_depth=3, periodic=True)
    prob = W.problem("vacuum", w_energy=10.0, energy_slice=16, energy_nt=2)
    plan = qp.Plan(circ, prob, path=path)
    sets = {"colloc": torch.tensor(W.uniform_points(600, 5, 1.5), device="cuda"),
            "ic": torch.tensor(W.ic_points_uniform(40, 6), device="cuda")}
    p0 = W.init_params(circ, 7)
    p1 = W.init_params(circ, 8)
    dp = torch.tensor(p0, device="cuda")
    loss = torch.empty(9 + 2, dtype=torch.float64, device="cuda")
    grad = torch.empty(plan.n_params, dtype=torch.float32, device="cuda")
    plan.reserve(640, torch.device("cuda"))
    l_ref, g_ref = [x.clone() for x in plan.loss_grad(dp, sets)]
    dp.copy_(torch.tensor(p1, device="cuda"))
    l_ref1, g_ref1 = [x.clone() for x in plan.loss_grad(dp, sets)]
    dp.copy_(torch.tensor(p0, device="cuda"))
    plan.loss_grad(dp, sets, out=(loss, grad))
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.loss_grad(dp, sets, out=(loss, grad))
    g.replay()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    assert _rel(loss.cpu().numpy(), l_ref.cpu().numpy()) < 1e-6
    assert _rel(grad.cpu().numpy(), g_ref.cpu().numpy()) < 1e-6
    dp.copy_(torch.tensor(p1, device="cuda"))
    g.replay()
    torch.cuda.synchronize()
    assert _rel(loss.cpu().numpy(), l_ref1.cpu().numpy()) < 1e-6
    assert _rel(grad.cpu().numpy(), g_ref1.cpu().numpy()) < 1e-6
