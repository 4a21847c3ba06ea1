"""GPU: sharded loss calls (whole-loss normalisers), the dielectric count and the batched
multi-instance step, through the C-ABI."""
import numpy as np
import pytest

from paper_2506_23246_b300 import dist as qdist
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


def test_count_dielectric_matches_oracle(torch_cuda, oracle):
    """Integer count, exact: points near the rim decide in the same float32 arithmetic."""
    from paper_2506_23246_b300 import qp
    torch = torch_cuda
    circ = W.c3_circuit(4, 2)
    prob = W.problem("dielectric", disk_x0=0.2, disk_r=0.6)
    plan = qp.Plan(circ, prob, path="simt")
    for n, seed in ((0, 1), (1, 2), (1000, 3), (70001, 4)):
        pts = W.uniform_points(n, seed, 1.0) if n else np.zeros((0, 3), np.float32)
        c = plan.count_dielectric(torch.tensor(pts, device="cuda"))
        assert int(c.item()) == oracle.count_dielectric(prob, pts)
    vac = qp.Plan(circ, W.problem("vacuum"), path="simt")
    assert int(vac.count_dielectric(torch.tensor(W.uniform_points(100, 5, 1.0), device="cuda")).item()) == 0


@pytest.mark.parametrize("n,L,path", [(6, 3, "simt"), (8, 4, "gemm_split"), (9, 2, "gemm_split")])
def test_sharded_calls_sum_to_whole(torch_cuda, n, L, path):
    """Three uneven shards of a dielectric loss with energy slices (one shard without IC
    points): with the whole-loss normalisers (counts, dielectric count, collocation offsets)
    the shards' loss terms and gradients add up to those of the whole batch."""
    from paper_2506_23246_b300 import qp
    torch = torch_cuda
    circ = W.c3_circuit(n, L)
    prob = W.problem("dielectric", disk_x0=0.2, disk_r=0.6, w_energy=10.0, energy_slice=64,
                     energy_nt=5)
    sets = {"colloc": W.uniform_points(300, n, 1.0), "ic": W.ic_points_uniform(40, n + 1),
            "bc": W.bc_points(20, n + 2)}
    params = W.init_params(circ, n)
    plan = qp.Plan(circ, prob, path=path)
    dp = torch.tensor(params, device="cuda")
    dsets = {k: torch.tensor(v, device="cuda") for k, v in sets.items()}
    lw, gw = plan.loss_grad(dp, dsets)
    lw, gw = lw.cpu().numpy(), gw.cpu().numpy()
    cuts = {"colloc": [0, 97, 211, 300], "ic": [0, 0, 25, 40], "bc": [0, 7, 14, 20]}
    shards = [{k: dsets[k][cuts[k][r]:cuts[k][r + 1]].contiguous() for k in dsets} for r in range(3)]
    nd = sum(int(plan.count_dielectric(s["colloc"]).item()) for s in shards)
    ls, gs, off = 0, 0, 0
    for s in shards:
        norm = {"n_colloc": 300, "n_ic": 40, "n_bc": 20, "n_diel": nd, "colloc_offset": off}
        l, g = plan.loss_grad(dp, s, norm=norm)
        ls = ls + l.cpu().numpy()
        gs = gs + g.cpu().numpy()
        off += s["colloc"].shape[0]
    assert plan.last_device_error() == 0
    assert _rel(ls, lw) < 2e-6
    assert _rel(gs, gw) < 2e-5


def test_sharding_arguments_checked(torch_cuda):
    from paper_2506_23246_b300 import qp
    torch = torch_cuda
    circ = W.c3_circuit(4, 2)
    plan = qp.Plan(circ, W.problem("dielectric"), path="simt")
    dp = torch.tensor(W.init_params(circ, 0), device="cuda")
    c = torch.tensor(W.uniform_points(50, 1, 1.0), device="cuda")
    bad = [{"n_colloc": 49, "n_diel": 0},                       # whole count below this call's
           {"n_colloc": 100, "n_diel": 101},                    # more inside than the whole set
           {"n_colloc": 100, "n_diel": 10, "colloc_offset": 60},  # runs past the whole set
           {"n_colloc": 0, "colloc_offset": 3},                 # offset without a whole count
           {"n_colloc": 100, "n_diel": -1}]
    for nm in bad:
        with pytest.raises(qp.QPError) as e:
            plan.loss_grad(dp, {"colloc": c}, norm=nm)
        assert e.value.code == 1
    plan.loss_grad(dp, {"colloc": c}, norm={"n_colloc": 100, "n_diel": 10, "colloc_offset": 50})
    torch.cuda.synchronize()


def test_batch_step_matches_single_calls(torch_cuda):
    """Uneven instances (4 to 9 qubits, both paths, different point counts) in one batched
    call equal the same instances called one by one."""
    from paper_2506_23246_b300 import qp
    torch = torch_cuda
    specs = [(4, 3, 900), (6, 2, 300), (8, 4, 500), (9, 2, 200), (5, 5, 1200), (7, 2, 64)]
    plans, params, sets, ref = [], [], [], []
    for i, (n, L, B) in enumerate(specs):
        circ = W.c3_circuit(n, L)
        prob = W.problem("vacuum", w_energy=10.0)
        p = qp.Plan(circ, prob)
        dp = torch.tensor(W.init_params(circ, i), device="cuda")
        ds = {"colloc": torch.tensor(W.uniform_points(B, 50 + i, 1.5), device="cuda"),
              "ic": torch.tensor(W.ic_points_uniform(max(B // 16, 1), 90 + i), device="cuda")}
        l, g = p.loss_grad(dp, ds)
        ref.append((l.clone(), g.clone()))
        plans.append(p)
        params.append(dp)
        sets.append(ds)
    out = qp.batch_step(plans, params, sets)
    torch.cuda.synchronize()
    for (l, g), (lr, gr) in zip(out, ref):
        assert _rel(l.cpu().numpy(), lr.cpu().numpy()) < 1e-6
        assert _rel(g.cpu().numpy(), gr.cpu().numpy()) < 1e-6
    with pytest.raises(qp.QPError):
        qp.batch_step([plans[0], plans[0]], [params[0], params[0]], [sets[0], sets[0]])
    assert qp.batch_step([], [], []) == []


TOL = 1e-5
CHAN_TOL = 1e-4


def _mix(torch, specs, seed0=0):
    """Plans, device parameters and device point sets of a list of (n, L, B, medium) instances
    (RFF64 + MLP32 premap, strongly entangling, energy term on the collocation points)."""
    from paper_2506_23246_b300 import qp
    plans, params, sets, host = [], [], [], []
    for i, (n, L, B, medium) in enumerate(specs):
        circ = W.c3_circuit(n, L)
        prob = W.problem(medium, disk_x0=0.2, disk_r=0.6, w_energy=10.0, energy_slice=max(B // 4, 1),
                         energy_nt=4)
        p = W.init_params(circ, seed0 + i)
        st = {"colloc": W.uniform_points(B, 300 + seed0 + i, 1.0),
              "ic": W.ic_points_uniform(max(B // 8, 1), 400 + seed0 + i),
              "bc": W.bc_points(max(B // 10, 1), 500 + seed0 + i)}
        plans.append(qp.Plan(circ, prob))
        params.append(torch.tensor(p, device="cuda"))
        sets.append({k: torch.tensor(v, device="cuda") for k, v in st.items()})
        host.append((circ, prob, p, st))
    return plans, params, sets, host


def test_grouped_batch_matches_oracle(torch_cuda, oracle):
    """A six-instance mix (4 to 8 qubits, vacuum and dielectric, energy slices, ragged point
    counts): four instances share the multi-instance launch, the 7- and 8-qubit ones take the
    tensor-core path on worker streams. Every instance's loss terms and gradient (all circuit
    and head parameters, a sample of the MLP's) against the FP64 oracle at 1e-5."""
    torch = torch_cuda
    specs = [(4, 3, 61, "vacuum"), (5, 2, 90, "dielectric"), (6, 2, 37, "vacuum"), (7, 2, 29, "dielectric"),
             (5, 4, 25, "vacuum"), (8, 2, 21, "vacuum")]
    plans, params, sets, host = _mix(torch, specs)
    assert [p.path for p in plans] == ["simt"] * 3 + ["gemm_split", "simt", "gemm_split"]
    out = qp_batch(plans, params, sets)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    for (loss, grad), pl, (circ, prob, p, st) in zip(out, plans, host):
        assert pl.last_device_error() == 0
        loss = loss.cpu().numpy().astype(np.float64)
        grad = grad.cpu().numpy()
        lo = np.asarray(oracle.loss(circ, prob, p, st), dtype=np.float64)
        for i in range(lo.shape[0]):
            err = abs(loss[i] - lo[i])
            if err < 1e-10:
                continue
            scale = max(abs(lo[i]), abs(lo[0])) if i < 9 else abs(lo[i])
            assert err <= TOL * scale and err <= CHAN_TOL * abs(lo[i]), (circ["n_qubits"], "loss", i)
        lay = oracle.param_layout(circ)
        mlp = rng.choice(np.arange(lay["fixed"], lay["circuit"]), 24, replace=False)
        idx = np.concatenate([np.sort(mlp), np.arange(lay["circuit"], lay["total"])])
        go = np.asarray(oracle.grad(circ, prob, p, st, idx), dtype=np.float64)
        gg = grad[idx].astype(np.float64)
        for lo_, hi_ in ((lay["fixed"], lay["circuit"]), (lay["circuit"], lay["head"]), (lay["head"], lay["total"])):
            sel = (idx >= lo_) & (idx < hi_)
            scale = float(np.max(np.abs(go[sel])))
            err = np.abs(gg[sel] - go[sel])
            assert np.all(err <= TOL * scale + CHAN_TOL * np.abs(go[sel])), (circ["n_qubits"], lo_, hi_)


def qp_batch(plans, params, sets, grouped=True):
    from paper_2506_23246_b300 import qp
    return qp.batch_step(plans, params, sets, grouped=grouped)


def test_grouped_equals_ungrouped_and_tuned(torch_cuda):
    """The multi-instance launch (default shape, then the tuner's choice) against every instance
    run as its own call: the same values up to FP32 summation order."""
    from paper_2506_23246_b300 import qp
    torch = torch_cuda
    specs = [(4, 2, 700, "vacuum"), (5, 3, 1500, "dielectric"), (6, 2, 333, "vacuum"), (7, 3, 900, "vacuum"),
             (7, 1, 50, "dielectric"), (3, 2, 128, "vacuum"), (9, 2, 100, "vacuum")]
    plans, params, sets, _ = _mix(torch, specs, 10)
    ref = [(l.clone(), g.clone()) for l, g in qp_batch(plans, params, sets, grouped=False)]
    got = [(l.clone(), g.clone()) for l, g in qp_batch(plans, params, sets)]
    w, k = qp.batch_tune(plans, params, sets)
    assert w in (4, 8, 12) and k in (1, 4, 16)
    tuned = qp_batch(plans, params, sets)
    torch.cuda.synchronize()
    for (lr, gr), (l1, g1), (l2, g2), pl in zip(ref, got, tuned, plans):
        assert pl.last_device_error() == 0
        for l, g in ((l1, g1), (l2, g2)):
            assert _rel(l.cpu().numpy(), lr.cpu().numpy()) < 1e-6
            assert _rel(g.cpu().numpy(), gr.cpu().numpy()) < 2e-6


def test_grouped_more_instances_than_one_launch(torch_cuda):
    """70 small instances of one qubit count: two launches of the multi-instance kernel (64
    instances at most each), every instance equal to its own call."""
    torch = torch_cuda
    specs = [(4, 1 + i % 3, 17 + 5 * i, "vacuum") for i in range(70)]
    plans, params, sets, _ = _mix(torch, specs, 20)
    ref = [(l.clone(), g.clone()) for l, g in qp_batch(plans, params, sets, grouped=False)]
    got = qp_batch(plans, params, sets)
    torch.cuda.synchronize()
    for (lr, gr), (l, g) in zip(ref, got):
        assert _rel(l.cpu().numpy(), lr.cpu().numpy()) < 1e-6
        assert _rel(g.cpu().numpy(), gr.cpu().numpy()) < 2e-6


def test_batch_flags_and_tuner_arguments(torch_cuda):
    """Unknown flag bits and a duplicated plan are refused before any launch; the tuner on a mix
    without gate-by-gate instances reports no shape."""
    from paper_2506_23246_b300 import qp
    torch = torch_cuda
    plans, params, sets, _ = _mix(torch, [(4, 2, 40, "vacuum"), (8, 2, 30, "vacuum")], 30)
    handles, arr, keep, res = qp._step_args(plans, params, sets, None, None)
    s = torch.cuda.current_stream()
    import ctypes
    rc = qp.lib().qp_batch_step_flags(handles, 2, arr, ctypes.c_void_p(s.cuda_stream), 2)
    assert rc == 1
    assert qp.batch_tune(plans[1:], params[1:], sets[1:]) == (0, 0)
    w, k = qp.batch_tune(plans, params, sets)
    assert w in (4, 8, 12) and k in (1, 4, 16)
    torch.cuda.synchronize()
