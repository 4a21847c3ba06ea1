"""Data-parallel sharding on the CPU: the whole-loss normalisers make the loss terms and the
gradient additive over shards (checked on the FP64 oracle), and the host logic of
paper_2506_23246_b300.dist reproduces the whole batch across two gloo ranks."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2506_23246_b300 import dist as qdist
from paper_2506_23246_b300 import workloads as W


def _case():
    circ = W.circuit(4, 2, 4, ansatz="strong_rot", enc="rx", scale="pi", premap="direct")
    prob = W.problem("dielectric", disk_x0=0.1, disk_r=0.5, w_energy=10.0, energy_slice=10,
                     energy_nt=4)
    sets = {"colloc": W.uniform_points(40, 11, 1.0), "ic": W.ic_points_uniform(9, 12),
            "bc": W.bc_points(6, 13)}
    return circ, prob, W.init_params(circ, 3), sets


def _shard_norms(oracle, prob, shards):
    nd = sum(oracle.count_dielectric(prob, s["colloc"]) for s in shards)
    tot = [sum(s[k].shape[0] for s in shards) for k in ("colloc", "ic", "bc")]
    out, off = [], 0
    for s in shards:
        out.append({"n_colloc": tot[0], "n_ic": tot[1], "n_bc": tot[2], "n_diel": nd, "colloc_offset": off})
        off += s["colloc"].shape[0]
    return out


def test_oracle_shards_sum_to_whole(oracle):
    """Uneven shards (one of them without BC points): loss terms, energy slices and the full
    gradient of the shards, each normalised by the whole-loss counts, add up to the whole."""
    circ, prob, params, sets = _case()
    cuts = {"colloc": [0, 17, 40], "ic": [0, 3, 9], "bc": [0, 6, 6]}
    shards = [{k: sets[k][cuts[k][r]:cuts[k][r + 1]] for k in sets} for r in range(2)]
    norms = _shard_norms(oracle, prob, shards)
    assert norms[0]["n_diel"] == oracle.count_dielectric(prob, sets["colloc"]) > 0
    lw, gw = oracle.loss(circ, prob, params, sets), oracle.grad(circ, prob, params, sets)
    ls = sum(oracle.loss(circ, prob, params, s, norm=nm) for s, nm in zip(shards, norms))
    gs = sum(oracle.grad(circ, prob, params, s, norm=nm) for s, nm in zip(shards, norms))
    assert np.allclose(ls, lw, rtol=1e-12, atol=1e-14)
    assert np.allclose(gs, gw, rtol=1e-11, atol=1e-13 * np.abs(gw).max())
    # without the normalisers the shards are two separate means: not the whole loss
    lo = sum(oracle.loss(circ, prob, params, s) for s in shards)
    assert not np.allclose(lo[:5], lw[:5], rtol=1e-6)


def test_shard_range_covers_all():
    for n in (0, 1, 7, 64, 65537):
        for world in (1, 2, 3, 8):
            spans = [qdist.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            sizes = [e - s for s, e in spans]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    from oracle import api as oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    circ, prob, params, sets = _case()
    local = qdist.shard_sets(sets, rank, world)

    def compute(ls, norm):
        loss = torch.tensor(oracle.loss(circ, prob, params, ls, norm=norm), dtype=torch.float64)
        grad = torch.tensor(oracle.grad(circ, prob, params, ls, norm=norm), dtype=torch.float64)
        return loss, grad

    def count_inside(colloc):
        return torch.tensor([oracle.count_dielectric(prob, colloc)], dtype=torch.int64)

    loss, grad = qdist.data_parallel_loss_grad(compute, count_inside, local)
    np.save(os.path.join(outdir, "loss%d.npy" % rank), loss.numpy())
    np.save(os.path.join(outdir, "grad%d.npy" % rank), grad.numpy())
    dist.destroy_process_group()


def test_gloo_two_ranks_match_whole_batch(oracle):
    """Two CPU ranks (gloo on 127.0.0.1) shard the point sets, gather the whole-loss counts,
    evaluate their shares on the oracle and all-reduce: every rank ends with the loss and
    gradient of the whole batch."""
    circ, prob, params, sets = _case()
    lw, gw = oracle.loss(circ, prob, params, sets), oracle.grad(circ, prob, params, sets)
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True,
                           start_method="spawn")
        for r in range(2):
            loss, grad = np.load(os.path.join(d, "loss%d.npy" % r)), np.load(os.path.join(d, "grad%d.npy" % r))
            assert np.allclose(loss, lw, rtol=1e-12, atol=1e-14)
            assert np.allclose(grad, gw, rtol=1e-11, atol=1e-13 * np.abs(gw).max())
