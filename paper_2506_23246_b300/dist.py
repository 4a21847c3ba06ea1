"""Data parallelism of the QPINN step over ranks (one process per GPU).

Every collocation, initial-condition and boundary point is independent, so a step shards by
points: each rank evaluates the loss terms and gradient of its own points, and one exchange
sums them. The loss terms are means over the whole point sets (Eqs. 11-17, 23) and the
dielectric split of Eq. 13 divides by the number of points inside and outside the disk, so a
rank must know the whole-loss counts before it evaluates: `shard_norm` gathers them once per
point layout (the counts of every rank, the collocation offsets that place each rank's points
in the energy slices of Eq. 31, and the whole set's number of points inside the disk). With
those normalisers the ranks' loss terms and gradients add up exactly to those of the whole
batch (`allreduce_loss_grad`).

The compute itself is the caller's: `Plan.loss_grad(..., norm=...)` on a GPU.
"""
import torch
import torch.distributed as dist


def shard_range(n, rank, world):
    """Contiguous [start, end) of n items owned by `rank` (the first n % world ranks get one more)."""
    q, r = divmod(int(n), int(world))
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def shard_sets(sets, rank, world):
    """This rank's contiguous slice of every point set of `sets` (dict of [n, 3] arrays/tensors)."""
    out = {}
    for k in ("colloc", "ic", "bc"):
        a = sets.get(k)
        if a is None:
            continue
        s, e = shard_range(a.shape[0], rank, world)
        out[k] = a[s:e]
    return out


def shard_norm(local_counts, n_diel_local, group=None, device=None):
    """Whole-loss normalisers of this rank's shard (collective over `group`).

    local_counts: (n_colloc, n_ic, n_bc) of this rank's sets; n_diel_local: a one-element
    int64 tensor (or int) with this rank's collocation points inside the dielectric disk.
    Returns the dict `Plan.loss_grad(norm=...)` takes: n_colloc, n_ic, n_bc, n_diel (whole
    loss) and colloc_offset (global index of this rank's first collocation point)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if torch.is_tensor(n_diel_local):
        dev = n_diel_local.device if device is None else device
        nd = n_diel_local.reshape(1).to(device=dev, dtype=torch.int64)
    else:
        dev = torch.device("cpu") if device is None else device
        nd = torch.tensor([int(n_diel_local)], dtype=torch.int64, device=dev)
    mine = torch.cat([torch.tensor([int(c) for c in local_counts], dtype=torch.int64, device=dev), nd])
    every = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(every, mine, group=group)
    table = torch.stack(every).cpu().tolist()
    tot = [sum(row[i] for row in table) for i in range(4)]
    off = sum(table[r][0] for r in range(rank))
    return {"n_colloc": tot[0], "n_ic": tot[1], "n_bc": tot[2], "n_diel": tot[3], "colloc_offset": off}


def allreduce_loss_grad(loss, grad, group=None):
    """Sum the ranks' loss terms (float64) and gradients (float32) in place: with whole-loss
    normalisers every entry is additive over the shards."""
    dist.all_reduce(loss, group=group)
    dist.all_reduce(grad, group=group)
    return loss, grad


def data_parallel_loss_grad(compute, count_inside, local_sets, group=None):
    """One loss and gradient of the union of every rank's `local_sets`.

    compute(local_sets, norm) -> (loss, grad) evaluates this rank's share with the whole-loss
    normalisers; count_inside(colloc) -> one-element int64 tensor counts this rank's
    collocation points inside the dielectric disk. Returns the summed (loss, grad)."""
    counts = tuple(int(local_sets[k].shape[0]) if local_sets.get(k) is not None else 0
                   for k in ("colloc", "ic", "bc"))
    device = next((t.device for t in local_sets.values() if torch.is_tensor(t)), None)
    colloc = local_sets.get("colloc")
    nd = count_inside(colloc) if colloc is not None and colloc.shape[0] > 0 else 0
    norm = shard_norm(counts, nd, group, device=device)
    loss, grad = compute(local_sets, norm)
    return allreduce_loss_grad(loss, grad, group)
