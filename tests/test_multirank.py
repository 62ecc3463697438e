"""Multi-process host logic on CPU (gloo, world size 2): the row-band split of
one image (its partial sums add up to the whole-image loss and gradient of
the FP64 oracle, Eq. 8 being a sum over pixels), the cost-balanced split of
a batch, and the max-over-ranks timing reduction of the benchmark."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2104_13715_gb300 import shard
from tests._helpers import field

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        m = 7
        d = field(61, 48, m, seed=5)
        spec = oracle.LossSpec(rho="cauchy", noise="ccd", sigma0=4.0, gain=1.3, var_floor=1e-6)
        theta = np.full(m * m + 1, 1.0 / (m * m))
        theta[-1] = float(np.median(d["I"]))
        rng = np.random.default_rng(0)
        mask = (rng.random(d["R"].shape) > 0.07).astype(np.uint8)
        v0, v1 = shard.band_partition(d["R"].shape[0], m, world)[rank]
        rows = shard.band_rows(v0, v1, m)
        L, g = oracle.loss_grad(d["R"][rows], d["I"][rows], m, theta, spec, mask=mask[rows])
        t = torch.tensor(np.concatenate([[L], g]), dtype=torch.float64)
        dist.all_reduce(t)   # the one collective a band-split evaluation needs
        ms, units = shard.reduce_max_sum(10.0 * (rank + 1), rank + 1)
        if rank == 0:
            L0, g0 = oracle.loss_grad(d["R"], d["I"], m, theta, spec, mask=mask)
            q.put(("ok", float(abs(t[0].item() - L0) / abs(L0)),
                   float(np.max(np.abs(t[1:].numpy() - g0)) / np.max(np.abs(g0))), ms, units))
    except Exception as e:   # surfaced in the parent
        q.put(("error", repr(e), 0.0, 0.0, 0.0))
        raise
    finally:
        dist.destroy_process_group()


def test_band_split_sums_to_whole_image_on_two_gloo_ranks():
    import oracle
    oracle.build()   # once, before the ranks start
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_worker, args=(WORLD, _free_port(), q), nprocs=WORLD, join=True,
                       start_method="spawn")
    status, rel_loss, rel_grad, ms, units = q.get()
    assert status == "ok", rel_loss
    assert rel_loss < 1e-12 and rel_grad < 1e-12, (rel_loss, rel_grad)
    assert (ms, units) == (20.0, 3.0)     # max of 10, 20; sum of 1, 2


@pytest.mark.parametrize("H,m,world", [(61, 7, 2), (61, 7, 3), (20, 5, 8), (128, 25, 5)])
def test_band_partition_covers_valid_rows_once(H, m, world):
    bands = shard.band_partition(H, m, world)
    nv = H - 2 * (m // 2)
    assert bands[0][0] == 0 and bands[-1][1] == nv
    assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
    sizes = [b - a for a, b in bands]
    assert max(sizes) - min(sizes) <= 1
    for a, b in bands:   # image rows read stay inside the image
        r = shard.band_rows(a, b, m)
        assert r.start >= 0 and r.stop <= H


def test_partition_by_cost_is_a_balanced_partition():
    rng = np.random.default_rng(1)
    sides = rng.integers(64, 513, size=512)
    ms = rng.choice(np.arange(7, 22, 2), size=512)
    costs = [shard.pair_cost(s, s, m) for s, m in zip(sides, ms)]
    for world in (1, 2, 4, 8):
        parts = shard.partition_by_cost(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(512))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: the largest load is at most the mean plus the largest unit
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9
    assert shard.partition_by_cost([5.0, 1.0, 1.0, 1.0], 2) == [[0], [1, 2, 3]]
