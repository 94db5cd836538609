"""Pair sharding for H_M across processes, on CPU ranks over gloo: the union
of the shards equals the single-process result, pair ids included."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2405_08578_gb300 import shard


class FakeCtx:
    """Stands in for lp.Context on CPU: a pair's entry depends only on the
    image indices and its RANSAC pair id, as lp_stitch_pairs_ids' does."""

    def lp_stitch_pairs(self, images, HM, n_in, valid, pairs=None, M_out=None, stream=None, pair_ids=None):
        ids = pair_ids if pair_ids is not None else range(len(pairs))
        for q, ((a, b), pid) in enumerate(zip(pairs, ids)):
            rng = np.random.default_rng(1000 * a + 10 * b + 7 * pid)
            HM[q] = torch.from_numpy(rng.standard_normal(9))
            n_in[q] = int(rng.integers(0, 50))
            valid[q] = int(n_in[q] >= 8)


def _single(n_img):
    pl = shard.all_pairs(n_img)
    P = len(pl)
    HM = torch.zeros((P, 9), dtype=torch.float64)
    n_in = torch.zeros(P, dtype=torch.int32)
    valid = torch.zeros(P, dtype=torch.uint8)
    FakeCtx().lp_stitch_pairs(None, HM, n_in, valid, pairs=pl, pair_ids=list(range(P)))
    return HM.reshape(P, 3, 3), n_in, valid


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_img, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        images = [(torch.zeros(1, dtype=torch.uint8), 1, 1, 16, 1) for _ in range(n_img)]
        HM, n_in, valid = shard.stitch_pairs_sharded(FakeCtx(), images, world, rank)
        q.put((rank, HM.numpy(), n_in.numpy(), valid.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n_img,world", [(9, 2), (4, 2), (2, 2), (5, 3)])
def test_union_of_shards_equals_single_process(n_img, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_img, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    HM, n_in, valid = _single(n_img)
    for _, h, n, v in got:
        assert np.array_equal(h, HM.numpy()) and np.array_equal(n, n_in.numpy()) and np.array_equal(v, valid.numpy())


def test_shard_partition():
    for P in [0, 1, 5, 36, 37]:
        for W in [1, 2, 3, 8]:
            parts = [shard.shard(P, W, r) for r in range(W)]
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(P))
            assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    with pytest.raises(ValueError):
        shard.shard(4, 2, 2)
    assert shard.all_pairs(4) == [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
