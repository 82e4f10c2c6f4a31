"""Multi-rank host logic on CPU: two gloo ranks split the SNPs, compute their
shard's hits and permutation minima with the oracle, and the merged result
equals the unsharded one; max-over-ranks timing agrees on every rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from paper_1307_3519_gb300 import shard


def test_shard_bounds_cover_exactly():
    for S in (0, 1, 7, 100, 500_001):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_bounds(S, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == S
            for (a, b), (c, _) in zip(spans, spans[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        d = synth.config(4, T=12, S=301, seed=77)
        perms = synth.make_perms(1307, 2, d["N"])
        b, e = shard.shard_bounds(d["S"], rank, world)
        snps = np.arange(b, e)
        r = oracle.scan(d["expr"], d["geno"], 0.01, snps=snps)
        a, c = np.nonzero(r["hit"])
        hits = np.stack([a, snps[c], r["d"][a, c, 0], r["d"][a, c, 1]], axis=1)
        part = (hits, r["H"][a, c], r["p"][a, c])
        minp = oracle.perm_minp(d["expr"], d["geno"], perms, snps=snps)
        parts = shard.gather_objects(part)
        mins = shard.gather_objects(minp)
        t = shard.max_over_ranks(1.5 + rank)
        if rank == 0:
            q.put((shard.merge_hits(parts), shard.merge_minp(mins), t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_the_unsharded_result():
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    (hits, H, P), minp, t = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 2.5
    d = synth.config(4, T=12, S=301, seed=77)
    r = oracle.scan(d["expr"], d["geno"], 0.01)
    a, c = np.nonzero(r["hit"])
    want = np.stack([a, c, r["d"][a, c, 0], r["d"][a, c, 1]], axis=1)
    order = np.lexsort((want[:, 0], want[:, 1]))
    assert np.array_equal(hits, want[order])
    assert np.array_equal(P, r["p"][a, c][order])
    perms = synth.make_perms(1307, 2, d["N"])
    assert np.array_equal(minp, oracle.perm_minp(d["expr"], d["geno"], perms))
