"""Host logic of the multi-process ensemble (world size 2, gloo, CPU only)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1612_00746_gb300.ensemble import combine_means, max_over_ranks, shard_realizations


def test_shards_are_disjoint_and_cover_everything():
    for total in (1, 5, 1024, 2049):
        for world in (1, 2, 3, 8):
            ids = [shard_realizations(total, world, r) for r in range(world)]
            flat = [i for s in ids for i in s]
            assert flat == list(range(total))
            assert max(map(len, ids)) - min(map(len, ids)) <= 1
    with pytest.raises(ValueError):
        shard_realizations(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank-local means over different realization counts per size group
        rng = np.random.default_rng(rank)
        counts = torch.tensor([3.0, 3.0, 0.0, 0.0] if rank == 0 else [1.0, 1.0, 2.0, 2.0],
                              dtype=torch.float64)
        P = torch.tensor(rng.uniform(size=(2, 4)), dtype=torch.float64)
        got = combine_means(P, counts)
        t = max_over_ranks(1.5 + rank)
        q.put((rank, P.numpy(), counts.numpy(), got.numpy(), t))
    finally:
        dist.destroy_process_group()


def test_combine_means_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in procs], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, P0, c0, g0, t0), (_, P1, c1, g1, t1) = res
    expect = (P0 * c0 + P1 * c1) / np.maximum(c0 + c1, 1)
    np.testing.assert_allclose(g0, expect, rtol=0, atol=1e-15)
    np.testing.assert_allclose(g1, expect, rtol=0, atol=1e-15)
    assert t0 == t1 == 2.5


def test_combine_means_single_process_is_identity():
    P = torch.rand(3, 5, dtype=torch.float64)
    c = torch.tensor([1.0, 2.0, 3.0, 4.0, 0.0], dtype=torch.float64)
    out = combine_means(P, c)
    np.testing.assert_allclose(out[:, :4].numpy(), P[:, :4].numpy())
    assert torch.all(out[:, 4] == 0)


def _graph_worker(rank, world, port, q):
    # each rank propagates its shard of a graph ensemble (the oracle stands in
    # for the per-rank GPU work) and the ranks combine their P means
    import ctqw_workloads as cw
    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = cw.get_graph("graph_small").with_(R=5, n_steps=20, obs_every=10)
        ids = shard_realizations(w.R, world, rank)
        out = oracle.graph_ensemble_run(w, realizations=ids)
        counts = torch.full((w.n_nodes(),), float(len(ids)), dtype=torch.float64)
        got = combine_means(torch.tensor(out["P"], dtype=torch.float64), counts)
        q.put((rank, got.numpy()))
    finally:
        dist.destroy_process_group()


def test_graph_ensemble_sharded_over_two_ranks_gloo():
    """Realization draws depend on the realization id only, so two ranks with
    disjoint shards reproduce the one-process ensemble mean of a graph
    workload (5 realizations: shards of 3 and 2)."""
    import ctqw_workloads as cw
    import oracle

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_graph_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in procs], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = cw.get_graph("graph_small").with_(R=5, n_steps=20, obs_every=10)
    full = oracle.graph_ensemble_run(w)["P"]
    for _, got in res:
        np.testing.assert_allclose(got, full, rtol=0, atol=1e-14)
