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


# ---------------------------------------------------------------- cost-balanced shards
def test_shard_by_cost_balances_a_ragged_batch():
    import ctqw_workloads as cw
    from paper_1612_00746_gb300.ensemble import shard_by_cost

    sizes = cw.get("ragged_n128_1024").sizes()
    cost = sizes.astype(np.float64) ** 2
    for world in (1, 2, 3, 8):
        shards = [shard_by_cost(sizes, 2, world, k) for k in range(world)]
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(sizes)))
        for s in shards:
            assert s == sorted(s)
        loads = np.array([cost[s].sum() for s in shards])
        # greedy largest-first: no rank above the mean by more than one realization
        assert loads.max() - loads.mean() <= cost.max()
        if world > 1:
            # contiguous blocks of ids would be far less even on this batch
            blocks = [cost[shard_realizations(len(sizes), world, k)].sum() for k in range(world)]
            assert loads.max() - loads.min() <= max(blocks) - min(blocks)
    with pytest.raises(ValueError):
        shard_by_cost(sizes, 2, 2, 5)


# ---------------------------------------------------------------- gradient reduction
def _grad_setup():
    import ctqw_workloads as cw

    w = cw.Workload(name="grad2", m=2, statistics=0, periodic=False, N=5, R=5, J0=1.0, U=1.0,
                    eps_halfwidth=0.5, J_halfwidth=0.2, sites=(1, 3), dt=0.05, K=6, n_steps=6,
                    obs_every=0, dtype=cw.C128, seed=11)
    target = np.random.default_rng(5).dirichlet(np.ones(w.N))
    return w, target


def _grad_worker(rank, world, port, q):
    # each rank stands in its oracle for the GPU work on its shard: forward
    # P at T, the global mean, the adjoint with the adjusted target, and the
    # gradient sums combined over the ranks
    import ctqw_workloads as cw
    import oracle
    from paper_1612_00746_gb300.ensemble import (adjoint_target, combine_gradients, global_loss,
                                                 shard_realizations as shard)

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, target = _grad_setup()
        ids = shard(w.R, world, rank)
        ue, uj = cw.uniform_draws(w.seed, ids, [w.N] * len(ids))
        params = [oracle.workload_parameters(w, ue[k], uj[k], w.N) for k in range(len(ids))]
        psi0 = oracle.initial_state(w.N, w.m, w.sites, w.statistics)
        P_local = np.zeros(w.N)
        for eps, J in params:
            H = oracle.many_particle_hamiltonian(oracle.single_particle_hamiltonian(eps, J, False), w.m, w.U)
            psi = psi0.copy()
            for _ in range(w.n_steps):
                psi = oracle.taylor_step(H, psi, w.dt, w.K)
            P_local += oracle.site_occupation(psi, w.N, w.m) / len(ids)
        counts = torch.full((w.N,), float(len(ids)), dtype=torch.float64)
        P_global = combine_means(torch.tensor(P_local), counts)
        tgt = adjoint_target(torch.tensor(target), torch.tensor(P_local), P_global)
        _, ge, gJ = oracle.loss_and_adjoint_gradient([p[0] for p in params], [p[1] for p in params],
                                                     w.N, w.m, False, w.U, psi0, w.dt, w.K, w.n_steps,
                                                     tgt.numpy())
        counts_all = combine_means(counts, torch.ones(w.N, dtype=torch.float64)) * world
        g_eps = combine_gradients(torch.tensor(ge.sum(0)), counts, counts_all)
        g_J = combine_gradients(torch.tensor(gJ.sum(0)), counts[:w.N - 1], counts_all[:w.N - 1])
        q.put((rank, global_loss(P_global, torch.tensor(target)), g_eps.numpy(), g_J.numpy()))
    finally:
        dist.destroy_process_group()


def test_gradient_of_the_global_loss_over_two_ranks_gloo():
    """Shards of 3 and 2 realizations: each rank runs its adjoint against the
    adjusted target, and the combined gradient sums equal the one-process
    gradient of the loss on the mean over all 5 realizations."""
    import ctqw_workloads as cw
    import oracle

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grad_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in procs], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w, target = _grad_setup()
    ue, uj = cw.uniform_draws(w.seed, range(w.R), [w.N] * w.R)
    params = [oracle.workload_parameters(w, ue[k], uj[k], w.N) for k in range(w.R)]
    psi0 = oracle.initial_state(w.N, w.m, w.sites, w.statistics)
    loss, ge, gJ = oracle.loss_and_adjoint_gradient([p[0] for p in params], [p[1] for p in params], w.N,
                                                    w.m, False, w.U, psi0, w.dt, w.K, w.n_steps, target)
    scale = max(np.abs(ge).max(), np.abs(gJ).max())
    for _, l, g_eps, g_J in res:
        assert abs(l - loss) <= 1e-14
        np.testing.assert_allclose(g_eps, ge.sum(0), rtol=0, atol=1e-13 * scale)
        np.testing.assert_allclose(g_J, gJ.sum(0), rtol=0, atol=1e-13 * scale)


# ---------------------------------------------------------------- a rank that stops
def _leaving_worker(rank, world, port, q, mode):
    import datetime
    from paper_1612_00746_gb300.ensemble import Heartbeat, RankFailure

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=3))
    hb = Heartbeat(timeout_s=2.0)
    try:
        hb.beat(0)
        hb.check(0)
        if rank == 1:
            q.put((rank, "left"))
            q.close()
            q.join_thread()
            os._exit(0)   # leaves between steps: no collective or launch of its own in flight
        t0 = __import__("time").time()
        try:
            if mode == "heartbeat":
                hb.beat(1)
                hb.check(1)
            else:
                combine_means(torch.ones(3, dtype=torch.float64), torch.ones(3, dtype=torch.float64))
            q.put((rank, "no failure"))
        except RankFailure as e:
            q.put((rank, f"RankFailure after {__import__('time').time() - t0:.1f} s: {e}"))
    finally:
        if rank == 0:
            q.close()
            q.join_thread()
            os._exit(0)   # the group cannot be destroyed cleanly without its peer


@pytest.mark.parametrize("mode", ["heartbeat", "collective"])
def test_a_rank_that_leaves_between_steps_is_reported(mode):
    """Rank 1 leaves after step 0.  Rank 0 learns it on the host, before its
    next launch (heartbeat: the store has no mark of rank 1 for step 1), or
    in the next exchange (the reduction times out); both raise RankFailure
    within seconds instead of blocking."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaving_worker, args=(r, 2, port, q, mode)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = dict(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    assert res[1] == "left"
    assert res[0].startswith("RankFailure"), res[0]
    if mode == "heartbeat":
        assert "rank(s) [1]" in res[0] and "step 1" in res[0]
