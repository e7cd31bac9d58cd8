"""Multi-rank host logic with two gloo ranks on CPU: baseline shards cover
every baseline once, the grid reduction sums the replicas, the timing is the
maximum over ranks, and sharded oracle gridding plus the reduction equals
gridding everything on one rank (the exchange step of multi-GPU gridding)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2502_17789_gb300 import parallel, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        obs = synth.config(1, seed=2, n_stations=10, n_timesteps=4)
        rng = np.random.default_rng(0)
        vis = synth.random_visibilities(rng, obs)
        mine = parallel.shard_baselines(obs.n_baselines, rank, world)
        sub = parallel.sub_observation(obs, mine)
        geom = oracle.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size)
        A = synth.aterms_identity(obs.n_intervals, obs.n_stations).astype(np.complex128)
        pl = oracle.plan(geom, sub.uvw, sub.freqs, sub.aterm_offsets)
        G = oracle.grid(geom, sub.n_stations, sub.baselines, sub.uvw, sub.freqs, sub.aterm_offsets, pl,
                        vis[mine].astype(np.complex128), A)
        Gt = torch.from_numpy(G.copy())
        parallel.reduce_grids(Gt)
        t = parallel.max_over_ranks(1.0 + rank)
        out[rank] = (mine.tolist(), Gt.numpy(), t)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_reduce_and_time():
    import oracle
    oracle.build()
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    shards = [set(out[r][0]) for r in range(world)]
    obs = synth.config(1, seed=2, n_stations=10, n_timesteps=4)
    assert set.union(*shards) == set(range(obs.n_baselines)) and not set.intersection(*shards)
    assert out[0][2] == out[1][2] == 2.0
    np.testing.assert_array_equal(out[0][1], out[1][1])
    rng = np.random.default_rng(0)
    vis = synth.random_visibilities(rng, obs)
    geom = oracle.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size)
    A = synth.aterms_identity(obs.n_intervals, obs.n_stations).astype(np.complex128)
    pl = oracle.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    G = oracle.grid(geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl,
                    vis.astype(np.complex128), A)
    assert np.linalg.norm(out[0][1] - G) / np.linalg.norm(G) < 1e-12


def test_shard_validation():
    with pytest.raises(ValueError):
        parallel.shard_baselines(10, 2, 2)
    assert parallel.shard_baselines(5, 1, 2).tolist() == [1, 3]


def _sharded_worker(rank, world, port, out):
    """The bench's multi-GPU step on CPU ranks, the oracle standing in for the
    library: shard_observation, then sharded_step (grid into the replica,
    all-reduce, degrid the shard from the model grid)."""
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        obs = synth.config(1, seed=3, n_stations=9, n_timesteps=4)
        rng = np.random.default_rng(1)
        vis = synth.random_visibilities(rng, obs).astype(np.complex128)
        A = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes).astype(np.complex128)
        sub, mine = parallel.shard_observation(obs, rank, world)
        geom = oracle.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size)
        pl = oracle.plan(geom, sub.uvw, sub.freqs, sub.aterm_offsets)
        args = (geom, sub.n_stations, sub.baselines, sub.uvw, sub.freqs, sub.aterm_offsets, pl)
        N = obs.grid_size
        model = torch.from_numpy(np.fft.fft2(rng.standard_normal((4, N, N))) * 1e-3)
        pred = {}

        def grid_fn(g):
            g += torch.from_numpy(oracle.grid(*args, vis[mine], A))

        def degrid_fn():
            pred["v"] = oracle.degrid(*args, model.numpy(), A)

        G = torch.full((4, N, N), 5.0 + 5.0j, dtype=torch.complex128)   # zeroed by the step
        parallel.sharded_step(grid_fn, degrid_fn, G, world)
        out[rank] = (mine.tolist(), G.numpy(), pred["v"], model.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_bench_sharded_step_on_gloo_ranks(world):
    """Every rank ends the step with the whole observation's grid (the sum of
    the shard replicas equals gridding all baselines at once), and the ranks'
    predicted visibilities together are the whole observation's."""
    import oracle
    oracle.build()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_sharded_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    obs = synth.config(1, seed=3, n_stations=9, n_timesteps=4)
    rng = np.random.default_rng(1)
    vis = synth.random_visibilities(rng, obs).astype(np.complex128)
    A = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes).astype(np.complex128)
    geom = oracle.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size)
    pl = oracle.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    args = (geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl)
    G = oracle.grid(*args, vis, A)
    V = oracle.degrid(*args, out[0][3], A)
    got_v = np.zeros_like(V)
    for r in range(world):
        mine, Gr, Vr, _ = out[r]
        assert np.linalg.norm(Gr - G) / np.linalg.norm(G) < 1e-12
        got_v[mine] = Vr
    assert sorted(sum((out[r][0] for r in range(world)), [])) == list(range(obs.n_baselines))
    assert np.linalg.norm(got_v - V) / np.linalg.norm(V) < 1e-12
    sub, bls = parallel.shard_observation(obs, 0, 1)
    assert sub is obs and bls.tolist() == list(range(obs.n_baselines))
