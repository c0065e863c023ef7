"""The N > 1 path on the CPU: sharding of views and uneven meshes over ranks, and the rank handshake (gloo,
world size 2).  Independent units need no collective (the ranks meet only at the timing barrier and at the
max-reduction of the step time); one mesh seen by views split over the ranks needs one sum of the world-space
vertex gradient over the ranks, checked here against the single-process gradient of all views."""
from __future__ import annotations

import itertools
import json
import os
import socket

import numpy as np
import pytest

from paper_2405_02508_gb300 import scenes, shard


def test_lpt_assigns_every_unit_exactly_once():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        costs = rng.uniform(1, 100, 37)
        shards = shard.lpt_assign(costs, world)
        assert len(shards) == world
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(37))
    assert shard.lpt_assign([], 4) == [[], [], [], []]
    with pytest.raises(ValueError):
        shard.lpt_assign([1.0], 0)


def test_lpt_within_grahams_bound_of_brute_force_optimum():
    """LPT makespan <= (4/3 - 1/(3m)) OPT, OPT found by enumerating every assignment of small instances."""
    rng = np.random.default_rng(1)
    for trial in range(30):
        m = 2 + trial % 2
        costs = rng.integers(1, 20, 7).astype(float)
        opt = min(max(sum(c for c, a in zip(costs, asg) if a == r) for r in range(m))
                  for asg in itertools.product(range(m), repeat=len(costs)))
        got = max(shard.loads(costs, shard.lpt_assign(costs, m)))
        assert got <= (4.0 / 3.0 - 1.0 / (3 * m)) * opt + 1e-9


def test_lpt_balances_the_uneven_batch():
    """Two ranks, 512 meshes of the uneven workload: loads within 1 % of each other."""
    nis, res = scenes.uneven_plan(512)
    costs = [shard.item_cost(8 * n * n, r, r) for n, r in zip(nis, res)]
    ld = shard.loads(costs, shard.lpt_assign(costs, 2))
    assert abs(ld[0] - ld[1]) <= 0.01 * max(ld)


def test_rank_subset_builds_the_same_items():
    """A rank builds exactly its own items, identical to the same items of the unsharded batch."""
    full = scenes.uneven_batch(n_items=6, t_max=3000, resolutions=(64, 128))
    part = scenes.uneven_batch(n_items=6, t_max=3000, resolutions=(64, 128), subset=[5, 2])
    for k, i in enumerate([5, 2]):
        assert np.array_equal(full[i].verts, part[k].verts)
        assert np.array_equal(full[i].tris, part[k].tris)
        assert (full[i].H, full[i].W) == (part[k].H, part[k].W)
        assert np.array_equal(full[i].cams, part[k].cams)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist

    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = shard.env_ranks()
    n_all = world * 3
    nis, res = scenes.uneven_plan(n_all, t_max=2000, resolutions=(32, 48))
    costs = [shard.item_cost(8 * n * n, x, x) for n, x in zip(nis, res)]
    mine = shard.lpt_assign(costs, w)[r]
    everyone = [None] * world
    dist.all_gather_object(everyone, mine)
    # each rank differentiates its own meshes with the oracle (no data exchange)
    items = scenes.uneven_batch(n_items=n_all, t_max=2000, resolutions=(32, 48), subset=mine)
    sums = {}
    for i, it in zip(mine, items):
        ov = oracle.render(it)[0]
        g = it.upstream()[0]
        gs, _, _ = oracle.backward(ov.scr, ov.snap, ov.flags, it.tris, ov.index, ov.image, g, it.attr, it.shading)
        sums[i] = float(np.abs(gs).sum())
    slowest = shard.max_over_ranks(1.5 + r)
    shard.barrier()
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "mine": mine, "everyone": everyone, "max": slowest,
                   "sums": {str(k): v for k, v in sums.items()}}, f)
    dist.destroy_process_group()


def test_two_rank_gloo_sharding(tmp_path):
    """Two gloo ranks: both compute the same assignment, the shards are disjoint and cover the batch, the step
    time reduces to the slowest rank's, and each rank's per-item results equal the single-process ones."""
    import torch.multiprocessing as mp

    import oracle

    oracle.build()
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    out = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [o["rank"] for o in out] == [0, 1] and all(o["world"] == world for o in out)
    assert out[0]["everyone"] == out[1]["everyone"] == [out[0]["mine"], out[1]["mine"]]
    assert sorted(out[0]["mine"] + out[1]["mine"]) == list(range(3 * world))
    assert all(o["max"] == 2.5 for o in out)
    # single process, same items
    items = scenes.uneven_batch(n_items=3 * world, t_max=2000, resolutions=(32, 48))
    for o in out:
        for k, v in o["sums"].items():
            it = items[int(k)]
            ov = oracle.render(it)[0]
            gs, _, _ = oracle.backward(ov.scr, ov.snap, ov.flags, it.tris, ov.index, ov.image, it.upstream()[0],
                                       it.attr, it.shading)
            assert float(np.abs(gs).sum()) == v


def test_view_seeds_differ_per_rank():
    """Weak scaling over views: each rank draws its own cameras."""
    a = scenes.cameras_on_sphere(4, 3.0, 64, 48, seed=shard.view_seed(6, 0))
    b = scenes.cameras_on_sphere(4, 3.0, 64, 48, seed=shard.view_seed(6, 1))
    assert not np.array_equal(a["R"], b["R"])


def test_split_views_covers_every_view_once():
    for n, world in [(32, 1), (32, 2), (32, 3), (32, 8), (5, 8), (0, 2)]:
        parts = shard.split_views(n, world)
        assert len(parts) == world
        assert [v for p in parts for v in p] == list(range(n))
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.split_views(4, 0)


def _mesh_worker(rank: int, world: int, port: int, out_dir: str):
    import torch
    import torch.distributed as dist

    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = shard.env_ranks()
    sc = scenes.head_multiview(n_views=5, H=40, W=36, n=6, tex_size=32)
    mine = shard.split_views(sc.n_views, w)[r]
    ovs = oracle.render(sc, mine)
    g = sc.upstream()
    # this rank's views only: their world-space vertex gradient, then the sum over the ranks
    _, gw, _, _ = oracle.backward_scene(sc, ovs, [g[v] for v in mine], mine)
    t = torch.from_numpy(gw.copy())
    shard.sum_over_ranks(t)
    np.save(os.path.join(out_dir, f"mesh_rank{r}.npy"), t.numpy())
    with open(os.path.join(out_dir, f"mesh_rank{r}.json"), "w") as f:
        json.dump({"mine": mine}, f)
    dist.destroy_process_group()


def test_two_rank_shared_mesh_gradient_sum(tmp_path):
    """One mesh, five views split over two gloo ranks: after the sum over the ranks both hold the same world
    gradient, equal to the single-process gradient of all five views (up to the order of the FP64 sums)."""
    import torch.multiprocessing as mp

    import oracle

    oracle.build()
    world = 2
    mp.spawn(_mesh_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    parts = [json.load(open(tmp_path / f"mesh_rank{r}.json"))["mine"] for r in range(world)]
    assert parts == [[0, 1, 2], [3, 4]]
    got = [np.load(tmp_path / f"mesh_rank{r}.npy") for r in range(world)]
    np.testing.assert_array_equal(got[0], got[1])
    sc = scenes.head_multiview(n_views=5, H=40, W=36, n=6, tex_size=32)
    ovs = oracle.render(sc)
    _, gw, _, _ = oracle.backward_scene(sc, ovs, list(sc.upstream()))
    assert np.abs(gw).max() > 0
    np.testing.assert_allclose(got[0], gw, rtol=1e-12, atol=1e-12 * np.abs(gw).max())
