"""The multi-GPU path's host logic on CPU: world-size-2 gloo ranks shard the
views, each computes its part of the gradient (here with the FP64 oracle's
finite differences, standing in for the device path), and the all-reduce
yields the gradient of the full batch of views."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2501_18630_gb300 import distributed, scenes

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    sc = scenes.config_scene(1, n=12, seed=3)
    cams = [scenes.ring_camera(3.0, 10.0, a, 24, 20) for a in (0.0, 0.7, 1.9, 3.1)]
    targets = scenes.target_images(cams, seed=4)
    return sc, cams, targets


def _rank_main(rank, port, out_path):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        sc, cams, targets = _problem()
        r, w = distributed.world()
        assert (r, w) == (rank, WORLD)
        mine = distributed.shard_views(range(len(cams)), r, w)
        g, _, _ = oracle.fd_grad(sc.planes, sc.n, sc.n_lobes, [cams[v] for v in mine],
                                 [targets[v] for v in mine], [0, 3, 10, 12], [0, 5, 9], local=False)
        grad = torch.from_numpy(g.copy())
        distributed.reduce_gradients(grad)
        t = distributed.max_over_ranks(float(rank + 1))
        if rank == 0:
            np.save(out_path, grad.numpy())
            assert t == float(WORLD)
    finally:
        dist.destroy_process_group()


def test_shard_views_partitions_the_batch():
    views = list(range(11))
    parts = [distributed.shard_views(views, r, 3) for r in range(3)]
    assert sorted(v for p in parts for v in p) == views
    with pytest.raises(ValueError):
        distributed.shard_views(views, 3, 3)


def test_single_rank_is_identity():
    g = torch.arange(6, dtype=torch.float32)
    assert torch.equal(distributed.reduce_gradients(g.clone()), g)
    assert distributed.world() == (0, 1)
    assert distributed.max_over_ranks(2.5) == 2.5


def test_two_rank_gradient_all_reduce_equals_full_batch(tmp_path):
    import oracle
    out = str(tmp_path / "grad.npy")
    mp.spawn(_rank_main, args=(_free_port(), out), nprocs=WORLD, join=True)
    sc, cams, targets = _problem()
    full, _, _ = oracle.fd_grad(sc.planes, sc.n, sc.n_lobes, cams, targets, [0, 3, 10, 12], [0, 5, 9],
                                local=False)
    got = np.load(out)
    assert np.abs(full).max() > 0
    # finite differences of a sum vs the sum of finite differences: equal up to FP64 rounding
    assert np.allclose(got, full, rtol=1e-6, atol=1e-9), np.abs(got - full).max()


def _rank_chunked(rank, port, out_path):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        sc, cams, targets = _problem()
        mine = distributed.shard_views(range(len(cams)), rank, WORLD)
        planes_ids = [0, 3, 10, 12]
        grad = torch.full((len(planes_ids), 16), -1.0, dtype=torch.float64)   # 12 primitives, pitch 16
        calls = []

        def produce(c0, c1):
            # the rank's gradient of its views for primitives [c0, c1)
            calls.append((c0, c1))
            g, _, _ = oracle.fd_grad(sc.planes, sc.n, sc.n_lobes, [cams[v] for v in mine],
                                     [targets[v] for v in mine], planes_ids, list(range(c0, c1)), local=False)
            grad[:, c0:c1] = torch.from_numpy(g)

        distributed.reduce_gradients_chunked(grad, produce, sc.n, chunk=5)
        assert calls == [(0, 8), (8, 12)]          # chunks start at multiples of 4
        if rank == 0:
            np.save(out_path, grad.numpy())
    finally:
        dist.destroy_process_group()


def test_chunk_ranges_cover_and_align():
    assert distributed.chunk_ranges(12, 5) == [(0, 8), (8, 12)]
    assert distributed.chunk_ranges(13, 4) == [(0, 4), (4, 8), (8, 12), (12, 13)]
    assert distributed.chunk_ranges(0, 4) == []
    for n, c in ((1, 1), (100, 7), (1000003, 125000)):
        r = distributed.chunk_ranges(n, c)
        assert r[0][0] == 0 and r[-1][1] == n and all(a % 4 == 0 for a, _ in r)
        assert all(r[k][1] == r[k + 1][0] for k in range(len(r) - 1))


def test_two_rank_chunked_all_reduce_equals_full_batch(tmp_path):
    """Chunked, asynchronous all-reduce (one per chunk of primitives, each
    started as soon as the chunk is produced): the summed gradient equals the
    full batch's; columns past the primitive count are left untouched."""
    import oracle
    out = str(tmp_path / "grad.npy")
    mp.spawn(_rank_chunked, args=(_free_port(), out), nprocs=WORLD, join=True)
    sc, cams, targets = _problem()
    full, _, _ = oracle.fd_grad(sc.planes, sc.n, sc.n_lobes, cams, targets, [0, 3, 10, 12], list(range(sc.n)),
                                local=False)
    got = np.load(out)
    assert np.allclose(got[:, :sc.n], full, rtol=1e-6, atol=1e-9), np.abs(got[:, :sc.n] - full).max()
    assert np.all(got[:, sc.n:] == -1.0)
