"""Multi-rank logic over gloo, world size 2: the round-robin brick shard of
the paper's multi-GPU chunk scheduling (Sec. III-D) reproduces the whole
volume when each rank filters only its bricks, and the benchmark's
whole-job reduction takes the slowest rank.

On CPU the per-brick filtering of each rank is the oracle's box mode over
the planner's bricks. Where a CUDA device is present (the gpu-marked test),
each rank runs its shard through libhp itself (hp_set_brick_shard on a host
volume, out of core on cuda:0); the ranks' kernels never wait on each
other, and the only exchange is the gather of the finished parts that the
test makes."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _bricks_worker(rank, world, port, out_dir):
    _init(rank, world, port)
    try:
        import oracle
        import paper_2511_11890_b300 as hp
        import synth
        f = synth.porous((24, 40, 56), 7)[0]
        sigma, r = 1.5, oracle.radius(1.5)
        cores, boxes = hp.plan_bricks(f.shape, r, 2, 4, 3 * 40 * 56 * 6 * 4, min_bricks=6)
        mine = hp.shard_bricks(len(cores), rank, world)
        part = np.full(f.shape, np.nan, np.float32)
        for i in mine:
            lo, hi = cores[i][:3], cores[i][3:]
            blo, bhi = boxes[i][:3], boxes[i][3:]
            src = f[blo[0]:bhi[0], blo[1]:bhi[1], blo[2]:bhi[2]]
            part[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = oracle.gaussian3d(
                src, sigma, gdims=f.shape, in_lo=list(blo), out_lo=list(lo),
                out_shape=tuple(int(h - l) for l, h in zip(lo, hi)))
        # gather every rank's part (no data exchange is needed to compute)
        parts = [torch.empty(f.size, dtype=torch.float32) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(part.ravel()))
        if rank == 0:
            whole = np.full(f.size, np.nan, np.float32)
            covered = np.zeros(f.size, np.int32)
            for p in parts:
                p = p.numpy()
                m = ~np.isnan(p)
                whole[m] = p[m]
                covered += m
            np.save(os.path.join(out_dir, "whole.npy"), whole.reshape(f.shape))
            np.save(os.path.join(out_dir, "covered.npy"), covered.reshape(f.shape))
            np.save(os.path.join(out_dir, "nbricks.npy"), np.array([len(cores)]))
    finally:
        dist.destroy_process_group()


def _libhp_shard_worker(rank, world, port, out_dir):
    _init(rank, world, port)
    try:
        import paper_2511_11890_b300 as hp
        import synth
        f = synth.porous((48, 64, 80), 7)[0]
        hp.set_memory_budget(6_000_000)
        hp.set_brick_shard(rank, world)
        part = np.full(f.shape, np.nan, np.float32)
        hp.gaussian3d(f, 1.5, out=part)               # host volume: this rank's bricks only
        nb = hp.stats()["bricks"]
        parts = [torch.empty(f.size, dtype=torch.float32) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(part.ravel()))
        counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(counts, torch.tensor([nb], dtype=torch.int64))
        if rank == 0:
            whole = np.full(f.size, np.nan, np.float32)
            covered = np.zeros(f.size, np.int32)
            for p in parts:
                p = p.numpy()
                m = ~np.isnan(p)
                whole[m] = p[m]
                covered += m
            np.save(os.path.join(out_dir, "whole.npy"), whole.reshape(f.shape))
            np.save(os.path.join(out_dir, "covered.npy"), covered.reshape(f.shape))
            np.save(os.path.join(out_dir, "counts.npy"), np.array([int(c) for c in counts]))
    finally:
        dist.destroy_process_group()


def _reduce_worker(rank, world, port, out_dir):
    _init(rank, world, port)
    try:
        import bench
        ms, value = bench.reduce_over_ranks(10.0 + 5.0 * rank, world, 1000.0)
        np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([ms, value]))
    finally:
        dist.destroy_process_group()


def test_round_robin_bricks_reproduce_whole_volume(tmp_path):
    pytest.importorskip("paper_2511_11890_b300")
    import oracle
    import synth
    mp.start_processes(_bricks_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2,
                       start_method="spawn")
    whole = np.load(tmp_path / "whole.npy")
    covered = np.load(tmp_path / "covered.npy")
    assert int(np.load(tmp_path / "nbricks.npy")[0]) >= 6
    assert (covered == 1).all(), "every voxel belongs to exactly one rank's bricks"
    f = synth.porous((24, 40, 56), 7)[0]
    ref = oracle.gaussian3d(f, 1.5).astype(np.float32)
    assert np.array_equal(whole.view(np.uint32), ref.view(np.uint32))


@pytest.mark.gpu
def test_libhp_shards_over_gloo_ranks_reproduce_whole_volume(tmp_path):
    """Two processes, each running its half of the bricks through libhp on
    cuda:0; the union equals one process running every brick, bit for bit."""
    hp = pytest.importorskip("paper_2511_11890_b300")
    import synth
    mp.start_processes(_libhp_shard_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2,
                       start_method="spawn")
    whole = np.load(tmp_path / "whole.npy")
    covered = np.load(tmp_path / "covered.npy")
    counts = np.load(tmp_path / "counts.npy")
    assert (covered == 1).all(), "every voxel belongs to exactly one rank's bricks"
    assert counts.min() >= 2 and abs(int(counts[0]) - int(counts[1])) <= 1
    f = synth.porous((48, 64, 80), 7)[0]
    ref = hp.gaussian3d(torch.from_numpy(f).cuda(), 1.5).cpu().numpy()
    assert np.array_equal(whole.view(np.uint32), ref.view(np.uint32))


def test_shard_is_a_partition():
    hp = pytest.importorskip("paper_2511_11890_b300")
    for n in (0, 1, 5, 37):
        for world in (1, 2, 3, 8):
            got = sorted(i for r in range(world) for i in hp.shard_bricks(n, r, world))
            assert got == list(range(n))
    with pytest.raises(ValueError):
        hp.shard_bricks(4, 2, 2)


def test_bench_reduction_takes_the_slowest_rank(tmp_path):
    mp.start_processes(_reduce_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2,
                       start_method="spawn")
    for rank in range(2):
        ms, value = np.load(tmp_path / f"r{rank}.npy")
        assert ms == 15.0
        assert value == pytest.approx(2 * 1000.0 / 0.015)
