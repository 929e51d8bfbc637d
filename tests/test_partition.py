"""Multi-rank partitioning of the search, on CPU with gloo (world size 2):
each rank searches its share with the oracle, the shares are gathered and
must equal the single-rank answer."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2112_03229_gb300 import partition
from paper_2112_03229_gb300 import workloads as wl


def test_target_slices_cover_exactly():
    for m in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            sl = [partition.target_slice(m, world, r) for r in range(world)]
            assert sl[0][0] == 0 and sl[-1][1] == m
            assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
            sizes = [e - s for s, e in sl]
            assert max(sizes) - min(sizes) <= 1


def test_lpt_balances_and_covers():
    rng = np.random.default_rng(0)
    counts = wl.zipf_counts(10_000, 1.1, 1000, 1_000_000, rng)
    for world in (2, 4, 8):
        parts = partition.lpt_tables(counts, world)
        allk = np.sort(np.concatenate(parts))
        np.testing.assert_array_equal(allk, np.arange(len(counts)))
        loads = np.array([counts[p].sum() for p in parts])
        # LPT bound: max load <= mean + largest item
        assert loads.max() <= loads.mean() + counts.max()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, outdir):
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = wl.batched_1d(ntables=40, count_scale=0.003, seed=11)
    X_off, X, Y_off, Y = b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy()
    counts = np.diff(Y_off)
    mine = partition.lpt_tables(counts, world)[rank]
    sx_off, sX, sy_off, sY, pos = partition.gather_batch(X_off, X, Y_off, Y, mine)
    got = oracle.search_1d_batched(sx_off, sX, sy_off, sY) if len(mine) else np.zeros(0, np.int32)
    # gather (positions, indices) from every rank
    n_local = torch.tensor([len(got)])
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n_local)
    mx = int(max(s.item() for s in sizes))
    buf = torch.full((2, mx), -1, dtype=torch.int64)
    buf[0, :len(got)] = torch.as_tensor(pos)
    buf[1, :len(got)] = torch.as_tensor(got.astype(np.int64))
    bufs = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf)
    if rank == 0:
        full = np.full(len(Y), -1, dtype=np.int64)
        for bb, sz in zip(bufs, sizes):
            n = int(sz.item())
            full[bb[0, :n].numpy()] = bb[1, :n].numpy()
        want = oracle.search_1d_batched(X_off, X, Y_off, Y)
        np.save(os.path.join(outdir, "ok.npy"), np.array([np.array_equal(full, want)]))
    # single-table slices
    X1, Y1 = wl.plain_1d(m=10_001, seed=2)
    s, e = partition.target_slice(len(Y1), world, rank)
    part = torch.as_tensor(oracle.search_1d(X1.numpy(), Y1.numpy()[s:e]).astype(np.int64))
    lens = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(lens, torch.tensor([e - s]))
    pad = torch.full((len(Y1),), -1, dtype=torch.int64)
    pad[:e - s] = part
    outs = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(outs, pad)
    if rank == 0:
        joined = np.concatenate([o[:int(l.item())].numpy() for o, l in zip(outs, lens)])
        np.save(os.path.join(outdir, "ok1.npy"),
                np.array([np.array_equal(joined, oracle.search_1d(X1.numpy(), Y1.numpy()))]))
    dist.destroy_process_group()


def test_two_rank_gloo_partition_matches_single_rank(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    assert bool(np.load(tmp_path / "ok.npy")[0])
    assert bool(np.load(tmp_path / "ok1.npy")[0])


def _bench_share_main(rank, world, port, outdir):
    # the split that `bench.py --scaling strong` gives each rank of the
    # batched workload: every table on exactly one rank, its data intact
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = wl.batched_1d(ntables=57, count_scale=0.002, seed=12)
    sub, tables = bench.share_of_batch(b, world, rank)
    X_off, Y_off = b.X_off.numpy(), b.Y_off.numpy()
    ok = len(sub.X_off) == len(tables) + 1 and len(sub.Y_off) == len(tables) + 1
    for i, k in enumerate(tables):
        xs, ys = sub.X[sub.X_off[i]:sub.X_off[i + 1]], sub.Y[sub.Y_off[i]:sub.Y_off[i + 1]]
        ok &= torch.equal(xs, b.X[X_off[k]:X_off[k + 1]]) and torch.equal(ys, b.Y[Y_off[k]:Y_off[k + 1]])
    got = [None] * world
    dist.all_gather_object(got, (list(map(int, tables)), bool(ok), int(sub.Y_off[-1])))
    if rank == 0:
        every = sorted(k for t, _, _ in got for k in t)
        total = sum(n for _, _, n in got)
        np.save(os.path.join(outdir, "share.npy"),
                np.array([every == list(range(57)), all(o for _, o, _ in got), total == int(Y_off[-1])]))
    dist.destroy_process_group()


def test_two_rank_gloo_bench_strong_split_covers_every_table_once(tmp_path):
    port = _free_port()
    mp.start_processes(_bench_share_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    assert np.load(tmp_path / "share.npy").all()
