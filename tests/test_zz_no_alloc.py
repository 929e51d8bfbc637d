"""The batched search that allocates no device memory
(ss_search_1d_batched_static), checked through the C ABI against the oracle
and against the plan-based batched search.  Callers such as plug-ins inside a
host framework that owns all device memory, or loops that cannot pay for
cudaMalloc's synchronisation, use it; its working set lives in a fixed array
inside the library.

This file is named so that pytest collects it last."""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_03229_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def ss():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_03229_gb300 as m
    return m


def from_oracle(b, side):
    return oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy(), side)


def from_plan(ss, b, side):
    plan = ss.Plan.create_1d(b.X_off, b.X.to(DEV), side=side)
    out = torch.empty(len(b.Y), dtype=torch.int32, device=DEV)
    plan.bind_1d(b.Y_off, b.Y.to(DEV), out)
    plan.execute()
    return out.cpu().numpy()


def test_static_matches_oracle_and_plan_on_two_calls_in_a_row(ss):
    # two different batches back to back: the second call must not see the
    # first call's tables, tiles or counter left in the shared array
    b1 = wl.batched_1d(ntables=40, count_scale=0.003, seed=21)
    b2 = wl.batched_1d(ntables=17, count_scale=0.005, seed=22)
    for b, side in ((b1, 0), (b2, 1)):
        want = from_oracle(b, side)
        np.testing.assert_array_equal(from_plan(ss, b, side), want)
        stat = ss.new_stat()
        out = torch.full((len(b.Y),), -1, dtype=torch.int32, device=DEV)
        ss.search_1d_batched_static(b.X_off, b.X.to(DEV), b.Y_off, b.Y.to(DEV), out=out, side=side, stat=stat)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        assert ss.read_stat(stat).flags == 0


def test_static_empty_tables_and_ragged_counts(ss):
    # tables without targets, a 2-entry table, targets on keys and at both ends
    X = torch.tensor([1.0, 2.0, 3.0, 10.0, 20.0, 30.0, 40.0, -5.0, 5.0], dtype=torch.float64)
    Y = torch.tensor([0.5, 2.5, 3.0, 25.0, 45.0, 40.0, 10.0, -7.0, 0.0, 5.0, 6.0], dtype=torch.float64)
    X_off, Y_off = np.array([0, 3, 7, 9]), np.array([0, 0, 6, 11])
    for side in (0, 1):
        want = oracle.search_1d_batched(X_off, X.numpy(), Y_off, Y.numpy(), side)
        got = ss.search_1d_batched_static(X_off, X.to(DEV), Y_off, Y.to(DEV), side=side)
        np.testing.assert_array_equal(got.cpu().numpy(), want)


def test_static_flags_an_unsorted_table(ss):
    # table 1 repeats a value: the flag reaches the caller's status record,
    # its indices stay in range and the other tables' indices stay exact
    b = wl.batched_1d(ntables=12, count_scale=0.002, seed=24)
    X = b.X.clone()
    lo, hi = int(b.X_off[1]), int(b.X_off[2])
    X[lo + 3] = X[lo + 2]
    stat = ss.new_stat()
    out = ss.search_1d_batched_static(b.X_off, X.to(DEV), b.Y_off, b.Y.to(DEV), stat=stat).cpu().numpy()
    assert ss.read_stat(stat).flags & ss.FLAG_NOT_SORTED
    want = from_oracle(b, 0)
    yo = b.Y_off.numpy()
    bad = slice(int(yo[1]), int(yo[2]))
    assert out[bad].min() >= 0 and out[bad].max() <= hi - lo - 1
    keep = np.ones(len(out), dtype=bool)
    keep[bad] = False
    np.testing.assert_array_equal(out[keep], want[keep])


def test_static_refuses_a_capturing_stream(ss):
    # refused before anything is queued: the caller's capture stays valid
    b = wl.batched_1d(ntables=5, count_scale=0.001, seed=25)
    X, Y = b.X.to(DEV), b.Y.to(DEV)
    out = torch.empty(len(b.Y), dtype=torch.int32, device=DEV)
    x = torch.zeros(8, device=DEV)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    codes = []
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            try:
                ss.search_1d_batched_static(b.X_off, X, b.Y_off, Y, out=out)
            except ss.SSError as e:
                codes.append((e.code, str(e)))
            x.add_(1.0)
    assert codes and codes[0][0] == 6 and "capturing" in codes[0][1]
    g.replay()
    torch.cuda.synchronize()
    assert float(x.sum()) == 8.0
    # and the entry point still works afterwards
    got = ss.search_1d_batched_static(b.X_off, X, b.Y_off, Y)
    np.testing.assert_array_equal(got.cpu().numpy(), from_oracle(b, 0))


def test_static_calls_on_two_streams_are_ordered(ss):
    # calls queued on two streams without synchronising in between share the
    # one array: each call's work waits for the previous call's, so every
    # result is still exact
    bs = [wl.batched_1d(ntables=30 + 7 * i, count_scale=0.004, seed=31 + i) for i in range(4)]
    wants = [from_oracle(b, i & 1) for i, b in enumerate(bs)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ins = [b.Y.to(DEV) for b in bs]
    Xs = [b.X.to(DEV) for b in bs]
    outs = [torch.full((len(b.Y),), -1, dtype=torch.int32, device=DEV) for b in bs]
    torch.cuda.synchronize()
    for rep in range(3):
        for i, b in enumerate(bs):
            ss.search_1d_batched_static(b.X_off, Xs[i], b.Y_off, ins[i], out=outs[i], side=i & 1,
                                        stream=streams[i & 1])
        torch.cuda.synchronize()
        for i in range(len(bs)):
            np.testing.assert_array_equal(outs[i].cpu().numpy(), wants[i])
            outs[i].fill_(-1)
        torch.cuda.synchronize()


def test_static_rejects_a_batch_over_its_limit(ss):
    b = wl.batched_1d(ntables=4000, count_scale=0.00005, seed=23)
    with pytest.raises(ss.SSError) as e:
        ss.search_1d_batched_static(b.X_off, b.X.to(DEV), b.Y_off, b.Y.to(DEV))
    assert e.value.code == 1 and "bytes" in str(e.value)
