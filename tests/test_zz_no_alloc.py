"""The batched search that allocates no device memory
(ss_search_1d_batched_static), checked against the plan-based batched search
through the C ABI.  Callers such as plug-ins inside a host framework that owns
all device memory, or loops that cannot pay for cudaMalloc's synchronisation,
use it; its working set lives in a fixed array inside the library.

This file is named so that pytest collects it last."""
import numpy as np
import pytest
import torch

from paper_2112_03229_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def ss():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_03229_gb300 as m
    return m


def reference(ss, b, side):
    plan = ss.Plan.create_1d(b.X_off, b.X.to(DEV), side=side)
    out = torch.empty(len(b.Y), dtype=torch.int32, device=DEV)
    plan.bind_1d(b.Y_off, b.Y.to(DEV), out)
    plan.execute()
    return out.cpu().numpy()


def test_static_matches_plan_on_two_calls_in_a_row(ss):
    # two different batches back to back: the second call must not see the
    # first call's tables, tiles or counter left in the shared array
    b1 = wl.batched_1d(ntables=40, count_scale=0.003, seed=21)
    b2 = wl.batched_1d(ntables=17, count_scale=0.005, seed=22)
    for b, side in ((b1, 0), (b2, 1)):
        want = reference(ss, b, side)
        stat = ss.new_stat()
        out = torch.full((len(b.Y),), -1, dtype=torch.int32, device=DEV)
        ss.search_1d_batched_static(b.X_off, b.X.to(DEV), b.Y_off, b.Y.to(DEV), out=out, side=side, stat=stat)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        assert ss.read_stat(stat).flags == 0


def test_static_calls_on_two_streams_are_ordered(ss):
    # calls queued on two streams without synchronising in between share the
    # one array: each call's work waits for the previous call's, so every
    # result is still exact
    bs = [wl.batched_1d(ntables=30 + 7 * i, count_scale=0.004, seed=31 + i) for i in range(4)]
    wants = [reference(ss, b, i & 1) for i, b in enumerate(bs)]
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
