"""Parity of the batched workloads at their full sizes, in the launch
configuration bench.py times (plans prepared with the autotuner, one graph
launch), on sampled outputs that the oracle computes one by one, plus
properties that hold at any size."""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_03229_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"
REL_TOL = 1e-12


@pytest.fixture(scope="module")
def ss():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_03229_gb300 as m
    return m


def sampled_positions(m, k, seed):
    """k random positions of [0, m) and the last 1000, sorted."""
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([rng.integers(0, m, size=k), np.arange(max(0, m - 1000), m)]))
    return idx


def check_batched_1d(b, out, k, seed):
    Y_off = b.Y_off.cpu().numpy()
    X_off = b.X_off.cpu().numpy()
    X = b.X.cpu().numpy()
    idx = sampled_positions(int(Y_off[-1]), k, seed)
    ti = torch.from_numpy(idx).to(DEV)
    got = out[ti].cpu().numpy()
    y = b.Y[ti].cpu().numpy() if b.Y.is_cuda else b.Y[torch.from_numpy(idx)].numpy()
    tab = np.searchsorted(Y_off, idx, side="right") - 1
    for t in np.unique(tab):
        sel = tab == t
        xt = X[X_off[t]:X_off[t + 1]]
        np.testing.assert_array_equal(got[sel], oracle.search_1d(xt, y[sel]))
        assert got[sel].min() >= 0 and got[sel].max() <= len(xt) - 1


def test_batched1d_full_size_sampled(ss):
    """The headline bench workload: two 10,000-table batches, 2,174,007,083
    targets; the plain plan (autotuned) and each position model's plan, as
    bench.py times them, on the same sampled targets."""
    b = wl.batched_1d_x2(seed=5, device=DEV)
    assert b.Y.numel() == 2_174_007_083
    X = b.X.to(DEV)
    out = torch.empty((b.Y.numel(),), dtype=torch.int32, device=DEV)
    for k, model in enumerate(("none", "spline", "mlp", "loghash")):
        plan = ss.Plan.create_1d(b.X_off, X, model=model, autotune=True)
        out.fill_(-1)
        stat = ss.new_stat()
        plan.bind_1d(b.Y_off, b.Y, out, stat=stat)
        plan.execute()
        torch.cuda.synchronize()
        assert int(out.min()) >= 0, model                 # every target written
        check_batched_1d(b, out, 1_000_000, seed=1 + k)
        assert ss.read_stat(stat).flags == 0
        del plan
    del out, b, X
    torch.cuda.empty_cache()


def test_sweep_full_size_sampled(ss):
    """The table-size sweep: 16, 256, 4096 and 65536 entries (the last
    through its wide section), 256M targets each."""
    tabs = [wl.sweep_table(n, seed=4) for n in (16, 256, 4096, 65536)]
    per = 256 << 20
    Ys = [wl.log_uniform(per, 0.5 * t[0].item(), 2 * t[-1].item(), seed=7 + i, device=DEV) for i, t in enumerate(tabs)]
    X_off = torch.tensor(np.concatenate([[0], np.cumsum([len(t) for t in tabs])]))
    Y_off = torch.tensor(np.concatenate([[0], np.cumsum([len(y) for y in Ys])]))
    b = wl.Batched1D(X_off, torch.cat(tabs), Y_off, torch.cat(Ys), None, None)
    del Ys
    plan = ss.Plan.create_1d(b.X_off, b.X.to(DEV), autotune=True)
    assert "wide" in [c[0] for c in plan.choices().values()]
    out = torch.full((b.Y.numel(),), -1, dtype=torch.int32, device=DEV)
    plan.bind_1d(b.Y_off, b.Y, out)
    plan.execute()
    torch.cuda.synchronize()
    assert int(out.min()) >= 0
    check_batched_1d(b, out, 2_000_000, seed=2)
    del out, b, plan
    torch.cuda.empty_cache()


@pytest.mark.parametrize("coherent", [False, True])
def test_batched2d_full_size_sampled(ss, coherent):
    """1,000 2D tables, 1M pairs each (1B pairs), random or coherent order:
    the plain plan (autotuned) and each position model's plan (the spline,
    the logarithm hash and the MLP in the lean kernel's instances when
    their windows allow, the hunt in the general kernel), sampled against
    the oracle."""
    b = wl.batched_2d(ntables=1000, pairs_per_table=1_000_000, coherent=coherent, seed=6, device=DEV)
    m = b.Y2.shape[0]
    idx = torch.empty((m, 2), dtype=torch.int32, device=DEV)
    val = torch.empty(m, dtype=torch.float64, device=DEV)
    pos = sampled_positions(m, 500_000, seed=3 + int(coherent))
    tp = torch.from_numpy(pos).to(DEV)
    y = b.Y2[tp].cpu().numpy()
    offs = [o.cpu().numpy() for o in (b.R_off, b.T_off, b.F_off, b.Y_off)]
    R, T, F = b.R.cpu().numpy(), b.T.cpu().numpy(), b.F.cpu().numpy()
    tab = np.searchsorted(offs[3], pos, side="right") - 1
    want_i = np.empty((len(pos), 2), dtype=np.int32)
    want_v = np.empty(len(pos))
    for t in np.unique(tab):
        sel = tab == t
        want_i[sel], want_v[sel] = oracle.search_interp_2d(R[offs[0][t]:offs[0][t + 1]], T[offs[1][t]:offs[1][t + 1]],
                                                           F[offs[2][t]:offs[2][t + 1]], y[sel])
    for model in ("none", "spline", "loghash", "mlp", "hunt"):
        plan = ss.Plan.create_2d(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV), model=model,
                                 autotune=model == "none")
        idx.fill_(-1)
        plan.bind_2d(b.Y_off, b.Y2, idx, val)
        plan.execute()
        torch.cuda.synchronize()
        assert int(idx.min()) >= 0, model                 # every pair written
        if model in ("spline", "loghash", "mlp"):
            assert plan.info().lean_kernel == (1 if plan.info().max_window <= 4 else 0), model
        np.testing.assert_array_equal(idx[tp].cpu().numpy(), want_i, err_msg=model)
        gv = val[tp].cpu().numpy()
        assert (np.abs(gv - want_v) <= REL_TOL * np.abs(want_v)).all(), model
        del plan
    del idx, val, b
    torch.cuda.empty_cache()
