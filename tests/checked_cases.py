"""Small plan cases run against the bounds-checked build of the library
(libsimdsearch_checked.so, selected with SS_CHECKED_LIBRARY=1): every answer
is compared with the oracle, and the run fails if any index was caught out
of range.  Run by tests/test_gpu_checked.py in a process of its own."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import paper_2112_03229_gb300 as ss  # noqa: E402
from paper_2112_03229_gb300 import workloads as wl  # noqa: E402

DEV = "cuda"
REL_TOL = 1e-12


def batch_1d(sizes, per, seed, walk=False):
    Xs, Ys = [], []
    for k, n in enumerate(sizes):
        X = wl.log_spaced_table(n, 1e-6, 1e4, 0.1, seed * 31 + k)
        Y = wl.walk_1d(per, 0.5e-6, 2e4, seed * 37 + k) if walk else wl.log_uniform(per, 0.5e-6, 2e4, seed * 37 + k)
        Xs.append(X)
        Ys.append(Y)
    X_off = torch.tensor(np.concatenate([[0], np.cumsum([len(x) for x in Xs])]))
    Y_off = torch.tensor(np.concatenate([[0], np.cumsum([len(y) for y in Ys])]))
    return wl.Batched1D(X_off, torch.cat(Xs), Y_off, torch.cat(Ys), None, None)


def check_1d(b, side=0, **opts):
    want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy(), side)
    plan = ss.Plan.create_1d(b.X_off, b.X.to(DEV), side=side, **opts)
    out = torch.full((b.Y.numel(),), -1, dtype=torch.int32, device=DEV)
    stat = ss.new_stat()
    plan.bind_1d(b.Y_off, b.Y.to(DEV), out, stat=stat)
    plan.execute()
    np.testing.assert_array_equal(out.cpu().numpy(), want, err_msg=str(opts))
    assert ss.read_stat(stat).flags == 0, opts


def check_2d(b, **opts):
    args = (b.R_off.numpy(), b.R.numpy(), b.T_off.numpy(), b.T.numpy(), b.F_off.numpy(), b.F.numpy(),
            b.Y_off.numpy(), b.Y2.numpy())
    wi, wv = oracle.search_interp_2d_batched(*args, extrap=int(opts.get("extrap", 0)),
                                             logspace=int(opts.get("logspace", 0)))
    plan = ss.Plan.create_2d(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV), **opts)
    m = b.Y2.shape[0]
    idx = torch.empty((m, 2), dtype=torch.int32, device=DEV)
    val = torch.empty(m, dtype=torch.float64, device=DEV)
    stat = ss.new_stat()
    plan.bind_2d(b.Y_off, b.Y2.to(DEV), idx, val, stat=stat)
    plan.execute()
    np.testing.assert_array_equal(idx.cpu().numpy(), wi, err_msg=str(opts))
    if not opts:
        assert (np.abs(val.cpu().numpy() - wv) / np.abs(wv)).max() <= REL_TOL
    assert ss.read_stat(stat).flags == 0, opts
    return plan


def main():
    assert ss.lib_path().endswith("libsimdsearch_checked.so")
    ss.checked_hits(reset=True)
    # the counter moves when an index is out of range (the check's own test)
    ss._check(ss.lib().ss_checked_selftest())
    assert ss.checked_hits(reset=True) == 1
    # 1D: staged tables of every size bucket, a wide-section table (30,000
    # entries) and a two-level table in global memory (100,000 entries)
    b = batch_1d((20, 64, 700, 2000, 8000, 30_000, 100_000), 20_011, seed=3)
    for side in (0, 1):
        check_1d(b, side)
        for model in ("spline", "mlp", "loghash", "hunt"):
            check_1d(b, side, model=model, mlp_epochs=60 if model == "mlp" else None)
        for algo in ("binary", "ballot"):
            check_1d(b, side, algo=algo)
    check_1d(batch_1d((64, 4000, 100_000), 30_011, seed=4, walk=True), model="hunt")
    check_1d(b, tile=997)
    # the batched search that allocates nothing runs the same kernel
    bs = wl.batched_1d(ntables=30, count_scale=0.003, seed=5)
    want = oracle.search_1d_batched(bs.X_off.numpy(), bs.X.numpy(), bs.Y_off.numpy(), bs.Y.numpy())
    got = ss.search_1d_batched_static(bs.X_off, bs.X.to(DEV), bs.Y_off, bs.Y.to(DEV))
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    # 2D: the lean kernel, the general one with each model, binary axes, the options
    b2 = wl.batched_2d(ntables=8, pairs_per_table=4001, seed=6)
    assert check_2d(b2).info().lean_kernel == 1
    for kw in (dict(model="spline"), dict(model="loghash"), dict(model="mlp", mlp_epochs=60), dict(model="hunt"),
               dict(algo="binary"), dict(extrap=True), dict(logspace=True)):
        check_2d(b2, **kw)
    check_2d(wl.batched_2d(ntables=4, pairs_per_table=4001, coherent=True, jump=0.02, seed=7), model="hunt")
    # one-shot 2D: the staged-grid kernel's lean path (bucket axes) and its out-of-line paths (binary axes)
    R, T, F, Y2 = wl.interp_2d(m=100_003, seed=8)
    wi, wv = oracle.search_interp_2d(R.numpy(), T.numpy(), F.numpy(), Y2.numpy())
    for algo in ("bucket", "binary"):
        idx, val = ss.search_interp_2d(R.to(DEV), T.to(DEV), F.to(DEV), Y2.to(DEV), algo=algo)
        np.testing.assert_array_equal(idx.cpu().numpy(), wi)
        assert (np.abs(val.cpu().numpy() - wv) / np.abs(wv)).max() <= REL_TOL
    # the one-call batched 2D lookup: the lean kernel, and the general one
    # when a grid value is outside the float-float range
    for big in (False, True):
        b3 = wl.batched_2d(ntables=5, pairs_per_table=3001, seed=9)
        if big:
            F3 = b3.F.clone()
            F3[7] = 1e250
            b3 = wl.Batched2D(b3.R_off, b3.R, b3.T_off, b3.T, b3.F_off, F3, b3.Y_off, b3.Y2)
        wi, wv = oracle.search_interp_2d_batched(b3.R_off.numpy(), b3.R.numpy(), b3.T_off.numpy(), b3.T.numpy(),
                                                 b3.F_off.numpy(), b3.F.numpy(), b3.Y_off.numpy(), b3.Y2.numpy())
        stat = ss.new_stat()
        idx, val = ss.search_interp_2d_batched(b3.R_off, b3.R.to(DEV), b3.T_off, b3.T.to(DEV), b3.F_off,
                                               b3.F.to(DEV), b3.Y_off, b3.Y2.to(DEV), stat=stat)
        np.testing.assert_array_equal(idx.cpu().numpy(), wi)
        assert (np.abs(val.cpu().numpy() - wv) / np.abs(wv)).max() <= REL_TOL
        assert ss.read_stat(stat).flags == 0
    hits = ss.checked_hits()
    assert hits == 0, "indices out of range: %d" % hits
    print("checked build: every case exact, 0 indices out of range")


if __name__ == "__main__":
    main()
