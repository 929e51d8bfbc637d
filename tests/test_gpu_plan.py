"""GPU parity of plans (prepared tables, learned proposals, persistent
batched kernel, CUDA graph, autotuner, save/load) against the CPU oracle."""
import ctypes
import os
import struct

import numpy as np
import pytest
import torch

import oracle
from paper_2112_03229_gb300 import PlanOpts
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


def run_plan_1d(ss, b, Y=None, **opts):
    plan = ss.Plan.create_1d(b.X_off, b.X.to(DEV), **opts)
    Yd = (b.Y if Y is None else Y).to(DEV)
    out = torch.full((Yd.numel(),), -1, dtype=torch.int32, device=DEV)
    stat = ss.new_stat()
    plan.bind_1d(b.Y_off, Yd, out, stat=stat)
    plan.execute()
    return plan, out.cpu().numpy(), ss.read_stat(stat)


def small_batch(seed=3, ntables=150, scale=0.003):
    return wl.batched_1d(ntables=ntables, count_scale=scale, seed=seed)


@pytest.mark.parametrize("model", ["none", "spline", "mlp", "loghash"])
@pytest.mark.parametrize("side", [0, 1])
def test_plan_1d_batched_models(ss, model, side):
    b = small_batch()
    want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy(), side)
    plan, got, st = run_plan_1d(ss, b, model=model, side=side, mlp_epochs=150 if model == "mlp" else None)
    np.testing.assert_array_equal(got, want)
    assert st.flags == 0
    inf = plan.info()
    if model == "none":
        assert inf.max_window == 0 and st.fallbacks == 0
    else:
        assert inf.max_window >= 1


@pytest.mark.parametrize("algo", ["bucket", "binary", "ballot"])
def test_plan_1d_plain_algorithms(ss, algo):
    b = small_batch(seed=4)
    want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy())
    _, got, st = run_plan_1d(ss, b, algo=algo)
    np.testing.assert_array_equal(got, want)


def sweep_batch(m_per=60_000):
    """The table-size sweep (16, 256, 4096, 65536 clustered entries) as one batch."""
    tabs = [wl.sweep_table(n) for n in (16, 256, 4096, 65536)]
    X = torch.cat(tabs)
    X_off = np.concatenate([[0], np.cumsum([len(t) for t in tabs])])
    Ys = [wl.log_uniform(m_per, 0.5 * t[0].item(), 2 * t[-1].item(), seed=len(t)) for t in tabs]
    Ys[-1][:2000] = tabs[-1][-2000:]                   # exact hits on the big table
    Y = torch.cat(Ys)
    Y_off = np.concatenate([[0], np.cumsum([len(y) for y in Ys])])
    return wl.Batched1D(torch.as_tensor(X_off), X, torch.as_tensor(Y_off), Y, None, None)


@pytest.mark.parametrize("model", ["none", "spline", "mlp", "loghash"])
def test_plan_table_size_sweep(ss, model):
    b = sweep_batch()
    want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy())
    plan, got, st = run_plan_1d(ss, b, model=model)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("tile", [0, 1000])
def test_plan_fitted_directory_and_wide_blocks(ss, side, tile):
    """A clustered 4096-entry table crowds the default bucket budget (up to 9
    keys in a bucket); the plan fits a finer directory to its keys (at most
    2 per bucket) and, with that table staged, runs 512-thread blocks.
    Smaller tables in the same batch, ragged tiles (tile=1000, not a multiple
    of the vector width) and a misaligned target array keep exact indices."""
    tabs = [wl.sweep_table(n) for n in (16, 256, 4096)]
    X = torch.cat(tabs)
    X_off = np.concatenate([[0], np.cumsum([len(t) for t in tabs])])
    Ys = [wl.log_uniform(50_001 + 7 * i, 0.5 * t[0].item(), 2 * t[-1].item(), seed=30 + i) for i, t in enumerate(tabs)]
    Ys[2][:4095] = tabs[2][1:]                               # exact hits on every searched key
    Ys[2][4095:8190] = torch.from_numpy(np.nextafter(tabs[2][1:].numpy(), -np.inf))
    Y = torch.cat(Ys)
    Y_off = np.concatenate([[0], np.cumsum([len(y) for y in Ys])])
    want = oracle.search_1d_batched(X_off, X.numpy(), Y_off, Y.numpy(), side)
    plan = ss.Plan.create_1d(X_off, X.to(DEV), side=side, tile=tile)
    inf = plan.info()
    assert inf.max_occupancy <= 2
    buf = torch.empty(Y.numel() + 1, dtype=torch.float64, device=DEV)
    Yd = buf[1:]                                              # 8-byte aligned, not 16
    Yd.copy_(Y)
    out = torch.full((Y.numel(),), -1, dtype=torch.int32, device=DEV)
    stat = ss.new_stat()
    plan.bind_1d(Y_off, Yd, out, stat=stat)
    assert plan.info().block_threads == 512
    plan.execute()
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    assert ss.read_stat(stat).flags == 0
    # the same batch with the default directory budget keeps 256-thread blocks
    plan2 = ss.Plan.create_1d(X_off, X.to(DEV), side=side, tile=tile, dir_cap=4096)
    assert plan2.info().max_occupancy > 2
    out2 = torch.full_like(out, -1)
    plan2.bind_1d(Y_off, Yd, out2)
    assert plan2.info().block_threads == 256
    plan2.execute()
    np.testing.assert_array_equal(out2.cpu().numpy(), want)


@pytest.mark.parametrize("model", ["none", "spline", "mlp", "loghash"])
@pytest.mark.parametrize("side", [0, 1])
def test_plan_every_layout_regime(ss, model, side, tmp_path):
    """One plan over tables of every layout regime: staged whole with fitted
    16-bit directories (2 .. 8128 entries, jittered and clustered), wide
    sections of different directory budgets (8129, 20000 and 65535
    entries), and a two-level table (80000 entries, searched in global
    memory); exact key hits and their neighbours in every table.  The plan
    also goes through a file: the load's layout checks accept every regime
    and the loaded plan gives the same answers."""
    rng = np.random.default_rng(77)
    tabs = [wl.log_spaced_table(n, 1e-4, 1e6, 0.2, seed=200 + n) for n in (2, 3, 17, 255, 1025, 8128, 8129, 20000)]
    tabs += [wl.sweep_table(4096, seed=9), wl.sweep_table(65535, seed=10), wl.log_spaced_table(80000, 1e-3, 1e7, 0.2, seed=11)]
    Ys = []
    for t in tabs:
        x = t.numpy()
        hits = x[rng.integers(0, len(x), 500)]
        Ys.append(np.concatenate([10 ** rng.uniform(np.log10(x[0]) - 1, np.log10(x[-1]) + 1, 6000), hits,
                                  np.nextafter(hits, np.inf), np.nextafter(hits, -np.inf)]))
    X = torch.cat(tabs)
    X_off = np.concatenate([[0], np.cumsum([len(t) for t in tabs])])
    Y = torch.as_tensor(np.concatenate(Ys))
    Y_off = np.concatenate([[0], np.cumsum([len(y) for y in Ys])])
    want = oracle.search_1d_batched(X_off, X.numpy(), Y_off, Y.numpy(), side)
    b = wl.Batched1D(torch.as_tensor(X_off), X, torch.as_tensor(Y_off), Y, None, None)
    plan, got, st = run_plan_1d(ss, b, model=model, side=side, mlp_epochs=60 if model == "mlp" else None)
    np.testing.assert_array_equal(got, want)
    assert st.flags == 0
    path = tmp_path / "regimes.bin"
    plan.save(path)
    re = ss.Plan.load(path)
    out = torch.full((len(Y),), -1, dtype=torch.int32, device=DEV)
    re.bind_1d(b.Y_off, Y.to(DEV), out)
    re.execute()
    np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_plan_wide_section_with_ties(ss):
    """Tables of 8129..~76K entries search a wide section (16-bit offsets in
    shared memory).  Runs of consecutive doubles inside a leaf whose other
    keys are far apart truncate to equal offsets, so targets at and next to
    those keys take the full-key comparison; both sides, indices exact."""
    rng = np.random.default_rng(21)
    base = np.logspace(0, 10, 10_000)
    runs = []
    for x in rng.choice(base[100:-100], 25, replace=False):
        v = x
        for _ in range(12):
            v = np.nextafter(v, np.inf)
            runs.append(v)
    X = np.unique(np.concatenate([base, runs]))
    assert np.all(np.diff(X) > 0) and len(X) > 8200
    near = np.concatenate([X, np.nextafter(X, np.inf), np.nextafter(X, -np.inf)])
    Y = np.concatenate([near, 10 ** rng.uniform(-1, 11, 200_000), [np.nan, -0.0, np.inf, -np.inf]])
    Xt, Yt = torch.from_numpy(X), torch.from_numpy(Y)
    b = wl.Batched1D(torch.tensor([0, len(X)]), Xt, torch.tensor([0, len(Y)]), Yt, None, None)
    for side in (0, 1):
        want = oracle.search_1d(X, Y, side)
        plan, got, st = run_plan_1d(ss, b, side=side)
        assert "wide" in [c[0] for c in plan.choices().values()]
        np.testing.assert_array_equal(got, want)
        assert st.flags == 0 and st.nan_targets == 1
    # the 65536-entry clustered table of the size sweep, through the wide section
    X = wl.sweep_table(65536)
    Y = wl.log_uniform(300_000, 0.5e-6, 2e4, seed=22)
    b = wl.Batched1D(torch.tensor([0, len(X)]), X, torch.tensor([0, len(Y)]), Y, None, None)
    plan, got, st = run_plan_1d(ss, b)
    assert plan.choices()[7][0] == "wide"
    np.testing.assert_array_equal(got, oracle.search_1d(X.numpy(), Y.numpy()))


def test_plan_empty_tiny_tiles_and_misaligned(ss):
    rng = np.random.default_rng(5)
    sizes = [2, 3, 17, 300, 2000, 5]
    counts = [0, 1, 63, 64, 65, 0, 1000, 3]
    sizes = sizes + [40, 50]
    tabs = [wl.log_spaced_table(n, 1e-3, 1e3, 0.1, seed=n) for n in sizes]
    X = torch.cat(tabs)
    X_off = np.concatenate([[0], np.cumsum(sizes)])
    Y = torch.as_tensor(10 ** rng.uniform(-4, 4, sum(counts)))
    Y_off = np.concatenate([[0], np.cumsum(counts)])
    want = oracle.search_1d_batched(X_off, X.numpy(), Y_off, Y.numpy())
    for model in ("none", "spline"):
        for off in (0, 1, 3):
            plan = ss.Plan.create_1d(X_off, X.to(DEV), model=model, tile=64)
            ybuf = torch.zeros(len(Y) + 4, dtype=torch.float64, device=DEV)
            ybuf[off:off + len(Y)] = Y.to(DEV)
            obuf = torch.full((len(Y) + 4,), -5, dtype=torch.int32, device=DEV)
            plan.bind_1d(Y_off, ybuf[off:off + len(Y)], obuf[off:off + len(Y)])
            plan.execute()
            o = obuf.cpu().numpy()
            np.testing.assert_array_equal(o[off:off + len(Y)], want)
            assert np.all(o[:off] == -5) and np.all(o[off + len(Y):] == -5)


@pytest.mark.parametrize("model", ["spline", "mlp", "loghash"])
@pytest.mark.parametrize("side", [0, 1])
def test_learned_windows_at_the_table_ends(ss, model, side):
    """Learned proposals on tables of 2..9 entries put their checked windows
    against both ends of the key array (window start 0, window end at the
    last key, where the check reads the sentinels after it).  Every entry,
    its neighbouring doubles, values between entries, far outside the range
    and IEEE specials; indices bit-exact for both sides."""
    sizes = list(range(2, 10))
    tabs = [wl.log_spaced_table(n, 0.5, 2.0 ** n, 0.2, seed=100 + n) for n in sizes]
    X = torch.cat(tabs)
    X_off = np.concatenate([[0], np.cumsum(sizes)])
    Ys = []
    for t in tabs:
        x = t.numpy()
        mids = np.sqrt(x[1:] * x[:-1])
        Ys.append(np.concatenate([x, np.nextafter(x, np.inf), np.nextafter(x, -np.inf), mids,
                                  [x[0] / 4, x[-1] * 4, 0.0, -0.0, -1.0, np.inf, -np.inf, np.nan]]))
    Y = torch.as_tensor(np.concatenate(Ys))
    Y_off = np.concatenate([[0], np.cumsum([len(y) for y in Ys])])
    want = oracle.search_1d_batched(X_off, X.numpy(), Y_off, Y.numpy(), side)
    b = wl.Batched1D(torch.as_tensor(X_off), X, torch.as_tensor(Y_off), Y, None, None)
    plan, got, st = run_plan_1d(ss, b, model=model, side=side, tile=1024,
                                mlp_epochs=100 if model == "mlp" else None)
    np.testing.assert_array_equal(got, want)
    assert st.nan_targets == len(sizes)


def test_plan_graph_replay_and_rebind(ss):
    b = small_batch(seed=6)
    plan = ss.Plan.create_1d(b.X_off, b.X.to(DEV), model="spline")
    Yd = b.Y.to(DEV)
    out = torch.empty(len(b.Y), dtype=torch.int32, device=DEV)
    plan.bind_1d(b.Y_off, Yd, out)
    plan.execute()
    first = out.clone()
    Yd.mul_(1.5)                                   # new targets in the bound buffer
    plan.execute()
    want2 = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), (b.Y * 1.5).numpy())
    np.testing.assert_array_equal(out.cpu().numpy(), want2)
    Yd.div_(1.5)
    plan.execute()
    assert torch.equal(out, first)


def test_plan_bound_to_page_locked_host_buffers(ss):
    """A plan bound to page-locked host buffers: the kernel streams targets in
    and indices out over the host link; same answers as device buffers."""
    b = small_batch(seed=13)
    want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy())
    plan = ss.Plan.create_1d(b.X_off, b.X.to(DEV))
    hY = b.Y.clone().pin_memory()
    hO = torch.full((b.Y.numel(),), -1, dtype=torch.int32).pin_memory()
    plan.bind_1d(b.Y_off, hY, hO)
    plan.execute()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hO.numpy(), want)
    with pytest.raises(TypeError):
        plan.bind_1d(b.Y_off, b.Y.clone(), hO)          # pageable host memory is refused
    b2 = wl.batched_2d(ntables=5, pairs_per_table=2001, seed=14)
    wi, wv = oracle.search_interp_2d_batched(b2.R_off.numpy(), b2.R.numpy(), b2.T_off.numpy(), b2.T.numpy(),
                                             b2.F_off.numpy(), b2.F.numpy(), b2.Y_off.numpy(), b2.Y2.numpy())
    p2 = ss.Plan.create_2d(b2.R_off, b2.R.to(DEV), b2.T_off, b2.T.to(DEV), b2.F_off, b2.F.to(DEV))
    m = b2.Y2.shape[0]
    hI = torch.empty((m, 2), dtype=torch.int32).pin_memory()
    hV = torch.empty(m, dtype=torch.float64).pin_memory()
    p2.bind_2d(b2.Y_off, b2.Y2.clone().pin_memory(), hI, hV)
    p2.execute()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hI.numpy(), wi)
    assert (np.abs(hV.numpy() - wv) / np.abs(wv)).max() <= REL_TOL


def walk_batch_1d(sizes, per_table, seed, order, side=0):
    """Tables of the given sizes (jittered log spacing) and per table a
    target sequence: a random walk in log space ("walk"), the same with 2 %
    of its steps leaping across up to the whole range ("jumps"), sorted
    log-uniform targets ("sorted") or log-uniform ones ("random")."""
    Xs, Ys = [], []
    for k, n in enumerate(sizes):
        lo, hi = 10.0 ** (-6 + k), 10.0 ** (4 + k)
        X = wl.log_spaced_table(n, lo, hi, 0.1, seed * 31 + k)
        a, b = 0.5 * lo, 2 * hi
        if order == "walk":
            Y = wl.walk_1d(per_table, a, b, seed * 37 + k)
        elif order == "jumps":
            Y = wl.walk_1d(per_table, a, b, seed * 37 + k, jump=0.02)
        else:
            Y = wl.log_uniform(per_table, a, b, seed * 37 + k)
            if order == "sorted":
                Y = torch.sort(Y).values
        Xs.append(X)
        Ys.append(Y)
    X_off = torch.tensor(np.concatenate([[0], np.cumsum([len(x) for x in Xs])]))
    Y_off = torch.tensor(np.concatenate([[0], np.cumsum([len(y) for y in Ys])]))
    return wl.Batched1D(X_off, torch.cat(Xs), Y_off, torch.cat(Ys), None, None)


@pytest.mark.parametrize("order", ["walk", "jumps", "sorted", "random"])
@pytest.mark.parametrize("side", [0, 1])
def test_hunt_1d_exact_on_every_order(ss, order, side):
    """Hunt and locate on 1D plans: tables staged whole (64, 2000 entries)
    and searched in global memory (20,000 and 100,000 entries), coherent,
    leaping, sorted and random targets; every index equals the oracle's."""
    b = walk_batch_1d((64, 2000, 20_000, 100_000), 30_011, seed=41, order=order)
    want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy(), side)
    for tile in (0, 997):                     # tuned tiles, and small odd ones (ragged warp runs)
        plan, got, st = run_plan_1d(ss, b, model="hunt", side=side, tile=tile)
        np.testing.assert_array_equal(got, want)
        assert st.flags == 0
    # off 16-byte alignment: the scalar head and tail of every tile
    Yd = torch.empty(b.Y.numel() + 1, dtype=torch.float64, device=DEV)
    Yd[1:] = b.Y.to(DEV)
    out = torch.full((b.Y.numel() + 1,), -1, dtype=torch.int32, device=DEV)
    plan.bind_1d(b.Y_off, Yd[1:], out[1:])
    plan.execute()
    np.testing.assert_array_equal(out[1:].cpu().numpy(), want)
    assert int(out[0]) == -1


def test_hunt_1d_starts_runs_with_the_bucket_search(ss):
    # the hunt reads the staged keys, which a table staged for the
    # breadth-first or ballot search does not carry: such plans are refused
    b = walk_batch_1d((300, 9000), 20_000, seed=43, order="jumps")
    for algo in ("binary", "ballot"):
        with pytest.raises(ss.SSError) as e:
            ss.Plan.create_1d(b.X_off, b.X.to(DEV), model="hunt", algo=algo)
        assert e.value.code == 1
    want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy())
    plan, got, _ = run_plan_1d(ss, b, model="hunt", algo="bucket", autotune=True)
    np.testing.assert_array_equal(got, want)
    assert all(c[0] == "bucket" for c in plan.choices().values())


@pytest.mark.parametrize("order", ["walk", "jumps", "random"])
def test_hunt_2d_exact_on_every_order(ss, order):
    """The 2D hunt: each axis hunts from the previous pair's index; walks,
    leaping walks and random pairs all give the oracle's indices and values
    within 1e-12, with bucket and binary axis searches."""
    b2 = wl.batched_2d(ntables=6, pairs_per_table=6001, coherent=order != "random", seed=18,
                       jump=0.02 if order == "jumps" else 0.0)
    wi, wv = oracle.search_interp_2d_batched(b2.R_off.numpy(), b2.R.numpy(), b2.T_off.numpy(), b2.T.numpy(),
                                             b2.F_off.numpy(), b2.F.numpy(), b2.Y_off.numpy(), b2.Y2.numpy())
    m = b2.Y2.shape[0]
    for algo in ("auto", "binary"):
        for tile in (0, 333):
            plan = ss.Plan.create_2d(b2.R_off, b2.R.to(DEV), b2.T_off, b2.T.to(DEV), b2.F_off, b2.F.to(DEV),
                                     model="hunt", algo=algo, tile=tile)
            idx = torch.full((m, 2), -1, dtype=torch.int32, device=DEV)
            val = torch.empty(m, dtype=torch.float64, device=DEV)
            stat = ss.new_stat()
            plan.bind_2d(b2.Y_off, b2.Y2.to(DEV), idx, val, stat=stat)
            plan.execute()
            np.testing.assert_array_equal(idx.cpu().numpy(), wi)
            assert (np.abs(val.cpu().numpy() - wv) / np.abs(wv)).max() <= REL_TOL
            assert ss.read_stat(stat).flags == 0


def test_plan_2d_binary_axes_with_options(ss):
    """Linear extrapolation reads axis entries on the fp64 path; with
    binary-search axes those entries must be staged too."""
    b = wl.batched_2d(ntables=5, pairs_per_table=3001, seed=19)
    rng = np.random.default_rng(20)
    Y2 = b.Y2.numpy() * np.exp(rng.uniform(-2.0, 2.0, size=b.Y2.shape))
    wi, wv = oracle.search_interp_2d_batched(b.R_off.numpy(), b.R.numpy(), b.T_off.numpy(), b.T.numpy(),
                                             b.F_off.numpy(), b.F.numpy(), b.Y_off.numpy(), Y2, extrap=1)
    plan = ss.Plan.create_2d(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV), algo="binary",
                             extrap=True)
    m = Y2.shape[0]
    idx = torch.empty((m, 2), dtype=torch.int32, device=DEV)
    val = torch.empty(m, dtype=torch.float64, device=DEV)
    plan.bind_2d(b.Y_off, torch.from_numpy(Y2).to(DEV), idx, val)
    plan.execute()
    np.testing.assert_array_equal(idx.cpu().numpy(), wi)
    v = val.cpu().numpy()
    outside = 0
    for k in range(5):
        y0, y1 = int(b.Y_off[k]), int(b.Y_off[k + 1])
        R = b.R.numpy()[int(b.R_off[k]):int(b.R_off[k + 1])]
        T = b.T.numpy()[int(b.T_off[k]):int(b.T_off[k + 1])]
        F2 = b.F.numpy()[int(b.F_off[k]):int(b.F_off[k + 1])].reshape(len(R), len(T))
        y = Y2[y0:y1]
        outside += int((~((y[:, 0] >= R[0]) & (y[:, 0] <= R[-1]) & (y[:, 1] >= T[0]) & (y[:, 1] <= T[-1]))).sum())
        cr = np.minimum(wi[y0:y1, 0], len(R) - 2)
        ct = np.minimum(wi[y0:y1, 1], len(T) - 2)
        wr = np.abs((y[:, 0] - R[cr]) / (R[cr + 1] - R[cr]))
        wt = np.abs((y[:, 1] - T[ct]) / (T[ct + 1] - T[ct]))
        lo = np.abs(1 - wt) * np.abs(F2[cr, ct]) + wt * np.abs(F2[cr, ct + 1])
        hi = np.abs(1 - wt) * np.abs(F2[cr + 1, ct]) + wt * np.abs(F2[cr + 1, ct + 1])
        assert (np.abs(v[y0:y1] - wv[y0:y1]) <= REL_TOL * (np.abs(1 - wr) * lo + wr * hi)).all()
    assert outside > 500


def test_plan_not_sorted_rejected(ss):
    X = torch.tensor([1.0, 2.0, 2.0, 3.0, 1.0, 5.0, 7.0], dtype=torch.float64, device=DEV)
    with pytest.raises(ss.SSError) as e:
        ss.Plan.create_1d([0, 4, 7], X)
    assert e.value.code == 2


def _blob_headers(raw):
    """Parse a saved plan file: returns (positions of blob headers, blob data start)."""
    pos = 8 + 4 * 3 + ctypes.sizeof(PlanOpts)  # magic, version/kind/ntables, options
    def vec(pos, fmt, size):
        n = struct.unpack_from("<q", raw, pos)[0]
        return list(struct.unpack_from("<%d%s" % (n, fmt), raw, pos + 8)), pos + 8 + n * size
    vals = {}
    for name, fmt, size in (("sizes", "i", 4), ("sizes_t", "i", 4), ("X_off", "q", 8), ("dir_cap", "i", 4),
                            ("algo", "i", 4), ("blob_off", "q", 8), ("grid_off", "q", 8)):
        vals[name], pos = vec(pos, fmt, size)
    pos += 3 * 8 * 4 + 4                      # bucket arrays, tuned
    pos += 8                                  # blob_bytes
    return vals["blob_off"], pos


def test_plan_save_load_and_forced_fallback(ss, tmp_path):
    b = small_batch(seed=7)
    want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy())
    plan, got, st = run_plan_1d(ss, b, model="mlp", mlp_epochs=100)
    np.testing.assert_array_equal(got, want)
    path = tmp_path / "plan.bin"
    plan.save(path)
    re = ss.Plan.load(path)
    out = torch.empty(len(b.Y), dtype=torch.int32, device=DEV)
    re.bind_1d(b.Y_off, b.Y.to(DEV), out)
    re.execute()
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    assert re.info().max_window == plan.info().max_window
    # corrupt every model (scrambled weights) and set its window to zero: the
    # exact check must reject the proposals and the plain search must take over
    raw = bytearray(path.read_bytes())
    offs, start = _blob_headers(bytes(raw))
    rng = np.random.default_rng(0)
    for o in offs:
        h = start + o
        struct.pack_into("<i", raw, h + 36, 0)                                     # E
        off_mlp = struct.unpack_from("<i", raw, h + 48)[0]
        struct.pack_into("<65f", raw, h + off_mlp, *rng.standard_normal(65).astype(np.float32))
    bad = tmp_path / "bad.bin"
    bad.write_bytes(bytes(raw))
    re2 = ss.Plan.load(bad)
    stat = ss.new_stat()
    out.fill_(-1)
    re2.bind_1d(b.Y_off, b.Y.to(DEV), out, stat=stat)
    re2.execute()
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    st = ss.read_stat(stat)
    assert st.fallbacks > len(b.Y) // 2


# byte offsets of blob header fields (the 128-byte header of every prepared table)
HDR_NB, HDR_OCC, HDR_E, HDR_S0, HDR_OFF_DIR, HDR_OFF_CELLS = 28, 32, 36, 40, 52, 112


def test_plan_load_refuses_inconsistent_layouts(ss, tmp_path):
    """A plan file whose layout does not hold together is refused by the
    load's host-side checks (SS_EINVAL) before any kernel could read outside
    it: a shifted blob offset, a bucket count above the budget, a directory
    that does not start at 0, a wrong occupancy, a negative window, a wrong
    ballot stride, a moved 2D cell table."""
    b = small_batch(seed=12, ntables=20)
    plan = ss.Plan.create_1d(b.X_off, b.X.to(DEV), model="spline")
    path = tmp_path / "ok.bin"
    plan.save(path)
    raw = path.read_bytes()
    offs, start = _blob_headers(raw)
    h = start + offs[3]
    blob_off_pos = raw.index(struct.pack("<q", len(offs)) + struct.pack("<%dq" % len(offs), *offs))

    def corrupt(edit):
        r = bytearray(raw)
        edit(r)
        bad = tmp_path / "bad.bin"
        bad.write_bytes(bytes(r))
        with pytest.raises(ss.SSError) as e:
            ss.Plan.load(bad)
        assert e.value.code == 1 and "corrupt plan file" in str(e.value)

    dir_cap = struct.unpack_from("<i", raw, h + 44)[0]
    off_dir = struct.unpack_from("<i", raw, h + HDR_OFF_DIR)[0]
    occ = struct.unpack_from("<i", raw, h + HDR_OCC)[0]
    corrupt(lambda r: struct.pack_into("<q", r, blob_off_pos + 8 + 8 * 2, offs[2] + 256))
    corrupt(lambda r: struct.pack_into("<i", r, h + HDR_NB, dir_cap + 1))
    corrupt(lambda r: struct.pack_into("<H", r, h + off_dir, 1))
    corrupt(lambda r: struct.pack_into("<i", r, h + HDR_OCC, occ + 1))
    corrupt(lambda r: struct.pack_into("<i", r, h + HDR_E, -1))
    corrupt(lambda r: struct.pack_into("<i", r, h + HDR_S0, 7))
    ss.Plan.load(path)   # the untouched file still loads

    b2 = wl.batched_2d(ntables=3, pairs_per_table=100, seed=13)
    plan2 = ss.Plan.create_2d(b2.R_off, b2.R.to(DEV), b2.T_off, b2.T.to(DEV), b2.F_off, b2.F.to(DEV))
    path2 = tmp_path / "ok2.bin"
    plan2.save(path2)
    raw = path2.read_bytes()
    offs, start = _blob_headers(raw)
    h = start + offs[1]
    cells = struct.unpack_from("<i", raw, h + HDR_OFF_CELLS)[0]
    corrupt(lambda r: struct.pack_into("<i", r, h + HDR_OFF_CELLS, cells + 16))
    ss.Plan.load(path2)


def test_plan_autotune_and_cache(ss, tmp_path):
    b = wl.batched_1d(ntables=60, count_scale=0.004, seed=8)
    want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy())
    cache = str(tmp_path / "tune.json")
    plan, got, _ = run_plan_1d(ss, b, autotune=True, tune_cache=cache)
    np.testing.assert_array_equal(got, want)
    inf = plan.info()
    assert inf.tuned == 1 and os.path.exists(cache)
    ch = plan.choices()
    assert ch and all(a in ss.BLOB_ALGOS[:5] and t >= 1024 for a, t, _ in ch.values())
    text = open(cache).read()
    assert '"buckets"' in text and '"tile_multiple"' in text
    plan2, got2, _ = run_plan_1d(ss, b, autotune=True, tune_cache=cache)
    np.testing.assert_array_equal(got2, want)
    assert {k: v[0] for k, v in plan2.choices().items()} == {k: v[0] for k, v in ch.items()}
    # a cache that lacks one of the plan's size buckets is not taken: the plan
    # is tuned afresh and the cache rewritten with every bucket
    lines = text.splitlines()
    entries = [i for i, ln in enumerate(lines) if '{"bucket": ' in ln]
    assert len(entries) >= 2
    partial = [ln for i, ln in enumerate(lines) if i != entries[-1]]
    partial[entries[-2]] = partial[entries[-2]].rstrip(",")
    open(cache, "w").write("\n".join(partial) + "\n")
    assert open(cache).read().count('{"bucket": ') == len(entries) - 1
    plan3, got3, _ = run_plan_1d(ss, b, autotune=True, tune_cache=cache)
    np.testing.assert_array_equal(got3, want)
    assert plan3.info().tuned == 1
    assert open(cache).read().count('{"bucket": ') == len(entries)


def test_learned_gain(ss):
    """What training buys: the trained MLP's fix-up window against the untrained
    initialisation (same architecture) on the 65536-entry clustered table."""
    X = wl.sweep_table(65536)
    b = wl.Batched1D(torch.tensor([0, len(X)]), X, torch.tensor([0, 200_000]),
                     wl.log_uniform(200_000, 0.5e-6, 2e4, seed=3), None, None)
    want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy())
    trained, got_t, st_t = run_plan_1d(ss, b, model="mlp", mlp_epochs=400)
    untrained, got_u, st_u = run_plan_1d(ss, b, model="mlp", mlp_epochs=0)
    spline, got_s, st_s = run_plan_1d(ss, b, model="spline")
    for g in (got_t, got_u, got_s):
        np.testing.assert_array_equal(g, want)
    Et, Eu = trained.info().max_window, untrained.info().max_window
    assert Et * 4 < Eu, (Et, Eu)
    assert trained.info().train_loss < 1e-3


def test_loghash_proposal(ss):
    """The logarithm hash of Sec. 3.4 (Eqs. 1-2) as an untrained proposal: on
    exactly log-spaced tables it is off by at most a step or two (rounding of
    the fp32 logarithm), on a table with no positive range it proposes 0 and
    the window spans the table; the indices are exact in both cases."""
    tabs = [wl.log_spaced_table(n, 1e-6, 1e4, 0.0, seed=n) for n in (17, 300, 2001)]
    counts = [5000, 7001, 9003]
    Y = torch.cat([wl.log_uniform(c, 0.5e-6, 2e4, seed=i) for i, c in enumerate(counts)])
    X_off = torch.tensor(np.concatenate([[0], np.cumsum([len(t) for t in tabs])]))
    Y_off = torch.tensor(np.concatenate([[0], np.cumsum(counts)]))
    b = wl.Batched1D(X_off, torch.cat(tabs), Y_off, Y, None, None)
    want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy())
    plan, got, st = run_plan_1d(ss, b, model="loghash")
    np.testing.assert_array_equal(got, want)
    assert 1 <= plan.info().max_window <= 3, plan.info().max_window
    assert st.fallbacks == 0
    # a table through zero: no positive range, a = c = 0
    Xn = torch.linspace(-5.0, 5.0, 64, dtype=torch.float64)
    Yn = torch.linspace(-6.0, 6.0, 1001, dtype=torch.float64)
    bn = wl.Batched1D(torch.tensor([0, 64]), Xn, torch.tensor([0, 1001]), Yn, None, None)
    want = oracle.search_1d_batched(bn.X_off.numpy(), bn.X.numpy(), bn.Y_off.numpy(), bn.Y.numpy())
    plan, got, st = run_plan_1d(ss, bn, model="loghash")
    np.testing.assert_array_equal(got, want)
    assert plan.info().max_window == 64 and st.fallbacks == 0


# ---------------------------------------------------------------- 2D plans

@pytest.mark.parametrize("coherent", [False, True])
@pytest.mark.parametrize("model", ["none", "spline", "mlp", "loghash", "hunt"])
def test_plan_2d_batched(ss, model, coherent):
    b = wl.batched_2d(ntables=12, pairs_per_table=4001, coherent=coherent, seed=9)
    wi, wv = oracle.search_interp_2d_batched(b.R_off.numpy(), b.R.numpy(), b.T_off.numpy(), b.T.numpy(),
                                             b.F_off.numpy(), b.F.numpy(), b.Y_off.numpy(), b.Y2.numpy())
    plan = ss.Plan.create_2d(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV), model=model,
                             mlp_epochs=150 if model == "mlp" else None)
    m = b.Y2.shape[0]
    idx = torch.empty((m, 2), dtype=torch.int32, device=DEV)
    val = torch.empty(m, dtype=torch.float64, device=DEV)
    stat = ss.new_stat()
    plan.bind_2d(b.Y_off, b.Y2.to(DEV), idx, val, stat=stat)
    plan.execute()
    np.testing.assert_array_equal(idx.cpu().numpy(), wi)
    rel = np.abs(val.cpu().numpy() - wv) / np.abs(wv)
    assert rel.max() <= REL_TOL
    assert ss.read_stat(stat).flags == 0


def test_plan_2d_lean_kernel(ss):
    """The lean kernel runs when every axis is a bucket search over a whole
    staged axis with at most two keys per bucket and float-float cells (the
    standard batch); it gives the oracle's indices and values, on aligned
    and misaligned arrays, with NaN pairs; so do its instances for the
    spline, MLP and logarithm-hash models, which run when every window is
    at most 4 keys, and for the hunt; plans outside its case (an
    interpolation option, a binary-search axis) run the general kernel."""
    b = wl.batched_2d(ntables=20, pairs_per_table=5003, seed=27)
    Y2 = b.Y2.clone()
    Y2[7, 0] = float("nan")                 # a NaN coordinate: value NaN, indices exact
    Y2[5000, 1] = float("nan")
    wi, wv = oracle.search_interp_2d_batched(b.R_off.numpy(), b.R.numpy(), b.T_off.numpy(), b.T.numpy(),
                                             b.F_off.numpy(), b.F.numpy(), b.Y_off.numpy(), Y2.numpy())
    m = Y2.shape[0]

    def run(plan, offset):
        Yd = torch.empty((m + offset, 2), dtype=torch.float64, device=DEV)
        Yd[offset:] = Y2.to(DEV)
        idx = torch.full((m + offset, 2), -1, dtype=torch.int32, device=DEV)
        val = torch.empty(m + offset, dtype=torch.float64, device=DEV)
        stat = ss.new_stat()
        plan.bind_2d(b.Y_off, Yd[offset:], idx[offset:], val[offset:], stat=stat)
        plan.execute()
        np.testing.assert_array_equal(idx[offset:].cpu().numpy(), wi)
        if offset:
            assert (idx[0].cpu().numpy() == -1).all()
        got = val[offset:].cpu().numpy()
        assert np.array_equal(np.isnan(got), np.isnan(wv))
        ok = ~np.isnan(wv)
        assert (np.abs(got[ok] - wv[ok]) / np.abs(wv[ok])).max() <= REL_TOL
        st = ss.read_stat(stat)
        assert st.flags == 0 and st.nan_targets == 2

    plan = ss.Plan.create_2d(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV))
    for offset in (0, 1):
        run(plan, offset)
        assert plan.info().lean_kernel == 1 and plan.info().max_occupancy <= 2
    run(ss.Plan.create_2d(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV), autotune=True), 0)
    for model in ("spline", "loghash", "mlp"):
        learned = ss.Plan.create_2d(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV), model=model)
        for offset in (0, 1):
            run(learned, offset)
        assert learned.info().lean_kernel == (1 if learned.info().max_window <= 4 else 0), model
    hunt = ss.Plan.create_2d(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV), model="hunt")
    for offset in (0, 1):
        run(hunt, offset)
        assert hunt.info().lean_kernel == 1
    for kw in (dict(algo="binary"), dict(extrap=True)):
        other = ss.Plan.create_2d(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV), **kw)
        if "extrap" not in kw:
            run(other, 0)
        else:
            other.bind_2d(b.Y_off, Y2.to(DEV), torch.empty((m, 2), dtype=torch.int32, device=DEV),
                          torch.empty(m, dtype=torch.float64, device=DEV))
        assert other.info().lean_kernel == 0, kw


@pytest.mark.parametrize("model", ["loghash", "mlp"])
def test_plan_2d_learned_lean_forced_fallback(ss, tmp_path, model):
    """The lean kernel's logarithm-hash and MLP instances with every
    proposal wrong: a saved 2D plan whose axes' coefficients (log hash) or
    parameters (MLP) are zeroed, so that every proposal is 0, and whose
    windows are set to 0 still runs the lean kernel, rejects the proposals
    (the walk of zero keys proves only an answer of 0) and gives the
    oracle's indices and values through the plain search, counting each
    rejected proposal as a fallback."""
    b = wl.batched_2d(ntables=9, pairs_per_table=4001, seed=31)
    wi, wv = oracle.search_interp_2d_batched(b.R_off.numpy(), b.R.numpy(), b.T_off.numpy(), b.T.numpy(),
                                             b.F_off.numpy(), b.F.numpy(), b.Y_off.numpy(), b.Y2.numpy())
    plan = ss.Plan.create_2d(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV), model=model,
                             mlp_epochs=40 if model == "mlp" else None)
    path = tmp_path / "plan2d.bin"
    plan.save(path)
    raw = bytearray(path.read_bytes())
    offs, start = _blob_headers(bytes(raw))
    assert len(offs) == 2 * 9
    for o in offs:
        h = start + o
        struct.pack_into("<i", raw, h + HDR_E, 0)
        off_mlp = struct.unpack_from("<i", raw, h + 48)[0]
        if model == "loghash":
            struct.pack_into("<2f", raw, h + off_mlp + 4 * 65, 0.0, 0.0)        # a = c = 0: proposal 0
        else:
            struct.pack_into("<65f", raw, h + off_mlp, *([0.0] * 65))           # network output 0: proposal 0
    bad = tmp_path / "bad2d.bin"
    bad.write_bytes(bytes(raw))
    re = ss.Plan.load(bad)
    m = b.Y2.shape[0]
    idx = torch.full((m, 2), -1, dtype=torch.int32, device=DEV)
    val = torch.empty(m, dtype=torch.float64, device=DEV)
    stat = ss.new_stat()
    re.bind_2d(b.Y_off, b.Y2.to(DEV), idx, val, stat=stat)
    re.execute()
    assert re.info().lean_kernel == 1
    np.testing.assert_array_equal(idx.cpu().numpy(), wi)
    assert (np.abs(val.cpu().numpy() - wv) / np.abs(wv)).max() <= REL_TOL
    # every coordinate whose answer is not 0 is a rejected proposal
    st = ss.read_stat(stat)
    assert st.fallbacks == int(np.count_nonzero(wi != 0)), (st.fallbacks, int(np.count_nonzero(wi != 0)))


@pytest.mark.parametrize("extrap,logspace", [(1, 0), (0, 1), (1, 1)])
def test_plan_2d_interpolation_options(ss, extrap, logspace):
    """2D plans with linear extrapolation / log-coordinate weights: pairs
    spread beyond the axes by up to a factor e^2 either way."""
    b = wl.batched_2d(ntables=7, pairs_per_table=3001, seed=15)
    rng = np.random.default_rng(16)
    Y2 = b.Y2.numpy() * np.exp(rng.uniform(-2.0, 2.0, size=b.Y2.shape))
    args = (b.R_off.numpy(), b.R.numpy(), b.T_off.numpy(), b.T.numpy(), b.F_off.numpy(), b.F.numpy(), b.Y_off.numpy())
    wi, wv = oracle.search_interp_2d_batched(*args, Y2, extrap=extrap, logspace=logspace)
    plan = ss.Plan.create_2d(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV), extrap=bool(extrap),
                             logspace=bool(logspace))
    m = Y2.shape[0]
    idx = torch.empty((m, 2), dtype=torch.int32, device=DEV)
    val = torch.empty(m, dtype=torch.float64, device=DEV)
    plan.bind_2d(b.Y_off, torch.from_numpy(Y2).to(DEV), idx, val)
    plan.execute()
    np.testing.assert_array_equal(idx.cpu().numpy(), wi)
    val = val.cpu().numpy()
    for k in range(7):
        r0, r1 = int(b.R_off[k]), int(b.R_off[k + 1])
        t0, t1 = int(b.T_off[k]), int(b.T_off[k + 1])
        f0, f1 = int(b.F_off[k]), int(b.F_off[k + 1])
        y0, y1 = int(b.Y_off[k]), int(b.Y_off[k + 1])
        R, T, F = b.R.numpy()[r0:r1], b.T.numpy()[t0:t1], b.F.numpy()[f0:f1]
        nr, nt = len(R), len(T)
        cr = np.minimum(wi[y0:y1, 0], nr - 2)
        ct = np.minimum(wi[y0:y1, 1], nt - 2)
        def w(X, c, x):
            if logspace:
                return np.abs((np.log(x) - np.log(X[c])) / (np.log(X[c + 1]) - np.log(X[c])))
            return np.abs((x - X[c]) / (X[c + 1] - X[c]))
        wr, wt = w(R, cr, Y2[y0:y1, 0]), w(T, ct, Y2[y0:y1, 1])
        F2 = F.reshape(nr, nt)
        lo = np.abs(1 - wt) * np.abs(F2[cr, ct]) + wt * np.abs(F2[cr, ct + 1])
        hi = np.abs(1 - wt) * np.abs(F2[cr + 1, ct]) + wt * np.abs(F2[cr + 1, ct + 1])
        scale = np.abs(1 - wr) * lo + wr * hi
        assert (np.abs(val[y0:y1] - wv[y0:y1]) <= REL_TOL * scale).all()


def test_plan_2d_save_load_and_autotune(ss, tmp_path):
    b = wl.batched_2d(ntables=6, pairs_per_table=3000, seed=10)
    wi, wv = oracle.search_interp_2d_batched(b.R_off.numpy(), b.R.numpy(), b.T_off.numpy(), b.T.numpy(),
                                             b.F_off.numpy(), b.F.numpy(), b.Y_off.numpy(), b.Y2.numpy())
    plan = ss.Plan.create_2d(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV), autotune=True)
    path = tmp_path / "p2.bin"
    plan.save(path)
    for p in (plan, ss.Plan.load(path)):
        m = b.Y2.shape[0]
        idx = torch.empty((m, 2), dtype=torch.int32, device=DEV)
        val = torch.empty(m, dtype=torch.float64, device=DEV)
        p.bind_2d(b.Y_off, b.Y2.to(DEV), idx, val)
        p.execute()
        np.testing.assert_array_equal(idx.cpu().numpy(), wi)
        assert (np.abs(val.cpu().numpy() - wv) / np.abs(wv)).max() <= REL_TOL


@pytest.mark.parametrize("side", [0, 1])
def test_oneshot_batched_1d(ss, side):
    # the one-call batched form: same answers as the oracle on ragged
    # per-table counts, and with target and output arrays off 16-byte alignment
    b = small_batch(seed=11, ntables=40, scale=0.002)
    want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy(), side)
    got = ss.search_1d_batched(b.X_off, b.X.to(DEV), b.Y_off, b.Y.to(DEV), side=side)
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    # misaligned: drop the first target and shift every table's range by one
    Yd = torch.empty(b.Y.numel() + 1, dtype=torch.float64, device=DEV)
    Yd[1:] = b.Y.to(DEV)
    out = torch.full((b.Y.numel() + 1,), -1, dtype=torch.int32, device=DEV)
    stat = ss.new_stat()
    ss.search_1d_batched(b.X_off, b.X.to(DEV), b.Y_off, Yd[1:], out=out[1:], side=side, stat=stat)
    np.testing.assert_array_equal(out[1:].cpu().numpy(), want)
    assert int(out[0]) == -1
    assert ss.read_stat(stat).flags == 0


def test_oneshot_batched_1d_empty_tables_and_unsorted(ss):
    X = torch.tensor([1.0, 2.0, 3.0, 10.0, 20.0, 30.0, 40.0], dtype=torch.float64)
    Y = torch.tensor([0.5, 2.5, 25.0, 45.0], dtype=torch.float64)
    got = ss.search_1d_batched([0, 3, 7], X.to(DEV), [0, 0, 4], Y.to(DEV))   # table 0 has no targets
    want = oracle.search_1d_batched(np.array([0, 3, 7]), X.numpy(), np.array([0, 0, 4]), Y.numpy())
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    # a table that is not strictly increasing is flagged on the GPU; the
    # other table's indices stay exact and every index stays in range
    bad = torch.tensor([1.0, 2.0, 2.0, 3.0, 1.0, 5.0, 7.0], dtype=torch.float64)
    stat = ss.new_stat()
    got = ss.search_1d_batched([0, 4, 7], bad.to(DEV), [0, 2, 4], Y.to(DEV), stat=stat).cpu().numpy()
    assert ss.read_stat(stat).flags & ss.FLAG_NOT_SORTED
    want = oracle.search_1d(bad.numpy()[4:], Y.numpy()[2:])
    np.testing.assert_array_equal(got[2:], want)
    assert got[:2].min() >= 0 and got[:2].max() <= 3


def test_oneshot_batched_1d_is_stream_ordered(ss):
    """The one-call batched search queues its work on the caller's stream and
    returns: several calls on a side stream, tables staged whole and searched
    in global memory (20,000 and 100,000 entries), read after one
    synchronisation; a capturing stream is refused before anything is queued."""
    bs = [wl.batched_1d(ntables=25 + 10 * i, count_scale=0.003, seed=40 + i) for i in range(3)]
    big = wl.Batched1D(torch.tensor([0, 20_000, 120_000]),
                       torch.cat([wl.log_spaced_table(20_000, 1e-5, 1e5, 0.1, 44),
                                  wl.log_spaced_table(100_000, 1e-3, 1e9, 0.1, 45)]),
                       torch.tensor([0, 50_000, 130_001]),
                       torch.cat([wl.log_uniform(50_000, 5e-6, 2e5, 46), wl.log_uniform(80_001, 5e-4, 2e9, 47)]),
                       None, None)
    bs.append(big)
    s = torch.cuda.Stream()
    ins = [(b.X.to(DEV), b.Y.to(DEV)) for b in bs]
    outs = [torch.full((len(b.Y),), -1, dtype=torch.int32, device=DEV) for b in bs]
    torch.cuda.synchronize()
    for k, b in enumerate(bs):
        ss.search_1d_batched(b.X_off, ins[k][0], b.Y_off, ins[k][1], out=outs[k], side=k & 1, stream=s)
    s.synchronize()
    for k, b in enumerate(bs):
        want = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy(), k & 1)
        np.testing.assert_array_equal(outs[k].cpu().numpy(), want)
    g = torch.cuda.CUDAGraph()
    x = torch.zeros(4, device=DEV)
    codes = []
    with torch.cuda.graph(g):
        try:
            ss.search_1d_batched(bs[0].X_off, ins[0][0], bs[0].Y_off, ins[0][1], out=outs[0])
        except ss.SSError as e:
            codes.append(e.code)
        x.add_(1.0)
    g.replay()
    torch.cuda.synchronize()
    assert codes == [6] and float(x.sum()) == 4.0


def test_oneshot_batched_2d(ss):
    b = wl.batched_2d(ntables=9, pairs_per_table=3001, seed=12)
    wi, wv = oracle.search_interp_2d_batched(b.R_off.numpy(), b.R.numpy(), b.T_off.numpy(), b.T.numpy(),
                                             b.F_off.numpy(), b.F.numpy(), b.Y_off.numpy(), b.Y2.numpy())
    stat = ss.new_stat()
    idx, val = ss.search_interp_2d_batched(b.R_off, b.R.to(DEV), b.T_off, b.T.to(DEV), b.F_off, b.F.to(DEV),
                                           b.Y_off, b.Y2.to(DEV), stat=stat)
    np.testing.assert_array_equal(idx.cpu().numpy(), wi)
    assert (np.abs(val.cpu().numpy() - wv) / np.abs(wv)).max() <= REL_TOL
    assert ss.read_stat(stat).flags == 0


def _oracle_2d(b):
    return oracle.search_interp_2d_batched(b.R_off.numpy(), b.R.numpy(), b.T_off.numpy(), b.T.numpy(),
                                           b.F_off.numpy(), b.F.numpy(), b.Y_off.numpy(), b.Y2.numpy())


def test_oneshot_batched_2d_is_stream_ordered(ss):
    """The one-call batched 2D lookup queues its work on the caller's stream
    and returns: batches on a side stream -- the common case (lean kernel),
    grid values outside the float-float range and an axis with a crowded
    bucket (both handed to the general kernel on the GPU), empty tables and
    arrays off 16-byte alignment -- read after one synchronisation, exact
    against the oracle; an axis that is not increasing is flagged on the GPU;
    a capturing stream is refused before anything is queued."""
    b1 = wl.batched_2d(ntables=7, pairs_per_table=2501, seed=21)
    b2 = wl.batched_2d(ntables=5, pairs_per_table=2003, seed=22)
    F = b2.F.clone()
    nt0 = int(b2.T_off[1] - b2.T_off[0])
    F[3 * nt0:5 * nt0] = 1e-200                      # table 0, rows 3 and 4: below the float-float range
    F[int(b2.F_off[2]) + 7] = 1e250                  # table 2: one value above it
    b2 = wl.Batched2D(b2.R_off, b2.R, b2.T_off, b2.T, b2.F_off, F, b2.Y_off, b2.Y2)
    base = np.geomspace(1e-6, 1e4, 60)
    Rc = np.sort(np.concatenate([base, base[30] * (1 + 1e-9 * np.arange(1, 13))]))
    Tc = wl.log_spaced_table(40, 1e-4, 1e4, 0.1, seed=23).numpy()
    Fc = wl.field_grid(torch.as_tensor(Rc), torch.as_tensor(Tc), wl.smooth_field(1e-6, 1e4, 1e-4, 1e4, seed=24))
    rng = np.random.default_rng(25)
    rho = np.exp(rng.uniform(np.log(0.5e-6), np.log(2e4), 3001))
    rho[::2] = base[30] * (1 + rng.uniform(0, 1.4e-8, len(rho[::2])))
    tem = np.exp(rng.uniform(np.log(0.5e-4), np.log(2e4), 3001))
    b3 = wl.Batched2D(torch.tensor([0, len(Rc)]), torch.as_tensor(Rc), torch.tensor([0, len(Tc)]), torch.as_tensor(Tc),
                      torch.tensor([0, len(Rc) * len(Tc)]), Fc.reshape(-1),
                      torch.tensor([0, 3001]), torch.as_tensor(np.stack([rho, tem], 1)))
    b4 = wl.batched_2d(ntables=4, pairs_per_table=777, seed=26)
    b4 = wl.Batched2D(b4.R_off, b4.R, b4.T_off, b4.T, b4.F_off, b4.F, torch.tensor([0, 0, 777, 777, 1554]),
                      b4.Y2[:1554])                  # tables 0 and 2 without pairs
    bs = [b1, b2, b3, b4]
    s = torch.cuda.Stream()
    ins, outs = [], []
    for k, b in enumerate(bs):
        m = len(b.Y2)
        off = k & 1                                  # odd batches: pairs, indices and values off 16-byte alignment
        y = torch.empty(2 * m + 2, dtype=torch.float64, device=DEV)
        y[off:off + 2 * m] = b.Y2.reshape(-1).to(DEV)
        ib = torch.full((2 * m + 4,), -7, dtype=torch.int32, device=DEV)
        vb = torch.full((m + 2,), -7.0, dtype=torch.float64, device=DEV)
        ins.append((b.R.to(DEV), b.T.to(DEV), b.F.to(DEV), y[off:off + 2 * m]))
        outs.append((ib, vb, off, m))
    stats = [ss.new_stat() for _ in bs]
    torch.cuda.synchronize()
    for k, b in enumerate(bs):
        R, T, F, y = ins[k]
        ib, vb, off, m = outs[k]
        ss.search_interp_2d_batched(b.R_off, R, b.T_off, T, b.F_off, F, b.Y_off, y, idx=ib[2 * off:2 * off + 2 * m],
                                    val=vb[off:off + m], stat=stats[k], stream=s)
    s.synchronize()
    for k, b in enumerate(bs):
        wi, wv = _oracle_2d(b)
        ib, vb, off, m = outs[k]
        np.testing.assert_array_equal(ib[2 * off:2 * off + 2 * m].cpu().numpy().reshape(-1, 2), wi)
        v = vb[off:off + m].cpu().numpy()
        assert (np.abs(v - wv) / np.abs(wv)).max(initial=0.0) <= REL_TOL
        assert torch.all(vb[:off] == -7.0) and torch.all(vb[off + m:] == -7.0)
        assert torch.all(ib[:2 * off] == -7) and torch.all(ib[2 * off + 2 * m:] == -7)
        assert ss.read_stat(stats[k]).flags == 0
    # an axis that is not strictly increasing: flagged, the other table exact
    bad = wl.batched_2d(ntables=2, pairs_per_table=1000, seed=27)
    R = bad.R.clone()
    R[5] = R[4]
    stat = ss.new_stat()
    idx, val = ss.search_interp_2d_batched(bad.R_off, R.to(DEV), bad.T_off, bad.T.to(DEV), bad.F_off, bad.F.to(DEV),
                                           bad.Y_off, bad.Y2.to(DEV), stat=stat)
    assert ss.read_stat(stat).flags & ss.FLAG_NOT_SORTED
    wi, wv = _oracle_2d(bad)
    np.testing.assert_array_equal(idx[1000:].cpu().numpy(), wi[1000:])
    assert (np.abs(val[1000:].cpu().numpy() - wv[1000:]) / np.abs(wv[1000:])).max() <= REL_TOL
    # a capturing stream is refused and the capture stays valid
    g = torch.cuda.CUDAGraph()
    x = torch.zeros(4, device=DEV)
    codes = []
    R, T, F, y = ins[0]
    with torch.cuda.graph(g):
        try:
            ss.search_interp_2d_batched(b1.R_off, R, b1.T_off, T, b1.F_off, F, b1.Y_off, y)
        except ss.SSError as e:
            codes.append(e.code)
        x.add_(1.0)
    g.replay()
    torch.cuda.synchronize()
    assert codes == [6] and float(x.sum()) == 4.0


def test_plan_auto_model_picks_per_bucket(ss):
    """SS_MODEL_AUTO: the tuner picks per table-size bucket among the plain
    searches and the untrained proposals (spline, log hash), timed on the
    bucket's own tables.  Indices are exact for every pick; the 64-entry
    table, staged whole, keeps a plain search, and the 1M-entry table,
    whose plain search finishes with dependent loads in global memory, takes
    a proposal (the log hash measured about twice the plain search there)."""
    tabs = [wl.log_spaced_table(64, 1e-6, 1e4, 0.1, seed=51), wl.log_spaced_table(1 << 20, 1e-6, 1e4, 0.1, seed=52)]
    Ys = [wl.log_uniform(1_500_001, 0.5e-6, 2e4, seed=53), wl.log_uniform(2_000_003, 0.5e-6, 2e4, seed=54)]
    X_off = torch.tensor([0, 64, 64 + (1 << 20)])
    Y_off = torch.tensor([0, len(Ys[0]), len(Ys[0]) + len(Ys[1])])
    X, Y = torch.cat(tabs), torch.cat(Ys)
    want = oracle.search_1d_batched(X_off.numpy(), X.numpy(), Y_off.numpy(), Y.numpy())
    plan = ss.Plan.create_1d(X_off, X.to(DEV), model="auto", autotune=True)
    out = torch.full((len(Y),), -1, dtype=torch.int32, device=DEV)
    stat = ss.new_stat()
    plan.bind_1d(Y_off, Y.to(DEV), out, stat=stat)
    plan.execute()
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    assert ss.read_stat(stat).flags == 0
    picks = sorted(plan.choices().items())
    assert len(picks) == 2, picks
    assert picks[0][1][0] in ("bucket", "binary", "ballot8", "ballot16", "ballot32"), picks
    assert picks[1][1][0] in ("spline", "loghash"), picks
    assert 1 <= plan.info().max_window <= 8
    # without the tuner the model is the plain search
    plain = ss.Plan.create_1d(X_off, X.to(DEV), model="auto")
    assert all(v[0] in ("bucket", "binary") for v in plain.choices().values())

