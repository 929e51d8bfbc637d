"""Pins of the CPU oracle against facts that do not come from the oracle
itself: brute-force counts on tiny tables, an independent bisection written
from the branchless-binary description of Sec. 3.2, IEEE special values,
invariants, the worked numbers of Sec. 5.2 / 5.5, closed forms of bilinear
interpolation, finite differences for the model gradient.

Each test is chosen so that a plausible slip in the oracle (a flipped
comparison, a dropped clamp, a wrong cell, a transposed grid, a missing
gradient term) fails at least one of them.
"""
import math
import os
import struct

import numpy as np
import pytest

import oracle
from paper_2112_03229_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (s.strip() for s in line.split("="))
                vals[k] = float(v)
    return vals


def special_targets(X):
    """Every entry, both neighbours in ulps, midpoints, and IEEE specials."""
    X = np.asarray(X, dtype=np.float64)
    t = [X, np.nextafter(X, -np.inf), np.nextafter(X, np.inf), (X[1:] + X[:-1]) / 2]
    t.append(np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, 5e-324, -5e-324,
                       2.2250738585072014e-308, X[0] / 2, X[-1] * 2, -X[-1], 1e300, -1e300]))
    return np.concatenate(t)


def brute(X, t, side):
    """max(0, #{X[j] below t} - 1) by a linear count (the Sec. 3 definition)."""
    out = np.empty(t.shape[0], dtype=np.int32)
    for i, y in enumerate(t):
        c = sum(1 for x in X if (x <= y if side else x < y))
        out[i] = max(0, c - 1)
    return out


def tiny_tables():
    rng = np.random.default_rng(7)
    tabs = []
    for n in (2, 3, 4, 5, 7, 8, 9, 16, 31, 32, 33, 63, 64):
        tabs.append(np.sort(rng.choice(np.arange(-1000, 1000), n, replace=False)).astype(np.float64) / 8)
        tabs.append(wl.log_spaced_table(n, 1e-6, 1e4, 0.1, seed=n).numpy())
    tabs.append(np.array([-np.inf, 0.0, np.inf]))
    tabs.append(np.array([-5e-324, 0.0, 5e-324, 1e-300]))
    tabs.append(np.array([-1.0, -0.0 + 0.0, 1.0]))
    return tabs


@pytest.mark.parametrize("side", [0, 1])
def test_search_1d_brute_force(side):
    for X in tiny_tables():
        t = special_targets(X[np.isfinite(X)] if np.isfinite(X).sum() >= 2 else X)
        got = oracle.search_1d(X, t, side=side)
        np.testing.assert_array_equal(got, brute(X, t, side), err_msg=f"n={len(X)} side={side}")


def bisection_le(X, y):
    """Branchless-binary search of Sec. 3.2 in my own words: keep
    X[lo] <= y < X[hi] while the bracket is wider than one, then apply the two
    end clamps.  Its result is the "<=" (Sec. 3) form of the answer."""
    n = len(X)
    lo, hi = 0, n
    while hi - lo > 1:
        mid = (lo + hi) // 2
        go_left = y < X[mid]
        hi = mid if go_left else hi
        lo = lo if go_left else mid
    if y < X[0]:
        lo = 0
    if y > X[n - 1]:
        lo = n - 1
    return lo


def test_le_side_matches_sec32_bisection():
    for X in tiny_tables():
        if not np.all(np.isfinite(X)):
            continue
        t = special_targets(X)
        t = t[~np.isnan(t)]          # the printed bisection has no NaN rule
        want = np.array([bisection_le(X, y) for y in t], dtype=np.int32)
        np.testing.assert_array_equal(oracle.search_1d(X, t, side=1), want)


def test_interval_invariant_and_monotone():
    X, Y = wl.plain_1d(m=200_000, seed=11)
    X, Y = X.numpy(), Y.numpy()
    n = len(X)
    idx = oracle.search_1d(X, Y)
    assert idx.min() >= 0 and idx.max() <= n - 1
    ok = ((idx == 0) | (X[idx] < Y)) & ((idx == n - 1) | (Y <= X[np.minimum(idx + 1, n - 1)]))
    assert ok.all()
    order = np.argsort(Y, kind="stable")
    assert np.all(np.diff(idx[order]) >= 0)
    # exact key hits go to the lower interval under "<": X[j] -> j-1 (j >= 1)
    np.testing.assert_array_equal(oracle.search_1d(X, X[1:]), np.arange(n - 1))
    np.testing.assert_array_equal(oracle.search_1d(X, X[:-1], side=1), np.arange(n - 1))


def test_special_values():
    X = np.array([1e-6, 1e-3, 1.0, 1e3])
    got = oracle.search_1d(X, [np.nan, -np.inf, np.inf, -0.0, 0.0, 5e-324, 1e-6, 1e3, 2e3])
    np.testing.assert_array_equal(got, [0, 0, 3, 0, 0, 0, 0, 2, 3])
    Xz = np.array([-1.0, 0.0, 1.0])
    assert oracle.search_1d(Xz, [-0.0])[0] == oracle.search_1d(Xz, [0.0])[0] == 0
    assert oracle.search_1d(Xz, [-0.0], side=1)[0] == oracle.search_1d(Xz, [0.0], side=1)[0] == 1


def test_paper_worked_numbers_exponent_hash():
    g = golden("paper_sec5_worked_numbers.txt")
    n = int(g["table_entries"])
    X = wl.log_spaced_table(n, g["table_min"], g["table_max"], 0.1, seed=3).numpy()
    base, L = oracle.bucket_directory(X, 52)
    B = len(L) - 1
    # number of powers of two spanned (Sec. 5.2): about 34
    assert abs(B - g["powers_of_two"]) <= 1
    assert abs(n / B - g["entries_per_bin"]) < 0.15
    # buckets at shift 52 are exactly the IEEE exponents (frexp is independent of the oracle)
    exps = np.array([math.frexp(x)[1] for x in X])
    assert B == exps.max() - exps.min() + 1
    occupied = np.count_nonzero(np.diff(L))
    assert occupied == len(np.unique(exps))
    # count form of the directory: entry j lies in [L[b_j], L[b_j + 1])
    for j, e in enumerate(exps):
        b = e - exps.min()
        assert L[b] <= j < L[b + 1]
    assert L[0] == 0 and L[-1] == n and np.all(np.diff(L) >= 0)


def test_paper_targets_half_out_of_range():
    g = golden("paper_sec5_worked_numbers.txt")
    X, Y = wl.paper_workload(m=200_000)
    Y = Y.numpy()
    out = np.mean((Y < X[0].item()) | (Y > X[-1].item()))
    assert abs(out - g["out_of_range_fraction"]) < 0.05


def _bits_key(x):
    """Order-preserving image via struct, written independently of the oracle."""
    if x == 0.0:
        x = 0.0
    u = struct.unpack("<Q", struct.pack("<d", x))[0]
    return (1 << 64) - u if u >> 63 else u | (1 << 63)


def test_order_key_preserves_order():
    rng = np.random.default_rng(5)
    vals = list(rng.standard_normal(200) * 10.0 ** rng.integers(-300, 300, 200))
    vals += [0.0, -0.0, 5e-324, -5e-324, np.inf, -np.inf, 1.0, -1.0, 2.2250738585072014e-308]
    keys = [oracle.order_key(v) for v in vals]
    for v, k in zip(vals, keys):
        assert k == _bits_key(v)
    for a, ka in zip(vals, keys):
        for b, kb in zip(vals, keys):
            assert (a < b) == (ka < kb)
    assert oracle.order_key(-0.0) == oracle.order_key(0.0)


def test_bucket_shift_and_directory_invariants():
    for n in (2, 64, 110, 2000):
        X = wl.log_spaced_table(n, 1e-8, 1e6, 0.1, seed=n).numpy()
        for cap in (2, 64, 1024, 1 << 16):
            s = oracle.bucket_shift(X, cap)
            base, L = oracle.bucket_directory(X, s)
            assert len(L) - 1 <= cap
            if s > 0:   # one bit finer would not fit
                k0, k1 = _bits_key(X[0]), _bits_key(X[-1])
                assert (k1 >> (s - 1)) - (k0 >> (s - 1)) + 1 > cap
            for j, x in enumerate(X):
                b = (_bits_key(x) >> s) - base
                assert L[b] <= j < L[b + 1]


def test_bucket_directory_wide_key_span():
    # a table from -1e300 to 1e300 covers most of the 64-bit key range
    X = np.array([-1e300, -1.0, -5e-324, 0.0, 5e-324, 1.0, 1e300])
    for cap in (2, 3, 64, 112, 4096):
        s = oracle.bucket_shift(X, cap)
        base, L = oracle.bucket_directory(X, s, cap=cap + 1)
        assert 1 <= len(L) - 1 <= cap
        k0, k1 = _bits_key(X[0]), _bits_key(X[-1])
        assert (k1 >> s) - (k0 >> s) + 1 == len(L) - 1
        for j, x in enumerate(X):
            b = (_bits_key(x) >> s) - base
            assert L[b] <= j < L[b + 1]


def test_spline_knots_closed_form():
    # entries exact powers of two: with K = n-1 segments, knot j (j >= 1) sits
    # one step above 2^j in the image, so j+1 entries lie below it
    n = 20
    X = 2.0 ** np.arange(n)
    delta, counts = oracle.spline_knots(X, n - 1)
    assert delta == (1 << 52) + 1
    np.testing.assert_array_equal(counts, np.concatenate([[0], np.arange(2, n + 1)]))
    X = wl.clustered_table(4096, 1e-6, 1e4, seed=9).numpy()
    delta, counts = oracle.spline_knots(X, 256)
    assert counts[0] == 0 and counts[-1] == len(X) and np.all(np.diff(counts) >= 0)


# ---------------------------------------------------------------- 2D lookup

def test_interp_affine_reproduced():
    R = wl.log_spaced_table(40, 1e-3, 1e3, 0.1, seed=1).numpy()
    T = wl.log_spaced_table(25, 1e-2, 1e2, 0.1, seed=2).numpy()
    a, b, c, d = 3.0, 0.25, 1.5, 0.125
    F = a + b * R[:, None] + c * T[None, :] + d * R[:, None] * T[None, :]
    Y = wl.pairs_log_uniform(20_000, R[0], R[-1], T[0], T[-1], seed=3).numpy()
    idx, val = oracle.search_interp_2d(R, T, F, Y)
    want = a + b * Y[:, 0] + c * Y[:, 1] + d * Y[:, 0] * Y[:, 1]
    np.testing.assert_allclose(val, want, rtol=1e-13, atol=0)
    np.testing.assert_array_equal(idx[:, 0], oracle.search_1d(R, Y[:, 0]))
    np.testing.assert_array_equal(idx[:, 1], oracle.search_1d(T, Y[:, 1]))


def test_interp_nodes_bounds_and_clamp():
    R = np.array([1.0, 2.0, 5.0, 10.0])
    T = np.array([0.1, 1.0, 3.0])
    F = np.arange(12, dtype=np.float64).reshape(4, 3) ** 2 + 1.0
    nodes = np.array([[r, t] for r in R for t in T])
    _, v = oracle.search_interp_2d(R, T, F, nodes)
    np.testing.assert_array_equal(v, F.reshape(-1))            # exact at nodes, row-major grid
    rng = np.random.default_rng(1)
    Y = np.stack([rng.uniform(0.5, 12, 5000), rng.uniform(0.05, 4, 5000)], 1)
    idx, v = oracle.search_interp_2d(R, T, F, Y)
    cr = np.minimum(idx[:, 0], 2)
    ct = np.minimum(idx[:, 1], 1)
    corners = np.stack([F[cr, ct], F[cr, ct + 1], F[cr + 1, ct], F[cr + 1, ct + 1]], 1)
    assert np.all(v >= corners.min(1) * (1 - 1e-15)) and np.all(v <= corners.max(1) * (1 + 1e-15))
    # constant extrapolation outside the grid: equals the value at the clamped
    # point.  The axes and grid sit at the front of NaN-filled buffers, so a
    # cell index one past the last cell would read NaN and show up here.
    padR = np.full(8, np.nan); padR[:4] = R
    padT = np.full(8, np.nan); padT[:3] = T
    padF = np.full(40, np.nan); padF[:12] = F.reshape(-1)
    Yc = np.stack([np.clip(Y[:, 0], R[0], R[-1]), np.clip(Y[:, 1], T[0], T[-1])], 1)
    L = oracle.lib()
    vo = np.empty(len(Y)); io = np.empty(2 * len(Y), dtype=np.int32)
    Yf = np.ascontiguousarray(Y.reshape(-1))
    L.oracle_search_interp_2d(oracle._p(padR, oracle._f64p), 4, oracle._p(padT, oracle._f64p), 3,
                              oracle._p(padF, oracle._f64p), oracle._p(Yf, oracle._f64p), len(Y),
                              oracle._p(io, oracle._i32p), oracle._p(vo, oracle._f64p))
    _, vc = oracle.search_interp_2d(R, T, F, Yc)
    assert not np.isnan(vo).any()
    np.testing.assert_allclose(vo, vc, rtol=1e-15)
    np.testing.assert_allclose(v, vc, rtol=1e-15)
    # separable 1D check along an edge: linear interpolation in rho at T = T[0]
    rr = np.linspace(1.0, 10.0, 101)
    _, ve = oracle.search_interp_2d(R, T, F, np.stack([rr, np.full_like(rr, T[0])], 1))
    np.testing.assert_allclose(ve, np.interp(rr, R, F[:, 0]), rtol=1e-14)
    # NaN in either coordinate: index 0, value NaN
    idx, v = oracle.search_interp_2d(R, T, F, np.array([[np.nan, 1.0], [2.0, np.nan]]))
    assert np.all(np.isnan(v)) and idx[0, 0] == 0 and idx[1, 1] == 0


def test_interp_linear_extrapolation_reproduces_affine():
    """Reading R6, extrap=1: without the clamp, bilinear interpolation on the
    edge cell continues the affine field a + b rho + c T + d rho T exactly
    beyond the grid; inside the grid nothing changes."""
    R = wl.log_spaced_table(30, 1e-3, 1e3, 0.1, seed=11).numpy()
    T = wl.log_spaced_table(20, 1e-2, 1e2, 0.1, seed=12).numpy()
    a, b, c, d = 3.0, 0.25, 1.5, 0.125
    F = a + b * R[:, None] + c * T[None, :] + d * R[:, None] * T[None, :]
    Y = wl.pairs_log_uniform(20_000, R[0] / 4, R[-1] * 4, T[0] / 4, T[-1] * 4, seed=13).numpy()
    idx, val = oracle.search_interp_2d(R, T, F, Y, extrap=1)
    want = a + b * Y[:, 0] + c * Y[:, 1] + d * Y[:, 0] * Y[:, 1]
    scale = abs(a) + abs(b * Y[:, 0]) + abs(c * Y[:, 1]) + abs(d * Y[:, 0] * Y[:, 1])
    assert (np.abs(val - want) <= 1e-12 * scale).all()
    outside = (Y[:, 0] < R[0]) | (Y[:, 0] > R[-1]) | (Y[:, 1] < T[0]) | (Y[:, 1] > T[-1])
    assert outside.sum() > 5000
    _, clamped = oracle.search_interp_2d(R, T, F, Y)
    np.testing.assert_array_equal(val[~outside], clamped[~outside])
    assert (np.abs(clamped[outside] - want[outside]) > 1e-6 * scale[outside]).any()
    np.testing.assert_array_equal(idx, oracle.search_interp_2d(R, T, F, Y)[0])


def test_interp_log_space_reproduces_log_affine():
    """Reading R6, logspace=1: weights in log coordinates reproduce a field
    that is bilinear in (ln rho, ln T); nodes are exact; outside the grid the
    clamp gives the edge value and extrap=1 continues the field."""
    R = wl.log_spaced_table(30, 1e-3, 1e3, 0.1, seed=14).numpy()
    T = wl.log_spaced_table(20, 1e-2, 1e2, 0.1, seed=15).numpy()
    a, b, c, d = 30.0, 0.5, -1.25, 0.2
    lr, lt = np.log(R), np.log(T)
    F = a + b * lr[:, None] + c * lt[None, :] + d * lr[:, None] * lt[None, :]
    Y = wl.pairs_log_uniform(20_000, R[0], R[-1], T[0], T[-1], seed=16).numpy()
    _, val = oracle.search_interp_2d(R, T, F, Y, logspace=1)
    ly0, ly1 = np.log(Y[:, 0]), np.log(Y[:, 1])
    want = a + b * ly0 + c * ly1 + d * ly0 * ly1
    scale = abs(a) + abs(b * ly0) + abs(c * ly1) + abs(d * ly0 * ly1)
    assert (np.abs(val - want) <= 1e-12 * scale).all()
    _, lin = oracle.search_interp_2d(R, T, F, Y)
    assert (np.abs(lin - want) > 1e-4 * scale).any()          # linear weights do not reproduce it
    nodes = np.array([[r, t] for r in R for t in T])
    np.testing.assert_array_equal(oracle.search_interp_2d(R, T, F, nodes, logspace=1)[1], F.reshape(-1))
    Yo = wl.pairs_log_uniform(5_000, R[0] / 10, R[-1] * 10, T[0] / 10, T[-1] * 10, seed=17).numpy()
    _, ext = oracle.search_interp_2d(R, T, F, Yo, extrap=1, logspace=1)
    ly0, ly1 = np.log(Yo[:, 0]), np.log(Yo[:, 1])
    want = a + b * ly0 + c * ly1 + d * ly0 * ly1
    scale = abs(a) + abs(b * ly0) + abs(c * ly1) + abs(d * ly0 * ly1)
    assert (np.abs(ext - want) <= 1e-12 * scale).all()
    Yc = np.stack([np.clip(Yo[:, 0], R[0], R[-1]), np.clip(Yo[:, 1], T[0], T[-1])], 1)
    np.testing.assert_allclose(oracle.search_interp_2d(R, T, F, Yo, logspace=1)[1],
                               oracle.search_interp_2d(R, T, F, Yc, logspace=1)[1], rtol=1e-15)


def test_batched_equals_per_table():
    b = wl.batched_1d(ntables=12, count_scale=0.002, seed=3)
    got = oracle.search_1d_batched(b.X_off.numpy(), b.X.numpy(), b.Y_off.numpy(), b.Y.numpy())
    for k in range(12):
        x = b.X[b.X_off[k]:b.X_off[k + 1]].numpy()
        y = b.Y[b.Y_off[k]:b.Y_off[k + 1]].numpy()
        np.testing.assert_array_equal(got[b.Y_off[k]:b.Y_off[k + 1]], brute(x, y, 0) if len(y) < 3000 else oracle.search_1d(x, y))


def test_batched_2d_equals_per_table():
    # every table of a 2D batch is looked up exactly as on its own (whose
    # values the closed-form pins above fix), options included
    b = wl.batched_2d(ntables=5, pairs_per_table=300, seed=4)
    Ro, To, Fo, Yo = (o.numpy() for o in (b.R_off, b.T_off, b.F_off, b.Y_off))
    R, T, F, Y2 = b.R.numpy(), b.T.numpy(), b.F.numpy(), b.Y2.numpy()
    for extrap, logspace in ((0, 0), (1, 0), (0, 1)):
        gi, gv = oracle.search_interp_2d_batched(Ro, R, To, T, Fo, F, Yo, Y2, extrap=extrap, logspace=logspace)
        for k in range(5):
            wi, wv = oracle.search_interp_2d(R[Ro[k]:Ro[k + 1]], T[To[k]:To[k + 1]], F[Fo[k]:Fo[k + 1]],
                                             Y2[Yo[k]:Yo[k + 1]], extrap=extrap, logspace=logspace)
            np.testing.assert_array_equal(gi[Yo[k]:Yo[k + 1]], wi)
            np.testing.assert_array_equal(gv[Yo[k]:Yo[k + 1]], wv)


def test_sampled_forms_equal_the_full_forms():
    rng = np.random.default_rng(8)
    X, Y = (t.numpy() for t in wl.plain_1d(m=5000, seed=6))
    sample = rng.choice(len(Y), 300, replace=False).astype(np.int64)
    for side in (0, 1):
        np.testing.assert_array_equal(oracle.search_1d_sampled(X, Y, sample, side), oracle.search_1d(X, Y, side)[sample])
    R, T, F, Y2 = (t.numpy() for t in wl.interp_2d(m=4000, seed=7))
    si, sv = oracle.search_interp_2d_sampled(R, T, F, Y2, sample[sample < 4000])
    fi, fv = oracle.search_interp_2d(R, T, F, Y2)
    np.testing.assert_array_equal(si, fi[sample[sample < 4000]])
    np.testing.assert_array_equal(sv, fv[sample[sample < 4000]])


# ---------------------------------------------------------------- position model

def test_mlp_features_closed_form():
    x0, x1 = oracle.mlp_features(1.5 * 2.0 ** -7, e_lo=-10.0, e_scale=0.5)
    assert x0 == (-7 + 10) * 0.5 and x1 == 0.5
    x0, x1 = oracle.mlp_features(1.0, 0.0, 1.0)
    assert x0 == 0.0 and x1 == 0.0


def test_mlp_gradient_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(65) * 0.5
    x = rng.uniform(0, 1, (256, 2))
    y = rng.uniform(0, 1, 256)
    loss, g = oracle.mlp_loss_grad(p, x, y)
    eps = 1e-6
    for k in range(65):
        q = p.copy(); q[k] += eps
        lp, _ = oracle.mlp_loss_grad(q, x, y)
        q[k] -= 2 * eps
        lm, _ = oracle.mlp_loss_grad(q, x, y)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), k
    # closed form: only the output bias is non-zero -> y = b2, dL/db2 = 2 mean(b2 - t)
    q = np.zeros(65); q[64] = 0.3
    loss, g = oracle.mlp_loss_grad(q, x, y)
    assert math.isclose(loss, np.mean((0.3 - y) ** 2), rel_tol=1e-14)
    assert math.isclose(g[64], 2 * np.mean(0.3 - y), rel_tol=1e-12)
    assert np.all(g[:64] == 0)


def test_adam_first_step_closed_form():
    p = np.linspace(-1, 1, 65)
    g = np.where(np.arange(65) % 2 == 0, 0.5, -2.0)
    m1, m2 = np.zeros(65), np.zeros(65)
    p0 = p.copy()
    oracle.adam_step(p, g, m1, m2, 1, lr=1e-2, eps=0.0)
    # bias-corrected first step moves every parameter by lr against the gradient sign
    np.testing.assert_allclose(p - p0, -1e-2 * np.sign(g), rtol=1e-12)
