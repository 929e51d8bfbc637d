"""CPU checks of the seeded input recipes, the synthetic stand-ins for the
paper's SESAME tables: sizes, ranges, strict order, gap jitter, exact-hit
fraction, clustering, count and step distributions match the stated recipe,
and the same seed gives the same inputs."""
import math

import numpy as np
import torch

from paper_2112_03229_gb300 import workloads as wl


def log_quartiles_match(v, lo, hi, atol):
    lv = np.log10(v)
    q = np.quantile(lv, [0.25, 0.5, 0.75])
    want = math.log10(lo) + (math.log10(hi) - math.log10(lo)) * np.array([0.25, 0.5, 0.75])
    return np.allclose(q, want, atol=atol)


def test_plain_1d_recipe():
    X, Y = wl.plain_1d(m=200_000, seed=1)
    x, y = X.numpy(), Y.numpy()
    assert len(x) == 64 and x[0] == 1e-6 and x[-1] == 1e4 and np.all(np.diff(x) > 0)
    pos = (np.log10(x) + 6.0) / (10.0 / 63)          # ideal positions 0..63 in log steps
    assert np.all(np.abs(pos - np.arange(64)) <= 0.1 + 1e-9)   # jitter within +-10 % of a step
    assert abs(np.isin(y, x).mean() - 0.01) < 0.002            # 1 % exact key hits
    assert y.min() >= 0.5e-6 and y.max() <= 2e4
    assert log_quartiles_match(y, 0.5e-6, 2e4, 0.05)          # log-uniform over [0.5 min, 2 max]
    X2, Y2 = wl.plain_1d(m=200_000, seed=1)
    assert torch.equal(X, X2) and torch.equal(Y, Y2)
    assert not torch.equal(Y, wl.plain_1d(m=200_000, seed=2)[1])


def test_interp_2d_recipe():
    R, T, F, Y2 = wl.interp_2d(m=100_000, seed=2)
    r, t, f, y = R.numpy(), T.numpy(), F.numpy(), Y2.numpy()
    assert r.shape == (200,) and t.shape == (100,) and f.shape == (200, 100) and y.shape == (100_000, 2)
    assert r[0] == 1e-6 and r[-1] == 1e4 and t[0] == 1e-4 and t[-1] == 1e4
    assert np.all(np.diff(r) > 0) and np.all(np.diff(t) > 0)
    assert f.min() >= 1.0 and f.max() <= 1.0 + 8 * 2.0       # 1 + eight Gaussians of height <= 2
    assert y[:, 0].min() >= 1e-6 and y[:, 0].max() <= 1e4 and y[:, 1].min() >= 1e-4 and y[:, 1].max() <= 1e4
    assert log_quartiles_match(y[:, 0], 1e-6, 1e4, 0.05) and log_quartiles_match(y[:, 1], 1e-4, 1e4, 0.05)


def test_sweep_tables_are_clustered():
    for n in (16, 256, 4096, 65536):
        x = wl.sweep_table(n).numpy()
        assert len(x) == n and x[0] == 1e-6 and x[-1] == 1e4 and np.all(np.diff(x) > 0)
    # the windows hold 8x the key density of the rest: with 64 bins of log
    # range, a bin inside a window holds 8x the keys of a bin outside
    x = wl.sweep_table(65536).numpy()
    counts = np.histogram((np.log10(x) + 6.0) / 10.0, bins=64, range=(0.0, 1.0))[0]
    assert 7.5 <= counts.max() / counts.min() <= 8.5


def test_zipf_counts_follow_the_truncated_law():
    lo, hi, a = 1000, 1_000_000, 1.1
    k = np.arange(lo, hi + 1, dtype=np.float64)
    p = k ** -a
    p /= p.sum()
    mean, sd = (k * p).sum(), math.sqrt(((k - (k * p).sum()) ** 2 * p).sum())
    c = wl.zipf_counts(400_000, a, lo, hi, np.random.default_rng(3))
    assert c.min() >= lo and c.max() <= hi
    assert abs(c.mean() - mean) < 4 * sd / math.sqrt(len(c))
    assert abs((c == lo).mean() - p[0]) < 4 * math.sqrt(p[0] * (1 - p[0]) / len(c))
    assert 105_000 < mean < 118_000          # about 1.1B targets over 10,000 tables


def test_batched_1d_recipe():
    b = wl.batched_1d(ntables=400, seed=5, count_scale=0.005)
    sizes, counts = np.diff(b.X_off.numpy()), np.diff(b.Y_off.numpy())
    assert sizes.min() >= 20 and sizes.max() <= 2000
    assert 150 <= np.median(sizes) <= 270                     # log-uniform on [20, 2000]: median near 200
    lo, hi = b.lo, b.hi
    assert np.all(lo >= 1e-8) and np.all(lo <= 1e-2)
    span = np.log10(hi / lo)
    assert np.all(span >= 4 - 1e-9) and np.all(span <= 12 + 1e-9)
    X, Y, Xo, Yo = b.X.numpy(), b.Y.numpy(), b.X_off.numpy(), b.Y_off.numpy()
    for k in range(0, 400, 13):
        x, y = X[Xo[k]:Xo[k + 1]], Y[Yo[k]:Yo[k + 1]]
        assert x[0] == lo[k] and x[-1] == hi[k] and np.all(np.diff(x) > 0)
        assert np.all(y >= 0.5 * lo[k] * (1 - 1e-12)) and np.all(y <= 2 * hi[k] * (1 + 1e-12))
    b2 = wl.batched_1d(ntables=400, seed=5, count_scale=0.005)
    assert torch.equal(b.X, b2.X) and torch.equal(b.Y, b2.Y)
    # a prefix of the same batch: the first tables keep their targets
    b3 = wl.batched_1d(ntables=400, seed=5, count_scale=0.005, max_targets=int(counts[:10].sum()))
    assert np.array_equal(np.diff(b3.Y_off.numpy())[:10], counts[:10]) and b3.Y_off[-1] == counts[:10].sum()


def test_batched_2d_recipe_random_and_coherent():
    for coherent in (False, True):
        b = wl.batched_2d(ntables=12, pairs_per_table=20_000, coherent=coherent, seed=6)
        nr, nt = np.diff(b.R_off.numpy()), np.diff(b.T_off.numpy())
        assert nr.min() >= 50 and nr.max() <= 500 and nt.min() >= 30 and nt.max() <= 300
        assert np.array_equal(np.diff(b.F_off.numpy()), nr * nt)
        assert np.all(b.F.numpy() >= 1.0)
        R, T, Y = b.R.numpy(), b.T.numpy(), b.Y2.numpy()
        Ro, To = b.R_off.numpy(), b.T_off.numpy()
        steps = []
        for k in range(12):
            r, t = R[Ro[k]:Ro[k + 1]], T[To[k]:To[k + 1]]
            y = Y[20_000 * k:20_000 * (k + 1)]
            assert np.all(np.diff(r) > 0) and np.all(np.diff(t) > 0)
            assert np.all(y[:, 0] >= r[0]) and np.all(y[:, 0] <= r[-1])
            assert np.all(y[:, 1] >= t[0]) and np.all(y[:, 1] <= t[-1])
            span_r, span_t = math.log10(r[-1] / r[0]), math.log10(t[-1] / t[0])
            assert 9 - 1e-9 <= span_r <= 11 + 1e-9 and 7 - 1e-9 <= span_t <= 9 + 1e-9
            steps.append(np.diff(np.log10(y), axis=0).ravel())
        s = np.concatenate(steps)
        if coherent:
            # a random walk of N(0, 0.01 decade) steps, reflected at the bounds (rarely)
            assert 0.0095 < np.std(s) < 0.0105
        else:
            assert np.std(s) > 1.0


def test_walk_1d_steps_and_jumps():
    lo, hi = 1e-6, 1e4
    y = wl.walk_1d(200_000, lo, hi, seed=3)
    assert torch.all((y >= lo) & (y <= hi))
    d = torch.diff(torch.log10(y))
    # N(0, 0.01 decade) steps (reflection only shortens a step)
    assert 0.0095 < float(d.std()) < 0.0105 and float(d.abs().max()) < 0.07
    y2 = wl.walk_1d(200_000, lo, hi, seed=3, jump=0.01)
    d2 = torch.diff(torch.log10(y2)).abs()
    big = int((d2 > 1.0).sum())                  # leaps of more than a decade
    assert 1000 < big < 2000 and float(d2.max()) > 5.0
    # the same seed without jumps is the plain walk, draw for draw
    assert torch.equal(wl.walk_1d(200_000, lo, hi, seed=3, jump=0.0), y)
