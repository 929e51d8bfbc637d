"""GPU parity of the one-shot 1D search and 2D lookup against the CPU oracle.

Indices must match bit for bit; interpolated values within 1e-12 relative.
All calls go through the C ABI (ctypes binding).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_03229_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12     # interpolated values, relative to the fp64 oracle


@pytest.fixture(scope="module")
def ss():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_03229_gb300 as m
    return m


DEV = "cuda"
VARIANTS = [("bucket", 0), ("binary", 0), ("branchy", 0), ("ballot", 8), ("ballot", 16), ("ballot", 32)]


def special_targets(X):
    X = np.asarray(X, dtype=np.float64)
    t = [X, np.nextafter(X, -np.inf), np.nextafter(X, np.inf), (X[1:] + X[:-1]) / 2]
    t.append(np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, 5e-324, -5e-324, 2.2250738585072014e-308,
                       X[0] / 2, X[-1] * 2, -X[-1], 1e300, -1e300, 1.0, -1.0]))
    return np.concatenate(t)


def run1d(ss, X, Y, side=0, algo="bucket", g=0, **kw):
    Xd = torch.as_tensor(X, dtype=torch.float64).to(DEV)
    Yd = torch.as_tensor(Y, dtype=torch.float64).to(DEV)
    return ss.search_1d(Xd, Yd, side=side, algo=algo, ballot_g=g, **kw).cpu().numpy()


@pytest.mark.parametrize("algo,g", VARIANTS)
@pytest.mark.parametrize("side", [0, 1])
def test_1d_sizes_and_specials(ss, algo, g, side):
    rng = np.random.default_rng(3)
    for n in (2, 3, 4, 31, 32, 33, 63, 64, 65, 110, 257, 1000):
        X = wl.log_spaced_table(n, 1e-6, 1e4, 0.1, seed=n).numpy()
        Y = np.concatenate([special_targets(X), 10 ** rng.uniform(-7, 5, 5000)])
        np.testing.assert_array_equal(run1d(ss, X, Y, side, algo, g), oracle.search_1d(X, Y, side),
                                      err_msg=f"{algo}/{g} n={n} side={side}")
    # tables with negatives, zero and subnormals
    for X in (np.array([-1e300, -1.0, -5e-324, 0.0, 5e-324, 1.0, 1e300]), np.array([-np.inf, 0.0, np.inf]),
              np.sort(rng.standard_normal(500) * 10.0 ** rng.integers(-200, 200, 500))):
        X = np.unique(X)
        Y = special_targets(X[np.isfinite(X)])
        np.testing.assert_array_equal(run1d(ss, X, Y, side, algo, g), oracle.search_1d(X, Y, side))


@pytest.mark.parametrize("algo,g", VARIANTS)
def test_1d_config0_full(ss, algo, g):
    # one table of 64 entries, 1M targets with 1% exact key hits (ragged m)
    X, Y = wl.plain_1d(m=(1 << 20) + 3, seed=1)
    np.testing.assert_array_equal(run1d(ss, X.numpy(), Y.numpy(), 0, algo, g), oracle.search_1d(X.numpy(), Y.numpy()))


@pytest.mark.parametrize("algo,g", [("bucket", 0), ("binary", 0), ("ballot", 32)])
def test_1d_ragged_and_misaligned(ss, algo, g):
    X, Y = wl.plain_1d(m=4099, seed=5)
    Xd, Yd = X.to(DEV), Y.to(DEV)
    want = oracle.search_1d(X.numpy(), Y.numpy())
    for m in (0, 1, 2, 3, 4, 5, 7, 8, 9, 4098):
        for yoff in (0, 1):
            for ooff in (0, 1, 2, 3):
                out = torch.full((m + 8,), -7, dtype=torch.int32, device=DEV)
                ys = Yd[yoff:yoff + m]
                ss.search_1d(Xd, ys, out=out[ooff:ooff + m], algo=algo, ballot_g=g)
                o = out.cpu().numpy()
                np.testing.assert_array_equal(o[ooff:ooff + m], want[yoff:yoff + m])
                assert np.all(o[:ooff] == -7) and np.all(o[ooff + m:] == -7)   # nothing written outside


@pytest.mark.parametrize("algo", ["binary", "bucket", "branchy"])
def test_1d_two_level_large_tables(ss, algo):
    # n-1 above the staged limit: sampled top level in shared memory, leaves in global memory
    for n in (8129, 8193, 20000, 65536):
        X = wl.sweep_table(n).numpy() if n == 65536 else wl.log_spaced_table(n, 1e-6, 1e4, 0.1, seed=n).numpy()
        Y = np.concatenate([special_targets(X[:2000]), special_targets(X[-2000:]),
                            10 ** np.random.default_rng(n).uniform(-7, 5, 200_000)])
        np.testing.assert_array_equal(run1d(ss, X, Y, 0, algo), oracle.search_1d(X, Y), err_msg=f"n={n}")


def test_1d_status_nan_and_unsorted(ss):
    X = wl.log_spaced_table(64, 1e-6, 1e4, 0.1, seed=1)
    Y = wl.log_uniform(10_000, 1e-7, 1e5, seed=2)
    Y[::100] = float("nan")
    Y[1::100] = -float("nan")
    stat = ss.new_stat()
    out = ss.search_1d(X.to(DEV), Y.to(DEV), stat=stat)
    st = ss.read_stat(stat)
    assert st.nan_targets == 200 and st.flags == 0
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.search_1d(X.numpy(), Y.numpy()))
    Xbad = X.clone()
    Xbad[10] = Xbad[9]
    stat = ss.new_stat()
    out = ss.search_1d(Xbad.to(DEV), Y.to(DEV), stat=stat)
    st = ss.read_stat(stat)
    assert st.flags & ss.FLAG_NOT_SORTED
    o = out.cpu().numpy()
    assert o.min() >= 0 and o.max() <= 63     # unspecified but in range


def test_1d_argument_errors(ss):
    X = torch.linspace(1, 2, 8, dtype=torch.float64, device=DEV)
    Y = torch.ones(4, dtype=torch.float64, device=DEV)
    with pytest.raises(ss.SSError):
        ss.search_1d(X[:1], Y)
    with pytest.raises(ss.SSError):
        ss.search_1d(X, Y, algo=9)


# ---------------------------------------------------------------- 2D lookup

def check_2d(idx, val, wi, wv):
    np.testing.assert_array_equal(idx, wi)
    nan = np.isnan(wv)
    assert np.array_equal(np.isnan(val), nan)
    rel = np.abs(val[~nan] - wv[~nan]) / np.abs(wv[~nan])
    assert rel.max(initial=0.0) <= REL_TOL, rel.max()


@pytest.mark.parametrize("algo,fp64", [("bucket", False), ("binary", False), ("bucket", True), ("binary", True)])
def test_2d_config1_small(ss, algo, fp64):
    R, T, F, Y2 = wl.interp_2d(m=(1 << 20) + 1, seed=2)
    # add out-of-range, exact-node and NaN pairs
    extra = np.array([[R[0].item(), T[0].item()], [R[-1].item(), T[-1].item()], [1e-9, 1e9], [1e9, 1e-9],
                      [np.nan, 1.0], [1.0, np.nan], [-0.0, 0.0], [np.inf, -np.inf], [R[5].item(), T[7].item()]])
    Y2 = torch.cat([Y2, torch.as_tensor(extra)])
    stat = ss.new_stat()
    idx, val = ss.search_interp_2d(R.to(DEV), T.to(DEV), F.to(DEV), Y2.to(DEV), algo=algo, fp64=fp64, stat=stat)
    wi, wv = oracle.search_interp_2d(R.numpy(), T.numpy(), F.numpy(), Y2.numpy())
    check_2d(idx.cpu().numpy(), val.cpu().numpy(), wi, wv)
    st = ss.read_stat(stat)
    assert st.flags == 0 and st.nan_targets == 2


def test_2d_float_float_preconditions(ss):
    """Axes or grids outside the float-float path's range fall back to fp64 and stay exact."""
    rng = np.random.default_rng(4)
    cases = []
    R = np.sort(rng.uniform(-5, 5, 40)); T = np.sort(rng.uniform(1, 50, 30))        # negative axis
    cases.append((R, T))
    R = np.array([1e-30, 1e-10, 1.0, 1e10, 1e30]); T = np.array([1.0, 2.0, 3.0])      # cells over 2^10 wide
    cases.append((R, T))
    R = np.geomspace(1e-25, 1e-20, 50); T = np.geomspace(1.0, 1e3, 20)               # axis below 2^-70
    cases.append((R, T))
    for R, T in cases:
        F = rng.uniform(0.5, 3.0, (len(R), len(T)))
        Y2 = np.stack([rng.uniform(R[0] * 1.5 - 1, R[-1] * 1.1, 20000) if R[0] < 0 else
                       np.exp(rng.uniform(np.log(R[0]) - 1, np.log(R[-1]) + 1, 20000)),
                       rng.uniform(T[0] - 1, T[-1] + 1, 20000)], 1)
        stat = ss.new_stat()
        idx, val = ss.search_interp_2d(*(torch.as_tensor(a).to(DEV) for a in (R, T, F.reshape(-1), Y2)), stat=stat)
        wi, wv = oracle.search_interp_2d(R, T, F, Y2)
        check_2d(idx.cpu().numpy(), val.cpu().numpy(), wi, wv)
        assert ss.read_stat(stat).flags & ss.FLAG_BAD_VALUE
    # grid values outside the splittable range (and zeros, negatives) on a float-float table
    R = wl.log_spaced_table(50, 1e-3, 1e3, 0.1, seed=1).numpy()
    T = wl.log_spaced_table(40, 1e-2, 1e2, 0.1, seed=2).numpy()
    F = rng.uniform(0.5, 3.0, (50, 40))
    F[3, :] = 1e-200; F[7, 5] = 0.0; F[9, 9] = -2.0; F[11, :] = 1e250
    Y2 = np.stack([np.exp(rng.uniform(np.log(1e-3), np.log(1e3), 50000)),
                   np.exp(rng.uniform(np.log(1e-2), np.log(1e2), 50000))], 1)
    idx, val = ss.search_interp_2d(*(torch.as_tensor(a).to(DEV) for a in (R, T, F.reshape(-1), Y2)))
    wi, wv = oracle.search_interp_2d(R, T, F, Y2)
    np.testing.assert_array_equal(idx.cpu().numpy(), wi)
    v = val.cpu().numpy()
    cr = np.minimum(wi[:, 0], 48)
    ct = np.minimum(wi[:, 1], 38)
    corners = np.abs(np.stack([F[cr, ct], F[cr, ct + 1], F[cr + 1, ct], F[cr + 1, ct + 1]], 1))
    # a convex blend is good to the rounding of its largest term; all-positive cells keep the relative bar
    assert np.all(np.abs(v - wv) <= 1e-12 * corners.max(1))
    pos = (corners.min(1) > 0) & (np.min(np.stack([F[cr, ct], F[cr, ct + 1], F[cr + 1, ct], F[cr + 1, ct + 1]], 1), 1) > 0)
    rel = np.abs(v - wv) / np.abs(wv)
    worst = np.argmax(np.where(pos, rel, 0.0))
    assert rel[worst] <= REL_TOL or not pos[worst], (
        "pair %s idx %s corners %s want %r got %r" % (Y2[worst].tolist(), wi[worst].tolist(),
                                                        [F[cr[worst], ct[worst]], F[cr[worst], ct[worst] + 1],
                                                         F[cr[worst] + 1, ct[worst]], F[cr[worst] + 1, ct[worst] + 1]],
                                                        wv[worst], v[worst]))


def test_2d_crowded_bucket_takes_bisection(ss):
    """Twenty entries packed inside one cell of the density axis leave a
    bucket with many keys: the staged-grid kernel leaves its lean two-key scan
    for the bounded bisection (and the binary layout), exact either way."""
    rng = np.random.default_rng(12)
    base = np.geomspace(1e-6, 1e4, 100)
    R = np.sort(np.concatenate([base, base[50] * (1 + 1e-9 * np.arange(1, 21))]))
    T = wl.log_spaced_table(90, 1e-4, 1e4, 0.1, seed=13).numpy()
    F = wl.field_grid(torch.as_tensor(R), torch.as_tensor(T), wl.smooth_field(1e-6, 1e4, 1e-4, 1e4, seed=14)).numpy()
    m = 300_001
    rho = np.exp(rng.uniform(np.log(0.5e-6), np.log(2e4), m))
    rho[::3] = base[50] * (1 + rng.uniform(0.0, 2.2e-8, len(rho[::3])))          # inside the crowded cell
    rho[1::7] = R[rng.integers(0, len(R), len(rho[1::7]))]                       # on entries
    tem = np.exp(rng.uniform(np.log(0.5e-4), np.log(2e4), m))
    Y2 = np.stack([rho, tem], 1)
    wi, wv = oracle.search_interp_2d(R, T, F, Y2)
    for algo in ("bucket", "binary"):
        idx, val = ss.search_interp_2d(*(torch.as_tensor(a).to(DEV) for a in (R, T, F.reshape(-1), Y2)), algo=algo)
        check_2d(idx.cpu().numpy(), val.cpu().numpy(), wi, wv)


def test_2d_ragged_misaligned_and_sizes(ss):
    for nr, nt in ((2, 2), (2, 3), (3, 2), (33, 65), (500, 300), (4096, 17)):
        R = wl.log_spaced_table(nr, 1e-6, 1e4, 0.1, seed=nr)
        T = wl.log_spaced_table(nt, 1e-4, 1e4, 0.1, seed=nt + 1)
        F = wl.field_grid(R, T, wl.smooth_field(1e-6, 1e4, 1e-4, 1e4, seed=3))
        Y2 = wl.pairs_log_uniform(2003, 0.5e-6, 2e4, 0.5e-4, 2e4, seed=4)
        wi, wv = oracle.search_interp_2d(R.numpy(), T.numpy(), F.numpy(), Y2.numpy())
        Rd, Td, Fd, Yd = R.to(DEV), T.to(DEV), F.to(DEV), Y2.reshape(-1).to(DEV)
        for m in (0, 1, 2, 3, 2002):
            for off in (0, 1):          # off=1 shifts pairs by one double: 8-byte aligned only
                ybuf = torch.empty(2 * m + 2, dtype=torch.float64, device=DEV)
                ybuf[off:off + 2 * m] = Yd[:2 * m]
                ib = torch.full((2 * m + 4,), -7, dtype=torch.int32, device=DEV)
                vb = torch.full((m + 2,), -7.0, dtype=torch.float64, device=DEV)
                ss.search_interp_2d(Rd, Td, Fd, ybuf[off:off + 2 * m], idx=ib[2 * off:2 * off + 2 * m],
                                    val=vb[off:off + m])
                check_2d(ib[2 * off:2 * off + 2 * m].cpu().numpy().reshape(-1, 2), vb[off:off + m].cpu().numpy(),
                         wi[:m], wv[:m])
                assert torch.all(vb[:off] == -7.0) and torch.all(vb[off + m:] == -7.0)


def test_2d_affine_field_exact(ss):
    R = wl.log_spaced_table(200, 1e-6, 1e4, 0.1, seed=1)
    T = wl.log_spaced_table(100, 1e-4, 1e4, 0.1, seed=2)
    F = 3.0 + 0.5 * R[:, None] + 2.0 * T[None, :] + 0.25 * R[:, None] * T[None, :]
    Y2 = wl.pairs_log_uniform(100_000, 1e-6, 1e4, 1e-4, 1e4, seed=3)
    _, val = ss.search_interp_2d(R.to(DEV), T.to(DEV), F.contiguous().to(DEV), Y2.to(DEV))
    want = 3.0 + 0.5 * Y2[:, 0] + 2.0 * Y2[:, 1] + 0.25 * Y2[:, 0] * Y2[:, 1]
    rel = ((val.cpu() - want).abs() / want).max().item()
    assert rel <= 1e-12


# ---------------------------------------------------------------- full sizes, sampled

def option_scale(R, T, F, Y, idx, logspace):
    """Per pair, the sum of |weight x corner| terms of the blend (unclamped
    weights): the size of the numbers the value is formed from, against
    which the 1e-12 bound is taken where extrapolation can cancel."""
    nr, nt = len(R), len(T)
    F2 = F.reshape(nr, nt)
    cr = np.minimum(idx[:, 0], nr - 2)
    ct = np.minimum(idx[:, 1], nt - 2)
    def w(X, c, x):
        if logspace:
            return (np.log(x) - np.log(X[c])) / (np.log(X[c + 1]) - np.log(X[c]))
        return (x - X[c]) / (X[c + 1] - X[c])
    wr, wt = np.abs(w(R, cr, Y[:, 0])), np.abs(w(T, ct, Y[:, 1]))
    lo = np.abs(1 - wt) * np.abs(F2[cr, ct]) + wt * np.abs(F2[cr, ct + 1])
    hi = np.abs(1 - wt) * np.abs(F2[cr + 1, ct]) + wt * np.abs(F2[cr + 1, ct + 1])
    return np.abs(1 - wr) * lo + wr * hi


@pytest.mark.parametrize("extrap,logspace", [(1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("fp64", [False, True])
def test_2d_interpolation_options(ss, extrap, logspace, fp64):
    """Linear extrapolation and log-coordinate weights against the oracle:
    indices exact, values within 1e-12 of the terms they are formed from,
    with pairs spread to 8x beyond both axes."""
    R, T, F, _ = wl.interp_2d(m=4, seed=21)
    Y = wl.pairs_log_uniform(300_001, float(R[0]) / 8, float(R[-1]) * 8, float(T[0]) / 8, float(T[-1]) * 8,
                             seed=22)
    Rn, Tn, Fn, Yn = R.numpy(), T.numpy(), F.numpy(), Y.numpy()
    wi, wv = oracle.search_interp_2d(Rn, Tn, Fn, Yn, extrap=extrap, logspace=logspace)
    idx, val = ss.search_interp_2d(R.to(DEV), T.to(DEV), F.to(DEV), Y.to(DEV), fp64=fp64, extrap=bool(extrap),
                                   logspace=bool(logspace))
    idx, val = idx.cpu().numpy(), val.cpu().numpy()
    np.testing.assert_array_equal(idx, wi)
    scale = option_scale(Rn, Tn, Fn, Yn, wi, logspace)
    err = np.abs(val - wv)
    assert (err <= REL_TOL * scale).all(), err.max()
    if extrap and not logspace:
        # inside the grid nothing changes: the default lookup's values, bit for bit
        inside = (Yn[:, 0] >= Rn[0]) & (Yn[:, 0] <= Rn[-1]) & (Yn[:, 1] >= Tn[0]) & (Yn[:, 1] <= Tn[-1])
        _, dv = ss.search_interp_2d(R.to(DEV), T.to(DEV), F.to(DEV), Y.to(DEV), fp64=fp64)
        np.testing.assert_array_equal(val[inside], dv.cpu().numpy()[inside])


def test_1d_one_billion_sampled(ss):
    """The bench-size 1D run (1B targets, bucket search) checked at 2M sampled positions."""
    m = 1 << 30
    X, Y = wl.plain_1d(m=m, seed=1, device=DEV)
    out = ss.search_1d(X, Y)
    sample = torch.randint(0, m, (2_000_000,), device=DEV)
    sample[:1000] = torch.arange(m - 1000, m, device=DEV)
    got = out[sample].cpu().numpy()
    want = oracle.search_1d_sampled(X.cpu().numpy(), Y[sample].cpu().numpy(), np.arange(len(sample)))
    np.testing.assert_array_equal(got, want)
    # properties at full size: range and the interval invariant on a second sample
    assert int(out.min()) >= 0 and int(out.max()) <= 63
    del out, Y
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_2d_full_size_sampled(ss):
    """The bench-size 2D run (64M pairs) checked at 1M sampled positions."""
    m = 64 << 20
    R, T, F, Y2 = wl.interp_2d(m=m, seed=2, device=DEV)
    idx, val = ss.search_interp_2d(R, T, F, Y2)
    sample = torch.randint(0, m, (1_000_000,), device=DEV)
    wi, wv = oracle.search_interp_2d(R.cpu().numpy(), T.cpu().numpy(), F.cpu().numpy(), Y2[sample].cpu().numpy())
    check_2d(idx[sample].cpu().numpy(), val[sample].cpu().numpy(), wi, wv)


# ---------------------------------------------------------------- host-array entry points

def test_host_entry_points_match_device_calls(ss):
    X, Y = wl.plain_1d(m=(1 << 24) + (1 << 23) + 5, seed=3)     # 1.5 chunks + ragged tail
    Yp = Y.pin_memory()
    got = ss.search_1d_host(X, Yp, out=torch.empty(len(Y), dtype=torch.int32).pin_memory())
    np.testing.assert_array_equal(got.numpy(), ss.search_1d(X.to(DEV), Y.to(DEV)).cpu().numpy())
    # pageable buffers work too
    got2 = ss.search_1d_host(X, Y[:1001].clone(), side=1)
    np.testing.assert_array_equal(got2.numpy(), oracle.search_1d(X.numpy(), Y[:1001].numpy(), side=1))
    R, T, F, Y2 = wl.interp_2d(m=(1 << 23) + 77, seed=4)
    idx, val = ss.search_interp_2d_host(R, T, F, Y2.pin_memory())
    di, dv = ss.search_interp_2d(R.to(DEV), T.to(DEV), F.to(DEV), Y2.to(DEV))
    np.testing.assert_array_equal(idx.numpy(), di.cpu().numpy())
    np.testing.assert_array_equal(val.numpy(), dv.cpu().numpy())


def test_host_entry_points_both_paths(ss):
    """Page-locked target and result buffers are streamed by the kernels over
    the host link; pageable (or mixed) ones go through the chunked copies.
    Both give the device call's answers, across chunk boundaries and at
    offsets that are not 16-byte aligned."""
    X, Y = wl.plain_1d(m=(1 << 24) + (1 << 23) + 3, seed=5)
    want = ss.search_1d(X.to(DEV), Y.to(DEV)).cpu().numpy()
    Yp = torch.empty(len(Y) + 1, dtype=torch.float64).pin_memory()
    Yp[1:] = Y
    Op = torch.full((len(Y) + 1,), -1, dtype=torch.int32).pin_memory()
    ss.search_1d_host(X, Yp[1:], out=Op[1:])                      # mapped, misaligned by 8 / 4 bytes
    np.testing.assert_array_equal(Op[1:].numpy(), want)
    assert int(Op[0]) == -1
    got = ss.search_1d_host(X, Y.clone())                          # pageable, 1.5 chunks
    np.testing.assert_array_equal(got.numpy(), want)
    got = ss.search_1d_host(X, Yp[1:], out=torch.empty(len(Y), dtype=torch.int32))   # mixed: chunked
    np.testing.assert_array_equal(got.numpy(), want)
    R, T, F, Y2 = wl.interp_2d(m=(1 << 23) + (1 << 22) + 9, seed=6)
    di, dv = ss.search_interp_2d(R.to(DEV), T.to(DEV), F.to(DEV), Y2.to(DEV))
    m = Y2.shape[0]
    Ip = torch.empty((m, 2), dtype=torch.int32).pin_memory()
    Vp = torch.empty(m, dtype=torch.float64).pin_memory()
    ss.search_interp_2d_host(R, T, F, Y2.pin_memory(), idx=Ip, val=Vp)   # mapped
    np.testing.assert_array_equal(Ip.numpy(), di.cpu().numpy())
    np.testing.assert_array_equal(Vp.numpy(), dv.cpu().numpy())
    idx, val = ss.search_interp_2d_host(R, T, F, Y2.clone())       # pageable, 1.5 chunks
    np.testing.assert_array_equal(idx.numpy(), di.cpu().numpy())
    np.testing.assert_array_equal(val.numpy(), dv.cpu().numpy())
