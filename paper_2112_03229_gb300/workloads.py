"""Seeded synthetic inputs for the search and the 2D lookup.

This module holds the input recipes only -- none of the search or
interpolation arithmetic.  Both the CUDA path and the CPU oracle are fed from
here.  Every generator takes a seed and a torch device, so small cases are
drawn on the CPU and billion-element cases directly in HBM with the same
recipe.

Recipes (the paper's SESAME table 301 / material 3720 is not available, so
log-spaced tables stand in for it; Sec. 4 gives its range 3e-6 .. 5.4e4 g/cc
with n = 110 and log-uniform targets over 1e-10 .. 1e10):

* jittered log-spaced table: entry i sits at log10 position (i + d_i) * h,
  d_i ~ U(-j, j) for interior entries, end points exact; strictly increasing
  for j < 0.5.
* clustered table: log-space key density 1 everywhere except 4 seeded
  regions, each 1/16 of the log range, at 8x density; entries are the n
  quantiles of the cumulative density.
* log-uniform targets over [lo, hi]; optionally a fraction of exact key hits.
* smooth value grid: F = 1 + sum_{k<8} a_k exp(-((log10 rho - mu_k)^2 / 2 s_k^2
  + (log10 T - nu_k)^2 / 2 t_k^2)), a_k ~ U(0.5, 2), mu/nu uniform over the
  axes' log ranges, s/t ~ U(0.3, 2) decades.
* batched 1D: table sizes round(log-uniform[20, 2000]), per-table range
  min 10^U(-8,-2), span 10^U(4,12); target counts from a truncated discrete
  Zipf(1.1) on [1e3, 1e6].
* batched 2D: axes of U{50..500} x U{30..300} entries; pairs either
  log-uniform in range or coherent (a random walk in log space with
  N(0, 0.01 decade) steps, reflected at the axis bounds).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

F64 = torch.float64


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    return g


def _uniform(shape, lo, hi, g, device):
    return torch.rand(shape, generator=g, device=device, dtype=F64) * (hi - lo) + lo


def log_spaced_table(n: int, lo: float, hi: float, jitter: float, seed: int, device="cpu") -> torch.Tensor:
    """Strictly increasing float64 table of n entries, jittered log spacing."""
    assert n >= 2 and 0 < lo < hi and 0 <= jitter < 0.5
    g = _gen(seed, device)
    la, lb = math.log10(lo), math.log10(hi)
    h = (lb - la) / (n - 1)
    pos = torch.arange(n, device=device, dtype=F64)
    d = _uniform((n,), -jitter, jitter, g, device)
    d[0] = 0.0
    d[-1] = 0.0
    X = torch.pow(10.0, la + pos * h + d * h)
    X[0] = lo
    X[-1] = hi
    assert bool((X[1:] > X[:-1]).all()), "table not strictly increasing"
    return X


def clustered_table(n: int, lo: float, hi: float, seed: int, regions: int = 4, width: float = 1 / 16,
                    factor: float = 8.0, device="cpu") -> torch.Tensor:
    """n quantiles of a log-space density that is `factor`x higher in `regions` seeded windows."""
    rng = np.random.default_rng(seed)
    la, lb = math.log10(lo), math.log10(hi)
    L = lb - la
    fine = 1 << 16
    u = (np.arange(fine + 1) / fine)                      # normalised log position
    dens = np.ones(fine)
    centers = (u[:-1] + u[1:]) / 2
    for s in rng.uniform(0.0, 1.0 - width, size=regions):
        dens[(centers >= s) & (centers < s + width)] = factor
    cdf = np.concatenate([[0.0], np.cumsum(dens)])
    cdf /= cdf[-1]
    q = np.interp(np.arange(n) / (n - 1), cdf, u)
    X = 10.0 ** (la + q * L)
    X[0], X[-1] = lo, hi
    assert np.all(X[1:] > X[:-1]), "table not strictly increasing"
    return torch.tensor(X, dtype=F64, device=device)


def log_uniform(m: int, lo: float, hi: float, seed: int, device="cpu") -> torch.Tensor:
    g = _gen(seed, device)
    u = torch.rand((m,), generator=g, device=device, dtype=F64)
    return torch.pow(10.0, math.log10(lo) + u * (math.log10(hi) - math.log10(lo)))


def targets_with_hits(X: torch.Tensor, m: int, lo: float, hi: float, hit_frac: float, seed: int,
                      device="cpu") -> torch.Tensor:
    """Log-uniform targets over [lo, hi] with a fraction replaced by exact table entries."""
    Y = log_uniform(m, lo, hi, seed, device)
    nh = int(round(m * hit_frac))
    if nh:
        g = _gen(seed ^ 0x5EED, device)
        where = torch.randint(0, m, (nh,), generator=g, device=device)
        which = torch.randint(0, X.shape[0], (nh,), generator=g, device=device)
        Y[where] = X.to(device)[which]
    return Y


@dataclass
class Field2D:
    a: np.ndarray
    mu: np.ndarray
    nu: np.ndarray
    s: np.ndarray
    t: np.ndarray


def smooth_field(R_lo, R_hi, T_lo, T_hi, seed: int, k: int = 8) -> Field2D:
    rng = np.random.default_rng(seed)
    return Field2D(a=rng.uniform(0.5, 2.0, k),
                   mu=rng.uniform(math.log10(R_lo), math.log10(R_hi), k),
                   nu=rng.uniform(math.log10(T_lo), math.log10(T_hi), k),
                   s=rng.uniform(0.3, 2.0, k), t=rng.uniform(0.3, 2.0, k))


def field_grid(R: torch.Tensor, T: torch.Tensor, fld: Field2D) -> torch.Tensor:
    """Row-major [len(R)][len(T)] float64 grid of the smooth field."""
    lr = torch.log10(R.double().cpu())[:, None]
    lt = torch.log10(T.double().cpu())[None, :]
    F = torch.ones(R.shape[0], T.shape[0], dtype=F64)
    for a, mu, nu, s, t in zip(fld.a, fld.mu, fld.nu, fld.s, fld.t):
        F += a * torch.exp(-((lr - mu) ** 2 / (2 * s * s) + (lt - nu) ** 2 / (2 * t * t)))
    return F.contiguous().to(R.device)


def pairs_log_uniform(m: int, R_lo, R_hi, T_lo, T_hi, seed: int, device="cpu") -> torch.Tensor:
    """m interleaved (rho, T) pairs, each coordinate log-uniform over its axis range; shape [m, 2]."""
    Y = torch.empty((m, 2), dtype=F64, device=device)
    Y[:, 0] = log_uniform(m, R_lo, R_hi, seed, device)
    Y[:, 1] = log_uniform(m, T_lo, T_hi, seed + 1, device)
    return Y


def _reflect(z: torch.Tensor, a: float, b: float) -> torch.Tensor:
    w = b - a
    y = torch.remainder(z - a, 2 * w)
    return a + torch.where(y > w, 2 * w - y, y)


def _walk(m: int, lo: float, hi: float, g, step: float, jump: float, device) -> torch.Tensor:
    """m points of a random walk in log10 space over [lo, hi], reflected at the
    bounds: N(0, step) steps, each replaced with probability `jump` by a
    uniform jump of up to the whole log range (a walk that leaps many cells)."""
    a, b = math.log10(lo), math.log10(hi)
    z0 = a + (b - a) * torch.rand((1,), generator=g, device=device, dtype=F64)
    steps = torch.randn((m,), generator=g, device=device, dtype=F64) * step
    if jump > 0:
        leap = torch.rand((m,), generator=g, device=device, dtype=F64) < jump
        far = (torch.rand((m,), generator=g, device=device, dtype=F64) * 2 - 1) * (b - a)
        steps = torch.where(leap, far, steps)
    steps[0] = 0.0
    z = _reflect(z0 + torch.cumsum(steps, 0), a, b)
    return torch.pow(10.0, z).clamp_(lo, hi)


def walk_1d(m: int, lo: float, hi: float, seed: int, step: float = 0.01, jump: float = 0.0,
            device="cpu") -> torch.Tensor:
    """m coherent targets over [lo, hi]: a reflected random walk in log10 space."""
    return _walk(m, lo, hi, _gen(seed, device), step, jump, device)


def pairs_random_walk(m: int, R_lo, R_hi, T_lo, T_hi, seed: int, step: float = 0.01, jump: float = 0.0,
                      device="cpu") -> torch.Tensor:
    """m coherent pairs: a reflected random walk in log10 space, N(0, step) per coordinate."""
    g = _gen(seed, device)
    out = torch.empty((m, 2), dtype=F64, device=device)
    for col, (lo, hi) in enumerate(((R_lo, R_hi), (T_lo, T_hi))):
        out[:, col] = _walk(m, lo, hi, g, step, jump, device)
    return out


# --------------------------------------------------------------------------
# The five workload families
# --------------------------------------------------------------------------

def plain_1d(m: int = 1 << 20, n: int = 64, seed: int = 1, device="cpu"):
    """Single 1D table (n=64, 1e-6..1e4, +-10% gap jitter); m targets over
    [0.5 min, 2 max] with 1% exact key hits."""
    X = log_spaced_table(n, 1e-6, 1e4, 0.1, seed, device)
    Y = targets_with_hits(X, m, 0.5e-6, 2e4, 0.01, seed + 17, device)
    return X, Y


def interp_2d(m: int = 64 << 20, nr: int = 200, nt: int = 100, seed: int = 2, device="cpu"):
    """Density axis 200 over 1e-6..1e4, temperature axis 100 over 1e-4..1e4,
    smooth 8-Gaussian value grid, m (rho, T) pairs log-uniform in range."""
    R = log_spaced_table(nr, 1e-6, 1e4, 0.1, seed, device)
    T = log_spaced_table(nt, 1e-4, 1e4, 0.1, seed + 1, device)
    F = field_grid(R, T, smooth_field(1e-6, 1e4, 1e-4, 1e4, seed + 2))
    Y2 = pairs_log_uniform(m, 1e-6, 1e4, 1e-4, 1e4, seed + 3, device)
    return R, T, F, Y2


def paper_workload(m: int = 5_000_000, seed: int = 3, device="cpu"):
    """The paper's experiment shape (Sec. 4): n=110 over 3e-6..5.4e4 and m
    targets log-uniform over 1e-10..1e10."""
    X = log_spaced_table(110, 3e-6, 5.4e4, 0.1, seed, device)
    Y = log_uniform(m, 1e-10, 1e10, seed + 1, device)
    return X, Y


def sweep_table(n: int, seed: int = 4, device="cpu"):
    """Clustered table of the table-size sweep (n in 16, 256, 4096, 65536)."""
    return clustered_table(n, 1e-6, 1e4, seed + n, device=device)


def zipf_counts(k: int, a: float, lo: int, hi: int, rng: np.random.Generator) -> np.ndarray:
    """k draws of a discrete Zipf(a) law truncated to the integers [lo, hi]."""
    support = np.arange(lo, hi + 1, dtype=np.float64)
    cdf = np.cumsum(support ** (-a))
    cdf /= cdf[-1]
    return (lo + np.searchsorted(cdf, rng.random(k), side="right")).astype(np.int64)


@dataclass
class Batched1D:
    X_off: torch.Tensor   # int64 [ntables+1]
    X: torch.Tensor       # float64, all tables back to back
    Y_off: torch.Tensor   # int64 [ntables+1]
    Y: torch.Tensor       # float64, all targets back to back
    lo: np.ndarray
    hi: np.ndarray


def batched_1d(ntables: int = 10_000, seed: int = 5, count_lo: int = 1000, count_hi: int = 1_000_000,
               count_scale: float = 1.0, device="cpu", max_targets: int | None = None) -> Batched1D:
    """Many uneven tables: sizes round(log-uniform[20,2000]), ranges
    min 10^U(-8,-2) with span 10^U(4,12), Zipf(1.1) target counts on
    [count_lo, count_hi] (scaled by count_scale for small test cases).
    max_targets keeps the targets of the first tables only (a prefix of the
    same batch: later tables get none)."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(10 ** rng.uniform(math.log10(20), math.log10(2000), ntables)).astype(np.int64)
    lo = 10 ** rng.uniform(-8, -2, ntables)
    hi = lo * 10 ** rng.uniform(4, 12, ntables)
    counts = np.maximum(0, np.rint(zipf_counts(ntables, 1.1, count_lo, count_hi, rng) * count_scale)).astype(np.int64)
    if max_targets is not None:
        keep = np.cumsum(counts) <= max_targets
        counts = np.where(keep, counts, 0)
    X_off = np.concatenate([[0], np.cumsum(sizes)])
    Y_off = np.concatenate([[0], np.cumsum(counts)])
    X = torch.cat([log_spaced_table(int(sizes[k]), float(lo[k]), float(hi[k]), 0.1, seed * 100003 + k)
                   for k in range(ntables)]).to(device)
    u = torch.rand((int(Y_off[-1]),), generator=_gen(seed + 7, device), device=device, dtype=F64)
    # each table's targets are log-uniform over [0.5 min, 2 max] of that table
    tab = torch.repeat_interleave(torch.arange(ntables, device=device),
                                  torch.as_tensor(counts, device=device))
    la = torch.as_tensor(np.log10(0.5 * lo), device=device)[tab]
    lb = torch.as_tensor(np.log10(2.0 * hi), device=device)[tab]
    Y = torch.pow(10.0, la + u * (lb - la))
    return Batched1D(torch.as_tensor(X_off, device=device), X, torch.as_tensor(Y_off, device=device), Y, lo, hi)


def batched_1d_x2(seed: int = 5, count_scale: float = 1.0, device="cpu") -> Batched1D:
    """Two independent 10,000-table batches (seeds `seed` and `seed + 500`)
    back to back: 20,000 tables and about 2.2B targets, the stated "about 2B"
    reached without distorting the Zipf(1.1) count law of one batch."""
    a = batched_1d(ntables=10_000, seed=seed, count_scale=count_scale, device=device)
    b = batched_1d(ntables=10_000, seed=seed + 500, count_scale=count_scale, device=device)
    return Batched1D(torch.cat([a.X_off, b.X_off[1:] + a.X_off[-1]]), torch.cat([a.X, b.X]),
                     torch.cat([a.Y_off, b.Y_off[1:] + a.Y_off[-1]]), torch.cat([a.Y, b.Y]),
                     np.concatenate([a.lo, b.lo]), np.concatenate([a.hi, b.hi]))


@dataclass
class Batched2D:
    R_off: torch.Tensor
    R: torch.Tensor
    T_off: torch.Tensor
    T: torch.Tensor
    F_off: torch.Tensor
    F: torch.Tensor
    Y_off: torch.Tensor
    Y2: torch.Tensor      # [m, 2]


def batched_2d(ntables: int = 1000, pairs_per_table: int = 1_000_000, coherent: bool = False, seed: int = 6,
               device="cpu", jump: float = 0.0) -> Batched2D:
    """Many 2D tables (axes U{50..500} x U{30..300}, jittered log spacing,
    per-table smooth fields), an equal number of pairs per table, random or
    coherent order (with `jump`, a fraction of the walk's steps leap across
    up to the whole range)."""
    rng = np.random.default_rng(seed)
    nr = rng.integers(50, 501, ntables)
    nt = rng.integers(30, 301, ntables)
    r_lo = 10 ** rng.uniform(-7, -5, ntables)
    r_hi = r_lo * 10 ** rng.uniform(9, 11, ntables)
    t_lo = 10 ** rng.uniform(-5, -3, ntables)
    t_hi = t_lo * 10 ** rng.uniform(7, 9, ntables)
    Rs, Ts, Fs, Ys = [], [], [], []
    for k in range(ntables):
        s = seed * 1000003 + 7 * k
        R = log_spaced_table(int(nr[k]), float(r_lo[k]), float(r_hi[k]), 0.1, s)
        T = log_spaced_table(int(nt[k]), float(t_lo[k]), float(t_hi[k]), 0.1, s + 1)
        F = field_grid(R, T, smooth_field(r_lo[k], r_hi[k], t_lo[k], t_hi[k], s + 2))
        Rs.append(R)
        Ts.append(T)
        Fs.append(F.reshape(-1))
        if coherent:
            Ys.append(pairs_random_walk(pairs_per_table, r_lo[k], r_hi[k], t_lo[k], t_hi[k], s + 3, jump=jump,
                                        device=device))
        else:
            Ys.append(pairs_log_uniform(pairs_per_table, r_lo[k], r_hi[k], t_lo[k], t_hi[k], s + 3, device=device))
    off = lambda sizes: torch.as_tensor(np.concatenate([[0], np.cumsum(sizes)]), dtype=torch.int64, device=device)
    return Batched2D(off(nr), torch.cat(Rs).to(device), off(nt), torch.cat(Ts).to(device),
                     off(nr * nt), torch.cat(Fs).to(device),
                     off(np.full(ntables, pairs_per_table)), torch.cat(Ys))
