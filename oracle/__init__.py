"""Plain CPU oracle for the sorted-table search (arXiv 2112.03229, Sec. 3)
and the bilinear lookup it feeds (Sec. 1, 2.2).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by the cpu_baseline leg of bench.py.  The product package never imports it.

Thin numpy/ctypes marshalling around oracle.c; all arithmetic is in the C file.
"""
import ctypes as C

import numpy as np

from . import build as _build_mod

_lib = None

_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_u64p = C.POINTER(C.c_uint64)
_f64p = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build_mod.build())
        L.oracle_search_1d.argtypes = [_f64p, C.c_int32, _f64p, C.c_int64, C.c_int32, _i32p]
        L.oracle_search_1d_sampled.argtypes = [_f64p, C.c_int32, _f64p, _i64p, C.c_int64, C.c_int32, _i32p]
        L.oracle_search_interp_2d.argtypes = [_f64p, C.c_int32, _f64p, C.c_int32, _f64p, _f64p,
                                              C.c_int64, _i32p, _f64p]
        L.oracle_search_interp_2d_sampled.argtypes = [_f64p, C.c_int32, _f64p, C.c_int32, _f64p, _f64p,
                                                      _i64p, C.c_int64, _i32p, _f64p]
        L.oracle_search_1d_batched.argtypes = [C.c_int32, _i64p, _f64p, _i64p, _f64p, C.c_int32, _i32p]
        L.oracle_search_interp_2d_batched.argtypes = [C.c_int32, _i64p, _f64p, _i64p, _f64p, _i64p, _f64p,
                                                      _i64p, _f64p, _i32p, _f64p]
        L.oracle_search_interp_2d_opts.argtypes = [_f64p, C.c_int32, _f64p, C.c_int32, _f64p, _f64p,
                                                   C.c_int64, C.c_int32, C.c_int32, _i32p, _f64p]
        L.oracle_search_interp_2d_batched_opts.argtypes = [C.c_int32, _i64p, _f64p, _i64p, _f64p, _i64p, _f64p,
                                                           _i64p, _f64p, C.c_int32, C.c_int32, _i32p, _f64p]
        L.oracle_order_key.argtypes = [C.c_double]
        L.oracle_order_key.restype = C.c_uint64
        L.oracle_bucket_directory.argtypes = [_f64p, C.c_int32, C.c_int32, _u64p, _i32p, C.c_int64]
        L.oracle_bucket_directory.restype = C.c_int64
        L.oracle_bucket_shift.argtypes = [_f64p, C.c_int32, C.c_int64]
        L.oracle_bucket_shift.restype = C.c_int32
        L.oracle_spline_knots.argtypes = [_f64p, C.c_int32, C.c_int32, _u64p, _i32p]
        L.oracle_mlp_features.argtypes = [C.c_double, C.c_double, C.c_double, _f64p, _f64p]
        L.oracle_mlp_forward.argtypes = [_f64p, _f64p, C.c_int64, _f64p]
        L.oracle_mlp_loss_grad.argtypes = [_f64p, _f64p, _f64p, C.c_int64, _f64p]
        L.oracle_mlp_loss_grad.restype = C.c_double
        L.oracle_adam_step.argtypes = [_f64p, _f64p, _f64p, _f64p, C.c_int64, C.c_double, C.c_double,
                                       C.c_double, C.c_double]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


SIDE_LT, SIDE_LE = 0, 1


def search_1d(X, Y, side=SIDE_LT):
    """Index of the largest entry of X below each target (Sec. 3), int32."""
    X, Y = _f64(X), _f64(Y)
    out = np.empty(Y.shape[0], dtype=np.int32)
    lib().oracle_search_1d(_p(X, _f64p), X.shape[0], _p(Y, _f64p), Y.shape[0], side, _p(out, _i32p))
    return out


def search_1d_sampled(X, Y, sample, side=SIDE_LT):
    """search_1d evaluated only at the target positions listed in sample."""
    X, Y = _f64(X), _f64(Y)
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    out = np.empty(sample.shape[0], dtype=np.int32)
    lib().oracle_search_1d_sampled(_p(X, _f64p), X.shape[0], _p(Y, _f64p), _p(sample, _i64p),
                                   sample.shape[0], side, _p(out, _i32p))
    return out


def search_interp_2d(R, T, F, Y2, extrap=0, logspace=0):
    """Per (rho, T) pair: the two lower-bound indices and the bilinear value.
    extrap=1: linear extrapolation (no weight clamp); logspace=1: weights in
    log axis coordinates (reading R6 of the C source)."""
    R, T, F, Y2 = _f64(R), _f64(T), _f64(F), _f64(Y2).reshape(-1)
    assert F.size == R.shape[0] * T.shape[0]
    m = Y2.shape[0] // 2
    idx = np.empty(2 * m, dtype=np.int32)
    val = np.empty(m, dtype=np.float64)
    if extrap or logspace:
        lib().oracle_search_interp_2d_opts(_p(R, _f64p), R.shape[0], _p(T, _f64p), T.shape[0], _p(F, _f64p),
                                           _p(Y2, _f64p), m, int(extrap), int(logspace), _p(idx, _i32p),
                                           _p(val, _f64p))
    else:
        lib().oracle_search_interp_2d(_p(R, _f64p), R.shape[0], _p(T, _f64p), T.shape[0], _p(F, _f64p),
                                      _p(Y2, _f64p), m, _p(idx, _i32p), _p(val, _f64p))
    return idx.reshape(m, 2), val


def search_interp_2d_sampled(R, T, F, Y2, sample):
    R, T, F, Y2 = _f64(R), _f64(T), _f64(F), _f64(Y2).reshape(-1)
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    ns = sample.shape[0]
    idx = np.empty(2 * ns, dtype=np.int32)
    val = np.empty(ns, dtype=np.float64)
    lib().oracle_search_interp_2d_sampled(_p(R, _f64p), R.shape[0], _p(T, _f64p), T.shape[0],
                                          _p(F, _f64p), _p(Y2, _f64p), _p(sample, _i64p), ns,
                                          _p(idx, _i32p), _p(val, _f64p))
    return idx.reshape(ns, 2), val


def search_1d_batched(X_off, X, Y_off, Y, side=SIDE_LT):
    X_off = np.ascontiguousarray(X_off, dtype=np.int64)
    Y_off = np.ascontiguousarray(Y_off, dtype=np.int64)
    X, Y = _f64(X), _f64(Y)
    out = np.empty(Y.shape[0], dtype=np.int32)
    lib().oracle_search_1d_batched(X_off.shape[0] - 1, _p(X_off, _i64p), _p(X, _f64p),
                                   _p(Y_off, _i64p), _p(Y, _f64p), side, _p(out, _i32p))
    return out


def search_interp_2d_batched(R_off, R, T_off, T, F_off, F, Y_off, Y2, extrap=0, logspace=0):
    offs = [np.ascontiguousarray(o, dtype=np.int64) for o in (R_off, T_off, F_off, Y_off)]
    R, T, F, Y2 = _f64(R), _f64(T), _f64(F), _f64(Y2).reshape(-1)
    m = Y2.shape[0] // 2
    idx = np.empty(2 * m, dtype=np.int32)
    val = np.empty(m, dtype=np.float64)
    lib().oracle_search_interp_2d_batched_opts(offs[0].shape[0] - 1, _p(offs[0], _i64p), _p(R, _f64p),
                                               _p(offs[1], _i64p), _p(T, _f64p), _p(offs[2], _i64p),
                                               _p(F, _f64p), _p(offs[3], _i64p), _p(Y2, _f64p),
                                               int(extrap), int(logspace), _p(idx, _i32p), _p(val, _f64p))
    return idx.reshape(m, 2), val


def order_key(x):
    return int(lib().oracle_order_key(float(x)))


def bucket_directory(X, shift, cap=1 << 22):
    """(base bucket, L[0..B]) of the exponent-style hash h = key >> shift (Sec. 3.5)."""
    X = _f64(X)
    L = np.empty(cap, dtype=np.int32)
    base = C.c_uint64()
    B = lib().oracle_bucket_directory(_p(X, _f64p), X.shape[0], shift, C.byref(base), _p(L, _i32p), cap)
    if B < 0:
        raise ValueError("directory larger than cap")
    return int(base.value), L[: B + 1].copy()


def bucket_shift(X, cap_buckets):
    X = _f64(X)
    return int(lib().oracle_bucket_shift(_p(X, _f64p), X.shape[0], cap_buckets))


def spline_knots(X, K):
    X = _f64(X)
    counts = np.empty(K + 1, dtype=np.int32)
    delta = C.c_uint64()
    lib().oracle_spline_knots(_p(X, _f64p), X.shape[0], K, C.byref(delta), _p(counts, _i32p))
    return int(delta.value), counts


def mlp_features(t, e_lo, e_scale):
    a, b = C.c_double(), C.c_double()
    lib().oracle_mlp_features(float(t), float(e_lo), float(e_scale), C.byref(a), C.byref(b))
    return a.value, b.value


def mlp_forward(params, x):
    params, x = _f64(params), _f64(x).reshape(-1)
    B = x.shape[0] // 2
    y = np.empty(B, dtype=np.float64)
    lib().oracle_mlp_forward(_p(params, _f64p), _p(x, _f64p), B, _p(y, _f64p))
    return y


def mlp_loss_grad(params, x, target):
    params, x, target = _f64(params), _f64(x).reshape(-1), _f64(target)
    grad = np.empty(65, dtype=np.float64)
    loss = lib().oracle_mlp_loss_grad(_p(params, _f64p), _p(x, _f64p), _p(target, _f64p),
                                      target.shape[0], _p(grad, _f64p))
    return loss, grad


def adam_step(params, grad, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of params, m1, m2 (float64 numpy arrays of 65)."""
    for a in (params, m1, m2):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    grad = _f64(grad)
    lib().oracle_adam_step(_p(params, _f64p), _p(grad, _f64p), _p(m1, _f64p), _p(m2, _f64p),
                           step, lr, beta1, beta2, eps)
