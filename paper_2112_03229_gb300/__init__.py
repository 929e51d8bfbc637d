"""GB300 (sm_103a) sorted-table search: Python binding of libsimdsearch.so.

Argument marshalling only: every step of the search and of the 2D lookup
runs in the CUDA kernels of the shared library; PyTorch supplies device
memory and the current stream.  There is no CPU fallback -- if the library
has not been built, every call raises.

The operation (arXiv 2112.03229, Sec. 3): for each target, the index of the
largest table entry below it, with both end clamps; the 2D form (Sec. 1,
2.2) searches a density and a temperature axis and interpolates bilinearly.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import _build

LIB_PATH = _build.LIB

SIDE_LT, SIDE_LE = 0, 1
ALGO_AUTO, ALGO_BINARY, ALGO_BUCKET, ALGO_BALLOT, ALGO_BRANCHY = 0, 1, 2, 3, 4
ALGOS = {"auto": ALGO_AUTO, "binary": ALGO_BINARY, "bucket": ALGO_BUCKET, "ballot": ALGO_BALLOT,
         "branchy": ALGO_BRANCHY}
FLAG_NOT_SORTED = 0x1
FLAG_BAD_VALUE = 0x2

STATUS = {0: "SS_OK", 1: "SS_EINVAL", 2: "SS_ENOTSORTED", 3: "SS_ENOMEM", 4: "SS_ECUDA", 5: "SS_ETIMEOUT",
          6: "SS_EUNSUPPORTED"}


class SSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class DevStat(C.Structure):
    _fields_ = [("nan_targets", C.c_ulonglong), ("fallbacks", C.c_ulonglong), ("flags", C.c_uint),
                ("max_window", C.c_uint)]


_lib = None
_vp, _i32, _i64 = C.c_void_p, C.c_int32, C.c_int64


def lib_path():
    """Path of the library this process loads: libsimdsearch.so, or the
    bounds-checked build when SS_CHECKED_LIBRARY=1 is set in the environment."""
    if os.environ.get("SS_CHECKED_LIBRARY") == "1":
        return os.path.join(os.path.dirname(LIB_PATH), "libsimdsearch_checked.so")
    return LIB_PATH


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("%s is not built (run __graft_entry__.build()); "
                               "this package has no CPU fallback" % os.path.basename(path))
        L = C.CDLL(path)
        L.ss_last_error.restype = C.c_char_p
        L.ss_version.restype = _i32
        L.ss_search_1d.argtypes = [_vp, _i32, _vp, _i64, _vp, _i32, _i32, _vp, _vp]
        L.ss_search_1d_tuned.argtypes = [_vp, _i32, _vp, _i64, _vp, _i32, _i32, _i32, _i32, _vp, _vp]
        L.ss_search_interp_2d.argtypes = [_vp, _i32, _vp, _i32, _vp, _vp, _i64, _vp, _vp, _i32, _vp, _vp]
        L.ss_search_interp_2d_fp64.argtypes = [_vp, _i32, _vp, _i32, _vp, _vp, _i64, _vp, _vp, _i32, _vp, _vp]
        L.ss_sync_status.argtypes = [_vp, _vp, _vp, _i32]
        L.ss_mlp_loss_grad.argtypes = [_vp, _vp, _vp, _i64, _vp, _vp, _vp]
        L.ss_mlp_forward.argtypes = [_vp, _vp, _i64, _vp, _vp]
        L.ss_mlp_adam_step.argtypes = [_vp, _vp, _vp, _vp, _i32, C.c_float, C.c_float, C.c_float, C.c_float, _vp]
        L.ss_checked_hits.argtypes = [C.POINTER(C.c_uint64), _i32]
        L.ss_checked_hits.restype = _i32
        L.ss_checked_selftest.argtypes = []
        L.ss_checked_selftest.restype = _i32
        for name in ("ss_search_1d", "ss_search_1d_tuned", "ss_search_interp_2d", "ss_search_interp_2d_fp64",
                     "ss_sync_status",
                     "ss_mlp_loss_grad", "ss_mlp_forward", "ss_mlp_adam_step"):
            getattr(L, name).restype = _i32
        _lib = L
    return _lib


def checked_hits(reset=False) -> int:
    """ss_checked_hits: indices caught out of range since the last reset
    (bounds-checked build only; raises SSError otherwise)."""
    v = C.c_uint64(0)
    _check(lib().ss_checked_hits(C.byref(v), 1 if reset else 0))
    return int(v.value)


def _check(code):
    if code != 0:
        raise SSError(code, lib().ss_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.device.index is not None and t.device.index != torch.cuda.current_device():
        raise ValueError("%s is on %s, but the library runs on the current device cuda:%d"
                         % (name, t.device, torch.cuda.current_device()))
    if t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return C.c_void_p(t.data_ptr())


def _dev_or_pinned(t, dtype, name):
    """A CUDA tensor, or a page-locked host tensor (mapped into the device's
    address space: the kernels stream it over the host link)."""
    if isinstance(t, torch.Tensor) and not t.is_cuda:
        if not t.is_pinned():
            raise TypeError("%s must be a CUDA tensor or a page-locked host tensor" % name)
        if t.dtype != dtype:
            raise TypeError("%s must be %s" % (name, dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        return C.c_void_p(t.data_ptr())
    return _dev(t, dtype, name)


def _algo(a):
    return ALGOS[a] if isinstance(a, str) else int(a)


def new_stat(device=None) -> torch.Tensor:
    """A zeroed device status record (24 bytes) to pass as `stat`."""
    return torch.zeros(C.sizeof(DevStat), dtype=torch.uint8, device=device or "cuda")


def read_stat(stat: torch.Tensor, stream=None, timeout_ms: int = 60_000) -> DevStat:
    out = DevStat()
    _check(lib().ss_sync_status(_stream(stream), C.c_void_p(stat.data_ptr()), C.byref(out), timeout_ms))
    return out


def _statp(stat):
    if stat is None:
        return None
    if not isinstance(stat, torch.Tensor) or not stat.is_cuda or not stat.is_contiguous():
        raise TypeError("stat must be a contiguous CUDA tensor (see new_stat)")
    if stat.numel() * stat.element_size() < C.sizeof(DevStat):
        raise ValueError("stat must hold at least %d bytes" % C.sizeof(DevStat))
    return _dev(stat, stat.dtype, "stat")


def _need(t, count, name):
    """The library reads or writes `count` elements of t."""
    if t.numel() < count:
        raise ValueError("%s holds %d elements, %d needed" % (name, t.numel(), count))


def search_1d(X: torch.Tensor, Y: torch.Tensor, out: torch.Tensor | None = None, side: int = SIDE_LT,
              algo="auto", stat=None, stream=None, dir_cap: int = 0, ballot_g: int = 0) -> torch.Tensor:
    """ss_search_1d: int32 index of the largest entry of X below each target of Y."""
    if out is None:
        out = torch.empty(Y.shape, dtype=torch.int32, device=Y.device)
    _need(out, Y.numel(), "out")
    args = (_dev(X, torch.float64, "X"), X.numel(), _dev(Y, torch.float64, "Y"), Y.numel(),
            _dev(out, torch.int32, "out"), side, _algo(algo))
    if dir_cap or ballot_g:
        _check(lib().ss_search_1d_tuned(*args, dir_cap, ballot_g, _statp(stat), _stream(stream)))
    else:
        _check(lib().ss_search_1d(*args, _statp(stat), _stream(stream)))
    return out


class InterpOpts(C.Structure):
    _fields_ = [("algo", C.c_int32), ("extrap", C.c_int32), ("logspace", C.c_int32), ("fp64", C.c_int32)]


def search_interp_2d(R, T, F, Y2, idx=None, val=None, algo="auto", stat=None, stream=None, fp64=False,
                     extrap=False, logspace=False):
    """ss_search_interp_2d: per (rho, T) pair the index pair and the bilinear value.
    fp64=True calls ss_search_interp_2d_fp64 (fp64 weights and blend); extrap /
    logspace select linear extrapolation / log-coordinate weights
    (ss_search_interp_2d_ex)."""
    m = Y2.numel() // 2
    if F.numel() != R.numel() * T.numel():
        raise ValueError("F must hold len(R) * len(T) values")
    if idx is None:
        idx = torch.empty((m, 2), dtype=torch.int32, device=Y2.device)
    if val is None:
        val = torch.empty((m,), dtype=torch.float64, device=Y2.device)
    _need(idx, 2 * m, "idx")
    _need(val, m, "val")
    if extrap or logspace:
        L = lib()
        L.ss_search_interp_2d_ex.argtypes = [_vp, _i32, _vp, _i32, _vp, _vp, _i64, _vp, _vp,
                                             C.POINTER(InterpOpts), _vp, _vp]
        L.ss_search_interp_2d_ex.restype = _i32
        o = InterpOpts(_algo(algo), int(bool(extrap)), int(bool(logspace)), int(bool(fp64)))
        _check(L.ss_search_interp_2d_ex(_dev(R, torch.float64, "R"), R.numel(), _dev(T, torch.float64, "T"),
                                        T.numel(), _dev(F, torch.float64, "F"), _dev(Y2, torch.float64, "Y2"), m,
                                        _dev(idx, torch.int32, "idx"), _dev(val, torch.float64, "val"),
                                        C.byref(o), _statp(stat), _stream(stream)))
        return idx, val
    fn = lib().ss_search_interp_2d_fp64 if fp64 else lib().ss_search_interp_2d
    _check(fn(_dev(R, torch.float64, "R"), R.numel(), _dev(T, torch.float64, "T"), T.numel(),
                                     _dev(F, torch.float64, "F"), _dev(Y2, torch.float64, "Y2"), m,
                                     _dev(idx, torch.int32, "idx"), _dev(val, torch.float64, "val"), _algo(algo),
                                     _statp(stat), _stream(stream)))
    return idx, val


# ---------------------------------------------------------------------------
# Position model (2 -> 16 -> 1 MLP) training kernels, exposed for checks
# ---------------------------------------------------------------------------
def mlp_loss_grad(params, x, y, stream=None):
    """Mean squared error of the MLP over (x, y) and its gradient (65 floats), on the GPU."""
    _need(params, 65, "params")
    _need(x, 2 * y.numel(), "x")
    grad = torch.empty(65, dtype=torch.float32, device=params.device)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    _check(lib().ss_mlp_loss_grad(_dev(params, torch.float32, "params"), _dev(x, torch.float32, "x"),
                                  _dev(y, torch.float32, "y"), y.numel(), _dev(grad, torch.float32, "grad"),
                                  _dev(loss, torch.float32, "loss"), _stream(stream)))
    return loss, grad


def mlp_forward(params, x, stream=None):
    _need(params, 65, "params")
    y = torch.empty(x.numel() // 2, dtype=torch.float32, device=x.device)
    _check(lib().ss_mlp_forward(_dev(params, torch.float32, "params"), _dev(x, torch.float32, "x"), y.numel(),
                                _dev(y, torch.float32, "y"), _stream(stream)))
    return y


def mlp_adam_step(params, grad, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    for t, name in ((params, "params"), (grad, "grad"), (m1, "m1"), (m2, "m2")):
        _need(t, 65, name)
    _check(lib().ss_mlp_adam_step(_dev(params, torch.float32, "params"), _dev(grad, torch.float32, "grad"),
                                  _dev(m1, torch.float32, "m1"), _dev(m2, torch.float32, "m2"), step, lr, beta1,
                                  beta2, eps, _stream(stream)))


# ---------------------------------------------------------------------------
# Plans: set-up once per set of tables, many batched searches
# ---------------------------------------------------------------------------
MODEL_NONE, MODEL_SPLINE, MODEL_MLP, MODEL_LOGHASH, MODEL_HUNT, MODEL_AUTO = 0, 1, 2, 3, 4, 5
MODELS = {"none": MODEL_NONE, "spline": MODEL_SPLINE, "mlp": MODEL_MLP, "loghash": MODEL_LOGHASH, "hunt": MODEL_HUNT,
          "auto": MODEL_AUTO}
BLOB_ALGOS = ["bucket", "binary", "ballot8", "ballot16", "ballot32", "spline", "mlp", "loghash", "wide"]


class PlanOpts(C.Structure):
    _fields_ = [("side", C.c_int32), ("algo", C.c_int32), ("model", C.c_int32), ("autotune", C.c_int32),
                ("tile", C.c_int32), ("mlp_epochs", C.c_int32), ("mlp_lr", C.c_float), ("dir_cap", C.c_int32),
                ("seed", C.c_uint64), ("tune_cache", C.c_char_p), ("extrap", C.c_int32), ("logspace", C.c_int32)]


class PlanInfo(C.Structure):
    _fields_ = [("kind", C.c_int32), ("ntables", C.c_int32), ("device_bytes", C.c_int64),
                ("max_window", C.c_int32), ("mean_window", C.c_float), ("train_loss", C.c_float),
                ("nbuckets", C.c_int32), ("bucket_algo", C.c_int32 * 8), ("bucket_tile", C.c_int32 * 8),
                ("bucket_tables", C.c_int32 * 8), ("ntiles", C.c_int64), ("tuned", C.c_int32),
                ("kernels", C.c_int32), ("block_threads", C.c_int32), ("smem_bytes", C.c_int32),
                ("max_occupancy", C.c_int32), ("lean_kernel", C.c_int32)]


def _plan_sigs(L):
    P = C.POINTER(C.c_void_p)
    i64p = C.POINTER(C.c_int64)
    L.ss_plan_opts_default.argtypes = [C.POINTER(PlanOpts)]
    L.ss_plan_opts_default.restype = None
    L.ss_plan_create_1d.argtypes = [P, _i32, i64p, _vp, C.POINTER(PlanOpts), _vp]
    L.ss_plan_create_2d.argtypes = [P, _i32, i64p, _vp, i64p, _vp, i64p, _vp, C.POINTER(PlanOpts), _vp]
    L.ss_plan_bind_1d.argtypes = [_vp, i64p, _vp, _vp, _vp, _vp]
    L.ss_plan_bind_2d.argtypes = [_vp, i64p, _vp, _vp, _vp, _vp, _vp]
    L.ss_plan_execute.argtypes = [_vp, _vp]
    L.ss_plan_info_get.argtypes = [_vp, C.POINTER(PlanInfo)]
    L.ss_plan_save.argtypes = [_vp, C.c_char_p]
    L.ss_plan_load.argtypes = [P, C.c_char_p, _vp]
    L.ss_plan_destroy.argtypes = [_vp]
    L.ss_plan_destroy.restype = None
    for n in ("ss_plan_create_1d", "ss_plan_create_2d", "ss_plan_bind_1d", "ss_plan_bind_2d", "ss_plan_execute",
              "ss_plan_info_get", "ss_plan_save", "ss_plan_load"):
        getattr(L, n).restype = _i32


def _offsets(off, name="offsets", length=None, data=None, per=1):
    """CSR offsets as a host int64 array and its pointer.  The library reads
    ntables + 1 of them (`length`, when the table count is already fixed), and
    the last one, times `per` elements, must lie within `data`."""
    import numpy as np
    a = np.ascontiguousarray(off.cpu().numpy() if isinstance(off, torch.Tensor) else off, dtype=np.int64)
    if a.ndim != 1 or len(a) < 2:
        raise ValueError("%s must list ntables + 1 >= 2 offsets" % name)
    if length is not None and len(a) != length:
        raise ValueError("%s has %d entries, %d expected (ntables + 1)" % (name, len(a), length))
    if a[0] < 0 or (np.diff(a) < 0).any():
        raise ValueError("%s must be non-negative and non-decreasing" % name)
    if data is not None and isinstance(data, torch.Tensor) and int(a[-1]) * per > data.numel():
        raise ValueError("%s end past the data (%d elements needed, %d held)" % (name, int(a[-1]) * per, data.numel()))
    return a, a.ctypes.data_as(C.POINTER(C.c_int64))


def plan_opts(side=SIDE_LT, algo="auto", model="none", autotune=False, tile=0, mlp_epochs=None, mlp_lr=0.0,
              dir_cap=0, seed=0x5EED, tune_cache=None, extrap=False, logspace=False) -> PlanOpts:
    o = PlanOpts()
    L = lib()
    if not hasattr(L, "_plan_sigs"):
        _plan_sigs(L)
        L._plan_sigs = True
    L.ss_plan_opts_default(C.byref(o))
    o.side = side
    o.algo = _algo(algo)
    o.model = MODELS[model] if isinstance(model, str) else int(model)
    o.autotune = int(bool(autotune))
    o.tile = tile
    if mlp_epochs is not None:
        o.mlp_epochs = mlp_epochs
    if mlp_lr:
        o.mlp_lr = mlp_lr
    o.dir_cap = dir_cap
    o.seed = seed
    o.tune_cache = tune_cache.encode() if tune_cache else None
    o.extrap = int(bool(extrap))
    o.logspace = int(bool(logspace))
    return o


class Plan:
    """ss_plan: prepared tables (and learned models) for repeated batched searches."""

    def __init__(self, handle, kind, ntables):
        self._h = handle
        self.kind = kind
        self.ntables = ntables
        self._keep = None

    @classmethod
    def create_1d(cls, X_off, X, stream=None, **opts):
        o = plan_opts(**opts)
        off, offp = _offsets(X_off, "X_off", data=X)
        h = C.c_void_p()
        _check(lib().ss_plan_create_1d(C.byref(h), len(off) - 1, offp, _dev(X, torch.float64, "X"), C.byref(o),
                                       _stream(stream)))
        return cls(h, 1, len(off) - 1)

    @classmethod
    def create_2d(cls, R_off, R, T_off, T, F_off, F, stream=None, **opts):
        o = plan_opts(**opts)
        ro, rp = _offsets(R_off, "R_off", data=R)
        to, tp = _offsets(T_off, "T_off", length=len(ro), data=T)
        fo, fp = _offsets(F_off, "F_off", length=len(ro), data=F)
        h = C.c_void_p()
        _check(lib().ss_plan_create_2d(C.byref(h), len(ro) - 1, rp, _dev(R, torch.float64, "R"), tp,
                                       _dev(T, torch.float64, "T"), fp, _dev(F, torch.float64, "F"), C.byref(o),
                                       _stream(stream)))
        return cls(h, 2, len(ro) - 1)

    @classmethod
    def load(cls, path, stream=None):
        plan_opts()   # registers signatures
        h = C.c_void_p()
        _check(lib().ss_plan_load(C.byref(h), str(path).encode(), _stream(stream)))
        p = cls(h, 0, 0)
        inf = p.info()
        p.kind, p.ntables = inf.kind, inf.ntables
        return p

    def bind_1d(self, Y_off, Y, out, stat=None, stream=None):
        off, offp = _offsets(Y_off, "Y_off", length=self.ntables + 1, data=Y)
        _need(out, int(off[-1]), "out")
        self._keep = (Y, out, stat)
        _check(lib().ss_plan_bind_1d(self._h, offp, _dev_or_pinned(Y, torch.float64, "Y"),
                                     _dev_or_pinned(out, torch.int32, "out"), _statp(stat), _stream(stream)))

    def bind_2d(self, Y_off, Y2, idx, val, stat=None, stream=None):
        off, offp = _offsets(Y_off, "Y_off", length=self.ntables + 1, data=Y2, per=2)
        _need(idx, 2 * int(off[-1]), "idx")
        _need(val, int(off[-1]), "val")
        self._keep = (Y2, idx, val, stat)
        _check(lib().ss_plan_bind_2d(self._h, offp, _dev_or_pinned(Y2, torch.float64, "Y2"),
                                     _dev_or_pinned(idx, torch.int32, "idx"), _dev_or_pinned(val, torch.float64, "val"),
                                     _statp(stat), _stream(stream)))

    def execute(self, stream=None):
        _check(lib().ss_plan_execute(self._h, _stream(stream)))

    def info(self) -> PlanInfo:
        inf = PlanInfo()
        _check(lib().ss_plan_info_get(self._h, C.byref(inf)))
        return inf

    def choices(self):
        inf = self.info()
        return {b: (BLOB_ALGOS[inf.bucket_algo[b]], inf.bucket_tile[b], inf.bucket_tables[b])
                for b in range(inf.nbuckets) if inf.bucket_tables[b]}

    def save(self, path):
        _check(lib().ss_plan_save(self._h, str(path).encode()))

    def close(self):
        if self._h:
            lib().ss_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batched_lib():
    L = lib()
    if not hasattr(L, "_batched_sig"):
        P64 = C.POINTER(C.c_int64)
        L.ss_search_1d_batched.argtypes = [_i32, P64, _vp, P64, _vp, _vp, _i32, _vp, _vp]
        L.ss_search_interp_2d_batched.argtypes = [_i32, P64, _vp, P64, _vp, P64, _vp, P64, _vp, _vp, _vp, _vp, _vp]
        L.ss_search_1d_batched.restype = _i32
        L.ss_search_interp_2d_batched.restype = _i32
        L._batched_sig = True
    return L


def search_1d_batched(X_off, X, Y_off, Y, out=None, side=SIDE_LT, stat=None, stream=None):
    """ss_search_1d_batched: one call over many tables (table k = X[X_off[k]:X_off[k+1]],
    its targets Y[Y_off[k]:Y_off[k+1]]); asynchronous on `stream` (default: the
    current stream); an unsorted table sets FLAG_NOT_SORTED in `stat`."""
    L = _batched_lib()
    xo, xp = _offsets(X_off, "X_off", data=X)
    yo, yp = _offsets(Y_off, "Y_off", length=len(xo), data=Y)
    if out is None:
        out = torch.empty(Y.shape, dtype=torch.int32, device=Y.device)
    _need(out, int(yo[-1]), "out")
    _check(L.ss_search_1d_batched(len(xo) - 1, xp, _dev(X, torch.float64, "X"), yp, _dev(Y, torch.float64, "Y"),
                                  _dev(out, torch.int32, "out"), side, _statp(stat), _stream(stream)))
    return out


def search_interp_2d_batched(R_off, R, T_off, T, F_off, F, Y_off, Y2, idx=None, val=None, stat=None, stream=None):
    """ss_search_interp_2d_batched: the 2D lookup over many tables in one call,
    queued on the stream (the current one by default).  Returns (idx [m, 2]
    int32, val [m] float64)."""
    L = _batched_lib()
    ro, rp = _offsets(R_off, "R_off", data=R)
    to, tp = _offsets(T_off, "T_off", length=len(ro), data=T)
    fo, fp = _offsets(F_off, "F_off", length=len(ro), data=F)
    yo, yp = _offsets(Y_off, "Y_off", length=len(ro), data=Y2, per=2)
    m = Y2.numel() // 2
    if idx is None:
        idx = torch.empty((m, 2), dtype=torch.int32, device=Y2.device)
    if val is None:
        val = torch.empty((m,), dtype=torch.float64, device=Y2.device)
    _need(idx, 2 * int(yo[-1]), "idx")
    _need(val, int(yo[-1]), "val")
    _check(L.ss_search_interp_2d_batched(len(ro) - 1, rp, _dev(R, torch.float64, "R"), tp, _dev(T, torch.float64, "T"),
                                         fp, _dev(F, torch.float64, "F"), yp, _dev(Y2, torch.float64, "Y2"),
                                         _dev(idx, torch.int32, "idx"), _dev(val, torch.float64, "val"),
                                         _statp(stat), _stream(stream)))
    return idx, val


def search_1d_batched_static(X_off, X, Y_off, Y, out=None, side=SIDE_LT, stat=None, stream=None):
    """ss_search_1d_batched_static: batched bucket search that allocates no
    device memory (its working set lives in a fixed 8 MiB array of the library)."""
    L = lib()
    if not hasattr(L, "_static_sig"):
        L.ss_search_1d_batched_static.argtypes = [_i32, C.POINTER(C.c_int64), _vp, C.POINTER(C.c_int64), _vp, _vp,
                                                  _i32, _vp, _vp]
        L.ss_search_1d_batched_static.restype = _i32
        L._static_sig = True
    xo, xp = _offsets(X_off, "X_off", data=X)
    yo, yp = _offsets(Y_off, "Y_off", length=len(xo), data=Y)
    if out is None:
        out = torch.empty(Y.shape, dtype=torch.int32, device=Y.device)
    _need(out, int(yo[-1]), "out")
    _check(L.ss_search_1d_batched_static(len(xo) - 1, xp, _dev(X, torch.float64, "X"), yp,
                                         _dev(Y, torch.float64, "Y"), _dev(out, torch.int32, "out"), side,
                                         _statp(stat), _stream(stream)))
    return out


# ---------------------------------------------------------------------------
# Host-array forms (pipelined copies + search inside the library)
# ---------------------------------------------------------------------------
def _host(t, dtype, name):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("%s must be a host (CPU) tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return C.c_void_p(t.data_ptr())


def _host_lib():
    L = lib()
    if not hasattr(L, "_host_sig"):
        L.ss_search_1d_host.argtypes = [_vp, _i32, _vp, _i64, _vp, _i32, _i32]
        L.ss_search_interp_2d_host.argtypes = [_vp, _i32, _vp, _i32, _vp, _vp, _i64, _vp, _vp, _i32]
        L.ss_search_1d_host.restype = _i32
        L.ss_search_interp_2d_host.restype = _i32
        L._host_sig = True
    return L


def search_1d_host(X, Y, out=None, side=SIDE_LT, algo="auto"):
    """ss_search_1d_host: all arrays in host memory (pin them for full copy speed)."""
    L = _host_lib()
    if out is None:
        out = torch.empty(Y.shape, dtype=torch.int32)
    _need(out, Y.numel(), "out")
    _check(L.ss_search_1d_host(_host(X, torch.float64, "X"), X.numel(), _host(Y, torch.float64, "Y"), Y.numel(),
                               _host(out, torch.int32, "out"), side, _algo(algo)))
    return out


def search_interp_2d_host(R, T, F, Y2, idx=None, val=None, algo="auto"):
    """ss_search_interp_2d_host: all arrays in host memory."""
    L = _host_lib()
    m = Y2.numel() // 2
    if F.numel() != R.numel() * T.numel():
        raise ValueError("F must hold len(R) * len(T) values")
    if idx is None:
        idx = torch.empty((m, 2), dtype=torch.int32)
    if val is None:
        val = torch.empty((m,), dtype=torch.float64)
    _need(idx, 2 * m, "idx")
    _need(val, m, "val")
    _check(L.ss_search_interp_2d_host(_host(R, torch.float64, "R"), R.numel(), _host(T, torch.float64, "T"), T.numel(),
                                      _host(F, torch.float64, "F"), _host(Y2, torch.float64, "Y2"), m,
                                      _host(idx, torch.int32, "idx"), _host(val, torch.float64, "val"), _algo(algo)))
    return idx, val
