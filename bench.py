#!/usr/bin/env python3
"""Throughput benchmark of the sorted-table search on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]
                [--scaling weak|strong]

Prints ONE JSON line (rank 0).  A step is one pass of the hot path over one
batch of synthetic input that is already resident in HBM; `value` is the
whole-job throughput in Gtargets/s (a 2D (rho, T) pair counts as one
target).  The headline workload is the batched plain-vs-learned case: two
independent batches of 10,000 tables of 20..2000 entries with Zipf(1.1)
target counts (about 2.2B targets in all), one graph launch of the
persistent plan kernel per step; the timed form is
the autotuned plain search, and the spline, MLP and log-hash proposal forms
and the '<=' side are timed on the same batch beside it.  Inputs are larger
than L2, so no flush is needed between steps.

After the headline, a default run (N=1) measures every other configuration
of the suite the same way and adds one record per configuration under
`configs`: the 64-entry table with 1M targets (L2 flushed between steps) and
scaled to 1B targets, the 200 x 100 2D lookup over 64M pairs, the 16..65536
table-size sweep, and the 1,000-table 2D batch in random and coherent order.
Each record carries its own value, CUDA-event times, roofline fraction,
end-to-end rate, the learned (and hunt) forms and the '<=' side beside the
plain search, and a CPU baseline whose outputs are compared element by
element with the GPU's at the same targets (the parity sample).

`e2e` is the same metric with the inputs in pinned host memory and the
outputs written back to pinned host memory inside the timed region: the
library's kernels stream page-locked buffers over the host link themselves
(the host-array entry points, or a plan bound to host buffers), so the
host-to-device and device-to-host traffic of a step is in flight at once.
`--impl reference` times the plain CPU oracle on host cores on a bounded
sample of the same workload (the oracle is test infrastructure; this arm and
`cpu_baseline` are its only uses here).  `--scaling strong` splits one
workload over the ranks (tables by longest processing time on their target
counts, or contiguous slices of one table's targets) instead of giving every
rank its own.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gtargets/s and HBM fraction of peak, learned vs plain search, same GB300"
UNIT = "Gtargets/s"


# ---------------------------------------------------------------------------
# Peaks
# ---------------------------------------------------------------------------
def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            v = float(json.load(f)["hbm_gbs"])
            return v, "measured"
    except Exception:
        return 6800.0, "fallback"


def sources_hash(files):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2112_03229_gb300", "csrc")
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded(kernel, workload, field="dram_bytes_per_launch"):
    """A per-launch (or per-unit) figure from the committed ncu summaries, or
    None when the kernel's source files changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f)[f"{kernel}@{workload}"]
        if rec.get("sources") != sources_hash(rec["files"]):
            return None
        return float(rec[field])
    except Exception:
        return None


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary (None once stale)."""
    return recorded(kernel, workload, "dram_bytes_per_launch")


FP64_NOMINAL_GOPS = 1250.0     # GB300 fp64: 1.25 TFLOP/s nominal (no measured figure in this pool's peaks)


def co_bound(wl_obj, value, sm_mhz):
    """Beside the HBM roofline, the instruction-issue bound of a kernel that
    computes per unit (the 2D lookups): warp instructions per unit from the
    committed ncu capture times the measured rate, against four issue slots
    per SM per clock at the sampled SM clock; and the fp64 instructions per
    unit against the nominal fp64 rate.  None when no current record exists."""
    w = recorded(wl_obj.kernel, wl_obj.name, "warp_inst_per_unit")
    if w is None:
        return None
    f64 = recorded(wl_obj.kernel, wl_obj.name, "fp64_thread_inst_per_unit")
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_mhz or 2070.0
    achieved = value * 1e9 * w / 1e12
    peak = sms * 4 * mhz * 1e6 / 1e12
    out = {"bound": "issue", "warp_inst_per_unit": w, "achieved": round(achieved, 4), "peak": round(peak, 4),
           "unit": "T warp instructions/s", "frac": round(achieved / peak, 4),
           "peak_source": "%d SMs x 4 issue slots x %.0f MHz (median SM clock sampled during this record)" % (sms, mhz)}
    if f64 is not None:
        g = value * f64
        out["fp64"] = {"thread_inst_per_unit": f64, "achieved_Gops": round(g, 1), "peak_Gops": FP64_NOMINAL_GOPS,
                       "frac": round(g / FP64_NOMINAL_GOPS, 4), "peak_source": "nominal"}
    return out


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout_s=3.0):
        """Block until the sampler has produced a line (nvidia-smi takes a
        moment to start), so that the timed region that follows is covered."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout_s:
            time.sleep(0.01)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, lo=0, hi=None):
        """Median and max SM clock and the throttle reasons seen in samples lo..hi."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[lo:hi]:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# The CPU oracle, timed as it stands (cpu_baseline and the reference arm).
# The outputs of the single-thread run are also compared, element by element,
# with the GPU's outputs at the same positions (taken right after the timed
# region): a sampled parity check of every benchmarked configuration.
# ---------------------------------------------------------------------------
REL_TOL = 1e-12                 # interpolated values against the fp64 oracle


def _batched_tables(Y_off, lo, hi):
    """Tables t0..t1-1 whose target ranges meet [lo, hi), and their offsets clipped to it."""
    t0 = max(int(np.searchsorted(Y_off, lo, side="right")) - 1, 0)
    t1 = max(int(np.searchsorted(Y_off, hi, side="left")), t0 + 1)
    return t0, t1, np.clip(Y_off[t0:t1 + 1], lo, hi) - lo


def _oracle_call(kind, a, lo, hi):
    """One oracle call on units [lo, hi) of a sample (targets, or pairs for 2D);
    returns the oracle's indices (and values for 2D)."""
    import oracle
    side = a.get("side", 0)
    if kind == "1d":
        return oracle.search_1d(a["X"], a["Y"][lo:hi], side)
    if kind == "2d":
        return oracle.search_interp_2d(a["R"], a["T"], a["F"], a["Y2"][lo:hi])
    if kind == "1d_batched":
        t0, t1, yo = _batched_tables(a["Y_off"], lo, hi)
        xo = a["X_off"][t0:t1 + 1]
        return oracle.search_1d_batched(xo - xo[0], a["X"][xo[0]:xo[-1]], yo, a["Y"][lo:hi], side)
    t0, t1, yo = _batched_tables(a["Y_off"], lo, hi)
    ro, to, fo = (a[k][t0:t1 + 1] for k in ("R_off", "T_off", "F_off"))
    return oracle.search_interp_2d_batched(ro - ro[0], a["R"][ro[0]:ro[-1]], to - to[0], a["T"][to[0]:to[-1]],
                                           fo - fo[0], a["F"][fo[0]:fo[-1]], yo, a["Y2"][lo:hi])


def oracle_rate_1thread(kind, a, n):
    """(units per second, outputs) of one single-thread oracle call on units [0, n)."""
    t0 = time.perf_counter()
    res = _oracle_call(kind, a, 0, n)
    return n / max(time.perf_counter() - t0, 1e-9), res


def sample_parity(kind, res, snap):
    """Oracle outputs on units [0, n) against the GPU's outputs there:
    indices bit-exact, values within REL_TOL relative."""
    if snap is None:
        return None
    if kind in ("1d", "1d_batched"):
        n = len(res)
        bad = int(np.count_nonzero(np.asarray(snap[:n]) != res))
        return {"units": n, "index_mismatches": bad, "ok": bad == 0}
    idx, val = res
    n = len(val)
    gi, gv = np.asarray(snap[0][:n]), np.asarray(snap[1][:n])
    bad = int(np.count_nonzero((gi != idx).any(axis=1)))
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.abs(gv - val) / np.abs(val)
    both_nan = np.isnan(gv) & np.isnan(val)
    rel = np.where(both_nan, 0.0, rel)
    worst = float(np.nanmax(rel)) if n else 0.0
    if np.isnan(rel).any():
        worst = float("inf")
    return {"units": n, "index_mismatches": bad, "max_rel_err": worst, "rel_tol": REL_TOL,
            "ok": bad == 0 and worst <= REL_TOL}


class OracleTimer:
    """Runs the oracle on a sample in one thread, and split over one thread
    per host core.  The oracle is C called through ctypes, which releases the
    interpreter lock for the call, so the threads run in parallel on shared
    arrays (no copies, no processes)."""

    def __init__(self):
        from concurrent.futures import ThreadPoolExecutor
        self.cores = os.cpu_count() or 1
        self.pool = ThreadPoolExecutor(self.cores)

    def parallel(self, kind, a, n):
        cuts = np.linspace(0, n, self.cores + 1).astype(np.int64)
        parts = [(int(cuts[i]), int(cuts[i + 1])) for i in range(self.cores) if cuts[i + 1] > cuts[i]]
        t0 = time.perf_counter()
        list(self.pool.map(lambda r: _oracle_call(kind, a, r[0], r[1]), parts))
        return n / max(time.perf_counter() - t0, 1e-9)

    def baseline_on(self, kind, a, n, desc, snap, reps=3):
        """cpu_baseline: all host cores (median of reps) on the sample, plus
        the single-thread rate; the single-thread outputs are checked against
        the GPU's outputs at the same units (snap)."""
        one, res = oracle_rate_1thread(kind, a, n)
        par = statistics.median([self.parallel(kind, a, n) for _ in range(reps)])
        return {"value": par / 1e9, "unit": UNIT, "cores": self.cores, "kind": "oracle",
                "sample": "%s, split over %d threads" % (desc, self.cores),
                "single_thread": {"value": one / 1e9, "cores": 1},
                "parity": sample_parity(kind, res, snap)}

    def close(self):
        self.pool.shutdown()


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
SNAP_MAX = 1 << 28          # most units whose GPU outputs are copied back for the parity sample


class Workload:
    name = ""
    kernel = ""               # dominant kernel (ncu name)
    bytes_per_target = 0      # algorithmic HBM bytes per target
    side = 0                  # 0: largest entry < target (default), 1: <= (SS_SIDE_LE)
    share = None              # (rank, world) under strong scaling: this rank's part of one workload
    snap = None               # GPU outputs of the oracle sample, taken right after the timed region
    flush = None              # buffer written between timed steps when the inputs fit in L2

    def setup(self, dev, seed):
        raise NotImplementedError

    def step(self):
        raise NotImplementedError

    def targets(self):
        raise NotImplementedError

    def release(self):
        """Drop every tensor and plan of this workload (the next one needs the memory)."""
        for k in list(vars(self)):
            if k not in ("name", "kernel", "m", "side", "share", "pairs", "coherent", "per_table", "model",
                         "autotune", "tile", "algo", "g"):
                setattr(self, k, None)
        import gc
        gc.collect()
        torch.cuda.empty_cache()


class Interp2D(Workload):
    """Fused 2D search + bilinear: 200 x 100 axes, 64M (rho, T) pairs (one table)."""
    name = "interp2d-200x100-64M"
    kernel = "k_search_interp_2d_sg"     # the grid fits shared memory: the staged-grid variant runs
    bytes_per_target = 16 + 8 + 8      # pair in, index pair out, value out

    def __init__(self, m=64 << 20):
        self.m = m

    def setup(self, dev, seed):
        from paper_2112_03229_gb300 import workloads as wl
        import paper_2112_03229_gb300 as ss
        self.ss = ss
        self.R, self.T, self.F, self.Y2 = wl.interp_2d(m=self.m, seed=2 + 1000 * seed, device=dev)
        self.idx = torch.empty((self.m, 2), dtype=torch.int32, device=dev)
        self.val = torch.empty((self.m,), dtype=torch.float64, device=dev)

    def step(self):
        self.ss.search_interp_2d(self.R, self.T, self.F, self.Y2, idx=self.idx, val=self.val)
        return 1

    def targets(self):
        return self.m

    def e2e_setup(self):
        """Host arrays (page-locked) through ss_search_interp_2d_host, which
        pipelines the copies and the search inside the library."""
        self.hY = torch.empty(self.Y2.shape, dtype=torch.float64, pin_memory=True)
        self.hY.copy_(self.Y2)
        self.hI = torch.empty(self.idx.shape, dtype=torch.int32, pin_memory=True)
        self.hV = torch.empty(self.val.shape, dtype=torch.float64, pin_memory=True)
        self.hR, self.hT, self.hF = self.R.cpu(), self.T.cpu(), self.F.cpu()
        return self.hY.numel() * 8, self.hI.numel() * 4 + self.hV.numel() * 8

    def e2e_step(self):
        self.ss.search_interp_2d_host(self.hR, self.hT, self.hF, self.hY, idx=self.hI, val=self.hV)

    def sample(self, ns):
        """Oracle inputs for the first ns pairs (same table)."""
        ns = int(min(ns, self.m))
        a = {"R": self.R.cpu().numpy(), "T": self.T.cpu().numpy(), "F": self.F.cpu().numpy(),
             "Y2": self.Y2[:ns].cpu().numpy()}
        return "2d", a, ns, "first %d of the %d pairs (same tables)" % (ns, self.m)

    def snapshot(self, ns):
        return self.idx[:ns].cpu().numpy(), self.val[:ns].cpu().numpy()


class Plain1D(Workload):
    """One 64-entry table, 1B float64 targets (bucket search)."""
    name = "plain1d-n64-1B"
    kernel = "k_search_1d_bucket"
    bytes_per_target = 8 + 4

    def __init__(self, m=1 << 30, algo="auto"):
        self.m, self.algo, self.g = m, algo, 0

    def set_algo(self, name):
        kern = {"auto": "bucket", "ballot8": "ballot", "ballot16": "ballot"}.get(name, name)
        self.kernel = "k_search_1d_" + kern
        self.algo = "ballot" if name.startswith("ballot") else name
        self.g = {"ballot8": 8, "ballot16": 16, "ballot": 32}.get(name, 0)
        self.name = "plain1d-n64-1B-" + name

    def setup(self, dev, seed):
        from paper_2112_03229_gb300 import workloads as wl
        import paper_2112_03229_gb300 as ss
        from paper_2112_03229_gb300 import partition
        self.ss = ss
        if self.share is None:
            self.X, self.Y = wl.plain_1d(m=self.m, seed=1 + 1000 * seed, device=dev)
        else:
            # strong scaling: every rank draws the same targets and keeps its contiguous slice
            rank, world = self.share
            X, Y = wl.plain_1d(m=self.m, seed=1, device=dev)
            a, b = partition.target_slice(self.m, world, rank)
            self.X, self.Y = X, Y[a:b].clone()
            del Y
        self.out = torch.empty(self.Y.shape, dtype=torch.int32, device=dev)

    def step(self, side=None):
        self.ss.search_1d(self.X, self.Y, out=self.out, algo=self.algo, ballot_g=self.g,
                          side=self.side if side is None else side)
        return 1

    def targets(self):
        return int(self.Y.numel())

    def e2e_setup(self):
        """Host arrays (page-locked) through ss_search_1d_host."""
        self.hY = torch.empty(self.Y.shape, dtype=torch.float64, pin_memory=True)
        self.hY.copy_(self.Y)
        self.hO = torch.empty(self.out.shape, dtype=torch.int32, pin_memory=True)
        self.hX = self.X.cpu()
        return self.hY.numel() * 8, self.hO.numel() * 4

    def e2e_step(self):
        self.ss.search_1d_host(self.hX, self.hY, out=self.hO, algo=self.algo)

    def sample(self, ns):
        ns = int(min(ns, self.targets()))
        a = {"X": self.X.cpu().numpy(), "Y": self.Y[:ns].cpu().numpy(), "side": self.side}
        return "1d", a, ns, "first %d of the %d targets (same table)" % (ns, self.targets())

    def snapshot(self, ns):
        return self.out[:ns].cpu().numpy()


class Plain1DSmall(Plain1D):
    """The 64-entry table with 1M targets as stated (the whole working set,
    12 MB, fits in L2): a 256 MB buffer is written between timed steps so
    that every step reads its targets from HBM."""
    name = "plain1d-n64-1M"

    def __init__(self):
        super().__init__(m=1 << 20)

    def setup(self, dev, seed):
        super().setup(dev, seed)
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)


def _per_table_sample(Y_off, ns):
    """Per table k, the first q_k of its targets, q_k proportional to its
    count (at least one for a table that has targets): a sample of about ns
    units that reaches every table.  Returns (start_k, q_k) arrays."""
    Y_off = np.asarray(Y_off, dtype=np.int64)
    cnt = np.diff(Y_off)
    total = int(cnt.sum())
    if total == 0:
        return Y_off[:-1], np.zeros_like(cnt)
    q = np.where(cnt > 0, np.maximum(1, np.floor(cnt * (ns / total))), 0).astype(np.int64)
    return Y_off[:-1], np.minimum(q, cnt)


def _gather(t, starts, q):
    """The rows [starts[k], starts[k] + q[k]) of t for every k, back to back."""
    parts = [t[int(s):int(s) + int(c)] for s, c in zip(starts, q) if c > 0]
    return torch.cat(parts) if parts else t[:0]


class PlanWorkload(Workload):
    """Common driver of the plan-based workloads: tables prepared once (not
    timed; Sec. 5.3 set-up), then each step is one graph launch of the
    persistent batched kernel over the bound batch."""
    kernel = "k_batched_1d"
    bytes_per_target = 8 + 4
    model = "none"
    compare_models = ("spline", "mlp", "loghash")     # timed beside the plain search

    def __init__(self, model=None, autotune=True):
        if model is not None:
            self.model = model
        self.autotune = autotune
        self.plans = {}

    tile = 0

    def make_plan(self, model, side=None):
        import paper_2112_03229_gb300 as ss
        side = self.side if side is None else side
        return ss.Plan.create_1d(self.b.X_off, self.b.X_dev, model=model, autotune=self.autotune, tile=self.tile,
                                 side=side, tune_cache=os.path.join(ROOT, "_build", "tune_%s_%s_%d.json"
                                                                    % (self.name, model, side)))

    def setup(self, dev, seed):
        import paper_2112_03229_gb300 as ss
        self.ss = ss
        if self.share is None:
            self.b = self.generate(dev, seed)
        else:
            # strong scaling: every rank draws the same batch and keeps the
            # tables that the longest-processing-time split gives it
            rank, world = self.share
            full = self.generate(dev, 0)
            self.b, self.tables = share_of_batch(full, world, rank)
            del full
        self.b.X_dev = self.b.X.to(dev)
        self.Y = self.b.Y.to(dev)
        self.out = torch.empty(self.Y.shape, dtype=torch.int32, device=dev)
        t0 = time.perf_counter()
        self.plan = self.make_plan(self.model)
        self.plan.bind_1d(self.b.Y_off, self.Y, self.out)
        torch.cuda.synchronize()
        self.setup_s = time.perf_counter() - t0

    def step(self):
        self.plan.execute()
        return self.kernels_per_step

    @property
    def kernels_per_step(self):
        """Kernels in the bound graph (read once; the binding used for timing does not change)."""
        if getattr(self, "_kps", None) is None:
            self._kps = self.plan.info().kernels
        return self._kps

    def targets(self):
        return int(self.b.Y_off[-1])

    def bind(self, plan):
        plan.bind_1d(self.b.Y_off, self.Y, self.out)

    def setup_reference(self, max_targets):
        """CPU-only inputs for the oracle arm: the first tables of the batch."""
        self.b = self.generate("cpu", 0, max_targets=max_targets)
        self.Y = self.b.Y

    def compare(self, stream, steps, model, side=None):
        """A plan with another position model (or none, or the other side) on
        the same bound batch, timed the same way."""
        other = self.make_plan(model, side)
        self.bind(other)
        for _ in range(3):
            other.execute()
        torch.cuda.synchronize()
        ms = time_loop(other.execute, stream, steps)[1]
        inf = other.info()
        res = {"model": model, "Gtargets_s": round(self.targets() / (ms / 1e3) / 1e9, 3),
               "ms_per_step": round(ms, 4), "choices": other.choices(), "max_window": inf.max_window,
               "mean_window": round(inf.mean_window, 2), "train_loss": inf.train_loss}
        if inf.kind == 2:
            res["lean_kernel"] = inf.lean_kernel
        self.bind(self.plan)
        del other
        return res

    def e2e_setup(self):
        """The plan bound to page-locked host buffers: each step's kernel reads
        the targets from host memory and writes the indices back there."""
        self.hY = torch.empty(self.Y.shape, dtype=torch.float64, pin_memory=True)
        self.hY.copy_(self.Y)
        self.hO = torch.empty(self.out.shape, dtype=torch.int32, pin_memory=True)
        self.plan.bind_1d(self.b.Y_off, self.hY, self.hO)
        return self.hY.numel() * 8, self.hO.numel() * 4

    def e2e_step(self):
        self.plan.execute()

    def e2e_finish(self):
        self.bind(self.plan)
        self.hY = self.hO = None

    def _sel(self, ns):
        if getattr(self, "_selection", None) is None or self._selection[0] != ns:
            self._selection = (ns,) + _per_table_sample(self.b.Y_off.cpu().numpy(), ns)
        return self._selection[1:]

    def sample(self, ns):
        """Oracle inputs: the first q_k targets of every table k (about ns in all)."""
        starts, q = self._sel(ns)
        yo = np.concatenate([[0], np.cumsum(q)]).astype(np.int64)
        a = {"X_off": self.b.X_off.cpu().numpy(), "X": self.b.X.cpu().numpy(), "Y_off": yo,
             "Y": _gather(self.Y, starts, q).cpu().numpy(), "side": self.side}
        n = int(yo[-1])
        return "1d_batched", a, n, "first %d targets of every table by its share (%d of %d targets, %d tables)" % (
            int(q.max()) if len(q) else 0, n, self.targets(), int(np.count_nonzero(q)))

    def snapshot(self, ns):
        starts, q = self._sel(ns)
        return _gather(self.out, starts, q).cpu().numpy()


def share_of_batch(b, world, rank):
    """Rank's tables of a 1D batch under the longest-processing-time split
    (partition.lpt_tables on the target counts): (the sub-batch with rebased
    offsets, the indices of its tables in the full batch)."""
    from paper_2112_03229_gb300 import partition
    from paper_2112_03229_gb300 import workloads as wl
    X_off, Y_off = b.X_off.cpu().numpy(), b.Y_off.cpu().numpy()
    tables = partition.lpt_tables(np.diff(Y_off), world)[rank]
    xo = np.concatenate([[0], np.cumsum(np.diff(X_off)[tables])]).astype(np.int64)
    yo = np.concatenate([[0], np.cumsum(np.diff(Y_off)[tables])]).astype(np.int64)
    X = _gather(b.X, X_off[tables], np.diff(X_off)[tables])
    Y = _gather(b.Y, Y_off[tables], np.diff(Y_off)[tables]).clone()
    return wl.Batched1D(torch.as_tensor(xo), X.cpu(), torch.as_tensor(yo), Y, None, None), tables


class Batched1D(PlanWorkload):
    """Two independent batches of 10,000 tables each (sizes log-uniform
    20..2000, Zipf(1.1) target counts on [1e3, 1e6]): a 10,000-table batch
    holds about 1.1B targets, so the second brings the total to the stated
    "about 2B" (2.2B) without distorting the count law; one persistent graph
    launch over all 20,000 tables, learned proposals vs plain.  --targets
    scales the counts (profiling cases)."""
    name = "batched1d-10k-zipf-x2"
    m = 0

    def generate(self, dev, seed, max_targets=None):
        from paper_2112_03229_gb300 import workloads as wl
        scale = self.m / 2.2e9 if self.m else 1.0
        if max_targets is not None:      # a prefix of the batch: the first tables only
            return wl.batched_1d(ntables=10_000, seed=5 + 1000 * seed, count_scale=scale, device=dev,
                                 max_targets=max_targets)
        return wl.batched_1d_x2(seed=5 + 1000 * seed, count_scale=scale, device=dev)


class Sweep1D(PlanWorkload):
    """Table-size sweep: clustered tables of 16, 256, 4096 and 65536 entries,
    256M log-uniform targets per table, learned proposals vs plain."""
    name = "sweep1d-16-65536-256M"
    m = 0                  # --targets: total targets of a smaller case (profiling)

    def __init__(self, per_table=256 << 20, **kw):
        super().__init__(**kw)
        self.per_table = per_table

    def generate(self, dev, seed, max_targets=None):
        from paper_2112_03229_gb300 import workloads as wl
        tabs = [wl.sweep_table(n, seed=4 + 1000 * seed) for n in (16, 256, 4096, 65536)]
        per = (self.m // 4 if self.m else self.per_table) if max_targets is None else max(1, max_targets // 4)
        Ys = [wl.log_uniform(per, 0.5 * t[0].item(), 2 * t[-1].item(), seed=7 + i + 1000 * seed,
                             device=dev) for i, t in enumerate(tabs)]
        X = torch.cat(tabs)
        X_off = torch.tensor(np.concatenate([[0], np.cumsum([len(t) for t in tabs])]))
        Y_off = torch.tensor(np.concatenate([[0], np.cumsum([len(y) for y in Ys])]))
        return wl.Batched1D(X_off, X, Y_off, torch.cat(Ys), None, None)


class Coherent1D(Sweep1D):
    """Hunt and locate's regime (Sec. 2.1, 5.5): jittered log-spaced tables of
    64, 4096, 65536 and 1M entries (the last searched in global memory), 64M
    coherent targets per table (a random walk in log space, N(0, 0.01
    decade) steps); plain search vs the hunt and the learned proposals."""
    name = "coherent1d-64-1M-64M"
    table_models = ("none", "hunt", "spline", "loghash")
    compare_models = ("hunt", "spline", "loghash", "auto")
    sizes = (64, 4096, 65536, 1 << 20)

    def __init__(self, per_table=64 << 20, **kw):
        super().__init__(per_table=per_table, **kw)

    def generate(self, dev, seed, max_targets=None):
        from paper_2112_03229_gb300 import workloads as wl
        tabs = [wl.log_spaced_table(n, 1e-6, 1e4, 0.1, seed=8 + n + 1000 * seed) for n in self.sizes]
        per = (self.m // 4 if self.m else self.per_table) if max_targets is None else max(1, max_targets // 4)
        Ys = [wl.walk_1d(per, 0.5e-6, 2e4, seed=9 + i + 1000 * seed, device=dev) for i in range(len(tabs))]
        X = torch.cat(tabs)
        X_off = torch.tensor(np.concatenate([[0], np.cumsum([len(t) for t in tabs])]))
        Y_off = torch.tensor(np.concatenate([[0], np.cumsum([len(y) for y in Ys])]))
        return wl.Batched1D(X_off, X, Y_off, torch.cat(Ys), None, None)


class Large1D(Sweep1D):
    """Tables too large for shared memory in any layout (262,144, 1M and 4M
    entries, jittered log spacing): the plain search finishes in the full
    keys in global memory with dependent loads, where a position proposal
    with a small window needs one; 64M log-uniform targets per table."""
    name = "large1d-256K-4M-64M"
    sizes = (1 << 18, 1 << 20, 1 << 22)
    table_models = ("none", "spline", "mlp", "loghash")
    compare_models = ("spline", "mlp", "loghash", "auto")

    def __init__(self, per_table=64 << 20, **kw):
        super().__init__(per_table=per_table, **kw)

    def generate(self, dev, seed, max_targets=None):
        from paper_2112_03229_gb300 import workloads as wl
        tabs = [wl.log_spaced_table(n, 1e-6, 1e4, 0.1, seed=10 + n + 1000 * seed) for n in self.sizes]
        per = (self.m // len(tabs) if self.m else self.per_table) if max_targets is None else \
            max(1, max_targets // len(tabs))
        Ys = [wl.log_uniform(per, 0.5e-6, 2e4, seed=11 + i + 1000 * seed, device=dev) for i in range(len(tabs))]
        X = torch.cat(tabs)
        X_off = torch.tensor(np.concatenate([[0], np.cumsum([len(t) for t in tabs])]))
        Y_off = torch.tensor(np.concatenate([[0], np.cumsum([len(y) for y in Ys])]))
        return wl.Batched1D(X_off, X, Y_off, torch.cat(Ys), None, None)


def sweep_per_table(wl_obj, stream, steps):
    """Per-table Gtargets/s of the sweep: one plan per table and model."""
    import paper_2112_03229_gb300 as ss
    b = wl_obj.b
    X_off, Y_off = b.X_off.tolist(), b.Y_off.tolist()
    res = {}
    for k in range(len(X_off) - 1):
        X = b.X_dev[X_off[k]:X_off[k + 1]]
        Y = wl_obj.Y[Y_off[k]:Y_off[k + 1]]
        out = wl_obj.out[Y_off[k]:Y_off[k + 1]]
        row = {}
        for model in getattr(wl_obj, "table_models", ("none", "spline", "mlp", "loghash")):
            plan = ss.Plan.create_1d([0, X.numel()], X, model=model, autotune=(model in ("none", "hunt")))
            plan.bind_1d([0, Y.numel()], Y, out)
            for _ in range(3):
                plan.execute()
            torch.cuda.synchronize()
            # three repetitions of the timed loop: the rate is their median,
            # and the spread between them is reported beside it
            rates = sorted(Y.numel() / (time_loop(plan.execute, stream, steps)[1] / 1e3) / 1e9 for _ in range(3))
            inf = plan.info()
            row[model] = {"Gtargets_s": round(rates[1], 2), "min_max": [round(rates[0], 2), round(rates[2], 2)],
                          "window": inf.max_window, "algo": list(plan.choices().values())[0][0]}
            del plan
        res[str(X.numel())] = row
    wl_obj.bind(wl_obj.plan)
    return res


class Batched2D(PlanWorkload):
    """1,000 2D tables (axes U{50..500} x U{30..300}), 1M (rho, T) pairs each
    (1B pairs), learned proposals on both axes and the coherent hunt vs plain."""
    name = "batched2d-1000-1B"
    kernel = "k_batched_2d_fast"     # every axis of this batch takes the lean kernel's path
    compare_models = ("spline", "mlp", "loghash", "hunt")
    bytes_per_target = 16 + 8 + 8
    m = 0                  # --targets: total pairs of a smaller case (profiling)

    def __init__(self, coherent=False, pairs=1_000_000, **kw):
        super().__init__(**kw)
        self.coherent = coherent
        self.pairs = pairs
        if coherent:
            self.name = "batched2d-1000-1B-coherent"

    def make_plan(self, model, side=None):
        import paper_2112_03229_gb300 as ss
        b = self.b
        return ss.Plan.create_2d(b.R_off, b.R_dev, b.T_off, b.T_dev, b.F_off, b.F_dev, model=model,
                                 autotune=self.autotune, tile=self.tile,
                                 tune_cache=os.path.join(ROOT, "_build", "tune_%s_%s.json" % (self.name, model)))

    def setup(self, dev, seed):
        import paper_2112_03229_gb300 as ss
        from paper_2112_03229_gb300 import workloads as wl
        self.ss = ss
        per = self.m // 1000 if self.m else self.pairs
        b = wl.batched_2d(ntables=1000, pairs_per_table=per, coherent=self.coherent, seed=6 + 1000 * seed,
                          device=dev)
        b.R_dev, b.T_dev, b.F_dev = b.R.to(dev), b.T.to(dev), b.F.to(dev)
        self.b = b
        self.Y = b.Y2
        self.m = b.Y2.shape[0]
        self.idx = torch.empty((self.m, 2), dtype=torch.int32, device=dev)
        self.val = torch.empty(self.m, dtype=torch.float64, device=dev)
        t0 = time.perf_counter()
        self.plan = self.make_plan(self.model)
        self.plan.bind_2d(b.Y_off, self.Y, self.idx, self.val)
        torch.cuda.synchronize()
        self.setup_s = time.perf_counter() - t0

    def bind(self, plan):
        plan.bind_2d(self.b.Y_off, self.Y, self.idx, self.val)

    def setup_reference(self, max_targets):
        from paper_2112_03229_gb300 import workloads as wl
        nt = max(1, min(1000, max_targets // self.pairs))
        self.b = wl.batched_2d(ntables=nt, pairs_per_table=self.pairs, coherent=self.coherent, seed=6, device="cpu")
        self.Y = self.b.Y2

    def e2e_setup(self):
        """The plan bound to page-locked host buffers (pairs in, index pairs and values out)."""
        self.hY = torch.empty(self.Y.shape, dtype=torch.float64, pin_memory=True)
        self.hY.copy_(self.Y)
        self.hI = torch.empty(self.idx.shape, dtype=torch.int32, pin_memory=True)
        self.hV = torch.empty(self.val.shape, dtype=torch.float64, pin_memory=True)
        self.plan.bind_2d(self.b.Y_off, self.hY, self.hI, self.hV)
        return self.hY.numel() * 8, self.hI.numel() * 4 + self.hV.numel() * 8

    def e2e_finish(self):
        self.bind(self.plan)
        self.hY = self.hI = self.hV = None

    def sample(self, ns):
        """Oracle inputs: the first q_k pairs of every table k (about ns in all)."""
        b = self.b
        starts, q = self._sel(ns)
        yo = np.concatenate([[0], np.cumsum(q)]).astype(np.int64)
        a = {"R_off": b.R_off.cpu().numpy(), "R": b.R.cpu().numpy(), "T_off": b.T_off.cpu().numpy(),
             "T": b.T.cpu().numpy(), "F_off": b.F_off.cpu().numpy(), "F": b.F.cpu().numpy(), "Y_off": yo,
             "Y2": _gather(self.Y, starts, q).cpu().numpy()}
        n = int(yo[-1])
        return "2d_batched", a, n, "first %d pairs of every table (%d of %d pairs, %d tables)" % (
            int(q.max()) if len(q) else 0, n, self.targets(), int(np.count_nonzero(q)))

    def snapshot(self, ns):
        starts, q = self._sel(ns)
        return _gather(self.idx, starts, q).cpu().numpy(), _gather(self.val, starts, q).cpu().numpy()


class Interp2DPlan(Batched2D):
    """The 200 x 100 table of the fused 2D lookup with its 64M pairs, run
    through a plan (one table, persistent launch, corner records in global
    memory) instead of the one-shot call that stages the grid per block."""
    name = "interp2d-200x100-64M-plan"

    def __init__(self, **kw):
        super().__init__(**kw)
        self.m = 0

    def setup(self, dev, seed):
        import paper_2112_03229_gb300 as ss
        from paper_2112_03229_gb300 import workloads as wl
        self.ss = ss
        m = self.m or (64 << 20)
        R, T, F, Y2 = wl.interp_2d(m=m, seed=2 + 1000 * seed, device=dev)
        off = lambda n: torch.tensor([0, n], dtype=torch.int64)
        b = wl.Batched2D(off(len(R)), R.cpu(), off(len(T)), T.cpu(), off(F.numel()), F.reshape(-1).cpu(), off(m), Y2)
        b.R_dev, b.T_dev, b.F_dev = R, T, F.reshape(-1)
        self.b = b
        self.Y = Y2
        self.m = m
        self.idx = torch.empty((m, 2), dtype=torch.int32, device=dev)
        self.val = torch.empty(m, dtype=torch.float64, device=dev)
        t0 = time.perf_counter()
        self.plan = self.make_plan(self.model)
        self.plan.bind_2d(b.Y_off, self.Y, self.idx, self.val)
        torch.cuda.synchronize()
        self.setup_s = time.perf_counter() - t0


WORKLOADS = {
    "interp2d": Interp2D,
    "plain1d": Plain1D,
    "plain1d-1m": Plain1DSmall,
    "batched1d": Batched1D,
    "sweep1d": Sweep1D,
    "batched2d": Batched2D,
    "batched2d-coherent": lambda: Batched2D(coherent=True),
    "coherent1d": Coherent1D,
    "large1d": Large1D,
    "interp2d-plan": Interp2DPlan,
}
DEFAULT_WORKLOAD = "batched1d"
# every configuration of the benchmark suite, in the order the default run
# measures them after the headline: (key, stated configuration)
SUITE = (
    ("plain1d-1m", "plain 1D search, 64-entry table, 1M targets (L2 flushed between steps)"),
    ("plain1d", "plain 1D search, 64-entry table, scaled to 1B targets (the >= 70% roofline bar)"),
    ("interp2d", "fused 2D search + bilinear, 200 x 100 axes, 64M pairs"),
    ("interp2d-plan", "the same 200 x 100 table and 64M pairs through a plan (corner records, persistent launch)"),
    ("sweep1d", "table-size sweep 16 / 256 / 4096 / 65536 entries, 256M targets each, learned vs plain"),
    ("batched2d", "1,000 2D tables, 1B pairs, random order, learned and hunt vs plain"),
    ("batched2d-coherent", "1,000 2D tables, 1B pairs, coherent order, learned and hunt vs plain"),
    ("coherent1d", "hunt and locate's regime: 64 .. 1M-entry tables, 64M coherent targets each, hunt vs plain"),
    ("large1d", "tables searched in global memory (256K .. 4M entries), 64M targets each, learned vs plain"),
)


# ---------------------------------------------------------------------------
# Timing
# ---------------------------------------------------------------------------
def time_loop(fn, stream, steps, flush=None):
    """Runs fn `steps` times on `stream` with CUDA events around every call.
    Returns (ms of the whole region, mean ms per call, calls' return values
    summed).  With `flush`, that buffer is written before every call, outside
    the per-call events; the region then counts the calls only."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    count = 0
    t0.record(stream)
    for i in range(steps):
        if flush is not None:
            flush.add_(1)
        starts[i].record(stream)
        count += fn() or 0
        ends[i].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total = sum(per) if flush is not None else t0.elapsed_time(t1)
    return total, statistics.mean(per), count


# ---------------------------------------------------------------------------
def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_over_ranks(x, world, op="max"):
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return t.item()


def max_over_ranks(x, world):
    return reduce_over_ranks(x, world, "max")


def sample_size(wl_obj, budget_s):
    """Units of the oracle sample: about budget_s seconds of single-thread
    oracle work, from the oracle's rate on a small probe sample."""
    kind, a, n, _ = wl_obj.sample(1 << 18)
    oracle_rate_1thread(kind, a, min(n, 1024))       # first call loads the oracle library
    rate, _ = oracle_rate_1thread(kind, a, n)
    return int(max(1 << 18, min(rate * budget_s, SNAP_MAX, wl_obj.targets())))


def run_reference(args, wl_obj):
    """Oracle arm: the plain CPU oracle on host cores, a bounded sample per step."""
    rank, world, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    # build the workload's inputs on the CPU at a bounded size (a prefix of the same workload)
    if isinstance(wl_obj, PlanWorkload):
        wl_obj.setup_reference(max_targets=1 << 24)
    else:
        wl_obj.m = min(wl_obj.m, 1 << 23)
        wl_obj.setup("cpu", 0)
    timer = OracleTimer()
    kind, a, n, desc = wl_obj.sample(sample_size(wl_obj, 4.0))
    rates = [timer.parallel(kind, a, n) for _ in range(args.warmup + args.steps)][args.warmup:]
    timer.close()
    value = statistics.median(rates) / 1e9
    sample = "%s, split over %d threads" % (desc, timer.cores)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": n / (value * 1e9) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl_obj.name},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": timer.cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def latency_table(dev):
    """Per-call latency for small batches (the set-up-dominated regime of
    Sec. 5.1 / 5.3): one-shot call (no set-up kept) vs a prepared plan
    replayed as a CUDA graph, on the 64-entry table; medians of 50 calls,
    each timed on the host including its synchronisation."""
    import paper_2112_03229_gb300 as ss
    from paper_2112_03229_gb300 import workloads as wl
    X, Y = wl.plain_1d(m=1 << 20, seed=1, device=dev)
    res = {}
    for m in (1, 100, 10_000, 1_000_000):
        y = Y[:m].contiguous()
        out = torch.empty(m, dtype=torch.int32, device=dev)
        plan = ss.Plan.create_1d([0, X.numel()], X)
        plan.bind_1d([0, m], y, out)
        row = {}
        for name, fn in (("one_shot", lambda: ss.search_1d(X, y, out=out)), ("plan_graph", plan.execute)):
            for _ in range(5):
                fn()
            torch.cuda.synchronize()
            ts = []
            for _ in range(50):
                t0 = time.perf_counter()
                fn()
                torch.cuda.synchronize()
                ts.append((time.perf_counter() - t0) * 1e6)
            row[name + "_us"] = round(statistics.median(ts), 2)
        res[str(m)] = row
        del plan
    return res


def small_m_latency(args):
    import __graft_entry__
    __graft_entry__.build()
    res = latency_table(torch.device("cuda", 0))
    print(json.dumps({"metric": "per-call latency (us), small target batches", "unit": "us", "n_gpus": 1,
                      "config": {"workload": "latency-n64", "table": 64}, "latency": res}), flush=True)


def measure(wl_obj, args, stream, world, cpu_budget, e2e_steps):
    """One configuration: W warm-up steps, K timed steps (per-step CUDA
    events on the launching stream, barrier and synchronise on both sides,
    max over ranks), the GPU outputs of the oracle sample copied back, then
    the end-to-end rate through the public API with host buffers."""
    ns = sample_size(wl_obj, cpu_budget) if cpu_budget else 0
    for _ in range(args.warmup):
        wl_obj.step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    total_ms, per_ms, launches = time_loop(wl_obj.step, stream, args.steps, flush=wl_obj.flush)
    barrier(world)
    total_ms = max_over_ranks(total_ms, world)
    mine = wl_obj.targets()
    units = reduce_over_ranks(float(mine), world, "sum") if wl_obj.share is not None else mine * world
    value = units * args.steps / (total_ms / 1e3) / 1e9
    if ns:
        wl_obj.sample_n = ns
        wl_obj.snap = wl_obj.snapshot(ns)
    peak, peak_kind = hbm_peak()
    achieved = mine * wl_obj.bytes_per_target / (per_ms / 1e3) / 1e9
    rec = {"value": round(value, 3), "ms_per_step": round(total_ms / args.steps, 4),
           "ms_per_launch": round(per_ms, 4), "targets_per_gpu": mine, "gpu_launches": launches,
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                        "traffic": recorded_traffic(wl_obj.kernel, wl_obj.name), "kernel": wl_obj.kernel,
                        "algorithmic_bytes_per_target": wl_obj.bytes_per_target}}
    if e2e_steps:
        h2d, d2h = wl_obj.e2e_setup()
        for _ in range(2):
            wl_obj.e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            wl_obj.e2e_step()
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, world)
        e2e_value = units * e2e_steps / (e2e_ms / 1e3) / 1e9
        rec["e2e"] = {"value": round(e2e_value, 3), "unit": UNIT,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps}
        if world == 1:
            # the same algorithmic bytes cross the host link: in and out in flight together
            link = host_link_peak(torch.device("cuda", torch.cuda.current_device()))
            moved = e2e_value * 1e9 * (h2d + d2h) / max(mine, 1) / 1e9
            peak = link_peak_for(h2d, d2h, link)
            rec["e2e"]["roofline"] = {"bound": "host link", "achieved": round(moved, 1), "peak": round(peak, 1),
                                      "unit": "GB/s", "frac": round(moved / peak, 4),
                                      "peak_source": "page-locked copies measured in this run (each direction "
                                                     "alone and both at once, best of 3), at this step's split "
                                                     "of bytes between the directions", "copies_GBs": dict(link)}
        if hasattr(wl_obj, "e2e_finish"):
            wl_obj.e2e_finish()
    return rec


_LINK = {}


def link_peak_for(h2d, d2h, link):
    """Total GB/s the host link can carry for a step that sends h2d bytes to
    the device and d2h bytes back with both directions in flight: each
    direction's own copy rate and the rate of both together bound the step
    time, and the slowest of the three decides (a 1D step sends twice the
    bytes it returns, so its host-to-device direction is the bound)."""
    if h2d + d2h <= 0:
        return float(link.get("both", 0.0))
    t = max(h2d / link["h2d"] if h2d else 0.0, d2h / link["d2h"] if d2h else 0.0, (h2d + d2h) / link["both"])
    return (h2d + d2h) / t


def host_link_peak(dev, nbytes=1 << 30, reps=3):
    """Host link copy rates (GB/s) measured here: page-locked host to device,
    device to host, and both at once on two streams (what an end-to-end step
    does: targets in and answers out in flight together); best of reps."""
    if _LINK:
        return _LINK
    h_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h_out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d_in = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d_out = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    best = {"h2d": 0.0, "d2h": 0.0, "both": 0.0}
    for _ in range(reps):
        for kind in ("h2d", "d2h", "both"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if kind in ("h2d", "both"):
                with torch.cuda.stream(s1):
                    d_in.copy_(h_in, non_blocking=True)
            if kind in ("d2h", "both"):
                with torch.cuda.stream(s2):
                    h_out.copy_(d_out, non_blocking=True)
            torch.cuda.synchronize()
            moved = nbytes * (2 if kind == "both" else 1)
            best[kind] = max(best[kind], moved / (time.perf_counter() - t0) / 1e9)
    _LINK.update({k: round(v, 1) for k, v in best.items()})
    del h_in, h_out, d_in, d_out
    return _LINK


def frac_of(wl_obj, ms):
    peak, _ = hbm_peak()
    return round(wl_obj.targets() * wl_obj.bytes_per_target / (ms / 1e3) / 1e9 / peak, 4)


def other_forms(wl_obj, stream, steps, value):
    """Beside the timed plain search on the same inputs: the learned
    proposals (and the hunt, for 2D plans) and the '<=' side."""
    extra = {}
    if isinstance(wl_obj, PlanWorkload):
        inf = wl_obj.plan.info()
        extra["plan"] = {"model": wl_obj.model, "setup_s": round(wl_obj.setup_s, 2), "choices": wl_obj.plan.choices(),
                         "max_window": inf.max_window, "mean_window": round(inf.mean_window, 2),
                         "train_loss": inf.train_loss, "ntiles": inf.ntiles}
        if wl_obj.model == "none":
            learned = {}
            models = wl_obj.compare_models
            for model in models:
                r = wl_obj.compare(stream, steps, model)
                r["frac"] = frac_of(wl_obj, r["ms_per_step"])
                learned[model] = r
            extra["learned"] = learned
            extra["learned_over_plain"] = {k: round(v["Gtargets_s"] / value, 3) for k, v in learned.items()}
        else:
            r = wl_obj.compare(stream, steps, "none")
            r["frac"] = frac_of(wl_obj, r["ms_per_step"])
            extra["plain"] = r
            extra["learned_over_plain"] = round(value / r["Gtargets_s"], 3)
        if isinstance(wl_obj, Sweep1D):
            extra["per_table"] = sweep_per_table(wl_obj, stream, steps)
        if not isinstance(wl_obj, Batched2D) and wl_obj.model == "none":
            r = wl_obj.compare(stream, steps, "none", side=1)
            extra["side_le"] = {"Gtargets_s": r["Gtargets_s"], "ms_per_step": r["ms_per_step"],
                                "frac": frac_of(wl_obj, r["ms_per_step"]),
                                "le_over_lt": round(r["Gtargets_s"] / value, 3), "choices": r["choices"]}
    elif isinstance(wl_obj, Plain1D):
        for _ in range(3):
            wl_obj.step(side=1)
        torch.cuda.synchronize()
        ms = time_loop(lambda: wl_obj.step(side=1), stream, steps, flush=wl_obj.flush)[1]
        g = wl_obj.targets() / (ms / 1e3) / 1e9
        extra["side_le"] = {"Gtargets_s": round(g, 3), "ms_per_step": round(ms, 4), "frac": frac_of(wl_obj, ms),
                            "le_over_lt": round(g / value, 3)}
        # the same table prepared once (a plan, Sec. 5.3) and replayed as a
        # graph: the one-shot call prepares the table in every block of every call
        plan = wl_obj.ss.Plan.create_1d([0, wl_obj.X.numel()], wl_obj.X)
        plan.bind_1d([0, wl_obj.targets()], wl_obj.Y, wl_obj.out)
        for _ in range(3):
            plan.execute()
        torch.cuda.synchronize()
        ms = time_loop(plan.execute, stream, steps, flush=wl_obj.flush)[1]
        g = wl_obj.targets() / (ms / 1e3) / 1e9
        extra["plan_graph"] = {"Gtargets_s": round(g, 3), "ms_per_step": round(ms, 4), "frac": frac_of(wl_obj, ms),
                               "over_one_shot": round(g / value, 3)}
        del plan
    return extra


def make_workload(key, args):
    wl_obj = WORKLOADS[key]()
    if args.targets:
        wl_obj.m = args.targets
    if args.model is not None and isinstance(wl_obj, PlanWorkload):
        wl_obj.model = args.model
    if args.tile and isinstance(wl_obj, PlanWorkload):
        wl_obj.tile = args.tile
    if args.algo is not None and isinstance(wl_obj, Plain1D):
        wl_obj.set_algo(args.algo)
    return wl_obj


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + ["latency"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: every rank runs the whole workload; strong: the ranks split one workload "
                         "(tables by longest processing time, or slices of one table's targets)")
    ap.add_argument("--cpu-budget", type=float, default=10.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--config-cpu-budget", type=float, default=1.5,
                    help="seconds of oracle work for each further configuration's baseline and parity sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-suite", action="store_true", help="time the chosen workload only (no configs records)")
    ap.add_argument("--targets", type=int, default=0, help="override the workload's target count (profiling cases)")
    ap.add_argument("--model", default=None, choices=["none", "spline", "mlp", "loghash", "hunt", "auto"],
                    help="position model of the timed plan (default none: plain search; the learned forms are "
                         "timed beside it)")
    ap.add_argument("--no-compare", action="store_true", help="skip the learned and '<=' forms beside the timed one")
    ap.add_argument("--tile", type=int, default=0, help="fixed targets per tile for plan workloads (0: tuned)")
    ap.add_argument("--algo", default=None, choices=["auto", "bucket", "binary", "branchy", "ballot", "ballot8", "ballot16"],
                    help="in-block search of the plain1d workload")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "latency":
        return small_m_latency(args)
    wl_obj = make_workload(args.workload, args)
    if args.impl == "reference":
        return run_reference(args, wl_obj)

    rank, world, local = dist_setup(args.gpus)
    if args.scaling == "strong":
        if not isinstance(wl_obj, (Batched1D, Plain1D)):
            raise SystemExit("--scaling strong splits the batched1d and plain1d workloads only")
        wl_obj.share = (rank, world)
    import __graft_entry__
    __graft_entry__.build()
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    wl_obj.setup(dev, rank)
    stream = torch.cuda.current_stream()
    # clocks are sampled from the warm-up through the last configuration
    # (nvidia-smi every 50 ms; a short timed region alone may fall between
    # two samples); each record carries the samples taken while it ran
    clk = ClockSampler(dev.index).__enter__()
    clk.wait_first()
    solo = rank == 0 and world == 1
    cpu_budget = args.cpu_budget if solo and not args.no_cpu_baseline else 0
    rec = measure(wl_obj, args, stream, world, cpu_budget, args.steps)
    extra = {}
    if world == 1 and not args.no_compare:
        extra = other_forms(wl_obj, stream, args.steps, rec["value"])
    cpu = None
    if cpu_budget:
        timer = OracleTimer()
        cpu = timer.baseline_on(*wl_obj.sample(wl_obj.sample_n), wl_obj.snap)
        timer.close()
    head_clocks = clk.summary()
    head_co = co_bound(wl_obj, rec["value"], head_clocks["sm_mhz"])
    name, targets, flushed = wl_obj.name, wl_obj.targets(), wl_obj.flush is not None
    model = getattr(wl_obj, "model", None)
    wl_obj.release()

    # the other configurations of the suite, one after another on this GPU
    configs = {}
    if solo and not args.no_suite and args.workload == DEFAULT_WORKLOAD and not args.targets:
        for key, what in SUITE:
            other = make_workload(key, args)
            lo = len(clk.lines)
            other.setup(dev, 0)
            budget = args.config_cpu_budget if not args.no_cpu_baseline else 0
            r = measure(other, args, stream, 1, budget, min(args.steps, 3))
            r["config"] = what
            if not args.no_compare:
                r.update(other_forms(other, stream, args.steps, r["value"]))
            if budget:
                timer = OracleTimer()
                r["cpu_baseline"] = timer.baseline_on(*other.sample(other.sample_n), other.snap, reps=1)
                timer.close()
            r["clocks"] = clk.summary(lo, len(clk.lines))
            cb = co_bound(other, r["value"], r["clocks"]["sm_mhz"])
            if cb is not None:
                r["co_bound"] = cb
            configs[other.name] = r
            other.release()
        # small batches (next row f4): per-call latency of one-shot calls and graph-replayed plans
        lo = len(clk.lines)
        configs["latency-n64"] = {"config": "64-entry table, 1 .. 1M targets per call: per-call latency (us)",
                                  "unit": "us", "latency": latency_table(dev),
                                  "clocks": clk.summary(lo, len(clk.lines))}
    clk.__exit__(None, None, None)

    if rank == 0:
        line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
                "scaling": args.scaling, "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": name, "targets_per_gpu": targets,
                           "l2": "256 MB buffer written between timed steps" if flushed
                           else "inputs larger than L2 (no flush needed)",
                           "parallelism": "dp%d" % world},
                "gpu_launches": rec["gpu_launches"], "roofline": rec["roofline"], "cpu_baseline": cpu,
                "e2e": rec["e2e"], "clocks": head_clocks}
        if model is not None:
            line["config"]["model"] = model
            line["config"]["setup"] = "tables prepared once before timing (plan creation, Sec. 5.3)"
        if head_co is not None:
            line["co_bound"] = head_co
        line.update(extra)
        if configs:
            line["configs"] = configs
            line["clocks_all"] = clk.summary()
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
