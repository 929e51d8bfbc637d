"""Mutation check of the oracle's pins, on the CPU.

Each case plants one plausible mistake in a copy of oracle/oracle.c (a
comparison of the wrong strictness, a dropped clamp, a transposed grid, a
wrong gradient term, ...), compiles the copy with the oracle's own flags,
and runs every pin of tests/test_oracle_pins.py against it: at least one
pin must fail.  The mistakes keep every access in bounds, so a mutant can
only give wrong answers.  The real oracle is left untouched and is used
again after each case.
"""
import importlib.util
import inspect
import os
import shutil
import subprocess

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")

# (name, text in oracle.c, replacement)
MUTATIONS = [
    ("strict comparison made non-strict",
     "int below = side ? (X[mid] <= t) : (X[mid] < t);",
     "int below = side ? (X[mid] <= t) : (X[mid] <= t);"),
    ("low end clamp wrong",
     "return (int32_t)(c > 0 ? c - 1 : 0);",
     "return (int32_t)(c > 1 ? c - 1 : 1);"),
    ("cell clamp off by one",
     "int32_t cr = ir < nr - 2 ? ir : nr - 2;",
     "int32_t cr = ir < nr - 3 ? ir : nr - 2;"),
    ("weight measured from the upper entry",
     "else w = (x - X[c]) / (X[c + 1] - X[c]);",
     "else w = (X[c + 1] - x) / (X[c + 1] - X[c]);"),
    ("weight clamp dropped",
     "return extrap ? w : clamp01(w);",
     "return w;"),
    ("grid transposed",
     "double f01 = F[(int64_t)cr * nt + ct + 1];\n  double f10 = F[(int64_t)(cr + 1) * nt + ct];",
     "double f01 = F[(int64_t)(cr + 1) * nt + ct];\n  double f10 = F[(int64_t)cr * nt + ct + 1];"),
    ("negative values keep their bit pattern as key",
     "if (u >> 63) return (uint64_t)0 - u;",
     "if (u >> 63) return u;"),
    ("directory counts its own bucket",
     "if ((oracle_order_key(X[j]) >> shift) < b0 + (uint64_t)b) ++c;",
     "if ((oracle_order_key(X[j]) >> shift) <= b0 + (uint64_t)b) ++c;"),
    ("spline knot spacing rounded down",
     "uint64_t delta = span / (uint64_t)K + (span % (uint64_t)K != 0);",
     "uint64_t delta = span / (uint64_t)K;"),
    ("exponent bias off by one",
     "double e = (double)((int64_t)((u >> 52) & 0x7FF) - 1023);",
     "double e = (double)((int64_t)((u >> 52) & 0x7FF) - 1022);"),
    ("ReLU dropped",
     "static double relu(double a) { return a > 0.0 ? a : 0.0; }",
     "static double relu(double a) { return a; }"),
    ("bias gradient scaled by a feature",
     "grad[2 * H + k] += dz;",
     "grad[2 * H + k] += dz * x0;"),
    ("Adam bias correction dropped",
     "double c1 = 1.0 - pow(beta1, (double)step);",
     "double c1 = 1.0;"),
    ("side <= searched as <",
     "int below = side ? (X[mid] <= t) : (X[mid] < t);",
     "int below = side ? (X[mid] < t) : (X[mid] < t);"),
    ("log-space weight measured from the upper entry",
     "if (logspace) w = (log(x) - log(X[c])) / (log(X[c + 1]) - log(X[c]));",
     "if (logspace) w = (log(X[c + 1]) - log(x)) / (log(X[c + 1]) - log(X[c]));"),
    ("extrapolation flag ignored",
     "return extrap ? w : clamp01(w);",
     "return clamp01(w);"),
    ("outer blend weighted by the T weight",
     "*v_out = (1.0 - wr) * lo_row + wr * hi_row;",
     "*v_out = (1.0 - wt) * lo_row + wt * hi_row;"),
    ("mantissa feature scaled by 2^-53",
     "/ 4503599627370496.0;",
     "/ 9007199254740992.0;"),
    ("output bias left out of the forward pass",
     "double y = b2;",
     "double y = 0.0;"),
    ("ReLU gradient passed through inactive units",
     "if (h[k] > 0.0) {",
     "if (h[k] >= 0.0) {"),
    ("loss summed instead of averaged",
     "return loss / (double)B;",
     "return loss;"),
    ("second Adam moment from the raw gradient",
     "(1.0 - beta2) * grad[k] * grad[k];",
     "(1.0 - beta2) * grad[k];"),
    ("bucket shift one step too coarse",
     "if ((k1 >> s) - (k0 >> s) < (uint64_t)cap_buckets) return s;",
     "if ((k1 >> s) - (k0 >> s) < (uint64_t)cap_buckets) return s + 1;"),
    ("spline knot counts its own key",
     "if (oracle_order_key(X[i]) < kappa) ++c;",
     "if (oracle_order_key(X[i]) <= kappa) ++c;"),
    ("2D batch options dropped",
     "Y2 + 2 * y0, Y_off[k + 1] - y0, extrap, logspace,",
     "Y2 + 2 * y0, Y_off[k + 1] - y0, 0, 0,"),
    ("2D batch pairs offset by one double per pair",
     "Y2 + 2 * y0, Y_off[k + 1] - y0, extrap, logspace,",
     "Y2 + y0, Y_off[k + 1] - y0, extrap, logspace,"),
    ("sampled 1D form reads the k-th target",
     "lowbounds[k] = lower_bound_index(X, n, Y[sample[k]], side);",
     "lowbounds[k] = lower_bound_index(X, n, Y[k], side);"),
    ("sampled 2D form reads the k-th pair",
     "int64_t i = sample[k];",
     "int64_t i = k;"),
]


def load_pins():
    spec = importlib.util.spec_from_file_location("oracle_pins_for_mutants", os.path.join(HERE, "test_oracle_pins.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def run_pins(pins):
    """Names of the pins that fail (any exception counts)."""
    failed = []
    for name, fn in sorted(vars(pins).items()):
        if not name.startswith("test_") or not callable(fn):
            continue
        params = list(inspect.signature(fn).parameters)
        calls = [{"side": 0}, {"side": 1}] if params == ["side"] else ([{}] if not params else [])
        for kw in calls:
            try:
                fn(**kw)
            except Exception:
                failed.append(name)
                break
    return failed


def test_the_pins_pass_on_the_real_oracle():
    assert run_pins(load_pins()) == []


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc missing")
@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_each_planted_mistake_fails_a_pin(tmp_path, monkeypatch, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found: " + name
    mutant_src = tmp_path / "oracle_mutant.c"
    mutant_src.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc"] + oracle._build_mod.CFLAGS + ["-o", str(lib), str(mutant_src), "-lm"],
                   check=True, capture_output=True)
    # the oracle module loads the mutant in place of the real library for this case
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle._build_mod, "build", lambda force=False: str(lib))
    try:
        failed = run_pins(load_pins())
    finally:
        oracle._lib = None
    assert failed, "no pin caught: " + name
