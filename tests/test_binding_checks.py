"""CPU checks of the Python binding's argument marshalling: offsets that the
library would read past, outputs too small for what the library writes,
and status records that are not device memory are refused with a Python
error before any call reaches the library or a kernel; without the built
library every call raises (there is no CPU fallback)."""
import numpy as np
import pytest
import torch

import paper_2112_03229_gb300 as ss


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2112_03229_gb300 import _build
    _build.build()


def test_offsets_are_checked():
    X = torch.zeros(10, dtype=torch.float64)
    a, _ = ss._offsets([0, 4, 10], "X_off", data=X)
    assert a.dtype == np.int64 and list(a) == [0, 4, 10]
    for bad, why in (([0], "ntables"), ([4, 2], "non-decreasing"), ([-1, 3], "non-negative"),
                     ([0, 11], "past the data"), (np.zeros((2, 2)), "ntables")):
        with pytest.raises(ValueError, match=why):
            ss._offsets(bad, "X_off", data=X)
    with pytest.raises(ValueError, match="3 expected"):
        ss._offsets([0, 1, 2, 3], "Y_off", length=3)
    # 2D pairs: the last offset counts pairs, the data holds two doubles per pair
    with pytest.raises(ValueError, match="past the data"):
        ss._offsets([0, 6], "Y_off", data=torch.zeros(11, dtype=torch.float64), per=2)


def test_batched_offsets_must_agree_in_length():
    X = torch.zeros(10, dtype=torch.float64)
    Y = torch.zeros(5, dtype=torch.float64)
    with pytest.raises(ValueError, match="expected"):
        ss.search_1d_batched([0, 4, 10], X, [0, 5], Y)
    with pytest.raises(ValueError, match="expected"):
        ss.search_1d_batched_static([0, 4, 10], X, [0, 2, 3, 5], Y)
    with pytest.raises(ValueError, match="past the data"):
        ss.search_1d_batched([0, 4, 10], X, [0, 2, 6], Y)
    R = torch.zeros(6, dtype=torch.float64)
    with pytest.raises(ValueError, match="expected"):
        ss.search_interp_2d_batched([0, 3, 6], R, [0, 3], R, [0, 9, 18], torch.zeros(18, dtype=torch.float64),
                                    [0, 1, 2], torch.zeros(4, dtype=torch.float64))


def test_outputs_must_hold_every_answer():
    X = torch.zeros(8, dtype=torch.float64)
    Y = torch.zeros(100, dtype=torch.float64)
    with pytest.raises(ValueError, match="out holds 99"):
        ss.search_1d(X, Y, out=torch.empty(99, dtype=torch.int32))
    with pytest.raises(ValueError, match="out holds 99"):
        ss.search_1d_host(X, Y, out=torch.empty(99, dtype=torch.int32))
    R, T = torch.zeros(4, dtype=torch.float64), torch.zeros(3, dtype=torch.float64)
    F, Y2 = torch.zeros(12, dtype=torch.float64), torch.zeros(20, dtype=torch.float64)
    with pytest.raises(ValueError, match="idx holds"):
        ss.search_interp_2d(R, T, F, Y2, idx=torch.empty(19, dtype=torch.int32))
    with pytest.raises(ValueError, match="val holds"):
        ss.search_interp_2d_host(R, T, F, Y2, val=torch.empty(9, dtype=torch.float64))
    with pytest.raises(ValueError, match="len\\(R\\) \\* len\\(T\\)"):
        ss.search_interp_2d_host(R, T, F[:11], Y2)
    with pytest.raises(ValueError, match="params holds"):
        ss.mlp_forward(torch.zeros(64, dtype=torch.float32), torch.zeros(8, dtype=torch.float32))
    with pytest.raises(ValueError, match="x holds"):
        ss.mlp_loss_grad(torch.zeros(65, dtype=torch.float32), torch.zeros(7, dtype=torch.float32),
                         torch.zeros(4, dtype=torch.float32))


def test_plan_binding_checks_its_table_count():
    plan = ss.Plan(None, 1, 3)          # no library handle: every check below comes first
    Y = torch.zeros(10, dtype=torch.float64)
    with pytest.raises(ValueError, match="4 expected"):
        plan.bind_1d([0, 5, 10], Y, torch.empty(10, dtype=torch.int32))
    with pytest.raises(ValueError, match="out holds 9"):
        plan.bind_1d([0, 2, 5, 10], Y, torch.empty(9, dtype=torch.int32))
    plan2 = ss.Plan(None, 2, 2)
    with pytest.raises(ValueError, match="idx holds"):
        plan2.bind_2d([0, 2, 5], Y, torch.empty(9, dtype=torch.int32), torch.empty(5, dtype=torch.float64))


def test_status_record_must_be_device_memory():
    with pytest.raises(TypeError, match="stat"):
        ss._statp(torch.zeros(24, dtype=torch.uint8))
    assert ss._statp(None) is None


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the built library every call raises
    monkeypatch.setattr(ss, "_lib", None)
    monkeypatch.setattr(ss, "LIB_PATH", str(tmp_path / "libsimdsearch.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        ss.lib()
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        ss.search_1d_host(torch.zeros(4, dtype=torch.float64), torch.zeros(3, dtype=torch.float64))
