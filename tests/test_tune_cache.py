"""Host logic of the launch-schedule autotuner, without a GPU: the cache key
names the device and the workload shape, a cached schedule is applied
without timing anything, and the cache file survives a round trip and a
corrupt file."""
import json
import types

import pytest

torch = pytest.importorskip("torch")

from paper_1907_02814_gb300 import tune  # noqa: E402


class FakeCtx:
    def __init__(self):
        self.calls = []

    def set_schedule(self, m, b):
        self.calls.append((m, b))


def _fake_torch(name="GB300 (fake)"):
    return types.SimpleNamespace(cuda=types.SimpleNamespace(get_device_name=lambda: name))


def _species(counts):
    return {k: types.SimpleNamespace(cell_count=torch.tensor(v, dtype=torch.int32)) for k, v in counts.items()}


def test_shape_key_names_device_cells_and_live_counts():
    k1 = tune.shape_key(_fake_torch(), 64, {"em": 10, "ion": 5})
    assert k1 == "GB300 (fake)|cells=64|em=10|ion=5"
    assert tune.shape_key(_fake_torch(), 64, {"ion": 5, "em": 10}) == k1          # order-free
    assert tune.shape_key(_fake_torch("other"), 64, {"em": 10, "ion": 5}) != k1
    assert tune.shape_key(_fake_torch(), 65, {"em": 10, "ion": 5}) != k1


def test_cached_schedule_is_applied_without_timing(tmp_path):
    species = _species({"em": [3, 4], "ep": [0, 0], "ph": [1, 0], "ion": [2, 2]})
    key = tune.shape_key(_fake_torch(), 2, {"em": 7, "ep": 0, "ph": 1, "ion": 4})
    path = str(tmp_path / "cache.json")
    tune._store(path, {key: {"schedule": [5, 4], "ms": {"5,4": 1.0}}})
    ctx = FakeCtx()
    pcc = types.SimpleNamespace(FP32_BATCHED=1)    # no collide: a timing run would fail
    out = tune.tune(ctx, pcc, _fake_torch(), 2, None, 1.0, species, 1e-15, 1, cache_path=path)
    assert out == {"schedule": (5, 4), "ms": {"5,4": 1.0}, "cached": True}
    assert ctx.calls == [(5, 4)]


def test_cache_round_trip_and_corrupt_file(tmp_path):
    path = str(tmp_path / "c.json")
    assert tune._load(path) == {}                    # missing file
    tune._store(path, {"a": {"schedule": [4, 0]}})
    assert tune._load(path) == {"a": {"schedule": [4, 0]}}
    assert json.load(open(path)) == {"a": {"schedule": [4, 0]}}
    with open(path, "w") as f:
        f.write("{not json")
    assert tune._load(path) == {}                    # corrupt file: start afresh


def test_candidates_are_valid_schedules():
    """Every candidate is a register budget the library compiles (2 to 6
    blocks per SM) and a grid cap that is 0 or at most that budget."""
    for m, b in tune.CANDIDATES:
        assert 2 <= m <= 6 and (b == 0 or 1 <= b <= m)
    assert len(set(tune.CANDIDATES)) == len(tune.CANDIDATES)
