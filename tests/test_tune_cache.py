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

    def set_scan_classes(self, g, t):
        self.calls.append(("classes", g, list(t)))


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
    tune._store(path, {key: {"schedule": [5, 4], "classes": {"0": [19, 17, 13, 0], "2": [18, 16, 14, 12]},
                             "ms": {"5,4": 1.0}}})
    ctx = FakeCtx()
    pcc = types.SimpleNamespace(FP32_BATCHED=1)    # no collide: a timing run would fail
    out = tune.tune(ctx, pcc, _fake_torch(), 2, None, 1.0, species, 1e-15, 1, cache_path=path)
    assert out == {"schedule": (5, 4), "classes": {0: [19, 17, 13, 0], 2: [18, 16, 14, 12]}, "ms": {"5,4": 1.0},
                   "cached": True}
    assert ctx.calls == [(5, 4), ("classes", 0, [19, 17, 13, 0]), ("classes", 2, [18, 16, 14, 12])]


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


def test_class_thresholds_validity():
    assert tune.valid_classes([20, 18, 14, 0]) and tune.valid_classes([34, 34, 34, 34])
    assert not tune.valid_classes([20, 21, 14, 0])        # g16 above warp
    assert not tune.valid_classes([35, 18, 14, 0]) and not tune.valid_classes([20, 18, 14, -1])


def test_descent_finds_the_minimum_of_a_separable_cost():
    """On a cost with its minimum at (24, 19, 12, 3) the descent from the
    default thresholds reaches it, measures every point once, keeps the
    ordering constraint, and stops when no move gains 1 %."""
    target = (24, 19, 12, 3)
    calls = []

    def cost(t):
        calls.append(tuple(t))
        assert tune.valid_classes(t)
        return 1.0 + sum((a - b) ** 2 for a, b in zip(t, target))

    best, c, seen = tune.descend([20, 18, 14, 0], cost, sweeps=10)
    assert tuple(best) == target and c == 1.0
    assert len(calls) == len(set(calls)) == len(seen)
    # a flat cost keeps the start
    best, c, _ = tune.descend([20, 18, 14, 0], lambda t: 1.0)
    assert best == [20, 18, 14, 0]
