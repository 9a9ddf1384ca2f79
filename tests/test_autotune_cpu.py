"""The autotuner's search on the host (no GPU): CUDA timing and the context are stand-ins whose
batch time depends on the tile widths, so that the search order and the winner can be checked."""
import sys
import types

import pytest


class _FakeEvent:
    clock = [0.0]

    def __init__(self, enable_timing=True):
        self.t = 0.0

    def record(self, stream=None):
        self.t = _FakeEvent.clock[0]

    def elapsed_time(self, other):
        return other.t - self.t


class _FakeStream:
    cuda_stream = 0

    def __init__(self, device=0):
        pass

    def synchronize(self):
        pass


def _fake_torch():
    cuda = types.SimpleNamespace(get_device_name=lambda d=0: "fake", Stream=_FakeStream, Event=_FakeEvent)
    return types.SimpleNamespace(cuda=cuda)


# batch time of a width assignment: per size, the cost of its width (lower is faster)
COST = {4: {32: 5.0, 8: 3.0, 16: 4.0}, 6: {32: 6.0, 8: 7.0, 16: 5.0}, 8: {32: 9.0, 8: 6.0, 16: 7.0},
        10: {32: 8.0, 8: 6.0}, 12: {32: 10.0, 4: 11.0}}


class _FakeContext:
    made = []

    def __init__(self, **kw):
        self.widths = {}
        _FakeContext.made.append(self)

    def set_sweep_order(self, order):
        pass

    def set_tile_width(self, L, w):
        self.widths[L] = w

    def init_disorder(self, dim, L, n, rid0=0):
        pass

    def set_launch(self, *a):
        pass

    def run_sweeps(self, n):
        _FakeEvent.clock[0] += sum(COST[L].get(self.widths.get(L, 32)) for L in COST)

    def close(self):
        pass


@pytest.fixture
def tuner(monkeypatch):
    from paper_2011_08560_gb300 import autotune, eamc
    monkeypatch.setitem(sys.modules, "torch", _fake_torch())
    monkeypatch.setattr(eamc, "Context", _FakeContext)
    widths = {4: [8, 16], 6: [8, 16], 8: [8, 16], 10: [8], 12: [4]}
    monkeypatch.setattr(eamc, "narrow_widths", lambda d, L, order=0: widths.get(L, []) if order else [])
    _FakeContext.made.clear()
    return autotune


def test_staged_search_finds_the_per_size_winners(tuner):
    groups = [(3, L, 100) for L in (4, 6, 8, 10, 12)]
    assert len(tuner.width_options(groups, 1)) > tuner.MAX_WIDTH_COMBOS
    best = tuner.tune(groups, sweeps=8, repeats=1, use_cache=False, order=1)
    assert best["widths"] == {"4": 8, "6": 16, "8": 8, "10": 8}
    # staged: the base, each size's narrow widths alone (2 + 2 + 2 + 1 + 1), the winners together
    assert len(_FakeContext.made) == 1 + 8 + 1


def test_small_products_are_tried_in_full(tuner):
    groups = [(3, 8, 100)]
    best = tuner.tune(groups, sweeps=8, repeats=1, use_cache=False, order=1)
    assert best["widths"] == {"8": 8}
    assert len(_FakeContext.made) == 3
