"""Host logic of the batch autotuner (no GPU): which candidates a form's accuracy bar allows,
that the fastest allowed (tile shape, K steps per unit) wins, and that the choice is cached
under the GPU name and the batch's shape signature and reused without timing again.  The
batch and the CUDA events are fakes driven by a fake clock, so the test runs on the CPU."""
import contextlib
import json
import types

import pytest


class FakeClock:
    def __init__(self):
        self.t = 0.0


class FakeBatch:
    """Each run advances the clock by the time the test assigns to the current settings."""

    def __init__(self, clock, cost):
        self.clock, self.cost = clock, cost
        self.tiles, self.ksteps = None, None
        self.runs = []

    def set_stage2_tiles(self, t):
        self.tiles = t

    def set_tuning(self, k):
        self.ksteps = k

    def run(self, stream=None):
        self.runs.append((self.tiles, self.ksteps))
        self.clock.t += self.cost(self.tiles, self.ksteps)


@pytest.fixture
def fake_cuda(monkeypatch):
    import torch
    clock = FakeClock()

    class Event:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = clock.t

        def elapsed_time(self, other):
            return other.t - self.t

    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    return clock


def _plans():
    P = lambda o, h, z: types.SimpleNamespace(obj_h=o, holo_h=h, n_layers=z)
    return [P(512, 1024, 16), P(128, 256, 4), P(1024, 2048, 28)]


def test_signature_is_order_free_and_names_the_form():
    from paper_2211_09938_gb300 import autotune
    a = autotune.signature(_plans(), "tc_fp16x3")
    b = autotune.signature(list(reversed(_plans())), "tc_fp16x3")
    assert a == b == "tc_fp16x3|128-256-4;512-1024-16;1024-2048-28"
    assert autotune.signature(_plans(), "tc_bf16x3") != a


@pytest.mark.parametrize("form,allowed", [("tc_fp16x3", {8, 16, 32}), ("tc_bf16x3", {8, 16, 32, 64, 128})])
def test_fastest_allowed_choice_is_taken_and_cached(tmp_path, fake_cuda, form, allowed):
    from paper_2211_09938_gb300 import autotune
    # the longest chains are fastest, pairs beat single CTAs: the winner is the longest chain
    # the form's accuracy bar allows, on pairs
    cost = lambda tiles, k: 10.0 / k + (0.5 if tiles == autotune.TILES["cta"] else 0.0)
    batch = FakeBatch(fake_cuda, cost)
    cache = tmp_path / "tune.json"
    entry = autotune.tune_batch(batch, _plans(), form, stream=None, cache_path=str(cache), reps=3)
    best_k = max(allowed)
    assert (entry["tiles"], entry["ksteps"]) == ("pair", best_k)
    assert (batch.tiles, batch.ksteps) == (autotune.TILES["pair"], best_k)  # applied to the batch
    assert {int(k.split("/")[1]) for k in entry["tried"]} == allowed  # nothing past the bar timed
    assert {k for _, k in batch.runs} == allowed
    assert entry["ms"] == pytest.approx(cost(autotune.TILES["pair"], best_k))
    key = "FakeGPU|" + autotune.signature(_plans(), form)
    assert json.loads(cache.read_text())[key]["ksteps"] == best_k

    # a second batch of the same shapes takes the cached choice without running
    again = FakeBatch(fake_cuda, cost)
    entry2 = autotune.tune_batch(again, _plans(), form, stream=None, cache_path=str(cache))
    assert again.runs == []
    assert (again.tiles, again.ksteps) == (autotune.TILES["pair"], best_k)
    assert entry2["ksteps"] == best_k


def test_single_cta_wins_when_faster_and_a_bad_cache_is_ignored(tmp_path, fake_cuda):
    from paper_2211_09938_gb300 import autotune
    cost = lambda tiles, k: {8: 3.0, 16: 1.0, 32: 2.0}[k] + (0.0 if tiles == autotune.TILES["cta"] else 0.25)
    cache = tmp_path / "tune.json"
    cache.write_text("{not json")
    batch = FakeBatch(fake_cuda, cost)
    entry = autotune.tune_batch(batch, _plans(), "tc_fp16x3", stream=None, cache_path=str(cache))
    assert (entry["tiles"], entry["ksteps"]) == ("cta", 16)
    assert json.loads(cache.read_text())  # rewritten as valid JSON
