"""The autotuner's selection and cache, without a GPU: fake volumes and a timer that charges a
known cost to each (brick, tile, refill) candidate."""
import json

import pytest

from paper_2509_26213_gb300 import tune


class FakeVolume:
    def __init__(self, brick):
        self.brick = brick
        self.closed = False

    def close(self):
        self.closed = True


def cost(vol, cams, tf, prm):
    """Fastest: brick 64, 8x4 tiles, refill 20; every candidate distinct."""
    return (10.0 + (0.0 if vol.brick == 64 else 3.0) + abs(prm["tile_w"] - 8) * 0.5 + abs(prm["tile_h"] - 4) * 0.25
            + abs(prm["refill"] - 20) * 0.01)


def test_picks_the_fastest_candidate_and_closes_the_rest(tmp_path):
    made = []

    def make(brick):
        made.append(FakeVolume(brick))
        return made[-1]

    calls = []

    def timer(vol, cams, tf, prm):
        calls.append((vol.brick, prm["tile_w"], prm["tile_h"], prm["refill"]))
        return cost(vol, cams, tf, prm)

    out = tune.autotune(make, cams=[], tf=None, params={"step": 0.5}, key="k", timer=timer, device_name="gpu",
                        cache_path=str(tmp_path / "cache.json"))
    assert (out["brick"], out["tile_w"], out["tile_h"], out["refill"]) == (64, 8, 4, 20)
    assert out["cached"] is False and out["volume"].brick == 64
    assert out["ms"] == pytest.approx(10.0)
    # every brick x tile x refill candidate timed once, with the caller's other parameters kept
    n = 2 * len(tune.DEFAULT_TILES) * len(tune.DEFAULT_REFILL)
    assert len(calls) == n == len(set(calls)) == len(out["timings"])
    assert [v.closed for v in made] == [True, False]


def test_winner_is_cached_per_device_and_key(tmp_path):
    path = str(tmp_path / "cache.json")
    tune.autotune(FakeVolume, [], None, {}, key="scene", timer=cost, device_name="gpu-a", cache_path=path)
    with open(path) as f:
        cached = json.load(f)
    assert list(cached) == ["gpu-a|scene"] and cached["gpu-a|scene"]["tile_w"] == 8

    def no_timing(*a):
        raise AssertionError("a cached result must not time anything")

    def no_volume(brick):
        raise AssertionError("a cached result must not build volumes")

    hit = tune.autotune(no_volume, [], None, {}, key="scene", timer=no_timing, device_name="gpu-a", cache_path=path)
    assert hit["cached"] is True and "volume" not in hit
    assert (hit["brick"], hit["tile_w"], hit["tile_h"], hit["refill"]) == (64, 8, 4, 20)
    # another device or another workload key is tuned afresh and added beside the first
    tune.autotune(FakeVolume, [], None, {}, key="scene", timer=cost, device_name="gpu-b", cache_path=path,
                  bricks=(32,))
    with open(path) as f:
        cached = json.load(f)
    assert sorted(cached) == ["gpu-a|scene", "gpu-b|scene"] and cached["gpu-b|scene"]["brick"] == 32
