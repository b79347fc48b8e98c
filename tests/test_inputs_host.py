"""The seeded input generators (synth/scenes.py) against the input recipe they promise: same
seed, same scene; shapes and types; layer indices inside the layer count; saliency maps of the
stated coverage; the batch mix; the per-point depth range and holes; the colour scene sharing
its layers and saliency with the grey one; the thresholds on the uint8 scale.  CPU only."""
import math

import numpy as np
import pytest

from synth import scenes


def _same(a, b):
    return all(np.array_equal(np.asarray(a[k]), np.asarray(b[k])) for k in ("intensity", "layer", "saliency", "z"))


def test_same_seed_same_scene_other_seed_other_scene():
    assert _same(scenes.paper_scene(), scenes.paper_scene())
    assert not np.array_equal(scenes.paper_scene(seed=2000)["intensity"], scenes.paper_scene(seed=2001)["intensity"])
    assert _same(scenes.random_scene(7, 128, 256, 5), scenes.random_scene(7, 128, 256, 5))


def test_paper_scene_recipe():
    sc = scenes.paper_scene()
    for k in ("intensity", "layer", "saliency"):
        assert sc[k].shape == (512, 512) and sc[k].dtype == np.uint8, k
    assert sc["holo"] == (1024, 1024)
    assert np.allclose(sc["z"], np.linspace(0.08, 0.20, 16))
    assert sc["layer"].max() < 16 and len(np.unique(sc["layer"])) > 8  # depth spread over the layers
    assert set(np.unique(sc["saliency"])) <= {0, 255}
    frac = (sc["saliency"] == 255).mean()
    assert 0.20 <= frac <= 0.35  # union of 3 ellipses, rejection-sampled to 20-35%
    assert sc["pitch"] == 8e-6 and sc["wavelength"] == 532e-9


def test_tiny_scene_recipe():
    sc = scenes.tiny_scene()
    assert sc["intensity"].shape == (64, 64) and sc["holo"] == (256, 256)
    assert np.allclose(sc["z"], [0.10, 0.11, 0.12, 0.13])
    assert sc["layer"].max() < 4
    assert abs((sc["saliency"] == 255).mean() - 0.25) < 0.03  # centred ellipse of 25% area


def test_batch_mix():
    b = scenes.batch_scenes()
    assert len(b) == 64
    edges = [s["intensity"].shape[0] for s in b]
    assert set(edges) <= {128, 256, 512, 1024} and len(set(edges)) >= 3
    for s in b:
        n = s["intensity"].shape[0]
        assert s["holo"] == (2 * n, 2 * n)
        assert 4 <= len(s["z"]) <= 32 and s["layer"].max() < len(s["z"])
        frac = (s["saliency"] == 255).mean()
        assert 0.03 <= frac <= 0.62  # ellipse area U[0.05, 0.6], up to pixel rounding


@pytest.mark.parametrize("holes", [0.0, 0.1])
def test_depth_map_range_and_holes(holes):
    z = scenes.depth_map(31, 128, holes=holes)
    assert z.dtype == np.float32 and z.shape == (128, 128)
    ok = np.isfinite(z) & (z > 0)
    assert np.all((z[ok] >= 0.08 - 1e-6) & (z[ok] <= 0.20 + 1e-6))
    if holes == 0.0:
        assert ok.all()
    else:
        assert abs((~ok).mean() - holes) < 0.01  # every hole (NaN, 0 or negative) is no depth


def test_rgb_scene_shares_layers_and_saliency():
    c = scenes.rgb_scene(9, 64, 128, 3)
    g = scenes.random_scene(9, 64, 128, 3)
    assert c["intensity"].shape == (3, 64, 64) and c["intensity"].dtype == np.uint8
    assert np.array_equal(c["layer"], g["layer"]) and np.array_equal(c["saliency"], g["saliency"])
    assert not np.array_equal(c["intensity"][0], c["intensity"][1])


def test_thresholds_are_floor_255_t():
    assert scenes.THRESHOLDS_U8 == {l: math.floor(255 * t) for l, t in ((3, 0.5), (2, 0.7), (1, 0.9))}
