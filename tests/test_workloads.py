"""The named workloads of workloads.json build the same inputs as the
constructions used so far (tiny_workload, scene_workload, the ring cameras of
the multi-view, precision and scene-batch forms), and scene files round-trip
bit for bit.  CPU only."""
import json
import math

import numpy as np
import pytest

from paper_2412_20522_gb300 import scenes

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh", "mask_logits")


def _same_gaussians(a, b):
    assert a.sh_degree == b.sh_degree
    for k in FIELDS:
        x, y = getattr(a, k), getattr(b, k)
        assert x.dtype == y.dtype and np.array_equal(x, y), k


def _same_camera(a, b):
    assert (a.width, a.height, a.fx, a.fy, a.cx, a.cy, a.near) == \
           (b.width, b.height, b.fx, b.fy, b.cx, b.cy, b.near)
    assert np.array_equal(a.viewmat, b.viewmat) and np.array_equal(a.cam_pos, b.cam_pos)


def test_c1_is_the_tiny_workload():
    w = scenes.workload("c1_tiny")
    g, cams, tgt = scenes.tiny_workload()
    _same_gaussians(w.gaussians, g)
    assert len(w.cams) == 1
    _same_camera(w.cams[0], cams[0])
    assert np.array_equal(w.targets[0], tgt) and w.view_ranges is None


def test_c2_and_c3_are_the_scene_view_and_its_ring():
    w2 = scenes.workload("c2_scene")
    g, cams, tgt = scenes.scene_workload()
    _same_gaussians(w2.gaussians, g)
    _same_camera(w2.cams[0], cams[0])
    assert np.array_equal(w2.targets[0], tgt)
    w3 = scenes.workload("c3_multiview")
    _same_gaussians(w3.gaussians, g)
    assert len(w3.cams) == 8 and w3.view_ranges is None
    for k, c in enumerate(w3.cams):
        _same_camera(c, scenes.ring_camera(2 * math.pi * k / 8, 4.0, 1557, 1038, 1150.0))
        assert np.array_equal(w3.targets[k], tgt)


def test_c4_precision_workload():
    w = scenes.workload("c4_precision")
    assert w.gaussians.n == 3_000_000 and w.storage == ("bf16", "fp16", "f32")
    _same_gaussians(w.gaussians, scenes.cluster_gaussians(3_000_000, seed=2024125))
    f4 = 1150.0 * 1957 / 1557
    for k, c in enumerate(w.cams):
        _same_camera(c, scenes.ring_camera(2 * math.pi * k / 4, 4.0, 1957, 1297, f4))
        assert np.array_equal(w.targets[k], scenes.target_image(1297, 1957, seed=2024126 + k))
    assert w.spec["error_crop"] == {"view": 0, "size": 64}


def test_c5_scene_batch_layout(tmp_path):
    """The scene batch on reduced sizes (same file layout): concatenation
    order, per-camera ranges, cameras and targets per scene."""
    spec = scenes.load_workloads()
    c5 = spec["c5_uneven"]
    assert [s["gaussians"] for s in c5["scenes"]] == [150_000, 400_000, 800_000, 1_200_000,
                                                      2_000_000, 3_000_000]
    assert c5["cameras"]["resolutions"][0] == [779, 519]
    small = json.loads(json.dumps(c5))
    for k, s in enumerate(small["scenes"]):
        s["gaussians"] = 1000 * (k + 1)
    path = tmp_path / "w.json"
    path.write_text(json.dumps({"c5_small": small}))
    w = scenes.workload("c5_small", str(path))
    sizes = [1000 * (k + 1) for k in range(6)]
    assert w.view_ranges == [(int(o), n) for o, n in
                             zip(np.concatenate([[0], np.cumsum(sizes)[:-1]]), sizes)]
    for k, (o, n) in enumerate(w.view_ranges):
        part = scenes.cluster_gaussians(n, seed=2024130 + k)
        _same_gaussians(w.gaussians.subset(slice(o, o + n)), part)
        _same_gaussians(w.parts[k][0], part)
        wk, hk = c5["cameras"]["resolutions"][k]
        _same_camera(w.cams[k], scenes.ring_camera(0.5 * k, 4.0, wk, hk, 1150.0 * wk / 1557))
        assert np.array_equal(w.targets[k], scenes.target_image(hk, wk, seed=2024140 + k))


def test_scene_file_round_trip(tmp_path):
    w = scenes.workload("c1_tiny")
    path = str(tmp_path / "scene.npz")
    scenes.save_npz(path, w.gaussians, w.cams, w.targets)
    g, cams, targets = scenes.load_npz(path)
    _same_gaussians(g, w.gaussians)
    assert len(cams) == 1 and len(targets) == 1
    _same_camera(cams[0], w.cams[0])
    assert np.array_equal(targets[0], w.targets[0])


def test_unknown_names_are_rejected(tmp_path):
    with pytest.raises(KeyError):
        scenes.workload("no_such_workload")
    bad = scenes.load_workloads()["c1_tiny"]
    bad = json.loads(json.dumps(bad))
    bad["scenes"][0]["distribution"] = "spiral"
    path = tmp_path / "w.json"
    path.write_text(json.dumps({"bad": bad}))
    with pytest.raises(ValueError):
        scenes.workload("bad", str(path))
