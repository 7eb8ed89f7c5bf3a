"""Seeded synthetic scenes, cameras and target images.

This module produces INPUTS only and holds none of the rasteriser's
arithmetic: no projection, no covariance, no compositing, no mask sampling.
It is the one piece shared by the CUDA path and the oracle, so that both see
bit-identical inputs.

The workloads stand in for the paper's real-world captures (Mip-NeRF360,
Tanks&Temples, Deep Blending; Sec. 4.1), which are not available: the Gaussian
counts mirror the paper's averages (1.2 M for MaskGaussian on Mip-NeRF360,
Table 1) and the attribute distributions are the ones stated for each named
workload below. No dataset item is reproduced.

Conventions (shared with the C ABI, ``include/maskgs.h``):
  * means f32[N][3]; log_scales f32[N][3]; quats f32[N][4] as (w, x, y, z);
    opacity_logit f32[N]; sh f32[N][(D+1)^2][3] (channel fastest);
    mask_logits f32[N][2] with index 0 = "present" (Sec. 3.3).
  * Cameras use OpenCV axes (x right, y down, z forward).  ``viewmat`` is the
    3x4 row-major world->camera transform t = R p + t_cam.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

SCENE_SEED = 2024122
TARGET_SEED = 2024123
GUMBEL_SEED = 2024124


@dataclass
class Gaussians:
    means: np.ndarray          # f32[N][3]
    log_scales: np.ndarray     # f32[N][3]
    quats: np.ndarray          # f32[N][4]  (w, x, y, z)
    opacity_logit: np.ndarray  # f32[N]
    sh: np.ndarray             # f32[N][(D+1)^2][3]
    mask_logits: np.ndarray    # f32[N][2]
    sh_degree: int = 3

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Gaussians":
        return Gaussians(self.means[idx].copy(), self.log_scales[idx].copy(),
                         self.quats[idx].copy(), self.opacity_logit[idx].copy(),
                         self.sh[idx].copy(), self.mask_logits[idx].copy(),
                         self.sh_degree)


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    viewmat: np.ndarray = field(repr=False)   # f32[3][4]
    cam_pos: np.ndarray = field(repr=False)   # f32[3]
    near: float = 0.2


def look_at_camera(eye, target, width, height, focal, near=0.2) -> Camera:
    """Pinhole camera at ``eye`` looking at ``target`` with world +y as 'down'."""
    eye = np.asarray(eye, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    z = target - eye
    z /= np.linalg.norm(z)
    down = np.array([0.0, 1.0, 0.0])
    if abs(float(np.dot(down, z))) > 0.999:
        down = np.array([0.0, 0.0, 1.0])
    x = np.cross(down, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=0)
    t = -R @ eye
    vm = np.concatenate([R, t[:, None]], axis=1).astype(np.float32)
    return Camera(width, height, float(focal), float(focal), width / 2.0, height / 2.0,
                  vm, eye.astype(np.float32), near)


def ring_camera(theta, radius, width, height, focal, near=0.2) -> Camera:
    eye = (radius * math.sin(theta), 0.0, -radius * math.cos(theta))
    return look_at_camera(eye, (0.0, 0.0, 0.0), width, height, focal, near)


def _random_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _attributes(rng, means, log_scale_mu, log_scale_sigma, sh_degree,
                mask_mu0=0.0):
    n = means.shape[0]
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, (n, 3)).astype(np.float32)
    quats = _random_quats(rng, n)
    opacity_logit = rng.standard_normal(n).astype(np.float32)
    nsh = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.1, (n, nsh, 3)).astype(np.float32)
    sh[:, 0, :] = rng.normal(0.5, 0.2, (n, 3)).astype(np.float32)
    mask_logits = rng.standard_normal((n, 2)).astype(np.float32)
    mask_logits[:, 0] += np.float32(mask_mu0)
    return Gaussians(means.astype(np.float32), log_scales, quats, opacity_logit,
                     sh, mask_logits, sh_degree)


def uniform_gaussians(n, seed=SCENE_SEED, sh_degree=3, log_scale_mu=-4.0,
                      log_scale_sigma=0.5) -> Gaussians:
    """Means uniform in [-1,1]^3, log-scales N(-4, 0.5), random unit quaternions,
    opacity sigmoid(N(0,1)), SH N(0, 0.1) with DC N(0.5, 0.2), mask logits N(0,1)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3))
    return _attributes(rng, means, log_scale_mu, log_scale_sigma, sh_degree)


def cluster_gaussians(n, seed=SCENE_SEED, sh_degree=3, n_clusters=64,
                      centre_radius=4.0, reject_radius=5.0, log_scale_mu=-5.0,
                      log_scale_sigma=1.0, mask_mu0=0.54) -> Gaussians:
    """Means from a mixture of ``n_clusters`` anisotropic clusters.

    Cluster centres are uniform in the radius-4 ball; each cluster has a random
    rotation and per-axis sigma log-uniform in [0.1, 1.0]; equal weights; samples
    outside radius 5 are redrawn.  Log-scales N(-5, 1).  Mask logits
    l0 ~ N(0.54, 1), l1 ~ N(0, 1), so that about 40 % of the Gaussians are
    sampled off.
    """
    rng = np.random.default_rng(seed)
    # centres: uniform in the ball by rejection from the cube
    centres = []
    while len(centres) < n_clusters:
        c = rng.uniform(-centre_radius, centre_radius, 3)
        if np.linalg.norm(c) <= centre_radius:
            centres.append(c)
    centres = np.array(centres)
    rots = []
    for _ in range(n_clusters):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        rots.append(np.array([
            [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
            [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
            [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]]))
    rots = np.array(rots)
    sig = np.exp(rng.uniform(math.log(0.1), math.log(1.0), (n_clusters, 3)))
    means = np.empty((n, 3))
    todo = np.arange(n)
    while todo.size:
        k = rng.integers(0, n_clusters, todo.size)
        z = rng.standard_normal((todo.size, 3)) * sig[k]
        p = centres[k] + np.einsum("nij,nj->ni", rots[k], z)
        ok = np.linalg.norm(p, axis=1) <= reject_radius
        means[todo[ok]] = p[ok]
        todo = todo[~ok]
    return _attributes(rng, means, log_scale_mu, log_scale_sigma, sh_degree,
                       mask_mu0=mask_mu0)


def target_image(height, width, seed=TARGET_SEED, channels=3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, (channels, height, width)).astype(np.float32)


# --- named workloads -------------------------------------------------------

def tiny_workload(n=10_000):
    """10k Gaussians in [-1,1]^3, one 128x128 camera at radius 3, 60 deg FoV."""
    g = uniform_gaussians(n)
    f = 64.0 / math.tan(math.radians(30.0))
    cam = look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 128, 128, f)
    return g, [cam], target_image(128, 128)


def scene_workload(n=1_200_000, views=1, width=1557, height=1038, focal=1150.0,
                   ring_radius=4.0):
    """1.2M clustered Gaussians, cameras on a radius-4 ring at 1557x1038, f=1150 px."""
    g = cluster_gaussians(n)
    cams = [ring_camera(2 * math.pi * k / max(views, 1), ring_radius, width, height,
                        focal) for k in range(views)]
    return g, cams, target_image(height, width)


def converged_mask_logits(n, absent_fraction=0.624, seed=SCENE_SEED + 7) -> np.ndarray:
    """Mask scores of the kind a trained model ends with (a stand-in: no
    trained weights are available): a fraction of the Gaussians with
    l_0 - l_1 ~ N(-7, 1) (almost never sampled), the rest ~ N(3, 1).  The
    default fraction is the pruning ratio the paper reports on Mip-NeRF360
    (62.4 %, Sec. 4.2)."""
    rng = np.random.default_rng(seed)
    absent = rng.random(n) < absent_fraction
    d = np.where(absent, rng.normal(-7.0, 1.0, n), rng.normal(3.0, 1.0, n))
    out = np.zeros((n, 2), np.float32)
    out[:, 0] = d.astype(np.float32)
    return out


# --- workload definitions (workloads.json) and scene files ------------------

WORKLOADS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")


@dataclass
class Workload:
    """A named workload: every scene's Gaussians concatenated, the cameras,
    one target image per camera, each camera's (first, count) range of the
    concatenation (None: every camera sees all of it), the storage types the
    workload is measured with, and per scene (Gaussians, cameras, targets)."""
    name: str
    gaussians: Gaussians
    cams: list
    targets: list
    view_ranges: list | None
    storage: tuple
    parts: list
    spec: dict


def load_workloads(path: str | None = None) -> dict:
    with open(path or WORKLOADS_FILE) as fh:
        return json.load(fh)


def concat_gaussians(gs) -> Gaussians:
    """One Gaussians holding the given ones in order (a scene batch)."""
    cat = {k: np.concatenate([getattr(s, k) for s in gs]) for k in
           ("means", "log_scales", "quats", "opacity_logit", "sh", "mask_logits")}
    return Gaussians(**cat, sh_degree=gs[0].sh_degree)


def _scene_of(spec: dict) -> Gaussians:
    kind = spec["distribution"]
    if kind == "uniform":
        return uniform_gaussians(spec["gaussians"], seed=spec["seed"])
    if kind == "clusters":
        return cluster_gaussians(spec["gaussians"], seed=spec["seed"])
    raise ValueError(f"unknown scene distribution {kind!r}")


def _cameras_of(spec: dict, n_scenes: int) -> list:
    kind = spec["kind"]
    if kind == "look_at":
        w, h = spec["width"], spec["height"]
        f = (w / 2.0) / math.tan(math.radians(spec["fov_deg"] / 2.0))
        return [look_at_camera(tuple(spec["eye"]), tuple(spec["target"]), w, h, f)]
    if kind == "ring":
        w, h, k_n = spec["width"], spec["height"], spec["count"]
        f = spec["focal"] * w / spec["focal_width"]
        return [ring_camera(2 * math.pi * k / k_n, spec["radius"], w, h, f) for k in range(k_n)]
    if kind == "ring_per_scene":
        res = spec["resolutions"]
        if len(res) != n_scenes:
            raise ValueError("one resolution per scene")
        return [ring_camera(spec["theta_step"] * k, spec["radius"], w, h,
                            spec["focal"] * w / spec["focal_width"])
                for k, (w, h) in enumerate(res)]
    raise ValueError(f"unknown camera kind {kind!r}")


def workload(name: str, path: str | None = None) -> Workload:
    """Build the named workload of workloads.json (c1_tiny ... c5_uneven)."""
    spec = load_workloads(path)[name]
    scs = [_scene_of(s) for s in spec["scenes"]]
    cams = _cameras_of(spec["cameras"], len(scs))
    seeds = spec["target_seeds"]
    if len(seeds) != len(cams):
        raise ValueError("one target seed per camera")
    targets = [target_image(c.height, c.width, seed=s) for c, s in zip(cams, seeds)]
    if len(scs) == 1:
        g, ranges, parts = scs[0], None, [(scs[0], cams, targets)]
    else:
        if len(cams) != len(scs):
            raise ValueError("a scene batch has one camera per scene")
        g = concat_gaussians(scs)
        offs = np.concatenate([[0], np.cumsum([s.n for s in scs])[:-1]])
        ranges = [(int(o), s.n) for o, s in zip(offs, scs)]
        parts = [(s, [c], [t]) for s, c, t in zip(scs, cams, targets)]
    return Workload(name, g, cams, targets, ranges, tuple(spec["storage"]), parts, spec)


def save_npz(path: str, g: Gaussians, cams=(), targets=()) -> None:
    """Write a scene (and optionally its cameras and target images) to one
    .npz file; ``load_npz`` gives back bit-identical arrays."""
    arrays = {k: getattr(g, k) for k in
              ("means", "log_scales", "quats", "opacity_logit", "sh", "mask_logits")}
    arrays["sh_degree"] = np.int64(g.sh_degree)
    for i, c in enumerate(cams):
        arrays[f"cam{i}_intrinsics"] = np.array([c.width, c.height, c.fx, c.fy, c.cx, c.cy,
                                                 c.near], dtype=np.float64)
        arrays[f"cam{i}_viewmat"] = c.viewmat
        arrays[f"cam{i}_pos"] = c.cam_pos
    for i, t in enumerate(targets):
        arrays[f"target{i}"] = t
    np.savez(path, **arrays)


def load_npz(path: str):
    """(Gaussians, cameras, targets) from a file written by ``save_npz``."""
    with np.load(path) as z:
        g = Gaussians(*(z[k].copy() for k in ("means", "log_scales", "quats", "opacity_logit",
                                               "sh", "mask_logits")),
                      sh_degree=int(z["sh_degree"]))
        cams, targets = [], []
        i = 0
        while f"cam{i}_intrinsics" in z:
            w, h, fx, fy, cx, cy, near = z[f"cam{i}_intrinsics"].tolist()
            cams.append(Camera(int(w), int(h), fx, fy, cx, cy, z[f"cam{i}_viewmat"].copy(),
                               z[f"cam{i}_pos"].copy(), near))
            i += 1
        i = 0
        while f"target{i}" in z:
            targets.append(z[f"target{i}"].copy())
            i += 1
    return g, cams, targets
