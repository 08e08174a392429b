"""Pins for the oracle's CPU ray tracer (CPU only): closed forms on the optical
axis, mirror symmetry of the empty scene, the analytic silhouette of one
sphere, black albedo, and the energy and path-length bounds."""
import math

import numpy as np
import pytest

import oracle
import synth

W, H = 33, 21          # odd sizes: pixel (16, 10) looks exactly along +z


def _scene(centres, radii, albedo, scale=(0.6, 0.4), cam=(0.5, 0.5, -1.5)):
    return {"centre": np.asarray(centres, np.float32).reshape(-1, 3), "radius": np.asarray(radii, np.float32),
            "albedo": np.asarray(albedo, np.float32).reshape(-1, 3), "scale": scale, "camera": cam}


def test_empty_scene_axis_pixel_closed_form():
    sc = _scene(np.zeros((0, 3)), [], np.zeros((0, 3)))
    rgb, segs = oracle.render_pixels(sc, W, H, [10 * W + 16])
    # d = (0, 0, 1): s = 0.5, sky = (0.5 + 0.25, 0.5 + 0.35, 0.5 + 0.5), all exact in binary
    assert rgb[0].tolist() == [0.75, 0.8500000238418579, 1.0]
    assert segs[0] == 1


def test_empty_scene_mirror_symmetry_and_vertical_order():
    sc = _scene(np.zeros((0, 3)), [], np.zeros((0, 3)))
    px = np.arange(W * H)
    rgb, segs = oracle.render_pixels(sc, W, H, px)
    img = rgb.reshape(H, W, 3)
    # u -> -u leaves d.y unchanged (up to the rounding of the pixel-centre arithmetic)
    assert np.allclose(img, img[:, ::-1], rtol=1e-6, atol=0)
    # rows higher in the image look more upward: red falls monotonically going up
    col = img[:, 16, 0]
    assert (np.diff(col) > 0).all()
    assert (segs == 1).all()


def test_single_sphere_silhouette_matches_analytic_cone():
    c, r = (0.5, 0.5, 0.0), 0.25
    sc = _scene([c], [r], [0.5, 0.5, 0.5])
    px = np.arange(W * H)
    rgb, segs = oracle.render_pixels(sc, W, H, px, max_bounces=0)
    hit = (rgb == 0).all(axis=1)                   # max_bounces = 0: a hit contributes 0
    # analytic: the primary ray hits iff its angle to the camera->centre axis is below asin(r / 1.5)
    pxx, pyy = px % W, px // W
    u = (2 * ((pxx + 0.5) / W) - 1) * 0.6
    v = (1 - 2 * ((pyy + 0.5) / H)) * 0.4
    cosang = 1.0 / np.sqrt(u * u + v * v + 1.0)
    ang = np.arccos(np.clip(cosang, -1, 1))
    lim = math.asin(r / 1.5)
    clear = np.abs(ang - lim) > 1e-3
    assert hit[clear].tolist() == (ang < lim)[clear].tolist()
    assert hit.sum() > 10


def test_black_albedo_gives_black_hits():
    sc = _scene([(0.5, 0.5, 0.0)], [0.25], [0.0, 0.0, 0.0])
    rgb, segs = oracle.render_pixels(sc, W, H, [10 * W + 16], max_bounces=8)
    assert rgb[0].tolist() == [0.0, 0.0, 0.0]


def test_random_scene_bounds():
    sc = synth.sphere_scene(512, seed=3)
    sc["scale"] = synth.camera_scale(64, 36)
    rgb, segs = oracle.render_pixels(sc, 64, 36, np.arange(64 * 36), max_bounces=4)
    assert (rgb >= 0).all()
    assert (rgb[:, 0] <= 1.0).all() and (rgb[:, 2] <= 1.0).all()   # albedo < 1, sky <= 1
    assert segs.max() <= 5 and segs.min() >= 1
    assert (segs > 1).mean() > 0.05                                 # some primary rays hit
