"""Tile-based wavefront ray tracing on the GPU against the oracle's sequential
CPU tracer (run with -m gpu).  Per-pixel radiance must agree within 1e-5
relative (both sides round every fp32 operation in the same order, so it is
expected to be bit-identical); every pixel must finish."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_01693_gb300 as gq
import synth

pytestmark = pytest.mark.gpu
KINDS = list(gq.READY_KINDS)


def _close(a, b, rel=1e-5):
    return np.abs(a - b) <= rel * np.maximum(np.abs(a), np.abs(b)) + 1e-30


def _render(kind, scene, W, H, tiles, bounces=8, seed=0):
    r = gq.Renderer(kind, scene, W, H, tiles=tiles, max_bounces=bounces, seed=seed)
    img = r.render().cpu().numpy()
    st = r.stats.cpu().numpy()
    for q in r.queues:
        assert q.sync_status() == 0
    assert st[2] == 0, "error flags %d" % st[2]
    assert st[1] == W * H
    return img, st


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("W,H,tiles,ns,bounces", [(96, 54, (4, 3), 512, 8), (41, 23, (2, 5), 64, 3),
                                                  (64, 64, (8, 8), 4096, 8)])
def test_small_image_matches_cpu_tracer(kind, W, H, tiles, ns, bounces):
    sc = synth.sphere_scene(ns, seed=ns)
    sc["scale"] = synth.camera_scale(W, H)
    img, st = _render(kind, sc, W, H, tiles, bounces, seed=5)
    want, segs = oracle.render_pixels(sc, W, H, np.arange(W * H), max_bounces=bounces, seed=5)
    got = img.reshape(-1, 3)
    assert _close(got, want).all()
    assert st[0] == int(segs.sum())
    assert (got == want).mean() > 0.999          # bit-identical in practice


def test_empty_scene_is_sky():
    sc = {"centre": np.zeros((0, 3), np.float32), "radius": np.zeros(0, np.float32),
          "albedo": np.zeros((0, 3), np.float32), "scale": synth.camera_scale(33, 21)}
    for kind in KINDS:
        img, st = _render(kind, sc, 33, 21, (3, 3))
        want, segs = oracle.render_pixels(sc, 33, 21, np.arange(33 * 21))
        assert (img.reshape(-1, 3) == want).all()
        assert st[0] == 33 * 21


@pytest.mark.parametrize("kind", KINDS)
def test_full_size_sampled_pixels(kind):
    # 1920 x 1080, 4096 spheres (radii lognormal mu -4, sigma 0.5), <= 8 bounces, 8 x 8 tile queues
    W, H = 1920, 1080
    sc = synth.sphere_scene(4096, seed=0)
    sc["scale"] = synth.camera_scale(W, H)
    img, st = _render(kind, sc, W, H, (8, 8))
    rng = np.random.default_rng(42)
    pix = np.concatenate([rng.integers(0, W * H, 3000), np.arange(0, W), np.arange(W * H - W, W * H)])
    want, segs = oracle.render_pixels(sc, W, H, pix)
    got = img.reshape(-1, 3)[pix]
    assert _close(got, want).all()
    assert st[0] > W * H                          # some rays bounced
