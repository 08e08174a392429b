"""Pins for the scatter step of the oracle's CPU ray tracer (CPU only).

The wavefront tracer's Lambertian bounce (Section V-B application; scene reading
of the ray-tracing workload): at a hit point p on sphere (c, r) the throughput
is multiplied by the sphere's albedo and the ray continues from p along
normalize(n + q), n = (p - c) / r the outward normal and q the first point of
the keyed rejection sequence that lies inside the unit ball; after
`max_bounces` scatterings a further hit contributes zero.

Pins that a wrong scatter step fails (each is also run against planted
mistakes compiled from a modified copy of oracle/rt.cpp, which must fail at
least one of them):
  * convex sphere, one bounce: a ray leaving a convex sphere along a direction
    with a positive normal component never meets it again, so every pixel whose
    primary ray hits the sphere traces exactly two segments and ends in the
    sky; its radiance is albedo * sky(d2), so blue equals the blue albedo and
    the sky parameter recovered from red and from green agree;
  * bounce limit: max_bounces = 0 makes hit pixels black after one segment;
    max_bounces = 1 does not;
  * float64 single bounce: the radiance of each hit pixel recomputed in float64
    from the scene, the camera and the keyed SplitMix64 draws;
  * mean direction: for q uniform in the unit ball, E[normalize(n + q)] = 0.8 n
    (closed form, also checked by numerical quadrature below), so regressing the
    recovered bounce direction's y on n.y over the hit pixels gives slope 0.8.
"""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")

W, H = 129, 81
SCALE = (0.6, 0.4)
CAM = (0.5, 0.5, -1.5)
CENTRE = (0.5, 0.5, 0.0)
RADIUS = 0.5
ALBEDO = (0.25, 0.5, 0.75)
SEED = 7


def _scene(albedo=ALBEDO):
    return {"centre": np.asarray([CENTRE], np.float32), "radius": np.asarray([RADIUS], np.float32),
            "albedo": np.asarray([albedo], np.float32), "scale": SCALE, "camera": CAM}


# ---------------------------------------------------------------------------
# float64 geometry of the primary rays (independent of the oracle's code)
# ---------------------------------------------------------------------------

def _primary():
    px = np.arange(W * H)
    pxx, pyy = px % W, px // W
    sx, sy = float(np.float32(SCALE[0])), float(np.float32(SCALE[1]))
    u = (2.0 * ((pxx + 0.5) / W) - 1.0) * sx
    v = (1.0 - 2.0 * ((pyy + 0.5) / H)) * sy
    d = np.stack([u, v, np.ones_like(u)], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.asarray(CAM, np.float64)
    c = np.asarray(CENTRE, np.float64)
    oc = o - c
    b = d @ oc
    cc = oc @ oc - RADIUS * RADIUS
    disc = b * b - cc
    hit = disc > 0
    t = -b - np.sqrt(np.where(hit, disc, 0.0))
    p = o + t[:, None] * d
    n = (p - c) / RADIUS
    # angle of the ray to the camera -> centre axis and the silhouette half angle
    axis = (c - o) / np.linalg.norm(c - o)
    ang = np.arccos(np.clip(d @ axis, -1.0, 1.0))
    lim = math.asin(RADIUS / np.linalg.norm(c - o))
    inner = ang < lim - 0.02          # comfortably inside the silhouette (no grazing hits)
    outer = ang > lim + 0.02
    return px, d, p, n, inner, outer


def _unit_ball_point(pix, bounce=0):
    """First candidate of the keyed rejection sequence inside the unit ball.
    The in-ball test is taken in fp32 with the tracer's summation order (a float
    comparison that decides which candidate is used)."""
    for a in range(32):
        key = (((pix * 16 + bounce) * 64 + a) * 4)
        r = synth.splitmix64(SEED, np.asarray([key, key + 1, key + 2], np.uint64)) >> np.uint64(40)
        cf = (np.float32(2.0) * (r.astype(np.float32) * np.float32(1.0 / 16777216.0)) - np.float32(1.0))
        s = cf[0] * cf[0]
        s = np.float32(s + cf[1] * cf[1])
        s = np.float32(s + cf[2] * cf[2])
        if s < np.float32(1.0):
            return cf.astype(np.float64)
    return np.zeros(3)


def _sky(d):
    s = 0.5 * (d[..., 1] + 1.0)
    return np.stack([(1 - s) + s * 0.5, (1 - s) + s * 0.7, (1 - s) + s * 1.0], axis=-1)


# ---------------------------------------------------------------------------
# renderers: the oracle, or a planted-mistake build of its tracer
# ---------------------------------------------------------------------------

def _render_with(lib):
    def render(scene, width, height, pixels, max_bounces=8, seed=0):
        centre = np.ascontiguousarray(scene["centre"], dtype=np.float32)
        radius = np.ascontiguousarray(scene["radius"], dtype=np.float32)
        albedo = np.ascontiguousarray(scene["albedo"], dtype=np.float32)
        cam = scene["camera"]
        S = oracle.RtScene(width, height, max_bounces, len(radius), cam[0], cam[1], cam[2], scene["scale"][0],
                           scene["scale"][1], seed, centre.ctypes.data, radius.ctypes.data, albedo.ctypes.data)
        pixels = np.ascontiguousarray(pixels, dtype=np.int64)
        rgb = np.zeros((len(pixels), 3), dtype=np.float32)
        segs = np.zeros(len(pixels), dtype=np.int32)
        lib.orc_render_pixels(ctypes.byref(S), pixels.ctypes.data, len(pixels), rgb.ctypes.data, segs.ctypes.data, 4)
        return rgb, segs
    return render


def _oracle_render(scene, width, height, pixels, max_bounces=8, seed=0):
    return oracle.render_pixels(scene, width, height, pixels, max_bounces=max_bounces, seed=seed)


# ---------------------------------------------------------------------------
# the pins
# ---------------------------------------------------------------------------

def pin_convex_one_bounce(render):
    px, d, p, n, inner, outer = _primary()
    a = np.asarray(ALBEDO, np.float64)
    for mb in (1, 8):
        rgb, segs = render(_scene(), W, H, px, max_bounces=mb, seed=SEED)
        assert (segs[outer] == 1).all(), "a miss traces one segment"
        assert (segs[inner] == 2).all(), "a hit on a convex sphere traces exactly two segments"
        c = rgb[inner].astype(np.float64)
        assert np.allclose(c[:, 2], a[2], rtol=2e-6, atol=0), "blue = albedo_b * sky_b = albedo_b"
        s_r = (1.0 - c[:, 0] / a[0]) / 0.5
        s_g = (1.0 - c[:, 1] / a[1]) / 0.3
        assert np.allclose(s_r, s_g, atol=1e-4), "one sky direction explains red and green"
        assert (s_r > -1e-5).all() and (s_r < 1 + 1e-5).all(), "radiance within albedo x [sky min, sky max]"


def pin_bounce_limit(render):
    px, d, p, n, inner, outer = _primary()
    rgb, segs = render(_scene(), W, H, px, max_bounces=0, seed=SEED)
    assert (rgb[inner] == 0).all() and (segs[inner] == 1).all(), "no scattering allowed: hits are black"
    rgb, segs = render(_scene(), W, H, px, max_bounces=1, seed=SEED)
    assert (rgb[inner] > 0).all(), "one scattering allowed: the bounced ray reaches the sky"


def pin_float64_single_bounce(render):
    px, d, p, n, inner, outer = _primary()
    sel = np.nonzero(inner)[0][::7]            # a sample of the hit pixels
    rgb, segs = render(_scene(), W, H, px[sel], max_bounces=1, seed=SEED)
    a = np.asarray(ALBEDO, np.float64)
    want = np.zeros((len(sel), 3))
    for j, i in enumerate(sel):
        q = _unit_ball_point(int(px[i]), 0)
        w = n[i] + q
        d2 = w / np.linalg.norm(w)
        want[j] = a * _sky(d2)
    assert np.allclose(rgb, want, rtol=0, atol=2e-5), np.abs(rgb - want).max()


def pin_mean_direction(render):
    px, d, p, n, inner, outer = _primary()
    rgb, segs = render(_scene(), W, H, px, max_bounces=1, seed=SEED)
    a = np.asarray(ALBEDO, np.float64)
    c = rgb[inner].astype(np.float64)
    s = (1.0 - c[:, 0] / a[0]) / 0.5
    dy = 2.0 * s - 1.0                         # y of the bounce direction
    ny = n[inner, 1]
    slope = np.polyfit(ny, dy, 1)[0]
    assert inner.sum() > 2000
    assert abs(slope - 0.8) < 0.05, slope
    resid = dy - 0.8 * ny
    assert abs(resid.mean()) < 4 * resid.std() / math.sqrt(len(resid)) + 1e-3


PINS = [pin_convex_one_bounce, pin_bounce_limit, pin_float64_single_bounce, pin_mean_direction]


def test_closed_form_mean_of_ball_bounce_by_quadrature():
    # E[n . normalize(n + q)] for q uniform in the unit ball, n a unit vector:
    # (3/2) int_0^1 int_{-1}^{1} r^2 (1 + r m) / sqrt(1 + r^2 + 2 r m) dm dr = 4/5
    from scipy import integrate
    val, err = integrate.dblquad(lambda m, r: 1.5 * r * r * (1 + r * m) / math.sqrt(1 + r * r + 2 * r * m),
                                 0.0, 1.0, -1.0, 1.0)
    assert abs(val - 0.8) < 1e-7
    # and the tangential mean vanishes by symmetry; a cosine-weighted sampler
    # (q on the unit sphere) would give 2/3 instead, which the 0.05 margin excludes
    val2, _ = integrate.quad(lambda m: 0.5 * (1 + m) / math.sqrt(2 + 2 * m), -1.0, 1.0)
    assert abs(val2 - 2.0 / 3.0) < 1e-7


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_oracle_passes(pin):
    pin(_oracle_render)


# planted mistakes: (name, original text, replacement) in oracle/rt.cpp
MUTANTS = [
    ("inverted_normal", "const V3 w = {n.x + q.x, n.y + q.y, n.z + q.z};",
     "const V3 w = {-n.x + q.x, -n.y + q.y, -n.z + q.z};"),
    ("n_minus_p", "const V3 w = {n.x + q.x, n.y + q.y, n.z + q.z};",
     "const V3 w = {n.x - q.x, n.y - q.y, n.z - q.z};"),
    ("bounce_limit_early", "if (bounce == S.max_bounces) {", "if (bounce + 1 >= S.max_bounces) {"),
    ("bounce_limit_late", "if (bounce == S.max_bounces) {", "if (bounce == S.max_bounces + 1) {"),
    ("albedo_channel_swap", "tp.y * S.albedo[3 * hit + 1]", "tp.y * S.albedo[3 * hit + 2]"),
    ("cube_not_ball", "if (dot3(c, c) < 1.0f) {", "if (dot3(c, c) < 3.0f) {"),
    ("normal_unscaled", "const float r = S.radius[hit];\n        const V3 n = {(p.x - S.centre[3 * hit]) / r,",
     "const float r = S.radius[hit] * 0.5f;\n        const V3 n = {(p.x - S.centre[3 * hit]) / r,"),
]


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    return tmp_path_factory.mktemp("rt_mutants")


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_rejected(mutant_dir, name, old, new):
    src = open(os.path.join(ORACLE_DIR, "rt.cpp")).read()
    assert src.count(old) == 1, "the planted mistake no longer matches the tracer's source"
    d = mutant_dir / name
    d.mkdir()
    (d / "rt.cpp").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ORACLE_DIR, "oracle.h"), d / "oracle.h")
    so = d / "librt_mutant.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                           "-o", str(so), str(d / "rt.cpp")])
    lib = ctypes.CDLL(str(so))
    lib.orc_render_pixels.argtypes = [ctypes.POINTER(oracle.RtScene), ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
    lib.orc_render_pixels.restype = None
    render = _render_with(lib)
    failed = []
    for pin in PINS:
        try:
            pin(render)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, "planted mistake %s passed every scatter pin" % name
