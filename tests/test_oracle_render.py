"""Pins of the oracle's rendering of a regular VDI from another viewpoint
(oracle.render_view / render_ray), on the CPU.

- From the generating view the rendering is the flattened VDI.
- A VDI whose every column holds the same shell [f, b] is one homogeneous
  emission-absorption medium filling (shell of G's eye) x (G's frustum): the
  opacity of a ray is 1 - (1 - A)^(L / (b - f)) with L the ray's length
  inside that region, computed here from ray-sphere and ray-plane
  intersections written independently of the oracle.
- A non-uniform VDI (lists with gaps, several records per column) against a
  brute-force Riemann integration of the same medium along the ray, with
  rays that pass G's eye at their closest point inside the frustum (so that
  the distance from G's eye first falls, then rises).
"""
import math
from dataclasses import dataclass

import numpy as np

import oracle
import synth


@dataclass
class Cam:
    eye: tuple
    center: tuple
    up: tuple
    fovy_deg: float
    width: int
    height: int


def frame(c):
    e = np.array(c.eye, float)
    fwd = np.array(c.center, float) - e
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.array(c.up, float))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    th = math.tan(math.radians(c.fovy_deg) / 2)
    return e, fwd, right, up, th, c.width / c.height


def orbit_cam(theta_deg, W, H, dist=3.0, fovy=40.0):
    t = math.radians(theta_deg)
    return Cam((dist * math.sin(t), 0.3 * dist * math.sin(t), -dist * math.cos(t)), (0.0, 0.0, 0.0),
               (0.0, 1.0, 0.0), fovy, W, H)


def random_vdi(W, H, n_s, seed, depth0=2.4, depth_len=1.2):
    """Regular VDI (counts, recs[W H, n_s, 6]) from the seeded synthetic lists, depths mapped to
    [depth0, depth0 + depth_len]."""
    counts = np.zeros(W * H, np.int32)
    recs = np.zeros((W * H, n_s, 6))
    for p in range(W * H):
        fb, rgba = synth.one_list(seed, 0, 0, p, n_s)
        n = len(fb)
        counts[p] = n
        recs[p, :n, 0:2] = depth0 + depth_len * fb.astype(np.float64)
        recs[p, :n, 2:6] = rgba
    return counts, recs


def test_generating_view_equals_flatten():
    W, H, n_s = 24, 18, 6
    gen = orbit_cam(0.0, W, H)
    counts, recs = random_vdi(W, H, n_s, 101)
    img = oracle.render_view(counts, recs, gen, gen)
    flat = oracle.flatten(counts, recs)
    assert np.abs(img - flat).max() < 1e-12


def frustum_interval(gen, o, d):
    """s-interval of the ray inside G's frustum, from the four side planes through G's eye."""
    e, fwd, right, up, th, asp = frame(gen)
    corners = [fwd + sx * th * asp * right + sy * th * up for sx, sy in ((-1, -1), (1, -1), (1, 1), (-1, 1))]
    lo, hi = 0.0, math.inf
    centre = fwd
    for a in range(4):
        n = np.cross(corners[a], corners[(a + 1) % 4])
        if np.dot(n, centre) < 0:
            n = -n
        # inside: n . (x - e) >= 0
        a0 = np.dot(n, o - e)
        b0 = np.dot(n, d)
        if b0 == 0:
            if a0 < 0:
                return 0.0, 0.0
            continue
        s = -a0 / b0
        if b0 > 0:
            lo = max(lo, s)
        else:
            hi = min(hi, s)
    return lo, hi


def shell_length(e, o, d, r0, r1, lo, hi):
    """Length of {s in [lo, hi] : r0 <= |o + s d - e| <= r1} (unit d)."""
    q = o - e
    bq = np.dot(q, d)
    cq = np.dot(q, q)

    def inside_ball(r):
        disc = bq * bq - (cq - r * r)
        if disc <= 0:
            return None
        sq = math.sqrt(disc)
        return (-bq - sq, -bq + sq)

    def clip(iv):
        if iv is None:
            return 0.0
        a, b = max(iv[0], lo), min(iv[1], hi)
        return max(0.0, b - a)

    return clip(inside_ball(r1)) - clip(inside_ball(r0))


def test_homogeneous_shell_closed_form():
    W, H, n_s = 16, 12, 2
    gen = orbit_cam(0.0, W, H)
    f, b, A = 2.7, 3.3, 0.6
    col = np.array([0.2, 0.5, 0.8])
    counts = np.ones(W * H, np.int32)
    recs = np.zeros((W * H, n_s, 6))
    recs[:, 0, 0], recs[:, 0, 1] = f, b
    recs[:, 0, 2:5] = A * col
    recs[:, 0, 5] = A
    e = np.array(gen.eye, float)
    checked = 0
    for theta in (0.0, 12.0, 35.0, 70.0):
        view = orbit_cam(theta, 20, 15, dist=3.4)
        for j in range(0, 15, 3):
            for i in range(0, 20, 3):
                o, d = oracle.ray(view, i, j)
                o, d = np.asarray(o), np.asarray(d)
                lo, hi = frustum_interval(gen, o, d)
                L = shell_length(e, o, d, f, b, lo, hi) if hi > lo else 0.0
                alpha = 1 - (1 - A) ** (L / (b - f))
                got = oracle.render_ray(counts, recs, gen, o, d)
                assert abs(got[3] - alpha) < 1e-9, (theta, i, j, got, alpha)
                assert np.abs(got[0:3] - col * alpha).max() < 1e-9
                checked += L > 0
    assert checked > 40


def brute_force(counts, recs, gen, o, d, s_max, steps):
    """Riemann sum of the VDI's emission-absorption medium along o + s d, s in [0, s_max]."""
    e, fwd, right, up, th, asp = frame(gen)
    W, H = gen.width, gen.height
    ds = s_max / steps
    T, C = 1.0, np.zeros(3)
    for m in range(steps):
        x = o + (m + 0.5) * ds * d
        q = x - e
        z = np.dot(q, fwd)
        if z <= 0:
            continue
        X, Y = np.dot(q, right) / z, np.dot(q, up) / z
        u = (X / (th * asp) + 1) * 0.5 * W
        v = (1 - Y / th) * 0.5 * H
        if not (0 <= u < W and 0 <= v < H):
            continue
        p = int(v) * W + int(u)
        rho = np.linalg.norm(q)
        for k in range(counts[p]):
            f, b, A = recs[p, k, 0], recs[p, k, 1], recs[p, k, 5]
            if f <= rho < b and A > 0:
                mu = -math.log1p(-A) / (b - f) if A < 1 else 1e9
                a = 1 - math.exp(-mu * ds)
                C += T * recs[p, k, 2:5] / A * a
                T *= 1 - a
                break
    return np.array([*C, 1 - T])


def test_against_brute_force_integration():
    W, H, n_s = 10, 8, 5
    gen = orbit_cam(0.0, W, H, fovy=50.0)
    counts, recs = random_vdi(W, H, n_s, 202, depth0=2.3, depth_len=1.4)
    rng = np.random.default_rng(7)
    worst = 0.0
    for theta in (25.0, 80.0):
        view = orbit_cam(theta, 12, 9, dist=3.2, fovy=50.0)
        for _ in range(6):
            i, j = int(rng.integers(0, 12)), int(rng.integers(0, 9))
            o, d = (np.asarray(x) for x in oracle.ray(view, i, j))
            got = oracle.render_ray(counts, recs, gen, o, d)
            ref = brute_force(counts, recs, gen, o, d, 8.0, 40000)
            worst = max(worst, float(np.abs(got - ref).max()))
    assert worst < 2e-3, worst
    # the distance from G's eye falls, then rises, along rays of the side view
    e = np.array(gen.eye, float)
    view = orbit_cam(80.0, 12, 9, dist=3.2, fovy=50.0)
    o, d = (np.asarray(x) for x in oracle.ray(view, 6, 4))
    s_star = -np.dot(o - e, d)
    lo, hi = frustum_interval(gen, o, d)
    assert lo < s_star < hi


def test_empty_and_outside():
    W, H, n_s = 8, 6, 3
    gen = orbit_cam(0.0, W, H)
    counts = np.zeros(W * H, np.int32)
    recs = np.zeros((W * H, n_s, 6))
    img = oracle.render_view(counts, recs, gen, orbit_cam(30.0, 10, 8))
    assert not img.any()
    # a ray pointing away from G's frustum sees nothing
    counts, recs = random_vdi(W, H, n_s, 5)
    out = oracle.render_ray(counts, recs, gen, np.array([0.0, 0.0, -3.0]), np.array([0.0, 0.0, -1.0]))
    assert not out.any()


def test_view_from_behind_reverses_the_order():
    # G looks at the origin from (0, 0, -3); V looks back from (0, 0, 3) towards G's eye, so along V's
    # centre ray the distance from G's eye falls: the record farther from G is met first.
    W = H = 3
    n_s = 2
    gen = Cam((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 40.0, W, H)
    view = Cam((0.0, 0.0, 3.0), (0.0, 0.0, -3.0), (0.0, 1.0, 0.0), 40.0, 1, 1)
    red, blue, A = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0]), 0.9
    counts = np.full(W * H, 2, np.int32)
    recs = np.zeros((W * H, n_s, 6))
    recs[:, 0, 0:2] = (2.5, 2.8)
    recs[:, 0, 2:5] = A * red
    recs[:, 0, 5] = A
    recs[:, 1, 0:2] = (3.2, 3.5)
    recs[:, 1, 2:5] = A * blue
    recs[:, 1, 5] = A
    got = oracle.render_view(counts, recs, gen, view)[0]
    # radial path: each record crossed over its full thickness, so each has opacity A
    want = np.array([*(A * blue + (1 - A) * A * red), 1 - (1 - A) ** 2])
    assert np.abs(got - want).max() < 1e-9, (got, want)
