"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

Each test checks the oracle against something other than itself: closed
forms, brute force on tiny inputs, invariants the paper states (associativity
of "over" makes a VDI exact from its generating view, sec. 2.3; lists are
depth-sorted per PE, sec. 5.2; at most N_S supersegments per list, sec. 2.4),
or textbook special cases.  They are chosen so that a dropped term, a wrong
sign or index, or a transposed operand in the oracle fails at least one of
them (tests/test_oracle_mutations.py plants such mistakes and checks that).
"""
import math

import numpy as np
import pytest

import oracle
import synth

RNG = np.random.default_rng(1234)


def over(pieces):
    """Front-to-back over of premultiplied (P[3], a) rows."""
    C = np.zeros(3)
    A = 0.0
    for P, a in pieces:
        C = C + (1 - A) * np.asarray(P)
        A = A + (1 - A) * a
    return C, A


def rand_pieces(n, rng, p_transparent=0.2, contiguous=True):
    t = 0.0
    rows = []
    for _ in range(n):
        l = rng.uniform(0.1, 1.0)
        a = 0.0 if rng.random() < p_transparent else rng.uniform(0.01, 0.9)
        c = rng.uniform(0, 1, 3)
        rows.append([t, t + l, *(c * a), a])
        t += l if contiguous else l + rng.uniform(0, 0.5)
    return np.array(rows)


# ----------------------------------------------------------------------------
# Rays and sampling
# ----------------------------------------------------------------------------

def test_ray_through_centre_pixel_hits_centre():
    cam = synth.Camera((10.0, -3.0, 4.0), (1.0, 2.0, 3.0), (0.0, 0.0, 1.0), 45.0, 5, 3)
    o, d = oracle.ray(cam, 2, 1)  # centre of a 5 x 3 image
    fwd = np.subtract(cam.center, cam.eye)
    fwd /= np.linalg.norm(fwd)
    assert np.allclose(o, cam.eye)
    assert np.allclose(d, fwd, atol=1e-15)


def test_ray_corner_angles_match_fovy():
    # top edge of the image is fovy/2 above the view axis, the left edge at the aspect-scaled angle
    W, H, fovy = 200, 100, 60.0
    cam = synth.Camera((0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 0.0, 1.0), fovy, W, H)
    _, d = oracle.ray(cam, W // 2, 0)  # top row, centre column (pixel centre is half a pixel in)
    el = math.degrees(math.atan2(d[2], d[0]))
    th = math.tan(math.radians(fovy / 2))
    expect = math.degrees(math.atan((1 - 1 / H) * th))
    assert abs(el - expect) < 1e-9
    _, d = oracle.ray(cam, 0, H // 2)  # left column: right = fwd x up = -y, so left is +y
    az = math.degrees(math.atan2(d[1], d[0]))
    expect = math.degrees(math.atan((1 - 1 / W) * th * W / H))
    assert abs(az - expect) < 1e-6  # row H//2 is half a pixel off the axis vertically


def test_slab_test_matches_brute_force():
    dims = (9, 5, 7)
    for _ in range(200):
        o = RNG.uniform(-20, 20, 3)
        d = RNG.normal(size=3)
        d /= np.linalg.norm(d)
        hit, tin, tout = oracle.hit_box(o, d, dims)
        ts = np.linspace(0, 80, 160001)
        pts = o[None, :] + ts[:, None] * d[None, :]
        inside = np.all((pts >= 0) & (pts <= np.array(dims) - 1), axis=1)
        if not inside.any():
            assert not hit or tout - tin < 1e-3
            continue
        assert hit
        assert abs(ts[inside][0] - tin) < 1e-3 and abs(ts[inside][-1] - tout) < 1e-3


def test_trilinear_exact_at_nodes_and_on_trilinear_fields():
    vol = RNG.uniform(0, 1, (4, 5, 6)).astype(np.float32)  # (Z, Y, X)
    for _ in range(20):
        x, y, z = RNG.integers(0, 6), RNG.integers(0, 5), RNG.integers(0, 4)
        assert oracle.value(vol, (x, y, z)) == pytest.approx(float(vol[z, y, x]), abs=0)
    # a trilinear polynomial is reproduced exactly by trilinear interpolation
    Z, Y, X = np.meshgrid(np.arange(4), np.arange(5), np.arange(6), indexing="ij")
    f = lambda x, y, z: 0.1 + 0.02 * x + 0.03 * y - 0.01 * z + 0.004 * x * y + 0.002 * y * z - 0.001 * x * z + 0.0005 * x * y * z
    vol = f(X, Y, Z).astype(np.float64)
    vol32 = vol.astype(np.float32)
    for _ in range(50):
        p = RNG.uniform([0, 0, 0], [5, 4, 3])
        exact = f(*p)
        # nodes are float32, so allow their rounding (< 1e-7 relative)
        assert abs(oracle.value(vol32, p) - exact) < 1e-7
    # clamping outside the box: value at the nearest face
    assert oracle.value(vol32, (-1.0, 0.0, 0.0)) == pytest.approx(float(vol32[0, 0, 0]))
    assert oracle.value(vol32, (9.0, 4.0, 3.0)) == pytest.approx(float(vol32[3, 4, 5]))


def test_uint16_volume_scaling():
    vol = np.array([[[0, 65535], [65535, 0]], [[32768, 0], [0, 65535]]], dtype=np.uint16)
    assert oracle.value(vol, (1, 0, 0)) == 1.0
    assert oracle.value(vol, (0, 0, 1)) == pytest.approx(32768 / 65535, abs=1e-15)


def test_lut_correction_and_classification():
    lut = synth.transfer_function(synth.SEED_TF)
    # step == reference length: unchanged
    c1 = oracle.lut_correct(lut, 1.0, 1.0)
    assert np.allclose(c1, lut.astype(np.float64), atol=1e-15)
    # two half steps composite to one full step: 1 - (1 - a')^2 == a
    ch = oracle.lut_correct(lut, 0.5, 1.0)
    a = lut[:, 3].astype(np.float64)
    assert np.allclose(1 - (1 - ch[:, 3]) ** 2, a, atol=1e-15)
    assert np.all(ch[:, 3] <= a + 1e-15)
    # colours are not touched
    assert np.array_equal(ch[:, :3], lut[:, :3].astype(np.float64))
    # at v = i/255 the table entry itself; half way between two entries the mean
    for i in [0, 1, 77, 200, 254, 255]:
        assert np.allclose(oracle.classify(ch, i / 255.0), ch[i], atol=1e-12)
    mid = oracle.classify(ch, 100.5 / 255.0)
    assert np.allclose(mid, 0.5 * (ch[100] + ch[101]), atol=1e-12)


def test_tiny_volume_dvr_closed_form():
    # constant 2x2x2 volume, axis-aligned ray through the box along +x at y = z = 0.5:
    # the chord is [0, 1] in x, step 0.25 gives 4 samples, A = 1 - (1 - a')^4.
    vol = np.full((2, 2, 2), 0.6, dtype=np.float32)
    lut = np.zeros((256, 4), dtype=np.float32)
    lut[:, 0] = 0.25
    lut[:, 1] = 0.5
    lut[:, 2] = 1.0
    lut[:, 3] = 0.3
    cam = synth.Camera((-5.0, 0.5, 0.5), (0.0, 0.5, 0.5), (0.0, 0.0, 1.0), 10.0, 1, 1)
    rgba = oracle.dvr(vol, lut, cam, 0.25, 1.0)[0]
    a_tab = float(np.float32(0.3))
    a = 1 - (1 - a_tab) ** 0.25
    A = 1 - (1 - a) ** 4
    assert rgba[3] == pytest.approx(A, abs=1e-15)
    assert np.allclose(rgba[:3], np.array([0.25, 0.5, 1.0], dtype=np.float32) * A, atol=1e-15)
    # the corrected opacity over the whole unit chord equals the table's per-unit opacity
    assert A == pytest.approx(a_tab, abs=1e-15)


def test_tiny_volume_dvr_linear_ramp_brute_force():
    # value ramps linearly in x; ray along x through node rows: sample values are
    # known exactly, so DVR is a hand-computable product
    vol = np.zeros((2, 2, 3), dtype=np.float32)
    vol[:, :, 0], vol[:, :, 1], vol[:, :, 2] = 0.0, 0.5, 1.0
    lut = np.zeros((256, 4), dtype=np.float32)
    lut[:, 3] = np.linspace(0, 0.5, 256, dtype=np.float32)
    lut[:, 0] = 1.0
    cam = synth.Camera((-3.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), 10.0, 1, 1)
    step = 0.5
    rgba = oracle.dvr(vol, lut, cam, step, 1.0)[0]
    lc = oracle.lut_correct(lut, step, 1.0)
    A = 0.0
    C = 0.0
    for k in range(4):  # chord [0, 2] in x, midpoints 0.25, 0.75, 1.25, 1.75 -> v = x/2
        v = (k + 0.5) * step / 2.0
        x = v * 255
        i = min(int(math.floor(x)), 254)
        w = x - i
        a = lc[i, 3] * (1 - w) + lc[i + 1, 3] * w
        C += (1 - A) * a
        A += (1 - A) * a
    assert rgba[3] == pytest.approx(A, abs=1e-15)
    assert rgba[0] == pytest.approx(C, abs=1e-15)


def test_sample_grid_midpoints_inside_chord():
    vol = np.zeros((33, 17, 9), dtype=np.float32)
    cam = synth.orbit((9, 17, 33), 1, 8, 8, 3)[0]
    for p in range(64):
        n, tin, tout = oracle.ray_sample_count(vol, cam, 0.5, p)
        if n == 0:
            continue
        # every midpoint t_in + (k + 1/2) step is inside; the next one is not
        assert tin + (n - 0.5) * 0.5 < tout <= tin + (n + 0.5) * 0.5


# ----------------------------------------------------------------------------
# Segmentation state machine (Eq. 1, Algorithm S1)
# ----------------------------------------------------------------------------

def test_gamma_zero_one_record_per_nontransparent_piece():
    pcs = rand_pieces(40, RNG)
    cnt, recs = oracle.segment(pcs, 0.0)
    nt = pcs[pcs[:, 5] > 0]
    assert cnt == len(nt) == len(recs)
    assert np.array_equal(recs[:, 0], nt[:, 0]) and np.array_equal(recs[:, 1], nt[:, 1])
    assert np.array_equal(recs[:, 2:6], nt[:, 2:6])


def test_gamma_two_single_record_is_over_of_all():
    pcs = rand_pieces(40, RNG)
    cnt, recs = oracle.segment(pcs, 2.0)
    assert cnt == 1
    nt = np.nonzero(pcs[:, 5] > 0)[0]
    assert recs[0, 0] == pcs[nt[0], 0] and recs[0, 1] == pcs[nt[-1], 1]
    C, A = over([(r[2:5], r[5]) for r in pcs])
    assert np.allclose(recs[0, 2:5], C, atol=1e-14) and recs[0, 5] == pytest.approx(A, abs=1e-14)


@pytest.mark.parametrize("alpha,length", [(0.3, 1.0), (0.05, 0.5), (0.9, 2.0)])
def test_homogeneous_medium_never_terminates(alpha, length):
    # identical pieces: S renormalised to the incoming length equals the piece,
    # so the distance is 0 and one supersegment absorbs all; A = 1 - (1 - a)^n.
    n = 50
    c = np.array([0.2, 0.7, 0.4])
    pcs = np.array([[i * length, (i + 1) * length, *(c * alpha), alpha] for i in range(n)])
    for g in [1e-9, 0.01, 0.05, 0.5]:
        cnt, recs = oracle.segment(pcs, g)
        assert cnt == 1
        assert recs[0, 5] == pytest.approx(1 - (1 - alpha) ** n, abs=1e-13)
        assert np.allclose(recs[0, 2:5], c * (1 - (1 - alpha) ** n), atol=1e-13)
        assert recs[0, 0] == 0.0 and recs[0, 1] == n * length


def test_unequal_lengths_renormalised():
    # a supersegment of two pieces of length 1 (opacity a each) compared with a piece
    # of length 2 and opacity 1 - (1 - a)^2 (the same medium): distance 0
    a = 0.4
    c = np.array([1.0, 0.5, 0.25])
    A2 = 1 - (1 - a) ** 2
    pcs = np.array([[0, 1, *(c * a), a], [1, 2, *(c * a), a], [2, 4, *(c * A2), A2]])
    cnt, recs = oracle.segment(pcs, 1e-9)
    assert cnt == 1
    # and a different medium of the same colour (higher density) is split off at small gamma
    pcs[2, 5] = 0.9
    pcs[2, 2:5] = c * 0.9
    cnt, _ = oracle.segment(pcs, 0.05)
    assert cnt == 2


def test_hand_case_three_pieces():
    # two equal red pieces then a blue one: gamma between 0 and the red/blue distance
    r = np.array([1.0, 0.0, 0.0]) * 0.5
    b = np.array([0.0, 0.0, 1.0]) * 0.5
    pcs = np.array([[0, 1, *r, 0.5], [1, 2, *r, 0.5], [2, 3, *b, 0.5]])
    cnt, recs = oracle.segment(pcs, 0.3)
    assert cnt == 2
    # first record: over of the two red pieces; second: the blue piece
    assert recs[0, 0] == 0 and recs[0, 1] == 2
    assert recs[0, 5] == pytest.approx(0.75)
    assert np.allclose(recs[0, 2:5], [0.75, 0, 0])
    assert np.allclose(recs[1], [2, 3, 0, 0, 0.5, 0.5])
    # distance red-S (renormalised 0.5 red) to blue piece = |(0.5,0,-0.5)| = 0.7071
    assert oracle.segment(pcs, 0.7071)[0] == 2
    assert oracle.segment(pcs, 0.7072)[0] == 1


def test_transparent_gap_absorbed_or_splits_and_back_is_last_opaque():
    c = np.array([0.5, 0.5, 0.5]) * 0.2
    pcs = np.array([[0, 1, *c, 0.2], [1, 2, 0, 0, 0, 0.0], [2, 3, *c, 0.2]])
    # gap distance = |C_S| * a~ with l_x / l_S = 1: |(0.5,0.5,0.5)| * 0.2 = 0.1732
    cnt, recs = oracle.segment(pcs, 0.2)
    assert cnt == 1 and recs[0, 1] == 3
    cnt, recs = oracle.segment(pcs, 0.17)
    assert cnt == 2 and recs[0, 1] == 1 and recs[1, 0] == 2
    # trailing transparency is absorbed but not part of the record's back depth
    pcs2 = np.array([[0, 1, *c, 0.2], [1, 2, 0, 0, 0, 0.0]])
    cnt, recs = oracle.segment(pcs2, 0.5)
    assert cnt == 1 and recs[0, 1] == 1


def test_cap_last_supersegment_absorbs_rest():
    pcs = rand_pieces(30, RNG, p_transparent=0.0)
    cnt, recs = oracle.segment(pcs, 0.0, cap=3)
    assert cnt == 3 and len(recs) == 3
    C, A = over([(r[2:5], r[5]) for r in pcs[2:]])
    assert np.allclose(recs[2, 2:5], C, atol=1e-14) and recs[2, 5] == pytest.approx(A, abs=1e-14)
    assert recs[2, 1] == pcs[-1, 1]


def test_break_closes_supersegment():
    c = np.array([0.3, 0.3, 0.3]) * 0.5
    pcs = np.array([[0, 1, *c, 0.5], [1, 2, *c, 0.5], [0, 0, 0, 0, 0, 0], [5, 6, *c, 0.5]])
    cnt, recs = oracle.segment(pcs, 2.0, brk=[0, 0, 1, 0])
    assert cnt == 2 and recs[0, 1] == 2 and recs[1, 0] == 5


def test_segmentation_preserves_over_any_gamma_cap():
    # associativity of over (sec. 2.3): flattening the records equals over of the pieces
    for _ in range(50):
        pcs = rand_pieces(int(RNG.integers(1, 60)), RNG)
        g = float(RNG.choice([0.0, RNG.uniform(0, 0.3), RNG.uniform(0, 2)]))
        cap = int(RNG.integers(1, 10))
        cnt, recs = oracle.segment(pcs, g, cap)
        assert cnt <= cap and len(recs) == cnt
        C, A = over([(r[2:5], r[5]) for r in recs])
        C0, A0 = over([(r[2:5], r[5]) for r in pcs])
        assert np.allclose(C, C0, atol=1e-13) and A == pytest.approx(A0, abs=1e-13)
        # records are disjoint, ordered, and span non-transparent pieces only
        for j in range(1, cnt):
            assert recs[j, 0] >= recs[j - 1, 1]


# ----------------------------------------------------------------------------
# gamma search (sec. 2.4)
# ----------------------------------------------------------------------------

def test_search_bracket_properties():
    iters = 16
    for trial in range(60):
        pcs = rand_pieces(int(RNG.integers(1, 80)), RNG, p_transparent=0.3)
        n_s = int(RNG.integers(1, 12))
        g, passes = oracle.search(pcs, n_s, iters)
        c0, _ = oracle.segment(pcs, 0.0)
        cg, _ = oracle.segment(pcs, g)
        assert 1 <= passes <= 1 + iters
        if c0 <= n_s:
            assert g == 0.0 and passes == 1
            continue
        assert cg <= n_s
        # the result is a dyadic point of the bisection grid on [0, 2]
        assert (g * 2 ** (iters - 1)) == int(g * 2 ** (iters - 1))
        if cg != n_s:
            # no early exit: the lower end of the final bracket was tested infeasible
            assert passes == 1 + iters
            lo = g - 2.0 ** (1 - iters)
            assert oracle.segment(pcs, lo)[0] > n_s


def test_search_full_bisection_closed_form():
    # red, green, red pieces of equal length and opacity a: for gamma <= D = a*sqrt(2) every
    # piece opens a supersegment (3 > n_s = 2); above D the green and then the second red are
    # absorbed (1 < n_s).  The count never equals n_s, so all 16 bisection steps run and the
    # result is the first grid point k * 2^-15 above D.
    for a in [0.3, 0.45, 0.6]:
        red, green = [a, 0.0, 0.0], [0.0, a, 0.0]
        pcs = np.array([[0, 1, *red, a], [1, 2, *green, a], [2, 3, *red, a]])
        D = a * math.sqrt(2.0)
        g, passes = oracle.search(pcs, 2, 16)
        assert passes == 17
        assert g == (math.floor(D * 2 ** 15) + 1) * 2.0 ** -15
        # with n_s = 1 the first midpoint above D (here 1.0) gives exactly one: early exit
        g1, passes1 = oracle.search(pcs, 1, 16)
        assert g1 == 1.0 and passes1 == 2


# ----------------------------------------------------------------------------
# Compositing pieces (sec. 5.2, Eq. 2)
# ----------------------------------------------------------------------------

def test_pieces_disjoint_records_unchanged_with_gaps():
    recs = np.array([[0.0, 0.5, 0.1, 0.2, 0.3, 0.4], [0.7, 1.0, 0.3, 0.2, 0.1, 0.5], [1.0, 1.5, 0.05, 0, 0, 0.1]])
    pcs = oracle.pieces(recs)
    assert len(pcs) == 4
    assert np.array_equal(pcs[0], recs[0])
    assert np.array_equal(pcs[1], [0.5, 0.7, 0, 0, 0, 0])
    assert np.array_equal(pcs[2], recs[1]) and np.array_equal(pcs[3], recs[2])


def test_pieces_ignore_empty_records():
    recs = np.array([[0.5, 0.5, 0.1, 0.1, 0.1, 0.3], [0.8, 0.2, 0.1, 0.1, 0.1, 0.3], [0, 1, 0.1, 0.1, 0.1, 0.2]])
    pcs = oracle.pieces(recs)
    assert len(pcs) == 1 and np.array_equal(pcs[0], recs[2])


def test_eq2_split_recomposes_exactly():
    # one record cut by the bounds of a disjoint neighbour list into 3 pieces (Eq. 2 per piece)
    A, c = 0.7, np.array([0.9, 0.3, 0.6])
    rec = [0.0, 3.0, *(c * A), A]
    other = [1.0, 1.0 + 1e-300, 0, 0, 0, 0]  # zero-length, ignored -> no cut
    pcs = oracle.pieces(np.array([rec, other]))
    assert len(pcs) == 1
    # a transparent-but-present record (A = 0) cuts the interval without changing it
    cutter = [1.0, 2.0, 0, 0, 0, 0.0]
    pcs = oracle.pieces(np.array([rec, cutter]))
    assert len(pcs) == 3
    # per-piece opacity is Eq. 2 with l = dt / l_record
    for p in pcs:
        assert p[5] == pytest.approx(1 - (1 - A) ** ((p[1] - p[0]) / 3.0), abs=1e-15)
        assert np.allclose(p[2:5] / p[5], c, atol=1e-15)
    C, Aa = over([(p[2:5], p[5]) for p in pcs])
    assert Aa == pytest.approx(A, abs=1e-15) and np.allclose(C, c * A, atol=1e-15)


def test_identical_overlap_doubles_optical_depth():
    A, c = 0.35, np.array([0.2, 0.4, 0.8])
    rec = [0.0, 1.0, *(c * A), A]
    pcs = oracle.pieces(np.array([rec, rec]))
    assert len(pcs) == 1
    assert pcs[0, 5] == pytest.approx(1 - (1 - A) ** 2, abs=1e-15)
    assert np.allclose(pcs[0, 2:5] / pcs[0, 5], c, atol=1e-15)


def test_opaque_record_dominates_overlap():
    r1 = [0.0, 1.0, 0.9, 0.0, 0.0, 1.0]
    r2 = [0.5, 1.5, 0.0, 0.5, 0.0, 0.5]
    pcs = oracle.pieces(np.array([r1, r2]))
    assert len(pcs) == 3
    assert np.allclose(pcs[1], [0.5, 1.0, 0.9, 0.0, 0.0, 1.0])


def _ea_integrate(recs, t0, t1, n=400000):
    """Euler integration of the emission-absorption ODE for piecewise-constant media:
    dT = -sum(mu_i) T dt, dC = T sum(mu_i c_i) dt, with mu_i = -ln(1 - A_i) / l_i."""
    ts = np.linspace(t0, t1, n + 1)
    mid = 0.5 * (ts[1:] + ts[:-1])
    dt = (t1 - t0) / n
    mu = np.zeros(n)
    em = np.zeros((n, 3))
    for r in recs:
        f, b, P, A = r[0], r[1], np.asarray(r[2:5]), r[4 + 1]
        inside = (mid >= f) & (mid < b)
        m = -math.log1p(-A) / (b - f)
        mu[inside] += m
        em[inside] += m * (P / A)
    T = np.exp(-np.concatenate([[0.0], np.cumsum(mu * dt)]))[:-1]
    C = (T[:, None] * em * dt).sum(0)
    return C, 1 - np.exp(-np.sum(mu * dt))


def test_mixture_matches_emission_absorption_integration():
    recs = np.array([[0.0, 0.6, 0.3 * 0.5, 0.1 * 0.5, 0.9 * 0.5, 0.5],
                     [0.2, 1.0, 0.8 * 0.3, 0.7 * 0.3, 0.1 * 0.3, 0.3],
                     [0.4, 0.5, 0.1 * 0.6, 0.9 * 0.6, 0.2 * 0.6, 0.6]])
    pcs = oracle.pieces(recs)
    C, A = over([(p[2:5], p[5]) for p in pcs])
    Ci, Ai = _ea_integrate(recs, 0.0, 1.0)
    assert A == pytest.approx(Ai, abs=1e-6)
    assert np.allclose(C, Ci, atol=2e-5)


# ----------------------------------------------------------------------------
# Compact layout (sec. 4, Fig. 2)
# ----------------------------------------------------------------------------

def test_exclusive_scan():
    c = RNG.integers(0, 30, 1000)
    off = oracle.exclusive_scan(c)
    assert off[0] == 0 and off[-1] == c.sum()
    assert np.array_equal(np.diff(off.astype(np.int64)), c)


def test_half_decoding():
    assert oracle.half_to_double(0x3C00) == 1.0
    assert oracle.half_to_double(0x3800) == 0.5
    assert oracle.half_to_double(0x0001) == 2.0 ** -24
    assert oracle.half_to_double(0x7BFF) == 65504.0
    assert oracle.half_to_double(0xC000) == -2.0
    for v in RNG.uniform(0, 1, 100):
        h = np.float16(v)
        assert oracle.half_to_double(int(h.view(np.uint16))) == float(h)


def test_split_boxes_near_equal_partition():
    for dims, g in [((512, 512, 512), (2, 2, 2)), ((64, 64, 64), (1, 1, 2)), ((1024, 1024, 1024), (4, 2, 2)),
                    ((37, 20, 11), (3, 2, 5))]:
        boxes = oracle.split_boxes(dims, g)
        assert len(boxes) == g[0] * g[1] * g[2]
        cover = np.zeros([d - 1 for d in dims][::-1], dtype=np.int32)
        for lo, hi in boxes:
            cover[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += 1
            for a in range(3):
                assert hi[a] > lo[a]
        assert np.all(cover == 1)
        for a in range(3):
            sizes = {hi[a] - lo[a] for lo, hi in boxes}
            assert max(sizes) - min(sizes) <= 1
