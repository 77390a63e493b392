"""End-to-end invariants of the oracle's generation + compositing.

 - Associativity of "over" (sec. 2.3): a VDI renders exactly from its generating
   view, so flatten(composite(sub-VDIs of all PEs)) equals DVR of the whole volume,
   for any N_S and gamma, convex or non-convex ownership (sec. 5.3).
 - gamma = 0 gives one supersegment per non-transparent sample (Eq. 1, >=).
 - A single PE composited alone is returned unchanged (K = 1 identity).
 - A homogeneous volume gives one supersegment per ray with A = 1 - (1 - a')^n.
 - At most N_S supersegments per PE list and per composited list (sec. 2.4, 5.1).
 - Compact layout: offsets are the exclusive prefix sum of the counts (sec. 4).
"""
import os

import numpy as np
import pytest

import oracle
import synth


def _gen(w, cam, n_s, gamma, boxes=None, pixels=None, owner_map=None, maxrec=None):
    return oracle.generate(w["vol"], boxes or w["boxes"], w["lut"], cam, w["step"], w["ref_len"], n_s, gamma,
                           pixels=pixels, owner_map=owner_map, maxrec=maxrec)


@pytest.mark.parametrize("n_s,gamma", [(8, 0.02), (8, -1.0), (3, -1.0), (1, 0.0), (20, 0.0), (2, 2.0)])
def test_flatten_of_composite_equals_dvr(tiny_workload, n_s, gamma):
    w = tiny_workload
    cam = w["cams"][1]
    npx = cam.width * cam.height
    cnt, _, recs, _ = _gen(w, cam, n_s, gamma, maxrec=max(n_s, 1))
    assert cnt.max() <= n_s
    cc, _, cr, _ = oracle.composite(oracle.lists_from_recs(cnt, recs), n_s, n_pix=npx)
    assert cc.max() <= n_s
    ref = oracle.dvr(w["vol"], w["lut"], cam, w["step"], w["ref_len"])
    assert np.abs(oracle.flatten(cc, cr) - ref).max() < 1e-12
    # and the sub-VDIs alone, flattened in depth order, give the same image
    assert ref[:, 3].max() > 0.5


def test_eight_bricks_uint16_invariant():
    dims = (48, 40, 56)
    vol = synth.volume(dims, 12, 3, 99, np.uint16)
    lut = synth.transfer_function(3)
    cam = synth.orbit(dims, 2, 40, 30, 5)[1]
    boxes = oracle.split_boxes(dims, (2, 2, 2))
    cnt, _, recs, _ = oracle.generate(vol, boxes, lut, cam, 0.5, 1.0, 6, -1.0)
    cc, _, cr, _ = oracle.composite(oracle.lists_from_recs(cnt, recs), 6, n_pix=40 * 30)
    ref = oracle.dvr(vol, lut, cam, 0.5, 1.0)
    assert np.abs(oracle.flatten(cc, cr) - ref).max() < 1e-12
    assert (cnt > 0).sum(0).max() >= 2  # some rays cross several bricks


def test_gamma_zero_one_record_per_nontransparent_sample(tiny_workload):
    w = tiny_workload
    cam = w["cams"][2]
    pixels = np.arange(0, cam.width * cam.height, 7, dtype=np.int32)
    cnt, _, recs, _ = _gen(w, cam, 10 ** 6, 0.0, pixels=pixels, maxrec=400)
    # count non-transparent samples per PE independently, from the DVR sample grid
    lc = oracle.lut_correct(w["lut"], w["step"], w["ref_len"])
    for q, p in enumerate(pixels[:200]):
        o, d = oracle.ray(cam, int(p) % cam.width, int(p) // cam.width)
        hit, tin, tout = oracle.hit_box(o, d, w["dims"])
        per_pe = [0, 0]
        if hit:
            k = 0
            while tin + (k + 0.5) * w["step"] < tout:
                t = tin + (k + 0.5) * w["step"]
                pt = o + t * d
                a = oracle.classify(lc, oracle.value(w["vol"], pt))[3]
                cz = min(max(int(np.floor(pt[2])), 0), w["dims"][2] - 2)
                pe = 0 if cz < w["boxes"][0][1][2] else 1
                per_pe[pe] += a > 0
                k += 1
        assert [cnt[0, q], cnt[1, q]] == per_pe
        for e in range(2):
            r = recs[e, q, :cnt[e, q]]
            assert np.allclose(r[:, 1] - r[:, 0], w["step"], atol=1e-9)


def test_single_pe_composite_is_identity(tiny_workload):
    w = tiny_workload
    cam = w["cams"][3]
    npx = cam.width * cam.height
    boxes = oracle.split_boxes(w["dims"], (1, 1, 1))
    for gamma in [0.02, -1.0]:
        cnt, _, recs, _ = _gen(w, cam, 8, gamma, boxes=boxes)
        cc, cg, cr, _ = oracle.composite(oracle.lists_from_recs(cnt, recs), 8, n_pix=npx)
        assert np.array_equal(cc, cnt[0])
        assert np.array_equal(cr, recs[0])  # bit-exact, including the zero tail
        assert np.all(cg == 0.0)


def test_homogeneous_volume_closed_form():
    dims = (20, 20, 20)
    vol = np.full(dims, 0.5, dtype=np.float32)
    lut = np.zeros((256, 4), dtype=np.float32)
    lut[:, :3] = [0.9, 0.5, 0.1]
    lut[:, 3] = 0.2
    cam = synth.orbit(dims, 1, 24, 24, 4)[0]
    boxes = oracle.split_boxes(dims, (2, 1, 1))
    step = 0.5
    cnt, gam, recs, _ = oracle.generate(vol, boxes, lut, cam, step, 1.0, 4, -1.0)
    a = 1 - (1 - float(np.float32(0.2))) ** step
    for e in range(2):
        for q in np.nonzero(cnt[e])[0]:
            if gam[e, q] == 0.0:  # at most N_S samples: gamma = 0 keeps one record per sample
                assert cnt[e, q] <= 4
                assert np.allclose(recs[e, q, :cnt[e, q], 5], a, atol=1e-15)
                continue
            assert cnt[e, q] == 1
            f, b = recs[e, q, 0, 0], recs[e, q, 0, 1]
            n = int(round((b - f) / step))
            assert n > 4
            assert recs[e, q, 0, 5] == pytest.approx(1 - (1 - a) ** n, abs=1e-12)
    # composited: the PEs' records are pieces of one medium (of different lengths); wherever
    # the search runs (more than N_S pieces), they merge into one record per ray
    cc, cg, cr, _ = oracle.composite(oracle.lists_from_recs(cnt, recs), 2, n_pix=24 * 24)
    searched = cg > 0
    assert searched.sum() > 20
    assert np.all(cc[searched] == 1)


def test_nonconvex_checkerboard_ownership(tiny_workload):
    # sec. 5.3: arbitrary ownership (here a 3-D checkerboard of 8^3-cell blocks over 3 PEs);
    # records end where the ray leaves a PE's domain, so depth ordering makes compositing exact
    w = tiny_workload
    cells = [d - 1 for d in w["dims"]]
    zz, yy, xx = np.meshgrid(*[np.arange(c) // 8 for c in cells[::-1]], indexing="ij")
    owner = ((xx + yy + zz) % 3).astype(np.int32)
    cam = w["cams"][4]
    npx = cam.width * cam.height
    boxes = [((0, 0, 0), (1, 1, 1))] * 3  # unused when an ownership map is given
    for n_s, gamma in [(8, -1.0), (40, 0.02)]:
        cnt, _, recs, _ = oracle.generate(w["vol"], boxes, w["lut"], cam, w["step"], w["ref_len"], n_s, gamma,
                                          owner_map=owner, maxrec=200)
        cc, _, cr, _ = oracle.composite(oracle.lists_from_recs(cnt, recs), n_s, n_pix=npx)
        ref = oracle.dvr(w["vol"], w["lut"], cam, w["step"], w["ref_len"])
        assert np.abs(oracle.flatten(cc, cr) - ref).max() < 1e-12
        # records of different PEs never overlap in depth
        for q in range(0, npx, 97):
            spans = sorted((recs[e, q, j, 0], recs[e, q, j, 1]) for e in range(3) for j in range(cnt[e, q]))
            for (f0, b0), (f1, b1) in zip(spans, spans[1:]):
                assert f1 >= b0


def test_nonconvex_lists_beyond_the_budget(tiny_workload):
    # sec. 5.3 with a budget smaller than a ray's domain runs: every re-entry still opens a
    # supersegment, so lists exceed N_S, the search ends at gamma = 2 for them, and the composite
    # of the sub-VDIs is still the DVR image
    w = tiny_workload
    cells = [d - 1 for d in w["dims"]]
    zz, yy, xx = np.meshgrid(*[np.arange(c) // 8 for c in cells[::-1]], indexing="ij")
    owner = ((xx + yy + zz) % 3).astype(np.int32)
    cam = w["cams"][4]
    npx = cam.width * cam.height
    boxes = [((0, 0, 0), (1, 1, 1))] * 3
    n_s = 2
    cnt, gam, recs, _ = oracle.generate(w["vol"], boxes, w["lut"], cam, w["step"], w["ref_len"], n_s, -1.0,
                                        owner_map=owner, maxrec=64)
    over = cnt > n_s
    assert over.any()
    assert np.all(gam[over] == 2.0)
    cc, _, cr, _ = oracle.composite(oracle.lists_from_recs(cnt, recs), n_s, n_pix=npx)
    ref = oracle.dvr(w["vol"], w["lut"], cam, w["step"], w["ref_len"])
    assert np.abs(oracle.flatten(cc, cr) - ref).max() < 1e-12


def test_flat_dvr_limit_case(tiny_workload):
    # sec. 5.3: one sub-supersegment per domain intersection (gamma = 2), composited into a
    # single supersegment per ray, is distributed DVR
    w = tiny_workload
    cam = w["cams"][5]
    npx = cam.width * cam.height
    cnt, _, recs, _ = _gen(w, cam, 8, 2.0)
    assert cnt.max() <= 1
    cc, _, cr, _ = oracle.composite(oracle.lists_from_recs(cnt, recs), 1, n_pix=npx)
    ref = oracle.dvr(w["vol"], w["lut"], cam, w["step"], w["ref_len"])
    assert cc.max() <= 1
    assert np.abs(cr[:, 0, 2:6] - ref).max() < 1e-12


def test_search_respects_budget_and_is_per_pe(tiny_workload):
    w = tiny_workload
    cam = w["cams"][6]
    cnt, gam, recs, passes = _gen(w, cam, 4, -1.0)
    assert cnt.max() <= 4
    # gamma is 0 exactly where the PE's list already fits at gamma = 0
    cnt0, _, _, _ = _gen(w, cam, 10 ** 6, 0.0, maxrec=400)
    assert np.array_equal(gam == 0.0, cnt0 <= 4)
    assert np.all(cnt[cnt0 <= 4] == cnt0[cnt0 <= 4])
    assert passes.max() <= 17


def test_compact_layout_matches_counts(tiny_workload):
    w = tiny_workload
    cam = w["cams"][7]
    cnt, _, recs, _ = _gen(w, cam, 8, 0.02)
    for cnt_e, off, fb, rgba, prec in oracle.lists_from_recs(cnt, recs):
        assert np.array_equal(off, oracle.exclusive_scan(cnt_e.astype(np.int32)))
        assert len(fb) == off[-1]
    # Fig. 2 of the paper: 6 lists of up to N_S = 3 supersegments take 18 regular slots,
    # of which the compact layout stores only the 11 generated ones
    counts = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "fig2_compact_counts.txt"),
                        dtype=np.int32)
    off = oracle.exclusive_scan(counts)
    assert len(counts) * 3 == 18 and off[-1] == 11


def test_records_lie_in_owning_brick():
    # gamma = 0: every record is one sample; the floor of its midpoint is a cell of the
    # PE's half-open box [lo, hi) (sec. 5.1: each PE raycasts only its own sub-volume)
    dims = (30, 26, 22)
    vol = synth.volume(dims, 10, 2, 5, np.float32)
    lut = synth.transfer_function(9)
    cam = synth.orbit(dims, 1, 32, 24, 8)[0]
    boxes = oracle.split_boxes(dims, (2, 2, 2))
    cnt, _, recs, _ = oracle.generate(vol, boxes, lut, cam, 0.5, 1.0, 10 ** 6, 0.0, maxrec=300)
    checked = 0
    for q in range(cam.width * cam.height):
        o, d = oracle.ray(cam, q % cam.width, q // cam.width)
        for e, (lo, hi) in enumerate(boxes):
            for j in range(cnt[e, q]):
                t = 0.5 * (recs[e, q, j, 0] + recs[e, q, j, 1])
                c = np.clip(np.floor(o + t * d), 0, np.array(dims) - 2)
                assert np.all(c >= lo) and np.all(c < hi)
                checked += 1
    assert checked > 1000


def test_transparent_ends_change_no_record():
    """Transparent samples before a ray's first non-transparent one and after its last one change no
    supersegment (sec. 2.4, Eq. 1 with readings G5 and G6): before the first, no supersegment is open;
    after the last, each is absorbed into the open supersegment or closes it, and neither moves its
    colour, opacity or back depth.  So the lists, and the searched gamma, of a ray equal those of the
    span between its first and last non-transparent sample -- the span the generation kernels record
    and emission marches."""
    rng = np.random.default_rng(29)
    for trial in range(60):
        n = int(rng.integers(8, 80))
        a = rng.uniform(0.0, 0.6, n) * (rng.uniform(size=n) < 0.6)
        lead, trail = int(rng.integers(0, 12)), int(rng.integers(0, 12))
        a[:lead] = 0.0
        a[n - trail:] = 0.0
        nz = np.nonzero(a)[0]
        if len(nz) == 0:
            continue
        first, last = nz[0], nz[-1]
        col = rng.uniform(size=(n, 3))
        k = np.arange(n, dtype=np.float64)
        pcs = np.column_stack([0.5 * k, 0.5 * (k + 1), col * a[:, None], a])
        span = pcs[first:last + 1]
        for gamma in (0.0, 0.05, 0.3, 1.0, 2.0):
            for cap in (2, 6, 1 << 30):
                c_full, r_full = oracle.segment(pcs, gamma, cap)
                c_span, r_span = oracle.segment(span, gamma, cap)
                assert c_full == c_span, (trial, gamma, cap)
                assert np.array_equal(r_full, r_span), (trial, gamma, cap)
        for n_s in (1, 3, 8):
            assert oracle.search(pcs, n_s)[0] == oracle.search(span, n_s)[0], (trial, n_s)
