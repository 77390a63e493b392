"""GPU sub-VDI generation (vdi_generate through the C ABI) against the FP64 oracle.

Sample positions on the GPU are exact to about 1e-12 voxel (double-float ray
setup, 20.44 fixed-point positions); what differs from the FP64 oracle is the
FP32 arithmetic of sampling, classification and the state machine, a few
units of 1e-7 in a sample's colour and opacity.  A decision of Eq. 1 (or of
the gamma search) whose margin is below that can flip, which changes a list's
count or a record's bounds.  Tolerances (the project's parity bar): per-(PE, ray)
counts identical, and counts plus depth bounds within 1e-5 of the ray's chord
identical, on at least 99.9% of lists; RGBA within 1e-5 on the records of
those lists; the flattened composite within 1e-5 of the oracle's DVR on every
pixel.  Measured on a GB300: RGBA 2.0e-6 (64^3) and 1.9e-6 (512^3), counts
100%, depth bounds 99.99% (one flipped boundary in 12,000 sampled lists at
512^3, one in 32,768 at 64^3 with N_S = 30).
"""
import numpy as np
import pytest

import oracle
import synth

from gpu_run import chords, compare_lists, composite, generate, per_pixel

pytestmark = pytest.mark.gpu

TOL = 1e-5  # RGBA, FP32 records
DEPTH_REL = 1e-5  # depth bounds, relative to the ray's chord


def _check_gen(g_lists, counts_o, recs_o, chord, pix=None):
    n_max = recs_o.shape[2]
    cg, rg = per_pixel(g_lists, n_max)
    if pix is not None:
        cg, rg = cg[:, pix], rg[:, pix]
    assert cg.max() <= n_max
    k = cg.shape[0]
    return compare_lists(cg, rg, counts_o, recs_o, np.tile(DEPTH_REL * chord, k), TOL)


def test_generate_fixed_gamma_tiny(tiny_workload):
    w = tiny_workload
    cam = w["cams"][0]
    lists, gam = generate(w["vol"], w["dims"], w["boxes"], w["lut"], cam, w["n_s"], w["gamma"], step=w["step"])
    cnt, ogam, recs, _ = oracle.generate(w["vol"], w["boxes"], w["lut"], cam, w["step"], w["ref_len"], w["n_s"],
                                         w["gamma"])
    _check_gen(lists, cnt, recs, chords(cam, w["dims"]))
    assert np.all(gam == np.float32(w["gamma"]))
    # offsets are the exclusive prefix sum of the counts
    for c, o, fb, rgba, _ in lists:
        assert o[0] == 0 and np.array_equal(np.diff(o.astype(np.int64)), c.astype(np.int64))


@pytest.mark.parametrize("n_s", [1, 3, 8, 30])
def test_generate_search_tiny(tiny_workload, n_s):
    w = tiny_workload
    cam = w["cams"][3]
    lists, gam = generate(w["vol"], w["dims"], w["boxes"], w["lut"], cam, n_s, -1.0, step=w["step"])
    cnt, ogam, recs, _ = oracle.generate(w["vol"], w["boxes"], w["lut"], cam, w["step"], w["ref_len"], n_s, -1.0)
    _check_gen(lists, cnt, recs, chords(cam, w["dims"]))
    same = np.stack([l[0] for l in lists]) == cnt
    assert np.mean(gam[same] == ogam[same]) >= 0.999


@pytest.mark.parametrize("gamma_mode", ["search", "given"])
def test_search_paths_agree(tiny_workload, gamma_mode):
    """The bisection runs over the sample cache when the workspace has room for it and re-marches the
    volume when it has not: the same decisions either way, so the counts, gammas and records agree bit
    for bit (with the search's own mode and with the given-gamma mode's fallback to it)."""
    import paper_2206_14503_gb300 as vdi

    w = tiny_workload
    cam = w["cams"][5]
    k, npix = len(w["boxes"]), cam.width * cam.height
    full = vdi.vdi_generate_workspace(k, cam.width, cam.height)
    no_cache = 512 + (8 * k * ((npix + 4095) // 4096) + 255) // 256 * 256  # the smallest workspace accepted
    assert no_cache < full
    given = None
    gamma = -1.0
    if gamma_mode == "given":
        gamma = -2.0  # VDI_GAMMA_GIVEN: a ray over the budget at its given gamma falls back to the search
        given = np.full((k, npix), 0.03, dtype=np.float32)
    runs = [generate(w["vol"], w["dims"], w["boxes"], w["lut"], cam, w["n_s"], gamma, step=w["step"],
                     given_gamma=given, ws_bytes=b) for b in (full, no_cache)]
    (ref_lists, ref_gam), (lists, gam) = runs
    searched = np.sum(ref_gam != np.float32(0.03)) if given is not None else np.sum(ref_gam > 0)
    assert searched > 1000
    assert np.array_equal(gam, ref_gam)
    for (c, o, fb, rgba, _), (c0, o0, fb0, rgba0, _) in zip(lists, ref_lists):
        assert np.array_equal(c, c0) and np.array_equal(o, o0)
        assert np.array_equal(fb, fb0) and np.array_equal(rgba, rgba0)


def test_emission_spans(tiny_workload):
    """Emission marches, for each ray with records, only the samples from its first to its last
    non-transparent one, as the count pass recorded them: the same call's, or the last vdi_choose_gamma's
    on the same workspace when it was for the same bricks, table and camera; with no such record it marches
    every sample.  The records are the same bit for bit in every case."""
    import torch

    import paper_2206_14503_gb300 as vdi
    from gpu_run import to_dev

    w = tiny_workload
    cam_a, cam_b = vdi.make_camera(w["cams"][6]), vdi.make_camera(w["cams"][7])
    npix = w["cams"][6].width * w["cams"][6].height
    n_s = w["n_s"]
    vb = [vdi.vdi_box(tuple(lo), tuple(hi)) for lo, hi in w["boxes"]]
    k = len(vb)
    br = vdi.Bricks(to_dev(w["vol"]), w["dims"], vb)
    lut = to_dev(w["lut"].astype(np.float32))
    params = vdi.make_params(step=w["step"])
    wsz = vdi.vdi_generate_workspace(k, w["cams"][6].width, w["cams"][6].height)

    def outs():
        return [vdi.Compact(npix, npix * n_s) for _ in vb]

    def structs(o):
        return [c.struct() for c in o]

    def records(o):
        torch.cuda.synchronize()
        res = []
        for c in o:
            fb, rgba = vdi.compact_records_f32(c)
            n = int(c.offsets[-1].item())
            res.append((c.counts.cpu().numpy(), c.offsets.cpu().numpy(), c.gamma.cpu().numpy(),
                        fb[:n].cpu().numpy(), rgba[:n].cpu().numpy()))
        return res

    # one call: the count pass records the spans, the emission of the same call uses them
    ws1 = vdi.Workspace(wsz)
    ref = outs()
    vdi.check(vdi.vdi_generate(br.bricks, lut.data_ptr(), cam_a, n_s, -1.0, structs(ref), params, ws1.ptr, ws1.nbytes),
              "one call")
    vdi.check(ws1.status(), "one call status")
    # the choice, then the emission on the same workspace: the choice's spans
    ws2 = vdi.Workspace(wsz)
    o2 = outs()
    vdi.check(vdi.vdi_choose_gamma(br.bricks, lut.data_ptr(), cam_a, n_s, -1.0, structs(o2), params, ws2.ptr,
                                   ws2.nbytes), "choice")
    vdi.check(vdi.vdi_generate(br.bricks, lut.data_ptr(), cam_a, n_s, vdi.VDI_GAMMA_CHOSEN, structs(o2), params,
                               ws2.ptr, ws2.nbytes), "chosen")
    vdi.check(ws2.status(), "chosen status")
    # the workspace's last choice was for another camera: every sample is marched
    ws3 = vdi.Workspace(wsz)
    o3, o3b = outs(), outs()
    vdi.check(vdi.vdi_choose_gamma(br.bricks, lut.data_ptr(), cam_a, n_s, -1.0, structs(o3), params, ws3.ptr,
                                   ws3.nbytes), "choice a")
    vdi.check(vdi.vdi_choose_gamma(br.bricks, lut.data_ptr(), cam_b, n_s, -1.0, structs(o3b), params, ws3.ptr,
                                   ws3.nbytes), "choice b")
    vdi.check(vdi.vdi_generate(br.bricks, lut.data_ptr(), cam_a, n_s, vdi.VDI_GAMMA_CHOSEN, structs(o3), params,
                               ws3.ptr, ws3.nbytes), "chosen, other record")
    vdi.check(ws3.status(), "chosen status")
    # a workspace without room for the spans
    small = 512 + (8 * k * ((npix + 4095) // 4096) + 255) // 256 * 256
    ws4 = vdi.Workspace(small)
    o4 = [vdi.Compact(npix, npix * n_s) for _ in vb]
    for c, r in zip(o4, o2):
        c.gamma.copy_(r.gamma)
        c.counts.copy_(r.counts)
    vdi.check(vdi.vdi_generate(br.bricks, lut.data_ptr(), cam_a, n_s, vdi.VDI_GAMMA_CHOSEN, structs(o4), params,
                               ws4.ptr, ws4.nbytes), "chosen, no spans")
    vdi.check(ws4.status(), "chosen status")
    r_ref = records(ref)
    assert sum(int(c[0].sum()) for c in r_ref) > 1000
    for o in (o2, o3, o4):
        for got, want in zip(records(o), r_ref):
            for g, x in zip(got, want):
                assert np.array_equal(g, x)


def test_end_to_end_equals_dvr_tiny(tiny_workload):
    # sec. 2.3: the composited VDI renders exactly from the generating view
    w = tiny_workload
    for view in (1, 5):
        cam = w["cams"][view]
        lists, _ = generate(w["vol"], w["dims"], w["boxes"], w["lut"], cam, w["n_s"], -1.0, step=w["step"])
        g = composite(lists, cam.width, cam.height, w["n_s"])
        ref = oracle.dvr(w["vol"], w["lut"], cam, w["step"], w["ref_len"])
        assert np.abs(g["image"] - ref).max() <= TOL


def test_generate_fp16_storage(tiny_workload):
    # FP16 records store the premultiplied colour and the optical depth tau = -log2(1 - A) in binary16:
    # colour within half an ulp (2^-11 relative), opacity within ln2 tau 2^-tau 2^-11 <= 1.8e-4
    w = tiny_workload
    cam = w["cams"][2]
    l32, _ = generate(w["vol"], w["dims"], w["boxes"], w["lut"], cam, w["n_s"], -1.0, step=w["step"])
    l16, _ = generate(w["vol"], w["dims"], w["boxes"], w["lut"], cam, w["n_s"], -1.0, step=w["step"], prec=1)
    for a, b in zip(l32, l16):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert np.array_equal(a[2], b[2])  # depths stay FP32
        assert np.abs(a[3][:, 0:3] - b[3][:, 0:3]).max() <= 2.0 ** -11 * np.abs(a[3][:, 0:3]).max() + 1e-7
        assert np.abs(a[3][:, 3] - b[3][:, 3]).max() <= 1.8e-4


def test_capacity_error_reported():
    import torch

    import paper_2206_14503_gb300 as vdi
    from gpu_run import to_dev

    dims = (24, 24, 24)
    vol = synth.volume(dims, 6, 2, 3, np.float32)
    lut = synth.transfer_function(synth.SEED_TF)
    cam = synth.orbit(dims, 1, 16, 16, 2)[0]
    boxes = [vdi.vdi_box(lo, hi) for lo, hi in oracle.split_boxes(dims, (1, 1, 1))]
    br = vdi.Bricks(to_dev(vol), dims, boxes)
    out = vdi.Compact(256, 3)
    ws = vdi.Workspace(vdi.vdi_generate_workspace(1, 16, 16))
    lut_d = to_dev(lut)
    # synchronous mode: the call itself returns VDI_ERR_CAPACITY with valid offsets
    s = vdi.vdi_generate(br.bricks, lut_d.data_ptr(), vdi.make_camera(cam), 4, 0.0, [out.struct()],
                         vdi.make_params(flags=vdi.VDI_FLAG_SYNC_CAPACITY), ws.ptr, ws.nbytes)
    assert s == vdi.VDI_ERR_CAPACITY
    need = int(out.offsets[-1].item())
    assert need > 3 and str(need) in vdi.last_error()
    # asynchronous mode: nothing past the capacity is written, the workspace status says why
    s = vdi.vdi_generate(br.bricks, lut_d.data_ptr(), vdi.make_camera(cam), 4, 0.0, [out.struct()],
                         vdi.make_params(), ws.ptr, ws.nbytes)
    assert s == vdi.VDI_OK
    assert ws.status() == vdi.VDI_ERR_CAPACITY
    # a large enough buffer clears it
    out2 = vdi.Compact(256, need)
    s = vdi.vdi_generate(br.bricks, lut_d.data_ptr(), vdi.make_camera(cam), 4, 0.0, [out2.struct()],
                         vdi.make_params(), ws.ptr, ws.nbytes)
    assert s == vdi.VDI_OK and ws.status() == vdi.VDI_OK
    torch.cuda.synchronize()
    # the overflowed sub-VDI's lists were cut to the records that fit: every span lies inside the
    # capacity and holds the records the large buffer got
    c_cut = out.counts.cpu().numpy().astype(np.int64)
    c_full = out2.counts.cpu().numpy().astype(np.int64)
    off = out.offsets.cpu().numpy().astype(np.int64)
    assert np.array_equal(off, out2.offsets.cpu().numpy().astype(np.int64))
    assert np.all((c_cut == 0) | (off[:-1] + c_cut <= 3)) and np.all(c_cut <= c_full) and c_cut.sum() == 3
    assert np.array_equal(c_cut, np.clip(3 - off[:-1], 0, c_full))
    assert torch.equal(out.rgba[:3], out2.rgba[:3]) and torch.equal(out.fb[:3], out2.fb[:3])
    # and composites without reading past it
    reg = vdi.Regular(256, 4)
    wsc = vdi.Workspace(vdi.vdi_composite_workspace(1, 16, 16, 4))
    vdi.check(vdi.vdi_composite([out.struct()], 16, 16, reg.struct(), vdi.make_params(), wsc.ptr, wsc.nbytes),
              "composite")
    vdi.check(wsc.status(), "composite status")


def test_given_gamma_with_fallback(tiny_workload):
    w = tiny_workload
    cam = w["cams"][4]
    npix = cam.width * cam.height
    k = len(w["boxes"])
    # given gamma = 0 everywhere: rays with more than N_S non-transparent samples fall back to the search,
    # so the result equals the plain search
    lists_s, gam_s = generate(w["vol"], w["dims"], w["boxes"], w["lut"], cam, w["n_s"], -1.0, step=w["step"])
    lists_g, gam_g = generate(w["vol"], w["dims"], w["boxes"], w["lut"], cam, w["n_s"], -2.0, step=w["step"],
                              given_gamma=np.zeros((k, npix), np.float32))
    for a, b in zip(lists_s, lists_g):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[3], b[3])
    assert np.array_equal(gam_s, gam_g)
    # given gamma = 2: one supersegment per PE ray (count at gamma 2 never exceeds N_S)
    lists_2, gam_2 = generate(w["vol"], w["dims"], w["boxes"], w["lut"], cam, w["n_s"], -2.0, step=w["step"],
                              given_gamma=np.full((k, npix), 2.0, np.float32))
    assert max(int(l[0].max()) for l in lists_2) == 1
    assert np.all(gam_2 == 2.0)


def test_plain_config_sampled_rays():
    # 512^3 uint16, 8 bricks, 1920 x 1080, N_S = 20, gamma searched in both phases; the oracle computes
    # 1500 sampled pixels of one view: the sub-VDIs (generation), the composite of the GPU's own
    # sub-VDIs (compositing, same inputs on both sides), and the DVR the flattened composite must equal
    dims = (512, 512, 512)
    vol = synth.volume(dims, 64, 3, synth.SEED_VOLUME + 1, np.uint16)
    lut = synth.transfer_function(synth.SEED_TF)
    cam = synth.orbit(dims, 16, 1920, 1080, synth.SEED_ORBIT)[0]
    boxes = oracle.split_boxes(dims, (2, 2, 2))
    n_s = 20
    lists, gam = generate(vol, dims, boxes, lut, cam, n_s, -1.0)
    g = composite(lists, 1920, 1080, n_s)
    rng = np.random.default_rng(3)
    pix = np.sort(rng.choice(1920 * 1080, 1500, replace=False)).astype(np.int32)
    ch = chords(cam, dims, pix)
    cnt, ogam, recs, _ = oracle.generate(vol, boxes, lut, cam, 0.5, 1.0, n_s, -1.0, pixels=pix)
    st = _check_gen(lists, cnt, recs, ch, pix)
    print("512^3 generation:", st)
    # compositing at the benchmarked size: the oracle composites the same FP32 sub-VDIs
    sub = []
    for c, o, fb, rgba, _ in lists:
        cs, os_ = c[pix], o[:-1][pix].astype(np.int64)
        idx = np.concatenate([np.arange(a, a + n) for a, n in zip(os_, cs.astype(np.int64))]) if cs.sum() else \
            np.zeros(0, np.int64)
        off = np.zeros(len(pix) + 1, np.uint64)
        off[1:] = np.cumsum(cs)
        sub.append((cs.astype(np.uint32), off, fb[idx], rgba[idx], 1))
    cc, _, crec, _ = oracle.composite(sub, n_s, n_pix=len(pix))
    gr = np.concatenate([g["fb"], g["rgba"]], -1)[pix]
    st_c = compare_lists(g["counts"][pix], gr, cc, crec, DEPTH_REL * ch, TOL)
    print("512^3 compositing:", st_c)
    ref = oracle.dvr(vol, lut, cam, 0.5, 1.0, pixels=pix)
    err = np.abs(g["image"][pix] - ref).max()
    assert err <= TOL, err


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("gamma_mode", ["search", "fixed"])
def test_generate_regular_equals_compact(tiny_workload, prec, gamma_mode):
    # generation straight into the regular layout (sec. 3.1) writes the records compact generation
    # writes, at pixel * n_s, with zeroed slots past each count
    import torch

    import paper_2206_14503_gb300 as vdi
    from gpu_run import to_dev

    w = tiny_workload
    cam = w["cams"][4]
    gamma = -1.0 if gamma_mode == "search" else w["gamma"]
    n_s = w["n_s"]
    lists, gam = generate(w["vol"], w["dims"], w["boxes"], w["lut"], cam, n_s, gamma, step=w["step"], prec=prec)
    npix = cam.width * cam.height
    vb = [vdi.vdi_box(tuple(lo), tuple(hi)) for lo, hi in w["boxes"]]
    br = vdi.Bricks(to_dev(w["vol"]), w["dims"], vb)
    outs = [vdi.Regular(npix, n_s, prec) for _ in vb]
    for o in outs:  # poison: every slot must be written
        o.rgba.fill_(-7)
        if o.fb is not None:
            o.fb.fill_(-7.0)
    ws = vdi.Workspace(vdi.vdi_generate_workspace(len(vb), cam.width, cam.height))
    lut_d = to_dev(w["lut"].astype(np.float32))
    vdi.check(vdi.vdi_generate_regular(br.bricks, lut_d.data_ptr(), vdi.make_camera(cam), n_s, gamma,
                                       [o.struct() for o in outs], vdi.make_params(step=w["step"]), ws.ptr,
                                       ws.nbytes), "vdi_generate_regular")
    vdi.check(ws.status(), "generate status")
    torch.cuda.synchronize()
    for e, o in enumerate(outs):
        c, off, fb_c, rgba_c, _ = lists[e]
        cnt = o.counts.cpu().numpy().astype(np.uint32)
        assert np.array_equal(cnt, c)
        assert np.array_equal(o.gamma.cpu().numpy(), gam[e])
        # decoded as the compact records were (FP16: the same decoder), so equal records decode equally
        fb_t, rgba_t = o.records_f32()
        fb_r = fb_t.cpu().numpy()
        raw_r = rgba_t.cpu().numpy()
        slot = np.arange(n_s)[None, :] < cnt[:, None].astype(np.int64)
        idx = off[:-1].astype(np.int64)[:, None] + np.arange(n_s)[None, :]
        idx = np.where(slot, idx, 0)
        assert np.array_equal(np.where(slot[..., None], fb_r, 0), np.where(slot[..., None], fb_c[idx], 0))
        assert np.array_equal(np.where(slot[..., None], raw_r, 0), np.where(slot[..., None], rgba_c[idx], 0))
        assert not np.any(fb_r[~slot]) and not np.any(raw_r[~slot])
