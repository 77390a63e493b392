"""Learned gamma on the GPU against the FP64 oracle.

The learned part is an extension (the paper searches gamma per ray, sec. 2.4):
tile features, tile labels from the search, a 40-64-64-1 MLP (inference on the
tensor cores with BF16 operands, training in FP32 with BF16-rounded weights),
and generation with the predicted gamma, the search remaining the fallback.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
import synth

from gpu_run import composite, generate, to_dev

pytestmark = pytest.mark.gpu


def _vdi():
    import torch

    import paper_2206_14503_gb300 as vdi

    return vdi, torch


def _bricks(vdi, vol, dims, boxes):
    return vdi.Bricks(to_dev(vol), dims, [vdi.vdi_box(lo, hi) for lo, hi in boxes])


def model_theta_bf16(vdi, torch, model):
    """The model's BF16 parameters as float64 (the weights every forward pass uses)."""
    n = vdi.vdi_model_nparams()
    raw = model[27648:27648 + 2 * n].cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    return raw.view(np.float32).astype(np.float64)


def new_model(vdi, torch, seed):
    m = torch.zeros(vdi.vdi_model_bytes(), dtype=torch.uint8, device="cuda")
    vdi.check(vdi.vdi_model_init(m.data_ptr(), seed), "init")
    return m


def test_features_match_oracle(tiny_workload):
    vdi, torch = _vdi()
    w = tiny_workload
    cam = w["cams"][0]
    br = _bricks(vdi, w["vol"], w["dims"], w["boxes"])
    k = len(w["boxes"])
    tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    F = torch.zeros((k, tiles, 40), dtype=torch.float32, device="cuda")
    V = torch.zeros((k, tiles), dtype=torch.uint8, device="cuda")
    lut = to_dev(w["lut"])
    vdi.check(vdi.vdi_tile_features(br.bricks, lut.data_ptr(), vdi.make_camera(cam), w["n_s"], vdi.make_params(),
                                    F.data_ptr(), V.data_ptr()), "features")
    torch.cuda.synchronize()
    Fo, Vo = oracle.tile_features(w["vol"], w["boxes"], w["lut"], cam, w["step"], w["ref_len"], w["n_s"])
    Fg, Vg = F.cpu().numpy().astype(np.float64), V.cpu().numpy()
    assert np.array_equal(Vg.astype(bool), Vo.astype(bool))
    assert Vo.sum() > 10
    assert np.abs(Fg[..., 32:] - Fo[..., 32:]).max() <= 1e-4
    # opacity histograms: a sample within rounding of a bin edge may change bin
    assert np.abs(Fg[..., :32] - Fo[..., :32]).sum(-1).max() <= 0.02


def test_labels_match_oracle(tiny_workload):
    vdi, torch = _vdi()
    w = tiny_workload
    cam = w["cams"][2]
    npix = cam.width * cam.height
    k = len(w["boxes"])
    br = _bricks(vdi, w["vol"], w["dims"], w["boxes"])
    outs = [vdi.Compact(npix, npix * w["n_s"]) for _ in range(k)]
    ws = vdi.Workspace(vdi.vdi_generate_workspace(k, cam.width, cam.height))
    lut = to_dev(w["lut"])
    vdi.check(vdi.vdi_choose_gamma(br.bricks, lut.data_ptr(), vdi.make_camera(cam), w["n_s"], vdi.VDI_GAMMA_SEARCH,
                                   [o.struct() for o in outs], vdi.make_params(), ws.ptr, ws.nbytes), "search")
    tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    L = torch.zeros((k, tiles), dtype=torch.float32, device="cuda")
    V = torch.zeros((k, tiles), dtype=torch.uint8, device="cuda")
    vdi.check(vdi.vdi_tile_labels([o.struct() for o in outs], cam.width, cam.height, L.data_ptr(), V.data_ptr()),
              "labels")
    torch.cuda.synchronize()
    g = np.stack([o.gamma.cpu().numpy() for o in outs]).astype(np.float64)
    c = np.stack([o.counts.cpu().numpy() for o in outs])
    Lo, Vo = oracle.tile_labels(g, c, cam.width, cam.height)
    assert np.array_equal(V.cpu().numpy().astype(bool), Vo.astype(bool))
    assert np.abs(L.cpu().numpy() - Lo)[Vo.astype(bool)].max() <= 1e-5


def test_inference_matches_fp64_forward():
    vdi, torch = _vdi()
    model = new_model(vdi, torch, 5)
    rng = np.random.default_rng(0)
    n = 1000  # not a multiple of 16: ragged last warp
    x = rng.uniform(0, 1, (n, 40)).astype(np.float32)
    X = torch.from_numpy(x).cuda()
    Y = torch.zeros(n, dtype=torch.float32, device="cuda")
    vdi.check(vdi.vdi_mlp_infer(model.data_ptr(), X.data_ptr(), n, 0.25, Y.data_ptr()), "infer")
    torch.cuda.synchronize()
    th = model_theta_bf16(vdi, torch, model)
    ref = oracle.mlp_forward(th, x.astype(np.float64)) - 0.25
    got = Y.cpu().numpy().astype(np.float64)
    # activations enter the tensor cores in BF16 (8 significant bits)
    assert np.all(np.abs(got - ref) <= 2e-2 * np.maximum(1.0, np.abs(ref))), np.abs(got - ref).max()
    assert np.std(ref) > 0.05


def test_gradient_matches_oracle():
    vdi, torch = _vdi()
    model = new_model(vdi, torch, 11)
    rng = np.random.default_rng(1)
    n = 333
    x = rng.uniform(0, 1, (n, 40)).astype(np.float32)
    y = rng.normal(-6, 2, n).astype(np.float32)
    v = (rng.uniform(size=n) < 0.8).astype(np.uint8)
    X, Yt, Vt = (torch.from_numpy(a).cuda() for a in (x, y, v))
    G = torch.zeros(vdi.vdi_model_nparams(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ws = vdi.Workspace(vdi.vdi_mlp_train_workspace(n))
    vdi.check(vdi.vdi_mlp_grad(model.data_ptr(), X.data_ptr(), Yt.data_ptr(), Vt.data_ptr(), n, G.data_ptr(),
                               loss.data_ptr(), ws.ptr, ws.nbytes), "grad")
    torch.cuda.synchronize()
    th = model_theta_bf16(vdi, torch, model)
    lo, go = oracle.mlp_loss_grad(th, x.astype(np.float64), y.astype(np.float64), v.astype(np.int32))
    gg = G.cpu().numpy().astype(np.float64)
    assert float(loss.item()) == pytest.approx(lo, rel=1e-5)
    scale = np.abs(go).max()
    assert np.abs(gg - go).max() <= 1e-5 * scale + 1e-6, np.abs(gg - go).max() / scale


def test_training_learns_and_resumes_bit_exact():
    vdi, torch = _vdi()
    rng = np.random.default_rng(2)
    n = 4096
    x = rng.uniform(0, 1, (n, 40)).astype(np.float32)
    w_true = rng.normal(0, 1, 40)
    y = (x @ w_true - 8.0 + 0.5 * np.sin(3 * x[:, 0])).astype(np.float32)
    v = np.ones(n, dtype=np.uint8)
    X, Yt, Vt = (torch.from_numpy(a).cuda() for a in (x, y, v))
    ws = vdi.Workspace(vdi.vdi_mlp_train_workspace(n))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def train(model, steps):
        losses = []
        for _ in range(steps):
            vdi.check(vdi.vdi_mlp_train_step(model.data_ptr(), X.data_ptr(), Yt.data_ptr(), Vt.data_ptr(), n, 3e-3,
                                             loss.data_ptr(), ws.ptr, ws.nbytes), "train step")
            losses.append(float(loss.item()))
        return losses

    a = new_model(vdi, torch, 3)
    l1 = train(a, 150)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "m.ckpt")
        vdi.check(vdi.vdi_model_save(a.data_ptr(), path), "save")
        l2 = train(a, 150)
        b = torch.zeros_like(a)
        vdi.check(vdi.vdi_model_load(b.data_ptr(), path), "load")
        l3 = train(b, 150)
    torch.cuda.synchronize()
    assert l2[-1] < 0.05 * l1[0]
    assert l2 == l3  # same losses, step by step
    assert torch.equal(a, b)  # same parameters, moments and step count
    # a corrupt file is rejected
    with tempfile.NamedTemporaryFile(suffix=".ckpt") as f:
        f.write(b"not a model")
        f.flush()
        assert vdi.vdi_model_load(b.data_ptr(), f.name) == vdi.VDI_ERR_MODEL


def _train_on(vdi, torch, vols, cams, boxes, lut, n_s, steps=600):
    """Features and search labels of (volume, view) pairs, then MLP training."""
    feats, labels, valids = [], [], []
    k = len(boxes)
    lut_d = to_dev(lut)
    for vol, dims in vols:
        br = _bricks(vdi, vol, dims, boxes)
        for cam in cams:
            npix = cam.width * cam.height
            tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
            outs = [vdi.Compact(npix, 1) for _ in range(k)]
            ws = vdi.Workspace(vdi.vdi_generate_workspace(k, cam.width, cam.height))
            c = vdi.make_camera(cam)
            vdi.check(vdi.vdi_choose_gamma(br.bricks, lut_d.data_ptr(), c, n_s, vdi.VDI_GAMMA_SEARCH,
                                           [o.struct() for o in outs], vdi.make_params(), ws.ptr, ws.nbytes), "s")
            F = torch.zeros((k, tiles, 40), dtype=torch.float32, device="cuda")
            FV = torch.zeros((k, tiles), dtype=torch.uint8, device="cuda")
            L = torch.zeros((k, tiles), dtype=torch.float32, device="cuda")
            LV = torch.zeros((k, tiles), dtype=torch.uint8, device="cuda")
            vdi.check(vdi.vdi_tile_features(br.bricks, lut_d.data_ptr(), c, n_s, vdi.make_params(), F.data_ptr(),
                                            FV.data_ptr()), "f")
            vdi.check(vdi.vdi_tile_labels([o.struct() for o in outs], cam.width, cam.height, L.data_ptr(),
                                          LV.data_ptr()), "l")
            feats.append(F.reshape(-1, 40))
            labels.append(L.reshape(-1))
            valids.append((FV & LV).reshape(-1))
    X = torch.cat(feats).contiguous()
    Y = torch.cat(labels).contiguous()
    V = torch.cat(valids).contiguous()
    n = X.shape[0]
    model = new_model(vdi, torch, 42)
    ws = vdi.Workspace(vdi.vdi_mlp_train_workspace(n))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    first = None
    for s in range(steps):
        vdi.check(vdi.vdi_mlp_train_step(model.data_ptr(), X.data_ptr(), Y.data_ptr(), V.data_ptr(), n,
                                         3e-3 if s < steps // 2 else 1e-3, loss.data_ptr(), ws.ptr, ws.nbytes), "t")
        if first is None:
            first = float(loss.item())
    return model, first, float(loss.item())


def test_learned_generation_is_exact_and_saves_work():
    vdi, torch = _vdi()
    dims = (96, 96, 96)
    lut = synth.transfer_function(synth.SEED_TF)
    boxes = oracle.split_boxes(dims, (2, 2, 1))
    k = len(boxes)
    n_s = 12
    train_vols = [(synth.volume(dims, 24, 3, 1000 + s, np.uint16), dims) for s in range(6)]
    cams = synth.orbit(dims, 6, 128, 128, 77)
    model, l0, l1 = _train_on(vdi, torch, train_vols, cams, boxes, lut, n_s)
    assert l1 < 0.5 * l0
    lut_d = to_dev(lut)
    census = vdi.make_params(flags=vdi.VDI_FLAG_CENSUS)

    def run(vol, cam, learned, offset=0.0, flags=0):
        npix = cam.width * cam.height
        br = _bricks(vdi, vol, dims, boxes)
        c = vdi.make_camera(cam)
        outs = [vdi.Compact(npix, npix * n_s) for _ in range(k)]
        gws = vdi.Workspace(vdi.vdi_generate_workspace(k, cam.width, cam.height))
        if learned:
            ws = vdi.Workspace(vdi.vdi_learned_workspace(k, cam.width, cam.height))
            p = vdi.make_params(flags=vdi.VDI_FLAG_CENSUS | flags)
            vdi.check(vdi.vdi_choose_gamma_learned(br.bricks, lut_d.data_ptr(), c, n_s, model.data_ptr(), offset,
                                                   [o.struct() for o in outs], p, ws.ptr, ws.nbytes), "learned")
            extra = ws.nbytes - vdi.vdi_generate_workspace(k, cam.width, cam.height)
            ctr = vdi.vdi_workspace_counters(ws.ptr + extra)
        else:
            vdi.check(vdi.vdi_choose_gamma(br.bricks, lut_d.data_ptr(), c, n_s, vdi.VDI_GAMMA_SEARCH,
                                           [o.struct() for o in outs], census, gws.ptr, gws.nbytes), "search")
            ctr = vdi.vdi_workspace_counters(gws.ptr)
        vdi.check(vdi.vdi_generate(br.bricks, lut_d.data_ptr(), c, n_s, vdi.VDI_GAMMA_CHOSEN,
                                   [o.struct() for o in outs], vdi.make_params(), gws.ptr, gws.nbytes), "emit")
        vdi.check(gws.status(), "status")
        lists = []
        for o in outs:
            tot = int(o.offsets[-1])
            lists.append((o.counts.cpu().numpy().astype(np.uint32), o.offsets.cpu().numpy().astype(np.uint64),
                          o.fb[:tot].cpu().numpy(), o.rgba[:tot].cpu().numpy(), 1))
        return lists, ctr

    def count_error(ls, ll):
        cs_ = np.stack([l[0] for l in ls]).astype(np.int64)
        cl_ = np.stack([l[0] for l in ll]).astype(np.int64)
        nz = cs_ > 0
        return np.abs(cl_ - cs_)[nz].sum() / max(cs_[nz].sum(), 1), cl_.max()

    # calibrate the offset on a training volume's view
    calib_vol, calib_cam = train_vols[0][0], cams[0]
    ls, _ = run(calib_vol, calib_cam, False)
    offset = None
    for off in (0.0, 0.5, 1.0, 1.5, 2.0, 3.0, 4.0):
        ll, _ = run(calib_vol, calib_cam, True, off)
        if count_error(ls, ll)[0] <= 0.04:
            offset = off
            break
    assert offset is not None
    # held-out volume and view
    vol = synth.volume(dims, 24, 3, 4242, np.uint16)
    cam = synth.orbit(dims, 1, 160, 120, 4243)[0]
    ls, cs = run(vol, cam, False)
    ll, cl = run(vol, cam, True, offset)
    err, cmax = count_error(ls, ll)
    assert cmax <= n_s
    assert err <= 0.05, (err, offset)
    # the composited VDI still renders the volume exactly from the generating view (sec. 2.3)
    g = composite(ll, cam.width, cam.height, n_s)
    ref = oracle.dvr(vol, lut, cam, 0.5, 1.0)
    assert np.abs(g["image"] - ref).max() <= 1e-5
    # gain: fewer rays need the bisection search, and less work is done -- fewer marches over a ray's
    # samples (volume or cached) and fewer state-machine steps than the search (census counters [2], [1])
    assert cl[4] < cs[4], (cl, cs)
    assert cl[2] < cs[2] and cl[1] < cs[1], (cl, cs)
    fell = cl[4] / max(cl[3], 1)
    print(f"learned: offset {offset}, count error {err:.4f}, fallback {fell:.3f}, marches {cl[2]} vs search {cs[2]}, "
          f"steps {cl[1]} vs {cs[1]}, volume samples {cl[0]} vs {cs[0]}")
    # the single-pass form (the prediction as it is, the search for rays over the budget): counts never
    # exceed the budget, and where the prediction is within it no search runs at all
    l1, c1 = run(vol, cam, True, offset, vdi.VDI_FLAG_LEARNED_SINGLE_PASS)
    err1, cmax1 = count_error(ls, l1)
    assert cmax1 <= n_s and c1[4] < cs[4], (c1, cs)
    print(f"learned single pass: count error {err1:.4f}, searched rays {c1[4]} vs {cs[4]}, marches {c1[2]}")


def test_learned_config_sampled_rays():
    # the learned-gamma workload at full size: 1024^3 uint16 (128 blobs, 4 octaves), K = 16 bricks, 1920 x
    # 1080, N_S = 32, gamma from the committed model; the composited VDI, flattened from the generating view,
    # must equal the FP64 oracle's DVR (whatever the gammas, sec. 2.3) on sampled pixels within 1e-5, every
    # list stays within the budget, and the count error against the search stays within 5%
    import json

    vdi, torch = _vdi()
    from synth import gpu_volume

    here = os.path.dirname(os.path.abspath(__file__))
    ckpt = os.path.join(here, "..", "paper_2206_14503_gb300", "models", "gamma_ns32_k16.ckpt")
    offset = json.load(open(os.path.splitext(ckpt)[0] + ".json"))["offset"]
    dims = (1024, 1024, 1024)
    W, H, n_s = 1920, 1080, 32
    npix = W * H
    torch.cuda.empty_cache()
    if torch.cuda.mem_get_info()[0] < 80e9:
        pytest.skip("needs 80 GB of free device memory")
    vol_d = gpu_volume.volume(dims, 128, 4, synth.SEED_VOLUME + 3)
    boxes = vdi.vdi_split_boxes(dims, (4, 2, 2))
    k = len(boxes)
    br = vdi.Bricks(vol_d, dims, boxes)
    lut = synth.transfer_function(synth.SEED_TF)
    lut_d = to_dev(lut)
    cam = synth.orbit(dims, 16, W, H, synth.SEED_ORBIT)[3]
    c = vdi.make_camera(cam)
    model = torch.zeros(vdi.vdi_model_bytes(), dtype=torch.uint8, device="cuda")
    vdi.check(vdi.vdi_model_load(model.data_ptr(), ckpt), "model load")
    cap = npix * n_s // 4
    outs_l = [vdi.Compact(npix, cap) for _ in range(k)]
    outs_s = [vdi.Compact(npix, 1) for _ in range(k)]
    lws = vdi.Workspace(vdi.vdi_learned_workspace(k, W, H))
    gws = vdi.Workspace(vdi.vdi_generate_workspace(k, W, H))
    vdi.check(vdi.vdi_choose_gamma_learned(br.bricks, lut_d.data_ptr(), c, n_s, model.data_ptr(), offset,
                                           [o.struct() for o in outs_l], vdi.make_params(), lws.ptr, lws.nbytes),
              "learned")
    vdi.check(vdi.vdi_generate(br.bricks, lut_d.data_ptr(), c, n_s, vdi.VDI_GAMMA_CHOSEN,
                               [o.struct() for o in outs_l], vdi.make_params(), gws.ptr, gws.nbytes), "emit")
    vdi.check(gws.status(), "emit status")
    vdi.check(vdi.vdi_choose_gamma(br.bricks, lut_d.data_ptr(), c, n_s, vdi.VDI_GAMMA_SEARCH,
                                   [o.struct() for o in outs_s], vdi.make_params(), gws.ptr, gws.nbytes), "search")
    torch.cuda.synchronize()
    cl = torch.stack([o.counts for o in outs_l]).long()
    cs = torch.stack([o.counts for o in outs_s]).long()
    nz = cs > 0
    err = float((cl - cs).abs()[nz].sum()) / max(float(cs[nz].sum()), 1.0)
    assert int(cl.max()) <= n_s and err <= 0.05, err
    del br, outs_s
    reg = vdi.Regular(npix, n_s)
    wsc = vdi.Workspace(vdi.vdi_composite_workspace(k, W, H, n_s))
    vdi.check(vdi.vdi_composite([o.struct() for o in outs_l], W, H, reg.struct(), vdi.make_params(), wsc.ptr,
                                wsc.nbytes), "composite")
    vdi.check(wsc.status(), "composite status")
    img = torch.zeros((npix, 4), dtype=torch.float32, device="cuda")
    vdi.check(vdi.vdi_render_view(reg.struct(), W, H, c, None, img.data_ptr()), "flatten")
    torch.cuda.synchronize()
    rng = np.random.default_rng(44)
    pix = np.sort(rng.choice(npix, 300, replace=False)).astype(np.int32)
    vol = vol_d.cpu().numpy().view(np.uint16).reshape(dims[2], dims[1], dims[0])
    ref = oracle.dvr(vol, lut, cam, 0.5, 1.0, pixels=pix)
    got = img.cpu().numpy().astype(np.float64)[pix]
    e_img = float(np.abs(got - ref).max())
    print(f"learned 1024^3: count error {err:.4f}, flattened VDI vs FP64 DVR on 300 pixels {e_img:.2e}")
    assert e_img <= 1e-5, e_img
