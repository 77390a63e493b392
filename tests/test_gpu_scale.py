"""Compositing at full size, through the C ABI, against the FP64 oracle on
sampled pixels (the oracle computes them one by one from the same seeded
lists, regenerated on the host).

- Precision and scale: 2048 x 2048, K = 32, N_S = 32, dense lists (every PE
  holds N_S records per pixel): first with FP32 records (103 GB of input),
  then with FP16 storage of colour and optical depth (69 GB).  The FP16 path
  is held to 2e-3 against the FP64 composite of the unrounded inputs (the
  project's bound for FP16 storage), and to the FP16 output's rounding
  against the oracle run on the stored FP16 inputs (the same bytes the GPU
  read).
- Batched: 64 requests of the seeded request table (W ~ U{256..1920},
  H ~ U{256..1080}, K ~ U{2..32}, N_S ~ U{8..64}, list lengths ~ U{0..N_S})
  in one persistent launch, captured in a CUDA graph and replayed, with the
  autotuner's schedules.  The lists are windows into a shared pool of sorted
  64-record runs, so the input fits in memory while every pixel still reads
  its own spans.

Both tests need well over 100 GB of device memory and skip when it is not
free.
"""
import numpy as np
import pytest

import oracle
import synth

from gpu_run import compare_lists

pytestmark = pytest.mark.gpu

SEED_SCALE = 0x5CA1E


def _free_gb():
    import torch

    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0] / 1e9


def _host_lists(per_pixel, prec):
    """Compact host lists of m pixels from per-pixel (fb, rgba) pairs, in the oracle's list format."""
    counts = np.array([len(fb) for fb, _ in per_pixel], dtype=np.uint32)
    offsets = np.zeros(len(counts) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(counts)
    fb = np.concatenate([fb for fb, _ in per_pixel]) if counts.sum() else np.zeros((0, 2), np.float32)
    rgba = np.concatenate([c for _, c in per_pixel]) if counts.sum() else np.zeros((0, 4), np.float32)
    return (counts, offsets, fb, rgba, prec)


def _gpu_records(out, pix):
    import torch

    fb, rgba = out.records_f32()
    idx = torch.from_numpy(pix.astype(np.int64)).cuda()
    recs = torch.cat([fb[idx], rgba[idx]], -1).double().cpu().numpy()
    return out.counts[idx].cpu().numpy(), recs


def _sample_pixels(w, h, crop, n_rand, seed):
    x0, y0, cw, ch = crop
    ys, xs = np.meshgrid(np.arange(y0, y0 + ch), np.arange(x0, x0 + cw), indexing="ij")
    crop_pix = (ys * w + xs).ravel()
    rng = np.random.default_rng(seed)
    rand = rng.choice(w * h, n_rand, replace=False)
    return np.unique(np.concatenate([crop_pix, rand])).astype(np.int64)


def test_precision_scale_full_size():
    import torch

    import paper_2206_14503_gb300 as vdi
    from synth import gpu_lists

    W = H = 2048
    K, NS = 32, 32
    npix = W * H
    if _free_gb() < 125:
        pytest.skip("needs 125 GB of free device memory")
    pix = _sample_pixels(W, H, (1024, 700, 24, 24), 600, 1)
    lists32 = [_host_lists([synth.one_list(SEED_SCALE, 0, e, int(p), NS, dense=True) for p in pix], 1)
               for e in range(K)]
    # FP32 records
    pes = []
    for e in range(K):
        c, o, fb, rgba = gpu_lists.dense_set(SEED_SCALE, 0, e, npix, NS)
        pes.append(vdi.Compact.from_tensors(c, o, rgba, fb, vdi.VDI_PREC_F32))
    out = vdi.Regular(npix, NS, vdi.VDI_PREC_F32)
    ws = vdi.Workspace(vdi.vdi_composite_workspace(K, W, H, NS))
    vdi.check(vdi.vdi_composite([p.struct() for p in pes], W, H, out.struct(), vdi.make_params(), ws.ptr, ws.nbytes),
              "composite f32")
    vdi.check(ws.status(), "composite f32 status")
    cnt_g, rec_g = _gpu_records(out, pix)
    cnt_o, _, rec_o, _ = oracle.composite(lists32, NS, n_pix=len(pix))
    st32 = compare_lists(cnt_g, rec_g, cnt_o, rec_o, 1e-5, 1e-5)
    print("precision/scale FP32:", st32)
    del out
    # FP16 storage of colour and optical depth (FP32 depth), converted PE by PE
    for e in range(K):
        rec = gpu_lists.pack_f16(pes[e].fb, pes[e].rgba)
        pes[e] = vdi.Compact.from_tensors(pes[e].counts, pes[e].offsets, rec, None, vdi.VDI_PREC_F16)
        torch.cuda.empty_cache()
    out16 = vdi.Regular(npix, NS, vdi.VDI_PREC_F16)
    vdi.check(vdi.vdi_composite([p.struct() for p in pes], W, H, out16.struct(), vdi.make_params(), ws.ptr,
                                ws.nbytes), "composite f16")
    vdi.check(ws.status(), "composite f16 status")
    cnt_g, rec_g = _gpu_records(out16, pix)
    # against the FP64 composite of the unrounded inputs: the storage error the 2e-3 bound is for
    st16_vs_64 = compare_lists(cnt_g, rec_g, cnt_o, rec_o, 1e-5, 2e-3, check=False)
    img16 = oracle.flatten(cnt_g, rec_g)
    img64 = oracle.flatten(cnt_o, rec_o)
    img_err = float(np.abs(img16 - img64).max())
    # against the oracle on the stored FP16 inputs of the sampled pixels (the bytes the GPU read)
    idx = torch.from_numpy((pix[:, None] * NS + np.arange(NS)[None, :]).ravel()).cuda()
    lists16 = []
    for e in range(K):
        raw = pes[e].rgba[idx].cpu().numpy()
        off = np.arange(len(pix) + 1, dtype=np.uint64) * NS
        lists16.append((np.full(len(pix), NS, np.uint32), off, None, raw, 2))
    cnt_o16, _, rec_o16, _ = oracle.composite(lists16, NS, n_pix=len(pix))
    st16 = compare_lists(cnt_g, rec_g, cnt_o16, rec_o16, 1e-5, 5e-4)
    print("precision/scale FP16: vs FP64 of the unrounded inputs", st16_vs_64, "image max err", img_err,
          "; vs the oracle on the stored inputs", st16)
    assert st16_vs_64["rgba_max"] <= 2e-3 and img_err <= 2e-3, (st16_vs_64, img_err)
    del pes, out16
    torch.cuda.empty_cache()


def test_batched_full_size():
    import torch

    import paper_2206_14503_gb300 as vdi
    from synth import gpu_lists

    runs = 1 << 22  # 268 M pooled records, 6.4 GB
    table = synth.requests(64)
    need = 12 + sum(w * h * (k * 12 + n_s * 24 + 8) for w, h, k, n_s in table) / 1e9
    if _free_gb() < need + 20:
        pytest.skip(f"needs {need + 20:.0f} GB of free device memory")
    pool_fb, pool_rgba = gpu_lists.pool(synth.SEED_REQUESTS, runs)
    reqs, outs = [], []
    for r, (w, h, k, n_s) in enumerate(table):
        pix = torch.arange(w * h, dtype=torch.int64, device="cuda")
        pes = []
        for e in range(k):
            n, first = gpu_lists.pool_picks(synth.SEED_REQUESTS, r, e, pix, n_s, runs)
            pes.append(vdi.Compact.from_tensors(n, first, pool_rgba, pool_fb, vdi.VDI_PREC_F32))
        reqs.append((w, h, k, n_s, pes))
        outs.append(vdi.Regular(w * h, n_s))
    items = [([p.struct() for p in pes], w, h, o.struct(), 0) for (w, h, k, n_s, pes), o in zip(reqs, outs)]
    R = vdi.Requests(items)
    tws = vdi.Workspace(vdi.vdi_composite_workspace(64, 1 << 20, 1, 64))
    vdi.check(vdi.vdi_composite_autotune(R, vdi.make_params(), tws.ptr, tws.nbytes), "autotune")
    host = vdi.vdi_batch_table_pack(R)
    dev = torch.frombuffer(bytearray(host), dtype=torch.uint8).cuda()
    ws = vdi.Workspace(vdi.vdi_composite_batched_workspace(host))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            vdi.check(vdi.vdi_composite_batched(dev.data_ptr(), host, vdi.make_params(), ws.ptr, ws.nbytes,
                                                stream=torch.cuda.current_stream()), "batched capture")
    g.replay()
    torch.cuda.synchronize()
    vdi.check(ws.status(), "batched status")
    # bit-exact against one vdi_composite call per request, on the smallest requests
    order = sorted(range(len(table)), key=lambda i: table[i][0] * table[i][1])
    for i in order[:3]:
        w, h, k, n_s, pes = reqs[i]
        one = vdi.Regular(w * h, n_s)
        cws = vdi.Workspace(vdi.vdi_composite_workspace(k, w, h, n_s))
        vdi.check(vdi.vdi_composite([p.struct() for p in pes], w, h, one.struct(), vdi.make_params(), cws.ptr,
                                    cws.nbytes), "single")
        for a, b in ((one.counts, outs[i].counts), (one.gamma, outs[i].gamma), (one.rgba, outs[i].rgba),
                     (one.fb, outs[i].fb)):
            assert torch.equal(a, b)
    # FP64 oracle on sampled pixels of every request
    rng = np.random.default_rng(3)
    agree = agree_d = tot = 0
    worst = 0.0
    for i, ((w, h, k, n_s, pes), o) in enumerate(zip(reqs, outs)):
        pix = np.sort(rng.choice(w * h, 24, replace=False)).astype(np.int64)
        lists = [_host_lists(synth.pooled_lists(synth.SEED_REQUESTS, i, e, pix, n_s, runs), 1) for e in range(k)]
        cnt_o, _, rec_o, _ = oracle.composite(lists, n_s, n_pix=len(pix))
        cnt_g, rec_g = _gpu_records(o, pix)
        st = compare_lists(cnt_g, rec_g, cnt_o, rec_o, 1e-5, 1e-5, check=False)
        agree += int(round(st["count_agree"] * len(pix)))
        agree_d += int(round(st["depth_agree"] * len(pix)))
        tot += len(pix)
        worst = max(worst, st["rgba_max"])
        assert st["rgba_max"] <= 1e-5, (i, st)
    print(f"batched full size: counts agree on {agree}/{tot}, counts and depths on {agree_d}/{tot}, "
          f"rgba max err {worst:.2e}")
    assert agree >= 0.999 * tot and agree_d >= 0.999 * tot
    del reqs, outs, pool_fb, pool_rgba
    torch.cuda.empty_cache()
