"""Test helpers that drive the library through its C ABI (via the binding) on
numpy inputs and return numpy outputs.  No method arithmetic here."""
from __future__ import annotations

import numpy as np


def _torch():
    import torch

    return torch


def to_dev(a):
    torch = _torch()
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def compact_from_numpy(counts, offsets, fb, rgba, prec=1):
    """Device compact sub-VDI from host arrays (fb float [n,2], rgba float [n,4]).  `prec` uses the
    oracle's codes: 0/1 (float64/float32 arrays) are stored as FP32 records, 2 as FP16 records (packed
    here from fb and rgba, or, with fb None, already packed in rgba as int32 [n, 4])."""
    import paper_2206_14503_gb300 as vdi

    n = len(rgba)
    c = to_dev(counts.astype(np.int32))
    o = to_dev(offsets.astype(np.int64))
    prec = vdi.VDI_PREC_F16 if prec == 2 else vdi.VDI_PREC_F32
    if prec == vdi.VDI_PREC_F32:
        r = np.ascontiguousarray(rgba, dtype=np.float32).reshape(-1, 4) if n else np.zeros((1, 4), np.float32)
        f = np.ascontiguousarray(fb, dtype=np.float32).reshape(-1, 2) if n else np.zeros((1, 2), np.float32)
        return vdi.Compact.from_tensors(c, o, to_dev(r), to_dev(f), prec)
    if fb is None:
        rec = np.ascontiguousarray(rgba).view(np.int32).reshape(-1, 4) if n else np.zeros((1, 4), np.int32)
    else:
        rec = pack_f16_records(fb, rgba) if n else np.zeros((1, 4), np.int32)
    return vdi.Compact.from_tensors(c, o, to_dev(rec), None, prec)


def pack_f16_records(fb, rgba):
    """16-byte records {float f, float b, half R, G, B, tau} as int32 [n, 4]: premultiplied colour and the
    optical depth tau = -log2(1 - A) (+inf for A = 1), each rounded to nearest even from float64."""
    n = len(fb)
    c = np.asarray(rgba, dtype=np.float64).reshape(n, 4).copy()
    with np.errstate(divide="ignore"):
        c[:, 3] = -np.log2(1.0 - c[:, 3])
    buf = np.zeros((n, 16), dtype=np.uint8)
    buf[:, 0:8] = np.ascontiguousarray(fb, dtype=np.float32).view(np.uint8).reshape(n, 8)
    buf[:, 8:16] = c.astype(np.float16).view(np.uint8).reshape(n, 8)
    return buf.view(np.int32).reshape(n, 4)


def unpack_f16_records(raw):
    """(fb float32 [n, 2], rgba float64 [n, 4]) of 16-byte records, opacity A = 1 - 2^-tau (in float64,
    so that packing the result again gives the same records)."""
    raw = np.ascontiguousarray(raw).view(np.uint8).reshape(-1, 16)
    fb = raw[:, 0:8].copy().view(np.float32).reshape(-1, 2)
    c = raw[:, 8:16].copy().view(np.float16).astype(np.float64).reshape(-1, 4)
    c[:, 3] = -np.expm1(-c[:, 3] * np.log(2.0))
    return fb, c


def composite(lists, w, h, n_s, prec_out=0, iters=16, schedule=0):
    """lists: per PE (counts, offsets, fb, rgba, prec).  Returns dict of numpy arrays."""
    import paper_2206_14503_gb300 as vdi

    torch = _torch()
    pes = [compact_from_numpy(*l) for l in lists]
    reg = vdi.Regular(w * h, n_s, prec_out)
    ws = vdi.Workspace(vdi.vdi_composite_workspace(len(pes), w, h, n_s))
    params = vdi.make_params(bisect_iters=iters, schedule=schedule)
    vdi.check(vdi.vdi_composite([p.struct() for p in pes], w, h, reg.struct(), params, ws.ptr, ws.nbytes),
              "vdi_composite")
    vdi.check(ws.status(), "composite status")
    img = torch.zeros((w * h, 4), dtype=torch.float32, device="cuda")
    vdi.check(vdi.vdi_render_view(reg.struct(), w, h, vdi.vdi_camera(), None, img.data_ptr()), "render")
    torch.cuda.synchronize()
    fb, rgba = reg.records_f32()
    return dict(counts=reg.counts.cpu().numpy(), gamma=reg.gamma.cpu().numpy(),
                fb=fb.cpu().numpy().astype(np.float64), rgba=rgba.cpu().numpy().astype(np.float64),
                image=img.cpu().numpy().astype(np.float64))


def generate(vol, dims, boxes, lut, cam, n_s, gamma, step=0.5, ref_len=1.0, prec=0, capacity=None, iters=16,
             given_gamma=None, ws_bytes=None):
    """Returns per-PE lists (counts, offsets, fb, rgba, prec) as numpy, plus gammas [k, npix].
    ws_bytes: the generation workspace's size (default: vdi_generate_workspace's)."""
    import paper_2206_14503_gb300 as vdi

    torch = _torch()
    W, H = cam.width, cam.height
    npix = W * H
    k = len(boxes)
    vb = [vdi.vdi_box(tuple(lo), tuple(hi)) for lo, hi in boxes]
    br = vdi.Bricks(to_dev(vol), dims, vb)
    cap = capacity if capacity is not None else npix * n_s
    outs = [vdi.Compact(npix, cap, prec) for _ in range(k)]
    if given_gamma is not None:
        for e in range(k):
            outs[e].gamma.copy_(torch.from_numpy(np.ascontiguousarray(given_gamma[e], dtype=np.float32)))
    ws = vdi.Workspace(ws_bytes if ws_bytes is not None else vdi.vdi_generate_workspace(k, W, H))
    lut_d = to_dev(lut.astype(np.float32))
    vdi.check(vdi.vdi_generate(br.bricks, lut_d.data_ptr(), vdi.make_camera(cam), n_s, gamma,
                               [o.struct() for o in outs], vdi.make_params(step=step, ref_len=ref_len,
                                                                           bisect_iters=iters),
                               ws.ptr, ws.nbytes), "vdi_generate")
    vdi.check(ws.status(), "generate status")
    torch.cuda.synchronize()
    lists, gammas = [], []
    for o in outs:
        counts = o.counts.cpu().numpy().astype(np.uint32)
        offsets = o.offsets.cpu().numpy().astype(np.uint64)
        total = int(offsets[-1])
        fb, rgba = vdi.compact_records_f32(o)
        lists.append((counts, offsets, fb[:total].cpu().numpy(), rgba[:total].cpu().numpy(), 1))
        gammas.append(o.gamma.cpu().numpy())
    return lists, np.stack(gammas)


def per_pixel(lists, n_s_max):
    """Compact lists -> counts [k, npix], recs [k, npix, n_s_max, 6] float64 (f, b, R, G, B, A)."""
    k = len(lists)
    npix = len(lists[0][0])
    counts = np.stack([l[0].astype(np.int64) for l in lists])
    recs = np.zeros((k, npix, n_s_max, 6))
    for e, (c, o, fb, rgba, _) in enumerate(lists):
        for j in range(n_s_max):
            sel = c > j
            idx = o[:-1][sel].astype(np.int64) + j
            recs[e, sel, j, 0:2] = fb[idx]
            recs[e, sel, j, 2:6] = rgba[idx]
    return counts, recs


def compare_lists(counts_g, recs_g, counts_o, recs_o, depth_tol, rgba_tol, min_agree=0.999, check=True):
    """Parity of per-list records (one list per pixel or per (PE, ray)) against the oracle's.

    depth_tol: absolute tolerance of the front and back depths, a scalar or one value per list (the
    tolerance is 1e-5 of the ray's chord t_out - t_in through the volume; synthetic lists lie on rays of
    length 1).  A list "agrees" when its count equals the oracle's and every depth bound is within
    depth_tol; RGBA is compared on the records of agreeing lists only.  With check, fails unless counts
    agree on at least min_agree of the lists, lists agree (counts and depths) on at least min_agree, and
    the largest RGBA error is within rgba_tol."""
    counts_g = np.asarray(counts_g).ravel()
    counts_o = np.asarray(counts_o).ravel()
    rg = recs_g.reshape(len(counts_g), -1, 6)
    ro = recs_o.reshape(len(counts_o), -1, 6)
    same = counts_g == counts_o
    n = rg.shape[1]
    mask = np.arange(n)[None, :] < counts_o[:, None]
    dd = np.where(mask, np.abs(rg[..., 0:2] - ro[..., 0:2]).max(-1), 0).max(-1)
    tol = np.broadcast_to(np.asarray(depth_tol, dtype=np.float64).ravel(), dd.shape) if np.ndim(depth_tol) else depth_tol
    match = same & (dd <= tol)
    err = np.where(mask[match][..., None], np.abs(rg[match][..., 2:6] - ro[match][..., 2:6]), 0)
    st = dict(count_agree=float(same.mean()) if len(same) else 1.0,
              depth_agree=float(match.mean()) if len(match) else 1.0,
              rgba_max=float(err.max()) if err.size else 0.0, n=len(counts_o))
    if check:
        assert st["count_agree"] >= min_agree and st["depth_agree"] >= min_agree and st["rgba_max"] <= rgba_tol, st
    return st


def chords(cam, dims, pixels=None):
    """Length t_out - t_in of each pixel's ray through the volume's box [0, dims - 1] (0 for a miss), from
    the oracle's ray and slab test."""
    import oracle

    W, H = cam.width, cam.height
    pixels = np.arange(W * H) if pixels is None else np.asarray(pixels)
    out = np.zeros(len(pixels))
    for n, p in enumerate(pixels):
        o, d = oracle.ray(cam, int(p) % W, int(p) // W)
        hit, tin, tout = oracle.hit_box(o, d, dims)
        out[n] = tout - tin if hit else 0.0
    return out
