"""Frame pipeline (vdi_pipeline_*): sub-VDI generation of one frame overlapping the
download of the previous frame's VDI (sec. 7) and the upload of the next volume.

Each frame's regular VDI, copied to host buffers by the pipeline, must equal bit for
bit the result of vdi_brick_build, vdi_generate and vdi_composite called one at a time
on the default stream (the compositing schedules agree bit for bit, so the pipeline's
autotuned choice does not matter).  Frames alternate volumes and repeat a volume
(volume NULL) so that both double buffers and the camera-only path are exercised.
"""
import numpy as np
import pytest

import synth

from gpu_run import to_dev

pytestmark = pytest.mark.gpu


def _one_by_one(vdi, torch, vol, dims, boxes, lut_d, cam, n_s, prec, gamma):
    w, h = cam.width, cam.height
    npix = w * h
    br = vdi.Bricks(to_dev(vol), dims, boxes)
    outs = [vdi.Compact(npix, npix * n_s, prec) for _ in boxes]
    ws = vdi.Workspace(vdi.vdi_generate_workspace(len(boxes), w, h))
    vdi.check(vdi.vdi_generate(br.bricks, lut_d.data_ptr(), cam, n_s, gamma, [o.struct() for o in outs],
                               vdi.make_params(), ws.ptr, ws.nbytes), "generate")
    vdi.check(ws.status(), "generate status")
    reg = vdi.Regular(npix, n_s, prec)
    wsc = vdi.Workspace(vdi.vdi_composite_workspace(len(boxes), w, h, n_s))
    vdi.check(vdi.vdi_composite([o.struct() for o in outs], w, h, reg.struct(), vdi.make_params(), wsc.ptr,
                                wsc.nbytes), "composite")
    vdi.check(wsc.status(), "composite status")
    torch.cuda.synchronize()
    return reg


@pytest.mark.parametrize("prec,gamma,schedule", [(0, -1.0, 0), (1, 0.02, 4)])
def test_pipeline_frames_equal_one_by_one(tiny_workload, prec, gamma, schedule):
    import torch

    import paper_2206_14503_gb300 as vdi

    w = tiny_workload
    dims = w["dims"]
    boxes = [vdi.vdi_box(tuple(lo), tuple(hi)) for lo, hi in w["boxes"]]
    n_s = w["n_s"]
    vol_a = w["vol"]
    vol_b = synth.volume(dims, 16, 3, synth.SEED_VOLUME + 5, np.float32)
    host = {"a": torch.from_numpy(vol_a).pin_memory(), "b": torch.from_numpy(vol_b).pin_memory()}
    lut_d = to_dev(w["lut"].astype(np.float32))
    cams = [vdi.make_camera(c) for c in w["cams"]]
    W, H = cams[0].width, cams[0].height
    pl = vdi.Pipeline(dims, vdi.VDI_VOL_F32, boxes, W, H, n_s, lut_d, prec=prec, gamma=gamma,
                      params=vdi.make_params(schedule=schedule))
    s_in, s_comp, s_out = pl.streams()
    assert len({s_in, s_comp, s_out}) == 3 and 0 not in (s_in, s_comp, s_out)
    frames = [("a", 0), (None, 1), ("b", 2), ("a", 3), (None, 4), ("b", 5)]
    dsts = [vdi.HostRegular(W * H, n_s, prec) for _ in frames]
    tickets = [pl.submit(None if v is None else host[v], cams[c], d) for (v, c), d in zip(frames, dsts)]
    assert tickets == list(range(len(frames)))
    assert vdi.vdi_pipeline_wait(pl.handle, len(frames)) == vdi.VDI_ERR_INVALID_ARG
    pl.wait(tickets[-1])
    pl.wait(0)  # older than the last two: the first error of any frame, none here
    last = None
    for (v, c), d in zip(frames, dsts):
        last = v or last
        ref = _one_by_one(vdi, torch, vol_a if last == "a" else vol_b, dims, boxes, lut_d, cams[c], n_s, prec,
                          gamma)
        assert torch.equal(d.counts, ref.counts.cpu())
        assert torch.equal(d.gamma, ref.gamma.cpu())
        assert torch.equal(d.rgba, ref.rgba.cpu())
        if prec == 0:
            assert torch.equal(d.fb, ref.fb.cpu())
        assert int(d.counts.sum()) > 0
    pl.close()


def test_pipeline_reports_capacity_overflow(tiny_workload):
    # a sub-VDI capacity below the frame's records: the frame reports VDI_ERR_CAPACITY, its lists are cut to
    # the records that fit, and the pipeline keeps going
    import torch

    import paper_2206_14503_gb300 as vdi

    w = tiny_workload
    boxes = [vdi.vdi_box(tuple(lo), tuple(hi)) for lo, hi in w["boxes"]]
    lut_d = to_dev(w["lut"].astype(np.float32))
    cam = vdi.make_camera(w["cams"][2])
    W, H = cam.width, cam.height
    pl = vdi.Pipeline(w["dims"], vdi.VDI_VOL_F32, boxes, W, H, w["n_s"], lut_d, capacity=200,
                      params=vdi.make_params(schedule=2))
    vol = torch.from_numpy(w["vol"]).pin_memory()
    d0, d1 = vdi.HostRegular(W * H, w["n_s"]), vdi.HostRegular(W * H, w["n_s"])
    t0 = pl.submit(vol, cam, d0)
    t1 = pl.submit(None, cam, d1)
    assert vdi.vdi_pipeline_wait(pl.handle, t0) == vdi.VDI_ERR_CAPACITY
    assert vdi.vdi_pipeline_wait(pl.handle, t1) == vdi.VDI_ERR_CAPACITY
    assert torch.equal(d0.counts, d1.counts) and int(d0.counts.sum()) > 0
    pl.close()
