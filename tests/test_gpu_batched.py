"""Batched persistent compositing (vdi_composite_batched): many requests with
different image sizes, K and N_S in one persistent launch, also captured in a
CUDA graph and replayed.  Outputs must equal one vdi_composite call per
request bit for bit, and agree with the FP64 oracle within the compositing
tolerance on sampled pixels.  The autotuner's schedules give identical
results (they differ only in how many bisection levels one march covers and
where the list heads live)."""
import numpy as np
import pytest

import oracle
import synth

from gpu_run import compact_from_numpy, compare_lists

pytestmark = pytest.mark.gpu


def make_requests(n, seed, max_w=96, max_h=64, dense=False):
    import paper_2206_14503_gb300 as vdi

    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(n):
        w, h = int(rng.integers(8, max_w + 1)), int(rng.integers(8, max_h + 1))
        k, n_s = int(rng.integers(2, 33)), int(rng.integers(8, 65))
        lists = []
        for e in range(k):
            c, o, fb, rgba = synth.lists_compact(synth.SEED_REQUESTS, r, e, w * h, n_s, dense)
            lists.append((c, o, fb, rgba, 1))
        reqs.append(dict(w=w, h=h, k=k, n_s=n_s, lists=lists, pes=[compact_from_numpy(*l) for l in lists]))
    return reqs


def run_single(vdi, q, schedule=0):
    out = vdi.Regular(q["w"] * q["h"], q["n_s"])
    ws = vdi.Workspace(vdi.vdi_composite_workspace(q["k"], q["w"], q["h"], q["n_s"]))
    vdi.check(vdi.vdi_composite([p.struct() for p in q["pes"]], q["w"], q["h"], out.struct(),
                                vdi.make_params(schedule=schedule), ws.ptr, ws.nbytes), "vdi_composite")
    return out


def outputs(out):
    return (out.counts.cpu().numpy(), out.gamma.cpu().numpy(), out.rgba.cpu().numpy(), out.fb.cpu().numpy())


def batched(vdi, torch, reqs, outs, schedules=None, graph=False, replays=1):
    items = []
    for i, (q, o) in enumerate(zip(reqs, outs)):
        items.append(([p.struct() for p in q["pes"]], q["w"], q["h"], o.struct(), 0 if schedules is None else schedules[i]))
    R = vdi.Requests(items)
    host = vdi.vdi_batch_table_pack(R)
    dev = torch.frombuffer(bytearray(host), dtype=torch.uint8).cuda()
    ws = vdi.Workspace(vdi.vdi_composite_batched_workspace(host))
    params = vdi.make_params()
    if not graph:
        vdi.check(vdi.vdi_composite_batched(dev.data_ptr(), host, params, ws.ptr, ws.nbytes), "batched")
        vdi.check(ws.status(), "batched status")
        return
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            vdi.check(vdi.vdi_composite_batched(dev.data_ptr(), host, params, ws.ptr, ws.nbytes,
                                                stream=torch.cuda.current_stream()), "batched capture")
    for _ in range(replays):
        for o in outs:  # clear outputs so each replay must rewrite them
            o.counts.zero_()
            o.rgba.zero_()
            o.fb.zero_()
        g.replay()
    torch.cuda.synchronize()
    vdi.check(ws.status(), "batched status")


def test_batched_equals_separate_calls():
    import torch

    import paper_2206_14503_gb300 as vdi

    reqs = make_requests(12, 1)
    ref = [outputs(run_single(vdi, q)) for q in reqs]
    outs = [vdi.Regular(q["w"] * q["h"], q["n_s"]) for q in reqs]
    batched(vdi, torch, reqs, outs)
    for r, o in zip(ref, outs):
        for a, b in zip(r, outputs(o)):
            assert np.array_equal(a, b)


def test_batched_graph_replay_bit_exact():
    import torch

    import paper_2206_14503_gb300 as vdi

    reqs = make_requests(9, 2)
    ref = [outputs(run_single(vdi, q)) for q in reqs]
    outs = [vdi.Regular(q["w"] * q["h"], q["n_s"]) for q in reqs]
    batched(vdi, torch, reqs, outs, graph=True, replays=2)
    for r, o in zip(ref, outs):
        for a, b in zip(r, outputs(o)):
            assert np.array_equal(a, b)


def test_schedules_and_autotuner_agree():
    import torch

    import paper_2206_14503_gb300 as vdi

    reqs = make_requests(6, 3)
    for q in reqs:
        base = outputs(run_single(vdi, q, schedule=0))
        for sched in (1, 2, 3, vdi.VDI_SCHED_STAGED):
            if sched == 1 and q["k"] > 8:
                continue
            got = outputs(run_single(vdi, q, schedule=sched))
            for a, b in zip(base, got):
                assert np.array_equal(a, b)
    # autotune fills in schedules for every request
    outs = [vdi.Regular(q["w"] * q["h"], q["n_s"]) for q in reqs]
    items = [([p.struct() for p in q["pes"]], q["w"], q["h"], o.struct(), 0) for q, o in zip(reqs, outs)]
    R = vdi.Requests(items)
    ws = vdi.Workspace(vdi.vdi_composite_workspace(64, 65536, 1, 64))
    vdi.check(vdi.vdi_composite_autotune(R, vdi.make_params(), ws.ptr, ws.nbytes), "autotune")
    scheds = [R.arr[i].schedule for i in range(len(R))]
    assert all(s in (1, 2, 3, vdi.VDI_SCHED_STAGED, vdi.VDI_SCHED_LANE) for s in scheds)
    assert all(not (s in (1, vdi.VDI_SCHED_LANE) and q["k"] > 8) for s, q in zip(scheds, reqs))
    ref = [outputs(run_single(vdi, q)) for q in reqs]
    outs2 = [vdi.Regular(q["w"] * q["h"], q["n_s"]) for q in reqs]
    batched(vdi, torch, reqs, outs2, schedules=scheds)
    for r, o in zip(ref, outs2):
        for a, b in zip(r, outputs(o)):
            assert np.array_equal(a, b)


def test_batched_matches_oracle():
    import torch

    import paper_2206_14503_gb300 as vdi

    reqs = make_requests(5, 4)
    outs = [vdi.Regular(q["w"] * q["h"], q["n_s"]) for q in reqs]
    batched(vdi, torch, reqs, outs)
    for q, o in zip(reqs, outs):
        npix = q["w"] * q["h"]
        pix = np.arange(0, npix, 3, dtype=np.int32)
        cnt, gam, recs, _ = oracle.composite(q["lists"], q["n_s"], pixels=pix, n_pix=npix)
        fb = o.fb.view(npix, q["n_s"], 2).cpu().numpy().astype(np.float64)[pix]
        rgba = o.rgba.view(npix, q["n_s"], 4).cpu().numpy().astype(np.float64)[pix]
        compare_lists(o.counts.cpu().numpy()[pix], np.concatenate([fb, rgba], -1), cnt, recs, 1e-5, 1e-5)
