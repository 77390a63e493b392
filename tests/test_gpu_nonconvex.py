"""Non-convex decompositions on the GPU (vdi_generate_owned, sec. 5.3) against the FP64 oracle.

The oracle takes ownership per cell; the GPU map per block of cells, expanded here
into the oracle's per-cell map.  Sub-VDIs must agree as in test_gpu_generate.py
(counts, and counts plus depth bounds within 1e-5 of the ray's chord, identical on
>= 99.9% of (PE, ray) pairs; records within GEN_TOL_TINY); composited,
they must reproduce the DVR image (records of different PEs never overlap in depth,
so depth ordering makes compositing exact, sec. 5.3), and at gamma = 2 with N_S = 1
they reduce to distributed DVR (the flat-DVR limit).  A map that encodes a box
decomposition must give vdi_generate's result bit for bit.
"""
import numpy as np
import pytest

import oracle

from gpu_run import chords, compare_lists, composite, per_pixel, to_dev

pytestmark = pytest.mark.gpu

GEN_TOL_TINY = 1e-5


def _cell_map(block_map, block, dims):
    cells = [d - 1 for d in dims]
    zz, yy, xx = np.meshgrid(*[np.arange(c) // block for c in cells[::-1]], indexing="ij")
    return block_map[zz, yy, xx].astype(np.int32)


def _bounding_boxes(block_map, block, dims, k):
    cells = [d - 1 for d in dims]
    boxes = []
    for e in range(k):
        bz, by, bx = np.nonzero(block_map == e)
        lo = [int(bx.min()) * block, int(by.min()) * block, int(bz.min()) * block]
        hi = [min((int(v.max()) + 1) * block, c) for v, c in zip((bx, by, bz), cells)]
        boxes.append((tuple(lo), tuple(hi)))
    return boxes


def _gen_owned(w, cam, n_s, gamma, block_map, block, k, maxrec):
    import torch

    import paper_2206_14503_gb300 as vdi

    dims = w["dims"]
    npix = cam.width * cam.height
    boxes = [vdi.vdi_box(lo, hi) for lo, hi in _bounding_boxes(block_map, block, dims, k)]
    br = vdi.Bricks(to_dev(w["vol"]), dims, boxes)
    map_d = torch.from_numpy(np.ascontiguousarray(block_map, dtype=np.uint8)).cuda()
    nb = block_map.shape[::-1]
    own = vdi.vdi_ownership(map_d.data_ptr(), block, tuple(int(x) for x in nb))
    outs = [vdi.Compact(npix, npix * maxrec) for _ in range(k)]
    ws = vdi.Workspace(vdi.vdi_generate_workspace(k, cam.width, cam.height))
    lut_d = to_dev(w["lut"].astype(np.float32))
    vdi.check(vdi.vdi_generate_owned(br.bricks, lut_d.data_ptr(), vdi.make_camera(cam), n_s, gamma, own,
                                     [o.struct() for o in outs], vdi.make_params(step=w["step"]), ws.ptr,
                                     ws.nbytes), "vdi_generate_owned")
    vdi.check(ws.status(), "generate status")
    torch.cuda.synchronize()
    lists, gammas = [], []
    for o in outs:
        offsets = o.offsets.cpu().numpy().astype(np.uint64)
        total = int(offsets[-1])
        lists.append((o.counts.cpu().numpy().astype(np.uint32), offsets, o.fb[:total].cpu().numpy(),
                      o.rgba[:total].cpu().numpy(), 1))
        gammas.append(o.gamma.cpu().numpy())
    return lists, np.stack(gammas)


def _checkerboard(dims, block, k):
    nb = [-(-(d - 1) // block) for d in dims]
    bz, by, bx = np.meshgrid(np.arange(nb[2]), np.arange(nb[1]), np.arange(nb[0]), indexing="ij")
    return ((bx + by + bz) % k).astype(np.uint8)


def _random_map(dims, block, k, seed):
    nb = [-(-(d - 1) // block) for d in dims]
    return np.random.default_rng(seed).integers(0, k, size=(nb[2], nb[1], nb[0])).astype(np.uint8)


# (map, block edge, K, N_S, gamma); with N_S = 2 some rays cross more domain runs of a PE (up to 5)
# than the budget allows, so their lists exceed N_S
CASES = [("checkerboard", 8, 3, 8, -1.0), ("checkerboard", 8, 3, 40, 0.02), ("checkerboard", 8, 3, 2, -1.0),
         ("random", 4, 4, 6, -1.0), ("random", 16, 2, 3, -1.0)]


@pytest.mark.parametrize("kind,block,k,n_s,gamma", CASES)
def test_owned_matches_oracle(tiny_workload, kind, block, k, n_s, gamma):
    w = tiny_workload
    dims = w["dims"]
    bmap = _checkerboard(dims, block, k) if kind == "checkerboard" else _random_map(dims, block, k, 11 + block)
    cam = w["cams"][4]
    maxrec = 200
    lists, gam = _gen_owned(w, cam, n_s, gamma, bmap, block, k, maxrec)
    boxes = [((0, 0, 0), (1, 1, 1))] * k  # unused under an ownership map
    cnt, ogam, recs, _ = oracle.generate(w["vol"], boxes, w["lut"], cam, w["step"], w["ref_len"], n_s, gamma,
                                         owner_map=_cell_map(bmap, block, dims), maxrec=maxrec)
    cg, rg = per_pixel(lists, maxrec)
    compare_lists(cg, rg, cnt, recs, np.tile(1e-5 * chords(cam, dims), k), GEN_TOL_TINY)
    if gamma < 0:
        same = cg == cnt
        assert np.mean(gam[same] == ogam[same]) >= 0.999
        if n_s == 2:
            # lists over the budget: the search ends at gamma = 2 with one record per domain run
            over = cnt > n_s
            assert over.any() and np.all(ogam[over] == 2.0) and np.all(gam[over & same] == 2.0)
    # composited, the sub-VDIs render the DVR image
    g = composite(lists, cam.width, cam.height, n_s)
    ref = oracle.dvr(w["vol"], w["lut"], cam, w["step"], w["ref_len"])
    assert np.abs(g["image"] - ref).max() <= GEN_TOL_TINY


def test_owned_flat_dvr_limit(tiny_workload):
    # gamma = 2: one sub-supersegment per domain run; composited into N_S = 1, distributed DVR
    w = tiny_workload
    dims = w["dims"]
    bmap = _checkerboard(dims, 8, 3)
    cam = w["cams"][5]
    lists, _ = _gen_owned(w, cam, 1, 2.0, bmap, 8, 3, 64)
    g = composite(lists, cam.width, cam.height, 1)
    ref = oracle.dvr(w["vol"], w["lut"], cam, w["step"], w["ref_len"])
    assert g["counts"].max() <= 1 and max(int(l[0].max()) for l in lists) > 1
    assert np.abs(g["rgba"][:, 0, :] - ref).max() <= GEN_TOL_TINY


@pytest.mark.parametrize("gamma", [-1.0, 0.02])
def test_box_map_equals_box_generation(tiny_workload, gamma):
    # a map encoding the z-slab boxes gives vdi_generate's sub-VDIs bit for bit
    from gpu_run import generate

    w = tiny_workload
    dims = w["dims"]
    cells = [d - 1 for d in dims]
    bmap = np.zeros((cells[2], cells[1], cells[0]), dtype=np.uint8)
    for e, (lo, hi) in enumerate(w["boxes"]):
        bmap[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = e
    cam = w["cams"][6]
    n_s = w["n_s"]
    lo_b, g_b = generate(w["vol"], dims, w["boxes"], w["lut"], cam, n_s, gamma, step=w["step"])
    lo_o, g_o = _gen_owned(w, cam, n_s, gamma, bmap, 1, len(w["boxes"]), n_s)
    assert np.array_equal(g_b, g_o)
    for a, b in zip(lo_b, lo_o):
        for x, y in zip(a[:4], b[:4]):
            assert np.array_equal(x, y)
