"""CPU checks of the C ABI: the library loads, exports every entry point that
include/vdi.h declares, and its host-side logic (decomposition, sizes,
argument validation) behaves as documented.  No kernel is launched."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vdi():
    import __graft_entry__

    __graft_entry__._builder().build()
    import paper_2206_14503_gb300 as v

    return v


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "vdi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vdi_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(vdi):
    names = declared_functions()
    assert len(names) >= 13
    lib = C.CDLL(vdi.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in vdi.h but not exported"
    assert set(vdi.SYMBOLS) <= set(names)


def test_library_is_sm103a_only(vdi):
    # the build compiles one gencode: sm_103a
    import __graft_entry__

    assert __graft_entry__._builder().ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_split_boxes_matches_oracle(vdi):
    import oracle

    for dims, g in [((512, 512, 512), (2, 2, 2)), ((1024, 1024, 1024), (4, 2, 2)), ((64, 64, 64), (1, 1, 2)),
                    ((37, 20, 11), (3, 2, 5))]:
        boxes = vdi.vdi_split_boxes(dims, g)
        assert [(tuple(b.lo), tuple(b.hi)) for b in boxes] == oracle.split_boxes(dims, g)


def test_split_boxes_rejects_bad_grid(vdi):
    with pytest.raises(vdi.VdiError):
        vdi.vdi_split_boxes((4, 4, 4), (5, 1, 1))
    with pytest.raises(vdi.VdiError):
        vdi.vdi_split_boxes((512, 512, 512), (8, 8, 2))  # more than 64 PEs


def test_brick_bytes(vdi):
    b = vdi.vdi_box((0, 0, 0), (255, 256, 10))
    assert vdi.vdi_brick_bytes(b) == 257 * 258 * 12 * 32
    assert vdi.vdi_brick_bytes(vdi.vdi_box((3, 0, 0), (3, 1, 1))) == 0


def test_workspace_sizes(vdi):
    assert vdi.vdi_generate_workspace(8, 1920, 1080) >= 256 + 8 * 8 * ((1920 * 1080 + 4095) // 4096)
    assert vdi.vdi_composite_workspace(8, 1920, 1080, 20) >= 256


def test_status_strings(vdi):
    for s in range(8):
        assert vdi.vdi_status_string(s)
    assert vdi.vdi_status_string(vdi.VDI_ERR_CAPACITY) == "output capacity too small"


def test_argument_errors_before_launch(vdi):
    # every one of these fails on the host, before any CUDA call
    cam = vdi.vdi_camera((0, 0, -10), (0, 0, 0), (0, 1, 0), 45.0, 8, 8)
    params = vdi.make_params()
    fake = 1 << 20  # never dereferenced: validation fails first
    bricks = (vdi.vdi_brick * 1)()
    out = vdi.vdi_compact(fake, fake, fake, fake, fake, 10, 0)
    # k out of range
    assert vdi.lib().vdi_generate(vdi._arr(bricks), 0, C.c_void_p(fake), vdi._ref(cam), 4, -1.0,
                                  vdi._arr((vdi.vdi_compact * 1)(out)), vdi._ref(params), C.c_void_p(fake), 1 << 20,
                                  None) == vdi.VDI_ERR_INVALID_ARG
    # n_s < 1
    assert vdi.vdi_generate(bricks, fake, cam, 0, -1.0, [out], params, fake, 1 << 20) == vdi.VDI_ERR_INVALID_ARG
    # bad gamma mode
    assert vdi.vdi_generate(bricks, fake, cam, 4, -4.0, [out], params, fake, 1 << 20) == vdi.VDI_ERR_INVALID_ARG
    assert vdi.vdi_choose_gamma(bricks, fake, cam, 4, -3.0, [out], params, fake, 1 << 20) == vdi.VDI_ERR_INVALID_ARG
    # degenerate camera (up parallel to the view direction)
    bad_cam = vdi.vdi_camera((0, 0, -10), (0, 0, 0), (0, 0, 1), 45.0, 8, 8)
    assert vdi.vdi_generate(bricks, fake, bad_cam, 4, -1.0, [out], params, fake, 1 << 20) == vdi.VDI_ERR_INVALID_ARG
    # bad params
    assert vdi.vdi_generate(bricks, fake, cam, 4, -1.0, [out], vdi.make_params(step=0.0), fake,
                            1 << 20) == vdi.VDI_ERR_INVALID_ARG
    # brick without cells
    assert vdi.vdi_generate(bricks, fake, cam, 4, -1.0, [out], params, fake, 1 << 20) == vdi.VDI_ERR_INVALID_ARG
    assert "brick 0" in vdi.last_error()
    # workspace too small
    bricks[0].cells = fake
    bricks[0].owned = vdi.vdi_box((0, 0, 0), (3, 3, 3))
    bricks[0].dims[:] = [4, 4, 4]
    bricks[0].value_scale = 1.0
    assert vdi.vdi_generate(bricks, fake, cam, 4, -1.0, [out], params, fake, 16) == vdi.VDI_ERR_WORKSPACE
    # regular generation: the output's N_S must be the call's, records present and aligned, no chosen-γ mode
    rout = vdi.vdi_regular(fake, fake, fake, fake, 4, 0)
    assert vdi.vdi_generate_regular(bricks, fake, cam, 5, -1.0, [rout], params, fake,
                                    1 << 20) == vdi.VDI_ERR_INVALID_ARG
    assert "n_s" in vdi.last_error()
    assert vdi.vdi_generate_regular(bricks, fake, cam, 4, vdi.VDI_GAMMA_CHOSEN, [rout], params, fake,
                                    1 << 20) == vdi.VDI_ERR_INVALID_ARG
    rout.rgba = fake + 4
    assert vdi.vdi_generate_regular(bricks, fake, cam, 4, -1.0, [rout], params, fake,
                                    1 << 20) == vdi.VDI_ERR_INVALID_ARG
    assert "misaligned" in vdi.last_error()
    rout.rgba, rout.fb = fake, None
    assert vdi.vdi_generate_regular(bricks, fake, cam, 4, -1.0, [rout], params, fake,
                                    1 << 20) == vdi.VDI_ERR_INVALID_ARG
    # ownership map: block a power of two, nb the blocks per axis of the brick's volume (dims 4: 3 cells)
    own = vdi.vdi_ownership(fake, 3, (1, 1, 1))
    assert vdi.vdi_generate_owned(bricks, fake, cam, 4, -1.0, own, [out], params, fake,
                                  1 << 20) == vdi.VDI_ERR_INVALID_ARG
    assert "block" in vdi.last_error()
    own = vdi.vdi_ownership(fake, 2, (1, 2, 2))
    assert vdi.vdi_generate_owned(bricks, fake, cam, 4, -1.0, own, [out], params, fake,
                                  1 << 20) == vdi.VDI_ERR_INVALID_ARG
    assert "nb[0]" in vdi.last_error()
    own = vdi.vdi_ownership(fake, 2, (2, 2, 2))
    assert vdi.vdi_generate_owned(bricks, fake, cam, 4, vdi.VDI_GAMMA_CHOSEN, own, [out], params, fake,
                                  1 << 20) == vdi.VDI_ERR_INVALID_ARG
    own.owner = None
    assert vdi.vdi_generate_owned(bricks, fake, cam, 4, -1.0, own, [out], params, fake,
                                  1 << 20) == vdi.VDI_ERR_INVALID_ARG
    # composite: n_s < 1, missing arrays
    reg = vdi.vdi_regular(fake, fake, fake, None, 0, 0)
    assert vdi.vdi_composite([out], 4, 4, reg, params, fake, 256) == vdi.VDI_ERR_INVALID_ARG
    reg.n_s = 4
    bad = vdi.vdi_compact(None, fake, fake, fake, None, 0, 0)
    assert vdi.vdi_composite([bad], 4, 4, reg, params, fake, 256) == vdi.VDI_ERR_INVALID_ARG
    assert vdi.vdi_composite([out], 4, 4, reg, params, None, 0) == vdi.VDI_ERR_WORKSPACE
    # rendering from a different view: the VDI's size must be its camera's, and the camera is required
    view = vdi.vdi_camera((1, 0, -10), (0, 0, 0), (0, 1, 0), 45.0, 8, 8)
    assert vdi.vdi_render_view(reg, cam.width + 1, cam.height, cam, view, fake) == vdi.VDI_ERR_INVALID_ARG
    assert vdi.vdi_render_view(reg, 8, 8, None, view, fake) == vdi.VDI_ERR_INVALID_ARG


def test_product_path_does_not_touch_oracle():
    # the library and its binding never import or load the oracle
    pkg = os.path.join(ROOT, "paper_2206_14503_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.replace("oracle is", ""), f


def _pipeline_desc(vdi):
    d = vdi.vdi_pipeline_desc()
    d.dims[:] = [33, 17, 9]
    d.type = vdi.VDI_VOL_U16
    boxes = vdi.vdi_split_boxes((33, 17, 9), (2, 1, 1))
    d.k = 2
    d.boxes[0], d.boxes[1] = boxes
    d.width, d.height, d.n_s, d.prec = 40, 30, 6, vdi.VDI_PREC_F32
    d.gamma = vdi.VDI_GAMMA_SEARCH
    d.params = vdi.make_params()
    return d


def test_pipeline_arena_layout(vdi):
    # the arena holds two volumes, the bricks, the sub-VDIs at full capacity, two regular VDIs and
    # both workspaces; an invalid description gives 0
    d = _pipeline_desc(vdi)
    n = vdi.vdi_pipeline_arena_bytes(d)
    npix, slots = 40 * 30, 40 * 30 * 6
    need = 2 * 33 * 17 * 9 * 2 + sum(vdi.vdi_brick_bytes(d.boxes[e]) for e in range(2)) + 4096
    need += 2 * (npix * 4 + (npix + 1) * 8 + npix * 4 + slots * 24) + 2 * (npix * 8 + slots * 24)
    need += vdi.vdi_generate_workspace(2, 40, 30) + vdi.vdi_composite_workspace(2, 40, 30, 6)
    assert need <= n <= need + 256 * 40
    d.capacity = 100
    assert vdi.vdi_pipeline_arena_bytes(d) < n
    d16 = _pipeline_desc(vdi)
    d16.prec = vdi.VDI_PREC_F16
    assert vdi.vdi_pipeline_arena_bytes(d16) < n
    for field, bad in [("k", 0), ("n_s", 0), ("prec", 2), ("gamma", -3.0), ("type", 5), ("width", 0)]:
        b = _pipeline_desc(vdi)
        setattr(b, field, bad)
        assert vdi.vdi_pipeline_arena_bytes(b) == 0, field
    b = _pipeline_desc(vdi)
    b.boxes[1] = vdi.vdi_box((0, 0, 0), (33, 16, 8))  # past the last cell
    assert vdi.vdi_pipeline_arena_bytes(b) == 0
    b = _pipeline_desc(vdi)
    b.params = vdi.make_params(schedule=vdi.VDI_SCHED_LANE + 1)  # no such schedule
    assert vdi.vdi_pipeline_arena_bytes(b) == 0


def test_pipeline_argument_errors(vdi):
    # every one of these fails on the host, before any CUDA call
    d = _pipeline_desc(vdi)
    n = vdi.vdi_pipeline_arena_bytes(d)
    fake = 1 << 20
    st, h = vdi.vdi_pipeline_create(d, fake + 16, n, fake)
    assert st == vdi.VDI_ERR_INVALID_ARG and "aligned" in vdi.last_error() and not h.value
    st, h = vdi.vdi_pipeline_create(d, fake, n - 1, fake)
    assert st == vdi.VDI_ERR_WORKSPACE and not h.value
    st, h = vdi.vdi_pipeline_create(d, fake, n, 0)
    assert st == vdi.VDI_ERR_INVALID_ARG
    d.n_s = 0
    st, h = vdi.vdi_pipeline_create(d, fake, n, fake)
    assert st == vdi.VDI_ERR_INVALID_ARG
    cam = vdi.vdi_camera((0, 0, -10), (0, 0, 0), (0, 1, 0), 45.0, 40, 30)
    dst = vdi.vdi_regular(fake, fake, fake, None, 6, 0)
    assert vdi.vdi_pipeline_submit(None, fake, cam, dst)[0] == vdi.VDI_ERR_INVALID_ARG
    assert vdi.vdi_pipeline_wait(None, 0) == vdi.VDI_ERR_INVALID_ARG
    assert vdi.vdi_pipeline_destroy(None) == vdi.VDI_ERR_INVALID_ARG
