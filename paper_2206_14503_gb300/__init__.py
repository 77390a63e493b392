"""Python binding of libvdi.so (include/vdi.h): GB300 generation and
compositing of distributed Volumetric Depth Images.

The functions named ``vdi_*`` mirror the C entry points one to one and only
marshal arguments (pointers come from torch CUDA tensors or integers).  The
helpers below them allocate buffers with torch and fill the C structs; every
step of the method runs in the library's CUDA kernels.  There is no CPU
fallback: importing this module fails if libvdi.so cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvdi.so")

VDI_OK = 0
VDI_ERR_INVALID_ARG = 1
VDI_ERR_CAPACITY = 2
VDI_ERR_WORKSPACE = 3
VDI_ERR_CUDA = 4
VDI_ERR_TIMEOUT = 5
VDI_ERR_MODEL = 6
VDI_ERR_UNSUPPORTED = 7
VDI_PREC_F32 = 0
VDI_PREC_F16 = 1
VDI_VOL_F32 = 0
VDI_VOL_U16 = 1
VDI_MAX_PE = 64
VDI_GAMMA_SEARCH = -1.0
VDI_GAMMA_GIVEN = -2.0
VDI_GAMMA_CHOSEN = -3.0
VDI_FLAG_SYNC_CAPACITY = 1
VDI_FLAG_CENSUS = 2
VDI_FLAG_LEARNED_SINGLE_PASS = 4
VDI_SCHED_STAGED = 4
VDI_SCHED_LANE = 5


class VdiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class vdi_box(C.Structure):
    _fields_ = [("lo", C.c_int32 * 3), ("hi", C.c_int32 * 3)]


class vdi_camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("center", C.c_double * 3), ("up", C.c_double * 3),
                ("fovy_deg", C.c_double), ("width", C.c_int32), ("height", C.c_int32)]


class vdi_params(C.Structure):
    _fields_ = [("step", C.c_float), ("ref_len", C.c_float), ("bisect_iters", C.c_int32),
                ("schedule", C.c_int32), ("flags", C.c_int32)]


class vdi_brick(C.Structure):
    _fields_ = [("cells", C.c_void_p), ("owned", vdi_box), ("dims", C.c_int32 * 3), ("value_scale", C.c_float)]


class vdi_ownership(C.Structure):
    _fields_ = [("owner", C.c_void_p), ("block", C.c_int32), ("nb", C.c_int32 * 3)]


class vdi_pipeline_desc(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("type", C.c_int32), ("k", C.c_int32), ("boxes", vdi_box * 64),
                ("width", C.c_int32), ("height", C.c_int32), ("n_s", C.c_int32), ("prec", C.c_int32),
                ("gamma", C.c_float), ("capacity", C.c_uint64), ("params", vdi_params)]


class vdi_compact(C.Structure):
    _fields_ = [("counts", C.c_void_p), ("offsets", C.c_void_p), ("rgba", C.c_void_p), ("fb", C.c_void_p),
                ("gamma", C.c_void_p), ("capacity", C.c_uint64), ("prec", C.c_int32)]


class vdi_regular(C.Structure):
    _fields_ = [("counts", C.c_void_p), ("rgba", C.c_void_p), ("fb", C.c_void_p), ("gamma", C.c_void_p),
                ("n_s", C.c_int32), ("prec", C.c_int32)]


class vdi_request(C.Structure):
    _fields_ = [("pe", C.c_void_p), ("k", C.c_int32), ("w", C.c_int32), ("h", C.c_int32), ("out", vdi_regular),
                ("schedule", C.c_int32)]


class vdi_gen_request(C.Structure):
    _fields_ = [("bricks", C.c_void_p), ("k", C.c_int32), ("tf_lut", C.c_void_p), ("cam", vdi_camera),
                ("n_s", C.c_int32), ("gamma", C.c_float), ("out", C.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvdi.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i32, sz, f32 = C.c_void_p, C.c_int32, C.c_size_t, C.c_float
    sigs = {
        "vdi_version": ([], i32),
        "vdi_status_string": ([i32], C.c_char_p),
        "vdi_last_error": ([C.c_char_p, sz], i32),
        "vdi_workspace_status": ([vp, vp], i32),
        "vdi_workspace_counters": ([vp, vp, vp], i32),
        "vdi_split_boxes": ([vp, vp, vp], i32),
        "vdi_brick_bytes": ([vp], sz),
        "vdi_brick_build": ([vp, i32, vp, i32, vp, vp, vp, vp], i32),
        "vdi_generate_workspace": ([i32, i32, i32], sz),
        "vdi_choose_gamma": ([vp, i32, vp, vp, i32, f32, vp, vp, vp, sz, vp], i32),
        "vdi_generate": ([vp, i32, vp, vp, i32, f32, vp, vp, vp, sz, vp], i32),
        "vdi_generate_static_scratch": ([vp, i32, vp, vp, i32, f32, vp, vp, vp], i32),
        "vdi_generate_regular": ([vp, i32, vp, vp, i32, f32, vp, vp, vp, sz, vp], i32),
        "vdi_generate_owned": ([vp, i32, vp, vp, i32, f32, vp, vp, vp, vp, sz, vp], i32),
        "vdi_composite_workspace": ([i32, i32, i32, i32], sz),
        "vdi_composite": ([vp, i32, i32, i32, vp, vp, vp, sz, vp], i32),
        "vdi_render_view": ([vp, i32, i32, vp, vp, vp, vp], i32),
        "vdi_batch_table_bytes": ([vp, i32], sz),
        "vdi_batch_table_pack": ([vp, i32, vp, sz], i32),
        "vdi_composite_batched_workspace": ([vp], sz),
        "vdi_composite_batched": ([vp, vp, vp, vp, sz, vp], i32),
        "vdi_composite_autotune": ([vp, i32, vp, vp, sz, vp], i32),
        "vdi_gen_batch_table_bytes": ([vp, i32], sz),
        "vdi_gen_batch_table_pack": ([vp, i32, vp, vp, sz], i32),
        "vdi_generate_batched_workspace": ([vp], sz),
        "vdi_generate_batched": ([vp, vp, vp, sz, vp], i32),
        "vdi_model_bytes": ([], sz),
        "vdi_model_nparams": ([], i32),
        "vdi_model_init": ([vp, C.c_uint64, vp], i32),
        "vdi_model_save": ([vp, C.c_char_p, vp], i32),
        "vdi_model_load": ([vp, C.c_char_p, vp], i32),
        "vdi_tile_features": ([vp, i32, vp, vp, i32, vp, vp, vp, vp], i32),
        "vdi_tile_labels": ([vp, i32, i32, i32, vp, vp, vp], i32),
        "vdi_mlp_infer": ([vp, vp, i32, f32, vp, vp], i32),
        "vdi_mlp_train_workspace": ([i32], sz),
        "vdi_mlp_grad": ([vp, vp, vp, vp, i32, vp, vp, vp, sz, vp], i32),
        "vdi_mlp_train_step": ([vp, vp, vp, vp, i32, f32, vp, vp, sz, vp], i32),
        "vdi_learned_workspace": ([i32, i32, i32], sz),
        "vdi_choose_gamma_learned": ([vp, i32, vp, vp, i32, vp, f32, vp, vp, vp, sz, vp], i32),
        "vdi_pipeline_arena_bytes": ([vp], sz),
        "vdi_pipeline_create": ([vp, vp, sz, vp, vp], i32),
        "vdi_pipeline_submit": ([vp, vp, vp, vp, vp], i32),
        "vdi_pipeline_wait": ([vp, C.c_uint64], i32),
        "vdi_pipeline_streams": ([vp, vp], i32),
        "vdi_pipeline_destroy": ([vp], i32),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()

# exported symbol names of the C ABI (checked by the tests against include/vdi.h)
SYMBOLS = ("vdi_version", "vdi_status_string", "vdi_last_error", "vdi_workspace_status", "vdi_workspace_counters",
           "vdi_split_boxes",
           "vdi_brick_bytes", "vdi_brick_build", "vdi_generate_workspace", "vdi_choose_gamma", "vdi_generate",
           "vdi_generate_static_scratch", "vdi_generate_regular", "vdi_generate_owned",
           "vdi_composite_workspace", "vdi_composite", "vdi_render_view", "vdi_batch_table_bytes",
           "vdi_batch_table_pack", "vdi_composite_batched_workspace", "vdi_composite_batched", "vdi_composite_autotune",
           "vdi_gen_batch_table_bytes", "vdi_gen_batch_table_pack", "vdi_generate_batched_workspace",
           "vdi_generate_batched",
           "vdi_model_bytes", "vdi_model_nparams", "vdi_model_init", "vdi_model_save", "vdi_model_load",
           "vdi_tile_features", "vdi_tile_labels", "vdi_mlp_infer", "vdi_mlp_train_workspace", "vdi_mlp_grad",
           "vdi_mlp_train_step", "vdi_learned_workspace", "vdi_choose_gamma_learned",
           "vdi_pipeline_arena_bytes", "vdi_pipeline_create", "vdi_pipeline_submit", "vdi_pipeline_wait",
           "vdi_pipeline_streams", "vdi_pipeline_destroy")


def lib():
    return _lib


def _ref(x):
    return None if x is None else C.cast(C.byref(x), C.c_void_p)


def _arr(x):
    return None if x is None else C.cast(x, C.c_void_p)


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def last_error() -> str:
    buf = C.create_string_buffer(512)
    _lib.vdi_last_error(buf, 512)
    return buf.value.decode()


def check(status: int, what: str = "vdi call"):
    if status != VDI_OK:
        raise VdiError(status, f"{what}: {_lib.vdi_status_string(status).decode()}: {last_error()}")
    return status


# --------------------------------------------------------------------------
# one-to-one wrappers of the C entry points (argument marshalling only)
# --------------------------------------------------------------------------

def vdi_version() -> int:
    return _lib.vdi_version()


def vdi_status_string(s: int) -> str:
    return _lib.vdi_status_string(s).decode()


def vdi_workspace_status(workspace_ptr: int, stream=None) -> int:
    return _lib.vdi_workspace_status(C.c_void_p(workspace_ptr), _stream(stream))


def vdi_workspace_counters(workspace_ptr: int, stream=None):
    out = (C.c_uint64 * 8)()
    check(_lib.vdi_workspace_counters(C.c_void_p(workspace_ptr), _arr(out), _stream(stream)), "vdi_workspace_counters")
    return list(out)


def vdi_split_boxes(dims, grid):
    k = grid[0] * grid[1] * grid[2]
    out = (vdi_box * k)()
    d = (C.c_int32 * 3)(*dims)
    g = (C.c_int32 * 3)(*grid)
    check(_lib.vdi_split_boxes(_arr(d), _arr(g), _arr(out)), "vdi_split_boxes")
    return list(out)


def vdi_brick_bytes(box: vdi_box) -> int:
    return _lib.vdi_brick_bytes(_ref(box))


def vdi_brick_build(volume_ptr: int, voltype: int, dims, boxes, cells_ptrs, stream=None):
    k = len(boxes)
    d = (C.c_int32 * 3)(*dims)
    bx = (vdi_box * k)(*boxes)
    cp = (C.c_void_p * k)(*cells_ptrs)
    bricks = (vdi_brick * k)()
    check(_lib.vdi_brick_build(C.c_void_p(volume_ptr), voltype, _arr(d), k, _arr(bx), _arr(cp), _arr(bricks),
                               _stream(stream)), "vdi_brick_build")
    return bricks


def vdi_generate_workspace(k: int, w: int, h: int) -> int:
    return _lib.vdi_generate_workspace(k, w, h)


def vdi_choose_gamma(bricks, lut_ptr, cam: vdi_camera, n_s, gamma, outs, params: vdi_params, ws_ptr, ws_bytes,
                     stream=None) -> int:
    k = len(outs)
    oarr = (vdi_compact * k)(*outs)
    return _lib.vdi_choose_gamma(_arr(bricks), k, C.c_void_p(lut_ptr), _ref(cam), n_s, gamma, _arr(oarr),
                                 _ref(params), C.c_void_p(ws_ptr), ws_bytes, _stream(stream))


def vdi_generate_owned(bricks, lut_ptr, cam: vdi_camera, n_s, gamma, own: vdi_ownership, outs, params: vdi_params,
                       ws_ptr, ws_bytes, stream=None) -> int:
    k = len(outs)
    oarr = (vdi_compact * k)(*outs)
    return _lib.vdi_generate_owned(_arr(bricks), k, C.c_void_p(lut_ptr), _ref(cam), n_s, gamma, _ref(own), _arr(oarr),
                                   _ref(params), C.c_void_p(ws_ptr), ws_bytes, _stream(stream))


def vdi_generate_regular(bricks, lut_ptr, cam: vdi_camera, n_s, gamma, outs, params: vdi_params, ws_ptr, ws_bytes,
                         stream=None) -> int:
    k = len(outs)
    oarr = (vdi_regular * k)(*outs)
    return _lib.vdi_generate_regular(_arr(bricks), k, C.c_void_p(lut_ptr), _ref(cam), n_s, gamma, _arr(oarr),
                                     _ref(params), C.c_void_p(ws_ptr), ws_bytes, _stream(stream))


def vdi_generate(bricks, lut_ptr, cam: vdi_camera, n_s, gamma, outs, params: vdi_params, ws_ptr, ws_bytes,
                 stream=None) -> int:
    k = len(outs)
    oarr = (vdi_compact * k)(*outs)
    return _lib.vdi_generate(_arr(bricks), k, C.c_void_p(lut_ptr), _ref(cam), n_s, gamma, _arr(oarr),
                             _ref(params), C.c_void_p(ws_ptr), ws_bytes, _stream(stream))


def vdi_generate_static_scratch(bricks, lut_ptr, cam: vdi_camera, n_s, gamma, outs, params: vdi_params,
                                stream=None) -> int:
    k = len(outs)
    oarr = (vdi_compact * k)(*outs)
    return _lib.vdi_generate_static_scratch(_arr(bricks), k, C.c_void_p(lut_ptr), _ref(cam), n_s, gamma,
                                            _arr(oarr), _ref(params), _stream(stream))


def vdi_composite_workspace(k, w, h, n_s) -> int:
    return _lib.vdi_composite_workspace(k, w, h, n_s)


def vdi_composite(pes, w, h, out: vdi_regular, params: vdi_params, ws_ptr, ws_bytes, stream=None) -> int:
    k = len(pes)
    arr = (vdi_compact * k)(*pes)
    return _lib.vdi_composite(_arr(arr), k, w, h, _ref(out), _ref(params), C.c_void_p(ws_ptr), ws_bytes,
                              _stream(stream))


class Requests:
    """A ctypes array of vdi_request plus the sub-VDI descriptor arrays it points to."""

    def __init__(self, items):
        """items: list of (list of vdi_compact, w, h, vdi_regular, schedule)."""
        self._pe_arrays = []
        self.arr = (vdi_request * len(items))()
        for i, (pes, w, h, out, sched) in enumerate(items):
            pa = (vdi_compact * len(pes))(*pes)
            self._pe_arrays.append(pa)
            self.arr[i].pe = C.cast(pa, C.c_void_p)
            self.arr[i].k = len(pes)
            self.arr[i].w, self.arr[i].h = w, h
            self.arr[i].out = out
            self.arr[i].schedule = sched

    def __len__(self):
        return len(self.arr)


def vdi_batch_table_bytes(reqs: Requests) -> int:
    return _lib.vdi_batch_table_bytes(_arr(reqs.arr), len(reqs))


def vdi_batch_table_pack(reqs: Requests):
    """Returns the packed table as a bytes-like ctypes buffer (host)."""
    n = vdi_batch_table_bytes(reqs)
    buf = (C.c_uint8 * n)()
    check(_lib.vdi_batch_table_pack(_arr(reqs.arr), len(reqs), _arr(buf), n), "vdi_batch_table_pack")
    return buf


def vdi_composite_batched_workspace(host_table) -> int:
    """Workspace bytes for a table packed by vdi_batch_table_pack."""
    return _lib.vdi_composite_batched_workspace(_arr(host_table))


def vdi_composite_batched(dev_table_ptr: int, host_table, params: vdi_params, ws_ptr, ws_bytes, stream=None) -> int:
    return _lib.vdi_composite_batched(C.c_void_p(dev_table_ptr), _arr(host_table), _ref(params), C.c_void_p(ws_ptr),
                                      ws_bytes, _stream(stream))


def vdi_composite_autotune(reqs: Requests, params: vdi_params, ws_ptr, ws_bytes, stream=None) -> int:
    return _lib.vdi_composite_autotune(_arr(reqs.arr), len(reqs), _ref(params), C.c_void_p(ws_ptr), ws_bytes,
                                       _stream(stream))


class GenRequests:
    """A ctypes array of vdi_gen_request plus the brick and sub-VDI descriptor arrays it points to."""

    def __init__(self, items):
        """items: list of (bricks (ctypes array or list of vdi_brick), lut_ptr, vdi_camera, n_s, gamma,
        list of vdi_compact)."""
        self._keep = []
        self.arr = (vdi_gen_request * len(items))()
        for i, (bricks, lut_ptr, cam, n_s, gamma, outs) in enumerate(items):
            ba = (vdi_brick * len(bricks))(*bricks)
            oa = (vdi_compact * len(outs))(*outs)
            self._keep += [ba, oa]
            r = self.arr[i]
            r.bricks = C.cast(ba, C.c_void_p)
            r.k = len(bricks)
            r.tf_lut = lut_ptr
            r.cam = cam
            r.n_s = n_s
            r.gamma = gamma
            r.out = C.cast(oa, C.c_void_p)

    def __len__(self):
        return len(self.arr)


def vdi_gen_batch_table_pack(reqs: GenRequests, params: vdi_params):
    """Checks and packs the generation requests; returns the table as a ctypes buffer (host)."""
    n = _lib.vdi_gen_batch_table_bytes(_arr(reqs.arr), len(reqs))
    buf = (C.c_uint8 * n)()
    check(_lib.vdi_gen_batch_table_pack(_arr(reqs.arr), len(reqs), _ref(params), _arr(buf), n),
          "vdi_gen_batch_table_pack")
    return buf


def vdi_generate_batched_workspace(host_table) -> int:
    return _lib.vdi_generate_batched_workspace(_arr(host_table))


def vdi_generate_batched(dev_table_ptr: int, host_table, ws_ptr, ws_bytes, stream=None) -> int:
    return _lib.vdi_generate_batched(C.c_void_p(dev_table_ptr), _arr(host_table), C.c_void_p(ws_ptr), ws_bytes,
                                     _stream(stream))


# ---- learned gamma ----
VDI_NFEAT = 40
VDI_GAMMA_TILE = 16


def vdi_model_bytes() -> int:
    return _lib.vdi_model_bytes()


def vdi_model_nparams() -> int:
    return _lib.vdi_model_nparams()


def vdi_model_init(model_ptr: int, seed: int, stream=None) -> int:
    return _lib.vdi_model_init(C.c_void_p(model_ptr), seed, _stream(stream))


def vdi_model_save(model_ptr: int, path: str, stream=None) -> int:
    return _lib.vdi_model_save(C.c_void_p(model_ptr), path.encode(), _stream(stream))


def vdi_model_load(model_ptr: int, path: str, stream=None) -> int:
    return _lib.vdi_model_load(C.c_void_p(model_ptr), path.encode(), _stream(stream))


def vdi_tile_features(bricks, lut_ptr, cam: vdi_camera, n_s, params: vdi_params, feats_ptr, valid_ptr,
                      stream=None) -> int:
    return _lib.vdi_tile_features(_arr(bricks), len(bricks), C.c_void_p(lut_ptr), _ref(cam), n_s, _ref(params),
                                  C.c_void_p(feats_ptr), C.c_void_p(valid_ptr), _stream(stream))


def vdi_tile_labels(searched, w, h, labels_ptr, valid_ptr, stream=None) -> int:
    arr = (vdi_compact * len(searched))(*searched)
    return _lib.vdi_tile_labels(_arr(arr), len(searched), w, h, C.c_void_p(labels_ptr), C.c_void_p(valid_ptr),
                                _stream(stream))


def vdi_mlp_infer(model_ptr, feats_ptr, n, offset, out_ptr, stream=None) -> int:
    return _lib.vdi_mlp_infer(C.c_void_p(model_ptr), C.c_void_p(feats_ptr), n, offset, C.c_void_p(out_ptr),
                              _stream(stream))


def vdi_mlp_train_workspace(n) -> int:
    return _lib.vdi_mlp_train_workspace(n)


def vdi_mlp_grad(model_ptr, feats_ptr, labels_ptr, valid_ptr, n, grad_ptr, loss_ptr, ws_ptr, ws_bytes,
                 stream=None) -> int:
    return _lib.vdi_mlp_grad(C.c_void_p(model_ptr), C.c_void_p(feats_ptr), C.c_void_p(labels_ptr),
                             C.c_void_p(valid_ptr), n, C.c_void_p(grad_ptr), C.c_void_p(loss_ptr), C.c_void_p(ws_ptr),
                             ws_bytes, _stream(stream))


def vdi_mlp_train_step(model_ptr, feats_ptr, labels_ptr, valid_ptr, n, lr, loss_ptr, ws_ptr, ws_bytes,
                       stream=None) -> int:
    return _lib.vdi_mlp_train_step(C.c_void_p(model_ptr), C.c_void_p(feats_ptr), C.c_void_p(labels_ptr),
                                   C.c_void_p(valid_ptr), n, lr, C.c_void_p(loss_ptr), C.c_void_p(ws_ptr), ws_bytes,
                                   _stream(stream))


def vdi_learned_workspace(k, w, h) -> int:
    return _lib.vdi_learned_workspace(k, w, h)


def vdi_choose_gamma_learned(bricks, lut_ptr, cam: vdi_camera, n_s, model_ptr, offset, outs, params: vdi_params,
                             ws_ptr, ws_bytes, stream=None) -> int:
    oarr = (vdi_compact * len(outs))(*outs)
    return _lib.vdi_choose_gamma_learned(_arr(bricks), len(outs), C.c_void_p(lut_ptr), _ref(cam), n_s,
                                         C.c_void_p(model_ptr), offset, _arr(oarr), _ref(params), C.c_void_p(ws_ptr),
                                         ws_bytes, _stream(stream))


def vdi_render_view(vdi: vdi_regular, w, h, gen: vdi_camera, view, rgba_ptr, stream=None) -> int:
    return _lib.vdi_render_view(_ref(vdi), w, h, _ref(gen), _ref(view) if view is not None else None,
                                C.c_void_p(rgba_ptr), _stream(stream))


def vdi_pipeline_arena_bytes(desc: vdi_pipeline_desc) -> int:
    return _lib.vdi_pipeline_arena_bytes(_ref(desc))


def vdi_pipeline_create(desc: vdi_pipeline_desc, arena_ptr: int, arena_bytes: int, lut_ptr: int):
    """Returns (status, handle)."""
    h = C.c_void_p()
    st = _lib.vdi_pipeline_create(_ref(desc), C.c_void_p(arena_ptr), arena_bytes, C.c_void_p(lut_ptr), C.byref(h))
    return st, h


def vdi_pipeline_submit(handle, volume_host_ptr, cam: vdi_camera, dst: vdi_regular):
    """volume_host_ptr: host address or None.  Returns (status, ticket)."""
    t = C.c_uint64()
    st = _lib.vdi_pipeline_submit(handle, None if volume_host_ptr is None else C.c_void_p(volume_host_ptr), _ref(cam),
                                  _ref(dst), C.byref(t))
    return st, t.value


def vdi_pipeline_wait(handle, ticket: int) -> int:
    return _lib.vdi_pipeline_wait(handle, ticket)


def vdi_pipeline_streams(handle):
    out = (C.c_void_p * 3)()
    check(_lib.vdi_pipeline_streams(handle, _arr(out)), "vdi_pipeline_streams")
    return [int(x or 0) for x in out]


def vdi_pipeline_destroy(handle) -> int:
    return _lib.vdi_pipeline_destroy(handle)


# --------------------------------------------------------------------------
# torch conveniences (buffer allocation and struct filling)
# --------------------------------------------------------------------------

def make_camera(cam) -> vdi_camera:
    c = vdi_camera()
    c.eye[:] = [float(x) for x in cam.eye]
    c.center[:] = [float(x) for x in cam.center]
    c.up[:] = [float(x) for x in cam.up]
    c.fovy_deg = float(cam.fovy_deg)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def make_params(step=0.5, ref_len=1.0, bisect_iters=16, schedule=0, flags=0) -> vdi_params:
    return vdi_params(step, ref_len, bisect_iters, schedule, flags)


class Compact:
    """Device buffers of one compact sub-VDI (torch tensors) and its C struct."""

    def __init__(self, npix: int, capacity: int, prec: int = VDI_PREC_F32, device="cuda"):
        import torch

        self.npix = npix
        self.capacity = capacity
        self.prec = prec
        self.counts = torch.zeros(npix, dtype=torch.int32, device=device)
        self.offsets = torch.zeros(npix + 1, dtype=torch.int64, device=device)
        self.gamma = torch.zeros(npix, dtype=torch.float32, device=device)
        if prec == VDI_PREC_F32:
            self.rgba = torch.zeros((max(capacity, 1), 4), dtype=torch.float32, device=device)
            self.fb = torch.zeros((max(capacity, 1), 2), dtype=torch.float32, device=device)
        else:
            self.rgba = torch.zeros((max(capacity, 1), 4), dtype=torch.int32, device=device)  # 16-byte records
            self.fb = None

    @classmethod
    def from_tensors(cls, counts, offsets, rgba, fb, prec=VDI_PREC_F32, gamma=None):
        self = cls.__new__(cls)
        self.npix = counts.numel()
        self.capacity = rgba.shape[0]
        self.prec = prec
        self.counts, self.offsets, self.rgba, self.fb, self.gamma = counts, offsets, rgba, fb, gamma
        return self

    def struct(self) -> vdi_compact:
        return vdi_compact(self.counts.data_ptr(), self.offsets.data_ptr(), self.rgba.data_ptr(),
                           None if self.fb is None else self.fb.data_ptr(),
                           None if self.gamma is None else self.gamma.data_ptr(), self.capacity, self.prec)


class Regular:
    """Device buffers of one regular VDI (torch tensors) and its C struct."""

    def __init__(self, npix: int, n_s: int, prec: int = VDI_PREC_F32, device="cuda"):
        import torch

        self.npix, self.n_s, self.prec = npix, n_s, prec
        self.counts = torch.zeros(npix, dtype=torch.int32, device=device)
        self.gamma = torch.zeros(npix, dtype=torch.float32, device=device)
        if prec == VDI_PREC_F32:
            self.rgba = torch.zeros((npix * n_s, 4), dtype=torch.float32, device=device)
            self.fb = torch.zeros((npix * n_s, 2), dtype=torch.float32, device=device)
        else:
            self.rgba = torch.zeros((npix * n_s, 4), dtype=torch.int32, device=device)
            self.fb = None

    def struct(self) -> vdi_regular:
        return vdi_regular(self.counts.data_ptr(), self.rgba.data_ptr(),
                           None if self.fb is None else self.fb.data_ptr(), self.gamma.data_ptr(), self.n_s, self.prec)

    def records_f32(self):
        """(fb [npix, n_s, 2], rgba [npix, n_s, 4]) as float32 tensors (FP16 records decoded)."""
        import torch

        if self.prec == VDI_PREC_F32:
            return self.fb.view(self.npix, self.n_s, 2), self.rgba.view(self.npix, self.n_s, 4)
        raw = self.rgba.view(self.npix, self.n_s, 4)
        return raw[..., 0:2].contiguous().view(torch.float32), _f16_colour(raw[..., 2:4])


def _f16_colour(raw):
    """float32 (R, G, B, A) of the colour halves (int32 [..., 2]) of 16-byte records {f, b, half R, G, B,
    tau}: premultiplied colour and the optical depth tau = -log2(1 - A), so A = 1 - 2^-tau."""
    import math

    import torch

    c = raw.contiguous().view(torch.float16).float()
    c[..., 3] = -torch.expm1(c[..., 3] * -math.log(2.0))
    return c


def compact_records_f32(c: Compact):
    """(fb [n, 2], rgba [n, 4]) float32 views of a compact sub-VDI's records (FP16 records decoded)."""
    import torch

    if c.prec == VDI_PREC_F32:
        return c.fb, c.rgba
    raw = c.rgba
    return raw[:, 0:2].contiguous().view(torch.float32), _f16_colour(raw[:, 2:4])


class Bricks:
    """Sampling bricks of K PEs built on the device from a whole volume."""

    def __init__(self, volume, dims, boxes, stream=None):
        import torch

        self.dims = tuple(int(d) for d in dims)
        self.boxes = list(boxes)
        voltype = VDI_VOL_U16 if volume.dtype in (torch.uint16, torch.int16) else VDI_VOL_F32
        self.cells = [torch.empty(vdi_brick_bytes(b) // 4, dtype=torch.float32, device=volume.device)
                      for b in self.boxes]
        self.bricks = vdi_brick_build(volume.data_ptr(), voltype, self.dims, self.boxes,
                                      [c.data_ptr() for c in self.cells], stream)

    def rebuild(self, volume, stream=None):
        import torch

        voltype = VDI_VOL_U16 if volume.dtype in (torch.uint16, torch.int16) else VDI_VOL_F32
        self.bricks = vdi_brick_build(volume.data_ptr(), voltype, self.dims, self.boxes,
                                      [c.data_ptr() for c in self.cells], stream)


class Workspace:
    def __init__(self, nbytes: int, device="cuda"):
        import torch

        self.nbytes = max(int(nbytes), 256)
        self.buf = torch.zeros(self.nbytes, dtype=torch.uint8, device=device)

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr()

    def status(self, stream=None) -> int:
        return vdi_workspace_status(self.ptr, stream)


class HostRegular:
    """Page-locked host buffers of one regular VDI (a pipeline's destination) and their C struct."""

    def __init__(self, npix: int, n_s: int, prec: int = VDI_PREC_F32, gamma: bool = True):
        import torch

        self.npix, self.n_s, self.prec = npix, n_s, prec
        self.counts = torch.zeros(npix, dtype=torch.int32).pin_memory()
        self.gamma = torch.zeros(npix, dtype=torch.float32).pin_memory() if gamma else None
        if prec == VDI_PREC_F32:
            self.rgba = torch.zeros((npix * n_s, 4), dtype=torch.float32).pin_memory()
            self.fb = torch.zeros((npix * n_s, 2), dtype=torch.float32).pin_memory()
        else:
            self.rgba = torch.zeros((npix * n_s, 4), dtype=torch.int32).pin_memory()
            self.fb = None

    def struct(self) -> vdi_regular:
        return vdi_regular(self.counts.data_ptr(), self.rgba.data_ptr(),
                           None if self.fb is None else self.fb.data_ptr(),
                           None if self.gamma is None else self.gamma.data_ptr(), self.n_s, self.prec)

    def nbytes(self) -> int:
        n = self.counts.numel() * 4 + self.rgba.numel() * 4
        if self.fb is not None:
            n += self.fb.numel() * 4
        if self.gamma is not None:
            n += self.gamma.numel() * 4
        return n


class Pipeline:
    """A frame pipeline (vdi_pipeline_*) with its device arena allocated by torch."""

    def __init__(self, dims, voltype, boxes, width, height, n_s, lut, prec=VDI_PREC_F32, gamma=VDI_GAMMA_SEARCH,
                 capacity=0, params=None, device="cuda"):
        import torch

        d = vdi_pipeline_desc()
        d.dims[:] = [int(x) for x in dims]
        d.type = voltype
        d.k = len(boxes)
        for e, b in enumerate(boxes):
            d.boxes[e] = b
        d.width, d.height, d.n_s, d.prec = width, height, n_s, prec
        d.gamma = gamma
        d.capacity = capacity
        d.params = params if params is not None else make_params()
        self.desc = d
        nbytes = vdi_pipeline_arena_bytes(d)
        if nbytes == 0:
            raise VdiError(VDI_ERR_INVALID_ARG, f"vdi_pipeline_arena_bytes: {last_error()}")
        self.arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.arena.data_ptr()
        self.arena_ptr = (base + 255) // 256 * 256
        self.lut = lut if lut.is_cuda else lut.to(device)
        st, self.handle = vdi_pipeline_create(d, self.arena_ptr, nbytes, self.lut.data_ptr())
        check(st, "vdi_pipeline_create")

    def submit(self, volume_host, cam: vdi_camera, dst: HostRegular) -> int:
        st, t = vdi_pipeline_submit(self.handle, None if volume_host is None else volume_host.data_ptr(), cam,
                                    dst.struct())
        check(st, "vdi_pipeline_submit")
        return t

    def wait(self, ticket: int):
        check(vdi_pipeline_wait(self.handle, ticket), "vdi_pipeline_wait")

    def streams(self):
        return vdi_pipeline_streams(self.handle)

    def close(self):
        if self.handle is not None:
            check(vdi_pipeline_destroy(self.handle), "vdi_pipeline_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
