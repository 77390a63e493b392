"""Python access to the FP64 CPU oracle (``vdi_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package's smoke check
and by the benchmark's CPU-baseline leg, never by the library.  The oracle is
the plain statement of the paper's method (generation, compact layout,
compositing with Eq. 2 subdivision and the gamma search of sec. 2.4/5.2,
flattening, DVR); see the C file's header for the section map.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vdi_oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
# A test may point the wrapper at another build of the oracle (a copy with a planted
# mistake, to check that the pins catch it).
_ALT = os.environ.get("VDI_ORACLE_LIB")
_lib = None

REC = 6  # f, b, R, G, B, A (premultiplied RGB)


class _Camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("center", C.c_double * 3), ("up", C.c_double * 3),
                ("fovy_deg", C.c_double), ("width", C.c_int), ("height", C.c_int)]


class _Volume(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int), ("dims", C.c_int * 3)]


class _Box(C.Structure):
    _fields_ = [("lo", C.c_int * 3), ("hi", C.c_int * 3)]


class _Piece(C.Structure):
    _fields_ = [("f", C.c_double), ("b", C.c_double), ("P", C.c_double * 3), ("a", C.c_double), ("brk", C.c_int)]


class _Lists(C.Structure):
    _fields_ = [("counts", C.c_void_p), ("offsets", C.c_void_p), ("fb", C.c_void_p), ("rgba", C.c_void_p),
                ("prec", C.c_int)]


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        if _ALT:
            lib = C.CDLL(_ALT)
        else:
            build()
            lib = C.CDLL(_LIB)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        lib.oc_generate.argtypes = [vp, vp, i, vp, vp, vp, d, d, i, d, i, vp, i, i, vp, vp, vp, vp]
        lib.oc_generate.restype = i
        lib.oc_composite.argtypes = [vp, i, vp, i, i, i, i, vp, vp, vp, vp]
        lib.oc_composite.restype = i
        lib.oc_segment.argtypes = [vp, i, d, i, vp, i, vp]
        lib.oc_segment.restype = i
        lib.oc_search.argtypes = [vp, i, i, i, vp]
        lib.oc_search.restype = d
        lib.oc_pieces.argtypes = [vp, i, vp, i, vp]
        lib.oc_pieces.restype = i
        lib.oc_flatten.argtypes = [vp, vp, i, i, vp]
        lib.oc_flatten.restype = None
        lib.oc_dvr.argtypes = [vp, vp, vp, d, d, vp, i, vp]
        lib.oc_dvr.restype = i
        lib.oc_ray.argtypes = [vp, i, i, vp, vp]
        lib.oc_ray.restype = None
        lib.oc_render_view.argtypes = [vp, vp, i, vp, vp, vp, i, vp]
        lib.oc_render_view.restype = None
        lib.oc_render_ray.argtypes = [vp, vp, i, d, vp, vp, vp, vp]
        lib.oc_render_ray.restype = None
        lib.oc_hit_box.argtypes = [vp, vp, vp, vp, vp]
        lib.oc_hit_box.restype = i
        lib.oc_value.argtypes = [vp, vp]
        lib.oc_value.restype = d
        lib.oc_lut_correct.argtypes = [vp, d, d, vp]
        lib.oc_lut_correct.restype = None
        lib.oc_classify.argtypes = [vp, d, vp]
        lib.oc_classify.restype = None
        lib.oc_exclusive_scan.argtypes = [vp, i, vp]
        lib.oc_exclusive_scan.restype = None
        lib.oc_half_to_double.argtypes = [C.c_uint16]
        lib.oc_half_to_double.restype = d
        lib.oc_ray_sample_count.argtypes = [vp, vp, d, i, vp]
        lib.oc_ray_sample_count.restype = i
        lib.oc_split_boxes.argtypes = [vp, vp, vp]
        lib.oc_split_boxes.restype = None
        lib.oc_tile_features.argtypes = [vp, vp, i, vp, vp, d, d, i, vp, vp]
        lib.oc_tile_features.restype = i
        lib.oc_tile_labels.argtypes = [vp, vp, i, i, i, vp, vp]
        lib.oc_tile_labels.restype = None
        lib.oc_mlp_nparams.argtypes = []
        lib.oc_mlp_nparams.restype = i
        lib.oc_mlp_forward.argtypes = [vp, vp, i, vp]
        lib.oc_mlp_forward.restype = None
        lib.oc_mlp_loss_grad.argtypes = [vp, vp, vp, vp, i, vp]
        lib.oc_mlp_loss_grad.restype = d
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _ref(s):
    return C.cast(C.byref(s), C.c_void_p)


def camera(cam) -> _Camera:
    c = _Camera()
    c.eye[:] = [float(x) for x in cam.eye]
    c.center[:] = [float(x) for x in cam.center]
    c.up[:] = [float(x) for x in cam.up]
    c.fovy_deg = float(cam.fovy_deg)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


class Volume:
    """Keeps the numpy array alive next to its C descriptor.  `vol` has shape (Z, Y, X)."""

    def __init__(self, vol: np.ndarray):
        self.arr = np.ascontiguousarray(vol)
        if self.arr.dtype == np.float32:
            code = 0
        elif self.arr.dtype == np.uint16:
            code = 1
        else:
            raise ValueError("volume must be float32 or uint16")
        Z, Y, X = self.arr.shape
        self.c = _Volume(self.arr.ctypes.data, code, (C.c_int * 3)(X, Y, Z))
        self.dims = (X, Y, Z)


def split_boxes(dims, grid):
    """Near-equal block decomposition of the cells; list of (lo, hi) per PE, x fastest."""
    k = grid[0] * grid[1] * grid[2]
    boxes = (_Box * k)()
    _load().oc_split_boxes(_p(np.asarray(dims, dtype=np.int32)), _p(np.asarray(grid, dtype=np.int32)),
                           C.cast(boxes, C.c_void_p))
    return [(tuple(b.lo), tuple(b.hi)) for b in boxes]


def _boxes(boxes):
    arr = (_Box * max(len(boxes), 1))()
    for e, (lo, hi) in enumerate(boxes):
        arr[e].lo[:] = list(lo)
        arr[e].hi[:] = list(hi)
    return arr


def generate(vol: np.ndarray, boxes, lut: np.ndarray, cam, step: float, ref_len: float, n_s: int,
             gamma: float, iters: int = 16, pixels=None, maxrec: int | None = None, owner_map=None,
             records: bool = True):
    """Phase-1 sub-VDIs.  gamma >= 0: fixed; gamma < 0: per-ray search.

    Returns (counts[k, np], gammas[k, np], recs[k, np, maxrec, 6], passes[k, np]).
    """
    V = Volume(vol)
    k = len(boxes)
    if pixels is None:
        pixels = np.arange(cam.width * cam.height, dtype=np.int32)
    pixels = np.ascontiguousarray(pixels, dtype=np.int32)
    np_ = len(pixels)
    if maxrec is None:
        maxrec = n_s
    counts = np.zeros((k, np_), dtype=np.int32)
    gammas = np.zeros((k, np_), dtype=np.float64)
    passes = np.zeros((k, np_), dtype=np.int32)
    recs = np.zeros((k, np_, maxrec, REC), dtype=np.float64) if records else None
    bx = _boxes(boxes)
    om = None if owner_map is None else np.ascontiguousarray(owner_map, dtype=np.int32)
    lut = np.ascontiguousarray(lut, dtype=np.float32)
    c = camera(cam)
    rc = _load().oc_generate(_ref(V.c), C.cast(bx, C.c_void_p), k, _p(om), _p(lut), _ref(c), step, ref_len, n_s,
                             gamma, iters, _p(pixels), np_, maxrec, _p(counts), _p(gammas), _p(recs), _p(passes))
    if rc != 0:
        raise RuntimeError(f"oc_generate failed ({rc})")
    return counts, gammas, recs, passes


def lists_from_recs(counts, recs):
    """Compact double-precision lists (one per PE) from generate()'s per-pixel arrays."""
    out = []
    k, np_, maxrec, _ = recs.shape
    for e in range(k):
        cnt = counts[e].astype(np.uint32)
        off = np.zeros(np_ + 1, dtype=np.uint64)
        off[1:] = np.cumsum(cnt, dtype=np.uint64)
        mask = np.arange(maxrec)[None, :] < cnt[:, None]
        flat = recs[e][mask]
        out.append((cnt, off, np.ascontiguousarray(flat[:, 0:2]), np.ascontiguousarray(flat[:, 2:6]), 0))
    return out


def composite(lists, n_s: int, iters: int = 16, pixels=None, n_pix=None, max_in=None):
    """Phase-2 compositing.  `lists`: per PE (counts u32, offsets u64, fb, rgba, prec) with
    prec 0 = float64 arrays, 1 = float32 arrays, 2 = 16-byte {f32 f, f32 b, f16 rgba} records in
    `rgba` (fb unused).  Returns (counts[np], gamma[np], recs[np, n_s, 6], passes[np])."""
    k = len(lists)
    if pixels is None:
        pixels = np.arange(n_pix, dtype=np.int32)
    pixels = np.ascontiguousarray(pixels, dtype=np.int32)
    np_ = len(pixels)
    keep = []
    arr = (_Lists * k)()
    for e, (cnt, off, fb, rgba, prec) in enumerate(lists):
        cnt = np.ascontiguousarray(cnt, dtype=np.uint32)
        off = np.ascontiguousarray(off, dtype=np.uint64)
        rgba = np.ascontiguousarray(rgba)
        fb = None if fb is None else np.ascontiguousarray(fb)
        keep += [cnt, off, fb, rgba]
        arr[e].counts = cnt.ctypes.data
        arr[e].offsets = off.ctypes.data
        arr[e].fb = None if fb is None else fb.ctypes.data
        arr[e].rgba = rgba.ctypes.data
        arr[e].prec = prec
    if max_in is None:
        max_in = max(1, sum(int(np.asarray(l[0])[pixels].max(initial=0)) for l in lists))
    counts = np.zeros(np_, dtype=np.int32)
    gam = np.zeros(np_, dtype=np.float64)
    passes = np.zeros(np_, dtype=np.int32)
    recs = np.zeros((np_, n_s, REC), dtype=np.float64)
    rc = _load().oc_composite(C.cast(arr, C.c_void_p), k, _p(pixels), np_, n_s, iters, max_in, _p(counts), _p(gam),
                              _p(recs), _p(passes))
    if rc != 0:
        raise RuntimeError(f"oc_composite failed ({rc})")
    return counts, gam, recs, passes


def pieces(recs):
    """Compositing pieces (f, b, P[3], a) of one pixel's records (array [n, 6])."""
    recs = np.ascontiguousarray(recs, dtype=np.float64).reshape(-1, REC)
    n = len(recs)
    out = (_Piece * (2 * n + 2))()
    bounds = np.zeros(2 * n + 2, dtype=np.float64)
    m = _load().oc_pieces(_p(recs), n, C.cast(out, C.c_void_p), 2 * n + 2, _p(bounds))
    return np.array([[p.f, p.b, p.P[0], p.P[1], p.P[2], p.a] for p in out[:m]], dtype=np.float64).reshape(-1, 6)


def _pieces_c(pcs, brk=None):
    pcs = np.asarray(pcs, dtype=np.float64).reshape(-1, 6)
    arr = (_Piece * max(len(pcs), 1))()
    for i, row in enumerate(pcs):
        arr[i].f, arr[i].b = row[0], row[1]
        arr[i].P[:] = list(row[2:5])
        arr[i].a = row[5]
        arr[i].brk = 0 if brk is None else int(brk[i])
    return arr, len(pcs)


def segment(pcs, gamma: float, cap: int = 1 << 30, brk=None):
    """State machine over pieces [n, 6] = (f, b, P[3], a).  Returns (count, records[m, 6])."""
    arr, n = _pieces_c(pcs, brk)
    out = np.zeros((max(n, 1) + 1, REC), dtype=np.float64)
    cnt = _load().oc_segment(C.cast(arr, C.c_void_p), n, gamma, cap, _p(out), len(out), None)
    m = min(cnt, len(out))
    # number written equals the number of supersegments opened (each is closed once)
    return cnt, out[:m].copy()


def search(pcs, n_s: int, iters: int = 16, brk=None):
    arr, n = _pieces_c(pcs, brk)
    passes = C.c_int(0)
    g = _load().oc_search(C.cast(arr, C.c_void_p), n, n_s, iters, C.cast(C.byref(passes), C.c_void_p))
    return g, passes.value


def flatten(counts, recs):
    """Front-to-back over of records: counts[np], recs[np, stride, 6] -> rgba[np, 4]."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    recs = np.ascontiguousarray(recs, dtype=np.float64)
    np_, stride = recs.shape[0], recs.shape[1]
    out = np.zeros((np_, 4), dtype=np.float64)
    _load().oc_flatten(_p(counts), _p(recs), np_, stride, _p(out))
    return out


def render_view(counts, recs, gen_cam, view_cam, pixels=None):
    """A regular VDI of camera gen_cam (counts[W H], recs[W H, n_s, 6]) rendered from view_cam:
    premultiplied rgba[np, 4] for the given pixels of view_cam (all by default)."""
    counts = np.ascontiguousarray(counts, dtype=np.int32).ravel()
    recs = np.ascontiguousarray(recs, dtype=np.float64)
    n_s = recs.shape[1]
    if pixels is None:
        pixels = np.arange(view_cam.width * view_cam.height, dtype=np.int32)
    pixels = np.ascontiguousarray(pixels, dtype=np.int32)
    out = np.zeros((len(pixels), 4), dtype=np.float64)
    g, v = camera(gen_cam), camera(view_cam)
    _load().oc_render_view(_p(counts), _p(recs), n_s, _ref(g), _ref(v), _p(pixels), len(pixels), _p(out))
    return out


def render_ray(counts, recs, gen_cam, o, d):
    """One ray o + s d (unit d) through the VDI of gen_cam: premultiplied rgba[4]."""
    counts = np.ascontiguousarray(counts, dtype=np.int32).ravel()
    recs = np.ascontiguousarray(recs, dtype=np.float64)
    o = np.ascontiguousarray(o, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(4, dtype=np.float64)
    g = camera(gen_cam)
    n_s = recs.shape[1]
    used = np.arange(n_s)[None, :] < counts[:, None]
    rho_max = float(recs[..., 1][used].max()) if used.any() else 0.0
    _load().oc_render_ray(_p(counts), _p(recs), n_s, rho_max, _ref(g), _p(o), _p(d), _p(out))
    return out


def dvr(vol, lut, cam, step: float, ref_len: float, pixels=None):
    V = Volume(vol)
    if pixels is None:
        pixels = np.arange(cam.width * cam.height, dtype=np.int32)
    pixels = np.ascontiguousarray(pixels, dtype=np.int32)
    out = np.zeros((len(pixels), 4), dtype=np.float64)
    c = camera(cam)
    lut = np.ascontiguousarray(lut, dtype=np.float32)
    _load().oc_dvr(_ref(V.c), _p(lut), _ref(c), step, ref_len, _p(pixels), len(pixels), _p(out))
    return out


def ray(cam, i, j):
    o = np.zeros(3)
    d = np.zeros(3)
    c = camera(cam)
    _load().oc_ray(_ref(c), i, j, _p(o), _p(d))
    return o, d


def hit_box(o, d, dims):
    tin = np.zeros(1)
    tout = np.zeros(1)
    hit = _load().oc_hit_box(_p(np.asarray(o, dtype=np.float64)), _p(np.asarray(d, dtype=np.float64)),
                             _p(np.asarray(dims, dtype=np.int32)), _p(tin), _p(tout))
    return bool(hit), float(tin[0]), float(tout[0])


def value(vol, p):
    V = Volume(vol)
    return _load().oc_value(_ref(V.c), _p(np.asarray(p, dtype=np.float64)))


def lut_correct(lut, step, ref_len):
    out = np.zeros((256, 4), dtype=np.float64)
    _load().oc_lut_correct(_p(np.ascontiguousarray(lut, dtype=np.float32)), step, ref_len, _p(out))
    return out


def classify(lutc, v):
    out = np.zeros(4)
    _load().oc_classify(_p(np.ascontiguousarray(lutc, dtype=np.float64)), float(v), _p(out))
    return out


def exclusive_scan(counts):
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    out = np.zeros(len(counts) + 1, dtype=np.uint64)
    _load().oc_exclusive_scan(_p(counts), len(counts), _p(out))
    return out


def half_to_double(h: int) -> float:
    return _load().oc_half_to_double(h)


def ray_sample_count(vol, cam, step, pixel):
    V = Volume(vol)
    c = camera(cam)
    t = np.zeros(2)
    n = _load().oc_ray_sample_count(_ref(V.c), _ref(c), step, pixel, _p(t))
    return n, float(t[0]), float(t[1])


# ----------------------------------------------------------------------------
# learned gamma (extension): tile features, labels, MLP
# ----------------------------------------------------------------------------
NF, NH, TILE = 40, 64, 16


def tile_features(vol, boxes, lut, cam, step, ref_len, n_s):
    """Features [k, tiles, 40] and valid [k, tiles] of every (PE, 16 x 16 tile)."""
    V = Volume(vol)
    k = len(boxes)
    tiles = ((cam.width + TILE - 1) // TILE) * ((cam.height + TILE - 1) // TILE)
    feats = np.zeros((k, tiles, NF))
    valid = np.zeros((k, tiles), dtype=np.int32)
    bx = _boxes(boxes)
    c = camera(cam)
    _load().oc_tile_features(_ref(V.c), C.cast(bx, C.c_void_p), k, _p(np.ascontiguousarray(lut, dtype=np.float32)),
                             _ref(c), step, ref_len, n_s, _p(feats), _p(valid))
    return feats, valid


def tile_labels(gammas, nts, W, H):
    """Per-tile median of log2(max(gamma, 2^-20)) over rays with nt > 0; gammas/nts [k, W*H]."""
    gammas = np.ascontiguousarray(gammas, dtype=np.float64)
    nts = np.ascontiguousarray(nts, dtype=np.int32)
    k = gammas.shape[0]
    tiles = ((W + TILE - 1) // TILE) * ((H + TILE - 1) // TILE)
    labels = np.zeros((k, tiles))
    valid = np.zeros((k, tiles), dtype=np.int32)
    _load().oc_tile_labels(_p(gammas), _p(nts), k, W, H, _p(labels), _p(valid))
    return labels, valid


def mlp_nparams():
    return _load().oc_mlp_nparams()


def mlp_forward(theta, x):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, NF)
    y = np.zeros(len(x))
    _load().oc_mlp_forward(_p(theta), _p(x), len(x), _p(y))
    return y


def mlp_loss_grad(theta, x, labels, valid=None):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, NF)
    labels = np.ascontiguousarray(labels, dtype=np.float64)
    valid = np.ones(len(x), dtype=np.int32) if valid is None else np.ascontiguousarray(valid, dtype=np.int32)
    g = np.zeros(mlp_nparams())
    loss = _load().oc_mlp_loss_grad(_p(theta), _p(x), _p(labels), _p(valid), len(x), _p(g))
    return loss, g
