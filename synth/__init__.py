"""Seeded synthetic inputs (volumes, transfer functions, camera orbits,
supersegment lists) shared by the oracle tests, the GPU tests and the
benchmark.  Nothing here implements any step of the VDI method.

The C source (``synth.c``) is compiled in-tree with gcc on first use (or by
``build()``); the functions below return numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lib = None

# Seeds of the standard workloads (volume seed = 0xC0FFEE + workload index).
SEED_VOLUME = 0xC0FFEE
SEED_TF = 7
SEED_ORBIT = 11
SEED_REQUESTS = 13
# request index of the record pool's runs (pooled lists)
POOL_REQ = 0xFFFF
POOL_RUN = 64


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
        build()
        lib = C.CDLL(_LIB)
        lib.synth_volume.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                     C.c_uint64, C.c_int, C.c_void_p]
        lib.synth_volume.restype = C.c_int
        lib.synth_tf.argtypes = [C.c_uint64, C.c_void_p]
        lib.synth_tf.restype = None
        lib.synth_orbit.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]
        lib.synth_orbit.restype = None
        lib.synth_list_len.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_int, C.c_int]
        lib.synth_list_len.restype = C.c_int
        lib.synth_list.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_int, C.c_int,
                                   C.c_void_p, C.c_void_p]
        lib.synth_list.restype = C.c_int
        lib.synth_lists_compact.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_int, C.c_int,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.synth_lists_compact.restype = C.c_uint64
        lib.synth_hash4.argtypes = [C.c_uint64] * 4
        lib.synth_hash4.restype = C.c_uint64
        lib.synth_pool_pick.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_int, C.c_uint64,
                                        C.c_void_p, C.c_void_p]
        lib.synth_pool_pick.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def volume(dims, n_blobs: int, octaves: int, seed: int, dtype=np.uint16,
           noise_amp: float = 0.1, base_freq: float = 4.0) -> np.ndarray:
    """Blob + value-noise field normalised to [0,1]; array shape (Z, Y, X).

    float32 volumes hold v in [0,1]; uint16 volumes hold round(v * 65535).
    """
    X, Y, Z = (int(d) for d in dims)
    out = np.empty((Z, Y, X), dtype=dtype)
    code = 0 if np.dtype(dtype) == np.float32 else 1
    if np.dtype(dtype) not in (np.dtype(np.float32), np.dtype(np.uint16)):
        raise ValueError("dtype must be float32 or uint16")
    rc = _load().synth_volume(X, Y, Z, n_blobs, octaves, noise_amp, base_freq, seed, code, _ptr(out))
    if rc != 0:
        raise RuntimeError("synth_volume failed")
    return out


def transfer_function(seed: int = SEED_TF) -> np.ndarray:
    """256 x 4 float32 RGBA: straight colour, opacity per unit (voxel) length."""
    lut = np.empty((256, 4), dtype=np.float32)
    _load().synth_tf(seed, _ptr(lut))
    return lut


@dataclass
class Camera:
    eye: tuple
    center: tuple
    up: tuple
    fovy_deg: float
    width: int
    height: int


def orbit(dims, n_views: int, width: int, height: int, seed: int = SEED_ORBIT, fovy_deg: float = 45.0):
    X, Y, Z = (int(d) for d in dims)
    raw = np.empty((n_views, 9), dtype=np.float64)
    _load().synth_orbit(seed, n_views, X, Y, Z, _ptr(raw))
    return [Camera(tuple(r[0:3]), tuple(r[3:6]), tuple(r[6:9]), fovy_deg, width, height) for r in raw]


def list_len(seed, req, set_, pixel, n_s, dense=False) -> int:
    return _load().synth_list_len(seed, req, set_, pixel, n_s, int(dense))


def one_list(seed, req, set_, pixel, n_s, dense=False):
    """(fb[n,2], rgba[n,4]) float32 of one synthetic list."""
    fb = np.empty((max(n_s, 1), 2), dtype=np.float32)
    rgba = np.empty((max(n_s, 1), 4), dtype=np.float32)
    n = _load().synth_list(seed, req, set_, pixel, n_s, int(dense), _ptr(fb), _ptr(rgba))
    if n < 0:
        raise ValueError("list too long")
    return fb[:n].copy(), rgba[:n].copy()


def lists_compact(seed, req, set_, n_pix, n_s, dense=False, with_records=True):
    """Compact arrays of one synthetic sub-VDI: counts[u32 n_pix],
    offsets[u64 n_pix+1], fb[f32 total,2], rgba[f32 total,4]."""
    lib = _load()
    counts = np.empty(n_pix, dtype=np.uint32)
    offsets = np.empty(n_pix + 1, dtype=np.uint64)
    total = lib.synth_lists_compact(seed, req, set_, n_pix, n_s, int(dense), _ptr(counts), _ptr(offsets), None, None)
    if not with_records:
        return counts, offsets, None, None
    fb = np.empty((total, 2), dtype=np.float32)
    rgba = np.empty((total, 4), dtype=np.float32)
    lib.synth_lists_compact(seed, req, set_, n_pix, n_s, int(dense), _ptr(counts), _ptr(offsets), _ptr(fb), _ptr(rgba))
    return counts, offsets, fb, rgba


def hash4(seed, a, b, c) -> int:
    return _load().synth_hash4(seed, a, b, c)


def pool_pick(seed, req, set_, pixel, n_s, runs):
    """(n, run, start) of the pooled list of (req, set, pixel): records
    [start, start + n) of pool run `run` (run r = one_list(seed, POOL_REQ, 0, r, POOL_RUN, dense=True))."""
    run = C.c_uint64(0)
    start = C.c_int(0)
    n = _load().synth_pool_pick(seed, req, set_, pixel, n_s, runs, C.byref(run), C.byref(start))
    return n, run.value, start.value


def pooled_lists(seed, req, set_, pixels, n_s, runs):
    """Per pixel (fb[n,2], rgba[n,4]) float32 of pooled lists, built on the host from the pool's runs."""
    out = []
    for p in pixels:
        n, r, s0 = pool_pick(seed, req, set_, int(p), n_s, runs)
        fb, rgba = one_list(seed, POOL_REQ, 0, r, POOL_RUN, dense=True)
        out.append((fb[s0:s0 + n], rgba[s0:s0 + n]))
    return out


def requests(n, seed=SEED_REQUESTS, w_range=(256, 1920), h_range=(256, 1080), k_range=(2, 32), n_s_range=(8, 64)):
    """Seeded request table of the batched workload: list of (w, h, k, n_s), each uniform on its range."""
    out = []
    for r in range(n):
        vals = []
        for i, (lo, hi) in enumerate((w_range, h_range, k_range, n_s_range)):
            vals.append(lo + hash4(seed, 0x72657173, r, i) % (hi - lo + 1))
        out.append(tuple(int(v) for v in vals))
    return out


# grids of K = 1, 2, 4, 8, 16 near-equal bricks
_GEN_GRIDS = ((1, 1, 1), (1, 1, 2), (1, 2, 2), (2, 2, 2), (4, 2, 2))


def gen_requests(n, seed=SEED_REQUESTS, sides=(128, 192, 256, 384), w_range=(256, 1920), h_range=(256, 1080),
                 n_s_range=(8, 64)):
    """Seeded table of uneven generation requests: list of (side, grid, w, h, n_s), the volume a side^3
    uint16 blob volume, K = product of grid in {1, 2, 4, 8, 16}, each field uniform on its set or range."""
    out = []
    for r in range(n):
        h = [hash4(seed, 0x67656E72, r, i) for i in range(5)]
        side = sides[h[0] % len(sides)]
        grid = _GEN_GRIDS[h[1] % len(_GEN_GRIDS)]
        w = w_range[0] + h[2] % (w_range[1] - w_range[0] + 1)
        hh = h_range[0] + h[3] % (h_range[1] - h_range[0] + 1)
        n_s = n_s_range[0] + h[4] % (n_s_range[1] - n_s_range[0] + 1)
        out.append((int(side), grid, int(w), int(hh), int(n_s)))
    return out
