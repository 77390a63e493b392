"""Helper of tests/test_zz_no_alloc.py, run as a child process: vdi_generate_static_scratch
in the device's primary context, then in a second context created on the same device with the
driver API (an in-situ host that keeps its own context), then in the primary context again after
the second one was destroyed.  Every buffer of a run is allocated in the context that is current
for it (cuMemAlloc), so no kernel touches another context's memory.  The three runs must give the
same counts, offsets, gamma and records.  Prints "OK <records>" and exits 0 on success.

The library looks up its static array's address in the context current at each call; an address
kept from the first context would be invalid in the second.
"""
import ctypes as C
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import paper_2206_14503_gb300 as vdi  # noqa: E402
import synth  # noqa: E402

cu = C.CDLL("libcuda.so.1")
for name in ("cuMemAlloc_v2", "cuMemFree_v2", "cuMemcpyHtoD_v2", "cuMemcpyDtoH_v2", "cuMemsetD8_v2"):
    getattr(cu, name).restype = C.c_int


def ck(r, what):
    if r != 0:
        raise RuntimeError(f"{what}: CUresult {r}")


class Buffers:
    """cuMemAlloc'ed buffers of the current context, freed together."""

    def __init__(self):
        self.ptrs = []

    def alloc(self, nbytes, host=None):
        p = C.c_uint64()
        ck(cu.cuMemAlloc_v2(C.byref(p), C.c_size_t(max(int(nbytes), 16))), "cuMemAlloc")
        self.ptrs.append(p.value)
        if host is not None:
            h = np.ascontiguousarray(host)
            ck(cu.cuMemcpyHtoD_v2(C.c_uint64(p.value), h.ctypes.data_as(C.c_void_p), C.c_size_t(h.nbytes)), "HtoD")
        else:
            ck(cu.cuMemsetD8_v2(C.c_uint64(p.value), C.c_ubyte(0), C.c_size_t(max(int(nbytes), 16))), "memset")
        return p.value

    def read(self, ptr, dtype, n):
        out = np.empty(n, dtype=dtype)
        ck(cu.cuMemcpyDtoH_v2(out.ctypes.data_as(C.c_void_p), C.c_uint64(ptr), C.c_size_t(out.nbytes)), "DtoH")
        return out

    def free(self):
        for p in self.ptrs:
            ck(cu.cuMemFree_v2(C.c_uint64(p)), "cuMemFree")
        self.ptrs = []


def run_once(vol, dims, boxes, lut, cam, n_s):
    b = Buffers()
    vol_d = b.alloc(vol.nbytes, vol)
    cells = [b.alloc(vdi.vdi_brick_bytes(bx)) for bx in boxes]
    bricks = vdi.vdi_brick_build(vol_d, vdi.VDI_VOL_U16, dims, boxes, cells, None)
    lut_d = b.alloc(lut.nbytes, lut)
    npix = cam.width * cam.height
    cap = npix * n_s
    outs, ptrs = [], []
    for _ in boxes:
        counts, offsets = b.alloc(npix * 4), b.alloc((npix + 1) * 8)
        gamma, rgba, fb = b.alloc(npix * 4), b.alloc(cap * 16), b.alloc(cap * 8)
        outs.append(vdi.vdi_compact(counts, offsets, rgba, fb, gamma, cap, vdi.VDI_PREC_F32))
        ptrs.append((counts, offsets, gamma, rgba, fb))
    vdi.check(vdi.vdi_generate_static_scratch(bricks, lut_d, vdi.make_camera(cam), n_s, vdi.VDI_GAMMA_SEARCH, outs,
                                              vdi.make_params()), "static scratch")
    ck(cu.cuCtxSynchronize(), "cuCtxSynchronize")
    res = []
    for counts, offsets, gamma, rgba, fb in ptrs:
        off = b.read(offsets, np.uint64, npix + 1)
        tot = int(off[-1])
        res.append((b.read(counts, np.uint32, npix), off, b.read(gamma, np.float32, npix),
                    b.read(rgba, np.float32, 4 * tot), b.read(fb, np.float32, 2 * tot)))
    b.free()
    return res


def main():
    dims = (48, 40, 56)
    vol = synth.volume(dims, 10, 3, 77, np.uint16)
    lut = np.ascontiguousarray(synth.transfer_function(synth.SEED_TF), dtype=np.float32)
    cam = synth.orbit(dims, 2, 72, 60, 21)[1]
    boxes = [vdi.vdi_box(lo, hi) for lo, hi in oracle.split_boxes(dims, (2, 1, 2))]
    n_s = 6
    ck(cu.cuInit(0), "cuInit")
    dev = C.c_int()
    ck(cu.cuDeviceGet(C.byref(dev), 0), "cuDeviceGet")
    primary = C.c_void_p()
    ck(cu.cuDevicePrimaryCtxRetain(C.byref(primary), dev), "cuDevicePrimaryCtxRetain")
    ck(cu.cuCtxSetCurrent(primary), "cuCtxSetCurrent(primary)")
    first = run_once(vol, dims, boxes, lut, cam, n_s)

    class CtxParams(C.Structure):
        _fields_ = [("execAffinityParams", C.c_void_p), ("numExecAffinityParams", C.c_int),
                    ("cigParams", C.c_void_p)]

    second_ctx = C.c_void_p()
    params = CtxParams(None, 0, None)
    ck(cu.cuCtxCreate_v4(C.byref(second_ctx), C.byref(params), C.c_uint(0), dev), "cuCtxCreate")
    ck(cu.cuCtxSetCurrent(second_ctx), "cuCtxSetCurrent(second)")
    second = run_once(vol, dims, boxes, lut, cam, n_s)
    ck(cu.cuCtxSetCurrent(primary), "cuCtxSetCurrent(primary again)")
    ck(cu.cuCtxDestroy_v2(second_ctx), "cuCtxDestroy")
    third = run_once(vol, dims, boxes, lut, cam, n_s)
    ck(cu.cuDevicePrimaryCtxRelease_v2(dev), "cuDevicePrimaryCtxRelease")
    records = 0
    for a, bb, c in zip(first, second, third):
        for x, y, z in zip(a, bb, c):
            assert np.array_equal(x, y) and np.array_equal(x, z)
        records += int(a[1][-1])
    assert records > 0
    print("OK", records)


if __name__ == "__main__":
    main()
