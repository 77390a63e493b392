// C ABI (include/vdi.h): argument checks on the host, then stream-ordered
// launches.  No entry point allocates device memory.
#include <math.h>
#include <map>
#include <mutex>
#include <stddef.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "vdi_internal.h"

namespace vdi {

static thread_local char g_msg[512];
static thread_local vdi_status g_last = VDI_OK;

vdi_status set_error(vdi_status s, const char* fmt, ...) {
    g_last = s;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return s;
}

vdi_status cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return VDI_OK;
    return set_error(VDI_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

CamDev make_cam(const vdi_camera& c) {
    double fwd[3], right[3], up[3];
    for (int a = 0; a < 3; ++a) fwd[a] = c.center[a] - c.eye[a];
    double n = sqrt(fwd[0] * fwd[0] + fwd[1] * fwd[1] + fwd[2] * fwd[2]);
    for (int a = 0; a < 3; ++a) fwd[a] /= n;
    right[0] = fwd[1] * c.up[2] - fwd[2] * c.up[1];
    right[1] = fwd[2] * c.up[0] - fwd[0] * c.up[2];
    right[2] = fwd[0] * c.up[1] - fwd[1] * c.up[0];
    n = sqrt(right[0] * right[0] + right[1] * right[1] + right[2] * right[2]);
    for (int a = 0; a < 3; ++a) right[a] /= n;
    up[0] = right[1] * fwd[2] - right[2] * fwd[1];
    up[1] = right[2] * fwd[0] - right[0] * fwd[2];
    up[2] = right[0] * fwd[1] - right[1] * fwd[0];
    double th = tan(0.5 * c.fovy_deg * 3.14159265358979323846 / 180.0);
    CamDev d;
    auto split = [](double v, float out[2]) {
        out[0] = (float)v;
        out[1] = (float)(v - (double)out[0]);
    };
    for (int a = 0; a < 3; ++a) {
        split(c.eye[a], d.eye[a]);
        split(fwd[a], d.fwd[a]);
        split(right[a], d.right[a]);
        split(up[a], d.up[a]);
    }
    split(th * (double)c.width / (double)c.height, d.sx);
    split(th, d.sy);
    d.W = c.width;
    d.H = c.height;
    return d;
}

static bool camera_ok(const vdi_camera* c) {
    if (!c || c->width < 1 || c->height < 1 || !(c->fovy_deg > 0.0 && c->fovy_deg < 180.0)) return false;
    double f[3] = {c->center[0] - c->eye[0], c->center[1] - c->eye[1], c->center[2] - c->eye[2]};
    double r[3] = {f[1] * c->up[2] - f[2] * c->up[1], f[2] * c->up[0] - f[0] * c->up[2], f[0] * c->up[1] - f[1] * c->up[0]};
    return (f[0] * f[0] + f[1] * f[1] + f[2] * f[2]) > 0.0 && (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) > 0.0;
}

static bool params_ok(const vdi_params* p) {
    return p && p->step > 0.f && p->ref_len > 0.f && p->bisect_iters >= 1 && p->bisect_iters <= 24;
}

BrickDev brick_dev(const vdi_brick& b) {
    BrickDev d;
    d.cells = b.cells;
    for (int a = 0; a < 3; ++a) {
        d.lo[a] = b.owned.lo[a];
        d.hi[a] = b.owned.hi[a];
    }
    d.nx = b.owned.hi[0] - b.owned.lo[0] + 2;
    d.ny = b.owned.hi[1] - b.owned.lo[1] + 2;
    d.nz = b.owned.hi[2] - b.owned.lo[2] + 2;
    d.ncells = d.nx * d.ny * d.nz;
    return d;
}

}  // namespace vdi

using namespace vdi;

extern "C" {

int32_t vdi_version(void) { return 100; }

const char* vdi_status_string(vdi_status s) {
    switch (s) {
        case VDI_OK: return "ok";
        case VDI_ERR_INVALID_ARG: return "invalid argument";
        case VDI_ERR_CAPACITY: return "output capacity too small";
        case VDI_ERR_WORKSPACE: return "workspace too small";
        case VDI_ERR_CUDA: return "CUDA error";
        case VDI_ERR_TIMEOUT: return "device wait timed out";
        case VDI_ERR_MODEL: return "model error";
        case VDI_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

vdi_status vdi_last_error(char* buf, size_t n) {
    if (buf && n > 0) {
        strncpy(buf, g_msg, n - 1);
        buf[n - 1] = 0;
    }
    return g_last;
}

// true if p is device (or managed) memory of the current context: a host or stray pointer handed to a
// device-to-host copy would otherwise be read as host memory
static bool device_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

vdi_status vdi_workspace_status(const void* workspace, vdi_stream stream) {
    if (!workspace) return set_error(VDI_ERR_INVALID_ARG, "vdi_workspace_status: workspace is NULL");
    if (!device_pointer(workspace))
        return set_error(VDI_ERR_INVALID_ARG, "vdi_workspace_status: workspace is not device memory");
    unsigned int s = 0;
    cudaStream_t st = (cudaStream_t)stream;
    vdi_status r = cuda_check(cudaMemcpyAsync(&s, workspace, sizeof s, cudaMemcpyDeviceToHost, st), "status read");
    if (r != VDI_OK) return r;
    r = cuda_check(cudaStreamSynchronize(st), "status sync");
    if (r != VDI_OK) return r;
    if (s != 0) return set_error((vdi_status)s, "device reported: %s", vdi_status_string((vdi_status)s));
    return VDI_OK;
}

vdi_status vdi_workspace_counters(const void* workspace, uint64_t counters[8], vdi_stream stream) {
    if (!workspace || !counters) return set_error(VDI_ERR_INVALID_ARG, "vdi_workspace_counters: NULL argument");
    if (!device_pointer(workspace))
        return set_error(VDI_ERR_INVALID_ARG, "vdi_workspace_counters: workspace is not device memory");
    cudaStream_t st = (cudaStream_t)stream;
    const char* src = static_cast<const char*>(workspace) + offsetof(WsHeader, counters);
    vdi_status r = cuda_check(cudaMemcpyAsync(counters, src, 8 * sizeof(uint64_t), cudaMemcpyDeviceToHost, st),
                              "counters read");
    if (r != VDI_OK) return r;
    return cuda_check(cudaStreamSynchronize(st), "counters sync");
}

vdi_status vdi_split_boxes(const int32_t dims[3], const int32_t grid[3], vdi_box* boxes_out) {
    if (!dims || !grid || !boxes_out) return set_error(VDI_ERR_INVALID_ARG, "vdi_split_boxes: NULL argument");
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2 || grid[a] < 1 || grid[a] > dims[a] - 1)
            return set_error(VDI_ERR_INVALID_ARG, "vdi_split_boxes: axis %d: dims %d grid %d", a, dims[a], grid[a]);
    if ((long)grid[0] * grid[1] * grid[2] > VDI_MAX_PE)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_split_boxes: more than %d PEs", VDI_MAX_PE);
    int e = 0;
    for (int z = 0; z < grid[2]; ++z)
        for (int y = 0; y < grid[1]; ++y)
            for (int x = 0; x < grid[0]; ++x) {
                int idx[3] = {x, y, z};
                for (int a = 0; a < 3; ++a) {
                    long cells = dims[a] - 1;
                    // run a of g gets cells [floor(a C / g), floor((a+1) C / g))
                    boxes_out[e].lo[a] = (int32_t)(cells * idx[a] / grid[a]);
                    boxes_out[e].hi[a] = (int32_t)(cells * (idx[a] + 1) / grid[a]);
                }
                ++e;
            }
    return VDI_OK;
}

size_t vdi_brick_bytes(const vdi_box* b) {
    if (!b) return 0;
    size_t n = 1;
    for (int a = 0; a < 3; ++a) {
        if (b->hi[a] <= b->lo[a]) return 0;
        n *= (size_t)(b->hi[a] - b->lo[a] + 2);
    }
    return n * 8 * sizeof(float);
}

vdi_status vdi_brick_build(const void* volume, vdi_voltype type, const int32_t dims[3], int32_t k,
                           const vdi_box* boxes, float* const* cells_out, vdi_brick* bricks_out, vdi_stream stream) {
    if (!volume || !dims || !boxes || !cells_out || !bricks_out)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_brick_build: NULL argument");
    if (k < 1 || k > VDI_MAX_PE) return set_error(VDI_ERR_INVALID_ARG, "vdi_brick_build: k = %d", k);
    if (type != VDI_VOL_F32 && type != VDI_VOL_U16) return set_error(VDI_ERR_INVALID_ARG, "vdi_brick_build: type");
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2) return set_error(VDI_ERR_INVALID_ARG, "vdi_brick_build: dims[%d] = %d", a, dims[a]);
    for (int e = 0; e < k; ++e) {
        for (int a = 0; a < 3; ++a)
            if (boxes[e].lo[a] < 0 || boxes[e].hi[a] > dims[a] - 1 || boxes[e].hi[a] <= boxes[e].lo[a])
                return set_error(VDI_ERR_INVALID_ARG, "vdi_brick_build: box %d axis %d [%d, %d)", e, a,
                                 boxes[e].lo[a], boxes[e].hi[a]);
        if (!cells_out[e]) return set_error(VDI_ERR_INVALID_ARG, "vdi_brick_build: cells_out[%d] NULL", e);
        if ((reinterpret_cast<uintptr_t>(cells_out[e]) & 15) != 0)
            return set_error(VDI_ERR_INVALID_ARG, "vdi_brick_build: cells_out[%d] not 16-byte aligned", e);
        if (vdi_brick_bytes(&boxes[e]) / 32 > (size_t)INT32_MAX)
            return set_error(VDI_ERR_INVALID_ARG, "vdi_brick_build: box %d too large", e);
    }
    vdi_status s = launch_brick_build(volume, type, dims, k, boxes, cells_out, (cudaStream_t)stream);
    if (s != VDI_OK) return s;
    for (int e = 0; e < k; ++e) {
        bricks_out[e].cells = cells_out[e];
        bricks_out[e].owned = boxes[e];
        for (int a = 0; a < 3; ++a) bricks_out[e].dims[a] = dims[a];
        bricks_out[e].value_scale = type == VDI_VOL_U16 ? (float)(1.0 / 65535.0) : 1.0f;
    }
    return VDI_OK;
}

static size_t gen_min_workspace(int k, int w, int h) { return kGenFixed + scan_workspace(k, w * h); }

size_t vdi_generate_workspace(int32_t k, int32_t w, int32_t h) {
    if (k < 1 || w < 0 || h < 0) return 0;
    int ctas = 0;
    size_t cache = 0;
    if (gen_count_grid(ctas) == VDI_OK) cache = gen_cache_bytes(ctas);
    size_t bytes = gen_min_workspace(k, w, h) + align_up(cache, 256);
    if (cache > 0) bytes += align_up(gen_span_bytes(k, w, h), 256) + 256;  // the recorded spans and their tag
    return bytes;
}

static vdi_status gen_check(const char* fn, const vdi_brick* bricks, int32_t k, const float* tf_lut,
                            const vdi_camera* cam, int32_t n_s, float gamma, const vdi_compact* out,
                            const vdi_params* params, bool need_records) {
    if (!bricks || !tf_lut || !cam || !out || !params) return set_error(VDI_ERR_INVALID_ARG, "%s: NULL argument", fn);
    if (k < 1 || k > VDI_MAX_PE) return set_error(VDI_ERR_INVALID_ARG, "%s: k = %d", fn, k);
    if (n_s < 1) return set_error(VDI_ERR_INVALID_ARG, "%s: n_s = %d", fn, n_s);
    if (!camera_ok(cam)) return set_error(VDI_ERR_INVALID_ARG, "%s: camera", fn);
    if (!params_ok(params)) return set_error(VDI_ERR_INVALID_ARG, "%s: params", fn);
    if (!(gamma >= 0.f || gamma == VDI_GAMMA_SEARCH || gamma == VDI_GAMMA_GIVEN ||
          (need_records && gamma == VDI_GAMMA_CHOSEN)) || isinf(gamma))
        return set_error(VDI_ERR_INVALID_ARG, "%s: gamma %g", fn, (double)gamma);
    if ((long long)cam->width * cam->height > (long long)INT32_MAX / 2)
        return set_error(VDI_ERR_INVALID_ARG, "%s: image too large", fn);
    for (int e = 0; e < k; ++e) {
        const vdi_brick& b = bricks[e];
        if (!b.cells) return set_error(VDI_ERR_INVALID_ARG, "%s: brick %d has no cells", fn, e);
        for (int a = 0; a < 3; ++a)
            if (b.dims[a] != bricks[0].dims[a] || b.dims[a] < 2 || b.owned.lo[a] < 0 ||
                b.owned.hi[a] > b.dims[a] - 1 || b.owned.hi[a] <= b.owned.lo[a])
                return set_error(VDI_ERR_INVALID_ARG, "%s: brick %d box/dims", fn, e);
        if (b.value_scale != bricks[0].value_scale) return set_error(VDI_ERR_INVALID_ARG, "%s: value_scale", fn);
        const vdi_compact& o = out[e];
        if (!o.counts || !o.gamma) return set_error(VDI_ERR_INVALID_ARG, "%s: out[%d] counts/gamma NULL", fn, e);
        if (need_records) {
            if (!o.offsets) return set_error(VDI_ERR_INVALID_ARG, "%s: out[%d].offsets NULL", fn, e);
            if (o.prec != VDI_PREC_F32 && o.prec != VDI_PREC_F16)
                return set_error(VDI_ERR_INVALID_ARG, "%s: out[%d].prec", fn, e);
            if (o.prec != out[0].prec) return set_error(VDI_ERR_INVALID_ARG, "%s: mixed precisions", fn);
            if (o.capacity > 0 && (!o.rgba || (o.prec == VDI_PREC_F32 && !o.fb)))
                return set_error(VDI_ERR_INVALID_ARG, "%s: out[%d] record arrays NULL", fn, e);
            if ((reinterpret_cast<uintptr_t>(o.rgba) & 15) || (reinterpret_cast<uintptr_t>(o.fb) & 7))
                return set_error(VDI_ERR_INVALID_ARG, "%s: out[%d] record arrays misaligned", fn, e);
        }
    }
    return VDI_OK;
}

static vdi_status gen_common(const char* fn, const vdi_brick* bricks, int32_t k, const float* tf_lut,
                             const vdi_camera* cam, int32_t n_s, float gamma, vdi_compact* out,
                             const vdi_params* params, void* workspace, size_t ws_bytes, bool need_records) {
    vdi_status s = gen_check(fn, bricks, k, tf_lut, cam, n_s, gamma, out, params, need_records);
    if (s != VDI_OK) return s;
    if (!workspace || ws_bytes < gen_min_workspace(k, cam->width, cam->height))
        return set_error(VDI_ERR_WORKSPACE, "%s: workspace %zu < %zu bytes", fn, ws_bytes,
                         gen_min_workspace(k, cam->width, cam->height));
    if (reinterpret_cast<uintptr_t>(workspace) & 255)
        return set_error(VDI_ERR_INVALID_ARG, "%s: workspace not 256-byte aligned", fn);
    return VDI_OK;
}

vdi_status vdi_choose_gamma(const vdi_brick* bricks, int32_t k, const float* tf_lut, const vdi_camera* cam,
                            int32_t n_s, float gamma, vdi_compact* out, const vdi_params* params, void* workspace,
                            size_t ws_bytes, vdi_stream stream) {
    vdi_status s = gen_common("vdi_choose_gamma", bricks, k, tf_lut, cam, n_s, gamma, out, params, workspace,
                              ws_bytes, false);
    if (s != VDI_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int* status = reinterpret_cast<unsigned int*>(workspace);
    s = cuda_check(cudaMemsetAsync(status, 0, kGenFixed, st), "status clear");
    if (s != VDI_OK) return s;
    BrickDev bd[VDI_MAX_PE];
    CompactDev od[VDI_MAX_PE];
    for (int e = 0; e < k; ++e) {
        bd[e] = brick_dev(bricks[e]);
        od[e] = CompactDev{out[e].counts, out[e].offsets, out[e].rgba, out[e].fb, out[e].gamma, out[e].capacity};
    }
    CamDev cd = make_cam(*cam);
    float scale255 = (float)(255.0 * (double)bricks[0].value_scale);
    const size_t fixed = gen_min_workspace(k, cam->width, cam->height);
    char* ws = static_cast<char*>(workspace);
    return launch_gen_count(bd, k, tf_lut, cd, bricks[0].dims, scale255, params->step, params->ref_len, n_s, gamma,
                            params->bisect_iters, od, status, (params->flags & VDI_FLAG_CENSUS) != 0,
                            reinterpret_cast<unsigned int*>(ws + kWsHeader), ws + fixed, ws_bytes - fixed, st);
}

static vdi_status generate_compact(const char* fn, const vdi_brick* bricks, int32_t k, const float* tf_lut,
                                   const vdi_camera* cam, int32_t n_s, float gamma, vdi_compact* out,
                                   const vdi_params* params, void* workspace, size_t ws_bytes, vdi_stream stream,
                                   const OwnerDev* own) {
    vdi_status s = gen_common(fn, bricks, k, tf_lut, cam, n_s, gamma, out, params, workspace, ws_bytes, true);
    if (s != VDI_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int* status = reinterpret_cast<unsigned int*>(workspace);
    s = cuda_check(cudaMemsetAsync(status, 0, kGenFixed, st), "status clear");
    if (s != VDI_OK) return s;
    BrickDev bd[VDI_MAX_PE];
    CompactDev od[VDI_MAX_PE];
    uint32_t* cnts[VDI_MAX_PE];
    uint64_t* offs[VDI_MAX_PE];
    for (int e = 0; e < k; ++e) {
        bd[e] = brick_dev(bricks[e]);
        od[e] = CompactDev{out[e].counts, out[e].offsets, out[e].rgba, out[e].fb, out[e].gamma, out[e].capacity};
        cnts[e] = out[e].counts;
        offs[e] = out[e].offsets;
    }
    CamDev cd = make_cam(*cam);
    float scale255 = (float)(255.0 * (double)bricks[0].value_scale);
    const int npix = cam->width * cam->height;
    const size_t fixed = gen_min_workspace(k, cam->width, cam->height);
    char* ws = static_cast<char*>(workspace);
    if (gamma != VDI_GAMMA_CHOSEN) {
        s = launch_gen_count(bd, k, tf_lut, cd, bricks[0].dims, scale255, params->step, params->ref_len, n_s, gamma,
                             params->bisect_iters, od, status, (params->flags & VDI_FLAG_CENSUS) != 0,
                             reinterpret_cast<unsigned int*>(ws + kWsHeader), ws + fixed, ws_bytes - fixed, st,
                             own);
        if (s != VDI_OK) return s;
    }
    s = launch_scan(k, npix, cnts, offs, ws + kGenFixed, st);
    if (s != VDI_OK) return s;
    if (params->flags & VDI_FLAG_SYNC_CAPACITY) {
        uint64_t tot[VDI_MAX_PE];
        for (int e = 0; e < k; ++e) {
            s = cuda_check(cudaMemcpyAsync(&tot[e], offs[e] + npix, sizeof(uint64_t), cudaMemcpyDeviceToHost, st),
                           "total read");
            if (s != VDI_OK) return s;
        }
        s = cuda_check(cudaStreamSynchronize(st), "total sync");
        if (s != VDI_OK) return s;
        for (int e = 0; e < k; ++e)
            if (tot[e] > out[e].capacity)
                return set_error(VDI_ERR_CAPACITY, "%s: PE %d needs %llu records, capacity %llu", fn, e,
                                 (unsigned long long)tot[e], (unsigned long long)out[e].capacity);
    }
    return launch_gen_emit(bd, k, tf_lut, cd, bricks[0].dims, scale255, params->step, params->ref_len, n_s,
                           out[0].prec, od, status, st, false, own, ws + fixed, ws_bytes - fixed);
}

vdi_status vdi_generate(const vdi_brick* bricks, int32_t k, const float* tf_lut, const vdi_camera* cam, int32_t n_s,
                        float gamma, vdi_compact* out, const vdi_params* params, void* workspace, size_t ws_bytes,
                        vdi_stream stream) {
    return generate_compact("vdi_generate", bricks, k, tf_lut, cam, n_s, gamma, out, params, workspace, ws_bytes,
                            stream, nullptr);
}

size_t vdi_gen_batch_table_bytes(const vdi_gen_request* reqs, int32_t n) {
    if (!reqs || n < 0) return 0;
    return gen_batch_table_bytes(reqs, n);
}

vdi_status vdi_gen_batch_table_pack(const vdi_gen_request* reqs, int32_t n, const vdi_params* params,
                                    void* host_table, size_t bytes) {
    if (!reqs || n < 0 || !params || !host_table)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_gen_batch_table_pack: NULL argument");
    char fn[64];
    for (int q = 0; q < n; ++q) {
        const vdi_gen_request& g = reqs[q];
        snprintf(fn, sizeof fn, "vdi_gen_batch_table_pack: request %d", q);
        if (g.gamma == VDI_GAMMA_CHOSEN) return set_error(VDI_ERR_INVALID_ARG, "%s: gamma", fn);
        vdi_status s = gen_check(fn, g.bricks, g.k, g.tf_lut, &g.cam, g.n_s, g.gamma, g.out, params, true);
        if (s != VDI_OK) return s;
    }
    return gen_batch_table_pack(reqs, n, params, host_table, bytes);
}

size_t vdi_generate_batched_workspace(const void* host_table) {
    if (!host_table) return 0;
    return gen_batched_workspace_bytes(host_table);
}

vdi_status vdi_generate_batched(const void* dev_table, const void* host_table, void* workspace, size_t ws_bytes,
                                vdi_stream stream) {
    if (!dev_table || !host_table || !workspace)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_batched: NULL argument");
    if (reinterpret_cast<uintptr_t>(workspace) & 255)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_batched: workspace not 256-byte aligned");
    if (reinterpret_cast<uintptr_t>(dev_table) & 63)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_batched: table not 64-byte aligned");
    return launch_gen_batched(dev_table, host_table, workspace, ws_bytes, (cudaStream_t)stream);
}

vdi_status vdi_generate_owned(const vdi_brick* bricks, int32_t k, const float* tf_lut, const vdi_camera* cam,
                              int32_t n_s, float gamma, const vdi_ownership* own, vdi_compact* out,
                              const vdi_params* params, void* workspace, size_t ws_bytes, vdi_stream stream) {
    if (!own || !own->owner || !bricks) return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_owned: NULL argument");
    if (gamma == VDI_GAMMA_CHOSEN)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_owned: gamma mode VDI_GAMMA_CHOSEN");
    int shift = 0;
    while (shift < 11 && (1 << shift) != own->block) ++shift;
    if (shift >= 11) return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_owned: block %d", own->block);
    if (k >= 1 && k <= VDI_MAX_PE)
        for (int a = 0; a < 3; ++a) {
            const int cells = bricks[0].dims[a] - 1;
            if (cells < 1 || own->nb[a] != (cells + own->block - 1) / own->block)
                return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_owned: nb[%d] = %d for %d cells", a, own->nb[a],
                                 cells);
        }
    const OwnerDev od{own->owner, shift, {own->nb[0], own->nb[1], own->nb[2]}};
    return generate_compact("vdi_generate_owned", bricks, k, tf_lut, cam, n_s, gamma, out, params, workspace,
                            ws_bytes, stream, &od);
}

vdi_status vdi_generate_regular(const vdi_brick* bricks, int32_t k, const float* tf_lut, const vdi_camera* cam,
                                int32_t n_s, float gamma, vdi_regular* out, const vdi_params* params,
                                void* workspace, size_t ws_bytes, vdi_stream stream) {
    if (!out) return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_regular: NULL argument");
    vdi_compact tmp[VDI_MAX_PE];
    const int kk = (k >= 1 && k <= VDI_MAX_PE) ? k : 0;
    for (int e = 0; e < kk; ++e)
        tmp[e] = vdi_compact{out[e].counts, nullptr, out[e].rgba, out[e].fb, out[e].gamma, 0, out[e].prec};
    vdi_status s = gen_common("vdi_generate_regular", bricks, k, tf_lut, cam, n_s, gamma, kk ? tmp : nullptr, params,
                              workspace, ws_bytes, false);
    if (s != VDI_OK) return s;
    if (gamma == VDI_GAMMA_CHOSEN) return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_regular: gamma mode");
    for (int e = 0; e < k; ++e) {
        const vdi_regular& o = out[e];
        if (o.n_s != n_s) return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_regular: out[%d].n_s != n_s", e);
        if ((o.prec != VDI_PREC_F32 && o.prec != VDI_PREC_F16) || o.prec != out[0].prec)
            return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_regular: out[%d].prec", e);
        if (!o.rgba || (o.prec == VDI_PREC_F32 && !o.fb))
            return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_regular: out[%d] record arrays NULL", e);
        if ((reinterpret_cast<uintptr_t>(o.rgba) & 15) || (reinterpret_cast<uintptr_t>(o.fb) & 7))
            return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_regular: out[%d] record arrays misaligned", e);
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int* status = reinterpret_cast<unsigned int*>(workspace);
    s = cuda_check(cudaMemsetAsync(status, 0, kGenFixed, st), "status clear");
    if (s != VDI_OK) return s;
    const uint64_t slots = (uint64_t)cam->width * (uint64_t)cam->height * (uint64_t)n_s;
    BrickDev bd[VDI_MAX_PE];
    CompactDev od[VDI_MAX_PE];
    for (int e = 0; e < k; ++e) {
        bd[e] = brick_dev(bricks[e]);
        od[e] = CompactDev{out[e].counts, nullptr, out[e].rgba, reinterpret_cast<float*>(out[e].fb), out[e].gamma,
                           slots};
    }
    CamDev cd = make_cam(*cam);
    float scale255 = (float)(255.0 * (double)bricks[0].value_scale);
    const size_t fixed = gen_min_workspace(k, cam->width, cam->height);
    char* ws = static_cast<char*>(workspace);
    s = launch_gen_count(bd, k, tf_lut, cd, bricks[0].dims, scale255, params->step, params->ref_len, n_s, gamma,
                         params->bisect_iters, od, status, (params->flags & VDI_FLAG_CENSUS) != 0,
                         reinterpret_cast<unsigned int*>(ws + kWsHeader), ws + fixed, ws_bytes - fixed, st);
    if (s != VDI_OK) return s;
    return launch_gen_emit(bd, k, tf_lut, cd, bricks[0].dims, scale255, params->step, params->ref_len, n_s,
                           out[0].prec, od, status, st, true, nullptr, ws + fixed, ws_bytes - fixed);
}

size_t vdi_composite_workspace(int32_t k, int32_t w, int32_t h, int32_t n_s) {
    (void)k; (void)n_s;
    if (w < 0 || h < 0) return 0;
    return composite_workspace_bytes(w, h);
}

vdi_status vdi_composite(const vdi_compact* pe, int32_t k, int32_t w, int32_t h, vdi_regular* out,
                         const vdi_params* params, void* workspace, size_t ws_bytes, vdi_stream stream) {
    if (!pe || !out || !params) return set_error(VDI_ERR_INVALID_ARG, "vdi_composite: NULL argument");
    if (k < 1 || k > VDI_MAX_PE) return set_error(VDI_ERR_INVALID_ARG, "vdi_composite: k = %d", k);
    if (w < 0 || h < 0 || (long long)w * h > (long long)INT32_MAX / 2)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_composite: image %d x %d", w, h);
    if (out->n_s < 1) return set_error(VDI_ERR_INVALID_ARG, "vdi_composite: n_s = %d", out->n_s);
    if (params->bisect_iters < 1 || params->bisect_iters > 24)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_composite: bisect_iters");
    if (params->schedule < 0 || params->schedule > VDI_SCHED_LANE)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_composite: schedule %d", params->schedule);
    for (int e = 0; e < k; ++e) {
        if (!pe[e].counts || !pe[e].offsets || !pe[e].rgba)
            return set_error(VDI_ERR_INVALID_ARG, "vdi_composite: pe[%d] NULL array", e);
        if (pe[e].prec != pe[0].prec || (pe[e].prec != VDI_PREC_F32 && pe[e].prec != VDI_PREC_F16))
            return set_error(VDI_ERR_INVALID_ARG, "vdi_composite: pe[%d].prec", e);
        if (pe[e].prec == VDI_PREC_F32 && !pe[e].fb)
            return set_error(VDI_ERR_INVALID_ARG, "vdi_composite: pe[%d].fb NULL", e);
        if ((reinterpret_cast<uintptr_t>(pe[e].rgba) & 15) || (reinterpret_cast<uintptr_t>(pe[e].fb) & 7))
            return set_error(VDI_ERR_INVALID_ARG, "vdi_composite: pe[%d] misaligned", e);
    }
    if (!out->counts || !out->rgba || (out->prec == VDI_PREC_F32 && !out->fb))
        return set_error(VDI_ERR_INVALID_ARG, "vdi_composite: output array NULL");
    if (out->prec != VDI_PREC_F32 && out->prec != VDI_PREC_F16)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_composite: out->prec");
    if (!workspace || ws_bytes < kWsHeader) return set_error(VDI_ERR_WORKSPACE, "vdi_composite: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int* status = reinterpret_cast<unsigned int*>(workspace);
    const bool census = (params->flags & VDI_FLAG_CENSUS) != 0;
    vdi_status s = cuda_check(cudaMemsetAsync(status, 0, census ? kWsHeader : sizeof(unsigned int), st),
                              "status clear");
    if (s != VDI_OK) return s;
    s = launch_composite(pe, k, w, h, out, params->bisect_iters, params->schedule, status, workspace, ws_bytes, st,
                         census);
    if (s == VDI_ERR_CUDA &&
        (params->schedule == 0 || params->schedule == VDI_SCHED_STAGED || params->schedule == VDI_SCHED_LANE) &&
        ws_bytes < composite_workspace_bytes(1, 1))
        return set_error(VDI_ERR_WORKSPACE, "vdi_composite: workspace too small for the staged and lane schedules");
    return s;
}

size_t vdi_batch_table_bytes(const vdi_request* reqs, int32_t n) {
    if (!reqs || n < 0) return 0;
    return batch_table_bytes(reqs, n);
}

static vdi_status check_request(const vdi_request& q, int idx, int prec0) {
    if (!q.pe || q.k < 1 || q.k > VDI_MAX_PE) return set_error(VDI_ERR_INVALID_ARG, "request %d: k = %d", idx, q.k);
    if (q.w < 0 || q.h < 0 || (long long)q.w * q.h > (long long)INT32_MAX / 2)
        return set_error(VDI_ERR_INVALID_ARG, "request %d: image %d x %d", idx, q.w, q.h);
    if (q.out.n_s < 1 || !q.out.counts || !q.out.rgba || (q.out.prec == VDI_PREC_F32 && !q.out.fb))
        return set_error(VDI_ERR_INVALID_ARG, "request %d: output", idx);
    if (q.schedule < 0 || q.schedule > VDI_SCHED_LANE)
        return set_error(VDI_ERR_INVALID_ARG, "request %d: schedule", idx);
    for (int e = 0; e < q.k; ++e) {
        const vdi_compact& c = q.pe[e];
        if (!c.counts || !c.offsets || !c.rgba || (c.prec == VDI_PREC_F32 && !c.fb))
            return set_error(VDI_ERR_INVALID_ARG, "request %d: pe[%d] NULL array", idx, e);
        if (c.prec != prec0) return set_error(VDI_ERR_INVALID_ARG, "request %d: mixed input precisions", idx);
        if ((reinterpret_cast<uintptr_t>(c.rgba) & 15) || (reinterpret_cast<uintptr_t>(c.fb) & 7))
            return set_error(VDI_ERR_INVALID_ARG, "request %d: pe[%d] misaligned", idx, e);
    }
    return VDI_OK;
}

vdi_status vdi_batch_table_pack(const vdi_request* reqs, int32_t n, void* host_table, size_t bytes) {
    if (!reqs || n < 1 || !host_table) return set_error(VDI_ERR_INVALID_ARG, "vdi_batch_table_pack: arguments");
    const int prec0 = reqs[0].pe ? reqs[0].pe[0].prec : 0;
    for (int r = 0; r < n; ++r) {
        vdi_status s = check_request(reqs[r], r, prec0);
        if (s != VDI_OK) return s;
    }
    return batch_table_pack(reqs, n, host_table, bytes);
}

size_t vdi_composite_batched_workspace(const void* host_table) {
    if (!host_table) return 0;
    return batched_workspace_bytes(host_table);
}

vdi_status vdi_composite_batched(const void* dev_table, const void* host_table, const vdi_params* params,
                                 void* workspace, size_t ws_bytes, vdi_stream stream) {
    if (!dev_table || !host_table || !params)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_composite_batched: NULL argument");
    if (params->bisect_iters < 1 || params->bisect_iters > 24)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_composite_batched: bisect_iters");
    if (!workspace || ws_bytes < batched_workspace_bytes(host_table))
        return set_error(VDI_ERR_WORKSPACE, "vdi_composite_batched: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int* status = reinterpret_cast<unsigned int*>(workspace);
    vdi_status s = cuda_check(cudaMemsetAsync(workspace, 0, kWsHeader, st), "batched: clear");
    if (s != VDI_OK) return s;
    return launch_composite_batched(dev_table, host_table, params->bisect_iters, status, workspace, ws_bytes, st);
}

static std::mutex g_tune_mu;
static std::map<long long, int> g_tune_cache;

static long long tune_key(const vdi_request& q) {
    int kb = q.k <= 8 ? 8 : (q.k <= 16 ? 16 : (q.k <= 32 ? 32 : 64));
    int nb = q.out.n_s <= 16 ? 16 : (q.out.n_s <= 32 ? 32 : (q.out.n_s <= 64 ? 64 : 128));
    return ((long long)kb << 32) | ((long long)nb << 8) | (long long)q.pe[0].prec;
}

vdi_status vdi_composite_autotune(vdi_request* reqs, int32_t n, const vdi_params* params, void* workspace,
                                  size_t ws_bytes, vdi_stream stream) {
    if (!reqs || n < 1 || !params) return set_error(VDI_ERR_INVALID_ARG, "vdi_composite_autotune: arguments");
    if (!workspace || ws_bytes < kWsHeader) return set_error(VDI_ERR_WORKSPACE, "vdi_composite_autotune: workspace");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int* status = reinterpret_cast<unsigned int*>(workspace);
    cudaEvent_t e0, e1;
    vdi_status s = cuda_check(cudaEventCreate(&e0), "event");
    if (s != VDI_OK) return s;
    s = cuda_check(cudaEventCreate(&e1), "event");
    if (s != VDI_OK) { cudaEventDestroy(e0); return s; }
    for (int r = 0; r < n && s == VDI_OK; ++r) {
        vdi_request& q = reqs[r];
        s = check_request(q, r, q.pe ? q.pe[0].prec : 0);
        if (s != VDI_OK) break;
        if (q.schedule != 0) continue;
        const long long key = tune_key(q);
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) { q.schedule = it->second; continue; }
        }
        // time each applicable schedule on up to 2^20 pixels of this request
        const long long npix = (long long)q.w * q.h;
        const int sub = (int)(npix < (1 << 20) ? npix : (1 << 20));
        int best = default_schedule(q.k);
        float best_ms = 3.0e38f;
        const bool staged_fits = ws_bytes >= composite_workspace_bytes(sub, 1);
        for (int sched = 1; sched <= VDI_SCHED_LANE && s == VDI_OK; ++sched) {
            if ((sched == 1 || sched == VDI_SCHED_LANE) && q.k > 8) continue;
            if ((sched == VDI_SCHED_STAGED || sched == VDI_SCHED_LANE) && !staged_fits) continue;
            float ms_min = 3.0e38f;
            for (int rep = 0; rep < 3 && s == VDI_OK; ++rep) {
                s = cuda_check(cudaEventRecord(e0, st), "event record");
                if (s == VDI_OK)
                    s = launch_composite(q.pe, q.k, sub, 1, &q.out, params->bisect_iters, sched, status, workspace,
                                         ws_bytes, st);
                if (s == VDI_OK) s = cuda_check(cudaEventRecord(e1, st), "event record");
                if (s == VDI_OK) s = cuda_check(cudaEventSynchronize(e1), "event sync");
                float ms = 0.f;
                if (s == VDI_OK) s = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
                if (ms < ms_min) ms_min = ms;
            }
            if (ms_min < best_ms) { best_ms = ms_min; best = sched; }
        }
        if (s != VDI_OK) break;
        q.schedule = best;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}

size_t vdi_model_bytes(void) { return model_bytes(); }
int32_t vdi_model_nparams(void) { return model_nparams(); }

vdi_status vdi_model_init(void* model, uint64_t seed, vdi_stream stream) {
    if (!model) return set_error(VDI_ERR_INVALID_ARG, "vdi_model_init: NULL model");
    return launch_model_init(model, seed, (cudaStream_t)stream);
}

vdi_status vdi_model_save(const void* model, const char* path, vdi_stream stream) {
    if (!model || !path) return set_error(VDI_ERR_INVALID_ARG, "vdi_model_save: NULL argument");
    return model_save(model, path, (cudaStream_t)stream);
}

vdi_status vdi_model_load(void* model, const char* path, vdi_stream stream) {
    if (!model || !path) return set_error(VDI_ERR_INVALID_ARG, "vdi_model_load: NULL argument");
    return model_load(model, path, (cudaStream_t)stream);
}

static vdi_status bricks_ok(const char* fn, const vdi_brick* bricks, int k) {
    if (!bricks || k < 1 || k > VDI_MAX_PE) return set_error(VDI_ERR_INVALID_ARG, "%s: bricks / k", fn);
    for (int e = 0; e < k; ++e) {
        const vdi_brick& b = bricks[e];
        if (!b.cells) return set_error(VDI_ERR_INVALID_ARG, "%s: brick %d has no cells", fn, e);
        for (int a = 0; a < 3; ++a)
            if (b.dims[a] != bricks[0].dims[a] || b.dims[a] < 2 || b.owned.lo[a] < 0 ||
                b.owned.hi[a] > b.dims[a] - 1 || b.owned.hi[a] <= b.owned.lo[a])
                return set_error(VDI_ERR_INVALID_ARG, "%s: brick %d box/dims", fn, e);
    }
    return VDI_OK;
}

vdi_status vdi_tile_features(const vdi_brick* bricks, int32_t k, const float* tf_lut, const vdi_camera* cam,
                             int32_t n_s, const vdi_params* params, float* feats, uint8_t* valid, vdi_stream stream) {
    vdi_status s = bricks_ok("vdi_tile_features", bricks, k);
    if (s != VDI_OK) return s;
    if (!tf_lut || !camera_ok(cam) || !params_ok(params) || !feats || !valid || n_s < 1)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_tile_features: arguments");
    BrickDev bd[VDI_MAX_PE];
    for (int e = 0; e < k; ++e) bd[e] = brick_dev(bricks[e]);
    CamDev cd = make_cam(*cam);
    return launch_tile_features(bd, k, tf_lut, cd, bricks[0].dims, (float)(255.0 * (double)bricks[0].value_scale),
                                params->step, params->ref_len, n_s, feats, valid, (cudaStream_t)stream);
}

vdi_status vdi_tile_labels(const vdi_compact* searched, int32_t k, int32_t w, int32_t h, float* labels,
                           uint8_t* valid, vdi_stream stream) {
    if (!searched || k < 1 || k > VDI_MAX_PE || w < 1 || h < 1 || !labels || !valid)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_tile_labels: arguments");
    for (int e = 0; e < k; ++e)
        if (!searched[e].counts || !searched[e].gamma)
            return set_error(VDI_ERR_INVALID_ARG, "vdi_tile_labels: searched[%d] counts/gamma NULL", e);
    return launch_tile_labels(searched, k, w, h, labels, valid, (cudaStream_t)stream);
}

vdi_status vdi_mlp_infer(const void* model, const float* feats, int32_t n, float offset, float* log2_gamma,
                         vdi_stream stream) {
    if (!model || n < 0 || (n > 0 && (!feats || !log2_gamma)))
        return set_error(VDI_ERR_INVALID_ARG, "vdi_mlp_infer: arguments");
    return launch_mlp_infer(model, feats, n, offset, log2_gamma, (cudaStream_t)stream);
}

size_t vdi_mlp_train_workspace(int32_t n) { return n < 0 ? 0 : train_workspace(n); }

vdi_status vdi_mlp_grad(const void* model, const float* feats, const float* labels, const uint8_t* valid, int32_t n,
                        float* grad, float* loss, void* workspace, size_t ws_bytes, vdi_stream stream) {
    if (!model || n < 1 || !feats || !labels || !valid || !grad)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_mlp_grad: arguments");
    if (!workspace || ws_bytes < train_workspace(n)) return set_error(VDI_ERR_WORKSPACE, "vdi_mlp_grad: workspace");
    return launch_mlp_grad(model, feats, labels, valid, n, grad, loss, workspace, (cudaStream_t)stream);
}

vdi_status vdi_mlp_train_step(void* model, const float* feats, const float* labels, const uint8_t* valid, int32_t n,
                              float lr, float* loss, void* workspace, size_t ws_bytes, vdi_stream stream) {
    if (!model || n < 1 || !feats || !labels || !valid || !(lr > 0.f))
        return set_error(VDI_ERR_INVALID_ARG, "vdi_mlp_train_step: arguments");
    if (!workspace || ws_bytes < train_workspace(n))
        return set_error(VDI_ERR_WORKSPACE, "vdi_mlp_train_step: workspace");
    return launch_train_step(model, feats, labels, valid, n, lr, loss, workspace, (cudaStream_t)stream);
}

static size_t learned_extra(int k, int w, int h) {
    size_t tiles = (size_t)((w + VDI_GAMMA_TILE - 1) / VDI_GAMMA_TILE) * ((h + VDI_GAMMA_TILE - 1) / VDI_GAMMA_TILE);
    size_t n = (size_t)k * tiles;
    return align_up(n * VDI_NFEAT * 4, 256) + align_up(n * 4, 256) + align_up(n, 256);
}

size_t vdi_learned_workspace(int32_t k, int32_t w, int32_t h) {
    if (k < 1 || w < 1 || h < 1) return 0;
    return learned_extra(k, w, h) + vdi_generate_workspace(k, w, h);
}

vdi_status vdi_choose_gamma_learned(const vdi_brick* bricks, int32_t k, const float* tf_lut, const vdi_camera* cam,
                                    int32_t n_s, const void* model, float offset, vdi_compact* out,
                                    const vdi_params* params, void* workspace, size_t ws_bytes, vdi_stream stream) {
    if (!model) return set_error(VDI_ERR_MODEL, "vdi_choose_gamma_learned: NULL model");
    if (!cam || cam->width < 1 || cam->height < 1) return set_error(VDI_ERR_INVALID_ARG, "vdi_choose_gamma_learned: camera");
    const size_t extra = learned_extra(k, cam->width, cam->height);
    if (!workspace || ws_bytes < extra) return set_error(VDI_ERR_WORKSPACE, "vdi_choose_gamma_learned: workspace");
    vdi_status s = gen_common("vdi_choose_gamma_learned", bricks, k, tf_lut, cam, n_s, VDI_GAMMA_GIVEN, out, params,
                              static_cast<char*>(workspace) + extra, ws_bytes - extra, false);
    if (s != VDI_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int tiles = ((cam->width + VDI_GAMMA_TILE - 1) / VDI_GAMMA_TILE) *
                      ((cam->height + VDI_GAMMA_TILE - 1) / VDI_GAMMA_TILE);
    const size_t n = (size_t)k * tiles;
    char* ws = static_cast<char*>(workspace);
    float* feats = reinterpret_cast<float*>(ws);
    float* pred = reinterpret_cast<float*>(ws + align_up(n * VDI_NFEAT * 4, 256));
    unsigned char* valid = reinterpret_cast<unsigned char*>(ws + align_up(n * VDI_NFEAT * 4, 256) + align_up(n * 4, 256));
    BrickDev bd[VDI_MAX_PE];
    CompactDev od[VDI_MAX_PE];
    float* gam[VDI_MAX_PE];
    for (int e = 0; e < k; ++e) {
        bd[e] = brick_dev(bricks[e]);
        od[e] = CompactDev{out[e].counts, out[e].offsets, out[e].rgba, out[e].fb, out[e].gamma, out[e].capacity};
        gam[e] = out[e].gamma;
    }
    CamDev cd = make_cam(*cam);
    const float scale255 = (float)(255.0 * (double)bricks[0].value_scale);
    s = launch_tile_features(bd, k, tf_lut, cd, bricks[0].dims, scale255, params->step, params->ref_len, n_s, feats,
                             valid, st);
    if (s != VDI_OK) return s;
    s = launch_mlp_infer(model, feats, (int)n, offset, pred, st);
    if (s != VDI_OK) return s;
    s = launch_gamma_expand(gam, k, cam->width, cam->height, pred, st);
    if (s != VDI_OK) return s;
    char* gws = ws + extra;
    const size_t gbytes = ws_bytes - extra;
    unsigned int* status = reinterpret_cast<unsigned int*>(gws);
    s = cuda_check(cudaMemsetAsync(status, 0, kGenFixed, st), "status clear");
    if (s != VDI_OK) return s;
    const size_t fixed = gen_min_workspace(k, cam->width, cam->height);
    // single pass: the prediction is the ray's gamma unless its count exceeds n_s (then the search);
    // default: the prediction brackets a short search over the cached samples
    const float mode = (params->flags & VDI_FLAG_LEARNED_SINGLE_PASS) ? VDI_GAMMA_GIVEN : kGammaLearnedBracket;
    return launch_gen_count(bd, k, tf_lut, cd, bricks[0].dims, scale255, params->step, params->ref_len, n_s, mode,
                            params->bisect_iters, od, status, (params->flags & VDI_FLAG_CENSUS) != 0,
                            reinterpret_cast<unsigned int*>(gws + kWsHeader), gws + fixed, gbytes - fixed, st);
}

vdi_status vdi_render_view(const vdi_regular* vdi, int32_t w, int32_t h, const vdi_camera* gen,
                           const vdi_camera* view, float* rgba_out, vdi_stream stream) {
    if (!vdi || !rgba_out || !vdi->counts || !vdi->rgba || vdi->n_s < 1)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_render_view: NULL argument");
    if (w < 0 || h < 0) return set_error(VDI_ERR_INVALID_ARG, "vdi_render_view: image size");
    if (!view || (gen && memcmp(view, gen, sizeof(vdi_camera)) == 0))
        return launch_flatten(vdi, w, h, rgba_out, (cudaStream_t)stream);
    if (!gen) return set_error(VDI_ERR_INVALID_ARG, "vdi_render_view: another view needs the generating camera");
    if (gen->width != w || gen->height != h)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_render_view: the VDI is %d x %d, its camera %d x %d", w, h,
                         gen->width, gen->height);
    if (!camera_ok(gen) || !camera_ok(view))
        return set_error(VDI_ERR_INVALID_ARG, "vdi_render_view: camera");
    if (vdi->prec == VDI_PREC_F32 && !vdi->fb) return set_error(VDI_ERR_INVALID_ARG, "vdi_render_view: fb NULL");
    return launch_novel_view(vdi, *gen, *view, rgba_out, (cudaStream_t)stream);
}

}  // extern "C"
