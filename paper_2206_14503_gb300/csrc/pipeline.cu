// Frame pipeline: sub-VDI generation of one frame overlaps the download of the
// previous frame's composited VDI and the upload of the next frame's volume.
// The paper overlaps sub-VDI generation with the final gather of the previous
// VDI (sec. 7); on one GPU that gather is the device-to-host copy of the
// regular VDI, so the overlap is between the copy engines and the SMs.
//
// Three streams per pipeline: copy-in (volume uploads), compute (brick build,
// generation, compositing, a snapshot of the status words), copy-out
// (regular-VDI downloads and the status read-back), ordered by events.  The
// volume and the regular VDI are double-buffered; the bricks, the sub-VDIs
// and the workspaces are used by the compute stream alone, so one copy of
// each suffices.  A submission first waits on the host for the frame two
// back, which frees its buffers: at most two frames are in flight and no
// device-side wait spans more than one frame.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "vdi_internal.h"

using vdi::cuda_check;
using vdi::set_error;

namespace {

constexpr int kDepth = 2;

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of every buffer in the caller's arena.
struct Layout {
    size_t vol[kDepth];
    size_t cells[VDI_MAX_PE];
    size_t lut;
    size_t sub_counts[VDI_MAX_PE], sub_offsets[VDI_MAX_PE], sub_gamma[VDI_MAX_PE];
    size_t sub_rgba[VDI_MAX_PE], sub_fb[VDI_MAX_PE];
    size_t reg_counts[kDepth], reg_gamma[kDepth], reg_rgba[kDepth], reg_fb[kDepth];
    size_t wsg, wsg_bytes, wsc, wsc_bytes;
    size_t status[kDepth];  // a frame's two status words, copied there by the compute stream
    size_t vol_bytes;
    uint64_t capacity;
    size_t total;
};

bool box_ok(const vdi_box& b, const int32_t dims[3]) {
    for (int a = 0; a < 3; ++a)
        if (b.lo[a] < 0 || b.hi[a] > dims[a] - 1 || b.hi[a] <= b.lo[a]) return false;
    return true;
}

// Checks the description and lays out the arena; false (with the error set)
// for an invalid description.
bool plan(const vdi_pipeline_desc* d, Layout& L) {
    if (!d) {
        set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline: NULL description");
        return false;
    }
    for (int a = 0; a < 3; ++a)
        if (d->dims[a] < 2) {
            set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline: dims[%d] = %d", a, d->dims[a]);
            return false;
        }
    if (d->type != VDI_VOL_F32 && d->type != VDI_VOL_U16) {
        set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline: volume type %d", d->type);
        return false;
    }
    if (d->k < 1 || d->k > VDI_MAX_PE) {
        set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline: k = %d", d->k);
        return false;
    }
    for (int e = 0; e < d->k; ++e)
        if (!box_ok(d->boxes[e], d->dims)) {
            set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline: box %d", e);
            return false;
        }
    if (d->width < 1 || d->height < 1 || (long long)d->width * d->height > (long long)INT32_MAX / 2) {
        set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline: image %d x %d", d->width, d->height);
        return false;
    }
    if (d->n_s < 1 || (d->prec != VDI_PREC_F32 && d->prec != VDI_PREC_F16)) {
        set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline: n_s %d / prec %d", d->n_s, d->prec);
        return false;
    }
    if (!(d->gamma >= 0.f || d->gamma == VDI_GAMMA_SEARCH) || std::isinf(d->gamma)) {
        set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline: gamma %g", (double)d->gamma);
        return false;
    }
    const vdi_params& p = d->params;
    if (!(p.step > 0.f) || !(p.ref_len > 0.f) || p.bisect_iters < 1 || p.bisect_iters > 24 || p.schedule < 0 ||
        p.schedule > VDI_SCHED_LANE) {
        set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline: params");
        return false;
    }
    const size_t npix = (size_t)d->width * (size_t)d->height;
    L.capacity = d->capacity ? d->capacity : (uint64_t)npix * (uint64_t)d->n_s;
    const size_t slots = npix * (size_t)d->n_s;
    L.vol_bytes = (size_t)d->dims[0] * d->dims[1] * d->dims[2] * (d->type == VDI_VOL_F32 ? 4 : 2);
    size_t at = 0;
    auto take = [&](size_t bytes) {
        const size_t o = at;
        at = round256(at + bytes);
        return o;
    };
    for (int s = 0; s < kDepth; ++s) L.vol[s] = take(L.vol_bytes);
    for (int e = 0; e < d->k; ++e) L.cells[e] = take(vdi_brick_bytes(&d->boxes[e]));
    L.lut = take(256 * 4 * sizeof(float));
    for (int e = 0; e < d->k; ++e) {
        L.sub_counts[e] = take(npix * 4);
        L.sub_offsets[e] = take((npix + 1) * 8);
        L.sub_gamma[e] = take(npix * 4);
        L.sub_rgba[e] = take((size_t)L.capacity * 16);
        L.sub_fb[e] = d->prec == VDI_PREC_F32 ? take((size_t)L.capacity * 8) : 0;
    }
    for (int s = 0; s < kDepth; ++s) {
        L.reg_counts[s] = take(npix * 4);
        L.reg_gamma[s] = take(npix * 4);
        L.reg_rgba[s] = take(slots * 16);
        L.reg_fb[s] = d->prec == VDI_PREC_F32 ? take(slots * 8) : 0;
    }
    L.wsg_bytes = vdi_generate_workspace(d->k, d->width, d->height);
    L.wsg = take(L.wsg_bytes);
    L.wsc_bytes = vdi_composite_workspace(d->k, d->width, d->height, d->n_s);
    L.wsc = take(L.wsc_bytes);
    for (int s = 0; s < kDepth; ++s) L.status[s] = take(2 * sizeof(unsigned int));
    L.total = at;
    return true;
}

// The status words of a frame's generation and compositing workspaces into the slot's snapshot.  A
// kernel, not a copy: a device-to-host copy on the compute stream would queue on the copy engine behind
// the previous frame's download and hold the compute stream until it ends.
__global__ void status_snapshot_kernel(const unsigned int* gen, const unsigned int* comp, unsigned int* dst) {
    if (threadIdx.x == 0) {
        dst[0] = *gen;
        dst[1] = *comp;
    }
}

}  // namespace

struct vdi_pipeline {
    vdi_pipeline_desc d;
    Layout L;
    char* arena = nullptr;
    int device = 0;
    cudaStream_t st[3] = {nullptr, nullptr, nullptr};  // copy-in, compute, copy-out
    cudaEvent_t vol_ready[kDepth] = {}, reg_ready[kDepth] = {}, done[kDepth] = {};
    unsigned int* mirror = nullptr;  // page-locked, 2 status words per slot
    float* cells[VDI_MAX_PE] = {};
    vdi_brick bricks[VDI_MAX_PE] = {};
    vdi_compact sub[VDI_MAX_PE] = {};
    vdi_regular reg[kDepth] = {};
    vdi_params params;
    bool tuned = false;
    uint64_t submitted = 0;  // frames submitted
    uint64_t harvested = 0;  // frames whose status was collected
    vdi_status host_err[kDepth] = {VDI_OK, VDI_OK};  // errors met while enqueuing the slot's frame
    vdi_status slot_status[kDepth] = {VDI_OK, VDI_OK};
    uint64_t slot_ticket[kDepth] = {~0ull, ~0ull};
    vdi_status sticky = VDI_OK;  // first error of any harvested frame
};

namespace {

// Makes the pipeline's device current for the scope of a call.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Waits for frame t (t == pl->harvested) and records its status.
vdi_status harvest(vdi_pipeline* pl, uint64_t t) {
    const int s = (int)(t % kDepth);
    vdi_status r = pl->host_err[s];
    vdi_status c = cuda_check(cudaEventSynchronize(pl->done[s]), "vdi_pipeline: frame wait");
    if (r == VDI_OK) r = c;
    if (r == VDI_OK) {
        for (int w = 0; w < 2 && r == VDI_OK; ++w) {
            const unsigned int v = pl->mirror[2 * s + w];
            if (v != 0) r = set_error((vdi_status)v, "vdi_pipeline: frame %llu: %s", (unsigned long long)t,
                                      vdi_status_string((vdi_status)v));
        }
    }
    pl->slot_status[s] = r;
    pl->slot_ticket[s] = t;
    if (r != VDI_OK && pl->sticky == VDI_OK) pl->sticky = r;
    pl->harvested = t + 1;
    return r;
}

void release(vdi_pipeline* pl) {
    for (int s = 0; s < kDepth; ++s) {
        if (pl->vol_ready[s]) cudaEventDestroy(pl->vol_ready[s]);
        if (pl->reg_ready[s]) cudaEventDestroy(pl->reg_ready[s]);
        if (pl->done[s]) cudaEventDestroy(pl->done[s]);
    }
    for (int i = 0; i < 3; ++i)
        if (pl->st[i]) cudaStreamDestroy(pl->st[i]);
    if (pl->mirror) cudaFreeHost(pl->mirror);
    delete pl;
}

}  // namespace

size_t vdi_pipeline_arena_bytes(const vdi_pipeline_desc* desc) {
    Layout L;
    return plan(desc, L) ? L.total : 0;
}

vdi_status vdi_pipeline_create(const vdi_pipeline_desc* desc, void* arena, size_t arena_bytes, const float* tf_lut,
                               vdi_pipeline** out) {
    if (!out || !arena || !tf_lut) return set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline_create: NULL argument");
    *out = nullptr;
    Layout L;
    if (!plan(desc, L)) return VDI_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(arena) & 255)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline_create: arena not 256-byte aligned");
    if (arena_bytes < L.total)
        return set_error(VDI_ERR_WORKSPACE, "vdi_pipeline_create: arena %zu < %zu bytes", arena_bytes, L.total);
    vdi_pipeline* pl = new (std::nothrow) vdi_pipeline;
    if (!pl) return set_error(VDI_ERR_CUDA, "vdi_pipeline_create: out of host memory");
    pl->d = *desc;
    pl->L = L;
    pl->arena = static_cast<char*>(arena);
    pl->params = desc->params;
    pl->tuned = desc->params.schedule != 0;
    vdi_status s = cuda_check(cudaGetDevice(&pl->device), "vdi_pipeline_create: device");
    for (int i = 0; i < 3 && s == VDI_OK; ++i)
        s = cuda_check(cudaStreamCreateWithFlags(&pl->st[i], cudaStreamNonBlocking), "vdi_pipeline_create: stream");
    for (int q = 0; q < kDepth && s == VDI_OK; ++q) {
        s = cuda_check(cudaEventCreateWithFlags(&pl->vol_ready[q], cudaEventDisableTiming), "event");
        if (s == VDI_OK) s = cuda_check(cudaEventCreateWithFlags(&pl->reg_ready[q], cudaEventDisableTiming), "event");
        if (s == VDI_OK) s = cuda_check(cudaEventCreateWithFlags(&pl->done[q], cudaEventDisableTiming), "event");
    }
    if (s == VDI_OK)
        s = cuda_check(cudaHostAlloc(reinterpret_cast<void**>(&pl->mirror), 2 * kDepth * sizeof(unsigned int),
                                     cudaHostAllocDefault),
                       "vdi_pipeline_create: status mirror");
    if (s == VDI_OK) std::memset(pl->mirror, 0, 2 * kDepth * sizeof(unsigned int));
    // the table is copied once, ordered after the caller's work on the device
    float* lut = reinterpret_cast<float*>(pl->arena + L.lut);
    if (s == VDI_OK) s = cuda_check(cudaDeviceSynchronize(), "vdi_pipeline_create: sync");
    if (s == VDI_OK)
        s = cuda_check(cudaMemcpyAsync(lut, tf_lut, 256 * 4 * sizeof(float), cudaMemcpyDeviceToDevice, pl->st[1]),
                       "vdi_pipeline_create: table copy");
    if (s == VDI_OK) s = cuda_check(cudaStreamSynchronize(pl->st[1]), "vdi_pipeline_create: sync");
    if (s != VDI_OK) {
        release(pl);
        return s;
    }
    char* a = pl->arena;
    const vdi_pipeline_desc& d = pl->d;
    for (int e = 0; e < d.k; ++e) {
        pl->cells[e] = reinterpret_cast<float*>(a + L.cells[e]);
        pl->sub[e] = vdi_compact{reinterpret_cast<uint32_t*>(a + L.sub_counts[e]),
                                 reinterpret_cast<uint64_t*>(a + L.sub_offsets[e]), a + L.sub_rgba[e],
                                 d.prec == VDI_PREC_F32 ? reinterpret_cast<float*>(a + L.sub_fb[e]) : nullptr,
                                 reinterpret_cast<float*>(a + L.sub_gamma[e]), L.capacity, d.prec};
    }
    for (int q = 0; q < kDepth; ++q)
        pl->reg[q] = vdi_regular{reinterpret_cast<uint32_t*>(a + L.reg_counts[q]), a + L.reg_rgba[q],
                                 d.prec == VDI_PREC_F32 ? reinterpret_cast<float*>(a + L.reg_fb[q]) : nullptr,
                                 reinterpret_cast<float*>(a + L.reg_gamma[q]), d.n_s, d.prec};
    *out = pl;
    return VDI_OK;
}

vdi_status vdi_pipeline_submit(vdi_pipeline* pl, const void* volume, const vdi_camera* cam, const vdi_regular* dst,
                               uint64_t* ticket) {
    if (!pl || !cam || !dst || !ticket) return set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline_submit: NULL argument");
    const vdi_pipeline_desc& d = pl->d;
    const Layout& L = pl->L;
    if (cam->width != d.width || cam->height != d.height)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline_submit: camera %d x %d, pipeline %d x %d", cam->width,
                         cam->height, d.width, d.height);
    if (!dst->counts || !dst->rgba || (d.prec == VDI_PREC_F32 && !dst->fb) || dst->n_s != d.n_s ||
        dst->prec != d.prec)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline_submit: destination buffers / n_s / prec");
    if (!volume && pl->submitted == 0)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline_submit: the first frame needs a volume");
    DeviceScope scope(pl->device);
    const uint64_t f = pl->submitted;
    const int s = (int)(f % kDepth);
    // the frame two back frees this slot's volume, regular VDI and status words
    while (f >= (uint64_t)kDepth && pl->harvested <= f - kDepth) harvest(pl, pl->harvested);
    const cudaStream_t cin = pl->st[0], comp = pl->st[1], cout = pl->st[2];
    char* a = pl->arena;
    const size_t npix = (size_t)d.width * (size_t)d.height;
    const size_t slots = npix * (size_t)d.n_s;
    vdi_status r = VDI_OK;
    if (volume) {
        void* vd = a + L.vol[s];
        r = cuda_check(cudaMemcpyAsync(vd, volume, L.vol_bytes, cudaMemcpyHostToDevice, cin), "volume upload");
        if (r == VDI_OK) r = cuda_check(cudaEventRecord(pl->vol_ready[s], cin), "event record");
        if (r == VDI_OK) r = cuda_check(cudaStreamWaitEvent(comp, pl->vol_ready[s], 0), "event wait");
        if (r == VDI_OK)
            r = vdi_brick_build(vd, (vdi_voltype)d.type, d.dims, d.k, d.boxes, pl->cells, pl->bricks,
                                (vdi_stream)comp);
    }
    const float* lut = reinterpret_cast<const float*>(a + L.lut);
    if (r == VDI_OK)
        r = vdi_generate(pl->bricks, d.k, lut, cam, d.n_s, d.gamma, pl->sub, &pl->params, a + L.wsg, L.wsg_bytes,
                         (vdi_stream)comp);
    if (r == VDI_OK && !pl->tuned) {
        // schedule 0: the autotuner picks the compositing schedule on the first frame (synchronises)
        vdi_request q{};
        q.pe = pl->sub;
        q.k = d.k;
        q.w = d.width;
        q.h = d.height;
        q.out = pl->reg[s];
        q.schedule = 0;
        r = vdi_composite_autotune(&q, 1, &pl->params, a + L.wsc, L.wsc_bytes, (vdi_stream)comp);
        if (r == VDI_OK) {
            pl->params.schedule = q.schedule;
            pl->tuned = true;
        }
    }
    if (r == VDI_OK)
        r = vdi_composite(pl->sub, d.k, d.width, d.height, &pl->reg[s], &pl->params, a + L.wsc, L.wsc_bytes,
                          (vdi_stream)comp);
    // the status words this frame's kernels left, kept in the slot before the next frame clears them;
    // the copy-out stream reads them back after the download
    unsigned int* snap = reinterpret_cast<unsigned int*>(a + L.status[s]);
    if (r == VDI_OK) {
        status_snapshot_kernel<<<1, 32, 0, comp>>>(reinterpret_cast<const unsigned int*>(a + L.wsg),
                                                   reinterpret_cast<const unsigned int*>(a + L.wsc), snap);
        r = cuda_check(cudaGetLastError(), "status snapshot");
    }
    // the completion events are recorded even after an error, so that waiting for the frame
    // waits for whatever part of it was enqueued
    vdi_status r2 = cuda_check(cudaEventRecord(pl->reg_ready[s], comp), "event record");
    if (r2 == VDI_OK) r2 = cuda_check(cudaStreamWaitEvent(cout, pl->reg_ready[s], 0), "event wait");
    if (r == VDI_OK && r2 == VDI_OK) {
        const vdi_regular& g = pl->reg[s];
        r = cuda_check(cudaMemcpyAsync(dst->counts, g.counts, npix * 4, cudaMemcpyDeviceToHost, cout), "download");
        if (r == VDI_OK)
            r = cuda_check(cudaMemcpyAsync(dst->rgba, g.rgba, slots * 16, cudaMemcpyDeviceToHost, cout), "download");
        if (r == VDI_OK && d.prec == VDI_PREC_F32)
            r = cuda_check(cudaMemcpyAsync(dst->fb, g.fb, slots * 8, cudaMemcpyDeviceToHost, cout), "download");
        if (r == VDI_OK && dst->gamma)
            r = cuda_check(cudaMemcpyAsync(dst->gamma, g.gamma, npix * 4, cudaMemcpyDeviceToHost, cout), "download");
        if (r == VDI_OK)
            r = cuda_check(cudaMemcpyAsync(pl->mirror + 2 * s, snap, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost,
                                           cout),
                           "status read");
    }
    vdi_status r3 = cuda_check(cudaEventRecord(pl->done[s], cout), "event record");
    if (r == VDI_OK) r = r2;
    if (r == VDI_OK) r = r3;
    pl->host_err[s] = r;
    *ticket = f;
    pl->submitted = f + 1;
    return r;
}

vdi_status vdi_pipeline_wait(vdi_pipeline* pl, uint64_t ticket) {
    if (!pl) return set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline_wait: NULL pipeline");
    if (ticket >= pl->submitted)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline_wait: frame %llu not submitted",
                         (unsigned long long)ticket);
    DeviceScope scope(pl->device);
    while (pl->harvested <= ticket) harvest(pl, pl->harvested);
    const int s = (int)(ticket % kDepth);
    return pl->slot_ticket[s] == ticket ? pl->slot_status[s] : pl->sticky;
}

vdi_status vdi_pipeline_streams(const vdi_pipeline* pl, vdi_stream streams[3]) {
    if (!pl || !streams) return set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline_streams: NULL argument");
    for (int i = 0; i < 3; ++i) streams[i] = (vdi_stream)pl->st[i];
    return VDI_OK;
}

vdi_status vdi_pipeline_destroy(vdi_pipeline* pl) {
    if (!pl) return set_error(VDI_ERR_INVALID_ARG, "vdi_pipeline_destroy: NULL pipeline");
    {
        DeviceScope scope(pl->device);
        while (pl->harvested < pl->submitted) harvest(pl, pl->harvested);
        release(pl);
    }
    return VDI_OK;
}
