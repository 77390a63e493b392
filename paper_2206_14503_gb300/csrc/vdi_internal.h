// Internal structures passed by value to the kernels, and host-side helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vdi.h"

namespace vdi {

// Camera basis as unevaluated pairs of floats (hi + lo, |lo| <= ulp(hi)/2):
// computed on the host in double and split, so the device sets rays up in
// double-float arithmetic without FP64 instructions.
struct CamDev {
    float eye[3][2];
    float fwd[3][2], right[3][2], up[3][2];
    float sx[2], sy[2];  // tan(fovy/2) * W/H, tan(fovy/2)
    int W, H;
};

// Non-convex ownership (sec. 5.3): the PE of each block of 2^shift cells per
// axis, x fastest, nb[] blocks per axis; map == nullptr means box ownership.
struct OwnerDev {
    const uint8_t* map;
    int shift;
    int nb[3];
};

// One PE's sampling brick: cells [lo-1, hi+1) per axis (a one-cell border),
// 8 corner values per cell as two float4 (v000 v100 v010 v110 | v001 v101 v011 v111).
struct BrickDev {
    const float* cells;
    int lo[3], hi[3];
    int nx, ny, nz;  // padded cell counts
    int ncells;
};

struct CompactDev {
    uint32_t* counts;
    uint64_t* offsets;
    void* rgba;
    float* fb;
    float* gamma;
    uint64_t capacity;
};

// Status word layout in the caller's workspace (first 256 bytes).
struct WsHeader {
    unsigned int status;  // vdi_status of the first device-side error
    unsigned int pad;
    unsigned long long counters[8];  // census (VDI_FLAG_CENSUS)
    unsigned long long pad2[23];
};
static_assert(sizeof(WsHeader) == 256, "workspace header is 256 bytes");
constexpr size_t kWsHeader = 256;

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// One list of a batched prefix sum: counts[0..n) -> offsets[0..n], its chunks
// of the partial sums starting at chunk_begin.
struct ScanList {
    const uint32_t* counts;
    uint64_t* offsets;
    int n;
    uint32_t chunk_begin;
};

// host helpers (api.cu)
CamDev make_cam(const vdi_camera& c);
BrickDev brick_dev(const vdi_brick& b);
vdi_status set_error(vdi_status s, const char* fmt, ...);
vdi_status cuda_check(cudaError_t e, const char* what);

// kernel launchers (one per .cu file)
vdi_status launch_brick_build(const void* volume, int type, const int dims[3], int k, const vdi_box* boxes,
                              float* const* cells, cudaStream_t st);
vdi_status launch_gen_count(const BrickDev* bricks, int k, const float* lut, const CamDev& cam, const int dims[3],
                            float scale255, float step, float ref_len, int n_s, float gamma, int iters,
                            const CompactDev* out, unsigned int* status, bool census, unsigned int* counter,
                            void* cache, size_t cache_bytes, cudaStream_t st, const OwnerDev* own = nullptr);
vdi_status gen_count_grid(int& ctas);
size_t gen_cache_bytes(int ctas);
size_t gen_span_bytes(int k, int w, int h);
// generation workspace: [0, 256) header, [256, 512) work counter, then the
// prefix sum's partial sums, then (optionally) the sample cache, the recorded
// spans (one uint2 per (PE, pixel)) and their 8-byte tag (a 256-byte slot)
constexpr size_t kGenFixed = 512;
// internal gamma mode of launch_gen_count: per-ray predicted gamma in out.gamma,
// refined by a short bracketed search over the sample cache (learned path)
constexpr float kGammaLearnedBracket = -5.0f;
vdi_status launch_gen_emit(const BrickDev* bricks, int k, const float* lut, const CamDev& cam, const int dims[3],
                           float scale255, float step, float ref_len, int n_s, int prec, const CompactDev* out,
                           unsigned int* status, cudaStream_t st, bool regular = false,
                           const OwnerDev* own = nullptr, void* cache = nullptr, size_t cache_bytes = 0);
size_t scan_workspace(int k, int n);
vdi_status launch_scan(int k, int n, uint32_t* const* counts, uint64_t* const* offsets, void* ws, cudaStream_t st);
uint32_t scan_chunks(int n);
vdi_status launch_scan_batched(const ScanList* dev_lists, int nlists, uint32_t total_chunks, uint64_t* partial,
                               cudaStream_t st);
// batched generation (generate.cu): host table of uneven requests, its workspace, the launches
size_t gen_batch_table_bytes(const vdi_gen_request* reqs, int n);
vdi_status gen_batch_table_pack(const vdi_gen_request* reqs, int n, const vdi_params* params, void* host_table,
                                size_t bytes);
size_t gen_batched_workspace_bytes(const void* host_table);
vdi_status launch_gen_batched(const void* dev_table, const void* host_table, void* workspace, size_t ws_bytes,
                              cudaStream_t st);

vdi_status launch_composite(const vdi_compact* pe, int k, int w, int h, const vdi_regular* out, int iters,
                            int schedule, unsigned int* status, void* workspace, size_t ws_bytes, cudaStream_t st,
                            bool census = false);
int default_schedule(int k);
size_t composite_workspace_bytes(int w, int h);
size_t batch_table_bytes(const vdi_request* reqs, int n);
vdi_status batch_table_pack(const vdi_request* reqs, int n, void* host_table, size_t bytes);
size_t batched_workspace_bytes(const void* host_table);
vdi_status launch_composite_batched(const void* dev_table, const void* host_table, int iters, unsigned int* status,
                                    void* workspace, size_t ws_bytes, cudaStream_t st);
vdi_status launch_flatten(const vdi_regular* v, int w, int h, float* rgba, cudaStream_t st);
vdi_status launch_novel_view(const vdi_regular* v, const vdi_camera& gen, const vdi_camera& view, float* rgba,
                             cudaStream_t st);

// learned gamma (learned.cu)
size_t model_bytes();
int model_nparams();
vdi_status launch_model_init(void* model, unsigned long long seed, cudaStream_t st);
vdi_status launch_tile_features(const BrickDev* bricks, int k, const float* lut, const CamDev& cam, const int dims[3],
                                float scale255, float step, float ref_len, int n_s, float* feats,
                                unsigned char* valid, cudaStream_t st);
vdi_status launch_tile_labels(const vdi_compact* searched, int k, int w, int h, float* labels, unsigned char* valid,
                              cudaStream_t st);
vdi_status launch_mlp_infer(const void* model, const float* feats, int n, float offset, float* out, cudaStream_t st);
vdi_status launch_gamma_expand(float* const* gammas, int k, int w, int h, const float* pred, cudaStream_t st);
size_t train_workspace(int n);
vdi_status launch_mlp_grad(const void* model, const float* x, const float* y, const unsigned char* valid, int n,
                           float* grad, float* loss, void* ws, cudaStream_t st);
vdi_status launch_train_step(void* model, const float* x, const float* y, const unsigned char* valid, int n, float lr,
                             float* loss, void* ws, cudaStream_t st);
vdi_status model_save(const void* model, const char* path, cudaStream_t st);
vdi_status model_load(void* model, const char* path, cudaStream_t st);

}  // namespace vdi
