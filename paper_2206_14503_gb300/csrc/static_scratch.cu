// vdi_generate_static_scratch: sub-VDI generation for callers that cannot
// allocate device memory.
//
// vdi_generate needs a caller-allocated workspace: a 256-byte status header
// plus the prefix sum's per-chunk partial sums.  Some callers have no way to
// provide it -- an in-situ simulation that reserves its whole device-memory
// budget at start-up and may not allocate during a time step, or a plugin
// that has no access to its host application's allocator.  This entry point
// uses instead a file-scope static device array of fixed size (every GPU that
// loads the library holds it until the process exits) and calls vdi_generate
// with it; nothing is allocated or freed.
//
// The array's host-side name is not a device address.  A module-scope device
// array has a different address in every CUDA context (a second context on
// the same device, or the primary context re-created after cudaDeviceReset),
// so every call looks the address up with cudaGetSymbolAddress in the
// context current at that call instead of caching it; the lookup is a table
// read in the runtime and allocates nothing.  The first call in a context
// loads the module, which is why that first call belongs before any stream
// capture begins.
#include "vdi_internal.h"

namespace vdi {

// status header, work counter and 65536 partial sums of 8 bytes:
// k * ceil(W*H / 4096) <= 65536, e.g. 64 PEs of 2048 x 2048 pixels or 8 PEs
// of 8192 x 8192.  There is no room for the sample cache, so the gamma search
// re-marches the volume (same result).
constexpr size_t kStaticPartials = 65536;
constexpr size_t kStaticScratchBytes = kGenFixed + kStaticPartials * sizeof(uint64_t);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static vdi_status static_scratch_address(void** out) {
    void* p = nullptr;
    vdi_status s = cuda_check(cudaGetSymbolAddress(&p, g_static_scratch),
                              "vdi_generate_static_scratch: cudaGetSymbolAddress");
    if (s != VDI_OK) return s;
    *out = p;
    return VDI_OK;
}

}  // namespace vdi

using namespace vdi;

extern "C" vdi_status vdi_generate_static_scratch(const vdi_brick* bricks, int32_t k, const float* tf_lut,
                                                  const vdi_camera* cam, int32_t n_s, float gamma, vdi_compact* out,
                                                  const vdi_params* params, vdi_stream stream) {
    if (!cam || !params) return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_static_scratch: NULL argument");
    if (k < 1 || k > VDI_MAX_PE) return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_static_scratch: k = %d", k);
    if (cam->width < 1 || cam->height < 1)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_static_scratch: image %d x %d", cam->width, cam->height);
    const size_t npix = (size_t)cam->width * (size_t)cam->height;
    const size_t chunks = (npix + 4095) / 4096;
    if ((size_t)k * chunks > kStaticPartials)
        return set_error(VDI_ERR_INVALID_ARG,
                         "vdi_generate_static_scratch: %d PEs x %zu pixels exceed the static scratch "
                         "(k * ceil(W*H / 4096) must be <= %zu); use vdi_generate with a workspace",
                         k, npix, kStaticPartials);
    if (kGenFixed + (size_t)k * chunks * sizeof(uint64_t) > kStaticScratchBytes)
        return set_error(VDI_ERR_INVALID_ARG, "vdi_generate_static_scratch: request exceeds the static scratch");
    void* scratch = nullptr;
    vdi_status s = static_scratch_address(&scratch);
    if (s != VDI_OK) return s;
    vdi_params p = *params;
    p.flags |= VDI_FLAG_SYNC_CAPACITY;  // the caller cannot read the status word: report capacity by return
    s = vdi_generate(bricks, k, tf_lut, cam, n_s, gamma, out, &p, scratch, kStaticScratchBytes, stream);
    if (s != VDI_OK) return s;
    // errors the kernels detect land in the status word at the start of the array, which the caller
    // cannot reach: read it back here and return it
    unsigned int word = 0;
    cudaStream_t st = (cudaStream_t)stream;
    s = cuda_check(cudaMemcpyAsync(&word, scratch, sizeof word, cudaMemcpyDeviceToHost, st),
                   "vdi_generate_static_scratch: status read");
    if (s != VDI_OK) return s;
    s = cuda_check(cudaStreamSynchronize(st), "vdi_generate_static_scratch: status sync");
    if (s != VDI_OK) return s;
    if (word != 0)
        return set_error((vdi_status)word, "vdi_generate_static_scratch: device reported: %s",
                         vdi_status_string((vdi_status)word));
    return VDI_OK;
}
