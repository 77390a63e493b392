// Rendering a regular VDI from its generating viewpoint: front-to-back "over"
// of each pixel's supersegments, which reproduces the volume rendering exactly
// by associativity of "over" (sec. 2.3).
#include <cuda_fp16.h>

#include "vdi_internal.h"

namespace vdi {

__global__ void flatten_kernel(const uint32_t* __restrict__ counts, const void* __restrict__ rgba, int n_s,
                               int prec, int npix, float4* __restrict__ out) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    uint32_t n = counts[p];
    if (n > (uint32_t)n_s) n = (uint32_t)n_s;
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
    for (uint32_t j = 0; j < n; ++j) {
        size_t idx = (size_t)p * n_s + j;
        float4 c;
        if (prec == VDI_PREC_F32) {
            c = __ldg(reinterpret_cast<const float4*>(rgba) + idx);
        } else {
            uint4 v = __ldg(reinterpret_cast<const uint4*>(rgba) + idx);
            float2 rg = __half22float2(*reinterpret_cast<__half2*>(&v.z));
            float2 ba = __half22float2(*reinterpret_cast<__half2*>(&v.w));
            c = make_float4(rg.x, rg.y, ba.x, ba.y);
        }
        float T = 1.f - A;
        C0 = fmaf(T, c.x, C0);
        C1 = fmaf(T, c.y, C1);
        C2 = fmaf(T, c.z, C2);
        A = fmaf(T, c.w, A);
    }
    out[p] = make_float4(C0, C1, C2, A);
}

vdi_status launch_flatten(const vdi_regular* v, int w, int h, float* rgba, cudaStream_t st) {
    int npix = w * h;
    if (npix == 0) return VDI_OK;
    int threads = 256;
    flatten_kernel<<<(npix + threads - 1) / threads, threads, 0, st>>>(v->counts, v->rgba, v->n_s, v->prec, npix,
                                                                     reinterpret_cast<float4*>(rgba));
    return cuda_check(cudaGetLastError(), "flatten_kernel launch");
}

}  // namespace vdi
