// Sampling bricks (decomposition of sec. 3): each PE's cells, padded by one
// cell on every side, in a cell-packed layout -- the 8 corner node values of a
// cell stored together (32 bytes) so that one trilinear sample is one pair of
// 16-byte loads.  Node coordinates outside the volume are clamped to its faces,
// which reproduces clamped trilinear interpolation at the volume's boundary.
#include "vdi_internal.h"

namespace vdi {

struct BrickBuildArgs {
    const void* vol;
    int type;  // vdi_voltype
    int dims[3];
    int k;
    int lo[VDI_MAX_PE][3];
    int n[VDI_MAX_PE][3];  // padded cell counts
    float* cells[VDI_MAX_PE];
};

__device__ __forceinline__ float node_value(const BrickBuildArgs& a, int x, int y, int z) {
    x = min(max(x, 0), a.dims[0] - 1);
    y = min(max(y, 0), a.dims[1] - 1);
    z = min(max(z, 0), a.dims[2] - 1);
    size_t i = ((size_t)z * a.dims[1] + y) * a.dims[0] + x;
    if (a.type == VDI_VOL_U16) return (float)__ldg(reinterpret_cast<const unsigned short*>(a.vol) + i);
    return __ldg(reinterpret_cast<const float*>(a.vol) + i);
}

// A brick holds fewer than 2^31 cells (vdi_brick_build checks), so cell indices
// and the grid stride fit 32-bit unsigned arithmetic (64-bit division per cell
// was a large part of this HBM-bound kernel's instructions).
__global__ void brick_build_kernel(const __grid_constant__ BrickBuildArgs a) {
    int e = blockIdx.y;
    const unsigned nx = (unsigned)a.n[e][0], ny = (unsigned)a.n[e][1], nz = (unsigned)a.n[e][2];
    const unsigned total = nx * ny * nz;
    float4* out = reinterpret_cast<float4*>(a.cells[e]);
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const unsigned row = idx / nx;
        int lx = (int)(idx - row * nx);
        int ly = (int)(row % ny);
        int lz = (int)(row / ny);
        int x = a.lo[e][0] - 1 + lx, y = a.lo[e][1] - 1 + ly, z = a.lo[e][2] - 1 + lz;
        float4 lo = make_float4(node_value(a, x, y, z), node_value(a, x + 1, y, z), node_value(a, x, y + 1, z),
                                node_value(a, x + 1, y + 1, z));
        float4 hi = make_float4(node_value(a, x, y, z + 1), node_value(a, x + 1, y, z + 1),
                                node_value(a, x, y + 1, z + 1), node_value(a, x + 1, y + 1, z + 1));
        out[2 * (size_t)idx] = lo;
        out[2 * (size_t)idx + 1] = hi;
    }
}

vdi_status launch_brick_build(const void* volume, int type, const int dims[3], int k, const vdi_box* boxes,
                              float* const* cells, cudaStream_t st) {
    BrickBuildArgs a;
    a.vol = volume;
    a.type = type;
    for (int i = 0; i < 3; ++i) a.dims[i] = dims[i];
    a.k = k;
    size_t maxcells = 0;
    for (int e = 0; e < k; ++e) {
        size_t c = 1;
        for (int i = 0; i < 3; ++i) {
            a.lo[e][i] = boxes[e].lo[i];
            a.n[e][i] = boxes[e].hi[i] - boxes[e].lo[i] + 2;
            c *= (size_t)a.n[e][i];
        }
        a.cells[e] = cells[e];
        if (c > maxcells) maxcells = c;
    }
    int threads = 256;
    size_t blocks = (maxcells + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    dim3 grid((unsigned)blocks, (unsigned)k);
    brick_build_kernel<<<grid, threads, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "brick_build_kernel launch");
}

}  // namespace vdi
