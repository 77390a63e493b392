// Exclusive prefix sum of the per-ray supersegment counts into 64-bit offsets
// (compact layout, sec. 4, Fig. 2b), for K PEs in one set of launches.  The
// paper computes it on the CPU; here it stays on the device so that
// generation needs no host round trip.
//
// Reduce-then-scan in three launches over chunks of 4096 counts: chunk sums,
// a scan of the chunk sums per PE (one CTA per PE), and a chunk-local scan
// plus the chunk's prefix.  Scratch: K x chunks 64-bit partial sums.
#include "vdi_internal.h"

namespace vdi {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

struct ScanArgs {
    const uint32_t* counts[VDI_MAX_PE];
    uint64_t* offsets[VDI_MAX_PE];
    uint64_t* partial;  // [k][chunks]
    int n, chunks;
};

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t& total) {
    __shared__ uint64_t warp_sums[kScanThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    uint64_t before = warp > 0 ? warp_sums[warp - 1] : 0;
    total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__device__ __forceinline__ void load_items(const uint32_t* c, int n, size_t base, uint32_t it[kScanItems]) {
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        size_t i = base + q;
        it[q] = i < (size_t)n ? __ldg(c + i) : 0u;
    }
}

__global__ void scan_reduce_kernel(const __grid_constant__ ScanArgs a) {
    int e = blockIdx.y, chunk = blockIdx.x;
    size_t base = (size_t)chunk * kScanChunk + (size_t)threadIdx.x * kScanItems;
    uint32_t it[kScanItems];
    load_items(a.counts[e], a.n, base, it);
    uint64_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) s += it[q];
    uint64_t total;
    block_exclusive_scan(s, total);
    if (threadIdx.x == 0) a.partial[(size_t)e * a.chunks + chunk] = total;
}

__global__ void scan_partials_kernel(const __grid_constant__ ScanArgs a) {
    int e = blockIdx.x;
    uint64_t* p = a.partial + (size_t)e * a.chunks;
    uint64_t carry = 0;
    for (int start = 0; start < a.chunks; start += kScanThreads) {
        int i = start + threadIdx.x;
        uint64_t v = i < a.chunks ? p[i] : 0;
        uint64_t total;
        uint64_t ex = block_exclusive_scan(v, total);
        if (i < a.chunks) p[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) a.offsets[e][a.n] = carry;
}

__global__ void scan_down_kernel(const __grid_constant__ ScanArgs a) {
    int e = blockIdx.y, chunk = blockIdx.x;
    size_t base = (size_t)chunk * kScanChunk + (size_t)threadIdx.x * kScanItems;
    uint32_t it[kScanItems];
    load_items(a.counts[e], a.n, base, it);
    uint64_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) s += it[q];
    uint64_t total;
    uint64_t ex = block_exclusive_scan(s, total) + a.partial[(size_t)e * a.chunks + chunk];
    uint64_t* out = a.offsets[e];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        size_t i = base + q;
        if (i < (size_t)a.n) out[i] = ex;
        ex += it[q];
    }
}

uint32_t scan_chunks(int n) { return (uint32_t)(((size_t)n + kScanChunk - 1) / kScanChunk); }

size_t scan_workspace(int k, int n) {
    size_t chunks = ((size_t)n + kScanChunk - 1) / kScanChunk;
    return align_up((size_t)k * chunks * sizeof(uint64_t), 256);
}

vdi_status launch_scan(int k, int n, uint32_t* const* counts, uint64_t* const* offsets, void* ws, cudaStream_t st) {
    ScanArgs a;
    for (int e = 0; e < k; ++e) {
        a.counts[e] = counts[e];
        a.offsets[e] = offsets[e];
    }
    a.n = n;
    a.chunks = (n + kScanChunk - 1) / kScanChunk;
    a.partial = reinterpret_cast<uint64_t*>(ws);
    if (a.chunks == 0) a.chunks = 1;
    dim3 grid((unsigned)a.chunks, (unsigned)k);
    scan_reduce_kernel<<<grid, kScanThreads, 0, st>>>(a);
    scan_partials_kernel<<<k, kScanThreads, 0, st>>>(a);
    scan_down_kernel<<<grid, kScanThreads, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "scan kernels launch");
}

// ---------------------------------------------------------------------------
// Batched: the lists of many (request, PE) pairs, each of its own length, in
// one set of three launches.  Chunk c belongs to the last list whose
// chunk_begin is <= c; partial sums are indexed by global chunk.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int list_of_chunk(const ScanList* L, int nl, uint32_t chunk) {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&L[mid].chunk_begin) <= chunk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void scan_reduce_batched_kernel(const ScanList* __restrict__ L, int nl, uint64_t* __restrict__ partial) {
    const uint32_t chunk = blockIdx.x;
    const ScanList& l = L[list_of_chunk(L, nl, chunk)];
    const size_t base = (size_t)(chunk - l.chunk_begin) * kScanChunk + (size_t)threadIdx.x * kScanItems;
    uint32_t it[kScanItems];
    load_items(l.counts, l.n, base, it);
    uint64_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) s += it[q];
    uint64_t total;
    block_exclusive_scan(s, total);
    if (threadIdx.x == 0) partial[chunk] = total;
}

__global__ void scan_partials_batched_kernel(const ScanList* __restrict__ L, uint64_t* __restrict__ partial) {
    const ScanList& l = L[blockIdx.x];
    const int chunks = (l.n + kScanChunk - 1) / kScanChunk;
    uint64_t* p = partial + l.chunk_begin;
    uint64_t carry = 0;
    for (int start = 0; start < chunks; start += kScanThreads) {
        const int i = start + threadIdx.x;
        const uint64_t v = i < chunks ? p[i] : 0;
        uint64_t total;
        const uint64_t ex = block_exclusive_scan(v, total);
        if (i < chunks) p[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) l.offsets[l.n] = carry;
}

__global__ void scan_down_batched_kernel(const ScanList* __restrict__ L, int nl, const uint64_t* __restrict__ partial) {
    const uint32_t chunk = blockIdx.x;
    const ScanList& l = L[list_of_chunk(L, nl, chunk)];
    const size_t base = (size_t)(chunk - l.chunk_begin) * kScanChunk + (size_t)threadIdx.x * kScanItems;
    uint32_t it[kScanItems];
    load_items(l.counts, l.n, base, it);
    uint64_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) s += it[q];
    uint64_t total;
    uint64_t ex = block_exclusive_scan(s, total) + partial[chunk];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        const size_t i = base + q;
        if (i < (size_t)l.n) l.offsets[i] = ex;
        ex += it[q];
    }
}

vdi_status launch_scan_batched(const ScanList* dev_lists, int nlists, uint32_t total_chunks, uint64_t* partial,
                               cudaStream_t st) {
    if (nlists <= 0 || total_chunks == 0) return VDI_OK;
    scan_reduce_batched_kernel<<<total_chunks, kScanThreads, 0, st>>>(dev_lists, nlists, partial);
    scan_partials_batched_kernel<<<nlists, kScanThreads, 0, st>>>(dev_lists, partial);
    scan_down_batched_kernel<<<total_chunks, kScanThreads, 0, st>>>(dev_lists, nlists, partial);
    return cuda_check(cudaGetLastError(), "batched scan kernels launch");
}

}  // namespace vdi
