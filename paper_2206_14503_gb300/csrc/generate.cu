// Phase 1: sub-VDI generation (sec. 4, sec. 5.1).
//
// gen_count_kernel: one thread per (PE, ray), 16 x 16 pixel tiles per CTA as in
// the paper's work-groups, each warp an 8 x 4 pixel block for coherent volume
// access.  It marches the PE's owned samples and runs the supersegment state
// machine (Eq. 1) to choose gamma: a fixed value, the per-ray bisection search
// of sec. 2.4, or a given per-ray value with the search as fallback.  The
// search replays sequential bisection exactly but evaluates two levels per
// march (midpoint and both quarter points), and the first march also counts
// the non-transparent samples, which is the count at gamma = 0.
//
// gen_emit_kernel: re-marches with the chosen gamma and writes the records at
// the prefix-sum offsets (compact layout, sec. 4).
#include <climits>
#include <float.h>

#include "vdi_device.cuh"

namespace vdi {

struct GenArgs {
    BrickDev b[VDI_MAX_PE];
    CompactDev out[VDI_MAX_PE];
    CamDev cam;
    int dims[3];
    const float* lut;  // 256 x 4, straight colour + opacity per ref_len
    float scale255, step, ref_len;
    int k, n_s, iters;
    int mode;  // 0 fixed, 1 search, 2 given (+ fallback)
    float gamma;
    int prec;
    int tiles_x;
    unsigned int* status;
};

constexpr int kTile = 16;

// Work census (VDI_FLAG_CENSUS): kept in registers; the kernel variant
// without the census never stores it, so the counting is compiled out.
struct Census {
    unsigned long long evals = 0, steps = 0, passes = 0;
};

// 257 entries of (colour/opacity, difference to the next entry); opacity
// corrected to the step length: a' = 1 - (1 - a)^(step / ref_len).
__device__ __forceinline__ void load_lut(const GenArgs& a, float4* lut2) {
    __shared__ float4 base[257];
    for (int i = threadIdx.x; i < 257; i += blockDim.x) {
        int s = min(i, 255);
        float4 v = reinterpret_cast<const float4*>(a.lut)[s];
        v.w = 1.f - powf(1.f - v.w, a.step / a.ref_len);
        base[i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 257; i += blockDim.x) {
        float4 v = base[i], w = base[min(i + 1, 256)];
        lut2[2 * i] = v;
        lut2[2 * i + 1] = make_float4(__fsub_rn(w.x, v.x), __fsub_rn(w.y, v.y), __fsub_rn(w.z, v.z),
                                      __fsub_rn(w.w, v.w));
    }
    __syncthreads();
}

__device__ __forceinline__ void tile_pixel(int tiles_x, int& i, int& j) {
    int t = blockIdx.x;
    int tx = t % tiles_x, ty = t / tiles_x;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    i = tx * kTile + (warp & 1) * 8 + (lane & 7);
    j = ty * kTile + (warp >> 1) * 4 + (lane >> 3);
}

// One march over samples [k0, k1): NC gamma candidates (squared) with the
// given cap, plus the number of non-transparent samples.
template <int NC>
__device__ __forceinline__ void count_pass(const Ray& r, float step, int k0, int k1, const BrickDev& b,
                                           const float4* lut2, float scale255, const float g2[NC], int cap,
                                           int cnt[NC], int& nt, Census& cs) {
    cs.evals += (unsigned long long)(k1 - k0);
    cs.steps += (unsigned long long)(k1 - k0) * NC;
    cs.passes += 1;
    GenCount st[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) gc_reset(st[c]);
    int n_nt = 0;
    long long P[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) P[a] = r.P0[a] + (long long)k0 * r.D[a];
    for (int k = k0; k < k1; ++k) {
        Sample s;
        sample_at(P, b, lut2, scale255, s);
#pragma unroll
        for (int a = 0; a < 3; ++a) P[a] += r.D[a];
        n_nt += s.a > 0.f;
#pragma unroll
        for (int c = 0; c < NC; ++c) gc_step(st[c], s, g2[c], cap);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) cnt[c] = st[c].cnt;
    nt = n_nt;
}

// Per-ray bisection search (sec. 2.4) given the count at gamma = 0 is above n_s.
// Returns gamma (upper end) and the count there.
__device__ __forceinline__ float search(const Ray& r, float step, int k0, int k1, const BrickDev& b,
                                        const float4* lut2, float scale255, int n_s, int iters, int c0,
                                        const int* first_counts, int& count, Census& cs) {
    Bisect bs;
    bs.lo = 0.f;
    bs.hi = 2.f;
    bs.it = 0;
    bs.cnt_hi = c0 > 0 ? 1 : 0;  // the distance never reaches 2: one supersegment
    bs.done = false;
    int c[3];
    if (first_counts) {
        c[0] = first_counts[0]; c[1] = first_counts[1]; c[2] = first_counts[2];
        bisect_apply(bs, c, n_s, iters);
    }
    while (!bs.done) {
        float g[3], g2[3];
        bisect_candidates(bs, g);
#pragma unroll
        for (int q = 0; q < 3; ++q) g2[q] = __fmul_rn(g[q], g[q]);
        int nt;
        count_pass<3>(r, step, k0, k1, b, lut2, scale255, g2, INT_MAX, c, nt, cs);
        bisect_apply(bs, c, n_s, iters);
    }
    count = bs.cnt_hi;
    return bs.hi;
}

template <bool CENSUS>
__global__ void __launch_bounds__(256, 2) gen_count_kernel(const __grid_constant__ GenArgs a) {
    __shared__ float4 lut2[2 * 257];
    load_lut(a, lut2);
    int i, j;
    tile_pixel(a.tiles_x, i, j);
    if (i >= a.cam.W || j >= a.cam.H) return;
    const int e = blockIdx.y;
    const BrickDev& b = a.b[e];
    const CompactDev& o = a.out[e];
    const size_t p = (size_t)j * a.cam.W + i;
    Ray r;
    int k0 = 0, k1 = 0;
    bool any = ray_setup(a.cam, i, j, a.dims, a.step, r) && owned_range(r, a.step, b, a.dims, k0, k1);
    float gamma = 0.f;
    int count = 0;
    Census cs;
    if (a.mode == 2) gamma = fmaxf(o.gamma[p], 0.f);
    if (any) {
        if (a.mode == 0) {
            float g2[1] = {__fmul_rn(a.gamma, a.gamma)};
            int c[1], nt;
            count_pass<1>(r, a.step, k0, k1, b, lut2, a.scale255, g2, a.n_s, c, nt, cs);
            gamma = a.gamma;
            count = c[0];
        } else if (a.mode == 2) {
            float g2[1] = {__fmul_rn(gamma, gamma)};
            int c[1], nt;
            count_pass<1>(r, a.step, k0, k1, b, lut2, a.scale255, g2, INT_MAX, c, nt, cs);
            if (c[0] <= a.n_s) {
                count = c[0];
            } else {
                // fallback: the full search (its first march re-counts gamma = 0)
                float g2s[3] = {1.f, 0.25f, 2.25f};
                int c3[3];
                count_pass<3>(r, a.step, k0, k1, b, lut2, a.scale255, g2s, INT_MAX, c3, nt, cs);
                if (nt <= a.n_s) {
                    gamma = 0.f;
                    count = nt;
                } else {
                    gamma = search(r, a.step, k0, k1, b, lut2, a.scale255, a.n_s, a.iters, nt, c3, count, cs);
                }
            }
        } else {
            // search: gamma = 0 (non-transparent count) and bisection levels 1-2 in one march
            float g2[3] = {1.f, 0.25f, 2.25f};
            int c[3], nt;
            count_pass<3>(r, a.step, k0, k1, b, lut2, a.scale255, g2, INT_MAX, c, nt, cs);
            if (nt <= a.n_s) {
                gamma = 0.f;
                count = nt;
            } else {
                gamma = search(r, a.step, k0, k1, b, lut2, a.scale255, a.n_s, a.iters, nt, c, count, cs);
            }
        }
    } else if (a.mode == 0) {
        gamma = a.gamma;
    }
    o.counts[p] = (uint32_t)count;
    if (o.gamma) o.gamma[p] = gamma;
    if (CENSUS) {
        unsigned long long* ctr = reinterpret_cast<WsHeader*>(a.status)->counters;
        atomicAdd(ctr + 0, cs.evals);
        atomicAdd(ctr + 1, cs.steps);
        atomicAdd(ctr + 2, cs.passes);
        atomicAdd(ctr + 3, any ? 1ull : 0ull);
    }
}

struct RecOut {
    float f, b, P[3], A;
};

__device__ __forceinline__ void store_record(const GenArgs& a, const CompactDev& o, uint64_t idx, const RecOut& r) {
    if (idx >= o.capacity) {
        atomicCAS(a.status, 0u, (unsigned)VDI_ERR_CAPACITY);
        return;
    }
    if (a.prec == VDI_PREC_F32) {
        reinterpret_cast<float4*>(o.rgba)[idx] = make_float4(r.P[0], r.P[1], r.P[2], r.A);
        reinterpret_cast<float2*>(o.fb)[idx] = make_float2(r.f, r.b);
    } else {
        __half2 rg = __floats2half2_rn(r.P[0], r.P[1]);
        __half2 ba = __floats2half2_rn(r.P[2], r.A);
        uint4 v;
        v.x = __float_as_uint(r.f);
        v.y = __float_as_uint(r.b);
        v.z = *reinterpret_cast<unsigned int*>(&rg);
        v.w = *reinterpret_cast<unsigned int*>(&ba);
        reinterpret_cast<uint4*>(o.rgba)[idx] = v;
    }
}

__global__ void __launch_bounds__(256, 2) gen_emit_kernel(const __grid_constant__ GenArgs a) {
    __shared__ float4 lut2[2 * 257];
    load_lut(a, lut2);
    int i, j;
    tile_pixel(a.tiles_x, i, j);
    if (i >= a.cam.W || j >= a.cam.H) return;
    const int e = blockIdx.y;
    const BrickDev& b = a.b[e];
    const CompactDev& o = a.out[e];
    const size_t p = (size_t)j * a.cam.W + i;
    const uint32_t want = o.counts[p];
    if (want == 0) return;
    Ray r;
    int k0 = 0, k1 = 0;
    if (!(ray_setup(a.cam, i, j, a.dims, a.step, r) && owned_range(r, a.step, b, a.dims, k0, k1))) return;
    const float gamma = o.gamma ? o.gamma[p] : a.gamma;
    const float g2 = __fmul_rn(gamma, gamma);
    const uint64_t base = o.offsets[p];
    const int cap = a.n_s;
    // state machine with record tracking (same decisions as GenCount)
    float P[3] = {0.f, 0.f, 0.f}, A = 0.f, L2 = 0.f, m = 0.f;
    int cnt = 0, kopen = 0, klast = 0;
    uint32_t written = 0;
    long long Pos[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) Pos[q] = r.P0[q] + (long long)k0 * r.D[q];
    for (int k = k0; k < k1; ++k) {
        Sample s;
        sample_at(Pos, b, lut2, a.scale255, s);
#pragma unroll
        for (int q = 0; q < 3; ++q) Pos[q] += r.D[q];
        bool open_new = false;
        if (m == 0.f) {
            open_new = s.a > 0.f;
        } else {
            float rr = rcp_approx(m);
            if (cnt < cap && criterion(P, A, L2, rr, s.P, g2)) {
                if (written < want) {
                    RecOut ro{sample_front(r, a.step, kopen), sample_front(r, a.step, klast + 1), {P[0], P[1], P[2]}, A};
                    store_record(a, o, base + written, ro);
                }
                ++written;
                m = 0.f;
                open_new = s.a > 0.f;
            } else {
                absorb(P, A, L2, s.P, s.a, s.lgT);
                m = __fadd_rn(m, 1.f);
                if (s.a > 0.f) klast = k;
            }
        }
        if (open_new) {
            P[0] = s.P[0]; P[1] = s.P[1]; P[2] = s.P[2];
            A = s.a; L2 = s.lgT; m = 1.f;
            kopen = k; klast = k;
            ++cnt;
        }
    }
    if (m != 0.f) {
        if (written < want) {
            RecOut ro{sample_front(r, a.step, kopen), sample_front(r, a.step, klast + 1), {P[0], P[1], P[2]}, A};
            store_record(a, o, base + written, ro);
        }
        ++written;
    }
    if (written != want) atomicCAS(a.status, 0u, (unsigned)VDI_ERR_CUDA);
}

static void fill_args(GenArgs& a, const BrickDev* bricks, int k, const float* lut, const CamDev& cam,
                      const int dims[3], float scale255, float step, float ref_len, int n_s, const CompactDev* out,
                      unsigned int* status) {
    for (int e = 0; e < k; ++e) {
        a.b[e] = bricks[e];
        a.out[e] = out[e];
    }
    a.cam = cam;
    for (int q = 0; q < 3; ++q) a.dims[q] = dims[q];
    a.lut = lut;
    a.scale255 = scale255;
    a.step = step;
    a.ref_len = ref_len;
    a.k = k;
    a.n_s = n_s;
    a.status = status;
    a.tiles_x = (cam.W + kTile - 1) / kTile;
}

vdi_status launch_gen_count(const BrickDev* bricks, int k, const float* lut, const CamDev& cam, const int dims[3],
                            float scale255, float step, float ref_len, int n_s, float gamma, int iters,
                            const CompactDev* out, unsigned int* status, bool census, cudaStream_t st) {
    GenArgs a;  // copied into the launch's parameter space
    fill_args(a, bricks, k, lut, cam, dims, scale255, step, ref_len, n_s, out, status);
    a.iters = iters;
    a.gamma = gamma;
    a.mode = gamma >= 0.f ? 0 : (gamma == VDI_GAMMA_GIVEN ? 2 : 1);
    a.prec = 0;
    int tiles_y = (cam.H + kTile - 1) / kTile;
    dim3 grid((unsigned)(a.tiles_x * tiles_y), (unsigned)k);
    if (census) gen_count_kernel<true><<<grid, 256, 0, st>>>(a);
    else gen_count_kernel<false><<<grid, 256, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "gen_count_kernel launch");
}

vdi_status launch_gen_emit(const BrickDev* bricks, int k, const float* lut, const CamDev& cam, const int dims[3],
                           float scale255, float step, float ref_len, int n_s, int prec, const CompactDev* out,
                           unsigned int* status, cudaStream_t st) {
    GenArgs a;
    fill_args(a, bricks, k, lut, cam, dims, scale255, step, ref_len, n_s, out, status);
    a.iters = 0;
    a.gamma = 0.f;
    a.mode = 0;
    a.prec = prec;
    int tiles_y = (cam.H + kTile - 1) / kTile;
    dim3 grid((unsigned)(a.tiles_x * tiles_y), (unsigned)k);
    gen_emit_kernel<<<grid, 256, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "gen_emit_kernel launch");
}

}  // namespace vdi
