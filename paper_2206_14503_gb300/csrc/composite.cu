// Phase 2: compositing of K compact sub-VDIs into one regular VDI (sec. 5.2,
// Eq. 2, Algorithm S1).
//
// One thread per pixel.  The paper's all-to-all exchange becomes a gather: the
// thread reads its K spans [offsets_e[p], offsets_e[p] + counts_e[p]) straight
// from the K PEs' record arrays.  A depth sweep over the K list heads (each PE's
// list is depth-sorted and non-overlapping, sec. 5.2) cuts the records at every
// front and back depth and yields the pieces in order:
//   - a gap between records: a transparent sample;
//   - an interval covered by one record whole: that record, unchanged;
//   - part of one record: opacity by Eq. 2, 1 - (1 - A)^(dt / l);
//   - an interval covered by several records: their emission-absorption
//     mixture (extinctions add; colour is the extinction-weighted mean).
// The pieces feed the supersegment state machine (Eq. 1) inside the per-pixel
// bisection search for gamma; each search march evaluates two bisection levels
// (midpoint and quarter points) and the first one also counts non-transparent
// pieces (the count at gamma = 0).  A final march emits at most n_s
// supersegments into the regular layout with a zero tail.
#include <climits>

#include "vdi_device.cuh"

namespace vdi {

struct PeIn {
    const uint32_t* counts;
    const uint64_t* offsets;
    const void* rgba;
    const float2* fb;
};

struct CompArgs {
    PeIn pe[VDI_MAX_PE];
    int k, npix, n_s, iters;
    int prec_out;
    uint32_t* out_counts;
    void* out_rgba;
    float2* out_fb;
    float* out_gamma;
    unsigned int* status;
};

struct Piece {
    float f, b;
    float P[3];
    float a;
    float lgT;  // log2(1 - a)
};

template <int PREC>
__device__ __forceinline__ void load_fb(const PeIn& pe, uint64_t idx, float& f, float& b) {
    if (PREC == VDI_PREC_F32) {
        float2 v = __ldg(pe.fb + idx);
        f = v.x;
        b = v.y;
    } else {
        float2 v = __ldg(reinterpret_cast<const float2*>(reinterpret_cast<const uint4*>(pe.rgba) + idx));
        f = v.x;
        b = v.y;
    }
}

template <int PREC>
__device__ __forceinline__ float4 load_rgba(const PeIn& pe, uint64_t idx) {
    if (PREC == VDI_PREC_F32) return __ldg(reinterpret_cast<const float4*>(pe.rgba) + idx);
    uint2 v = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const uint4*>(pe.rgba) + idx) + 1);
    __half2 rg = *reinterpret_cast<__half2*>(&v.x);
    __half2 ba = *reinterpret_cast<__half2*>(&v.y);
    float2 a = __half22float2(rg), b2 = __half22float2(ba);
    return make_float4(a.x, a.y, b2.x, b2.y);
}

// Sweep state: one head per PE.
template <int KMAX>
struct Heads {
    uint64_t cur[KMAX];
    uint32_t rem[KMAX];
    float hf[KMAX], hb[KMAX];
};

// advance PE e's head to its next record with b > f (records with b <= f are ignored)
template <int KMAX, int PREC>
__device__ __forceinline__ void next_valid(const CompArgs& a, Heads<KMAX>& h, int e) {
    while (h.rem[e] > 0) {
        float f, b;
        load_fb<PREC>(a.pe[e], h.cur[e], f, b);
        if (b > f) {
            h.hf[e] = f;
            h.hb[e] = b;
            return;
        }
        ++h.cur[e];
        --h.rem[e];
    }
}

// Calls visit(piece) for every piece of pixel p in depth order.
template <int KMAX, int PREC, typename V>
__device__ __forceinline__ void sweep(const CompArgs& a, const uint32_t* cnt0, const uint64_t* off0, V& visit) {
    Heads<KMAX> h;
    const int k = a.k;
    float t = 3.0e38f;
#pragma unroll
    for (int e = 0; e < KMAX; ++e) {
        if (e < k) {
            h.cur[e] = off0[e];
            h.rem[e] = cnt0[e];
            next_valid<KMAX, PREC>(a, h, e);
            if (h.rem[e] > 0) t = fminf(t, h.hf[e]);
        }
    }
    while (true) {
        float t1 = 3.0e38f;
        int nact = 0, last = -1;
#pragma unroll
        for (int e = 0; e < KMAX; ++e) {
            if (e < k && h.rem[e] > 0) {
                if (h.hf[e] <= t) {
                    ++nact;
                    last = e;
                    t1 = fminf(t1, h.hb[e]);
                } else {
                    t1 = fminf(t1, h.hf[e]);
                }
            }
        }
        if (t1 >= 3.0e38f) break;
        Piece x;
        x.f = t;
        x.b = t1;
        if (nact == 0) {
            x.P[0] = x.P[1] = x.P[2] = 0.f;
            x.a = 0.f;
            x.lgT = 0.f;
        } else if (nact == 1 && h.hf[last] == t && h.hb[last] == t1) {
            float4 c = load_rgba<PREC>(a.pe[last], h.cur[last]);
            x.P[0] = c.x; x.P[1] = c.y; x.P[2] = c.z;
            x.a = c.w;
            x.lgT = lg2_approx(__fsub_rn(1.f, c.w));
        } else {
            // emission-absorption mixture over [t, t1]; extinction in log2 units
            float M = 0.f, MC[3] = {0.f, 0.f, 0.f}, OC[3] = {0.f, 0.f, 0.f};
            int nop = 0;
            const float dt = __fsub_rn(t1, t);
#pragma unroll
            for (int e = 0; e < KMAX; ++e) {
                if (e < k && h.rem[e] > 0 && h.hf[e] <= t) {
                    float4 c = load_rgba<PREC>(a.pe[e], h.cur[e]);
                    if (c.w >= 1.f) {
                        ++nop;
                        OC[0] += c.x; OC[1] += c.y; OC[2] += c.z;
                    } else if (c.w > 0.f) {
                        float ia = rcp_approx(c.w);
                        float mu = __fmul_rn(-lg2_approx(__fsub_rn(1.f, c.w)), rcp_approx(__fsub_rn(h.hb[e], h.hf[e])));
                        M = __fadd_rn(M, mu);
                        MC[0] = __fmaf_rn(mu, __fmul_rn(c.x, ia), MC[0]);
                        MC[1] = __fmaf_rn(mu, __fmul_rn(c.y, ia), MC[1]);
                        MC[2] = __fmaf_rn(mu, __fmul_rn(c.z, ia), MC[2]);
                    }
                }
            }
            if (nop > 0) {
                float inv = 1.f / (float)nop;
                x.a = 1.f;
                x.P[0] = OC[0] * inv; x.P[1] = OC[1] * inv; x.P[2] = OC[2] * inv;
                x.lgT = -INFINITY;
            } else if (M > 0.f) {
                x.lgT = -__fmul_rn(M, dt);
                x.a = __fsub_rn(1.f, ex2_approx(x.lgT));
                float s = __fmul_rn(x.a, rcp_approx(M));
                x.P[0] = __fmul_rn(MC[0], s); x.P[1] = __fmul_rn(MC[1], s); x.P[2] = __fmul_rn(MC[2], s);
            } else {
                x.P[0] = x.P[1] = x.P[2] = 0.f;
                x.a = 0.f;
                x.lgT = 0.f;
            }
        }
        visit(x);
        // advance heads that end at t1
#pragma unroll
        for (int e = 0; e < KMAX; ++e) {
            if (e < k && h.rem[e] > 0 && h.hf[e] <= t && h.hb[e] <= t1) {
                ++h.cur[e];
                --h.rem[e];
                next_valid<KMAX, PREC>(a, h, e);
            }
        }
        t = t1;
    }
}

// Counting state of one gamma candidate over pieces of arbitrary length.
struct CompCount {
    float P[3], A, L2, fS, bS;
    int cnt;
    bool open;
};

__device__ __forceinline__ void cc_step(CompCount& s, const Piece& x, float g2, int cap) {
    if (!s.open) {
        if (x.a > 0.f) {
            s.P[0] = x.P[0]; s.P[1] = x.P[1]; s.P[2] = x.P[2];
            s.A = x.a; s.L2 = x.lgT; s.fS = x.f; s.bS = x.b; s.open = true;
            ++s.cnt;
        }
        return;
    }
    float lx = __fsub_rn(x.b, x.f), lS = __fsub_rn(s.bS, s.fS);
    float r = (lx > 0.f && lS > 0.f) ? __fmul_rn(lx, rcp_approx(lS)) : 1.f;
    if (s.cnt < cap && criterion(s.P, s.A, s.L2, r, x.P, g2)) {
        if (x.a > 0.f) {
            s.P[0] = x.P[0]; s.P[1] = x.P[1]; s.P[2] = x.P[2];
            s.A = x.a; s.L2 = x.lgT; s.fS = x.f; s.bS = x.b;
            ++s.cnt;
        } else {
            s.open = false;
        }
    } else {
        absorb(s.P, s.A, s.L2, x.P, x.a, x.lgT);
        s.bS = x.b;
    }
}

template <int NC>
struct CountVisitor {
    CompCount st[NC];
    float g2[NC];
    int nt;
    __device__ __forceinline__ void operator()(const Piece& x) {
        nt += x.a > 0.f;
#pragma unroll
        for (int c = 0; c < NC; ++c) cc_step(st[c], x, g2[c], INT_MAX);
    }
};

struct EmitVisitor {
    CompCount s;
    float g2;
    int cap;
    float bt;
    int written;
    size_t base;  // first slot of the pixel
    const CompArgs* a;

    __device__ __forceinline__ void store(float f, float b, const float P[3], float A) {
        size_t idx = base + written;
        if (a->prec_out == VDI_PREC_F32) {
            reinterpret_cast<float4*>(a->out_rgba)[idx] = make_float4(P[0], P[1], P[2], A);
            a->out_fb[idx] = make_float2(f, b);
        } else {
            __half2 rg = __floats2half2_rn(P[0], P[1]);
            __half2 ba = __floats2half2_rn(P[2], A);
            uint4 v;
            v.x = __float_as_uint(f);
            v.y = __float_as_uint(b);
            v.z = *reinterpret_cast<unsigned int*>(&rg);
            v.w = *reinterpret_cast<unsigned int*>(&ba);
            reinterpret_cast<uint4*>(a->out_rgba)[idx] = v;
        }
        ++written;
    }

    __device__ __forceinline__ void operator()(const Piece& x) {
        if (!s.open) {
            if (x.a > 0.f) {
                s.P[0] = x.P[0]; s.P[1] = x.P[1]; s.P[2] = x.P[2];
                s.A = x.a; s.L2 = x.lgT; s.fS = x.f; s.bS = x.b; s.open = true;
                bt = x.b;
                ++s.cnt;
            }
            return;
        }
        float lx = __fsub_rn(x.b, x.f), lS = __fsub_rn(s.bS, s.fS);
        float r = (lx > 0.f && lS > 0.f) ? __fmul_rn(lx, rcp_approx(lS)) : 1.f;
        if (s.cnt < cap && criterion(s.P, s.A, s.L2, r, x.P, g2)) {
            if (written < cap) store(s.fS, bt, s.P, s.A);
            if (x.a > 0.f) {
                s.P[0] = x.P[0]; s.P[1] = x.P[1]; s.P[2] = x.P[2];
                s.A = x.a; s.L2 = x.lgT; s.fS = x.f; s.bS = x.b;
                bt = x.b;
                ++s.cnt;
            } else {
                s.open = false;
            }
        } else {
            absorb(s.P, s.A, s.L2, x.P, x.a, x.lgT);
            s.bS = x.b;
            if (x.a > 0.f) bt = x.b;
        }
    }
};

template <int KMAX, int PREC>
__global__ void __launch_bounds__(128) composite_kernel(const __grid_constant__ CompArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.npix) return;
    uint32_t cnt0[KMAX];
    uint64_t off0[KMAX];
#pragma unroll
    for (int e = 0; e < KMAX; ++e) {
        if (e < a.k) {
            cnt0[e] = __ldg(a.pe[e].counts + p);
            off0[e] = __ldg(a.pe[e].offsets + p);
        }
    }
    // search (sec. 2.4 applied to the pieces, sec. 5.2)
    float gamma = 0.f;
    int count;
    {
        CountVisitor<3> v;
        v.g2[0] = 1.f; v.g2[1] = 0.25f; v.g2[2] = 2.25f;
        v.nt = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) { v.st[c].cnt = 0; v.st[c].open = false; }
        sweep<KMAX, PREC>(a, cnt0, off0, v);
        if (v.nt <= a.n_s) {
            count = v.nt;
        } else {
            Bisect bs;
            bs.lo = 0.f; bs.hi = 2.f; bs.it = 0; bs.cnt_hi = 1; bs.done = false;
            int c[3] = {v.st[0].cnt, v.st[1].cnt, v.st[2].cnt};
            bisect_apply(bs, c, a.n_s, a.iters);
            while (!bs.done) {
                float g[3];
                bisect_candidates(bs, g);
                CountVisitor<3> w;
                w.nt = 0;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    w.g2[q] = __fmul_rn(g[q], g[q]);
                    w.st[q].cnt = 0;
                    w.st[q].open = false;
                }
                sweep<KMAX, PREC>(a, cnt0, off0, w);
                c[0] = w.st[0].cnt; c[1] = w.st[1].cnt; c[2] = w.st[2].cnt;
                bisect_apply(bs, c, a.n_s, a.iters);
            }
            gamma = bs.hi;
            count = bs.cnt_hi;
        }
    }
    // emission
    EmitVisitor em;
    em.s.cnt = 0;
    em.s.open = false;
    em.g2 = __fmul_rn(gamma, gamma);
    em.cap = a.n_s;
    em.bt = 0.f;
    em.written = 0;
    em.base = (size_t)p * a.n_s;
    em.a = &a;
    sweep<KMAX, PREC>(a, cnt0, off0, em);
    if (em.s.open && em.written < a.n_s) em.store(em.s.fS, em.bt, em.s.P, em.s.A);
    // zero tail
    for (int j = em.written; j < a.n_s; ++j) {
        size_t idx = (size_t)p * a.n_s + j;
        if (a.prec_out == VDI_PREC_F32) {
            reinterpret_cast<float4*>(a.out_rgba)[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
            a.out_fb[idx] = make_float2(0.f, 0.f);
        } else {
            reinterpret_cast<uint4*>(a.out_rgba)[idx] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    a.out_counts[p] = (uint32_t)em.written;
    if (a.out_gamma) a.out_gamma[p] = gamma;
    if (em.written != count) atomicCAS(a.status, 0u, (unsigned)VDI_ERR_CUDA);
}

vdi_status launch_composite(const vdi_compact* pe, int k, int w, int h, const vdi_regular* out, int iters,
                            int schedule, unsigned int* status, cudaStream_t st) {
    CompArgs a;
    for (int e = 0; e < k; ++e) {
        a.pe[e].counts = pe[e].counts;
        a.pe[e].offsets = pe[e].offsets;
        a.pe[e].rgba = pe[e].rgba;
        a.pe[e].fb = reinterpret_cast<const float2*>(pe[e].fb);
    }
    a.k = k;
    a.npix = w * h;
    a.n_s = out->n_s;
    a.iters = iters;
    a.prec_out = out->prec;
    a.out_counts = out->counts;
    a.out_rgba = out->rgba;
    a.out_fb = reinterpret_cast<float2*>(out->fb);
    a.out_gamma = out->gamma;
    a.status = status;
    const int prec_in = pe[0].prec;
    (void)schedule;
    const int threads = 128;
    const unsigned blocks = (unsigned)((a.npix + threads - 1) / threads);
    if (a.npix == 0) return VDI_OK;
    if (k <= 8) {
        if (prec_in == VDI_PREC_F32) composite_kernel<8, VDI_PREC_F32><<<blocks, threads, 0, st>>>(a);
        else composite_kernel<8, VDI_PREC_F16><<<blocks, threads, 0, st>>>(a);
    } else {
        if (prec_in == VDI_PREC_F32) composite_kernel<VDI_MAX_PE, VDI_PREC_F32><<<blocks, threads, 0, st>>>(a);
        else composite_kernel<VDI_MAX_PE, VDI_PREC_F16><<<blocks, threads, 0, st>>>(a);
    }
    return cuda_check(cudaGetLastError(), "composite_kernel launch");
}

}  // namespace vdi
