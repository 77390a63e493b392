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
// bisection search for gamma.  A search march evaluates the next NLEV
// bisection levels at once (the 2^NLEV - 1 midpoints of the subtree) and
// records, per candidate, the interval of gamma over which all of its
// decisions would repeat; the sequential bisection is replayed from the
// recorded counts, marching again only for a midpoint no record covers, so
// the result is that of plain bisection.  The first march also counts
// non-transparent pieces, which is the count at gamma = 0.  A final march emits at most n_s
// supersegments into the regular layout with a zero tail.
//
// Schedules (chosen per request by the autotuner, vdi_composite_autotune):
//   1: list heads in registers (K <= 8), 2 levels per march;
//   2: list heads in local memory (K <= 64), 2 levels per march;
//   3: list heads in local memory, 3 levels per march (7 candidates).
//
// composite_batched_kernel runs many requests (different sizes, K, N_S) in one
// persistent launch: CTAs pull (request, 128-pixel tile) items from an atomic
// counter until none are left.
#include <climits>

#include "vdi_device.cuh"

namespace vdi {

struct PeIn {
    const uint32_t* counts;
    const uint64_t* offsets;
    const void* rgba;
    const float2* fb;
};

struct OutDev {
    uint32_t* counts;
    void* rgba;
    float2* fb;
    float* gamma;
    int n_s;
    int prec;
};

struct CompArgs {
    PeIn pe[VDI_MAX_PE];
    OutDev out;
    int k, npix, iters;
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

// Sweep state: one head per PE.  KMAX <= 16: unrolled, in registers;
// larger: runtime loops, in local memory.
template <int KMAX>
struct Heads {
    uint64_t cur[KMAX];
    uint32_t rem[KMAX];
    float hf[KMAX], hb[KMAX];
};

#define VDI_UNROLL_K _Pragma("unroll")
template <int KMAX>
struct Unroll {
    static constexpr int N = KMAX <= 16 ? KMAX : 1;
};

// advance PE e's head to its next record with b > f (records with b <= f are ignored)
template <int KMAX, int PREC>
__device__ __forceinline__ void next_valid(const PeIn* pe, Heads<KMAX>& h, int e) {
    while (h.rem[e] > 0) {
        float f, b;
        load_fb<PREC>(pe[e], h.cur[e], f, b);
        if (b > f) {
            h.hf[e] = f;
            h.hb[e] = b;
            return;
        }
        ++h.cur[e];
        --h.rem[e];
    }
}

// Calls visit(piece) for every piece of one pixel in depth order.
template <int KMAX, int PREC, typename V>
__device__ __forceinline__ void sweep(const PeIn* pe, int k, const uint32_t* cnt0, const uint64_t* off0, V& visit) {
    Heads<KMAX> h;
    float t = 3.0e38f;
#pragma unroll Unroll<KMAX>::N
    for (int e = 0; e < KMAX; ++e) {
        if (e < k) {
            h.cur[e] = off0[e];
            h.rem[e] = cnt0[e];
            next_valid<KMAX, PREC>(pe, h, e);
            if (h.rem[e] > 0) t = fminf(t, h.hf[e]);
        }
    }
    while (true) {
        float t1 = 3.0e38f;
        int nact = 0, last = -1;
#pragma unroll Unroll<KMAX>::N
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
            float4 c = load_rgba<PREC>(pe[last], h.cur[last]);
            x.P[0] = c.x; x.P[1] = c.y; x.P[2] = c.z;
            x.a = c.w;
            x.lgT = lg2_approx(__fsub_rn(1.f, c.w));
        } else {
            // emission-absorption mixture over [t, t1]; extinction in log2 units
            float M = 0.f, MC[3] = {0.f, 0.f, 0.f}, OC[3] = {0.f, 0.f, 0.f};
            int nop = 0;
            const float dt = __fsub_rn(t1, t);
#pragma unroll Unroll<KMAX>::N
            for (int e = 0; e < KMAX; ++e) {
                if (e < k && h.rem[e] > 0 && h.hf[e] <= t) {
                    float4 c = load_rgba<PREC>(pe[e], h.cur[e]);
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
#pragma unroll Unroll<KMAX>::N
        for (int e = 0; e < KMAX; ++e) {
            if (e < k && h.rem[e] > 0 && h.hf[e] <= t && h.hb[e] <= t1) {
                ++h.cur[e];
                --h.rem[e];
                next_valid<KMAX, PREC>(pe, h, e);
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

// Counting with decision intervals (see GenCountQ): qlo / qhi bound the
// gamma^2 for which every decision of the march repeats.
struct CompCountQ {
    float P[3], A, L2, fS, bS;
    float qlo, qhi;
    int cnt;
    bool open;
};

__device__ __forceinline__ void cq_step(CompCountQ& s, const Piece& x, float g2) {
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
    float q;
    if (criterion_q(s.P, s.A, s.L2, r, x.P, g2, q)) {
        s.qhi = fminf(s.qhi, q);
        if (x.a > 0.f) {
            s.P[0] = x.P[0]; s.P[1] = x.P[1]; s.P[2] = x.P[2];
            s.A = x.a; s.L2 = x.lgT; s.fS = x.f; s.bS = x.b;
            ++s.cnt;
        } else {
            s.open = false;
        }
    } else {
        s.qlo = fmaxf(s.qlo, q);
        absorb(s.P, s.A, s.L2, x.P, x.a, x.lgT);
        s.bS = x.b;
    }
}

template <int NC>
struct CountVisitorQ {
    CompCountQ st[NC];
    float g2[NC];
    int nt;
    __device__ __forceinline__ void reset() {
        nt = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            st[c].cnt = 0;
            st[c].open = false;
            st[c].qlo = -1.f;
            st[c].qhi = 3.0e38f;
        }
    }
    __device__ __forceinline__ void operator()(const Piece& x) {
        nt += x.a > 0.f;
#pragma unroll
        for (int c = 0; c < NC; ++c) cq_step(st[c], x, g2[c]);
    }
};

template <int NC>
struct CountVisitor {
    CompCount st[NC];
    float g2[NC];
    int nt;
    __device__ __forceinline__ void reset() {
        nt = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            st[c].cnt = 0;
            st[c].open = false;
        }
    }
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
    const OutDev* out;

    __device__ __forceinline__ void store(float f, float b, const float P[3], float A) {
        size_t idx = base + written;
        if (out->prec == VDI_PREC_F32) {
            reinterpret_cast<float4*>(out->rgba)[idx] = make_float4(P[0], P[1], P[2], A);
            out->fb[idx] = make_float2(f, b);
        } else {
            __half2 rg = __floats2half2_rn(P[0], P[1]);
            __half2 ba = __floats2half2_rn(P[2], A);
            uint4 v;
            v.x = __float_as_uint(f);
            v.y = __float_as_uint(b);
            v.z = *reinterpret_cast<unsigned int*>(&rg);
            v.w = *reinterpret_cast<unsigned int*>(&ba);
            reinterpret_cast<uint4*>(out->rgba)[idx] = v;
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

// Midpoints of the complete bisection subtree of NLEV levels below [lo, hi]
// in heap order (node 1 = midpoint, node 2i / 2i+1 = its left / right child).
template <int NLEV>
__device__ __forceinline__ void tree_candidates(float lo, float hi, float g[(1 << NLEV) - 1]) {
    float L[(1 << NLEV)], H[(1 << NLEV)];
    L[1] = lo;
    H[1] = hi;
#pragma unroll
    for (int i = 1; i < (1 << NLEV); ++i) {
        float m = 0.5f * (L[i] + H[i]);
        g[i - 1] = m;
        if (2 * i + 1 < (1 << NLEV)) {
            L[2 * i] = L[i]; H[2 * i] = m;
            L[2 * i + 1] = m; H[2 * i + 1] = H[i];
        }
    }
}

// The whole per-pixel composite: search, emission, zero tail.
template <int KMAX, int NLEV, int PREC>
__device__ __forceinline__ void composite_pixel(const PeIn* pe, int k, const OutDev& out, int iters,
                                                unsigned int* status, uint32_t p) {
    constexpr int NC = (1 << NLEV) - 1;
    uint32_t cnt0[KMAX];
    uint64_t off0[KMAX];
#pragma unroll Unroll<KMAX>::N
    for (int e = 0; e < KMAX; ++e) {
        if (e < k) {
            cnt0[e] = __ldg(pe[e].counts + p);
            off0[e] = __ldg(pe[e].offsets + p);
        }
    }
    // search (sec. 2.4 applied to the pieces, sec. 5.2): sequential bisection;
    // a midpoint's count comes from the table of earlier marches when one of
    // their decision intervals holds it, else from a march over the NLEV-level
    // subtree below the current bracket.
    float gamma = 0.f;
    int count;
    {
        CountTable t;
        t.n = 0;
        CountVisitorQ<NC> v;
        float g[NC];
        v.reset();
        tree_candidates<NLEV>(0.f, 2.f, g);
#pragma unroll
        for (int q = 0; q < NC; ++q) v.g2[q] = __fmul_rn(g[q], g[q]);
        sweep<KMAX, PREC>(pe, k, cnt0, off0, v);
#pragma unroll
        for (int q = 0; q < NC; ++q) t.add(v.g2[q], v.st[q].qlo, v.st[q].qhi, v.st[q].cnt);
        if (v.nt <= out.n_s) {
            count = v.nt;
        } else {
            float lo = 0.f, hi = 2.f;
            int cnt_hi = 1;  // the distance never reaches 2: one supersegment
            for (int it = 0; it < iters; ++it) {
                float mid = 0.5f * (lo + hi);
                int c = t.lookup(__fmul_rn(mid, mid));
                if (c < 0) {
                    tree_candidates<NLEV>(lo, hi, g);
                    v.reset();
#pragma unroll
                    for (int q = 0; q < NC; ++q) v.g2[q] = __fmul_rn(g[q], g[q]);
                    sweep<KMAX, PREC>(pe, k, cnt0, off0, v);
#pragma unroll
                    for (int q = 0; q < NC; ++q) t.add(v.g2[q], v.st[q].qlo, v.st[q].qhi, v.st[q].cnt);
                    c = v.st[0].cnt;
                }
                if (c <= out.n_s) {
                    hi = mid;
                    cnt_hi = c;
                    if (c == out.n_s) break;
                } else {
                    lo = mid;
                }
            }
            gamma = hi;
            count = cnt_hi;
        }
    }
    EmitVisitor em;
    em.s.cnt = 0;
    em.s.open = false;
    em.g2 = __fmul_rn(gamma, gamma);
    em.cap = out.n_s;
    em.bt = 0.f;
    em.written = 0;
    em.base = (size_t)p * out.n_s;
    em.out = &out;
    sweep<KMAX, PREC>(pe, k, cnt0, off0, em);
    if (em.s.open && em.written < out.n_s) em.store(em.s.fS, em.bt, em.s.P, em.s.A);
    for (int j = em.written; j < out.n_s; ++j) {
        size_t idx = (size_t)p * out.n_s + j;
        if (out.prec == VDI_PREC_F32) {
            reinterpret_cast<float4*>(out.rgba)[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
            out.fb[idx] = make_float2(0.f, 0.f);
        } else {
            reinterpret_cast<uint4*>(out.rgba)[idx] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    out.counts[p] = (uint32_t)em.written;
    if (out.gamma) out.gamma[p] = gamma;
    if (em.written != count) atomicCAS(status, 0u, (unsigned)VDI_ERR_CUDA);
}

template <int PREC>
__device__ __forceinline__ void composite_pixel_sched(int sched, const PeIn* pe, int k, const OutDev& out, int iters,
                                                      unsigned int* status, uint32_t p) {
    if (sched == 1) composite_pixel<8, 2, PREC>(pe, k, out, iters, status, p);
    else if (sched == 3) composite_pixel<VDI_MAX_PE, 3, PREC>(pe, k, out, iters, status, p);
    else composite_pixel<VDI_MAX_PE, 2, PREC>(pe, k, out, iters, status, p);
}

template <int KMAX, int NLEV, int PREC>
__global__ void __launch_bounds__(128) composite_kernel(const __grid_constant__ CompArgs a) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (uint32_t)a.npix) return;
    composite_pixel<KMAX, NLEV, PREC>(a.pe, a.k, a.out, a.iters, a.status, p);
}

// ---------------------------------------------------------------------------
// Batched persistent compositing
// ---------------------------------------------------------------------------
struct ReqDev {
    OutDev out;
    uint32_t npix;
    uint32_t item_begin;  // first work item of the request
    uint32_t pe_begin;    // index of its first PE descriptor
    int k, schedule;
};

struct BatchArgs {
    const ReqDev* reqs;
    const PeIn* pes;
    int n;
    uint32_t total_items;
    unsigned int* counter;
    unsigned int* status;
    int iters;
};

constexpr int kBatchTile = 128;

template <int PREC>
__global__ void __launch_bounds__(kBatchTile) composite_batched_kernel(const __grid_constant__ BatchArgs a) {
    __shared__ uint32_t s_item;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= a.total_items) return;
        // request holding the item: last r with item_begin <= item
        int lo = 0, hi = a.n - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (__ldg(&a.reqs[mid].item_begin) <= item) lo = mid;
            else hi = mid - 1;
        }
        const ReqDev& r = a.reqs[lo];
        const uint32_t p = (item - r.item_begin) * kBatchTile + threadIdx.x;
        if (p < r.npix)
            composite_pixel_sched<PREC>(r.schedule, a.pes + r.pe_begin, r.k, r.out, a.iters, a.status, p);
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int default_schedule(int k) { return k <= 8 ? 1 : 2; }

static OutDev out_dev(const vdi_regular* out) {
    OutDev o;
    o.counts = out->counts;
    o.rgba = out->rgba;
    o.fb = reinterpret_cast<float2*>(out->fb);
    o.gamma = out->gamma;
    o.n_s = out->n_s;
    o.prec = out->prec;
    return o;
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
    a.iters = iters;
    a.out = out_dev(out);
    a.status = status;
    const int prec_in = pe[0].prec;
    if (schedule == 0 || (schedule == 1 && k > 8)) schedule = default_schedule(k);
    const int threads = 128;
    const unsigned blocks = (unsigned)((a.npix + threads - 1) / threads);
    if (a.npix == 0) return VDI_OK;
    const bool f32 = prec_in == VDI_PREC_F32;
    switch (schedule) {
        case 1:
            if (f32) composite_kernel<8, 2, VDI_PREC_F32><<<blocks, threads, 0, st>>>(a);
            else composite_kernel<8, 2, VDI_PREC_F16><<<blocks, threads, 0, st>>>(a);
            break;
        case 3:
            if (f32) composite_kernel<VDI_MAX_PE, 3, VDI_PREC_F32><<<blocks, threads, 0, st>>>(a);
            else composite_kernel<VDI_MAX_PE, 3, VDI_PREC_F16><<<blocks, threads, 0, st>>>(a);
            break;
        default:
            if (f32) composite_kernel<VDI_MAX_PE, 2, VDI_PREC_F32><<<blocks, threads, 0, st>>>(a);
            else composite_kernel<VDI_MAX_PE, 2, VDI_PREC_F16><<<blocks, threads, 0, st>>>(a);
            break;
    }
    return cuda_check(cudaGetLastError(), "composite_kernel launch");
}

// Device table: [BatchHeader][ReqDev x n][PeIn x sum k]
struct BatchHeader {
    uint32_t n, total_items, total_pes, prec_in;
    uint64_t reqs_off, pes_off;
};

size_t batch_table_bytes(const vdi_request* reqs, int n) {
    size_t pes = 0;
    for (int r = 0; r < n; ++r) pes += (size_t)reqs[r].k;
    return align_up(sizeof(BatchHeader), 64) + align_up(sizeof(ReqDev) * (size_t)n, 64) + sizeof(PeIn) * pes;
}

vdi_status batch_table_pack(const vdi_request* reqs, int n, void* host_table, size_t bytes) {
    if (bytes < batch_table_bytes(reqs, n)) return set_error(VDI_ERR_INVALID_ARG, "batch table: buffer too small");
    char* base = static_cast<char*>(host_table);
    BatchHeader* hd = reinterpret_cast<BatchHeader*>(base);
    hd->reqs_off = align_up(sizeof(BatchHeader), 64);
    hd->pes_off = hd->reqs_off + align_up(sizeof(ReqDev) * (size_t)n, 64);
    ReqDev* rd = reinterpret_cast<ReqDev*>(base + hd->reqs_off);
    PeIn* pd = reinterpret_cast<PeIn*>(base + hd->pes_off);
    uint64_t items = 0, pes = 0;
    for (int r = 0; r < n; ++r) {
        const vdi_request& q = reqs[r];
        rd[r].out = out_dev(&q.out);
        rd[r].npix = (uint32_t)((uint64_t)q.w * (uint64_t)q.h);
        rd[r].item_begin = (uint32_t)items;
        rd[r].pe_begin = (uint32_t)pes;
        rd[r].k = q.k;
        rd[r].schedule = (q.schedule == 0 || (q.schedule == 1 && q.k > 8)) ? default_schedule(q.k) : q.schedule;
        for (int e = 0; e < q.k; ++e) {
            pd[pes + e].counts = q.pe[e].counts;
            pd[pes + e].offsets = q.pe[e].offsets;
            pd[pes + e].rgba = q.pe[e].rgba;
            pd[pes + e].fb = reinterpret_cast<const float2*>(q.pe[e].fb);
        }
        pes += (uint64_t)q.k;
        items += ((uint64_t)rd[r].npix + kBatchTile - 1) / kBatchTile;
    }
    if (items > 0xFFFFFFFFull) return set_error(VDI_ERR_INVALID_ARG, "batch table: too many work items");
    hd->n = (uint32_t)n;
    hd->total_items = (uint32_t)items;
    hd->total_pes = (uint32_t)pes;
    hd->prec_in = n > 0 ? (uint32_t)reqs[0].pe[0].prec : 0u;
    return VDI_OK;
}

vdi_status launch_composite_batched(const void* dev_table, const void* host_table, int iters, unsigned int* counter,
                                    unsigned int* status, int device_sms, cudaStream_t st) {
    const BatchHeader* hd = static_cast<const BatchHeader*>(host_table);
    if (hd->n == 0 || hd->total_items == 0) return VDI_OK;
    BatchArgs a;
    a.reqs = reinterpret_cast<const ReqDev*>(static_cast<const char*>(dev_table) + hd->reqs_off);
    a.pes = reinterpret_cast<const PeIn*>(static_cast<const char*>(dev_table) + hd->pes_off);
    a.n = (int)hd->n;
    a.total_items = hd->total_items;
    a.counter = counter;
    a.status = status;
    a.iters = iters;
    int per_sm = 1;
    cudaError_t e;
    if (hd->prec_in == VDI_PREC_F32)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, composite_batched_kernel<VDI_PREC_F32>, kBatchTile, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, composite_batched_kernel<VDI_PREC_F16>, kBatchTile, 0);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    unsigned blocks = (unsigned)(device_sms * per_sm);
    if (blocks > hd->total_items) blocks = hd->total_items;
    if (hd->prec_in == VDI_PREC_F32) composite_batched_kernel<VDI_PREC_F32><<<blocks, kBatchTile, 0, st>>>(a);
    else composite_batched_kernel<VDI_PREC_F16><<<blocks, kBatchTile, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "composite_batched_kernel launch");
}

}  // namespace vdi
