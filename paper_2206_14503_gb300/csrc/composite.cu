// Phase 2: compositing of K compact sub-VDIs into one regular VDI (sec. 5.2,
// Eq. 2, Algorithm S1).
//
// The paper's all-to-all exchange becomes a gather: pixel p's input is its K
// spans [offsets_e[p], offsets_e[p] + counts_e[p]) in the K PEs' record
// arrays.  A depth sweep over the K lists (each depth-sorted, sec. 5.2) cuts
// the records at every front and back depth and yields the pieces in order:
//   - a gap between records: a transparent sample;
//   - an interval covered by one record whole: that record, unchanged;
//   - part of one record: opacity by Eq. 2, 1 - (1 - A)^(dt / l);
//   - an interval covered by several records: their emission-absorption
//     mixture (extinctions add; colour is the extinction-weighted mean), summed
//     exactly in 128-bit fixed point so that every schedule gets the same bits.
// The pieces feed the supersegment state machine (Eq. 1) inside the per-pixel
// bisection search for gamma: a march evaluates the next two bisection levels
// at once (midpoint and both children) and records, per candidate, the
// interval of gamma over which all of its decisions repeat; the sequential
// bisection is replayed from the recorded counts, marching again only for a
// midpoint no record covers, so the result is that of plain bisection.  The
// first march also counts non-transparent pieces (the count at gamma = 0).  A
// final sweep emits at most n_s supersegments into the regular layout with a
// zero tail.
//
// Schedules (the same result, bit for bit; chosen per request by the
// autotuner, vdi_composite_autotune; the default is the lane schedule for
// K <= 8 and the staged one above):
//   VDI_SCHED_LANE (5, K <= 8): composite_lane_kernel copies a warp's 32
//     pixels' records into shared memory with asynchronous coalesced copies
//     and sweeps each pixel there once (a lane each; depth-disjoint lists, as
//     every box decomposition gives, without the K-head merge): the pixels
//     whose gamma = 0 count is within n_s are emitted, the others' pieces go
//     to a pool in the workspace; the list of those pixels is sorted by piece
//     count (list_hist / list_offsets / list_scatter) and
//     composite_flat_kernel searches and emits them;
//   VDI_SCHED_STAGED (4): composite_build_kernel builds each pixel's pieces
//     with the whole warp (coalesced span loads, merge-path sort of the bounds,
//     exact prefix scan of the mixture terms) into the pool, and
//     composite_flat_kernel searches and emits every pixel; the host runs the
//     pixels in chunks whose pieces fit the pool;
//   both list pixels they cannot stage (more than 480 / 1024 records, pieces
//     beyond the pool, lists out of depth order) for composite_marked_kernel,
//     the direct sweep;
//   1, 2, 3 (direct, composite_kernel): one thread per pixel re-sweeps its K
//     lists on every march, heads in registers (1, K <= 8) or in shared memory
//     under a winner tree (2; 3 with three levels per march).
// composite_flat_kernel runs the search and the emission as one loop whose
// body handles one piece of a lane's current march, so lanes at different
// marches or pixels execute the same instructions; lanes at the end of a
// march wait for others to end theirs together, and a lane that finishes its
// pixel takes the next one.
//
// The batched path runs many requests (different sizes, K, N_S) as the pooled
// staged schedule does: composite_batched_build_kernel pulls (request, 32-pixel
// batch) items from an atomic counter and builds them into the pool,
// composite_batched_flat_kernel searches and emits, and requests with a direct
// schedule (and pixels the stage cannot hold) go to
// composite_batched_marked_kernel.
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

// A record's premultiplied colour and opacity, and its optical depth tau =
// -log2(1 - A): computed from A for FP32 records, stored for FP16 ones.  A
// record is opaque iff tau is not finite (A >= 1 for FP32 records).
struct RecC {
    float4 c;
    float tau;
};

template <int PREC>
__device__ __forceinline__ RecC load_rec(const PeIn& pe, uint64_t idx) {
    RecC r;
    if (PREC == VDI_PREC_F32) {
        r.c = __ldg(reinterpret_cast<const float4*>(pe.rgba) + idx);
        r.tau = -lg2_approx(__fsub_rn(1.f, r.c.w));
    } else {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const uint4*>(pe.rgba) + idx) + 1);
        f16_unpack_col(v, r.c, r.tau);
    }
    return r;
}

__device__ __forceinline__ bool rec_opaque(const RecC& r) { return !(r.tau < INFINITY); }

// ---------------------------------------------------------------------------
// Piece sweep
// ---------------------------------------------------------------------------
// The pieces of a pixel are the intervals between consecutive distinct record
// bounds of its K lists.  A sweep keeps one head per PE (its current record)
// and processes the bounds in depth order as events: a record's front starts
// it, its back ends it and moves the head to the PE's next record with b > f.
// The emission-absorption mixture of the active records is kept as exact
// running sums, updated once per event: the extinction mu = -log2(1 - A) / l
// and mu times the unpremultiplied colour of every non-opaque record are
// summed in 128-bit fixed point (64 integer and 64 fraction bits; a record's
// terms are computed the same way at its start and at its end, so the sum of
// the active records is exact however many events came before).  Opaque
// records (A >= 1) are counted, with their colours summed.

struct U128 {
    unsigned long long hi, lo;
};

__device__ __forceinline__ void u128_add(U128& s, const U128& x) {
    const unsigned long long lo = s.lo + x.lo;
    s.hi += x.hi + (lo < s.lo ? 1ull : 0ull);
    s.lo = lo;
}

__device__ __forceinline__ void u128_sub(U128& s, const U128& x) {
    const unsigned long long lo = s.lo - x.lo;
    s.hi -= x.hi + (s.lo < x.lo ? 1ull : 0ull);
    s.lo = lo;
}

// v in [0, 2^56] as fixed point: exact for v >= 2^-41 (the 24-bit significand
// fits in the 64 fraction bits), truncated below
__device__ __forceinline__ U128 to_fixed(float v) {
    const float ip = truncf(v);
    U128 r;
    r.hi = __float2ull_rz(ip);
    r.lo = __float2ull_rz(__fmul_rn(__fsub_rn(v, ip), 18446744073709551616.f));
    return r;
}

__device__ __forceinline__ float from_fixed(const U128& s) {
    return __fmaf_rn(__ull2float_rn(s.lo), 5.421010862427522e-20f, __ull2float_rn(s.hi));
}

// Clamp of a record's extinction terms (per unit depth): a record shorter than
// ~3e-16 depth units with non-zero opacity is treated as having mu = 2^56, so
// that 64 PEs' sums stay below 2^64.
constexpr float kMuMax = 72057594037927936.f;  // 2^56

// A record's terms: extinction mu = -log2(1 - A) / (b - f) and mu times the
// unpremultiplied colour (non-opaque records), or its colour (opaque records).
struct Contrib {
    U128 M, MC[3], OC[3];
    int op;  // 1 if opaque
};

__device__ __forceinline__ void u128_zero(U128& x) { x.hi = x.lo = 0ull; }

__device__ __forceinline__ Contrib contrib(const RecC& x, float f, float b) {
    Contrib r;
    u128_zero(r.M);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        u128_zero(r.MC[q]);
        u128_zero(r.OC[q]);
    }
    r.op = 0;
    const float4& c = x.c;
    const float col[3] = {c.x, c.y, c.z};
    if (rec_opaque(x)) {
        r.op = 1;
#pragma unroll
        for (int q = 0; q < 3; ++q) r.OC[q] = to_fixed(fminf(fmaxf(col[q], 0.f), kMuMax));
    } else if (c.w > 0.f) {
        const float ia = rcp_approx(c.w);
        const float mu = fminf(__fmul_rn(x.tau, rcp_approx(__fsub_rn(b, f))), kMuMax);
        r.M = to_fixed(mu);
#pragma unroll
        for (int q = 0; q < 3; ++q) r.MC[q] = to_fixed(fminf(fmaxf(__fmul_rn(mu, __fmul_rn(col[q], ia)), 0.f), kMuMax));
    }
    return r;
}

// Sums over the active records.
struct MixSums {
    U128 M, MC[3], OC[3];
    int nop, nact;
};

__device__ __forceinline__ void sums_reset(MixSums& m) {
    u128_zero(m.M);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        u128_zero(m.MC[q]);
        u128_zero(m.OC[q]);
    }
    m.nop = m.nact = 0;
}

// OPQ = false: the caller knows that no record is opaque (the OC sums stay 0)
template <bool ADD, bool OPQ = true>
__device__ __forceinline__ void sums_update(MixSums& m, const Contrib& x) {
    if (ADD) {
        u128_add(m.M, x.M);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            u128_add(m.MC[q], x.MC[q]);
            if (OPQ) u128_add(m.OC[q], x.OC[q]);
        }
        m.nop += x.op;
        ++m.nact;
    } else {
        u128_sub(m.M, x.M);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            u128_sub(m.MC[q], x.MC[q]);
            if (OPQ) u128_sub(m.OC[q], x.OC[q]);
        }
        m.nop -= x.op;
        --m.nact;
    }
}

// The piece [t, t1] of an active set with sums m; `whole` when exactly one
// record is active and it spans [t, t1] (its colour and opacity are wc).
__device__ __forceinline__ void piece_from(const MixSums& m, bool whole, const RecC& wr, float t, float t1,
                                           Piece& x) {
    x.f = t;
    x.b = t1;
    if (whole) {
        // one record covering the piece exactly: the record itself
        x.P[0] = wr.c.x;
        x.P[1] = wr.c.y;
        x.P[2] = wr.c.z;
        x.a = wr.c.w;
        x.lgT = -wr.tau;
        return;
    }
    if (m.nop > 0) {
        // opaque records: the mean of their colours
        const float inv = 1.f / (float)m.nop;
        x.a = 1.f;
#pragma unroll
        for (int q = 0; q < 3; ++q) x.P[q] = __fmul_rn(from_fixed(m.OC[q]), inv);
        x.lgT = -INFINITY;
        return;
    }
    const float M = m.nact > 0 ? from_fixed(m.M) : 0.f;
    if (M > 0.f) {
        // emission-absorption mixture (Eq. 2 when one record covers the piece in part)
        x.lgT = -__fmul_rn(M, __fsub_rn(t1, t));
        x.a = __fsub_rn(1.f, ex2_approx(x.lgT));
        const float s = __fmul_rn(x.a, rcp_approx(M));
#pragma unroll
        for (int q = 0; q < 3; ++q) x.P[q] = __fmul_rn(from_fixed(m.MC[q]), s);
    } else {
        // a gap, or only fully transparent records
        x.P[0] = x.P[1] = x.P[2] = 0.f;
        x.a = 0.f;
        x.lgT = 0.f;
    }
}

// Direct sweeps: the sums plus the record started last (for the whole-record case).
struct Mix {
    MixSums s;
    float lt_f, lt_b;  // bounds of the record started last
    RecC lt_c;         // and its colour, opacity and optical depth
};

__device__ __forceinline__ void mix_reset(Mix& m) {
    sums_reset(m.s);
    m.lt_f = m.lt_b = -1.f;
    m.lt_c.c = make_float4(0.f, 0.f, 0.f, 0.f);
    m.lt_c.tau = 0.f;
}

__device__ __forceinline__ void mix_piece(const Mix& m, float t, float t1, Piece& x) {
    piece_from(m.s, m.s.nact == 1 && m.lt_f == t && m.lt_b == t1, m.lt_c, t, t1, x);
}

__device__ __forceinline__ void mix_start(Mix& m, const RecC& c, float f, float b) {
    sums_update<true>(m.s, contrib(c, f, b));
    m.lt_f = f;
    m.lt_b = b;
    m.lt_c = c;
}

__device__ __forceinline__ void mix_end(Mix& m, const RecC& c, float f, float b) {
    sums_update<false>(m.s, contrib(c, f, b));
}

constexpr float kNoEvent = 3.0e38f;

// Heads in registers (K <= KMAX, fully unrolled; KMAX <= 8).
template <int KMAX>
struct RegHeads {
    uint64_t cur[KMAX];
    uint32_t rem[KMAX];
    float hf[KMAX], hb[KMAX];
};

// advance PE e's head to its next record with b > f (records with b <= f are ignored)
template <int KMAX, int PREC>
__device__ __forceinline__ void reg_next_valid(const PeIn* pe, RegHeads<KMAX>& h, int e) {
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


struct ActiveRec {
    uint64_t cur;
    float f, b;
    int e;
};

// The piece [t, t1] covered by the n active records ar: the opaque records'
// colour sum if any is opaque, else the extinction sums (each in exact fixed
// point, as the running sums of the other sweeps).
template <int PREC>
__device__ __forceinline__ void mixture_piece(const PeIn* pe, const ActiveRec* ar, int n, float t, float t1,
                                              Piece& x) {
    MixSums m;
    sums_reset(m);
    m.nact = n;
    for (int i = 0; i < n; ++i) {
        if (rec_opaque(load_rec<PREC>(pe[ar[i].e], ar[i].cur))) ++m.nop;
    }
    if (m.nop > 0) {
        for (int i = 0; i < n; ++i) {
            const RecC r = load_rec<PREC>(pe[ar[i].e], ar[i].cur);
            if (rec_opaque(r)) {
                const float col[3] = {r.c.x, r.c.y, r.c.z};
#pragma unroll
                for (int q = 0; q < 3; ++q) u128_add(m.OC[q], to_fixed(fminf(fmaxf(col[q], 0.f), kMuMax)));
            }
        }
    } else {
        for (int i = 0; i < n; ++i) {
            const Contrib c = contrib(load_rec<PREC>(pe[ar[i].e], ar[i].cur), ar[i].f, ar[i].b);
            u128_add(m.M, c.M);
#pragma unroll
            for (int q = 0; q < 3; ++q) u128_add(m.MC[q], c.MC[q]);
        }
    }
    piece_from(m, false, RecC{make_float4(0.f, 0.f, 0.f, 0.f), 0.f}, t, t1, x);
}

// Calls visit(piece) for every piece of one pixel in depth order; returns the
// number of pieces.  The heads' bounds give each piece; the mixture sums of a
// piece covered by several records (or part of one) are summed from its
// active records (exactly, so the result equals the running sums of the other
// sweeps), which costs nothing for the common piece that is a whole record
// or a gap.
template <int KMAX, int PREC, typename V>
__device__ __forceinline__ int sweep_reg(const PeIn* pe, int k, const uint32_t* cnt0, const uint64_t* off0, V& visit) {
    RegHeads<KMAX> h;
    float t = kNoEvent;
#pragma unroll
    for (int e = 0; e < KMAX; ++e) {
        h.rem[e] = 0;
        if (e < k) {
            h.cur[e] = off0[e];
            h.rem[e] = cnt0[e];
            reg_next_valid<KMAX, PREC>(pe, h, e);
            if (h.rem[e] > 0) t = fminf(t, h.hf[e]);
        }
    }
    int npieces = 0;
    while (true) {
        float t1 = kNoEvent;
        int nact = 0, last = 0;
        unsigned act = 0u;
#pragma unroll
        for (int e = 0; e < KMAX; ++e) {
            if (e < k && h.rem[e] > 0) {
                if (h.hf[e] <= t) {
                    ++nact;
                    last = e;
                    act |= 1u << e;
                    t1 = fminf(t1, h.hb[e]);
                } else {
                    t1 = fminf(t1, h.hf[e]);
                }
            }
        }
        if (t1 >= kNoEvent) break;
        Piece x;
        if (nact == 0) {
            x.f = t;
            x.b = t1;
            x.P[0] = x.P[1] = x.P[2] = 0.f;
            x.a = 0.f;
            x.lgT = 0.f;
        } else {
            float lf = 0.f, lb = 0.f;
            uint64_t lc = 0;
#pragma unroll
            for (int e = 0; e < KMAX; ++e) {
                if (e == last) {
                    lf = h.hf[e];
                    lb = h.hb[e];
                    lc = h.cur[e];
                }
            }
            if (nact == 1 && lf == t && lb == t1) {
                MixSums m;
                sums_reset(m);
                piece_from(m, true, load_rec<PREC>(pe[last], lc), t, t1, x);
            } else {
                ActiveRec ar[KMAX];
                int na = 0;
#pragma unroll
                for (int e = 0; e < KMAX; ++e) {
                    if ((act >> e) & 1u) {
                        ar[na].cur = h.cur[e];
                        ar[na].f = h.hf[e];
                        ar[na].b = h.hb[e];
                        ar[na].e = e;
                        ++na;
                    }
                }
                mixture_piece<PREC>(pe, ar, na, t, t1, x);
            }
        }
        visit(x);
        ++npieces;
        // advance the heads that end at t1
#pragma unroll
        for (int e = 0; e < KMAX; ++e) {
            if (((act >> e) & 1u) && h.hb[e] <= t1) {
                ++h.cur[e];
                --h.rem[e];
                reg_next_valid<KMAX, PREC>(pe, h, e);
            }
        }
        t = t1;
    }
    return npieces;
}

// Heads in shared memory with a winner tree over P leaves (K <= P <= 64), one
// lane's arrays interleaved with its warp's other lanes (element i of lane l
// at word i * 32 + l), so that every access is free of bank conflicts.
template <int P>
struct SmemHeads {
    float* key;      // next event depth of each head (kNoEvent when exhausted)
    float* oth;      // the other bound of the head's record
    uint32_t* pos;   // record index within the PE's list; top bit: record active
    uint32_t* node;  // node[n], 1 <= n < P: winning head of the subtree n
    __device__ __forceinline__ float& K(int i) const { return key[i * 32]; }
    __device__ __forceinline__ float& O(int i) const { return oth[i * 32]; }
    __device__ __forceinline__ uint32_t& S(int i) const { return pos[i * 32]; }
    __device__ __forceinline__ uint32_t& N(int i) const { return node[i * 32]; }
};

constexpr uint32_t kActive = 0x80000000u;

// words of dynamic shared memory per thread for P leaves
template <int P>
constexpr int smem_words_per_thread() {
    return 4 * P;
}

template <int P>
__device__ __forceinline__ SmemHeads<P> smem_heads(uint32_t* smem) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* base = smem + (size_t)warp * (4 * P * 32) + lane;
    SmemHeads<P> h;
    h.key = reinterpret_cast<float*>(base);
    h.oth = reinterpret_cast<float*>(base + P * 32);
    h.pos = base + 2 * P * 32;
    h.node = base + 3 * P * 32;
    return h;
}

template <int P>
__device__ __forceinline__ int tree_winner_of(const SmemHeads<P>& h, int n) {
    return n >= P ? n - P : (int)h.N(n);
}

// recompute the winners on the path from leaf e to the root
template <int P>
__device__ __forceinline__ void tree_update(const SmemHeads<P>& h, int e) {
    int c = P + e;
    int w = e;
    float kw = h.K(e);
#pragma unroll
    for (int lev = 0; lev < 6; ++lev) {
        if ((P >> lev) <= 1) break;
        const int ws = tree_winner_of(h, c ^ 1);
        const float ks = h.K(ws);
        if (ks < kw || (ks == kw && ws < w)) {
            w = ws;
            kw = ks;
        }
        c >>= 1;
        h.N(c) = (uint32_t)w;
    }
}

template <int P>
__device__ __forceinline__ void tree_build(const SmemHeads<P>& h) {
    for (int n = P - 1; n >= 1; --n) {
        const int a = tree_winner_of(h, 2 * n), b = tree_winner_of(h, 2 * n + 1);
        const float ka = h.K(a), kb = h.K(b);
        h.N(n) = (uint32_t)((kb < ka || (kb == ka && b < a)) ? b : a);
    }
}

// move head e to its first record at or after index j with b > f
template <int P, int PREC>
__device__ __forceinline__ void smem_seek(const SmemHeads<P>& h, const PeIn& pe, uint32_t p, int e, uint32_t j) {
    const uint32_t cnt = __ldg(pe.counts + p);
    const uint64_t base = __ldg(pe.offsets + p);
    while (j < cnt) {
        float f, b;
        load_fb<PREC>(pe, base + j, f, b);
        if (b > f) {
            h.K(e) = f;
            h.O(e) = b;
            h.S(e) = j;
            return;
        }
        ++j;
    }
    h.K(e) = kNoEvent;
    h.S(e) = j;
}

template <int P, int PREC, typename V>
__device__ __forceinline__ int sweep_smem(const PeIn* pe, int k, uint32_t p, const SmemHeads<P>& h, V& visit) {
    for (int e = 0; e < P; ++e) {
        if (e < k) smem_seek<P, PREC>(h, pe[e], p, e, 0u);
        else h.K(e) = kNoEvent;
    }
    tree_build<P>(h);
    Mix m;
    mix_reset(m);
    int npieces = 0;
    float t = h.K(h.N(1));
    while (t < kNoEvent) {
        // events at depth t, in ascending PE order (the tree breaks ties by index)
        float t1;
        while (true) {
            const int e = (int)h.N(1);
            t1 = h.K(e);
            if (t1 != t) break;
            const uint32_t s = h.S(e);
            const uint32_t j = s & ~kActive;
            const RecC c = load_rec<PREC>(pe[e], __ldg(pe[e].offsets + p) + j);
            if (!(s & kActive)) {
                const float b = h.O(e);
                mix_start(m, c, t, b);
                h.K(e) = b;
                h.O(e) = t;
                h.S(e) = s | kActive;
            } else {
                mix_end(m, c, h.O(e), t);
                smem_seek<P, PREC>(h, pe[e], p, e, j + 1);
            }
            tree_update<P>(h, e);
        }
        if (t1 >= kNoEvent) break;
        Piece x;
        mix_piece(m, t, t1, x);
        visit(x);
        ++npieces;
        t = t1;
    }
    return npieces;
}

// Work census of the compositing kernels (VDI_FLAG_CENSUS).
struct CompCensus {
    unsigned long long pixels = 0, searched = 0, sweeps = 0, pieces = 0, cand_steps = 0, records = 0,
                       table_hits = 0;
};

// Counting state of one gamma candidate over pieces of arbitrary length.
struct CompCount {
    float P[3], A, L2, fS, bS;
    int cnt;
    bool open;
};

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

// cq_step written without branches: every outcome
// is computed with the same rounded operations and selected, so the decisions
// are bit for bit those of the branchy steps, and a visitor's candidates form
// straight-line code whose dependency chains interleave.
struct StepSel {
    bool fresh, close;
};

// A step that neither opens S (fresh) nor absorbs into it leaves S closed, and the colour, opacity,
// optical depth and bounds of a closed S are never read again (the next fresh piece overwrites all of
// them), so those steps may take the absorbing form as well: one select per value instead of two.
template <typename S>
__device__ __forceinline__ void apply_step(S& s, const Piece& x, StepSel d) {
    const float T = __fsub_rn(1.f, s.A);
#pragma unroll
    for (int c = 0; c < 3; ++c) s.P[c] = d.fresh ? x.P[c] : __fmaf_rn(T, x.P[c], s.P[c]);
    s.A = d.fresh ? x.a : __fmaf_rn(T, x.a, s.A);
    s.L2 = d.fresh ? x.lgT : __fadd_rn(s.L2, x.lgT);
    s.fS = d.fresh ? x.f : s.fS;
    s.bS = x.b;
    s.open = d.fresh || (s.open && !d.close);
    s.cnt += d.fresh ? 1 : 0;
}

template <typename S>
__device__ __forceinline__ float piece_ratio(const S& s, const Piece& x) {
    const float lx = __fsub_rn(x.b, x.f), lS = __fsub_rn(s.bS, s.fS);
    return (lx > 0.f && lS > 0.f) ? __fmul_rn(lx, rcp_approx(lS)) : 1.f;
}

__device__ __forceinline__ void cq_step_select(CompCountQ& s, const Piece& x, float g2) {
    float q = 0.f;
    const bool crit = s.open && criterion_q(s.P, s.A, s.L2, piece_ratio(s, x), x.P, g2, q);
    s.qhi = crit ? fminf(s.qhi, q) : s.qhi;               // crit implies an open S
    s.qlo = (s.open && !crit) ? fmaxf(s.qlo, q) : s.qlo;
    const bool opaque = x.a > 0.f;
    apply_step(s, x, StepSel{opaque && (!s.open || crit), crit && !opaque});
}

// SELECT: the branch-free steps (faster where the pieces come from the staged
// buffer, 2.46 vs 2.76 s at 2048^2, K = 32; slower in the direct sweepers, 8.1
// vs 7.5 ms on the 512^3 frame, whose piece generation interleaves with them)
template <int NC, bool SELECT>
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
        for (int c = 0; c < NC; ++c) {
            if constexpr (SELECT) cq_step_select(st[c], x, g2[c]);
            else cq_step(st[c], x, g2[c]);
        }
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

    // L2 = log2(1 - A), the record's optical depth (stored by the FP16 form)
    __device__ __forceinline__ void store(float f, float b, const float P[3], float A, float L2) {
        size_t idx = base + written;
        if (out->prec == VDI_PREC_F32) {
            reinterpret_cast<float4*>(out->rgba)[idx] = make_float4(P[0], P[1], P[2], A);
            out->fb[idx] = make_float2(f, b);
        } else {
            reinterpret_cast<uint4*>(out->rgba)[idx] = f16_pack(f, b, P[0], P[1], P[2], L2);
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
            if (written < cap) store(s.fS, bt, s.P, s.A, s.L2);
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

// One pixel's sweeps: heads in registers (KMAX > 0, K <= KMAX) or in shared
// memory with P leaves (KMAX == 0, K <= P).
template <int KMAX, int P, int PREC>
struct Sweeper {
    static constexpr bool kSelectSteps = false;  // counting steps with branches (see CountVisitorQ)
    const PeIn* pe;
    int k;
    uint32_t p;
    uint32_t cnt0[KMAX > 0 ? KMAX : 1];
    uint64_t off0[KMAX > 0 ? KMAX : 1];
    SmemHeads<P> sh;

    __device__ __forceinline__ void init(const PeIn* pe_, int k_, uint32_t p_, uint32_t* smem) {
        pe = pe_;
        k = k_;
        p = p_;
        if constexpr (KMAX > 0) {
#pragma unroll
            for (int e = 0; e < KMAX; ++e) {
                if (e < k) {
                    cnt0[e] = __ldg(pe[e].counts + p);
                    off0[e] = __ldg(pe[e].offsets + p);
                }
            }
        } else {
            sh = smem_heads<P>(smem);
        }
    }
    __device__ __forceinline__ unsigned long long records() const {
        unsigned long long n = 0;
        for (int e = 0; e < k; ++e) n += __ldg(pe[e].counts + p);
        return n;
    }
    template <typename V>
    __device__ __forceinline__ int run(V& v) {
        if constexpr (KMAX > 0) return sweep_reg<KMAX, PREC>(pe, k, cnt0, off0, v);
        else return sweep_smem<P, PREC>(pe, k, p, sh, v);
    }
};

// The whole per-pixel composite: search, emission, zero tail.
// The whole per-pixel composite over the pieces that sw.run(visit) produces:
// search, emission, zero tail.
template <int NLEV, bool CENSUS, typename SW>
__device__ __forceinline__ void composite_search_emit(SW& sw, const OutDev& out, int iters, unsigned int* status,
                                                      uint32_t p, CompCensus* cs) {
    constexpr int NC = (1 << NLEV) - 1;
    // search (sec. 2.4 applied to the pieces, sec. 5.2): sequential bisection;
    // a midpoint's count comes from the table of earlier marches when one of
    // their decision intervals holds it, else from a march over the NLEV-level
    // subtree below the current bracket.
    float gamma = 0.f;
    int count;
    {
        CountTable t;
        t.n = 0;
        CountVisitorQ<NC, SW::kSelectSteps> v;
        float g[NC];
        v.reset();
        tree_candidates<NLEV>(0.f, 2.f, g);
#pragma unroll
        for (int q = 0; q < NC; ++q) v.g2[q] = __fmul_rn(g[q], g[q]);
        {
            const int np = sw.run(v);
            if (CENSUS) {
                cs->sweeps += 1;
                cs->pieces += (unsigned long long)np;
                cs->cand_steps += (unsigned long long)np * NC;
            }
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) t.add(v.g2[q], v.st[q].qlo, v.st[q].qhi, v.st[q].cnt);
        if (v.nt <= out.n_s) {
            count = v.nt;
        } else {
            if (CENSUS) cs->searched += 1;
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
                    const int np = sw.run(v);
                    if (CENSUS) {
                        cs->sweeps += 1;
                        cs->pieces += (unsigned long long)np;
                        cs->cand_steps += (unsigned long long)np * NC;
                    }
#pragma unroll
                    for (int q = 0; q < NC; ++q) t.add(v.g2[q], v.st[q].qlo, v.st[q].qhi, v.st[q].cnt);
                    c = v.st[0].cnt;
                } else if (CENSUS) {
                    cs->table_hits += 1;
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
    {
        const int np = sw.run(em);
        if (CENSUS) {
            cs->sweeps += 1;
            cs->pieces += (unsigned long long)np;
        }
    }
    if (em.s.open && em.written < out.n_s) em.store(em.s.fS, em.bt, em.s.P, em.s.A, em.s.L2);
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

// Direct path: the pieces are swept from the K lists on every march.
template <int KMAX, int P, int NLEV, int PREC, bool CENSUS = false>
__device__ __forceinline__ void composite_pixel(const PeIn* pe, int k, const OutDev& out, int iters,
                                                unsigned int* status, uint32_t p, uint32_t* smem,
                                                CompCensus* cs = nullptr) {
    Sweeper<KMAX, P, PREC> sw;
    sw.init(pe, k, p, smem);
    if (CENSUS) {
        cs->pixels += 1;
        cs->records += sw.records();
    }
    composite_search_emit<NLEV, CENSUS>(sw, out, iters, status, p, cs);
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void census_flush(const CompCensus& cs, unsigned long long* ctr) {
    const unsigned long long v[7] = {cs.pixels, cs.searched, cs.sweeps, cs.pieces, cs.cand_steps, cs.records,
                                     cs.table_hits};
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const unsigned long long w = warp_sum(v[i]);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(ctr + i, w);
    }
}

template <int KMAX, int P, int NLEV, int PREC, bool CENSUS>
__global__ void __launch_bounds__(128, NLEV > 2 ? 2 : 3) composite_kernel(const __grid_constant__ CompArgs a) {
    extern __shared__ uint32_t smem[];
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    CompCensus cs;
    if (p < (uint32_t)a.npix)
        composite_pixel<KMAX, P, NLEV, PREC, CENSUS>(a.pe, a.k, a.out, a.iters, a.status, p, smem, &cs);
    if (CENSUS) census_flush(cs, reinterpret_cast<WsHeader*>(a.status)->counters);
}


// ---------------------------------------------------------------------------
// Staged path
// ---------------------------------------------------------------------------
// A warp takes 32 consecutive pixels at a time.  Phase G builds the pieces of
// each of them in turn, the whole warp on one pixel: it loads the pixel's
// records from all K lists, drops those with b <= f, sorts their bounds (each
// list's bounds are already in order, so a stable merge of the K runs: log2 K
// rounds in which every bound finds its place in its partner run by binary
// search; ties go to the lower PE) and obtains the active set's sums after
// every bound by an exact prefix scan of the records' terms.  The pieces go to
// the warp's piece buffer, pixel i of the batch in column i.  Phase S: lane i
// runs the search and the emission of pixel i over column i.  The pieces are
// bit for bit those of the direct sweep.  Pixels with more records than the
// stage holds are listed for the direct path (a second launch).

constexpr int kStageRMax = 1024;           // records per pixel held by the stage
constexpr int kStageWarps = 8;             // warps per CTA

struct StageSmem {
    uint16_t pay[2][2 * kStageRMax];  // bounds: (valid record << 1) | is_back
    float2 rfb[kStageRMax];           // bounds of the valid records
    uint32_t rloc[kStageRMax];        // (PE << 16) | index in the PE's list, of the valid records
    uint32_t pref[VDI_MAX_PE + 1];    // records before PE e
    uint32_t vpref[VDI_MAX_PE + 1];   // valid records before PE e
    uint64_t off[VDI_MAX_PE];         // start of PE e's list for the pixel
};

__device__ __forceinline__ float bound_key(const StageSmem& S, uint32_t w) {
    const float2 fb = S.rfb[w >> 1];
    return (w & 1u) ? fb.y : fb.x;
}

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

__device__ __forceinline__ U128 shfl_up_u128(const U128& v, int d) {
    U128 r;
    r.hi = __shfl_up_sync(0xffffffffu, v.hi, d);
    r.lo = __shfl_up_sync(0xffffffffu, v.lo, d);
    return r;
}

// running state of the stage's scan
struct ScanState {
    MixSums s;
    uint32_t xr;   // xor of the active records' indices
    uint32_t nb;   // bounds followed by a larger one (pieces)
};

__device__ __forceinline__ void scan_reset(ScanState& a) {
    sums_reset(a.s);
    a.xr = 0u;
    a.nb = 0u;
}

// a + b (element-wise, modulo 2^128 for the sums)
template <bool OPQ>
__device__ __forceinline__ void scan_add(ScanState& a, const ScanState& b) {
    u128_add(a.s.M, b.s.M);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        u128_add(a.s.MC[q], b.s.MC[q]);
        if (OPQ) u128_add(a.s.OC[q], b.s.OC[q]);
    }
    a.s.nop += b.s.nop;
    a.s.nact += b.s.nact;
    a.xr ^= b.xr;
    a.nb += b.nb;
}

template <bool OPQ>
__device__ __forceinline__ ScanState shfl_up_state(const ScanState& v, int d) {
    ScanState r;
    r.s.M = shfl_up_u128(v.s.M, d);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        r.s.MC[q] = shfl_up_u128(v.s.MC[q], d);
        if (OPQ) r.s.OC[q] = shfl_up_u128(v.s.OC[q], d);
        else u128_zero(r.s.OC[q]);
    }
    r.s.nop = __shfl_up_sync(0xffffffffu, v.s.nop, d);
    r.s.nact = __shfl_up_sync(0xffffffffu, v.s.nact, d);
    r.xr = __shfl_up_sync(0xffffffffu, v.xr, d);
    r.nb = __shfl_up_sync(0xffffffffu, v.nb, d);
    return r;
}

// applies bound w (sorted position i) to the state
template <int PREC, bool OPQ>
__device__ __forceinline__ void stage_apply(const PeIn* pe, const StageSmem& S, uint32_t w, ScanState& a) {
    const uint32_t c = w >> 1;
    const uint32_t loc = S.rloc[c];
    const int e = (int)(loc >> 16);
    const float2 fb = S.rfb[c];
    const Contrib x = contrib(load_rec<PREC>(pe[e], S.off[e] + (loc & 0xFFFFu)), fb.x, fb.y);
    if (w & 1u) sums_update<false, OPQ>(a.s, x);
    else sums_update<true, OPQ>(a.s, x);
    a.xr ^= c;
}

// Where phase G writes a pixel's pieces: a column of a warp's piece buffer
// (rows 32 elements apart), or (POOL) a run of the pool allocated once the
// pixel's piece count is known; base receives the run's first piece, and a
// pixel whose run does not fit the pool gets npieces = -1 and no writes.
struct PoolRun {
    uint32_t* counter;
    uint32_t cap;
    uint32_t base;
};

// Phase G after the merge: exact prefix scan of the records' terms over the
// sorted bounds (srt, E of them; nv valid records), in contiguous chunks per
// lane, and the pieces written to the column (or the pool).
template <int PREC, bool OPQ, bool POOL = false>
__device__ __forceinline__ void stage_scan(const PeIn* pe, const StageSmem& S, const uint16_t* srt, uint32_t E,
                                           uint32_t nv, float4* colA, float2* colB, int& npieces, int& nt,
                                           float& f0, PoolRun* run = nullptr) {
    constexpr size_t kStride = POOL ? 1 : 32;
    const int lane = threadIdx.x & 31;
    // exact prefix scan of the records' terms over the sorted bounds, in
    // contiguous chunks per lane
    const uint32_t chunk = (E + 31) / 32;
    const uint32_t i0 = min(E, lane * chunk), i1 = min(E, i0 + chunk);
    ScanState loc;
    scan_reset(loc);
#pragma unroll 4
    for (uint32_t i = i0; i < i1; ++i) {
        stage_apply<PREC, OPQ>(pe, S, srt[i], loc);
        if (i + 1 < E && bound_key(S, srt[i]) < bound_key(S, srt[i + 1])) ++loc.nb;
    }
    // exclusive prefix of the lanes' totals
    ScanState inc = loc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const ScanState o = shfl_up_state<OPQ>(inc, d);
        if (lane >= d) {
            ScanState t = o;
            scan_add<OPQ>(t, inc);
            inc = t;
        }
    }
    ScanState st = shfl_up_state<OPQ>(inc, 1);
    if (lane == 0) scan_reset(st);
    const uint32_t total_pieces = __shfl_sync(0xffffffffu, inc.nb, 31);
    if constexpr (POOL) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(run->counter, total_pieces);
        base = __shfl_sync(0xffffffffu, base, 0);
        run->base = base;
        if ((uint64_t)base + total_pieces > (uint64_t)run->cap) {
            npieces = -1;
            nt = 0;
            f0 = 0.f;
            return;
        }
        colA += base;
        colB += base;
    }
    // the pieces: after bound i the active set is that of [key_i, key_{i+1}]
    int my_nt = 0;
    uint32_t row = st.nb;
    for (uint32_t i = i0; i < i1; ++i) {
        stage_apply<PREC, OPQ>(pe, S, srt[i], st);
        if (i + 1 >= E) break;
        const float t = bound_key(S, srt[i]), t1 = bound_key(S, srt[i + 1]);
        if (!(t < t1)) continue;
        bool whole = false;
        RecC wc{make_float4(0.f, 0.f, 0.f, 0.f), 0.f};
        if (st.s.nact == 1) {
            const uint32_t c = min(st.xr, nv - 1);
            const float2 fb = S.rfb[c];
            if (fb.x == t && fb.y == t1) {
                const uint32_t l = S.rloc[c];
                const int e = (int)(l >> 16);
                wc = load_rec<PREC>(pe[e], S.off[e] + (l & 0xFFFFu));
                whole = true;
            }
        }
        Piece x;
        piece_from(st.s, whole, wc, t, t1, x);
        colA[(size_t)row * kStride] = make_float4(x.P[0], x.P[1], x.P[2], x.a);
        colB[(size_t)row * kStride] = make_float2(x.b, x.lgT);
        my_nt += x.a > 0.f;
        ++row;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) my_nt += __shfl_xor_sync(0xffffffffu, my_nt, d);
    npieces = (int)total_pieces;
    nt = my_nt;
    f0 = bound_key(S, srt[0]);
}

// Phase G for pixel p into one column of the piece buffer (colA/colB point at
// row 0 of the column; rows are 32 elements apart).  Returns false when the
// pixel has more than kStageRMax records.
template <int PREC, bool POOL = false>
__device__ bool stage_pixel(const PeIn* pe, int k, uint32_t p, StageSmem& S, float4* colA, float2* colB, int rows,
                            int& npieces, int& nt, float& f0, PoolRun* run = nullptr) {
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    // counts and list starts, prefix over PEs
    uint32_t c0 = 0, c1 = 0;
    if (lane < k) {
        c0 = __ldg(pe[lane].counts + p);
        S.off[lane] = __ldg(pe[lane].offsets + p);
    }
    if (lane + 32 < k) {
        c1 = __ldg(pe[lane + 32].counts + p);
        S.off[lane + 32] = __ldg(pe[lane + 32].offsets + p);
    }
    const uint32_t x0 = warp_incl_scan_u32(c0);
    const uint32_t t0 = __shfl_sync(0xffffffffu, x0, 31);
    const uint32_t x1 = warp_incl_scan_u32(c1);
    const uint32_t R = t0 + __shfl_sync(0xffffffffu, x1, 31);
    S.pref[lane] = x0 - c0;
    S.pref[lane + 32] = t0 + x1 - c1;
    if (lane == 0) S.pref[VDI_MAX_PE] = R;
    __syncwarp();
    if (R > (uint32_t)kStageRMax) return false;
    // bounds of every record; the valid ones (b > f) compacted in list order
    uint32_t nv = 0;
    bool opaque = false;
    for (uint32_t r0 = 0; r0 < R; r0 += 32) {
        const uint32_t r = r0 + lane;
        bool valid = false;
        float f = 0.f, b = 0.f;
        int e = 0;
        uint32_t j = 0;
        if (r < R) {
            int lo = 0, hi = k - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (S.pref[mid] <= r) lo = mid;
                else hi = mid - 1;
            }
            e = lo;
            j = r - S.pref[e];
            load_fb<PREC>(pe[e], S.off[e] + j, f, b);
            valid = b > f;
            if (valid) opaque |= rec_opaque(load_rec<PREC>(pe[e], S.off[e] + j));
        }
        const unsigned m = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const uint32_t c = nv + __popc(m & lt_mask);
            S.rfb[c] = make_float2(f, b);
            S.rloc[c] = ((uint32_t)e << 16) | j;
        }
        nv += __popc(m);
    }
    __syncwarp();
    if (nv > 0 && 2 * nv - 1 > (uint32_t)rows) return false;  // more pieces than the column holds
    // each list must be in depth order (b of a record <= f of the next): else
    // the merge below would not be a permutation; such pixels go to the
    // direct path
    bool unsorted = false;
    for (uint32_t c = lane + 1; c < nv; c += 32)
        unsorted |= (S.rloc[c] >> 16) == (S.rloc[c - 1] >> 16) && !(S.rfb[c].x >= S.rfb[c - 1].y);
    if (__any_sync(0xffffffffu, unsorted)) return false;
    opaque = __any_sync(0xffffffffu, opaque);
    // valid records before PE e: the first compacted record of a PE >= e
    for (int e = lane; e <= k; e += 32) {
        uint32_t lo = 0, hi = nv;
        const uint32_t key = (uint32_t)e << 16;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (S.rloc[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        S.vpref[e] = lo;
    }
    const uint32_t E = 2 * nv;
    for (uint32_t i = lane; i < E; i += 32) S.pay[0][i] = (uint16_t)i;
    __syncwarp();
    if (E == 0) {
        npieces = 0;
        nt = 0;
        f0 = 0.f;
        return true;
    }
    // stable merge of the PEs' runs of bounds: round r merges the groups of
    // 2^r PEs pairwise (merge path: every lane takes an equal share of the
    // output, finds where it starts in the two runs by binary search and
    // merges sequentially from there; ties go to the lower run)
    int src = 0;
    for (int r = 0; (1 << r) < k; ++r) {
        const uint16_t* in = S.pay[src];
        uint16_t* outp = S.pay[src ^ 1];
        const int span = 2 << r;
        const int ngroups = (k + span - 1) / span;
        const uint32_t per = (E + 31) / 32;
        uint32_t o = min(E, (uint32_t)lane * per);
        const uint32_t o_end = min(E, o + per);
        while (o < o_end) {
            // the merged group holding output o: the last one starting at or before o
            int qlo = 0, qhi = ngroups - 1;
            while (qlo < qhi) {
                const int mid = (qlo + qhi + 1) >> 1;
                if (2u * S.vpref[mid * span] <= o) qlo = mid;
                else qhi = mid - 1;
            }
            const int e0 = qlo * span, em = min(e0 + (span >> 1), k), e1 = min(e0 + span, k);
            const uint32_t a0 = 2u * S.vpref[e0], b0 = 2u * S.vpref[em], b1 = 2u * S.vpref[e1];
            const uint32_t la = b0 - a0, lb = b1 - b0, d = o - a0;
            uint32_t lo = d > lb ? d - lb : 0u, hi = min(d, la);
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (bound_key(S, in[a0 + mid]) <= bound_key(S, in[b0 + d - mid - 1])) lo = mid + 1;
                else hi = mid;
            }
            uint32_t i = lo, j = d - lo;
            float ka = i < la ? bound_key(S, in[a0 + i]) : 0.f;
            float kb = j < lb ? bound_key(S, in[b0 + j]) : 0.f;
            const uint32_t stop = min(o_end, b1);
            for (; o < stop; ++o) {
                if (i < la && (j >= lb || ka <= kb)) {
                    outp[o] = in[a0 + i];
                    ++i;
                    if (i < la) ka = bound_key(S, in[a0 + i]);
                } else {
                    outp[o] = in[b0 + j];
                    ++j;
                    if (j < lb) kb = bound_key(S, in[b0 + j]);
                }
            }
        }
        src ^= 1;
        __syncwarp();
    }
    const uint16_t* srt = S.pay[src];
    if (opaque) stage_scan<PREC, true, POOL>(pe, S, srt, E, nv, colA, colB, npieces, nt, f0, run);
    else stage_scan<PREC, false, POOL>(pe, S, srt, E, nv, colA, colB, npieces, nt, f0, run);
    __syncwarp();
    return true;
}


// storage of the pieces of the pixels the lane and pooled staged paths search
struct PiecePool {
    float4* A;  // (P.rgb, a)
    float2* B;  // (b, log2(1 - a))
    uint32_t cap;
};

// list entry of a pixel for the flat search: pixel (top bit: composite it by the direct sweep), first
// piece in the pool, number of pieces, front of the first piece
struct FlatEntry {
    uint32_t p, base, n;
    float f0;
};

// ---------------------------------------------------------------------------
// Lane-staged path (short lists: K <= kLaneKMax).  Two passes.
//
// Batch pass (composite_lane_kernel): a warp takes 32 consecutive pixels,
// reads their counts and offsets (coalesced over the pixels) and copies their
// records into its shared-memory slab with asynchronous copies (cp.async:
// every copy of a round is in flight before the warp waits once), PE by PE:
// the spans of consecutive pixels of one PE are consecutive in the PE's record
// array (the layout generation writes), so the copies are coalesced 16- and
// 8-byte runs; other layouts find each record's pixel by a binary search over
// the lanes.  A lane sweeps its pixel's K lists in the slab into pieces and
// counts the non-transparent ones: at most n_s means gamma = 0 (sec. 2.4: the
// count at gamma = 0 is within the budget), and a second sweep emits the
// pixel's records straight away.  A pixel that needs the gamma search gets
// its pieces written, once, to a pool in the workspace and is listed.
//
// Search pass (composite_flat_kernel, below): the listed pixels' searches and
// emissions over their pooled pieces, a lane per pixel, lanes taking new
// pixels as they finish.  Pixels whose records exceed the slab, or whose
// pieces do not fit the pool, are listed for the direct sweep
// (composite_marked_kernel).  The pieces are those of every other schedule,
// bit for bit, so is the result.
// ---------------------------------------------------------------------------
constexpr int kLaneKMax = 8;        // PEs the lane path handles (heads in registers)
constexpr int kLaneWarps = 4;       // warps per CTA
constexpr int kLaneRCap = 480;      // records per warp slab

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// A warp's slab of CAP records: F32 as rgba[] then fb[], F16 as the raw
// 16-byte records.
template <int PREC, int CAP>
struct LaneSlab;
template <int CAP>
struct LaneSlab<VDI_PREC_F32, CAP> {
    float4 rgba[CAP];
    float2 fb[CAP];
    __device__ __forceinline__ float2 bounds(uint32_t i) const { return fb[i]; }
    __device__ __forceinline__ RecC rec(uint32_t i) const {
        RecC r;
        r.c = rgba[i];
        r.tau = -lg2_approx(__fsub_rn(1.f, r.c.w));
        return r;
    }
    __device__ __forceinline__ void copy(const PeIn& pe, uint64_t src, uint32_t dst) {
        cp_async16(rgba + dst, reinterpret_cast<const float4*>(pe.rgba) + src);
        cp_async8(fb + dst, pe.fb + src);
    }
};
template <int CAP>
struct LaneSlab<VDI_PREC_F16, CAP> {
    uint4 raw[CAP];
    __device__ __forceinline__ float2 bounds(uint32_t i) const {
        return make_float2(__uint_as_float(raw[i].x), __uint_as_float(raw[i].y));
    }
    __device__ __forceinline__ RecC rec(uint32_t i) const {
        RecC r;
        f16_unpack_col(make_uint2(raw[i].z, raw[i].w), r.c, r.tau);
        return r;
    }
    __device__ __forceinline__ void copy(const PeIn& pe, uint64_t src, uint32_t dst) {
        cp_async16(raw + dst, reinterpret_cast<const uint4*>(pe.rgba) + src);
    }
};

// moves a head to its next record with b > f (records with b <= f are ignored)
template <class SLAB>
__device__ __forceinline__ void slab_next_valid(const SLAB& S, uint32_t& cur, uint32_t& rem, float& hf, float& hb) {
    while (rem > 0) {
        const float2 fb = S.bounds(cur);
        if (fb.y > fb.x) {
            hf = fb.x;
            hb = fb.y;
            return;
        }
        ++cur;
        --rem;
    }
}

// The pieces of one pixel from its K lists in the slab (list e: slab entries
// [st[e], st[e] + cnt[e])), in depth order: the sweep of sweep_reg with the
// records read from shared memory.
template <class SLAB, typename V>
__device__ __forceinline__ int sweep_slab(const SLAB& S, int k, const uint32_t st[kLaneKMax],
                                          const uint32_t cnt[kLaneKMax], V& visit) {
    uint32_t cur[kLaneKMax], rem[kLaneKMax];
    float hf[kLaneKMax], hb[kLaneKMax];
    float t = kNoEvent;
#pragma unroll
    for (int e = 0; e < kLaneKMax; ++e) {
        rem[e] = 0;
        hf[e] = hb[e] = 0.f;
        cur[e] = 0;
        if (e < k) {
            cur[e] = st[e];
            rem[e] = cnt[e];
            slab_next_valid(S, cur[e], rem[e], hf[e], hb[e]);
            if (rem[e] > 0) t = fminf(t, hf[e]);
        }
    }
    int npieces = 0;
    while (true) {
        float t1 = kNoEvent;
        int nact = 0, last = 0;
        unsigned act = 0u;
#pragma unroll
        for (int e = 0; e < kLaneKMax; ++e) {
            if (e < k && rem[e] > 0) {
                if (hf[e] <= t) {
                    ++nact;
                    last = e;
                    act |= 1u << e;
                    t1 = fminf(t1, hb[e]);
                } else {
                    t1 = fminf(t1, hf[e]);
                }
            }
        }
        if (t1 >= kNoEvent) break;
        Piece x;
        if (nact == 0) {
            x.f = t;
            x.b = t1;
            x.P[0] = x.P[1] = x.P[2] = 0.f;
            x.a = 0.f;
            x.lgT = 0.f;
        } else {
            float lf = 0.f, lb = 0.f;
            uint32_t lc = 0;
#pragma unroll
            for (int e = 0; e < kLaneKMax; ++e) {
                if (e == last) {
                    lf = hf[e];
                    lb = hb[e];
                    lc = cur[e];
                }
            }
            MixSums m;
            sums_reset(m);
            if (nact == 1 && lf == t && lb == t1) {
                piece_from(m, true, S.rec(lc), t, t1, x);
            } else {
                // the active records' mixture, summed exactly (as mixture_piece)
                m.nact = nact;
#pragma unroll
                for (int e = 0; e < kLaneKMax; ++e)
                    if ((act >> e) & 1u) m.nop += rec_opaque(S.rec(cur[e])) ? 1 : 0;
                if (m.nop > 0) {
#pragma unroll
                    for (int e = 0; e < kLaneKMax; ++e) {
                        if ((act >> e) & 1u) {
                            const RecC r = S.rec(cur[e]);
                            if (rec_opaque(r)) {
                                const float col[3] = {r.c.x, r.c.y, r.c.z};
#pragma unroll
                                for (int q = 0; q < 3; ++q)
                                    u128_add(m.OC[q], to_fixed(fminf(fmaxf(col[q], 0.f), kMuMax)));
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < kLaneKMax; ++e) {
                        if ((act >> e) & 1u) {
                            const Contrib c = contrib(S.rec(cur[e]), hf[e], hb[e]);
                            u128_add(m.M, c.M);
#pragma unroll
                            for (int q = 0; q < 3; ++q) u128_add(m.MC[q], c.MC[q]);
                        }
                    }
                }
                piece_from(m, false, RecC{make_float4(0.f, 0.f, 0.f, 0.f), 0.f}, t, t1, x);
            }
        }
        visit(x);
        ++npieces;
#pragma unroll
        for (int e = 0; e < kLaneKMax; ++e) {
            if (((act >> e) & 1u) && hb[e] <= t1) {
                ++cur[e];
                --rem[e];
                slab_next_valid(S, cur[e], rem[e], hf[e], hb[e]);
            }
        }
        t = t1;
    }
    return npieces;
}

// One pixel's sweeps over the slab.  When the pixel's K lists are disjoint
// in depth -- each list sorted with
// non-overlapping records, and the PEs' depth ranges not overlapping (every
// convex decomposition gives such lists: a ray crosses each box in one
// stretch) -- no interval is covered by two records, so the pieces are the
// records themselves, in the order of the PEs' ranges, with a transparent gap
// piece wherever one record ends before the next begins: exactly the pieces
// the sweep would cut, without comparing K list heads per piece.  Other
// pixels take the sweep.
template <class SLAB>
struct SlabSweeper {
    static constexpr bool kSelectSteps = false;  // counting steps with branches (see CountVisitorQ)
    const SLAB* S;
    int k;
    uint32_t st[kLaneKMax], cnt[kLaneKMax];
    bool disjoint;
    uint32_t order;  // PEs by the front of their first record, 4 bits each
    int nonempty;    // PEs with a record of positive length
    int nvalid;      // records of positive length
    int nto;         // of them, those of positive opacity (the non-transparent pieces, if disjoint)

    __device__ __forceinline__ void prepare() {
        float lo[kLaneKMax], hi[kLaneKMax];
        bool ok = true;
        int nz = 0;
        nvalid = 0;
        nto = 0;
#pragma unroll
        for (int e = 0; e < kLaneKMax; ++e) {
            lo[e] = kNoEvent;
            hi[e] = -kNoEvent;
            if (e < k) {
                float prev = -kNoEvent;
                for (uint32_t r = st[e]; r < st[e] + cnt[e]; ++r) {
                    const float2 fb = S->bounds(r);
                    if (!(fb.y > fb.x)) continue;
                    ++nvalid;
                    nto += S->rec(r).c.w > 0.f;
                    ok = ok && fb.x >= prev;
                    prev = fb.y;
                    lo[e] = fminf(lo[e], fb.x);
                    hi[e] = fb.y;
                }
                nz += lo[e] < kNoEvent;
            }
        }
        // insertion sort of the PEs by their first front (ties by index, as the sweep's heads)
        uint32_t ord = 0;
        int n = 0;
#pragma unroll
        for (int e = 0; e < kLaneKMax; ++e) {
            if (e < k && lo[e] < kNoEvent) {
                int pos = n;
                while (pos > 0) {
                    const int q = (int)((ord >> (4 * (pos - 1))) & 15u);
                    float lq = lo[0];
#pragma unroll
                    for (int w = 1; w < kLaneKMax; ++w)
                        if (w == q) lq = lo[w];
                    if (!(lq > lo[e])) break;
                    const uint32_t sh = 4u * (uint32_t)pos;
                    ord = (ord & ~(15u << sh)) | ((uint32_t)q << sh);
                    --pos;
                }
                const uint32_t sh = 4u * (uint32_t)pos;
                ord = (ord & ~(15u << sh)) | ((uint32_t)e << sh);
                ++n;
            }
        }
        // consecutive ranges must not overlap
        float end = -kNoEvent;
        for (int i = 0; i < n; ++i) {
            const int e = (int)((ord >> (4 * i)) & 15u);
            float le = lo[0], he = hi[0];
#pragma unroll
            for (int w = 1; w < kLaneKMax; ++w)
                if (w == e) {
                    le = lo[w];
                    he = hi[w];
                }
            ok = ok && le >= end;
            end = he;
        }
        disjoint = ok;
        order = ord;
        nonempty = n;
    }

    template <typename V>
    __device__ __forceinline__ int run(V& v) const {
        if (!disjoint) return sweep_slab(*S, k, st, cnt, v);
        const int n = nonempty;
        int np = 0;
        float t = 0.f;
        bool first = true;
        for (int i = 0; i < n; ++i) {
            const int e = (int)((order >> (4 * i)) & 15u);
            uint32_t s0 = st[0], c0 = cnt[0];
#pragma unroll
            for (int w = 1; w < kLaneKMax; ++w)
                if (w == e) {
                    s0 = st[w];
                    c0 = cnt[w];
                }
            for (uint32_t r = s0; r < s0 + c0; ++r) {
                const float2 fb = S->bounds(r);
                if (!(fb.y > fb.x)) continue;
                Piece x;
                if (!first && fb.x > t) {
                    x.f = t;
                    x.b = fb.x;
                    x.P[0] = x.P[1] = x.P[2] = 0.f;
                    x.a = 0.f;
                    x.lgT = 0.f;
                    v(x);
                    ++np;
                }
                MixSums m;
                sums_reset(m);
                piece_from(m, true, S->rec(r), fb.x, fb.y, x);
                v(x);
                ++np;
                t = fb.y;
                first = false;
            }
        }
        return np;
    }
};

struct NtVisitor {
    int nt;
    __device__ __forceinline__ void operator()(const Piece& x) { nt += x.a > 0.f; }
};

// One sweep of the batch pass for every lane, whichever way its pixel goes.  A pixel whose
// non-transparent pieces number at most N_S takes gamma = 0 (sec. 2.4), and then every
// non-transparent piece is one output record, itself: each one terminates the open supersegment
// (Eq. 1 with gamma = 0: the distance is >= 0, reading G2) and each transparent piece closes it,
// so EmitVisitor with gamma = 0 stores exactly these pieces' values.  A pixel that needs the search
// writes all its pieces to its pool run.
struct LaneSink {
    const OutDev* out;
    size_t base;  // first output slot of the pixel
    int written;
    bool emit;
    float4* A;  // the pixel's pool run
    float2* B;
    bool pool;
    float f0;  // front of the first piece
    uint32_t np;
    __device__ __forceinline__ void operator()(const Piece& x) {
        if (np == 0) f0 = x.f;
        if (pool) {
            A[np] = make_float4(x.P[0], x.P[1], x.P[2], x.a);
            B[np] = make_float2(x.b, x.lgT);
        }
        if (emit && x.a > 0.f) {
            const size_t idx = base + written;
            if (out->prec == VDI_PREC_F32) {
                reinterpret_cast<float4*>(out->rgba)[idx] = make_float4(x.P[0], x.P[1], x.P[2], x.a);
                out->fb[idx] = make_float2(x.f, x.b);
            } else {
                reinterpret_cast<uint4*>(out->rgba)[idx] = f16_pack(x.f, x.b, x.P[0], x.P[1], x.P[2], x.lgT);
            }
            ++written;
        }
        ++np;
    }
};

// writes the zero tail, count and gamma of pixel p after an emission of `written` records
__device__ __forceinline__ void finish_pixel(const OutDev& out, uint32_t p, int written, float gamma) {
    for (int j = written; j < out.n_s; ++j) {
        const size_t idx = (size_t)p * out.n_s + j;
        if (out.prec == VDI_PREC_F32) {
            reinterpret_cast<float4*>(out.rgba)[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
            out.fb[idx] = make_float2(0.f, 0.f);
        } else {
            reinterpret_cast<uint4*>(out.rgba)[idx] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    out.counts[p] = (uint32_t)written;
    if (out.gamma) out.gamma[p] = gamma;
}

// list: [0] entries, [1] next entry for the search pass, [2] pieces taken from the pool, [3] unused,
// then FlatEntry entries from word 4
struct LaneArgs {
    unsigned int* counter;  // batch counter of the batch pass
    uint32_t* list;
    PiecePool pool;
};


// appends an entry for each lane with `flag` set (one atomic per warp)
__device__ __forceinline__ void list_push(uint32_t* list, bool flag, const FlatEntry& en) {
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(list, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (flag) reinterpret_cast<FlatEntry*>(list + 4)[base + __popc(m & ((1u << lane) - 1u))] = en;
}

// Copies the records of the lanes with `take` set into the slab, PE-major,
// and sets st[e] to each lane's first slab entry of PE e.  The copies are
// asynchronous; the caller waits once for all of them.
template <class SLAB>
__device__ __forceinline__ void slab_stage(const PeIn* pe, int k, SLAB& S, bool take, const uint32_t cnt[kLaneKMax],
                                           const uint64_t off[kLaneKMax], uint32_t st[kLaneKMax]) {
    const int lane = threadIdx.x & 31;
    uint32_t base_e = 0;
#pragma unroll
    for (int e = 0; e < kLaneKMax; ++e) {
        st[e] = 0;
        if (e < k) {
            const uint32_t ce = take ? cnt[e] : 0u;
            const uint32_t ie = warp_incl_scan_u32(ce);
            const uint32_t pre = ie - ce;
            const uint32_t n_e = __shfl_sync(0xffffffffu, ie, 31);
            st[e] = base_e + pre;
            // PE e's spans of this round are one run of its record array iff every non-empty span starts
            // where the previous ones leave off
            const unsigned nz = __ballot_sync(0xffffffffu, ce > 0);
            if (nz) {
                const int f = __ffs(nz) - 1;
                const uint64_t o0 = __shfl_sync(0xffffffffu, off[e], f);
                const bool run = !__any_sync(0xffffffffu, ce > 0 && off[e] != o0 + pre);
                for (uint32_t r0 = 0; r0 < n_e; r0 += 32) {
                    const uint32_t r = r0 + (uint32_t)lane;
                    uint64_t src = o0 + r;
                    if (!run) {
                        // the lane whose span holds record r: the last with pre <= r
                        int lo = 0, hi = 31;
#pragma unroll
                        for (int it = 0; it < 5; ++it) {
                            const int mid = (lo + hi + 1) >> 1;
                            const uint32_t pm = __shfl_sync(0xffffffffu, pre, mid);
                            if (pm <= r) lo = mid;
                            else hi = mid - 1;
                        }
                        const uint64_t oq = __shfl_sync(0xffffffffu, off[e], lo);
                        const uint32_t pq = __shfl_sync(0xffffffffu, pre, lo);
                        src = oq + (r - pq);
                    }
                    if (r < n_e) S.copy(pe[e], src, base_e + r);
                }
            }
            base_e += n_e;
        }
    }
}

// the listed pixels marked for the direct sweep (records beyond a slab, pieces beyond the pool, lists
// out of depth order), list heads in registers (KMAX > 0) or in shared memory under a winner tree of P
// leaves (KMAX == 0)
template <int KMAX, int P, int PREC, bool CENSUS>
__global__ void __launch_bounds__(128) composite_marked_kernel(const __grid_constant__ CompArgs a,
                                                               const uint32_t* __restrict__ list) {
    extern __shared__ uint32_t smem[];
    const uint32_t n = *list;
    const FlatEntry* entries = reinterpret_cast<const FlatEntry*>(list + 4);
    CompCensus cs;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i - threadIdx.x < n; i += gridDim.x * blockDim.x) {
        const uint32_t v = i < n ? entries[i].p : 0u;
        if (v & 0x80000000u)
            composite_pixel<KMAX, P, 2, PREC, CENSUS>(a.pe, a.k, a.out, a.iters, a.status, v & 0x7FFFFFFFu, smem,
                                                      &cs);
    }
    if (CENSUS) census_flush(cs, reinterpret_cast<WsHeader*>(a.status)->counters);
}

template <int PREC, int CAP>
constexpr size_t lane_smem_bytes() {
    return kLaneWarps * sizeof(LaneSlab<PREC, CAP>);
}

template <int PREC, bool CENSUS>
__global__ void __launch_bounds__(kLaneWarps * 32) composite_lane_kernel(const __grid_constant__ CompArgs a,
                                                                        const __grid_constant__ LaneArgs la) {
    using Slab = LaneSlab<PREC, kLaneRCap>;
    extern __shared__ __align__(16) unsigned char lane_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Slab& S = reinterpret_cast<Slab*>(lane_smem)[warp];
    const int k = a.k;
    const uint32_t nitems = ((uint32_t)a.npix + 31u) / 32u;
    CompCensus cs;
    while (true) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(la.counter, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nitems) break;
        const uint32_t p = item * 32u + (uint32_t)lane;
        const bool valid = p < (uint32_t)a.npix;
        uint32_t cnt[kLaneKMax];
        uint64_t off[kLaneKMax];
        uint32_t tot = 0;
#pragma unroll
        for (int e = 0; e < kLaneKMax; ++e) {
            cnt[e] = 0;
            off[e] = 0;
            if (e < k && valid) {
                cnt[e] = __ldg(a.pe[e].counts + p);
                off[e] = __ldg(a.pe[e].offsets + p);
                tot += cnt[e];
            }
        }
        // records beyond the slab: the direct sweep composites the pixel
        const bool big = valid && tot > (uint32_t)kLaneRCap;
        list_push(la.list, big, FlatEntry{p | 0x80000000u, 0u, 0u, 0.f});
        bool pending = valid && !big;
        while (__any_sync(0xffffffffu, pending)) {
            // this round: the pending lanes, in order, whose records fit the slab together
            const uint32_t incl = warp_incl_scan_u32(pending ? tot : 0u);
            const bool take = pending && incl <= (uint32_t)kLaneRCap;
            pending = pending && !take;
            uint32_t st[kLaneKMax];
            slab_stage(a.pe, k, S, take, cnt, off, st);
            cp_async_wait_all();
            __syncwarp();
            SlabSweeper<Slab> sw;
            sw.S = &S;
            sw.k = k;
#pragma unroll
            for (int e = 0; e < kLaneKMax; ++e) {
                sw.st[e] = st[e];
                sw.cnt[e] = take ? cnt[e] : 0u;
            }
            sw.prepare();
            bool emit = false, search = false;
            uint32_t bound = 0;  // pieces the pixel's pool run must hold
            int nt = 0;
            if (take) {
                if (sw.disjoint) {
                    // the pieces are the valid records with a gap between some of them
                    nt = sw.nto;
                    bound = sw.nvalid > 0 ? 2u * (uint32_t)sw.nvalid - 1u : 0u;
                } else {
                    NtVisitor nv{0};
                    bound = (uint32_t)sw.run(nv);
                    nt = nv.nt;
                }
                emit = nt <= a.out.n_s;
                search = !emit;
            }
            // the searching lanes' pool runs (one atomic per warp)
            uint32_t base = 0;
            bool fits = false;
            if (__any_sync(0xffffffffu, search)) {
                const uint32_t mine = search ? bound : 0u;
                const uint32_t inc = warp_incl_scan_u32(mine);
                if (lane == 31) base = atomicAdd(la.list + 2, inc);
                base = __shfl_sync(0xffffffffu, base, 31) + inc - mine;
                fits = search && (uint64_t)base + mine <= (uint64_t)la.pool.cap;
            }
            // one sweep: the gamma = 0 pixels' records, the searched pixels' pieces
            LaneSink snk{&a.out, (size_t)p * a.out.n_s, 0, emit, la.pool.A + base, la.pool.B + base, fits, 0.f, 0u};
            if (emit || fits) sw.run(snk);
            if (emit) {
                if (snk.written != nt) atomicCAS(a.status, 0u, (unsigned)VDI_ERR_CUDA);
                finish_pixel(a.out, p, snk.written, 0.f);
                if (CENSUS) {
                    const unsigned sweeps = sw.disjoint ? 1u : 2u;
                    cs.pixels += 1;
                    cs.records += tot;
                    cs.sweeps += sweeps;
                    cs.pieces += (unsigned long long)sweeps * snk.np;
                }
            }
            if (__any_sync(0xffffffffu, search))
                list_push(la.list, search, FlatEntry{fits ? p : (p | 0x80000000u), base, snk.np, snk.f0});
            __syncwarp();
        }
    }
    if (CENSUS) census_flush(cs, reinterpret_cast<WsHeader*>(a.status)->counters);
}

// ---------------------------------------------------------------------------
// Pooled staged path (K > kLaneKMax): composite_build_kernel builds each
// pixel's pieces as phase G of the staged schedule does -- the whole warp on
// one pixel: coalesced span loads, a stable merge of the bounds, the exact
// prefix scan of the mixture terms -- but writes them as one run of the pool
// and lists the pixel; composite_flat_kernel then searches and emits every
// listed pixel, a lane each.  The host runs the pixels in chunks whose pieces
// fit the pool.
// ---------------------------------------------------------------------------
struct BuildArgs {
    unsigned int* counter;  // batch counter
    uint32_t* list;         // as LaneArgs::list
    PiecePool pool;
    uint32_t p0, p1;        // the chunk's pixels
};

template <int PREC, bool CENSUS>
__global__ void __launch_bounds__(kStageWarps * 32, 1) composite_build_kernel(const __grid_constant__ CompArgs a,
                                                                              const __grid_constant__ BuildArgs ba) {
    extern __shared__ __align__(16) unsigned char stage_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    StageSmem& S = reinterpret_cast<StageSmem*>(stage_smem)[warp];
    const uint32_t nbatch = (ba.p1 - ba.p0 + 31u) / 32u;
    CompCensus cs;
    while (true) {
        uint32_t batch = 0;
        if (lane == 0) batch = atomicAdd(ba.counter, 1u);
        batch = __shfl_sync(0xffffffffu, batch, 0);
        if (batch >= nbatch) break;
        const uint32_t base = ba.p0 + batch * 32u;
        FlatEntry mine{0u, 0u, 0u, 0.f};
        bool have = false;
        for (int col = 0; col < 32; ++col) {
            const uint32_t p = base + (uint32_t)col;
            if (p >= ba.p1) break;
            PoolRun run{ba.list + 2, ba.pool.cap, 0u};
            int n = 0, nt = 0;
            float f0 = 0.f;
            const bool ok = stage_pixel<PREC, true>(a.pe, a.k, p, S, ba.pool.A, ba.pool.B, 0x7FFFFFFF, n, nt, f0, &run);
            if (lane == col) {
                if (!ok || n < 0) {
                    mine = FlatEntry{p | 0x80000000u, 0u, 0u, 0.f};
                    have = true;
                } else if (n == 0) {
                    finish_pixel(a.out, p, 0, 0.f);  // no record: an empty list
                    if (CENSUS) cs.pixels += 1;
                } else {
                    mine = FlatEntry{p, run.base, (uint32_t)n, f0};
                    have = true;
                }
            }
        }
        list_push(ba.list, have, mine);
    }
    if (CENSUS) census_flush(cs, reinterpret_cast<WsHeader*>(a.status)->counters);
}

// ---------------------------------------------------------------------------
// Flat search: composite_search_emit<2> for one pixel per lane, written as one
// loop whose body handles one piece of the lane's current march.  Lanes at
// different marches, or at different pixels, execute the same loop body, so
// a warp's lanes stay busy however many marches their pixels need; a lane
// that finishes its pixel takes the next one from the list.  The decisions,
// the table of decision intervals and the replay of sequential bisection are
// those of composite_search_emit, step for step, so the output is the same,
// bit for bit.  The pieces come from a pool in the workspace (written by the
// batch pass), one contiguous run per pixel.
// ---------------------------------------------------------------------------
enum : int { kFlatIdle = 0, kFlatFirst = 1, kFlatSearch = 2, kFlatEmit = 3 };

#ifndef VDI_FLAT_END_BATCH
#define VDI_FLAT_END_BATCH 16
#endif
// resident CTAs of the flat pass per SM over the dense pieces of the pooled and batched paths (the lane
// path takes as many as the registers allow): with 2047-piece runs, more lanes per SM evict each
// other's pool lines and decision tables from L1 (dense 512^2, K = 32: 137.7 ms at 5 CTAs, 150.8 at 6;
// the plain frame: 3.20 ms at 6, 3.36 at 5)
#ifndef VDI_FLAT_CTAS_PER_SM
#define VDI_FLAT_CTAS_PER_SM 5
#endif

struct FlatLane {
    const OutDev* out;  // the pixel's output (its request's, in a batch)
    uint32_t p, base, n, j;
    float f, f0;
    int phase;
    float g2[3];
    CompCountQ st[3];  // a counting march's candidates; st[0] also holds the emission's supersegment
    int nt;
    float bt;  // emission: back of the last non-transparent piece of the open supersegment
    int written;
    float lo, hi, gamma;
    int cnt_hi, it, count;
};

__device__ __forceinline__ void flat_start_count(FlatLane& L, float lo, float hi) {
    float g[3];
    tree_candidates<2>(lo, hi, g);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        L.g2[q] = __fmul_rn(g[q], g[q]);
        L.st[q].cnt = 0;
        L.st[q].open = false;
        L.st[q].qlo = -1.f;
        L.st[q].qhi = 3.0e38f;
    }
    L.nt = 0;
    L.j = 0;
    L.f = L.f0;
}

__device__ __forceinline__ void flat_start_emit(FlatLane& L) {
    L.phase = kFlatEmit;
    L.g2[0] = __fmul_rn(L.gamma, L.gamma);
    L.st[0].cnt = 0;
    L.st[0].open = false;
    L.bt = 0.f;
    L.written = 0;
    L.j = 0;
    L.f = L.f0;
}

__device__ __forceinline__ void flat_store(const OutDev& out, uint32_t p, int written, float f, float b,
                                           const float P[3], float A, float L2) {
    const size_t idx = (size_t)p * out.n_s + written;
    if (out.prec == VDI_PREC_F32) {
        reinterpret_cast<float4*>(out.rgba)[idx] = make_float4(P[0], P[1], P[2], A);
        out.fb[idx] = make_float2(f, b);
    } else {
        reinterpret_cast<uint4*>(out.rgba)[idx] = f16_pack(f, b, P[0], P[1], P[2], L2);
    }
}

// Continues the bisection replay from level L.it: levels whose midpoint a recorded decision interval
// answers need no march; returns with the next march started, or with the emission started.
template <bool CENSUS>
__device__ __forceinline__ void flat_advance(FlatLane& L, CountTable& t, int iters, int n_s, CompCensus& cs) {
    while (L.it < iters) {
        const float mid = 0.5f * (L.lo + L.hi);
        const int c = t.lookup(__fmul_rn(mid, mid));
        if (c < 0) {
            L.phase = kFlatSearch;
            flat_start_count(L, L.lo, L.hi);
            return;
        }
        if (CENSUS) cs.table_hits += 1;
        ++L.it;
        if (c <= n_s) {
            L.hi = mid;
            L.cnt_hi = c;
            if (c == n_s) break;
        } else {
            L.lo = mid;
        }
    }
    L.gamma = L.hi;
    L.count = L.cnt_hi;
    flat_start_emit(L);
}

template <bool CENSUS>
__device__ __forceinline__ void flat_end_march(FlatLane& L, CountTable& t, const OutDev& out, int iters,
                                               unsigned int* status, CompCensus& cs) {
    if (CENSUS) {
        cs.sweeps += 1;
        cs.pieces += L.n;
        if (L.phase != kFlatEmit) cs.cand_steps += (unsigned long long)L.n * 3;
    }
    if (L.phase == kFlatFirst) {
#pragma unroll
        for (int q = 0; q < 3; ++q) t.add(L.g2[q], L.st[q].qlo, L.st[q].qhi, L.st[q].cnt);
        if (L.nt <= out.n_s) {
            L.gamma = 0.f;
            L.count = L.nt;
            flat_start_emit(L);
        } else {
            if (CENSUS) cs.searched += 1;
            L.lo = 0.f;
            L.hi = 2.f;
            L.cnt_hi = 1;  // the distance never reaches 2: one supersegment
            L.it = 0;
            flat_advance<CENSUS>(L, t, iters, out.n_s, cs);
        }
    } else if (L.phase == kFlatSearch) {
#pragma unroll
        for (int q = 0; q < 3; ++q) t.add(L.g2[q], L.st[q].qlo, L.st[q].qhi, L.st[q].cnt);
        const int c = L.st[0].cnt;
        const float mid = 0.5f * (L.lo + L.hi);
        ++L.it;
        if (c <= out.n_s) {
            L.hi = mid;
            L.cnt_hi = c;
            if (c == out.n_s) {
                L.it = iters;  // done
            }
        } else {
            L.lo = mid;
        }
        flat_advance<CENSUS>(L, t, iters, out.n_s, cs);
    } else {
        // the emission: the open supersegment, the zero tail, count and gamma
        CompCountQ& s = L.st[0];
        if (s.open && L.written < out.n_s) {
            flat_store(out, L.p, L.written, s.fS, L.bt, s.P, s.A, s.L2);
            ++L.written;
        }
        finish_pixel(out, L.p, L.written, L.gamma);
        if (L.written != L.count) atomicCAS(status, 0u, (unsigned)VDI_ERR_CUDA);
        L.phase = kFlatIdle;
    }
}

// Where the flat loop finds its pixels: the list's entries (one request) ...
struct FlatSrcOne {
    const FlatEntry* entries;
    const OutDev* out;
    const PeIn* pe;
    int k;
    __device__ __forceinline__ bool get(uint32_t i, FlatLane& L) const {
        const FlatEntry en = entries[i];
        if (en.p & 0x80000000u) return false;  // the direct sweep's
        L.p = en.p;
        L.base = en.base;
        L.n = en.n;
        L.f0 = en.f0;
        L.out = out;
        return true;
    }
    __device__ __forceinline__ unsigned long long records(uint32_t p) const {
        unsigned long long r = 0;
        for (int e = 0; e < k; ++e) r += __ldg(pe[e].counts + p);
        return r;
    }
};

// The search and emission of the listed pixels, a lane each (list: [count, next-entry counter, ...]
// then the entries SRC reads).
template <bool CENSUS, class SRC>
__device__ __forceinline__ void flat_loop(const SRC& src, const PiecePool& pool, uint32_t* list, int iters,
                                          unsigned int* status, CompCensus& cs) {
    const uint32_t n_list = list[0];
    const int lane = threadIdx.x & 31;
    FlatLane L;
    L.phase = kFlatIdle;
    L.out = nullptr;
    CountTable t;
    t.n = 0;
    bool exhausted = false;
    float4 cA = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 cB = make_float2(0.f, 0.f);
    while (true) {
        // idle lanes take the next entries, one atomic per warp (in a list sorted by piece count, the
        // entries one fetch hands to a warp's lanes have nearly equal counts)
        const unsigned need = __ballot_sync(0xffffffffu, L.phase == kFlatIdle && !exhausted);
        if (need) {
            const int leader = __ffs(need) - 1;
            uint32_t first = 0;
            if (lane == leader) first = atomicAdd(list + 1, (uint32_t)__popc(need));
            first = __shfl_sync(0xffffffffu, first, leader);
            if ((need >> lane) & 1u) {
                const uint32_t idx = first + (uint32_t)__popc(need & ((1u << lane) - 1u));
                if (idx >= n_list) {
                    exhausted = true;
                } else if (src.get(idx, L)) {  // (a marked entry leaves the lane idle: it takes another)
                    L.phase = kFlatFirst;
                    t.n = 0;
                    flat_start_count(L, 0.f, 2.f);
                    if (CENSUS) {
                        cs.pixels += 1;
                        cs.records += src.records(L.p);
                    }
                }
            }
        }
        const bool active = L.phase != kFlatIdle;
        const unsigned act = __ballot_sync(0xffffffffu, active);
        if (!act) {
            if (__all_sync(0xffffffffu, exhausted)) break;
            continue;  // lanes that drew a marked entry draw again
        }
        // a lane at the end of its march waits until VDI_FLAT_END_BATCH lanes (or all active ones) are
        // there: the end of a march (table updates, the replay of bisection levels, the next march's
        // candidates) runs once for all of them instead of once per lane while the others idle
        const bool at_end = active && L.j == L.n;
        const unsigned pend = __ballot_sync(0xffffffffu, at_end);
        if (pend != 0u && (pend == act || __popc(pend) >= VDI_FLAT_END_BATCH)) {
            if (at_end) flat_end_march<CENSUS>(L, t, *L.out, iters, status, cs);
            continue;
        }
        if (!active || at_end) continue;
        // one piece of the lane's march
        if (L.j == 0) {
            cA = pool.A[L.base];
            cB = pool.B[L.base];
        }
        Piece x;
        x.f = L.f;
        x.b = cB.x;
        x.P[0] = cA.x;
        x.P[1] = cA.y;
        x.P[2] = cA.z;
        x.a = cA.w;
        x.lgT = cB.y;
        if (L.j + 1 < L.n) {
            cA = pool.A[L.base + L.j + 1];
            cB = pool.B[L.base + L.j + 1];
        }
        // one instruction stream for counting and emitting lanes: candidate 0 carries the budget (none
        // while counting) and, emitting, writes the supersegment a termination closes -- EmitVisitor's
        // decisions, in select form; candidates 1 and 2 only count
        {
            const bool emitting = L.phase == kFlatEmit;
            const int cap = emitting ? L.out->n_s : INT_MAX;
            CompCountQ& s = L.st[0];
            float q = 0.f;
            const bool crit = s.open && s.cnt < cap &&
                              criterion_q(s.P, s.A, s.L2, piece_ratio(s, x), x.P, L.g2[0], q);
            if (emitting && crit && L.written < cap) {
                flat_store(*L.out, L.p, L.written, s.fS, L.bt, s.P, s.A, s.L2);
                ++L.written;
            }
            s.qhi = crit ? fminf(s.qhi, q) : s.qhi;
            s.qlo = (s.open && !crit) ? fmaxf(s.qlo, q) : s.qlo;
            const bool opaque = x.a > 0.f;
            const bool fresh = opaque && (!s.open || crit);
            const bool absorbing = s.open && !crit;
            L.bt = (fresh || (absorbing && opaque)) ? x.b : L.bt;
            apply_step(s, x, StepSel{fresh, crit && !opaque});
            L.nt += opaque;
            cq_step_select(L.st[1], x, L.g2[1]);
            cq_step_select(L.st[2], x, L.g2[2]);
        }
        L.f = x.b;
        ++L.j;
    }
}

template <bool CENSUS>
__global__ void __launch_bounds__(128) composite_flat_kernel(const __grid_constant__ CompArgs a,
                                                             const __grid_constant__ PiecePool pool,
                                                             uint32_t* list) {
    CompCensus cs;
    const FlatSrcOne src{reinterpret_cast<const FlatEntry*>(list + 4), &a.out, a.pe, a.k};
    flat_loop<CENSUS>(src, pool, list, a.iters, a.status, cs);
    if (CENSUS) census_flush(cs, reinterpret_cast<WsHeader*>(a.status)->counters);
}

// ---------------------------------------------------------------------------
// Order of the search pass: the listed pixels sorted by piece count, longest
// first (a counting sort into a second list with the same header).  A warp's
// lanes then take pixels of (nearly) equal piece counts, so their marches end
// together and no lane waits for the others at the end of a march; the
// longest pixels start first, so the last wave holds the shortest.  The order
// of pixels with equal counts is that of the atomics, which is free to vary:
// each pixel's result is independent of when it runs.  Marked pixels (the
// direct sweep's) stay out of the sorted list.
// ---------------------------------------------------------------------------
constexpr int kSortBins = 2048;

__device__ __forceinline__ uint32_t sort_bin(uint32_t n) {
    return (uint32_t)(kSortBins - 1) - (n < (uint32_t)(kSortBins - 1) ? n : (uint32_t)(kSortBins - 1));
}

// hist[b] += entries of bin b (hist zeroed by the caller)
template <class E, int HW>
__global__ void __launch_bounds__(256) list_hist_kernel(const uint32_t* __restrict__ list, uint32_t* hist) {
    __shared__ uint32_t h[kSortBins];
    for (int i = threadIdx.x; i < kSortBins; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    const uint32_t n = list[0];
    const E* en = reinterpret_cast<const E*>(list + HW);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const E e = en[i];
        if (!(e.p & 0x80000000u)) atomicAdd(&h[sort_bin(e.n)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSortBins; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// hist -> exclusive offsets (in place); the sorted list's header: [0] entries, [1] next entry = 0
__global__ void __launch_bounds__(1024) list_offsets_kernel(uint32_t* hist, uint32_t* sorted) {
    __shared__ uint32_t wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kPer = kSortBins / 1024;
    uint32_t v[kPer], s = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        v[q] = hist[tid * kPer + q];
        s += v[q];
    }
    const uint32_t incl = warp_incl_scan_u32(s);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = warp_incl_scan_u32(wsum[lane]);
        wsum[lane] = w;
    }
    __syncthreads();
    uint32_t ex = (warp > 0 ? wsum[warp - 1] : 0u) + incl - s;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        hist[tid * kPer + q] = ex;
        ex += v[q];
    }
    if (tid == 0) {
        sorted[0] = wsum[31];
        sorted[1] = 0u;
    }
}

// every unmarked entry to its bin's next slot (one atomic per bin and warp)
template <class E, int HW>
__global__ void __launch_bounds__(256) list_scatter_kernel(const uint32_t* __restrict__ list, uint32_t* pos,
                                                           uint32_t* sorted) {
    const uint32_t n = list[0];
    const E* en = reinterpret_cast<const E*>(list + HW);
    E* out = reinterpret_cast<E*>(sorted + HW);
    const int lane = threadIdx.x & 31;
    for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
        const uint32_t i = i0 + threadIdx.x;
        E e{};
        bool take = false;
        if (i < n) {
            e = en[i];
            take = !(e.p & 0x80000000u);
        }
        const unsigned act = __ballot_sync(0xffffffffu, take);
        if (take) {
            const uint32_t b = sort_bin(e.n);
            const unsigned grp = __match_any_sync(act, b);
            const int leader = __ffs(grp) - 1;
            uint32_t slot = 0;
            if (lane == leader) slot = atomicAdd(&pos[b], (uint32_t)__popc(grp));
            slot = __shfl_sync(grp, slot, leader) + (uint32_t)__popc(grp & ((1u << lane) - 1u));
            out[slot] = e;
        }
    }
}

static int device_sms();

// bytes of the sort's scratch: the histogram / offsets
constexpr size_t kSortScratch = kSortBins * sizeof(uint32_t);

// sorts list (HW header words, entries E) into sorted; hist: kSortScratch bytes
template <class E, int HW>
static cudaError_t launch_sort(const uint32_t* list, uint32_t* sorted, uint32_t* hist, uint64_t max_entries,
                               cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(hist, 0, kSortScratch, st);
    if (e != cudaSuccess) return e;
    uint64_t b = (max_entries + 255) / 256;
    const uint64_t cap = (uint64_t)device_sms() * 4u;
    if (b > cap) b = cap;
    if (b == 0) b = 1;
    list_hist_kernel<E, HW><<<(unsigned)b, 256, 0, st>>>(list, hist);
    list_offsets_kernel<<<1, 1024, 0, st>>>(hist, sorted);
    list_scatter_kernel<E, HW><<<(unsigned)b, 256, 0, st>>>(list, hist, sorted);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched persistent compositing
// ---------------------------------------------------------------------------
struct ReqDev {
    OutDev out;
    uint32_t npix;
    uint32_t item_begin;  // first 32-pixel batch of the request
    uint32_t pe_begin;    // index of its first PE descriptor
    int k, schedule;
};

struct BatchArgs {
    const ReqDev* reqs;
    const PeIn* pes;
    int n;
    uint32_t total_items;
    unsigned int* status;
    int iters;
};

__device__ __forceinline__ int request_of(const BatchArgs& a, uint32_t item) {
    int lo = 0, hi = a.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&a.reqs[mid].item_begin) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Pooled batched path: composite_batched_build_kernel takes (request,
// 32-pixel batch) items of a chunk from an atomic counter and builds each
// pixel's pieces into the pool as composite_build_kernel does (requests with
// a direct schedule, and pixels the stage cannot hold, are listed for the
// direct sweep); composite_batched_flat_kernel searches and emits the listed
// pixels, a lane each, each into its request's output; composite_batched_
// marked_kernel sweeps the pixels listed for the direct path.
struct BatchEntry {
    uint32_t p, base, n;
    float f0;
    uint32_t req, pad0, pad1, pad2;
};

struct BatchBuildArgs {
    unsigned int* counter;  // item counter
    uint32_t* list;         // [0] entries, [1] next entry of the flat pass, [2] pool pieces taken; entries from word 8
    PiecePool pool;
    uint32_t item0, item1;  // the chunk's items
};

__device__ __forceinline__ void batch_push(uint32_t* list, bool flag, const BatchEntry& en) {
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(list, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (flag) reinterpret_cast<BatchEntry*>(list + 8)[base + __popc(m & ((1u << lane) - 1u))] = en;
}

template <int PREC>
__global__ void __launch_bounds__(kStageWarps * 32, 1) composite_batched_build_kernel(
    const __grid_constant__ BatchArgs a, const __grid_constant__ BatchBuildArgs bb) {
    extern __shared__ __align__(16) unsigned char stage_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    StageSmem& S = reinterpret_cast<StageSmem*>(stage_smem)[warp];
    while (true) {
        uint32_t item = 0;
        if (lane == 0) item = bb.item0 + atomicAdd(bb.counter, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= bb.item1) break;
        const int rq = request_of(a, item);
        const ReqDev& r = a.reqs[rq];
        const uint32_t base = (item - r.item_begin) * 32u;
        BatchEntry mine{0u, 0u, 0u, 0.f, (uint32_t)rq, 0u, 0u, 0u};
        bool have = false;
        if (r.schedule == VDI_SCHED_STAGED) {
            for (int col = 0; col < 32; ++col) {
                const uint32_t p = base + (uint32_t)col;
                if (p >= r.npix) break;
                PoolRun run{bb.list + 2, bb.pool.cap, 0u};
                int n = 0, nt = 0;
                float f0 = 0.f;
                const bool ok = stage_pixel<PREC, true>(a.pes + r.pe_begin, r.k, p, S, bb.pool.A, bb.pool.B,
                                                        0x7FFFFFFF, n, nt, f0, &run);
                if (lane == col) {
                    if (!ok || n < 0) {
                        mine.p = p | 0x80000000u;
                        have = true;
                    } else if (n == 0) {
                        finish_pixel(r.out, p, 0, 0.f);  // no record: an empty list
                    } else {
                        mine.p = p;
                        mine.base = run.base;
                        mine.n = (uint32_t)n;
                        mine.f0 = f0;
                        have = true;
                    }
                }
            }
        } else {
            const uint32_t p = base + (uint32_t)lane;
            have = p < r.npix;
            mine.p = p | 0x80000000u;
        }
        batch_push(bb.list, have, mine);
    }
}

struct FlatSrcBatch {
    const BatchEntry* entries;
    const ReqDev* reqs;
    __device__ __forceinline__ bool get(uint32_t i, FlatLane& L) const {
        const BatchEntry en = entries[i];
        if (en.p & 0x80000000u) return false;  // the direct sweep's
        L.p = en.p;
        L.base = en.base;
        L.n = en.n;
        L.f0 = en.f0;
        L.out = &reqs[en.req].out;
        return true;
    }
    __device__ __forceinline__ unsigned long long records(uint32_t) const { return 0; }
};

__global__ void __launch_bounds__(128) composite_batched_flat_kernel(const __grid_constant__ BatchArgs a,
                                                                     const __grid_constant__ PiecePool pool,
                                                                     uint32_t* list) {
    CompCensus cs;
    const FlatSrcBatch src{reinterpret_cast<const BatchEntry*>(list + 8), a.reqs};
    flat_loop<false>(src, pool, list, a.iters, a.status, cs);
}

template <int P, int PREC>
__global__ void __launch_bounds__(128) composite_batched_marked_kernel(const __grid_constant__ BatchArgs a,
                                                                       const uint32_t* __restrict__ list) {
    extern __shared__ uint32_t smem[];
    const uint32_t n = *list;
    const BatchEntry* entries = reinterpret_cast<const BatchEntry*>(list + 8);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i - threadIdx.x < n; i += gridDim.x * blockDim.x) {
        const BatchEntry en = i < n ? entries[i] : BatchEntry{0u, 0u, 0u, 0.f, 0u, 0u, 0u, 0u};
        if (en.p & 0x80000000u) {
            const ReqDev& r = a.reqs[en.req];
            composite_pixel<0, P, 2, PREC>(a.pes + r.pe_begin, r.k, r.out, a.iters, a.status, en.p & 0x7FFFFFFFu,
                                           smem);
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int default_schedule(int k) { return k <= kLaneKMax ? VDI_SCHED_LANE : VDI_SCHED_STAGED; }

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

// leaves of the winner tree for K PEs
static int tree_leaves(int k) { return k <= 16 ? 16 : (k <= 32 ? 32 : 64); }

template <int P>
static size_t heads_smem_bytes(int threads) {
    return (size_t)threads * smem_words_per_thread<P>() * sizeof(uint32_t);
}

static int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    return sms;
}

// Workspace of the staged path: [header][batch counter][overflow count, pad,
// entries][piece buffers], for `batches` 32-pixel batches and `entries`
// overflow entries of `entry_bytes`.
static size_t stage_ctas(uint64_t batches) {
    const uint64_t need = (batches + kStageWarps - 1) / kStageWarps;
    const uint64_t sms = (uint64_t)device_sms();
    return (size_t)(need < sms ? (need > 0 ? need : 1) : sms);
}

// pixels per chunk of the pooled staged path that the queried workspace holds at the stage's worst case
constexpr uint64_t kPoolChunkPixels = 131072;

size_t composite_workspace_bytes(int w, int h) {
    const uint64_t npix = (uint64_t)w * (uint64_t)h;
    const size_t piece = sizeof(float4) + sizeof(float2);
    // pooled staged path: a chunk of up to kPoolChunkPixels pixels, each with room for the stage's pieces
    const uint64_t chunk = npix < kPoolChunkPixels ? npix : kPoolChunkPixels;
    const size_t pooled = kWsHeader + 512 + (size_t)chunk * (sizeof(FlatEntry) + 2 * kStageRMax * piece);
    // lane path: the list of every pixel, its sorted copy and a pool of 16 pieces per pixel
    const size_t lane = kWsHeader + 256 + 2 * align_up(16 + npix * sizeof(FlatEntry), 256) + kSortScratch +
                        (size_t)npix * 16 * piece;
    return pooled > lane ? pooled : lane;
}


template <int KMAX, int P, int NLEV, int PREC>
static cudaError_t launch_cs(bool census, unsigned blocks, int threads, cudaStream_t st, const CompArgs& a) {
    const size_t sm = KMAX > 0 ? 0 : heads_smem_bytes<P>(threads);
    auto kern = census ? composite_kernel<KMAX, P, NLEV, PREC, true> : composite_kernel<KMAX, P, NLEV, PREC, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<blocks, threads, sm, st>>>(a);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t launch_sched(int schedule, int k, bool census, unsigned blocks, int threads, cudaStream_t st,
                                const CompArgs& a) {
    if (schedule == 1) return launch_cs<8, 16, 2, PREC>(census, blocks, threads, st, a);
    const int P = tree_leaves(k);
    if (schedule == 3) {
        if (P == 16) return launch_cs<0, 16, 3, PREC>(census, blocks, threads, st, a);
        if (P == 32) return launch_cs<0, 32, 3, PREC>(census, blocks, threads, st, a);
        return launch_cs<0, 64, 3, PREC>(census, blocks, threads, st, a);
    }
    if (P == 16) return launch_cs<0, 16, 2, PREC>(census, blocks, threads, st, a);
    if (P == 32) return launch_cs<0, 32, 2, PREC>(census, blocks, threads, st, a);
    return launch_cs<0, 64, 2, PREC>(census, blocks, threads, st, a);
}


template <int KMAX, int P, int PREC>
static cudaError_t launch_marked(bool census, const CompArgs& a, const uint32_t* list, uint64_t npix,
                                 cudaStream_t st) {
    const size_t sm = KMAX > 0 ? 0 : heads_smem_bytes<P>(128);
    auto kern = census ? composite_marked_kernel<KMAX, P, PREC, true> : composite_marked_kernel<KMAX, P, PREC, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    unsigned b = (unsigned)((npix + 127) / 128);
    const unsigned cap = (unsigned)device_sms() * 2u;
    if (b > cap) b = cap;
    kern<<<b, 128, sm, st>>>(a, list);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t launch_flat(bool census, const CompArgs& a, const PiecePool& pool, uint32_t* list, uint64_t lanes,
                               cudaStream_t st, int max_per_sm = 0) {
    auto k2 = census ? composite_flat_kernel<true> : composite_flat_kernel<false>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k2, 128, 0);
    if (e != cudaSuccess) return e;
    if (max_per_sm > 0 && per_sm > max_per_sm) per_sm = max_per_sm;
    uint64_t b = (uint64_t)device_sms() * (uint64_t)(per_sm > 0 ? per_sm : 1);
    const uint64_t need = (lanes + 127) / 128;
    if (b > need) b = need > 0 ? need : 1;
    k2<<<(unsigned)b, 128, 0, st>>>(a, pool, list);
    return cudaGetLastError();
}

// pieces a pixel of the pooled staged path may need (the stage holds kStageRMax records)
constexpr uint64_t kPoolPiecesPerPixel = 2 * kStageRMax;

template <int PREC>
static cudaError_t launch_staged_pool(bool census, const CompArgs& a, void* workspace, size_t ws_bytes,
                                     cudaStream_t st) {
    // workspace: [header][counters][list: 4 words, entries of a chunk][pool: float4 x cap][pool: float2 x cap]
    // (the list stays in build order: dense pixels have equal piece counts, and a warp's lanes then read
    // pool runs that one warp wrote next to each other)
    const uint64_t npix = (uint64_t)a.npix;
    char* base = static_cast<char*>(workspace);
    // the chunk: as many pixels as the pool holds at the stage's worst case, all of them if they fit
    const size_t head = kWsHeader + 256;
    if (ws_bytes < head + 256) return cudaErrorInvalidValue;
    const size_t per_pixel = sizeof(FlatEntry) + kPoolPiecesPerPixel * (sizeof(float4) + sizeof(float2));
    uint64_t chunk = (ws_bytes - head - 256) / per_pixel;
    if (chunk > npix) chunk = npix;
    if (chunk == 0) return cudaErrorInvalidValue;
    const size_t list_bytes = align_up(16 + chunk * sizeof(FlatEntry), 256);
    size_t cap = (ws_bytes - head - list_bytes) / (sizeof(float4) + sizeof(float2));
    if (cap > 0x7FFFFFFFu) cap = 0x7FFFFFFFu;
    BuildArgs ba;
    ba.counter = reinterpret_cast<unsigned int*>(base + kWsHeader);
    ba.list = reinterpret_cast<uint32_t*>(base + head);
    ba.pool.cap = (uint32_t)cap;
    ba.pool.A = reinterpret_cast<float4*>(base + head + list_bytes);
    ba.pool.B = reinterpret_cast<float2*>(base + head + list_bytes + cap * sizeof(float4));
    const size_t sm = kStageWarps * sizeof(StageSmem);
    auto kb = census ? composite_build_kernel<PREC, true> : composite_build_kernel<PREC, false>;
    cudaError_t e = cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int P = tree_leaves(a.k);
    for (uint64_t p0 = 0; p0 < npix; p0 += chunk) {
        const uint64_t p1 = p0 + chunk < npix ? p0 + chunk : npix;
        ba.p0 = (uint32_t)p0;
        ba.p1 = (uint32_t)p1;
        e = cudaMemsetAsync(ba.counter, 0, 256, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(ba.list, 0, 16, st);
        if (e != cudaSuccess) return e;
        kb<<<(unsigned)stage_ctas((p1 - p0 + 31) / 32), kStageWarps * 32, sm, st>>>(a, ba);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_flat<PREC>(census, a, ba.pool, ba.list, p1 - p0, st, VDI_FLAT_CTAS_PER_SM);
        if (e == cudaSuccess) {
            if (P == 16) e = launch_marked<0, 16, PREC>(census, a, ba.list, p1 - p0, st);
            else if (P == 32) e = launch_marked<0, 32, PREC>(census, a, ba.list, p1 - p0, st);
            else e = launch_marked<0, 64, PREC>(census, a, ba.list, p1 - p0, st);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int PREC>
static cudaError_t launch_lane(bool census, const CompArgs& a, void* workspace, size_t ws_bytes, cudaStream_t st) {
    // workspace: [header][counters][list: 4 words, npix entries][the list sorted][sort scratch]
    // [pool: float4 x cap][pool: float2 x cap]
    const uint64_t npix = (uint64_t)a.npix;
    const size_t list_bytes = align_up(16 + npix * sizeof(FlatEntry), 256);
    const size_t fixed = kWsHeader + 256 + 2 * list_bytes + kSortScratch;
    if (ws_bytes < fixed) return cudaErrorInvalidValue;
    char* base = static_cast<char*>(workspace);
    LaneArgs la;
    la.counter = reinterpret_cast<unsigned int*>(base + kWsHeader);
    la.list = reinterpret_cast<uint32_t*>(base + kWsHeader + 256);
    uint32_t* sorted = reinterpret_cast<uint32_t*>(base + kWsHeader + 256 + list_bytes);
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + kWsHeader + 256 + 2 * list_bytes);
    size_t cap = (ws_bytes - fixed) / (sizeof(float4) + sizeof(float2));
    if (cap > 0x7FFFFFFFu) cap = 0x7FFFFFFFu;
    la.pool.cap = (uint32_t)cap;
    la.pool.A = reinterpret_cast<float4*>(base + fixed);
    la.pool.B = reinterpret_cast<float2*>(base + fixed + cap * sizeof(float4));
    cudaError_t e = cudaMemsetAsync(la.counter, 0, 256 + 16, st);
    if (e != cudaSuccess) return e;
    // batch pass
    const size_t sm = lane_smem_bytes<PREC, kLaneRCap>();
    auto k1 = census ? composite_lane_kernel<PREC, true> : composite_lane_kernel<PREC, false>;
    e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1, kLaneWarps * 32, sm);
    if (e != cudaSuccess) return e;
    const uint64_t batches = (npix + 31) / 32;
    uint64_t blocks = (uint64_t)device_sms() * (uint64_t)(per_sm > 0 ? per_sm : 1);
    const uint64_t need = (batches + kLaneWarps - 1) / kLaneWarps;
    if (blocks > need) blocks = need > 0 ? need : 1;
    k1<<<(unsigned)blocks, kLaneWarps * 32, sm, st>>>(a, la);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // search pass over the list sorted by piece count: a persistent grid; the list's length is known
    // only on the device
    e = launch_sort<FlatEntry, 4>(la.list, sorted, hist, npix, st);
    if (e == cudaSuccess) e = launch_flat<PREC>(census, a, la.pool, sorted, npix, st);
    if (e != cudaSuccess) return e;
    return launch_marked<kLaneKMax, 16, PREC>(census, a, la.list, npix, st);
}

vdi_status launch_composite(const vdi_compact* pe, int k, int w, int h, const vdi_regular* out, int iters,
                            int schedule, unsigned int* status, void* workspace, size_t ws_bytes, cudaStream_t st,
                            bool census) {
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
    const bool automatic = schedule == 0;
    if (schedule == 0 || (schedule == 1 && k > 8)) schedule = default_schedule(k);
    // an automatic choice falls back to a direct schedule when the workspace holds no list or stage
    if (automatic && schedule == VDI_SCHED_LANE &&
        ws_bytes < kWsHeader + 256 + 2 * align_up(16 + (uint64_t)w * h * sizeof(FlatEntry), 256) + kSortScratch)
        schedule = 1;
    if (automatic && schedule == VDI_SCHED_STAGED && ws_bytes < composite_workspace_bytes(1, 1)) schedule = 2;
    if (a.npix == 0) return VDI_OK;
    const bool f32 = prec_in == VDI_PREC_F32;
    cudaError_t e;
    if (schedule == VDI_SCHED_LANE && k > kLaneKMax) schedule = VDI_SCHED_STAGED;
    if (schedule == VDI_SCHED_STAGED) {
        e = f32 ? launch_staged_pool<VDI_PREC_F32>(census, a, workspace, ws_bytes, st)
                : launch_staged_pool<VDI_PREC_F16>(census, a, workspace, ws_bytes, st);
    } else if (schedule == VDI_SCHED_LANE) {
        e = f32 ? launch_lane<VDI_PREC_F32>(census, a, workspace, ws_bytes, st)
                : launch_lane<VDI_PREC_F16>(census, a, workspace, ws_bytes, st);
    } else {
        const int threads = 128;
        const unsigned blocks = (unsigned)((a.npix + threads - 1) / threads);
        e = f32 ? launch_sched<VDI_PREC_F32>(schedule, k, census, blocks, threads, st, a)
                : launch_sched<VDI_PREC_F16>(schedule, k, census, blocks, threads, st, a);
    }
    return cuda_check(e, "composite launch");
}

// Device table: [BatchHeader][ReqDev x n][PeIn x sum k]
struct BatchHeader {
    uint32_t n, total_items, total_pes, prec_in;
    uint32_t max_k, pad;
    uint64_t total_pixels;
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
    uint64_t items = 0, pes = 0, pixels = 0;
    uint32_t max_k = 0;
    for (int r = 0; r < n; ++r) {
        const vdi_request& q = reqs[r];
        rd[r].out = out_dev(&q.out);
        rd[r].npix = (uint32_t)((uint64_t)q.w * (uint64_t)q.h);
        rd[r].item_begin = (uint32_t)items;
        rd[r].pe_begin = (uint32_t)pes;
        rd[r].k = q.k;
        rd[r].schedule =
            q.schedule == VDI_SCHED_STAGED || q.schedule == VDI_SCHED_LANE || q.schedule == 0 ? VDI_SCHED_STAGED : 2;
        for (int e = 0; e < q.k; ++e) {
            pd[pes + e].counts = q.pe[e].counts;
            pd[pes + e].offsets = q.pe[e].offsets;
            pd[pes + e].rgba = q.pe[e].rgba;
            pd[pes + e].fb = reinterpret_cast<const float2*>(q.pe[e].fb);
        }
        pes += (uint64_t)q.k;
        pixels += rd[r].npix;
        items += ((uint64_t)rd[r].npix + 31) / 32;
        if ((uint32_t)q.k > max_k) max_k = (uint32_t)q.k;
    }
    if (items > 0xFFFFFFFFull) return set_error(VDI_ERR_INVALID_ARG, "batch table: too many work items");
    hd->n = (uint32_t)n;
    hd->total_items = (uint32_t)items;
    hd->total_pes = (uint32_t)pes;
    hd->prec_in = n > 0 ? (uint32_t)reqs[0].pe[0].prec : 0u;
    hd->max_k = max_k;
    hd->pad = 0;
    hd->total_pixels = pixels;
    return VDI_OK;
}

// Pooled batched path: pieces a request's pixel is expected to need (its K lists of at most N_S records
// cut into at most 2 K N_S - 1 pieces, at most the stage's), and the workspace: [header][counter]
// [list: 8 words, kBatchListCap entries at most][pool]
constexpr uint64_t kBatchListCap = 1u << 22;
constexpr uint64_t kBatchPoolCap = 1u << 28;

static uint64_t batch_pixel_pieces(const ReqDev& r) {
    const uint64_t est = 2ull * (uint64_t)r.k * (uint64_t)(r.out.n_s > 0 ? r.out.n_s : 1) + 1;
    return est < kPoolPiecesPerPixel ? est : kPoolPiecesPerPixel;
}

static size_t batch_list_bytes(const BatchHeader* hd) {
    const uint64_t n = hd->total_pixels < kBatchListCap ? hd->total_pixels : kBatchListCap;
    return align_up(32 + n * sizeof(BatchEntry), 256);
}

size_t batched_workspace_bytes(const void* host_table) {
    const BatchHeader* hd = static_cast<const BatchHeader*>(host_table);
    const ReqDev* rd = reinterpret_cast<const ReqDev*>(static_cast<const char*>(host_table) + hd->reqs_off);
    uint64_t est = 0;
    for (uint32_t q = 0; q < hd->n; ++q) est += (uint64_t)rd[q].npix * batch_pixel_pieces(rd[q]);
    if (est > kBatchPoolCap) est = kBatchPoolCap;
    if (est < kPoolPiecesPerPixel * 32) est = kPoolPiecesPerPixel * 32;
    return kWsHeader + 256 + batch_list_bytes(hd) + (size_t)est * (sizeof(float4) + sizeof(float2));
}

template <int PREC>
static cudaError_t launch_batched(const BatchArgs& a, const BatchHeader* hd, const ReqDev* rd, void* workspace,
                                  size_t ws_bytes, cudaStream_t st) {
    // workspace: [header][counter][list][pool: float4 x cap][pool: float2 x cap] (the list in build order, as
    // the pooled path's)
    char* base = static_cast<char*>(workspace);
    const size_t fixed = kWsHeader + 256 + batch_list_bytes(hd);
    if (ws_bytes < fixed) return cudaErrorInvalidValue;
    uint64_t cap = (ws_bytes - fixed) / (sizeof(float4) + sizeof(float2));
    if (cap > 0x7FFFFFFFu) cap = 0x7FFFFFFFu;
    if (cap < kPoolPiecesPerPixel * 32) return cudaErrorInvalidValue;  // one item's worst case
    const uint64_t list_cap = hd->total_pixels < kBatchListCap ? hd->total_pixels : kBatchListCap;
    BatchBuildArgs bb;
    bb.counter = reinterpret_cast<unsigned int*>(base + kWsHeader);
    bb.list = reinterpret_cast<uint32_t*>(base + kWsHeader + 256);
    bb.pool.cap = (uint32_t)cap;
    bb.pool.A = reinterpret_cast<float4*>(base + fixed);
    bb.pool.B = reinterpret_cast<float2*>(base + fixed + cap * sizeof(float4));
    const size_t sm = kStageWarps * sizeof(StageSmem);
    cudaError_t e = cudaFuncSetAttribute(composite_batched_build_kernel<PREC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int P = tree_leaves((int)hd->max_k);
    const size_t smd = P == 16 ? heads_smem_bytes<16>(128) : (P == 32 ? heads_smem_bytes<32>(128)
                                                                        : heads_smem_bytes<64>(128));
    auto km = P == 16 ? composite_batched_marked_kernel<16, PREC>
                      : (P == 32 ? composite_batched_marked_kernel<32, PREC> : composite_batched_marked_kernel<64, PREC>);
    e = cudaFuncSetAttribute(km, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smd);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, composite_batched_flat_kernel, 128, 0);
    if (e != cudaSuccess) return e;
    if (VDI_FLAT_CTAS_PER_SM > 0 && per_sm > VDI_FLAT_CTAS_PER_SM) per_sm = VDI_FLAT_CTAS_PER_SM;
    // chunks of whole items whose expected pieces fit the pool and whose pixels fit the list
    uint32_t item = 0;
    int q = 0;
    while (item < hd->total_items) {
        const uint32_t item0 = item;
        uint64_t pieces = 0, pixels = 0;
        while (item < hd->total_items) {
            while (q + 1 < (int)hd->n && rd[q + 1].item_begin <= item) ++q;
            const uint64_t px = 32;
            const uint64_t pc = px * batch_pixel_pieces(rd[q]);
            if (item > item0 && (pieces + pc > cap || pixels + px > list_cap)) break;
            pieces += pc;
            pixels += px;
            ++item;
        }
        BatchBuildArgs c = bb;
        c.item0 = item0;
        c.item1 = item;
        e = cudaMemsetAsync(bb.counter, 0, 256, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(bb.list, 0, 32, st);
        if (e != cudaSuccess) return e;
        composite_batched_build_kernel<PREC><<<(unsigned)stage_ctas(item - item0), kStageWarps * 32, sm, st>>>(a, c);
        uint64_t b = (uint64_t)device_sms() * (uint64_t)(per_sm > 0 ? per_sm : 1);
        const uint64_t need = (pixels + 127) / 128;
        if (b > need) b = need > 0 ? need : 1;
        composite_batched_flat_kernel<<<(unsigned)b, 128, 0, st>>>(a, bb.pool, bb.list);
        unsigned b3 = (unsigned)((pixels + 127) / 128);
        const unsigned cap3 = (unsigned)device_sms() * 2u;
        if (b3 > cap3) b3 = cap3;
        km<<<b3, 128, smd, st>>>(a, bb.list);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

vdi_status launch_composite_batched(const void* dev_table, const void* host_table, int iters, unsigned int* status,
                                    void* workspace, size_t ws_bytes, cudaStream_t st) {
    const BatchHeader* hd = static_cast<const BatchHeader*>(host_table);
    if (hd->n == 0 || hd->total_items == 0) return VDI_OK;
    BatchArgs a;
    a.reqs = reinterpret_cast<const ReqDev*>(static_cast<const char*>(dev_table) + hd->reqs_off);
    a.pes = reinterpret_cast<const PeIn*>(static_cast<const char*>(dev_table) + hd->pes_off);
    a.n = (int)hd->n;
    a.total_items = hd->total_items;
    a.status = status;
    a.iters = iters;
    const ReqDev* rd = reinterpret_cast<const ReqDev*>(static_cast<const char*>(host_table) + hd->reqs_off);
    const cudaError_t e = hd->prec_in == VDI_PREC_F32
                              ? launch_batched<VDI_PREC_F32>(a, hd, rd, workspace, ws_bytes, st)
                              : launch_batched<VDI_PREC_F16>(a, hd, rd, workspace, ws_bytes, st);
    return cuda_check(e, "composite_batched launch");
}

}  // namespace vdi
