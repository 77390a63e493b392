// Phase 1: sub-VDI generation (sec. 4, sec. 5.1).
//
// gen_count_kernel chooses gamma per (PE, ray): a fixed value, the per-ray
// bisection search of sec. 2.4, or a given per-ray value with the search as
// fallback.  It is a persistent kernel: CTAs of 64 threads take (PE, 16 x 4
// pixel tile) work items from an atomic counter (the paper used 16 x 16
// work-groups); each warp is an 8 x 4 pixel block so its rays read
// neighbouring cells.  Every thread owns a fixed slot of the sample cache in
// the workspace:
//   - the first march over the PE's owned samples counts the non-transparent
//     samples (the count at gamma = 0) and stores each of them, with the
//     number of transparent samples before it, in the slot (entry-major, so
//     a warp's later reads are coalesced).  An entry is 8 bytes: the
//     sample's table coordinate x = v * 255 and that gap.  Classification is
//     a function of x alone, so a cached march re-classifies x from the
//     table in shared memory (about 13 operations against the 24-byte
//     classified sample it replaces) and gets the volume march's colour and
//     opacity bit for bit;
//   - every bisection march then runs over the cached samples instead of
//     re-sampling the volume.  It evaluates a midpoint and both its children;
//     the sequential bisection choices are replayed from those counts.
// Rays with more non-transparent samples than a slot holds, and calls whose
// workspace has no room for the cache, re-march the volume instead (same
// decisions, same result).
//
// A run of transparent samples inside an open supersegment S is decided by
// its first sample: the criterion's distance |C_S| (1 - T_S^(1/m)) decreases
// strictly as the run lengthens S (m grows, nothing else changes), so if the
// first one is absorbed, so are the rest.  Every GPU path applies this rule,
// so cached, re-marched and emitting marches take identical decisions.
//
// gen_emit_kernel re-marches with the chosen gamma and writes the records at
// the prefix-sum offsets (compact layout, sec. 4).  The count kernel's first
// march records, per (PE, ray), the span from the first to the last
// non-transparent sample; emission marches only that span when the record is
// for its own inputs (samples outside it change no record).
//
// Non-convex ownership (sec. 5.3; the OWNED instantiations): a PE marches the
// samples of its bounding box and keeps those whose cell lies in one of its
// blocks.  Where the ray leaves the PE's domain and comes back, the open
// supersegment ends (a "break"): every candidate closes, emission writes the
// record, and the next non-transparent sample opens a new supersegment even
// when the budget is spent.  The cache marks a break by a negative gap on
// the next cached sample; at gamma = 2 each run of the domain that holds a
// non-transparent sample gives one supersegment, so the search's upper end
// counts those runs.
#include <climits>
#include <float.h>

#include "vdi_device.cuh"

namespace vdi {

// One generation request's parameters, shared by its PEs.
struct GenReq {
    CamDev cam;
    int dims[3];
    const float* lut;  // 256 x 4, straight colour + opacity per ref_len
    float scale255, step, ref_len;
    int k, n_s, iters;
    int mode;  // 0 fixed, 1 search, 2 given (+ fallback), 3 learned bracket (+ fallback)
    float gamma;
    int prec;
    int tiles_x, tiles_y;
    OwnerDev own;  // non-convex ownership (own.map != nullptr): b[e] is the bounding box of PE e's blocks
};

struct GenArgs {
    GenReq r;
    BrickDev b[VDI_MAX_PE];
    CompactDev out[VDI_MAX_PE];
    unsigned int* status;
    unsigned int* counter;  // work-item counter (persistent kernel)
    float2* cache;          // sample cache: [cap][slots] (table coordinate x, transparent samples before it)
    int cache_cap, slots;
    // each (PE, ray)'s samples from its first to its last non-transparent one, [x, y) (PE-major), and the
    // tag of the inputs they were recorded for: the count kernel records them, the emit kernel marches
    // only that span when the tag matches its own inputs' (nullptr: neither)
    uint2* ranges;
    unsigned long long* range_tag;
    unsigned long long tag;
};

// gen_count_kernel: CTAs of two warps on 16 x 4 tiles, VDI_COUNT_MIN_BLOCKS per SM (the register
// bound follows), so that a tile's barrier waits on one other warp's searches; gen_emit_kernel: four
// warps on 16 x 8 tiles
#ifndef VDI_COUNT_MIN_BLOCKS
#define VDI_COUNT_MIN_BLOCKS 12
#endif
constexpr int kTileW = 16, kCountTileH = 4, kCountThreads = 64, kEmitTileH = 8, kEmitThreads = 128;
constexpr int kCacheCap = 1024;  // cached non-transparent samples per (PE, ray)

// Work census (VDI_FLAG_CENSUS): kept in registers; the kernel variant
// without the census never stores it, so the counting is compiled out.
struct Census {
    unsigned long long evals = 0, steps = 0, passes = 0, searched = 0, overflow = 0, cached = 0, remarched = 0;
};

// 257 entries of colour/opacity, then their differences to the next entry; opacity
// corrected to the step length: a' = 1 - (1 - a)^(step / ref_len).
__device__ __forceinline__ void load_lut(const GenReq& a, float4* lut2) {
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
        lut2[i] = v;
        lut2[257 + i] = make_float4(__fsub_rn(w.x, v.x), __fsub_rn(w.y, v.y), __fsub_rn(w.z, v.z),
                                      __fsub_rn(w.w, v.w));
    }
    __syncthreads();
}

// pixel of this thread in tile `tile` (th rows): warps are 8 x 4 blocks, two per row of blocks
__device__ __forceinline__ void tile_pixel(int tiles_x, int tile, int th, int& i, int& j) {
    int tx = tile % tiles_x, ty = tile / tiles_x;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    i = tx * kTileW + (warp & 1) * 8 + (lane & 7);
    j = ty * th + (warp >> 1) * 4 + (lane >> 3);
}

// PE owning the cell of fixed-point midpoint P (clamped to the volume's cells).
__device__ __forceinline__ int owner_at(const GenReq& a, const long long P[3]) {
    int bl[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        int c = fixed_cell(P[q]);
        c = c < 0 ? 0 : (c > a.dims[q] - 2 ? a.dims[q] - 2 : c);
        bl[q] = c >> a.own.shift;
    }
    return __ldg(a.own.map + ((size_t)bl[2] * a.own.nb[1] + bl[1]) * a.own.nb[0] + bl[0]);
}

// Number of samples, from the one at fixed-point position P on, whose
// midpoints stay in the same block of 2^shift cells on every axis (at least
// 1, at most limit).  Blocks are taken on the unclamped cell index: every
// sample of such a run also has the same clamped cell block, hence one owner.
__device__ __forceinline__ int block_span(const long long P[3], const long long D[3], int shift, int limit) {
    const int S = kFrac + shift;
    long long n = limit;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const long long d = D[q];
        if (d == 0) continue;
        const long long blk = P[q] >> S;  // floor
        long long m;
        if (d > 0) m = (((blk + 1) << S) - P[q] + d - 1) / d;  // first m with P + m d >= next boundary
        else m = (P[q] - (blk << S)) / (-d) + 1;                // first m with P + m d < this boundary
        n = m < n ? m : n;
    }
    return (int)(n > 1 ? n : 1);
}

// march() restricted to the samples PE e owns, block by block: a block PE e
// does not own is passed over in one step; on_break() is called before the
// first owned sample after a stretch of samples the PE does not own.
template <typename F, typename B>
__device__ __forceinline__ void march_owned(const Ray& r, int k0, int k1, const BrickDev& b,
                                            const float4* __restrict__ lut2, float scale255, const GenReq& a, int e,
                                            F&& f, B&& on_break) {
    long long P[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) P[q] = r.P0[q] + (long long)k0 * r.D[q];
    bool seen = false, away = false;
    int k = k0;
    while (k < k1) {
        const int n = block_span(P, r.D, a.own.shift, k1 - k);
        if (owner_at(a, P) != e) {
            away = seen;
            k += n;
#pragma unroll
            for (int q = 0; q < 3; ++q) P[q] += (long long)n * r.D[q];
            continue;
        }
        if (away) {
            on_break();
            away = false;
        }
        seen = true;
        // the block's samples; the next cell is loaded while the current one is processed
        float4 clo, chi;
        cell_load(P, b, clo, chi);
        for (int j = 0; j < n; ++j, ++k) {
            const float w0 = fixed_frac(P[0]), w1 = fixed_frac(P[1]), w2 = fixed_frac(P[2]);
#pragma unroll
            for (int q = 0; q < 3; ++q) P[q] += r.D[q];
            float4 nlo, nhi;
            cell_load(P, b, nlo, nhi);
            Sample s;
            sample_from(w0, w1, w2, clo, chi, lut2, scale255, s);
            f(k, s);
            clo = nlo;
            chi = nhi;
        }
    }
}

// ---------------------------------------------------------------------------
// State machine of one gamma candidate over generation samples (all of one
// step's length): m = samples in S (0: closed), r = 1/m; `run` = S is inside
// a transparent run whose first sample was absorbed.
// ---------------------------------------------------------------------------
struct GenCount {
    float P[3], A, L2, m;
    int cnt;
    bool run;
};

__device__ __forceinline__ void gc_reset(GenCount& s) {
    s.m = 0.f;
    s.cnt = 0;
    s.run = false;
}

__device__ __forceinline__ void gc_open(GenCount& s, const float P[3], float a, float lgT) {
    s.P[0] = P[0]; s.P[1] = P[1]; s.P[2] = P[2];
    s.A = a; s.L2 = lgT; s.m = 1.f;
    s.run = false;
    ++s.cnt;
}

// one sample (P premultiplied, opacity a, lgT = log2(1 - a))
__device__ __forceinline__ void gc_step(GenCount& s, const float P[3], float a, float lgT, float g2, int cap) {
    if (s.m == 0.f) {
        if (a > 0.f) gc_open(s, P, a, lgT);
        return;
    }
    if (a == 0.f && s.run) {  // rest of an absorbed transparent run
        s.m = __fadd_rn(s.m, 1.f);
        return;
    }
    if (s.cnt < cap && criterion(s.P, s.A, s.L2, rcp_approx(s.m), P, g2)) {
        if (a > 0.f) gc_open(s, P, a, lgT);
        else s.m = 0.f;
    } else if (a > 0.f) {
        absorb(s.P, s.A, s.L2, P, a, lgT);
        s.m = __fadd_rn(s.m, 1.f);
        s.run = false;
    } else {
        s.m = __fadd_rn(s.m, 1.f);
        s.run = true;
    }
}

// a run of n >= 1 transparent samples, all at once (same decisions as n gc_step calls)
__device__ __forceinline__ void gc_run(GenCount& s, float n, float g2, int cap) {
    if (s.m == 0.f) return;
    if (s.cnt < cap && criterion_clear(s.P, s.A, s.L2, rcp_approx(s.m), g2)) {
        s.m = 0.f;
    } else {
        s.m = __fadd_rn(s.m, n);
        s.run = true;
    }
}

// The same steps without branches, for the cached marches (every cached sample
// is non-transparent, no budget): both outcomes are computed with the same
// rounded operations and one is selected, so the decisions are gc_run's and
// gc_step's bit for bit, and the three candidates of a march form straight-line
// code whose dependency chains the compiler can interleave.  A closed S (m = 0)
// takes 1/0 = inf into the criterion, whose result is then not used (a closed S
// neither closes nor absorbs: the sample opens a new one).
__device__ __forceinline__ void gc_run_select(GenCount& s, float n, float g2) {
    const bool open = s.m != 0.f;
    const bool close = open && criterion_clear(s.P, s.A, s.L2, rcp_approx(s.m), g2);
    s.m = close ? 0.f : (open ? __fadd_rn(s.m, n) : s.m);
    s.run = open && !close;
}

__device__ __forceinline__ void gc_step_opaque_select(GenCount& s, const float P[3], float a, float lgT, float g2) {
    const bool open = s.m != 0.f;
    const bool fresh = !open || criterion(s.P, s.A, s.L2, rcp_approx(s.m), P, g2);
    const float T = __fsub_rn(1.f, s.A);
#pragma unroll
    for (int c = 0; c < 3; ++c) s.P[c] = fresh ? P[c] : __fmaf_rn(T, P[c], s.P[c]);
    s.A = fresh ? a : __fmaf_rn(T, a, s.A);
    s.L2 = fresh ? lgT : __fadd_rn(s.L2, lgT);
    s.m = fresh ? 1.f : __fadd_rn(s.m, 1.f);
    s.cnt += fresh ? 1 : 0;
    s.run = false;
}

// ---------------------------------------------------------------------------
// Marches
// ---------------------------------------------------------------------------
struct CacheRef {
    float2* e;
    int slot, slots, cap;
    __device__ __forceinline__ size_t at(int j) const { return (size_t)j * slots + slot; }
};

// First march: counts non-transparent samples and, if `c` is given, caches
// them (up to c->cap).  NC gamma candidates ride along (NC may be 0).  OWNED:
// PE e's samples under the ownership map of *ga; *runs receives the number of
// domain runs holding a non-transparent sample (the count at gamma = 2).
template <int NC, bool OWNED = false>
__device__ __forceinline__ int first_march(const Ray& r, int k0, int k1, const BrickDev& b, const float4* lut2,
                                           float scale255, const float* g2, int cap, const CacheRef* c, int* cnt,
                                           Census& cs, const GenReq* ga = nullptr, int e = 0, int* runs = nullptr,
                                           int* kspan = nullptr) {
    cs.evals += (unsigned long long)(k1 - k0);
    cs.steps += (unsigned long long)(k1 - k0) * NC;
    cs.passes += 1;
    GenCount st[NC > 0 ? NC : 1];
#pragma unroll
    for (int q = 0; q < NC; ++q) gc_reset(st[q]);
    int nt = 0, gap = 0, nruns = 0, kf = 0, kl = 0;
    bool brk = false;
    auto visit = [&](int k, const Sample& s) {
        if (s.a > 0.f) {
            if (kspan) {
                kf = nt == 0 ? k : kf;
                kl = k;
            }
            if (c && nt < c->cap) c->e[c->at(nt)] = make_float2(s.x, (OWNED && brk) ? -1.f : (float)gap);
            if (OWNED && (nruns == 0 || brk)) ++nruns;
            brk = false;
            ++nt;
            gap = 0;
        } else {
            ++gap;
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) gc_step(st[q], s.P, s.a, s.lgT, g2[q], cap);
    };
    if constexpr (OWNED) {
        march_owned(r, k0, k1, b, lut2, scale255, *ga, e, visit, [&]() {
            brk = true;
            gap = 0;
#pragma unroll
            for (int q = 0; q < NC; ++q) st[q].m = 0.f;
        });
        *runs = nruns;
    } else {
        march(r, k0, k1, b, lut2, scale255, visit);
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) cnt[q] = st[q].cnt;
    if (kspan) {
        kspan[0] = kf;
        kspan[1] = kl + 1;
    }
    return nt;
}

// entries of the sample cache loaded ahead of their use in a cached march: a ring of registers that the
// unrolled loop indexes statically (4 ahead: 19.1 ms for the plain frame's search, against 19.5 ms with a
// pair of registers shifted two ahead)
#ifndef VDI_GEN_PREFETCH
#define VDI_GEN_PREFETCH 4
#endif

// Bisection march over the cached samples: three candidates.  Entries are
// read VDI_GEN_PREFETCH ahead of their use so the loads overlap the
// state-machine work, and re-classified from the table.  OWNED: a negative
// gap marks a break before the entry.
template <bool OWNED = false>
__device__ __forceinline__ void cached_march(const CacheRef& c, int nt, const float4* __restrict__ lut2,
                                             const float g2[3], int cnt[3], Census& cs) {
    cs.steps += (unsigned long long)nt * 3;
    cs.passes += 1;
    GenCount st[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) gc_reset(st[q]);
    auto entry = [&](const float2 y) {
        Sample s;
        classify_x(y.x, lut2, s);
        if (OWNED && y.y < 0.f) {
#pragma unroll
            for (int q = 0; q < 3; ++q) st[q].m = 0.f;
        }
        if (y.y > 0.f) {
#pragma unroll
            for (int q = 0; q < 3; ++q) gc_run_select(st[q], y.y, g2[q]);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) gc_step_opaque_select(st[q], s.P, s.a, s.lgT, g2[q]);
    };
    constexpr int PF = VDI_GEN_PREFETCH;
    float2 y[PF];
    const float2* ld = c.e + c.slot;  // entry j of the slot at ld + j * slots
    const size_t stride = (size_t)c.slots;
#pragma unroll
    for (int u = 0; u < PF; ++u) {
        y[u] = u < nt ? __ldcg(ld) : make_float2(0.f, 0.f);
        ld += stride;
    }
    for (int j0 = 0; j0 < nt; j0 += PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            if (j0 + u < nt) {
                const float2 yy = y[u];
                if (j0 + u + PF < nt) y[u] = __ldcg(ld);
                ld += stride;
                entry(yy);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) cnt[q] = st[q].cnt;
}


// Bisection march over the volume: three candidates.
template <bool OWNED = false>
__device__ __forceinline__ void volume_march(const Ray& r, int k0, int k1, const BrickDev& b, const float4* lut2,
                                             float scale255, const float g2[3], int cnt[3], Census& cs,
                                             const GenReq* ga, int e) {
    int runs = 0;
    first_march<3, OWNED>(r, k0, k1, b, lut2, scale255, g2, INT_MAX, nullptr, cnt, cs, ga, e, &runs);
}

// Per-ray bisection of gamma, two levels per march (each march evaluates the
// midpoint and both of its children), in one of three phases that share the
// march's call sites, so that the learned instantiation inlines one cached and
// one volume march, as the search does:
//   kBisSearch: the search of sec. 2.4, called when the count at gamma = 0
//     (nt) exceeds n_s: sequential bisection of [0, 2] for `iters` levels;
//     `runs` is the count at gamma = 2 (OWNED; otherwise 1).
//   kBisBracket (learned): the prediction gp is feasible (count cp <= n_s):
//     six levels of bisection of log2 gamma over [log2 gp - 4, log2 gp].
//   kBisTop (learned): gp is infeasible: one march evaluates log2 gp + 4 (the
//     bracket's top), its midpoint and left quarter; an infeasible top falls
//     back to the search, otherwise the bisection continues in the bracket.
// A midpoint whose count is within n_s becomes the upper end, and stops the
// bisection if its count is exactly n_s.  Returns the upper end's gamma (the
// smallest feasible gamma found; for the learned brackets within a factor
// 2^(1/16) of the bracket's threshold) and its count.  The census counts a
// fallback from kBisTop as a searched ray.
enum : int { kBisTop = 0, kBisBracket = 1, kBisSearch = 2 };

// the learned bracket: its width in octaves of gamma and its levels of bisection (1024^3, K = 16,
// N_S = 32: 4 octaves in 6 levels give 1.43% supersegment-count error against the search; 4 levels,
// one cached march fewer, 1.14x faster but 5.3-6.2% count error at 2-4 octaves; 5 levels cost as much
// as 6)
#ifndef VDI_LEARNED_OCTAVES
#define VDI_LEARNED_OCTAVES 4.f
#endif
#ifndef VDI_LEARNED_LEVELS
#define VDI_LEARNED_LEVELS 6
#endif

template <bool LEARNED, bool OWNED = false>
__device__ __forceinline__ float bisect_gamma(const Ray& r, int k0, int k1, const BrickDev& b, const float4* lut2,
                                              float scale255, int n_s, int iters, int nt, const CacheRef* c,
                                              int phase, float gp, int cp, int& count, Census& cs,
                                              const GenReq* ga = nullptr, int e = 0, int runs = 1) {
    constexpr float R = VDI_LEARNED_OCTAVES;   // learned bracket: octaves of gamma
    constexpr int kLevels = VDI_LEARNED_LEVELS;  // learned bracket: levels of bisection in log2 gamma
    float lo, hi, ghi;
    int cnt_hi, it, levels;
    if (LEARNED && phase != kBisSearch) {
        const float lg = log2f(fmaxf(gp, 0x1p-30f));
        it = 0;
        levels = kLevels;
        lo = lg;
        hi = lg + R;
        ghi = 0.f;
        cnt_hi = 0;
        if (phase == kBisBracket) {
            hi = lg;
            ghi = gp;
            cnt_hi = cp;
            lo = lg - R;
            if (cp == n_s) it = levels;
        }
    } else {
        phase = kBisSearch;
        lo = 0.f;
        hi = 2.f;
        ghi = 2.f;
        // the distance never reaches 2: one supersegment per domain run
        cnt_hi = nt > 0 ? (OWNED ? runs : 1) : 0;
        it = 0;
        levels = iters;
    }
    while (it < levels) {
        float x[3];
        if (LEARNED && phase == kBisTop) {
            x[0] = hi;
            x[1] = lo + 0.5f * R;
            x[2] = lo + 0.25f * R;
        } else {
            const float mid = 0.5f * (lo + hi);
            x[0] = mid;
            x[1] = 0.5f * (lo + mid);
            x[2] = 0.5f * (mid + hi);
        }
        float g[3], g2[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            g[q] = (LEARNED && phase != kBisSearch) ? exp2f(x[q]) : x[q];
            g2[q] = __fmul_rn(g[q], g[q]);
        }
        int cnt[3];
        if (c) {
            cached_march<OWNED>(*c, nt, lut2, g2, cnt, cs);
            cs.cached += 1;
        } else {
            volume_march<OWNED>(r, k0, k1, b, lut2, scale255, g2, cnt, cs, ga, e);
            cs.remarched += 1;
        }
        if (LEARNED && phase == kBisTop) {
            if (cnt[0] > n_s) {
                // no feasible gamma in the bracket: the full search
                cs.searched += 1;
                cs.overflow += c ? 0 : 1;
                phase = kBisSearch;
                lo = 0.f;
                hi = 2.f;
                ghi = 2.f;
                cnt_hi = nt > 0 ? (OWNED ? runs : 1) : 0;
                it = 0;
                levels = iters;
                continue;
            }
            phase = kBisBracket;
            hi = x[0];
            ghi = g[0];
            cnt_hi = cnt[0];
            ++it;
            if (cnt[1] <= n_s) {
                hi = x[1];
                ghi = g[1];
                cnt_hi = cnt[1];
                if (cnt[1] != n_s) {
                    ++it;
                    if (cnt[2] <= n_s) {
                        hi = x[2];
                        ghi = g[2];
                        cnt_hi = cnt[2];
                    } else {
                        lo = x[2];
                    }
                }
            } else {
                lo = x[1];
            }
            if (cnt_hi == n_s) break;
            continue;
        }
        // level 1: the midpoint
        ++it;
        int child;
        if (cnt[0] <= n_s) {
            hi = x[0];
            ghi = g[0];
            cnt_hi = cnt[0];
            if (cnt[0] == n_s) break;
            child = 1;
        } else {
            lo = x[0];
            child = 2;
        }
        if (it >= levels) break;
        // level 2: the child inside the new bracket
        ++it;
        const int cc = cnt[child];
        if (cc <= n_s) {
            hi = x[child];
            ghi = g[child];
            cnt_hi = cc;
            if (cc == n_s) break;
        } else {
            lo = x[child];
        }
    }
    count = cnt_hi;
    return ghi;
}

// gamma and count of one (PE, ray): the body of the count kernels.  The
// learned-gamma refinement (mode 3) is compiled only into the LEARNED
// instantiation so that the search kernel keeps its register budget.  Every
// march is inlined: out-of-line calls in this persistent loop cost far more
// than the spills inlining brings (the learned choice took 80.6 ms with the
// refinement, its marches and the search fallback out of line, 65.6 ms inlined).
template <bool LEARNED, bool OWNED>
__device__ __forceinline__ void count_ray(const GenReq& a, const BrickDev& b, const CompactDev& o, int e, int i, int j,
                                          const float4* __restrict__ lut2, const CacheRef& cref, Census& cs,
                                          unsigned long long& rays, uint2* rng) {
    const int mode = LEARNED ? 3 : a.mode;
    const size_t p = (size_t)j * a.cam.W + i;
    Ray r;
    int k0 = 0, k1 = 0;
    const bool any = ray_setup(a.cam, i, j, a.dims, a.step, r) && owned_range(r, a.step, b, a.dims, k0, k1);
    float gamma = mode == 0 ? a.gamma : (mode >= 2 ? fmaxf(o.gamma[p], 0.f) : 0.f);
    int count = 0;
    int runs = 1;
    // the span from the first to the last non-transparent sample (box domains): samples outside it change
    // no count and no record
    int kspan[2] = {0, 0};
    int* ks = OWNED ? nullptr : kspan;
    if (any) {
        rays += 1;
        if (mode == 0) {
            const float g2[1] = {__fmul_rn(a.gamma, a.gamma)};
            int c[1];
            const int nt = first_march<1, OWNED>(r, k0, k1, b, lut2, a.scale255, g2, a.n_s, nullptr, c, cs, &a, e,
                                                 &runs, ks);
            count = c[0];
            if (!OWNED && rng && nt > 0) *rng = make_uint2((unsigned)kspan[0], (unsigned)kspan[1]);
        } else {
            const bool use_cache = cref.e != nullptr;
            int nt;
            bool searched = true;
            int phase = kBisSearch, cp = 0;
            if (mode >= 2) {
                // one march: count at the given gamma, non-transparent count, cache
                const float g2[1] = {__fmul_rn(gamma, gamma)};
                int c[1];
                nt = first_march<1, OWNED>(r, k0, k1, b, lut2, a.scale255, g2, INT_MAX, use_cache ? &cref : nullptr,
                                           c, cs, &a, e, &runs, ks);
                cp = c[0];
                if (mode == 2) {
                    if (c[0] <= a.n_s) {
                        count = c[0];
                        searched = false;
                    }
                } else if (LEARNED && nt > a.n_s && use_cache && nt <= cref.cap) {
                    phase = c[0] <= a.n_s ? kBisBracket : kBisTop;
                }
            } else {
                int dummy[1];
                nt = first_march<0, OWNED>(r, k0, k1, b, lut2, a.scale255, nullptr, INT_MAX,
                                           use_cache ? &cref : nullptr, dummy, cs, &a, e, &runs, ks);
            }
            if (!OWNED && nt > 0) {
                if (rng) *rng = make_uint2((unsigned)kspan[0], (unsigned)kspan[1]);
                // a search that re-marches the volume marches the span only (same counts)
                k0 = kspan[0];
                k1 = kspan[1];
            }
            if (searched) {
                if (nt <= a.n_s) {
                    gamma = 0.f;
                    count = nt;
                } else {
                    const CacheRef* c = (use_cache && nt <= cref.cap) ? &cref : nullptr;
                    if (phase == kBisSearch) {
                        cs.searched += 1;
                        cs.overflow += c ? 0 : 1;
                    }
                    gamma = bisect_gamma<LEARNED, OWNED>(r, k0, k1, b, lut2, a.scale255, a.n_s, a.iters, nt, c, phase,
                                                         gamma, cp, count, cs, &a, e, runs);
                }
            }
        }
    }
    o.counts[p] = (uint32_t)count;
    if (o.gamma) o.gamma[p] = gamma;
}

__device__ __forceinline__ void census_flush_gen(const Census& cs, unsigned long long rays, unsigned int* status) {
    unsigned long long* ctr = reinterpret_cast<WsHeader*>(status)->counters;
    atomicAdd(ctr + 0, cs.evals);
    atomicAdd(ctr + 1, cs.steps);
    atomicAdd(ctr + 2, cs.passes);
    atomicAdd(ctr + 3, rays);
    atomicAdd(ctr + 4, cs.searched);
    atomicAdd(ctr + 5, cs.overflow);
    atomicAdd(ctr + 6, cs.cached);
    atomicAdd(ctr + 7, cs.remarched);
}

// the learned instantiation's block bound (its first march at the prediction adds live state)
#ifndef VDI_LEARNED_MIN_BLOCKS
#define VDI_LEARNED_MIN_BLOCKS 10
#endif
template <bool CENSUS, bool LEARNED, bool OWNED = false>
__global__ void __launch_bounds__(kCountThreads, LEARNED ? VDI_LEARNED_MIN_BLOCKS : VDI_COUNT_MIN_BLOCKS)
    gen_count_kernel(
    const __grid_constant__ GenArgs a) {
    __shared__ float4 lut2[2 * 257];
    __shared__ unsigned int s_item;
    if (a.range_tag && blockIdx.x == 0 && threadIdx.x == 0) *a.range_tag = a.tag;
    load_lut(a.r, lut2);
    const unsigned tiles = (unsigned)(a.r.tiles_x * a.r.tiles_y);
    const unsigned total = tiles * (unsigned)a.r.k;
    CacheRef cref;
    cref.e = a.cache;
    cref.slot = blockIdx.x * blockDim.x + threadIdx.x;
    cref.slots = a.slots;
    cref.cap = a.cache_cap;
    Census cs;
    unsigned long long rays = 0;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u);
        __syncthreads();
        const unsigned item = s_item;
        __syncthreads();
        if (item >= total) break;
        const int e = (int)(item / tiles);
        int i, j;
        tile_pixel(a.r.tiles_x, (int)(item % tiles), kCountTileH, i, j);
        if (i >= a.r.cam.W || j >= a.r.cam.H) continue;
        count_ray<LEARNED, OWNED>(a.r, a.b[e], a.out[e], e, i, j, lut2, cref, cs, rays,
                                  a.ranges ? a.ranges + (size_t)e * a.r.cam.W * a.r.cam.H +
                                                 ((size_t)j * a.r.cam.W + i)
                                           : nullptr);
    }
    if (CENSUS) census_flush_gen(cs, rays, a.status);
}

struct RecOut {
    float f, b, P[3], A;
    float L2;  // log2(1 - A) of the record: its FP16 form stores -L2
};

__device__ __forceinline__ void store_record(unsigned int* status, int prec, const CompactDev& o, uint64_t idx,
                                             const RecOut& r) {
    if (idx >= o.capacity) {
        atomicCAS(status, 0u, (unsigned)VDI_ERR_CAPACITY);
        return;
    }
    if (prec == VDI_PREC_F32) {
        reinterpret_cast<float4*>(o.rgba)[idx] = make_float4(r.P[0], r.P[1], r.P[2], r.A);
        reinterpret_cast<float2*>(o.fb)[idx] = make_float2(r.f, r.b);
    } else {
        reinterpret_cast<uint4*>(o.rgba)[idx] = f16_pack(r.f, r.b, r.P[0], r.P[1], r.P[2], r.L2);
    }
}

// Emission of pixel (i, j) of PE e (one CTA = one tile of kEmitThreads pixels of one PE; `inside`:
// the pixel lies in the image).  REGULAR: records at p * n_s with a zero tail.  Compile-time, so that
// the compact path carries none of it (as a run-time flag it cost the compact emission 70%).
template <bool OWNED, bool REGULAR>
__device__ __forceinline__ void emit_ray(const GenReq& a, const BrickDev& b, const CompactDev& o, int e, int i, int j,
                                         bool inside, float4* lut2, unsigned int* status, const uint2* rng) {
    const size_t p = inside ? (size_t)j * a.cam.W + i : 0;
    const uint32_t want = inside ? o.counts[p] : 0u;
    // most (PE, tile) pairs hold no record (rays that miss the PE's box): such a CTA of the compact
    // layout leaves before building the table
    if constexpr (!REGULAR) {
        if (!__syncthreads_or(want > 0)) return;
    }
    load_lut(a, lut2);
    if (!inside) return;
    uint32_t written = 0;
    // regular layout: the slots after the pixel's records are zero
    auto zero_tail = [&]() {
        if constexpr (REGULAR) {
            const RecOut z{0.f, 0.f, {0.f, 0.f, 0.f}, 0.f, 0.f};
            for (uint32_t q = min(written, (uint32_t)a.n_s); q < (uint32_t)a.n_s; ++q)
                store_record(status, a.prec, o, (uint64_t)p * (uint64_t)a.n_s + q, z);
        }
    };
    if (want == 0) {
        zero_tail();
        return;
    }
    // records that fit: a pixel of the regular layout owns n_s slots (counts never exceed n_s for
    // box-shaped domains); a compact list cut by the capacity keeps the records that fit as its
    // count, so the sub-VDI stays valid input for compositing, and the status reports the overflow
    uint64_t base;
    uint32_t room = want;
    if constexpr (REGULAR) {
        base = (uint64_t)p * (uint64_t)a.n_s;
        room = min(want, (uint32_t)a.n_s);
    } else {
        base = o.offsets[p];
        if (base + want > o.capacity) {
            room = base >= o.capacity ? 0u : (uint32_t)(o.capacity - base);
            o.counts[p] = room;
            atomicCAS(status, 0u, (unsigned)VDI_ERR_CAPACITY);
        }
    }
    Ray r;
    int k0 = 0, k1 = 0;
    if (!(ray_setup(a.cam, i, j, a.dims, a.step, r) && owned_range(r, a.step, b, a.dims, k0, k1))) {
        zero_tail();
        return;
    }
    if (!OWNED && rng) {
        // the span the count kernel recorded: before its first non-transparent sample no supersegment is
        // open, and after its last one transparent samples only absorb into or close the open one, whose
        // values and back depth they leave unchanged
        const uint2 g = rng[p];
        k0 = max(k0, (int)g.x);
        k1 = min(k1, (int)g.y);
    }
    const float gamma = o.gamma ? o.gamma[p] : a.gamma;
    const float g2 = __fmul_rn(gamma, gamma);
    const int cap = a.n_s;
    // the GenCount state machine (same decisions), tracking the records
    GenCount st;
    gc_reset(st);
    int kopen = 0, klast = 0;
    auto visit = [&](int k, const Sample& s) {
        const bool was_open = st.m != 0.f;
        const int before = st.cnt;
        const RecOut cur{sample_front(r, a.step, kopen), sample_front(r, a.step, klast + 1),
                         {st.P[0], st.P[1], st.P[2]}, st.A, st.L2};
        gc_step(st, s.P, s.a, s.lgT, g2, cap);
        // S closed by this sample: either it was shut (m = 0) or a new one opened
        const bool closed = was_open && (st.m == 0.f || st.cnt != before);
        if (closed) {
            if (written < room) store_record(status, a.prec, o, base + written, cur);
            ++written;
        }
        if (st.cnt != before) {
            kopen = k;
            klast = k;
        } else if (st.m != 0.f && s.a > 0.f) {
            klast = k;
        }
    };
    if constexpr (OWNED) {
        // leaving the PE's domain ends the open supersegment (sec. 5.3)
        march_owned(r, k0, k1, b, lut2, a.scale255, a, e, visit, [&]() {
            if (st.m == 0.f) return;
            const RecOut cur{sample_front(r, a.step, kopen), sample_front(r, a.step, klast + 1),
                             {st.P[0], st.P[1], st.P[2]}, st.A, st.L2};
            if (written < room) store_record(status, a.prec, o, base + written, cur);
            ++written;
            st.m = 0.f;
        });
    } else {
        march(r, k0, k1, b, lut2, a.scale255, visit);
    }
    if (st.m != 0.f) {
        if (written < room) {
            RecOut ro{sample_front(r, a.step, kopen), sample_front(r, a.step, klast + 1), {st.P[0], st.P[1], st.P[2]},
                      st.A, st.L2};
            store_record(status, a.prec, o, base + written, ro);
        }
        ++written;
    }
    if (written != want) atomicCAS(status, 0u, (unsigned)VDI_ERR_CUDA);
    zero_tail();
}

template <bool OWNED, bool REGULAR>
#ifndef VDI_EMIT_MIN_BLOCKS
#define VDI_EMIT_MIN_BLOCKS 8
#endif
__global__ void __launch_bounds__(kEmitThreads, VDI_EMIT_MIN_BLOCKS) gen_emit_kernel(const __grid_constant__ GenArgs a) {
    __shared__ float4 lut2[2 * 257];
    int i, j;
    tile_pixel(a.r.tiles_x, blockIdx.x, kEmitTileH, i, j);
    const bool inside = i < a.r.cam.W && j < a.r.cam.H;
    const int e = blockIdx.y;
    const bool spans = !OWNED && a.ranges && *a.range_tag == a.tag;
    emit_ray<OWNED, REGULAR>(a.r, a.b[e], a.out[e], e, i, j, inside, lut2, a.status,
                             spans ? a.ranges + (size_t)e * a.r.cam.W * a.r.cam.H : nullptr);
}

// ---------------------------------------------------------------------------
// Batched generation: uneven requests (their own volumes, cameras, image
// sizes, K, N_S, gamma modes and precisions) in one persistent count launch
// over (request, PE, 16 x 4 tile) items, one batched prefix sum and one emit
// launch over (request, PE, 16 x 8 tile) items.  The table (host and device
// copies, the same bytes): [header][GenBatchReq x n][GenBatchPe x sum k]
// [ScanList x sum k].
// ---------------------------------------------------------------------------
struct GenBatchReq {
    GenReq r;
    uint32_t item_begin;   // first count item of the request
    uint32_t eitem_begin;  // first emit item
    uint32_t pe_begin;     // first PE descriptor
    int etiles_y;          // emit tile rows
};

struct GenBatchPe {
    BrickDev b;
    CompactDev out;
};

struct GenBatchHeader {
    uint32_t n, total_items, total_eitems, total_pes;
    uint32_t total_chunks, pad;
    uint64_t reqs_off, pes_off, lists_off;
};

struct GenBatchArgs {
    const GenBatchReq* reqs;
    const GenBatchPe* pes;
    int n;
    uint32_t total_items;
    unsigned int* status;
    unsigned int* counter;
    float2* cache;
    int cache_cap, slots;
};

// the request holding work item `item` (the last one beginning at or before it)
template <bool EMIT>
__device__ __forceinline__ int batch_request(const GenBatchReq* reqs, int n, uint32_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const uint32_t b = EMIT ? __ldg(&reqs[mid].eitem_begin) : __ldg(&reqs[mid].item_begin);
        if (b <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kCountThreads, VDI_COUNT_MIN_BLOCKS) gen_count_batched_kernel(const __grid_constant__ GenBatchArgs a) {
    __shared__ float4 lut2[2 * 257];
    __shared__ unsigned int s_item;
    CacheRef cref;
    cref.e = a.cache;
    cref.slot = blockIdx.x * blockDim.x + threadIdx.x;
    cref.slots = a.slots;
    cref.cap = a.cache_cap;
    Census cs;
    unsigned long long rays = 0;
    int cur = -1;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u);
        __syncthreads();
        const unsigned item = s_item;
        __syncthreads();
        if (item >= a.total_items) break;
        const int q = batch_request<false>(a.reqs, a.n, item);
        const GenBatchReq& br = a.reqs[q];
        if (q != cur) {  // the CTA's table follows its request (q is the same for the whole CTA)
            load_lut(br.r, lut2);
            cur = q;
        }
        const unsigned tiles = (unsigned)(br.r.tiles_x * br.r.tiles_y);
        const unsigned local = item - br.item_begin;
        const int e = (int)(local / tiles);
        int i, j;
        tile_pixel(br.r.tiles_x, (int)(local % tiles), kCountTileH, i, j);
        if (i >= br.r.cam.W || j >= br.r.cam.H) continue;
        const GenBatchPe& pe = a.pes[br.pe_begin + e];
        count_ray<false, false>(br.r, pe.b, pe.out, e, i, j, lut2, cref, cs, rays, nullptr);
    }
}

__global__ void __launch_bounds__(kEmitThreads, VDI_EMIT_MIN_BLOCKS) gen_emit_batched_kernel(const __grid_constant__ GenBatchArgs a) {
    __shared__ float4 lut2[2 * 257];
    const uint32_t item = blockIdx.x;
    const int q = batch_request<true>(a.reqs, a.n, item);
    const GenBatchReq& br = a.reqs[q];
    const unsigned etiles = (unsigned)(br.r.tiles_x * br.etiles_y);
    const unsigned local = item - br.eitem_begin;
    const int e = (int)(local / etiles);
    int i, j;
    tile_pixel(br.r.tiles_x, (int)(local % etiles), kEmitTileH, i, j);
    const bool inside = i < br.r.cam.W && j < br.r.cam.H;
    const GenBatchPe& pe = a.pes[br.pe_begin + e];
    emit_ray<false, false>(br.r, pe.b, pe.out, e, i, j, inside, lut2, a.status, nullptr);
}

static void fill_req(GenReq& r, int k, const float* lut, const CamDev& cam, const int dims[3], float scale255,
                     float step, float ref_len, int n_s) {
    r.cam = cam;
    for (int q = 0; q < 3; ++q) r.dims[q] = dims[q];
    r.lut = lut;
    r.scale255 = scale255;
    r.step = step;
    r.ref_len = ref_len;
    r.k = k;
    r.n_s = n_s;
    r.iters = 0;
    r.mode = 0;
    r.gamma = 0.f;
    r.prec = 0;
    r.tiles_x = (cam.W + kTileW - 1) / kTileW;
    r.tiles_y = (cam.H + kCountTileH - 1) / kCountTileH;  // the count kernel's; the emit launch sets its own
    r.own = OwnerDev{nullptr, 0, {0, 0, 0}};
}

static void fill_args(GenArgs& a, const BrickDev* bricks, int k, const float* lut, const CamDev& cam,
                      const int dims[3], float scale255, float step, float ref_len, int n_s, const CompactDev* out,
                      unsigned int* status) {
    for (int e = 0; e < k; ++e) {
        a.b[e] = bricks[e];
        a.out[e] = out[e];
    }
    fill_req(a.r, k, lut, cam, dims, scale255, step, ref_len, n_s);
    a.status = status;
    a.counter = nullptr;
    a.cache = nullptr;
    a.cache_cap = 0;
    a.slots = 0;
    a.ranges = nullptr;
    a.range_tag = nullptr;
    a.tag = 0;
}

// The recorded spans in a generation workspace: after the sample cache, one uint2 per (PE, pixel) and
// the 8-byte tag (nullptr when the workspace has no room for them).
static void gen_span_refs(void* cache, size_t cache_bytes, int k, int w, int h, uint2*& ranges,
                          unsigned long long*& tag) {
    ranges = nullptr;
    tag = nullptr;
    int ctas = 0;
    if (!cache || gen_count_grid(ctas) != VDI_OK) return;
    const size_t cache_sz = align_up(gen_cache_bytes(ctas), 256);
    const size_t span_sz = align_up(gen_span_bytes(k, w, h), 256);
    if (cache_bytes < cache_sz + span_sz + 256) return;
    char* b = static_cast<char*>(cache);
    ranges = reinterpret_cast<uint2*>(b + cache_sz);
    tag = reinterpret_cast<unsigned long long*>(b + cache_sz + span_sz);
}

// Tag of the inputs that decide which samples are non-transparent (bricks, table, camera, sampling): a
// 64-bit FNV-1a hash of their values (pointers, not contents), never 0.
static unsigned long long gen_span_tag(const GenArgs& a) {
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    };
    mix(&a.r.k, sizeof a.r.k);
    mix(&a.r.cam, sizeof a.r.cam);
    mix(a.r.dims, sizeof a.r.dims);
    mix(&a.r.lut, sizeof a.r.lut);
    mix(&a.r.scale255, sizeof a.r.scale255);
    mix(&a.r.step, sizeof a.r.step);
    mix(&a.r.ref_len, sizeof a.r.ref_len);
    mix(a.b, sizeof(BrickDev) * (size_t)a.r.k);
    return h ? h : 1ull;
}

// count-kernel mode of a gamma argument
static int gamma_mode(float gamma) {
    return gamma >= 0.f ? 0 : (gamma == VDI_GAMMA_GIVEN ? 2 : (gamma == kGammaLearnedBracket ? 3 : 1));
}

// persistent grid of gen_count_kernel on the current device
vdi_status gen_count_grid(int& ctas) {
    int dev = 0, sms = 0, per_sm = 0, per_sm_c = 0;
    vdi_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != VDI_OK) return s;
    s = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    if (s != VDI_OK) return s;
    void (*const kernels[6])(GenArgs) = {gen_count_kernel<false, false>, gen_count_kernel<true, false>,
                                         gen_count_kernel<false, true>,  gen_count_kernel<true, true>,
                                         gen_count_kernel<false, false, true>, gen_count_kernel<true, false, true>};
    for (int q = 0; q < 6; ++q) {
        s = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_c, kernels[q], kCountThreads, 0),
                       "occupancy");
        if (s != VDI_OK) return s;
        if (per_sm_c > per_sm) per_sm = per_sm_c;
    }
    s = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_c, gen_count_batched_kernel, kCountThreads,
                                                                 0),
                   "occupancy");
    if (s != VDI_OK) return s;
    if (per_sm_c > per_sm) per_sm = per_sm_c;
    ctas = sms * (per_sm > 0 ? per_sm : 1);
    return VDI_OK;
}

size_t gen_span_bytes(int k, int w, int h) { return (size_t)k * (size_t)w * (size_t)h * sizeof(uint2); }

size_t gen_cache_bytes(int ctas) {
    return (size_t)ctas * kCountThreads * kCacheCap * sizeof(float2);
}

vdi_status launch_gen_count(const BrickDev* bricks, int k, const float* lut, const CamDev& cam, const int dims[3],
                            float scale255, float step, float ref_len, int n_s, float gamma, int iters,
                            const CompactDev* out, unsigned int* status, bool census, unsigned int* counter,
                            void* cache, size_t cache_bytes, cudaStream_t st, const OwnerDev* own) {
    GenArgs a;  // copied into the launch's parameter space
    fill_args(a, bricks, k, lut, cam, dims, scale255, step, ref_len, n_s, out, status);
    if (own) a.r.own = *own;
    a.r.iters = iters;
    a.r.gamma = gamma;
    a.r.mode = gamma_mode(gamma);
    a.counter = counter;
    int ctas = 0;
    vdi_status s = gen_count_grid(ctas);
    if (s != VDI_OK) return s;
    const unsigned items = (unsigned)(a.r.tiles_x * a.r.tiles_y) * (unsigned)k;
    if (items == 0) return VDI_OK;
    if (cache && cache_bytes >= gen_cache_bytes(ctas)) {
        a.slots = ctas * kCountThreads;
        a.cache_cap = kCacheCap;
        a.cache = reinterpret_cast<float2*>(cache);
    }
    if ((unsigned)ctas > items) ctas = (int)items;
    const bool learned = a.r.mode == 3;
    if (a.r.own.map && learned) return set_error(VDI_ERR_UNSUPPORTED, "learned gamma with an ownership map");
    // the spans: every count launch invalidates the recorded ones; box domains record their own
    gen_span_refs(cache, cache_bytes, k, cam.W, cam.H, a.ranges, a.range_tag);
    if (a.range_tag) {
        s = cuda_check(cudaMemsetAsync(a.range_tag, 0, sizeof(unsigned long long), st), "span tag clear");
        if (s != VDI_OK) return s;
        if (a.r.own.map) {
            a.ranges = nullptr;
            a.range_tag = nullptr;
        } else {
            a.tag = gen_span_tag(a);
        }
    }
    if (a.r.own.map && census) gen_count_kernel<true, false, true><<<ctas, kCountThreads, 0, st>>>(a);
    else if (a.r.own.map) gen_count_kernel<false, false, true><<<ctas, kCountThreads, 0, st>>>(a);
    else if (census && learned) gen_count_kernel<true, true><<<ctas, kCountThreads, 0, st>>>(a);
    else if (census) gen_count_kernel<true, false><<<ctas, kCountThreads, 0, st>>>(a);
    else if (learned) gen_count_kernel<false, true><<<ctas, kCountThreads, 0, st>>>(a);
    else gen_count_kernel<false, false><<<ctas, kCountThreads, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "gen_count_kernel launch");
}

vdi_status launch_gen_emit(const BrickDev* bricks, int k, const float* lut, const CamDev& cam, const int dims[3],
                           float scale255, float step, float ref_len, int n_s, int prec, const CompactDev* out,
                           unsigned int* status, cudaStream_t st, bool regular, const OwnerDev* own, void* cache,
                           size_t cache_bytes) {
    GenArgs a;
    fill_args(a, bricks, k, lut, cam, dims, scale255, step, ref_len, n_s, out, status);
    if (own) a.r.own = *own;
    // the spans the last count launch on this workspace recorded, used when they are for these inputs
    if (!a.r.own.map) {
        gen_span_refs(cache, cache_bytes, k, cam.W, cam.H, a.ranges, a.range_tag);
        if (a.range_tag) a.tag = gen_span_tag(a);
    }
    a.r.prec = prec;
    a.r.tiles_y = (cam.H + kEmitTileH - 1) / kEmitTileH;
    dim3 grid((unsigned)(a.r.tiles_x * a.r.tiles_y), (unsigned)k);
    if (grid.x == 0) return VDI_OK;
    if (a.r.own.map) gen_emit_kernel<true, false><<<grid, kEmitThreads, 0, st>>>(a);
    else if (regular) gen_emit_kernel<false, true><<<grid, kEmitThreads, 0, st>>>(a);
    else gen_emit_kernel<false, false><<<grid, kEmitThreads, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "gen_emit_kernel launch");
}

size_t gen_batch_table_bytes(const vdi_gen_request* reqs, int n) {
    size_t pes = 0;
    for (int q = 0; q < n; ++q) pes += (size_t)(reqs[q].k > 0 ? reqs[q].k : 0);
    return align_up(sizeof(GenBatchHeader), 64) + align_up(sizeof(GenBatchReq) * (size_t)n, 64) +
           align_up(sizeof(GenBatchPe) * pes, 64) + sizeof(ScanList) * pes;
}

// The caller has checked every request (vdi_gen_batch_table_pack in api.cu).
vdi_status gen_batch_table_pack(const vdi_gen_request* reqs, int n, const vdi_params* params, void* host_table,
                                size_t bytes) {
    if (bytes < gen_batch_table_bytes(reqs, n))
        return set_error(VDI_ERR_INVALID_ARG, "generation batch table: buffer too small");
    char* base = static_cast<char*>(host_table);
    GenBatchHeader* hd = reinterpret_cast<GenBatchHeader*>(base);
    size_t pes = 0;
    for (int q = 0; q < n; ++q) pes += (size_t)reqs[q].k;
    hd->reqs_off = align_up(sizeof(GenBatchHeader), 64);
    hd->pes_off = hd->reqs_off + align_up(sizeof(GenBatchReq) * (size_t)n, 64);
    hd->lists_off = hd->pes_off + align_up(sizeof(GenBatchPe) * pes, 64);
    GenBatchReq* rd = reinterpret_cast<GenBatchReq*>(base + hd->reqs_off);
    GenBatchPe* pd = reinterpret_cast<GenBatchPe*>(base + hd->pes_off);
    ScanList* ld = reinterpret_cast<ScanList*>(base + hd->lists_off);
    uint64_t items = 0, eitems = 0, chunks = 0;
    uint32_t pe = 0;
    for (int q = 0; q < n; ++q) {
        const vdi_gen_request& g = reqs[q];
        GenBatchReq& r = rd[q];
        const CamDev cam = make_cam(g.cam);
        fill_req(r.r, g.k, g.tf_lut, cam, g.bricks[0].dims, (float)(255.0 * (double)g.bricks[0].value_scale),
                 params->step, params->ref_len, g.n_s);
        r.r.iters = params->bisect_iters;
        r.r.gamma = g.gamma;
        r.r.mode = gamma_mode(g.gamma);
        r.r.prec = g.out[0].prec;
        r.etiles_y = (cam.H + kEmitTileH - 1) / kEmitTileH;
        r.item_begin = (uint32_t)items;
        r.eitem_begin = (uint32_t)eitems;
        r.pe_begin = pe;
        items += (uint64_t)(r.r.tiles_x * r.r.tiles_y) * (uint64_t)g.k;
        eitems += (uint64_t)(r.r.tiles_x * r.etiles_y) * (uint64_t)g.k;
        const int npix = cam.W * cam.H;
        for (int e = 0; e < g.k; ++e, ++pe) {
            pd[pe].b = brick_dev(g.bricks[e]);
            const vdi_compact& o = g.out[e];
            pd[pe].out = CompactDev{o.counts, o.offsets, o.rgba, o.fb, o.gamma, o.capacity};
            ld[pe].counts = o.counts;
            ld[pe].offsets = o.offsets;
            ld[pe].n = npix;
            ld[pe].chunk_begin = (uint32_t)chunks;
            chunks += scan_chunks(npix);
        }
    }
    if (items > 0xFFFFFFFFull || eitems > 0x7FFFFFFFull || chunks > 0x7FFFFFFFull)
        return set_error(VDI_ERR_INVALID_ARG, "generation batch table: too many work items");
    hd->n = (uint32_t)n;
    hd->total_items = (uint32_t)items;
    hd->total_eitems = (uint32_t)eitems;
    hd->total_pes = pe;
    hd->total_chunks = (uint32_t)chunks;
    hd->pad = 0;
    return VDI_OK;
}

// [0, 256) status header, [256, 512) work counter, the prefix sum's partial
// sums, then (optionally) the sample cache
size_t gen_batched_workspace_bytes(const void* host_table) {
    const GenBatchHeader* hd = static_cast<const GenBatchHeader*>(host_table);
    int ctas = 0;
    size_t cache = 0;
    if (gen_count_grid(ctas) == VDI_OK) cache = gen_cache_bytes(ctas);
    return kGenFixed + align_up((size_t)hd->total_chunks * sizeof(uint64_t), 256) + align_up(cache, 256);
}

vdi_status launch_gen_batched(const void* dev_table, const void* host_table, void* workspace, size_t ws_bytes,
                              cudaStream_t st) {
    const GenBatchHeader* hd = static_cast<const GenBatchHeader*>(host_table);
    const size_t fixed = kGenFixed + align_up((size_t)hd->total_chunks * sizeof(uint64_t), 256);
    if (ws_bytes < fixed)
        return set_error(VDI_ERR_WORKSPACE, "vdi_generate_batched: workspace %zu < %zu bytes", ws_bytes, fixed);
    char* ws = static_cast<char*>(workspace);
    vdi_status s = cuda_check(cudaMemsetAsync(ws, 0, kGenFixed, st), "status clear");
    if (s != VDI_OK || hd->n == 0 || hd->total_items == 0) return s;
    const char* t = static_cast<const char*>(dev_table);
    GenBatchArgs a;
    a.reqs = reinterpret_cast<const GenBatchReq*>(t + hd->reqs_off);
    a.pes = reinterpret_cast<const GenBatchPe*>(t + hd->pes_off);
    a.n = (int)hd->n;
    a.total_items = hd->total_items;
    a.status = reinterpret_cast<unsigned int*>(ws);
    a.counter = reinterpret_cast<unsigned int*>(ws + kWsHeader);
    a.cache = nullptr;
    a.cache_cap = 0;
    a.slots = 0;
    int ctas = 0;
    s = gen_count_grid(ctas);
    if (s != VDI_OK) return s;
    if (ws_bytes >= fixed + gen_cache_bytes(ctas)) {
        a.slots = ctas * kCountThreads;
        a.cache_cap = kCacheCap;
        a.cache = reinterpret_cast<float2*>(ws + fixed);
    }
    if ((unsigned)ctas > hd->total_items) ctas = (int)hd->total_items;
    gen_count_batched_kernel<<<ctas, kCountThreads, 0, st>>>(a);
    s = cuda_check(cudaGetLastError(), "gen_count_batched_kernel launch");
    if (s != VDI_OK) return s;
    s = launch_scan_batched(reinterpret_cast<const ScanList*>(t + hd->lists_off), (int)hd->total_pes,
                            hd->total_chunks, reinterpret_cast<uint64_t*>(ws + kGenFixed), st);
    if (s != VDI_OK) return s;
    if (hd->total_eitems == 0) return VDI_OK;
    gen_emit_batched_kernel<<<hd->total_eitems, kEmitThreads, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "gen_emit_batched_kernel launch");
}

}  // namespace vdi
