// Device-side building blocks shared by the generation and compositing kernels.
//
// The supersegment state machine (Eq. 1 with the renormalised opacity of
// Algorithm S1) and the sampling arithmetic are written with explicitly
// rounded intrinsics (__fmaf_rn, __fmul_rn, ...) so that every kernel that
// re-runs them -- the gamma search and the later emission pass -- takes the
// same decision on the same sample, whatever the compiler's contraction
// choices in the surrounding code.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "vdi_internal.h"

namespace vdi {

// ---------------------------------------------------------------------------
// SFU approximations (hardware instructions; relative error ~2^-22)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// FP16 record codec.  A 16-byte record is {float f, float b, binary16 R, G, B,
// binary16 tau}: premultiplied colour and the opacity A stored as its base-2
// optical depth tau = -log2(1 - A) (+inf for A = 1).  Rounding A itself to
// binary16 would put every A above 1 - 2^-12 at exactly 1 (an opaque record)
// and move the extinction -log2(1 - A) / l of the compositing mixture, whose
// sensitivity to A is 1 / (1 - A), by up to the whole value; tau keeps a
// relative precision of 2^-11 at every opacity, and A = 1 - 2^-tau then moves
// by at most ln2 tau 2^-tau 2^-11 <= 1.8e-4.
// ---------------------------------------------------------------------------
// A = 1 - 2^-tau, written as -expm1(-tau ln 2) so that small opacities keep
// their relative precision (colour is P / A)
__device__ __forceinline__ float f16_opacity(float tau) {
    return -expm1f(__fmul_rn(-tau, 0.693147180559945309f));
}

// record -> 16 bytes; L2 = log2(1 - A) of the record (tau = -L2, written as
// 0 - L2 so that L2 = 0 stores +0)
__device__ __forceinline__ uint4 f16_pack(float f, float b, float R, float G, float B, float L2) {
    const __half2 rg = __floats2half2_rn(R, G);
    const __half2 bt = __floats2half2_rn(B, __fsub_rn(0.f, L2));
    uint4 v;
    v.x = __float_as_uint(f);
    v.y = __float_as_uint(b);
    v.z = *reinterpret_cast<const unsigned int*>(&rg);
    v.w = *reinterpret_cast<const unsigned int*>(&bt);
    return v;
}

// colour half of a record (its last 8 bytes) -> premultiplied colour, opacity, tau
__device__ __forceinline__ void f16_unpack_col(uint2 v, float4& c, float& tau) {
    const float2 rg = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    const float2 bt = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    tau = bt.y;
    c = make_float4(rg.x, rg.y, bt.x, f16_opacity(tau));
}

// floor of x (|x| < 2^22) without the conversion pipe: (x - 1/2) rounded to the
// nearest integer by adding 1.5 * 2^23.  Returns the integer and its float.
// At exact integers the tie may resolve to x - 1 (then the weight x - floor is 1),
// which gives the same interpolated value.
__device__ __forceinline__ int floor_magic(float x, float& fl) {
    const float M = 12582912.0f;  // 1.5 * 2^23
    float m = __fadd_rn(__fadd_rn(x, -0.5f), M);
    fl = __fadd_rn(m, -M);
    return __float_as_int(m) - 0x4B400000;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (unevaluated sums hi + lo of two floats) from the
// error-free transformations TwoSum (Knuth) and TwoProduct via FMA (Dekker's
// double-length arithmetic).  Used once per ray, so that sample positions are
// exact to ~1e-12 voxel without FP64 instructions.
// ---------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {  // requires |a| >= |b|
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    s = quick_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return quick_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_div(df a, df b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    df r = df_sub(a, df_mul(df{q1, 0.f}, b));
    float q2 = __fdiv_rn(r.hi, b.hi);
    r = df_sub(r, df_mul(df{q2, 0.f}, b));
    float q3 = __fdiv_rn(r.hi, b.hi);
    return df_add(quick_two_sum(q1, q2), df{q3, 0.f});
}
__device__ __forceinline__ df df_sqrt(df a) {
    if (a.hi <= 0.f) return {0.f, 0.f};
    float s = __fsqrt_rn(a.hi);
    df r = df_sub(a, df_mul(df{s, 0.f}, df{s, 0.f}));
    return quick_two_sum(s, __fdiv_rn(r.hi, __fmul_rn(2.f, s)));
}
__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ df df_f(float x) { return {x, 0.f}; }

// Fixed-point sample positions: 64-bit signed, 44 fractional bits (20.44).
// Integer addition is exact and associative, so P0 + k D is the same whether
// it is stepped sample by sample or computed directly, in every kernel.
constexpr int kFrac = 44;
__device__ __forceinline__ long long df_to_fixed(df v) {
    const float S = 17592186044416.0f;  // 2^44, exact scaling
    return __float2ll_rn(__fmul_rn(v.hi, S)) + __float2ll_rn(__fmul_rn(v.lo, S));
}
__device__ __forceinline__ int fixed_cell(long long P) { return (int)(P >> kFrac); }
// top 23 fractional bits as a float in [0, 1)
__device__ __forceinline__ float fixed_frac(long long P) {
    unsigned lo = (unsigned)P, hi = (unsigned)(P >> 32);
    unsigned m = __funnelshift_r(lo, hi, kFrac - 23) & 0x7FFFFFu;
    return __fsub_rn(__uint_as_float(m | 0x3F800000u), 1.f);
}

// ---------------------------------------------------------------------------
// Rays (pinhole camera, one ray per pixel through its centre)
// ---------------------------------------------------------------------------
struct Ray {
    long long P0[3], D[3];  // fixed point: midpoint of sample 0, step vector
    float tin_hi, tin_lo;   // entry depth (double-float)
    float o[3], d[3];       // float eye and direction, for range estimates only
    int n;                  // samples on the global grid
};

// Slab test against [0, dims-1]^3 in double-float; returns false on a miss.
__device__ __forceinline__ bool ray_setup(const CamDev& c, int i, int j, const int dims[3], float step, Ray& r) {
    df x = df_mul(df_sub(df_div(df_f((float)(2 * i + 1)), df_f((float)c.W)), df_f(1.f)), df{c.sx[0], c.sx[1]});
    df y = df_mul(df_sub(df_f(1.f), df_div(df_f((float)(2 * j + 1)), df_f((float)c.H))), df{c.sy[0], c.sy[1]});
    df v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        v[a] = df_add(df_add(df{c.fwd[a][0], c.fwd[a][1]}, df_mul(x, df{c.right[a][0], c.right[a][1]})),
                      df_mul(y, df{c.up[a][0], c.up[a][1]}));
    df nn = df_sqrt(df_add(df_add(df_mul(v[0], v[0]), df_mul(v[1], v[1])), df_mul(v[2], v[2])));
    df d[3], o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d[a] = df_div(v[a], nn);
        o[a] = df{c.eye[a][0], c.eye[a][1]};
        r.o[a] = o[a].hi;
        r.d[a] = d[a].hi;
    }
    df tin = df_f(0.f), tout = df_f(3.0e38f);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        df hi = df_f((float)(dims[a] - 1));
        if (d[a].hi == 0.f) {
            if (df_lt(o[a], df_f(0.f)) || df_lt(hi, o[a])) { r.n = 0; return false; }
            continue;
        }
        df t0 = df_div(df_neg(o[a]), d[a]);
        df t1 = df_div(df_sub(hi, o[a]), d[a]);
        if (df_lt(t1, t0)) { df t = t0; t0 = t1; t1 = t; }
        if (df_lt(tin, t0)) tin = t0;
        if (df_lt(t1, tout)) tout = t1;
    }
    r.tin_hi = tin.hi;
    r.tin_lo = tin.lo;
    if (!df_lt(tin, tout)) { r.n = 0; return false; }
    // number of k with midpoint tin + (k + 1/2) step < tout
    df len = df_sub(tout, tin);
    int n = (int)ceilf(__fsub_rn(__fdiv_rn(len.hi, step), 0.5f));
    if (n < 0) n = 0;
    auto mid = [&](int k) { return df_add(tin, df_mul(df_f((float)k + 0.5f), df_f(step))); };
    while (n > 0 && !df_lt(mid(n - 1), tout)) --n;
    while (df_lt(mid(n), tout)) ++n;
    r.n = n;
    if (n <= 0) return false;
    df t0 = mid(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r.P0[a] = df_to_fixed(df_add(o[a], df_mul(t0, d[a])));
        r.D[a] = df_to_fixed(df_mul(df_f(step), d[a]));
    }
    return true;
}

// depth of the front of sample k: t_in + k step (to FP32)
__device__ __forceinline__ float sample_front(const Ray& r, float step, int k) {
    return __fadd_rn(__fmaf_rn((float)k, step, r.tin_hi), r.tin_lo);
}

// global cell (clamped to the volume's cells) of sample k's midpoint
__device__ __forceinline__ void sample_cell(const Ray& r, int k, const int dims[3], int c[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int ci = fixed_cell(r.P0[a] + (long long)k * r.D[a]);
        c[a] = ci < 0 ? 0 : (ci > dims[a] - 2 ? dims[a] - 2 : ci);
    }
}

__device__ __forceinline__ bool owns(const BrickDev& b, const int c[3]) {
    return c[0] >= b.lo[0] && c[0] < b.hi[0] && c[1] >= b.lo[1] && c[1] < b.hi[1] && c[2] >= b.lo[2] &&
           c[2] < b.hi[2];
}

// Owned sample range [k0, k1) of brick b on ray r (boxes are convex and cell
// coordinates are monotone along the ray, so the owned samples are one run).
__device__ __forceinline__ bool owned_range(const Ray& r, float step, const BrickDev& b, const int dims[3], int& k0,
                                            int& k1) {
    // estimate with a float slab test against the brick's cells widened by a cell
    float tlo = r.tin_hi, thi = 3.0e38f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float lo = (float)b.lo[a] - 1.0f, hi = (float)b.hi[a] + 1.0f;
        if (r.d[a] == 0.f) {
            if (r.o[a] < lo || r.o[a] > hi) return false;
            continue;
        }
        float t0 = (lo - r.o[a]) / r.d[a], t1 = (hi - r.o[a]) / r.d[a];
        if (t0 > t1) { float t = t0; t0 = t1; t1 = t; }
        tlo = fmaxf(tlo, t0);
        thi = fminf(thi, t1);
    }
    if (!(thi >= tlo)) return false;
    float ka = floorf((tlo - r.tin_hi) / step) - 1.f, kb = ceilf((thi - r.tin_hi) / step) + 1.f;
    int a0 = (int)fmaxf(ka, 0.f);
    int a1 = (int)fminf(kb, (float)r.n);
    // first owned sample, then the end of the run by bisection
    int c[3];
    int k = a0;
    for (; k < a1; ++k) {
        sample_cell(r, k, dims, c);
        if (owns(b, c)) break;
    }
    if (k >= a1) return false;
    k0 = k;
    int lo = k0 + 1, hi = a1;  // samples < lo owned; samples >= hi not owned
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        sample_cell(r, mid, dims, c);
        if (owns(b, c)) lo = mid + 1;
        else hi = mid;
    }
    k1 = lo;
    return true;
}

// ---------------------------------------------------------------------------
// Sampling one brick: trilinear from cell-packed corners, classification
// ---------------------------------------------------------------------------
struct Sample {
    float P[3];  // premultiplied colour
    float a;     // opacity over the step
    float lgT;   // log2(1 - a)
    float x;     // table coordinate v * 255 (clamped): the sample's classification is a function of x alone
};

// Corner values of the cell holding the fixed-point position P (two float4
// loads).  The index is clamped to the brick, so the load is always in bounds.
__device__ __forceinline__ void cell_load(const long long P[3], const BrickDev& b, float4& lo, float4& hi) {
    int lx = fixed_cell(P[0]) - b.lo[0] + 1, ly = fixed_cell(P[1]) - b.lo[1] + 1, lz = fixed_cell(P[2]) - b.lo[2] + 1;
    int idx = (lz * b.ny + ly) * b.nx + lx;
    idx = min(max(idx, 0), b.ncells - 1);
    const float4* cp = reinterpret_cast<const float4*>(b.cells) + 2 * (size_t)idx;
    lo = __ldg(cp);
    hi = __ldg(cp + 1);
}

// Classification of table coordinate x in [0, 255]: the step-corrected table
// (257 entries, then their 257 differences to the next entry; two halves so
// that a warp's 16-byte reads of different entries spread over all banks)
// interpolated at x, premultiplied
// colour, log-transmittance.  A function of x alone, so a cached x gives the
// sample's colour and opacity bit for bit.
__device__ __forceinline__ void classify_x(float x, const float4* __restrict__ lut2, Sample& s) {
    s.x = x;
    float fl;
    int i = floor_magic(x, fl);
    float wt = __fsub_rn(x, fl);
    float4 base = lut2[i], dl = lut2[257 + i];
    float R = __fmaf_rn(wt, dl.x, base.x);
    float G = __fmaf_rn(wt, dl.y, base.y);
    float B = __fmaf_rn(wt, dl.z, base.z);
    float A = __fmaf_rn(wt, dl.w, base.w);
    s.a = A;
    s.P[0] = __fmul_rn(R, A);
    s.P[1] = __fmul_rn(G, A);
    s.P[2] = __fmul_rn(B, A);
    s.lgT = lg2_approx(__fsub_rn(1.f, A));
}

// Sample at fixed-point midpoint P from its cell's corners (lo = v000 v100 v010
// v110, hi = v001 v101 v011 v111): trilinear value, then classification.
__device__ __forceinline__ void sample_from(float w0, float w1, float w2, const float4& lo, const float4& hi,
                                            const float4* __restrict__ lut2, float scale255, Sample& s) {
    float c00 = __fmaf_rn(w0, __fsub_rn(lo.y, lo.x), lo.x);
    float c10 = __fmaf_rn(w0, __fsub_rn(lo.w, lo.z), lo.z);
    float c01 = __fmaf_rn(w0, __fsub_rn(hi.y, hi.x), hi.x);
    float c11 = __fmaf_rn(w0, __fsub_rn(hi.w, hi.z), hi.z);
    float c0 = __fmaf_rn(w1, __fsub_rn(c10, c00), c00);
    float c1 = __fmaf_rn(w1, __fsub_rn(c11, c01), c01);
    float v = __fmaf_rn(w2, __fsub_rn(c1, c0), c0);
    classify_x(fminf(fmaxf(__fmul_rn(v, scale255), 0.f), 255.f), lut2, s);
}

// March over samples [k0, k1) of ray r in brick b, calling f(k, sample) in
// order.  The next sample's cell is loaded while the current one is
// processed, so the load latency overlaps the state-machine work.
template <typename F>
__device__ __forceinline__ void march(const Ray& r, int k0, int k1, const BrickDev& b, const float4* __restrict__ lut2,
                                      float scale255, F&& f) {
    long long P[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) P[a] = r.P0[a] + (long long)k0 * r.D[a];
    float4 clo, chi;
    cell_load(P, b, clo, chi);
    for (int k = k0; k < k1; ++k) {
        const float w0 = fixed_frac(P[0]), w1 = fixed_frac(P[1]), w2 = fixed_frac(P[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) P[a] += r.D[a];
        float4 nlo, nhi;
        cell_load(P, b, nlo, nhi);  // next sample's cell, in flight during this sample's work
        Sample s;
        sample_from(w0, w1, w2, clo, chi, lut2, scale255, s);
        f(k, s);
        clo = nlo;
        chi = nhi;
    }
}

// ---------------------------------------------------------------------------
// Supersegment state machine (Eq. 1, Algorithm S1)
// ---------------------------------------------------------------------------
// Decision for an open supersegment S (premultiplied P, opacity A, optical
// depth L2 = log2(1 - A) summed over its pieces, extent length lS) and an
// incoming piece x (P_x, a_x, length lx): with a~ = 1 - 2^(L2 lx / lS),
//   terminate  <=>  || P a~ - A P_x ||^2 >= gamma^2 A^2
// which is Eq. 1's || (P/A) a~ - P_x || >= gamma multiplied through by A > 0.
__device__ __forceinline__ bool criterion(const float P[3], float A, float L2, float r, const float Px[3],
                                          float g2) {
    float at = __fsub_rn(1.f, ex2_approx(__fmul_rn(L2, r)));
    float e0 = __fmaf_rn(P[0], at, -__fmul_rn(A, Px[0]));
    float e1 = __fmaf_rn(P[1], at, -__fmul_rn(A, Px[1]));
    float e2 = __fmaf_rn(P[2], at, -__fmul_rn(A, Px[2]));
    float D = __fmaf_rn(e2, e2, __fmaf_rn(e1, e1, __fmul_rn(e0, e0)));
    return D >= __fmul_rn(g2, __fmul_rn(A, A));
}

// The same decision for a transparent piece (Px = 0): each channel's term
// fma(P, at, -(A * 0)) is the rounded product P * at (adding -0 changes no
// rounded result), so this is criterion(P, A, L2, r, {0, 0, 0}, g2) bit for
// bit with three multiplications fewer.
__device__ __forceinline__ bool criterion_clear(const float P[3], float A, float L2, float r, float g2) {
    float at = __fsub_rn(1.f, ex2_approx(__fmul_rn(L2, r)));
    float e0 = __fmul_rn(P[0], at);
    float e1 = __fmul_rn(P[1], at);
    float e2 = __fmul_rn(P[2], at);
    float D = __fmaf_rn(e2, e2, __fmaf_rn(e1, e1, __fmul_rn(e0, e0)));
    return D >= __fmul_rn(g2, __fmul_rn(A, A));
}

// The same decision, also returning the decision ratio q ~= D / A^2 (one
// approximate reciprocal): every gamma with gamma^2 on the same side of q
// takes the same decision at this step.
__device__ __forceinline__ bool criterion_q(const float P[3], float A, float L2, float r, const float Px[3], float g2,
                                            float& q) {
    float at = __fsub_rn(1.f, ex2_approx(__fmul_rn(L2, r)));
    float e0 = __fmaf_rn(P[0], at, -__fmul_rn(A, Px[0]));
    float e1 = __fmaf_rn(P[1], at, -__fmul_rn(A, Px[1]));
    float e2 = __fmaf_rn(P[2], at, -__fmul_rn(A, Px[2]));
    float D = __fmaf_rn(e2, e2, __fmaf_rn(e1, e1, __fmul_rn(e0, e0)));
    float AA = __fmul_rn(A, A);
    q = __fmul_rn(D, rcp_approx(AA));
    return D >= __fmul_rn(g2, AA);
}

// absorb piece x into S ("over")
__device__ __forceinline__ void absorb(float P[3], float& A, float& L2, const float Px[3], float ax, float lgTx) {
    float T = __fsub_rn(1.f, A);
    P[0] = __fmaf_rn(T, Px[0], P[0]);
    P[1] = __fmaf_rn(T, Px[1], P[1]);
    P[2] = __fmaf_rn(T, Px[2], P[2]);
    A = __fmaf_rn(T, ax, A);
    L2 = __fadd_rn(L2, lgTx);
}

// Known counts: exact candidates and their decision intervals.
#ifndef VDI_TABLE_N
#define VDI_TABLE_N 27
#endif
struct CountTable {
    static constexpr int N = VDI_TABLE_N;  // 27: 9 marches of 3 candidates cover 16 levels
    float g2[N], lo[N], hi[N];  // lo, hi: the interval narrowed by the margin below
    int c[N];
    int n;
    // The interval is narrowed by a relative margin of 2^-16, far above the ratio's approximation
    // error; the narrowed bounds are kept.
    __device__ __forceinline__ void add(float g2v, float qlo, float qhi, int cnt) {
        if (n >= N) n = 0;  // full (more than 16 levels): start over, dropping the oldest
        {
            g2[n] = g2v;
            lo[n] = qlo * (1.f + 1.0f / 65536.f);
            hi[n] = qhi * (1.f - 1.0f / 65536.f);
            c[n] = cnt;
            ++n;
        }
    }
    // count at gamma^2 = x if known, else -1
    __device__ __forceinline__ int lookup(float x) const {
        for (int i = 0; i < n; ++i) {
            if (x == g2[i]) return c[i];
            if (x > lo[i] && x <= hi[i]) return c[i];
        }
        return -1;
    }
};

}  // namespace vdi
