// Rendering a regular VDI.  From its generating viewpoint: front-to-back
// "over" of each pixel's supersegments, which reproduces the volume rendering
// exactly by associativity of "over" (sec. 2.3).  From another viewpoint: the
// VDI read as a view-dependent volume (below).
#include <cuda_fp16.h>
#include <math.h>

#include "vdi_device.cuh"

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
            const uint2 v = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const uint4*>(rgba) + idx) + 1);
            float tau;
            f16_unpack_col(v, c, tau);
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


// ---------------------------------------------------------------------------
// Rendering from another viewpoint
// ---------------------------------------------------------------------------
// The VDI of camera G read as a view-dependent volume: pixel (i, j)'s frustum
// column (the points whose projection through G's eye falls in the pixel's
// square on G's image plane) holds its supersegments, supersegment (f, b, P,
// A) filling the points at distance f..b from G's eye as a homogeneous
// emission-absorption medium: a path of length l through it has opacity
// 1 - (1 - A)^(l / (b - f)) (the length correction of Eq. 2) and straight
// colour P / A.  One thread per pixel of the viewing camera V walks its ray
// through G's columns (a DDA over G's pixel grid, whose face crossings are
// linear in the ray parameter), cuts each column's part at the closest
// approach to G's eye (where the distance from it stops falling), and
// composites the supersegments it crosses front to back (sec. 2.3).  Lengths
// use u = |s - s*|, the ray's offset from its closest approach s*: the
// distance c from G's eye is reached at u = sqrt((c - rho*)(c + rho*)), with
// s* and rho* in double-float so that shells grazed by the ray keep their
// extent.
struct NovelArgs {
    const uint32_t* counts;
    const void* rgba;
    const float2* fb;
    int n_s, prec, GW, GH;
    float gx[2], gy[2];           // G: tan(fovy / 2) * aspect, tan(fovy / 2), double-float
    float q[3][2];                // V's eye minus G's eye, in G's frame (right, up, forward)
    float vr[3][2], vu[3][2], vf[3][2];  // V's right, up, forward axes in G's frame
    float vx[2], vy[2];           // V: tan(fovy / 2) * aspect, tan(fovy / 2)
    int VW, VH;
    float4* out;
};

__device__ __forceinline__ df dfp(const float v[2]) { return df{v[0], v[1]}; }
__device__ __forceinline__ float df_to_f(df a) { return __fadd_rn(a.hi, a.lo); }

// ray parameter at which the line q + s d meets the plane {x = B z} (or {y = B z}): -(qa - B qz) / (da - B dz)
__device__ __forceinline__ df face_cross(df qa, df qz, df da, df dz, df B, bool& ok) {
    const df den = df_sub(da, df_mul(B, dz));
    ok = den.hi != 0.f;
    if (!ok) return df_f(0.f);
    return df_neg(df_div(df_sub(qa, df_mul(B, qz)), den));
}

// face position of column face (or row face) index k of n: (2 k / n - 1) * t, rows (1 - 2 k / n) * t
__device__ __forceinline__ df face_pos(int k, int n, df t, bool row) {
    const df r = df_div(df_f((float)(2 * k)), df_f((float)n));
    return df_mul(row ? df_sub(df_f(1.f), r) : df_sub(r, df_f(1.f)), t);
}

__device__ __forceinline__ void load_rec(const NovelArgs& a, size_t idx, float& f, float& b) {
    if (a.prec == VDI_PREC_F32) {
        const float2 v = __ldg(a.fb + idx);
        f = v.x;
        b = v.y;
    } else {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const uint4*>(a.rgba) + idx));
        f = __uint_as_float(v.x);
        b = __uint_as_float(v.y);
    }
}

// premultiplied colour and opacity of record idx, and its optical depth tau = -log2(1 - A)
__device__ __forceinline__ float4 load_col(const NovelArgs& a, size_t idx, float& tau) {
    if (a.prec == VDI_PREC_F32) {
        const float4 c = __ldg(reinterpret_cast<const float4*>(a.rgba) + idx);
        tau = -log2f(1.f - c.w);
        return c;
    }
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const uint4*>(a.rgba) + idx) + 1);
    float4 c;
    f16_unpack_col(v, c, tau);
    return c;
}

// offset u >= 0 from the closest approach at which the distance from G's eye is c
__device__ __forceinline__ float shell_offset(float c, df rho) {
    const df dc = df_sub(df_f(c), rho);
    if (dc.hi <= 0.f) return 0.f;
    return __fsqrt_rn(__fmul_rn(__fadd_rn(dc.hi, dc.lo), __fadd_rn(c, rho.hi)));
}

__global__ void __launch_bounds__(128) novel_view_kernel(const __grid_constant__ NovelArgs a) {
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= a.VW * a.VH) return;
    const int i = pix % a.VW, j = pix / a.VW;
    // ray direction in G's frame, in double-float: for a view ray nearly parallel to G's columns the
    // face crossings move by the direction's error divided by the small angle between them
    const df x = df_mul(df_sub(df_div(df_f((float)(2 * i + 1)), df_f((float)a.VW)), df_f(1.f)), dfp(a.vx));
    const df y = df_mul(df_sub(df_f(1.f), df_div(df_f((float)(2 * j + 1)), df_f((float)a.VH))), dfp(a.vy));
    df D[3];
    df n2 = df_f(0.f);
    for (int c = 0; c < 3; ++c) {
        D[c] = df_add(df_add(df_mul(x, dfp(a.vr[c])), df_mul(y, dfp(a.vu[c]))), dfp(a.vf[c]));
        n2 = df_add(n2, df_mul(D[c], D[c]));
    }
    const df nn = df_sqrt(n2);
    float d[3];
    for (int c = 0; c < 3; ++c) {
        D[c] = df_div(D[c], nn);
        d[c] = D[c].hi;
    }
    const df Q[3] = {dfp(a.q[0]), dfp(a.q[1]), dfp(a.q[2])};
    const float qx = a.q[0][0], qy = a.q[1][0], qz = a.q[2][0];
    const df X1 = dfp(a.gx), Y0 = dfp(a.gy);
    // the part of the ray inside G's frustum: four half-spaces through G's eye, A + s B >= 0
    const df Ac[4] = {df_add(Q[0], df_mul(X1, Q[2])), df_sub(df_mul(X1, Q[2]), Q[0]),
                      df_sub(df_mul(Y0, Q[2]), Q[1]), df_add(Q[1], df_mul(Y0, Q[2]))};
    const df Bc[4] = {df_add(D[0], df_mul(X1, D[2])), df_sub(df_mul(X1, D[2]), D[0]),
                      df_sub(df_mul(Y0, D[2]), D[1]), df_add(D[1], df_mul(Y0, D[2]))};
    float s_in = 0.f, s_out = INFINITY;
    bool hit = true;
    for (int c = 0; c < 4; ++c) {
        if (Bc[c].hi == 0.f) {
            if (Ac[c].hi < 0.f) hit = false;
            continue;
        }
        const float s = df_to_f(df_neg(df_div(Ac[c], Bc[c])));
        if (Bc[c].hi > 0.f) s_in = fmaxf(s_in, s);
        else s_out = fminf(s_out, s);
    }
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
    if (hit && s_out > s_in) {
        // closest approach to G's eye
        df sdot = df_f(0.f);
        for (int c = 0; c < 3; ++c) sdot = df_add(sdot, df_mul(Q[c], D[c]));
        const df s_star = df_neg(sdot);
        df rho2 = df_f(0.f);
        for (int c = 0; c < 3; ++c) {
            const df pc = df_add(Q[c], df_mul(s_star, D[c]));
            rho2 = df_add(rho2, df_mul(pc, pc));
        }
        const df rho = df_sqrt(rho2);
        const float ss = s_star.hi;
        // DDA over G's columns; du, dv: signs of dX/ds, dY/ds (v grows downwards)
        const df du = df_sub(df_mul(D[0], Q[2]), df_mul(Q[0], D[2]));
        const df dv = df_sub(df_mul(D[1], Q[2]), df_mul(Q[1], D[2]));
        const int stepu = du.hi > 0.f ? 1 : -1, stepv = dv.hi > 0.f ? -1 : 1;
        float s = s_in;
        int iu, iv;
        {
            const float sm = isinf(s_out) ? s_in + 1.f : 0.5f * (s_in + s_out);
            const float zm = fmaf(sm, d[2], qz);
            const float Xm = fmaf(sm, d[0], qx) / zm, Ym = fmaf(sm, d[1], qy) / zm;
            // column of the entry point (on the frustum face or inside)
            const float z0 = fmaf(s_in, d[2], qz);
            const float X0 = z0 > 0.f ? fmaf(s_in, d[0], qx) / z0 : Xm, Y0p = z0 > 0.f ? fmaf(s_in, d[1], qy) / z0 : Ym;
            iu = min(max((int)floorf((X0 / X1.hi + 1.f) * 0.5f * a.GW), 0), a.GW - 1);
            iv = min(max((int)floorf((1.f - Y0p / Y0.hi) * 0.5f * a.GH), 0), a.GH - 1);
        }
        const int max_steps = a.GW + a.GH + 4;
        for (int it = 0; it < max_steps && s < s_out; ++it) {
            // next column face in u and v (none along an axis the ray does not move in: a ray from G's
            // eye lies in no face it meets there)
            float sx = INFINITY, sy = INFINITY;
            const int bu = stepu > 0 ? iu + 1 : iu, bv = stepv > 0 ? iv + 1 : iv;
            if (du.hi != 0.f && bu > 0 && bu < a.GW) {
                bool ok;
                const df c = face_cross(Q[0], Q[2], D[0], D[2], face_pos(bu, a.GW, X1, false), ok);
                if (ok) {
                    sx = df_to_f(c);
                    if (!(fmaf(sx, d[2], qz) > 0.f)) sx = INFINITY;  // the face's plane met behind G's eye
                }
            }
            if (dv.hi != 0.f && bv > 0 && bv < a.GH) {
                bool ok;
                const df c = face_cross(Q[1], Q[2], D[1], D[2], face_pos(bv, a.GH, Y0, true), ok);
                if (ok) {
                    sy = df_to_f(c);
                    if (!(fmaf(sy, d[2], qz) > 0.f)) sy = INFINITY;
                }
            }
            // the next event decides the step before the segment end is clamped to s (a face
            // crossing rounded to just behind s is still crossed)
            float sn = fminf(fminf(sx, sy), s_out);
            bool cross_u = sx < s_out && sx <= sy, cross_v = sy < s_out && sy <= sx;
            if (ss > s && ss < sn) {
                sn = ss;
                cross_u = cross_v = false;
            }
            const bool exits = !cross_u && !cross_v && sn >= s_out;
            sn = fmaxf(sn, s);
            // the piece [s, sn] of column (iu, iv)
            const size_t p = (size_t)iv * a.GW + iu;
            const int n = (int)min(__ldg(a.counts + p), (uint32_t)a.n_s);
            if (n > 0 && sn > s) {
                const bool rising = s >= ss;
                const float ua = fabsf(df_sub(df_f(s), s_star).hi), ub = isinf(sn) ? INFINITY : fabsf(df_sub(df_f(sn), s_star).hi);
                const float ulo = fminf(ua, ub), uhi = fmaxf(ua, ub);
                // The column's records are sorted and disjoint in depth, and shell_offset is
                // non-decreasing in depth, so the records this piece overlaps are one run: rising, from
                // the first whose back lies beyond ulo to the first whose front reaches uhi; falling
                // (records in reverse), from the last whose front lies below uhi down to the first whose
                // back reaches down to ulo.  The run's start is found by bisection; the records skipped
                // have no overlap (l <= 0), so the sum is that of the full loop.
                int k0;
                {
                    int lo_k = 0, hi_k = n;
                    while (lo_k < hi_k) {
                        const int mid = (lo_k + hi_k) >> 1;
                        float f, b;
                        load_rec(a, p * a.n_s + mid, f, b);
                        const bool before = rising ? !(shell_offset(b, rho) > ulo) : shell_offset(f, rho) < uhi;
                        if (before) lo_k = mid + 1;
                        else hi_k = mid;
                    }
                    k0 = rising ? lo_k : lo_k - 1;
                }
                for (int k = k0; rising ? k < n : k >= 0; k += rising ? 1 : -1) {
                    const size_t idx = p * a.n_s + k;
                    float f, b;
                    load_rec(a, idx, f, b);
                    if (!(b > f)) continue;
                    const float so_f = shell_offset(f, rho), so_b = shell_offset(b, rho);
                    if (rising ? so_f >= uhi : so_b <= ulo) break;
                    const float lo = fmaxf(so_f, ulo);
                    const float hi = fminf(so_b, uhi);
                    const float l = hi - lo;
                    if (!(l > 0.f)) continue;
                    float tau;
                    const float4 c = load_col(a, idx, tau);
                    if (c.w <= 0.f) continue;
                    float alpha;
                    if (!(tau < INFINITY)) alpha = 1.f;
                    else alpha = 1.f - exp2f(-tau * (l / (b - f)));
                    const float w = T * alpha / c.w;
                    C0 = fmaf(w, c.x, C0);
                    C1 = fmaf(w, c.y, C1);
                    C2 = fmaf(w, c.z, C2);
                    T *= 1.f - alpha;
                }
            }
            if (exits) break;
            if (cross_u) iu += stepu;
            if (cross_v) iv += stepv;
            if (iu < 0 || iu >= a.GW || iv < 0 || iv >= a.GH) break;
            s = sn;
        }
    }
    a.out[pix] = make_float4(C0, C1, C2, 1.f - T);
}

vdi_status launch_novel_view(const vdi_regular* v, const vdi_camera& gen, const vdi_camera& view, float* rgba,
                             cudaStream_t st) {
    auto frame = [](const vdi_camera& c, double fwd[3], double right[3], double up[3]) {
        for (int k = 0; k < 3; ++k) fwd[k] = c.center[k] - c.eye[k];
        double n = sqrt(fwd[0] * fwd[0] + fwd[1] * fwd[1] + fwd[2] * fwd[2]);
        for (int k = 0; k < 3; ++k) fwd[k] /= n;
        right[0] = fwd[1] * c.up[2] - fwd[2] * c.up[1];
        right[1] = fwd[2] * c.up[0] - fwd[0] * c.up[2];
        right[2] = fwd[0] * c.up[1] - fwd[1] * c.up[0];
        n = sqrt(right[0] * right[0] + right[1] * right[1] + right[2] * right[2]);
        for (int k = 0; k < 3; ++k) right[k] /= n;
        up[0] = right[1] * fwd[2] - right[2] * fwd[1];
        up[1] = right[2] * fwd[0] - right[0] * fwd[2];
        up[2] = right[0] * fwd[1] - right[1] * fwd[0];
    };
    double gf[3], gr[3], gu[3], vf[3], vr[3], vu[3];
    frame(gen, gf, gr, gu);
    frame(view, vf, vr, vu);
    auto dot = [](const double* x, const double* y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
    NovelArgs a;
    a.counts = v->counts;
    a.rgba = v->rgba;
    a.fb = reinterpret_cast<const float2*>(v->fb);
    a.n_s = v->n_s;
    a.prec = v->prec;
    a.GW = gen.width;
    a.GH = gen.height;
    auto split = [](double x, float out[2]) {
        out[0] = (float)x;
        out[1] = (float)(x - (double)out[0]);
    };
    const double gth = tan(0.5 * gen.fovy_deg * 3.14159265358979323846 / 180.0);
    split(gth * (double)gen.width / (double)gen.height, a.gx);
    split(gth, a.gy);
    double q[3] = {view.eye[0] - gen.eye[0], view.eye[1] - gen.eye[1], view.eye[2] - gen.eye[2]};
    const double qg[3] = {dot(q, gr), dot(q, gu), dot(q, gf)};
    for (int k = 0; k < 3; ++k) split(qg[k], a.q[k]);
    const double* vb[3] = {vr, vu, vf};
    float (*dst[3])[2] = {a.vr, a.vu, a.vf};
    for (int m = 0; m < 3; ++m) {
        split(dot(vb[m], gr), dst[m][0]);
        split(dot(vb[m], gu), dst[m][1]);
        split(dot(vb[m], gf), dst[m][2]);
    }
    const double vth = tan(0.5 * view.fovy_deg * 3.14159265358979323846 / 180.0);
    split(vth * (double)view.width / (double)view.height, a.vx);
    split(vth, a.vy);
    a.VW = view.width;
    a.VH = view.height;
    a.out = reinterpret_cast<float4*>(rgba);
    const int npix = view.width * view.height;
    if (npix == 0) return VDI_OK;
    novel_view_kernel<<<(npix + 127) / 128, 128, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "novel_view_kernel launch");
}

}  // namespace vdi
