/*
 * CPU oracle for distributed Volumetric Depth Image (VDI) generation and
 * compositing (Gupta et al., "Parallel Compositing of Volumetric Depth Images
 * for Interactive Visualization of Distributed Volumes at High Frame Rates").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, FP64 statement of
 * what the GPU library computes.  Only the tests, the package's smoke check
 * and the benchmark's CPU-baseline leg may load it; the library never does.
 * It shares no code, header or table with the CUDA sources.
 *
 * Everything is double precision and follows the paper's steps in its order:
 *   - rays and samples: sec. 2.4 (one list per pixel, N_L = w h), sec. 5.1
 *     (all PEs share the camera; each PE raycasts its own sub-volume);
 *   - classification with length-adjusted opacity: sec. 2.4 (after Eq. 1);
 *   - supersegment termination criterion tau: Eq. 1;
 *   - iterative bisection search for gamma: sec. 2.4 and sec. 5.2;
 *   - compact layout (counts + exclusive prefix sum): sec. 4, Fig. 2;
 *   - compositing of sub-supersegments: sec. 5.2, Eq. 2 and Algorithm S1
 *     (K-way depth ordering, gaps as transparent samples, re-segmentation);
 *   - non-convex ownership: sec. 5.3 (a sub-supersegment ends where the ray
 *     leaves the PE's domain);
 *   - flattening by front-to-back "over" and ground-truth DVR: sec. 2.3.
 * Where the paper is silent or its pseudocode is inconsistent, the readings
 * are marked below where they are used (G1..G19: the opacity compared in
 * Eq. 1, the tie rule, premultiplied colour, the units of Eq. 2, the control
 * flow of Algorithm S1, gaps, overlapping PEs, the search constants, what is
 * counted, the budget, sampling, ownership, depth, camera, early termination,
 * the regular layout, FP16 storage, synthetic lists and the learned features).
 *
 * Parity status: every function here is pinned by tests in tests/ against
 * closed forms, brute force or invariants, except the places marked
 * "parity unpinned" (none at present in this file).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double eye[3], center[3], up[3];
    double fovy_deg;
    int width, height;
} oc_camera;

typedef struct {
    const void* data; /* node values, x fastest, then y, then z */
    int dtype;        /* 0: float32 in [0,1]; 1: uint16, value = u / 65535 */
    int dims[3];      /* nodes per axis; the volume spans [0, dims-1] per axis */
} oc_volume;

typedef struct {
    int lo[3], hi[3]; /* owned cells [lo, hi) per axis; cell c spans [c, c+1] */
} oc_box;

typedef struct {
    double f, b;  /* front and back depth along the ray */
    double P[3];  /* premultiplied colour */
    double a;     /* opacity over [f, b] */
    int brk;      /* 1: marker "the ray left this PE's domain here" */
} oc_piece;

/* output / input record: f, b, R, G, B, A (premultiplied RGB) */
#define REC 6

/* ---------------------------------------------------------------------- */
/* Vector helpers                                                          */
/* ---------------------------------------------------------------------- */
static void v_sub(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static void v_cross(const double* a, const double* b, double* o) {
    double t[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    o[0] = t[0]; o[1] = t[1]; o[2] = t[2];
}
static void v_norm(double* a) {
    double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    a[0] /= n; a[1] /= n; a[2] /= n;
}

/* ---------------------------------------------------------------------- */
/* Rays (sec. 2.4: one ray per pixel; sec. 5.1: shared camera)             */
/* Pixel (i, j), j = 0 at the top row, through the pixel centre.           */
/* ---------------------------------------------------------------------- */
void oc_ray(const oc_camera* c, int i, int j, double* o, double* d) {
    double fwd[3], right[3], up2[3];
    v_sub(c->center, c->eye, fwd);
    v_norm(fwd);
    v_cross(fwd, c->up, right);
    v_norm(right);
    v_cross(right, fwd, up2);
    double th = tan(0.5 * c->fovy_deg * 3.14159265358979323846 / 180.0);
    double x = (2.0 * (i + 0.5) / c->width - 1.0) * th * (double)c->width / (double)c->height;
    double y = (1.0 - 2.0 * (j + 0.5) / c->height) * th;
    for (int a = 0; a < 3; ++a) d[a] = x * right[a] + y * up2[a] + fwd[a];
    v_norm(d);
    o[0] = c->eye[0]; o[1] = c->eye[1]; o[2] = c->eye[2];
}

/* Slab test against [0, dims-1]^3.  Returns 1 and [t_in, t_out] on a hit. */
int oc_hit_box(const double* o, const double* d, const int* dims, double* t_in, double* t_out) {
    double tin = 0.0, tout = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double hi = (double)(dims[a] - 1);
        if (d[a] == 0.0) {
            if (o[a] < 0.0 || o[a] > hi) return 0;
            continue;
        }
        double t0 = (0.0 - o[a]) / d[a], t1 = (hi - o[a]) / d[a];
        if (t0 > t1) { double t = t0; t0 = t1; t1 = t; }
        if (t0 > tin) tin = t0;
        if (t1 < tout) tout = t1;
    }
    *t_in = tin;
    *t_out = tout;
    return tout > tin;
}

/* ---------------------------------------------------------------------- */
/* Volume sampling: node-centred trilinear interpolation (reading G12)     */
/* ---------------------------------------------------------------------- */
static double node(const oc_volume* v, int x, int y, int z) {
    size_t idx = ((size_t)z * v->dims[1] + y) * v->dims[0] + x;
    if (v->dtype == 0) return (double)((const float*)v->data)[idx];
    return (double)((const uint16_t*)v->data)[idx] / 65535.0;
}

/* cell index of a point: floor, clamped to [0, dims-2] */
static void cell_of(const oc_volume* v, const double* p, int* c) {
    for (int a = 0; a < 3; ++a) {
        double fl = floor(p[a]);
        int ci = fl < 0 ? 0 : (fl > v->dims[a] - 2 ? v->dims[a] - 2 : (int)fl);
        c[a] = ci;
    }
}

double oc_value(const oc_volume* v, const double* p) {
    int c[3];
    double w[3];
    cell_of(v, p, c);
    for (int a = 0; a < 3; ++a) {
        double t = p[a] - c[a];
        w[a] = t < 0 ? 0 : (t > 1 ? 1 : t);
    }
    double acc = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double wt = (dx ? w[0] : 1 - w[0]) * (dy ? w[1] : 1 - w[1]) * (dz ? w[2] : 1 - w[2]);
                acc += wt * node(v, c[0] + dx, c[1] + dy, c[2] + dz);
            }
    return acc;
}

/* ---------------------------------------------------------------------- */
/* Classification (sec. 2.4: "length-adjusted opacity"; reading G11):      */
/* the 256-entry table's opacity, given per reference length, is corrected */
/* to the step length, alpha' = 1 - (1 - alpha)^(step / ref_len), and the  */
/* table is then interpolated linearly at x = 255 v.                       */
/* ---------------------------------------------------------------------- */
void oc_lut_correct(const float* lut, double step, double ref_len, double* out) {
    for (int e = 0; e < 256; ++e) {
        out[4 * e + 0] = lut[4 * e + 0];
        out[4 * e + 1] = lut[4 * e + 1];
        out[4 * e + 2] = lut[4 * e + 2];
        out[4 * e + 3] = 1.0 - pow(1.0 - (double)lut[4 * e + 3], step / ref_len);
    }
}

/* straight colour and opacity of value v in [0,1] */
void oc_classify(const double* lutc, double v, double* rgba) {
    double x = v * 255.0;
    int i = (int)floor(x);
    if (i > 254) i = 254;
    if (i < 0) i = 0;
    double w = x - i;
    for (int c = 0; c < 4; ++c) rgba[c] = lutc[4 * i + c] * (1.0 - w) + lutc[4 * (i + 1) + c] * w;
}

/* ---------------------------------------------------------------------- */
/* Supersegment state machine: Eq. 1 and Algorithm S1 (readings G1-G6,     */
/* G9, G10).  Pieces are samples (generation) or sub-supersegment pieces   */
/* and transparent gaps (compositing), in depth order.                     */
/*                                                                         */
/* The open supersegment S keeps its front f_S, its extent end b_S (which  */
/* includes absorbed transparent pieces), the back b_t of its last          */
/* non-transparent piece, its premultiplied colour P_S and opacity A_S     */
/* (accumulated with "over" as in Algorithm S1).                          */
/* For an incoming piece x of length l_x, S's opacity is renormalised to   */
/* x's length (G1): a~ = 1 - (1 - A_S)^(l_x / l_S), and S's straight colour */
/* is C_S = P_S / A_S.  Eq. 1 then compares the premultiplied colours:     */
/* x starts a new supersegment iff || C_S a~ - P_x || >= gamma (G2), as     */
/* long as fewer than `cap` supersegments were opened (G10).  A piece with  */
/* zero opacity never opens a supersegment (G5).  Returns the number of    */
/* supersegments opened; writes them to `out` (if non-NULL, at most        */
/* max_out) as f_S, b_t, P_S, A_S.                                         */
/* ---------------------------------------------------------------------- */
int oc_segment(const oc_piece* x, int n, double gamma, int cap, double* out, int max_out, int* overflow) {
    int count = 0, open = 0, written = 0;
    double fS = 0, bS = 0, bt = 0, P[3] = {0, 0, 0}, A = 0, L = 0;
    if (overflow) *overflow = 0;
#define EMIT()                                                                         \
    do {                                                                               \
        if (out) {                                                                     \
            if (written < max_out) {                                                   \
                double* r = out + (size_t)REC * written;                               \
                r[0] = fS; r[1] = bt; r[2] = P[0]; r[3] = P[1]; r[4] = P[2]; r[5] = A; \
            } else if (overflow) *overflow = 1;                                        \
        }                                                                              \
        ++written;                                                                     \
    } while (0)
#define OPEN(px)                                                                       \
    do {                                                                               \
        fS = (px)->f; bS = (px)->b; bt = (px)->b;                                      \
        P[0] = (px)->P[0]; P[1] = (px)->P[1]; P[2] = (px)->P[2]; A = (px)->a;          \
        L = log1p(-(px)->a);                                                           \
        open = 1; ++count;                                                             \
    } while (0)
    for (int i = 0; i < n; ++i) {
        const oc_piece* p = x + i;
        if (p->brk) { /* sec. 5.3: the ray leaves the PE's domain */
            if (open) { EMIT(); open = 0; }
            continue;
        }
        if (!open) {
            if (p->a > 0.0) OPEN(p);
            continue;
        }
        double lx = p->b - p->f, lS = bS - fS;
        double r = (lx > 0.0 && lS > 0.0) ? lx / lS : 1.0;
        /* a~ = 1 - (1 - A_S)^r, with ln(1 - A_S) carried as the summed optical
           depth L of S's pieces (equal in exact arithmetic; stays accurate when
           A_S rounds to 1) */
        double at = -expm1(r * L);
        double cs[3];
        for (int c = 0; c < 3; ++c) cs[c] = A > 0.0 ? P[c] / A : 0.0;
        double d2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            double e = cs[c] * at - p->P[c];
            d2 += e * e;
        }
        double d = sqrt(d2);
        if (d >= gamma && count < cap) {
            EMIT();
            open = 0;
            if (p->a > 0.0) OPEN(p);
        } else {
            double T = 1.0 - A;
            for (int c = 0; c < 3; ++c) P[c] += T * p->P[c];
            A += T * p->a;
            L += log1p(-p->a);
            bS = p->b;
            if (p->a > 0.0) bt = p->b;
        }
    }
    if (open) EMIT();
#undef EMIT
#undef OPEN
    return count;
}

/* ---------------------------------------------------------------------- */
/* Per-ray iterative bisection search for gamma (sec. 2.4; sec. 5.2;       */
/* reading G8): if gamma = 0 yields at most n_s supersegments, gamma = 0.  */
/* Otherwise bisect [0, 2] (the criterion's distance never exceeds sqrt 3, */
/* so gamma = 2 opens at most one supersegment per domain run) for `iters` */
/* steps: a midpoint with count <= n_s becomes the upper end (and stops    */
/* the search if count == n_s), otherwise the lower end.  The result is    */
/* the upper end, which always satisfies the budget when any value does.  */
/* ---------------------------------------------------------------------- */
double oc_search(const oc_piece* x, int n, int n_s, int iters, int* n_passes) {
    int passes = 1;
    int c0 = oc_segment(x, n, 0.0, 1 << 30, NULL, 0, NULL);
    if (c0 <= n_s) {
        if (n_passes) *n_passes = passes;
        return 0.0;
    }
    double lo = 0.0, hi = 2.0;
    for (int it = 0; it < iters; ++it) {
        double mid = 0.5 * (lo + hi);
        int c = oc_segment(x, n, mid, 1 << 30, NULL, 0, NULL);
        ++passes;
        if (c <= n_s) {
            hi = mid;
            if (c == n_s) break;
        } else {
            lo = mid;
        }
    }
    if (n_passes) *n_passes = passes;
    return hi;
}

/* ---------------------------------------------------------------------- */
/* Samples along a ray (reading G11, G12): global grid t_k = t_in + (k+1/2) */
/* step for every k whose midpoint lies before t_out; sample k covers       */
/* [t_in + k step, t_in + (k+1) step].  Its owner is the PE whose cells     */
/* contain the floor of the midpoint (clamped to the volume's cells).       */
/* ---------------------------------------------------------------------- */
typedef struct {
    double f, b, P[3], a;
    int owner;
} oc_sample;

static int owner_of(const oc_volume* v, const oc_box* boxes, int k, const int* owner_map, const double* p) {
    int c[3];
    cell_of(v, p, c);
    if (owner_map) {
        size_t idx = ((size_t)c[2] * (v->dims[1] - 1) + c[1]) * (v->dims[0] - 1) + c[0];
        return owner_map[idx];
    }
    for (int e = 0; e < k; ++e) {
        const oc_box* bx = boxes + e;
        if (c[0] >= bx->lo[0] && c[0] < bx->hi[0] && c[1] >= bx->lo[1] && c[1] < bx->hi[1] && c[2] >= bx->lo[2] &&
            c[2] < bx->hi[2])
            return e;
    }
    return -1;
}

/* Returns the number of samples written to s (at most max_s; -1 if more). */
static int ray_samples(const oc_volume* v, const oc_box* boxes, int k, const int* owner_map, const double* lutc,
                       double step, const double* o, const double* d, oc_sample* s, int max_s) {
    double tin, tout;
    if (!oc_hit_box(o, d, v->dims, &tin, &tout)) return 0;
    int n = 0;
    for (long kk = 0;; ++kk) {
        double tm = tin + ((double)kk + 0.5) * step;
        if (!(tm < tout)) break;
        if (n >= max_s) return -1;
        double p[3] = {o[0] + tm * d[0], o[1] + tm * d[1], o[2] + tm * d[2]};
        double rgba[4];
        oc_classify(lutc, oc_value(v, p), rgba);
        oc_sample* q = s + n++;
        q->f = tin + (double)kk * step;
        q->b = tin + (double)(kk + 1) * step;
        q->a = rgba[3];
        for (int c = 0; c < 3; ++c) q->P[c] = rgba[c] * rgba[3];
        q->owner = owner_of(v, boxes, k, owner_map, p);
    }
    return n;
}

/* ---------------------------------------------------------------------- */
/* Phase 1: sub-VDI generation (sec. 5.1, sec. 4).  For every PE e and    */
/* every requested pixel: the PE's own samples in depth order (with a      */
/* break wherever the ray left the PE's domain and came back), gamma fixed */
/* (gamma >= 0) or searched (gamma < 0), then emission with cap n_s.       */
/* Outputs are indexed [e][q] for pixel q of `pixels`:                     */
/*   counts[e*np+q], gammas[e*np+q], recs[((e*np+q)*maxrec + j)*6 + c].     */
/* Returns 0, or -2 if a list exceeded maxrec, -3 if a ray had too many    */
/* samples.                                                                */
/* ---------------------------------------------------------------------- */
int oc_generate(const oc_volume* v, const oc_box* boxes, int k, const int* owner_map, const float* lut,
                const oc_camera* cam, double step, double ref_len, int n_s, double gamma, int iters,
                const int* pixels, int np, int maxrec, int* counts, double* gammas, double* recs, int* passes_out) {
    double lutc[256 * 4];
    oc_lut_correct(lut, step, ref_len, lutc);
    int max_s = 0;
    for (int a = 0; a < 3; ++a) max_s += v->dims[a];
    max_s = (int)(2.0 * max_s / step) + 16;
    int err = 0;
#pragma omp parallel
    {
        oc_sample* s = malloc(sizeof(oc_sample) * (size_t)max_s);
        oc_piece* pc = malloc(sizeof(oc_piece) * (size_t)max_s);
#pragma omp for schedule(dynamic, 16)
        for (int q = 0; q < np; ++q) {
            int i = pixels[q] % cam->width, j = pixels[q] / cam->width;
            double o[3], d[3];
            oc_ray(cam, i, j, o, d);
            int ns = ray_samples(v, boxes, k, owner_map, lutc, step, o, d, s, max_s);
            if (ns < 0) {
#pragma omp atomic write
                err = -3;
                ns = 0;
            }
            for (int e = 0; e < k; ++e) {
                int n = 0, seen = 0, away = 0;
                for (int t = 0; t < ns; ++t) {
                    if (s[t].owner != e) {
                        if (seen) away = 1;
                        continue;
                    }
                    if (away) { /* left the domain and came back (sec. 5.3) */
                        memset(pc + n, 0, sizeof(oc_piece));
                        pc[n++].brk = 1;
                        away = 0;
                    }
                    seen = 1;
                    pc[n].f = s[t].f; pc[n].b = s[t].b; pc[n].a = s[t].a;
                    pc[n].P[0] = s[t].P[0]; pc[n].P[1] = s[t].P[1]; pc[n].P[2] = s[t].P[2];
                    pc[n].brk = 0;
                    ++n;
                }
                int np_ = 0;
                double g = gamma >= 0.0 ? gamma : oc_search(pc, n, n_s, iters, &np_);
                int ovf = 0;
                int cnt = oc_segment(pc, n, g, n_s, recs ? recs + (size_t)(e * (size_t)np + q) * maxrec * REC : NULL,
                                     maxrec, &ovf);
                if (ovf) {
#pragma omp atomic write
                    err = -2;
                }
                size_t idx = (size_t)e * np + q;
                if (counts) counts[idx] = cnt;
                if (gammas) gammas[idx] = g;
                if (passes_out) passes_out[idx] = np_;
            }
        }
        free(s);
        free(pc);
    }
    return err;
}

/* ---------------------------------------------------------------------- */
/* Compact layout (sec. 4, Fig. 2b): exclusive prefix sum of the counts.   */
/* offsets has n+1 entries; the last one is the total.                     */
/* ---------------------------------------------------------------------- */
void oc_exclusive_scan(const int* counts, int n, uint64_t* offsets) {
    uint64_t acc = 0;
    for (int i = 0; i < n; ++i) {
        offsets[i] = acc;
        acc += (uint64_t)counts[i];
    }
    offsets[n] = acc;
}

/* ---------------------------------------------------------------------- */
/* Input lists for compositing: one compact sub-VDI per PE.                */
/* prec 0: fb double[2], rgba double[4]; 1: fb float[2], rgba float[4];    */
/* 2: 16-byte records {float f, float b, binary16 R, G, B, tau} in `rgba`:  */
/* premultiplied colour and the opacity as its base-2 optical depth         */
/* tau = -log2(1 - A), so A = 1 - 2^-tau (reading G17: FP16 storage).      */
/* The list of pixel p is records [offsets[p], offsets[p] + counts[p]).   */
/* ---------------------------------------------------------------------- */
typedef struct {
    const uint32_t* counts;
    const uint64_t* offsets;
    const void* fb;
    const void* rgba;
    int prec;
} oc_lists;

/* IEEE 754 binary16 -> double, from the format's definition */
double oc_half_to_double(uint16_t h) {
    int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp((double)(1024 + m), e - 25);
    return s ? -v : v;
}

static void read_rec(const oc_lists* L, uint64_t r, double* out) {
    if (L->prec == 0) {
        const double* fb = (const double*)L->fb + 2 * r;
        const double* c = (const double*)L->rgba + 4 * r;
        out[0] = fb[0]; out[1] = fb[1];
        out[2] = c[0]; out[3] = c[1]; out[4] = c[2]; out[5] = c[3];
    } else if (L->prec == 1) {
        const float* fb = (const float*)L->fb + 2 * r;
        const float* c = (const float*)L->rgba + 4 * r;
        out[0] = fb[0]; out[1] = fb[1];
        out[2] = c[0]; out[3] = c[1]; out[4] = c[2]; out[5] = c[3];
    } else {
        const unsigned char* base = (const unsigned char*)L->rgba + 16 * r;
        float f, b;
        uint16_t h[4];
        memcpy(&f, base, 4);
        memcpy(&b, base + 4, 4);
        memcpy(h, base + 8, 8);
        out[0] = f; out[1] = b;
        for (int c = 0; c < 3; ++c) out[2 + c] = oc_half_to_double(h[c]);
        out[5] = -expm1(-oc_half_to_double(h[3]) * log(2.0));
    }
}

/* ---------------------------------------------------------------------- */
/* Phase 2 pieces (sec. 5.2, Eq. 2, reading G7): all sub-supersegments of a */
/* pixel with b > f, cut at every front and back depth.  On each interval:  */
/*  - no record covers it: a transparent gap;                               */
/*  - one record covers it whole: that record unchanged;                    */
/*  - otherwise the emission-absorption mixture of the covering records:    */
/*    each has extinction mu_i = -ln(1 - A_i) / l_i, so the interval's      */
/*    opacity is 1 - exp(-sum mu_i dt) and its colour the mu-weighted mean  */
/*    of the records' colours C_i = P_i / A_i.  With one record this is     */
/*    Eq. 2 with l = dt / l_i.  Records with A_i = 1 are opaque: the piece   */
/*    is opaque with their mean colour.                                      */
/* Writes at most max_pc pieces; returns the count (or -1 on overflow).    */
/* ---------------------------------------------------------------------- */
static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

int oc_pieces(const double* recs, int nr, oc_piece* out, int max_pc, double* bounds_scratch) {
    int nb = 0;
    for (int i = 0; i < nr; ++i) {
        const double* r = recs + (size_t)REC * i;
        if (!(r[1] > r[0])) continue;
        bounds_scratch[nb++] = r[0];
        bounds_scratch[nb++] = r[1];
    }
    qsort(bounds_scratch, nb, sizeof(double), cmp_double);
    int nu = 0;
    for (int i = 0; i < nb; ++i)
        if (nu == 0 || bounds_scratch[i] != bounds_scratch[nu - 1]) bounds_scratch[nu++] = bounds_scratch[i];
    int np = 0;
    for (int j = 0; j + 1 < nu; ++j) {
        double t0 = bounds_scratch[j], t1 = bounds_scratch[j + 1], dt = t1 - t0;
        int nact = 0, last = -1, nopaque = 0;
        double M = 0.0, MC[3] = {0, 0, 0}, OC[3] = {0, 0, 0};
        for (int i = 0; i < nr; ++i) {
            const double* r = recs + (size_t)REC * i;
            if (!(r[1] > r[0])) continue;
            if (r[0] <= t0 && r[1] >= t1) {
                ++nact;
                last = i;
                double A = r[5], l = r[1] - r[0];
                if (A >= 1.0) {
                    ++nopaque;
                    for (int c = 0; c < 3; ++c) OC[c] += r[2 + c] / A;
                } else if (A > 0.0) {
                    double mu = -log1p(-A) / l;
                    M += mu;
                    for (int c = 0; c < 3; ++c) MC[c] += mu * (r[2 + c] / A);
                }
            }
        }
        if (np >= max_pc) return -1;
        oc_piece* p = out + np++;
        memset(p, 0, sizeof *p);
        p->f = t0;
        p->b = t1;
        if (nact == 0) continue; /* transparent gap */
        const double* r = recs + (size_t)REC * last;
        if (nact == 1 && r[0] == t0 && r[1] == t1) { /* whole record, unchanged */
            p->a = r[5];
            for (int c = 0; c < 3; ++c) p->P[c] = r[2 + c];
            continue;
        }
        if (nopaque > 0) {
            p->a = 1.0;
            for (int c = 0; c < 3; ++c) p->P[c] = OC[c] / nopaque;
        } else if (M > 0.0) {
            double a = -expm1(-M * dt);
            p->a = a;
            for (int c = 0; c < 3; ++c) p->P[c] = (MC[c] / M) * a;
        }
    }
    return np;
}

/* ---------------------------------------------------------------------- */
/* Phase 2: compositing (sec. 5.2, Algorithm S1).  For each requested      */
/* pixel: gather its K lists, build the pieces, search gamma for n_s       */
/* supersegments, emit them (regular layout, zero tail).                   */
/*   out_counts[q], out_gamma[q], out_recs[(q*n_s + j)*6 + c].              */
/* Returns 0, or -1 if a pixel had more than max_in records in total.      */
/* ---------------------------------------------------------------------- */
int oc_composite(const oc_lists* lists, int k, const int* pixels, int np, int n_s, int iters, int max_in,
                 int* out_counts, double* out_gamma, double* out_recs, int* passes_out) {
    int err = 0;
#pragma omp parallel
    {
        double* recs = malloc(sizeof(double) * REC * (size_t)max_in);
        double* bounds = malloc(sizeof(double) * 2 * (size_t)max_in + 2);
        oc_piece* pc = malloc(sizeof(oc_piece) * (2 * (size_t)max_in + 2));
#pragma omp for schedule(dynamic, 16)
        for (int q = 0; q < np; ++q) {
            int p = pixels[q], nr = 0, bad = 0;
            for (int e = 0; e < k; ++e) {
                uint32_t c = lists[e].counts[p];
                uint64_t o = lists[e].offsets[p];
                for (uint32_t t = 0; t < c; ++t) {
                    if (nr >= max_in) { bad = 1; break; }
                    read_rec(&lists[e], o + t, recs + (size_t)REC * nr++);
                }
            }
            if (bad) {
#pragma omp atomic write
                err = -1;
            }
            int npc = oc_pieces(recs, nr, pc, 2 * max_in + 2, bounds);
            int passes = 0;
            double g = oc_search(pc, npc, n_s, iters, &passes);
            double* dst = out_recs + (size_t)q * n_s * REC;
            memset(dst, 0, sizeof(double) * REC * (size_t)n_s);
            int cnt = oc_segment(pc, npc, g, n_s, dst, n_s, NULL);
            out_counts[q] = cnt;
            if (out_gamma) out_gamma[q] = g;
            if (passes_out) passes_out[q] = passes;
        }
        free(recs);
        free(bounds);
        free(pc);
    }
    return err;
}

/* ---------------------------------------------------------------------- */
/* Flattening from the generating view: front-to-back "over" of the        */
/* records (sec. 2.3).  recs[(q*stride + j)*6 + c] for j < counts[q].      */
/* ---------------------------------------------------------------------- */
void oc_flatten(const int* counts, const double* recs, int np, int stride, double* rgba) {
    for (int q = 0; q < np; ++q) {
        double C[3] = {0, 0, 0}, A = 0.0;
        for (int j = 0; j < counts[q]; ++j) {
            const double* r = recs + ((size_t)q * stride + j) * REC;
            double T = 1.0 - A;
            for (int c = 0; c < 3; ++c) C[c] += T * r[2 + c];
            A += T * r[5];
        }
        rgba[4 * q + 0] = C[0]; rgba[4 * q + 1] = C[1]; rgba[4 * q + 2] = C[2]; rgba[4 * q + 3] = A;
    }
}

/* ---------------------------------------------------------------------- */
/* Ground-truth direct volume rendering: the same samples as generation,   */
/* all of them, composited front to back with "over" (sec. 2.3, sec. 7's   */
/* emission-absorption model).  Premultiplied RGB + A per pixel.           */
/* ---------------------------------------------------------------------- */
int oc_dvr(const oc_volume* v, const float* lut, const oc_camera* cam, double step, double ref_len,
           const int* pixels, int np, double* rgba) {
    double lutc[256 * 4];
    oc_lut_correct(lut, step, ref_len, lutc);
#pragma omp parallel for schedule(dynamic, 16)
    for (int q = 0; q < np; ++q) {
        int i = pixels[q] % cam->width, j = pixels[q] / cam->width;
        double o[3], d[3], tin, tout, C[3] = {0, 0, 0}, A = 0.0;
        oc_ray(cam, i, j, o, d);
        if (oc_hit_box(o, d, v->dims, &tin, &tout)) {
            for (long kk = 0;; ++kk) {
                double tm = tin + ((double)kk + 0.5) * step;
                if (!(tm < tout)) break;
                double p[3] = {o[0] + tm * d[0], o[1] + tm * d[1], o[2] + tm * d[2]};
                double s[4];
                oc_classify(lutc, oc_value(v, p), s);
                double T = 1.0 - A;
                for (int c = 0; c < 3; ++c) C[c] += T * s[c] * s[3];
                A += T * s[3];
            }
        }
        rgba[4 * q + 0] = C[0]; rgba[4 * q + 1] = C[1]; rgba[4 * q + 2] = C[2]; rgba[4 * q + 3] = A;
    }
    return 0;
}

/* Sample count along one pixel's ray (for the tests and work accounting). */
int oc_ray_sample_count(const oc_volume* v, const oc_camera* cam, double step, int pixel, double* t_in_out) {
    double o[3], d[3], tin, tout;
    oc_ray(cam, pixel % cam->width, pixel / cam->width, o, d);
    if (!oc_hit_box(o, d, v->dims, &tin, &tout)) return 0;
    int n = 0;
    while (tin + (n + 0.5) * step < tout) ++n;
    if (t_in_out) { t_in_out[0] = tin; t_in_out[1] = tout; }
    return n;
}

/* Near-equal block decomposition (sec. 3): the cells of each axis are split
 * into g[a] runs whose sizes differ by at most one; boxes are ordered with x
 * fastest.  Fills k = g0*g1*g2 boxes.                                      */
void oc_split_boxes(const int* dims, const int* g, oc_box* boxes) {
    int e = 0;
    for (int z = 0; z < g[2]; ++z)
        for (int y = 0; y < g[1]; ++y)
            for (int x = 0; x < g[0]; ++x) {
                int idx[3] = {x, y, z};
                for (int a = 0; a < 3; ++a) {
                    int cells = dims[a] - 1;
                    boxes[e].lo[a] = (int)(((long)cells * idx[a]) / g[a]);
                    boxes[e].hi[a] = (int)(((long)cells * (idx[a] + 1)) / g[a]);
                }
                ++e;
            }
}

/* ====================================================================== */
/* Learned gamma (an extension of the method; the paper searches gamma per */
/* ray, sec. 2.4).  Per (PE, 16 x 16 pixel tile) features feed a small     */
/* MLP that predicts log2 gamma for the tile; the search remains the       */
/* fallback and the judge.                                                 */
/* ====================================================================== */
#define OC_NF 40
#define OC_NH 64
#define OC_TILE 16

/* Features of one (PE, tile) from the owned samples of the tile's rays at
 * even pixel offsets (8 x 8 of its 16 x 16 rays), in order:
 *  [0..31]  histogram of the opacity a' of non-transparent samples, bins of
 *           width 1/64 (bin 31 holds a' >= 31/64), normalised to sum 1;
 *  [32],[33] mean and standard deviation over rays with a non-transparent
 *           sample of the depth of the first one, (k_first - k0) step / diag;
 *  [34],[35] the same for the back of the last one, (k_last + 1 - k0) step / diag;
 *  [36]     log1p(mean non-transparent samples per ray with owned samples) / 8;
 *  [37]     n_s / 64;
 *  [38]     fraction of rays with owned samples that have a non-transparent one;
 *  [39]     mean |P_k - P_prev| over consecutive non-transparent samples.
 * diag is the volume box's diagonal.  A tile whose rays own no sample has all
 * features 0 and valid = 0.  Per-ray search results (gamma_ray, nt_ray, from
 * oc_generate with gamma < 0) give the label: the median over rays with
 * nt > 0 of log2(max(gamma, 2^-20)), the lower middle element for an even
 * number of rays.                                                         */
int oc_tile_features(const oc_volume* v, const oc_box* boxes, int k, const float* lut, const oc_camera* cam,
                     double step, double ref_len, int n_s, double* feats, int* valid) {
    double lutc[256 * 4];
    oc_lut_correct(lut, step, ref_len, lutc);
    const int W = cam->width, H = cam->height;
    const int tx = (W + OC_TILE - 1) / OC_TILE, ty = (H + OC_TILE - 1) / OC_TILE, nt_tiles = tx * ty;
    int max_s = 0;
    for (int a = 0; a < 3; ++a) max_s += v->dims[a];
    max_s = (int)(2.0 * max_s / step) + 16;
    double diag = 0.0;
    for (int a = 0; a < 3; ++a) diag += (double)(v->dims[a] - 1) * (v->dims[a] - 1);
    diag = sqrt(diag);
#pragma omp parallel
    {
        oc_sample* s = malloc(sizeof(oc_sample) * (size_t)max_s);
#pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < nt_tiles; ++t) {
            for (int e = 0; e < k; ++e) {
                double hist[32] = {0}, sf = 0, sf2 = 0, sl = 0, sl2 = 0, var = 0;
                long ntot = 0, pairs = 0, rays_own = 0, rays_nt = 0;
                for (int jj = 0; jj < OC_TILE; jj += 2)
                    for (int ii = 0; ii < OC_TILE; ii += 2) {
                        int i = (t % tx) * OC_TILE + ii, j = (t / tx) * OC_TILE + jj;
                        if (i >= W || j >= H) continue;
                        double o[3], d[3];
                        oc_ray(cam, i, j, o, d);
                        int ns = ray_samples(v, boxes, k, NULL, lutc, step, o, d, s, max_s);
                        int k0 = -1, kf = -1, kl = -1, nt = 0;
                        double prev[3] = {0, 0, 0};
                        for (int q = 0; q < ns; ++q) {
                            if (s[q].owner != e) continue;
                            if (k0 < 0) k0 = q;
                            if (s[q].a > 0.0) {
                                int bin = (int)floor(s[q].a * 64.0);
                                if (bin > 31) bin = 31;
                                hist[bin] += 1.0;
                                if (nt > 0) {
                                    double dd = 0;
                                    for (int c = 0; c < 3; ++c) dd += (s[q].P[c] - prev[c]) * (s[q].P[c] - prev[c]);
                                    var += sqrt(dd);
                                    ++pairs;
                                }
                                for (int c = 0; c < 3; ++c) prev[c] = s[q].P[c];
                                if (kf < 0) kf = q;
                                kl = q;
                                ++nt;
                            }
                        }
                        if (k0 < 0) continue;
                        ++rays_own;
                        ntot += nt;
                        if (nt > 0) {
                            ++rays_nt;
                            double f = (kf - k0) * step / diag, l = (kl + 1 - k0) * step / diag;
                            sf += f; sf2 += f * f; sl += l; sl2 += l * l;
                        }
                    }
                double* F = feats + ((size_t)e * nt_tiles + t) * OC_NF;
                for (int c = 0; c < OC_NF; ++c) F[c] = 0.0;
                valid[(size_t)e * nt_tiles + t] = rays_own > 0;
                if (rays_own == 0) continue;
                if (ntot > 0)
                    for (int c = 0; c < 32; ++c) F[c] = hist[c] / (double)ntot;
                if (rays_nt > 0) {
                    double mf = sf / rays_nt, ml = sl / rays_nt;
                    F[32] = mf;
                    F[33] = sqrt(fmax(sf2 / rays_nt - mf * mf, 0.0));
                    F[34] = ml;
                    F[35] = sqrt(fmax(sl2 / rays_nt - ml * ml, 0.0));
                }
                F[36] = log1p((double)ntot / (double)rays_own) / 8.0;
                F[37] = n_s / 64.0;
                F[38] = (double)rays_nt / (double)rays_own;
                F[39] = pairs > 0 ? var / (double)pairs : 0.0;
            }
        }
        free(s);
    }
    return 0;
}

static int cmp_dbl(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Tile labels from per-ray search results: gammas[e][p], nts[e][p] (the
 * count at gamma = 0, i.e. non-transparent samples).  labels[e][t], valid[e][t]. */
void oc_tile_labels(const double* gammas, const int* nts, int k, int W, int H, double* labels, int* valid) {
    const int tx = (W + OC_TILE - 1) / OC_TILE, ty = (H + OC_TILE - 1) / OC_TILE;
    double buf[OC_TILE * OC_TILE];
    for (int e = 0; e < k; ++e)
        for (int t = 0; t < tx * ty; ++t) {
            int n = 0;
            for (int jj = 0; jj < OC_TILE; ++jj)
                for (int ii = 0; ii < OC_TILE; ++ii) {
                    int i = (t % tx) * OC_TILE + ii, j = (t / tx) * OC_TILE + jj;
                    if (i >= W || j >= H) continue;
                    size_t p = (size_t)e * W * H + (size_t)j * W + i;
                    if (nts[p] <= 0) continue;
                    double g = gammas[p] > 0x1p-20 ? gammas[p] : 0x1p-20;
                    buf[n++] = log2(g);
                }
            size_t o = (size_t)e * tx * ty + t;
            valid[o] = n > 0;
            if (n == 0) { labels[o] = 0.0; continue; }
            qsort(buf, n, sizeof(double), cmp_dbl);
            labels[o] = buf[(n - 1) / 2];
        }
}

/* MLP 40 -> 64 -> 64 -> 1 with ReLU; parameters in one array:
 * W1[64][40], b1[64], W2[64][64], b2[64], w3[64], b3 (6849 values).
 * y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 = predicted log2 gamma.      */
#define OC_NPARAM (OC_NH * OC_NF + OC_NH + OC_NH * OC_NH + OC_NH + OC_NH + 1)

int oc_mlp_nparams(void) { return OC_NPARAM; }

static void mlp_fwd1(const double* th, const double* x, double* h1, double* h2, double* y) {
    const double *W1 = th, *b1 = W1 + OC_NH * OC_NF, *W2 = b1 + OC_NH, *b2 = W2 + OC_NH * OC_NH, *w3 = b2 + OC_NH,
                 *b3 = w3 + OC_NH;
    for (int o = 0; o < OC_NH; ++o) {
        double a = b1[o];
        for (int i = 0; i < OC_NF; ++i) a += W1[o * OC_NF + i] * x[i];
        h1[o] = a > 0 ? a : 0;
    }
    for (int o = 0; o < OC_NH; ++o) {
        double a = b2[o];
        for (int i = 0; i < OC_NH; ++i) a += W2[o * OC_NH + i] * h1[i];
        h2[o] = a > 0 ? a : 0;
    }
    double a = b3[0];
    for (int i = 0; i < OC_NH; ++i) a += w3[i] * h2[i];
    *y = a;
}

void oc_mlp_forward(const double* th, const double* x, int n, double* y) {
    for (int s = 0; s < n; ++s) {
        double h1[OC_NH], h2[OC_NH];
        mlp_fwd1(th, x + (size_t)s * OC_NF, h1, h2, y + s);
    }
}

/* Mean squared error over the rows with valid != 0 and its gradient with
 * respect to every parameter (backpropagation through the two ReLU layers;
 * ReLU'(0) = 0).  Returns the loss; grad has OC_NPARAM entries. */
double oc_mlp_loss_grad(const double* th, const double* x, const double* label, const int* valid, int n, double* grad) {
    const double *W2 = th + OC_NH * OC_NF + OC_NH, *w3 = W2 + OC_NH * OC_NH + OC_NH;
    double *gW1 = grad, *gb1 = gW1 + OC_NH * OC_NF, *gW2 = gb1 + OC_NH, *gb2 = gW2 + OC_NH * OC_NH, *gw3 = gb2 + OC_NH,
           *gb3 = gw3 + OC_NH;
    for (int i = 0; i < OC_NPARAM; ++i) grad[i] = 0.0;
    int m = 0;
    for (int s = 0; s < n; ++s) m += valid[s] != 0;
    if (m == 0) return 0.0;
    double loss = 0.0;
    for (int s = 0; s < n; ++s) {
        if (!valid[s]) continue;
        const double* xs = x + (size_t)s * OC_NF;
        double h1[OC_NH], h2[OC_NH], y;
        mlp_fwd1(th, xs, h1, h2, &y);
        double r = y - label[s];
        loss += r * r / m;
        double dy = 2.0 * r / m;
        gb3[0] += dy;
        double dh2[OC_NH], dh1[OC_NH];
        for (int i = 0; i < OC_NH; ++i) {
            gw3[i] += dy * h2[i];
            dh2[i] = h2[i] > 0 ? dy * w3[i] : 0.0;
        }
        for (int i = 0; i < OC_NH; ++i) dh1[i] = 0.0;
        for (int o = 0; o < OC_NH; ++o) {
            gb2[o] += dh2[o];
            for (int i = 0; i < OC_NH; ++i) {
                gW2[o * OC_NH + i] += dh2[o] * h1[i];
                dh1[i] += W2[o * OC_NH + i] * dh2[o];
            }
        }
        for (int o = 0; o < OC_NH; ++o) {
            double g = h1[o] > 0 ? dh1[o] : 0.0;
            gb1[o] += g;
            for (int i = 0; i < OC_NF; ++i) gW1[o * OC_NF + i] += g * xs[i];
        }
    }
    return loss;
}

/* ====================================================================== */
/* Rendering a regular VDI from another viewpoint.  The paper renders its   */
/* VDIs from deviated viewpoints to judge them (sec. 5.2, the comparison    */
/* with DVR at viewpoint deviations) with a renderer from earlier work that */
/* it does not restate; this is the plain reading of a VDI as a             */
/* view-dependent volume:                                                   */
/*  - the generating camera G splits space into frustum columns, one per   */
/*    pixel: the points whose projection through G's eye falls in the      */
/*    pixel's square on G's image plane (the plane at unit distance along  */
/*    G's forward axis);                                                    */
/*  - within pixel p's column, supersegment (f, b, P, A) occupies the      */
/*    points at distance f..b from G's eye (reading R1: the depth of a     */
/*    point off the column's centre ray is its distance from G's eye, which*/
/*    is the generation depth on the centre ray) and is a homogeneous      */
/*    emission-absorption medium: a path of length l through it has        */
/*    opacity 1 - (1 - A)^(l / (b - f)) (the length correction of Eq. 2)   */
/*    and straight colour P / A;                                           */
/*  - a ray of the viewing camera V is cut where it crosses column faces   */
/*    and supersegment shells, and the pieces are composited front to back */
/*    with "over" (sec. 2.3).  Everything outside the columns, and between */
/*    supersegments, is empty.                                              */
/* With V = G every ray stays on its column's centre line and the result   */
/* is the flattened VDI (oc_flatten).                                       */
/* ====================================================================== */
typedef struct {
    double eye[3], fwd[3], right[3], up[3];
    double th, asp;
    int W, H;
} oc_frame;

static void oc_frame_of(const oc_camera* c, oc_frame* F) {
    for (int a = 0; a < 3; ++a) F->eye[a] = c->eye[a];
    v_sub(c->center, c->eye, F->fwd);
    v_norm(F->fwd);
    v_cross(F->fwd, c->up, F->right);
    v_norm(F->right);
    v_cross(F->right, F->fwd, F->up);
    F->th = tan(0.5 * c->fovy_deg * 3.14159265358979323846 / 180.0);
    F->asp = (double)c->width / (double)c->height;
    F->W = c->width;
    F->H = c->height;
}

static double v_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static int cmp_dbl_up(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* One ray o + s d (unit d, s >= 0) through the VDI of G: counts[W_G H_G],  */
/* recs[W_G H_G][n_s][REC], rho_max at least the largest back depth.        */
/* Writes premultiplied RGBA to rgba[4].                                    */
void oc_render_ray(const int* counts, const double* recs, int n_s, double rho_max, const oc_camera* gen,
                   const double* o, const double* d, double* rgba) {
    oc_frame G;
    oc_frame_of(gen, &G);
    double q0[3];
    v_sub(o, G.eye, q0);
    const double qx = v_dot(q0, G.right), qy = v_dot(q0, G.up), qz = v_dot(q0, G.fwd);
    const double dx = v_dot(d, G.right), dy = v_dot(d, G.up), dz = v_dot(d, G.fwd);
    const double X0 = -G.th * G.asp, X1 = G.th * G.asp, Y0 = G.th, Y1 = -G.th;
    /* inside the frustum: x - X0 z >= 0, X1 z - x >= 0, Y0 z - y >= 0, y - Y1 z >= 0, all linear in s */
    double s_in = 0.0, s_out = INFINITY;
    const double A[4] = {qx - X0 * qz, X1 * qz - qx, Y0 * qz - qy, qy - Y1 * qz};
    const double B[4] = {dx - X0 * dz, X1 * dz - dx, Y0 * dz - dy, dy - Y1 * dz};
    rgba[0] = rgba[1] = rgba[2] = rgba[3] = 0.0;
    for (int c = 0; c < 4; ++c) {
        if (B[c] == 0.0) {
            if (A[c] < 0.0) return;
            continue;
        }
        double s = -A[c] / B[c];
        if (B[c] > 0.0) { if (s > s_in) s_in = s; }
        else if (s < s_out) s_out = s;
    }
    /* beyond |q0| + rho_max the distance from G's eye exceeds every back depth */
    const double s_far = sqrt(v_dot(q0, q0)) + rho_max + 1.0;
    if (s_out > s_far) s_out = s_far;
    if (!(s_out > s_in)) return;
    /* cut points: column faces, row faces, closest approach to G's eye */
    const int ncut_max = G.W + G.H + 4;
    double* cut = (double*)malloc(sizeof(double) * (size_t)ncut_max);
    int nc = 0;
    cut[nc++] = s_in;
    cut[nc++] = s_out;
    for (int i = 1; i < G.W; ++i) {
        const double Xi = (2.0 * i / G.W - 1.0) * G.th * G.asp;
        const double den = dx - Xi * dz;
        if (den == 0.0) continue;
        const double s = -(qx - Xi * qz) / den;
        if (s > s_in && s < s_out) cut[nc++] = s;
    }
    for (int j = 1; j < G.H; ++j) {
        const double Yj = (1.0 - 2.0 * j / G.H) * G.th;
        const double den = dy - Yj * dz;
        if (den == 0.0) continue;
        const double s = -(qy - Yj * qz) / den;
        if (s > s_in && s < s_out) cut[nc++] = s;
    }
    const double s_star = -v_dot(q0, d); /* closest approach of the line to G's eye */
    if (s_star > s_in && s_star < s_out) cut[nc++] = s_star;
    qsort(cut, nc, sizeof(double), cmp_dbl_up);
    double perp[3];
    for (int a = 0; a < 3; ++a) perp[a] = q0[a] + s_star * d[a];
    const double rho_star = sqrt(v_dot(perp, perp));
    double T = 1.0, C[3] = {0.0, 0.0, 0.0};
    for (int m = 0; m + 1 < nc; ++m) {
        const double sa = cut[m], sb = cut[m + 1];
        if (!(sb > sa)) continue;
        const double sm = 0.5 * (sa + sb);
        const double zm = qz + sm * dz;
        const double Xm = (qx + sm * dx) / zm, Ym = (qy + sm * dy) / zm;
        int iu = (int)floor((Xm / (G.th * G.asp) + 1.0) * 0.5 * G.W);
        int iv = (int)floor((1.0 - Ym / G.th) * 0.5 * G.H);
        if (iu < 0) iu = 0;
        if (iu >= G.W) iu = G.W - 1;
        if (iv < 0) iv = 0;
        if (iv >= G.H) iv = G.H - 1;
        const size_t p = (size_t)iv * G.W + iu;
        const int n = counts[p];
        const int rising = sm >= s_star; /* distance from G's eye grows with s on this piece */
        for (int t = 0; t < n; ++t) {
            const int k = rising ? t : n - 1 - t;
            const double* r = recs + ((size_t)p * n_s + k) * REC;
            const double f = r[0], b = r[1], Ar = r[5];
            if (!(b > f) || Ar <= 0.0) continue;
            /* s-interval of the piece where the distance lies in [f, b] */
            double lo, hi;
            const double cf = f > rho_star ? sqrt((f - rho_star) * (f + rho_star)) : 0.0;
            const double cb = b > rho_star ? sqrt((b - rho_star) * (b + rho_star)) : 0.0;
            if (b <= rho_star) continue;
            if (rising) { lo = s_star + cf; hi = s_star + cb; }
            else { lo = s_star - cb; hi = s_star - cf; }
            if (lo < sa) lo = sa;
            if (hi > sb) hi = sb;
            const double l = hi - lo;
            if (!(l > 0.0)) continue;
            double alpha;
            if (Ar >= 1.0) alpha = 1.0;
            else alpha = -expm1(log1p(-Ar) * l / (b - f));
            for (int c = 0; c < 3; ++c) C[c] += T * (r[2 + c] / Ar) * alpha;
            T *= 1.0 - alpha;
        }
    }
    free(cut);
    rgba[0] = C[0];
    rgba[1] = C[1];
    rgba[2] = C[2];
    rgba[3] = 1.0 - T;
}

/* Pixels (i, j) of V (pixel index j W_V + i) through the VDI of G. */
void oc_render_view(const int* counts, const double* recs, int n_s, const oc_camera* gen, const oc_camera* view,
                    const int* pixels, int np, double* rgba) {
    double rho_max = 0.0;
    for (size_t p = 0; p < (size_t)gen->width * gen->height; ++p)
        for (int k = 0; k < counts[p]; ++k) {
            const double b = recs[(p * n_s + k) * REC + 1];
            if (b > rho_max) rho_max = b;
        }
#pragma omp parallel for schedule(dynamic, 16)
    for (int q = 0; q < np; ++q) {
        double o[3], d[3];
        oc_ray(view, pixels[q] % view->width, pixels[q] / view->width, o, d);
        oc_render_ray(counts, recs, n_s, rho_max, gen, o, d, rgba + (size_t)4 * q);
    }
}
