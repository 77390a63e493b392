/*
 * Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.
 *
 * This file holds only input generation: volumes, transfer functions, camera
 * orbits and synthetic supersegment lists.  It contains none of the VDI
 * method's arithmetic (no raycasting, no compositing, no termination
 * criterion), so both sides of every parity test can consume its output.
 *
 * Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014): a sequential
 * stream for the few host-drawn parameters, and its output mixer applied to
 * hashed counters for everything that is generated per voxel or per pixel,
 * so that any element can be regenerated independently (and on any device).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no fast-math, so
 * results do not depend on FMA contraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SM64_GAMMA 0x9E3779B97F4A7C15ULL

/* SplitMix64 output function applied to x + golden gamma. */
static inline uint64_t sm64_mix(uint64_t x) {
    uint64_t z = x + SM64_GAMMA;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Sequential SplitMix64 stream. */
static inline uint64_t sm64_next(uint64_t* s) {
    *s += SM64_GAMMA;
    uint64_t z = *s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform double in [0,1) with 53 bits */
static inline double u53(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }
/* uniform float in [0,1) with 24 bits: exactly representable, identical on any device */
static inline float u24(uint64_t h) { return (float)(uint32_t)(h >> 40) * (1.0f / 16777216.0f); }

uint64_t synth_hash4(uint64_t seed, uint64_t a, uint64_t b, uint64_t c) {
    uint64_t h = sm64_mix(seed);
    h = sm64_mix(h ^ a);
    h = sm64_mix(h ^ b);
    h = sm64_mix(h ^ c);
    return h;
}

/* ------------------------------------------------------------------------ */
/* Volumes: sum of anisotropic axis-aligned Gaussian blobs plus value noise.  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int X, Y, Z, n_blobs, octaves;
    double noise_amp, base_freq;
    uint64_t seed;
    double* gx; /* [X][n_blobs] separable blob factors */
    double* gy; /* [Y][n_blobs] */
    double* gz; /* [Z][n_blobs] */
    double* lat[8]; /* per-octave lattice values, (f+1)^3 */
    int freq[8];
} vol_ctx;

static double smoothstep01(double t) { return t * t * (3.0 - 2.0 * t); }

static double noise_at(const vol_ctx* c, int o, double ux, double uy, double uz) {
    int f = c->freq[o];
    double x = ux * f, y = uy * f, z = uz * f;
    int i = (int)floor(x), j = (int)floor(y), k = (int)floor(z);
    if (i > f - 1) i = f - 1;
    if (j > f - 1) j = f - 1;
    if (k > f - 1) k = f - 1;
    double sx = smoothstep01(x - i), sy = smoothstep01(y - j), sz = smoothstep01(z - k);
    const double* L = c->lat[o];
    int n = f + 1;
#define LAT(a, b, d) L[((size_t)(d) * n + (b)) * n + (a)]
    double c00 = LAT(i, j, k) * (1 - sx) + LAT(i + 1, j, k) * sx;
    double c10 = LAT(i, j + 1, k) * (1 - sx) + LAT(i + 1, j + 1, k) * sx;
    double c01 = LAT(i, j, k + 1) * (1 - sx) + LAT(i + 1, j, k + 1) * sx;
    double c11 = LAT(i, j + 1, k + 1) * (1 - sx) + LAT(i + 1, j + 1, k + 1) * sx;
#undef LAT
    double c0 = c00 * (1 - sy) + c10 * sy;
    double c1 = c01 * (1 - sy) + c11 * sy;
    return c0 * (1 - sz) + c1 * sz;
}

static double raw_value(const vol_ctx* c, int x, int y, int z, const double* wyz) {
    double s = 0.0;
    const double* g = c->gx + (size_t)x * c->n_blobs;
    for (int b = 0; b < c->n_blobs; ++b) s += g[b] * wyz[b];
    double ux = c->X > 1 ? (double)x / (c->X - 1) : 0.0;
    double uy = c->Y > 1 ? (double)y / (c->Y - 1) : 0.0;
    double uz = c->Z > 1 ? (double)z / (c->Z - 1) : 0.0;
    double amp = 1.0, nz = 0.0;
    for (int o = 0; o < c->octaves; ++o) {
        nz += amp * noise_at(c, o, ux, uy, uz);
        amp *= 0.5;
    }
    return s + c->noise_amp * nz;
}

/*
 * Fill `out` (x fastest, then y, then z) with the normalised blob+noise field.
 * dtype 0: float32 in [0,1]; dtype 1: uint16 = round(v * 65535).
 * Returns 0 on success, -1 on bad arguments / allocation failure.
 */
int synth_volume(int X, int Y, int Z, int n_blobs, int octaves, double noise_amp, double base_freq,
                 uint64_t seed, int dtype, void* out) {
    if (X < 2 || Y < 2 || Z < 2 || n_blobs < 0 || octaves < 0 || octaves > 8 || !out) return -1;
    vol_ctx c;
    memset(&c, 0, sizeof c);
    c.X = X; c.Y = Y; c.Z = Z; c.n_blobs = n_blobs; c.octaves = octaves;
    c.noise_amp = noise_amp; c.base_freq = base_freq; c.seed = seed;
    int nb = n_blobs > 0 ? n_blobs : 1;
    c.gx = calloc((size_t)X * nb, sizeof(double));
    c.gy = calloc((size_t)Y * nb, sizeof(double));
    c.gz = calloc((size_t)Z * nb, sizeof(double));
    if (!c.gx || !c.gy || !c.gz) return -1;
    uint64_t st = seed;
    for (int b = 0; b < n_blobs; ++b) {
        double cx = u53(sm64_next(&st)), cy = u53(sm64_next(&st)), cz = u53(sm64_next(&st));
        double sx = 0.03 + 0.12 * u53(sm64_next(&st));
        double sy = 0.03 + 0.12 * u53(sm64_next(&st));
        double sz = 0.03 + 0.12 * u53(sm64_next(&st));
        for (int x = 0; x < X; ++x) { double u = (double)x / (X - 1) - cx; c.gx[(size_t)x * nb + b] = exp(-u * u / (2 * sx * sx)); }
        for (int y = 0; y < Y; ++y) { double u = (double)y / (Y - 1) - cy; c.gy[(size_t)y * nb + b] = exp(-u * u / (2 * sy * sy)); }
        for (int z = 0; z < Z; ++z) { double u = (double)z / (Z - 1) - cz; c.gz[(size_t)z * nb + b] = exp(-u * u / (2 * sz * sz)); }
    }
    for (int o = 0; o < octaves; ++o) {
        int f = (int)(base_freq * (double)(1 << o) + 0.5);
        if (f < 1) f = 1;
        c.freq[o] = f;
        size_t n = (size_t)(f + 1) * (f + 1) * (f + 1);
        c.lat[o] = malloc(n * sizeof(double));
        if (!c.lat[o]) return -1;
        for (int k = 0; k <= f; ++k)
            for (int j = 0; j <= f; ++j)
                for (int i = 0; i <= f; ++i)
                    c.lat[o][((size_t)k * (f + 1) + j) * (f + 1) + i] =
                        u53(synth_hash4(seed ^ 0x6e6f697365ULL, (uint64_t)o, (uint64_t)i | ((uint64_t)j << 21), (uint64_t)k));
    }

    double vmin = INFINITY, vmax = -INFINITY;
    for (int pass = 0; pass < 2; ++pass) {
        double lo = vmin, inv = (vmax > vmin) ? 1.0 / (vmax - vmin) : 0.0;
        double pmin = INFINITY, pmax = -INFINITY;
#pragma omp parallel
        {
            double* wyz = malloc(sizeof(double) * nb);
            double tmin = INFINITY, tmax = -INFINITY;
#pragma omp for schedule(dynamic, 1) collapse(2)
            for (int z = 0; z < Z; ++z)
                for (int y = 0; y < Y; ++y) {
                    for (int b = 0; b < n_blobs; ++b) wyz[b] = c.gy[(size_t)y * nb + b] * c.gz[(size_t)z * nb + b];
                    size_t row = ((size_t)z * Y + y) * X;
                    for (int x = 0; x < X; ++x) {
                        double r = raw_value(&c, x, y, z, wyz);
                        if (pass == 0) {
                            if (r < tmin) tmin = r;
                            if (r > tmax) tmax = r;
                        } else {
                            double v = (r - lo) * inv;
                            if (v < 0) v = 0;
                            if (v > 1) v = 1;
                            if (dtype == 0) ((float*)out)[row + x] = (float)v;
                            else ((uint16_t*)out)[row + x] = (uint16_t)floor(v * 65535.0 + 0.5);
                        }
                    }
                }
#pragma omp critical
            {
                if (tmin < pmin) pmin = tmin;
                if (tmax > pmax) pmax = tmax;
            }
            free(wyz);
        }
        if (pass == 0) { vmin = pmin; vmax = pmax; }
    }
    free(c.gx); free(c.gy); free(c.gz);
    for (int o = 0; o < octaves; ++o) free(c.lat[o]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Transfer function: 256 RGBA entries, straight colour, opacity per voxel    */
/* length.  Multi-hue colour ramp; 4-6 Gaussian opacity bumps capped at 0.6;  */
/* fully transparent below v = 0.2 and wherever the bumps sum below 1e-3.     */
/* ------------------------------------------------------------------------ */

static void hsv2rgb(double h, double s, double v, double* r, double* g, double* b) {
    h = fmod(h, 360.0);
    if (h < 0) h += 360.0;
    double c = v * s, x = c * (1 - fabs(fmod(h / 60.0, 2.0) - 1)), m = v - c;
    double rr = 0, gg = 0, bb = 0;
    if (h < 60) { rr = c; gg = x; }
    else if (h < 120) { rr = x; gg = c; }
    else if (h < 180) { gg = c; bb = x; }
    else if (h < 240) { gg = x; bb = c; }
    else if (h < 300) { rr = x; bb = c; }
    else { rr = c; bb = x; }
    *r = rr + m; *g = gg + m; *b = bb + m;
}

void synth_tf(uint64_t seed, float* lut) {
    uint64_t st = seed;
    int nb = 4 + (int)(sm64_next(&st) % 3);
    double m[6], s[6], a[6];
    for (int i = 0; i < nb; ++i) {
        m[i] = 0.25 + 0.70 * u53(sm64_next(&st));
        s[i] = 0.02 + 0.06 * u53(sm64_next(&st));
        a[i] = 0.2 + 0.4 * u53(sm64_next(&st));
    }
    double h0 = 360.0 * u53(sm64_next(&st));
    for (int e = 0; e < 256; ++e) {
        double v = e / 255.0, al = 0.0;
        if (v >= 0.2) {
            for (int i = 0; i < nb; ++i) al += a[i] * exp(-(v - m[i]) * (v - m[i]) / (2 * s[i] * s[i]));
            if (al > 0.6) al = 0.6;
            if (al < 1e-3) al = 0.0;
        }
        double r, g, b;
        hsv2rgb(h0 + 300.0 * v, 0.8, 1.0, &r, &g, &b);
        lut[4 * e + 0] = (float)r;
        lut[4 * e + 1] = (float)g;
        lut[4 * e + 2] = (float)b;
        lut[4 * e + 3] = (float)al;
    }
}

/* ------------------------------------------------------------------------ */
/* Camera orbit: eye on a sphere of radius 1.8 x the box half-diagonal about  */
/* the box centre, azimuth U[0,360), elevation U[-30,30] degrees, up = +z.    */
/* out: n_views x 9 doubles (eye, centre, up).                                */
/* ------------------------------------------------------------------------ */
void synth_orbit(uint64_t seed, int n_views, int X, int Y, int Z, double* out) {
    uint64_t st = seed;
    double cx = 0.5 * (X - 1), cy = 0.5 * (Y - 1), cz = 0.5 * (Z - 1);
    double hd = 0.5 * sqrt((double)(X - 1) * (X - 1) + (double)(Y - 1) * (Y - 1) + (double)(Z - 1) * (Z - 1));
    double R = 1.8 * hd, pi = 3.14159265358979323846;
    for (int v = 0; v < n_views; ++v) {
        double az = 2 * pi * u53(sm64_next(&st));
        double el = (pi / 6) * (2 * u53(sm64_next(&st)) - 1);
        double* o = out + 9 * v;
        o[0] = cx + R * cos(el) * cos(az);
        o[1] = cy + R * cos(el) * sin(az);
        o[2] = cz + R * sin(el);
        o[3] = cx; o[4] = cy; o[5] = cz;
        o[6] = 0; o[7] = 0; o[8] = 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Synthetic supersegment lists.                                              */
/* One list per (seed, request, set, pixel).  Length n = n_s when dense, else */
/* U{0..n_s}.  2n draws from U[0,1) (24-bit, exact in float) are sorted and   */
/* paired as f0 < b0 <= f1 < b1 ...  Opacity A ~ U[0,1), premultiplied colour */
/* RGB = A * U[0,1) per channel (one float multiply each).                    */
/* ------------------------------------------------------------------------ */

static inline uint64_t list_key(uint64_t seed, uint32_t req, uint32_t set, uint64_t pixel) {
    return synth_hash4(seed, ((uint64_t)req << 32) | set, pixel, 0x6c697374ULL);
}

int synth_list_len(uint64_t seed, uint32_t req, uint32_t set, uint64_t pixel, int n_s, int dense) {
    if (dense) return n_s;
    uint64_t key = list_key(seed, req, set, pixel);
    return (int)(sm64_mix(key ^ 0x4c454e47ULL) % (uint64_t)(n_s + 1));
}

/* Writes n records: fb[2*i] = f, fb[2*i+1] = b, rgba[4*i..] premultiplied. Returns n. */
int synth_list(uint64_t seed, uint32_t req, uint32_t set, uint64_t pixel, int n_s, int dense, float* fb, float* rgba) {
    int n = synth_list_len(seed, req, set, pixel, n_s, dense);
    uint64_t key = list_key(seed, req, set, pixel);
    float t[256];
    int m = 2 * n;
    if (m > 256) return -1;
    for (int j = 0; j < m; ++j) t[j] = u24(sm64_mix(key + 2 * (uint64_t)j + 1));
    /* insertion sort (n is small) */
    for (int j = 1; j < m; ++j) {
        float v = t[j];
        int i = j - 1;
        while (i >= 0 && t[i] > v) { t[i + 1] = t[i]; --i; }
        t[i + 1] = v;
    }
    for (int i = 0; i < n; ++i) {
        fb[2 * i] = t[2 * i];
        fb[2 * i + 1] = t[2 * i + 1];
        uint64_t kc = sm64_mix(key ^ (0x636f6c6fULL + 8 * (uint64_t)i));
        float A = u24(kc);
        float r = u24(sm64_mix(kc + 1)), g = u24(sm64_mix(kc + 2)), b = u24(sm64_mix(kc + 3));
        rgba[4 * i + 0] = A * r;
        rgba[4 * i + 1] = A * g;
        rgba[4 * i + 2] = A * b;
        rgba[4 * i + 3] = A;
    }
    return n;
}

/*
 * Compact arrays for pixels [0, n_pix) of one (request, set): counts[p],
 * offsets[p] (exclusive prefix sum, n_pix + 1 entries, the last one the
 * total), fb[2*rec], rgba[4*rec].  Pass fb/rgba
 * NULL to get counts/offsets only.  Returns the total record count.
 */
uint64_t synth_lists_compact(uint64_t seed, uint32_t req, uint32_t set, uint64_t n_pix, int n_s, int dense,
                             uint32_t* counts, uint64_t* offsets, float* fb, float* rgba) {
#pragma omp parallel for schedule(static)
    for (long long p = 0; p < (long long)n_pix; ++p) counts[p] = (uint32_t)synth_list_len(seed, req, set, (uint64_t)p, n_s, dense);
    uint64_t acc = 0;
    for (uint64_t p = 0; p < n_pix; ++p) { offsets[p] = acc; acc += counts[p]; }
    offsets[n_pix] = acc;
    if (fb && rgba) {
#pragma omp parallel for schedule(dynamic, 256)
        for (long long p = 0; p < (long long)n_pix; ++p) {
            uint64_t o = offsets[p];
            synth_list(seed, req, set, (uint64_t)p, n_s, dense, fb + 2 * o, rgba + 4 * o);
        }
    }
    return acc;
}

/*
 * Pooled lists (the batched workload, whose lists would not fit in memory if
 * every one were stored): a pool of `runs` sorted 64-record runs, run r being
 * synth_list(seed, SYNTH_POOL_REQ, 0, r, 64, dense).  The list of (req, set,
 * pixel) is the window of n = synth_list_len(...) consecutive records of run
 * `run`, starting at `start`; returns n and writes run and start.
 */
int synth_pool_pick(uint64_t seed, uint32_t req, uint32_t set, uint64_t pixel, int n_s, uint64_t runs,
                    uint64_t* run, int* start) {
    int n = synth_list_len(seed, req, set, pixel, n_s, 0);
    uint64_t key = list_key(seed, req, set, pixel);
    *run = sm64_mix(key ^ 0x706f6f6cULL) % runs;
    *start = (int)(sm64_mix(key ^ 0x73747274ULL) % (uint64_t)(64 - n + 1));
    return n;
}
