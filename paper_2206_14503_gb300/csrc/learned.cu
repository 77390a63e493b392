// Learned gamma: per (PE, 16 x 16 tile) features, a 40-64-64-1 MLP that
// predicts log2 gamma for the tile, its training, and generation with the
// predicted gamma (the bisection search of sec. 2.4 stays as the fallback
// for rays whose count at the predicted gamma exceeds N_S, and as the source
// of the training labels).  The paper has no learned component; this is an
// extension on top of its method.
//
// Model buffer (caller-allocated, vdi_model_bytes()):
//   FP32 master parameters theta[6849] in the order W1[64][40], b1[64],
//   W2[64][64], b2[64], w3[64], b3; a BF16 copy used by every forward pass;
//   Adam moments m, v; the Adam step count and the init seed.
//
// Inference (mlp_infer_kernel) runs the two hidden layers on the tensor
// cores with mma.sync m16n8k16 (BF16 operands, FP32 accumulation): 16 tiles
// per warp, the first layer's accumulators re-packed in registers as the
// second layer's A operand.  Training (mlp_fwdbwd_kernel, mlp_reduce_kernel,
// adam_kernel) uses FP32 arithmetic with the BF16-rounded weights, per-block
// partial gradients and a fixed-order reduction, so a step is deterministic.
#include <cuda_bf16.h>
#include <stdio.h>
#include <string.h>

#include "vdi_device.cuh"

namespace vdi {

constexpr int kNF = 40, kNFP = 48, kNH = 64, kFT = 16;
constexpr int kNP = kNH * kNF + kNH + kNH * kNH + kNH + kNH + 1;  // 6849
constexpr int oW1 = 0, oB1 = oW1 + kNH * kNF, oW2 = oB1 + kNH, oB2 = oW2 + kNH * kNH, oW3 = oB2 + kNH, oB3 = oW3 + kNH;

// byte offsets in the model buffer
constexpr size_t kMaster = 0;
constexpr size_t kBf16 = 27648;
constexpr size_t kMomM = kBf16 + 13824;
constexpr size_t kMomV = kMomM + 27648;
constexpr size_t kState = kMomV + 27648;  // uint64 step, uint64 seed
constexpr size_t kModelBytes = kState + 256;
static_assert(kNP * 4 <= 27648 && kNP * 2 <= 13824, "model layout");

struct ModelState {
    unsigned long long step, seed;
};

// ---------------------------------------------------------------------------
// Initialisation: He-uniform weights (bound sqrt(6 / fan_in)), zero biases and
// moments.  Uniforms from the SplitMix64 output mixer applied to (seed, index).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void model_init_kernel(unsigned char* model, unsigned long long seed) {
    float* th = reinterpret_cast<float*>(model + kMaster);
    __nv_bfloat16* tb = reinterpret_cast<__nv_bfloat16*>(model + kBf16);
    float* m = reinterpret_cast<float*>(model + kMomM);
    float* v = reinterpret_cast<float*>(model + kMomV);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kNP; p += gridDim.x * blockDim.x) {
        int fan = p < oB1 ? kNF : (p >= oW2 && p < oB2 ? kNH : (p >= oW3 && p < oB3 ? kNH : 0));
        float x = 0.f;
        if (fan > 0) {
            unsigned long long h = mix64(mix64(seed) ^ (unsigned long long)p);
            float u = (float)(unsigned)(h >> 40) * (1.0f / 16777216.0f);
            x = (2.f * u - 1.f) * sqrtf(6.f / (float)fan);
        }
        th[p] = x;
        tb[p] = __float2bfloat16_rn(x);
        m[p] = 0.f;
        v[p] = 0.f;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ModelState* s = reinterpret_cast<ModelState*>(model + kState);
        s->step = 0;
        s->seed = seed;
    }
}

// ---------------------------------------------------------------------------
// Tile features (one CTA of 8 x 8 threads per (tile, PE): the tile's rays at
// even pixel offsets): opacity histogram of
// non-transparent samples, first/last non-transparent depth statistics, mean
// count, N_S, coverage, colour change.
// ---------------------------------------------------------------------------
struct FeatArgs {
    BrickDev b[VDI_MAX_PE];
    CamDev cam;
    int dims[3];
    const float* lut;
    float scale255, step, ref_len, inv_diag;
    int k, n_s, tiles_x, tiles_y;
    float* feats;          // [k][tiles][40]
    unsigned char* valid;  // [k][tiles]
};

__device__ __forceinline__ float block_sum(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

__global__ void __launch_bounds__(64) tile_features_kernel(const __grid_constant__ FeatArgs a) {
    __shared__ float4 lut2[2 * 257];
    __shared__ float base[257][4];
    __shared__ int hist[32];
    __shared__ float red[8];
    for (int i = threadIdx.x; i < 257; i += blockDim.x) {
        int s = min(i, 255);
        float4 v = reinterpret_cast<const float4*>(a.lut)[s];
        base[i][0] = v.x; base[i][1] = v.y; base[i][2] = v.z;
        base[i][3] = 1.f - powf(1.f - v.w, a.step / a.ref_len);
    }
    if (threadIdx.x < 32) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < 257; i += blockDim.x) {
        int n = min(i + 1, 256);
        lut2[i] = make_float4(base[i][0], base[i][1], base[i][2], base[i][3]);
        lut2[257 + i] = make_float4(__fsub_rn(base[n][0], base[i][0]), __fsub_rn(base[n][1], base[i][1]),
                                      __fsub_rn(base[n][2], base[i][2]), __fsub_rn(base[n][3], base[i][3]));
    }
    __syncthreads();
    const int tile = blockIdx.x, e = blockIdx.y;
    const int i = (tile % a.tiles_x) * kFT + 2 * (threadIdx.x & 7), j = (tile / a.tiles_x) * kFT + 2 * (threadIdx.x >> 3);
    float own = 0.f, nt = 0.f, has = 0.f, f = 0.f, l = 0.f, var = 0.f, pairs = 0.f;
    if (i < a.cam.W && j < a.cam.H) {
        Ray r;
        int k0 = 0, k1 = 0;
        if (ray_setup(a.cam, i, j, a.dims, a.step, r) && owned_range(r, a.step, a.b[e], a.dims, k0, k1)) {
            own = 1.f;
            int kf = -1, kl = -1, cnt = 0;
            float pv[3] = {0.f, 0.f, 0.f};
            march(r, k0, k1, a.b[e], lut2, a.scale255, [&](int k, const Sample& s) {
                if (s.a > 0.f) {
                    atomicAdd(&hist[min((int)(s.a * 64.f), 31)], 1);
                    if (cnt > 0) {
                        float d0 = s.P[0] - pv[0], d1 = s.P[1] - pv[1], d2 = s.P[2] - pv[2];
                        var += sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
                        pairs += 1.f;
                    }
                    pv[0] = s.P[0]; pv[1] = s.P[1]; pv[2] = s.P[2];
                    if (kf < 0) kf = k;
                    kl = k;
                    ++cnt;
                }
            });
            nt = (float)cnt;
            if (cnt > 0) {
                has = 1.f;
                f = (float)(kf - k0) * a.step * a.inv_diag;
                l = (float)(kl + 1 - k0) * a.step * a.inv_diag;
            }
        }
    }
    const float s_own = block_sum(own, red), s_nt = block_sum(nt, red), s_has = block_sum(has, red);
    const float s_f = block_sum(f, red), s_f2 = block_sum(f * f, red), s_l = block_sum(l, red);
    const float s_l2 = block_sum(l * l, red), s_var = block_sum(var, red), s_pairs = block_sum(pairs, red);
    __syncthreads();
    float* F = a.feats + ((size_t)e * a.tiles_x * a.tiles_y + tile) * kNF;
    if (threadIdx.x < kNF) {
        float v = 0.f;
        const int c = threadIdx.x;
        if (s_own > 0.f) {
            if (c < 32) v = s_nt > 0.f ? (float)hist[c] / s_nt : 0.f;
            else if (c == 32) v = s_has > 0.f ? s_f / s_has : 0.f;
            else if (c == 33) v = s_has > 0.f ? sqrtf(fmaxf(s_f2 / s_has - (s_f / s_has) * (s_f / s_has), 0.f)) : 0.f;
            else if (c == 34) v = s_has > 0.f ? s_l / s_has : 0.f;
            else if (c == 35) v = s_has > 0.f ? sqrtf(fmaxf(s_l2 / s_has - (s_l / s_has) * (s_l / s_has), 0.f)) : 0.f;
            else if (c == 36) v = log1pf(s_nt / s_own) / 8.f;
            else if (c == 37) v = (float)a.n_s / 64.f;
            else if (c == 38) v = s_has / s_own;
            else v = s_pairs > 0.f ? s_var / s_pairs : 0.f;
        }
        F[c] = v;
    }
    if (threadIdx.x == 0) a.valid[(size_t)e * a.tiles_x * a.tiles_y + tile] = s_own > 0.f ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Tile labels: lower median over the tile's rays with a supersegment of
// log2(max(gamma, 2^-20)), from a searched generation's counts and gammas.
// ---------------------------------------------------------------------------
struct LabelArgs {
    const uint32_t* counts[VDI_MAX_PE];
    const float* gamma[VDI_MAX_PE];
    int W, H, tiles_x, tiles_y;
    float* labels;
    unsigned char* valid;
};

__global__ void __launch_bounds__(256) tile_labels_kernel(const __grid_constant__ LabelArgs a) {
    __shared__ float val[256];
    __shared__ int ok[256];
    __shared__ float red[8];
    const int tile = blockIdx.x, e = blockIdx.y;
    const int i = (tile % a.tiles_x) * kFT + (threadIdx.x & 15), j = (tile / a.tiles_x) * kFT + (threadIdx.x >> 4);
    float v = 0.f;
    int good = 0;
    if (i < a.W && j < a.H) {
        size_t p = (size_t)j * a.W + i;
        if (a.counts[e][p] > 0) {
            good = 1;
            v = log2f(fmaxf(a.gamma[e][p], 0x1p-20f));
        }
    }
    val[threadIdx.x] = v;
    ok[threadIdx.x] = good;
    const float n = block_sum((float)good, red);
    __syncthreads();
    const size_t o = (size_t)e * a.tiles_x * a.tiles_y + tile;
    if (threadIdx.x == 0) {
        a.valid[o] = n > 0.f ? 1 : 0;
        if (n == 0.f) a.labels[o] = 0.f;
    }
    if (good) {
        int rank = 0;
        for (int q = 0; q < 256; ++q)
            if (ok[q] && (val[q] < v || (val[q] == v && q < (int)threadIdx.x))) ++rank;
        if (rank == ((int)n - 1) / 2) a.labels[o] = v;
    }
}

// ---------------------------------------------------------------------------
// Inference on the tensor cores
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned*>(&v);
}

__global__ void __launch_bounds__(128) mlp_infer_kernel(const unsigned char* __restrict__ model,
                                                        const float* __restrict__ feats, int n, float offset,
                                                        float* __restrict__ out_log2g) {
    __shared__ __nv_bfloat16 w1[kNH][kNFP];
    __shared__ __nv_bfloat16 w2[kNH][kNH];
    __shared__ float b1[kNH], b2[kNH], w3[kNH];
    __shared__ float b3;
    const __nv_bfloat16* tb = reinterpret_cast<const __nv_bfloat16*>(model + kBf16);
    for (int q = threadIdx.x; q < kNH * kNFP; q += blockDim.x) {
        int o = q / kNFP, c = q % kNFP;
        w1[o][c] = c < kNF ? tb[oW1 + o * kNF + c] : __float2bfloat16_rn(0.f);
    }
    for (int q = threadIdx.x; q < kNH * kNH; q += blockDim.x) w2[q / kNH][q % kNH] = tb[oW2 + q];
    for (int q = threadIdx.x; q < kNH; q += blockDim.x) {
        b1[q] = __bfloat162float(tb[oB1 + q]);
        b2[q] = __bfloat162float(tb[oB2 + q]);
        w3[q] = __bfloat162float(tb[oW3 + q]);
    }
    if (threadIdx.x == 0) b3 = __bfloat162float(tb[oB3]);
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int r0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 16; r0 < n; r0 += warps * 16) {
        const int ra = r0 + g, rb = r0 + g + 8;
        auto X = [&](int r, int c) -> float { return (r < n && c < kNF) ? __ldg(feats + (size_t)r * kNF + c) : 0.f; };
        // layer 1: [16 x 48] . [48 x 64]
        float c1[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) c1[nt][0] = c1[nt][1] = c1[nt][2] = c1[nt][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
            const int c0 = 16 * kk + 2 * t;
            unsigned A[4] = {pack_bf16(X(ra, c0), X(ra, c0 + 1)), pack_bf16(X(rb, c0), X(rb, c0 + 1)),
                             pack_bf16(X(ra, c0 + 8), X(ra, c0 + 9)), pack_bf16(X(rb, c0 + 8), X(rb, c0 + 9))};
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int o = 8 * nt + g;
                unsigned b0 = *reinterpret_cast<const unsigned*>(&w1[o][c0]);
                unsigned b1r = *reinterpret_cast<const unsigned*>(&w1[o][c0 + 8]);
                mma_bf16(c1[nt], A, b0, b1r);
            }
        }
        // bias + ReLU, re-packed as layer 2's A operand
        unsigned A2[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int o = 8 * nt + 2 * t;
            float h0 = fmaxf(c1[nt][0] + b1[o], 0.f), h1 = fmaxf(c1[nt][1] + b1[o + 1], 0.f);
            float h2 = fmaxf(c1[nt][2] + b1[o], 0.f), h3 = fmaxf(c1[nt][3] + b1[o + 1], 0.f);
            const int kk = nt >> 1, half = nt & 1;
            A2[kk][2 * half] = pack_bf16(h0, h1);
            A2[kk][2 * half + 1] = pack_bf16(h2, h3);
        }
        // layer 2: [16 x 64] . [64 x 64]
        float c2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) c2[nt][0] = c2[nt][1] = c2[nt][2] = c2[nt][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int c0 = 16 * kk + 2 * t;
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int o = 8 * nt + g;
                unsigned b0 = *reinterpret_cast<const unsigned*>(&w2[o][c0]);
                unsigned b1r = *reinterpret_cast<const unsigned*>(&w2[o][c0 + 8]);
                mma_bf16(c2[nt], A2[kk], b0, b1r);
            }
        }
        // output layer: dot with w3 over the quad's columns, then across the quad
        float ya = 0.f, yb = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int o = 8 * nt + 2 * t;
            ya += fmaxf(c2[nt][0] + b2[o], 0.f) * w3[o] + fmaxf(c2[nt][1] + b2[o + 1], 0.f) * w3[o + 1];
            yb += fmaxf(c2[nt][2] + b2[o], 0.f) * w3[o] + fmaxf(c2[nt][3] + b2[o + 1], 0.f) * w3[o + 1];
        }
        ya += __shfl_xor_sync(0xffffffffu, ya, 1);
        ya += __shfl_xor_sync(0xffffffffu, ya, 2);
        yb += __shfl_xor_sync(0xffffffffu, yb, 1);
        yb += __shfl_xor_sync(0xffffffffu, yb, 2);
        if (t == 0) {
            if (ra < n) out_log2g[ra] = ya + b3 - offset;
            if (rb < n) out_log2g[rb] = yb + b3 - offset;
        }
    }
}

// per-ray gamma of a learned generation: 2^(prediction of the ray's tile)
struct ExpandArgs {
    float* gamma[VDI_MAX_PE];
    const float* pred;  // [k][tiles]
    int W, H, tiles_x, tiles;
};

__global__ void gamma_expand_kernel(const __grid_constant__ ExpandArgs a) {
    const int e = blockIdx.y;
    const size_t npix = (size_t)a.W * a.H;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(p % a.W), j = (int)(p / a.W);
        int t = (j / kFT) * a.tiles_x + i / kFT;
        a.gamma[e][p] = exp2f(a.pred[(size_t)e * a.tiles + t]);
    }
}

// ---------------------------------------------------------------------------
// Training: forward + backward per block of rows into per-block partial
// gradients; fixed-order reduction; Adam.
// ---------------------------------------------------------------------------
constexpr int kTrainRows = 64;

__global__ void count_valid_kernel(const unsigned char* valid, int n, float* m) {
    __shared__ float red[8];
    float c = 0.f;
    for (int r = threadIdx.x; r < n; r += blockDim.x) c += valid[r] ? 1.f : 0.f;
    float s = block_sum(c, red);
    if (threadIdx.x == 0) *m = s;
}

__global__ void __launch_bounds__(256) mlp_fwdbwd_kernel(const unsigned char* __restrict__ model,
                                                         const float* __restrict__ x, const float* __restrict__ y,
                                                         const unsigned char* __restrict__ valid, int n,
                                                         const float* __restrict__ mcount, float* __restrict__ partial) {
    extern __shared__ float sm[];
    float* W = sm;                              // kNP (BF16-rounded weights as FP32)
    float* X = W + kNP;                         // [rows][40]
    float* H1 = X + kTrainRows * kNF;           // [rows][64]
    float* H2 = H1 + kTrainRows * kNH;          // [rows][64]
    float* D2 = H2 + kTrainRows * kNH;          // [rows][64]
    float* D1 = D2 + kTrainRows * kNH;          // [rows][64]
    float* DY = D1 + kTrainRows * kNH;          // [rows]
    float* LS = DY + kTrainRows;                // [rows] loss terms
    const __nv_bfloat16* tb = reinterpret_cast<const __nv_bfloat16*>(model + kBf16);
    for (int q = threadIdx.x; q < kNP; q += blockDim.x) W[q] = __bfloat162float(tb[q]);
    const int r0 = blockIdx.x * kTrainRows;
    for (int q = threadIdx.x; q < kTrainRows * kNF; q += blockDim.x) {
        int r = r0 + q / kNF;
        X[q] = r < n ? x[(size_t)r0 * kNF + q] : 0.f;
    }
    __syncthreads();
    const float m = fmaxf(*mcount, 1.f);
    // layer 1
    for (int q = threadIdx.x; q < kTrainRows * kNH; q += blockDim.x) {
        int r = q / kNH, o = q % kNH;
        float s = W[oB1 + o];
        for (int i = 0; i < kNF; ++i) s = fmaf(W[oW1 + o * kNF + i], X[r * kNF + i], s);
        H1[q] = fmaxf(s, 0.f);
    }
    __syncthreads();
    // layer 2
    for (int q = threadIdx.x; q < kTrainRows * kNH; q += blockDim.x) {
        int r = q / kNH, o = q % kNH;
        float s = W[oB2 + o];
        for (int i = 0; i < kNH; ++i) s = fmaf(W[oW2 + o * kNH + i], H1[r * kNH + i], s);
        H2[q] = fmaxf(s, 0.f);
    }
    __syncthreads();
    // output and loss derivative (MSE over valid rows, normalised by their count)
    float* part = partial + (size_t)blockIdx.x * (kNP + 1);
    if (threadIdx.x < kTrainRows) {
        int rr = threadIdx.x, r = r0 + rr;
        float s = W[oB3];
        for (int i = 0; i < kNH; ++i) s = fmaf(W[oW3 + i], H2[rr * kNH + i], s);
        float d = (r < n && valid[r]) ? s - y[r] : 0.f;
        DY[rr] = 2.f * d / m;
        LS[rr] = d * d / m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int rr = 0; rr < kTrainRows; ++rr) l += LS[rr];
        part[kNP] = l;
    }
    __syncthreads();
    // delta of layer 2 pre-activations
    for (int q = threadIdx.x; q < kTrainRows * kNH; q += blockDim.x) {
        int r = q / kNH, o = q % kNH;
        D2[q] = H2[q] > 0.f ? DY[r] * W[oW3 + o] : 0.f;
    }
    __syncthreads();
    // delta of layer 1 pre-activations
    for (int q = threadIdx.x; q < kTrainRows * kNH; q += blockDim.x) {
        int r = q / kNH, i = q % kNH;
        float s = 0.f;
        for (int o = 0; o < kNH; ++o) s = fmaf(W[oW2 + o * kNH + i], D2[r * kNH + o], s);
        D1[q] = H1[q] > 0.f ? s : 0.f;
    }
    __syncthreads();
    // parameter gradients of this block (sums over its rows in fixed order)
    for (int p = threadIdx.x; p < kNP; p += blockDim.x) {
        float s = 0.f;
        if (p < oB1) {
            int o = p / kNF, i = p % kNF;
            for (int r = 0; r < kTrainRows; ++r) s = fmaf(D1[r * kNH + o], X[r * kNF + i], s);
        } else if (p < oW2) {
            int o = p - oB1;
            for (int r = 0; r < kTrainRows; ++r) s += D1[r * kNH + o];
        } else if (p < oB2) {
            int o = (p - oW2) / kNH, i = (p - oW2) % kNH;
            for (int r = 0; r < kTrainRows; ++r) s = fmaf(D2[r * kNH + o], H1[r * kNH + i], s);
        } else if (p < oW3) {
            int o = p - oB2;
            for (int r = 0; r < kTrainRows; ++r) s += D2[r * kNH + o];
        } else if (p < oB3) {
            int i = p - oW3;
            for (int r = 0; r < kTrainRows; ++r) s = fmaf(DY[r], H2[r * kNH + i], s);
        } else {
            for (int r = 0; r < kTrainRows; ++r) s += DY[r];
        }
        part[p] = s;
    }
}

__global__ void mlp_reduce_kernel(const float* __restrict__ partial, int blocks, float* __restrict__ grad,
                                  float* __restrict__ loss) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kNP) return;
    float s = 0.f;
    for (int b = 0; b < blocks; ++b) s += partial[(size_t)b * (kNP + 1) + p];
    if (p < kNP) grad[p] = s;
    else if (loss) *loss = s;
}

__global__ void adam_kernel(unsigned char* model, const float* __restrict__ grad, float lr, float b1, float b2,
                            float eps) {
    float* th = reinterpret_cast<float*>(model + kMaster);
    __nv_bfloat16* tb = reinterpret_cast<__nv_bfloat16*>(model + kBf16);
    float* m = reinterpret_cast<float*>(model + kMomM);
    float* v = reinterpret_cast<float*>(model + kMomV);
    ModelState* st = reinterpret_cast<ModelState*>(model + kState);
    const unsigned long long t = st->step + 1;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kNP; p += gridDim.x * blockDim.x) {
        float g = grad[p];
        float mm = b1 * m[p] + (1.f - b1) * g;
        float vv = b2 * v[p] + (1.f - b2) * g * g;
        m[p] = mm;
        v[p] = vv;
        float w = th[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        th[p] = w;
        tb[p] = __float2bfloat16_rn(w);
    }
}

__global__ void step_increment_kernel(unsigned char* model) {
    reinterpret_cast<ModelState*>(model + kState)->step += 1;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
size_t model_bytes() { return kModelBytes; }
int model_nparams() { return kNP; }

vdi_status launch_model_init(void* model, unsigned long long seed, cudaStream_t st) {
    model_init_kernel<<<8, 256, 0, st>>>(static_cast<unsigned char*>(model), seed);
    return cuda_check(cudaGetLastError(), "model_init_kernel launch");
}

vdi_status launch_tile_features(const BrickDev* bricks, int k, const float* lut, const CamDev& cam, const int dims[3],
                                float scale255, float step, float ref_len, int n_s, float* feats,
                                unsigned char* valid, cudaStream_t st) {
    FeatArgs a;
    for (int e = 0; e < k; ++e) a.b[e] = bricks[e];
    a.cam = cam;
    double d2 = 0.0;
    for (int q = 0; q < 3; ++q) {
        a.dims[q] = dims[q];
        d2 += (double)(dims[q] - 1) * (dims[q] - 1);
    }
    a.inv_diag = (float)(1.0 / sqrt(d2));
    a.lut = lut;
    a.scale255 = scale255;
    a.step = step;
    a.ref_len = ref_len;
    a.k = k;
    a.n_s = n_s;
    a.tiles_x = (cam.W + kFT - 1) / kFT;
    a.tiles_y = (cam.H + kFT - 1) / kFT;
    a.feats = feats;
    a.valid = valid;
    dim3 grid((unsigned)(a.tiles_x * a.tiles_y), (unsigned)k);
    tile_features_kernel<<<grid, 64, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "tile_features_kernel launch");
}

vdi_status launch_tile_labels(const vdi_compact* searched, int k, int w, int h, float* labels, unsigned char* valid,
                              cudaStream_t st) {
    LabelArgs a;
    for (int e = 0; e < k; ++e) {
        a.counts[e] = searched[e].counts;
        a.gamma[e] = searched[e].gamma;
    }
    a.W = w;
    a.H = h;
    a.tiles_x = (w + kFT - 1) / kFT;
    a.tiles_y = (h + kFT - 1) / kFT;
    a.labels = labels;
    a.valid = valid;
    dim3 grid((unsigned)(a.tiles_x * a.tiles_y), (unsigned)k);
    tile_labels_kernel<<<grid, 256, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "tile_labels_kernel launch");
}

vdi_status launch_mlp_infer(const void* model, const float* feats, int n, float offset, float* out,
                            cudaStream_t st) {
    if (n <= 0) return VDI_OK;
    int blocks = (n + 63) / 64;  // 4 warps x 16 rows
    if (blocks > 2048) blocks = 2048;
    mlp_infer_kernel<<<blocks, 128, 0, st>>>(static_cast<const unsigned char*>(model), feats, n, offset, out);
    return cuda_check(cudaGetLastError(), "mlp_infer_kernel launch");
}

vdi_status launch_gamma_expand(float* const* gammas, int k, int w, int h, const float* pred, cudaStream_t st) {
    ExpandArgs a;
    for (int e = 0; e < k; ++e) a.gamma[e] = gammas[e];
    a.pred = pred;
    a.W = w;
    a.H = h;
    a.tiles_x = (w + kFT - 1) / kFT;
    a.tiles = a.tiles_x * ((h + kFT - 1) / kFT);
    size_t npix = (size_t)w * h;
    unsigned blocks = (unsigned)((npix + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks == 0) return VDI_OK;
    gamma_expand_kernel<<<dim3(blocks, (unsigned)k), 256, 0, st>>>(a);
    return cuda_check(cudaGetLastError(), "gamma_expand_kernel launch");
}

size_t train_workspace(int n) {
    size_t blocks = ((size_t)n + kTrainRows - 1) / kTrainRows;
    return 256 + align_up(blocks * (kNP + 1) * sizeof(float), 256) + align_up((kNP + 1) * sizeof(float), 256);
}

static size_t fwdbwd_smem() { return (size_t)(kNP + kTrainRows * kNF + 4 * kTrainRows * kNH + 2 * kTrainRows) * 4; }

// gradient (and loss) of the mean squared error into grad[kNP], loss (device)
vdi_status launch_mlp_grad(const void* model, const float* x, const float* y, const unsigned char* valid, int n,
                           float* grad, float* loss, void* ws, cudaStream_t st) {
    const int blocks = (n + kTrainRows - 1) / kTrainRows;
    float* mcount = reinterpret_cast<float*>(ws);
    float* partial = reinterpret_cast<float*>(static_cast<char*>(ws) + 256);
    count_valid_kernel<<<1, 256, 0, st>>>(valid, n, mcount);
    vdi_status s = cuda_check(cudaGetLastError(), "count_valid_kernel launch");
    if (s != VDI_OK || blocks == 0) return s;
    const size_t smem = fwdbwd_smem();
    s = cuda_check(cudaFuncSetAttribute(mlp_fwdbwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                   "smem attribute");
    if (s != VDI_OK) return s;
    mlp_fwdbwd_kernel<<<blocks, 256, smem, st>>>(static_cast<const unsigned char*>(model), x, y, valid, n, mcount,
                                                 partial);
    s = cuda_check(cudaGetLastError(), "mlp_fwdbwd_kernel launch");
    if (s != VDI_OK) return s;
    mlp_reduce_kernel<<<(kNP + 1 + 255) / 256, 256, 0, st>>>(partial, blocks, grad, loss);
    return cuda_check(cudaGetLastError(), "mlp_reduce_kernel launch");
}

vdi_status launch_train_step(void* model, const float* x, const float* y, const unsigned char* valid, int n, float lr,
                             float* loss, void* ws, cudaStream_t st) {
    const int blocks = (n + kTrainRows - 1) / kTrainRows;
    float* grad = reinterpret_cast<float*>(static_cast<char*>(ws) + 256 +
                                           align_up((size_t)blocks * (kNP + 1) * sizeof(float), 256));
    vdi_status s = launch_mlp_grad(model, x, y, valid, n, grad, loss, ws, st);
    if (s != VDI_OK) return s;
    adam_kernel<<<(kNP + 255) / 256, 256, 0, st>>>(static_cast<unsigned char*>(model), grad, lr, 0.9f, 0.999f, 1e-8f);
    s = cuda_check(cudaGetLastError(), "adam_kernel launch");
    if (s != VDI_OK) return s;
    step_increment_kernel<<<1, 1, 0, st>>>(static_cast<unsigned char*>(model));
    return cuda_check(cudaGetLastError(), "step_increment_kernel launch");
}

// checkpoint: "VDIMLP01", format version, parameter count, byte size, then the model buffer
struct CkptHeader {
    char magic[8];
    uint32_t version, nparams;
    uint64_t bytes;
};

vdi_status model_save(const void* model, const char* path, cudaStream_t st) {
    unsigned char* host = (unsigned char*)malloc(kModelBytes);
    if (!host) return set_error(VDI_ERR_MODEL, "vdi_model_save: host buffer");
    vdi_status s = cuda_check(cudaMemcpyAsync(host, model, kModelBytes, cudaMemcpyDeviceToHost, st), "model read");
    if (s == VDI_OK) s = cuda_check(cudaStreamSynchronize(st), "model read sync");
    if (s == VDI_OK) {
        FILE* f = fopen(path, "wb");
        if (!f) {
            s = set_error(VDI_ERR_MODEL, "vdi_model_save: cannot open %s", path);
        } else {
            CkptHeader h;
            memcpy(h.magic, "VDIMLP01", 8);
            h.version = 1;
            h.nparams = kNP;
            h.bytes = kModelBytes;
            if (fwrite(&h, sizeof h, 1, f) != 1 || fwrite(host, 1, kModelBytes, f) != kModelBytes)
                s = set_error(VDI_ERR_MODEL, "vdi_model_save: write failed");
            if (fclose(f) != 0 && s == VDI_OK) s = set_error(VDI_ERR_MODEL, "vdi_model_save: close failed");
        }
    }
    free(host);
    return s;
}

vdi_status model_load(void* model, const char* path, cudaStream_t st) {
    FILE* f = fopen(path, "rb");
    if (!f) return set_error(VDI_ERR_MODEL, "vdi_model_load: cannot open %s", path);
    CkptHeader h;
    vdi_status s = VDI_OK;
    unsigned char* host = nullptr;
    if (fread(&h, sizeof h, 1, f) != 1 || memcmp(h.magic, "VDIMLP01", 8) != 0 || h.version != 1 ||
        h.nparams != (uint32_t)kNP || h.bytes != kModelBytes) {
        s = set_error(VDI_ERR_MODEL, "vdi_model_load: %s is not a version-1 model checkpoint", path);
    } else {
        host = (unsigned char*)malloc(kModelBytes);
        if (!host || fread(host, 1, kModelBytes, f) != kModelBytes)
            s = set_error(VDI_ERR_MODEL, "vdi_model_load: truncated %s", path);
    }
    fclose(f);
    if (s == VDI_OK) s = cuda_check(cudaMemcpyAsync(model, host, kModelBytes, cudaMemcpyHostToDevice, st), "model write");
    if (s == VDI_OK) s = cuda_check(cudaStreamSynchronize(st), "model write sync");
    free(host);
    return s;
}

}  // namespace vdi
