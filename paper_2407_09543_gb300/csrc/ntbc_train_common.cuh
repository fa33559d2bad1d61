// Device helpers shared by the training kernels (the FP32 layer-by-layer path and the
// fused BF16 tensor-core path): sample coordinates, palettes and the straight-through
// argmax of the losses (Sec. 3.2, App. A), the QAT straight-through mask (Sec. 3.3) and
// the bilinear adjoint with warp-aggregated atomics.
#pragma once

#include "ntbc_internal.cuh"
#include "ntbc_kernels.cuh"

namespace ntbc {

constexpr float kNormGuard = 1e-6f;

// sample k of the colour network is texel (k & 15) of block ids[k >> 4];
// sample k of the endpoint network is block ids[k]
__device__ __forceinline__ void sample_coords(const ModelView& mv, bool color, const int32_t* ids, int k, float& u,
                                              float& v, int& x, int& y) {
    if (color) {
        int b = ids[k >> 4], i = k & 15;
        x = 4 * (b % mv.bw) + (i & 3);
        y = 4 * (b / mv.bw) + (i >> 2);
        u = ((float)x + 0.5f) / (float)mv.width;
        v = ((float)y + 0.5f) / (float)mv.height;
    } else {
        int b = ids[k];
        x = b % mv.bw;
        y = b / mv.bw;
        u = ((float)x + 0.5f) / (float)mv.bw;
        v = ((float)y + 0.5f) / (float)mv.bh;
    }
}

// linear-order float palette P_n = a_n e0 + b_n e1 + const_n (Eq. palette / Eq. weightBC4)
__device__ __forceinline__ int palette_coeffs(int fmt, bool eight, float a[8], float b[8], float c[8]) {
    if (fmt == NTBC_BC1) {
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            float w = (float)n / 3.f;
            a[n] = 1.f - w;
            b[n] = w;
            c[n] = 0.f;
        }
        return 4;
    }
    if (eight) {
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            float w = (float)n / 7.f;
            a[n] = 1.f - w;
            b[n] = w;
            c[n] = 0.f;
        }
    } else {
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            bool interp = n >= 1 && n <= 6;
            float w = interp ? (float)(n - 1) / 5.f : 0.f;
            a[n] = interp ? 1.f - w : 0.f;
            b[n] = interp ? w : 0.f;
            c[n] = n == 7 ? 1.f : 0.f;
        }
    }
    return 8;
}

// decoded reference endpoints in [0, 1] (stored order) of block b of texture t
__device__ __forceinline__ void ref_endpoints(int fmt, const uint8_t* blocks, int b, float e0[3], float e1[3]) {
    uint32_t lo = *reinterpret_cast<const uint32_t*>(blocks + (long long)b * 8);
    if (fmt == NTBC_BC1) {
        int r, g, bb;
        expand565(lo & 0xFFFF, r, g, bb);
        e0[0] = r / 255.f; e0[1] = g / 255.f; e0[2] = bb / 255.f;
        expand565(lo >> 16, r, g, bb);
        e1[0] = r / 255.f; e1[1] = g / 255.f; e1[2] = bb / 255.f;
    } else {
        e0[0] = (float)(lo & 0xFF) / 255.f;
        e1[0] = (float)((lo >> 8) & 0xFF) / 255.f;
    }
}

__device__ __forceinline__ float texel_value(const uint8_t* tex, int fmt, int w, int x, int y, int ch) {
    int C = fmt == NTBC_BC1 ? 3 : 1;
    return (float)tex[((long long)y * w + x) * C + ch] / 255.f;
}

struct TexPtrs {
    const uint8_t* texels[NTBC_MAX_TEXTURES];
    const uint8_t* blocks[NTBC_MAX_TEXTURES];
};

__device__ __forceinline__ void block_reduce_add(double* acc, float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, (double)v);
}

// Softmax-expectation backward of the hard decode dec = P_{argmax d}:
// g_d[n] = (1/T) sigma_n sum_c g_dec[c] (P[n][c] - sum_i sigma_i P[i][c])
__device__ __forceinline__ void ste_grad(int K, int C, const float d[8], const float P[8][3], const float g_dec[3],
                                         float T, float g_d[8]) {
    float m = d[0];
    for (int n = 1; n < K; ++n) m = fmaxf(m, d[n]);
    float sig[8], sum = 0.f;
    for (int n = 0; n < K; ++n) {
        sig[n] = expf((d[n] - m) / T);
        sum += sig[n];
    }
    float pbar[3] = {0.f, 0.f, 0.f};
    for (int n = 0; n < K; ++n) {
        sig[n] /= sum;
        for (int c = 0; c < C; ++c) pbar[c] += sig[n] * P[n][c];
    }
    for (int n = 0; n < K; ++n) {
        float s = 0.f;
        for (int c = 0; c < C; ++c) s += g_dec[c] * (P[n][c] - pbar[c]);
        g_d[n] = sig[n] * s / T;
    }
}

// Fire-and-forget vector reduction into global memory (8-byte aligned address): no value
// comes back, so the thread does not wait for the L2 round trip.
__device__ __forceinline__ void red_add_f32x2(float* addr, float2 v) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// Bilinear adjoint: d loss / d features back to the 4 corners of every level.
// Colour network: the 16 texels of a block sit in one half-warp and their corner
// indices are non-decreasing in x (lane & 3) and in y (lane >> 2), so equal corners form
// contiguous runs; a segmented scan along x, then along y, leaves each distinct corner's
// total in the last lane of its run, which issues the only atomic for that corner.
// The keys of those runs (the neighbours' corner indices) are recomputed from the
// neighbours' coordinates, shuffled once per sample (`Neighbours`), with the same arithmetic
// the neighbour uses, so only the gradient values travel through shuffles per level.
struct Neighbours {
    float u_m1, u_m2, u_p1;      // u of the texels 1 and 2 to the left and 1 to the right
    float v_m1, v_m2, v_p1;      // v of the texels 1 and 2 rows up and 1 row down
};

__device__ __forceinline__ Neighbours neighbours(float u, float v) {
    Neighbours n;
    n.u_m1 = __shfl_up_sync(0xffffffffu, u, 1);
    n.u_m2 = __shfl_up_sync(0xffffffffu, u, 2);
    n.u_p1 = __shfl_down_sync(0xffffffffu, u, 1);
    n.v_m1 = __shfl_up_sync(0xffffffffu, v, 4);
    n.v_m2 = __shfl_up_sync(0xffffffffu, v, 8);
    n.v_p1 = __shfl_down_sync(0xffffffffu, v, 4);
    return n;
}

__device__ __forceinline__ int cell_of(float t, int res) { return min((int)floorf(t * (float)(res - 1)), res - 2); }

// One level l: (g0, g1) = d loss / d features of the sample at this level. All 32 lanes of
// the warp must call it together.
__device__ __forceinline__ void scatter_level(const NetView& nv, bool color, int l, float u, float v, int lane_k,
                                              bool valid, float g0, float g1, const GridSrc& src, int qat_bits,
                                              float* __restrict__ ggrad, const Neighbours& nb = Neighbours()) {
    const int lx = lane_k & 3, ly = (lane_k >> 2) & 3;
    int res = nv.res[l];
    float px = u * (float)(res - 1), py = v * (float)(res - 1);
    int ix = min((int)floorf(px), res - 2), iy = min((int)floorf(py), res - 2);
    int kx_m1 = 0, kx_m2 = 0, kx_p1 = 0, ky_m1 = 0, ky_m2 = 0, ky_p1 = 0;
    if (color) {
        kx_m1 = cell_of(nb.u_m1, res);
        kx_m2 = cell_of(nb.u_m2, res);
        kx_p1 = cell_of(nb.u_p1, res);
        ky_m1 = cell_of(nb.v_m1, res);
        ky_m2 = cell_of(nb.v_m2, res);
        ky_p1 = cell_of(nb.v_p1, res);
    }
    float fx = px - (float)ix, fy = py - (float)iy;
    if (!valid) g0 = g1 = 0.f;
    float w[4] = {(1.f - fx) * (1.f - fy), fx * (1.f - fy), (1.f - fx) * fy, fx * fy};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int cx = ix + (j & 1), cy = iy + (j >> 1);
        long long corner = nv.grid_off[l] + ((long long)cy * res + cx) * 2;
        // QAT (Sec. 3.3): the straight-through factor is 1 where the quantiser does not clamp.
        // alpha and beta are this level's own min and max, recomputed every step, so no grid
        // value is ever clamped and the factor is 1 throughout; testing the clamp in FP32 instead
        // could mark a level's maximum as clamped (round(beta / s) + z rounding to 2^b).
        float2 add = make_float2(w[j] * g0, w[j] * g1);
        bool issue = valid;
        if (color) {
            const int dx = j & 1, dy = j >> 1;
#pragma unroll
            for (int dd = 1; dd <= 2; dd <<= 1) {          // runs along x
                float px0 = __shfl_up_sync(0xffffffffu, add.x, dd), px1 = __shfl_up_sync(0xffffffffu, add.y, dd);
                int pk = (dd == 1 ? kx_m1 : kx_m2) + dx;
                if (lx >= dd && pk == cx) {
                    add.x += px0;
                    add.y += px1;
                }
            }
            bool last_x = lx == 3 || kx_p1 + dx != cx;
            if (!last_x) add = make_float2(0.f, 0.f);
#pragma unroll
            for (int dd = 4; dd <= 8; dd <<= 1) {          // runs along y
                float py0 = __shfl_up_sync(0xffffffffu, add.x, dd), py1 = __shfl_up_sync(0xffffffffu, add.y, dd);
                int pk = (dd == 4 ? ky_m1 : ky_m2) + dy;
                if (ly >= dd / 4 && pk == cy) {
                    add.x += py0;
                    add.y += py1;
                }
            }
            bool last_y = ly == 3 || ky_p1 + dy != cy;
            issue = valid && last_x && last_y;
        }
        if (issue) red_add_f32x2(ggrad + corner, add);
    }
}

// All levels of one sample. kc: the sample (for its coordinates); lane_k: any index whose
// low 4 bits are the texel's position in its block's half-warp (colour); g: d loss /
// d features of this sample, level-major, 2 per level (registers: the loop is unrolled).
__device__ __forceinline__ void scatter_sample(const ModelView& mv, bool color, const int32_t* __restrict__ ids, int kc,
                                               int lane_k, bool valid, const float* g, const GridSrc& src,
                                               float* __restrict__ ggrad) {
    const NetView& nv = color ? mv.color : mv.endpoint;
    float u, v;
    int x, y;
    sample_coords(mv, color, ids, kc, u, v, x, y);
    const int qat_bits = src.qat_bits;
    const Neighbours nb = color ? neighbours(u, v) : Neighbours();
#pragma unroll
    for (int l = 0; l < NTBC_MAX_LEVELS; ++l) {              // unrolled: g stays in registers
        if (l >= nv.levels) break;
        scatter_level(nv, color, l, u, v, lane_k, valid, g[2 * l], g[2 * l + 1], src, qat_bits, ggrad, nb);
    }
}

}  // namespace ntbc
