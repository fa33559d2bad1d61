// Fused tensor-core training pass of one network (BF16 operands, FP32 accumulation in
// TMEM): the grid gather with QAT fake quantisation (Sec. 3.3), the MLP forward, the loss
// with the straight-through argmax (Sec. 3.2, App. A), the backward through every layer
// and the grid scatter-add, for tiles of 128 samples, with every intermediate kept on chip.
//
// A persistent CTA per SM runs one or two independent warpgroups. A warpgroup takes a tile
// of 128 samples (texels of 8 sampled blocks, or 128 sampled blocks for the endpoint
// network); row r of every tile is thread r's sample. Shared memory holds, per group, the
// input features X [128][K0], the hidden activations A_l [128][80] (64 units + the bias
// column, constant 1) and one delta tile D, all BF16 in the canonical no-swizzle core-matrix
// layout, plus the CTA's copy of the BF16 weight image (each layer's [N][K] tile).
//
// MMAs (M = 128; one elected thread issues, the group waits on its mbarrier):
//   forward      Z_l = A_{l-1} W_l^T      A K-major (rows = samples), B = the W_l tile
//   data grad    dA_{l-1} = D_l W_l       A = D (K-major), B = the same W_l tile read
//                                         MN-major (N = inputs along the tile's columns)
//   weight grad  dW_l^T += A_{l-1}^T D_l  both operands MN-major: K = the 128 samples;
//                                         M = the 80 input columns (rows 80..127 of the
//                                         accumulator are never read), N = the outputs
//   layer 0      dW_0 += D_0^T X          M = the 64 units (rows 64..127 unused), N = K0
// The weight-gradient accumulators stay in TMEM across all tiles of the group and are
// added to the global gradient once, at the end.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "ntbc_internal.cuh"
#include "ntbc_kernels.cuh"
#include "ntbc_train_common.cuh"
#include "ntbc_train_tc.cuh"
#include "tcgen05.cuh"

namespace ntbc {

constexpr int kTrRows = 128;
constexpr int kTrHidCols = 80;            // 64 hidden units + the bias K block (column 64 = 1)
constexpr int kTrMaxGroups = 2;
constexpr int kTrPad = 1024;              // bytes after a group's tiles: MN-major reads of the
                                          // unused accumulator rows run past the last tile

// byte offset of the core-matrix chunk (8 columns starting at 8 * kg) of row r, tile of C columns
__host__ __device__ __forceinline__ int chunk_byte(int r, int kg, int C) {
    return (((r >> 3) * (C >> 3) + kg) * 64 + (r & 7) * 8) * 2;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void st_chunk_bf16(unsigned char* tile, int r, int kg, int C, const float* v) {
    uint4 u = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                         pack_bf16x2(v[6], v[7]));
    *reinterpret_cast<uint4*>(tile + chunk_byte(r, kg, C)) = u;
}

// the BF16 pair nearest to what the BF16 pair `hi` leaves of (a, b): hi + lo carries about 16
// significant bits of each value (the differences are exact in FP32)
__device__ __forceinline__ uint32_t pack_bf16x2_lo(float a, float b, uint32_t hi) {
    const float2 h = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&hi));
    return pack_bf16x2(a - h.x, b - h.y);
}

// one chunk as a hi tile of C columns and a lo tile of Clo columns (the endpoint network's
// split forward operands)
__device__ __forceinline__ void st_chunk_bf16_split(unsigned char* hi_tile, int C, unsigned char* lo_tile, int Clo, int r,
                                                    int kg, const float* v) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        h[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
        l[j] = pack_bf16x2_lo(v[2 * j], v[2 * j + 1], h[j]);
    }
    *reinterpret_cast<uint4*>(hi_tile + chunk_byte(r, kg, C)) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo_tile + chunk_byte(r, kg, Clo)) = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void ld_chunk_bf16(const unsigned char* tile, int r, int kg, int C, float* v) {
    uint4 u = *reinterpret_cast<const uint4*>(tile + chunk_byte(r, kg, C));
    uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w[j]);
        float2 f = __bfloat1622float2(h);
        v[2 * j] = f.x;
        v[2 * j + 1] = f.y;
    }
}

__device__ __forceinline__ float tmem_ld1f(uint32_t taddr) {
    uint32_t v;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(taddr));
    return __uint_as_float(v);
}

struct TrGroup {
    unsigned char* X;
    unsigned char* X2;        // colour: the other input tile (tiles alternate between X and X2)
    unsigned char* A[3];
    unsigned char* D;
    uint64_t* bar;
    uint32_t tmem, row;       // group's TMEM base column; this thread's lane address
    int g, r;
};

// Colour pass: each tile warpgroup g has a helper warpgroup that gathers the group's next tile
// into the other input tile (X / X2 alternate) and scatters the grid gradients of the group's
// current tile (read from the group's delta tile, where the backward leaves them), so the group
// itself runs only the forward, the loss and the backward. Named barriers over the pair's 256
// threads hand the tiles over: XFULL (an input tile is gathered: the helper arrives, the group
// waits), FULL (the tile's gradients are ready and its input tile is free: the group arrives,
// the helper waits) and EMPTY (the helper has read its row of gradients into registers: it
// arrives, then scatters; the group waits before its next loss writes the delta tile). Both
// walk the same tile sequence and every arrival is matched by a wait, on the abort path too
// (the group passes a stop flag and consumes the input tile gathered ahead).
__device__ __forceinline__ int pair_full_id(int g) { return 4 + g; }
__device__ __forceinline__ int pair_empty_id(int g) { return 6 + g; }
__device__ __forceinline__ int pair_xfull_id(int g) { return 8 + g; }
// bar.arrive releases the arriving thread's prior shared-memory writes to the threads that
// complete the barrier with bar.sync; it takes no fence (a fence would also wait for the
// helper's global gradient reductions still in flight)
__device__ __forceinline__ void pair_arrive(int id) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(2 * kTrRows) : "memory");
}
__device__ __forceinline__ void pair_sync(int id) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(2 * kTrRows) : "memory"); }

__device__ __forceinline__ bool tr_barrier(int g, volatile int* abort_flag) {
    proxy_fence();
    tc_fence_before();
    group_sync(g);
    return abort_flag[g] == 0;
}

// the endpoint kernel's forward and backward run on all 16 warps (one tile per CTA): a CTA
// barrier instead of the warpgroup's
__device__ __forceinline__ bool tr_cta_barrier(volatile int* abort_flag) {
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    return abort_flag[0] == 0;
}

__device__ __forceinline__ void tr_wait(const TrGroup& G, uint32_t& phase, volatile int* abort_flag) {
    if (!mbar_wait(G.bar, phase)) abort_flag[G.g] = 1;
    phase ^= 1;
    tc_fence_after();
}

// ---------------------------------------------------------------------------
// fast arithmetic (MUFU); every result feeds a BF16 operand or a loss gradient whose
// comparison bar is far above these errors (relative ~2^-22)
// ---------------------------------------------------------------------------

constexpr float kL2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_fast(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_fast(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// ||x - P_n|| and its guarded inverse 1 / max(||x - P_n||, 1e-6) from the squared distance
// with one reciprocal square root: r = 1 / sqrt(max(sq, 1e-12)), norm = sq r (below the
// guard the norm itself is < 1e-6 and only enters the softmax, where 1e-6 / T is negligible)
__device__ __forceinline__ float norm_and_inverse(float sq, float& inv) {
    inv = rsqrt_fast(fmaxf(sq, kNormGuard * kNormGuard));
    return sq * inv;
}
// the hidden activation on a pair with packed FP32 (two lanes per instruction): SELU as
// lambda (z - m) + lambda alpha (2^(m log2 e) - 1) with m = min(z, 0), which is lambda z for z > 0
// (the exponential term is exactly 0) and lambda alpha (e^z - 1) for z <= 0 (z - m is exactly 0)
__device__ __forceinline__ float2 act_fast2(float2 z, int act) {
    if (act != NTBC_ACT_SELU) return make_float2(fmaxf(z.x, 0.f), fmaxf(z.y, 0.f));
    const float2 m = make_float2(fminf(z.x, 0.f), fminf(z.y, 0.f));
    const float2 ml = __fmul2_rn(m, make_float2(kL2e, kL2e));
    const float2 e = make_float2(ex2_fast(ml.x), ex2_fast(ml.y));
    const float2 t = __ffma2_rn(make_float2(kSeluLA, kSeluLA), e, make_float2(-kSeluLA, -kSeluLA));
    return __ffma2_rn(make_float2(kSeluLambda, kSeluLambda), __ffma2_rn(m, make_float2(-1.f, -1.f), z), t);
}
__device__ __forceinline__ float sigmoid_fast(float z) { return rcp_fast(1.f + ex2_fast(-z * kL2e)); }

// ---------------------------------------------------------------------------
// losses: every palette / softmax loop runs over a compile-time entry count (4 for BC1,
// C = 3; 8 for BC4, C = 1) and channel count, so nothing leaves the registers
// ---------------------------------------------------------------------------

// Softmax-expectation backward of the hard decode (App. A, corrected form):
// g_d[n] = (1/T) sigma_n sum_c g_dec[c] (P[n][c] - sum_i sigma_i P[i][c]), sigma = softmax(d / T),
// evaluated as (1/T) sigma_n (v_n - sum_i sigma_i v_i) with v_n = sum_c g_dec[c] P[n][c].
// Returned already divided by the guarded distance: s_n = g_d[n] inv[n], since every caller
// goes on through d d_n / d P_n = (x - P_n) / max(||x - P_n||, 1e-6).
template <int C>
__device__ __forceinline__ void ste_fast(int K, const float d[8], const float P[8][C], const float g_dec[C], float invT,
                                         const float inv[8], float s[8]) {
    constexpr int KM = C == 3 ? 4 : 8;
    float m = d[0];
#pragma unroll
    for (int n = 1; n < KM; ++n)
        if (n < K) m = fmaxf(m, d[n]);
    const float k = invT * kL2e, mk = m * k;
    float e[8], v[8], sum = 0.f, vbar = 0.f;
#pragma unroll
    for (int n = 0; n < KM; ++n) {
        e[n] = n < K ? ex2_fast(fmaf(d[n], k, -mk)) : 0.f;
        sum += e[n];
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < C; ++q) t = fmaf(g_dec[q], P[n][q], t);
        v[n] = t;
        vbar = fmaf(e[n], t, vbar);
    }
    const float r = rcp_fast(sum);
    vbar *= r;
    const float c = r * invT;
#pragma unroll
    for (int n = 0; n < KM; ++n) s[n] = e[n] * c * (v[n] - vbar) * inv[n];
}

// linear palette P_n = a_n e0 + b_n e1 + c_n (Eq. palette / Eq. weightBC4), distances
// d_n = -||x - P_n|| (n < K) and their inverse norms, and the argmax (ties: lowest n)
template <int C>
__device__ __forceinline__ int palette_distances(int fmt, const float* e0, const float* e1, const float* x, float P[8][C],
                                                 float a8[8], float b8[8], float d[8], float inv[8], int& best) {
    float c8[8];
#pragma unroll
    for (int n = 0; n < (C == 3 ? 4 : 8); ++n) a8[n] = b8[n] = c8[n] = 0.f;       // BC1 fills only n < 4
    int K = palette_coeffs(fmt, e0[0] > e1[0], a8, b8, c8);
    float bestsq = 3.0e38f;
    best = 0;
#pragma unroll
    for (int n = 0; n < (C == 3 ? 4 : 8); ++n) {
        float sq = 0.f;
#pragma unroll
        for (int q = 0; q < C; ++q) {
            P[n][q] = fmaf(a8[n], e0[q], fmaf(b8[n], e1[q], c8[n]));
            float df = x[q] - P[n][q];
            sq = fmaf(df, df, sq);
        }
        float nrm = norm_and_inverse(sq, inv[n]);
        d[n] = n < K ? -nrm : -3.0e38f;
        if (n < K && sq < bestsq) {           // argmax of -||.|| = argmin of the squared distance
            bestsq = sq;
            best = n;
        }
    }
    return K;
}

template <int C>
__device__ __forceinline__ void pick(const float P[8][C], int best, float* out) {
#pragma unroll
    for (int q = 0; q < C; ++q) out[q] = P[0][q];
#pragma unroll
    for (int n = 1; n < (C == 3 ? 4 : 8); ++n)
        if (n == best)
#pragma unroll
            for (int q = 0; q < C; ++q) out[q] = P[n][q];
}

// colour network, one texture of a texel sample: L_c + L_cd with distances from c_hat to
// the reference palette; dz = d loss / d z_out (through the sigmoid)
template <int C>
__device__ __forceinline__ void color_texture(int fmt, const float* ch, const float* c, const float* e0, const float* e1,
                                              float invT, float inv_n, bool valid, float* dz, float& lc, float& lcd) {
    float P[8][C], a8[8], b8[8], d[8], inv[8];
    int best;
    int K = palette_distances<C>(fmt, e0, e1, ch, P, a8, b8, d, inv, best);
    float pb[C], g_dec[C], g[C];
    pick<C>(P, best, pb);
#pragma unroll
    for (int q = 0; q < C; ++q) {
        float rr = c[q] - pb[q], e = ch[q] - c[q];
        if (valid) {
            lcd = fmaf(rr, rr, lcd);
            lc = fmaf(e, e, lc);
        }
        g_dec[q] = -2.f * rr * inv_n;
        g[q] = 2.f * e * inv_n;
    }
    float sd[8];
    ste_fast<C>(K, d, P, g_dec, invT, inv, sd);
#pragma unroll
    for (int n = 0; n < (C == 3 ? 4 : 8); ++n)
#pragma unroll
        for (int q = 0; q < C; ++q) g[q] = fmaf(-sd[n], ch[q] - P[n][q], g[q]);
#pragma unroll
    for (int q = 0; q < C; ++q) dz[q] = valid ? g[q] * ch[q] * (1.f - ch[q]) : 0.f;
}

__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// start the global reads of every texture a loss row needs (the reference block's endpoints
// and the texel) before the per-texture arithmetic, so they overlap instead of chaining
__device__ __forceinline__ void prefetch_row(const TrArgs& a, int b, int x, int y) {
    const ModelView& mv = a.mv;
    for (int t = 0; t < mv.n_textures; ++t) {
        prefetch_l1(a.tp.blocks[t] + (long long)b * 8);
        prefetch_l1(a.tp.texels[t] + ((long long)y * mv.width + x) * (mv.formats[t] == NTBC_BC1 ? 3 : 1));
    }
}

__device__ __forceinline__ void st_bf16(unsigned char* tile, int r, int col, int C, float v) {
    *reinterpret_cast<__nv_bfloat16*>(tile + chunk_byte(r, col >> 3, C) + (col & 7) * 2) = __float2bfloat16_rn(v);
}

// colour loss of texel sample s (row r): writes the output deltas of every texture
__device__ __forceinline__ void color_loss_row(const TrArgs& a, int s, bool valid, uint32_t zrow, unsigned char* D,
                                               int r, float& lc, float& lcd) {
    const ModelView& mv = a.mv;
    int b = a.ids[s >> 4], i = s & 15;
    int x = 4 * (b % mv.bw) + (i & 3), y = 4 * (b / mv.bw) + (i >> 2);
    const float inv_n = 1.f / ((float)a.B * (float)a.net.out_dim), invT = 1.f / a.T;
    prefetch_row(a, b, x, y);
    for (int t = 0; t < mv.n_textures; ++t) {
        const int fmt = mv.formats[t], co = mv.coff[t];
        float e0[3], e1[3];
        ref_endpoints(fmt, a.tp.blocks[t], b, e0, e1);
        if (fmt == NTBC_BC1) {
            float ch[3], c[3], dz[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) ch[q] = tmem_ld1f(zrow + co + q);
            tmem_wait_ld_regs<3>(ch);
            const uint8_t* tp = a.tp.texels[t] + ((long long)y * mv.width + x) * 3;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                ch[q] = sigmoid_fast(ch[q]);
                c[q] = (float)tp[q] * (1.f / 255.f);
            }
            color_texture<3>(fmt, ch, c, e0, e1, invT, inv_n, valid, dz, lc, lcd);
#pragma unroll
            for (int q = 0; q < 3; ++q) st_bf16(D, r, co + q, a.net.out_pad, dz[q]);
        } else {
            float ch[1], c[1], dz[1];
            ch[0] = tmem_ld1f(zrow + co);
            tmem_wait_ld_regs<1>(ch);
            ch[0] = sigmoid_fast(ch[0]);
            c[0] = (float)a.tp.texels[t][(long long)y * mv.width + x] * (1.f / 255.f);
            color_texture<1>(fmt, ch, c, e0, e1, invT, inv_n, valid, dz, lc, lcd);
            st_bf16(D, r, co, a.net.out_pad, dz[0]);
        }
    }
}

// endpoint network, one (block, texture) item: the L_cd terms of the block's 16 texels,
// with distances to the palette of the predicted endpoints (eh0, eh1) and the decode from
// the reference palette (both palettes built once per item); the item's gradient
// d loss / d (eh0, eh1), summed over the texels, goes to grow.
template <int C>
__device__ __forceinline__ void endpoint_item(const TrArgs& a, int fmt, int b, int eo, const float* yrow,
                                              const uint8_t* blocks, const uint8_t* tex, bool valid, float* grow,
                                              float& lcd) {
    constexpr int KM = C == 3 ? 4 : 8;
    const ModelView& mv = a.mv;
    const float inv_ncd = 1.f / ((float)a.B * 16.f * (float)mv.color.out_dim), invT = 1.f / a.T;
    const int bx = b % mv.bw, by = b / mv.bw;
    const uint8_t* row0 = tex + ((long long)(4 * by) * mv.width + 4 * bx) * C;
#pragma unroll
    for (int yy = 0; yy < 4; ++yy) {
        prefetch_l1(row0 + (long long)yy * mv.width * C);
        prefetch_l1(row0 + (long long)yy * mv.width * C + 4 * C - 1);
    }
    float eh0[3] = {0.f, 0.f, 0.f}, eh1[3] = {0.f, 0.f, 0.f}, e0[3], e1[3];
#pragma unroll
    for (int q = 0; q < C; ++q) {
        eh0[q] = yrow[eo + q];
        eh1[q] = yrow[eo + C + q];
    }
    ref_endpoints(fmt, blocks, b, e0, e1);
    float ah[8], bh[8], chh[8], ar[8], br[8], cr[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) ah[n] = bh[n] = chh[n] = ar[n] = br[n] = cr[n] = 0.f;
    const int K = palette_coeffs(fmt, eh0[0] > eh1[0], ah, bh, chh);
    palette_coeffs(fmt, e0[0] > e1[0], ar, br, cr);
    float Ph[8][C], Pr[8][C];
#pragma unroll
    for (int n = 0; n < KM; ++n)
#pragma unroll
        for (int q = 0; q < C; ++q) {
            Ph[n][q] = fmaf(ah[n], eh0[q], fmaf(bh[n], eh1[q], chh[n]));
            Pr[n][q] = fmaf(ar[n], e0[q], fmaf(br[n], e1[q], cr[n]));
        }
    float g0[C], g1[C];
#pragma unroll
    for (int q = 0; q < C; ++q) g0[q] = g1[q] = 0.f;
#pragma unroll 2
    for (int i = 0; i < 16; ++i) {
        const uint8_t* tp = row0 + ((long long)(i >> 2) * mv.width + (i & 3)) * C;
        float c[C];
#pragma unroll
        for (int q = 0; q < C; ++q) c[q] = (float)tp[q] * (1.f / 255.f);
        float d[8], inv[8];
        float bestsq = 3.0e38f;
        int best = 0;
#pragma unroll
        for (int n = 0; n < KM; ++n) {
            float sq = 0.f;
#pragma unroll
            for (int q = 0; q < C; ++q) {
                float df = c[q] - Ph[n][q];
                sq = fmaf(df, df, sq);
            }
            d[n] = -norm_and_inverse(sq, inv[n]);
            if (sq < bestsq) {                // argmax of -||.|| = argmin of the squared distance
                bestsq = sq;
                best = n;
            }
        }
        float pb[C], g_dec[C];
        pick<C>(Pr, best, pb);
#pragma unroll
        for (int q = 0; q < C; ++q) {
            float rr = c[q] - pb[q];
            if (valid) lcd = fmaf(rr, rr, lcd);
            g_dec[q] = valid ? -2.f * rr * inv_ncd : 0.f;
        }
        float sd[8];
        ste_fast<C>(K, d, Pr, g_dec, invT, inv, sd);
#pragma unroll
        for (int n = 0; n < KM; ++n)
#pragma unroll
            for (int q = 0; q < C; ++q) {
                float gp = sd[n] * (c[q] - Ph[n][q]);   // d d_n / d P_n = (c - P_n) / ||.||
                g0[q] = fmaf(ah[n], gp, g0[q]);
                g1[q] = fmaf(bh[n], gp, g1[q]);
            }
    }
#pragma unroll
    for (int q = 0; q < C; ++q) {
        grow[eo + q] = g0[q];
        grow[eo + C + q] = g1[q];
    }
}

// endpoint block row r: L_e and the output deltas from the summed L_cd gradients
__device__ __forceinline__ void endpoint_block_row(const TrArgs& a, int s, bool valid, int r, const float* Ys,
                                                   const float* Gs, unsigned char* D, float& le) {
    const ModelView& mv = a.mv;
    const int od = mv.endpoint.out_dim;
    int b = a.ids[s];
    const float inv_ne = 1.f / ((float)a.B * (float)od);
    for (int t = 0; t < mv.n_textures; ++t) {
        const int fmt = mv.formats[t], C = fmt == NTBC_BC1 ? 3 : 1, eo = mv.eoff[t];
        float e0[3], e1[3];
        ref_endpoints(fmt, a.tp.blocks[t], b, e0, e1);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (q < C)
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    int col = eo + k * C + q;
                    float yh = Ys[r * od + col], ref = k ? e1[q] : e0[q];
                    float rr = yh - ref;
                    if (valid) le = fmaf(rr, rr, le);
                    float g = Gs[r * od + col] + 2.f * rr * inv_ne;
                    st_bf16(D, r, col, a.net.out_pad, valid ? g * yh * (1.f - yh) : 0.f);
                }
    }
}

// grid features of one sample (FP32 master grid, QAT fake quantisation while active)
// straight into the BF16 X row: level l -> columns 2l, 2l + 1
// the two features of level l at (u, v) (bilinear over the FP32 grid, fake-quantised in the
// QAT phase) as one BF16 pair in row r of the X tile (and, with Xlo, their lo parts in Xlo)
__device__ __forceinline__ void gather_level_train(const NetView& nv, const GridSrc& src, int l, float u, float v,
                                                   unsigned char* X, int r, int K0, int qat_bits,
                                                   unsigned char* Xlo = nullptr) {
    Bilinear bl = bilinear_at(nv.res[l], u, v);
    const float* gp = src.f32 + nv.grid_off[l] + bl.base;
    float2 p00 = __ldg(reinterpret_cast<const float2*>(gp));
    float2 p01 = __ldg(reinterpret_cast<const float2*>(gp + 2));
    float2 p10 = __ldg(reinterpret_cast<const float2*>(gp + bl.row));
    float2 p11 = __ldg(reinterpret_cast<const float2*>(gp + bl.row + 2));
    if (qat_bits > 0) {
        float sc = src.scale[l], z = src.zero[l], qm = (float)((1 << qat_bits) - 1);
        p00 = make_float2(fake_quant(p00.x, sc, z, qm), fake_quant(p00.y, sc, z, qm));
        p01 = make_float2(fake_quant(p01.x, sc, z, qm), fake_quant(p01.y, sc, z, qm));
        p10 = make_float2(fake_quant(p10.x, sc, z, qm), fake_quant(p10.y, sc, z, qm));
        p11 = make_float2(fake_quant(p11.x, sc, z, qm), fake_quant(p11.y, sc, z, qm));
    }
    float f0 = bl.w00 * p00.x + bl.w01 * p01.x + bl.w10 * p10.x + bl.w11 * p11.x;
    float f1 = bl.w00 * p00.y + bl.w01 * p01.y + bl.w10 * p10.y + bl.w11 * p11.y;
    const int off = chunk_byte(r, (2 * l) >> 3, K0) + ((2 * l) & 7) * 2;
    const uint32_t hi = pack_bf16x2(f0, f1);
    *reinterpret_cast<uint32_t*>(X + off) = hi;
    if (Xlo) *reinterpret_cast<uint32_t*>(Xlo + off) = pack_bf16x2_lo(f0, f1, hi);
}

__device__ __forceinline__ void gather_row_train(const NetView& nv, const GridSrc& src, float u, float v,
                                                 unsigned char* X, int r, int K0) {
    const int qat_bits = src.qat_bits;
    for (int l = 0; l < nv.levels; ++l) {               // both corner rows of every level into L1
        Bilinear bl = bilinear_at(nv.res[l], u, v);
        const float* gp = src.f32 + nv.grid_off[l] + bl.base;
        prefetch_l1(gp);
        prefetch_l1(gp + bl.row);
    }
#pragma unroll 4
    for (int l = 0; l < nv.levels; ++l) gather_level_train(nv, src, l, u, v, X, r, K0, qat_bits);
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

constexpr int kTrEndpointThreads = 512;   // endpoint CTA: warpgroup 0 runs the tile, all 16 warps the loss

template <bool COLOR>
__global__ void __launch_bounds__(COLOR ? 2 * kTrRows * kTrMaxGroups : kTrEndpointThreads, 1)
    train_tc_kernel(const __grid_constant__ TrArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag[kTrMaxGroups];
    __shared__ int pair_stop[kTrMaxGroups];
    const TrNet& net = a.net;
    const TrSmem& sl = a.sl;
    const NetView& nv = COLOR ? a.mv.color : a.mv.endpoint;
    const int act = a.mv.activation;
    const bool tile_thread = threadIdx.x < a.groups * kTrRows;
    const bool helper = COLOR && !tile_thread && threadIdx.x < 2 * a.groups * kTrRows;

    // weight image -> shared memory; tiles zeroed (no stale NaN bit patterns ever reach an MMA)
    for (int i = threadIdx.x; i < net.img_bytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = reinterpret_cast<const uint4*>(a.img)[i];
    for (int i = threadIdx.x; i < a.groups * sl.group_bytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem + sl.group_off)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();

    TrGroup G;
    G.g = tile_thread ? threadIdx.x / kTrRows : (helper ? threadIdx.x / kTrRows - a.groups : 0);
    G.r = threadIdx.x % kTrRows;
    unsigned char* gb = smem + sl.group_off + G.g * sl.group_bytes;
    G.X = gb + sl.x_off;
    G.X2 = gb + sl.x2_off;
    for (int l = 0; l < 3; ++l) G.A[l] = gb + sl.a_off[l];
    G.D = gb + sl.d_off;
    G.bar = reinterpret_cast<uint64_t*>(gb + sl.bar_off);
    // endpoint: lo parts of the hidden activations, [128][64] over the delta tile (dead during
    // the forward: the loss writes it after the last forward MMA has completed)
    unsigned char* const Alo = gb + sl.alo_off;
    const int r = G.r;
    if (tile_thread) {
        // constant columns: the bias column of every hidden tile (64 = 1) and of X (in_dim = 1)
        for (int l = 0; l < net.n_layers - 1; ++l) {
            float v8[8] = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            st_chunk_bf16(G.A[l], r, 8, kTrHidCols, v8);
        }
        for (int kg = net.in_dim / 8; kg < net.K0 / 8; ++kg) {
            float v8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v8[j] = kg * 8 + j == net.in_dim ? 1.f : 0.f;
            st_chunk_bf16(G.X, r, kg, net.K0, v8);
            if (COLOR) st_chunk_bf16(G.X2, r, kg, net.K0, v8);   // endpoint: X2 holds lo parts (0 here)
        }
        if (r == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(G.bar)), "r"(1));
            asm volatile("fence.mbarrier_init.release.cluster;");
            abort_flag[G.g] = 0;
        }
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    G.tmem = tmem_slot + (uint32_t)(G.g * 256);
    G.row = G.tmem + ((uint32_t)((r / 32) * 32) << 16);
    volatile int* abort = abort_flag;

    const int L = net.n_layers;
    const uint32_t R = G.tmem;                 // forward / data-gradient accumulator (64 columns)
    const int od = net.out_dim;
    float* Ys = reinterpret_cast<float*>(smem + sl.stage_off);   // endpoint only
    float* Gs = Ys + kTrRows * od;
    float2* UV = reinterpret_cast<float2*>(Gs + kTrRows * od);    // endpoint only: block coordinates
    uint32_t phase = 0;
    bool ok = true, first = true;
    float loss0 = 0.f, loss1 = 0.f;
    const int tile0 = COLOR ? blockIdx.x * a.groups + G.g : blockIdx.x;
    const int tstep = COLOR ? gridDim.x * a.groups : gridDim.x;

    bool pending = false;                   // colour: a FULL arrival whose EMPTY is still owed
    if (helper) {
        // the grid scatter of the paired group's tiles (texels, warp-aggregated along the
        // block's rows and columns), one tile behind the group
        const int qat_bits = a.src.qat_bits;
        const float* gs = reinterpret_cast<const float*>(G.D) + r * 33;
        auto gather = [&](int t, unsigned char* X) {
            const int sr = t * kTrRows + r;
            float gu, gv2;
            int x, y;
            sample_coords(a.mv, true, a.ids, sr < a.B ? sr : a.B - 1, gu, gv2, x, y);
            gather_row_train(nv, a.src, gu, gv2, X, r, net.K0);
            proxy_fence();                            // the tensor core reads the tile
            pair_arrive(pair_xfull_id(G.g));
        };
        if (tile0 < a.tiles) gather(tile0, G.X);
        int k = 0;
        for (int tile = tile0; tile < a.tiles; tile += tstep, ++k) {
            // the next tile's input goes to the tile the group finished with one tile ago
            if (tile + tstep < a.tiles) gather(tile + tstep, (k & 1) ? G.X : G.X2);
            pair_sync(pair_full_id(G.g));
            if (pair_stop[G.g]) break;
            float gv[2 * NTBC_MAX_LEVELS];
#pragma unroll
            for (int j = 0; j < 2 * NTBC_MAX_LEVELS; ++j) gv[j] = gs[j];
            pair_arrive(pair_empty_id(G.g));          // the delta tile is free again
            const int s_raw = tile * kTrRows + r;
            const bool valid = s_raw < a.B;
            float su, sv;
            int x, y;
            sample_coords(a.mv, true, a.ids, valid ? s_raw : a.B - 1, su, sv, x, y);
            const Neighbours nbr = neighbours(su, sv);
#pragma unroll 1
            for (int lv = 0; lv < nv.levels; ++lv)
                scatter_level(nv, true, lv, su, sv, r, valid, gv[2 * lv], gv[2 * lv + 1], a.src, qat_bits, a.grads, nbr);
        }
    } else
    for (int tile = tile0, kk = 0; tile < a.tiles; tile += tstep, ++kk) {
        const int s_raw = tile * kTrRows + r;
        const bool valid = s_raw < a.B;
        const int s = valid ? s_raw : a.B - 1;

        if (!COLOR) {
            // ---- gather of the tile's 128 blocks, one (block, level) item per thread over all
            // 16 warps; the blocks' coordinates stay in shared memory for the scatter
            const int qat_bits = a.src.qat_bits;
            for (int p = threadIdx.x; p < kTrRows * nv.levels; p += blockDim.x) {
                const int rr = p % kTrRows, lv = p / kTrRows, sb = tile * kTrRows + rr;
                float u, v;
                int x, y;
                sample_coords(a.mv, false, a.ids, sb < a.B ? sb : a.B - 1, u, v, x, y);
                if (lv == 0) UV[rr] = make_float2(u, v);
                gather_level_train(nv, a.src, lv, u, v, G.X, rr, net.K0, qat_bits, G.X2);
            }
            proxy_fence();
            __syncthreads();
        }
        unsigned char* Xt = (COLOR && (kk & 1)) ? G.X2 : G.X;    // this tile's input tile
        // colour: the tile warpgroup; endpoint: all 16 warps, warpgroup qw taking accumulator
        // columns [16 qw, 16 qw + 16) of every row in the epilogues (TMEM lane quarters are the
        // warp's index mod 4, so every warp reaches its rows)
        const bool mma_thread = COLOR ? tile_thread : true;
        const int qw = COLOR ? 0 : (int)threadIdx.x / kTrRows;
        if (mma_thread && ok) {
            // ---- gather (colour: gathered ahead by the helper)
            if (COLOR) pair_sync(pair_xfull_id(G.g));
            // ---- forward
            for (int l = 0; l < L; ++l) {
                const TrLayer& Ly = net.layer[l];
                if (!(COLOR ? tr_barrier(G.g, abort) : tr_cta_barrier(abort))) {
                    ok = false;
                    break;
                }
                if (r == 0 && qw == 0) {
                    tc_fence_after();
                    const unsigned char* src = l == 0 ? Xt : G.A[l - 1];
                    const int C = l == 0 ? net.K0 : kTrHidCols;
                    const uint32_t idesc = umma_idesc_kind(Ly.N, 1, 0, 0);
                    for (int kc = 0; kc < Ly.K / 16; ++kc) {
                        uint64_t ad = umma_desc(smem_u32(src) + kc * 256, 128, (C / 8) * 128);
                        uint64_t bd = umma_desc(smem_u32(smem + Ly.img) + kc * 256, 128, (Ly.K / 8) * 128);
                        umma_f16(R, ad, bd, idesc, kc > 0);
                    }
                    if constexpr (!COLOR) {
                        // split operands: + A_lo W_hi (over the 64 units of a hidden tile: the
                        // constant bias input has no lo part) + A_hi W_lo (the lo x lo term,
                        // ~2^-16 of the product, is left out)
                        const unsigned char* src_lo = l == 0 ? G.X2 : Alo;
                        const int Clo = l == 0 ? net.K0 : 64;
                        for (int kc = 0; kc < Clo / 16; ++kc) {
                            uint64_t al = umma_desc(smem_u32(src_lo) + kc * 256, 128, (Clo / 8) * 128);
                            uint64_t bd = umma_desc(smem_u32(smem + Ly.img) + kc * 256, 128, (Ly.K / 8) * 128);
                            umma_f16(R, al, bd, idesc, 1);
                        }
                        for (int kc = 0; kc < Ly.K / 16; ++kc) {
                            uint64_t ad = umma_desc(smem_u32(src) + kc * 256, 128, (C / 8) * 128);
                            uint64_t bl = umma_desc(smem_u32(smem + net.lo_img + Ly.img) + kc * 256, 128,
                                                    (Ly.K / 8) * 128);
                            umma_f16(R, ad, bl, idesc, 1);
                        }
                    }
                    umma_commit(G.bar);
                }
                tr_wait(G, phase, abort);
                if (l + 1 < L) {
                    if constexpr (COLOR) {
#pragma unroll
                        for (int c0 = 0; c0 < 64; c0 += 32) {
                            float z[32];
                            tmem_ld16(G.row + c0, z);
                            tmem_ld16(G.row + c0 + 16, z + 16);
                            tmem_wait_ld_regs<32>(z);
#pragma unroll
                            for (int j = 0; j < 32; j += 2) {
                                const float2 y = act_fast2(make_float2(z[j], z[j + 1]), act);
                                z[j] = y.x;
                                z[j + 1] = y.y;
                            }
#pragma unroll
                            for (int q = 0; q < 4; ++q) st_chunk_bf16(G.A[l], r, c0 / 8 + q, kTrHidCols, z + 8 * q);
                        }
                    } else {
                        float z[16];
                        tmem_ld16(G.row + 16 * qw, z);
                        tmem_wait_ld_regs<16>(z);
#pragma unroll
                        for (int j = 0; j < 16; j += 2) {
                            const float2 y = act_fast2(make_float2(z[j], z[j + 1]), act);
                            z[j] = y.x;
                            z[j + 1] = y.y;
                        }
                        // hi parts for the next layer and the backward, lo parts for the next layer
                        // (layer l's MMAs, the last readers of the lo tile, have completed)
                        st_chunk_bf16_split(G.A[l], kTrHidCols, Alo, 64, r, 2 * qw, z);
                        st_chunk_bf16_split(G.A[l], kTrHidCols, Alo, 64, r, 2 * qw + 1, z + 8);
                    }
                }
            }
        }
        // the helper is done with the delta tile (the previous tile's gradients) before the
        // loss writes it
        if (COLOR && tile_thread && pending) {
            pair_sync(pair_empty_id(G.g));
            pending = false;
        }
        if (mma_thread && ok) {
            // ---- outputs -> loss (colour) or staging (endpoint)
            {
                if (COLOR) {
#pragma unroll
                    for (int kg = 0; kg < 6; ++kg) {
                        if (kg * 8 >= net.out_pad) break;
                        float zero8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                        st_chunk_bf16(G.D, r, kg, net.out_pad, zero8);
                    }
                    color_loss_row(a, s, valid, G.row, G.D, r, loss0, loss1);
                } else {
                    const int c0 = 16 * qw;                      // warp-uniform
                    if (c0 < net.out_pad) {
                        float z[16];
                        tmem_ld16(G.row + c0, z);
                        tmem_wait_ld_regs<16>(z);
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < od) Ys[r * od + c0 + j] = sigmoid_fast(z[j]);
                    }
                }
            }
        }

        if (!COLOR) {
            // ---- endpoint L_cd over the tile's 128 blocks x 16 texels, shared by all 16 warps
            __syncthreads();
            if (abort[0]) break;
            // one (block, texture) item per thread; a warp holds 32 blocks of one texture
            for (int item = threadIdx.x; item < kTrRows * a.mv.n_textures; item += blockDim.x) {
                const int t = item / kTrRows, bb = item % kTrRows, sb = tile * kTrRows + bb;
                const bool pv = sb < a.B;
                const int b = a.ids[pv ? sb : a.B - 1];
                if (a.mv.formats[t] == NTBC_BC1)
                    endpoint_item<3>(a, NTBC_BC1, b, a.mv.eoff[t], Ys + bb * od, a.tp.blocks[t], a.tp.texels[t], pv,
                                     Gs + bb * od, loss1);
                else
                    endpoint_item<1>(a, NTBC_BC4, b, a.mv.eoff[t], Ys + bb * od, a.tp.blocks[t], a.tp.texels[t], pv,
                                     Gs + bb * od, loss1);
            }
            __syncthreads();
            if (tile_thread) {
#pragma unroll
                for (int kg = 0; kg < 6; ++kg) {
                    if (kg * 8 >= net.out_pad) break;
                    float zero8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    st_chunk_bf16(G.D, r, kg, net.out_pad, zero8);
                }
                endpoint_block_row(a, s, valid, r, Ys, Gs, G.D, loss0);
            }
        }

        if (mma_thread && ok) {
            // ---- backward
            for (int l = L - 1; l >= 0; --l) {
                const TrLayer& Ly = net.layer[l];
                const int CD = l == L - 1 ? net.out_pad : 64;       // columns of the delta tile
                if (!(COLOR ? tr_barrier(G.g, abort) : tr_cta_barrier(abort))) {
                    ok = false;
                    break;
                }
                if (r == 0 && qw == 0) {
                    tc_fence_after();
                    const uint32_t dw = G.tmem + (uint32_t)Ly.dw_col;
                    const uint32_t d_base = smem_u32(G.D);
                    const uint32_t dstride = (uint32_t)(CD / 8) * 128;
                    if (l > 0) {          // dW_l^T[i][o] += sum_s A_{l-1}[s][i] D_l[s][o]
                        const uint32_t a_base = smem_u32(G.A[l - 1]);
                        const uint32_t idw = umma_idesc_kind(Ly.N, 1, 1, 1);
                        for (int ks = 0; ks < kTrRows / 16; ++ks) {
                            uint64_t ad = umma_desc(a_base + ks * 2 * (kTrHidCols / 8) * 128, (kTrHidCols / 8) * 128, 128);
                            uint64_t bd = umma_desc(d_base + ks * 2 * dstride, dstride, 128);
                            umma_f16(dw, ad, bd, idw, !(first && ks == 0));
                        }
                    } else {              // dW_0[o][i] += sum_s D_0[s][o] X[s][i]
                        const uint32_t x_base = smem_u32(Xt);
                        const uint32_t xstride = (uint32_t)(net.K0 / 8) * 128;
                        const uint32_t idw = umma_idesc_kind(net.K0, 1, 1, 1);
                        for (int ks = 0; ks < kTrRows / 16; ++ks) {
                            uint64_t ad = umma_desc(d_base + ks * 2 * dstride, dstride, 128);
                            uint64_t bd = umma_desc(x_base + ks * 2 * xstride, xstride, 128);
                            umma_f16(dw, ad, bd, idw, !(first && ks == 0));
                        }
                    }
                    // dA_{l-1} = D_l W_l (N = the layer's inputs, incl. the bias column for l = 0)
                    const int n_in = l > 0 ? 64 : net.K0;
                    const uint32_t idd = umma_idesc_kind(n_in, 1, 0, 1);
                    const uint32_t wstride = (uint32_t)(Ly.K / 8) * 128;
                    for (int kc = 0; kc < CD / 16; ++kc) {
                        uint64_t ad = umma_desc(d_base + kc * 256, 128, dstride);
                        uint64_t bd = umma_desc(smem_u32(smem + Ly.img) + kc * 2 * wstride, wstride, 128);
                        umma_f16(R, ad, bd, idd, kc > 0);
                    }
                    umma_commit(G.bar);
                }
                tr_wait(G, phase, abort);
                if (!COLOR && l > 0) {    // quarter qw of D_{l-1} = dA_{l-1} * act'(A_{l-1})
                    float dA[16];
                    tmem_ld16(G.row + 16 * qw, dA);
                    tmem_wait_ld_regs<16>(dA);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        float av[8];
                        ld_chunk_bf16(G.A[l - 1], r, 2 * qw + q, kTrHidCols, av);
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            dA[8 * q + j] = valid ? dA[8 * q + j] * act_grad_from_out(av[j], act) : 0.f;
                    }
                    st_chunk_bf16(G.D, r, 2 * qw, 64, dA);
                    st_chunk_bf16(G.D, r, 2 * qw + 1, 64, dA + 8);
                } else if (!COLOR) {      // quarters 0, 1: d loss / d features (32 columns)
                    if (qw < 2) {
                        float gx[16];
                        tmem_ld16(G.row + 16 * qw, gx);
                        tmem_wait_ld_regs<16>(gx);
                        float* gs = reinterpret_cast<float*>(G.D) + r * 33 + 16 * qw;
#pragma unroll
                        for (int j = 0; j < 16; ++j) gs[j] = gx[j];
                    }
                } else if (l > 0) {       // D_{l-1} = dA_{l-1} * act'(A_{l-1})
#pragma unroll
                    for (int c0 = 0; c0 < 64; c0 += 32) {
                        float dA[32];
                        tmem_ld16(G.row + c0, dA);
                        tmem_ld16(G.row + c0 + 16, dA + 16);
                        tmem_wait_ld_regs<32>(dA);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            float av[8];
                            ld_chunk_bf16(G.A[l - 1], r, c0 / 8 + q, kTrHidCols, av);
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                dA[8 * q + j] = valid ? dA[8 * q + j] * act_grad_from_out(av[j], act) : 0.f;
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) st_chunk_bf16(G.D, r, c0 / 8 + q, 64, dA + 8 * q);
                    }
                } else {                  // d loss / d features -> grid scatter-add
                    float gx[32];
                    tmem_ld16(G.row, gx);
                    tmem_ld16(G.row + 16, gx + 16);
                    tmem_wait_ld_regs<32>(gx);
                    float* gs = reinterpret_cast<float*>(G.D) + r * 33;    // the delta tile is free now
#pragma unroll
                    for (int j = 0; j < 32; ++j) gs[j] = gx[j];
                    // (colour: the helper warpgroup scatters gs; endpoint: all warps, below)
                }
            }
            if (ok) first = false;
        }
        if (COLOR && tile_thread) {         // hand the tile's gradients (or the stop) to the helper
            if (r == 0) pair_stop[G.g] = ok ? 0 : 1;
            __threadfence_block();
            pair_arrive(pair_full_id(G.g));
            pending = ok;
            if (!ok && tile + tstep < a.tiles) pair_sync(pair_xfull_id(G.g));   // the tile gathered ahead
        }
        if (!COLOR) {
            // blocks: the (sample, level) scatter items spread over all 16 warps
            __syncthreads();
            if (abort[0]) break;
            const int qat_bits = a.src.qat_bits;
            const float* gs_all = reinterpret_cast<const float*>(G.D);
            for (int p = threadIdx.x; p < kTrRows * nv.levels; p += blockDim.x) {
                const int rr = p % kTrRows, lv = p / kTrRows, sb = tile * kTrRows + rr;
                const bool pv = sb < a.B;
                const float2 uv = UV[rr];
                scatter_level(nv, false, lv, uv.x, uv.y, rr, pv, gs_all[rr * 33 + 2 * lv], gs_all[rr * 33 + 2 * lv + 1],
                              a.src, qat_bits, a.grads);
            }
            __syncthreads();                // staging reused by the next tile
        } else if (!ok) {
            break;
        }
    }

    if (COLOR && tile_thread && pending) pair_sync(pair_empty_id(G.g));

    // ---- losses: warp sums, then one double atomic per CTA and term
    {
        __shared__ float loss_red[2][kTrEndpointThreads / 32];
        const float n0 = (float)a.B * (float)od;
        const float n1 = COLOR ? n0 : (float)a.B * 16.f * (float)a.mv.color.out_dim;
        float v0 = loss0 / n0, v1 = loss1 / n1;
        for (int o = 16; o > 0; o >>= 1) {
            v0 += __shfl_xor_sync(0xffffffffu, v0, o);
            v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        }
        if ((threadIdx.x & 31) == 0) {
            loss_red[0][threadIdx.x >> 5] = v0;
            loss_red[1][threadIdx.x >> 5] = v1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s0 = 0.0, s1 = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                s0 += loss_red[0][w];
                s1 += loss_red[1][w];
            }
            atomicAdd(&a.acc[COLOR ? 2 : 0], s0);
            atomicAdd(&a.acc[COLOR ? 3 : 1], s1);
        }
    }

    // ---- weight gradients: this group's TMEM accumulators -> its row of partial sums (plain
    // stores; a second kernel adds the rows of all groups, so no address sees contention).
    // Layer 0 holds dW_0 (lane = unit o, column = input i, the bias at i = in); later layers
    // hold dW_l^T (lane = input i, the bias at i = in, column = unit o). Warps whose 32 lanes
    // hold nothing skip the layer; the others read only the columns that hold gradients.
    // In the endpoint kernel the four warps that reach one TMEM lane quarter (w, w + 4,
    // w + 8, w + 12) share the column chunks, so all 16 warps flush.
    bool flush = tile_thread && ok, no_tiles = first;
    int part_id = 0, nparts = 1;
    if (!COLOR) {
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        flush = abort[0] == 0;
        no_tiles = (int)blockIdx.x >= a.tiles;
        part_id = threadIdx.x / kTrRows;
        nparts = blockDim.x / kTrRows;
    }
    if (flush) {
        float* part = a.partials + (long long)(blockIdx.x * a.groups + G.g) * net.mlp_params;
        const int lane0 = r & ~31;
        for (int l = 0; l < L; ++l) {
            const TrLayer& Ly = net.layer[l];
            const int lanes = l == 0 ? Ly.out : Ly.in + 1;
            if (lane0 >= lanes) continue;                    // warp-uniform
            const int ncol = l == 0 ? Ly.in + 1 : Ly.out;
            const bool lane_ok = r < lanes;
            float* wrow = part + (Ly.w_off - net.mlp_base) + (l == 0 ? (long long)r * Ly.in : (long long)r);
            float* brow = part + (Ly.b_off - net.mlp_base);
            for (int c0 = 0, ci = 0; c0 < ncol; c0 += 16, ++ci) {
                if (ci % nparts != part_id) continue;            // warp-uniform
                float v[16];
                if (!no_tiles) {
                    tmem_ld16(G.row + (uint32_t)Ly.dw_col + c0, v);
                    tmem_wait_ld_regs<16>(v);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0.f;      // a group without tiles adds nothing
                }
                if (!lane_ok) continue;
                if (l == 0) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int c = c0 + j;
                        if (c < Ly.in) wrow[c] = v[j];
                        else if (c == Ly.in) brow[r] = v[j];
                    }
                } else if (r < Ly.in) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c0 + j < Ly.out) wrow[(long long)(c0 + j) * Ly.in] = v[j];
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c0 + j < Ly.out) brow[c0 + j] = v[j];
                }
            }
        }
    }

    // ---- teardown: a group whose wait gave up lets its in-flight MMAs land before TMEM is freed
    if (tile_thread && !ok) {
        if (r == 0) atomicExch(a.err, 1);
        mbar_wait(G.bar, phase ^ 1);
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot), "r"(512));
}

// grads[base + j] += sum over a network's partial rows. blockIdx.x: 32 columns of the colour
// network's parameters, then of the endpoint network's; blockIdx.y: a chunk of kReduceRows
// rows, split over the 8 warps (each row read is one 128-byte line); the chunk's sum is added
// atomically (the rows of a column are spread over several chunks).
constexpr int kReduceWarps = 8;
constexpr int kReduceRows = 32;
struct ReducePart {
    const float* part;
    float* grads;             // grads + the network's mlp_base
    int rows, n, col_blocks;
};
__global__ void __launch_bounds__(32 * kReduceWarps) reduce_partials_kernel(ReducePart c, ReducePart e) {
    __shared__ float sums[kReduceWarps][32];
    const bool ep = (int)blockIdx.x >= c.col_blocks;
    const ReducePart& q = ep ? e : c;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = ((int)blockIdx.x - (ep ? c.col_blocks : 0)) * 32 + lane;
    const int r0 = blockIdx.y * kReduceRows, r1 = min(r0 + kReduceRows, q.rows);
    if (r0 >= r1) return;                                  // CTA-uniform
    float acc = 0.f;
    if (j < q.n)
        for (int p = r0 + w; p < r1; p += kReduceWarps) acc += __ldcs(q.part + (long long)p * q.n + j);
    sums[w][lane] = acc;
    __syncthreads();
    if (w == 0 && j < q.n) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kReduceWarps; ++k) t += sums[k][lane];
        atomicAdd(q.grads + j, t);
    }
}

ntbc_status train_tc_reduce(const TrNet& cnet, const float* cpart, int crows, const TrNet& enet, const float* epart,
                            int erows, float* grads, cudaStream_t s) {
    ReducePart c{cpart, grads + cnet.mlp_base, crows, cnet.mlp_params, (cnet.mlp_params + 31) / 32};
    ReducePart e{epart, grads + enet.mlp_base, erows, enet.mlp_params, (enet.mlp_params + 31) / 32};
    const int chunks = (std::max(crows, erows) + kReduceRows - 1) / kReduceRows;
    if (chunks < 1) return NTBC_OK;
    reduce_partials_kernel<<<dim3(c.col_blocks + e.col_blocks, chunks), 32 * kReduceWarps, 0, s>>>(c, e);
    NTBC_CHECK_LAUNCH("weight-gradient partials");
    return NTBC_OK;
}

// BF16 weight images of both networks (blockIdx.y: colour, endpoint): per layer the [N][K]
// tile (W in columns 0..in-1, the bias in column `in`, zeros elsewhere), canonical K-major
// core-matrix layout; a network with lo_img also gets the lo parts, w - bf16(w) in BF16
__global__ void train_image_kernel(const float* __restrict__ params, TrNet net0, TrNet net1,
                                   __nv_bfloat16* __restrict__ img0, __nv_bfloat16* __restrict__ img1) {
    const TrNet& net = blockIdx.y ? net1 : net0;
    __nv_bfloat16* img = blockIdx.y ? img1 : img0;
    for (int l = 0; l < net.n_layers; ++l) {
        const TrLayer& Ly = net.layer[l];
        __nv_bfloat16* t = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(img) + Ly.img);
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ly.N * Ly.K; e += gridDim.x * blockDim.x) {
            int n = e / Ly.K, k = e % Ly.K;
            float w = 0.f;
            if (n < Ly.out) {
                if (k < Ly.in) w = params[Ly.w_off + (long long)n * Ly.in + k];
                else if (k == Ly.in) w = params[Ly.b_off + n];
            }
            const __nv_bfloat16 hi = __float2bfloat16_rn(w);
            t[core_byte(n, k, Ly.K) / 2] = hi;
            if (net.lo_img)
                t[(net.lo_img + core_byte(n, k, Ly.K)) / 2] = __float2bfloat16_rn(w - __bfloat162float(hi));
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

TrNet train_tc_net_desc(const ModelView& mv, bool color) {
    const NetView& nv = color ? mv.color : mv.endpoint;
    TrNet n;
    memset(&n, 0, sizeof(n));
    n.n_layers = nv.n_layers;
    n.in_dim = nv.in_dim;
    n.out_dim = nv.out_dim;
    n.out_pad = (nv.out_dim + 15) / 16 * 16;
    n.K0 = (nv.in_dim + 1 + 15) / 16 * 16;
    int img = 0, col = 64;
    for (int l = 0; l < nv.n_layers; ++l) {
        TrLayer& L = n.layer[l];
        L.in = nv.layer_in[l];
        L.out = nv.layer_out[l];
        L.K = l == 0 ? n.K0 : kTrHidCols;
        L.N = l + 1 == nv.n_layers ? n.out_pad : 64;
        L.img = img;
        img += L.N * L.K * 2;
        L.w_off = nv.w_off[l];
        L.b_off = nv.b_off[l];
        L.dw_col = col;
        col += l == 0 ? n.K0 : L.N;
    }
    n.mlp_base = n.layer[0].w_off;
    n.mlp_params = (int)(n.layer[nv.n_layers - 1].b_off + n.layer[nv.n_layers - 1].out - n.mlp_base);
    img = (img + 127) & ~127;
    // the endpoint network's forward takes split operands (its outputs steer the straight-through
    // softmax, where an output error is amplified 1/T): a second image of the weights' lo parts
    n.lo_img = color ? 0 : img;
    n.img_bytes = color ? img : 2 * img;
    return n;
}

int train_tc_tmem_cols(const TrNet& n) { return n.layer[n.n_layers - 1].dw_col + n.layer[n.n_layers - 1].N; }

static TrSmem train_tc_smem(const TrNet& n) {
    TrSmem s;
    memset(&s, 0, sizeof(s));
    s.group_off = n.img_bytes;
    int o = 0;
    s.x_off = o;
    o += kTrRows * n.K0 * 2;
    s.x2_off = o;
    o += kTrRows * n.K0 * 2;
    for (int l = 0; l < 3; ++l) {
        s.a_off[l] = o;
        if (l < n.n_layers - 1) o += kTrRows * kTrHidCols * 2;
    }
    s.d_off = o;
    s.alo_off = o;      // split forward: the lo activations [128][64] share the delta tile
    o += kTrRows * 64 * 2 + kTrPad;
    s.bar_off = o;
    o += 16;
    s.group_bytes = (o + 127) & ~127;
    s.stage_off = 0;
    return s;
}

ntbc_status train_tc_images(const float* params, const TrNet& cnet, unsigned char* cimg, const TrNet& enet,
                            unsigned char* eimg, cudaStream_t s) {
    train_image_kernel<<<dim3(32, 2), 256, 0, s>>>(params, cnet, enet, reinterpret_cast<__nv_bfloat16*>(cimg),
                                                   reinterpret_cast<__nv_bfloat16*>(eimg));
    NTBC_CHECK_LAUNCH("training weight images");
    return NTBC_OK;
}

int train_tc_max_partial_rows() { return 2 * 152; }

ntbc_status train_tc_launch(const ModelView& mv, bool color, const TrNet& net, const unsigned char* img,
                            const GridSrc& src, const TexPtrs& tp, const int32_t* ids, int B, float T, float* grads,
                            double* acc, int* err, float* partials, int max_rows, int* rows, cudaStream_t s) {
    *rows = 0;
    if (net.in_dim > 2 * NTBC_MAX_LEVELS || net.out_pad > 48)
        return fail(NTBC_EUNSUPPORTED, "tensor-core training: network shape outside the kernel's tiles");
    const int cols = train_tc_tmem_cols(net);
    if (cols > 512) return fail(NTBC_EUNSUPPORTED, "tensor-core training: accumulators exceed TMEM");
    TrArgs a;
    memset(&a, 0, sizeof(a));
    a.mv = mv;
    a.net = net;
    a.sl = train_tc_smem(net);
    a.src = src;
    a.tp = tp;
    a.ids = ids;
    a.B = B;
    a.tiles = (B + kTrRows - 1) / kTrRows;
    a.color = color;
    a.T = T;
    a.grads = grads;
    a.acc = acc;
    a.err = err;
    a.img = img;
    a.partials = partials;
    size_t smem = (size_t)a.sl.group_off + 2 * (size_t)a.sl.group_bytes;
    // colour: two warpgroups when their accumulators fit; endpoint: one tile per CTA
    // (the loss then runs on all 16 warps) with the FP32 staging of outputs and gradients
    a.groups = (color && cols <= 256 && smem + 1024 <= 227 * 1024) ? 2 : 1;
    smem = (size_t)a.sl.group_off + (size_t)a.groups * a.sl.group_bytes;
    if (!color) {
        a.sl.stage_off = (int)smem;
        smem += 2 * (size_t)kTrRows * net.out_dim * sizeof(float) + (size_t)kTrRows * sizeof(float2);
    }
    if (smem + 1024 > 227 * 1024) return fail(NTBC_EUNSUPPORTED, "tensor-core training: shared memory too small");
    smem = std::max(smem, (size_t)116 * 1024);     // one CTA per SM: each CTA allocates all 512 TMEM columns
    int dev = 0, sms = 0;
    NTBC_CHECK_CUDA(cudaGetDevice(&dev));
    NTBC_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int grid = std::min(sms, (a.tiles + a.groups - 1) / a.groups);
    if (grid < 1) return NTBC_OK;
    grid = std::min(grid, max_rows / a.groups);
    if (color) {
        NTBC_CHECK_CUDA(ensure_dynamic_smem(reinterpret_cast<const void*>(train_tc_kernel<true>), smem));
        train_tc_kernel<true><<<grid, 2 * kTrRows * a.groups, smem, s>>>(a);   // tile groups + their helpers
    } else {
        NTBC_CHECK_CUDA(ensure_dynamic_smem(reinterpret_cast<const void*>(train_tc_kernel<false>), smem));
        train_tc_kernel<false><<<grid, kTrEndpointThreads, smem, s>>>(a);
    }
    NTBC_CHECK_LAUNCH(color ? "tensor-core training (colour)" : "tensor-core training (endpoint)");
    *rows = grid * a.groups;
    return NTBC_OK;
}

}  // namespace ntbc
