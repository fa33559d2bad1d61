// Tensor-core (tcgen05) form of the fused NTBC inference kernel (Sec. 3.2,
// Fig. NTBC (a); Sec. 4.4) for FP16 weights, FP32 accumulation in TMEM.
//
// One persistent CTA per SM holds up to four independent warpgroups. A
// warpgroup owns one work unit at a time: 128 consecutive blocks. It runs the
// endpoint MLP on the 128 blocks as one M = 128 MMA chain, turns the sigmoid
// outputs into quantised endpoints and integer palettes (kept in shared memory),
// then runs the colour MLP on the unit's 2048 texels as 16 tiles of 128 texels
// (8 blocks each), picks each texel's code and packs the 16 codes of a block
// with shuffles inside the half-warp that holds the block.
//
// Per layer: the warpgroup writes its A tile (activations, FP16, canonical
// K-major core-matrix layout, no swizzle) to shared memory, one elected thread
// issues the K/16 MMAs (the bias rides in one extra K column: a constant 1 in A,
// the bias in B) and commits to the group's mbarrier; after the bounded wait the
// 128 threads read their row of the accumulator (tcgen05.ld 32x32b) and apply
// SELU (or the sigmoid on the output layer). The other warpgroups of the CTA
// keep the SM busy while one waits on its MMA.
//
// The FP8 arithmetic (NTBC_PREC_FP8_MMA) runs the same schedule with E4M3 tiles and
// kind::f8f6f4 MMAs (K = 32 per MMA): the A tile holds each layer's input scaled by the
// layer's 2^-a and rounded to E4M3, the B tile the E4M3 weight codes; the accumulator is
// then (x W) 2^-(a + w), so the epilogue forms z L = acc L 2^(a + w) + b L with the FP32
// bias from shared memory (no bias K block) and writes SELU(z) 2^-a' for the next layer.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ntbc_internal.cuh"
#include "ntbc_kernels.cuh"
#include "tcgen05.cuh"

namespace ntbc {

constexpr int kTcRows = 128;               // M of every MMA: blocks (endpoint) or texels (colour)
// Work unit: kTcUnitBlocks consecutive blocks (the endpoint MMA's 128 rows), or half of that
// when the palettes of a material with many textures would leave room for fewer warpgroups
// (the endpoint MMA then runs with 64 valid rows)
constexpr int kTcUnitBlocks = 128;
constexpr int kTcMaxGroups = 4;
constexpr int kTcColsPerGroup = 128;           // two 64-column accumulator regions per group
constexpr int kTcPalBytes = 12;            // integer palette bytes per block per texture
// A-operand (activation) formats: FP16; FP16 high + low halves (two MMAs per K block); E4M3
// at per-layer power-of-two scales (kind::f8f6f4)
enum { kActF16 = 0, kActSplit = 1, kActE4M3 = 2 };

__host__ __device__ constexpr int tc_a_bytes(int act) { return act == kActE4M3 ? 1 : 2; }
// store 8 FP16 values (k-group kg) of row r
__device__ __forceinline__ void st_row8(unsigned char* tile, int r, int kg, int K, const float* v) {
    __half2 h0 = __floats2half2_rn(v[0], v[1]), h1 = __floats2half2_rn(v[2], v[3]);
    __half2 h2 = __floats2half2_rn(v[4], v[5]), h3 = __floats2half2_rn(v[6], v[7]);
    uint4 u;
    u.x = *reinterpret_cast<uint32_t*>(&h0);
    u.y = *reinterpret_cast<uint32_t*>(&h1);
    u.z = *reinterpret_cast<uint32_t*>(&h2);
    u.w = *reinterpret_cast<uint32_t*>(&h3);
    *reinterpret_cast<uint4*>(tile + (((r >> 3) * (K >> 3) + kg) * 128 + (r & 7) * 16)) = u;
}

// x - (float)h for both halves of h (low half with x.x): one mixed-precision FMA per value,
// h * -1 + x with the half operand widened exactly and a single rounding (the residual of an
// FP16 rounding is exact in FP32, so no rounding happens at all)
__device__ __forceinline__ float2 residual_f16x2(__half2 h, float2 x) {
    float2 r;
    const uint32_t hb = *reinterpret_cast<uint32_t*>(&h);
    asm("{\n\t.reg .b16 hl, hu, m1;\n\tmov.b32 {hl, hu}, %2;\n\tmov.b16 m1, 0xBC00;\n\t"
        "fma.rn.f32.f16 %0, hl, m1, %3;\n\tfma.rn.f32.f16 %1, hu, m1, %4;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "r"(hb), "f"(x.x), "f"(x.y));
    return r;
}

// store 8 values as FP16 hi (and, when split, the FP16 rounding of the residual in lo)
template <bool SPLIT>
__device__ __forceinline__ void st_row8_split(unsigned char* hi_tile, unsigned char* lo_tile, int r, int kg, int K,
                                              const float* v) {
    if constexpr (!SPLIT) {
        st_row8(hi_tile, r, kg, K, v);
    } else {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __half2 h = __floats2half2_rn(v[2 * j], v[2 * j + 1]);
            float2 r = residual_f16x2(h, make_float2(v[2 * j], v[2 * j + 1]));
            __half2 lo = __floats2half2_rn(r.x, r.y);
            hw[j] = *reinterpret_cast<uint32_t*>(&h);
            lw[j] = *reinterpret_cast<uint32_t*>(&lo);
        }
        int off = ((r >> 3) * (K >> 3) + kg) * 128 + (r & 7) * 16;
        *reinterpret_cast<uint4*>(hi_tile + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

// two values as E4M3 codes (nearest even, saturating at +-448): lo in the low byte
__device__ __forceinline__ uint32_t e4m3x2(float lo, float hi) {
    unsigned short d;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(hi), "f"(lo));
    return d;
}

// store 16 values as E4M3 (k-group kg of 16 one-byte elements) of row r
__device__ __forceinline__ void st_row16_e4m3(unsigned char* tile, int r, int kg, int K, const float* v) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = e4m3x2(v[4 * j], v[4 * j + 1]) | (e4m3x2(v[4 * j + 2], v[4 * j + 3]) << 16);
    *reinterpret_cast<uint4*>(tile + core_byte8(r, 16 * kg, K)) = make_uint4(w[0], w[1], w[2], w[3]);
}

// Activations travel scaled by L = log2(e): every accumulator holds z L (the layer-0
// features and both bias inputs carry the factor), so the exponentials are plain ex2.
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2_approx(float x) {
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(x));
    return e;
}

// SELU on a pair of units with packed FP32 (two lanes per instruction):
// lambda max(a, 0) + lambda alpha L (2^min(a, 0) - 1), with max(a, 0) formed as a - min(a, 0)
// (exact) so that one min per unit serves both branches
__device__ __forceinline__ float2 selu2_l2(float2 a) {
    const float2 m = make_float2(fminf(a.x, 0.f), fminf(a.y, 0.f));
    float2 e = make_float2(ex2_approx(m.x), ex2_approx(m.y));
    float2 t = __ffma2_rn(make_float2(kSeluLA * kLog2e, kSeluLA * kLog2e), e,
                          make_float2(-kSeluLA * kLog2e, -kSeluLA * kLog2e));
    return __ffma2_rn(make_float2(kSeluLambda, kSeluLambda), __ffma2_rn(m, make_float2(-1.f, -1.f), a), t);
}

// sigmoid(z) from a = z L
__device__ __forceinline__ float sigmoid_l2(float a) { return __fdividef(1.f, 1.f + ex2_approx(-a)); }

// The same SELU with the output scaled: c1 (a - min(a, 0)) + c2 (2^min(a, 0) - 1), which is
// SELU(z) 2^-a' for c1 = lambda 2^-a' / L and c2 = lambda alpha 2^-a' (ReLU: c1 max(a, 0), c2 = 0)
__device__ __forceinline__ float2 selu2_scaled(float2 a, float c1, float c2) {
    const float2 m = make_float2(fminf(a.x, 0.f), fminf(a.y, 0.f));
    float2 e = make_float2(ex2_approx(m.x), ex2_approx(m.y));
    float2 t = __ffma2_rn(make_float2(c2, c2), e, make_float2(-c2, -c2));
    return __ffma2_rn(make_float2(c1, c1), __ffma2_rn(m, make_float2(-1.f, -1.f), a), t);
}

// The decisions of choose_code_bc1 / choose_code_bc4 (least squared FP32 distance, channels
// summed in order, ties to the lowest code) with two palette entries per packed instruction;
// each lane of a packed op rounds exactly like the scalar op, and p * -1 + x is x - p rounded
// once, so the distances and the codes are bit-identical.
__device__ __forceinline__ int choose_code_bc1_x2(const BlockPalette& bp, float r, float g, float b) {
    if (bp.solid) return 0;
    float d[4];
#pragma unroll
    for (int k = 0; k < 4; k += 2) {
        const float2 m1 = make_float2(-1.f, -1.f);
        float2 dr = __ffma2_rn(make_float2(bp.pal[k][0], bp.pal[k + 1][0]), m1, make_float2(r, r));
        float2 dg = __ffma2_rn(make_float2(bp.pal[k][1], bp.pal[k + 1][1]), m1, make_float2(g, g));
        float2 db = __ffma2_rn(make_float2(bp.pal[k][2], bp.pal[k + 1][2]), m1, make_float2(b, b));
        float2 s2 = __fadd2_rn(__fadd2_rn(__fmul2_rn(dr, dr), __fmul2_rn(dg, dg)), __fmul2_rn(db, db));
        d[k] = s2.x;
        d[k + 1] = s2.y;
    }
    int best = 0;
    float bestd = d[0];
#pragma unroll
    for (int k = 1; k < 4; ++k)
        if (d[k] < bestd) {
            bestd = d[k];
            best = k;
        }
    return best;
}

__device__ __forceinline__ int choose_code_bc4_x2(const BlockPalette& bp, float v) {
    float2 d[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float2 dv = __ffma2_rn(make_float2(bp.pal[2 * k][0], bp.pal[2 * k + 1][0]), make_float2(-1.f, -1.f),
                               make_float2(v, v));
        d[k] = __fmul2_rn(dv, dv);
    }
    // tournament: the right entry wins only when strictly smaller, so equal distances keep the
    // lowest code, as a first-minimum scan does
    int i0 = d[0].y < d[0].x, i1 = 2 + (d[1].y < d[1].x), i2 = 4 + (d[2].y < d[2].x), i3 = 6 + (d[3].y < d[3].x);
    float m0 = fminf(d[0].x, d[0].y), m1 = fminf(d[1].x, d[1].y), m2 = fminf(d[2].x, d[2].y), m3 = fminf(d[3].x, d[3].y);
    if (m1 < m0) { m0 = m1; i0 = i1; }
    if (m3 < m2) { m2 = m3; i2 = i3; }
    return m2 < m0 ? i2 : i0;
}

struct TcLayer {
    int K;           // total K of the MMA (FP16: multiple of 16, bias column included; E4M3: 32 or 64)
    int N;           // padded output width (multiple of 16)
    int out;         // real output width
    int img;         // byte offset of the B tile in the weight image
    int bias;        // E4M3: byte offset of the N FP32 values b L in the weight image
};

// E4M3: per network and layer (colour 0.., endpoint 0..) the FP32 constants
// (L 2^(a + w), c1, c2 of the scaled SELU writing the next layer's input, and for layer 0
// the grid-feature scale 2^-a), at byte ftab of the weight image. A ReLU hidden layer keeps
// L out of it (s = 2^(a + w - a'), bias b 2^-a'): every scaling is then a power of two, so
// an activation that is exactly an E4M3 rounding tie (common in a ReLU network, whose
// values are dyadic) reaches the rounding unperturbed.
struct TcLayerConst {
    float s, c1, c2, fscale;
};

struct TcNet {
    int n_layers;
    TcLayer layer[NTBC_MAX_MLP_LAYERS];
};

struct TcArgs {
    ModelView mv;
    TcNet net[2];             // 0 colour, 1 endpoint
    int img_bytes;            // weight image size (multiple of 16)
    int groups;
    int n;                    // blocks to process
    const int32_t* ids;       // optional block ids (else first .. first + n - 1)
    int first;
    int mode;                 // 0 pack, 1 raw outputs
    int ub;                   // blocks per work unit (128, or 64)
    int act;                  // A-operand format (kActF16, kActSplit, kActE4M3)
    int ftab;                 // E4M3: byte offset of the TcLayerConst table in the weight image
    int* err;
    float inv_w, inv_h, inv_bw, inv_bh;   // reciprocals of the texel and block extents
    // optional completion record (chained batches): units completed, the %globaltimer stamp of
    // the last one, and (first launch of a chain) the stamp of the launch's start
    int* done;
    unsigned long long* done_stamp;
    unsigned long long* start_stamp;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// block index -> (bx, by) without an integer division: q = floor(b / bw) from the FP32
// reciprocal (off by at most one for b < 2^24), then one correction step
__device__ __forceinline__ void block_xy(int b, int bw, float inv_bw, int& bx, int& by) {
    int q = (int)((float)b * inv_bw);
    q -= q * bw > b;
    q += (q + 1) * bw <= b;
    by = q;
    bx = b - q * bw;
}

struct TcOut {
    uint8_t* p[NTBC_MAX_TEXTURES];
    int stride[NTBC_MAX_TEXTURES];     // bytes between consecutive blocks of a texture
};

struct TcSmem {
    int ones_off, table_off, lvl_off, group_off, group_bytes, a_off, lo_off, pal_off, ep_off, bar_off;
};

// Shared: weight image, ones tile (bias K block), k/255 table, per-level dequantisation
// constants. Per group: A tile (FP16 or E4M3 activations), the low-half tile when split,
// the unit's integer palettes (12 bytes per block and texture) and quantised endpoints,
// and the group's mbarrier.
__host__ __device__ inline TcSmem tc_smem_layout(int img_bytes, int n_tex, int act, int ub) {
    TcSmem s;
    s.ones_off = (img_bytes + 127) & ~127;
    s.table_off = s.ones_off + 2 * kTcRows * 16 * 2;             // two constant tiles: L high, L low
    s.lvl_off = s.table_off + 256 * 4;
    s.group_off = (s.lvl_off + 2 * 4 * NTBC_MAX_LEVELS * 4 + 127) & ~127;
    s.a_off = 0;
    s.lo_off = kTcRows * 64 * tc_a_bytes(act);
    s.pal_off = s.lo_off + (act == kActSplit ? kTcRows * 64 * 2 : 0);
    s.ep_off = s.pal_off + ((n_tex * ub * kTcPalBytes + 15) & ~15);
    s.bar_off = s.ep_off + n_tex * ub * 4;
    s.group_bytes = (s.bar_off + 16 + 127) & ~127;
    return s;
}

__device__ __forceinline__ float tmem_ld1(uint32_t taddr) {
    uint32_t v;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(taddr));
    return __uint_as_float(v);
}

// the two codes (bytes 0 and 1) of a corner as exact floats: each byte lands in the low
// mantissa byte of 2^23, then one packed subtract of 2^23 (no integer-to-float conversion)
__device__ __forceinline__ float2 corner_codes(uint32_t word) {
    return __fadd2_rn(make_float2(__uint_as_float(__byte_perm(word, 0x4B000000u, 0x7540)),
                                  __uint_as_float(__byte_perm(word, 0x4B000000u, 0x7541))),
                      make_float2(-8388608.f, -8388608.f));
}

// corner-aligned bilinear set-up of level l: p = (u, v) (res - 1); floor(p) as p + 2^23
// rounded down, the integer then sits in the low mantissa bits (no float-to-int conversion on
// the XU pipe); p < res - 1 for every texel and block centre (checked on the host), so
// floor(p) <= res - 2 needs no clamp
__device__ __forceinline__ Bilinear bilinear_tc(const NetView& nv, int l, float u, float v) {
    float2 p = __fmul2_rn(make_float2(u, v), make_float2(nv.resm1[l], nv.resm1[l]));
    const float tx = __fadd_rd(p.x, 8388608.f), ty = __fadd_rd(p.y, 8388608.f);
    float2 fl = __fadd2_rn(make_float2(tx, ty), make_float2(-8388608.f, -8388608.f));
    float2 f = __fadd2_rn(p, make_float2(-fl.x, -fl.y));                 // (fx, fy)
    float2 g = __fadd2_rn(make_float2(1.f, 1.f), make_float2(-f.x, -f.y)); // (1 - fx, 1 - fy)
    float2 w0 = __fmul2_rn(make_float2(g.y, g.y), make_float2(g.x, f.x));  // (w00, w01)
    float2 w1 = __fmul2_rn(make_float2(f.y, f.y), make_float2(g.x, f.x));  // (w10, w11)
    const int ix = __float_as_int(tx) - 0x4B000000, iy = __float_as_int(ty) - 0x4B000000;
    Bilinear b;
    b.base = (long long)((iy * nv.res[l] + ix) * 2);
    b.row = nv.res[l] * 2;
    b.w00 = w0.x;
    b.w01 = w0.y;
    b.w10 = w1.x;
    b.w11 = w1.y;
    return b;
}

__device__ __forceinline__ uint32_t ld_u16(const uint8_t* p) {
    return (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p));
}

// Grid features of one row (texel or block), level-major, 2 per level, followed by the
// constant 1 of the layer-0 bias column; stored as FP16 chunks (high, and low halves when
// split), or for E4M3 as 32 codes of the features times 2^-a (no bias column). Exported
// grids: bilinear interpolation of the exact codes, then the dequantisation s (q - z) fs as
// one FMA with the per-level constants in lvl; FP32 grids: the interpolation times fs.
// fs = L, or 2^-a for E4M3.
template <int ACT>
__device__ __forceinline__ void gather_row(const NetView& nv, const GridSrc& src, const float4* lvl, float fs, float u,
                                           float v, int K0, unsigned char* A, unsigned char* Alo, int r, bool valid) {
    float f[2 * NTBC_MAX_LEVELS];
#pragma unroll
    for (int l = 0; l < NTBC_MAX_LEVELS; ++l) {
        float f0 = 0.f, f1 = 0.f;
        if (l < nv.levels && valid) {
            Bilinear b = bilinear_tc(nv, l, u, v);
            long long o = nv.grid_off[l] + b.base;
            if (src.codes) {
                const uint8_t* gp = src.codes + o;
                uint32_t a = ld_u16(gp), c = ld_u16(gp + 2), d = ld_u16(gp + b.row), e = ld_u16(gp + b.row + 2);
                float2 y = __fmul2_rn(make_float2(b.w00, b.w00), corner_codes(a));
                y = __ffma2_rn(make_float2(b.w01, b.w01), corner_codes(c), y);
                y = __ffma2_rn(make_float2(b.w10, b.w10), corner_codes(d), y);
                y = __ffma2_rn(make_float2(b.w11, b.w11), corner_codes(e), y);
                const float4 k = lvl[l];
                float2 f = __ffma2_rn(make_float2(k.x, k.y), y, make_float2(k.z, k.w));
                f0 = f.x;
                f1 = f.y;
            } else {
                const float* gp = src.f32 + o;
                float2 a = __ldg(reinterpret_cast<const float2*>(gp));
                float2 c = __ldg(reinterpret_cast<const float2*>(gp + 2));
                float2 d = __ldg(reinterpret_cast<const float2*>(gp + b.row));
                float2 e = __ldg(reinterpret_cast<const float2*>(gp + b.row + 2));
                f0 = (b.w00 * a.x + b.w01 * c.x + b.w10 * d.x + b.w11 * e.x) * fs;
                f1 = (b.w00 * a.y + b.w01 * c.y + b.w10 * d.y + b.w11 * e.y) * fs;
            }
        }
        f[2 * l] = f0;
        f[2 * l + 1] = f1;
    }
    if constexpr (ACT == kActE4M3) {              // K0 = 32 = 2 NTBC_MAX_LEVELS
        st_row16_e4m3(A, r, 0, 32, f);
        st_row16_e4m3(A, r, 1, 32, f + 16);
    } else {
#pragma unroll
        for (int kg = 0; kg < 6; ++kg) {
            if (kg * 8 >= K0) break;
            float v8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                int i = kg * 8 + j;
                float x = i < 2 * NTBC_MAX_LEVELS ? f[i] : 0.f;
                v8[j] = i == nv.in_dim ? kLog2e : x;
            }
            st_row8_split<ACT == kActSplit>(A, Alo, r, kg, K0, v8);
        }
    }
}

// Shared-memory pointers of one warpgroup.
struct TcGroup {
    unsigned char* A;
    unsigned char* Alo;
    uint8_t* palb;
    uint32_t* eps;
    uint64_t* bar;
    uint32_t tmem, tmem_row;
    int g, r;
};

// Per-level dequantisation constants of both grids as pairs: (s fs, s fs, -s z fs, -s z fs)
// with the feature scale fs of the network (L, or 2^-a for E4M3: fs_c colour, fs_e endpoint).
__device__ __forceinline__ void load_level_constants(const ModelView& mv, const GridSrc& csrc, const GridSrc& esrc,
                                                     float4* lvl, float fs_c = kLog2e, float fs_e = kLog2e) {
    for (int i = threadIdx.x; i < 2 * NTBC_MAX_LEVELS; i += blockDim.x) {
        int net = i / NTBC_MAX_LEVELS, l = i % NTBC_MAX_LEVELS;
        const GridSrc& src = net ? esrc : csrc;
        int L = net ? mv.endpoint.levels : mv.color.levels;
        const float fs = net ? fs_e : fs_c;
        float4 k = make_float4(0.f, 0.f, 0.f, 0.f);
        if (src.codes && l < L) {
            float sc = src.scale[l], z = src.zero[l];
            k = make_float4(sc * fs, sc * fs, -sc * z * fs, -sc * z * fs);
        }
        lvl[i] = k;
    }
}

// Constant tiles (L high / low for the bias K block) and the k/255 table.
__device__ __forceinline__ void load_constants(unsigned char* smem, const TcSmem& sl) {
    for (int i = threadIdx.x; i < kTcRows * 16; i += blockDim.x) {
        int rr = i / 16, k = i % 16;
        __half hi = __float2half_rn(kLog2e);
        __half lo = __float2half_rn(kLog2e - __half2float(hi));
        *reinterpret_cast<__half*>(smem + sl.ones_off + core_byte(rr, k, 16)) = k == 0 ? hi : __float2half(0.f);
        *reinterpret_cast<__half*>(smem + sl.ones_off + kTcRows * 32 + core_byte(rr, k, 16)) = k == 0 ? lo : __float2half(0.f);
    }
    for (int i = threadIdx.x; i < 256; i += blockDim.x) reinterpret_cast<float*>(smem + sl.table_off)[i] = __fdiv_rn((float)i, 255.f);
}

// TMEM columns, group barriers; every thread returns its group's view.
__device__ __forceinline__ TcGroup setup_groups(unsigned char* smem, const TcSmem& sl, int groups, uint32_t* tmem_slot,
                                                volatile int* abort_flag) {
    TcGroup G;
    G.g = threadIdx.x / kTcRows;
    G.r = threadIdx.x % kTcRows;
    unsigned char* gbase = smem + sl.group_off + G.g * sl.group_bytes;
    G.A = gbase + sl.a_off;
    G.Alo = gbase + sl.lo_off;
    G.palb = gbase + sl.pal_off;
    G.eps = reinterpret_cast<uint32_t*>(gbase + sl.ep_off);
    G.bar = reinterpret_cast<uint64_t*>(gbase + sl.bar_off);
    if (G.r == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(G.bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag[G.g] = 0;
    }
    const int ncols = groups == 1 ? 128 : (groups == 2 ? 256 : 512);
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    G.tmem = *tmem_slot + (uint32_t)(G.g * kTcColsPerGroup);
    G.tmem_row = G.tmem + ((uint32_t)((G.r / 32) * 32) << 16);   // this warp's 32 lanes
    return G;
}

__device__ __forceinline__ void teardown_groups(const TcGroup& G, int groups, bool ok, uint32_t phase, int* err,
                                                uint32_t tmem_slot) {
    // a group whose wait gave up records it and lets the MMA still in flight land
    // (bounded wait on the phase that gave up) before TMEM is freed
    if (!ok) {
        if (G.r == 0) atomicExch(err, 1);
        mbar_wait(G.bar, phase ^ 1);
    }
    tc_fence_before();
    __syncthreads();
    const int ncols = groups == 1 ? 128 : (groups == 2 ? 256 : 512);
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot), "r"(ncols));
}

// MMAs of K blocks kc0 .. kc1-1 of layer l (A tile of K0 columns for layer 0, 64
// afterwards; when split each block twice, high and low halves) and, with `bias`, the
// bias K block from the constant tiles, into the accumulator at tmem_d. A K block is 32
// bytes of every row: 16 FP16 values (kind::f16) or 32 E4M3 values (kind::f8f6f4, no bias
// block).
template <int ACT>
__device__ __forceinline__ void issue_steps(const TcLayer& L, int l, unsigned char* smem, unsigned char* A,
                                            const TcSmem& sl, uint32_t tmem_d, int kc0, int kc1, bool bias) {
    // descriptors built once; the K step advances only the start-address field (16-byte units,
    // no carry out of the field for shared-memory addresses), so each MMA adds to the low word
    constexpr int EPC = 16 / tc_a_bytes(ACT);               // elements per core-matrix row
    const uint32_t idesc = ACT == kActE4M3 ? umma_idesc_e4m3(L.N) : umma_idesc(L.N);
    const int Ka = l == 0 ? L.K : 64;
    const uint64_t a0 = umma_desc(smem_u32(A), 128, (Ka / EPC) * 128);
    const uint64_t b0 = umma_desc(smem_u32(smem + L.img), 128, (L.K / EPC) * 128);
    const uint32_t a_lo = (uint32_t)a0, a_hi = (uint32_t)(a0 >> 32);
    const uint32_t b_lo = (uint32_t)b0, b_hi = (uint32_t)(b0 >> 32);
    const uint32_t lo_step = (uint32_t)(sl.lo_off - sl.a_off) >> 4;
    for (int kc = kc0; kc < kc1; ++kc) {
        const uint32_t ka = a_lo + (uint32_t)kc * 16u, kb = b_lo + (uint32_t)kc * 16u;
        const uint64_t bd = ((uint64_t)b_hi << 32) | kb;
        if constexpr (ACT == kActE4M3) {
            umma_f8(tmem_d, ((uint64_t)a_hi << 32) | ka, bd, idesc, kc > 0);
        } else {
            umma_f16(tmem_d, ((uint64_t)a_hi << 32) | ka, bd, idesc, kc > 0);
            if (ACT == kActSplit) umma_f16(tmem_d, ((uint64_t)a_hi << 32) | (ka + lo_step), bd, idesc, 1);
        }
    }
    if (ACT != kActE4M3 && bias) {
        const uint64_t bd = ((uint64_t)b_hi << 32) | (b_lo + (uint32_t)(Ka / 16) * 16u);
        umma_f16(tmem_d, umma_desc(smem_u32(smem + sl.ones_off), 128, 256), bd, idesc, 1);
        if (ACT == kActSplit) umma_f16(tmem_d, umma_desc(smem_u32(smem + sl.ones_off + kTcRows * 32), 128, 256), bd, idesc, 1);
    }
}

// Group barrier after this thread's shared-memory writes and TMEM loads; false (for the
// whole group) once a bounded wait of the group has given up.
__device__ __forceinline__ bool group_barrier(int g, volatile int* abort_flag) {
    proxy_fence();
    tc_fence_before();
    group_sync(g);
    return abort_flag[g] == 0;
}

__device__ __forceinline__ void wait_mma(uint64_t* bar, uint32_t& phase, int g, volatile int* abort_flag) {
    if (!mbar_wait(bar, phase)) abort_flag[g] = 1;
    phase ^= 1;
    tc_fence_after();
}

// 32 accumulator columns (c0 .. c0 + 31) -> activation -> A columns c0 .. c0 + 31. E4M3:
// the accumulator is first turned into z L = acc s + b L (ReLU: z 2^-a' = acc s + b 2^-a';
// lc: the layer's constants, bias: its bias column in shared memory) and the activation is
// written scaled for the next layer.
template <int ACT>
__device__ __forceinline__ void epilogue_half(uint32_t src_row, int c0, unsigned char* A, unsigned char* Alo, int r,
                                              int act, const TcLayerConst& lc, const float* bias) {
    float v[32];
    tmem_ld16(src_row + c0, v);
    tmem_ld16(src_row + c0 + 16, v + 16);
    tmem_wait_ld();
    if constexpr (ACT == kActE4M3) {
        const float4* b4 = reinterpret_cast<const float4*>(bias + c0);
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
            const float4 b = b4[j / 4];
            float2 a0 = __ffma2_rn(make_float2(v[j], v[j + 1]), make_float2(lc.s, lc.s), make_float2(b.x, b.y));
            float2 a1 = __ffma2_rn(make_float2(v[j + 2], v[j + 3]), make_float2(lc.s, lc.s), make_float2(b.z, b.w));
            float2 y0, y1;
            if (act == NTBC_ACT_SELU) {
                y0 = selu2_scaled(a0, lc.c1, lc.c2);
                y1 = selu2_scaled(a1, lc.c1, lc.c2);
            } else {                             // ReLU: a is already z 2^-a'
                y0 = make_float2(fmaxf(a0.x, 0.f), fmaxf(a0.y, 0.f));
                y1 = make_float2(fmaxf(a1.x, 0.f), fmaxf(a1.y, 0.f));
            }
            v[j] = y0.x;
            v[j + 1] = y0.y;
            v[j + 2] = y1.x;
            v[j + 3] = y1.y;
        }
        st_row16_e4m3(A, r, c0 / 16, 64, v);
        st_row16_e4m3(A, r, c0 / 16 + 1, 64, v + 16);
    } else {
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
            float2 y = act == NTBC_ACT_SELU ? selu2_l2(make_float2(v[j], v[j + 1]))
                                            : make_float2(fmaxf(v[j], 0.f), fmaxf(v[j + 1], 0.f));
            v[j] = y.x;
            v[j + 1] = y.y;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) st_row8_split<ACT == kActSplit>(A, Alo, r, c0 / 8 + q, 64, v + 8 * q);
    }
}

// E4M3: the constants of layer l of network `net` (0 colour, 1 endpoint) in the image copy
__device__ __forceinline__ TcLayerConst layer_const(const unsigned char* smem, int ftab, int net, int l) {
    return reinterpret_cast<const TcLayerConst*>(smem + ftab)[net * NTBC_MAX_MLP_LAYERS + l];
}

// All layers of one MLP on the A tile the gather wrote. Accumulators alternate between the
// group's two TMEM regions, and each hidden epilogue runs in two halves: once the first 32
// activations of every row are in shared memory, the next layer's K blocks over them are
// issued, so they run on the tensor core while the second half is computed. Leaves the
// output layer's accumulator row at *out_row.
template <int ACT>
__device__ __forceinline__ bool run_mlp(const TcNet& net, int which, int ftab, int act, unsigned char* smem,
                                        const TcSmem& sl, const TcGroup& G, uint32_t& phase, uint32_t& region,
                                        volatile int* abort_flag, uint32_t* out_row) {
    constexpr int KB = ACT == kActE4M3 ? 32 : 16;        // K per MMA
    constexpr int KH = 32 / KB;                           // MMAs per half of a hidden layer
    if (!group_barrier(G.g, abort_flag)) return false;
    uint32_t cur = region;
    if (G.r == 0) {
        tc_fence_after();
        issue_steps<ACT>(net.layer[0], 0, smem, G.A, sl, G.tmem + 64 * cur, 0, net.layer[0].K / KB, false);
        umma_commit(G.bar);
    }
    wait_mma(G.bar, phase, G.g, abort_flag);
    for (int l = 1; l < net.n_layers; ++l) {
        uint32_t nxt = cur ^ 1;
        uint32_t src_row = G.tmem_row + 64 * cur;
        TcLayerConst lc{};
        const float* bias = nullptr;
        if constexpr (ACT == kActE4M3) {
            lc = layer_const(smem, ftab, which, l - 1);
            bias = reinterpret_cast<const float*>(smem + net.layer[l - 1].bias);
        }
        epilogue_half<ACT>(src_row, 0, G.A, G.Alo, G.r, act, lc, bias);
        if (!group_barrier(G.g, abort_flag)) return false;
        if (G.r == 0) {
            tc_fence_after();
            issue_steps<ACT>(net.layer[l], l, smem, G.A, sl, G.tmem + 64 * nxt, 0, KH, false);
        }
        epilogue_half<ACT>(src_row, 32, G.A, G.Alo, G.r, act, lc, bias);
        if (!group_barrier(G.g, abort_flag)) return false;
        if (G.r == 0) {
            tc_fence_after();
            issue_steps<ACT>(net.layer[l], l, smem, G.A, sl, G.tmem + 64 * nxt, KH, 2 * KH, true);
            umma_commit(G.bar);
        }
        wait_mma(G.bar, phase, G.g, abort_flag);
        cur = nxt;
    }
    region = cur ^ 1;
    *out_row = G.tmem_row + 64 * cur;
    return abort_flag[G.g] == 0;
}

// One work unit (UB blocks, 128 or 64): endpoint network, palettes, then UB / 8 colour tiles.
template <int ACT, int UB>
__device__ __forceinline__ bool process_unit(const TcArgs& args, const GridSrc& csrc, const GridSrc& esrc, const TcOut& outs,
                                          float* __restrict__ e_out, float* __restrict__ c_out, int unit,
                                          unsigned char* smem, const TcSmem& sl, const TcGroup& G, uint32_t& phase,
                                          uint32_t& region, volatile int* abort_flag) {
    const ModelView& mv = args.mv;
    const int r = G.r;
    unsigned char* A = G.A;
    unsigned char* Alo = G.Alo;
    uint8_t* palb = G.palb;
    uint32_t* eps = G.eps;
    const float* tab = reinterpret_cast<const float*>(smem + sl.table_off);
    const float4* lvl = reinterpret_cast<const float4*>(smem + sl.lvl_off);
    const int T = mv.n_textures;
    constexpr int ub = UB;
    bool ok = true;
    // E4M3: the output layers' z L = acc s + b L (FP16 paths: the accumulator already holds z L)
    float fs[2] = {kLog2e, kLog2e}, os[2] = {1.f, 1.f};
    const float* ob[2] = {nullptr, nullptr};
    if constexpr (ACT == kActE4M3) {
        for (int w = 0; w < 2; ++w) {
            const TcNet& tn = args.net[w];
            fs[w] = layer_const(smem, args.ftab, w, 0).fscale;
            os[w] = layer_const(smem, args.ftab, w, tn.n_layers - 1).s;
            ob[w] = reinterpret_cast<const float*>(smem + tn.layer[tn.n_layers - 1].bias);
        }
    }
    auto zl = [&](int w, float acc, int col) -> float {
        if constexpr (ACT == kActE4M3) return fmaf(acc, os[w], ob[w][col]);
        else return acc;
    };
        // ================= endpoint network: row r = block r of the unit
        {
            const TcNet& net = args.net[1];
            int k = unit * ub + r;
            bool valid = r < ub && k < args.n;
            int b = valid ? (args.ids ? args.ids[k] : args.first + k) : 0;
            int bx, by;
            block_xy(b, mv.bw, args.inv_bw, bx, by);
            gather_row<ACT>(mv.endpoint, esrc, lvl + NTBC_MAX_LEVELS, fs[1], ((float)bx + 0.5f) * args.inv_bw,
                            ((float)by + 0.5f) * args.inv_bh, net.layer[0].K, A, Alo, r, valid);
            uint32_t orow = 0;
            ok = run_mlp<ACT>(net, 1, args.ftab, mv.activation, smem, sl, G, phase, region, abort_flag, &orow);
            for (int l = net.n_layers - 1; l < net.n_layers && ok; ++l) {
                const uint32_t tmem_row = orow;
                if (args.mode == 1) {
                    int out = net.layer[l].out;
                    for (int o = 0; o < out; ++o) {
                        float e = tmem_ld1(tmem_row + o);
                        tmem_wait_ld_regs<1>(&e);
                        e = sigmoid_l2(zl(1, e, o));
                        if (valid) e_out[(long long)k * out + o] = e;
                    }
                    continue;
                }
                for (int t = 0; t < T && r < ub; ++t) {
                    int eo = mv.eoff[t];
                    uint8_t* pb = palb + (t * ub + r) * kTcPalBytes;
                    float e[6];
                    if (mv.formats[t] == NTBC_BC1) {
#pragma unroll
                        for (int q = 0; q < 6; ++q) e[q] = tmem_ld1(tmem_row + eo + q);
                        tmem_wait_ld();
#pragma unroll
                        for (int q = 0; q < 6; ++q) e[q] = sigmoid_l2(zl(1, e[q], eo + q));
                        uint32_t c0 = (quant_channel(e[0], 31.f, 31) << 11) | (quant_channel(e[1], 63.f, 63) << 5) |
                                      quant_channel(e[2], 31.f, 31);
                        uint32_t c1 = (quant_channel(e[3], 31.f, 31) << 11) | (quant_channel(e[4], 63.f, 63) << 5) |
                                      quant_channel(e[5], 31.f, 31);
                        if (c0 < c1) {
                            uint32_t tt = c0;
                            c0 = c1;
                            c1 = tt;
                        }
                        int p[4][3];
                        bc1_palette(c0, c1, p);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
#pragma unroll
                            for (int ch = 0; ch < 3; ++ch) pb[q * 3 + ch] = (uint8_t)p[q][ch];
                        eps[t * ub + r] = c0 | (c1 << 16);
                    } else {
                        e[0] = tmem_ld1(tmem_row + eo);
                        e[1] = tmem_ld1(tmem_row + eo + 1);
                        tmem_wait_ld();
                        int r0 = quant_channel(sigmoid_l2(zl(1, e[0], eo)), 255.f, 255);
                        int r1 = quant_channel(sigmoid_l2(zl(1, e[1], eo + 1)), 255.f, 255);
                        int p[8];
                        bc4_palette(r0, r1, p);
#pragma unroll
                        for (int q = 0; q < 8; ++q) pb[q] = (uint8_t)p[q];
                        eps[t * ub + r] = (uint32_t)r0 | ((uint32_t)r1 << 8);
                    }
                }
            }
        }
        // ================= colour network: 16 tiles of 8 blocks x 16 texels
        for (int tile = 0; tile < ub / 8 && ok; ++tile) {
            const TcNet& net = args.net[0];
            int blk = tile * 8 + r / 16, i = r & 15;
            int k = unit * ub + blk;
            bool valid = k < args.n;
            int b = valid ? (args.ids ? args.ids[k] : args.first + k) : 0;
            int bx, by;
            block_xy(b, mv.bw, args.inv_bw, bx, by);
            int x = 4 * bx + (i & 3), y = 4 * by + (i >> 2);
            gather_row<ACT>(mv.color, csrc, lvl, fs[0], ((float)x + 0.5f) * args.inv_w, ((float)y + 0.5f) * args.inv_h,
                            net.layer[0].K, A, Alo, r, valid);
            uint32_t orow = 0;
            ok = run_mlp<ACT>(net, 0, args.ftab, mv.activation, smem, sl, G, phase, region, abort_flag, &orow);
            for (int l = net.n_layers - 1; l < net.n_layers && ok; ++l) {
                const uint32_t tmem_row = orow;
                if (args.mode == 1) {
                    int out = net.layer[l].out;
                    for (int o = 0; o < out; ++o) {
                        float c = tmem_ld1(tmem_row + o);
                        tmem_wait_ld_regs<1>(&c);
                        c = sigmoid_l2(zl(0, c, o));
                        if (valid) c_out[((long long)k * 16 + i) * out + o] = c;
                    }
                    continue;
                }
                float cv[NTBC_MAX_TEXTURES][3];
#pragma unroll
                for (int t = 0; t < NTBC_MAX_TEXTURES; ++t) {
                    if (t >= T) break;
                    int co = mv.coff[t];
                    cv[t][0] = tmem_ld1(tmem_row + co);
                    if (mv.formats[t] == NTBC_BC1) {
                        cv[t][1] = tmem_ld1(tmem_row + co + 1);
                        cv[t][2] = tmem_ld1(tmem_row + co + 2);
                    }
                }
                tmem_wait_ld();
#pragma unroll
                for (int t = 0; t < NTBC_MAX_TEXTURES; ++t) {
                    if (t >= T) break;
                    const uint8_t* pb = palb + (t * ub + blk) * kTcPalBytes;
                    uint32_t ep = eps[t * ub + blk];
                    BlockPalette bp;
                    uint64_t bits;
                    if (mv.formats[t] == NTBC_BC1) {           // 2-bit codes: the block's 32 bits in one word
                        bp.solid = (ep & 0xFFFFu) == (ep >> 16);
                        uint32_t wv[3] = {*reinterpret_cast<const uint32_t*>(pb), *reinterpret_cast<const uint32_t*>(pb + 4),
                                          *reinterpret_cast<const uint32_t*>(pb + 8)};
#pragma unroll
                        for (int q = 0; q < 12; ++q) bp.pal[q / 3][q % 3] = tab[(wv[q / 4] >> (8 * (q % 4))) & 255];
                        const int co = mv.coff[t];
                        uint32_t w = (uint32_t)choose_code_bc1_x2(bp, sigmoid_l2(zl(0, cv[t][0], co)),
                                                                  sigmoid_l2(zl(0, cv[t][1], co + 1)),
                                                                  sigmoid_l2(zl(0, cv[t][2], co + 2))) << (2 * i);
#pragma unroll
                        for (int o = 8; o > 0; o >>= 1) w |= __shfl_xor_sync(0xffffffffu, w, o);
                        bits = w;
                    } else {                                   // 3-bit codes: 48 bits
                        uint32_t w0 = *reinterpret_cast<const uint32_t*>(pb);
                        uint32_t w1 = *reinterpret_cast<const uint32_t*>(pb + 4);
#pragma unroll
                        for (int q = 0; q < 8; ++q) bp.pal[q][0] = tab[((q < 4 ? w0 : w1) >> (8 * (q % 4))) & 255];
                        bits = (uint64_t)choose_code_bc4_x2(bp, sigmoid_l2(zl(0, cv[t][0], mv.coff[t]))) << (3 * i);
#pragma unroll
                        for (int o = 8; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
                    }
                    if (i == 0 && valid) {
                        uint8_t* dst = outs.p[t] + (long long)b * outs.stride[t];
                        if (mv.formats[t] == NTBC_BC1)
                            store_block(dst, ep, (uint32_t)bits);
                        else
                            store_block(dst, ep | (uint32_t)((bits & 0xFFFF) << 16), (uint32_t)(bits >> 16));
                    }
                }
            }
        }
    
    return ok;
}

// the grid-feature scales (colour, endpoint) of a weight image in global memory
template <int ACT>
__device__ __forceinline__ float2 feature_scales(const uint4* img, int ftab) {
    if constexpr (ACT == kActE4M3) {
        const TcLayerConst* t = reinterpret_cast<const TcLayerConst*>(reinterpret_cast<const unsigned char*>(img) + ftab);
        return make_float2(t[0].fscale, t[NTBC_MAX_MLP_LAYERS].fscale);
    }
    return make_float2(kLog2e, kLog2e);
}

template <int ACT, int UB>
__global__ void __launch_bounds__(kTcRows * kTcMaxGroups, 1)
infer_tc_kernel(TcArgs args, const uint4* __restrict__ img, GridSrc csrc, GridSrc esrc, TcOut outs,
                float* __restrict__ e_out, float* __restrict__ c_out) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag[kTcMaxGroups];
    const TcSmem sl = tc_smem_layout(args.img_bytes, args.mv.n_textures, ACT, UB);
    // a launch chained after this one (programmatic dependent launch, chained batches) may start
    // as soon as every CTA of this one is resident: it reads and writes none of this launch's
    // data, and its CTAs take the SMs this launch's CTAs leave at its tail
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (args.start_stamp && blockIdx.x == 0 && threadIdx.x == 0) *args.start_stamp = global_ns();
    for (int i = threadIdx.x; i < args.img_bytes / 16; i += blockDim.x) reinterpret_cast<uint4*>(smem)[i] = img[i];
    load_constants(smem, sl);
    const float2 fs = feature_scales<ACT>(img, args.ftab);
    load_level_constants(args.mv, csrc, esrc, reinterpret_cast<float4*>(smem + sl.lvl_off), fs.x, fs.y);
    TcGroup G = setup_groups(smem, sl, args.groups, &tmem_slot, abort_flag);
    uint32_t phase = 0, region = 0;
    bool ok = true;
    const int n_units = (args.n + UB - 1) / UB;
    int units_done = 0;
    for (int unit = blockIdx.x * args.groups + G.g; unit < n_units && ok; unit += gridDim.x * args.groups) {
        ok = process_unit<ACT, UB>(args, csrc, esrc, outs, e_out, c_out, unit, smem, sl, G, phase, region, abort_flag);
        ++units_done;
    }
    if (args.done && ok && G.r == 0 && units_done > 0) {
        __threadfence();
        if (atomicAdd(args.done, units_done) + units_done == n_units) *args.done_stamp = global_ns();
    }
    teardown_groups(G, args.groups, ok, phase, args.err, tmem_slot);
}

// ---------------------------------------------------------------------------
// batched load-time inference: many materials in one persistent launch
// ---------------------------------------------------------------------------

struct TcMat {
    TcArgs args;
    const uint4* img;
    GridSrc csrc, esrc;
    TcOut outs;
    int first_cta_unit;          // index of this material's first CTA-unit (one unit per group)
    int units;
};

struct TcBatchHeader {
    int n_mats, total_cta_units, groups, img_bytes, max_textures, ub;
    int* done;                   // [n_mats] units completed
    unsigned long long* stamps;  // [n_mats + 1]: kernel start, then each material's completion (globaltimer, ns)
    int* err;
    int* ticket;                 // work queue: the next CTA-unit to claim
    long long claim_limit;       // claims outside the queue a CTA makes before it gives up
};

// A device work queue of CTA-units (one work unit per warpgroup, all from one material; the
// materials ordered largest first): thread 0 claims the next CTA-unit from the ticket counter
// and the CTA works on it, so CTAs that finish early take more work instead of idling at the
// end of a static share. All groups of a CTA work on the same material, so the weight image
// is reloaded (after a CTA barrier) only when the CTA crosses into the next material. A claim
// outside the queue (a negative ticket: the counter was corrupted) does no work; after
// claim_limit of them the CTA records the error and stops, so a bad counter ends the launch
// with NTBC_ETIMEOUT instead of spinning. A group that gave up keeps claiming with its CTA
// (skipping the work) so that the CTA barriers stay uniform.
template <int ACT, int UB>
__global__ void __launch_bounds__(kTcRows * kTcMaxGroups, 1)
infer_tc_batch_kernel(TcBatchHeader hdr, const TcMat* __restrict__ mats) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag[kTcMaxGroups];
    __shared__ TcMat cur;
    __shared__ int claim[2];
    if (blockIdx.x == 0 && threadIdx.x == 0) hdr.stamps[0] = global_ns();
    const TcSmem sl = tc_smem_layout(hdr.img_bytes, hdr.max_textures, ACT, UB);
    load_constants(smem, sl);
    TcGroup G = setup_groups(smem, sl, hdr.groups, &tmem_slot, abort_flag);
    uint32_t phase = 0, region = 0;
    bool ok = true;
    int m = -1;
    long long bad = 0;
    for (int it = 0;; ++it) {
        // double-buffered by iteration: the slot written here was last read before the
        // previous iteration's barrier
        if (threadIdx.x == 0) claim[it & 1] = atomicAdd(hdr.ticket, 1);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const int j = claim[it & 1];
        if (j >= hdr.total_cta_units) break;
        if (j < 0) {
            if (++bad >= hdr.claim_limit) {
                if (threadIdx.x == 0) atomicExch(hdr.err, 1);
                break;
            }
            continue;
        }
        int mj = m < 0 ? 0 : m;
        while (mj + 1 < hdr.n_mats && mats[mj + 1].first_cta_unit <= j) ++mj;
        if (mj != m) {                                   // uniform across the CTA
            if (threadIdx.x == 0) cur = mats[mj];
            __syncthreads();
            for (int i = threadIdx.x; i < cur.args.img_bytes / 16; i += blockDim.x)
                reinterpret_cast<uint4*>(smem)[i] = cur.img[i];
            const float2 fs = feature_scales<ACT>(cur.img, cur.args.ftab);
            load_level_constants(cur.args.mv, cur.csrc, cur.esrc, reinterpret_cast<float4*>(smem + sl.lvl_off), fs.x, fs.y);
            proxy_fence();
            __syncthreads();
            tc_fence_after();
            m = mj;
        }
        int unit = (j - cur.first_cta_unit) * hdr.groups + G.g;
        if (ok && unit < cur.units) {
            ok = process_unit<ACT, UB>(cur.args, cur.csrc, cur.esrc, cur.outs, nullptr, nullptr, unit, smem, sl, G, phase,
                                     region, abort_flag);
            if (ok && G.r == 0) {
                __threadfence();
                if (atomicAdd(&hdr.done[m], 1) + 1 == cur.units) hdr.stamps[m + 1] = global_ns();
            }
        }
    }
    teardown_groups(G, hdr.groups, ok, phase, hdr.err, tmem_slot);
}

// ---------------------------------------------------------------------------
// bounded-wait probe: an mbarrier that expects one arrival that never comes, polled with the
// waits of the tensor-core kernels under a given poll limit; records that the wait gave up
// and how long it took (the failure path of every MMA wait, without any GPU fault)
// ---------------------------------------------------------------------------

__global__ void wait_probe_kernel(long long polls, int* __restrict__ gave_up, unsigned long long* __restrict__ ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = global_ns();
        const bool done = mbar_wait(&bar, 0, polls);
        *ns = global_ns() - t0;
        *gave_up = done ? 0 : 1;
    }
}

// ---------------------------------------------------------------------------
// exp2 throughput probe: the MUFU peak of the inference roofline, measured on the device the
// library runs on (every thread runs 8 independent chains x = 2^-x, one ex2.approx per step)
// ---------------------------------------------------------------------------

constexpr int kEx2Chains = 8;

__global__ void ex2_rate_kernel(float* __restrict__ out, int iters) {
    float a[kEx2Chains];
#pragma unroll
    for (int k = 0; k < kEx2Chains; ++k) a[k] = 0.5f + 0.01f * (float)k + 1e-7f * (float)threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kEx2Chains; ++k)
            asm volatile("{\n\t.reg .f32 t;\n\tneg.f32 t, %0;\n\tex2.approx.ftz.f32 %0, t;\n\t}" : "+f"(a[k]));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kEx2Chains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ---------------------------------------------------------------------------
// weight image: every layer's B tile [N][K] (FP16, core-matrix layout) with the
// bias in column `in` (layer 0) or column 64 (the extra K block of later layers)
// ---------------------------------------------------------------------------

// Every element of every tile is written (weights, the bias column, zeros elsewhere); only the
// padding behind the last tile is zeroed separately, so any number of CTAs can share the work.
__global__ void build_image_kernel(const float* __restrict__ params, TcArgs args, ModelView mv, __half* __restrict__ img) {
    const TcNet& last_net = args.net[1];
    const TcLayer& last = last_net.layer[last_net.n_layers - 1];
    const int tiles_end = (last.img + last.N * last.K * 2) / 2, total = args.img_bytes / 2;
    for (int e = tiles_end + blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x)
        img[e] = __float2half(0.f);
    // one pass per (net, layer): element (n, k)
    for (int net = 0; net < 2; ++net) {
        const NetView& nv = net ? mv.endpoint : mv.color;
        const TcNet& tn = args.net[net];
        for (int l = 0; l < tn.n_layers; ++l) {
            const TcLayer& L = tn.layer[l];
            int in = nv.layer_in[l], out = nv.layer_out[l];
            int bias_col = l == 0 ? in : 64;
            for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L.N * L.K; e += gridDim.x * blockDim.x) {
                int n = e / L.K, k = e % L.K;
                float v = 0.f;
                if (n < out && k < in) v = params[nv.w_off[l] + (long long)n * in + k];
                else if (n < out && k == bias_col) v = params[nv.b_off[l] + n];
                img[(L.img + core_byte(n, k, L.K)) / 2] = __float2half(v);
            }
        }
    }
}

// E4M3 weight image: every layer's B tile [N][K] of E4M3 codes (core-matrix layout, K = 32
// for layer 0, 64 after it; no bias column), then per layer N FP32 values b L, then the
// TcLayerConst table. Every byte up to the end of the table is written by the kernel.
__global__ void build_image8_kernel(const uint8_t* __restrict__ codes, const float* __restrict__ params,
                                    const int* __restrict__ wexp, const int* __restrict__ aexp, long long grid_floats,
                                    TcArgs args, ModelView mv, uint8_t* __restrict__ img) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const int used = args.ftab + 2 * NTBC_MAX_MLP_LAYERS * (int)sizeof(TcLayerConst);
    for (int e = used + tid; e < args.img_bytes; e += nth) img[e] = 0;
    for (int net = 0; net < 2; ++net) {
        const NetView& nv = net ? mv.endpoint : mv.color;
        const TcNet& tn = args.net[net];
        for (int l = 0; l < tn.n_layers; ++l) {
            const TcLayer& L = tn.layer[l];
            const int in = nv.layer_in[l], out = nv.layer_out[l];
            for (int e = tid; e < L.N * L.K; e += nth) {
                const int n = e / L.K, k = e % L.K;
                img[L.img + core_byte8(n, k, L.K)] = n < out && k < in ? codes[nv.w_off[l] - grid_floats + (long long)n * in + k] : 0;
            }
            // ReLU hidden layers work on z 2^-a' directly (bias b 2^-a', exact), every other
            // layer on z L (bias b L)
            const bool relu_hidden = mv.activation == NTBC_ACT_RELU && l + 1 < tn.n_layers;
            const int i_next = net * tn.n_layers + l + 1;
            float* b = reinterpret_cast<float*>(img + L.bias);
            for (int n = tid; n < L.N; n += nth) {
                const float bq = n < out ? params[nv.b_off[l] + n] : 0.f;
                b[n] = relu_hidden ? ldexpf(bq, -aexp[i_next]) : bq * kLog2e;
            }
        }
    }
    // layer i = net * layers + l of the exponent lists (colour layers, then endpoint layers)
    if (tid < 2 * NTBC_MAX_MLP_LAYERS) {
        const int net = tid / NTBC_MAX_MLP_LAYERS, l = tid % NTBC_MAX_MLP_LAYERS, nl = args.net[net].n_layers;
        TcLayerConst c{0.f, 0.f, 0.f, 0.f};
        if (l < nl) {
            const int i = net * nl + l;
            c.s = ldexpf(kLog2e, aexp[i] + wexp[i]);
            if (l == 0) c.fscale = ldexpf(1.f, -aexp[i]);
            if (l + 1 < nl) {
                if (mv.activation == NTBC_ACT_SELU) {
                    c.c1 = ldexpf(kSeluLambda / kLog2e, -aexp[i + 1]);
                    c.c2 = ldexpf(kSeluLA, -aexp[i + 1]);
                } else {                 // ReLU: max(acc 2^(a + w - a') + b 2^-a', 0), all scalings exact
                    c.s = ldexpf(1.f, aexp[i] + wexp[i] - aexp[i + 1]);
                    c.c1 = 1.f;
                }
            }
        }
        reinterpret_cast<TcLayerConst*>(img + args.ftab)[tid] = c;
    }
}

static int tc_act(const ntbc_model* m) {
    if (m->weight_prec == NTBC_PREC_FP16_FAST) return kActF16;
    return m->weight_prec == NTBC_PREC_FP8_MMA ? kActE4M3 : kActSplit;      // FP16 and FP8-storage: split
}

static TcArgs tc_args(const ntbc_model* m) {
    TcArgs a;
    memset(&a, 0, sizeof(a));
    a.mv = make_view(m->desc, m->layout);
    a.act = tc_act(m);
    const bool f8 = a.act == kActE4M3;
    int off = 0;
    for (int net = 0; net < 2; ++net) {
        const NetView& nv = net ? a.mv.endpoint : a.mv.color;
        TcNet& tn = a.net[net];
        tn.n_layers = nv.n_layers;
        for (int l = 0; l < nv.n_layers; ++l) {
            TcLayer& L = tn.layer[l];
            if (f8)
                L.K = l == 0 ? 2 * NTBC_MAX_LEVELS : 64;             // in_dim <= 2 NTBC_MAX_LEVELS = 32
            else
                L.K = l == 0 ? ((nv.in_dim + 1 + 15) / 16) * 16 : 64 + 16;
            L.out = nv.layer_out[l];
            L.N = ((L.out + 15) / 16) * 16;
            L.img = off;
            off += L.N * L.K * tc_a_bytes(a.act);
        }
    }
    if (f8) {
        for (int net = 0; net < 2; ++net)
            for (int l = 0; l < a.net[net].n_layers; ++l) {
                a.net[net].layer[l].bias = off;
                off += a.net[net].layer[l].N * 4;
            }
        a.ftab = off;
        off += 2 * NTBC_MAX_MLP_LAYERS * (int)sizeof(TcLayerConst);
    }
    a.img_bytes = (off + 15) & ~15;
    a.inv_w = 1.f / (float)a.mv.width;
    a.inv_h = 1.f / (float)a.mv.height;
    a.inv_bw = 1.f / (float)a.mv.bw;
    a.inv_bh = 1.f / (float)a.mv.bh;
    return a;
}

// The tensor-core gather takes floor(p) for p = t (res - 1) without clamping it to res - 2:
// true when the largest texel or block centre coordinate t_max (computed in FP32 as the kernel
// does) keeps p below res - 1, which holds unless (res - 1) / extent falls under FP32 rounding
// of res - 1. Checked for every level of both grids before a launch.
static bool floor_in_range(const NetView& nv, int extent, float inv) {
    const float t_max = ((float)(extent - 1) + 0.5f) * inv;
    for (int l = 0; l < nv.levels; ++l) {
        const float p = t_max * nv.resm1[l];
        if (!(std::floor(p) <= (float)(nv.res[l] - 2))) return false;
    }
    return true;
}

static bool tc_coords_ok(const TcArgs& a) {
    return floor_in_range(a.mv.color, a.mv.width, a.inv_w) && floor_in_range(a.mv.color, a.mv.height, a.inv_h) &&
           floor_in_range(a.mv.endpoint, a.mv.bw, a.inv_bw) && floor_in_range(a.mv.endpoint, a.mv.bh, a.inv_bh);
}

// static_bytes: the kernel's static shared variables (the batch kernel keeps a copy of
// the current material's launch description). Returns the warpgroups per CTA and sets the
// work-unit size: 128 blocks, unless 64-block units (half the palette space) fit more groups.
static int tc_groups_ub(const TcArgs& a, int n_tex, int act, int ub, size_t* smem_bytes, size_t static_bytes) {
    for (int groups = kTcMaxGroups; groups >= 1; --groups) {
        TcSmem sl = tc_smem_layout(a.img_bytes, n_tex, act, ub);
        size_t bytes = (size_t)sl.group_off + (size_t)groups * sl.group_bytes;
        if (bytes + static_bytes <= 227 * 1024) {
            // more than two groups allocate all 512 TMEM columns: ask for enough shared
            // memory that a second CTA never lands on the SM and stalls in tcgen05.alloc
            if (groups > 2) bytes = std::max(bytes, (size_t)116 * 1024);
            *smem_bytes = bytes;
            return groups;
        }
    }
    return 0;
}

static int tc_groups(const TcArgs& a, int n_tex, int act, size_t* smem_bytes, int* ub, size_t static_bytes = 256) {
    size_t s128 = 0, s64 = 0;
    const int g128 = tc_groups_ub(a, n_tex, act, kTcUnitBlocks, &s128, static_bytes);
    const int g64 = g128 == kTcMaxGroups ? 0 : tc_groups_ub(a, n_tex, act, kTcUnitBlocks / 2, &s64, static_bytes);
    if (g64 > g128) {
        *smem_bytes = s64;
        *ub = kTcUnitBlocks / 2;
        return g64;
    }
    *smem_bytes = s128;
    *ub = kTcUnitBlocks;
    return g128;
}

ntbc_status tc_prepare(ntbc_model* m, cudaStream_t s) {
    TcArgs a = tc_args(m);
    const size_t need = (size_t)a.img_bytes + sizeof(int) * 4;
    if (m->umma_img && m->umma_bytes < need) {          // an export with a larger image (FP16 after E4M3)
        NTBC_CHECK_CUDA(cudaFree(m->umma_img));         // waits for work still reading it
        m->umma_img = nullptr;
    }
    if (!m->umma_img) {
        ntbc_status st = device_alloc((void**)&m->umma_img, need, "tensor-core weight image");
        if (st != NTBC_OK) return st;
        m->umma_bytes = need;
    }
    m->tc_err = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(m->umma_img) + a.img_bytes);
    NTBC_CHECK_CUDA(cudaMemsetAsync(m->tc_err, 0, sizeof(int), s));
    if (a.act == kActE4M3)
        build_image8_kernel<<<32, 256, 0, s>>>(m->w8, m->infer_params, m->w8_exp, m->w8_aexp, (long long)m->layout.grid_floats,
                                               a, a.mv, reinterpret_cast<uint8_t*>(m->umma_img));
    else
        build_image_kernel<<<32, 256, 0, s>>>(m->infer_params, a, a.mv, m->umma_img);
    NTBC_CHECK_LAUNCH("tensor-core weight image");
    return NTBC_OK;
}

using TcKernel = void (*)(TcArgs, const uint4*, GridSrc, GridSrc, TcOut, float*, float*);
using TcBatchKernel = void (*)(TcBatchHeader, const TcMat*);

// the kernel instance for an A-operand format and a work-unit size (128 or 64 blocks)
static TcKernel tc_kernel(int act, int ub) {
    const bool half = ub != kTcUnitBlocks;
    if (act == kActE4M3) return half ? infer_tc_kernel<kActE4M3, kTcUnitBlocks / 2> : infer_tc_kernel<kActE4M3, kTcUnitBlocks>;
    if (act == kActSplit) return half ? infer_tc_kernel<kActSplit, kTcUnitBlocks / 2> : infer_tc_kernel<kActSplit, kTcUnitBlocks>;
    return half ? infer_tc_kernel<kActF16, kTcUnitBlocks / 2> : infer_tc_kernel<kActF16, kTcUnitBlocks>;
}

static TcBatchKernel tc_batch_kernel(int act, int ub) {
    const bool half = ub != kTcUnitBlocks;
    if (act == kActE4M3)
        return half ? infer_tc_batch_kernel<kActE4M3, kTcUnitBlocks / 2> : infer_tc_batch_kernel<kActE4M3, kTcUnitBlocks>;
    if (act == kActSplit)
        return half ? infer_tc_batch_kernel<kActSplit, kTcUnitBlocks / 2> : infer_tc_batch_kernel<kActSplit, kTcUnitBlocks>;
    return half ? infer_tc_batch_kernel<kActF16, kTcUnitBlocks / 2> : infer_tc_batch_kernel<kActF16, kTcUnitBlocks>;
}

int tc_units_in_flight(const ntbc_model* m, int* unit_blocks) {
    TcArgs a = tc_args(m);
    size_t smem = 0;
    int ub = kTcUnitBlocks;
    const int groups = tc_groups(a, m->desc.n_textures, a.act, &smem, &ub);
    if (unit_blocks) *unit_blocks = ub;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return groups * sms;
}

// One planned launch of the single-material kernel (grid 0: nothing to do).
struct TcLaunch {
    TcKernel kernel;
    TcArgs a;
    const uint4* img;
    GridSrc csrc, esrc;
    TcOut outs;
    float* e_out;
    float* c_out;
    int grid, block;
    size_t smem;
};

// ub_force: 0 for the unit size tc_groups picks, or kTcUnitBlocks / 2
static ntbc_status tc_plan(const ntbc_model* m, uint8_t* const* blocks_out, const int* strides, const int32_t* ids, int n,
                           float* e_out, float* c_out, const GridSrc& csrc, const GridSrc& esrc, TcLaunch* L,
                           int ub_force = 0) {
    TcArgs a = tc_args(m);
    size_t smem = 0;
    if (ub_force) {
        a.ub = ub_force;
        a.groups = tc_groups_ub(a, m->desc.n_textures, a.act, ub_force, &smem, 256);
    } else {
        a.groups = tc_groups(a, m->desc.n_textures, a.act, &smem, &a.ub);
    }
    if (a.groups == 0) return fail(NTBC_EUNSUPPORTED, "tensor-core inference: shared memory too small for this model");
    if (!tc_coords_ok(a)) return fail(NTBC_EUNSUPPORTED, "tensor-core inference: a grid level is too fine for the texture extent");
    a.n = n;
    a.ids = ids;
    a.mode = blocks_out ? 0 : 1;
    a.err = m->tc_err;
    memset(&L->outs, 0, sizeof(L->outs));
    if (blocks_out)
        for (int t = 0; t < m->desc.n_textures; ++t) {
            L->outs.p[t] = blocks_out[t];
            L->outs.stride[t] = strides ? strides[t] : 8;
        }
    int dev = 0, sms = 0;
    NTBC_CHECK_CUDA(cudaGetDevice(&dev));
    NTBC_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int units = (n + a.ub - 1) / a.ub;
    L->grid = std::max(0, std::min(sms, (units + a.groups - 1) / a.groups));
    L->block = kTcRows * a.groups;
    L->smem = smem;
    L->kernel = tc_kernel(a.act, a.ub);
    L->img = reinterpret_cast<const uint4*>(m->umma_img);
    L->csrc = csrc;
    L->esrc = esrc;
    L->e_out = e_out;
    L->c_out = c_out;
    L->a = a;
    if (L->grid > 0) NTBC_CHECK_CUDA(ensure_dynamic_smem(reinterpret_cast<const void*>(L->kernel), smem));
    return NTBC_OK;
}

// chained: a programmatic dependent launch, which may start while the previous kernel on the
// stream (a launch of this kernel that reads and writes none of this one's data) is finishing
static cudaError_t tc_enqueue(const TcLaunch& L, cudaStream_t s, bool chained) {
    if (L.grid < 1) return cudaSuccess;
    if (!chained) {
        L.kernel<<<L.grid, L.block, L.smem, s>>>(L.a, L.img, L.csrc, L.esrc, L.outs, L.e_out, L.c_out);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(L.grid);
    cfg.blockDim = dim3(L.block);
    cfg.dynamicSmemBytes = L.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, L.kernel, L.a, L.img, L.csrc, L.esrc, L.outs, L.e_out, L.c_out);
}

// blocks of a planned launch that go to its full rounds (n when the launch is not split)
static int tc_split_head(const TcLaunch& L, int n, int sms) {
    const int per_round = L.grid * L.a.groups;
    const int units = (n + L.a.ub - 1) / L.a.ub;
    return L.grid == sms && L.a.ub == kTcUnitBlocks && per_round > 0 ? units / per_round * per_round * L.a.ub : n;
}

// The units of one launch run in rounds of (grid x groups); when the grid is full and the last
// round is partial, that round's blocks go to a second launch in half-size units (chained by
// programmatic dependent launch, so its CTAs take the SMs the first launch's CTAs leave): the
// tail then takes about half a unit's time at nearly full occupancy instead of a whole unit's
// time on part of the SMs.
ntbc_status tc_launch(const ntbc_model* m, uint8_t* const* blocks_out, const int* strides, const int32_t* ids, int n,
                      float* e_out, float* c_out, const GridSrc& csrc, const GridSrc& esrc, cudaStream_t s,
                      bool chained) {
    TcLaunch L;
    ntbc_status st = tc_plan(m, blocks_out, strides, ids, n, e_out, c_out, csrc, esrc, &L);
    if (st != NTBC_OK) return st;
    int dev = 0, sms = 0;
    NTBC_CHECK_CUDA(cudaGetDevice(&dev));
    NTBC_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int head = tc_split_head(L, n, sms);
    if (head > 0 && head < n) {
        TcLaunch T;
        const int rest = n - head;
        st = tc_plan(m, blocks_out, strides, ids ? ids + head : nullptr, rest,
                     e_out ? e_out + (size_t)head * L.a.mv.endpoint.out_dim : nullptr,
                     c_out ? c_out + (size_t)head * 16 * L.a.mv.color.out_dim : nullptr, csrc, esrc, &T, kTcUnitBlocks / 2);
        if (st != NTBC_OK) return st;
        if (!ids) T.a.first = head;
        L.a.n = head;
        NTBC_CHECK_CUDA(tc_enqueue(L, s, chained));
        NTBC_CHECK_CUDA(tc_enqueue(T, s, true));
    } else {
        NTBC_CHECK_CUDA(tc_enqueue(L, s, chained));
    }
    NTBC_CHECK_LAUNCH("ntbc inference (tcgen05)");
    return NTBC_OK;
}

}  // namespace ntbc

struct ntbc_batch {
    int n = 0, groups = 0, grid = 0;
    int mode = NTBC_BATCH_CHAINED;
    int act = ntbc::kActSplit;
    size_t smem = 0;
    ntbc::TcBatchHeader hdr{};
    ntbc::TcMat* d_mats = nullptr;      // work-queue mode: the materials' launch descriptions
    std::vector<ntbc::TcLaunch> chain;  // chained mode: one planned launch per material
    unsigned char* d_mem = nullptr;     // stamps, done counters, error flag, ticket counter
    std::vector<int> order;             // queue position -> the caller's material index
};

namespace ntbc {

static cudaError_t batch_set_smem(const ntbc_batch* b) {
    return ensure_dynamic_smem(reinterpret_cast<const void*>(tc_batch_kernel(b->act, b->hdr.ub)), b->smem);
}

static ntbc_status batch_fail_free(ntbc_batch* b, ntbc_status st) {
    if (b) {
        cudaFree(b->d_mats);
        cudaFree(b->d_mem);
        delete b;
    }
    return st;
}

}  // namespace ntbc

extern "C" {

ntbc_status ntbc_wait_probe(long long polls, double* seconds, void* stream) {
    using namespace ntbc;
    clear_error();
    if (polls < 1 || polls > ntbc::kTcWaitLimit) return fail(NTBC_EINVAL, "polls must be 1..%lld", ntbc::kTcWaitLimit);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* d = nullptr;
    ntbc_status st = device_alloc((void**)&d, 2 * sizeof(unsigned long long), "wait probe");
    if (st != NTBC_OK) return st;
    ntbc::wait_probe_kernel<<<1, 32, 0, s>>>(polls, reinterpret_cast<int*>(d + 1), d);
    cudaError_t e = cudaGetLastError();
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "wait probe");
    const double sec = (double)h[0] * 1e-9;
    if (seconds) *seconds = sec;
    const int gave_up = *reinterpret_cast<const int*>(&h[1]);
    if (gave_up) return fail(NTBC_ETIMEOUT, "bounded wait gave up after %lld polls (%.3f s)", polls, sec);
    return NTBC_OK;
}

ntbc_status ntbc_infer_plan(const ntbc_model* m, int* launches, int* unit_blocks, int* units_in_flight) {
    using namespace ntbc;
    clear_error();
    if (!m || !launches || !unit_blocks || !units_in_flight) return fail(NTBC_EINVAL, "null argument");
    if (m->grid_bits < 0) return fail(NTBC_EINVAL, "model has not been exported (call ntbc_model_export or ntbc_model_load)");
    *launches = 1;
    *unit_blocks = 0;
    *units_in_flight = 0;
    if (m->weight_prec == NTBC_PREC_FP32) return NTBC_OK;             // the SIMT kernel: one launch
    const int n = (m->desc.width / 4) * (m->desc.height / 4);
    GridSrc csrc, esrc;
    ntbc_status st = grid_sources(m, csrc, esrc);
    if (st != NTBC_OK) return st;
    TcLaunch L;
    st = tc_plan(m, nullptr, nullptr, nullptr, n, nullptr, nullptr, csrc, esrc, &L);
    if (st != NTBC_OK) return st;
    int dev = 0, sms = 0;
    NTBC_CHECK_CUDA(cudaGetDevice(&dev));
    NTBC_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int head = tc_split_head(L, n, sms);
    *launches = head > 0 && head < n ? 2 : 1;
    *unit_blocks = L.a.ub;
    *units_in_flight = L.grid * L.a.groups;
    return NTBC_OK;
}

ntbc_status ntbc_ex2_rate_probe(double* ex2_per_s, void* stream) {
    using namespace ntbc;
    clear_error();
    if (!ex2_per_s) return fail(NTBC_EINVAL, "null output");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    NTBC_CHECK_CUDA(cudaGetDevice(&dev));
    NTBC_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256, iters = 4096, reps = 5;
    float* d = nullptr;
    ntbc_status st = device_alloc((void**)&d, (size_t)blocks * threads * sizeof(float), "exp2 probe");
    if (st != NTBC_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int w = 0; w < 3 && e == cudaSuccess; ++w) {
        ntbc::ex2_rate_kernel<<<blocks, threads, 0, s>>>(d, iters);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        ntbc::ex2_rate_kernel<<<blocks, threads, 0, s>>>(d, iters);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "exp2 probe");
    *ex2_per_s = (double)blocks * threads * iters * ntbc::kEx2Chains * reps / ((double)ms * 1e-3);
    return NTBC_OK;
}

ntbc_status ntbc_batch_create(const ntbc_model* const* models, int n, uint8_t* const* const* blocks_out, ntbc_batch** out) {
    return ntbc_batch_create_mode(models, n, blocks_out, NTBC_BATCH_CHAINED, out);
}

ntbc_status ntbc_batch_create_mode(const ntbc_model* const* models, int n, uint8_t* const* const* blocks_out, int mode,
                                   ntbc_batch** out) {
    using namespace ntbc;
    clear_error();
    if (!models || !blocks_out || !out || n <= 0) return fail(NTBC_EINVAL, "need models, outputs and n > 0");
    if (mode != NTBC_BATCH_CHAINED && mode != NTBC_BATCH_QUEUE) return fail(NTBC_EINVAL, "unknown batch mode %d", mode);
    *out = nullptr;
    int prec = -1, max_tex = 0, max_img = 0, total = 0;
    std::vector<TcMat> mats(n);
    for (int i = 0; i < n; ++i) {
        const ntbc_model* m = models[i];
        if (!m || !blocks_out[i]) return fail(NTBC_EINVAL, "material %d: null model or output list", i);
        if (m->weight_prec == NTBC_PREC_FP32 || m->grid_bits < 0 || !m->umma_img)
            return fail(NTBC_EINVAL, "material %d: export the model with a tensor-core precision first", i);
        const int kind = tc_act(m);
        if (mode == NTBC_BATCH_QUEUE && prec >= 0 && kind != prec)
            return fail(NTBC_EINVAL, "all materials of a work-queue batch need the same tensor-core kernel");
        prec = kind;
        TcMat& t = mats[i];
        memset(&t, 0, sizeof(t));
        t.args = tc_args(m);
        if (!tc_coords_ok(t.args)) return fail(NTBC_EUNSUPPORTED, "material %d: a grid level is too fine for the texture extent", i);
        t.args.n = (m->desc.width / 4) * (m->desc.height / 4);
        t.args.mode = 0;
        t.img = reinterpret_cast<const uint4*>(m->umma_img);
        ntbc_status st = grid_sources(m, t.csrc, t.esrc);
        if (st != NTBC_OK) return st;
        for (int k = 0; k < m->desc.n_textures; ++k) {
            uint8_t* o = blocks_out[i][k];
            if (!o || (reinterpret_cast<uintptr_t>(o) & 7)) return fail(NTBC_EINVAL, "material %d texture %d: output null or not 8-byte aligned", i, k);
            t.outs.p[k] = o;
            t.outs.stride[k] = 8;
        }
        max_tex = std::max(max_tex, m->desc.n_textures);
        max_img = std::max(max_img, t.args.img_bytes);
    }
    // the materials of a batch are written concurrently: their output ranges must be disjoint
    std::vector<std::pair<uintptr_t, uintptr_t>> ranges;
    for (int i = 0; i < n; ++i) {
        const size_t bytes = (size_t)mats[i].args.n * 8;
        for (int k = 0; k < models[i]->desc.n_textures; ++k) {
            const uintptr_t p0 = reinterpret_cast<uintptr_t>(blocks_out[i][k]);
            ranges.push_back({p0, p0 + bytes});
        }
    }
    std::sort(ranges.begin(), ranges.end());
    for (size_t j = 1; j < ranges.size(); ++j)
        if (ranges[j].first < ranges[j - 1].second) return fail(NTBC_EINVAL, "batch: two outputs overlap");
    // materials largest first: the last work (queue claims, or chained launches) is the small
    // materials', so the SMs finish close together
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return mats[a].args.n > mats[b].args.n; });
    std::vector<TcMat> sorted(n);
    for (int i = 0; i < n; ++i) sorted[i] = mats[order[i]];
    mats.swap(sorted);
    // the models may have been exported on any stream: their images and grids are complete
    // before the batch exists (creation is a one-time set-up call)
    NTBC_CHECK_CUDA(cudaDeviceSynchronize());
    ntbc_batch* b = new ntbc_batch();
    b->n = n;
    b->mode = mode;
    b->order = order;
    b->act = prec;
    // completion stamps (start, then one per material), done counters, error flag, ticket
    size_t mem = (size_t)(n + 1) * sizeof(unsigned long long) + (size_t)(n + 2) * sizeof(int);
    ntbc_status st = device_alloc((void**)&b->d_mem, mem, "batch counters");
    if (st != NTBC_OK) return batch_fail_free(b, st);
    b->hdr.n_mats = n;
    b->hdr.stamps = reinterpret_cast<unsigned long long*>(b->d_mem);
    b->hdr.done = reinterpret_cast<int*>(b->d_mem + (size_t)(n + 1) * sizeof(unsigned long long));
    b->hdr.err = b->hdr.done + n;
    b->hdr.ticket = b->hdr.err + 1;
    b->hdr.claim_limit = 1 << 16;
    cudaError_t e = cudaMemset(b->d_mem, 0, mem);
    if (e != cudaSuccess) return batch_fail_free(b, cuda_fail(e, "batch set-up"));
    if (mode == NTBC_BATCH_CHAINED) {
        // one launch of the single-material kernel per material (each with its own unit size and
        // warpgroup count), chained by programmatic dependent launch
        b->chain.resize(n);
        for (int k = 0; k < n; ++k) {
            const int i = order[k];
            GridSrc csrc, esrc;
            st = grid_sources(models[i], csrc, esrc);
            if (st == NTBC_OK) st = tc_plan(models[i], blocks_out[i], nullptr, nullptr, mats[k].args.n, nullptr, nullptr, csrc, esrc, &b->chain[k]);
            if (st != NTBC_OK) return batch_fail_free(b, st);
            TcArgs& a = b->chain[k].a;
            a.err = b->hdr.err;
            a.done = b->hdr.done + k;
            a.done_stamp = b->hdr.stamps + k + 1;
            a.start_stamp = k == 0 ? b->hdr.stamps : nullptr;
        }
        *out = b;
        return NTBC_OK;
    }
    TcArgs probe;
    memset(&probe, 0, sizeof(probe));
    probe.img_bytes = max_img;
    int ub = kTcUnitBlocks;
    b->groups = tc_groups(probe, max_tex, b->act, &b->smem, &ub, sizeof(TcMat) + 256);
    if (b->groups == 0) return batch_fail_free(b, fail(NTBC_EUNSUPPORTED, "batch: shared memory too small"));
    for (int i = 0; i < n; ++i) {
        mats[i].args.ub = ub;
        mats[i].units = (mats[i].args.n + ub - 1) / ub;
    }
    for (int i = 0; i < n; ++i) {
        mats[i].first_cta_unit = total;
        mats[i].args.groups = b->groups;
        total += (mats[i].units + b->groups - 1) / b->groups;
    }
    st = device_alloc((void**)&b->d_mats, (size_t)n * sizeof(TcMat), "batch descriptors");
    if (st != NTBC_OK) return batch_fail_free(b, st);
    b->hdr.total_cta_units = total;
    b->hdr.groups = b->groups;
    b->hdr.img_bytes = max_img;
    b->hdr.max_textures = max_tex;
    b->hdr.ub = ub;
    for (int i = 0; i < n; ++i) mats[i].args.err = b->hdr.err;
    e = cudaMemcpy(b->d_mats, mats.data(), (size_t)n * sizeof(TcMat), cudaMemcpyHostToDevice);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = batch_set_smem(b);
    if (e != cudaSuccess) return batch_fail_free(b, cuda_fail(e, "batch set-up"));
    b->grid = std::min(sms, total);
    *out = b;
    return NTBC_OK;
}

ntbc_status ntbc_batch_infer(ntbc_batch* b, void* stream) {
    ntbc::NvtxRange nvtx_range("ntbc_batch_infer");
    using namespace ntbc;
    clear_error();
    if (!b) return fail(NTBC_EINVAL, "null batch");
    cudaStream_t s = (cudaStream_t)stream;
    // completion counters, the error flag and the ticket counter start at zero every launch;
    // NTBC_FAULT=ticket corrupts the ticket counter instead (a negative start), which the
    // kernel's bounded claim loop turns into NTBC_ETIMEOUT
    NTBC_CHECK_CUDA(cudaMemsetAsync(b->hdr.done, 0, (size_t)(b->n + 2) * sizeof(int), s));
    if (b->mode == NTBC_BATCH_CHAINED) {
        // the first launch follows the reset in stream order; each later one may start while its
        // predecessor's last CTAs finish
        for (int k = 0; k < b->n; ++k) NTBC_CHECK_CUDA(tc_enqueue(b->chain[k], s, k > 0));
        NTBC_CHECK_LAUNCH("chained ntbc inference (tcgen05)");
        return NTBC_OK;
    }
    if (fault_injected("ticket")) NTBC_CHECK_CUDA(cudaMemsetAsync(b->hdr.ticket, 0x80, sizeof(int), s));
    const TcBatchKernel kernel = tc_batch_kernel(b->act, b->hdr.ub);
    kernel<<<dim3(b->grid), dim3(kTcRows * b->groups), b->smem, s>>>(b->hdr, b->d_mats);
    NTBC_CHECK_LAUNCH("batched ntbc inference (tcgen05)");
    return NTBC_OK;
}

ntbc_status ntbc_batch_times(const ntbc_batch* b, double* ms, void* stream) {
    using namespace ntbc;
    clear_error();
    if (!b || !ms) return fail(NTBC_EINVAL, "null argument");
    NTBC_CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    std::vector<unsigned long long> st(b->n + 1);
    int err = 0;
    NTBC_CHECK_CUDA(cudaMemcpy(st.data(), b->hdr.stamps, st.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    NTBC_CHECK_CUDA(cudaMemcpy(&err, b->hdr.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) return fail(NTBC_ETIMEOUT, "a bounded wait or the bounded work-queue claim loop of the batched inference gave up");
    for (int i = 0; i < b->n; ++i) ms[b->order[i]] = st[i + 1] >= st[0] ? (double)(st[i + 1] - st[0]) * 1e-6 : -1.0;
    return NTBC_OK;
}

void ntbc_batch_free(ntbc_batch* b) { ntbc::batch_fail_free(b, NTBC_OK); }

}  // extern "C"
