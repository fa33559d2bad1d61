// Internal declarations shared by the CUDA translation units of libntbc.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "../../include/ntbc.h"

namespace ntbc {

// ---------------------------------------------------------------------------
// host-side error plumbing
// ---------------------------------------------------------------------------

ntbc_status fail(ntbc_status st, const char* fmt, ...);
ntbc_status cuda_fail(cudaError_t err, const char* what);
void clear_error();
bool fault_injected(const char* what);   // NTBC_FAULT=alloc|launch|... host-side fault injection

#define NTBC_CHECK_CUDA(expr)                                  \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) return ::ntbc::cuda_fail(_e, #expr); \
    } while (0)

#define NTBC_CHECK_LAUNCH(what)                                            \
    do {                                                                   \
        if (::ntbc::fault_injected("launch"))                              \
            return ::ntbc::fail(NTBC_ECUDA, "injected launch failure: %s", what); \
        cudaError_t _e = cudaGetLastError();                               \
        if (_e != cudaSuccess) return ::ntbc::cuda_fail(_e, what);         \
    } while (0)

ntbc_status device_alloc(void** ptr, size_t bytes, const char* what);

// NVTX range over one C-ABI call (host timeline of a profiler; the NVTX v3 calls are no-ops
// unless a tool is attached)
// cudaFuncAttributeMaxDynamicSharedMemorySize belongs to a kernel instance, process-wide: it is
// only ever raised (to the largest size any launch or batch of that instance has asked for on
// this device), so a later, smaller request never invalidates a batch created earlier
inline cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> granted;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = granted[{dev, fn}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

inline int channels_of(int fmt) { return fmt == NTBC_BC1 ? 3 : (fmt == NTBC_BC4 ? 1 : 0); }

ntbc_status check_texture_args(int fmt, const void* a, const void* b, int w, int h);

// ---------------------------------------------------------------------------
// model state
// ---------------------------------------------------------------------------

constexpr int kHidden = NTBC_HIDDEN_WIDTH;
constexpr int kMaxIn = 32;              // features * levels, padded
constexpr int kMaxOutC = 24;            // colour outputs (3 per BC1, 1 per BC4)
constexpr int kMaxOutE = 48;            // endpoint outputs

}  // namespace ntbc

struct ntbc_model {
    ntbc_model_desc desc;
    ntbc_layout layout;
    float* params = nullptr;            // FP32 master parameters [layout.total]
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    // exported (inference) form
    int grid_bits = -1;                 // -1: not exported; 0: FP32 grids; 8 / 4: codes
    int weight_prec = NTBC_PREC_FP32;
    uint8_t* qgrid = nullptr;           // codes [layout.grid_floats]
    float* qscale = nullptr;            // [color_levels + endpoint_levels]
    float* qzero = nullptr;
    float* infer_params = nullptr;      // FP32 copy used by inference: FP32 grids (grid_bits 0)
                                        // and the MLP weights rounded to the export precision
    __half* w16 = nullptr;              // MLP part in FP16 (weight_prec FP16, and FP8 expanded)
    uint8_t* w8 = nullptr;              // MLP part as E4M3 codes (weight_prec FP8 / FP8_MMA), then
    int* w8_exp = nullptr;              // the per-layer weight scale exponents, the activation
    int* w8_aexp = nullptr;             // scale exponents (FP8_MMA) and the calibration maxima
    unsigned* w8_amax = nullptr;        // (all inside the w8 allocation)
    __half* umma_img = nullptr;         // weights in the tensor-core shared-memory layout (FP16, or
                                        // E4M3 codes followed by FP32 biases and layer constants)
    size_t umma_bytes = 0;              // its allocation size
    int* tc_err = nullptr;              // set by the tensor-core kernel when a bounded wait gives up
    struct ntbc_train_state* train = nullptr;   // training scratch (allocated on first use)
    long long next_step = 0;            // the encode step a resumed ntbc_train_range starts at
    struct ntbc_host_io* host_io = nullptr;     // staging of ntbc_infer_to_host (allocated on first use)
};

namespace ntbc {

// Kernel-side view of a model (plain pointers and sizes; passed by value).
struct NetView {
    int levels;
    int res[NTBC_MAX_LEVELS];
    float resm1[NTBC_MAX_LEVELS];            // res - 1 and res - 2 as floats
    float resm2[NTBC_MAX_LEVELS];
    long long grid_off[NTBC_MAX_LEVELS];     // element offset of each level in its grid buffer
    int features;
    int in_dim, out_dim, hidden_layers;
    // MLP spans (float offsets inside the parameter buffer)
    long long w_off[NTBC_MAX_MLP_LAYERS], b_off[NTBC_MAX_MLP_LAYERS];
    int layer_in[NTBC_MAX_MLP_LAYERS], layer_out[NTBC_MAX_MLP_LAYERS];
    int n_layers;
};

struct ModelView {
    int width, height, bw, bh, n_textures;
    int formats[NTBC_MAX_TEXTURES];
    int coff[NTBC_MAX_TEXTURES];         // colour output offset per texture
    int eoff[NTBC_MAX_TEXTURES];         // endpoint output offset per texture
    int activation;
    NetView color, endpoint;
};

ModelView make_view(const ntbc_model_desc& d, const ntbc_layout& L);
void host_io_release(ntbc_model* m);

// ---------------------------------------------------------------------------
// device helpers: SELU, sigmoid, BC palettes, packing, output decisions
// ---------------------------------------------------------------------------

constexpr float kSeluLambda = 1.0507009873554804934f;
constexpr float kSeluAlpha = 1.6732632423543772848f;
constexpr float kSeluLA = 1.7580993408473766f;   // lambda * alpha

__device__ __forceinline__ float selu_f(float z) {
    return z > 0.f ? kSeluLambda * z : kSeluLA * expm1f(z);
}
__device__ __forceinline__ float act_f(float z, int act) {
    return act == NTBC_ACT_SELU ? selu_f(z) : fmaxf(z, 0.f);
}
// derivative from the activation's output a: SELU a > 0 -> lambda, else a + lambda*alpha
__device__ __forceinline__ float act_grad_from_out(float a, int act) {
    if (act == NTBC_ACT_SELU) return a > 0.f ? kSeluLambda : a + kSeluLA;
    return a > 0.f ? 1.f : 0.f;
}
__device__ __forceinline__ float sigmoid_f(float z) { return 1.f / (1.f + expf(-z)); }

__device__ __forceinline__ void expand565(uint32_t c, int& r, int& g, int& b) {
    int r5 = (c >> 11) & 31, g6 = (c >> 5) & 63, b5 = c & 31;
    r = (r5 << 3) | (r5 >> 2);
    g = (g6 << 2) | (g6 >> 4);
    b = (b5 << 3) | (b5 >> 2);
}

// BC1 integer palette in hardware-code order, [code][channel]
__device__ __forceinline__ void bc1_palette(uint32_t c0, uint32_t c1, int pal[4][3]) {
    int e0[3], e1[3];
    expand565(c0, e0[0], e0[1], e0[2]);
    expand565(c1, e1[0], e1[1], e1[2]);
    bool four = c0 > c1;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        pal[0][ch] = e0[ch];
        pal[1][ch] = e1[ch];
        pal[2][ch] = four ? (2 * e0[ch] + e1[ch] + 1) / 3 : (e0[ch] + e1[ch] + 1) / 2;
        pal[3][ch] = four ? (e0[ch] + 2 * e1[ch] + 1) / 3 : 0;
    }
}

// BC4 integer palette in hardware-code order
__device__ __forceinline__ void bc4_palette(int r0, int r1, int pal[8]) {
    pal[0] = r0;
    pal[1] = r1;
    if (r0 > r1) {
#pragma unroll
        for (int k = 1; k <= 6; ++k) pal[k + 1] = ((7 - k) * r0 + k * r1 + 3) / 7;
    } else {
#pragma unroll
        for (int k = 1; k <= 4; ++k) pal[k + 1] = ((5 - k) * r0 + k * r1 + 2) / 5;
        pal[6] = 0;
        pal[7] = 255;
    }
}

__device__ __forceinline__ void store_block(uint8_t* dst, uint32_t lo, uint32_t hi) {
    // 8-byte aligned (block index * 8 from a cudaMalloc'd base)
    *reinterpret_cast<uint2*>(dst) = make_uint2(lo, hi);
}

// FP32 quantisation of a predicted endpoint channel: floor(e * levels + 0.5), clamped
__device__ __forceinline__ int quant_channel(float e, float levels, int maxv) {
    float q = floorf(__fadd_rn(__fmul_rn(e, levels), 0.5f));
    q = fminf(fmaxf(q, 0.f), (float)maxv);
    return (int)q;
}

// Decision state of one block of one texture: quantised endpoints and the FP32
// palette of the integer palette / 255 (hardware-code order).
struct BlockPalette {
    uint32_t ep;            // BC1: c0 | c1 << 16 ; BC4: r0 | r1 << 8
    float pal[8][3];        // BC1 uses [0..3][0..2]; BC4 uses [0..7][0]
    bool solid;             // BC1 c0 == c1 -> all codes 0
};

__device__ __forceinline__ void make_palette_bc1(const float* e, BlockPalette& bp) {
    uint32_t c0 = (quant_channel(e[0], 31.f, 31) << 11) | (quant_channel(e[1], 63.f, 63) << 5) |
                  quant_channel(e[2], 31.f, 31);
    uint32_t c1 = (quant_channel(e[3], 31.f, 31) << 11) | (quant_channel(e[4], 63.f, 63) << 5) |
                  quant_channel(e[5], 31.f, 31);
    if (c0 < c1) {
        uint32_t t = c0;
        c0 = c1;
        c1 = t;
    }
    int pal[4][3];
    bc1_palette(c0, c1, pal);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) bp.pal[k][ch] = __fdiv_rn((float)pal[k][ch], 255.f);
    bp.ep = c0 | (c1 << 16);
    bp.solid = (c0 == c1);
}

__device__ __forceinline__ void make_palette_bc4(const float* e, BlockPalette& bp) {
    int r0 = quant_channel(e[0], 255.f, 255);
    int r1 = quant_channel(e[1], 255.f, 255);
    int pal[8];
    bc4_palette(r0, r1, pal);
#pragma unroll
    for (int k = 0; k < 8; ++k) bp.pal[k][0] = __fdiv_rn((float)pal[k], 255.f);
    bp.ep = (uint32_t)r0 | ((uint32_t)r1 << 8);
    bp.solid = false;
}

// least squared FP32 distance, channels summed in order, ties to the lowest code
__device__ __forceinline__ int choose_code_bc1(const BlockPalette& bp, float r, float g, float b) {
    if (bp.solid) return 0;
    int best = 0;
    float bestd = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float dr = __fsub_rn(r, bp.pal[k][0]);
        float dg = __fsub_rn(g, bp.pal[k][1]);
        float db = __fsub_rn(b, bp.pal[k][2]);
        float d = __fadd_rn(__fadd_rn(__fmul_rn(dr, dr), __fmul_rn(dg, dg)), __fmul_rn(db, db));
        if (k == 0 || d < bestd) {
            bestd = d;
            best = k;
        }
    }
    return best;
}

__device__ __forceinline__ int choose_code_bc4(const BlockPalette& bp, float v) {
    int best = 0;
    float bestd = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float dv = __fsub_rn(v, bp.pal[k][0]);
        float d = __fmul_rn(dv, dv);
        if (k == 0 || d < bestd) {
            bestd = d;
            best = k;
        }
    }
    return best;
}

}  // namespace ntbc
