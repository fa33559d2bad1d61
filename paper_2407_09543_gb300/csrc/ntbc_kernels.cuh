// Device code shared by the inference and training translation units:
// level tables, multi-resolution grid lookup, host hooks of the training state.
#pragma once

#include "ntbc_internal.cuh"

namespace ntbc {

constexpr int kMaxAllLevels = 2 * NTBC_MAX_LEVELS;

struct LevelTable {
    int levels;
    long long offset[kMaxAllLevels];
    long long count[kMaxAllLevels];
};

LevelTable level_table(const ntbc_model_desc& d, const ntbc_layout& L);
// per-level QAT scale / zero point
ntbc_status launch_level_scale_zero(const float* grid, const LevelTable& lt, int bits, unsigned* mm, float* scale,
                                    float* zero, cudaStream_t s);

// Where a network's grid comes from.
//   f32:  FP32 features (parameter buffer), optional QAT fake quantisation (qat_bits > 0 with
//         scale / zero per level, Eq. quantizer)
//   codes: exported integer codes with per-level scale / zero (Eq. dequantize after the
//         bilinear interpolation, which is linear)
struct GridSrc {
    const float* f32;
    const uint8_t* codes;
    const float* scale;      // indexed by level (already offset for the network)
    const float* zero;
    int qat_bits;
};

// Corner-aligned bilinear lookup of level l at normalised (u, v):
// p = u (res - 1), i0 = min(floor p, res - 2), f = p - i0.
struct Bilinear {
    long long base;          // element offset of corner (ix, iy) within the level
    int row;                 // elements per grid row (res * 2)
    float w00, w01, w10, w11;
};

__device__ __forceinline__ Bilinear bilinear_at(int res, float u, float v) {
    float px = u * (float)(res - 1);
    float py = v * (float)(res - 1);
    int ix = min((int)floorf(px), res - 2);
    int iy = min((int)floorf(py), res - 2);
    float fx = px - (float)ix, fy = py - (float)iy;
    Bilinear b;
    b.base = ((long long)iy * res + ix) * 2;
    b.row = res * 2;
    b.w00 = (1.f - fx) * (1.f - fy);
    b.w01 = fx * (1.f - fy);
    b.w10 = (1.f - fx) * fy;
    b.w11 = fx * fy;
    return b;
}

__device__ __forceinline__ float fake_quant(float r, float s, float z, float qmax) {
    float q = fminf(fmaxf(roundf(__fdiv_rn(r, s)) + z, 0.f), qmax);
    return s * (q - z);
}

// features of every level, level-major, 2 per level, into out[0 .. 2*levels)
__device__ __forceinline__ void grid_features(const NetView& nv, const GridSrc& src, float u, float v, float* out) {
    const int qat_bits = src.qat_bits;
#pragma unroll
    for (int l = 0; l < NTBC_MAX_LEVELS; ++l) {
        if (l >= nv.levels) break;
        Bilinear b = bilinear_at(nv.res[l], u, v);
        long long o = nv.grid_off[l] + b.base;
        float f0, f1;
        if (src.codes) {
            const uint8_t* g = src.codes + o;
            uchar2 a = *reinterpret_cast<const uchar2*>(g);
            uchar2 c = *reinterpret_cast<const uchar2*>(g + 2);
            uchar2 d = *reinterpret_cast<const uchar2*>(g + b.row);
            uchar2 e = *reinterpret_cast<const uchar2*>(g + b.row + 2);
            float q0 = b.w00 * a.x + b.w01 * c.x + b.w10 * d.x + b.w11 * e.x;
            float q1 = b.w00 * a.y + b.w01 * c.y + b.w10 * d.y + b.w11 * e.y;
            float s = src.scale[l], z = src.zero[l];
            f0 = s * (q0 - z);
            f1 = s * (q1 - z);
        } else {
            const float* g = src.f32 + o;
            float2 a = __ldg(reinterpret_cast<const float2*>(g));
            float2 c = __ldg(reinterpret_cast<const float2*>(g + 2));
            float2 d = __ldg(reinterpret_cast<const float2*>(g + b.row));
            float2 e = __ldg(reinterpret_cast<const float2*>(g + b.row + 2));
            if (qat_bits > 0) {
                float s = src.scale[l], z = src.zero[l], qm = (float)((1 << qat_bits) - 1);
                a.x = fake_quant(a.x, s, z, qm); a.y = fake_quant(a.y, s, z, qm);
                c.x = fake_quant(c.x, s, z, qm); c.y = fake_quant(c.y, s, z, qm);
                d.x = fake_quant(d.x, s, z, qm); d.y = fake_quant(d.y, s, z, qm);
                e.x = fake_quant(e.x, s, z, qm); e.y = fake_quant(e.y, s, z, qm);
            }
            f0 = b.w00 * a.x + b.w01 * c.x + b.w10 * d.x + b.w11 * e.x;
            f1 = b.w00 * a.y + b.w01 * c.y + b.w10 * d.y + b.w11 * e.y;
        }
        out[2 * l] = f0;
        out[2 * l + 1] = f1;
    }
}

void ntbc_train_release(ntbc_model* m);

// grid sources of an exported model (codes + scale / zero, or FP32 grids)
ntbc_status grid_sources(const ntbc_model* m, GridSrc& csrc, GridSrc& esrc);

// per-layer activation exponents of NTBC_PREC_FP8_MMA (into m->w8_aexp) from the calibration
// sample of the exported model (grids and FP8 weights already in place)
ntbc_status fp8_calibrate(ntbc_model* m, cudaStream_t s);

// tensor-core inference (FP16 or FP8 weights): weight image preparation and launch
ntbc_status tc_prepare(ntbc_model* m, cudaStream_t s);
// work units the tensor-core inference processes at once (groups x SMs; 0 on error) and the
// blocks per work unit (unit_blocks, optional)
int tc_units_in_flight(const ntbc_model* m, int* unit_blocks);
// blocks_out: per texture the first block; strides: bytes between its blocks (NULL: 8);
// chained: a programmatic dependent launch, which may start while the previous launch on the
// stream is finishing (only where the two share no data, e.g. the ranges of one material)
ntbc_status tc_launch(const ntbc_model* m, uint8_t* const* blocks_out, const int* strides, const int32_t* ids, int n,
                      float* e_out, float* c_out, const GridSrc& csrc, const GridSrc& esrc, cudaStream_t s,
                      bool chained = false);

}  // namespace ntbc
