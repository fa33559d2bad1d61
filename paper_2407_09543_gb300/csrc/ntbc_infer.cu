// NTBC inference to BC blocks (Sec. 3.2, Fig. NTBC (a); Sec. 4.4): one fused
// launch performs the grid lookup and dequantisation, the endpoint MLP per
// block, the colour MLP per texel, endpoint quantisation, the per-texel argmax
// of -||c_hat - p_n|| and the packing into 8-byte blocks.
//
// This translation unit holds the FP32 SIMT form of the fused kernel: one
// thread owns one block (its endpoint network and its 16 texels), the weights
// of the running network sit in shared memory and each thread keeps a private
// column of shared memory for the 64 hidden activations.
#include "ntbc_internal.cuh"
#include "ntbc_kernels.cuh"

namespace ntbc {

constexpr int kInPad = kMaxIn;          // layer-0 rows padded to 32 inputs
constexpr int kSimtThreads = 128;
constexpr int kPalFloats = 12;          // per texture: BC1 4x3, BC4 8

// Shared-memory image of one network's weights: layer 0 [64][32] zero padded,
// hidden layers [64][64], output [out][64], then the biases.
struct WeightImage {
    int w[NTBC_MAX_MLP_LAYERS], b[NTBC_MAX_MLP_LAYERS], cols[NTBC_MAX_MLP_LAYERS];
    int floats;
};

static WeightImage weight_image(const NetView& nv) {
    WeightImage wi;
    int off = 0;
    for (int l = 0; l < nv.n_layers; ++l) {
        wi.cols[l] = l == 0 ? kInPad : kHidden;
        wi.w[l] = off;
        off += nv.layer_out[l] * wi.cols[l];
    }
    for (int l = 0; l < nv.n_layers; ++l) {
        wi.b[l] = off;
        off += nv.layer_out[l];
    }
    wi.floats = (off + 3) & ~3;
    return wi;
}

__device__ void load_weight_image(const NetView& nv, const WeightImage& wi, const float* __restrict__ params,
                                  float* __restrict__ img) {
    for (int l = 0; l < nv.n_layers; ++l) {
        int rows = nv.layer_out[l], in = nv.layer_in[l], cols = wi.cols[l];
        for (int i = threadIdx.x; i < rows * cols; i += blockDim.x) {
            int r = i / cols, c = i % cols;
            img[wi.w[l] + i] = c < in ? params[nv.w_off[l] + (long long)r * in + c] : 0.f;
        }
        for (int i = threadIdx.x; i < rows; i += blockDim.x) img[wi.b[l] + i] = params[nv.b_off[l] + i];
    }
}

// Evaluate the MLP of one sample. x0: layer-0 input (32, zero padded). The hidden
// activations live in the thread's shared-memory column col[k * stride]; the
// sigmoid outputs are written to col[0 .. out).
__device__ void mlp_eval(const NetView& nv, const WeightImage& wi, const float* __restrict__ img, int act,
                         const float (&x0)[kInPad], float* col, int stride) {
    // layer 0
    {
        const float* W = img + wi.w[0];
        const float* B = img + wi.b[0];
        bool last = nv.n_layers == 1;
        int rows = nv.layer_out[0];
#pragma unroll 1
        for (int o = 0; o < rows; ++o) {
            const float4* w4 = reinterpret_cast<const float4*>(W + o * kInPad);
            float acc = B[o];
#pragma unroll
            for (int i = 0; i < kInPad / 4; ++i) {
                float4 w = w4[i];
                acc = fmaf(w.x, x0[4 * i], acc);
                acc = fmaf(w.y, x0[4 * i + 1], acc);
                acc = fmaf(w.z, x0[4 * i + 2], acc);
                acc = fmaf(w.w, x0[4 * i + 3], acc);
            }
            col[o * stride] = last ? sigmoid_f(acc) : act_f(acc, act);
        }
    }
    for (int l = 1; l < nv.n_layers; ++l) {
        float x[kHidden];
#pragma unroll
        for (int i = 0; i < kHidden; ++i) x[i] = col[i * stride];
        const float* W = img + wi.w[l];
        const float* B = img + wi.b[l];
        bool last = l + 1 == nv.n_layers;
        int rows = nv.layer_out[l];
#pragma unroll 1
        for (int o = 0; o < rows; ++o) {
            const float4* w4 = reinterpret_cast<const float4*>(W + o * kHidden);
            float acc = B[o];
#pragma unroll
            for (int i = 0; i < kHidden / 4; ++i) {
                float4 w = w4[i];
                acc = fmaf(w.x, x[4 * i], acc);
                acc = fmaf(w.y, x[4 * i + 1], acc);
                acc = fmaf(w.z, x[4 * i + 2], acc);
                acc = fmaf(w.w, x[4 * i + 3], acc);
            }
            col[o * stride] = last ? sigmoid_f(acc) : act_f(acc, act);
        }
    }
}

struct OutPtrs {
    uint8_t* p[NTBC_MAX_TEXTURES];
    int stride[NTBC_MAX_TEXTURES];     // bytes between consecutive blocks of a texture
};

// MODE_PACK: write BC blocks; MODE_RAW: write e_hat / c_hat of the listed blocks
enum { MODE_PACK = 0, MODE_RAW = 1 };

template <int MODE>
__global__ void __launch_bounds__(kSimtThreads)
infer_simt_kernel(ModelView mv, const float* __restrict__ params, GridSrc csrc, GridSrc esrc, WeightImage wic,
                  WeightImage wie, OutPtrs outs, const int32_t* __restrict__ ids, int n, float* __restrict__ e_out,
                  float* __restrict__ c_out) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const int stride = blockDim.x;
    int wfloats = max(wic.floats, wie.floats);
    float* img = smem;
    float* colbase = smem + wfloats;                              // [64][stride]
    float* palbase = colbase + kHidden * stride;                  // [T][12][stride]
    uint32_t* epbase = reinterpret_cast<uint32_t*>(palbase + mv.n_textures * kPalFloats * stride);
    const int tid = threadIdx.x;
    float* col = colbase + tid;
    int idx_in = blockIdx.x * blockDim.x + tid;
    bool valid = idx_in < n;
    int b = valid ? (ids ? ids[idx_in] : idx_in) : 0;
    int bx = b % mv.bw, by = b / mv.bw;

    // ---- endpoint network (per block)
    load_weight_image(mv.endpoint, wie, params, img);
    __syncthreads();
    if (valid) {
        float x0[kInPad];
        float feats[kInPad];
        grid_features(mv.endpoint, esrc, ((float)bx + 0.5f) / (float)mv.bw, ((float)by + 0.5f) / (float)mv.bh, feats);
#pragma unroll
        for (int i = 0; i < kInPad; ++i) x0[i] = i < mv.endpoint.in_dim ? feats[i] : 0.f;
        mlp_eval(mv.endpoint, wie, img, mv.activation, x0, col, stride);
        if (MODE == MODE_RAW) {
            for (int o = 0; o < mv.endpoint.out_dim; ++o) e_out[(long long)idx_in * mv.endpoint.out_dim + o] = col[o * stride];
        } else {
            for (int t = 0; t < mv.n_textures; ++t) {
                BlockPalette bp;
                float e[6];
                int eo = mv.eoff[t];
                float* pal = palbase + t * kPalFloats * stride + tid;
                if (mv.formats[t] == NTBC_BC1) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) e[k] = col[(eo + k) * stride];
                    make_palette_bc1(e, bp);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) pal[(k * 3 + ch) * stride] = bp.pal[k][ch];
                    epbase[t * stride + tid] = bp.ep;
                } else {
                    e[0] = col[eo * stride];
                    e[1] = col[(eo + 1) * stride];
                    make_palette_bc4(e, bp);
#pragma unroll
                    for (int k = 0; k < 8; ++k) pal[k * stride] = bp.pal[k][0];
                    epbase[t * stride + tid] = bp.ep;
                }
            }
        }
    }
    __syncthreads();

    // ---- colour network (per texel) + argmax + pack
    load_weight_image(mv.color, wic, params, img);
    __syncthreads();
    if (!valid) return;
    uint64_t idx[NTBC_MAX_TEXTURES];
#pragma unroll
    for (int t = 0; t < NTBC_MAX_TEXTURES; ++t) idx[t] = 0;
    for (int i = 0; i < 16; ++i) {
        int x = 4 * bx + (i & 3), y = 4 * by + (i >> 2);
        float x0[kInPad];
        float feats[kInPad];
        grid_features(mv.color, csrc, ((float)x + 0.5f) / (float)mv.width, ((float)y + 0.5f) / (float)mv.height, feats);
#pragma unroll
        for (int k = 0; k < kInPad; ++k) x0[k] = k < mv.color.in_dim ? feats[k] : 0.f;
        mlp_eval(mv.color, wic, img, mv.activation, x0, col, stride);
        if (MODE == MODE_RAW) {
            for (int o = 0; o < mv.color.out_dim; ++o)
                c_out[((long long)idx_in * 16 + i) * mv.color.out_dim + o] = col[o * stride];
            continue;
        }
#pragma unroll
        for (int t = 0; t < NTBC_MAX_TEXTURES; ++t) {
            if (t >= mv.n_textures) break;
            const float* pal = palbase + t * kPalFloats * stride + tid;
            int co = mv.coff[t];
            BlockPalette bp;
            int code;
            if (mv.formats[t] == NTBC_BC1) {
                uint32_t ep = epbase[t * stride + tid];
                bp.solid = (ep & 0xFFFFu) == (ep >> 16);
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) bp.pal[k][ch] = pal[(k * 3 + ch) * stride];
                code = choose_code_bc1(bp, col[co * stride], col[(co + 1) * stride], col[(co + 2) * stride]);
                idx[t] |= (uint64_t)code << (2 * i);
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) bp.pal[k][0] = pal[k * stride];
                code = choose_code_bc4(bp, col[co * stride]);
                idx[t] |= (uint64_t)code << (3 * i);
            }
        }
    }
    if (MODE == MODE_PACK) {
#pragma unroll
        for (int t = 0; t < NTBC_MAX_TEXTURES; ++t) {
            if (t >= mv.n_textures) break;
            uint32_t ep = epbase[t * stride + tid];
            uint8_t* dst = outs.p[t] + (long long)b * outs.stride[t];
            if (mv.formats[t] == NTBC_BC1) {
                store_block(dst, ep, (uint32_t)idx[t]);       // equal colours carry all-zero codes
            } else {
                store_block(dst, ep | (uint32_t)((idx[t] & 0xFFFF) << 16), (uint32_t)(idx[t] >> 16));
            }
        }
    }
}

static size_t simt_smem_bytes(const ModelView& mv, const WeightImage& wic, const WeightImage& wie, int threads) {
    size_t wf = (size_t)std::max(wic.floats, wie.floats);
    return (wf + (size_t)kHidden * threads + (size_t)mv.n_textures * kPalFloats * threads) * sizeof(float) +
           (size_t)mv.n_textures * threads * sizeof(uint32_t);
}

ntbc_status grid_sources(const ntbc_model* m, GridSrc& csrc, GridSrc& esrc) {
    if (m->grid_bits < 0) return fail(NTBC_EINVAL, "model has not been exported (call ntbc_model_export or ntbc_model_load)");
    memset(&csrc, 0, sizeof(csrc));
    memset(&esrc, 0, sizeof(esrc));
    if (m->grid_bits > 0) {
        csrc.codes = m->qgrid;
        esrc.codes = m->qgrid;
        csrc.scale = m->qscale;
        csrc.zero = m->qzero;
        esrc.scale = m->qscale + m->desc.color_levels;
        esrc.zero = m->qzero + m->desc.color_levels;
    } else {
        csrc.f32 = m->infer_params;
        esrc.f32 = m->infer_params;
    }
    return NTBC_OK;
}

template <int MODE>
static ntbc_status launch_simt(const ntbc_model* m, const OutPtrs& outs, const int32_t* ids, int n, float* e_out,
                               float* c_out, cudaStream_t s) {
    GridSrc csrc, esrc;
    ntbc_status st = grid_sources(m, csrc, esrc);
    if (st != NTBC_OK) return st;
    ModelView mv = make_view(m->desc, m->layout);
    WeightImage wic = weight_image(mv.color), wie = weight_image(mv.endpoint);
    int threads = kSimtThreads;
    size_t smem = simt_smem_bytes(mv, wic, wie, threads);
    NTBC_CHECK_CUDA(ensure_dynamic_smem(reinterpret_cast<const void*>(infer_simt_kernel<MODE>), smem));
    int grid = (n + threads - 1) / threads;
    infer_simt_kernel<MODE><<<grid, threads, smem, s>>>(mv, m->infer_params, csrc, esrc, wic, wie, outs, ids, n, e_out, c_out);
    NTBC_CHECK_LAUNCH("ntbc inference (SIMT)");
    return NTBC_OK;
}

// ---------------------------------------------------------------------------
// calibration of the FP8 activation scales (NTBC_PREC_FP8_MMA): the largest |input| of every
// layer over a fixed sample of the material, in FP32 with the FP8 weights and unrounded
// activations; then per layer the smallest a with 2 max|x| <= 448 2^a
// ---------------------------------------------------------------------------

constexpr int kFp8CalibBlocks = 2048;
constexpr unsigned long long kFp8CalibStride = 2654435761ull;     // prime: the sampled ids are distinct

// One thread per sample row: rows [0, count) run the endpoint network on the sampled blocks'
// centres, rows [count, 17 count) the colour network on their 16 texels. amax: per network
// (colour, endpoint) and layer the largest |input| as FP32 bits (non-negative floats order
// like their bit patterns).
__global__ void __launch_bounds__(128) fp8_calib_kernel(ModelView mv, const float* __restrict__ params, GridSrc csrc,
                                                        GridSrc esrc, int count, unsigned* __restrict__ amax) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = row < 17 * count;
    const bool endpoint = row < count;
    float m[NTBC_MAX_MLP_LAYERS];
#pragma unroll
    for (int l = 0; l < NTBC_MAX_MLP_LAYERS; ++l) m[l] = 0.f;
    if (valid) {
        const int k = endpoint ? row : (row - count) / 16, i = endpoint ? 0 : (row - count) % 16;
        const unsigned long long nb = (unsigned long long)mv.bw * (unsigned long long)mv.bh;
        const long long b = (long long)((unsigned long long)k * kFp8CalibStride % nb);
        const int bx = (int)(b % mv.bw), by = (int)(b / mv.bw);
        const NetView& nv = endpoint ? mv.endpoint : mv.color;
        float u, v;
        if (endpoint) {
            u = ((float)bx + 0.5f) / (float)mv.bw;
            v = ((float)by + 0.5f) / (float)mv.bh;
        } else {
            u = ((float)(4 * bx + (i & 3)) + 0.5f) / (float)mv.width;
            v = ((float)(4 * by + (i >> 2)) + 0.5f) / (float)mv.height;
        }
        float f[kMaxIn], x[kHidden], y[kHidden];
        grid_features(nv, endpoint ? esrc : csrc, u, v, f);
        for (int j = 0; j < kHidden; ++j) x[j] = j < nv.in_dim ? f[j] : 0.f;
        for (int l = 0; l < nv.n_layers; ++l) {
            const int in = nv.layer_in[l], out = nv.layer_out[l];
            float mx = 0.f;
            for (int j = 0; j < in; ++j) mx = fmaxf(mx, fabsf(x[j]));
            m[l] = mx;
            if (l + 1 == nv.n_layers) break;                 // the output layer's result feeds no layer
            for (int o = 0; o < out; ++o) {
                float acc = params[nv.b_off[l] + o];
                for (int j = 0; j < in; ++j) acc = fmaf(params[nv.w_off[l] + (long long)o * in + j], x[j], acc);
                y[o] = act_f(acc, mv.activation);
            }
            for (int o = 0; o < out; ++o) x[o] = y[o];
        }
    }
    for (int net = 0; net < 2; ++net)
#pragma unroll
        for (int l = 0; l < NTBC_MAX_MLP_LAYERS; ++l) {
            unsigned w = valid && endpoint == (net == 1) ? __float_as_uint(m[l]) : 0u;
            w = __reduce_max_sync(0xffffffffu, w);
            if ((threadIdx.x & 31) == 0 && w) atomicMax(amax + net * NTBC_MAX_MLP_LAYERS + l, w);
        }
}

// aexp[net * n_layers + l] (the order of the FP8 weight exponents): smallest a with
// 2 max <= 448 2^a, compared exactly (powers of two scale exactly); 0 for an all-zero input
__global__ void fp8_act_exponent_kernel(const unsigned* __restrict__ amax, int n_layers, int* __restrict__ aexp) {
    for (int net = 0; net < 2; ++net)
        for (int l = 0; l < n_layers; ++l) {
            const float m = 2.f * __uint_as_float(amax[net * NTBC_MAX_MLP_LAYERS + l]);
            int e = 0;
            if (m > 0.f) {
                e = ilogbf(fminf(m, 3.0e38f)) - 8;
                for (int it = 0; it < 64 && m > ldexpf(448.f, e); ++it) ++e;
                for (int it = 0; it < 64 && m <= ldexpf(448.f, e - 1); ++it) --e;
            }
            aexp[net * n_layers + l] = e;
        }
}

ntbc_status fp8_calibrate(ntbc_model* m, cudaStream_t s) {
    GridSrc csrc, esrc;
    ntbc_status st = grid_sources(m, csrc, esrc);
    if (st != NTBC_OK) return st;
    const ModelView mv = make_view(m->desc, m->layout);
    const long long nb = (long long)mv.bw * mv.bh;
    const int count = (int)std::min<long long>(nb, kFp8CalibBlocks);
    NTBC_CHECK_CUDA(cudaMemsetAsync(m->w8_amax, 0, 2 * NTBC_MAX_MLP_LAYERS * sizeof(unsigned), s));
    const int rows = 17 * count;
    fp8_calib_kernel<<<(rows + 127) / 128, 128, 0, s>>>(mv, m->infer_params, csrc, esrc, count, m->w8_amax);
    fp8_act_exponent_kernel<<<1, 1, 0, s>>>(m->w8_amax, mv.color.n_layers, m->w8_aexp);
    NTBC_CHECK_LAUNCH("FP8 activation calibration");
    return NTBC_OK;
}

// ---------------------------------------------------------------------------
// host delivery (ntbc_infer_to_host): device staging of the blocks, block ids 0 .. n-1 for
// the ranged launches, a copy stream and its events, kept by the model
// ---------------------------------------------------------------------------

constexpr int kHostIoMaxChunks = 16;

}  // namespace ntbc

struct ntbc_host_io {
    uint8_t* stage = nullptr;                         // n_textures x n blocks x 8 bytes
    int32_t* ids = nullptr;                           // 0 .. n - 1
    cudaStream_t copy = nullptr;
    cudaEvent_t done[ntbc::kHostIoMaxChunks] = {};    // range c computed
    cudaEvent_t copied = nullptr;                     // every range on the host
};

namespace ntbc {

__global__ void iota_kernel(int32_t* __restrict__ ids, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) ids[i] = i;
}

static void host_io_destroy(ntbc_host_io* io) {
    if (!io) return;
    if (io->copy) {
        cudaStreamSynchronize(io->copy);
        cudaStreamDestroy(io->copy);
    }
    for (int c = 0; c < kHostIoMaxChunks; ++c)
        if (io->done[c]) cudaEventDestroy(io->done[c]);
    if (io->copied) cudaEventDestroy(io->copied);
    cudaFree(io->stage);
    cudaFree(io->ids);
    delete io;
}

void host_io_release(ntbc_model* m) {
    host_io_destroy(m->host_io);
    m->host_io = nullptr;
}

static ntbc_status host_io_prepare(ntbc_model* m, int n, cudaStream_t s) {
    if (m->host_io) return NTBC_OK;
    ntbc_host_io* io = new ntbc_host_io();
    ntbc_status st = device_alloc((void**)&io->stage, (size_t)m->desc.n_textures * n * 8, "host-delivery staging");
    if (st == NTBC_OK) st = device_alloc((void**)&io->ids, (size_t)n * sizeof(int32_t), "block ids");
    cudaError_t e = cudaSuccess;
    if (st == NTBC_OK) e = cudaStreamCreateWithFlags(&io->copy, cudaStreamNonBlocking);
    for (int c = 0; c < kHostIoMaxChunks && st == NTBC_OK && e == cudaSuccess; ++c)
        e = cudaEventCreateWithFlags(&io->done[c], cudaEventDisableTiming);
    if (st == NTBC_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&io->copied, cudaEventDisableTiming);
    if (st == NTBC_OK && e == cudaSuccess) {
        iota_kernel<<<(unsigned)std::min((n + 255) / 256, 152 * 8), 256, 0, s>>>(io->ids, n);
        e = cudaGetLastError();
    }
    if (st != NTBC_OK || e != cudaSuccess) {
        host_io_destroy(io);
        return st != NTBC_OK ? st : cuda_fail(e, "host-delivery set-up");
    }
    m->host_io = io;
    return NTBC_OK;
}

}  // namespace ntbc

using namespace ntbc;

extern "C" {

ntbc_status ntbc_infer_to_bc_strided(const ntbc_model* m, uint8_t* const* blocks_out, const int* block_stride,
                                     void* stream) {
    ntbc::NvtxRange nvtx_range("ntbc_infer_to_bc_strided");
    clear_error();
    if (!m || !blocks_out) return fail(NTBC_EINVAL, "null argument");
    OutPtrs outs;
    memset(&outs, 0, sizeof(outs));
    for (int t = 0; t < m->desc.n_textures; ++t) {
        if (!blocks_out[t]) return fail(NTBC_EINVAL, "null output pointer for texture %d", t);
        if (reinterpret_cast<uintptr_t>(blocks_out[t]) & 7) return fail(NTBC_EINVAL, "output %d not 8-byte aligned", t);
        outs.p[t] = blocks_out[t];
        outs.stride[t] = block_stride ? block_stride[t] : 8;
        if (outs.stride[t] < 8 || (outs.stride[t] & 7))
            return fail(NTBC_EINVAL, "block stride of texture %d must be a positive multiple of 8, got %d", t, outs.stride[t]);
    }
    int n = (m->desc.width / 4) * (m->desc.height / 4);
    if (m->weight_prec != NTBC_PREC_FP32) {
        GridSrc csrc, esrc;
        ntbc_status st = grid_sources(m, csrc, esrc);
        if (st != NTBC_OK) return st;
        return tc_launch(m, blocks_out, outs.stride, nullptr, n, nullptr, nullptr, csrc, esrc, (cudaStream_t)stream);
    }
    return launch_simt<MODE_PACK>(m, outs, nullptr, n, nullptr, nullptr, (cudaStream_t)stream);
}

ntbc_status ntbc_infer_to_bc(const ntbc_model* m, uint8_t* const* blocks_out, void* stream) {
    return ntbc_infer_to_bc_strided(m, blocks_out, nullptr, stream);
}

ntbc_status ntbc_infer_to_host(ntbc_model* m, uint8_t* const* host_out, int chunks, void* stream) {
    ntbc::NvtxRange nvtx_range("ntbc_infer_to_host");
    clear_error();
    if (!m || !host_out) return fail(NTBC_EINVAL, "null argument");
    if (chunks < 1 || chunks > kHostIoMaxChunks) return fail(NTBC_EINVAL, "chunks must be 1..%d", kHostIoMaxChunks);
    if (m->grid_bits < 0) return fail(NTBC_EINVAL, "model has not been exported (call ntbc_model_export or ntbc_model_load)");
    for (int t = 0; t < m->desc.n_textures; ++t)
        if (!host_out[t]) return fail(NTBC_EINVAL, "null output pointer for texture %d", t);
    const int n = (m->desc.width / 4) * (m->desc.height / 4);
    cudaStream_t s = (cudaStream_t)stream;
    ntbc_status st = host_io_prepare(m, n, s);
    if (st != NTBC_OK) return st;
    ntbc_host_io* io = m->host_io;
    const int T = m->desc.n_textures;
    uint8_t* stage[NTBC_MAX_TEXTURES];
    int strides[NTBC_MAX_TEXTURES];
    for (int t = 0; t < T; ++t) {
        stage[t] = io->stage + (size_t)t * n * 8;
        strides[t] = 8;
    }
    // ranges of whole work units (128 blocks, or the tensor-core kernel's unit size); on the
    // tensor-core path every range but the last is a whole number of rounds of the units in
    // flight, so the ranged launches take no more rounds than one launch over the material would
    int ub = 128;
    const int flight = m->weight_prec != NTBC_PREC_FP32 ? tc_units_in_flight(m, &ub) : 0;
    const int units = (n + ub - 1) / ub;
    int per_units = (units + chunks - 1) / chunks;
    if (flight > 0) {
        const int rounds = (units + flight - 1) / flight;
        per_units = (rounds + chunks - 1) / chunks * flight;
    }
    const int per = per_units * ub;
    GridSrc csrc, esrc;
    if (m->weight_prec != NTBC_PREC_FP32) {
        st = grid_sources(m, csrc, esrc);
        if (st != NTBC_OK) return st;
    }
    int c = 0;
    for (int first = 0; first < n; first += per, ++c) {
        const int cnt = std::min(per, n - first);
        if (m->weight_prec != NTBC_PREC_FP32) {
            // every range after the first is chained to the one before it (the ranges write
            // disjoint blocks; a range's copy waits for its event, recorded after its launch)
            st = tc_launch(m, stage, strides, io->ids + first, cnt, nullptr, nullptr, csrc, esrc, s, first > 0);
        } else {
            OutPtrs outs;
            memset(&outs, 0, sizeof(outs));
            for (int t = 0; t < T; ++t) {
                outs.p[t] = stage[t];
                outs.stride[t] = 8;
            }
            st = launch_simt<MODE_PACK>(m, outs, io->ids + first, cnt, nullptr, nullptr, s);
        }
        if (st != NTBC_OK) return st;
        // this range's blocks go to the host on the copy stream while the next range runs
        NTBC_CHECK_CUDA(cudaEventRecord(io->done[c], s));
        NTBC_CHECK_CUDA(cudaStreamWaitEvent(io->copy, io->done[c], 0));
        for (int t = 0; t < T; ++t)
            NTBC_CHECK_CUDA(cudaMemcpyAsync(host_out[t] + (size_t)first * 8, stage[t] + (size_t)first * 8,
                                            (size_t)cnt * 8, cudaMemcpyDeviceToHost, io->copy));
    }
    NTBC_CHECK_CUDA(cudaEventRecord(io->copied, io->copy));
    NTBC_CHECK_CUDA(cudaStreamWaitEvent(s, io->copied, 0));
    return NTBC_OK;
}

ntbc_status ntbc_forward(const ntbc_model* m, const int32_t* block_ids, int n, float* e_hat, float* c_hat, void* stream) {
    ntbc::NvtxRange nvtx_range("ntbc_forward");
    clear_error();
    if (!m) return fail(NTBC_EINVAL, "null model");
    if (n < 0) return fail(NTBC_EINVAL, "negative count");
    if (n == 0) return NTBC_OK;                       // nothing to read or write
    if (!block_ids || !e_hat || !c_hat) return fail(NTBC_EINVAL, "null argument");
    if (m->weight_prec != NTBC_PREC_FP32) {
        GridSrc csrc, esrc;
        ntbc_status st = grid_sources(m, csrc, esrc);
        if (st != NTBC_OK) return st;
        return tc_launch(m, nullptr, nullptr, block_ids, n, e_hat, c_hat, csrc, esrc, (cudaStream_t)stream);
    }
    OutPtrs outs;
    memset(&outs, 0, sizeof(outs));
    return launch_simt<MODE_RAW>(m, outs, block_ids, n, e_hat, c_hat, (cudaStream_t)stream);
}

}  // extern "C"
