// NTBC model state: parameter layout, allocation, the QAT export to the stored
// form (Sec. 2.3 Eq. quantize / scaling_factor, Sec. 3.3 per-level asymmetric
// quantisation) and the stored blob (Sec. 3.3: grids stored as 8-bit integers,
// half-precision MLP weights, Sec. 3.4).
#include <cuda_fp8.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "ntbc_internal.cuh"
#include "ntbc_kernels.cuh"

namespace ntbc {

static ntbc_status validate_desc(const ntbc_model_desc* d) {
    if (!d) return fail(NTBC_EINVAL, "null model description");
    if (d->width <= 0 || d->height <= 0 || (d->width & 3) || (d->height & 3))
        return fail(NTBC_EINVAL, "width and height must be positive multiples of 4 (got %dx%d)", d->width, d->height);
    if ((long long)d->width * d->height > (1LL << 30)) return fail(NTBC_EINVAL, "texture too large");
    if (d->n_textures < 1 || d->n_textures > NTBC_MAX_TEXTURES)
        return fail(NTBC_EINVAL, "n_textures must be 1..%d", NTBC_MAX_TEXTURES);
    for (int t = 0; t < d->n_textures; ++t)
        if (d->formats[t] != NTBC_BC1 && d->formats[t] != NTBC_BC4)
            return fail(NTBC_EINVAL, "texture %d: format must be NTBC_BC1 or NTBC_BC4", t);
    if (d->features != 2) return fail(NTBC_EUNSUPPORTED, "features per level must be 2");
    for (int net = 0; net < 2; ++net) {
        int L = net ? d->endpoint_levels : d->color_levels;
        const int* res = net ? d->endpoint_res : d->color_res;
        if (L < 1 || L > NTBC_MAX_LEVELS || L * d->features > kMaxIn)
            return fail(NTBC_EINVAL, "%s grid: 1..%d levels with features*levels <= %d", net ? "endpoint" : "colour",
                        NTBC_MAX_LEVELS, kMaxIn);
        for (int l = 0; l < L; ++l)
            if (res[l] < 2 || res[l] > 16384)
                return fail(NTBC_EINVAL, "%s grid level %d: resolution %d outside 2..16384", net ? "endpoint" : "colour",
                            l, res[l]);
    }
    if (d->hidden_width != kHidden) return fail(NTBC_EUNSUPPORTED, "hidden width must be %d", kHidden);
    if (d->hidden_layers < 1 || d->hidden_layers > 3) return fail(NTBC_EUNSUPPORTED, "hidden layers must be 1..3");
    if (d->activation != NTBC_ACT_SELU && d->activation != NTBC_ACT_RELU)
        return fail(NTBC_EINVAL, "activation must be NTBC_ACT_SELU or NTBC_ACT_RELU");
    return NTBC_OK;
}

ModelView make_view(const ntbc_model_desc& d, const ntbc_layout& L) {
    ModelView mv;
    memset(&mv, 0, sizeof(mv));
    mv.width = d.width;
    mv.height = d.height;
    mv.bw = d.width / 4;
    mv.bh = d.height / 4;
    mv.n_textures = d.n_textures;
    mv.activation = d.activation;
    int co = 0;
    for (int t = 0; t < d.n_textures; ++t) {
        mv.formats[t] = d.formats[t];
        mv.coff[t] = co;
        mv.eoff[t] = 2 * co;
        co += channels_of(d.formats[t]);
    }
    for (int net = 0; net < 2; ++net) {
        NetView& nv = net ? mv.endpoint : mv.color;
        nv.levels = net ? d.endpoint_levels : d.color_levels;
        nv.features = d.features;
        const ntbc_span* gs = net ? L.endpoint_grid : L.color_grid;
        for (int l = 0; l < nv.levels; ++l) {
            nv.res[l] = net ? d.endpoint_res[l] : d.color_res[l];
            nv.resm1[l] = (float)(nv.res[l] - 1);
            nv.resm2[l] = (float)(nv.res[l] - 2);
            nv.grid_off[l] = (long long)gs[l].offset;
        }
        nv.in_dim = net ? L.in_endpoint : L.in_color;
        nv.out_dim = net ? L.out_endpoint : L.out_color;
        nv.hidden_layers = d.hidden_layers;
        nv.n_layers = d.hidden_layers + 1;
        const ntbc_span* ws = net ? L.endpoint_w : L.color_w;
        const ntbc_span* bs = net ? L.endpoint_b : L.color_b;
        for (int l = 0; l < nv.n_layers; ++l) {
            nv.w_off[l] = (long long)ws[l].offset;
            nv.b_off[l] = (long long)bs[l].offset;
            nv.layer_in[l] = l == 0 ? nv.in_dim : kHidden;
            nv.layer_out[l] = l + 1 == nv.n_layers ? nv.out_dim : kHidden;
        }
    }
    return mv;
}

// ---------------------------------------------------------------------------
// per-level min / max (order-preserving unsigned encoding; both start at the
// encoding of 0.0 so the range always contains zero) and scale / zero point
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned enc_f(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float dec_f(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

__global__ void level_minmax_kernel(const float* __restrict__ grid, LevelTable lt, unsigned* __restrict__ mm) {
    int l = blockIdx.y;
    long long n = lt.count[l];
    const float* g = grid + lt.offset[l];
    float lo = 0.f, hi = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float v = g[i];
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&mm[2 * l], enc_f(lo));
        atomicMax(&mm[2 * l + 1], enc_f(hi));
    }
}

__global__ void level_minmax_init_kernel(unsigned* mm, int levels) {
    int i = threadIdx.x;
    if (i < 2 * levels) mm[i] = enc_f(0.f);
}

// s = (beta - alpha) / (2^b - 1), z = round(-alpha / s); all-zero level: s = 1, z = 0
__global__ void level_scale_zero_kernel(const unsigned* __restrict__ mm, int levels, int bits,
                                        float* __restrict__ scale, float* __restrict__ zero) {
    int l = threadIdx.x;
    if (l >= levels) return;
    float a = dec_f(mm[2 * l]), b = dec_f(mm[2 * l + 1]);
    float range = __fsub_rn(b, a);
    if (range == 0.f) {
        scale[l] = 1.f;
        zero[l] = 0.f;
        return;
    }
    float s = __fdiv_rn(range, (float)((1 << bits) - 1));
    scale[l] = s;
    zero[l] = roundf(__fdiv_rn(-a, s));
}

__global__ void quantize_levels_kernel(const float* __restrict__ grid, LevelTable lt, const float* __restrict__ scale,
                                       const float* __restrict__ zero, int bits, uint8_t* __restrict__ codes) {
    int l = blockIdx.y;
    long long n = lt.count[l];
    float s = scale[l], z = zero[l], qmax = (float)((1 << bits) - 1);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float q = roundf(__fdiv_rn(grid[lt.offset[l] + i], s)) + z;
        q = fminf(fmaxf(q, 0.f), qmax);
        codes[lt.offset[l] + i] = (uint8_t)q;
    }
}

__global__ void round_half_kernel(const float* __restrict__ src, float* __restrict__ dst, __half* __restrict__ h,
                                  long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        __half v = __float2half_rn(src[i]);
        h[i] = v;
        dst[i] = __half2float(v);
    }
}

// 4-bit grid codes in the blob: two per byte, the lower-indexed code in the low nibble
__global__ void pack_nibbles_kernel(const uint8_t* __restrict__ codes, uint8_t* __restrict__ packed, long long n) {
    const long long pairs = (n + 1) / 2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < pairs; i += (long long)gridDim.x * blockDim.x) {
        uint8_t lo = codes[2 * i] & 15, hi = 2 * i + 1 < n ? codes[2 * i + 1] & 15 : 0;
        packed[i] = (uint8_t)(lo | (hi << 4));
    }
}

__global__ void unpack_nibbles_kernel(const uint8_t* __restrict__ packed, uint8_t* __restrict__ codes, long long n) {
    const long long pairs = (n + 1) / 2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < pairs; i += (long long)gridDim.x * blockDim.x) {
        uint8_t b = packed[i];
        codes[2 * i] = b & 15;
        if (2 * i + 1 < n) codes[2 * i + 1] = b >> 4;
    }
}

// the packed staging area of 4-bit blobs sits behind the codes in the same allocation
static size_t qgrid_codes_bytes(const ntbc_layout& L) { return (L.grid_floats + 15) & ~(size_t)15; }

__global__ void half_to_float_kernel(const __half* __restrict__ h, float* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = __half2float(h[i]);
}

LevelTable level_table(const ntbc_model_desc& d, const ntbc_layout& L) {
    LevelTable lt;
    memset(&lt, 0, sizeof(lt));
    lt.levels = d.color_levels + d.endpoint_levels;
    for (int l = 0; l < d.color_levels; ++l) {
        lt.offset[l] = (long long)L.color_grid[l].offset;
        lt.count[l] = (long long)L.color_grid[l].count;
    }
    for (int l = 0; l < d.endpoint_levels; ++l) {
        lt.offset[d.color_levels + l] = (long long)L.endpoint_grid[l].offset;
        lt.count[d.color_levels + l] = (long long)L.endpoint_grid[l].count;
    }
    return lt;
}

ntbc_status launch_level_scale_zero(const float* grid, const LevelTable& lt, int bits, unsigned* mm, float* scale,
                                    float* zero, cudaStream_t s) {
    level_minmax_init_kernel<<<1, 64, 0, s>>>(mm, lt.levels);
    dim3 g(64, lt.levels);
    level_minmax_kernel<<<g, 256, 0, s>>>(grid, lt, mm);
    level_scale_zero_kernel<<<1, 32, 0, s>>>(mm, lt.levels, bits, scale, zero);
    NTBC_CHECK_LAUNCH("grid level scale / zero point");
    return NTBC_OK;
}

// FP8 E4M3 weights with one power-of-two scale per layer. A layer is its weight matrix and
// bias (two spans of the parameter buffer); one CTA per layer.
struct Fp8Layers {
    int n;
    long long w_off[2 * NTBC_MAX_MLP_LAYERS], w_cnt[2 * NTBC_MAX_MLP_LAYERS];
    long long b_off[2 * NTBC_MAX_MLP_LAYERS], b_cnt[2 * NTBC_MAX_MLP_LAYERS];
};

static Fp8Layers fp8_layers(const ntbc_model_desc& d, const ntbc_layout& L) {
    Fp8Layers f;
    memset(&f, 0, sizeof(f));
    int per_net = d.hidden_layers + 1;
    for (int net = 0; net < 2; ++net)
        for (int l = 0; l < per_net; ++l) {
            const ntbc_span& w = net ? L.endpoint_w[l] : L.color_w[l];
            const ntbc_span& b = net ? L.endpoint_b[l] : L.color_b[l];
            f.w_off[f.n] = (long long)w.offset;
            f.w_cnt[f.n] = (long long)w.count;
            f.b_off[f.n] = (long long)b.offset;
            f.b_cnt[f.n] = (long long)b.count;
            ++f.n;
        }
    return f;
}

__device__ __forceinline__ long long fp8_index(const Fp8Layers& f, int l, long long j) {
    return j < f.w_cnt[l] ? f.w_off[l] + j : f.b_off[l] + (j - f.w_cnt[l]);
}

__device__ __forceinline__ float e4m3_value(uint8_t q) {
    __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q, __NV_E4M3);
    return __half2float(__half(h));
}

// quantise (codes == written) or expand stored codes; writes the exact values q 2^e as
// FP32 (dst, same indexing as the parameter buffer) and FP16 (h, MLP part only)
__global__ void __launch_bounds__(256) fp8_layers_kernel(const float* __restrict__ params, Fp8Layers f,
                                                         long long grid_floats, int quantise, uint8_t* __restrict__ codes,
                                                         int* __restrict__ exps, float* __restrict__ dst,
                                                         __half* __restrict__ h) {
    __shared__ float wmax[8];
    __shared__ int e_sh;
    const int l = blockIdx.x;
    const long long n = f.w_cnt[l] + f.b_cnt[l];
    if (quantise) {
        float m = 0.f;
        for (long long j = threadIdx.x; j < n; j += blockDim.x) m = fmaxf(m, fabsf(params[fp8_index(f, l, j)]));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmax[w]);
            int e = 0;
            if (m > 0.f) {                 // smallest e with m <= 448 * 2^e (exact comparisons)
                e = ilogbf(m) - 8;
                while (m > ldexpf(448.f, e)) ++e;
                while (m <= ldexpf(448.f, e - 1)) --e;
            }
            e_sh = e;
            exps[l] = e;
        }
    } else if (threadIdx.x == 0) {
        e_sh = exps[l];
    }
    __syncthreads();
    const int e = e_sh;
    for (long long j = threadIdx.x; j < n; j += blockDim.x) {
        long long i = fp8_index(f, l, j);
        uint8_t q;
        if (quantise) {
            q = (uint8_t)__nv_cvt_float_to_fp8(ldexpf(params[i], -e), __NV_SATFINITE, __NV_E4M3);
            codes[i - grid_floats] = q;
        } else {
            q = codes[i - grid_floats];
        }
        float v = ldexpf(e4m3_value(q), e);
        dst[i] = v;
        h[i - grid_floats] = __float2half_rn(v);
    }
}

static bool is_fp8(int prec) { return prec == NTBC_PREC_FP8 || prec == NTBC_PREC_FP8_MMA; }

// exponent bytes of an FP8 blob: the weight exponents, and for FP8_MMA the activation ones
static size_t fp8_exp_bytes(int prec) {
    return (prec == NTBC_PREC_FP8_MMA ? 4 : 2) * NTBC_MAX_MLP_LAYERS * sizeof(int);
}

static int grid_blocks(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 8); }

}  // namespace ntbc

using namespace ntbc;

extern "C" {

ntbc_status ntbc_level_resolutions(int levels, int n_min, int n_max, int* out) {
    clear_error();
    if (!out || levels < 1 || levels > NTBC_MAX_LEVELS || n_min < 2 || n_max < n_min)
        return fail(NTBC_EINVAL, "need 1..%d levels and 2 <= n_min <= n_max", NTBC_MAX_LEVELS);
    for (int l = 0; l < levels; ++l) {
        double r = levels == 1 ? (double)n_min
                               : (double)n_min * std::pow((double)n_max / n_min, (double)l / (levels - 1));
        out[l] = (int)std::floor(r + 0.5);
    }
    return NTBC_OK;
}

ntbc_status ntbc_model_layout(const ntbc_model_desc* desc, ntbc_layout* out) {
    clear_error();
    if (!out) return fail(NTBC_EINVAL, "null layout");
    ntbc_status st = validate_desc(desc);
    if (st != NTBC_OK) return st;
    ntbc_layout L;
    memset(&L, 0, sizeof(L));
    size_t off = 0;
    for (int l = 0; l < desc->color_levels; ++l) {
        size_t n = (size_t)desc->color_res[l] * desc->color_res[l] * desc->features;
        L.color_grid[l] = {off, n};
        off += n;
    }
    for (int l = 0; l < desc->endpoint_levels; ++l) {
        size_t n = (size_t)desc->endpoint_res[l] * desc->endpoint_res[l] * desc->features;
        L.endpoint_grid[l] = {off, n};
        off += n;
    }
    L.grid_floats = off;
    int outc = 0;
    for (int t = 0; t < desc->n_textures; ++t) outc += channels_of(desc->formats[t]);
    L.in_color = desc->features * desc->color_levels;
    L.in_endpoint = desc->features * desc->endpoint_levels;
    L.out_color = outc;
    L.out_endpoint = 2 * outc;
    if (L.out_color > kMaxOutC || L.out_endpoint > kMaxOutE)
        return fail(NTBC_EUNSUPPORTED, "too many output channels (%d colour, max %d)", outc, kMaxOutC);
    for (int net = 0; net < 2; ++net) {
        int nl = desc->hidden_layers + 1;
        for (int l = 0; l < nl; ++l) {
            int in = l == 0 ? (net ? L.in_endpoint : L.in_color) : desc->hidden_width;
            int o = l + 1 == nl ? (net ? L.out_endpoint : L.out_color) : desc->hidden_width;
            ntbc_span* w = net ? L.endpoint_w : L.color_w;
            ntbc_span* b = net ? L.endpoint_b : L.color_b;
            w[l] = {off, (size_t)in * o};
            off += (size_t)in * o;
            b[l] = {off, (size_t)o};
            off += o;
        }
    }
    L.total = off;
    *out = L;
    return NTBC_OK;
}

ntbc_status ntbc_model_create(const ntbc_model_desc* desc, ntbc_model** out) {
    clear_error();
    if (!out) return fail(NTBC_EINVAL, "null output handle");
    *out = nullptr;
    ntbc_layout L;
    ntbc_status st = ntbc_model_layout(desc, &L);
    if (st != NTBC_OK) return st;
    ntbc_model* m = new ntbc_model();
    m->desc = *desc;
    m->layout = L;
    st = device_alloc((void**)&m->params, L.total * sizeof(float), "model parameters");
    if (st == NTBC_OK) {
        cudaError_t e = cudaMemset(m->params, 0, L.total * sizeof(float));
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemset(parameters)");
    }
    if (st != NTBC_OK) {
        ntbc_model_free(m);
        return st;
    }
    *out = m;
    return NTBC_OK;
}

void ntbc_model_free(ntbc_model* m) {
    if (!m) return;
    cudaFree(m->params);
    cudaFree(m->adam_m);
    cudaFree(m->adam_v);
    cudaFree(m->qgrid);
    cudaFree(m->qscale);   // also holds the zero points and the min / max scratch
    cudaFree(m->infer_params);
    cudaFree(m->w16);
    cudaFree(m->w8);                     // also holds w8_exp
    cudaFree(m->umma_img);               // also holds tc_err
    ntbc_train_release(m);
    host_io_release(m);
    delete m;
}

ntbc_status ntbc_model_params(ntbc_model* m, float** params, size_t* count) {
    clear_error();
    if (!m || !params || !count) return fail(NTBC_EINVAL, "null argument");
    *params = m->params;
    *count = m->layout.total;
    return NTBC_OK;
}

ntbc_status ntbc_model_set_params(ntbc_model* m, const float* src, size_t count, void* stream) {
    clear_error();
    if (!m || !src) return fail(NTBC_EINVAL, "null argument");
    if (count != m->layout.total) return fail(NTBC_EINVAL, "expected %zu floats, got %zu", m->layout.total, count);
    NTBC_CHECK_CUDA(cudaMemcpyAsync(m->params, src, count * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return NTBC_OK;
}

ntbc_status ntbc_model_get_params(const ntbc_model* m, float* dst, size_t count, void* stream) {
    clear_error();
    if (!m || !dst) return fail(NTBC_EINVAL, "null argument");
    if (count != m->layout.total) return fail(NTBC_EINVAL, "expected %zu floats, got %zu", m->layout.total, count);
    NTBC_CHECK_CUDA(cudaMemcpyAsync(dst, m->params, count * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return NTBC_OK;
}

static ntbc_status ensure_export_buffers(ntbc_model* m) {
    const ntbc_layout& L = m->layout;
    int levels = m->desc.color_levels + m->desc.endpoint_levels;
    ntbc_status st = NTBC_OK;
    if (!m->qgrid) st = device_alloc((void**)&m->qgrid, qgrid_codes_bytes(L) + (L.grid_floats + 1) / 2, "grid codes");
    if (st == NTBC_OK && !m->qscale) st = device_alloc((void**)&m->qscale, levels * sizeof(float) * 2 + 2 * levels * sizeof(unsigned), "grid scales");
    if (st == NTBC_OK && !m->qzero) m->qzero = m->qscale + levels;
    if (st == NTBC_OK && !m->infer_params) st = device_alloc((void**)&m->infer_params, L.total * sizeof(float), "inference parameters");
    if (st == NTBC_OK && !m->w16) st = device_alloc((void**)&m->w16, (L.total - L.grid_floats) * sizeof(__half), "half weights");
    if (st == NTBC_OK && !m->w8) {
        size_t codes = ((L.total - L.grid_floats) + 15) & ~(size_t)15;
        st = device_alloc((void**)&m->w8, codes + 6 * NTBC_MAX_MLP_LAYERS * sizeof(int), "FP8 weights");
        if (st == NTBC_OK) {
            m->w8_exp = reinterpret_cast<int*>(m->w8 + codes);
            m->w8_aexp = m->w8_exp + 2 * NTBC_MAX_MLP_LAYERS;
            m->w8_amax = reinterpret_cast<unsigned*>(m->w8_aexp + 2 * NTBC_MAX_MLP_LAYERS);
        }
    }
    return st;
}

ntbc_status ntbc_model_export(ntbc_model* m, int grid_bits, int weight_prec, void* stream) {
    ntbc::NvtxRange nvtx_range("ntbc_model_export");
    clear_error();
    if (!m) return fail(NTBC_EINVAL, "null model");
    if (grid_bits != 0 && grid_bits != 8 && grid_bits != 4) return fail(NTBC_EINVAL, "grid_bits must be 0, 4 or 8");
    if (weight_prec < NTBC_PREC_FP32 || weight_prec > NTBC_PREC_FP8_MMA)
        return fail(NTBC_EINVAL, "weight precision must be NTBC_PREC_FP32, NTBC_PREC_FP16, NTBC_PREC_FP16_FAST, "
                                 "NTBC_PREC_FP8 or NTBC_PREC_FP8_MMA");
    ntbc_status st = ensure_export_buffers(m);
    if (st != NTBC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const ntbc_layout& L = m->layout;
    int levels = m->desc.color_levels + m->desc.endpoint_levels;
    // grids: FP32 copy (always, for grid_bits 0) and codes
    NTBC_CHECK_CUDA(cudaMemcpyAsync(m->infer_params, m->params, L.grid_floats * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (grid_bits > 0) {
        LevelTable lt = level_table(m->desc, L);
        unsigned* mm = reinterpret_cast<unsigned*>(m->qscale + 2 * levels);
        st = launch_level_scale_zero(m->params, lt, grid_bits, mm, m->qscale, m->qzero, s);
        if (st != NTBC_OK) return st;
        dim3 g(64, lt.levels);
        quantize_levels_kernel<<<g, 256, 0, s>>>(m->params, lt, m->qscale, m->qzero, grid_bits, m->qgrid);
        NTBC_CHECK_LAUNCH("quantize grid levels");
    }
    // MLP weights
    long long nw = (long long)(L.total - L.grid_floats);
    m->weight_prec = weight_prec;
    if (is_fp8(weight_prec)) {
        Fp8Layers f = fp8_layers(m->desc, L);
        fp8_layers_kernel<<<f.n, 256, 0, s>>>(m->params, f, (long long)L.grid_floats, 1, m->w8, m->w8_exp,
                                              m->infer_params, m->w16);
        NTBC_CHECK_LAUNCH("quantise weights to FP8");
        if (weight_prec == NTBC_PREC_FP8_MMA) {
            m->grid_bits = grid_bits;          // the calibration reads the exported grids
            st = fp8_calibrate(m, s);
            if (st != NTBC_OK) return st;
        }
        st = tc_prepare(m, s);
        if (st != NTBC_OK) return st;
    } else if (weight_prec != NTBC_PREC_FP32) {
        round_half_kernel<<<grid_blocks(nw), 256, 0, s>>>(m->params + L.grid_floats, m->infer_params + L.grid_floats, m->w16, nw);
        NTBC_CHECK_LAUNCH("round weights to half");
        st = tc_prepare(m, s);
        if (st != NTBC_OK) return st;
    } else {
        NTBC_CHECK_CUDA(cudaMemcpyAsync(m->infer_params + L.grid_floats, m->params + L.grid_floats, nw * sizeof(float),
                                        cudaMemcpyDeviceToDevice, s));
    }
    m->grid_bits = grid_bits;
    m->weight_prec = weight_prec;
    return NTBC_OK;
}

ntbc_status ntbc_model_exported_grid(const ntbc_model* m, uint8_t* codes, float* scales, float* zeros, void* stream) {
    clear_error();
    if (!m || !codes || !scales || !zeros) return fail(NTBC_EINVAL, "null argument");
    if (m->grid_bits <= 0) return fail(NTBC_EINVAL, "model has no quantised export");
    cudaStream_t s = (cudaStream_t)stream;
    int levels = m->desc.color_levels + m->desc.endpoint_levels;
    NTBC_CHECK_CUDA(cudaMemcpyAsync(codes, m->qgrid, m->layout.grid_floats, cudaMemcpyDeviceToDevice, s));
    NTBC_CHECK_CUDA(cudaMemcpyAsync(scales, m->qscale, levels * sizeof(float), cudaMemcpyDeviceToDevice, s));
    NTBC_CHECK_CUDA(cudaMemcpyAsync(zeros, m->qzero, levels * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return NTBC_OK;
}

// blob: magic, version, desc, grid_bits, weight_prec | scales, zeros | grid | weights
struct BlobHeader {
    char magic[4];
    int version;
    ntbc_model_desc desc;
    int grid_bits, weight_prec;
};

static size_t blob_parts(const ntbc_model* m, size_t* grid_b, size_t* sz_b, size_t* w_b) {
    const ntbc_layout& L = m->layout;
    int levels = m->desc.color_levels + m->desc.endpoint_levels;
    *sz_b = 2 * levels * sizeof(float);
    *grid_b = m->grid_bits == 4 ? (L.grid_floats + 1) / 2
                                : (m->grid_bits > 0 ? L.grid_floats : L.grid_floats * sizeof(float));
    size_t nw = L.total - L.grid_floats;
    if (is_fp8(m->weight_prec))
        *w_b = fp8_exp_bytes(m->weight_prec) + nw;                 // exponents, then codes
    else
        *w_b = nw * (m->weight_prec != NTBC_PREC_FP32 ? sizeof(__half) : sizeof(float));
    return sizeof(BlobHeader) + *sz_b + *grid_b + *w_b;
}

ntbc_status ntbc_model_blob_size(const ntbc_model* m, size_t* size) {
    clear_error();
    if (!m || !size) return fail(NTBC_EINVAL, "null argument");
    if (m->grid_bits < 0) return fail(NTBC_EINVAL, "model not exported");
    size_t g, z, w;
    *size = blob_parts(m, &g, &z, &w);
    return NTBC_OK;
}

ntbc_status ntbc_model_save(const ntbc_model* m, uint8_t* blob, size_t size, void* stream) {
    clear_error();
    if (!m || !blob) return fail(NTBC_EINVAL, "null argument");
    if (m->grid_bits < 0) return fail(NTBC_EINVAL, "model not exported");
    size_t gb, zb, wb;
    size_t need = blob_parts(m, &gb, &zb, &wb);
    if (size < need) return fail(NTBC_EINVAL, "blob buffer too small (%zu < %zu)", size, need);
    cudaStream_t s = (cudaStream_t)stream;
    BlobHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "NTBC", 4);
    h.version = ntbc_abi_version();
    h.desc = m->desc;
    h.grid_bits = m->grid_bits;
    h.weight_prec = m->weight_prec;
    memcpy(blob, &h, sizeof(h));
    uint8_t* p = blob + sizeof(h);
    if (m->grid_bits == 4) {
        uint8_t* packed = m->qgrid + qgrid_codes_bytes(m->layout);
        pack_nibbles_kernel<<<grid_blocks((long long)gb), 256, 0, s>>>(m->qgrid, packed, (long long)m->layout.grid_floats);
        NTBC_CHECK_LAUNCH("pack 4-bit grid codes");
        NTBC_CHECK_CUDA(cudaMemcpyAsync(p, m->qscale, zb, cudaMemcpyDeviceToHost, s));
        NTBC_CHECK_CUDA(cudaMemcpyAsync(p + zb, packed, gb, cudaMemcpyDeviceToHost, s));
    } else if (m->grid_bits > 0) {
        NTBC_CHECK_CUDA(cudaMemcpyAsync(p, m->qscale, zb, cudaMemcpyDeviceToHost, s));
        NTBC_CHECK_CUDA(cudaMemcpyAsync(p + zb, m->qgrid, gb, cudaMemcpyDeviceToHost, s));
    } else {
        memset(p, 0, zb);
        NTBC_CHECK_CUDA(cudaMemcpyAsync(p + zb, m->infer_params, gb, cudaMemcpyDeviceToHost, s));
    }
    const ntbc_layout& L = m->layout;
    if (is_fp8(m->weight_prec)) {
        // weight exponents, then (FP8_MMA) the activation exponents that follow them in w8
        const size_t eb = fp8_exp_bytes(m->weight_prec);
        NTBC_CHECK_CUDA(cudaMemcpyAsync(p + zb + gb, m->w8_exp, eb, cudaMemcpyDeviceToHost, s));
        NTBC_CHECK_CUDA(cudaMemcpyAsync(p + zb + gb + eb, m->w8, wb - eb, cudaMemcpyDeviceToHost, s));
    } else if (m->weight_prec != NTBC_PREC_FP32)
        NTBC_CHECK_CUDA(cudaMemcpyAsync(p + zb + gb, m->w16, wb, cudaMemcpyDeviceToHost, s));
    else
        NTBC_CHECK_CUDA(cudaMemcpyAsync(p + zb + gb, m->infer_params + L.grid_floats, wb, cudaMemcpyDeviceToHost, s));
    NTBC_CHECK_CUDA(cudaStreamSynchronize(s));
    return NTBC_OK;
}

ntbc_status ntbc_model_load(ntbc_model* m, const uint8_t* blob, size_t size, void* stream) {
    ntbc::NvtxRange nvtx_range("ntbc_model_load");
    clear_error();
    if (!m || !blob) return fail(NTBC_EINVAL, "null argument");
    if (size < sizeof(BlobHeader)) return fail(NTBC_EINVAL, "blob too small");
    BlobHeader h;
    memcpy(&h, blob, sizeof(h));
    if (memcmp(h.magic, "NTBC", 4) != 0 || h.version != ntbc_abi_version()) return fail(NTBC_EINVAL, "not an NTBC blob of this version");
    if (memcmp(&h.desc, &m->desc, sizeof(ntbc_model_desc)) != 0) return fail(NTBC_EINVAL, "blob describes a different model");
    if (h.grid_bits != 0 && h.grid_bits != 4 && h.grid_bits != 8) return fail(NTBC_EINVAL, "blob has grid_bits %d", h.grid_bits);
    if (h.weight_prec < NTBC_PREC_FP32 || h.weight_prec > NTBC_PREC_FP8_MMA)
        return fail(NTBC_EINVAL, "blob has weight precision %d", h.weight_prec);
    ntbc_status st = ensure_export_buffers(m);
    if (st != NTBC_OK) return st;
    m->grid_bits = h.grid_bits;
    m->weight_prec = h.weight_prec;
    size_t gb, zb, wb;
    size_t need = blob_parts(m, &gb, &zb, &wb);
    if (size < need) return fail(NTBC_EINVAL, "blob truncated (%zu < %zu)", size, need);
    cudaStream_t s = (cudaStream_t)stream;
    const uint8_t* p = blob + sizeof(h);
    const ntbc_layout& L = m->layout;
    if (m->grid_bits == 4) {
        uint8_t* packed = m->qgrid + qgrid_codes_bytes(L);
        NTBC_CHECK_CUDA(cudaMemcpyAsync(m->qscale, p, zb, cudaMemcpyHostToDevice, s));
        NTBC_CHECK_CUDA(cudaMemcpyAsync(packed, p + zb, gb, cudaMemcpyHostToDevice, s));
        unpack_nibbles_kernel<<<grid_blocks((long long)gb), 256, 0, s>>>(packed, m->qgrid, (long long)L.grid_floats);
        NTBC_CHECK_LAUNCH("unpack 4-bit grid codes");
    } else if (m->grid_bits > 0) {
        NTBC_CHECK_CUDA(cudaMemcpyAsync(m->qscale, p, zb, cudaMemcpyHostToDevice, s));
        NTBC_CHECK_CUDA(cudaMemcpyAsync(m->qgrid, p + zb, gb, cudaMemcpyHostToDevice, s));
    } else {
        NTBC_CHECK_CUDA(cudaMemcpyAsync(m->infer_params, p + zb, gb, cudaMemcpyHostToDevice, s));
    }
    long long nw = (long long)(L.total - L.grid_floats);
    if (is_fp8(m->weight_prec)) {
        const size_t eb = fp8_exp_bytes(m->weight_prec);
        NTBC_CHECK_CUDA(cudaMemcpyAsync(m->w8_exp, p + zb + gb, eb, cudaMemcpyHostToDevice, s));
        NTBC_CHECK_CUDA(cudaMemcpyAsync(m->w8, p + zb + gb + eb, wb - eb, cudaMemcpyHostToDevice, s));
        Fp8Layers f = fp8_layers(m->desc, L);
        fp8_layers_kernel<<<f.n, 256, 0, s>>>(m->params, f, (long long)L.grid_floats, 0, m->w8, m->w8_exp,
                                              m->infer_params, m->w16);
        NTBC_CHECK_LAUNCH("expand FP8 weights");
        st = tc_prepare(m, s);
        if (st != NTBC_OK) return st;
    } else if (m->weight_prec != NTBC_PREC_FP32) {
        NTBC_CHECK_CUDA(cudaMemcpyAsync(m->w16, p + zb + gb, wb, cudaMemcpyHostToDevice, s));
        half_to_float_kernel<<<grid_blocks(nw), 256, 0, s>>>(m->w16, m->infer_params + L.grid_floats, nw);
        NTBC_CHECK_LAUNCH("expand half weights");
        st = tc_prepare(m, s);
        if (st != NTBC_OK) return st;
    } else {
        NTBC_CHECK_CUDA(cudaMemcpyAsync(m->infer_params + L.grid_floats, p + zb + gb, wb, cudaMemcpyHostToDevice, s));
    }
    return NTBC_OK;
}

}  // extern "C"
