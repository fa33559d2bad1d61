// NTBC training (encode): batch sampling, forward of both networks, the losses
// L_endpoint = L_e + L_cd and L_color = L_c + L_cd (Sec. 3.2, Eq. lossNTBC_e /
// lossNTBC_c) with the straight-through argmax (Eq. softmax, App. A), the hand-
// written backward (MLP weight / input gradients, grid scatter-add), QAT fake
// quantisation of the grids (Sec. 3.3) and dense Adam with warm-up + cosine
// schedule (Sec. 3.4).
//
// Layout: every activation buffer is feature-major, [unit][sample], so that
// consecutive threads (samples) touch consecutive addresses. The colour network
// runs on 16 samples per sampled block (all its texels), the endpoint network on
// one sample per block.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "ntbc_internal.cuh"
#include "ntbc_kernels.cuh"
#include "ntbc_train_common.cuh"
#include "ntbc_train_tc.cuh"
#include "tcgen05.cuh"

namespace ntbc {

constexpr double kAdamB1 = 0.9, kAdamB2 = 0.999;
constexpr float kAdamEps = 1e-15f;

struct StepState {
    long long step;          // current step index (0-based)
    float lr_grid, lr_mlp;   // scheduled learning rates of this step
    float bc1, bc2;          // Adam bias corrections 1 - beta^(step+1)
};

// The scheduled quantities of one step, copied into StepState at the start of the step.
struct StepSchedule {
    float lr_grid, lr_mlp, bc1, bc2;
};

struct NetBuffers {
    int cap;                 // sample capacity
    float* X;                // [32][cap] grid features
    float* A[3];             // [64][cap] hidden activations (post-activation)
    float* Y;                // [out][cap] sigmoid outputs
    float* D0;               // [64][cap] deltas (ping)
    float* D1;               // [64][cap] deltas (pong)
};

}  // namespace ntbc

struct ntbc_train_state {
    int cap_blocks = 0;
    ntbc::NetBuffers color{}, endpoint{};
    int32_t* ids = nullptr;
    float* grads = nullptr;
    double* loss_acc = nullptr;       // [6]
    float* losses = nullptr;          // [6]
    ntbc::StepState* st = nullptr;
    float* qscale = nullptr;          // [levels] QAT scale / zero of this step
    float* qzero = nullptr;
    unsigned* qmm = nullptr;
    unsigned char* tc_img = nullptr;  // BF16 weight images of both networks (tensor-core training)
    float* tc_part = nullptr;         // weight-gradient partial sums of the tensor-core pass
    int tc_part_rows = 0;
    int* tc_err = nullptr;            // set when a bounded wait of the tensor-core training gives up
    ntbc::StepSchedule* sched = nullptr;   // per-step schedule of the current ntbc_train call
    long long sched_cap = 0;
};

namespace ntbc {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al. 2011)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        if (r < 9) {
            k.x += W0;
            k.y += W1;
        }
    }
    return c;
}

// With a schedule table (a captured training step) thread 0 also publishes the step's LR and
// bias corrections into the step state and clears the step's six loss accumulators, before
// anything of the step reads them.
__global__ void sample_kernel(uint64_t seed, StepState* __restrict__ st, const StepSchedule* __restrict__ tab,
                              long long total_steps, long long explicit_step, int n, int n_blocks,
                              int32_t* __restrict__ ids, double* __restrict__ loss_acc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long step = st ? st->step : explicit_step;
    if (tab && i == 0 && step >= 0 && step < total_steps) {
        const StepSchedule q = tab[step];
        st->lr_grid = q.lr_grid;
        st->lr_mlp = q.lr_mlp;
        st->bc1 = q.bc1;
        st->bc2 = q.bc2;
        for (int k = 0; k < 6; ++k) loss_acc[k] = 0.0;
    }
    uint4 w = philox4x32_10(make_uint4((uint32_t)(i >> 2), (uint32_t)step, 0u, 0u),
                            make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    uint32_t word = (i & 3) == 0 ? w.x : (i & 3) == 1 ? w.y : (i & 3) == 2 ? w.z : w.w;
    ids[i] = (int32_t)(((uint64_t)word * (uint64_t)n_blocks) >> 32);
}

// ---------------------------------------------------------------------------
// step bookkeeping: schedule and bias corrections
// ---------------------------------------------------------------------------

// LR (linear warm-up, then cosine to 0 over all steps, Sec. 3.4) and Adam bias corrections
// of step t
__device__ __forceinline__ StepSchedule schedule_of(long long t, long long total_steps, float lr_grid, float lr_mlp,
                                                    int warmup) {
    double f;
    if (t < warmup) {
        f = (double)(t + 1) / warmup;
    } else {
        long long span = total_steps - warmup > 0 ? total_steps - warmup : 1;
        f = 0.5 * (1.0 + cos(3.14159265358979323846 * (double)(t - warmup) / (double)span));
    }
    StepSchedule q;
    q.lr_grid = (float)(lr_grid * f);
    q.lr_mlp = (float)(lr_mlp * f);
    q.bc1 = (float)(1.0 - pow(kAdamB1, (double)(t + 1)));
    q.bc2 = (float)(1.0 - pow(kAdamB2, (double)(t + 1)));
    return q;
}

// every step's schedule at once (one thread per step), before the step loop
__global__ void schedule_kernel(StepSchedule* tab, long long total_steps, float lr_grid, float lr_mlp, int warmup) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total_steps;
         t += (long long)gridDim.x * blockDim.x)
        tab[t] = schedule_of(t, total_steps, lr_grid, lr_mlp, warmup);
}

// The schedule of step t = explicit_step into the step state (the single-step Adam call).
__global__ void step_begin_kernel(StepState* st, long long explicit_step, long long total_steps, float lr_grid,
                                  float lr_mlp, int warmup) {
    if (threadIdx.x != 0) return;
    st->step = explicit_step;
    const StepSchedule q = schedule_of(explicit_step, total_steps, lr_grid, lr_mlp, warmup);
    st->lr_grid = q.lr_grid;
    st->lr_mlp = q.lr_mlp;
    st->bc1 = q.bc1;
    st->bc2 = q.bc2;
}


// ---------------------------------------------------------------------------
// batch gather of grid features
// ---------------------------------------------------------------------------

__global__ void gather_kernel(ModelView mv, bool color, GridSrc src, const int32_t* __restrict__ ids, int B,
                              float* __restrict__ X) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= B) return;
    const NetView& nv = color ? mv.color : mv.endpoint;
    float u, v;
    int x, y;
    sample_coords(mv, color, ids, k, u, v, x, y);
    float f[kMaxIn];
    grid_features(nv, src, u, v, f);
#pragma unroll
    for (int i = 0; i < kMaxIn; ++i)
        if (i < nv.in_dim) X[(long long)i * B + k] = f[i];
}

// ---------------------------------------------------------------------------
// dense layers
// ---------------------------------------------------------------------------

// Y[o][k] = act(b[o] + sum_i W[o][i] X[i][k]); act: 0 SELU, 1 ReLU, 2 sigmoid
template <int IN_PAD>
__global__ void dense_fwd_kernel(const float* __restrict__ X, int in, int B, const float* __restrict__ W,
                                 const float* __restrict__ bias, int out, int act, float* __restrict__ Y) {
    __shared__ __align__(16) float Ws[kHidden * IN_PAD];
    __shared__ float bs[kHidden];
    for (int i = threadIdx.x; i < out * IN_PAD; i += blockDim.x) {
        int r = i / IN_PAD, c = i % IN_PAD;
        Ws[i] = c < in ? W[r * in + c] : 0.f;
    }
    for (int i = threadIdx.x; i < out; i += blockDim.x) bs[i] = bias[i];
    __syncthreads();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= B) return;
    float x[IN_PAD];
#pragma unroll
    for (int i = 0; i < IN_PAD; ++i) x[i] = i < in ? X[(long long)i * B + k] : 0.f;
#pragma unroll 1
    for (int o = 0; o < out; ++o) {
        const float4* w4 = reinterpret_cast<const float4*>(Ws + o * IN_PAD);
        float acc = bs[o];
#pragma unroll
        for (int i = 0; i < IN_PAD / 4; ++i) {
            float4 w = w4[i];
            acc = fmaf(w.x, x[4 * i], acc);
            acc = fmaf(w.y, x[4 * i + 1], acc);
            acc = fmaf(w.z, x[4 * i + 2], acc);
            acc = fmaf(w.w, x[4 * i + 3], acc);
        }
        Y[(long long)o * B + k] = act == 2 ? sigmoid_f(acc) : act_f(acc, act);
    }
}

// Dprev[i][k] = (sum_o W[o][i] D[o][k]) * act'(Aprev[i][k])   (no factor when Aprev == null)
__global__ void dense_bwd_data_kernel(const float* __restrict__ D, int out, int B, const float* __restrict__ W, int in,
                                      const float* __restrict__ Aprev, int act, float* __restrict__ Dprev) {
    __shared__ __align__(16) float WT[kHidden * kHidden];    // [i][o], o padded to 64
    for (int j = threadIdx.x; j < in * kHidden; j += blockDim.x) {
        int i = j / kHidden, o = j % kHidden;
        WT[j] = o < out ? W[o * in + i] : 0.f;
    }
    __syncthreads();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= B) return;
    float d[kHidden];
#pragma unroll
    for (int o = 0; o < kHidden; ++o) d[o] = o < out ? D[(long long)o * B + k] : 0.f;
#pragma unroll 1
    for (int i = 0; i < in; ++i) {
        const float4* w4 = reinterpret_cast<const float4*>(WT + i * kHidden);
        float acc = 0.f;
#pragma unroll
        for (int o = 0; o < kHidden / 4; ++o) {
            float4 w = w4[o];
            acc = fmaf(w.x, d[4 * o], acc);
            acc = fmaf(w.y, d[4 * o + 1], acc);
            acc = fmaf(w.z, d[4 * o + 2], acc);
            acc = fmaf(w.w, d[4 * o + 3], acc);
        }
        if (Aprev) acc *= act_grad_from_out(Aprev[(long long)i * B + k], act);
        Dprev[(long long)i * B + k] = acc;
    }
}

// dW[o][i] += sum_k D[o][k] A[i][k], db[o] += sum_k D[o][k] over this CTA's chunk of samples
constexpr int kWgChunk = 512;
constexpr int kWgTile = 32;

__global__ void __launch_bounds__(256) dense_bwd_weight_kernel(const float* __restrict__ D, int out,
                                                               const float* __restrict__ A, int in, int B,
                                                               float* __restrict__ dW, float* __restrict__ db) {
    __shared__ float Ds[kHidden][kWgTile + 1];
    __shared__ float As[kHidden][kWgTile + 1];
    int ob = threadIdx.x / 16, ib = threadIdx.x % 16;   // 4 x 4 tile of (o, i)
    float acc[4][4] = {};
    float bacc[4] = {};
    long long k0 = (long long)blockIdx.x * kWgChunk;
    long long k1 = min((long long)B, k0 + kWgChunk);
    for (long long kt = k0; kt < k1; kt += kWgTile) {
        for (int j = threadIdx.x; j < kHidden * kWgTile; j += blockDim.x) {
            int r = j / kWgTile, c = j % kWgTile;
            long long k = kt + c;
            bool ok = k < k1;
            Ds[r][c] = (r < out && ok) ? D[(long long)r * B + k] : 0.f;
            As[r][c] = (r < in && ok) ? A[(long long)r * B + k] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int c = 0; c < kWgTile; ++c) {
            float d[4], a[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                d[j] = Ds[4 * ob + j][c];
                a[j] = As[4 * ib + j][c];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                bacc[p] += d[p];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(d[p], a[q], acc[p][q]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        int o = 4 * ob + p;
        if (o >= out) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int i = 4 * ib + q;
            if (i < in) atomicAdd(&dW[o * in + i], acc[p][q]);
        }
        if (ib == 0) atomicAdd(&db[o], bacc[p]);
    }
}

// ---------------------------------------------------------------------------
// losses with the straight-through argmax
// ---------------------------------------------------------------------------

// colour network: per texel sample, L_c + L_cd with distances from c_hat to the
// reference palette; writes D[o][k] = dL/dz_out (through the sigmoid)
__global__ void color_loss_kernel(ModelView mv, TexPtrs tp, const int32_t* __restrict__ ids, int B,
                                  const float* __restrict__ Y, float T, float* __restrict__ D, double* __restrict__ acc) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = k < B;
    float lc = 0.f, lcd = 0.f;
    if (ok) {
        int b = ids[k >> 4], i = k & 15;
        int x = 4 * (b % mv.bw) + (i & 3), y = 4 * (b / mv.bw) + (i >> 2);
        float n_el = (float)B * (float)mv.color.out_dim;
        for (int t = 0; t < mv.n_textures; ++t) {
            int fmt = mv.formats[t], C = fmt == NTBC_BC1 ? 3 : 1, co = mv.coff[t];
            float c[3], ch[3], e0[3], e1[3], g[3];
            for (int q = 0; q < C; ++q) {
                c[q] = texel_value(tp.texels[t], fmt, mv.width, x, y, q);
                ch[q] = Y[(long long)(co + q) * B + k];
            }
            ref_endpoints(fmt, tp.blocks[t], b, e0, e1);
            float A[8], Bc[8], Cc[8], P[8][3], d[8], nrm[8];
            int K = palette_coeffs(fmt, e0[0] > e1[0], A, Bc, Cc);
            int best = 0;
            for (int n = 0; n < K; ++n) {
                float s = 0.f;
                for (int q = 0; q < C; ++q) {
                    P[n][q] = A[n] * e0[q] + Bc[n] * e1[q] + Cc[n];
                    float df = ch[q] - P[n][q];
                    s += df * df;
                }
                nrm[n] = sqrtf(s);
                d[n] = -nrm[n];
                if (d[n] > d[best]) best = n;
            }
            float g_dec[3];
            for (int q = 0; q < C; ++q) {
                float r = c[q] - P[best][q];
                lcd += r * r;
                g_dec[q] = -2.f * r / n_el;
                float e = ch[q] - c[q];
                lc += e * e;
                g[q] = 2.f * e / n_el;
            }
            float g_d[8];
            ste_grad(K, C, d, P, g_dec, T, g_d);
            for (int n = 0; n < K; ++n) {
                float inv = 1.f / fmaxf(nrm[n], kNormGuard);
                for (int q = 0; q < C; ++q) g[q] -= g_d[n] * (ch[q] - P[n][q]) * inv;
            }
            for (int q = 0; q < C; ++q) D[(long long)(co + q) * B + k] = g[q] * ch[q] * (1.f - ch[q]);
        }
    }
    float n_el = (float)B * (float)mv.color.out_dim;
    block_reduce_add(&acc[2], lc / n_el);
    block_reduce_add(&acc[3], lcd / n_el);
}

// endpoint network: one thread per (sampled block, texel) -- thread k is texel k & 15 of
// sample k >> 4, so a block's 16 texels sit in one half-warp. L_cd uses distances from the
// texel colours to the palette of the predicted (unquantised) endpoints and decodes with
// the reference endpoints; the half-warp sums the 16 texels' contributions to the
// endpoint gradient, and its first lane adds L_e and writes D (through the sigmoid).
__global__ void endpoint_loss_kernel(ModelView mv, TexPtrs tp, const int32_t* __restrict__ ids, int Bn,
                                     const float* __restrict__ Y, float T, float* __restrict__ D,
                                     double* __restrict__ acc) {
    int kk = blockIdx.x * blockDim.x + threadIdx.x;
    int bi = kk >> 4, i = kk & 15;
    bool ok = bi < Bn;
    if (!ok) bi = 0;
    float okf = ok ? 1.f : 0.f;
    float le = 0.f, lcd = 0.f;
    int b = ids[bi];
    int x = 4 * (b % mv.bw) + (i & 3), y = 4 * (b / mv.bw) + (i >> 2);
    float n_e = (float)Bn * (float)mv.endpoint.out_dim;
    float n_cd = (float)Bn * 16.f * (float)mv.color.out_dim;
    for (int t = 0; t < mv.n_textures; ++t) {
        int fmt = mv.formats[t], C = fmt == NTBC_BC1 ? 3 : 1, eo = mv.eoff[t];
        float eh0[3] = {0.f, 0.f, 0.f}, eh1[3] = {0.f, 0.f, 0.f}, e0[3] = {0.f, 0.f, 0.f}, e1[3] = {0.f, 0.f, 0.f};
        float g0[3] = {0.f, 0.f, 0.f}, g1[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
        ref_endpoints(fmt, tp.blocks[t], b, e0, e1);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (q < C) {
                eh0[q] = Y[(long long)(eo + q) * Bn + bi];
                eh1[q] = Y[(long long)(eo + C + q) * Bn + bi];
                c[q] = texel_value(tp.texels[t], fmt, mv.width, x, y, q);
            }
        float Ah[8], Bh[8], Ch[8], Ar[8], Br[8], Cr[8];
        int K = palette_coeffs(fmt, eh0[0] > eh1[0], Ah, Bh, Ch);
        palette_coeffs(fmt, e0[0] > e1[0], Ar, Br, Cr);
        float Ph[8][3], Pr[8][3], d[8], nrm[8];
        int best = 0;
        for (int n = 0; n < K; ++n) {
            float sq = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                Ph[n][q] = Ah[n] * eh0[q] + Bh[n] * eh1[q] + Ch[n];
                Pr[n][q] = Ar[n] * e0[q] + Br[n] * e1[q] + Cr[n];
                float df = q < C ? c[q] - Ph[n][q] : 0.f;
                sq += df * df;
            }
            nrm[n] = sqrtf(sq);
            d[n] = -nrm[n];
            if (d[n] > d[best]) best = n;
        }
        float g_dec[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (q < C) {
                float rr = c[q] - Pr[best][q];
                lcd += okf * rr * rr;
                g_dec[q] = -2.f * okf * rr / n_cd;
            }
        float g_d[8];
        ste_grad(K, C, d, Pr, g_dec, T, g_d);
        for (int n = 0; n < K; ++n) {
            float inv = 1.f / fmaxf(nrm[n], kNormGuard);
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (q < C) {
                    float gp = g_d[n] * (c[q] - Ph[n][q]) * inv;      // d d_n / d p_n = (c - p_n)/||.||
                    g0[q] += Ah[n] * gp;
                    g1[q] += Bh[n] * gp;
                }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                g0[q] += __shfl_xor_sync(0xffffffffu, g0[q], o);
                g1[q] += __shfl_xor_sync(0xffffffffu, g1[q], o);
            }
        if (i == 0 && ok) {
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (q < C) {
                    float r0 = eh0[q] - e0[q], r1 = eh1[q] - e1[q];
                    le += r0 * r0 + r1 * r1;
                    g0[q] += 2.f * r0 / n_e;
                    g1[q] += 2.f * r1 / n_e;
                    D[(long long)(eo + q) * Bn + bi] = g0[q] * eh0[q] * (1.f - eh0[q]);
                    D[(long long)(eo + C + q) * Bn + bi] = g1[q] * eh1[q] * (1.f - eh1[q]);
                }
        }
    }
    block_reduce_add(&acc[0], le / n_e);
    block_reduce_add(&acc[1], lcd / n_cd);
}

__global__ void loss_finalize_kernel(const double* __restrict__ acc, float* __restrict__ losses) {
    if (threadIdx.x != 0) return;
    losses[0] = (float)acc[0];
    losses[1] = (float)acc[1];
    losses[2] = (float)acc[2];
    losses[3] = (float)acc[3];
    losses[4] = (float)(acc[0] + acc[1]);
    losses[5] = (float)(acc[2] + acc[3]);
}

// ---------------------------------------------------------------------------
// grid scatter-add (bilinear adjoint), with the QAT straight-through mask
// ---------------------------------------------------------------------------

// grid scatter-add of the batch's feature gradients G (feature-major [2L][B])
__global__ void grid_scatter_kernel(ModelView mv, bool color, const int32_t* __restrict__ ids, int B,
                                    const float* __restrict__ G, GridSrc src, float* __restrict__ ggrad) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = k < B;
    int kc = valid ? k : 0;
    const NetView& nv = color ? mv.color : mv.endpoint;
    float g[2 * NTBC_MAX_LEVELS];
#pragma unroll
    for (int i = 0; i < 2 * NTBC_MAX_LEVELS; ++i) g[i] = (valid && i < 2 * nv.levels) ? G[(long long)i * B + kc] : 0.f;
    scatter_sample(mv, color, ids, kc, k, valid, g, src, ggrad);
}

// ---------------------------------------------------------------------------
// Adam (dense)
// ---------------------------------------------------------------------------

// one Adam update; step = lr / (1 - beta1^t), rsb2 = 1 / sqrt(1 - beta2^t):
// p -= lr (m / bc1) / (sqrt(v / bc2) + eps), rearranged so that each element costs one
// square root and one (fast) division
__device__ __forceinline__ void adam_one(float& p, float g, float& m, float& v, float step, float rsb2) {
    m = fmaf(0.9f, m, 0.1f * g);
    v = fmaf(0.999f, v, 0.001f * g * g);
    p -= step * __fdividef(m, fmaf(sqrtf(v), rsb2, kAdamEps));
}

__device__ __forceinline__ void adam4(float4& P, float4 G, float4& M, float4& V, long long e, long long grid_floats,
                                      float step_g, float step_m, float rsb2) {
    adam_one(P.x, G.x, M.x, V.x, e < grid_floats ? step_g : step_m, rsb2);
    adam_one(P.y, G.y, M.y, V.y, e + 1 < grid_floats ? step_g : step_m, rsb2);
    adam_one(P.z, G.z, M.z, V.z, e + 2 < grid_floats ? step_g : step_m, rsb2);
    adam_one(P.w, G.w, M.w, V.w, e + 3 < grid_floats ? step_g : step_m, rsb2);
}

// dense Adam over all parameters, two float4 of every array in flight per thread; the
// streams are touched once per step, so they bypass L2 retention (evict-first hints)
// advance: a captured training step, whose last kernel this is, moves the step counter on
// gclear (the training step's own gradient buffer, = g): every gradient read is cleared for
// the next step where it is nonzero, so the buffer stays zero without a dense clear (a step's
// grid scatter touches a few million of the 16.8 M entries)
// the BF16 weight images of the tensor-core pass (both networks), rewritten by the training
// step's Adam for the MLP parameters it updates, so no per-step image kernel is needed
struct AdamImages {
    TrNet net[2];
    unsigned char* img[2];
    long long lo, hi;         // the MLP parameters: [lo, hi) of the parameter buffer
    int on;
};

// image element of parameter e (W[o][i] at row o, column i; b[o] at row o, column in), and its
// lo part where the network has one
__device__ __forceinline__ void image_store(const AdamImages& im, long long e, float w) {
#pragma unroll 1
    for (int k = 0; k < 2; ++k) {
        const TrNet& n = im.net[k];
#pragma unroll 1
        for (int l = 0; l < n.n_layers; ++l) {
            const TrLayer& L = n.layer[l];
            long long d = e - L.w_off;
            int row = -1, col = 0;
            if (d >= 0 && d < (long long)L.out * L.in) {
                row = (int)(d / L.in);
                col = (int)(d % L.in);
            } else if (e >= L.b_off && e < L.b_off + L.out) {
                row = (int)(e - L.b_off);
                col = L.in;
            }
            if (row >= 0) {
                unsigned char* t = im.img[k] + L.img + core_byte(row, col, L.K);
                const __nv_bfloat16 hi = __float2bfloat16_rn(w);
                *reinterpret_cast<__nv_bfloat16*>(t) = hi;
                if (n.lo_img)          // the endpoint network's lo parts
                    *reinterpret_cast<__nv_bfloat16*>(t + n.lo_img) = __float2bfloat16_rn(w - __bfloat162float(hi));
                return;
            }
        }
    }
}

__device__ __forceinline__ void image_update(const AdamImages& im, long long e, float4 P) {
    if (!im.on || e + 3 < im.lo || e >= im.hi) return;
    const float w[4] = {P.x, P.y, P.z, P.w};
#pragma unroll 1
    for (int j = 0; j < 4; ++j)
        if (e + j >= im.lo && e + j < im.hi) image_store(im, e + j, w[j]);
}

__device__ __forceinline__ void clear_used(float* gclear, long long i4, float4 G) {
    if (gclear && (G.x != 0.f || G.y != 0.f || G.z != 0.f || G.w != 0.f))
        __stcs(reinterpret_cast<float4*>(gclear) + i4, make_float4(0.f, 0.f, 0.f, 0.f));
}

__global__ void adam_kernel(float* __restrict__ p, const float* g, float* __restrict__ m,
                            float* __restrict__ v, long long n, long long grid_floats, StepState* __restrict__ st,
                            int advance, float* gclear, const __grid_constant__ AdamImages im) {
    const float inv_bc1 = 1.f / st->bc1, rsb2 = rsqrtf(st->bc2);
    const float step_g = st->lr_grid * inv_bc1, step_m = st->lr_mlp * inv_bc1;
    const long long n4 = n / 4;
    float4* P4 = reinterpret_cast<float4*>(p);
    const float4* G4 = reinterpret_cast<const float4*>(g);
    float4* M4 = reinterpret_cast<float4*>(m);
    float4* V4 = reinterpret_cast<float4*>(v);
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + stride < n4; i += 2 * stride) {
        const long long j = i + stride;
        float4 Pa = __ldcs(P4 + i), Ga = __ldcs(G4 + i), Ma = __ldcs(M4 + i), Va = __ldcs(V4 + i);
        float4 Pb = __ldcs(P4 + j), Gb = __ldcs(G4 + j), Mb = __ldcs(M4 + j), Vb = __ldcs(V4 + j);
        adam4(Pa, Ga, Ma, Va, 4 * i, grid_floats, step_g, step_m, rsb2);
        adam4(Pb, Gb, Mb, Vb, 4 * j, grid_floats, step_g, step_m, rsb2);
        clear_used(gclear, i, Ga);
        clear_used(gclear, j, Gb);
        image_update(im, 4 * i, Pa);
        image_update(im, 4 * j, Pb);
        __stcs(P4 + i, Pa);
        __stcs(M4 + i, Ma);
        __stcs(V4 + i, Va);
        __stcs(P4 + j, Pb);
        __stcs(M4 + j, Mb);
        __stcs(V4 + j, Vb);
    }
    if (i < n4) {
        float4 Pa = __ldcs(P4 + i), Ga = __ldcs(G4 + i), Ma = __ldcs(M4 + i), Va = __ldcs(V4 + i);
        adam4(Pa, Ga, Ma, Va, 4 * i, grid_floats, step_g, step_m, rsb2);
        clear_used(gclear, i, Ga);
        image_update(im, 4 * i, Pa);
        __stcs(P4 + i, Pa);
        __stcs(M4 + i, Ma);
        __stcs(V4 + i, Va);
    }
    if (blockIdx.x == 0 && threadIdx.x < n - 4 * n4) {
        long long e = 4 * n4 + threadIdx.x;
        adam_one(p[e], g[e], m[e], v[e], e < grid_floats ? step_g : step_m, rsb2);
        if (gclear) gclear[e] = 0.f;
        if (im.on && e >= im.lo && e < im.hi) image_store(im, e, p[e]);
    }
    if (advance && blockIdx.x == 0 && threadIdx.x == 0) st->step += 1;   // nothing of this kernel reads it
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static void free_net(NetBuffers& nb) {
    cudaFree(nb.X);
    for (int l = 0; l < 3; ++l) cudaFree(nb.A[l]);
    cudaFree(nb.Y);
    cudaFree(nb.D0);
    cudaFree(nb.D1);
    memset(&nb, 0, sizeof(nb));
}

void ntbc_train_release(ntbc_model* m) {
    ntbc_train_state* ts = m->train;
    if (!ts) return;
    free_net(ts->color);
    free_net(ts->endpoint);
    cudaFree(ts->ids);
    cudaFree(ts->grads);
    cudaFree(ts->loss_acc);
    cudaFree(ts->st);
    cudaFree(ts->qscale);
    cudaFree(ts->tc_img);
    cudaFree(ts->tc_part);
    cudaFree(ts->sched);
    delete ts;
    m->train = nullptr;
}

static ntbc_status alloc_net(NetBuffers& nb, int cap, int out_dim) {
    nb.cap = cap;
    ntbc_status st = device_alloc((void**)&nb.X, (size_t)kMaxIn * cap * sizeof(float), "features");
    for (int l = 0; l < 3 && st == NTBC_OK; ++l) st = device_alloc((void**)&nb.A[l], (size_t)kHidden * cap * sizeof(float), "activations");
    if (st == NTBC_OK) st = device_alloc((void**)&nb.Y, (size_t)out_dim * cap * sizeof(float), "outputs");
    if (st == NTBC_OK) st = device_alloc((void**)&nb.D0, (size_t)kHidden * cap * sizeof(float), "deltas");
    if (st == NTBC_OK) st = device_alloc((void**)&nb.D1, (size_t)kHidden * cap * sizeof(float), "deltas");
    return st;
}

static ntbc_status ensure_train_state(ntbc_model* m, int n_blocks) {
    ntbc_train_state* ts = m->train;
    if (ts && ts->cap_blocks >= n_blocks) return NTBC_OK;
    int levels = m->desc.color_levels + m->desc.endpoint_levels;
    float* grads_keep = nullptr;
    if (ts) {
        free_net(ts->color);
        free_net(ts->endpoint);
        cudaFree(ts->ids);
        ts->ids = nullptr;
    } else {
        ts = new ntbc_train_state();
        m->train = ts;
        ntbc_status st = device_alloc((void**)&ts->grads, m->layout.total * sizeof(float), "gradients");
        if (st == NTBC_OK) st = device_alloc((void**)&ts->loss_acc, 6 * sizeof(double) + 6 * sizeof(float), "losses");
        if (st == NTBC_OK) st = device_alloc((void**)&ts->st, sizeof(StepState), "step state");
        if (st == NTBC_OK) st = device_alloc((void**)&ts->qscale, levels * (2 * sizeof(float) + 2 * sizeof(unsigned)), "QAT scales");
        if (st != NTBC_OK) {
            ntbc_train_release(m);
            return st;
        }
        ts->losses = reinterpret_cast<float*>(ts->loss_acc + 6);
        ts->qzero = ts->qscale + levels;
        ts->qmm = reinterpret_cast<unsigned*>(ts->qscale + 2 * levels);
        NTBC_CHECK_CUDA(cudaMemset(ts->st, 0, sizeof(StepState)));
        ModelView mv = make_view(m->desc, m->layout);
        size_t img = (size_t)train_tc_net_desc(mv, true).img_bytes + train_tc_net_desc(mv, false).img_bytes;
        st = device_alloc((void**)&ts->tc_img, img + 16, "training weight images");
        if (st != NTBC_OK) {
            ntbc_train_release(m);
            return st;
        }
        ts->tc_err = reinterpret_cast<int*>(ts->tc_img + img);
        NTBC_CHECK_CUDA(cudaMemset(ts->tc_err, 0, sizeof(int)));
        TrNet cn = train_tc_net_desc(mv, true), en = train_tc_net_desc(mv, false);
        ts->tc_part_rows = train_tc_max_partial_rows();
        // one scratch per network: both are reduced by one launch after the two passes
        size_t part = (size_t)ts->tc_part_rows * ((size_t)cn.mlp_params + en.mlp_params) * sizeof(float);
        st = device_alloc((void**)&ts->tc_part, part, "weight-gradient partials");
        if (st != NTBC_OK) {
            ntbc_train_release(m);
            return st;
        }
    }
    (void)grads_keep;
    ts->cap_blocks = n_blocks;
    const ntbc_layout& L = m->layout;
    ntbc_status st = alloc_net(ts->color, n_blocks * 16, L.out_color);
    if (st == NTBC_OK) st = alloc_net(ts->endpoint, n_blocks, L.out_endpoint);
    if (st == NTBC_OK) st = device_alloc((void**)&ts->ids, (size_t)n_blocks * sizeof(int32_t), "batch ids");
    if (st != NTBC_OK) ntbc_train_release(m);
    return st;
}

static ntbc_status ensure_adam(ntbc_model* m) {
    if (m->adam_m) return NTBC_OK;
    size_t bytes = m->layout.total * sizeof(float);
    ntbc_status st = device_alloc((void**)&m->adam_m, bytes, "Adam m");
    if (st == NTBC_OK) st = device_alloc((void**)&m->adam_v, bytes, "Adam v");
    if (st != NTBC_OK) return st;
    NTBC_CHECK_CUDA(cudaMemset(m->adam_m, 0, bytes));
    NTBC_CHECK_CUDA(cudaMemset(m->adam_v, 0, bytes));
    return NTBC_OK;
}

static inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

static ntbc_status check_material(const ntbc_model* m, const ntbc_material* mat) {
    if (!mat) return fail(NTBC_EINVAL, "null material");
    if (mat->width != m->desc.width || mat->height != m->desc.height || mat->n_textures != m->desc.n_textures)
        return fail(NTBC_EINVAL, "material does not match the model (size or texture count)");
    for (int t = 0; t < mat->n_textures; ++t) {
        if (mat->formats[t] != m->desc.formats[t]) return fail(NTBC_EINVAL, "texture %d: format differs from the model", t);
        if (!mat->texels[t] || !mat->ref_blocks[t]) return fail(NTBC_EINVAL, "texture %d: null texels or reference blocks", t);
    }
    return NTBC_OK;
}

// gather + dense layers of one network on the batch: features in nb.X, hidden
// activations in nb.A, sigmoid outputs in nb.Y (feature-major)
static void net_forward(const float* params, const ModelView& mv, bool color, NetBuffers& nb, const int32_t* ids,
                        int B, GridSrc src, cudaStream_t s) {
    const NetView& nv = color ? mv.color : mv.endpoint;
    const int thr = 128;
    unsigned g = blocks_for(B, thr);
    gather_kernel<<<g, thr, 0, s>>>(mv, color, src, ids, B, nb.X);
    const float* prev = nb.X;
    int nl = nv.n_layers;
    for (int l = 0; l < nl; ++l) {
        bool last = l + 1 == nl;
        float* outbuf = last ? nb.Y : nb.A[l];
        int act = last ? 2 : mv.activation;
        if (l == 0)
            dense_fwd_kernel<kMaxIn><<<g, thr, 0, s>>>(prev, nv.layer_in[l], B, params + nv.w_off[l], params + nv.b_off[l], nv.layer_out[l], act, outbuf);
        else
            dense_fwd_kernel<kHidden><<<g, thr, 0, s>>>(prev, nv.layer_in[l], B, params + nv.w_off[l], params + nv.b_off[l], nv.layer_out[l], act, outbuf);
        prev = outbuf;
    }
}

// backward from the output-layer deltas in nb.D0 (d loss / d pre-sigmoid): weight and
// bias gradients, input gradients, and the grid scatter-add (through the QAT mask)
static void net_backward(const float* params, const ModelView& mv, bool color, NetBuffers& nb, const int32_t* ids,
                         int B, GridSrc src, float* grads, cudaStream_t s) {
    const NetView& nv = color ? mv.color : mv.endpoint;
    const int thr = 128;
    unsigned g = blocks_for(B, thr);
    float* D = nb.D0;
    float* Dn = nb.D1;
    unsigned gw = blocks_for(B, kWgChunk);
    for (int l = nv.n_layers - 1; l >= 0; --l) {
        const float* Ain = l == 0 ? nb.X : nb.A[l - 1];
        dense_bwd_weight_kernel<<<gw, 256, 0, s>>>(D, nv.layer_out[l], Ain, nv.layer_in[l], B, grads + nv.w_off[l], grads + nv.b_off[l]);
        dense_bwd_data_kernel<<<g, thr, 0, s>>>(D, nv.layer_out[l], B, params + nv.w_off[l], nv.layer_in[l],
                                                 l == 0 ? nullptr : nb.A[l - 1], mv.activation, Dn);
        float* t = D;
        D = Dn;
        Dn = t;
    }
    grid_scatter_kernel<<<g, thr, 0, s>>>(mv, color, ids, B, D, src, grads);
}

// one network's forward + loss + backward on the gathered batch, on given parameters and
// buffers (the model's training state, or the allocation-free entry point's scratch)
static void net_step(const float* params, const ModelView& mv, bool color, const TexPtrs& tp, const int32_t* ids,
                     int B, GridSrc src, float T, NetBuffers& nb, float* grads, double* acc, cudaStream_t s) {
    net_forward(params, mv, color, nb, ids, B, src, s);
    const int thr = 128;
    if (color)
        color_loss_kernel<<<blocks_for(B, thr), thr, 0, s>>>(mv, tp, ids, B, nb.Y, T, nb.D0, acc);
    else
        endpoint_loss_kernel<<<blocks_for((long long)B * 16, thr), thr, 0, s>>>(mv, tp, ids, B, nb.Y, T, nb.D0, acc);
    net_backward(params, mv, color, nb, ids, B, src, grads, s);
}

static ntbc_status run_net(ntbc_model* m, const ModelView& mv, bool color, const TexPtrs& tp, const int32_t* ids, int B,
                           GridSrc src, float T, float* grads, double* acc, cudaStream_t s) {
    net_step(m->params, mv, color, tp, ids, B, src, T, color ? m->train->color : m->train->endpoint, grads, acc, s);
    NTBC_CHECK_LAUNCH(color ? "colour network step" : "endpoint network step");
    return NTBC_OK;
}

// outputs to the row-major [k][o] layout of ntbc_forward and, with an upstream gradient g
// (same layout), the output-layer deltas D[o][k] = g[k][o] y (1 - y)
__global__ void vjp_seed_kernel(const float* __restrict__ Y, int out, int B, const float* __restrict__ g,
                                float* __restrict__ D, float* __restrict__ y_out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * out) return;
    long long k = i / out;
    int o = (int)(i % out);
    float y = Y[(long long)o * B + k];
    if (y_out) y_out[i] = y;
    if (g) D[(long long)o * B + k] = g[i] * y * (1.f - y);
}

// grid sources of the FP32 master parameters, with static QAT fake quantisation
static ntbc_status train_sources(ntbc_model* m, int qat_bits, GridSrc& csrc, GridSrc& esrc,
                                 cudaStream_t s) {
    ntbc_train_state* ts = m->train;
    memset(&csrc, 0, sizeof(csrc));
    csrc.f32 = m->params;
    csrc.qat_bits = qat_bits;
    esrc = csrc;
    if (qat_bits > 0) {
        LevelTable lt = level_table(m->desc, m->layout);
        ntbc_status st = launch_level_scale_zero(m->params, lt, qat_bits, ts->qmm, ts->qscale, ts->qzero, s);
        if (st != NTBC_OK) return st;
        csrc.scale = ts->qscale;
        csrc.zero = ts->qzero;
        esrc.scale = ts->qscale + m->desc.color_levels;
        esrc.zero = ts->qzero + m->desc.color_levels;
    }
    return NTBC_OK;
}

// in_step: inside a captured training step, whose sampler clears the loss accumulators and
// whose losses are turned into floats once after the last step
static ntbc_status grads_on_ids(ntbc_model* m, const ntbc_material* mat, const int32_t* ids, int nb, int qat_bits,
                                float T, int precision, float* grads, cudaStream_t s, bool in_step = false) {
    ntbc_train_state* ts = m->train;
    ModelView mv = make_view(m->desc, m->layout);
    TexPtrs tp;
    memset(&tp, 0, sizeof(tp));
    for (int t = 0; t < mat->n_textures; ++t) {
        tp.texels[t] = mat->texels[t];
        tp.blocks[t] = mat->ref_blocks[t];
    }
    GridSrc csrc, esrc;
    ntbc_status st0 = train_sources(m, qat_bits, csrc, esrc, s);
    if (st0 != NTBC_OK) return st0;
    // a captured step's gradients start at zero: the step's Adam clears every entry it used
    if (!in_step) NTBC_CHECK_CUDA(cudaMemsetAsync(grads, 0, m->layout.total * sizeof(float), s));
    if (!in_step) NTBC_CHECK_CUDA(cudaMemsetAsync(ts->loss_acc, 0, 6 * sizeof(double), s));
    ntbc_status st;
    if (precision == NTBC_TRAIN_BF16) {
        TrNet cn = train_tc_net_desc(mv, true), en = train_tc_net_desc(mv, false);
        unsigned char* cimg = ts->tc_img;
        unsigned char* eimg = ts->tc_img + cn.img_bytes;
        float* cpart = ts->tc_part;
        float* epart = ts->tc_part + (size_t)ts->tc_part_rows * cn.mlp_params;
        int crows = 0, erows = 0;
        // a captured step reads the images its previous step's Adam rewrote (built once before
        // the first step of a range)
        st = in_step ? NTBC_OK : train_tc_images(m->params, cn, cimg, en, eimg, s);
        if (st == NTBC_OK)
            st = train_tc_launch(mv, true, cn, cimg, csrc, tp, ids, nb * 16, T, grads, ts->loss_acc, ts->tc_err,
                                 cpart, ts->tc_part_rows, &crows, s);
        if (st == NTBC_OK)
            st = train_tc_launch(mv, false, en, eimg, esrc, tp, ids, nb, T, grads, ts->loss_acc, ts->tc_err,
                                 epart, ts->tc_part_rows, &erows, s);
        if (st == NTBC_OK) st = train_tc_reduce(cn, cpart, crows, en, epart, erows, grads, s);
    } else {
        st = run_net(m, mv, true, tp, ids, nb * 16, csrc, T, grads, ts->loss_acc, s);
        if (st == NTBC_OK) st = run_net(m, mv, false, tp, ids, nb, esrc, T, grads, ts->loss_acc, s);
    }
    if (st != NTBC_OK) return st;
    if (in_step) return NTBC_OK;
    loss_finalize_kernel<<<1, 32, 0, s>>>(ts->loss_acc, ts->losses);
    NTBC_CHECK_LAUNCH("loss finalize");
    return NTBC_OK;
}

static ntbc_status adam_launch(ntbc_model* m, const float* grads, cudaStream_t s, int advance = 0,
                               float* clear = nullptr, const AdamImages* images = nullptr) {
    long long n = (long long)m->layout.total;
    unsigned g = (unsigned)std::min<long long>(blocks_for(n, 256), 152LL * 16);
    AdamImages im;
    memset(&im, 0, sizeof(im));
    if (images) im = *images;
    adam_kernel<<<g, 256, 0, s>>>(m->params, grads, m->adam_m, m->adam_v, n, (long long)m->layout.grid_floats, m->train->st,
                                  advance, clear, im);
    NTBC_CHECK_LAUNCH("adam");
    return NTBC_OK;
}

// A stream created for one call: drained and destroyed on every return path.
struct OwnedStream {
    cudaStream_t s = nullptr;
    ~OwnedStream() {
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
};

// Capture one training step (qbits > 0: a QAT-phase step) as a graph on `cap`.
// the training step's weight images and their MLP parameter range (BF16 pass)
static AdamImages step_images(const ntbc_model* m) {
    AdamImages im;
    memset(&im, 0, sizeof(im));
    const ModelView mv = make_view(m->desc, m->layout);
    im.net[0] = train_tc_net_desc(mv, true);
    im.net[1] = train_tc_net_desc(mv, false);
    im.img[0] = m->train->tc_img;
    im.img[1] = m->train->tc_img + im.net[0].img_bytes;
    im.lo = std::min(im.net[0].mlp_base, im.net[1].mlp_base);
    im.hi = std::max(im.net[0].mlp_base + im.net[0].mlp_params, im.net[1].mlp_base + im.net[1].mlp_params);
    im.on = 1;
    return im;
}

static ntbc_status capture_step(ntbc_model* m, const ntbc_material* mat, const ntbc_train_config* cfg, int nb,
                                int n_blocks, long long total, int qbits, cudaStream_t cap, cudaGraphExec_t* exec) {
    ntbc_train_state* ts = m->train;
    cudaGraph_t graph = nullptr;
    NTBC_CHECK_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    sample_kernel<<<blocks_for(nb, 256), 256, 0, cap>>>(cfg->seed, ts->st, ts->sched, total, 0, nb, n_blocks, ts->ids,
                                                        ts->loss_acc);
    ntbc_status st = grads_on_ids(m, mat, ts->ids, nb, qbits, cfg->temperature, cfg->precision, ts->grads, cap, true);
    // Adam clears the gradients it used and, for the BF16 pass, rewrites the weight images
    const AdamImages im = step_images(m);
    if (st == NTBC_OK)
        st = adam_launch(m, ts->grads, cap, 1, ts->grads, cfg->precision == NTBC_TRAIN_BF16 ? &im : nullptr);
    cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    if (st != NTBC_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return st != NTBC_OK ? st : cuda_fail(ce, "cudaStreamEndCapture");
    }
    ce = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        *exec = nullptr;
        return cuda_fail(ce, "cudaGraphInstantiate");
    }
    return NTBC_OK;
}

}  // namespace ntbc

using namespace ntbc;

extern "C" {

ntbc_status ntbc_sample_blocks(uint64_t seed, long step, int n, int n_blocks, int32_t* ids, void* stream) {
    clear_error();
    if (!ids || n < 0 || n_blocks <= 0) return fail(NTBC_EINVAL, "need ids, n >= 0 and n_blocks > 0");
    if (n == 0) return NTBC_OK;
    sample_kernel<<<blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(seed, nullptr, nullptr, 0, step, n, n_blocks, ids,
                                                                        nullptr);
    NTBC_CHECK_LAUNCH("sample blocks");
    return NTBC_OK;
}

ntbc_status ntbc_train_grads(ntbc_model* m, const ntbc_material* mat, const int32_t* block_ids, int n_blocks,
                             int qat_bits, float temperature, int precision, float* grads, float* losses, void* stream) {
    ntbc::NvtxRange nvtx_range("ntbc_train_grads");
    clear_error();
    if (!m || !block_ids || !grads) return fail(NTBC_EINVAL, "null argument");
    ntbc_status st = check_material(m, mat);
    if (st != NTBC_OK) return st;
    if (n_blocks <= 0) return fail(NTBC_EINVAL, "need at least one block");
    if (qat_bits != 0 && qat_bits != 8 && qat_bits != 4) return fail(NTBC_EINVAL, "qat_bits must be 0, 4 or 8");
    if (!(temperature > 0.f)) return fail(NTBC_EINVAL, "temperature must be positive");
    if (precision != NTBC_TRAIN_FP32 && precision != NTBC_TRAIN_BF16) return fail(NTBC_EINVAL, "unknown training precision");
    st = ensure_train_state(m, n_blocks);
    if (st != NTBC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = grads_on_ids(m, mat, block_ids, n_blocks, qat_bits, temperature, precision, grads, s);
    if (st != NTBC_OK) return st;
    if (losses) NTBC_CHECK_CUDA(cudaMemcpyAsync(losses, m->train->losses, 6 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return NTBC_OK;
}

ntbc_status ntbc_vjp(ntbc_model* m, const int32_t* block_ids, int n_blocks, int qat_bits, const float* g_e,
                     const float* g_c, float* grads, float* e_hat, float* c_hat, void* stream) {
    clear_error();
    if (!m || !block_ids) return fail(NTBC_EINVAL, "null argument");
    if (n_blocks <= 0) return fail(NTBC_EINVAL, "need at least one block");
    if (qat_bits != 0 && qat_bits != 8 && qat_bits != 4) return fail(NTBC_EINVAL, "qat_bits must be 0, 4 or 8");
    if ((g_e == nullptr) != (g_c == nullptr)) return fail(NTBC_EINVAL, "give both upstream gradients or neither");
    if (g_e && !grads) return fail(NTBC_EINVAL, "upstream gradients need a gradient buffer");
    ntbc_status st = ensure_train_state(m, n_blocks);
    if (st != NTBC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    GridSrc csrc, esrc;
    st = train_sources(m, qat_bits, csrc, esrc, s);
    if (st != NTBC_OK) return st;
    ModelView mv = make_view(m->desc, m->layout);
    if (g_e) NTBC_CHECK_CUDA(cudaMemsetAsync(grads, 0, m->layout.total * sizeof(float), s));
    for (int net = 0; net < 2; ++net) {
        const bool color = net == 0;
        NetBuffers& nb = color ? m->train->color : m->train->endpoint;
        const int B = color ? n_blocks * 16 : n_blocks;
        const int out = color ? m->layout.out_color : m->layout.out_endpoint;
        net_forward(m->params, mv, color, nb, block_ids, B, color ? csrc : esrc, s);
        vjp_seed_kernel<<<blocks_for((long long)B * out, 256), 256, 0, s>>>(nb.Y, out, B, color ? g_c : g_e, nb.D0,
                                                                            color ? c_hat : e_hat);
        if (g_e) net_backward(m->params, mv, color, nb, block_ids, B, color ? csrc : esrc, grads, s);
        NTBC_CHECK_LAUNCH(color ? "colour network vjp" : "endpoint network vjp");
    }
    return NTBC_OK;
}

ntbc_status ntbc_adam_step(ntbc_model* m, const float* grads, long step, long total_steps, const ntbc_train_config* cfg,
                           void* stream) {
    clear_error();
    if (!m || !grads || !cfg) return fail(NTBC_EINVAL, "null argument");
    if (step < 0 || total_steps <= 0 || step >= total_steps) return fail(NTBC_EINVAL, "step outside [0, total_steps)");
    ntbc_status st = ensure_train_state(m, 1);
    if (st == NTBC_OK) st = ensure_adam(m);
    if (st != NTBC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (step == 0) {
        NTBC_CHECK_CUDA(cudaMemsetAsync(m->adam_m, 0, m->layout.total * sizeof(float), s));
        NTBC_CHECK_CUDA(cudaMemsetAsync(m->adam_v, 0, m->layout.total * sizeof(float), s));
    }
    step_begin_kernel<<<1, 32, 0, s>>>(m->train->st, step, total_steps, cfg->lr_grid, cfg->lr_mlp, cfg->warmup);
    NTBC_CHECK_LAUNCH("step begin");
    return adam_launch(m, grads, s);
}

ntbc_status ntbc_train_range(ntbc_model* m, const ntbc_material* mat, const ntbc_train_config* cfg, long first_step,
                             long last_step, float* losses_out, void* stream) {
    ntbc::NvtxRange nvtx_range("ntbc_train_range");
    clear_error();
    if (!m || !cfg) return fail(NTBC_EINVAL, "null argument");
    ntbc_status st = check_material(m, mat);
    if (st != NTBC_OK) return st;
    if (cfg->steps <= 0 || cfg->batch_texels < 16 || (cfg->batch_texels & 15))
        return fail(NTBC_EINVAL, "need steps > 0 and batch_texels a positive multiple of 16");
    if (cfg->qat_fraction < 0.f || (cfg->qat_fraction > 0.f && cfg->grid_bits != 8 && cfg->grid_bits != 4))
        return fail(NTBC_EINVAL, "QAT needs grid_bits 8 or 4");
    if (!(cfg->temperature > 0.f) || cfg->warmup < 0) return fail(NTBC_EINVAL, "bad temperature or warm-up");
    if (cfg->precision != NTBC_TRAIN_FP32 && cfg->precision != NTBC_TRAIN_BF16)
        return fail(NTBC_EINVAL, "unknown training precision");
    int nb = cfg->batch_texels / 16;
    int n_blocks = (m->desc.width / 4) * (m->desc.height / 4);
    long long qat_steps = cfg->qat_fraction > 0.f ? (long long)std::ceil((double)cfg->qat_fraction * (double)cfg->steps) : 0;
    long long total = cfg->steps + qat_steps;
    int qbits = qat_steps > 0 ? cfg->grid_bits : 0;
    if (first_step < 0 || last_step <= first_step || last_step > total)
        return fail(NTBC_EINVAL, "step range [%ld, %ld) outside the schedule's %lld steps", first_step, last_step, total);
    if (first_step > 0 && !m->adam_m)
        return fail(NTBC_EINVAL, "resuming at step %ld needs the Adam state (train the earlier steps or load a checkpoint)",
                    first_step);
    st = ensure_train_state(m, nb);
    if (st == NTBC_OK) st = ensure_adam(m);
    if (st != NTBC_OK) return st;
    ntbc_train_state* ts = m->train;
    cudaStream_t s = (cudaStream_t)stream;
    OwnedStream owned;
    NTBC_CHECK_CUDA(cudaStreamCreateWithFlags(&owned.s, cudaStreamNonBlocking));
    cudaStream_t cap = owned.s;
    NTBC_CHECK_CUDA(cudaStreamSynchronize(s));
    if (first_step == 0) {          // a fresh encode: Adam moments start at zero
        NTBC_CHECK_CUDA(cudaMemsetAsync(m->adam_m, 0, m->layout.total * sizeof(float), cap));
        NTBC_CHECK_CUDA(cudaMemsetAsync(m->adam_v, 0, m->layout.total * sizeof(float), cap));
    }
    // the captured steps' gradient buffer starts at zero (each step's Adam keeps it so), and
    // the BF16 weight images start from the current parameters (each step's Adam keeps them)
    NTBC_CHECK_CUDA(cudaMemsetAsync(ts->grads, 0, m->layout.total * sizeof(float), cap));
    if (cfg->precision == NTBC_TRAIN_BF16) {
        const AdamImages im = step_images(m);
        st = train_tc_images(m->params, im.net[0], im.img[0], im.net[1], im.img[1], cap);
        if (st != NTBC_OK) return st;
    }
    {                               // the step counter the sampler, schedule and Adam read
        StepState st0;
        memset(&st0, 0, sizeof(st0));
        st0.step = first_step;
        NTBC_CHECK_CUDA(cudaMemcpyAsync(ts->st, &st0, sizeof(StepState), cudaMemcpyHostToDevice, cap));
        NTBC_CHECK_CUDA(cudaStreamSynchronize(cap));
    }
    if (ts->sched_cap < total) {
        cudaFree(ts->sched);
        ts->sched = nullptr;
        ts->sched_cap = 0;
        st = device_alloc((void**)&ts->sched, (size_t)total * sizeof(StepSchedule), "step schedule");
        if (st != NTBC_OK) return st;
        ts->sched_cap = total;
    }
    schedule_kernel<<<(unsigned)std::min<long long>((total + 255) / 256, 1024), 256, 0, cap>>>(
        ts->sched, total, cfg->lr_grid, cfg->lr_mlp, cfg->warmup);
    NTBC_CHECK_LAUNCH("step schedule");
    // one graph per phase (the main phase without the QAT kernels, the QAT phase with them),
    // each launched once per step; every quantity that changes per step lives in StepState
    cudaGraphExec_t exec_main = nullptr, exec_qat = nullptr;
    // the main-phase steps of the range, then its QAT-phase steps
    const long long main_n = std::max(0LL, std::min((long long)last_step, (long long)cfg->steps) - first_step);
    const long long qat_n = (long long)last_step - first_step - main_n;
    if (main_n > 0) st = capture_step(m, mat, cfg, nb, n_blocks, total, 0, cap, &exec_main);
    if (st == NTBC_OK && qat_n > 0) st = capture_step(m, mat, cfg, nb, n_blocks, total, qbits, cap, &exec_qat);
    cudaError_t ce = cudaSuccess;
    if (st == NTBC_OK) {
        for (long long t = 0; t < main_n && ce == cudaSuccess; ++t) ce = cudaGraphLaunch(exec_main, cap);
        for (long long t = 0; t < qat_n && ce == cudaSuccess; ++t) ce = cudaGraphLaunch(exec_qat, cap);
        if (ce == cudaSuccess) {              // the last step's losses
            loss_finalize_kernel<<<1, 32, 0, cap>>>(ts->loss_acc, ts->losses);
            ce = cudaGetLastError();
            // host-side fault injection of a diverged encode: NTBC_FAULT=nan overwrites the
            // finalised losses with NaN, so the non-finite check below is exercised
            if (ce == cudaSuccess && fault_injected("nan")) ce = cudaMemsetAsync(ts->losses, 0xFF, 6 * sizeof(float), cap);
        }
    }
    cudaError_t se = cudaStreamSynchronize(cap);
    if (exec_main) cudaGraphExecDestroy(exec_main);
    if (exec_qat) cudaGraphExecDestroy(exec_qat);
    if (st != NTBC_OK) return st;
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphLaunch");
    if (se != cudaSuccess) return cuda_fail(se, "training steps");
    int tc_err = 0;
    NTBC_CHECK_CUDA(cudaMemcpy(&tc_err, ts->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (tc_err) return fail(NTBC_ETIMEOUT, "tensor-core training: a bounded wait gave up");
    float host_losses[6];
    NTBC_CHECK_CUDA(cudaMemcpy(host_losses, ts->losses, sizeof(host_losses), cudaMemcpyDeviceToHost));
    if (losses_out) memcpy(losses_out, host_losses, sizeof(host_losses));
    m->next_step = last_step;
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(host_losses[i])) return fail(NTBC_ENONFINITE, "non-finite loss after training");
    return NTBC_OK;
}


ntbc_status ntbc_train(ntbc_model* m, const ntbc_material* mat, const ntbc_train_config* cfg, float* losses_out,
                       void* stream) {
    ntbc::NvtxRange nvtx_range("ntbc_train");
    clear_error();
    if (!cfg) return fail(NTBC_EINVAL, "null argument");
    const long long qat_steps =
        cfg->qat_fraction > 0.f ? (long long)std::ceil((double)cfg->qat_fraction * (double)cfg->steps) : 0;
    return ntbc_train_range(m, mat, cfg, 0, (long)(cfg->steps + qat_steps), losses_out, stream);
}

namespace {

// Training checkpoint: header, then the FP32 master parameters, Adam m and Adam v.
struct CheckpointHeader {
    char magic[4];               // "NTCK"
    int version;                 // ntbc_abi_version()
    ntbc_model_desc desc;        // the model it belongs to
    unsigned long long total;    // floats per array
    long long next_step;         // the step a resumed encode starts at
};

}  // namespace

ntbc_status ntbc_checkpoint_size(const ntbc_model* m, size_t* size) {
    clear_error();
    if (!m || !size) return fail(NTBC_EINVAL, "null argument");
    *size = sizeof(CheckpointHeader) + 3 * m->layout.total * sizeof(float);
    return NTBC_OK;
}

ntbc_status ntbc_checkpoint_save(ntbc_model* m, uint8_t* buf, size_t size, void* stream) {
    ntbc::NvtxRange nvtx_range("ntbc_checkpoint_save");
    clear_error();
    size_t need = 0;
    ntbc_status st = ntbc_checkpoint_size(m, &need);
    if (st != NTBC_OK) return st;
    if (!buf || size != need) return fail(NTBC_EINVAL, "checkpoint buffer must be %zu bytes", need);
    st = ensure_adam(m);               // a model that never trained saves zero moments
    if (st != NTBC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CheckpointHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "NTCK", 4);
    h.version = ntbc_abi_version();
    h.desc = m->desc;
    h.total = m->layout.total;
    h.next_step = m->next_step;
    const size_t bytes = m->layout.total * sizeof(float);
    memcpy(buf, &h, sizeof(h));
    uint8_t* p = buf + sizeof(h);
    NTBC_CHECK_CUDA(cudaMemcpyAsync(p, m->params, bytes, cudaMemcpyDeviceToHost, s));
    NTBC_CHECK_CUDA(cudaMemcpyAsync(p + bytes, m->adam_m, bytes, cudaMemcpyDeviceToHost, s));
    NTBC_CHECK_CUDA(cudaMemcpyAsync(p + 2 * bytes, m->adam_v, bytes, cudaMemcpyDeviceToHost, s));
    NTBC_CHECK_CUDA(cudaStreamSynchronize(s));
    return NTBC_OK;
}

ntbc_status ntbc_checkpoint_load(ntbc_model* m, const uint8_t* buf, size_t size, long* next_step, void* stream) {
    ntbc::NvtxRange nvtx_range("ntbc_checkpoint_load");
    clear_error();
    size_t need = 0;
    ntbc_status st = ntbc_checkpoint_size(m, &need);
    if (st != NTBC_OK) return st;
    if (!buf || size != need) return fail(NTBC_EINVAL, "checkpoint must be %zu bytes", need);
    CheckpointHeader h;
    memcpy(&h, buf, sizeof(h));
    if (memcmp(h.magic, "NTCK", 4) != 0 || h.version != ntbc_abi_version())
        return fail(NTBC_EINVAL, "not an NTBC checkpoint of this version");
    if (memcmp(&h.desc, &m->desc, sizeof(ntbc_model_desc)) != 0 || h.total != m->layout.total)
        return fail(NTBC_EINVAL, "the checkpoint belongs to another model");
    if (h.next_step < 0) return fail(NTBC_EINVAL, "bad step in checkpoint");
    st = ensure_adam(m);
    if (st != NTBC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = m->layout.total * sizeof(float);
    const uint8_t* p = buf + sizeof(h);
    NTBC_CHECK_CUDA(cudaMemcpyAsync(m->params, p, bytes, cudaMemcpyHostToDevice, s));
    NTBC_CHECK_CUDA(cudaMemcpyAsync(m->adam_m, p + bytes, bytes, cudaMemcpyHostToDevice, s));
    NTBC_CHECK_CUDA(cudaMemcpyAsync(m->adam_v, p + 2 * bytes, bytes, cudaMemcpyHostToDevice, s));
    NTBC_CHECK_CUDA(cudaStreamSynchronize(s));
    m->next_step = h.next_step;
    if (next_step) *next_step = (long)h.next_step;
    return NTBC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of the training-gradient call.
//
// Some callers cannot allocate device memory: an engine's texture-streaming
// thread that works inside a fixed, pre-reserved VRAM budget, or a real-time
// thread that cannot afford the device-wide synchronisation cudaMalloc implies.
// For them the scratch of one gradient evaluation (features, activations,
// deltas, loss accumulators, QAT scales) lives in the file-scope array below,
// sized for at most kNoAllocMaxBlocks blocks per call. Every GPU that loads the
// library holds the array until the process exits.
// ---------------------------------------------------------------------------

namespace ntbc {

constexpr int kNoAllocMaxBlocks = 128;                         // 2048 texels per call
constexpr int kNoAllocColor = kNoAllocMaxBlocks * 16;
constexpr size_t kNoAllocNetFloats(int cap, int out) { return (size_t)(kMaxIn + 3 * kHidden + out + 2 * kHidden) * cap; }
constexpr size_t kNoAllocFloats = kNoAllocNetFloats(kNoAllocColor, kMaxOutC) + kNoAllocNetFloats(kNoAllocMaxBlocks, kMaxOutE);
constexpr int kNoAllocLevels = 2 * NTBC_MAX_LEVELS;
// floats of both networks, then 6 double loss accumulators, then QAT scale / zero / min-max words
constexpr size_t kNoAllocBytes = kNoAllocFloats * sizeof(float) + 6 * sizeof(double) + kNoAllocLevels * 4 * sizeof(float);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static void* g_noalloc_addr[kNoAllocMaxDevices];
static std::mutex g_noalloc_mutex;

// Device address of the scratch array on the current device; looked up once per
// device (with that device current) on the first call.
static ntbc_status noalloc_scratch(unsigned char** out) {
    int dev = 0;
    NTBC_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(NTBC_EUNSUPPORTED, "device ordinal %d beyond %d", dev, kNoAllocMaxDevices);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
    return NTBC_OK;
}

static NetBuffers carve_net(float*& cursor, int cap, int out) {
    NetBuffers nb;
    nb.cap = cap;
    nb.X = cursor;
    cursor += (size_t)kMaxIn * cap;
    for (int l = 0; l < 3; ++l) {
        nb.A[l] = cursor;
        cursor += (size_t)kHidden * cap;
    }
    nb.Y = cursor;
    cursor += (size_t)out * cap;
    nb.D0 = cursor;
    cursor += (size_t)kHidden * cap;
    nb.D1 = cursor;
    cursor += (size_t)kHidden * cap;
    return nb;
}

}  // namespace ntbc

extern "C" {

ntbc_status ntbc_train_grads_noalloc(const ntbc_model_desc* desc, const float* params, const ntbc_material* mat,
                                     const int32_t* block_ids, int n_blocks, int qat_bits, float temperature,
                                     float* grads, float* losses, void* stream) {
    clear_error();
    ntbc_layout L;
    ntbc_status st = ntbc_model_layout(desc, &L);
    if (st != NTBC_OK) return st;
    if (!params || !mat || !block_ids || !grads || !losses) return fail(NTBC_EINVAL, "null argument");
    if (n_blocks <= 0) return fail(NTBC_EINVAL, "need at least one block");
    if (n_blocks > kNoAllocMaxBlocks)
        return fail(NTBC_EINVAL, "n_blocks %d exceeds the allocation-free limit of %d blocks (%d texels) per call",
                    n_blocks, kNoAllocMaxBlocks, kNoAllocMaxBlocks * 16);
    if (qat_bits != 0 && qat_bits != 8 && qat_bits != 4) return fail(NTBC_EINVAL, "qat_bits must be 0, 4 or 8");
    if (!(temperature > 0.f)) return fail(NTBC_EINVAL, "temperature must be positive");
    if (mat->width != desc->width || mat->height != desc->height || mat->n_textures != desc->n_textures)
        return fail(NTBC_EINVAL, "material does not match the model (size or texture count)");
    TexPtrs tp;
    memset(&tp, 0, sizeof(tp));
    for (int t = 0; t < mat->n_textures; ++t) {
        if (mat->formats[t] != desc->formats[t]) return fail(NTBC_EINVAL, "texture %d: format differs from the model", t);
        if (!mat->texels[t] || !mat->ref_blocks[t]) return fail(NTBC_EINVAL, "texture %d: null texels or reference blocks", t);
        tp.texels[t] = mat->texels[t];
        tp.blocks[t] = mat->ref_blocks[t];
    }
    unsigned char* base = nullptr;
    st = noalloc_scratch(&base);
    if (st != NTBC_OK) return st;
    float* cursor = reinterpret_cast<float*>(base);
    NetBuffers cbuf = carve_net(cursor, kNoAllocColor, kMaxOutC);
    NetBuffers ebuf = carve_net(cursor, kNoAllocMaxBlocks, kMaxOutE);
    double* acc = reinterpret_cast<double*>(base + kNoAllocFloats * sizeof(float));
    float* qscale = reinterpret_cast<float*>(acc + 6);
    float* qzero = qscale + kNoAllocLevels;
    unsigned* qmm = reinterpret_cast<unsigned*>(qzero + kNoAllocLevels);

    cudaStream_t s = (cudaStream_t)stream;
    ModelView mv = make_view(*desc, L);
    GridSrc csrc;
    memset(&csrc, 0, sizeof(csrc));
    csrc.f32 = params;
    csrc.qat_bits = qat_bits;
    GridSrc esrc = csrc;
    if (qat_bits > 0) {
        LevelTable lt = level_table(*desc, L);
        st = launch_level_scale_zero(params, lt, qat_bits, qmm, qscale, qzero, s);
        if (st != NTBC_OK) return st;
        csrc.scale = qscale;
        csrc.zero = qzero;
        esrc.scale = qscale + desc->color_levels;
        esrc.zero = qzero + desc->color_levels;
    }
    // the array keeps the previous call's contents: clear what accumulates
    NTBC_CHECK_CUDA(cudaMemsetAsync(grads, 0, L.total * sizeof(float), s));
    NTBC_CHECK_CUDA(cudaMemsetAsync(acc, 0, 6 * sizeof(double), s));
    net_step(params, mv, true, tp, block_ids, n_blocks * 16, csrc, temperature, cbuf, grads, acc, s);
    net_step(params, mv, false, tp, block_ids, n_blocks, esrc, temperature, ebuf, grads, acc, s);
    loss_finalize_kernel<<<1, 32, 0, s>>>(acc, losses);
    NTBC_CHECK_LAUNCH("allocation-free training gradients");
    return NTBC_OK;
}

}  // extern "C"
