// BC1 / BC4 reference encoder, decoder and the output-to-block stage of NTBC
// inference; host error plumbing of the library.
//
// Format: Sec. 2.1 (8-byte blocks, RGB565 + 2-bit codes, 8-bit + 3-bit codes,
// palettes of Eq. palette / Eq. weightBC4). The reference encoder stands in for
// the Compressonator encoder of Sec. 4.1 and is bit-exact with the CPU oracle:
// its FP64 arithmetic uses explicit round-to-nearest intrinsics (no fused
// multiply-add) in the same order as the oracle's.
#include <cstdlib>
#include <cstring>

#include "ntbc_internal.cuh"

namespace ntbc {

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------

static thread_local std::string g_last_error;

ntbc_status fail(ntbc_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

ntbc_status cuda_fail(cudaError_t err, const char* what) {
    if (err == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(NTBC_ENOMEM, "%s: %s", what, cudaGetErrorString(err));
    }
    return fail(NTBC_ECUDA, "%s: %s", what, cudaGetErrorString(err));
}

void clear_error() { g_last_error.clear(); }

bool fault_injected(const char* what) {
    const char* env = std::getenv("NTBC_FAULT");
    return env && std::strstr(env, what) != nullptr;
}

ntbc_status device_alloc(void** ptr, size_t bytes, const char* what) {
    *ptr = nullptr;
    if (fault_injected("alloc")) return fail(NTBC_ENOMEM, "injected allocation failure: %s", what);
    if (bytes == 0) return NTBC_OK;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(NTBC_ENOMEM, "cudaMalloc(%zu) for %s: %s", bytes, what, cudaGetErrorString(e));
    }
    return NTBC_OK;
}

ntbc_status check_texture_args(int fmt, const void* a, const void* b, int w, int h) {
    if (fmt != NTBC_BC1 && fmt != NTBC_BC4 && fmt != NTBC_BC3 && fmt != NTBC_BC5)
        return fail(NTBC_EINVAL, "format must be NTBC_BC1, NTBC_BC3, NTBC_BC4 or NTBC_BC5, got %d", fmt);
    if (w <= 0 || h <= 0 || (w & 3) || (h & 3))
        return fail(NTBC_EINVAL, "width and height must be positive multiples of 4, got %dx%d", w, h);
    if ((long long)w * h > (1LL << 30)) return fail(NTBC_EINVAL, "texture too large (%dx%d)", w, h);
    if (!a || !b) return fail(NTBC_EINVAL, "null data pointer");
    return NTBC_OK;
}

// ---------------------------------------------------------------------------
// reference encoder
// ---------------------------------------------------------------------------

constexpr int kPowerIterations = 8;

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }

// BC1 codes of least integer squared RGB distance (ties: lowest code) for c0 >= c1
// (c0 == c1: all codes 0), and the block's total squared error
__device__ __forceinline__ void bc1_codes(const int x[16][3], uint32_t c0, uint32_t c1, uint32_t& idx, int& sse) {
    int pal[4][3];
    bc1_palette(c0, c1, pal);
    idx = 0;
    sse = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        int best = 0, bestd = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int dr = x[i][0] - pal[k][0], dg = x[i][1] - pal[k][1], db = x[i][2] - pal[k][2];
            int d = dr * dr + dg * dg + db * db;
            if (k == 0 || d < bestd) {
                bestd = d;
                best = k;
            }
        }
        if (c0 == c1) {
            best = 0;
            int dr = x[i][0] - pal[0][0], dg = x[i][1] - pal[0][1], db = x[i][2] - pal[0][2];
            bestd = dr * dr + dg * dg + db * db;
        }
        idx |= (uint32_t)best << (2 * i);
        sse += bestd;
    }
}

// Least-squares refinement (optional; the reading of Compressonator's "refine steps"):
// endpoints a, b minimising sum_i |x_i - ((D - w_i) a + w_i b) / D|^2 for the current codes
// (w_i: the code's weight of the second endpoint in units of 1/D) are, with A11 = sum
// (D-w)^2, A12 = sum (D-w) w, A22 = sum w^2, R1 = sum (D-w) x, R2 = sum w x and det = A11 A22 -
// A12^2: a = D (A22 R1 - A12 R2) / det, b = D (A11 R2 - A12 R1) / det. The quantised value
// round-half-up(a L / 255), clamped to [0, L], is taken in exact integer arithmetic.
__device__ __forceinline__ int quantise_ls(long long num, long long det, int D, int L) {
    if (num <= 0) return 0;
    long long q = (2LL * D * num * L + 255LL * det) / (510LL * det);
    return (int)(q < L ? q : L);
}

// texels: ts bytes per texel, the encoded channel(s) from byte to; blocks bs bytes apart;
// refine: least-squares refinement steps (kept while the squared error strictly falls)
__global__ void bc1_encode_kernel(const uint8_t* __restrict__ tex, int w, int h, int ts, int to,
                                  uint8_t* __restrict__ out, int bs, int refine) {
    int bw = w >> 2, bh = h >> 2;
    long long nb = (long long)bw * bh;
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int bx = (int)(b % bw), by = (int)(b / bw);
    int x[16][3];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint8_t* p = tex + ((long long)(4 * by + (i >> 2)) * w + 4 * bx + (i & 3)) * ts + to;
        x[i][0] = p[0];
        x[i][1] = p[1];
        x[i][2] = p[2];
    }
    // integer covariance of 16 * deviation
    int s[3] = {0, 0, 0}, mn[3] = {255, 255, 255}, mx[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 16; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            s[c] += x[i][c];
            mn[c] = min(mn[c], x[i][c]);
            mx[c] = max(mx[c], x[i][c]);
        }
    long long cov[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            long long acc = 0;
#pragma unroll
            for (int i = 0; i < 16; ++i) acc += (long long)(16 * x[i][j] - s[j]) * (16 * x[i][k] - s[k]);
            cov[j][k] = acc;
        }
    double C[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) C[j][k] = (double)cov[j][k];
    int widest = 0;
    int r0 = mx[0] - mn[0], r1 = mx[1] - mn[1], r2 = mx[2] - mn[2];
    if (r1 > r0) widest = 1;
    if (r2 > (widest == 0 ? r0 : r1)) widest = 2;
    double v[3] = {(double)r0, (double)r1, (double)r2};
#pragma unroll
    for (int c = 0; c < 3; ++c)
        if (c != widest && cov[widest][c] < 0) v[c] = -v[c];
    bool live = true;
    for (int it = 0; it < kPowerIterations; ++it) {
        double wv[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) wv[j] = dadd(dadd(dmul(C[j][0], v[0]), dmul(C[j][1], v[1])), dmul(C[j][2], v[2]));
        double m = fmax(fmax(fabs(wv[0]), fabs(wv[1])), fabs(wv[2]));
        live = live && (m > 0.0);
        if (live) {
#pragma unroll
            for (int j = 0; j < 3; ++j) v[j] = __ddiv_rn(wv[j], m);
        }
    }
    int imax = 0, imin = 0;
    double pmax = 0.0, pmin = 0.0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        double p = dadd(dadd(dmul((double)x[i][0], v[0]), dmul((double)x[i][1], v[1])), dmul((double)x[i][2], v[2]));
        if (i == 0 || p > pmax) {
            pmax = p;
            imax = i;
        }
        if (i == 0 || p < pmin) {
            pmin = p;
            imin = i;
        }
    }
    auto q565 = [&](int i) -> uint32_t {
        return (uint32_t)(((x[i][0] * 31 + 127) / 255) << 11) | (uint32_t)(((x[i][1] * 63 + 127) / 255) << 5) |
               (uint32_t)((x[i][2] * 31 + 127) / 255);
    };
    uint32_t c0 = q565(imax), c1 = q565(imin);
    if (c0 < c1) {
        uint32_t t = c0;
        c0 = c1;
        c1 = t;
    }
    uint32_t idx;
    int sse;
    bc1_codes(x, c0, c1, idx, sse);
    for (int it = 0; it < refine; ++it) {
        const int w3[4] = {0, 3, 1, 2};             // code -> weight of colour1, in thirds
        long long A11 = 0, A12 = 0, A22 = 0, R1[3] = {0, 0, 0}, R2[3] = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            int wi = w3[(idx >> (2 * i)) & 3], ui = 3 - wi;
            A11 += ui * ui;
            A12 += ui * wi;
            A22 += wi * wi;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                R1[c] += ui * x[i][c];
                R2[c] += wi * x[i][c];
            }
        }
        long long det = A11 * A22 - A12 * A12;
        if (det <= 0) break;
        const int L[3] = {31, 63, 31};
        int qa[3], qb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            qa[c] = quantise_ls(A22 * R1[c] - A12 * R2[c], det, 3, L[c]);
            qb[c] = quantise_ls(A11 * R2[c] - A12 * R1[c], det, 3, L[c]);
        }
        uint32_t a0 = ((uint32_t)qa[0] << 11) | ((uint32_t)qa[1] << 5) | (uint32_t)qa[2];
        uint32_t a1 = ((uint32_t)qb[0] << 11) | ((uint32_t)qb[1] << 5) | (uint32_t)qb[2];
        uint32_t n0 = a0 > a1 ? a0 : a1, n1 = a0 > a1 ? a1 : a0;
        uint32_t nidx;
        int nsse;
        bc1_codes(x, n0, n1, nidx, nsse);
        if (nsse >= sse) break;
        c0 = n0;
        c1 = n1;
        idx = nidx;
        sse = nsse;
    }
    store_block(out + b * bs, c0 | (c1 << 16), idx);
}

__device__ __forceinline__ void bc4_codes(const int x[16], int r0, int r1, uint64_t& idx, int& sse) {
    int pal[8];
    bc4_palette(r0, r1, pal);
    idx = 0;
    sse = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        int best = 0, bestd = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            int d = abs(x[i] - pal[k]);
            if (k == 0 || d < bestd) {
                bestd = d;
                best = k;
            }
        }
        idx |= (uint64_t)best << (3 * i);
        sse += bestd * bestd;
    }
}

__global__ void bc4_encode_kernel(const uint8_t* __restrict__ tex, int w, int h, int ts, int to,
                                  uint8_t* __restrict__ out, int bs, int refine) {
    int bw = w >> 2, bh = h >> 2;
    long long nb = (long long)bw * bh;
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int bx = (int)(b % bw), by = (int)(b / bw);
    int x[16];
    int mx = 0, mn = 255, lo = 256, hi = -1;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        x[i] = tex[((long long)(4 * by + (i >> 2)) * w + 4 * bx + (i & 3)) * ts + to];
        mx = max(mx, x[i]);
        mn = min(mn, x[i]);
        if (x[i] != 0 && x[i] != 255) {
            lo = min(lo, x[i]);
            hi = max(hi, x[i]);
        }
    }
    int r0, r1, sse = 0;
    uint64_t idx;
    if (mx == mn) {
        r0 = r1 = mx;
        idx = 0;
    } else {
        if (hi < 0) {
            lo = 0;
            hi = 255;
        }
        uint64_t ia, ib;
        int sa, sb;
        bc4_codes(x, mx, mn, ia, sa);
        bc4_codes(x, lo, hi, ib, sb);
        if (sa <= sb) {
            r0 = mx;
            r1 = mn;
            idx = ia;
            sse = sa;
        } else {
            r0 = lo;
            r1 = hi;
            idx = ib;
            sse = sb;
        }
    }
    for (int it = 0; it < refine; ++it) {          // the block keeps its mode
        const bool eight = r0 > r1;
        const int D = eight ? 7 : 5;
        const int w8[8] = {0, 7, 1, 2, 3, 4, 5, 6}, w6[8] = {0, 5, 1, 2, 3, 4, -1, -1};
        long long A11 = 0, A12 = 0, A22 = 0, R1 = 0, R2 = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            int code = (int)((idx >> (3 * i)) & 7);
            int wi = eight ? w8[code] : w6[code];
            if (wi < 0) continue;                      // the constants 0 and 255 of the six-value mode
            int ui = D - wi;
            A11 += ui * ui;
            A12 += ui * wi;
            A22 += wi * wi;
            R1 += ui * x[i];
            R2 += wi * x[i];
        }
        long long det = A11 * A22 - A12 * A12;
        if (det <= 0) break;
        int qa = quantise_ls(A22 * R1 - A12 * R2, det, D, 255), qb = quantise_ls(A11 * R2 - A12 * R1, det, D, 255);
        int n0 = eight ? max(qa, qb) : min(qa, qb), n1 = eight ? min(qa, qb) : max(qa, qb);
        if (eight && n0 <= n1) break;
        uint64_t nidx;
        int nsse;
        bc4_codes(x, n0, n1, nidx, nsse);
        if (nsse >= sse) break;
        r0 = n0;
        r1 = n1;
        idx = nidx;
        sse = nsse;
    }
    uint32_t wlo = (uint32_t)r0 | ((uint32_t)r1 << 8) | (uint32_t)((idx & 0xFFFF) << 16);
    uint32_t whi = (uint32_t)(idx >> 16);
    store_block(out + b * bs, wlo, whi);
}

// ---------------------------------------------------------------------------
// decoder: one thread per block, 16 texels written
// ---------------------------------------------------------------------------

// blocks bs bytes apart; texels ts bytes apart, channel(s) from byte to. four: the BC1
// colour block always uses the four-colour palette (the colour block of BC3).
__global__ void bc_decode_kernel(int fmt, const uint8_t* __restrict__ blocks, int bs, int w, int h,
                                 uint8_t* __restrict__ tex, int ts, int to, int four) {
    int bw = w >> 2, bh = h >> 2;
    long long nb = (long long)bw * bh;
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int bx = (int)(b % bw), by = (int)(b / bw);
    uint2 blk = *reinterpret_cast<const uint2*>(blocks + b * bs);
    if (fmt == NTBC_BC1) {
        int pal[4][3];
        uint32_t c0 = blk.x & 0xFFFF, c1 = blk.x >> 16;
        if (four && c0 <= c1) {                  // interpolants at 1/3 and 2/3 whatever the order
            int e0[3], e1[3];
            expand565(c0, e0[0], e0[1], e0[2]);
            expand565(c1, e1[0], e1[1], e1[2]);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                pal[0][c] = e0[c];
                pal[1][c] = e1[c];
                pal[2][c] = (2 * e0[c] + e1[c] + 1) / 3;
                pal[3][c] = (e0[c] + 2 * e1[c] + 1) / 3;
            }
        } else {
            bc1_palette(c0, c1, pal);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            int code = (blk.y >> (2 * i)) & 3;
            uint8_t* p = tex + ((long long)(4 * by + (i >> 2)) * w + 4 * bx + (i & 3)) * ts + to;
            p[0] = (uint8_t)pal[code][0];
            p[1] = (uint8_t)pal[code][1];
            p[2] = (uint8_t)pal[code][2];
        }
    } else {
        int pal[8];
        bc4_palette(blk.x & 0xFF, (blk.x >> 8) & 0xFF, pal);
        uint64_t idx = (uint64_t)(blk.x >> 16) | ((uint64_t)blk.y << 16);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            int code = (int)((idx >> (3 * i)) & 7);
            tex[((long long)(4 * by + (i >> 2)) * w + 4 * bx + (i & 3)) * ts + to] = (uint8_t)pal[code];
        }
    }
}

// ---------------------------------------------------------------------------
// outputs -> blocks (steps a6-a8) for given network outputs
// ---------------------------------------------------------------------------

__global__ void outputs_to_bc_kernel(int fmt, const float* __restrict__ e_hat, const float* __restrict__ c_hat,
                                     int n, uint8_t* __restrict__ out) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    BlockPalette bp;
    if (fmt == NTBC_BC1) {
        float e[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) e[k] = e_hat[(long long)b * 6 + k];
        make_palette_bc1(e, bp);
        uint32_t idx = 0;
        const float* c = c_hat + (long long)b * 48;
#pragma unroll
        for (int i = 0; i < 16; ++i) idx |= (uint32_t)choose_code_bc1(bp, c[3 * i], c[3 * i + 1], c[3 * i + 2]) << (2 * i);
        store_block(out + (long long)b * 8, bp.ep, idx);
    } else {
        float e[2] = {e_hat[(long long)b * 2], e_hat[(long long)b * 2 + 1]};
        make_palette_bc4(e, bp);
        uint64_t idx = 0;
        const float* c = c_hat + (long long)b * 16;
#pragma unroll
        for (int i = 0; i < 16; ++i) idx |= (uint64_t)choose_code_bc4(bp, c[i]) << (3 * i);
        store_block(out + (long long)b * 8, bp.ep | (uint32_t)((idx & 0xFFFF) << 16), (uint32_t)(idx >> 16));
    }
}

}  // namespace ntbc

using namespace ntbc;

extern "C" {

const char* ntbc_last_error(void) { return g_last_error.c_str(); }

int ntbc_abi_version(void) { return 1; }

ntbc_status bc_reference_encode(int fmt, const uint8_t* texels, int w, int h, uint8_t* blocks, void* stream) {
    ntbc::NvtxRange nvtx_range("bc_reference_encode");
    return bc_reference_encode_refined(fmt, texels, w, h, 0, blocks, stream);
}

ntbc_status bc_reference_encode_refined(int fmt, const uint8_t* texels, int w, int h, int refine, uint8_t* blocks,
                                        void* stream) {
    ntbc::NvtxRange nvtx_range("bc_reference_encode_refined");
    clear_error();
    ntbc_status st = check_texture_args(fmt, texels, blocks, w, h);
    if (st != NTBC_OK) return st;
    if (refine < 0 || refine > 16) return fail(NTBC_EINVAL, "refinement steps must be in 0..16, got %d", refine);
    long long nb = (long long)(w / 4) * (h / 4);
    int threads = 128;
    unsigned grid = (unsigned)((nb + threads - 1) / threads);
    cudaStream_t s = (cudaStream_t)stream;
    switch (fmt) {
        case NTBC_BC1: bc1_encode_kernel<<<grid, threads, 0, s>>>(texels, w, h, 3, 0, blocks, 8, refine); break;
        case NTBC_BC4: bc4_encode_kernel<<<grid, threads, 0, s>>>(texels, w, h, 1, 0, blocks, 8, refine); break;
        case NTBC_BC3:   // alpha (byte 3 of RGBA) as BC4, then the colour as BC1
            bc4_encode_kernel<<<grid, threads, 0, s>>>(texels, w, h, 4, 3, blocks, 16, refine);
            bc1_encode_kernel<<<grid, threads, 0, s>>>(texels, w, h, 4, 0, blocks + 8, 16, refine);
            break;
        default:         // BC5: one BC4 block per channel
            bc4_encode_kernel<<<grid, threads, 0, s>>>(texels, w, h, 2, 0, blocks, 16, refine);
            bc4_encode_kernel<<<grid, threads, 0, s>>>(texels, w, h, 2, 1, blocks + 8, 16, refine);
    }
    NTBC_CHECK_LAUNCH("bc_reference_encode");
    return NTBC_OK;
}

ntbc_status bc_decode(int fmt, const uint8_t* blocks, int w, int h, uint8_t* texels, void* stream) {
    ntbc::NvtxRange nvtx_range("bc_decode");
    clear_error();
    ntbc_status st = check_texture_args(fmt, blocks, texels, w, h);
    if (st != NTBC_OK) return st;
    long long nb = (long long)(w / 4) * (h / 4);
    int threads = 128;
    unsigned grid = (unsigned)((nb + threads - 1) / threads);
    cudaStream_t s = (cudaStream_t)stream;
    switch (fmt) {
        case NTBC_BC1: bc_decode_kernel<<<grid, threads, 0, s>>>(NTBC_BC1, blocks, 8, w, h, texels, 3, 0, 0); break;
        case NTBC_BC4: bc_decode_kernel<<<grid, threads, 0, s>>>(NTBC_BC4, blocks, 8, w, h, texels, 1, 0, 0); break;
        case NTBC_BC3:
            bc_decode_kernel<<<grid, threads, 0, s>>>(NTBC_BC4, blocks, 16, w, h, texels, 4, 3, 0);
            bc_decode_kernel<<<grid, threads, 0, s>>>(NTBC_BC1, blocks + 8, 16, w, h, texels, 4, 0, 1);
            break;
        default:
            bc_decode_kernel<<<grid, threads, 0, s>>>(NTBC_BC4, blocks, 16, w, h, texels, 2, 0, 0);
            bc_decode_kernel<<<grid, threads, 0, s>>>(NTBC_BC4, blocks + 8, 16, w, h, texels, 2, 1, 0);
    }
    NTBC_CHECK_LAUNCH("bc_decode");
    return NTBC_OK;
}

ntbc_status ntbc_outputs_to_bc(int fmt, const float* e_hat, const float* c_hat, int n, uint8_t* blocks, void* stream) {
    clear_error();
    if (fmt != NTBC_BC1 && fmt != NTBC_BC4) return fail(NTBC_EINVAL, "format must be NTBC_BC1 or NTBC_BC4");
    if (n < 0) return fail(NTBC_EINVAL, "negative block count");
    if (n == 0) return NTBC_OK;
    if (!e_hat || !c_hat || !blocks) return fail(NTBC_EINVAL, "null data pointer");
    int threads = 128;
    outputs_to_bc_kernel<<<(n + threads - 1) / threads, threads, 0, (cudaStream_t)stream>>>(fmt, e_hat, c_hat, n, blocks);
    NTBC_CHECK_LAUNCH("ntbc_outputs_to_bc");
    return NTBC_OK;
}

}  // extern "C"
