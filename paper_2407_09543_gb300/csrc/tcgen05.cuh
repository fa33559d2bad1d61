// tcgen05 / mbarrier primitives shared by the tensor-core kernels (inline PTX for
// sm_100-family tensor cores: descriptors, MMA issue, commit, bounded waits, TMEM loads,
// fences) and the canonical no-swizzle core-matrix tile layout.
#pragma once

#include <cstdint>

namespace ntbc {

// polls of an mbarrier before a wait gives up (the caller then records an error,
// lets in-flight MMAs land and returns instead of hanging the GPU); an unsuccessful
// try_wait suspends the thread for ~3.8 us on GB300, so the limit is about one second
constexpr long long kTcWaitLimit = 1LL << 18;


__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// UMMA shared-memory descriptor, no swizzle. A core matrix is 8 rows of 16 bytes
// (128 contiguous bytes). k_stride: bytes between core matrices adjacent along K;
// mn_stride: bytes between core matrices adjacent along M (or N). The same reading
// holds for K-major operands (rows along M/N, 16 bytes of K each) and for MN-major ones
// (rows along K, 16 bytes of M/N each).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t k_stride, uint32_t mn_stride) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((k_stride >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((mn_stride >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16 with M = 128, D = F32: A and B both F16 (bf16 = 0) or
// both BF16 (bf16 = 1); a_mn / b_mn select the MN-major (transposed) operand layout
__host__ __device__ constexpr uint32_t umma_idesc_kind(int n, int bf16, int a_mn, int b_mn) {
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)a_mn << 15) |
           ((uint32_t)b_mn << 16) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__host__ __device__ constexpr uint32_t umma_idesc(int n) { return umma_idesc_kind(n, 0, 0, 0); }
// kind::f8f6f4 with A and B both E4M3 (format code 0 in the same fields), D = F32, M = 128,
// both operands K-major: the same bits as the FP16 descriptor
__host__ __device__ constexpr uint32_t umma_idesc_e4m3(int n) { return umma_idesc_kind(n, 0, 0, 0); }

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// one MMA of kind::f8f6f4: K = 32 one-byte elements per row (the same 32 bytes per row as a
// kind::f16 MMA's K = 16)
__device__ __forceinline__ void umma_f8(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, long long limit = kTcWaitLimit) {
    uint32_t done = 0;
    for (long long it = 0; it < limit; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(phase));
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// tcgen05.wait::ld, then tie the loaded registers to it so that no use of them can be
// scheduled above the wait
template <int N>
__device__ __forceinline__ void tmem_wait_ld_regs(float* v) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < N; ++i) asm volatile("" : "+f"(v[i]));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// named barrier g + 1 over one warpgroup (128 threads)
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(128) : "memory"); }

// byte offset of element (r, k) in a tile of K columns (16-bit elements)
__host__ __device__ __forceinline__ int core_byte(int r, int k, int K) {
    return (((r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7)) * 2;
}

// byte offset of element (r, k) in a tile of K columns (8-bit elements: a core matrix row
// holds 16 of them)
__host__ __device__ __forceinline__ int core_byte8(int r, int k, int K) {
    return ((r >> 3) * (K >> 4) + (k >> 4)) * 128 + (r & 7) * 16 + (k & 15);
}

}  // namespace ntbc
