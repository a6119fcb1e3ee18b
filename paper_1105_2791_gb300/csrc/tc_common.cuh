// Shared pieces of the tcgen05 kernels: PTX wrappers (mbarrier, bulk copy, tcgen05
// MMA/commit/ld/fences), shared-memory and instruction descriptors, the split-precision
// element conversions and the per-map fp16 range scale.
#pragma once

#include "modal_internal.cuh"

#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace modal {

constexpr int TC_MAPS = 8;                 // maps per work item of the adjoint Legendre kernel (N = 16 P)
constexpr int TC_MAX_MAPS = 32;            // most maps per work item of the forward kernel (tunable, N = 2 P G <= 256)
constexpr int TC_PROD_WARPS = 8;           // epilogue warps
constexpr int TC_THREADS = 32 * (2 + TC_PROD_WARPS);
constexpr int TC_STAGES = 4;
constexpr int TC_KB = 64;                  // bytes of K per row per stage (4 core matrices)
constexpr int TC_SBO = 8 * TC_KB;          // bytes between 8-row groups
constexpr int TC_A_TILE = 128 * TC_KB;     // bytes: 128 rows x TC_KB bytes of K
constexpr int TC_A_STAGE = 2 * TC_A_TILE;  // hi, lo
constexpr float TC_LAMBDA_SCALE = 2048.f;  // |lambda| * 2^11 stays inside fp16 range
constexpr long long TC_WAIT_CYCLES = 1ll << 31;

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the CTA is aborting or the wait gave up (then it aborts).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > TC_WAIT_CYCLES) {
            atomicOr(err, MODAL_DEVERR_TIMEOUT);
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// Shared-memory matrix descriptor: K-major, no swizzle; LBO = 128 B (next core matrix
// along K), SBO = TC_SBO (next 8-row group: 8 rows x TC_KB bytes), descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(TC_SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: fp32 accumulate, K-major A and B, M = 128, N = n.
// fmt: 0 = f16, 1 = bf16 (kind::f16); 2 = tf32 (kind::tf32).
__host__ __device__ constexpr uint32_t umma_idesc(int fmt, int n) {
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if (TF32) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    }
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ element splitting
// PREC: MODAL_FP16X3, MODAL_BF16X3, MODAL_BF16 (16-bit elements), MODAL_3XTF32 (32-bit).
template <int PREC>
struct Split;

template <>
struct Split<MODAL_FP16X3> {
    static constexpr int E = 2, FMT = 0, PRODUCTS = 3;
    __device__ static void split(float x, uint16_t& hi, uint16_t& lo) {
        const __half h = __float2half_rn(x);
        const __half l = __float2half_rn(x - __half2float(h));
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(l);
    }
};
template <>
struct Split<MODAL_BF16X3> {
    static constexpr int E = 2, FMT = 1, PRODUCTS = 3;
    __device__ static void split(float x, uint16_t& hi, uint16_t& lo) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(l);
    }
};
template <>
struct Split<MODAL_BF16> {
    static constexpr int E = 2, FMT = 1, PRODUCTS = 1;
    __device__ static void split(float x, uint16_t& hi, uint16_t& lo) {
        hi = __bfloat16_as_ushort(__float2bfloat16_rn(x));
        lo = 0;
    }
};
template <>
struct Split<MODAL_3XTF32> {
    static constexpr int E = 4, FMT = 2, PRODUCTS = 3;
    // Both parts rounded to nearest tf32 (unbiased), so the tensor core reads them exactly.
    __device__ static uint32_t to_tf32(float x) {
        uint32_t r;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
        return r;
    }
    __device__ static void split(float x, uint32_t& hi, uint32_t& lo) {
        hi = to_tf32(x);
        lo = to_tf32(x - __uint_as_float(hi));
    }
};

// Power-of-two exponent k that brings the map's largest |f_p(l) a_lm| into [2^14, 2^15)
// (fp16 keeps 11 significant bits down to 2^-14; the lo parts stay normal well below
// the largest values).  amax_bits: the float bits of that maximum (0 for an empty map).
__device__ __forceinline__ int tc_scale_exp(unsigned amax_bits) {
    if (amax_bits == 0u) return 0;
    const int e = (int)((amax_bits >> 23) & 0xFF);             // biased exponent
    return max(-120, min(120, 141 - e));
}

template <int E>
struct ElemT;
template <>
struct ElemT<2> { using T = uint16_t; };
template <>
struct ElemT<4> { using T = uint32_t; };

}  // namespace modal
