// Throughput probes for the roofline denominators that no library kernel can supply:
// the FP32 SIMT rate (packed f32x2 FMA), the FP64 SIMT rate, and the tcgen05 tensor rate
// for tf32 and f16 inputs (M = 128, N = 256, FP32 accumulate, operands in shared memory),
// plus the tf32 rate at N = 16, the narrow shape of the adjoint's pixel-weight product.
// Each probe runs a fixed amount of independent work on every SM and is timed with CUDA
// events on the caller's stream; the result is the work over the elapsed time.
#include "modal_internal.cuh"

#include "tc_common.cuh"

namespace modal {

constexpr int PK_THREADS = 256;

// 8 independent packed FMA chains per thread (the dependency latency is covered by the
// chains and by 2048 threads per SM); the result feeds a store that never happens unless
// the sum is exactly 1234.5, so the compiler keeps the work.
__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma2(int iters, float* sink) {
    float2 a[8];
    const float2 m = make_float2(0.999999f, 1.000001f), c = make_float2(1e-7f, -1e-7f);
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = make_float2((float)threadIdx.x + i, (float)blockIdx.x - i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = __ffma2_rn(a[i], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i].x + a[i].y;
    if (s == 1234.5f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_dfma(int iters, double* sink) {
    double a[8];
    const double m = 0.9999999999, c = 1e-12;
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (double)threadIdx.x + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fma(a[i], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == 1234.5) sink[threadIdx.x] = s;
}

// One CTA per SM: a single thread issues `iters` MMAs (M = 128, N = 256 or 16, K = 8 tf32
// or 16 f16 per instruction) on zeroed shared-memory operands into one TMEM accumulator,
// then one commit, and waits (bounded) for it before TMEM is freed.
template <bool TF32, int N>
__global__ void __launch_bounds__(128, 1) k_peak_mma(int iters, int* err) {
    extern __shared__ __align__(1024) char pk_smem[];
    char* ops = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(pk_smem) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t done;
    __shared__ uint32_t tmem_slot;
    constexpr int A_BYTES = 128 * 32, B_BYTES = N * 32;      // one K step (32 bytes of K per row)
    for (int i = threadIdx.x; i < (A_BYTES + B_BYTES) / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(ops)[i] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_proxy_async();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x == 0) {
        // K-major core-matrix layout of one K step: rows of 32 bytes, 8-row groups 256 B apart
        auto desc = [](uint32_t saddr) {
            uint64_t d = 0;
            d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
            d |= (uint64_t)(128 >> 4) << 16;
            d |= (uint64_t)(256 >> 4) << 32;
            d |= (uint64_t)1 << 46;
            return d;
        };
        const uint64_t ad = desc(smem_u32(ops)), bd = desc(smem_u32(ops + A_BYTES));
        const uint32_t idesc = umma_idesc(TF32 ? 2 : 0, N);
        for (int it = 0; it < iters; ++it) umma<TF32>(tmem, ad, bd, idesc, it == 0 ? 0u : 1u);
        umma_commit(&done);                              // one commit tracks every MMA issued above
        const long long t0 = clock64();
        bool ok = false;
        while (!(ok = mbar_try_wait(&done, 0)) && clock64() - t0 < TC_WAIT_CYCLES) {
        }
        if (!ok) atomicOr(err, MODAL_DEVERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
    }
}

}  // namespace modal

using namespace modal;

extern "C" modal_status modal_peak_probe(int kind, double* tflops, void* stream) {
    if (!tflops || kind < 0 || kind > 4) return set_error(MODAL_EINVAL, "kind in [0, 4] and tflops required");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    modal_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != MODAL_OK) return s;
    s = cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
    if (s != MODAL_OK) return s;
    void* buf = nullptr;
    s = cuda_check(cudaMallocAsync(&buf, 4096, st), "probe buffer");
    if (s != MODAL_OK) return s;
    cudaMemsetAsync(buf, 0, 4096, st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double flop = 0.0;
    auto launch = [&](bool timed) -> cudaError_t {
        if (timed) cudaEventRecord(e0, st);
        if (kind == 0) {                                 // FP32 SIMT: 8 ctas x 256 threads per SM
            const int iters = 4096;
            k_peak_ffma2<<<nsm * 8, PK_THREADS, 0, st>>>(iters, static_cast<float*>(buf));
            flop = (double)nsm * 8 * PK_THREADS * iters * 16 * 8 * 2 * 2;
        } else if (kind == 1) {                          // FP64 SIMT
            const int iters = 256;
            k_peak_dfma<<<nsm * 8, PK_THREADS, 0, st>>>(iters, static_cast<double*>(buf));
            flop = (double)nsm * 8 * PK_THREADS * iters * 16 * 8 * 2;
        } else {                                         // tcgen05: tf32 (2), f16 (3), tf32 at N = 16 (4)
            const int iters = 65536;
            const int n = kind == 4 ? 16 : 256;
            const size_t smem = 1024 + 128 * 32 + (size_t)n * 32;
            const bool tf32 = kind != 3;
            cudaError_t e;
            if (kind == 2) {
                e = cudaFuncSetAttribute(k_peak_mma<true, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e == cudaSuccess) k_peak_mma<true, 256><<<nsm, 128, smem, st>>>(iters, static_cast<int*>(buf));
            } else if (kind == 3) {
                e = cudaFuncSetAttribute(k_peak_mma<false, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e == cudaSuccess) k_peak_mma<false, 256><<<nsm, 128, smem, st>>>(iters, static_cast<int*>(buf));
            } else {
                e = cudaFuncSetAttribute(k_peak_mma<true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e == cudaSuccess) k_peak_mma<true, 16><<<nsm, 128, smem, st>>>(iters, static_cast<int*>(buf));
            }
            if (e != cudaSuccess) return e;
            flop = (double)nsm * iters * 2.0 * 128 * n * (tf32 ? 8 : 16);
        }
        if (timed) cudaEventRecord(e1, st);
        return cudaGetLastError();
    };
    cudaError_t e = launch(false);                       // warm-up (clocks, first-launch costs)
    if (e == cudaSuccess) e = launch(true);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    int flag = 0;
    if (e == cudaSuccess && kind >= 2) e = cudaMemcpyAsync(&flag, buf, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(buf, st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s = cuda_check(e, "peak probe");
    if (s != MODAL_OK) return s;
    if (flag) return set_error(MODAL_ETIMEOUT, "peak probe: the tensor-core wait gave up");
    *tflops = flop / (ms * 1e-3) / 1e12;
    return MODAL_OK;
}
