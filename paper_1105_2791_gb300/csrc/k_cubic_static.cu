// Allocation-free variant of the cubic-term reduction.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned entirely by
// another allocator (a framework's caching pool, a fixed budget carved out at start-up),
// and latency-critical loops where an allocation, which may synchronise the device, is
// not acceptable.  modal_cubic_static serves them: it reduces caller-provided maps to
// the cubic coefficients beta_prs = sum_x W_x M_p M_r M_s using a scratch area that is
// a file-scope static device array, so the call allocates nothing.
//
// The scratch holds per-CTA partial sums (every entry the call reads is written by the
// same call first, so nothing needs clearing).  It is one array per device, shared by
// every call: calls that overlap on the GPU (different streams, different threads)
// race on it.  Its device address is looked up once per device with
// cudaGetSymbolAddress on the first call made with that device current; make that
// first call before any stream capture.  Every GPU that loads this library holds the
// array (MODAL_STATIC_SCRATCH_DOUBLES doubles = 32 MiB) until the process exits.
#include "modal_internal.cuh"

#include <algorithm>
#include <mutex>

#define MODAL_STATIC_SCRATCH_DOUBLES (4u << 20)
#define MODAL_STATIC_MAX_DEVICES 64

#define CUDA_TRY_STATUS(expr, what)                             \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return cuda_check(_e, (what));   \
    } while (0)

namespace modal {

static __device__ __align__(256) double g_modal_static_scratch[MODAL_STATIC_SCRATCH_DOUBLES];

constexpr int CS_TX = 64;       // pixels per shared-memory tile
constexpr int CS_LANES = 8;     // pixel lanes per register tile

// Pairs (p, r), p <= r, in colex order (sorted by r, then p): c -> (p, r).
__device__ __forceinline__ void cs_colex(int c, int& p, int& r) {
    r = 0;
    while ((r + 1) * (r + 2) / 2 <= c) ++r;
    p = c - r * (r + 1) / 2;
}

// Lexicographic index of the mode (p, r, s), p <= r <= s < P.
__device__ __forceinline__ int cs_mode(int p, int r, int s, int P) {
    int n = 0;
    for (int q = 0; q < p; ++q) n += (P - q) * (P - q + 1) / 2;
    for (int q = p; q < r; ++q) n += P - q;
    return n + (s - r);
}

// Register tiles of 8 colex pairs x 4 values of s that hold at least one s >= r.
__host__ __device__ inline int cs_tiles(int P, int* out) {
    const int npair = P * (P + 1) / 2, npg = (npair + 7) / 8, nsq = (P + 3) / 4;
    int n = 0;
    for (int pg = 0; pg < npg; ++pg)
        for (int sq = 0; sq < nsq; ++sq) {
            bool any = false;
            for (int c = pg * 8; c < pg * 8 + 8 && c < npair; ++c) {
                int r = 0;
                while ((r + 1) * (r + 2) / 2 <= c) ++r;
                for (int s = sq * 4; s < sq * 4 + 4 && s < P; ++s)
                    if (s >= r) any = true;
            }
            if (any) {
                if (out) out[n] = pg | (sq << 8);
                ++n;
            }
        }
    return n;
}

__global__ void __launch_bounds__(320)
k_cubic_static(int P, int64_t npix, int64_t px_per_cta, const float* __restrict__ maps, const float* __restrict__ W,
               double* __restrict__ partial, int n_max) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_tiles[64];
    __shared__ int s_ntiles;
    const int npair = P * (P + 1) / 2;
    const int SU = ((npair + 7) / 8) * 8, SM = ((P + 3) / 4) * 4;
    float* sU = smem;                     // [CS_TX][SU]
    float* sM = sU + CS_TX * SU;          // [CS_TX][SM]
    float* sW = sM + CS_TX * SM;          // [CS_TX]
    if (threadIdx.x == 0) s_ntiles = cs_tiles(P, s_tiles);
    __syncthreads();
    const int ntiles = s_ntiles;
    const int b = blockIdx.y;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int tile = tid % ntiles;
    const int lane = tid / ntiles;
    const bool computes = lane < CS_LANES;
    const int pg = s_tiles[tile] & 0xff, sq = s_tiles[tile] >> 8;
    const int64_t x_begin = (int64_t)blockIdx.x * px_per_cta;
    const int64_t x_end = min(npix, x_begin + px_per_cta);
    const float* mb = maps + (int64_t)b * P * npix;

    float acc[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) acc[e] = 0.f;

    for (int64_t x0 = x_begin; x0 < x_end; x0 += CS_TX) {
        for (int i = tid; i < CS_TX * SM; i += nthr) {
            const int xl = i % CS_TX, s = i / CS_TX;
            const int64_t x = x0 + xl;
            sM[xl * SM + s] = (s < P && x < x_end) ? mb[(int64_t)s * npix + x] : 0.f;
        }
        for (int i = tid; i < CS_TX; i += nthr) sW[i] = (x0 + i < x_end) ? W[x0 + i] : 0.f;
        __syncthreads();
        for (int i = tid; i < CS_TX * SU; i += nthr) {
            const int xl = i / SU, c = i % SU;
            float v = 0.f;
            if (c < npair) {
                int p, r;
                cs_colex(c, p, r);
                v = sW[xl] * sM[xl * SM + p] * sM[xl * SM + r];
            }
            sU[i] = v;
        }
        __syncthreads();
        if (computes) {
            float tmp[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) tmp[e] = 0.f;
            for (int xi = lane; xi < CS_TX; xi += CS_LANES) {
                const float4 u0 = *reinterpret_cast<const float4*>(sU + xi * SU + pg * 8);
                const float4 u1 = *reinterpret_cast<const float4*>(sU + xi * SU + pg * 8 + 4);
                const float4 mv = *reinterpret_cast<const float4*>(sM + xi * SM + sq * 4);
                const float u[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                const float mm[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k) tmp[i * 4 + k] = fmaf(u[i], mm[k], tmp[i * 4 + k]);
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) acc[e] += tmp[e];
        }
        __syncthreads();
    }
    float* red = smem;   // [CS_LANES][ntiles][32]
    if (computes) {
#pragma unroll
        for (int e = 0; e < 32; ++e) red[(lane * ntiles + tile) * 32 + e] = acc[e];
    }
    __syncthreads();
    for (int i = tid; i < ntiles * 32; i += nthr) {
        const int t = i / 32, e = i % 32;
        float v = 0.f;
        for (int ln = 0; ln < CS_LANES; ++ln) v += red[(ln * ntiles + t) * 32 + e];
        const int c = (s_tiles[t] & 0xff) * 8 + e / 4, s = (s_tiles[t] >> 8) * 4 + e % 4;
        if (c >= npair || s >= P) continue;
        int p, r;
        cs_colex(c, p, r);
        if (s < r) continue;
        partial[((int64_t)b * gridDim.x + blockIdx.x) * n_max + cs_mode(p, r, s, P)] = (double)v;
    }
}

__global__ void k_cubic_static_finalize(int B, int n_max, int nctas, const double* __restrict__ partial,
                                        double* __restrict__ beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * n_max) return;
    const int b = i / n_max, n = i % n_max;
    double v = 0.0;
    for (int c = 0; c < nctas; ++c) v += partial[((int64_t)b * nctas + c) * n_max + n];
    beta[i] = v;
}

// Device address of the static scratch for the current device, looked up once per device.
static modal_status static_scratch(double** out) {
    static std::mutex mu;
    static double* addr[MODAL_STATIC_MAX_DEVICES] = {};
    int dev = 0;
    CUDA_TRY_STATUS(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= MODAL_STATIC_MAX_DEVICES) return set_error(MODAL_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        CUDA_TRY_STATUS(cudaGetSymbolAddress(&p, g_modal_static_scratch), "cudaGetSymbolAddress(static scratch)");
        addr[dev] = static_cast<double*>(p);
    }
    *out = addr[dev];
    return MODAL_OK;
}

}  // namespace modal

using namespace modal;

extern "C" modal_status modal_cubic_static(const float* maps, const float* W, long long npix, int P, int B,
                                           double* beta, void* stream) {
    if (P < 1 || P > MODAL_MAXP) return set_error(MODAL_EINVAL, "P must be in [1, 16]");
    if (npix < 1 || B < 0) return set_error(MODAL_EINVAL, "npix must be >= 1 and B >= 0");
    if (B == 0) return MODAL_OK;
    if (B > 65535) return set_error(MODAL_EINVAL, "B must be <= 65535");
    if (!maps || !W || !beta) return set_error(MODAL_EINVAL, "null pointer");
    const int n_max = P * (P + 1) * (P + 2) / 6;
    if ((long long)B * n_max > (long long)MODAL_STATIC_SCRATCH_DOUBLES)
        return set_error(MODAL_EINVAL, "B * n_max exceeds the static scratch (4 Mi doubles)");
    long long nctas = std::max<long long>(1, std::min<long long>(npix / 16384, 128));
    nctas = std::min<long long>(nctas, (long long)MODAL_STATIC_SCRATCH_DOUBLES / ((long long)B * n_max));
    double* scratch = nullptr;
    modal_status s = static_scratch(&scratch);
    if (s != MODAL_OK) return s;
    const int ntiles = cs_tiles(P, nullptr);
    const int nthr = ((ntiles * CS_LANES + 31) / 32) * 32;
    const int npair = P * (P + 1) / 2;
    const size_t tilebuf = (size_t)CS_TX * (((npair + 7) / 8) * 8 + ((P + 3) / 4) * 4 + 1) * sizeof(float);
    const size_t redbuf = (size_t)CS_LANES * ntiles * 32 * sizeof(float);
    const size_t smem = std::max(tilebuf, redbuf);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaFuncSetAttribute(k_cubic_static, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(e, "cubic_static attribute");
    const long long ppc = ((npix + nctas - 1) / nctas + CS_TX - 1) / CS_TX * CS_TX;
    k_cubic_static<<<dim3((unsigned)nctas, (unsigned)B), nthr, smem, st>>>(P, npix, ppc, maps, W, scratch, n_max);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(e, "cubic_static launch");
    k_cubic_static_finalize<<<(B * n_max + 127) / 128, 128, 0, st>>>(B, n_max, (int)nctas, scratch, beta);
    return cuda_check(cudaGetLastError(), "cubic_static finalize launch");
}
