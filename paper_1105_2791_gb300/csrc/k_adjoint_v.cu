// Pixel weights of the adjoint on the tensor cores (tcgen05, sm_103a), split plans.
//
// The derivative of sum_n g_n beta_n (Eq. bbispect with its linear term) with respect to the
// filtered map M_t(x) is U_t(x) = W_x sum_c h_{t,c} (M_a M_b - <M_a M_b>_x), c = (a <= b),
// with h_{t,c} = 3 k_c h_tab from k_adjoint_weights.  It is split in two by linearity:
//
//   map part   U^M_t(x) = W_x sum_a M_a(x) V_{t,a}(x),   V_{t,a}(x) = sum_b G_t[a][b] M_b(x),
//              G_t[a][b] = h_{t,(a,b)} for a <= b and 0 otherwise.  Per map, V is a GEMM with
//              M = 128 pixels, N = 16 P columns (t, a), K = 16 (b, zero-padded): six tcgen05
//              MMAs per pixel tile (two K steps of 8 tf32, hi*hi + hi*lo + lo*hi) at the wide
//              N where an MMA instruction is cheapest per flop; the epilogue forms U^M_t from
//              V in FP32 and writes it over the maps.
//   mean part  U^pm_t(x) = sum_c h_{t,c} W_x <c>_x depends on the map only through h; it is
//              applied in harmonic space after the transposed Legendre sums
//              (k_pm_harmonic.cu: launch_adjoint_pm).
//
// Every wait is bounded as in the Legendre kernels; on expiry the kernel records
// MODAL_DEVERR_TIMEOUT and its roles drain.
#include "modal_internal.cuh"

#include "tc_common.cuh"

#include <cuda.h>
#include <algorithm>
#include <mutex>

namespace modal {

constexpr int AV_PM = 16;                         // b (K) and a padded to 16
constexpr int AV_GROUPS = 2;                      // converter/epilogue groups (one TMEM accumulator each)
constexpr int AV_GW = 8;                          // warps per group: two per TMEM lane quarter, split by t
constexpr int AV_THREADS = 32 * (AV_GW * AV_GROUPS + 2);   // groups, the loader warp, the MMA warp
constexpr int AV_MAPS = 4;                        // maps per CTA (their G operands stay in shared memory)
constexpr int AV_ROW = 64;                        // bytes of K per operand row (16 tf32)
constexpr int AV_SBO = 8 * AV_ROW;                // bytes between 8-row groups (512 = TC_SBO)
constexpr int AV_GT = 256 * AV_ROW;               // one G tile: N <= 256 rows (16 KB)
constexpr int AV_BMAP = 2 * AV_GT;                // G operand of one map: [hi, lo] (32 KB)
constexpr int AV_AT = 128 * AV_ROW;               // one A tile: 128 pixels (8 KB)
constexpr int AV_ABUF = 2 * AV_AT;                // A operand of one group: [hi, lo] (16 KB)
constexpr int AV_STAGES = 6;                      // map tiles in flight (TMA ring)
constexpr int AV_MT = AV_PM * 128 * 4;            // one map tile: 16 rows (p) x 128 pixels (8 KB)
static_assert(AV_SBO == TC_SBO, "the operand tiles use the shared descriptor geometry");

// Round-to-nearest tf32 (ties away from zero) by integer arithmetic on the float bits, and
// the remainder rounded the same way: x ~ hi + lo with both exact in tf32.
__device__ __forceinline__ void av_split(float x, uint32_t& hi, uint32_t& lo) {
    hi = (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
    lo = (__float_as_uint(x - __uint_as_float(hi)) + 0x1000u) & 0xFFFFE000u;
}

// Two 16-column TMEM loads (this lane's row of columns c .. c + 31) and one wait; the wait
// names the destination registers, so no use of them moves above it.
#define AV_R16(o) "=r"(r[o + 0]), "=r"(r[o + 1]), "=r"(r[o + 2]), "=r"(r[o + 3]), "=r"(r[o + 4]), "=r"(r[o + 5]), \
    "=r"(r[o + 6]), "=r"(r[o + 7]), "=r"(r[o + 8]), "=r"(r[o + 9]), "=r"(r[o + 10]), "=r"(r[o + 11]),           \
    "=r"(r[o + 12]), "=r"(r[o + 13]), "=r"(r[o + 14]), "=r"(r[o + 15])
#define AV_W16(o) "+r"(r[o + 0]), "+r"(r[o + 1]), "+r"(r[o + 2]), "+r"(r[o + 3]), "+r"(r[o + 4]), "+r"(r[o + 5]), \
    "+r"(r[o + 6]), "+r"(r[o + 7]), "+r"(r[o + 8]), "+r"(r[o + 9]), "+r"(r[o + 10]), "+r"(r[o + 11]),           \
    "+r"(r[o + 12]), "+r"(r[o + 13]), "+r"(r[o + 14]), "+r"(r[o + 15])
#define AV_LD16 "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
__device__ __forceinline__ void av_ld32(uint32_t c, uint32_t (&r)[32]) {
    asm volatile(AV_LD16 : AV_R16(0) : "r"(c));
    asm volatile(AV_LD16 : AV_R16(16) : "r"(c + 16));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : AV_W16(0), AV_W16(16) :: "memory");
}
#undef AV_R16
#undef AV_W16
#undef AV_LD16

// Byte offset of element (row r, k) in a K-major no-swizzle operand tile of AV_ROW bytes per row.
__host__ __device__ constexpr int av_off(int r, int k) { return (r / 8) * AV_SBO + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4; }

// G operands: [map][hi tile, lo tile]; row n = 16 t + a, column k = b.
__global__ void __launch_bounds__(256) k_adjv_gprep(int P, int n_pair, const float* __restrict__ hk, char* __restrict__ out) {
    const int bmap = blockIdx.x;
    char* dst = out + (int64_t)bmap * AV_BMAP;
    for (int e = threadIdx.x; e < 256 * AV_PM; e += blockDim.x) {
        const int n = e / AV_PM, k = e % AV_PM, t = n / AV_PM, a = n % AV_PM;
        float v = 0.f;
        if (t < P && a < P && k < P && a <= k) {
            const int c = a * P - a * (a - 1) / 2 + (k - a);
            v = hk[((int64_t)bmap * P + t) * n_pair + c];
        }
        uint32_t hi, lo;
        av_split(v, hi, lo);
        *reinterpret_cast<uint32_t*>(dst + av_off(n, k)) = hi;
        *reinterpret_cast<uint32_t*>(dst + AV_GT + av_off(n, k)) = lo;
    }
}

struct AdjVArgs {
    int P, b_first, B, n_quads, G;
    int64_t npix, ntiles;
    const char* gops;              // [B][AV_BMAP] from k_adjv_gprep
    const float* W;                // [npix]
    float* maps;                   // [B][P][npix]: M in, U^M out (in place)
    int* err;
};

// grid: n_quads * G CTAs; CTA (quad q, column c) keeps maps b_first + 4 q .. + 3 and walks
// pixel tiles c, c + G, ...; its tile-maps n = (tile index) * nbq + (map of the quad) are
// dealt to the two groups alternately.  One thread of its own warp issues every MMA (its
// warp-mates wait at the final barrier: a lane spinning on an mbarrier in the issuer's warp
// would hold each issue back).  The loader warp streams each tile-map's 16 x 128
// map values into a ring of AV_STAGES shared-memory tiles by 2D TMA (maps_map: rows b P + p
// of the chunk's maps, boxes of 128 pixels x 16 rows; rows and pixels past the end read as
// zero), so that several tiles per SM are in flight.
__global__ void __launch_bounds__(AV_THREADS, 1) k_adjoint_v(const __grid_constant__ CUtensorMap maps_map, AdjVArgs a) {
    extern __shared__ __align__(1024) char av_smem[];
    char* sG = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(av_smem) + 1023) & ~uintptr_t(1023));
    char* sA = sG + AV_MAPS * AV_BMAP;             // [AV_GROUPS][hi, lo]
    const float* sM = reinterpret_cast<const float*>(sA + AV_GROUPS * AV_ABUF);   // [AV_STAGES][16][128]
    __shared__ uint64_t a_full[AV_GROUPS], mma_done[AV_GROUPS], gbar, m_full[AV_STAGES], m_empty[AV_STAGES];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_word;
    volatile int* abort_flag = &abort_word;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int mq = blockIdx.x % a.n_quads;
    const int64_t tile0 = blockIdx.x / a.n_quads;
    const int b0 = a.b_first + mq * AV_MAPS;
    const int nbq = min(AV_MAPS, a.b_first + a.B - b0);
    const int64_t ntile_cta = (tile0 < a.ntiles) ? (a.ntiles - tile0 + a.G - 1) / a.G : 0;
    const int64_t n_tm = (nbq > 0) ? ntile_cta * nbq : 0;
    constexpr uint32_t tmem_cols = 512;

    if (threadIdx.x == 0) {
        for (int i = 0; i < AV_GROUPS; ++i) {
            mbar_init(&a_full[i], AV_GW);                // the group's warps, once per tile-map
            mbar_init(&mma_done[i], 1);
        }
        mbar_init(&gbar, 1);
        for (int i = 0; i < AV_STAGES; ++i) {
            mbar_init(&m_full[i], 1);
            mbar_init(&m_empty[i], AV_GW);               // the consuming group's warps
        }
        abort_word = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == AV_GW * AV_GROUPS) {
        // ---------------- loader: the quad's G operands once, then every tile-map's map values
        if (lane == 0 && n_tm > 0) {
            mbar_arrive_expect_tx(&gbar, (uint32_t)(nbq * AV_BMAP));
            bulk_copy_g2s(sG, a.gops + (int64_t)(b0 - a.b_first) * AV_BMAP, (uint32_t)(nbq * AV_BMAP), &gbar);
            int64_t n_issued = 0;
            for (int64_t n = 0; n < n_tm && !*abort_flag; ++n) {
                const int s = (int)(n % AV_STAGES);
                const uint32_t ph = (uint32_t)((n / AV_STAGES) & 1);
                if (!mbar_wait(&m_empty[s], ph ^ 1, abort_flag, a.err)) break;
                mbar_arrive_expect_tx(&m_full[s], (uint32_t)AV_MT);
                const int x0 = (int)((tile0 + (n / nbq) * a.G) * 128);
                const int y0 = (b0 - a.b_first + (int)(n % nbq)) * a.P;
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
                        "r"(smem_u32(sM + (int64_t)s * AV_PM * 128)), "l"(reinterpret_cast<uint64_t>(&maps_map)),
                        "r"(x0), "r"(y0), "r"(smem_u32(&m_full[s]))
                    : "memory");
                n_issued = n + 1;
            }
            // copies still in flight complete before the CTA exits
            const long long t0 = clock64();
            while (!mbar_try_wait(&gbar, 0) && clock64() - t0 < TC_WAIT_CYCLES) {
            }
            for (int64_t n = (n_issued > AV_STAGES ? n_issued - AV_STAGES : 0); n < n_issued; ++n) {
                const long long t1 = clock64();
                while (!mbar_try_wait(&m_full[n % AV_STAGES], (uint32_t)((n / AV_STAGES) & 1)) &&
                       clock64() - t1 < TC_WAIT_CYCLES) {
                }
            }
        }
    } else if (warp == AV_GW * AV_GROUPS + 1) {
        // ---------------- MMA issuer: tile-map n goes to group n % 2's accumulator
        if (lane == 0 && n_tm > 0) {
            const uint32_t idesc = umma_idesc(2, AV_PM * a.P);
            bool ok = mbar_wait(&gbar, 0, abort_flag, a.err);
            for (int64_t n = 0; ok && n < n_tm; ++n) {
                const int g = (int)(n % AV_GROUPS);
                const uint32_t k = (uint32_t)(n / AV_GROUPS);
                ok = mbar_wait(&a_full[g], k & 1, abort_flag, a.err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t dcol = tmem + (uint32_t)(g * 256);
                const uint32_t aHi_s = smem_u32(sA + g * AV_ABUF), aLo_s = aHi_s + AV_AT;
                const uint32_t gHi_s = smem_u32(sG + (int)(n % nbq) * AV_BMAP), gLo_s = gHi_s + AV_GT;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const uint32_t ko = (uint32_t)(s * 2 * 128);     // two core matrices = 8 tf32 of K
                    const uint64_t ah = umma_desc(aHi_s + ko), al = umma_desc(aLo_s + ko);
                    const uint64_t bh = umma_desc(gHi_s + ko), bl = umma_desc(gLo_s + ko);
                    umma<true>(dcol, ah, bh, idesc, s > 0 ? 1u : 0u);
                    umma<true>(dcol, ah, bl, idesc, 1u);
                    umma<true>(dcol, al, bh, idesc, 1u);
                }
                umma_commit(&mma_done[g]);
            }
        }
    } else {
        // ---------------- converter / epilogue groups: warp (quarter, half) converts K values
        // 8 half .. + 7 of its pixels and forms U^M_t for t = 8 half .. + 7
        const int g = warp / AV_GW, quarter = warp % 4, half = (warp % AV_GW) / 4;
        const int xl = quarter * 32 + lane;              // pixel within the tile = TMEM lane
        const uint32_t dcol = tmem + (uint32_t)(g * 256);
        const uint32_t lane_base = dcol + ((uint32_t)(quarter * 32) << 16);
        char* aHi = sA + g * AV_ABUF;
        char* aLo = aHi + AV_AT;
        uint32_t u = 0;                                  // tile-maps this group has handed to the MMA warp
        bool ok = true;
        for (int64_t n = g; ok && n < n_tm; n += AV_GROUPS, ++u) {
            const int j = (int)(n % nbq);
            const int64_t x = (tile0 + (n / nbq) * a.G) * 128 + xl;
            const bool in = x < a.npix;
            // this tile-map's map values from the TMA ring (rows p >= P belong to the next map)
            const int s = (int)(n % AV_STAGES);
            ok = !*abort_flag && mbar_wait(&m_full[s], (uint32_t)((n / AV_STAGES) & 1), abort_flag, a.err);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            float M[AV_PM];
            const float* ms = sM + (int64_t)s * AV_PM * 128 + xl;
#pragma unroll
            for (int p = 0; p < AV_PM; ++p) M[p] = (p < a.P) ? ms[p * 128] : 0.f;
            __syncwarp();
            if (lane == 0) mbar_arrive(&m_empty[s]);
            // A operand: this pixel's row of M (k = b), tf32 hi and lo, this half's K values
#pragma unroll
            for (int kc = 0; kc < AV_PM / 4; ++kc) {
                if ((kc >> 1) != half) continue;         // (compile-time kc keeps M in registers)
                uint4 hv, lv;
                av_split(M[4 * kc + 0], hv.x, lv.x);
                av_split(M[4 * kc + 1], hv.y, lv.y);
                av_split(M[4 * kc + 2], hv.z, lv.z);
                av_split(M[4 * kc + 3], hv.w, lv.w);
                *reinterpret_cast<uint4*>(aHi + av_off(xl, 4 * kc)) = hv;
                *reinterpret_cast<uint4*>(aLo + av_off(xl, 4 * kc)) = lv;
            }
            fence_proxy_async();                         // generic-proxy stores -> the MMA's reads
            tc_fence_before();                           // this warp's reads of the accumulator are done
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_full[g]);
            ok = !*abort_flag && mbar_wait(&mma_done[g], u & 1, abort_flag, a.err);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc_fence_after();
            // epilogue: U^M_t = W_x sum_a M_a V[x, 16 t + a], two t per TMEM wait, two
            // partial sums per t (columns past 16 P lie inside the group's 256 and are unused)
            const float w = in ? __ldg(a.W + x) : 0.f;
            float* out = a.maps + (int64_t)(b0 + j) * a.P * a.npix + x;
            for (int t0 = 8 * half; t0 < min(a.P, 8 * half + 8); t0 += 2) {
                uint32_t r[32];
                av_ld32(lane_base + (uint32_t)(16 * t0), r);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int q = 0; q < AV_PM / 2; ++q) {
                        s0 = fmaf(M[q], __uint_as_float(r[16 * i + q]), s0);
                        s1 = fmaf(M[q + 8], __uint_as_float(r[16 * i + q + 8]), s1);
                    }
                    if (in && t0 + i < a.P) out[(int64_t)(t0 + i) * a.npix] = w * (s0 + s1);
                }
            }
        }
        if (!ok && lane == 0) atomicOr(a.err, MODAL_DEVERR_TIMEOUT);   // tile-maps left undone: never silent
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
    }
}

size_t adjoint_v_workspace_bytes(const Plan& pl, int chunk) {
    return pl.prec == MODAL_FP32 ? 0 : (size_t)chunk * AV_BMAP;
}

// cuTensorMapEncodeTiled from the CUDA driver API, looked up once through the runtime.
typedef CUresult (*AvEncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static AvEncodeTiledFn av_encode_tiled() {
    static std::once_flag once;
    static AvEncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<AvEncodeTiledFn>(p);
    });
    return fn;
}

cudaError_t launch_adjoint_v(Plan& pl, int B, const float* hk, float* maps, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    // the map rows' pitch (npix floats) must be a multiple of 16 bytes for the tensor map
    if (!pl.adj_gops || B > pl.chunk || pl.P > AV_PM || pl.npix % 4 != 0) return cudaErrorInvalidValue;
    k_adjv_gprep<<<B, 256, 0, st>>>(pl.P, pl.n_pair, hk, pl.adj_gops);
    note_launch(pl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = 1024 + (size_t)AV_MAPS * AV_BMAP + (size_t)AV_GROUPS * AV_ABUF + (size_t)AV_STAGES * AV_MT;
    e = cudaFuncSetAttribute(k_adjoint_v, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    AvEncodeTiledFn enc = av_encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    AdjVArgs a;
    a.P = pl.P;
    a.npix = pl.npix;
    a.ntiles = (pl.npix + 127) / 128;
    a.gops = pl.adj_gops;
    a.W = pl.W;
    a.maps = maps;
    a.err = pl.d_err;
    const int nsm = std::max(pl.nsm, 1);
    // one CTA per SM (each holds all 512 TMEM columns): launches of up to nsm map quads
    const int quads = (B + AV_MAPS - 1) / AV_MAPS;
    for (int q0 = 0; q0 < quads; q0 += nsm) {
        const int nq = std::min(nsm, quads - q0);
        a.b_first = q0 * AV_MAPS;
        a.B = std::min(B - a.b_first, nq * AV_MAPS);
        a.n_quads = nq;
        a.G = (int)std::max<int64_t>(1, std::min<int64_t>(nsm / nq, a.ntiles));
        a.gops = pl.adj_gops + (int64_t)a.b_first * AV_BMAP;
        // rows of this launch's maps: b P + p for b in [b_first, b_first + B)
        alignas(64) CUtensorMap mm;
        const cuuint64_t dims[2] = {(cuuint64_t)pl.npix, (cuuint64_t)a.B * pl.P};
        const cuuint64_t strides[1] = {(cuuint64_t)pl.npix * sizeof(float)};
        const cuuint32_t box[2] = {128, (cuuint32_t)AV_PM};
        const cuuint32_t estr[2] = {1, 1};
        const CUresult r = enc(&mm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, maps + (int64_t)a.b_first * pl.P * pl.npix, dims,
                               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        k_adjoint_v<<<nq * a.G, AV_THREADS, smem, st>>>(mm, a);
        note_launch(pl);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace modal
