// Tensor-core (tcgen05, sm_103a) pixel weights of the adjoint with 3xTF32 operands:
//
//   U_t(x) = W_x sum_c h_{b,t,c} Q_c(x),  Q_c = M_a M_b' - <M_a M_b'>_x,  c = (a <= b')
//
// (the derivative of sum_n g_n beta_n with respect to M_t(x), Eq. bbispect with its linear
// term; h_{b,t,c} = 3 k_c h_tab as formed by k_adjoint_weights).  Per map b this is a GEMM
// with M = 128 pixels, N = 16 (t), K = 144 pairs (136 zero-padded):
//   D[x, t] = sum_c Q[x, c] H_b[c, t],   U_t(x) = W_x D[x, t].
// Each output is a fresh 136-term sum, so the tensor core's FP32 accumulator needs no
// hand-off to register sums.
//
// A (Q) lives in tensor memory: a converter thread owns one pixel (one TMEM lane), forms
// its pair products in FP32 (one fmaf with the pair mean, as the SIMT kernel), splits each
// into tf32 hi + lo (both rounded to nearest) and stores them along the lane's columns with
// tcgen05.st, so the operand never passes through shared memory.  B (H_b, split the same
// way, core-matrix K-major layout) stays in shared memory for the CTA's 4 maps.
// K runs in three stages of 48 pairs.  Four groups of four converter warps (one per TMEM
// lane quarter) each own an A region of one stage (48 hi + 48 lo columns) and a 16-column
// accumulator; a group converts a stage, its leader thread issues the 6 K-steps x 3
// products (hi*hi, hi*lo, lo*hi, kind::tf32, A from TMEM) and commits to the group's
// mbarrier; after the third stage the group reads its accumulator, scales by W_x and
// writes U in place over the maps (tile by tile; a tile's maps are read before its U is
// written).  The CTA's tile-maps (pixel tile, map of the quad) are dealt to the groups
// round-robin, so with a full quad group g takes map g of every tile; a loader warp brings
// each tile's pair means into shared memory by TMA (double-buffered), and every group walks
// every tile of the CTA, so the pair-mean buffers' phases stay in step.
//
// Work: the CTA keeps one quad of maps (its B operands) and walks pixel tiles c / n_quads,
// + G, ...; CTAs next to each other take the same tile for different quads.  Every wait is
// bounded as in the Legendre kernels; on expiry the kernel records MODAL_DEVERR_TIMEOUT.
#include "modal_internal.cuh"

#include "tc_common.cuh"

#include <cuda.h>
#include <algorithm>
#include <cstring>
#include <mutex>

namespace modal {

constexpr int AT_PM = 16;                       // K laid out for 16 modes: k <-> (a <= b'), lexicographic
constexpr int AT_NPAIR = AT_PM * (AT_PM + 1) / 2;   // 136
constexpr int AT_SK = 48;                       // pairs per stage
constexpr int AT_NST = 3;                       // stages (144 >= 136)
constexpr int AT_GROUPS = 4;
constexpr int AT_THREADS = 32 * (4 * AT_GROUPS + 1);   // converter groups + the loader warp
constexpr int AT_MAPS = 4;                      // maps per CTA
constexpr int AT_SBO = (AT_SK / 4) * 128;       // bytes between 8-row groups of a B tile (1536)
constexpr int AT_BT = 16 * AT_SK * 4;           // bytes of one B tile (16 rows x 48 tf32)
constexpr int AT_BMAP = AT_NST * 2 * AT_BT;     // bytes of one map's B operand (18432)
constexpr int AT_ACOLS = 2 * AT_SK;             // TMEM columns of one A stage (hi, lo)
constexpr int AT_DCOL0 = AT_GROUPS * AT_ACOLS;  // first accumulator column (384)

__host__ __device__ constexpr int at_pair_a(int k) {
    int a = 0;
    while (a < AT_PM && k >= AT_PM - a) {
        k -= AT_PM - a;
        ++a;
    }
    return a;
}
__host__ __device__ constexpr int at_pair_b(int k) {
    int a = 0;
    while (a < AT_PM && k >= AT_PM - a) {
        k -= AT_PM - a;
        ++a;
    }
    return a + k;
}

// B operand of every map: [map][stage][hi tile, lo tile], element (t, k) of a tile at
// (t / 8) AT_SBO + (k / 4) 128 + (t % 8) 16 + (k % 4) 4 bytes; k = pair within the stage.
__global__ void __launch_bounds__(256) k_adj_hprep(int P, int n_pair, const float* __restrict__ hk,
                                                   char* __restrict__ out) {
    const int b = blockIdx.x;
    char* dst = out + (int64_t)b * AT_BMAP;
    for (int e = threadIdx.x; e < AT_NST * 16 * AT_SK; e += blockDim.x) {
        const int S = e / (16 * AT_SK), rem = e % (16 * AT_SK), t = rem / AT_SK, kk = rem % AT_SK;
        const int k = S * AT_SK + kk;
        float v = 0.f;
        if (k < AT_NPAIR && t < P) {
            const int a = at_pair_a(k), bb = at_pair_b(k);
            if (a < P && bb < P) v = hk[((int64_t)b * P + t) * n_pair + a * P - a * (a - 1) / 2 + (bb - a)];
        }
        uint32_t hi, lo;
        Split<MODAL_3XTF32>::split(v, hi, lo);
        const int off = S * 2 * AT_BT + (t >> 3) * AT_SBO + (kk >> 2) * 128 + (t & 7) * 16 + (kk & 3) * 4;
        *reinterpret_cast<uint32_t*>(dst + off) = hi;
        *reinterpret_cast<uint32_t*>(dst + off + AT_BT) = lo;
    }
}

struct AdjTcArgs {
    int P, n_pair, B, b_first;       // maps b_first .. b_first + B - 1 of the chunk
    int n_quads, G;                  // map quads in this launch; CTAs per quad
    int64_t npix, ntiles;
    const char* hops;                // [chunk][AT_BMAP] (k_adj_hprep)
    const float* pm;                 // [n_pair][npix] pair means, or null
    const float* W;                  // [npix]
    float* maps;                     // [chunk][P][npix], U written in place
    int* err;
};

__device__ __forceinline__ uint64_t at_bdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(AT_SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void at_mma(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void at_st8(uint32_t taddr, const uint32_t (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

// tf32 hi part of x rounded to nearest (ties away from zero): add half an ulp of the
// 10-bit mantissa to the magnitude bits and clear the 13 bits below it.  x - hi is exact
// in FP32; the tensor core reads that lo part's top 19 bits.
__device__ __forceinline__ void at_split(float x, uint32_t& hi, uint32_t& lo) {
    hi = (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}

// Q of pair K at this thread's pixel, split into tf32 hi/lo.  spm: the pixel's column of the
// tile's pair means in shared memory ([row][128 pixels]) or null; with all 16 modes (FULL)
// row = K, otherwise rows[K] is the lexicographic pair row for the plan's P (-1: a mode past
// P, whose map values are zero and whose mean does not exist).
template <int K, bool FULL>
__device__ __forceinline__ void at_q(const float (&M)[AT_PM], const float* spm, const short* rows, uint32_t& hi,
                                     uint32_t& lo) {
    float q = 0.f;
    if constexpr (K < AT_NPAIR) {
        constexpr int A = at_pair_a(K), Bb = at_pair_b(K);
        float pv = 0.f;
        if (spm) {
            if constexpr (FULL) {
                pv = spm[K * 128];
            } else {
                const int row = rows[K];
                if (row >= 0) pv = spm[row * 128];
            }
        }
        q = fmaf(M[A], M[Bb], -pv);
    }
    at_split(q, hi, lo);
}

// One 8-pair column block (pairs K0 .. K0 + 7) of a stage, stored at columns col, col + AT_SK.
template <int K0, bool FULL>
__device__ __forceinline__ void at_block(const float (&M)[AT_PM], const float* spm, const short* rows, uint32_t taddr) {
    uint32_t hi[8], lo[8];
    at_q<K0 + 0, FULL>(M, spm, rows, hi[0], lo[0]);
    at_q<K0 + 1, FULL>(M, spm, rows, hi[1], lo[1]);
    at_q<K0 + 2, FULL>(M, spm, rows, hi[2], lo[2]);
    at_q<K0 + 3, FULL>(M, spm, rows, hi[3], lo[3]);
    at_q<K0 + 4, FULL>(M, spm, rows, hi[4], lo[4]);
    at_q<K0 + 5, FULL>(M, spm, rows, hi[5], lo[5]);
    at_q<K0 + 6, FULL>(M, spm, rows, hi[6], lo[6]);
    at_q<K0 + 7, FULL>(M, spm, rows, hi[7], lo[7]);
    at_st8(taddr, hi);
    at_st8(taddr + AT_SK, lo);
}

template <int S, int BLK, bool FULL>
__device__ __forceinline__ void at_stage(const float (&M)[AT_PM], const float* spm, const short* rows, uint32_t taddr) {
    if constexpr (BLK < AT_SK / 8) {
        at_block<S * AT_SK + BLK * 8, FULL>(M, spm, rows, taddr + BLK * 8);
        at_stage<S, BLK + 1, FULL>(M, spm, rows, taddr);
    }
}

template <bool FULL>
__global__ void __launch_bounds__(AT_THREADS, 1) k_adjoint_tc(const __grid_constant__ CUtensorMap pm_map, AdjTcArgs a) {
    extern __shared__ __align__(1024) char at_smem[];
    char* sB = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(at_smem) + 1023) & ~uintptr_t(1023));
    float* sPM = reinterpret_cast<float*>(sB + AT_MAPS * AT_BMAP);       // [2][n_pair][128]
    __shared__ uint64_t a_full[AT_GROUPS], mma_done[AT_GROUPS], hbar, pm_full[2], pm_empty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_word;
    __shared__ short rows[AT_NST * AT_SK];
    volatile int* abort_flag = &abort_word;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int g = warp / 4, quarter = warp % 4;
    const int mq = blockIdx.x % a.n_quads;
    const int64_t tile0 = blockIdx.x / a.n_quads;
    const int b0 = a.b_first + mq * AT_MAPS;
    const int nbq = min(AT_MAPS, a.b_first + a.B - b0);
    const int64_t ntile_cta = (tile0 < a.ntiles) ? (a.ntiles - tile0 + a.G - 1) / a.G : 0;
    const int64_t n_tm = ntile_cta * nbq;                 // tile-maps of this CTA
    const bool use_pm = a.pm != nullptr;
    constexpr uint32_t tmem_cols = 512;

    if (threadIdx.x == 0) {
        for (int i = 0; i < AT_GROUPS; ++i) {
            mbar_init(&a_full[i], 4);
            mbar_init(&mma_done[i], 1);
        }
        mbar_init(&hbar, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&pm_full[i], 1);
            mbar_init(&pm_empty[i], 4 * AT_GROUPS);       // every converter warp, once per tile
        }
        abort_word = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int k = threadIdx.x; k < AT_NST * AT_SK; k += blockDim.x) {
        int row = -1;
        if (k < AT_NPAIR) {
            const int pa = at_pair_a(k), pb = at_pair_b(k);
            if (pa < a.P && pb < a.P) row = pa * a.P - pa * (pa - 1) / 2 + (pb - pa);
        }
        rows[k] = (short)row;
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

    if (warp == 4 * AT_GROUPS) {
        // ---------------- loader: the maps' B operands once, the pair means of every tile
        if (lane == 0 && n_tm > 0) {
            mbar_arrive_expect_tx(&hbar, (uint32_t)(nbq * AT_BMAP));
            bulk_copy_g2s(sB, a.hops + (int64_t)b0 * AT_BMAP, (uint32_t)(nbq * AT_BMAP), &hbar);
            int64_t n_issued = 0;
            for (int64_t i = 0; use_pm && i < ntile_cta && !*abort_flag; ++i) {
                const int buf = (int)(i & 1);
                const uint32_t ph = (uint32_t)((i >> 1) & 1);
                if (!mbar_wait(&pm_empty[buf], ph ^ 1, abort_flag, a.err)) break;
                // one 2D tensor copy: 128 pixels x n_pair rows (pixels past npix read as zero)
                const int x0 = (int)((tile0 + i * a.G) * 128);
                mbar_arrive_expect_tx(&pm_full[buf], (uint32_t)(128 * a.n_pair * 4));
                float* dst = sPM + (int64_t)buf * a.n_pair * 128;
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
                        "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(&pm_map)), "r"(x0), "r"(0),
                        "r"(smem_u32(&pm_full[buf]))
                    : "memory");
                n_issued = i + 1;
            }
            // copies still in flight complete before the CTA exits
            const long long t0 = clock64();
            while (!mbar_try_wait(&hbar, 0) && clock64() - t0 < TC_WAIT_CYCLES) {
            }
            for (int64_t i = (n_issued > 2 ? n_issued - 2 : 0); i < n_issued; ++i) {   // the last fill of each buffer
                const long long t1 = clock64();
                while (!mbar_try_wait(&pm_full[i & 1], (uint32_t)((i >> 1) & 1)) && clock64() - t1 < TC_WAIT_CYCLES) {
                }
            }
        }
    } else {
        // ---------------- converter groups (MMA issued by each group's leader thread)
        const uint32_t idesc = umma_idesc(2, 16);
        const uint32_t colA = (uint32_t)(g * AT_ACOLS), colD = (uint32_t)(AT_DCOL0 + g * 16);
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        const bool leader = (quarter == 0) && lane == 0;
        const int xl = quarter * 32 + lane;                // pixel within the tile = TMEM lane
        uint32_t u = 0;                                   // stages this group has issued
        bool ok = true, have_prev = false;
        int64_t prev_x = 0;
        int prev_b = 0;
        // U of the group's previous tile-map: accumulator -> W_x D[x, t] -> maps (in place)
        auto epilogue = [&]() {
            float v[16];
            tmem_ld16(lane_base + colD, v);
            if (prev_x < a.npix) {
                const float w = __ldg(a.W + prev_x);
                float* out = a.maps + (int64_t)prev_b * a.P * a.npix + prev_x;
#pragma unroll
                for (int t = 0; t < 16; ++t)
                    if (t < a.P) out[(int64_t)t * a.npix] = v[t] * w;
            }
        };
        // Every group walks every tile of the CTA in order: it waits for the tile's pair means,
        // converts its own tile-maps of that tile (n = ti nbq + j with n = g mod AT_GROUPS, none
        // for some tiles when nbq < AT_GROUPS) and releases the buffer, so each buffer's fills
        // are observed one phase at a time and no tile can overtake another on a buffer.
        // The map values of the group's next tile-map are loaded one tile-map ahead.
        float Mn[AT_PM];
        auto load_maps = [&](int64_t n) {
            const int64_t x = (tile0 + (n / nbq) * a.G) * 128 + xl;
            const bool in = n < n_tm && x < a.npix;
            const float* mb = a.maps + (int64_t)(b0 + (int)(n % nbq)) * a.P * a.npix + x;
#pragma unroll
            for (int p = 0; p < AT_PM; ++p) Mn[p] = (in && p < a.P) ? mb[(int64_t)p * a.npix] : 0.f;
        };
        int64_t next_n = g;
        load_maps(next_n);
        for (int64_t ti = 0; ok && ti < ntile_cta; ++ti) {
            const float* spm_tile = nullptr;
            if (use_pm) {
                ok = !*abort_flag && mbar_wait(&pm_full[ti & 1], (uint32_t)((ti >> 1) & 1), abort_flag, a.err);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                spm_tile = sPM + (int64_t)(ti & 1) * a.n_pair * 128 + xl;
            }
            for (; next_n < n_tm && next_n / nbq == ti; ) {
                const int64_t n = next_n;
                next_n += AT_GROUPS;
                const int64_t tile = tile0 + ti * a.G;
                const int b = b0 + (int)(n % nbq);
                const int64_t x = tile * 128 + xl;
                const bool in = x < a.npix;
                float M[AT_PM];
#pragma unroll
                for (int p = 0; p < AT_PM; ++p) M[p] = Mn[p];
                load_maps(next_n);
                const float* spm = in ? spm_tile : nullptr;
#pragma unroll
                for (int S = 0; S < AT_NST; ++S) {
                    if (u > 0) {                          // the group's previous stage is consumed
                        ok = ok && !*abort_flag && mbar_wait(&mma_done[g], (u - 1) & 1, abort_flag, a.err);
                        ok = __all_sync(0xffffffffu, ok);
                        if (!ok) break;
                        tc_fence_after();
                        if (S == 0 && have_prev) epilogue();
                    }
                    if (S == 0) at_stage<0, 0, FULL>(M, spm, rows, lane_base + colA);
                    else if (S == 1) at_stage<1, 0, FULL>(M, spm, rows, lane_base + colA);
                    else at_stage<2, 0, FULL>(M, spm, rows, lane_base + colA);
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&a_full[g]);
                    if (leader) {
                        bool go = mbar_wait(&a_full[g], u & 1, abort_flag, a.err);
                        if (go && u == 0) go = mbar_wait(&hbar, 0, abort_flag, a.err);
                        if (go) {
                            tc_fence_after();
                            const uint32_t bh0 = smem_u32(sB + (int64_t)(b - b0) * AT_BMAP + S * 2 * AT_BT);
                            const uint32_t dcol = tmem + colD;
#pragma unroll
                            for (int i = 0; i < AT_SK / 8; ++i) {
                                const uint32_t ah = tmem + colA + i * 8, al = ah + AT_SK;
                                const uint64_t bh = at_bdesc(bh0 + i * 256), bl = at_bdesc(bh0 + AT_BT + i * 256);
                                at_mma(dcol, ah, bh, idesc, (S == 0 && i == 0) ? 0u : 1u);
                                at_mma(dcol, ah, bl, idesc, 1u);
                                at_mma(dcol, al, bh, idesc, 1u);
                            }
                        }
                        umma_commit(&mma_done[g]);        // also on abort: keeps the phases in step
                    }
                    __syncwarp();
                    ++u;
                }
                if (!ok) break;
                have_prev = true;
                prev_x = x;
                prev_b = b;
            }
            if (!ok) break;
            // this warp's last read of the tile's pair means is done (its stores to TMEM waited)
            if (use_pm && lane == 0) mbar_arrive(&pm_empty[ti & 1]);
        }
        if (ok && have_prev) {
            ok = mbar_wait(&mma_done[g], (u - 1) & 1, abort_flag, a.err);
            ok = __all_sync(0xffffffffu, ok);
            if (ok) {
                tc_fence_after();
                epilogue();
            }
        }
        if (!ok && lane == 0) atomicOr(a.err, MODAL_DEVERR_TIMEOUT);    // tile-maps left undone: never silent
        if (leader && u > 0) {                            // the group's MMAs complete before TMEM is freed
            const long long t0 = clock64();
            while (!mbar_try_wait(&mma_done[g], (u - 1) & 1) && clock64() - t0 < TC_WAIT_CYCLES) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Tensor map of the pair-mean panel [n_pair][npix] float: boxes of 128 pixels x n_pair rows.
static cudaError_t pair_mean_map(const Plan& pl, CUtensorMap* map) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)pl.npix, (cuuint64_t)pl.n_pair};
    const cuuint64_t strides[1] = {(cuuint64_t)pl.npix * sizeof(float)};
    const cuuint32_t box[2] = {128, (cuuint32_t)pl.n_pair};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, pl.pair_mean, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t adjoint_tc_workspace_bytes(const Plan& pl, int chunk) {
    return pl.prec == MODAL_FP32 ? 0 : (size_t)chunk * AT_BMAP;
}

cudaError_t launch_adjoint_tc(Plan& pl, int B, const float* hk, int use_linear, float* maps, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    if (!pl.adj_hops || B > pl.chunk || pl.P > AT_PM || pl.npix % 4 != 0) return cudaErrorInvalidValue;
    k_adj_hprep<<<B, 256, 0, st>>>(pl.P, pl.n_pair, hk, pl.adj_hops);
    note_launch(pl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = 1024 + (size_t)AT_MAPS * AT_BMAP + (use_linear ? (size_t)2 * pl.n_pair * 128 * 4 : 0);
    const bool full = pl.P == AT_PM;
    e = full ? cudaFuncSetAttribute(k_adjoint_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
             : cudaFuncSetAttribute(k_adjoint_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    AdjTcArgs a;
    a.P = pl.P;
    a.n_pair = pl.n_pair;
    a.npix = pl.npix;
    a.ntiles = (pl.npix + 127) / 128;
    a.hops = pl.adj_hops;
    a.pm = use_linear ? pl.pair_mean : nullptr;
    a.W = pl.W;
    a.maps = maps;
    a.err = pl.d_err;
    alignas(64) CUtensorMap pm_map;
    std::memset(&pm_map, 0, sizeof(pm_map));
    if (a.pm) {
        e = pair_mean_map(pl, &pm_map);
        if (e != cudaSuccess) return e;
    }
    const int nsm = std::max(pl.nsm, 1);
    // at most one CTA per SM (each holds all 512 TMEM columns): launches of up to nsm map quads
    const int quads = (B + AT_MAPS - 1) / AT_MAPS;
    for (int q0 = 0; q0 < quads; q0 += nsm) {
        const int nq = std::min(nsm, quads - q0);
        a.b_first = q0 * AT_MAPS;
        a.B = std::min(B - a.b_first, nq * AT_MAPS);
        a.n_quads = nq;
        a.G = (int)std::max<int64_t>(1, std::min<int64_t>(nsm / nq, a.ntiles));
        const int grid = nq * a.G;
        if (full) k_adjoint_tc<true><<<grid, AT_THREADS, smem, st>>>(pm_map, a);
        else k_adjoint_tc<false><<<grid, AT_THREADS, smem, st>>>(pm_map, a);
        note_launch(pl);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace modal
