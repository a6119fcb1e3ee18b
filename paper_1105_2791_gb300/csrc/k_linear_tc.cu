// Tensor-core (tcgen05, sm_103a) linear-term GEMM with 3xTF32 operands.
//
//   G[(b, c), (ab)] = sum_x maps_{b,c}(x) * W_x <M_a M_b>_x        (Eq. bispectrumest linear term)
//
// M = 128 rows of (map, basis function), N = 144 (pairs, zero-padded), K = pixels.
// Work item = (row tile, pixel range), row tile fastest, so that the CTAs working on the
// row tiles of one pixel range run side by side and read its B blocks once from HBM and
// then from L2; a persistent CTA loops over items.  The B
// operand, W <M_a M_b> split into tf32 hi/lo in the no-swizzle K-major core-matrix
// layout, is the same for every map: k_lt_presplit builds it once per finalised mean,
// one block of 32 pixels per stage, and a loader thread streams each stage's block into
// shared memory with one cp.async.bulk.  Per stage eight converter warps load the maps'
// FP32 rows, split each value into two tf32 parts rounded to nearest and store them in
// the same layout; one thread issues tcgen05.mma (kind::tf32, hi*hi + hi*lo + lo*hi) into
// one of two TMEM accumulators.  Because the tensor core
// rounds its FP32 accumulator once per MMA, every 4 stages (16 MMA steps) the
// accumulator is handed to eight epilogue warps that add it into FP32 register sums
// and release it; the MMAs continue in the other buffer.  At the end of an item the
// register sums are written (FP64) to the split-K partials read by k_beta_finalize.
// All waits are bounded as in the Legendre kernels.
#include "modal_internal.cuh"

#include "tc_common.cuh"

#include <algorithm>

namespace modal {

constexpr int LT_N = 144;                  // pair columns (n_pair <= 136, padded to 16)
constexpr int LT_CONV_WARPS = 8;
constexpr int LT_EPI_WARPS = 8;
constexpr int LT_THREADS = 32 * (2 + LT_CONV_WARPS + LT_EPI_WARPS);
constexpr int LT_KPX = 32;                 // pixels per stage (128 bytes of fp32 per row)
constexpr int LT_A_TILE = 128 * 128;       // bytes
constexpr int LT_B_TILE = LT_N * 128;      // bytes
constexpr int LT_STAGE = 2 * LT_A_TILE + 2 * LT_B_TILE;
constexpr int LT_FLUSH = 4;                // stages per accumulator hand-off
constexpr int LT_COLS_PER_WARP = LT_N / 2; // epilogue: two warps per TMEM lane quarter

struct LinArgs {
    int nrows, ncols, n_pair;              // rows = n_pair (pairs), cols = B * P
    int64_t npix, krange;                  // pixels per item
    int n_mt, n_kr;
    const char* bsplit;                    // [npix / 32][hi B tile, lo B tile] (k_lt_presplit)
    const float* maps;                     // [cols][npix]
    double* out;                           // [n_kr][n_pair][ncols]
    int* err;
};

// One 32-pixel stage of the B operand per CTA: W_x <pair>_x split into tf32 hi/lo, rows
// 0..143 (pairs, zero past n_pair), stored as [hi tile][lo tile] with the converters'
// chunk order and core-matrix offsets.
__global__ void __launch_bounds__(256) k_lt_presplit(int n_pair, int64_t npix, const float* __restrict__ panel,
                                                     const float* __restrict__ W, char* __restrict__ out) {
    const int64_t xs = (int64_t)blockIdx.x * LT_KPX;
    char* base = out + (int64_t)blockIdx.x * 2 * LT_B_TILE;
    for (int c = threadIdx.x; c < LT_N * 8; c += blockDim.x) {
        const int row = ((c >> 6) << 3) + (c & 7), kc = (c >> 3) & 7;
        const int64_t x = xs + kc * 4;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (row < n_pair)
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (x + i < npix) v[i] = panel[(int64_t)row * npix + x + i] * W[x + i];
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) Split<MODAL_3XTF32>::split(v[i], hv[i], lv[i]);
        const int off = (row >> 3) * 1024 + kc * 128 + (row & 7) * 16;
        *reinterpret_cast<uint4*>(base + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<uint4*>(base + LT_B_TILE + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
}

__device__ __forceinline__ uint64_t lt_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(LT_THREADS, 1) k_linear_tc(LinArgs a) {
    extern __shared__ __align__(1024) char smem[];
    char* stages = smem;                                    // [2][A hi, A lo, B hi, B lo]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * LT_STAGE);
    uint64_t* full = bars;                                  // [2]
    uint64_t* empty = bars + 2;                             // [2]
    uint64_t* acc_full = bars + 4;                          // [2]
    uint64_t* acc_empty = bars + 6;                         // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    constexpr uint32_t tmem_cols = 512;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&full[s], LT_CONV_WARPS + 1);         // converters + the B loader's expect_tx
            mbar_init(&empty[s], 1);
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], LT_EPI_WARPS);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t n_items = (int64_t)a.n_mt * a.n_kr;

    if (warp == 0) {
        // ---------------- B loader (one thread): the pre-split pair-mean block of each stage
        if (lane == 0) {
            uint32_t it = 0;
            uint32_t last_phase[2] = {0, 0};
            bool issued[2] = {false, false};
            for (int64_t item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x) {
                const int kr = (int)(item / a.n_mt);
                const int64_t x0 = (int64_t)kr * a.krange, x1 = min(a.npix, x0 + a.krange);
                const int nst = (int)(((x1 > x0 ? x1 - x0 : (int64_t)0) + LT_KPX - 1) / LT_KPX);
                for (int st = 0; st < nst; ++st, ++it) {
                    const int s = it & 1;
                    const uint32_t ph = (it >> 1) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, a.err)) break;
                    mbar_arrive_expect_tx(&full[s], 2 * LT_B_TILE);
                    bulk_copy_g2s(stages + s * LT_STAGE + 2 * LT_A_TILE,
                                  a.bsplit + (x0 / LT_KPX + st) * (int64_t)(2 * LT_B_TILE), 2 * LT_B_TILE, &full[s]);
                    last_phase[s] = ph;
                    issued[s] = true;
                }
            }
            // copies still in flight complete before the CTA exits
            for (int s = 0; s < 2; ++s) {
                if (!issued[s]) continue;
                const long long t0 = clock64();
                while (!mbar_try_wait(&full[s], last_phase[s]) && clock64() - t0 < TC_WAIT_CYCLES) {
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = umma_idesc(2, LT_N);
            uint32_t it = 0, nflush = 0;
            for (int64_t item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x) {
                const int kr = (int)(item / a.n_mt);
                const int64_t x0 = (int64_t)kr * a.krange, x1 = min(a.npix, x0 + a.krange);
                const int nst = (int)(((x1 > x0 ? x1 - x0 : (int64_t)0) + LT_KPX - 1) / LT_KPX);
                const int nfl = max(1, (nst + LT_FLUSH - 1) / LT_FLUSH);    // hand-offs (one even if empty)
                for (int f = 0; f < nfl; ++f, ++nflush) {
                    const int buf = nflush & 1;
                    const uint32_t d = tmem + (uint32_t)(buf * 256);
                    if (!mbar_wait(&acc_empty[buf], ((nflush >> 1) & 1) ^ 1, abort_flag, a.err)) break;
                    tc_fence_after();
                    const int s0 = f * LT_FLUSH, s1 = min(nst, s0 + LT_FLUSH);
                    for (int st = s0; st < s1; ++st, ++it) {
                        const int s = it & 1;
                        const uint32_t ph = (it >> 1) & 1;
                        if (!mbar_wait(&full[s], ph, abort_flag, a.err)) break;
                        tc_fence_after();
                        const uint32_t base = smem_u32(stages + s * LT_STAGE);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint32_t koff = ks * 2 * 128;
                            const uint64_t ah = lt_desc(base + koff);
                            const uint64_t al = lt_desc(base + LT_A_TILE + koff);
                            const uint64_t bh = lt_desc(base + 2 * LT_A_TILE + koff);
                            const uint64_t bl = lt_desc(base + 2 * LT_A_TILE + LT_B_TILE + koff);
                            const uint32_t acc = (st == s0 && ks == 0) ? 0u : 1u;
                            umma<true>(d, ah, bh, idesc, acc);
                            umma<true>(d, ah, bl, idesc, 1u);
                            umma<true>(d, al, bh, idesc, 1u);
                        }
                        umma_commit(&empty[s]);
                    }
                    umma_commit(&acc_full[buf]);
                }
            }
        }
    } else if (warp >= 2 && warp < 2 + LT_CONV_WARPS) {
        // ---------------- converters: the maps' FP32 rows -> tf32 hi/lo core matrices (A)
        const int ct = threadIdx.x - 64;                    // 0 .. 255
        uint32_t it = 0;
        for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
            if (*abort_flag) break;
            const int mt = (int)(item % a.n_mt), kr = (int)(item / a.n_mt);
            const int64_t x0 = (int64_t)kr * a.krange, x1 = min(a.npix, x0 + a.krange);
            const int nst = (int)(((x1 > x0 ? x1 - x0 : (int64_t)0) + LT_KPX - 1) / LT_KPX);
            for (int st = 0; st < nst; ++st, ++it) {
                const int s = it & 1;
                const uint32_t ph = (it >> 1) & 1;
                bool ok = !*abort_flag && mbar_wait(&empty[s], ph ^ 1, abort_flag, a.err);
                if (ok) {
                    char* base = stages + s * LT_STAGE;
                    const int64_t xs = x0 + (int64_t)st * LT_KPX;
                    // A: 128 rows x 8 chunks of 4 pixels.  Chunk index c runs over blocks of 8 rows,
                    // and within a block kc-major: c = 64 (row / 8) + 8 kc + row % 8, so that 8
                    // consecutive threads store the 8 rows of one core matrix (128 contiguous bytes)
                    // and a warp's 16-byte stores are free of bank conflicts.  Thread ct owns chunk
                    // column kc = (ct / 8) % 8 in every row it touches (stride 256 keeps kc fixed);
                    // all loads of the stage are issued before any value is split.
                    constexpr int NCH = 128 * 8;
                    constexpr int NU = NCH / (32 * LT_CONV_WARPS);
                    const int kc = (ct >> 3) & 7;
                    const int64_t x = xs + kc * 4;
                    const bool whole = (x + 3 < x1);            // x is a multiple of 4: 16-byte aligned
                    float4 vals[NU];
#pragma unroll
                    for (int u = 0; u < NU; ++u) {
                        const int c = ct + u * 32 * LT_CONV_WARPS;
                        const int row = ((c >> 6) << 3) + (c & 7);
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        const float* src = nullptr;
                        const int gr = mt * 128 + row;
                        if (gr < a.ncols) src = a.maps + (int64_t)gr * a.npix + x;
                        if (src) {
                            if (whole) v = *reinterpret_cast<const float4*>(src);
                            else {
                                if (x + 0 < x1) v.x = src[0];
                                if (x + 1 < x1) v.y = src[1];
                                if (x + 2 < x1) v.z = src[2];
                            }
                        }
                        vals[u] = v;
                    }
#pragma unroll
                    for (int u = 0; u < NU; ++u) {
                        const int c = ct + u * 32 * LT_CONV_WARPS;
                        const int row = ((c >> 6) << 3) + (c & 7);
                        const float4 v = vals[u];
                        uint32_t hv[4], lv[4];
                        Split<MODAL_3XTF32>::split(v.x, hv[0], lv[0]);
                        Split<MODAL_3XTF32>::split(v.y, hv[1], lv[1]);
                        Split<MODAL_3XTF32>::split(v.z, hv[2], lv[2]);
                        Split<MODAL_3XTF32>::split(v.w, hv[3], lv[3]);
                        const int off = (row >> 3) * 1024 + kc * 128 + (row & 7) * 16;
                        *reinterpret_cast<uint4*>(base + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                        *reinterpret_cast<uint4*>(base + LT_A_TILE + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                    }
                    fence_proxy_async();
                }
                __syncwarp();
                if (ok && lane == 0) mbar_arrive(&full[s]);
            }
        }
    } else if (warp >= 2 + LT_CONV_WARPS) {
        // ---------------- epilogue: TMEM hand-offs -> FP32 register sums -> FP64 partials
        const int ew = warp - 2 - LT_CONV_WARPS;            // 0 .. 7
        const int quarter = warp % 4;
        const int half = ew / 4;                            // column half
        const int row = quarter * 32 + lane;                // TMEM lane = row within the tile
        uint32_t nflush = 0;
        for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
            const int mt = (int)(item % a.n_mt), kr = (int)(item / a.n_mt);
            const int64_t x0 = (int64_t)kr * a.krange, x1 = min(a.npix, x0 + a.krange);
            const int nst = (int)(((x1 > x0 ? x1 - x0 : (int64_t)0) + LT_KPX - 1) / LT_KPX);
            const int nfl = max(1, (nst + LT_FLUSH - 1) / LT_FLUSH);
            float sum[LT_COLS_PER_WARP];
#pragma unroll
            for (int i = 0; i < LT_COLS_PER_WARP; ++i) sum[i] = 0.f;
            bool ok = true;
            for (int f = 0; f < nfl; ++f, ++nflush) {
                const int buf = nflush & 1;
                ok = !*abort_flag && mbar_wait(&acc_full[buf], (nflush >> 1) & 1, abort_flag, a.err);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc_fence_after();
                if (nst > 0) {
                    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + buf * 256 + half * LT_COLS_PER_WARP;
#pragma unroll
                    for (int c = 0; c < LT_COLS_PER_WARP; c += 8) {
                        float v[8];
                        tmem_ld8(taddr + c, v);
#pragma unroll
                        for (int i = 0; i < 8; ++i) sum[c + i] += v[i];
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[buf]);
            }
            if (!ok) {                                      // items left undone: never silent
                if (lane == 0) atomicOr(a.err, MODAL_DEVERR_TIMEOUT);
                break;
            }
            const int gr = mt * 128 + row;                  // (map, basis) column of G
            if (gr < a.ncols) {
#pragma unroll
                for (int i = 0; i < LT_COLS_PER_WARP; ++i) {
                    const int pr = half * LT_COLS_PER_WARP + i;
                    if (pr < a.n_pair) a.out[((int64_t)kr * a.n_pair + pr) * a.ncols + gr] = (double)sum[i];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
    }
}

// Pixel ranges: by default one per SM, so the n_mt * nsm items of equal size spread evenly
// over the nsm persistent CTAs, n_mt each; the plan's tuning may choose another count (the
// partial-sum buffer holds max(nsm, lt_ranges) ranges).
int linear_tc_splits(const Plan& pl, int B) {
    (void)B;
    const int r = pl.lt_ranges > 0 ? pl.lt_ranges : pl.nsm;
    return (int)std::max<int64_t>(1, std::min<int64_t>(r, pl.npix / LT_KPX));
}

size_t linear_presplit_bytes(const Plan& pl) {
    return (size_t)((pl.npix + LT_KPX - 1) / LT_KPX) * 2 * LT_B_TILE;
}

cudaError_t launch_linear_presplit(Plan& pl, cudaStream_t st) {
    if (pl.n_pair > LT_N || !pl.lin_bsplit) return cudaErrorInvalidValue;
    const int64_t nst = (pl.npix + LT_KPX - 1) / LT_KPX;
    k_lt_presplit<<<(unsigned)nst, 256, 0, st>>>(pl.n_pair, pl.npix, pl.pair_mean, pl.W, pl.lin_bsplit);
    note_launch(pl);
    return cudaGetLastError();
}

cudaError_t launch_linear_tc(Plan& pl, const float* maps, int B, double* partial, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    if (pl.n_pair > LT_N || !pl.lin_bsplit) return cudaErrorInvalidValue;
    LinArgs a;
    a.nrows = pl.n_pair;
    a.ncols = B * pl.P;
    a.n_pair = pl.n_pair;
    a.npix = pl.npix;
    a.n_mt = (a.ncols + 127) / 128;
    a.n_kr = linear_tc_splits(pl, B);
    a.krange = ((pl.npix + a.n_kr - 1) / a.n_kr + LT_KPX - 1) / LT_KPX * LT_KPX;
    a.bsplit = pl.lin_bsplit;
    a.maps = maps;
    a.out = partial;
    a.err = pl.d_err;
    const size_t smem = 1024 + 2 * LT_STAGE + 8 * 8 + 16;
    cudaError_t e = cudaFuncSetAttribute(k_linear_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, pl.dev);
    const int64_t items = (int64_t)a.n_mt * a.n_kr;
    const int grid = (int)std::min<int64_t>(items, (int64_t)std::max(nsm, 1));
    k_linear_tc<<<grid, LT_THREADS, smem, st>>>(a);
    note_launch(pl);
    return cudaGetLastError();
}

}  // namespace modal
