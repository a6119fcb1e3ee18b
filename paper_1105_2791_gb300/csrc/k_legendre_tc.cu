// Tensor-core (tcgen05, sm_103a) Legendre sums with compensated split precision.
//
// For every order m and parity pi of l - m the contraction
//     D_pi[j, n] = sum_{l = m + pi (mod 2)} lambda_lm(theta_j) * F[l, n],
//     F[l, (b, p, c)] = f_p(l) * (Re, Im)_c a_{b,lm}
// is a GEMM with M = ring pairs j, N = 2 P x (8 maps), K = l.  The north ring gets
// E + O, its mirror south ring E - O (lambda_lm(-mu) = (-1)^{l+m} lambda_lm(mu)).
//
// Work item = (m, parity, tile of 128 ring pairs, group of 8 maps).  A persistent CTA
// loops over items.  Per pipeline stage (TC_STAGES of them) it holds TC_KB bytes of K per row:
//   A (lambda, pre-split hi/lo, pre-tiled in HBM): fetched with one cp.async.bulk;
//   B (filtered a_lm, scaled and split hi/lo): built once per chunk by k_tc_prep_b in
//      the same layout and shared by all ring tiles; fetched with cp.async.bulk.
// One thread issues tcgen05.mma: hi*hi into TMEM accumulator D1 (columns 0..N-1) and
// the cross products hi*lo + lo*hi into D2 (columns N..2N-1).  The tensor core rounds
// its FP32 accumulator once per MMA; keeping the small cross terms apart makes their
// rounding 2^-11 smaller, so the error of a sum over ~10^3 values of l stays near
// (K/16) 2^-24 instead of three times that.  The 8 epilogue warps drain TMEM (two
// column blocks of D1 and D2 per wait), release it before their last stores so that the
// next item's MMAs start, form D1 + D2, undo the scaling and write the even (E) or odd
// (O) row for the ring pairs; the ring FFT forms north = E + O and south = E - O.
// Operands use the no-swizzle K-major core-matrix layout: element (row r, k) at
// (r/8)*TC_SBO + (k/(16/E))*128 + (r%8)*16 + (k%(16/E))*E bytes (E = element bytes).
//
// Every mbarrier wait is bounded (~1 s of clock): on expiry the kernel records
// MODAL_DEVERR_TIMEOUT, the roles drain, in-flight copies are awaited (bounded) and
// TMEM is freed before exit.
#include "modal_internal.cuh"

#include "tc_common.cuh"

namespace modal {

// ------------------------------------------------------------------ table builder
// Number of values of l in [m, L] with l - m = pi (mod 2), and K blocks of KPS of them
// (at least one, zero-padded, so that every item writes its row).
__host__ __device__ inline int tc_nkb(int L, int m, int pi, int kps) {
    const int k = (L - m - pi >= 0) ? (L - m - pi) / 2 + 1 : 0;
    return k > 0 ? (k + kps - 1) / kps : 1;
}

// Stage block (m, pi, rt, kb) = [hi tile, lo tile] of 128 ring pairs x KPS values of
// l = m + pi + 2 (kb KPS + k), KPS = 128 / E; lambda scaled by 2^11 for 16-bit formats.
template <int PREC>
__global__ void k_build_tc_table(int L, int R_half, int RH, int n_rt, const float* __restrict__ lam,
                                 const int64_t* __restrict__ blk_base, void* __restrict__ out) {
    using S = Split<PREC>;
    using T = typename ElemT<S::E>::T;
    constexpr int KPS = TC_KB / S::E;
    constexpr int CM = 16 / S::E;            // K values per core matrix
    const int m = blockIdx.y >> 1, pi = blockIdx.y & 1;
    const int nkb = tc_nkb(L, m, pi, KPS);
    const int64_t base_m = d_alm_index(m, m, L);
    const float scale = (S::E == 2) ? TC_LAMBDA_SCALE : 1.f;
    for (int64_t blk = blockIdx.x; blk < (int64_t)n_rt * nkb; blk += gridDim.x) {
        const int rt = (int)(blk / nkb), kb = (int)(blk % nkb);
        char* dst = reinterpret_cast<char*>(out) + (blk_base[2 * m + pi] + blk) * TC_A_STAGE;
        for (int e = threadIdx.x; e < 128 * KPS; e += blockDim.x) {
            const int r = e / KPS, k = e % KPS;
            const int l = m + pi + 2 * (kb * KPS + k);
            const int j = rt * 128 + r;
            float v = 0.f;
            if (l <= L && j < R_half) v = lam[(base_m + (l - m)) * (int64_t)RH + j] * scale;
            T hi, lo;
            S::split(v, hi, lo);
            const int off = (r / 8) * TC_SBO + (k / CM) * 128 + (r % 8) * 16 + (k % CM) * S::E;
            *reinterpret_cast<T*>(dst + off) = hi;
            *reinterpret_cast<T*>(dst + TC_A_TILE + off) = lo;
        }
    }
}

// ------------------------------------------------------------------ per-map scale
// amax[b] = max_{l,m,p} |f_p(l) a_{b,lm}| as float bits (positive floats order as ints).
// grid (AM_BLOCKS, B): block x takes orders m = x, x + AM_BLOCKS, ...; one atomic per warp.
constexpr int AM_BLOCKS = 64;
__global__ void __launch_bounds__(256) k_alm_amax(int L, const float* __restrict__ fmax_l, const float2* __restrict__ alm,
                                                  int64_t n_alm, unsigned* __restrict__ amax) {
    const int b = blockIdx.y;
    float v = 0.f;
    for (int m = blockIdx.x; m <= L; m += gridDim.x) {
        const float2* row = alm + (int64_t)b * n_alm + d_alm_index(m, m, L);
        for (int k = threadIdx.x; k <= L - m; k += blockDim.x) {
            const float2 a = row[k];
            v = fmaxf(v, fmaxf(fabsf(a.x), fabsf(a.y)) * fmax_l[m + k]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(&amax[b], __float_as_uint(v));
}

// ------------------------------------------------------------------ B operand blocks
// Stage block (g, m, pi, kb) of the filtered a_lm for maps G g .. G g + G - 1 (G maps per
// group, the plan's tunable): [hi tile, lo tile], each N = 2 P G rows (b, p, re/im) x TC_KB
// bytes of K (KPS values l = m + pi + 2 (kb KPS + k)), the same core-matrix layout the MMA
// reads.  Built once per chunk and shared by every ring tile.
struct PrepArgs {
    int L, P, B, G, n_groups;
    int64_t n_alm, total_bkb;      // stage blocks per map group
    const int64_t* bblk_base;      // [2 (L+1)] first stage block of (m, parity)
    const float* filt;             // [P][L+1]
    const float2* alm;             // [B][n_alm]
    const unsigned* amax;          // [B] float bits
    char* out;                     // [n_groups][total_bkb][2][N][128 bytes]
};

template <int PREC>
__global__ void __launch_bounds__(256) k_tc_prep_b(PrepArgs a) {
    using S = Split<PREC>;
    using T = typename ElemT<S::E>::T;
    constexpr int KPS = TC_KB / S::E;
    constexpr int CM = 16 / S::E;
    constexpr int NKC = TC_KB / 16;
    __shared__ float2 s_a[TC_MAX_MAPS * 32];
    __shared__ float s_f[64 * 16];
    __shared__ float s_scale[TC_MAX_MAPS];
    __shared__ int s_dec[16 * 16];                              // per column n: (map row of s_a, p, Re/Im)
    const int N = 2 * a.P * a.G;
    const int b_tile = N * TC_KB;
    const int m = blockIdx.y >> 1, pi = blockIdx.y & 1, g = blockIdx.z;
    const int nkb = tc_nkb(a.L, m, pi, KPS);
    const int64_t base_m = d_alm_index(m, m, a.L);
    if (threadIdx.x < a.G) {
        const int b = g * a.G + threadIdx.x;
        s_scale[threadIdx.x] = (b < a.B) ? exp2f((float)tc_scale_exp(a.amax[b])) : 0.f;
    }
    // column n = (map bl, p, Re/Im) = 2 (bl P + p) + comp, decoded once per CTA
    for (int n = threadIdx.x; n < N; n += blockDim.x)
        s_dec[n] = ((n / (2 * a.P)) * KPS) << 16 | ((n / 2) % a.P) << 1 | (n & 1);
    // this thread's first (chunk column, n) and its stride over c = kc N + n, divided once
    const int kc0 = threadIdx.x / N, n0 = threadIdx.x % N;
    const int dkc = blockDim.x / N, dn = blockDim.x % N;
    for (int kb = blockIdx.x; kb < nkb; kb += gridDim.x) {
        const int l0 = m + pi + 2 * kb * KPS;                   // l of K index k: l0 + 2 k
        __syncthreads();
        for (int i = threadIdx.x; i < a.G * KPS; i += blockDim.x) {
            const int bl = i / KPS, k = i % KPS;
            const int b = g * a.G + bl, l = l0 + 2 * k;
            float2 v = make_float2(0.f, 0.f);
            if (b < a.B && l <= a.L) {
                v = a.alm[(int64_t)b * a.n_alm + base_m + (l - m)];
                v.x *= s_scale[bl];
                v.y *= s_scale[bl];
            }
            s_a[i] = v;
        }
        for (int i = threadIdx.x; i < KPS * 16; i += blockDim.x) {
            const int k = i / 16, p = i % 16, l = l0 + 2 * k;
            s_f[i] = (p < a.P && l <= a.L) ? a.filt[(int64_t)p * (a.L + 1) + l] : 0.f;
        }
        __syncthreads();
        char* bt = a.out + ((int64_t)g * a.total_bkb + a.bblk_base[2 * m + pi] + kb) * (int64_t)(2 * b_tile);
        for (int kc = kc0, n = n0; kc < NKC;) {
            const int dec = s_dec[n];
            const int arow = dec >> 16, p = (dec >> 1) & 0x7fff, comp = dec & 1;
            T hv[CM], lv[CM];
#pragma unroll
            for (int i = 0; i < CM; ++i) {
                const int k = kc * CM + i;
                const float2 av = s_a[arow + k];
                const float x = s_f[k * 16 + p] * (comp ? av.y : av.x);
                S::split(x, hv[i], lv[i]);
            }
            const int off = (n >> 3) * TC_SBO + kc * 128 + (n & 7) * 16;
            *reinterpret_cast<uint4*>(bt + off) = *reinterpret_cast<const uint4*>(hv);
            *reinterpret_cast<uint4*>(bt + b_tile + off) = *reinterpret_cast<const uint4*>(lv);
            kc += dkc;
            n += dn;
            if (n >= N) {
                n -= N;
                ++kc;
            }
        }
    }
}

// ------------------------------------------------------------------ main kernel
// Four 16-column TMEM loads (D1 and D2 of two column blocks) and one wait; the waits
// carry the destination registers as operands, so no use of them is scheduled before
// the loads have landed.
#define TC_R16(o) "=r"(r[o + 0]), "=r"(r[o + 1]), "=r"(r[o + 2]), "=r"(r[o + 3]), "=r"(r[o + 4]), "=r"(r[o + 5]), \
    "=r"(r[o + 6]), "=r"(r[o + 7]), "=r"(r[o + 8]), "=r"(r[o + 9]), "=r"(r[o + 10]), "=r"(r[o + 11]),           \
    "=r"(r[o + 12]), "=r"(r[o + 13]), "=r"(r[o + 14]), "=r"(r[o + 15])
#define TC_W16(o) "+r"(r[o + 0]), "+r"(r[o + 1]), "+r"(r[o + 2]), "+r"(r[o + 3]), "+r"(r[o + 4]), "+r"(r[o + 5]), \
    "+r"(r[o + 6]), "+r"(r[o + 7]), "+r"(r[o + 8]), "+r"(r[o + 9]), "+r"(r[o + 10]), "+r"(r[o + 11]),           \
    "+r"(r[o + 12]), "+r"(r[o + 13]), "+r"(r[o + 14]), "+r"(r[o + 15])
#define TC_LD16 "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"

__device__ __forceinline__ void tmem_ld16x4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t (&r)[64]) {
    asm volatile(TC_LD16 : TC_R16(0) : "r"(a0));
    asm volatile(TC_LD16 : TC_R16(16) : "r"(a1));
    asm volatile(TC_LD16 : TC_R16(32) : "r"(a2));
    asm volatile(TC_LD16 : TC_R16(48) : "r"(a3));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : TC_W16(0), TC_W16(16) :: "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" : TC_W16(32), TC_W16(48) :: "memory");
}
#undef TC_R16
#undef TC_W16
#undef TC_LD16

struct TcArgs {
    int L, P, R, R_half, RH, n_rt, B, G, n_groups;
    int64_t n_items, total_bkb;
    const char* table;             // pre-tiled A blocks
    const int64_t* blk_base;       // [2 (L+1)] first A block of (m, parity)
    const char* bops;              // B stage blocks (k_tc_prep_b)
    const int64_t* bblk_base;      // [2 (L+1)] first B block of (m, parity)
    const unsigned* amax;          // [B] float bits
    float2* delta;                 // [B][P][L+1][2][RH]: E and O rows per ring pair
    int* err;
};

// item -> (m, pi, rt, g); consecutive items share the lambda tiles (same m, pi, rt).
__device__ __forceinline__ void tc_item(const TcArgs& a, int64_t item, int& m, int& pi, int& rt, int& g) {
    g = (int)(item % a.n_groups);
    int64_t t = item / a.n_groups;
    rt = (int)(t % a.n_rt);
    t /= a.n_rt;
    pi = (int)(t & 1);
    m = (int)(t >> 1);
}

template <int PREC>
__global__ void __launch_bounds__(TC_THREADS, 1) k_legendre_tc(TcArgs a) {
    using S = Split<PREC>;
    constexpr bool TF32 = (PREC == MODAL_3XTF32);
    constexpr int KPS = TC_KB / S::E;     // K values per stage
    constexpr int NKC = TC_KB / 16;       // core matrices along K per stage
    const int N = 2 * a.P * a.G;          // 2 (re, im) x P x G maps
    const int b_tile = N * TC_KB;         // bytes of one B tile
    const uint32_t stage_tx = TC_A_STAGE + 2 * b_tile;

    extern __shared__ __align__(1024) char smem[];
    char* sA = smem;                                        // [TC_STAGES][hi, lo]
    char* sB = sA + TC_STAGES * TC_A_STAGE;                 // [TC_STAGES][hi, lo][b_tile]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + TC_STAGES * 2 * 256 * TC_KB);
    uint64_t* full = bars;                                  // [TC_STAGES]
    uint64_t* empty = bars + TC_STAGES;                     // [TC_STAGES]
    uint64_t* tmem_full = bars + 2 * TC_STAGES;
    uint64_t* tmem_empty = tmem_full + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tmem_empty + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tmem_cols = (2 * N <= 256) ? 256u : 512u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tmem_full, 1);
        mbar_init(tmem_empty, TC_PROD_WARPS);
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

    if (warp == 0) {
        // ---------------- loader (one thread): A and B stage blocks by cp.async.bulk
        if (lane == 0) {
            uint32_t it = 0;
            uint32_t last_phase[TC_STAGES] = {};
            bool issued[TC_STAGES] = {};
            for (int64_t item = blockIdx.x; item < a.n_items && !*abort_flag; item += gridDim.x) {
                int m, pi, rt, g;
                tc_item(a, item, m, pi, rt, g);
                const int nkb = tc_nkb(a.L, m, pi, KPS);
                const char* srcA = a.table + (a.blk_base[2 * m + pi] + (int64_t)rt * nkb) * TC_A_STAGE;
                const char* srcB = a.bops + ((int64_t)g * a.total_bkb + a.bblk_base[2 * m + pi]) * (int64_t)(2 * b_tile);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % TC_STAGES;
                    const uint32_t ph = (it / TC_STAGES) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, a.err)) break;
                    mbar_arrive_expect_tx(&full[s], stage_tx);
                    bulk_copy_g2s(sA + s * TC_A_STAGE, srcA + (int64_t)kb * TC_A_STAGE, TC_A_STAGE, &full[s]);
                    bulk_copy_g2s(sB + s * 2 * b_tile, srcB + (int64_t)kb * 2 * b_tile, 2 * b_tile, &full[s]);
                    last_phase[s] = ph;
                    issued[s] = true;
                }
            }
            // copies still in flight complete before the CTA exits
            for (int s = 0; s < TC_STAGES; ++s) {
                if (!issued[s]) continue;
                const long long t0 = clock64();
                while (!mbar_try_wait(&full[s], last_phase[s]) && clock64() - t0 < TC_WAIT_CYCLES) {
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (one thread)
        if (lane == 0) {
            const uint32_t idesc = umma_idesc(S::FMT, N);
            const uint32_t d1 = tmem, d2 = tmem + (uint32_t)N;
            uint32_t it = 0, nitem = 0;
            for (int64_t item = blockIdx.x; item < a.n_items && !*abort_flag; item += gridDim.x, ++nitem) {
                int m, pi, rt, g;
                tc_item(a, item, m, pi, rt, g);
                const int nkb = tc_nkb(a.L, m, pi, KPS);
                if (!mbar_wait(tmem_empty, (nitem & 1) ^ 1, abort_flag, a.err)) break;
                tc_fence_after();
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % TC_STAGES;
                    const uint32_t ph = (it / TC_STAGES) & 1;
                    if (!mbar_wait(&full[s], ph, abort_flag, a.err)) break;
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + s * TC_A_STAGE);
                    const uint32_t b0 = smem_u32(sB + s * 2 * b_tile);
#pragma unroll
                    for (int ks = 0; ks < NKC / 2; ++ks) {
                        const uint32_t koff = ks * 2 * 128;          // 2 core matrices (32 B of K) per MMA
                        const uint64_t ah = umma_desc(a0 + koff);
                        const uint64_t al = umma_desc(a0 + TC_A_TILE + koff);
                        const uint64_t bh = umma_desc(b0 + koff);
                        const uint64_t bl = umma_desc(b0 + b_tile + koff);
                        const uint32_t first = (kb == 0 && ks == 0) ? 0u : 1u;
                        umma<TF32>(d1, ah, bh, idesc, first);
                        if (S::PRODUCTS == 3) {
                            umma<TF32>(d2, ah, bl, idesc, first);
                            umma<TF32>(d2, al, bh, idesc, 1u);
                        }
                    }
                    umma_commit(&empty[s]);
                }
                umma_commit(tmem_full);
            }
        }
    } else {
        // ---------------- epilogue (TC_PROD_WARPS warps): TMEM -> D1 + D2 -> E or O row
        // Columns are ordered (map bl, basis p, re/im); column pair cp = bl P + p maps to
        // the delta row (G g P + cp) (L+1) 2 RH + (2 m + pi) RH, so addresses advance by a
        // fixed stride per column pair.
        const int quarter = warp % 4;                       // TMEM lanes 32 quarter .. + 31
        const int half = (warp - 2) / 4;                    // column half
        const int nblk = N / 16;                            // 16-column blocks
        const int blk_lo = half ? (nblk + 1) / 2 : 0, blk_hi = half ? nblk : (nblk + 1) / 2;
        const int64_t row_stride = (int64_t)(a.L + 1) * 2 * a.RH;
        const float lam_inv = (S::E == 2) ? (1.f / TC_LAMBDA_SCALE) : 1.f;
        uint32_t nitem = 0;
        for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x, ++nitem) {
            int m, pi, rt, g;
            tc_item(a, item, m, pi, rt, g);
            // per-map unscale factors of this map group (lane bl holds map G g + bl)
            float inv_lane = 0.f;
            if (lane < a.G && g * a.G + lane < a.B)
                inv_lane = exp2f((float)-tc_scale_exp(a.amax[g * a.G + lane])) * lam_inv;
            bool ok = !*abort_flag && mbar_wait(tmem_full, nitem & 1, abort_flag, a.err);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {                                       // items left undone: never silent
                if (lane == 0) atomicOr(a.err, MODAL_DEVERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            const int jn = rt * 128 + quarter * 32 + lane;   // TMEM lane = ring pair within the tile
            const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
            const int cp_valid = (a.B - g * a.G) * a.P;       // column pairs that belong to real maps
            float2* base = a.delta + ((int64_t)g * a.G * a.P) * row_stride + (int64_t)(2 * m + pi) * a.RH + jn;
            auto store_block = [&](int blk, const float* d) {
                const int cp0 = blk * 8;
                int bl = cp0 / a.P, p = cp0 - bl * a.P;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float inv = __shfl_sync(0xffffffffu, inv_lane, bl);
                    if (jn < a.R_half && cp0 + q < cp_valid)
                        base[(int64_t)(cp0 + q) * row_stride] = make_float2(d[2 * q] * inv, d[2 * q + 1] * inv);
                    if (++p == a.P) { p = 0; ++bl; }
                }
            };
            auto release = [&]() {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tmem_empty);
            };
            if (S::PRODUCTS == 3) {
                // pairs of column blocks; TMEM is released as soon as the last pair is read
                if (blk_hi <= blk_lo) release();
                for (int blk = blk_lo; blk < blk_hi; blk += 2) {
                    const bool two = blk + 1 < blk_hi;             // warp-uniform
                    const uint32_t c0 = lane_addr + blk * 16, c1 = lane_addr + (two ? blk + 1 : blk) * 16;
                    uint32_t r[64];
                    tmem_ld16x4(c0, c0 + N, c1, c1 + N, r);
                    float d0[16], d1[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        d0[i] = __uint_as_float(r[i]) + __uint_as_float(r[16 + i]);
                        d1[i] = __uint_as_float(r[32 + i]) + __uint_as_float(r[48 + i]);
                    }
                    if (blk + 2 >= blk_hi) release();
                    store_block(blk, d0);
                    if (two) store_block(blk + 1, d1);
                }
            } else {
                for (int blk = blk_lo; blk < blk_hi; ++blk) {
                    float d[16];
                    tmem_ld16(lane_addr + blk * 16, d);
                    store_block(blk, d);
                }
                release();
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

static size_t tc_smem_bytes() {
    return 1024 /*alignment slack*/ + TC_STAGES * TC_A_STAGE + TC_STAGES * 2 * 256 * TC_KB +
           8 * (2 * TC_STAGES + 2) + 16;
}

// ------------------------------------------------------------------ host side
static int kps_for(int prec) { return prec == MODAL_3XTF32 ? TC_KB / 4 : TC_KB / 2; }

size_t tc_b_workspace_bytes(const Plan& pl, int chunk) {
    if (pl.prec == MODAL_FP32) return 0;
    const int KPS = kps_for(pl.prec);
    int64_t total = 0;
    for (int m = 0; m <= pl.lmax; ++m)
        for (int pi = 0; pi < 2; ++pi) total += tc_nkb(pl.lmax, m, pi, KPS);
    const int groups = (chunk + pl.tc_maps - 1) / pl.tc_maps;
    return (size_t)groups * total * 2 * (2 * pl.P * pl.tc_maps) * TC_KB;
}

bool tc_maps_valid(int P, int G) {
    const int n = 2 * P * G;
    return G >= 1 && G <= TC_MAX_MAPS && n % 16 == 0 && n <= 256;
}

size_t tc_table_bytes(const Plan& pl) {
    if (pl.prec == MODAL_FP32) return 0;
    const int KPS = kps_for(pl.prec);
    const int64_t n_rt = (pl.R_half + 127) / 128;
    int64_t total = 0;
    for (int m = 0; m <= pl.lmax; ++m)
        for (int pi = 0; pi < 2; ++pi) total += n_rt * tc_nkb(pl.lmax, m, pi, KPS);
    return (size_t)total * TC_A_STAGE;
}

cudaError_t build_tc_tables(Plan& pl, cudaStream_t st) {
    const int L = pl.lmax;
    const int KPS = kps_for(pl.prec);
    pl.tc.n_rt = (pl.R_half + 127) / 128;
    pl.tc.kb_off.assign(2 * (L + 1), 0);
    std::vector<int64_t> bb(2 * (L + 1), 0);
    int64_t total = 0, btotal = 0;
    for (int m = 0; m <= L; ++m)
        for (int pi = 0; pi < 2; ++pi) {
            pl.tc.kb_off[2 * m + pi] = total;
            bb[2 * m + pi] = btotal;
            const int nkb = tc_nkb(L, m, pi, KPS);
            total += (int64_t)pl.tc.n_rt * nkb;
            btotal += nkb;
        }
    pl.tc.n_kb = total;
    pl.tc.total_bkb = btotal;
    pl.tc.bytes = (size_t)total * TC_A_STAGE;
    cudaError_t e = cudaMalloc(&pl.tc.hi, pl.tc.bytes);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&pl.tc.d_kb_off, 2 * (L + 1) * sizeof(int64_t));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&pl.tc.d_bkb_off, 2 * (L + 1) * sizeof(int64_t));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&pl.tc.d_amax, 4096 * sizeof(unsigned));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&pl.tc.d_fmax, (L + 1) * sizeof(float));
    if (e != cudaSuccess) return e;
    pl.device_bytes += pl.tc.bytes + (L + 1) * (4 * sizeof(int64_t) + sizeof(float)) + 4096 * sizeof(unsigned);
    e = cudaMemcpy(pl.tc.d_kb_off, pl.tc.kb_off.data(), 2 * (L + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(pl.tc.d_bkb_off, bb.data(), 2 * (L + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    {
        std::vector<float> fm(L + 1, 0.f);
        for (int l = 0; l <= L; ++l) {
            if (pl.cl[l] <= 0) continue;
            for (int p = 0; p < pl.P; ++p)
                fm[l] = std::max(fm[l], (float)std::fabs(pl.basis[(size_t)p * (L + 1) + l] / std::sqrt(pl.cl[l])));
        }
        e = cudaMemcpy(pl.tc.d_fmax, fm.data(), (L + 1) * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(std::min(pl.tc.n_rt * 64, 1024), 2 * (L + 1));
    switch (pl.prec) {
        case MODAL_FP16X3:
            k_build_tc_table<MODAL_FP16X3><<<grid, 256, 0, st>>>(L, pl.R_half, pl.RH, pl.tc.n_rt, pl.lam, pl.tc.d_kb_off, pl.tc.hi);
            break;
        case MODAL_BF16X3:
            k_build_tc_table<MODAL_BF16X3><<<grid, 256, 0, st>>>(L, pl.R_half, pl.RH, pl.tc.n_rt, pl.lam, pl.tc.d_kb_off, pl.tc.hi);
            break;
        case MODAL_BF16:
            k_build_tc_table<MODAL_BF16><<<grid, 256, 0, st>>>(L, pl.R_half, pl.RH, pl.tc.n_rt, pl.lam, pl.tc.d_kb_off, pl.tc.hi);
            break;
        case MODAL_3XTF32:
            k_build_tc_table<MODAL_3XTF32><<<grid, 256, 0, st>>>(L, pl.R_half, pl.RH, pl.tc.n_rt, pl.lam, pl.tc.d_kb_off, pl.tc.hi);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

void free_tc_tables(Plan& pl) {
    if (pl.tc.hi) cudaFree(pl.tc.hi);
    if (pl.tc.d_kb_off) cudaFree(pl.tc.d_kb_off);
    if (pl.tc.d_bkb_off) cudaFree(pl.tc.d_bkb_off);
    if (pl.tc.d_amax) cudaFree(pl.tc.d_amax);
    if (pl.tc.d_fmax) cudaFree(pl.tc.d_fmax);
    pl.tc = TcTable();
}

template <int PREC>
static cudaError_t launch_tc(const Plan& pl, const PrepArgs& pa, const TcArgs& args, int part, cudaStream_t st) {
    if (part & 1) {
        const int maxkb = tc_nkb(pl.lmax, 0, 0, kps_for(pl.prec));
        dim3 grid(std::min(maxkb, 8), 2 * (pl.lmax + 1), pa.n_groups);
        k_tc_prep_b<PREC><<<grid, 256, 0, st>>>(pa);
        note_launch(pl);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (!(part & 2)) return cudaSuccess;
    const size_t smem = tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_legendre_tc<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, pl.dev);
    const int grid = (int)std::min<int64_t>(args.n_items, (int64_t)std::max(nsm, 1));
    k_legendre_tc<PREC><<<grid, TC_THREADS, smem, st>>>(args);
    note_launch(pl);
    return cudaGetLastError();
}

cudaError_t launch_legendre_tc(const Plan& pl, const float2* alm, int B, float2* delta, int part, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    if (B > 4096 || B > pl.chunk || !tc_maps_valid(pl.P, pl.tc_maps)) return cudaErrorInvalidValue;
    if (part & 1) {
        cudaError_t e = cudaMemsetAsync(pl.tc.d_amax, 0, B * sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        k_alm_amax<<<dim3(AM_BLOCKS, B), 256, 0, st>>>(pl.lmax, pl.tc.d_fmax, alm, pl.n_alm, pl.tc.d_amax);
        note_launch(pl);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    PrepArgs pa;
    pa.L = pl.lmax;
    pa.P = pl.P;
    pa.B = B;
    pa.G = pl.tc_maps;
    pa.n_groups = (B + pa.G - 1) / pa.G;
    pa.n_alm = pl.n_alm;
    pa.total_bkb = pl.tc.total_bkb;
    pa.bblk_base = pl.tc.d_bkb_off;
    pa.filt = pl.filt;
    pa.alm = alm;
    pa.amax = pl.tc.d_amax;
    pa.out = static_cast<char*>(pl.tc.bops);
    TcArgs a;
    a.L = pl.lmax;
    a.P = pl.P;
    a.R = pl.nrings;
    a.R_half = pl.R_half;
    a.RH = pl.RH;
    a.n_rt = pl.tc.n_rt;
    a.B = B;
    a.G = pa.G;
    a.n_groups = pa.n_groups;
    a.n_items = (int64_t)(pl.lmax + 1) * 2 * a.n_rt * a.n_groups;
    a.total_bkb = pl.tc.total_bkb;
    a.table = static_cast<const char*>(pl.tc.hi);
    a.blk_base = pl.tc.d_kb_off;
    a.bops = static_cast<const char*>(pl.tc.bops);
    a.bblk_base = pl.tc.d_bkb_off;
    a.amax = pl.tc.d_amax;
    a.delta = delta;
    a.err = pl.d_err;
    switch (pl.prec) {
        case MODAL_FP16X3: return launch_tc<MODAL_FP16X3>(pl, pa, a, part, st);
        case MODAL_BF16X3: return launch_tc<MODAL_BF16X3>(pl, pa, a, part, st);
        case MODAL_BF16: return launch_tc<MODAL_BF16>(pl, pa, a, part, st);
        case MODAL_3XTF32: return launch_tc<MODAL_3XTF32>(pl, pa, a, part, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace modal
