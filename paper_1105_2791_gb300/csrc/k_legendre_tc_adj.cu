// Tensor-core (tcgen05, sm_103a) transposed Legendre sums for the adjoint.
//
// For order m and parity pi the adjoint needs, per map b and basis function t,
//     G_{b,t}(l) = sum_j lambda_lm(theta_j) U^pi_{b,t,m}(j),   l = m + pi (mod 2),
// where U^0 = U~_north + U~_south and U^1 = U~_north - U~_south are the ring-pair
// Fourier coefficients from the r2c transform, and then
//     grad_{b,lm} = c_m sum_t f_t(l) G_{b,t}(l),   c_0 = 1, c_m = 2.
// This is a GEMM with M = 128 values of l (one parity), K = ring pairs j, N = 16 P
// columns (8 maps x P basis functions x re/im).  Work item = (m, pi, l tile, map
// group).  The kernel mirrors k_legendre_tc: lambda^T tiles (a second pre-split,
// pre-tiled table) and the scaled, split U operand blocks (built by k_tc_prep_adj)
// arrive by cp.async.bulk; one thread issues tcgen05.mma into TMEM (hi*hi in D1,
// cross terms in D2); four warps read TMEM, form D1 + D2, contract the P columns of
// each map with f_t(l), undo the scaling and store the gradient.  Waits are bounded
// as in the forward kernel.
#include "modal_internal.cuh"

#include "tc_common.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace modal {

constexpr int TA_EPI_WARPS = 4;
constexpr int TA_THREADS = 32 * (2 + 2 * TA_EPI_WARPS);   // same shape as the forward kernel
// bytes after the operand stages: 2 TC_STAGES + 2 mbarriers, the TMEM slot and the abort
// flag, rounded up to 16; the epilogue's filter table follows
constexpr int TA_BAR_BYTES = ((8 * (2 * TC_STAGES + 2) + 8 + 15) / 16) * 16;

__host__ __device__ inline int ta_kpar(int L, int m, int pi) {
    return (L - m - pi >= 0) ? (L - m - pi) / 2 + 1 : 0;       // values of l with this parity
}
__host__ __device__ inline int ta_nlt(int L, int m, int pi) {
    const int k = ta_kpar(L, m, pi);
    return k > 0 ? (k + 127) / 128 : 1;
}

// ------------------------------------------------------------------ transposed table
// Stage block (m, pi, lt, kb) = [hi, lo] tiles of 128 values of l (l = m + pi + 2 (128 lt + r))
// x KPS ring pairs (j = kb KPS + k), lambda scaled by 2^11 for 16-bit formats.
template <int PREC>
__global__ void k_build_tc_adj_table(int L, int R_half, int RH, int nkb, const float* __restrict__ lam,
                                     const int64_t* __restrict__ blk_base, void* __restrict__ out) {
    using S = Split<PREC>;
    using T = typename ElemT<S::E>::T;
    constexpr int KPS = TC_KB / S::E;
    constexpr int CM = 16 / S::E;
    const int m = blockIdx.y >> 1, pi = blockIdx.y & 1;
    const int nlt = ta_nlt(L, m, pi);
    const int64_t base_m = d_alm_index(m, m, L);
    const float scale = (S::E == 2) ? TC_LAMBDA_SCALE : 1.f;
    for (int64_t blk = blockIdx.x; blk < (int64_t)nlt * nkb; blk += gridDim.x) {
        const int lt = (int)(blk / nkb), kb = (int)(blk % nkb);
        char* dst = reinterpret_cast<char*>(out) + (blk_base[2 * m + pi] + blk) * TC_A_STAGE;
        for (int e = threadIdx.x; e < 128 * KPS; e += blockDim.x) {
            const int r = e / KPS, k = e % KPS;
            const int l = m + pi + 2 * (lt * 128 + r);
            const int j = kb * KPS + k;
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

// ------------------------------------------------------------------ operand preparation
// amax[b] = max |U| over the valid ring pairs of map b (float bits).
__global__ void k_ut_amax(int L, int P, int R_half, int RH, const float2* __restrict__ ut, unsigned* __restrict__ amax) {
    const int b = blockIdx.y;
    const int64_t rows = (int64_t)P * (L + 1) * 2;
    float v = 0.f;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const float2* u = ut + ((int64_t)b * rows + row) * RH;
        for (int j = threadIdx.x; j < R_half; j += blockDim.x) v = fmaxf(v, fmaxf(fabsf(u[j].x), fabsf(u[j].y)));
    }
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(&amax[b], __float_as_uint(v));
}

struct AdjPrepArgs {
    int L, P, R_half, RH, B, nkb;
    const float2* ut;              // [B][P][L+1][2][RH]
    const unsigned* amax;
    char* out;                     // [(g (L+1) + m) 2 + pi][kb][2][N][128 bytes]
};

// B block (g, m, pi, kb): rows n = (bl, t, re/im), K = ring pairs j = kb KPS + k.
// A thread takes one (bl, t) and one core-matrix column kc: it reads the CM values of
// U~ there as 16-byte vectors and writes the hi and lo parts of both the Re row (n = 2q)
// and the Im row (n = 2q + 1) (one 32-byte sector per part).  Consecutive threads take
// consecutive kc of one row, so a row's KPS values are read as one contiguous run.
template <int PREC>
__global__ void __launch_bounds__(256) k_tc_prep_adj(AdjPrepArgs a) {
    using S = Split<PREC>;
    using T = typename ElemT<S::E>::T;
    constexpr int KPS = TC_KB / S::E;
    constexpr int CM = 16 / S::E;
    constexpr int NKC = TC_KB / 16;
    static_assert(CM % 2 == 0, "CM values of U~ are read as float4 pairs");
    __shared__ float s_scale[TC_MAPS];
    const int N = 16 * a.P;
    const int NQ = N / 2;                                  // (bl, t) rows
    const int b_tile = N * TC_KB;
    const int m = blockIdx.y >> 1, pi = blockIdx.y & 1, g = blockIdx.z;
    if (threadIdx.x < TC_MAPS) {
        const int b = g * TC_MAPS + threadIdx.x;
        s_scale[threadIdx.x] = (b < a.B) ? exp2f((float)tc_scale_exp(a.amax[b])) : 0.f;
    }
    __syncthreads();
    for (int kb = blockIdx.x; kb < a.nkb; kb += gridDim.x) {
        char* bt = a.out + ((((int64_t)g * (a.L + 1) + m) * 2 + pi) * a.nkb + kb) * (int64_t)(2 * b_tile);
        for (int c = threadIdx.x; c < NKC * NQ; c += blockDim.x) {
            const int kc = c % NKC, q = c / NKC;           // the NKC threads of a row read it contiguously
            const int bl = q / a.P, t = q % a.P;
            const int b = g * TC_MAPS + bl;
            const float sc = s_scale[bl];
            const int j0 = kb * KPS + kc * CM;
            float re[CM], im[CM];
            if (b < a.B && j0 + CM <= a.R_half) {
                // whole core-matrix row inside the ring range: 16-byte loads (RH is a multiple of 32)
                const float4* u4 = reinterpret_cast<const float4*>(
                    a.ut + ((((int64_t)(b * a.P + t)) * (a.L + 1) + m) * 2 + pi) * a.RH + j0);
#pragma unroll
                for (int i = 0; i < CM / 2; ++i) {
                    const float4 v = u4[i];
                    re[2 * i] = v.x * sc;
                    im[2 * i] = v.y * sc;
                    re[2 * i + 1] = v.z * sc;
                    im[2 * i + 1] = v.w * sc;
                }
            } else {
                const float2* u = a.ut + ((((int64_t)(b * a.P + t)) * (a.L + 1) + m) * 2 + pi) * a.RH;
#pragma unroll
                for (int i = 0; i < CM; ++i) {
                    const int j = j0 + i;
                    float2 v = make_float2(0.f, 0.f);
                    if (b < a.B && j < a.R_half) v = u[j];
                    re[i] = v.x * sc;
                    im[i] = v.y * sc;
                }
            }
            T hr[CM], lr[CM], hm[CM], lm[CM];
#pragma unroll
            for (int i = 0; i < CM; ++i) {
                S::split(re[i], hr[i], lr[i]);
                S::split(im[i], hm[i], lm[i]);
            }
            const int n = 2 * q;                             // Re row; the Im row n + 1 is 16 bytes on
            const int off = (n / 8) * TC_SBO + kc * 128 + (n % 8) * 16;
            *reinterpret_cast<uint4*>(bt + off) = *reinterpret_cast<const uint4*>(hr);
            *reinterpret_cast<uint4*>(bt + off + 16) = *reinterpret_cast<const uint4*>(hm);
            *reinterpret_cast<uint4*>(bt + b_tile + off) = *reinterpret_cast<const uint4*>(lr);
            *reinterpret_cast<uint4*>(bt + b_tile + off + 16) = *reinterpret_cast<const uint4*>(lm);
        }
    }
}

// ------------------------------------------------------------------ main kernel
struct AdjArgs {
    int L, P, B, n_groups, nkb;
    int64_t n_items, n_alm;
    const int64_t* item_base;      // [2 (L+1) + 1] prefix sums of l tiles over (m, pi)
    const char* table;             // transposed lambda blocks
    const int64_t* blk_base;       // [2 (L+1)] first block of (m, pi)
    const char* bops;              // U operand blocks
    const float* filt;             // [P][L+1]
    const unsigned* amax;          // [B]
    float2* grad;                  // [B][n_alm]
    int* err;
};

// item -> (m, pi, lt, g): items of one (m, pi, lt) are consecutive (they share lambda tiles).
__device__ __forceinline__ void ta_item(const AdjArgs& a, int64_t item, int& m, int& pi, int& lt, int& g) {
    g = (int)(item % a.n_groups);
    const int64_t t = item / a.n_groups;
    int lo = 0, hi = 2 * (a.L + 1) - 1;                    // largest mp with item_base[mp] <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.item_base[mid] <= t) lo = mid; else hi = mid - 1;
    }
    m = lo >> 1;
    pi = lo & 1;
    lt = (int)(t - a.item_base[lo]);
}

template <int PREC>
__global__ void __launch_bounds__(TA_THREADS, 1) k_legendre_tc_adj(AdjArgs a) {
    using S = Split<PREC>;
    constexpr bool TF32 = (PREC == MODAL_3XTF32);
    constexpr int NKC = TC_KB / 16;
    const int N = 16 * a.P;
    const int b_tile = N * TC_KB;
    const uint32_t stage_tx = TC_A_STAGE + 2 * b_tile;

    extern __shared__ __align__(1024) char smem[];
    char* sA = smem;
    char* sB = sA + TC_STAGES * TC_A_STAGE;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + TC_STAGES * 2 * 256 * TC_KB);
    uint64_t* full = bars;
    uint64_t* empty = bars + TC_STAGES;
    uint64_t* tmem_full = bars + 2 * TC_STAGES;
    uint64_t* tmem_empty = tmem_full + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tmem_empty + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* sF = reinterpret_cast<float*>(smem + TC_STAGES * TC_A_STAGE + TC_STAGES * 2 * 256 * TC_KB +
                                         TA_BAR_BYTES);                                              // [128][17]

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tmem_cols = (2 * N <= 256) ? 256u : 512u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tmem_full, 1);
        mbar_init(tmem_empty, TA_EPI_WARPS);
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
        if (lane == 0) {
            uint32_t it = 0;
            uint32_t last_phase[TC_STAGES] = {};
            bool issued[TC_STAGES] = {};
            for (int64_t item = blockIdx.x; item < a.n_items && !*abort_flag; item += gridDim.x) {
                int m, pi, lt, g;
                ta_item(a, item, m, pi, lt, g);
                const char* srcA = a.table + (a.blk_base[2 * m + pi] + (int64_t)lt * a.nkb) * TC_A_STAGE;
                const char* srcB = a.bops + (((int64_t)g * (a.L + 1) + m) * 2 + pi) * a.nkb * (int64_t)(2 * b_tile);
                for (int kb = 0; kb < a.nkb; ++kb, ++it) {
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
            for (int s = 0; s < TC_STAGES; ++s) {
                if (!issued[s]) continue;
                const long long t0 = clock64();
                while (!mbar_try_wait(&full[s], last_phase[s]) && clock64() - t0 < TC_WAIT_CYCLES) {
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = umma_idesc(S::FMT, N);
            const uint32_t d1 = tmem, d2 = tmem + (uint32_t)N;
            uint32_t it = 0, nitem = 0;
            for (int64_t item = blockIdx.x; item < a.n_items && !*abort_flag; item += gridDim.x, ++nitem) {
                if (!mbar_wait(tmem_empty, (nitem & 1) ^ 1, abort_flag, a.err)) break;
                tc_fence_after();
                for (int kb = 0; kb < a.nkb; ++kb, ++it) {
                    const int s = it % TC_STAGES;
                    const uint32_t ph = (it / TC_STAGES) & 1;
                    if (!mbar_wait(&full[s], ph, abort_flag, a.err)) break;
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + s * TC_A_STAGE);
                    const uint32_t b0 = smem_u32(sB + s * 2 * b_tile);
#pragma unroll
                    for (int ks = 0; ks < NKC / 2; ++ks) {
                        const uint32_t koff = ks * 2 * 128;
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
    } else if (warp < 2 + TA_EPI_WARPS) {
        // ---------------- epilogue: lane = one l; reduce each map's P columns with f_t(l)
        const int quarter = warp % 4;
        const float lam_inv = (S::E == 2) ? (1.f / TC_LAMBDA_SCALE) : 1.f;
        uint32_t nitem = 0;
        for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x, ++nitem) {
            int m, pi, lt, g;
            ta_item(a, item, m, pi, lt, g);
            const int l = m + pi + 2 * (lt * 128 + quarter * 32 + lane);
            float inv_lane = 0.f;
            if (lane < TC_MAPS && g * TC_MAPS + lane < a.B)
                inv_lane = exp2f((float)-tc_scale_exp(a.amax[g * TC_MAPS + lane])) * lam_inv;
            float* my_f = sF + (threadIdx.x - 64) * 17;      // this lane's f_t(l), t < P
            for (int t = 0; t < a.P; ++t) my_f[t] = (l <= a.L) ? a.filt[(int64_t)t * (a.L + 1) + l] : 0.f;
            bool ok = !*abort_flag && mbar_wait(tmem_full, nitem & 1, abort_flag, a.err);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {                                       // items left undone: never silent
                if (lane == 0) atomicOr(a.err, MODAL_DEVERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
            float acc_re = 0.f, acc_im = 0.f;
            int bl = 0, t = 0;
            for (int blk = 0; blk < a.P; ++blk) {                // N = 16 P columns in blocks of 16
                float d[16], d2[16];
                tmem_ld16(lane_addr + blk * 16, d);
                if (S::PRODUCTS == 3) {
                    tmem_ld16(lane_addr + N + blk * 16, d2);
#pragma unroll
                    for (int i = 0; i < 16; ++i) d[i] += d2[i];
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float ft = my_f[t];
                    acc_re = fmaf(ft, d[2 * q], acc_re);
                    acc_im = fmaf(ft, d[2 * q + 1], acc_im);
                    if (++t == a.P) {
                        // map bl complete
                        const float inv = __shfl_sync(0xffffffffu, inv_lane, bl);
                        const int b = g * TC_MAPS + bl;
                        if (l <= a.L && b < a.B) {
                            const float cm = (m == 0) ? 1.f : 2.f;
                            a.grad[(int64_t)b * a.n_alm + d_alm_index(l, m, a.L)] =
                                make_float2(cm * acc_re * inv, (m == 0) ? 0.f : cm * acc_im * inv);
                        }
                        acc_re = acc_im = 0.f;
                        t = 0;
                        ++bl;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tmem_empty);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
    }
}

static size_t ta_smem_bytes() {
    return 1024 + TC_STAGES * TC_A_STAGE + TC_STAGES * 2 * 256 * TC_KB + TA_BAR_BYTES + 128 * 17 * sizeof(float);
}

static int ta_kps(int prec) { return prec == MODAL_3XTF32 ? TC_KB / 4 : TC_KB / 2; }

size_t tc_adj_workspace_bytes(const Plan& pl, int chunk) {
    if (pl.prec == MODAL_FP32) return 0;
    const int nkb = (pl.R_half + ta_kps(pl.prec) - 1) / ta_kps(pl.prec);
    const int groups = (chunk + TC_MAPS - 1) / TC_MAPS;
    return (size_t)groups * (pl.lmax + 1) * 2 * nkb * 2 * (16 * pl.P) * TC_KB;
}

size_t tc_adj_table_bytes(const Plan& pl) {
    if (pl.prec == MODAL_FP32) return 0;
    const int L = pl.lmax;
    const int64_t nkb = (pl.R_half + ta_kps(pl.prec) - 1) / ta_kps(pl.prec);
    int64_t total = 0;
    for (int m = 0; m <= L; ++m)
        for (int pi = 0; pi < 2; ++pi) total += (int64_t)ta_nlt(L, m, pi) * nkb;
    return (size_t)total * TC_A_STAGE;
}

cudaError_t build_tc_adj_tables(Plan& pl, cudaStream_t st) {
    const int L = pl.lmax;
    const int KPS = ta_kps(pl.prec);
    const int nkb = (pl.R_half + KPS - 1) / KPS;
    std::vector<int64_t> base(2 * (L + 1)), ibase(2 * (L + 1) + 1);
    int64_t total = 0, items = 0;
    for (int m = 0; m <= L; ++m)
        for (int pi = 0; pi < 2; ++pi) {
            base[2 * m + pi] = total;
            ibase[2 * m + pi] = items;
            total += (int64_t)ta_nlt(L, m, pi) * nkb;
            items += ta_nlt(L, m, pi);
        }
    ibase[2 * (L + 1)] = items;
    pl.tca.nkb = nkb;
    pl.tca.n_lt_total = items;
    pl.tca.bytes = (size_t)total * TC_A_STAGE;
    cudaError_t e = cudaMalloc(&pl.tca.table, pl.tca.bytes);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&pl.tca.d_blk_base, base.size() * sizeof(int64_t));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&pl.tca.d_item_base, ibase.size() * sizeof(int64_t));
    if (e != cudaSuccess) return e;
    pl.device_bytes += pl.tca.bytes + (base.size() + ibase.size()) * sizeof(int64_t);
    e = cudaMemcpy(pl.tca.d_blk_base, base.data(), base.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(pl.tca.d_item_base, ibase.data(), ibase.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    dim3 grid(std::min(nkb * 16, 1024), 2 * (L + 1));
    switch (pl.prec) {
        case MODAL_FP16X3:
            k_build_tc_adj_table<MODAL_FP16X3><<<grid, 256, 0, st>>>(L, pl.R_half, pl.RH, nkb, pl.lam, pl.tca.d_blk_base, pl.tca.table);
            break;
        case MODAL_BF16X3:
            k_build_tc_adj_table<MODAL_BF16X3><<<grid, 256, 0, st>>>(L, pl.R_half, pl.RH, nkb, pl.lam, pl.tca.d_blk_base, pl.tca.table);
            break;
        case MODAL_BF16:
            k_build_tc_adj_table<MODAL_BF16><<<grid, 256, 0, st>>>(L, pl.R_half, pl.RH, nkb, pl.lam, pl.tca.d_blk_base, pl.tca.table);
            break;
        case MODAL_3XTF32:
            k_build_tc_adj_table<MODAL_3XTF32><<<grid, 256, 0, st>>>(L, pl.R_half, pl.RH, nkb, pl.lam, pl.tca.d_blk_base, pl.tca.table);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

void free_tc_adj_tables(Plan& pl) {
    if (pl.tca.table) cudaFree(pl.tca.table);
    if (pl.tca.d_blk_base) cudaFree(pl.tca.d_blk_base);
    if (pl.tca.d_item_base) cudaFree(pl.tca.d_item_base);
    pl.tca = TcAdjTable();
}

template <int PREC>
static cudaError_t launch_adj(const Plan& pl, const AdjPrepArgs& pa, const AdjArgs& a, int part, cudaStream_t st) {
    cudaError_t e;
    if (part & 1) {
        dim3 pgrid(std::min(pa.nkb, 8), 2 * (pl.lmax + 1), a.n_groups);
        k_tc_prep_adj<PREC><<<pgrid, 256, 0, st>>>(pa);
        note_launch(pl);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (!(part & 2)) return cudaSuccess;
    const size_t smem = ta_smem_bytes();
    e = cudaFuncSetAttribute(k_legendre_tc_adj<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, pl.dev);
    const int grid = (int)std::min<int64_t>(a.n_items, (int64_t)std::max(nsm, 1));
    k_legendre_tc_adj<PREC><<<grid, TA_THREADS, smem, st>>>(a);
    note_launch(pl);
    return cudaGetLastError();
}

cudaError_t launch_legendre_adjoint_tc(const Plan& pl, const float2* ut, int B, float2* grad, bool amax_ready,
                                       int part, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    if (B > 4096 || B > pl.chunk) return cudaErrorInvalidValue;
    if (!amax_ready && (part & 1)) {
        cudaError_t e = cudaMemsetAsync(pl.tc.d_amax, 0, B * sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        k_ut_amax<<<dim3(256, B), 256, 0, st>>>(pl.lmax, pl.P, pl.R_half, pl.RH, ut, pl.tc.d_amax);
        note_launch(pl);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    AdjPrepArgs pa;
    pa.L = pl.lmax;
    pa.P = pl.P;
    pa.R_half = pl.R_half;
    pa.RH = pl.RH;
    pa.B = B;
    pa.nkb = pl.tca.nkb;
    pa.ut = ut;
    pa.amax = pl.tc.d_amax;
    pa.out = static_cast<char*>(pl.tca.bops);
    AdjArgs a;
    a.L = pl.lmax;
    a.P = pl.P;
    a.B = B;
    a.n_groups = (B + TC_MAPS - 1) / TC_MAPS;
    a.nkb = pl.tca.nkb;
    a.n_items = pl.tca.n_lt_total * a.n_groups;
    a.n_alm = pl.n_alm;
    a.item_base = pl.tca.d_item_base;
    a.table = static_cast<const char*>(pl.tca.table);
    a.blk_base = pl.tca.d_blk_base;
    a.bops = static_cast<const char*>(pl.tca.bops);
    a.filt = pl.filt;
    a.amax = pl.tc.d_amax;
    a.grad = grad;
    a.err = pl.d_err;
    switch (pl.prec) {
        case MODAL_FP16X3: return launch_adj<MODAL_FP16X3>(pl, pa, a, part, st);
        case MODAL_BF16X3: return launch_adj<MODAL_BF16X3>(pl, pa, a, part, st);
        case MODAL_BF16: return launch_adj<MODAL_BF16>(pl, pa, a, part, st);
        case MODAL_3XTF32: return launch_adj<MODAL_3XTF32>(pl, pa, a, part, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace modal
