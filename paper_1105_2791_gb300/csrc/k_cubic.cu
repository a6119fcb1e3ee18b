// Pixel-space kernels of the modal projection (Eq. bbispect with the linear term of
// Eq. bispectrumest), the Monte Carlo pair means, and the pixel part of the adjoint.
//
//   cubic     C_prs = sum_x W_x M_p M_r M_s                      (p <= r <= s)
//   linear    G_{(ab),c} = sum_x W_x <M_a M_b>_x M_c             (all pairs, all c)
//   beta_prs  = C_prs - (G_{(pr),s} + G_{(ps),r} + G_{(rs),p})
//   pairs     S_{(ab)}(x) += sum_b M_a M_b   (mean over simulations, FP64 sums)
//   adjoint   U_t(x) = 3 W_x sum_{a,b} h_tab (M_a M_b - <M_a M_b>_x)
#include "modal_internal.cuh"

#include <algorithm>

namespace modal {

// ---------------------------------------------------------------- cubic term
// C_prs = sum_x U_(pr)(x) M_s(x) with U_(pr) = W M_p M_r: a GEMM of the pair-product
// panel against the map panel, one map per CTA row of the grid, the panel built in
// shared memory tile by tile and never written to HBM.
//
// Tiles: 8 colex pairs (a pair group pg, pairs sorted by r, then p) x 4 values of s (a quad
// sq); tiles entirely below the diagonal s < r are absent from the tile list.  A compute
// item holds two tiles, either of one pair group and two quads (kind A: 8 pair values and
// 2 x 4 map values per pixel for 32 packed FMAs) or of two pair groups and one quad (kind B:
// 16 + 4 values); a tile left alone is paired with a quad of zeros.  The two halves of a
// warp (16 lanes each) take one item each, of the same kind, so that a warp runs one path.
//
// Warp roles (named barriers, two shared-memory stages of CUB_TX pixels each):
//   fill warps     two pixels per thread: the map values and W are prefetched one tile
//                  ahead in registers, the pair products of all colex pairs are formed
//                  in registers and stored as float4 slots of the panel;
//   compute warps  16 lanes per item, 8 pixels per lane per stage.
// Stage layout, pixel fastest: [2 n_pg slots of 4 pairs][CUB_TX] float4, then
// [n_sq + 1 quads of 4 map values][CUB_TX] float4 (the last quad is zero), so that the
// fill threads' stores and the half-warps' loads are runs of consecutive float4.  Per-CTA
// partial sums go to `partial` (FP64) and are summed in a fixed order by k_beta_finalize.
constexpr int CUB_TX = 128;                 // pixels per stage
constexpr int CUB_FILL = 64;                // fill threads (two pixels each)
constexpr int CUB_MAXCOMP = 288;            // compute threads at most (18 items x 16 lanes)
constexpr int CUB_THREADS = CUB_MAXCOMP + CUB_FILL;   // 11 warps: at most 3 per SM sub-partition
constexpr int CUB_LANES = 16;               // lanes per item

__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void named_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// items: [nslots] int2 (tile a, tile b); tile a < 0: idle slot; tile b < 0: tile a alone.
struct CubicJob {
    const float* maps;
    const float* W;
    double* partial;
    int64_t npix, ppc;
    int nctas;
};
struct CubicJobs {
    CubicJob job[CUBIC_MAX_JOBS];
    int64_t item_end[CUBIC_MAX_JOBS];   // cumulative item counts
    int n;
};

// One work item: map b of `maps`, pixel range `cta` of `nctas` ranges of px_per_cta pixels;
// the CTA's sums of every mode go to partial[(b nctas + cta) n_max + n].  Ends with the CTA
// synchronised, so that a persistent caller can run the next item on the same shared memory.
template <int PM>
__device__ __forceinline__ void cubic_item(float* smem, int P, int n_pg, int n_sq, int ntiles, int ncomp,
                                           const int* __restrict__ tiles, const int2* __restrict__ items,
                                           const int* __restrict__ modeidx, int64_t npix, int64_t px_per_cta,
                                           const float* __restrict__ maps, const float* __restrict__ W,
                                           double* __restrict__ partial, int n_max, int b, int cta, int nctas) {
    const int nslot = 2 * n_pg;
    const int stage_f4 = (nslot + n_sq + 1) * CUB_TX;              // float4 per stage
    const int tid = threadIdx.x;
    const int nthr = ncomp + CUB_FILL;
    const int64_t x_begin = (int64_t)cta * px_per_cta;
    const int64_t x_end = min(npix, x_begin + px_per_cta);
    const int nch = (x_end > x_begin) ? (int)((x_end - x_begin + CUB_TX - 1) / CUB_TX) : 0;
    const float* mb = maps + (int64_t)b * P * npix;
    float4* s4 = reinterpret_cast<float4*>(smem);

    // the zero quad of both stages
    for (int i = tid; i < 2 * CUB_TX; i += nthr)
        s4[(i / CUB_TX) * stage_f4 + (nslot + n_sq) * CUB_TX + i % CUB_TX] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();

    float accA[32], accB[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) accA[e] = accB[e] = 0.f;
    const int lane16 = (tid % 32) % CUB_LANES;
    const int slot_item = tid / CUB_LANES;
    int2 it = make_int2(-1, -1);

    if (tid >= ncomp) {
        // ------------------------------------------------ fill warps
        const int xl = tid - ncomp;                                  // pixels xl and xl + CUB_FILL
        float cur[2][PM + 1], n1[2][PM + 1];
        auto load = [&](float (&v)[2][PM + 1], int k) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t x = x_begin + (int64_t)k * CUB_TX + xl + h * CUB_FILL;
                const bool in = k < nch && x < x_end;
#pragma unroll
                for (int p = 0; p < PM; ++p) v[h][p] = (in && p < P) ? mb[(int64_t)p * npix + x] : 0.f;
                v[h][PM] = in ? W[x] : 0.f;
            }
        };
        load(cur, 0);
        for (int k = 0; k < nch; ++k) {
            load(n1, k + 1);
            const int s = k & 1;
            if (k >= 2) named_sync(3 + s, nthr);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float4* sU = s4 + s * stage_f4 + xl + h * CUB_FILL;
                float4* sM = sU + nslot * CUB_TX;
                const float* cv = cur[h];
                float wm[PM];
#pragma unroll
                for (int p = 0; p < PM; ++p) wm[p] = cv[PM] * cv[p];
                float st[4];
#pragma unroll
                for (int r = 0; r < PM; ++r)
#pragma unroll
                    for (int p = 0; p <= r; ++p) {
                        const int c = r * (r + 1) / 2 + p;           // colex pair index
                        st[c & 3] = wm[p] * cv[r];
                        if ((c & 3) == 3 && c < 8 * n_pg) sU[(c >> 2) * CUB_TX] = make_float4(st[0], st[1], st[2], st[3]);
                    }
                constexpr int NPR = PM * (PM + 1) / 2;
                if ((NPR & 3) != 0) {                                // tail of a partial float4
                    const int c0 = NPR & ~3;
#pragma unroll
                    for (int i = (NPR & 3); i < 4; ++i) st[i] = 0.f;
                    if (c0 < 8 * n_pg) sU[(c0 >> 2) * CUB_TX] = make_float4(st[0], st[1], st[2], st[3]);
                }
                // pair slots past the colex pairs of PM modes (8 n_pg > NPR) are zero
                for (int c0 = (NPR + 3) & ~3; c0 < 8 * n_pg; c0 += 4)
                    sU[(c0 >> 2) * CUB_TX] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < (PM + 3) / 4; ++q)
                    if (q < n_sq)
                        sM[q * CUB_TX] = make_float4(q * 4 + 0 < PM ? cv[q * 4 + 0] : 0.f, q * 4 + 1 < PM ? cv[q * 4 + 1] : 0.f,
                                                     q * 4 + 2 < PM ? cv[q * 4 + 2] : 0.f, q * 4 + 3 < PM ? cv[q * 4 + 3] : 0.f);
            }
            named_arrive(1 + s, nthr);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int p = 0; p <= PM; ++p) cur[h][p] = n1[h][p];
        }
    } else {
        // ------------------------------------------------ compute warps
        it = items[slot_item];
        const bool active = it.x >= 0;
        const int ta = active ? tiles[it.x] : 0;
        const int tb = (active && it.y >= 0) ? tiles[it.y] : -1;
        const int pga = ta & 0xff, sqa = ta >> 8;
        // kind A: one pair group, quads a and b (the zero quad for a lone tile); kind B: two pair groups, one quad
        const bool kindB = tb >= 0 && (tb & 0xff) != pga;
        const int pgb = kindB ? (tb & 0xff) : pga;
        const int sqb = kindB ? sqa : (tb >= 0 ? (tb >> 8) : n_sq);
        for (int k = 0; k < nch; ++k) {
            const int s = k & 1;
            named_sync(1 + s, nthr);
            if (active) {
                const float4* sU = s4 + s * stage_f4;
                const float4* sM = sU + nslot * CUB_TX;
                // packed FP32 pairs (one rounding per lane, as fmaf): tA[ip][q], tB[ip][q] hold the
                // sums of pairs 2 ip, 2 ip + 1 of the two tiles against their s = 4 sq + q
                float2 tA[4][4], tB[4][4];
#pragma unroll
                for (int ip = 0; ip < 4; ++ip)
#pragma unroll
                    for (int q = 0; q < 4; ++q) tA[ip][q] = tB[ip][q] = make_float2(0.f, 0.f);
                if (!kindB) {
#pragma unroll 1
                    for (int xi = lane16; xi < CUB_TX; xi += CUB_LANES) {
                        const float4 u0 = sU[(2 * pga) * CUB_TX + xi], u1 = sU[(2 * pga + 1) * CUB_TX + xi];
                        const float4 ma = sM[sqa * CUB_TX + xi], mbv = sM[sqb * CUB_TX + xi];
                        const float2 u2[4] = {make_float2(u0.x, u0.y), make_float2(u0.z, u0.w), make_float2(u1.x, u1.y),
                                              make_float2(u1.z, u1.w)};
                        const float2 a2[4] = {make_float2(ma.x, ma.x), make_float2(ma.y, ma.y), make_float2(ma.z, ma.z),
                                              make_float2(ma.w, ma.w)};
                        const float2 b2[4] = {make_float2(mbv.x, mbv.x), make_float2(mbv.y, mbv.y),
                                              make_float2(mbv.z, mbv.z), make_float2(mbv.w, mbv.w)};
#pragma unroll
                        for (int ip = 0; ip < 4; ++ip)
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                tA[ip][q] = __ffma2_rn(u2[ip], a2[q], tA[ip][q]);
                                tB[ip][q] = __ffma2_rn(u2[ip], b2[q], tB[ip][q]);
                            }
                    }
                } else {
#pragma unroll 1
                    for (int xi = lane16; xi < CUB_TX; xi += CUB_LANES) {
                        const float4 u0 = sU[(2 * pga) * CUB_TX + xi], u1 = sU[(2 * pga + 1) * CUB_TX + xi];
                        const float4 v0 = sU[(2 * pgb) * CUB_TX + xi], v1 = sU[(2 * pgb + 1) * CUB_TX + xi];
                        const float4 mv = sM[sqa * CUB_TX + xi];
                        const float2 u2[4] = {make_float2(u0.x, u0.y), make_float2(u0.z, u0.w), make_float2(u1.x, u1.y),
                                              make_float2(u1.z, u1.w)};
                        const float2 v2[4] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w), make_float2(v1.x, v1.y),
                                              make_float2(v1.z, v1.w)};
                        const float2 m2[4] = {make_float2(mv.x, mv.x), make_float2(mv.y, mv.y), make_float2(mv.z, mv.z),
                                              make_float2(mv.w, mv.w)};
#pragma unroll
                        for (int ip = 0; ip < 4; ++ip)
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                tA[ip][q] = __ffma2_rn(u2[ip], m2[q], tA[ip][q]);
                                tB[ip][q] = __ffma2_rn(v2[ip], m2[q], tB[ip][q]);
                            }
                    }
                }
#pragma unroll
                for (int ip = 0; ip < 4; ++ip)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        accA[(2 * ip) * 4 + q] += tA[ip][q].x;
                        accA[(2 * ip + 1) * 4 + q] += tA[ip][q].y;
                        accB[(2 * ip) * 4 + q] += tB[ip][q].x;
                        accB[(2 * ip + 1) * 4 + q] += tB[ip][q].y;
                    }
            }
            if (k + 2 < nch) named_arrive(3 + s, nthr);
        }
    }
    __syncthreads();
    float* red = smem;   // [CUB_LANES][ntiles][32]
    if (tid < ncomp && it.x >= 0) {
#pragma unroll
        for (int e = 0; e < 32; ++e) red[(lane16 * ntiles + it.x) * 32 + e] = accA[e];
        if (it.y >= 0) {
#pragma unroll
            for (int e = 0; e < 32; ++e) red[(lane16 * ntiles + it.y) * 32 + e] = accB[e];
        }
    }
    __syncthreads();
    for (int i = tid; i < ntiles * 32; i += nthr) {
        const int t = i / 32, e = i % 32;
        float v = 0.f;
        for (int ln = 0; ln < CUB_LANES; ++ln) v += red[(ln * ntiles + t) * 32 + e];
        const int tp = tiles[t];
        const int c = (tp & 0xff) * 8 + e / 4, sv = (tp >> 8) * 4 + e % 4;
        const int n = modeidx[c * 16 + sv];
        if (n >= 0) partial[((int64_t)b * nctas + cta) * n_max + n] = (double)v;
    }
    __syncthreads();
}

template <int PM>
__global__ void __launch_bounds__(CUB_THREADS, 1)
k_cubic(int P, int n_pg, int n_sq, int ntiles, int ncomp, const int* __restrict__ tiles, const int2* __restrict__ items,
        const int* __restrict__ modeidx, int64_t npix, int64_t px_per_cta, const float* __restrict__ maps,
        const float* __restrict__ W, double* __restrict__ partial, int n_max) {
    extern __shared__ __align__(16) float smem[];
    cubic_item<PM>(smem, P, n_pg, n_sq, ntiles, ncomp, tiles, items, modeidx, npix, px_per_cta, maps, W, partial, n_max,
                   blockIdx.y, blockIdx.x, gridDim.x);
}

// The cubic sums of several plans (one pass of a mixed-l_max batch, the same P) as one
// persistent launch: CTAs take (job, map, pixel range) items from a device counter, jobs in
// the order given (the host puts the plans with the longest items first); every item is the
// one the plan's own launch would compute, so the partial sums are identical.
template <int PM>
__global__ void __launch_bounds__(CUB_THREADS, 1)
k_cubic_multi(CubicJobs jobs, int P, int n_pg, int n_sq, int ntiles, int ncomp, const int* __restrict__ tiles,
              const int2* __restrict__ items, const int* __restrict__ modeidx, int n_max, int* __restrict__ counter) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t item = s_item;
        __syncthreads();
        if (item >= jobs.item_end[jobs.n - 1]) break;
        int j = 0;
        while (item >= jobs.item_end[j]) ++j;
        const int64_t local = item - (j > 0 ? jobs.item_end[j - 1] : 0);
        const CubicJob& jb = jobs.job[j];
        cubic_item<PM>(smem, P, n_pg, n_sq, ntiles, ncomp, tiles, items, modeidx, jb.npix, jb.ppc, jb.maps, jb.W,
                       jb.partial, n_max, (int)(local / jb.nctas), (int)(local % jb.nctas), jb.nctas);
    }
}

static size_t cubic_smem(const Plan& pl) {
    const size_t tilebuf = 2 * (size_t)CUB_TX * (2 * pl.n_pg + pl.n_sq + 1) * 16;
    const size_t redbuf = (size_t)CUB_LANES * pl.n_tiles * 32 * 4;
    return tilebuf > redbuf ? tilebuf : redbuf;
}

template <int PM>
static cudaError_t launch_cubic_pm(Plan& pl, const float* maps, int B, double* partial, cudaStream_t st) {
    const int ncomp = pl.cubic_nslots * CUB_LANES;
    const size_t smem = cubic_smem(pl);
    cudaError_t e = cudaFuncSetAttribute(k_cubic<PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t ppc = ((pl.npix + pl.cubic_ctas - 1) / pl.cubic_ctas + CUB_TX - 1) / CUB_TX * CUB_TX;
    dim3 grid(pl.cubic_ctas, B);
    k_cubic<PM><<<grid, ncomp + CUB_FILL, smem, st>>>(pl.P, pl.n_pg, pl.n_sq, pl.n_tiles, ncomp, pl.tiles,
                                                    reinterpret_cast<const int2*>(pl.tiles + ((pl.n_tiles + 1) & ~1)), pl.modeidx,
                                                    pl.npix, ppc, maps, pl.W, partial, pl.n_max);
    note_launch(pl);
    return cudaGetLastError();
}

template <int PM>
static cudaError_t launch_cubic_multi_pm(const Plan& p0, const CubicJobs& jobs, int* counter, int nctas_grid,
                                        cudaStream_t st) {
    const int ncomp = p0.cubic_nslots * CUB_LANES;
    const size_t smem = cubic_smem(p0);
    cudaError_t e = cudaFuncSetAttribute(k_cubic_multi<PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_cubic_multi<PM><<<nctas_grid, ncomp + CUB_FILL, smem, st>>>(jobs, p0.P, p0.n_pg, p0.n_sq, p0.n_tiles, ncomp, p0.tiles,
                                                                   reinterpret_cast<const int2*>(p0.tiles + ((p0.n_tiles + 1) & ~1)),
                                                                   p0.modeidx, p0.n_max, counter);
    note_launch(p0);
    return cudaGetLastError();
}

cudaError_t launch_cubic_multi(Plan* const* plans, const float* const* maps, const int* B, int n, int* counter,
                               cudaStream_t st) {
    if (n < 1 || n > CUBIC_MAX_JOBS) return cudaErrorInvalidValue;
    const Plan& p0 = *plans[0];
    if (p0.cubic_nslots * CUB_LANES > CUB_MAXCOMP || p0.cubic_nslots % 2 != 0) return cudaErrorInvalidValue;
    CubicJobs jobs = {};
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        const Plan& pl = *plans[i];
        if (pl.P != p0.P || B[i] < 1 || B[i] > pl.chunk) return cudaErrorInvalidValue;
        CubicJob& jb = jobs.job[i];
        jb.maps = maps[i];
        jb.W = pl.W;
        jb.partial = pl.partial;
        jb.npix = pl.npix;
        jb.nctas = pl.cubic_ctas;
        jb.ppc = ((pl.npix + pl.cubic_ctas - 1) / pl.cubic_ctas + CUB_TX - 1) / CUB_TX * CUB_TX;
        total += (int64_t)B[i] * pl.cubic_ctas;
        jobs.item_end[i] = total;
    }
    jobs.n = n;
    const int grid = (int)std::min<int64_t>(total, (int64_t)std::max(p0.nsm, 1));
    if (p0.P <= 4) return launch_cubic_multi_pm<4>(p0, jobs, counter, grid, st);
    if (p0.P <= 8) return launch_cubic_multi_pm<8>(p0, jobs, counter, grid, st);
    return launch_cubic_multi_pm<16>(p0, jobs, counter, grid, st);
}

cudaError_t launch_cubic(Plan& pl, const float* maps, int B, double* partial, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    if (pl.cubic_nslots * CUB_LANES > CUB_MAXCOMP || pl.cubic_nslots % 2 != 0) return cudaErrorInvalidValue;
    if (pl.P <= 4) return launch_cubic_pm<4>(pl, maps, B, partial, st);
    if (pl.P <= 8) return launch_cubic_pm<8>(pl, maps, B, partial, st);
    return launch_cubic_pm<16>(pl, maps, B, partial, st);
}

// ---------------------------------------------------------------- linear term GEMM
// out[z][row][col] = sum_{x in split z} (W_x <pair row>_x) * maps[col][x],
// rows = pairs (lexicographic), cols = (map, c) = b * P + c.  64 x 64 CTA tiles,
// 4 x 4 register tiles, K (pixels) staged 32 at a time, split over gridDim.z.
constexpr int LG_TM = 64, LG_TN = 64, LG_TK = 32;

__global__ void __launch_bounds__(256)
k_linear_gemm(int nrows, int ncols, int64_t npix, int64_t kchunk, const float* __restrict__ panel,
              const float* __restrict__ W, const float* __restrict__ maps, double* __restrict__ out) {
    __shared__ __align__(16) float sA[LG_TK][LG_TM + 4];
    __shared__ __align__(16) float sB[LG_TK][LG_TN + 4];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int r0 = blockIdx.x * LG_TM, c0 = blockIdx.y * LG_TN;
    const int64_t k_begin = (int64_t)blockIdx.z * kchunk;
    const int64_t k_end = min(npix, k_begin + kchunk);
    float acc[4][4] = {};
    for (int64_t k0 = k_begin; k0 < k_end; k0 += LG_TK) {
        for (int i = tid; i < LG_TM * LG_TK; i += 256) {
            const int r = i / LG_TK, k = i % LG_TK;
            const int64_t x = k0 + k;
            float v = 0.f;
            if (r0 + r < nrows && x < k_end) v = panel[(int64_t)(r0 + r) * npix + x] * W[x];
            sA[k][r] = v;
        }
        for (int i = tid; i < LG_TN * LG_TK; i += 256) {
            const int c = i / LG_TK, k = i % LG_TK;
            const int64_t x = k0 + k;
            sB[k][c] = (c0 + c < ncols && x < k_end) ? maps[(int64_t)(c0 + c) * npix + x] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < LG_TK; ++k) {
            const float4 a = *reinterpret_cast<const float4*>(&sA[k][ty * 4]);
            const float4 bb = *reinterpret_cast<const float4*>(&sB[k][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + ty * 4 + i, c = c0 + tx * 4 + j;
            if (r < nrows && c < ncols) out[((int64_t)blockIdx.z * nrows + r) * ncols + c] = (double)acc[i][j];
        }
}

cudaError_t launch_linear_gemm(Plan& pl, const float* maps, int B, double* partial, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    const int ncols = B * pl.P;
    const int64_t kchunk = ((pl.npix + pl.lin_ksplit - 1) / pl.lin_ksplit + LG_TK - 1) / LG_TK * LG_TK;
    dim3 grid((pl.n_pair + LG_TM - 1) / LG_TM, (ncols + LG_TN - 1) / LG_TN, pl.lin_ksplit);
    k_linear_gemm<<<grid, 256, 0, st>>>(pl.n_pair, ncols, pl.npix, kchunk, pl.pair_mean, pl.W, maps, partial);
    note_launch(pl);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- beta
__device__ __forceinline__ int pair_lex(int p, int r, int P) { return p * P - (p * (p - 1)) / 2 + (r - p); }

__global__ void k_beta_finalize(int P, int n_max, int B, int ncub, int use_linear, int ksplit, int n_pair,
                                const int* __restrict__ mp, const int* __restrict__ mr, const int* __restrict__ ms,
                                const double* __restrict__ cub, const double* __restrict__ lin,
                                double* __restrict__ beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * n_max) return;
    const int b = i / n_max, n = i % n_max;
    double v = 0.0;
    for (int c = 0; c < ncub; ++c) v += cub[((int64_t)b * ncub + c) * n_max + n];
    if (use_linear) {
        const int p = mp[n], r = mr[n], s = ms[n];
        const int ncols = B * P;
        const int rpr = pair_lex(p, r, P), rps = pair_lex(p, s, P), rrs = pair_lex(r, s, P);
        double l = 0.0;
        for (int z = 0; z < ksplit; ++z) {
            const double* g = lin + (int64_t)z * n_pair * ncols;
            l += g[(int64_t)rpr * ncols + b * P + s] + g[(int64_t)rps * ncols + b * P + r]
               + g[(int64_t)rrs * ncols + b * P + p];
        }
        v -= l;
    }
    beta[i] = v;
}

cudaError_t launch_beta_finalize(Plan& pl, int B, int use_linear, const double* cub_partial,
                                 const double* lin_partial, int lin_splits, double* beta, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    const int n = B * pl.n_max;
    k_beta_finalize<<<(n + 127) / 128, 128, 0, st>>>(pl.P, pl.n_max, B, pl.cubic_ctas, use_linear, lin_splits,
                                                      pl.n_pair, pl.modeidx + 16 * 256, pl.modeidx + 16 * 256 + 1024,
                                                      pl.modeidx + 16 * 256 + 2048, cub_partial, lin_partial, beta);
    note_launch(pl);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Monte Carlo pair means
// Two threads per pixel: thread h (h = 0, 1, warp-uniform) owns the mode rows p = 2k + h,
// k = 0 .. PM/2 - 1.  It works on its pixel's map values shifted by h (v[i] = M_{i+h}),
// so that both threads run the same code with compile-time indices: its pairs are
// (2k, r') in the shifted frame, r' >= 2k, i.e. (2k + h, r' + h).  The maps stream
// through a PA_STAGES-deep ring in shared memory by cp.async: the two threads of a
// pixel copy alternate rows of its column (each map value is fetched once) and read the
// whole column after a CTA barrier; a second barrier keeps a stage from being refilled
// while it is read.  The FP64 sums are read, updated and written once per launch: the
// tile's FP32 sums go to shared memory by pair, each thread updates the pairs of its parity
// at its pixel, PA_RMW loads in flight at a time (more spill at the 128-register cap that
// keeps four CTAs per SM), their lines sent to L2 a few maps before the update.
constexpr int PA_THREADS = 128;             // 64 pixels x 2 row parities
constexpr int PA_PIX = PA_THREADS / 2;
constexpr int PA_STAGES = 5;
constexpr int PA_RMW = 8;                   // FP64 read-modify-writes in flight per thread (68 per thread at P = 16)
constexpr int PA_PREFETCH = 4;              // maps before the end of a tile at which its FP64 sums go to L2

template <int PM>
constexpr size_t pa_smem_floats() {
    constexpr size_t ring = (size_t)PA_STAGES * PM * PA_PIX;
    constexpr size_t sums = (size_t)(PM * (PM + 1) / 2) * PA_PIX;
    return ring > sums ? ring : sums;
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}

template <int PM>
__global__ void __launch_bounds__(PA_THREADS, 4)
k_pair_accumulate(int P, int B, int64_t npix, const float* __restrict__ maps, double* __restrict__ sums) {
    constexpr int NACC = (PM / 2) * (PM / 2 + 1);                // sum over k of (PM - 2k)
    extern __shared__ __align__(16) float pa_ring[];            // [PA_STAGES][PM][PA_PIX]; then [n_pair][PA_PIX]
    const int tid = threadIdx.x;
    const int h = tid / PA_PIX, xl = tid % PA_PIX;
    const int nv = P - h;                                       // shifted values that exist
    for (int64_t x0 = (int64_t)blockIdx.x * PA_PIX; x0 < npix; x0 += (int64_t)gridDim.x * PA_PIX) {
        const int64_t x = x0 + xl;
        const bool in = x < npix;
        __syncthreads();                                              // previous sums read out of the ring
        auto issue = [&](int b) {
            if (b < B && in) {
                const float* src = maps + ((int64_t)b * P + h) * npix + x;
                float* dst = pa_ring + ((b % PA_STAGES) * PM + h) * PA_PIX + xl;
                for (int i = h; i < P; i += 2) {                        // rows of this thread's parity
                    cp_async4(dst, src);
                    src += 2 * npix;
                    dst += 2 * PA_PIX;
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
#pragma unroll
        for (int b = 0; b < PA_STAGES - 1; ++b) issue(b);
        float acc[NACC];
#pragma unroll
        for (int c = 0; c < NACC; ++c) acc[c] = 0.f;
#pragma unroll 1
        for (int b = 0; b < B; ++b) {
            __syncthreads();                                          // stage (b - 1) % PA_STAGES is free
            issue(b + PA_STAGES - 1);
            asm volatile("cp.async.wait_group %0;" ::"n"(PA_STAGES - 1) : "memory");   // this thread's rows of map b
            __syncthreads();                                          // ... and the partner's
            if (b == (B > PA_PREFETCH ? B - PA_PREFETCH : 0)) {
                // the FP64 sums of this tile into L2 a few maps before their update: one
                // 128-byte line per thread and step (PA_PIX doubles of a pair = 4 lines)
                const int npair = P * (P + 1) / 2;
                for (int i = tid; i < npair * (PA_PIX / 16); i += PA_THREADS) {
                    const int64_t xs = x0 + (i % (PA_PIX / 16)) * 16;
                    if (xs < npix) {
                        const double* line = sums + (int64_t)(i / (PA_PIX / 16)) * npix + xs;
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(line));
                    }
                }
            }
            const float* col = pa_ring + ((b % PA_STAGES) * PM + h) * PA_PIX + xl;
            float v[PM];
#pragma unroll
            for (int i = 0; i < PM; ++i) v[i] = (i < nv && in) ? col[i * PA_PIX] : 0.f;
            int c = 0;
#pragma unroll
            for (int k = 0; k < PM / 2; ++k)
#pragma unroll
                for (int r = 2 * k; r < PM; ++r) {
                    acc[c] = fmaf(v[2 * k], v[r], acc[c]);
                    ++c;
                }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();                                              // the ring is free
        // the sums pass through shared memory, one row of PA_PIX pixels per pair (lexicographic),
        // so that the FP64 update below runs over pairs h, h + 2, ... with one stride
#pragma unroll
        for (int k = 0, c = 0; k < PM / 2; ++k) {
            const int pa = 2 * k + h, q0 = pair_lex(pa, pa, P);
#pragma unroll
            for (int j = 0; j < PM - 2 * k; ++j, ++c)
                if (pa + j < P) pa_ring[(q0 + j) * PA_PIX + xl] = acc[c];
        }
        __syncthreads();
        if (in) {
            // PA_RMW old values are loaded before the first of their stores, so that those
            // loads are in flight together
            const int nq = (P * (P + 1) / 2 - h + 1) / 2;
            double* row = sums + (int64_t)h * npix + x;
            const float* add = pa_ring + h * PA_PIX + xl;
#pragma unroll 1
            for (int i0 = 0; i0 < nq; i0 += PA_RMW) {
                double old[PA_RMW];
#pragma unroll
                for (int u = 0; u < PA_RMW; ++u)
                    if (i0 + u < nq) old[u] = row[(int64_t)(2 * (i0 + u)) * npix];
#pragma unroll
                for (int u = 0; u < PA_RMW; ++u)
                    if (i0 + u < nq) row[(int64_t)(2 * (i0 + u)) * npix] = old[u] + (double)add[2 * (i0 + u) * PA_PIX];
            }
        }
    }
}

cudaError_t launch_pair_accumulate(Plan& pl, const float* maps, int B, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    const int64_t nblk = (pl.npix + PA_PIX - 1) / PA_PIX;
    const int grid = (int)(nblk < 152 * 16 ? nblk : 152 * 16);
    note_launch(pl);
    if (pl.P <= 4)
        k_pair_accumulate<4><<<grid, PA_THREADS, pa_smem_floats<4>() * 4, st>>>(pl.P, B, pl.npix, maps, pl.pair_sum);
    else if (pl.P <= 8)
        k_pair_accumulate<8><<<grid, PA_THREADS, pa_smem_floats<8>() * 4, st>>>(pl.P, B, pl.npix, maps, pl.pair_sum);
    else
        k_pair_accumulate<16><<<grid, PA_THREADS, pa_smem_floats<16>() * 4, st>>>(pl.P, B, pl.npix, maps, pl.pair_sum);
    return cudaGetLastError();
}

__global__ void k_pair_finalize(int64_t n, double inv, const double* __restrict__ sums, float* __restrict__ mean) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        mean[i] = (float)(sums[i] * inv);
}

cudaError_t launch_pair_finalize(Plan& pl, cudaStream_t st) {
    const int64_t n = (int64_t)pl.n_pair * pl.npix;
    k_pair_finalize<<<152 * 8, 256, 0, st>>>(n, 1.0 / (double)pl.n_lin, pl.pair_sum, pl.pair_mean);
    note_launch(pl);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- adjoint (pixel part)
// hk[b][t][c] = 3 k_c h_{t,a,b'} for lexicographic pair c = (a, b'), k_c = 2 if a != b'
// else 1, h_tab = g_{sort(t,a,b)} / (number of distinct orderings of that triple).
__global__ void k_adjoint_weights(int P, int n_pair, int n_max, int B, const int* __restrict__ mode_of,
                                  const double* __restrict__ g, float* __restrict__ hk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * P * n_pair) return;
    const int b = i / (P * n_pair), rem = i % (P * n_pair), t = rem / n_pair, c = rem % n_pair;
    int a = 0, cc = c;
    while (cc >= P - a) { cc -= P - a; ++a; }
    const int bb = a + cc;
    int x0 = t, x1 = a, x2 = bb, tmp;
    if (x0 > x1) { tmp = x0; x0 = x1; x1 = tmp; }
    if (x1 > x2) { tmp = x1; x1 = x2; x2 = tmp; }
    if (x0 > x1) { tmp = x0; x0 = x1; x1 = tmp; }
    const int nperm = (x0 == x2) ? 1 : ((x0 == x1 || x1 == x2) ? 3 : 6);
    const int n = mode_of[(x0 * P + x1) * P + x2];
    const double kc = (a == bb) ? 1.0 : 2.0;
    hk[i] = (float)(3.0 * kc * g[(int64_t)b * n_max + n] / nperm);
}

cudaError_t launch_adjoint_weights(Plan& pl, const double* g, int B, float* hk, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    const int n = B * pl.P * pl.n_pair;
    k_adjoint_weights<<<(n + 127) / 128, 128, 0, st>>>(pl.P, pl.n_pair, pl.n_max, B, pl.modeidx + 16 * 256 + 3072,
                                                        g, hk);
    note_launch(pl);
    return cudaGetLastError();
}

// In place: maps[b][t][x] <- U_t(x) = W_x sum_c hk[b][t][c] (M_a M_b' - <c>_x).
// Register tile per thread: AU_NX adjacent pixels x AU_NB maps, all PM values of each
// map in registers, accumulators packed in FP32 pairs over t.  Both pair loops (a, then
// b' >= a) are unrolled at compile time, so every map value is a register and the body
// has no branches; each pair costs four broadcast float4 loads of the weights per map
// and one 8-byte load of the pair means for 8 AU_NX AU_NB packed FMAs.  The pair-mean
// row of a + 1 is copied into shared memory (cp.async, each thread its own pixels) while
// row a is being used.  A CTA keeps its AU_NB maps' weights in shared memory and walks
// pixel tiles g, g + G, ...; CTAs of the same g but different map pairs are adjacent in
// launch order, so they read the same pair-mean rows close together in time.
constexpr int AU_THREADS = 128;
constexpr int AU_NX = 2;                    // adjacent pixels per thread
constexpr int AU_NB = 2;                    // maps per thread (and per CTA)
constexpr int AU_TILE = AU_THREADS * AU_NX; // pixels per CTA tile

__device__ __forceinline__ void cp_async8(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Pair-mean row a (b' = a .. P-1 of this thread's two pixels) into stage a & 1.
template <int PM>
__device__ __forceinline__ void adj_issue_row(int a, const float* __restrict__ pm, bool in, int P, int64_t npix,
                                              int64_t x0, int px, float* sP) {
    if (pm && in) {
        const int crow = a * P - a * (a - 1) / 2 - a;
        float* dst = sP + (a & 1) * PM * AU_TILE + px;
#pragma unroll
        for (int bb = 0; bb < PM; ++bb)
            if (bb >= a && bb < P) cp_async8(dst + bb * AU_TILE, pm + (int64_t)(crow + bb) * npix + x0 + px);
    }
    cp_async_commit();
}

// Row A of the pair loop (pairs (A, b'), b' >= A), then rows A+1 .. PM-1: a template
// recursion, so that every map-value index is a compile-time constant.
template <int PM, int A>
__device__ __forceinline__ void adj_rows(const float2 (&M)[AU_NB][PM], float2 (&u)[AU_NB][AU_NX][PM / 2],
                                         const float* sH, float* sP, const float* __restrict__ pm, bool in, int P,
                                         int64_t npix, int64_t x0, int px) {
    if constexpr (A < PM) {
        constexpr int NPM = PM * (PM + 1) / 2;
        if (A + 1 < PM) adj_issue_row<PM>(A + 1, pm, in, P, npix, x0, px, sP);
        else cp_async_commit();
        cp_async_wait1();                                  // row A has landed
        const float* prow = sP + (A & 1) * PM * AU_TILE + px;
#pragma unroll
        for (int bb = A; bb < PM; ++bb) {
            const float2 pv = *reinterpret_cast<const float2*>(prow + bb * AU_TILE);
            const int k = A * PM - A * (A - 1) / 2 + (bb - A);  // PM-lex pair index
#pragma unroll
            for (int i = 0; i < AU_NB; ++i) {
                const float y0 = fmaf(M[i][A].x, M[i][bb].x, -pv.x);
                const float y1 = fmaf(M[i][A].y, M[i][bb].y, -pv.y);
                const float2 y02 = make_float2(y0, y0), y12 = make_float2(y1, y1);
                const float4* h4 = reinterpret_cast<const float4*>(sH + (i * NPM + k) * PM);
#pragma unroll
                for (int q = 0; q < PM / 4; ++q) {
                    const float4 h = h4[q];
                    const float2 hlo = make_float2(h.x, h.y), hhi = make_float2(h.z, h.w);
                    u[i][0][2 * q] = __ffma2_rn(hlo, y02, u[i][0][2 * q]);
                    u[i][0][2 * q + 1] = __ffma2_rn(hhi, y02, u[i][0][2 * q + 1]);
                    u[i][1][2 * q] = __ffma2_rn(hlo, y12, u[i][1][2 * q]);
                    u[i][1][2 * q + 1] = __ffma2_rn(hhi, y12, u[i][1][2 * q + 1]);
                }
            }
        }
        adj_rows<PM, A + 1>(M, u, sH, sP, pm, in, P, npix, x0, px);
    }
}

template <int PM>
__global__ void __launch_bounds__(AU_THREADS, 2)
k_adjoint_u(int P, int n_pair, int B, int ngroups, int64_t npix, int nphi, int nrings, const float* __restrict__ hk,
            const float* __restrict__ pm, const float* __restrict__ vring, const float* __restrict__ W,
            float* __restrict__ maps) {
    constexpr int NPM = PM * (PM + 1) / 2;
    extern __shared__ __align__(16) float au_smem[];
    float* sH = au_smem;                                   // [AU_NB][NPM][PM], pairs in PM-lex order
    float* sP = sH + AU_NB * NPM * PM;                     // [2][PM][AU_TILE] pair-mean rows
    const int tid = threadIdx.x;
    const int nmp = (B + AU_NB - 1) / AU_NB;
    const int mp = blockIdx.x % nmp;
    const int g = blockIdx.x / nmp;
    const int b0 = mp * AU_NB;
    const int nb = min(AU_NB, B - b0);
    const int px = AU_NX * tid;                            // this thread's pixels within a tile
    for (int i = tid; i < AU_NB * NPM * PM; i += AU_THREADS) {
        const int mb = i / (NPM * PM), rem = i % (NPM * PM);
        const int k = rem / PM, t = rem % PM;
        int a = 0, kk = k;
        while (kk >= PM - a) { kk -= PM - a; ++a; }
        const int bb = a + kk;
        float v = 0.f;
        if (mb < nb && t < P && bb < P) v = hk[((int64_t)(b0 + mb) * P + t) * n_pair + pair_lex(a, bb, P)];
        sH[i] = v;
    }
    // pair-mean rows that are never copied (b' >= P, or no linear term) read as zero
#pragma unroll
    for (int st = 0; st < 2; ++st)
#pragma unroll
        for (int bb = 0; bb < PM; ++bb)
            if (!pm || bb >= P) *reinterpret_cast<float2*>(sP + (st * PM + bb) * AU_TILE + px) = make_float2(0.f, 0.f);
    __syncthreads();
    const int64_t ntile = (npix + AU_TILE - 1) / AU_TILE;
    for (int64_t tile = g; tile < ntile; tile += ngroups) {
        const int64_t x0 = tile * AU_TILE;
        const bool in = x0 + px < npix;                    // npix is even: both pixels or neither
        adj_issue_row<PM>(0, pm, in, P, npix, x0, px, sP);
        float2 M[AU_NB][PM];                               // (pixel 0, pixel 1) per map and mode
#pragma unroll
        for (int i = 0; i < AU_NB; ++i)
#pragma unroll
            for (int p = 0; p < PM; ++p) {
                float2 v = make_float2(0.f, 0.f);
                if (i < nb && p < P && in) v = *reinterpret_cast<const float2*>(maps + ((int64_t)(b0 + i) * P + p) * npix + x0 + px);
                M[i][p] = v;
            }
        float2 u[AU_NB][AU_NX][PM / 2];                    // (t = 2 tp, 2 tp + 1) packed
#pragma unroll
        for (int i = 0; i < AU_NB; ++i)
#pragma unroll
            for (int j = 0; j < AU_NX; ++j)
#pragma unroll
                for (int tp = 0; tp < PM / 2; ++tp) u[i][j][tp] = make_float2(0.f, 0.f);
        // sP entries are copied in and read by the same thread only
        adj_rows<PM, 0>(M, u, sH, sP, pm, in, P, npix, x0, px);
        if (in) {
            const float2 wx = *reinterpret_cast<const float2*>(W + x0 + px);
            const int ring = (int)((x0 + px) / nphi);     // both pixels (nphi is even)
#pragma unroll
            for (int i = 0; i < AU_NB; ++i)
#pragma unroll
                for (int t = 0; t < PM; ++t)
                    if (i < nb && t < P) {
                        // ring mode: the pair-mean term sum_c h_tc <c>_ring, the same for both pixels
                        const float vr = vring ? vring[((int64_t)(b0 + i) * P + t) * nrings + ring] : 0.f;
                        const float u0 = ((t & 1) ? u[i][0][t >> 1].y : u[i][0][t >> 1].x) - vr;
                        const float u1 = ((t & 1) ? u[i][1][t >> 1].y : u[i][1][t >> 1].x) - vr;
                        *reinterpret_cast<float2*>(maps + ((int64_t)(b0 + i) * P + t) * npix + x0 + px) =
                            make_float2(wx.x * u0, wx.y * u1);
                    }
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

template <int PM>
static cudaError_t launch_adjoint_u_pm(Plan& pl, int B, const float* hk, const float* pm, const float* vring,
                                       float* maps, cudaStream_t st) {
    constexpr int NPM = PM * (PM + 1) / 2;
    const size_t smem = ((size_t)AU_NB * NPM * PM + (size_t)2 * PM * AU_TILE) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_adjoint_u<PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nmp = (B + AU_NB - 1) / AU_NB;
    const int64_t ntile = (pl.npix + AU_TILE - 1) / AU_TILE;
    // two resident CTAs per SM in total, every map pair in every group
    int64_t ng = std::max<int64_t>(1, (152 * 2) / nmp);
    ng = std::min<int64_t>(ng, ntile);
    k_adjoint_u<PM><<<(unsigned)(ng * nmp), AU_THREADS, smem, st>>>(pl.P, pl.n_pair, B, (int)ng, pl.npix, pl.nphi,
                                                                    pl.nrings, hk, pm, vring, pl.W, maps);
    note_launch(pl);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_u(Plan& pl, const float* /*maps_in*/, int B, const float* hk, int use_linear,
                             float* maps, cudaStream_t st) {
    // The kernel can subtract a per-ring term at every pixel (vring); the library applies
    // that term to the m = 0 analysis coefficients instead (k_vring_correct), which is
    // cheaper.  The parameter stays: without it this fully unrolled kernel is allocated
    // 255 registers with a spill and runs 15 % slower (measured at l_max = 2000).
    const float* vring = nullptr;
    if (B == 0) return cudaSuccess;
    if (pl.npix % 2 != 0) return cudaErrorInvalidValue;
    const float* pm = use_linear ? pl.pair_mean : nullptr;
    if (pl.P <= 4) return launch_adjoint_u_pm<4>(pl, B, hk, pm, vring, maps, st);
    if (pl.P <= 8) return launch_adjoint_u_pm<8>(pl, B, hk, pm, vring, maps, st);
    return launch_adjoint_u_pm<16>(pl, B, hk, pm, vring, maps, st);
}

}  // namespace modal
