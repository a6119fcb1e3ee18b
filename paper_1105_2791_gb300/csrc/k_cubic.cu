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
// Register tiles of 8 pairs x 4 values of s over pairs in colex order (by r, then p),
// so that tiles entirely below the diagonal s < r are skipped; each thread of a CTA
// owns one tile and one of 8 pixel lanes.  Pair products W M_p M_r are formed once
// per pixel in shared memory.  Per-CTA partial sums go to `partial` (FP64) and are
// summed in a fixed order by k_beta_finalize.
constexpr int CUB_TX = 64;
constexpr int CUB_LANES = 8;

__global__ void __launch_bounds__(320)
k_cubic(int P, int SU, int SM, int ntiles, const int* __restrict__ tiles, const int* __restrict__ pair_ab,
        const int* __restrict__ modeidx, int64_t npix, int64_t px_per_cta, const float* __restrict__ maps,
        const float* __restrict__ W, double* __restrict__ partial, int n_max) {
    extern __shared__ __align__(16) float smem[];
    float* sU = smem;                         // [CUB_TX][SU]
    float* sM = sU + CUB_TX * SU;             // [CUB_TX][SM]
    float* sW = sM + CUB_TX * SM;             // [CUB_TX]
    const int b = blockIdx.y;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int tile = tid % ntiles;
    const int lane = tid / ntiles;
    const bool computes = lane < CUB_LANES;
    const int tpk = tiles[tile];
    const int pg = tpk & 0xff, sq = tpk >> 8;
    const int64_t x_begin = (int64_t)blockIdx.x * px_per_cta;
    const int64_t x_end = min(npix, x_begin + px_per_cta);
    const float* mb = maps + (int64_t)b * P * npix;
    // pair-product fill: thread -> (pair column, block of pixels), fixed for the CTA
    const int nsplit = max(1, nthr / SU);
    const int fill_c = (tid < nsplit * SU) ? tid % SU : -1;
    const int fill_part = (tid < nsplit * SU) ? tid / SU : 0;
    const int fill_nx = (CUB_TX + nsplit - 1) / nsplit;
    const int fill_x0 = fill_part * fill_nx;
    const int fill_ab = (fill_c >= 0) ? pair_ab[fill_c] : -1;

    float acc[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) acc[e] = 0.f;

    for (int64_t x0 = x_begin; x0 < x_end; x0 += CUB_TX) {
        for (int i = tid; i < CUB_TX * SM; i += nthr) {
            const int xl = i % CUB_TX, s = i / CUB_TX;
            const int64_t x = x0 + xl;
            sM[xl * SM + s] = (s < P && x < x_end) ? mb[(int64_t)s * npix + x] : 0.f;
        }
        for (int i = tid; i < CUB_TX; i += nthr) sW[i] = (x0 + i < x_end) ? W[x0 + i] : 0.f;
        __syncthreads();
        if (fill_c >= 0) {
            for (int xl = fill_x0; xl < fill_x0 + fill_nx && xl < CUB_TX; ++xl)
                sU[xl * SU + fill_c] = (fill_ab >= 0) ? sW[xl] * sM[xl * SM + (fill_ab & 0xff)] * sM[xl * SM + (fill_ab >> 8)]
                                                      : 0.f;
        }
        __syncthreads();
        if (computes) {
            float tmp[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) tmp[e] = 0.f;
            for (int xi = lane; xi < CUB_TX; xi += CUB_LANES) {
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
    float* red = smem;   // [CUB_LANES][ntiles][32]
    if (computes) {
#pragma unroll
        for (int e = 0; e < 32; ++e) red[(lane * ntiles + tile) * 32 + e] = acc[e];
    }
    __syncthreads();
    for (int i = tid; i < ntiles * 32; i += nthr) {
        const int t = i / 32, e = i % 32;
        float v = 0.f;
        for (int ln = 0; ln < CUB_LANES; ++ln) v += red[(ln * ntiles + t) * 32 + e];
        const int tp = tiles[t];
        const int c = (tp & 0xff) * 8 + e / 4, s = (tp >> 8) * 4 + e % 4;
        const int n = modeidx[c * 16 + s];
        if (n >= 0) partial[((int64_t)b * gridDim.x + blockIdx.x) * n_max + n] = (double)v;
    }
}

static size_t cubic_smem(const Plan& pl) {
    const size_t tilebuf = (size_t)CUB_TX * (pl.n_pg * 8 + pl.n_sq * 4 + 1) * 4;
    const size_t redbuf = (size_t)CUB_LANES * pl.n_tiles * 32 * 4;
    return tilebuf > redbuf ? tilebuf : redbuf;
}

cudaError_t launch_cubic(Plan& pl, const float* maps, int B, double* partial, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    const int nthr = ((pl.n_tiles * CUB_LANES + 31) / 32) * 32;
    const size_t smem = cubic_smem(pl);
    cudaError_t e = cudaFuncSetAttribute(k_cubic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t ppc = ((pl.npix + pl.cubic_ctas - 1) / pl.cubic_ctas + CUB_TX - 1) / CUB_TX * CUB_TX;
    dim3 grid(pl.cubic_ctas, B);
    k_cubic<<<grid, nthr, smem, st>>>(pl.P, pl.n_pg * 8, pl.n_sq * 4, pl.n_tiles, pl.tiles, pl.pair_ab, pl.modeidx,
                                      pl.npix, ppc, maps, pl.W, partial, pl.n_max);
    return cudaGetLastError();
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
                                 const double* lin_partial, double* beta, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    const int n = B * pl.n_max;
    k_beta_finalize<<<(n + 127) / 128, 128, 0, st>>>(pl.P, pl.n_max, B, pl.cubic_ctas, use_linear, pl.lin_ksplit,
                                                      pl.n_pair, pl.modeidx + 16 * 256, pl.modeidx + 16 * 256 + 1024,
                                                      pl.modeidx + 16 * 256 + 2048, cub_partial, lin_partial, beta);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Monte Carlo pair means
template <int PM>
__global__ void __launch_bounds__(128)
k_pair_accumulate(int P, int B, int64_t npix, const float* __restrict__ maps, double* __restrict__ sums) {
    constexpr int NPM = PM * (PM + 1) / 2;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < npix; x += (int64_t)gridDim.x * blockDim.x) {
        float acc[NPM];
#pragma unroll
        for (int c = 0; c < NPM; ++c) acc[c] = 0.f;
        for (int b = 0; b < B; ++b) {
            float mv[PM];
#pragma unroll
            for (int p = 0; p < PM; ++p) mv[p] = (p < P) ? maps[((int64_t)b * P + p) * npix + x] : 0.f;
            int c = 0;
#pragma unroll
            for (int p = 0; p < PM; ++p)
#pragma unroll
                for (int r = p; r < PM; ++r) {
                    acc[c] = fmaf(mv[p], mv[r], acc[c]);
                    ++c;
                }
        }
        int c = 0;
#pragma unroll
        for (int p = 0; p < PM; ++p)
#pragma unroll
            for (int r = p; r < PM; ++r) {
                if (r < P) sums[(int64_t)pair_lex(p, r, P) * npix + x] += (double)acc[c];
                ++c;
            }
    }
}

cudaError_t launch_pair_accumulate(Plan& pl, const float* maps, int B, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    const int64_t nblk = (pl.npix + 127) / 128;
    const int grid = (int)(nblk < 152 * 16 ? nblk : 152 * 16);
    if (pl.P <= 4)
        k_pair_accumulate<4><<<grid, 128, 0, st>>>(pl.P, B, pl.npix, maps, pl.pair_sum);
    else if (pl.P <= 8)
        k_pair_accumulate<8><<<grid, 128, 0, st>>>(pl.P, B, pl.npix, maps, pl.pair_sum);
    else
        k_pair_accumulate<16><<<grid, 128, 0, st>>>(pl.P, B, pl.npix, maps, pl.pair_sum);
    return cudaGetLastError();
}

__global__ void k_pair_finalize(int64_t n, double inv, const double* __restrict__ sums, float* __restrict__ mean) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        mean[i] = (float)(sums[i] * inv);
}

cudaError_t launch_pair_finalize(Plan& pl, cudaStream_t st) {
    const int64_t n = (int64_t)pl.n_pair * pl.npix;
    k_pair_finalize<<<152 * 8, 256, 0, st>>>(n, 1.0 / (double)pl.n_lin, pl.pair_sum, pl.pair_mean);
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
    return cudaGetLastError();
}

// In place: maps[b][t][x] <- U_t(x) = W_x sum_c hk[b][t][c] (M_a M_b' - <c>_x).
// A block handles AU_MB maps for a range of pixels, so the pair-mean panel <c>_x is
// read once per AU_MB maps.  One thread per pixel; the maps' values sit in a
// shared-memory column; pairs are taken 8 at a time and each weight row is read as
// two float4 (4 FMAs per shared load).
constexpr int AU_THREADS = 128;
constexpr int AU_MB = 4;
constexpr int AU_SC = 136;                  // pairs padded to a multiple of 8 (P <= 16)

__global__ void __launch_bounds__(AU_THREADS)
k_adjoint_u(int P, int n_pair, int B, int64_t npix, const float* __restrict__ hk, const float* __restrict__ pm,
            const float* __restrict__ W, float* __restrict__ maps) {
    extern __shared__ __align__(16) float au_smem[];
    float* sH = au_smem;                                     // [AU_MB][MAXP][AU_SC]
    float* sM = sH + AU_MB * MODAL_MAXP * AU_SC;            // [AU_MB][MAXP][AU_THREADS]
    __shared__ int s_pa[AU_SC], s_pb[AU_SC];
    const int tid = threadIdx.x;
    const int b0 = blockIdx.y * AU_MB;
    const int nb = min(AU_MB, B - b0);
    for (int i = tid; i < AU_MB * MODAL_MAXP * AU_SC; i += AU_THREADS) {
        const int mb = i / (MODAL_MAXP * AU_SC), rem = i % (MODAL_MAXP * AU_SC);
        const int t = rem / AU_SC, c = rem % AU_SC;
        sH[i] = (mb < nb && t < P && c < n_pair) ? hk[((int64_t)(b0 + mb) * P + t) * n_pair + c] : 0.f;
    }
    for (int c = tid; c < AU_SC; c += AU_THREADS) {
        int pa = 0, pb = 0;
        if (c < n_pair) {
            int cc = c;
            while (cc >= P - pa) { cc -= P - pa; ++pa; }
            pb = pa + cc;
        }
        s_pa[c] = pa;
        s_pb[c] = pb;
    }
    for (int i = tid; i < AU_MB * MODAL_MAXP * AU_THREADS; i += AU_THREADS) sM[i] = 0.f;
    __syncthreads();
    const float4* H4 = reinterpret_cast<const float4*>(sH);
    for (int64_t x0 = (int64_t)blockIdx.x * AU_THREADS; x0 < npix; x0 += (int64_t)gridDim.x * AU_THREADS) {
        const int64_t x = x0 + tid;
        const bool in = x < npix;
        for (int mb = 0; mb < nb; ++mb)
            for (int p = 0; p < P; ++p)
                sM[(mb * MODAL_MAXP + p) * AU_THREADS + tid] = in ? maps[((int64_t)(b0 + mb) * P + p) * npix + x] : 0.f;
        float u[AU_MB][MODAL_MAXP];
#pragma unroll
        for (int mb = 0; mb < AU_MB; ++mb)
#pragma unroll
            for (int t = 0; t < MODAL_MAXP; ++t) u[mb][t] = 0.f;
        for (int c0 = 0; c0 < n_pair; c0 += 8) {
            float pv[8];
            int pa[8], pb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c = c0 + i;
                pa[i] = s_pa[c];
                pb[i] = s_pb[c];
                pv[i] = (pm && in && c < n_pair) ? pm[(int64_t)c * npix + x] : 0.f;
            }
#pragma unroll
            for (int mb = 0; mb < AU_MB; ++mb) {
                float y[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    y[i] = (c0 + i < n_pair)
                               ? sM[(mb * MODAL_MAXP + pa[i]) * AU_THREADS + tid] * sM[(mb * MODAL_MAXP + pb[i]) * AU_THREADS + tid] - pv[i]
                               : 0.f;
#pragma unroll
                for (int t = 0; t < MODAL_MAXP; ++t) {
                    const int h = ((mb * MODAL_MAXP + t) * AU_SC + c0) / 4;
                    const float4 h0 = H4[h], h1 = H4[h + 1];
                    u[mb][t] = fmaf(h0.x, y[0], u[mb][t]);
                    u[mb][t] = fmaf(h0.y, y[1], u[mb][t]);
                    u[mb][t] = fmaf(h0.z, y[2], u[mb][t]);
                    u[mb][t] = fmaf(h0.w, y[3], u[mb][t]);
                    u[mb][t] = fmaf(h1.x, y[4], u[mb][t]);
                    u[mb][t] = fmaf(h1.y, y[5], u[mb][t]);
                    u[mb][t] = fmaf(h1.z, y[6], u[mb][t]);
                    u[mb][t] = fmaf(h1.w, y[7], u[mb][t]);
                }
            }
        }
        if (in) {
            const float wx = W[x];
#pragma unroll
            for (int mb = 0; mb < AU_MB; ++mb)
#pragma unroll
                for (int t = 0; t < MODAL_MAXP; ++t)
                    if (mb < nb && t < P) maps[((int64_t)(b0 + mb) * P + t) * npix + x] = wx * u[mb][t];
        }
    }
}

cudaError_t launch_adjoint_u(Plan& pl, const float* /*maps_in*/, int B, const float* hk, int use_linear, float* maps,
                             cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    const size_t smem = (size_t)AU_MB * MODAL_MAXP * (AU_SC + AU_THREADS) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_adjoint_u, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t nblk = (pl.npix + AU_THREADS - 1) / AU_THREADS;
    const int ng = (B + AU_MB - 1) / AU_MB;
    const int64_t want = (152 * 8 + ng - 1) / ng;            // about 8 blocks per SM in total
    dim3 grid((unsigned)std::min<int64_t>(nblk, std::max<int64_t>(want, 152)), ng);
    const float* pm = use_linear ? pl.pair_mean : nullptr;
    k_adjoint_u<<<grid, AU_THREADS, smem, st>>>(pl.P, pl.n_pair, B, pl.npix, hk, pm, pl.W, maps);
    return cudaGetLastError();
}

}  // namespace modal
