// The Monte Carlo pair means in harmonic space (split plans, per-pixel means).
//
// Both places where the per-pixel pair means <c>_x (c = (a <= b)) enter the path are linear
// in a quantity that does not depend on the map values:
//
//   linear term  G_{(c),t} = sum_x W_x <c>_x M_t(x) (Eq. bispectrumest's linear term, read 3 of
//                the readings) is linear in the map's a_lm through M_t = synthesis of f_t a;
//   adjoint      the pair-mean part of the pixel weights, -W_x sum_c h_{t,c} <c>_x, is linear
//                in the adjoint weights h and passes through the rest of the adjoint (ring r2c,
//                transposed Legendre sums, filter), which is linear.
//
// With F_c the adjoint transform of the weighted row W<c> (r2c without ring weights, then the
// transposed Legendre sums without the filter: the same two steps the adjoint applies to the
// pixel weights), the adjoint's image of a field V is c_m sum_t f_t(l) (transform of V_t)[lm],
// and for any field V and map a, sum_x V(x) M_t(x) = sum_lm c_m f_t(l) Re(conj(G_V[lm]) a_lm)
// (c_0 = 1, c_m = 2; Im a_l0 does not enter): the sums are the same finite sums in another
// order.  So
//
//   G_{(c),t}   = sum_l f_t(l) S_c(l),    S_c(l) = sum_m c_m Re(conj(F_c[lm]) a_lm)
//   grad^pm[lm] = c_m sum_c K_c(l) F_c[lm],   K_c(l) = sum_t f_t(l) h_{t,c}
//
// a 136-term sum per coefficient (and per pair and l) in place of a 2176-term sum per pixel.
// F is built once per finalised mean (build_pm_table) and stored l-major, [c][l (l+1)/2 + m],
// so that the loops over m read it contiguously.
#include "modal_internal.cuh"

#include <algorithm>
#include <vector>

namespace modal {

constexpr int AP_MAPS = 32;                       // maps per block of the gradient correction
constexpr int AP_THREADS = 128;                   // m values per block of that kernel
constexpr int LH_MC = 32;                         // m values per shared-memory chunk of the linear term
constexpr int LH_MAPS = 32;                       // maps per block of the linear term
constexpr int LH_THREADS = 288;                   // (maps / 4) x (pairs / 4) register tiles, 8 x 34 at most
constexpr int LH_FPT = (136 * LH_MC + LH_THREADS - 1) / LH_THREADS;     // table values a thread loads per block
constexpr int LH_APT = (LH_MAPS * LH_MC + LH_THREADS - 1) / LH_THREADS;  // a_lm values a thread loads per block

__host__ __device__ inline int64_t av_lidx(int64_t l, int64_t m) { return l * (l + 1) / 2 + m; }

// in[c][x] = W_x <c>_x
__global__ void k_adjpm_weighted(int64_t npix, int n_pair, const float* __restrict__ W, const float* __restrict__ pm,
                                 float* __restrict__ out) {
    const int64_t n = (int64_t)n_pair * npix;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = W[i % npix] * pm[i];
}

// F[c][l (l+1)/2 + m] = in[c][alm index (l, m)]: the l-major copy read by k_adjpm_grad
__global__ void k_adjpm_lmajor(int L, int64_t n_alm, const float2* __restrict__ in, float2* __restrict__ F) {
    const int c = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_alm; i += (int64_t)gridDim.x * blockDim.x) {
        // i = m (2 L + 3 - m) / 2 + (l - m): recover m by the closed form, then correct by one
        int m = (int)((2.0 * L + 3.0 - sqrt((2.0 * L + 3.0) * (2.0 * L + 3.0) - 8.0 * (double)i)) / 2.0);
        m = max(0, min(L, m));
        while (m > 0 && d_alm_index(m, m, L) > i) --m;
        while (m < L && d_alm_index(m + 1, m + 1, L) <= i) ++m;
        const int l = m + (int)(i - d_alm_index(m, m, L));
        F[(int64_t)c * n_alm + av_lidx(l, m)] = in[(int64_t)c * n_alm + i];
    }
}

cudaError_t build_pm_table(Plan& pl, cudaStream_t st) {
    if (!pl.pair_mean) return cudaErrorInvalidValue;
    if (!pl.adj_pm) {
        cudaError_t e = cudaMalloc(&pl.adj_pm, (size_t)pl.n_pair * pl.n_alm * sizeof(float2));
        if (e != cudaSuccess) {
            pl.adj_pm = nullptr;
            return e;
        }
        pl.device_bytes += (size_t)pl.n_pair * pl.n_alm * sizeof(float2);
        ++pl.generation;
        // blocks of k_adjpm_grad: (l, m block) packed as l << 8 | block, largest l first
        std::vector<int> blk;
        for (int l = pl.lmax; l >= 0; --l)
            for (int q = 0; q * AP_THREADS <= l; ++q) blk.push_back(l << 8 | q);
        e = cudaMalloc(&pl.adj_pm_blk, blk.size() * sizeof(int));
        if (e != cudaSuccess) {
            pl.adj_pm_blk = nullptr;
            return e;
        }
        pl.device_bytes += blk.size() * sizeof(int);
        pl.adj_pm_nblk = (int)blk.size();
        e = cudaMemcpy(pl.adj_pm_blk, blk.data(), blk.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    const size_t L1 = pl.lmax + 1;
    float* win = nullptr;
    float2* ut = nullptr;
    float2* fm = nullptr;
    cudaError_t e = cudaMallocAsync(&win, (size_t)pl.n_pair * pl.npix * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&ut, (size_t)pl.n_pair * L1 * 2 * pl.RH * sizeof(float2), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&fm, (size_t)pl.n_pair * pl.n_alm * sizeof(float2), st);
    if (e == cudaSuccess) {
        k_adjpm_weighted<<<pl.nsm * 8, 256, 0, st>>>(pl.npix, pl.n_pair, pl.W, pl.pair_mean, win);
        note_launch(pl);
        e = cudaGetLastError();
    }
    // the adjoint's own transforms without the filter: ring r2c (no ring weights: W is in
    // the rows), then the transposed Legendre sums of each row
    if (e == cudaSuccess) e = launch_ring_r2c(pl, win, pl.n_pair, nullptr, ut, nullptr, st);
    if (e == cudaSuccess) e = launch_legendre_adjoint_simt(pl, ut, pl.n_pair, nullptr, 1, fm, st);
    if (e == cudaSuccess) {
        k_adjpm_lmajor<<<dim3(std::max(1, std::min(pl.nsm * 2, (int)((pl.n_alm + 255) / 256))), pl.n_pair), 256, 0, st>>>(
            pl.lmax, pl.n_alm, fm, pl.adj_pm);
        note_launch(pl);
        e = cudaGetLastError();
    }
    if (win) cudaFreeAsync(win, st);
    if (ut) cudaFreeAsync(ut, st);
    if (fm) cudaFreeAsync(fm, st);
    if (e == cudaSuccess) pl.adj_pm_ready = 1;
    return e;
}

// K[l][b][c] = sum_t f_t(l) h_{b,t,c}
__global__ void k_adjpm_k(int L, int P, int n_pair, int B, const float* __restrict__ filt, const float* __restrict__ hk,
                          float* __restrict__ K) {
    const int64_t n = (int64_t)(L + 1) * B * n_pair;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % n_pair);
        const int b = (int)((i / n_pair) % B);
        const int l = (int)(i / ((int64_t)n_pair * B));
        float s = 0.f;
        for (int t = 0; t < P; ++t) s = fmaf(filt[(int64_t)t * (L + 1) + l], hk[((int64_t)b * P + t) * n_pair + c], s);
        K[i] = s;
    }
}

// T[b][l (l+1)/2 + m] = c_m sum_c K[l][b][c] F_c[lm] for up to AP_MAPS maps per block; block =
// (one l, AP_THREADS consecutive m), the largest l first so that the longest rows start early.
// K[l] sits in shared memory as [c][b], read four maps per broadcast load; T is l-major like
// F, so both the loads of F and the stores of T are contiguous in m.
__global__ void __launch_bounds__(AP_THREADS) k_adjpm_grad(int n_pair, int B, int64_t n_alm, const int* __restrict__ blk_l,
                                                           const float* __restrict__ K, const float2* __restrict__ F,
                                                           float2* __restrict__ T) {
    __shared__ __align__(16) float sK[136 * AP_MAPS];
    const int code = blk_l[blockIdx.x];
    const int l = code >> 8, m = ((code & 0xff) * AP_THREADS) + threadIdx.x;
    const int bg = blockIdx.y * AP_MAPS;
    const int nb = min(AP_MAPS, B - bg);
    for (int i = threadIdx.x; i < n_pair * AP_MAPS; i += blockDim.x) {
        const int c = i / AP_MAPS, b = i % AP_MAPS;
        sK[i] = (b < nb) ? K[((int64_t)l * B + bg + b) * n_pair + c] : 0.f;
    }
    __syncthreads();
    if (m > l) return;
    float2 acc[AP_MAPS];
#pragma unroll
    for (int b = 0; b < AP_MAPS; ++b) acc[b] = make_float2(0.f, 0.f);
    const float2* f = F + av_lidx(l, m);
    // eight pair rows per round: their loads are all in flight before the first is used
    for (int c0 = 0; c0 < n_pair; c0 += 8) {
        float2 v8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v8[i] = (c0 + i < n_pair) ? f[(int64_t)(c0 + i) * n_alm] : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = min(c0 + i, n_pair - 1);       // a row past the end carries v = 0
            const float2 v = v8[i];
            const float4* k4 = reinterpret_cast<const float4*>(sK + c * AP_MAPS);
#pragma unroll
            for (int q = 0; q < AP_MAPS / 4; ++q) {
                const float4 k = k4[q];
                acc[4 * q + 0].x = fmaf(k.x, v.x, acc[4 * q + 0].x); acc[4 * q + 0].y = fmaf(k.x, v.y, acc[4 * q + 0].y);
                acc[4 * q + 1].x = fmaf(k.y, v.x, acc[4 * q + 1].x); acc[4 * q + 1].y = fmaf(k.y, v.y, acc[4 * q + 1].y);
                acc[4 * q + 2].x = fmaf(k.z, v.x, acc[4 * q + 2].x); acc[4 * q + 2].y = fmaf(k.z, v.y, acc[4 * q + 2].y);
                acc[4 * q + 3].x = fmaf(k.w, v.x, acc[4 * q + 3].x); acc[4 * q + 3].y = fmaf(k.w, v.y, acc[4 * q + 3].y);
            }
        }
    }
    const float cm = (m == 0) ? 1.f : 2.f;
    const int64_t li = av_lidx(l, m);
#pragma unroll
    for (int b = 0; b < AP_MAPS; ++b)
        if (b < nb) T[(int64_t)(bg + b) * n_alm + li] = make_float2(cm * acc[b].x, m > 0 ? cm * acc[b].y : 0.f);
}

// grad[b][alm index (l, m)] -= T[b][l (l+1)/2 + m], through 32 x 32 tiles of (l, m) in shared
// memory so that T is read contiguous in m and grad written contiguous in l.
__global__ void __launch_bounds__(256) k_adjpm_apply(int L, int64_t n_alm, const float2* __restrict__ T,
                                                     float2* __restrict__ grad) {
    __shared__ float2 tile[32][33];
    const int nlb = (L + 32) / 32;
    const int lb = blockIdx.x / nlb, mb = blockIdx.x % nlb;
    if (mb > lb) return;
    const int b = blockIdx.y;
    const float2* tb = T + (int64_t)b * n_alm;
    float2* gb = grad + (int64_t)b * n_alm;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    for (int i = ty; i < 32; i += 8) {                     // row l = 32 lb + i, column m = 32 mb + tx
        const int l = 32 * lb + i, m = 32 * mb + tx;
        tile[tx][i] = (l <= L && m <= l) ? tb[av_lidx(l, m)] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {                     // row m = 32 mb + j, column l = 32 lb + tx
        const int m = 32 * mb + j, l = 32 * lb + tx;
        if (l <= L && m <= l) {
            float2* o = gb + d_alm_index(l, m, L);
            const float2 d = tile[j][tx];
            float2 r = *o;
            r.x -= d.x;
            r.y -= d.y;
            *o = r;
        }
    }
}

// K of the adjoint correction and S of the linear term, [lmax+1][chunk][n_pair] / [chunk][n_pair][lmax+1]
size_t adjoint_pm_workspace_bytes(const Plan& pl, int chunk) {
    return pl.prec == MODAL_FP32 ? 0 : (size_t)(pl.lmax + 1) * chunk * pl.n_pair * sizeof(float);
}

cudaError_t launch_adjoint_pm(Plan& pl, int B, const float* hk, float2* grad, float2* scratch, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    if (!pl.adj_pm_ready || !pl.adj_pmk || !pl.adj_pm_blk || B > pl.chunk || pl.n_pair > 136) return cudaErrorInvalidValue;
    const int64_t n = (int64_t)(pl.lmax + 1) * B * pl.n_pair;
    k_adjpm_k<<<(unsigned)std::min<int64_t>((n + 255) / 256, 65535), 256, 0, st>>>(pl.lmax, pl.P, pl.n_pair, B, pl.filt, hk,
                                                                                  pl.adj_pmk);
    note_launch(pl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adjpm_grad<<<dim3(pl.adj_pm_nblk, (B + AP_MAPS - 1) / AP_MAPS), AP_THREADS, 0, st>>>(
        pl.n_pair, B, pl.n_alm, pl.adj_pm_blk, pl.adj_pmk, pl.adj_pm, scratch);
    note_launch(pl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nlb = (pl.lmax + 32) / 32;
    k_adjpm_apply<<<dim3(nlb * nlb, B), 256, 0, st>>>(pl.lmax, pl.n_alm, scratch, grad);
    note_launch(pl);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ linear term
// S[b][c][l] = sum_m c_m Re(conj(F_c[lm]) a_b[lm]) (only Re a at m = 0), one block per l (the
// largest first) and up to LH_MAPS maps; thread = register tile of 4 maps x 4 pairs (pairs
// ct + q n_pair/4, so that a warp reads consecutive rows of the staged table); chunks of
// LH_MC values of m staged in shared memory, each thread's loads of a chunk issued together;
// the per-chunk FP32 sums are added with compensation (sums of up to l_max + 1 terms of
// both signs).
__global__ void __launch_bounds__(LH_THREADS) k_linh_s(int L, int n_pair, int B, int64_t n_alm, const float2* __restrict__ F,
                                                       const float2* __restrict__ alm, float* __restrict__ S) {
    // sF[c][j]: pair c at order m0 + j (a row per pair, as in F; the odd row length keeps the
    // compute reads of 32 different rows on distinct banks)
    __shared__ __align__(16) float2 sF[136][LH_MC + 1];
    __shared__ float2 sA[LH_MAPS][LH_MC + 1];
    const int l = L - (int)blockIdx.x;
    const int bg = blockIdx.y * LH_MAPS;
    const int nb = min(LH_MAPS, B - bg);
    const int nct = (n_pair + 3) / 4, nbt = (nb + 3) / 4;
    const int tid = threadIdx.x;
    const bool active = tid < nbt * nct;
    const int bt = tid / nct, ct = tid % nct;
    float sum[4][4], comp[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sum[i][j] = comp[i][j] = 0.f;
    // the table rows and a_lm of the next block of orders are loaded into registers while
    // the current block is summed (LH_FPT + LH_APT loads in flight per thread)
    float2 pf[LH_FPT], pa[LH_APT];
    auto fetch = [&](int m0) {
#pragma unroll
        for (int u = 0; u < LH_FPT; ++u) {
            const int i = tid + u * LH_THREADS, c = i / LH_MC, m = m0 + i % LH_MC;
            pf[u] = (i < 136 * LH_MC && c < n_pair && m <= l) ? F[(int64_t)c * n_alm + (int64_t)l * (l + 1) / 2 + m]
                                                            : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < LH_APT; ++u) {
            const int i = tid + u * LH_THREADS, b = i / LH_MC, m = m0 + i % LH_MC;
            float2 v = make_float2(0.f, 0.f);
            if (i < LH_MAPS * LH_MC && b < nb && m <= l) {
                v = alm[(int64_t)(bg + b) * n_alm + d_alm_index(l, m, L)];
                if (m == 0) v.y = 0.f;
                else { v.x *= 2.f; v.y *= 2.f; }
            }
            pa[u] = v;
        }
    };
    for (int m0 = 0; m0 <= l; m0 += LH_MC) {
        fetch(m0);
        __syncthreads();
#pragma unroll
        for (int u = 0; u < LH_FPT; ++u) {
            const int i = tid + u * LH_THREADS;
            if (i < 136 * LH_MC) sF[i / LH_MC][i % LH_MC] = pf[u];
        }
#pragma unroll
        for (int u = 0; u < LH_APT; ++u) {
            const int i = tid + u * LH_THREADS;
            if (i < LH_MAPS * LH_MC) sA[i / LH_MC][i % LH_MC] = pa[u];
        }
        __syncthreads();
        if (active) {
            float part[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) part[i][j] = 0.f;
#pragma unroll 4
            for (int j = 0; j < LH_MC; ++j) {
                float2 fv[4];
#pragma unroll
                for (int qc = 0; qc < 4; ++qc) fv[qc] = sF[ct + qc * nct][j];
#pragma unroll
                for (int qb = 0; qb < 4; ++qb) {
                    const float2 av = sA[4 * bt + qb][j];
#pragma unroll
                    for (int qc = 0; qc < 4; ++qc) part[qb][qc] = fmaf(fv[qc].x, av.x, fmaf(fv[qc].y, av.y, part[qb][qc]));
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {           // compensated: sum += part
                    const float y = part[i][j] - comp[i][j];
                    const float t = sum[i][j] + y;
                    comp[i][j] = (t - sum[i][j]) - y;
                    sum[i][j] = t;
                }
        }
    }
    if (!active) return;
#pragma unroll
    for (int qb = 0; qb < 4; ++qb)
#pragma unroll
        for (int qc = 0; qc < 4; ++qc) {
            const int b = 4 * bt + qb, c = ct + qc * nct;
            if (b < nb && c < n_pair) S[((int64_t)(bg + b) * n_pair + c) * (L + 1) + l] = sum[qb][qc];
        }
}

// lin[c][b P + t] = sum_l f_t(l) S[b][c][l] (the layout k_beta_finalize reads, one K split).
// Blocks of 32 values of l are summed in FP32 arithmetic without losing the accuracy of an
// FP64 sum: each product's rounding error is recovered exactly by an FMA and each
// addition's by Knuth's two-sum, the errors are added up beside the sum, and every block
// goes to an FP64 accumulator.  (FP64 throughput on sm_103a is near 1 TF/s; a plain FP64
// chain per output took 0.84 ms at l_max = 2000, 32 maps.)
__global__ void k_linh_g(int L, int P, int n_pair, int B, const float* __restrict__ filt, const float* __restrict__ S,
                         double* __restrict__ lin) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * n_pair * P) return;
    const int t = i % P, bc = i / P, c = bc % n_pair, b = bc / n_pair;
    const float* srow = S + ((int64_t)b * n_pair + c) * (L + 1);
    const float* frow = filt + (int64_t)t * (L + 1);
    double acc = 0.0;
    for (int l0 = 0; l0 <= L; l0 += 32) {
        float sum = 0.f, err = 0.f;
        const int l1 = min(L + 1, l0 + 32);
        for (int l = l0; l < l1; ++l) {
            const float f = frow[l], v = srow[l];
            // _rn intrinsics: no operation below may be contracted into an FMA
            const float p = __fmul_rn(f, v);
            const float pe = fmaf(f, v, -p);        // f v - p exactly
            const float s2 = __fadd_rn(sum, p);     // two-sum: sum + p = s2 + se exactly
            const float z = __fsub_rn(s2, sum);
            const float se = __fadd_rn(__fsub_rn(sum, __fsub_rn(s2, z)), __fsub_rn(p, z));
            sum = s2;
            err = __fadd_rn(err, __fadd_rn(se, pe));
        }
        acc += (double)sum + (double)err;
    }
    lin[(int64_t)c * (B * P) + b * P + t] = acc;
}

cudaError_t launch_linear_harmonic(Plan& pl, const float2* alm, int B, double* lin, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    if (!pl.adj_pm_ready || !pl.adj_pmk || B > pl.chunk || pl.n_pair > 136) return cudaErrorInvalidValue;
    k_linh_s<<<dim3(pl.lmax + 1, (B + LH_MAPS - 1) / LH_MAPS), LH_THREADS, 0, st>>>(pl.lmax, pl.n_pair, B, pl.n_alm,
                                                                                  pl.adj_pm, alm, pl.adj_pmk);
    note_launch(pl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n = B * pl.n_pair * pl.P;
    k_linh_g<<<(n + 127) / 128, 128, 0, st>>>(pl.lmax, pl.P, pl.n_pair, B, pl.filt, pl.adj_pmk, lin);
    note_launch(pl);
    return cudaGetLastError();
}

}  // namespace modal
