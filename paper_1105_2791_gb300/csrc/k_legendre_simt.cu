// Plain FP32 SIMT Legendre sums (forward and transposed), one thread per ring
// pair (forward) or per multipole l (transposed).
//
// Forward:  D_{b,p,m}(theta) = sum_{l>=m} lambda_lm(theta) f_p(l) a_{b,lm},
// split by the parity of l - m into E (even) and O (odd) so that one table row
// serves the north ring (E + O) and its mirror south ring (E - O), since
// lambda_lm(-mu) = (-1)^{l+m} lambda_lm(mu).  E and O are stored per ring pair
// (delta layout [B][P][lmax+1][2][RH]); the ring FFT combines them.  This is the
// separable evaluation of the filtered maps whose cube gives Eq. bbispect.
#include "modal_internal.cuh"

namespace modal {

template <int PM>
__global__ void __launch_bounds__(128)
k_legendre_simt(int L, int P, int R, int R_half, int RH, const float* __restrict__ lam,
                const float* __restrict__ filt, const float2* __restrict__ alm, int64_t n_alm,
                float2* __restrict__ delta) {
    constexpr int CH = 64;
    __shared__ float2 sa[CH];
    __shared__ __align__(16) float sf[CH][PM];
    const int m = blockIdx.y, b = blockIdx.z;
    const int j = blockIdx.x * 128 + threadIdx.x;
    const int64_t base = d_alm_index(m, m, L);
    const float2* a = alm + (int64_t)b * n_alm + base;
    const bool active = j < R_half;
    const float* lp = lam + base * (int64_t)RH + (active ? j : 0);

    float2 accE[PM], accO[PM];
#pragma unroll
    for (int p = 0; p < PM; ++p) {
        accE[p] = make_float2(0.f, 0.f);
        accO[p] = make_float2(0.f, 0.f);
    }
    for (int l0 = m; l0 <= L; l0 += CH) {
        const int n = min(CH, L + 1 - l0);
        __syncthreads();
        for (int i = threadIdx.x; i < CH; i += 128) sa[i] = (i < n) ? a[l0 - m + i] : make_float2(0.f, 0.f);
        for (int i = threadIdx.x; i < CH * PM; i += 128) {
            const int li = i / PM, p = i % PM;
            sf[li][p] = (li < n && p < P) ? filt[(int64_t)p * (L + 1) + l0 + li] : 0.f;
        }
        __syncthreads();
        if (active) {
            // l0 - m is a multiple of CH (even), so i + u has the parity of u.
            for (int i = 0; i < n; i += 8) {
                float lv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) lv[u] = (i + u < n) ? lp[(int64_t)(l0 - m + i + u) * RH] : 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float2 t = make_float2(lv[u] * sa[i + u].x, lv[u] * sa[i + u].y);
                    float2* acc = (u & 1) ? accO : accE;
                    const float4* f4 = reinterpret_cast<const float4*>(&sf[i + u][0]);
#pragma unroll
                    for (int q = 0; q < PM / 4; ++q) {
                        const float4 f = f4[q];
                        acc[4 * q + 0].x = fmaf(f.x, t.x, acc[4 * q + 0].x);
                        acc[4 * q + 0].y = fmaf(f.x, t.y, acc[4 * q + 0].y);
                        acc[4 * q + 1].x = fmaf(f.y, t.x, acc[4 * q + 1].x);
                        acc[4 * q + 1].y = fmaf(f.y, t.y, acc[4 * q + 1].y);
                        acc[4 * q + 2].x = fmaf(f.z, t.x, acc[4 * q + 2].x);
                        acc[4 * q + 2].y = fmaf(f.z, t.y, acc[4 * q + 2].y);
                        acc[4 * q + 3].x = fmaf(f.w, t.x, acc[4 * q + 3].x);
                        acc[4 * q + 3].y = fmaf(f.w, t.y, acc[4 * q + 3].y);
                    }
                }
            }
        }
    }
    if (!active) return;
#pragma unroll
    for (int p = 0; p < PM; ++p) {
        if (p < P) {
            const int64_t row = ((int64_t)(b * P + p) * (L + 1) + m) * 2 * RH;
            delta[row + j] = accE[p];
            delta[row + RH + j] = accO[p];
        }
    }
}

cudaError_t launch_legendre_simt(const Plan& pl, const float2* alm, int B, float2* delta, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    dim3 grid((pl.R_half + 127) / 128, pl.lmax + 1, B);
    note_launch(pl);
    if (pl.P <= 4)
        k_legendre_simt<4><<<grid, 128, 0, st>>>(pl.lmax, pl.P, pl.nrings, pl.R_half, pl.RH, pl.lam, pl.filt,
                                                 alm, pl.n_alm, delta);
    else if (pl.P <= 8)
        k_legendre_simt<8><<<grid, 128, 0, st>>>(pl.lmax, pl.P, pl.nrings, pl.R_half, pl.RH, pl.lam, pl.filt,
                                                 alm, pl.n_alm, delta);
    else
        k_legendre_simt<16><<<grid, 128, 0, st>>>(pl.lmax, pl.P, pl.nrings, pl.R_half, pl.RH, pl.lam, pl.filt,
                                                  alm, pl.n_alm, delta);
    return cudaGetLastError();
}

// Transposed sums:  G_{b,t,lm} = sum_j lambda_lm(theta_j) U^{par(l-m)}_{b,t,m}(j), where
// U^0 = U_north + U_south and U^1 = U_north - U_south per ring pair (the mirror
// symmetry again).  Output per (b, l, m):
//   rowfilt != NULL:  c_m sum_t rowfilt[t][l] G_t   (adjoint: c_0 = 1, c_m = 2)
//   rowfilt == NULL:  G_0                           (quadrature analysis, nt = 1)
// ut layout: [B][nt][lmax+1][2][RH] complex.
template <int PM>
__global__ void __launch_bounds__(128)
k_legendre_adj_simt(int L, int nt, int R_half, int RH, const float* __restrict__ lam,
                    const float2* __restrict__ ut, const float* __restrict__ rowfilt, int64_t n_alm,
                    float2* __restrict__ out) {
    constexpr int JT = 32;
    __shared__ float sl[128][JT + 1];
    __shared__ float2 su[PM][2][JT + 1];
    const int m = blockIdx.y, b = blockIdx.z;
    const int l0 = m + blockIdx.x * 128;
    if (l0 > L) return;
    const int nl = min(128, L + 1 - l0);
    const int tid = threadIdx.x;
    const int l = l0 + tid;
    const int par = (l - m) & 1;
    const int64_t base = d_alm_index(m, m, L);
    const float* lrow = lam + (base + (l0 - m)) * (int64_t)RH;
    const float2* ub = ut + ((int64_t)b * nt * (L + 1) + m) * 2 * RH;   // + t*(L+1)*2*RH + par*RH + j

    float2 acc[PM];
#pragma unroll
    for (int t = 0; t < PM; ++t) acc[t] = make_float2(0.f, 0.f);

    const int warp = tid >> 5, lane = tid & 31;
    for (int j0 = 0; j0 < R_half; j0 += JT) {
        __syncthreads();
        for (int r = warp; r < 128; r += 4)
            sl[r][lane] = (r < nl && j0 + lane < R_half) ? lrow[(int64_t)r * RH + j0 + lane] : 0.f;
        for (int i = tid; i < PM * 2 * JT; i += 128) {
            const int t = i / (2 * JT), pj = i % (2 * JT), pr = pj / JT, jj = pj % JT;
            su[t][pr][jj] = (t < nt && j0 + jj < R_half)
                                ? ub[((int64_t)t * (L + 1)) * 2 * RH + (int64_t)pr * RH + j0 + jj]
                                : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < JT; ++jj) {
            const float lv = sl[tid][jj];
#pragma unroll
            for (int t = 0; t < PM; ++t) {
                const float2 u = su[t][par][jj];
                acc[t].x = fmaf(lv, u.x, acc[t].x);
                acc[t].y = fmaf(lv, u.y, acc[t].y);
            }
        }
    }
    if (tid >= nl) return;
    float2 r = make_float2(0.f, 0.f);
    if (rowfilt) {
#pragma unroll
        for (int t = 0; t < PM; ++t) {
            if (t < nt) {
                const float f = rowfilt[(int64_t)t * (L + 1) + l];
                r.x = fmaf(f, acc[t].x, r.x);
                r.y = fmaf(f, acc[t].y, r.y);
            }
        }
        const float cm = (m == 0) ? 1.f : 2.f;
        r.x *= cm;
        r.y *= cm;
        if (m == 0) r.y = 0.f;
    } else {
        r = acc[0];
    }
    out[(int64_t)b * n_alm + base + (l - m)] = r;
}

cudaError_t launch_legendre_adjoint_simt(const Plan& pl, const float2* ut, int B, const float* rowfilt,
                                         int nt, float2* out, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    dim3 grid((pl.lmax + 1 + 127) / 128, pl.lmax + 1, B);
    note_launch(pl);
    if (nt <= 4)
        k_legendre_adj_simt<4><<<grid, 128, 0, st>>>(pl.lmax, nt, pl.R_half, pl.RH, pl.lam, ut, rowfilt, pl.n_alm, out);
    else if (nt <= 8)
        k_legendre_adj_simt<8><<<grid, 128, 0, st>>>(pl.lmax, nt, pl.R_half, pl.RH, pl.lam, ut, rowfilt, pl.n_alm, out);
    else
        k_legendre_adj_simt<16><<<grid, 128, 0, st>>>(pl.lmax, nt, pl.R_half, pl.RH, pl.lam, ut, rowfilt, pl.n_alm, out);
    return cudaGetLastError();
}

}  // namespace modal
