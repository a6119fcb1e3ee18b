// Ring Fourier transforms in shared memory (power-of-two N = nphi).
//
// Synthesis (c2r):  M(theta, phi_k) = D_0 + 2 Re sum_{m=1}^{lmax} D_m e^{i m phi_k}
// = sum_{m=-lmax}^{lmax} D_m e^{2 pi i m k / N} with D_{-m} = conj(D_m).  The north
// and south rings of one ring pair share one complex transform:
// Z = X_north + i X_south (both Hermitian), z = IDFT(Z), north = Re z, south = Im z.
//
// Analysis (r2c):  U~_m = sum_k U(k) e^{-2 pi i m k / N}, m = 0..lmax, for a pair of
// real rings packed as z = U_north + i U_south; U~_north,m = (Z_m + conj Z_{N-m}) / 2,
// U~_south,m = (Z_m - conj Z_{N-m}) / 2i.  The output is stored per ring pair as
// (U~_north + U~_south, U~_north - U~_south), the even/odd-l combinations the
// transposed Legendre sum consumes.
//
// Both use an in-place Stockham radix-4 (plus one radix-2 stage when log2 N is odd):
// every thread loads its butterfly inputs, the block synchronises, every thread
// stores its outputs.
#include "modal_internal.cuh"

namespace modal {

constexpr int FFT_THREADS = 512;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Stockham passes over `ntr` transforms of length N stored back to back in buf.
// sign = +1: e^{+2 pi i ...} (synthesis); sign = -1: e^{-2 pi i ...} (analysis).
// tw[q] = e^{+2 pi i q / N}.
template <int SIGN>
__device__ void stockham_inplace(float2* buf, int N, int log2N, int ntr, const float2* __restrict__ tw) {
    int Ns = 1, log2Ns = 0;
    if (log2N & 1) {
        // radix-2 stage at Ns = 1: no twiddles
        const int half = N >> 1, lh = log2N - 1;
        for (int base = 0; base < ntr * half; base += FFT_THREADS * 8) {
            float2 v0[8], v1[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = base + threadIdx.x + u * FFT_THREADS;
                if (idx < ntr * half) {
                    const int q = idx >> lh, jj = idx & (half - 1);
                    v0[u] = buf[(q << log2N) + jj];
                    v1[u] = buf[(q << log2N) + jj + half];
                }
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = base + threadIdx.x + u * FFT_THREADS;
                if (idx < ntr * half) {
                    const int q = idx >> lh, jj = idx & (half - 1);
                    buf[(q << log2N) + 2 * jj] = make_float2(v0[u].x + v1[u].x, v0[u].y + v1[u].y);
                    buf[(q << log2N) + 2 * jj + 1] = make_float2(v0[u].x - v1[u].x, v0[u].y - v1[u].y);
                }
            }
            __syncthreads();
        }
        Ns = 2;
        log2Ns = 1;
    }
    const int quarter = N >> 2, lq = log2N - 2;
    for (; Ns < N; Ns <<= 2, log2Ns += 2) {
        const int lstride = log2N - log2Ns - 2;       // twiddle index step for r * k is 2^lstride
        for (int base = 0; base < ntr * quarter; base += FFT_THREADS * 4) {
            float2 v[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = base + threadIdx.x + u * FFT_THREADS;
                if (idx < ntr * quarter) {
                    const int q = idx >> lq, jj = idx & (quarter - 1);
                    const int k = jj & (Ns - 1);
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        float2 x = buf[(q << log2N) + jj + r * quarter];
                        if (r > 0) {
                            float2 w = __ldg(&tw[(r * k) << lstride]);
                            if (SIGN < 0) w.y = -w.y;
                            x = cmul(x, w);
                        }
                        v[u][r] = x;
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = base + threadIdx.x + u * FFT_THREADS;
                if (idx < ntr * quarter) {
                    const int q = idx >> lq, jj = idx & (quarter - 1);
                    const int k = jj & (Ns - 1);
                    const int d = ((jj >> log2Ns) << (log2Ns + 2)) + k;
                    const float2 a0 = make_float2(v[u][0].x + v[u][2].x, v[u][0].y + v[u][2].y);
                    const float2 a1 = make_float2(v[u][0].x - v[u][2].x, v[u][0].y - v[u][2].y);
                    const float2 a2 = make_float2(v[u][1].x + v[u][3].x, v[u][1].y + v[u][3].y);
                    const float2 df = make_float2(v[u][1].x - v[u][3].x, v[u][1].y - v[u][3].y);
                    // a3 = SIGN * i * (v1 - v3)
                    const float2 a3 = (SIGN > 0) ? make_float2(-df.y, df.x) : make_float2(df.y, -df.x);
                    float2* o = buf + (q << log2N) + d;
                    o[0] = make_float2(a0.x + a2.x, a0.y + a2.y);
                    o[Ns] = make_float2(a1.x + a3.x, a1.y + a3.y);
                    o[2 * Ns] = make_float2(a0.x - a2.x, a0.y - a2.y);
                    o[3 * Ns] = make_float2(a1.x - a3.x, a1.y - a3.y);
                }
            }
            __syncthreads();
        }
    }
}

__host__ __device__ inline int fft_rings_per_block(int N) {
    int r = 16384 / N;
    return r < 1 ? 1 : (r > 16 ? 16 : r);
}

// grid: (ceil(R_half / RPB), nmp); nmp = number of (map, p) rows.
// delta layout [nmp][L+1][2][RH]: even (E) and odd (O) Legendre sums per ring pair;
// north = E + O, south = E - O.
__global__ void __launch_bounds__(FFT_THREADS)
k_ring_c2r(int L, int R, int R_half, int RH, int N, int log2N, const float2* __restrict__ delta,
           const float2* __restrict__ tw, float* __restrict__ maps) {
    extern __shared__ float2 buf[];
    const int RPB = fft_rings_per_block(N);
    const int mp = blockIdx.y;
    const int j0 = blockIdx.x * RPB;
    const int ntr = min(RPB, R_half - j0);
    for (int i = threadIdx.x; i < ntr * N; i += FFT_THREADS) buf[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const float2* d = delta + (int64_t)mp * (L + 1) * 2 * RH;
    for (int i = threadIdx.x; i < (L + 1) * ntr; i += FFT_THREADS) {
        const int m = i / ntr, q = i % ntr;
        const float2 e = d[(int64_t)m * 2 * RH + j0 + q];
        const float2 o = d[(int64_t)m * 2 * RH + RH + j0 + q];
        const float2 dn = make_float2(e.x + o.x, e.y + o.y);
        const float2 ds = make_float2(e.x - o.x, e.y - o.y);
        if (m == 0) {
            buf[q * N] = make_float2(dn.x, ds.x);
        } else {
            buf[q * N + m] = make_float2(dn.x - ds.y, dn.y + ds.x);       // X_n + i X_s
            buf[q * N + N - m] = make_float2(dn.x + ds.y, ds.x - dn.y);   // conj(X_n) + i conj(X_s)
        }
    }
    __syncthreads();
    stockham_inplace<+1>(buf, N, log2N, ntr, tw);
    float* out = maps + (int64_t)mp * R * N;
    for (int q = 0; q < ntr; ++q) {
        const int jn = j0 + q, js = R - 1 - jn;
        for (int k = threadIdx.x; k < N; k += FFT_THREADS) {
            const float2 z = buf[q * N + k];
            out[(int64_t)jn * N + k] = z.x;
            if (js != jn) out[(int64_t)js * N + k] = z.y;
        }
    }
}

// grid: (ceil(R_half / RPB), nmp).  ut layout [nmp][L+1][2][RH].
__global__ void __launch_bounds__(FFT_THREADS)
k_ring_r2c(int L, int R, int R_half, int RH, int N, int log2N, const float* __restrict__ maps,
           const float* __restrict__ ring_weight, const float2* __restrict__ tw, float2* __restrict__ ut) {
    extern __shared__ float2 buf[];
    const int RPB = fft_rings_per_block(N);
    const int mp = blockIdx.y;
    const int j0 = blockIdx.x * RPB;
    const int ntr = min(RPB, R_half - j0);
    const float* in = maps + (int64_t)mp * R * N;
    for (int q = 0; q < ntr; ++q) {
        const int jn = j0 + q, js = R - 1 - jn;
        const float wn = ring_weight ? ring_weight[jn] : 1.f;
        const float ws = ring_weight ? ring_weight[js] : 1.f;
        for (int k = threadIdx.x; k < N; k += FFT_THREADS) {
            const float xn = wn * in[(int64_t)jn * N + k];
            const float xs = (js != jn) ? ws * in[(int64_t)js * N + k] : 0.f;
            buf[q * N + k] = make_float2(xn, xs);
        }
    }
    __syncthreads();
    stockham_inplace<-1>(buf, N, log2N, ntr, tw);
    float2* o = ut + (int64_t)mp * (L + 1) * 2 * RH;
    for (int i = threadIdx.x; i < (L + 1) * ntr; i += FFT_THREADS) {
        const int m = i / ntr, q = i % ntr;
        const float2 zm = buf[q * N + m];
        const float2 zc = buf[q * N + ((N - m) & (N - 1))];
        // U~_n = (Z_m + conj Z_{N-m}) / 2 ; U~_s = (Z_m - conj Z_{N-m}) / 2i
        const float2 un = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
        const float2 us = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
        o[((int64_t)m * 2 + 0) * RH + j0 + q] = make_float2(un.x + us.x, un.y + us.y);
        o[((int64_t)m * 2 + 1) * RH + j0 + q] = make_float2(un.x - us.x, un.y - us.y);
    }
}

static int ilog2(int n) {
    int r = 0;
    while ((1 << r) < n) ++r;
    return r;
}

cudaError_t launch_ring_c2r(const Plan& pl, const float2* delta, int nmp, float* maps, cudaStream_t st) {
    if (nmp == 0) return cudaSuccess;
    const int N = pl.nphi, RPB = fft_rings_per_block(N);
    const size_t smem = (size_t)RPB * N * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_ring_c2r, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((pl.R_half + RPB - 1) / RPB, nmp);
    k_ring_c2r<<<grid, FFT_THREADS, smem, st>>>(pl.lmax, pl.nrings, pl.R_half, pl.RH, N, ilog2(N), delta, pl.twiddle,
                                                maps);
    return cudaGetLastError();
}

cudaError_t launch_ring_r2c(const Plan& pl, const float* maps, int nmp, const float* ring_weight, float2* ut,
                            cudaStream_t st) {
    if (nmp == 0) return cudaSuccess;
    const int N = pl.nphi, RPB = fft_rings_per_block(N);
    const size_t smem = (size_t)RPB * N * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_ring_r2c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((pl.R_half + RPB - 1) / RPB, nmp);
    k_ring_r2c<<<grid, FFT_THREADS, smem, st>>>(pl.lmax, pl.nrings, pl.R_half, pl.RH, N, ilog2(N), maps, ring_weight,
                                                pl.twiddle, ut);
    return cudaGetLastError();
}

}  // namespace modal
