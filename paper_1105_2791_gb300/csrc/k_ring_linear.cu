// Ring-only ("axisymmetric") linear term.  When the weights W_x, the noise and the mask
// depend on the ring alone, the Monte Carlo pair means <M_a M_b>(x) are functions of the
// ring in expectation, and they are kept per ring:
//     <ab>_j = (1 / (N_lin N_phi)) sum_sims sum_k M_a M_b (theta_j, phi_k).
// The linear part of beta then needs only ring sums of the maps, which the m = 0 Legendre
// sums give exactly (sum_k e^{i m phi_k} = 0 for 0 < m < N_phi):
//     G[(ab), (b, c)] = sum_j W_j <ab>_j R_{b,c}(j),   R_{b,c}(j) = N_phi Re D_{b,c,0}(theta_j),
// north ring j: D_0 = E + O, its mirror R-1-j: D_0 = E - O.  For the adjoint the pair-mean
// term of U_t is the per-ring V_{b,t}(j) = sum_c hk[b][t][c] <c>_j, constant on each ring,
// so it is taken off the m = 0 analysis coefficients (k_vring_correct).
#include "modal_internal.cuh"

namespace modal {

__device__ __forceinline__ int rl_pair_lex(int p, int r, int P) { return p * P - (p * (p - 1)) / 2 + (r - p); }

// ring_sum[c][j] += sum_b sum_k M_a M_b (j, k), c = (a <= b) lexicographic.  One CTA per
// ring: each thread sums the products of its longitudes over all maps in FP32 registers,
// then one warp per pair reduces the threads' sums by a fixed shuffle tree (deterministic)
// and adds the result to the FP64 sums.
constexpr int RP_THREADS = 128;

template <int PM>
__global__ void __launch_bounds__(RP_THREADS)
k_pair_ring(int P, int B, int nphi, int64_t npix, int nrings, const float* __restrict__ maps,
            double* __restrict__ ring_sum) {
    constexpr int NPM = PM * (PM + 1) / 2;
    extern __shared__ __align__(16) float rp_red[];          // [NPM][RP_THREADS + 4]
    const int j = blockIdx.x, tid = threadIdx.x;
    float acc[NPM];
#pragma unroll
    for (int c = 0; c < NPM; ++c) acc[c] = 0.f;
    for (int b = 0; b < B; ++b) {
        const float* mb = maps + (int64_t)b * P * npix + (int64_t)j * nphi;
        for (int k = tid; k < nphi; k += RP_THREADS) {
            float v[PM];
#pragma unroll
            for (int p = 0; p < PM; ++p) v[p] = (p < P) ? mb[(int64_t)p * npix + k] : 0.f;
            int c = 0;
#pragma unroll
            for (int p = 0; p < PM; ++p)
#pragma unroll
                for (int r = p; r < PM; ++r) {
                    acc[c] = fmaf(v[p], v[r], acc[c]);
                    ++c;
                }
        }
    }
#pragma unroll
    for (int c = 0; c < NPM; ++c) rp_red[c * (RP_THREADS + 4) + tid] = acc[c];
    __syncthreads();
    // one warp per pair row: four partial sums per lane, then a shuffle tree (FP32, fixed
    // order), stored in FP64
    const int warp = tid / 32, lane = tid % 32;
    for (int c = warp; c < NPM; c += RP_THREADS / 32) {
        const float4 v = *reinterpret_cast<const float4*>(rp_red + c * (RP_THREADS + 4) + 4 * lane);
        float t = (v.x + v.y) + (v.z + v.w);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane != 0) continue;
        int p = 0, cc = c;
        while (cc >= PM - p) { cc -= PM - p; ++p; }
        const int r = p + cc;
        if (r >= P) continue;
        const double s = (double)t;
        ring_sum[(int64_t)rl_pair_lex(p, r, P) * nrings + j] += s;
    }
}

cudaError_t launch_pair_ring(Plan& pl, const float* maps, int B, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    note_launch(pl);
    if (pl.P <= 4) {
        const size_t smem = 10 * (RP_THREADS + 4) * sizeof(float);
        k_pair_ring<4><<<pl.nrings, RP_THREADS, smem, st>>>(pl.P, B, pl.nphi, pl.npix, pl.nrings, maps, pl.ring_sum);
    } else if (pl.P <= 8) {
        const size_t smem = 36 * (RP_THREADS + 4) * sizeof(float);
        k_pair_ring<8><<<pl.nrings, RP_THREADS, smem, st>>>(pl.P, B, pl.nphi, pl.npix, pl.nrings, maps, pl.ring_sum);
    } else {
        const size_t smem = 136 * (RP_THREADS + 4) * sizeof(float);
        cudaError_t e = cudaFuncSetAttribute(k_pair_ring<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_pair_ring<16><<<pl.nrings, RP_THREADS, smem, st>>>(pl.P, B, pl.nphi, pl.npix, pl.nrings, maps, pl.ring_sum);
    }
    return cudaGetLastError();
}

__global__ void k_ring_finalize(int64_t n, double inv, const double* __restrict__ sum, double* __restrict__ mean) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        mean[i] = sum[i] * inv;
}

cudaError_t launch_ring_finalize(Plan& pl, cudaStream_t st) {
    const int64_t n = (int64_t)pl.n_pair * pl.nrings;
    k_ring_finalize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, 1.0 / ((double)pl.n_lin * pl.nphi), pl.ring_sum,
                                                                  pl.ring_mean);
    note_launch(pl);
    return cudaGetLastError();
}

// lin[(c) ncols + b P + s] = sum_j W_j <c>_j R_{b,s}(j), ncols = B P (one split of the
// layout k_beta_finalize reads).  Grid: (ceil(n_pair P / 128), B).
__global__ void k_linear_ring(int P, int n_pair, int B, int L, int R, int R_half, int RH, int nphi,
                              const float2* __restrict__ delta, const float* __restrict__ W,
                              const double* __restrict__ ring_mean, double* __restrict__ lin) {
    const int b = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pair * P) return;
    const int c = i / P, s = i % P;
    const float2* d0 = delta + ((int64_t)(b * P + s) * (L + 1) + 0) * 2 * RH;    // m = 0: [E][RH], [O][RH]
    const double* mc = ring_mean + (int64_t)c * R;
    double acc = 0.0;
    for (int jp = 0; jp < R_half; ++jp) {
        const double e = d0[jp].x, o = d0[RH + jp].x;
        const int jn = jp, js = R - 1 - jp;
        acc += (double)W[(int64_t)jn * nphi] * mc[jn] * (e + o);
        if (js != jn) acc += (double)W[(int64_t)js * nphi] * mc[js] * (e - o);
    }
    lin[(int64_t)c * B * P + b * P + s] = acc * nphi;
}

cudaError_t launch_linear_ring(Plan& pl, int B, double* lin, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    dim3 grid((pl.n_pair * pl.P + 127) / 128, B);
    k_linear_ring<<<grid, 128, 0, st>>>(pl.P, pl.n_pair, B, pl.lmax, pl.nrings, pl.R_half, pl.RH, pl.nphi, pl.delta,
                                         pl.W, pl.ring_mean, lin);
    note_launch(pl);
    return cudaGetLastError();
}

// vring[(b P + t) R + j] = sum_c hk[(b P + t) n_pair + c] <c>_j.  Grid: (ceil(R / 128), B P).
__global__ void k_vring(int n_pair, int R, const float* __restrict__ hk, const double* __restrict__ ring_mean,
                        float* __restrict__ vring) {
    const int row = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= R) return;
    const float* h = hk + (int64_t)row * n_pair;
    double acc = 0.0;
    for (int c = 0; c < n_pair; ++c) acc += (double)h[c] * ring_mean[(int64_t)c * R + j];
    vring[(int64_t)row * R + j] = (float)acc;
}

cudaError_t launch_vring(Plan& pl, const float* hk, int B, float* vring, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    dim3 grid((pl.nrings + 127) / 128, B * pl.P);
    k_vring<<<grid, 128, 0, st>>>(pl.n_pair, pl.nrings, hk, pl.ring_mean, vring);
    note_launch(pl);
    return cudaGetLastError();
}

// Ring mode of the adjoint: U_t = W (u_t - V_t(ring)) with V constant on a ring, so the
// subtraction changes only the m = 0 coefficient of each ring, by nphi W_j V_t(j)
// (sum_k e^{-i m phi_k} = 0 for 0 < m < nphi).  The analysis stores (U~_n + U~_s, U~_n - U~_s)
// per ring pair; the equator has no south ring.  amax (split precisions) is raised to the
// corrected values.
__global__ void k_vring_correct(int P, int nrows, int R, int R_half, int RH, int L, int nphi,
                                const float* __restrict__ vring, const float* __restrict__ W,
                                float2* __restrict__ ut, unsigned* __restrict__ amax) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = blockIdx.y;
    if (q >= R_half || row >= nrows) return;
    const int jn = q, js = R - 1 - q;
    const float* v = vring + (int64_t)row * R;
    const float cn = (float)nphi * W[(int64_t)jn * nphi] * v[jn];
    const float cs = (js != jn) ? (float)nphi * W[(int64_t)js * nphi] * v[js] : 0.f;
    float2* e = ut + (int64_t)row * (L + 1) * 2 * RH + q;     // m = 0: E row, then O row
    float2 ev = e[0], ov = e[RH];
    ev.x -= cn + cs;
    ov.x -= cn - cs;
    e[0] = ev;
    e[RH] = ov;
    if (amax) {
        const float m = fmaxf(fmaxf(fabsf(ev.x), fabsf(ev.y)), fmaxf(fabsf(ov.x), fabsf(ov.y)));
        if (m > 0.f) atomicMax(&amax[row / P], __float_as_uint(m));
    }
}

cudaError_t launch_vring_correct(Plan& pl, const float* vring, int nrows, float2* ut, unsigned* amax, cudaStream_t st) {
    if (nrows == 0) return cudaSuccess;
    dim3 grid((pl.R_half + 127) / 128, nrows);
    k_vring_correct<<<grid, 128, 0, st>>>(pl.P, nrows, pl.nrings, pl.R_half, pl.RH, pl.lmax, pl.nphi, vring, pl.W, ut,
                                          amax);
    note_launch(pl);
    return cudaGetLastError();
}

__global__ void k_ring_mean_float(int64_t n, const double* __restrict__ mean, float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)mean[i];
}

cudaError_t launch_ring_mean_float(Plan& pl, float* out, cudaStream_t st) {
    const int64_t n = (int64_t)pl.n_pair * pl.nrings;
    k_ring_mean_float<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, pl.ring_mean, out);
    note_launch(pl);
    return cudaGetLastError();
}

}  // namespace modal
