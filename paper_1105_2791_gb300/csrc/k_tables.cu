// Legendre tables: lambda_lm(theta_j) by the FP64 three-term recurrence with
// exponent rescaling (normalised associated Legendre functions with the
// Condon-Shortley phase, Y_lm = lambda_lm e^{i m phi}; the Gaunt integral of
// Sec. II is built from these Y_lm), stored as FP32 for the SIMT path and
// re-tiled for the tensor-core path.
#include "modal_internal.cuh"

namespace modal {

__device__ __forceinline__ float emit_scaled(double v, int e) {
    if (e < -1100) return 0.f;
    return (float)ldexp(v, e);
}

// One thread per (ring pair j, order m); the recurrence runs over l = m..lmax.
// lambda = v 2^e with v renormalised by 2^-200 whenever |v| > 2^200, so that
// lambda_mm may underflow FP64 while later lambda_lm stay exact.
__global__ void k_lambda_table(int L, int R_half, int RH, const double* __restrict__ mu,
                               const double* __restrict__ log2c, const double* __restrict__ ca,
                               const double* __restrict__ cb, float* __restrict__ lam) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (j >= RH) return;
    const int64_t base = d_alm_index(m, m, L);
    const int K = L - m + 1;
    float* out = lam + base * (int64_t)RH + j;
    if (j >= R_half) {
        for (int d = 0; d < K; ++d) out[(int64_t)d * RH] = 0.f;
        return;
    }
    const double x = mu[j];
    const double s2 = 1.0 - x * x;
    const double l2 = log2c[m] + (m > 0 ? 0.5 * (double)m * log2(s2) : 0.0);
    int e = (int)floor(l2);
    double v_prev = 0.0;
    double v = ((m & 1) ? -1.0 : 1.0) * exp2(l2 - (double)e);
    out[0] = emit_scaled(v, e);
    for (int d = 1; d < K; ++d) {
        const double a = ca[base + d], b = cb[base + d];
        const double vn = a * (x * v - b * v_prev);
        v_prev = v;
        v = vn;
        if (fabs(v) > 0x1p200) {
            v *= 0x1p-200;
            v_prev *= 0x1p-200;
            e += 200;
        }
        out[(int64_t)d * RH] = emit_scaled(v, e);
    }
}

cudaError_t launch_lambda_table(const Plan& pl, const double* d_mu_north, const double* d_log2c,
                                const double* d_a, const double* d_b, cudaStream_t st) {
    dim3 grid((pl.RH + 127) / 128, pl.lmax + 1);
    k_lambda_table<<<grid, 128, 0, st>>>(pl.lmax, pl.R_half, pl.RH, d_mu_north, d_log2c, d_a, d_b, pl.lam);
    return cudaGetLastError();
}

}  // namespace modal
