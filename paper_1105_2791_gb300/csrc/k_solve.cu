// Monte Carlo covariance and the estimator solve, in FP64 on the GPU.
//   S1 += sum_b beta_b,  S2 += sum_b beta_b beta_b^T                 (Eq. linearterm)
//   zeta = (S2 - S1 S1^T / N) / (N - 1) / 6                           (zeta = <beta beta^T>/6)
//   zeta = L L^T;  alpha' = L^-1 alpha,  beta'_b = L^-1 beta_b        (Eq. Cholrot)
//   fNL_b = alpha'.beta'_b / |alpha'|^2,  sigma^2 = 6 / |alpha'|^2   (Eq. modalest, modalvariance)
#include "modal_internal.cuh"

namespace modal {

__global__ void k_cov_accumulate(int n, int B, const double* __restrict__ beta, double* __restrict__ S1,
                                 double* __restrict__ S2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * n) return;
    const int r = (int)(i / n), c = (int)(i % n);
    double s = 0.0;
    for (int b = 0; b < B; ++b) s = fma(beta[(int64_t)b * n + r], beta[(int64_t)b * n + c], s);
    S2[i] += s;
    if (c == 0) {
        double t = 0.0;
        for (int b = 0; b < B; ++b) t += beta[(int64_t)b * n + r];
        S1[r] += t;
    }
}

cudaError_t launch_cov_accumulate(Plan& pl, const double* beta, int B, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    const int64_t n2 = (int64_t)pl.n_max * pl.n_max;
    k_cov_accumulate<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(pl.n_max, B, beta, pl.S1, pl.S2);
    return cudaGetLastError();
}

__global__ void k_zeta(int n, double N, const double* __restrict__ S1, const double* __restrict__ S2,
                       double* __restrict__ zeta) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * n) return;
    const int r = (int)(i / n), c = (int)(i % n);
    zeta[i] = (S2[i] - S1[r] * S1[c] / N) / (N - 1.0) / 6.0;
}

cudaError_t launch_zeta(Plan& pl, double* zeta, cudaStream_t st) {
    const int64_t n2 = (int64_t)pl.n_max * pl.n_max;
    k_zeta<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(pl.n_max, (double)pl.n_cov, pl.S1, pl.S2, zeta);
    return cudaGetLastError();
}

// Right-looking Cholesky of the lower triangle of A (row-major n x n), one CTA.
// On a pivot <= 0 (or NaN) the factorisation stops and MODAL_DEVERR_NOTPD is set.
__global__ void __launch_bounds__(1024) k_cholesky(int n, double* __restrict__ A, int* __restrict__ err) {
    extern __shared__ double col[];
    __shared__ int bad;
    __shared__ double piv;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double d = A[(int64_t)k * n + k];
            if (!(d > 0.0)) {
                bad = 1;
                atomicOr(err, MODAL_DEVERR_NOTPD);
            } else {
                piv = sqrt(d);
                A[(int64_t)k * n + k] = piv;
            }
        }
        __syncthreads();
        if (bad) return;
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
            const double v = A[(int64_t)i * n + k] / piv;
            A[(int64_t)i * n + k] = v;
            col[i] = v;
        }
        __syncthreads();
        const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
        for (int i = k + 1 + ty; i < n; i += 32) {
            const double ci = col[i];
            double* row = A + (int64_t)i * n;
            for (int j = k + 1 + tx; j <= i; j += 32) row[j] -= ci * col[j];
        }
        __syncthreads();
    }
}

cudaError_t launch_cholesky(Plan& pl, double* A, int n, cudaStream_t st) {
    k_cholesky<<<1, 1024, (size_t)n * sizeof(double), st>>>(n, A, pl.d_err);
    return cudaGetLastError();
}

// Forward substitution L y = v in place for each right-hand side (one CTA per column of
// rhs [nrhs][n]); column-oriented: after y_i is known every thread updates its v_k, k > i.
__global__ void __launch_bounds__(256) k_solve_rhs(int n, const double* __restrict__ Lc, double* __restrict__ rhs) {
    double* v = rhs + (int64_t)blockIdx.x * n;
    __shared__ double yi;
    for (int i = 0; i < n; ++i) {
        if (threadIdx.x == 0) {
            yi = v[i] / Lc[(int64_t)i * n + i];
            v[i] = yi;
        }
        __syncthreads();
        for (int k = i + 1 + threadIdx.x; k < n; k += blockDim.x) v[k] -= Lc[(int64_t)k * n + i] * yi;
        __syncthreads();
    }
}

cudaError_t launch_solve_rhs(Plan& pl, const double* Lc, int n, double* rhs, int nrhs, cudaStream_t st) {
    if (nrhs == 0) return cudaSuccess;
    k_solve_rhs<<<nrhs, 256, 0, st>>>(n, Lc, rhs);
    return cudaGetLastError();
}

// out[0] = |alpha'|^2, out[1 + b] = alpha'.beta'_b / |alpha'|^2; rhs = [alpha'; beta'_0; ...].
__global__ void __launch_bounds__(256) k_estimates(int n, int B, const double* __restrict__ rhs, double* __restrict__ out) {
    __shared__ double red[256];
    __shared__ double norm;
    const double* a = rhs;
    for (int b = -1; b < B; ++b) {
        const double* y = (b < 0) ? rhs : rhs + (int64_t)(b + 1) * n;
        double s = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(a[i], y[i], s);
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (b < 0) {
                norm = red[0];
                out[0] = red[0];
            } else {
                out[1 + b] = red[0] / norm;
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_estimates(Plan& pl, const double* rhs, int n, int B, double* out, cudaStream_t st) {
    k_estimates<<<1, 256, 0, st>>>(n, B, rhs, out);
    return cudaGetLastError();
}

// Bounded wait on a flag that nothing sets: after spin_limit polls the thread records
// MODAL_DEVERR_TIMEOUT and returns (no trap, no fault).
__global__ void k_wait_selftest(int* err, int spin_limit) {
    __shared__ volatile int flag;
    if (threadIdx.x == 0) flag = 0;
    __syncthreads();
    if (threadIdx.x != 0) return;
    int polls = 0;
    while (flag == 0) {
        if (++polls >= spin_limit) {
            atomicOr(err, MODAL_DEVERR_TIMEOUT);
            return;
        }
        __nanosleep(100);
    }
}

cudaError_t launch_wait_selftest(int* d_err, int spin_limit, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(d_err, spin_limit);
    return cudaGetLastError();
}

}  // namespace modal
