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
    note_launch(pl);
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
    note_launch(pl);
    return cudaGetLastError();
}

// Blocked right-looking Cholesky of the lower triangle of A (row-major n x n), 32-column
// panels: (1) the diagonal block is factored in shared memory by one CTA, (2) the rows
// below it are solved against it, (3) the trailing lower triangle is updated by a grid of
// 32 x 32 tiles.  On a pivot <= 0 (or NaN) MODAL_DEVERR_NOTPD is set and every later
// launch of the factorisation returns at once.
constexpr int CH_NB = 32;

__global__ void __launch_bounds__(CH_NB * CH_NB) k_chol_diag(int n, int k0, double* __restrict__ A, int* __restrict__ err) {
    __shared__ double s[CH_NB][CH_NB + 1];
    __shared__ int bad;
    if (*err & MODAL_DEVERR_NOTPD) return;
    const int tx = threadIdx.x % CH_NB, ty = threadIdx.x / CH_NB;
    const int kn = min(CH_NB, n - k0);
    if (ty < kn && tx < kn) s[ty][tx] = A[(int64_t)(k0 + ty) * n + k0 + tx];
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < kn; ++k) {
        if (threadIdx.x == 0) {
            const double d = s[k][k];
            if (!(d > 0.0)) {
                bad = 1;
                atomicOr(err, MODAL_DEVERR_NOTPD);
            } else {
                s[k][k] = sqrt(d);
            }
        }
        __syncthreads();
        if (bad) return;
        if (ty == 0 && tx > k && tx < kn) s[tx][k] /= s[k][k];
        __syncthreads();
        if (tx > k && ty > k && tx <= ty && ty < kn) s[ty][tx] -= s[ty][k] * s[tx][k];
        __syncthreads();
    }
    if (ty < kn && tx <= ty) A[(int64_t)(k0 + ty) * n + k0 + tx] = s[ty][tx];
}

// Rows i >= k0 + 32 of the panel: solve x L11^T = a for x (one 32-thread warp per row).
__global__ void __launch_bounds__(256) k_chol_panel(int n, int k0, double* __restrict__ A, const int* __restrict__ err) {
    __shared__ double L11[CH_NB][CH_NB + 1];
    if (*err & MODAL_DEVERR_NOTPD) return;
    const int kn = CH_NB;                                   // panel rows exist only below a full block
    for (int i = threadIdx.x; i < CH_NB * CH_NB; i += blockDim.x) {
        const int r = i / CH_NB, c = i % CH_NB;
        L11[r][c] = (c <= r) ? A[(int64_t)(k0 + r) * n + k0 + c] : 0.0;
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int row = k0 + kn + blockIdx.x * 8 + warp;
    if (row >= n) return;
    double* a = A + (int64_t)row * n + k0;
    double x = a[lane];
    for (int j = 0; j < kn; ++j) {
        // x_j = (a_j - sum_{i<j} x_i L_ji) / L_jj: lanes > j subtract lane j's finished value
        const double xj = __shfl_sync(0xffffffffu, x, j) / L11[j][j];
        if (lane == j) x = xj;
        if (lane > j) x -= xj * L11[lane][j];
    }
    a[lane] = x;
}

// Trailing update A22 -= A21 A21^T on 32 x 32 tiles (rb >= cb), K = 32.
__global__ void __launch_bounds__(256) k_chol_update(int n, int k0, double* __restrict__ A, const int* __restrict__ err) {
    __shared__ double Ar[CH_NB][CH_NB + 1], Ac[CH_NB][CH_NB + 1];
    if (*err & MODAL_DEVERR_NOTPD) return;
    const int nt = (n - k0 - CH_NB + CH_NB - 1) / CH_NB;
    // blockIdx.x enumerates the lower triangle of tiles: (rb, cb), cb <= rb
    int rb = 0, rem = blockIdx.x;
    while (rem > rb) { rem -= rb + 1; ++rb; }
    const int cb = rem;
    if (rb >= nt) return;
    const int r0 = k0 + CH_NB + rb * CH_NB, c0 = k0 + CH_NB + cb * CH_NB;
    for (int i = threadIdx.x; i < CH_NB * CH_NB; i += blockDim.x) {
        const int r = i / CH_NB, k = i % CH_NB;
        Ar[r][k] = (r0 + r < n) ? A[(int64_t)(r0 + r) * n + k0 + k] : 0.0;
        Ac[r][k] = (c0 + r < n) ? A[(int64_t)(c0 + r) * n + k0 + k] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < CH_NB * CH_NB; i += blockDim.x) {
        const int r = i / CH_NB, c = i % CH_NB;
        if (r0 + r >= n || c0 + c >= n || c0 + c > r0 + r) continue;
        double acc = 0.0;
#pragma unroll 8
        for (int k = 0; k < CH_NB; ++k) acc = fma(Ar[r][k], Ac[c][k], acc);
        A[(int64_t)(r0 + r) * n + c0 + c] -= acc;
    }
}

cudaError_t launch_cholesky(Plan& pl, double* A, int n, cudaStream_t st) {
    for (int k0 = 0; k0 < n; k0 += CH_NB) {
        k_chol_diag<<<1, CH_NB * CH_NB, 0, st>>>(n, k0, A, pl.d_err + 1);
        note_launch(pl);
        const int below = n - k0 - CH_NB;
        if (below > 0) {
            k_chol_panel<<<(below + 7) / 8, 256, 0, st>>>(n, k0, A, pl.d_err + 1);
            note_launch(pl);
            const int nt = (below + CH_NB - 1) / CH_NB;
            k_chol_update<<<nt * (nt + 1) / 2, 256, 0, st>>>(n, k0, A, pl.d_err + 1);
            note_launch(pl);
        }
    }
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
    note_launch(pl);
    return cudaGetLastError();
}

// Back substitution L^T x = y in place (one CTA): after x_i is known every thread updates
// its y_k, k < i, with L_ik (row i of the lower factor).
__global__ void __launch_bounds__(256) k_solve_rhs_t(int n, const double* __restrict__ Lc, double* __restrict__ v) {
    __shared__ double xi;
    for (int i = n - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            xi = v[i] / Lc[(int64_t)i * n + i];
            v[i] = xi;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < i; k += blockDim.x) v[k] -= Lc[(int64_t)i * n + k] * xi;
        __syncthreads();
    }
}

// w = x / norm[0] (one CTA).
__global__ void __launch_bounds__(256) k_scale_by(int n, const double* __restrict__ x, const double* __restrict__ norm,
                                                  double* __restrict__ w) {
    const double inv = 1.0 / norm[0];
    for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = x[i] * inv;
}

cudaError_t launch_fnl_weights(Plan& pl, const double* Lc, int n, double* v, const double* norm, double* w,
                               cudaStream_t st) {
    k_solve_rhs_t<<<1, 256, 0, st>>>(n, Lc, v);
    note_launch(pl);
    k_scale_by<<<1, 256, 0, st>>>(n, v, norm, w);
    note_launch(pl);
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
    note_launch(pl);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- bivector form (Sec. III.B)
// zeta ~ L0 (I + bt bt^T) L0^T with an ideal covariance zeta0 = L0 L0^T.

__global__ void k_transpose(int n, const double* __restrict__ in, double* __restrict__ out) {
    __shared__ double tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = by + k, c = bx + threadIdx.x;
        if (r < n && c < n) tile[k][threadIdx.x] = in[(int64_t)r * n + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = bx + k, c = by + threadIdx.x;
        if (r < n && c < n) out[(int64_t)r * n + c] = tile[threadIdx.x][k];
    }
}

cudaError_t launch_transpose(Plan& pl, int n, const double* in, double* out, cudaStream_t st) {
    dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
    k_transpose<<<grid, block, 0, st>>>(n, in, out);
    note_launch(pl);
    return cudaGetLastError();
}

// Power iteration on the whitened Z (eigenvalues 1 + l_i > 0, so the dominant one is
// the largest): w = Z v, one warp per row.
__global__ void __launch_bounds__(256) k_matvec(int n, const double* __restrict__ Z, const double* __restrict__ v,
                                                double* __restrict__ w) {
    const int row = blockIdx.x * 8 + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (row >= n) return;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s = fma(Z[(int64_t)row * n + j], v[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[row] = s;
}

__device__ __forceinline__ double block_sum256(double x, double* red) {
    red[threadIdx.x] = x;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// One CTA: lam = v.w (the Rayleigh quotient of the unit v), res = |w - lam v|, then v = w / |w|.
// stat = {lam, res}.
__global__ void __launch_bounds__(256) k_normalize(int n, const double* __restrict__ w, double* __restrict__ v,
                                                   double* __restrict__ stat) {
    __shared__ double red[256];
    double s = 0.0, d = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        s = fma(w[i], w[i], s);
        d = fma(v[i], w[i], d);
    }
    const double ww = block_sum256(s, red), lam = block_sum256(d, red);
    double r = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double e = w[i] - lam * v[i];
        r = fma(e, e, r);
    }
    const double rr = block_sum256(r, red);
    if (threadIdx.x == 0) {
        stat[0] = lam;
        stat[1] = sqrt(rr);
    }
    const double inv = ww > 0.0 ? 1.0 / sqrt(ww) : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = w[i] * inv;
}

cudaError_t launch_power_step(Plan& pl, int n, const double* Z, double* v, double* w, double* stat, cudaStream_t st) {
    k_matvec<<<(n + 7) / 8, 256, 0, st>>>(n, Z, v, w);
    note_launch(pl);
    k_normalize<<<1, 256, 0, st>>>(n, w, v, stat);
    note_launch(pl);
    return cudaGetLastError();
}

// rhs = [alpha'; beta'_0; ...] (whitened), bt: out[0] = alpha'^T Z^-1 alpha' and
// out[1 + b] = alpha'^T Z^-1 beta'_b / out[0], Z^-1 = I - bt bt^T / (1 + |bt|^2) (Eq. ic_bivectorinv).
__global__ void __launch_bounds__(256) k_bivector_estimates(int n, int B, const double* __restrict__ rhs,
                                                            const double* __restrict__ bt, double* __restrict__ out) {
    __shared__ double red[256];
    const double* a = rhs;
    double bb = 0.0, ab = 0.0, aa = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        bb = fma(bt[i], bt[i], bb);
        ab = fma(a[i], bt[i], ab);
        aa = fma(a[i], a[i], aa);
    }
    bb = block_sum256(bb, red);
    ab = block_sum256(ab, red);
    aa = block_sum256(aa, red);
    const double norm = aa - ab * ab / (1.0 + bb);
    if (threadIdx.x == 0) out[0] = norm;
    for (int b = 0; b < B; ++b) {
        const double* y = rhs + (int64_t)(b + 1) * n;
        double ay = 0.0, by = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            ay = fma(a[i], y[i], ay);
            by = fma(bt[i], y[i], by);
        }
        ay = block_sum256(ay, red);
        by = block_sum256(by, red);
        if (threadIdx.x == 0) out[1 + b] = (ay - ab * by / (1.0 + bb)) / norm;
    }
}

cudaError_t launch_bivector_estimates(Plan& pl, const double* rhs, int n, int B, const double* bt, double* out,
                                      cudaStream_t st) {
    k_bivector_estimates<<<1, 256, 0, st>>>(n, B, rhs, bt, out);
    note_launch(pl);
    return cudaGetLastError();
}

// x <- Lt^-1 x for the analytic Cholesky factor Lt of I + bt bt^T (Sec. III.B):
// with S_0 = 1, S_i = S_{i-1} + b_i^2, Lt_ii = sqrt(S_i / S_{i-1}) and
// Lt_ik = b_i b_k / sqrt(S_{k-1} S_k) (k < i), forward substitution needs only the running
// sum t_i = sum_{k<i} b_k y_k / sqrt(S_{k-1} S_k): O(n) per vector, one thread each.
__global__ void k_bivector_rotate(int n, int B, const double* __restrict__ bt, double* __restrict__ x) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double* v = x + (int64_t)b * n;
    double S = 1.0, t = 0.0;
    for (int i = 0; i < n; ++i) {
        const double bi = bt[i], Sn = fma(bi, bi, S);
        const double y = (v[i] - bi * t) * sqrt(S / Sn);
        t = fma(bi * y, 1.0 / sqrt(S * Sn), t);
        v[i] = y;
        S = Sn;
    }
}

cudaError_t launch_bivector_rotate(Plan& pl, int n, int B, const double* bt, double* x, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    k_bivector_rotate<<<(B + 63) / 64, 64, 0, st>>>(n, B, bt, x);
    note_launch(pl);
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
