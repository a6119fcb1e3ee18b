// Ring Fourier transforms in shared memory (power-of-two N = nphi, 16 <= N <= 8192).
//
// Synthesis (c2r):  M(theta, phi_k) = D_0 + 2 Re sum_{m=1}^{lmax} D_m e^{i m phi_k}
// = sum_{m=-lmax}^{lmax} D_m e^{2 pi i m k / N} with D_{-m} = conj(D_m).  The north
// and south rings of one ring pair share one complex transform:
// Z = X_north + i X_south (both Hermitian), z = IDFT(Z), north = Re z, south = Im z,
// where X_north = E + O and X_south = E - O from the even/odd Legendre sums.
//
// Analysis (r2c):  U~_m = sum_k U(k) e^{-2 pi i m k / N}, m = 0..lmax, for a pair of
// real rings packed as z = U_north + i U_south; U~_north,m = (Z_m + conj Z_{N-m}) / 2,
// U~_south,m = (Z_m - conj Z_{N-m}) / 2i.  The output is stored per ring pair as
// (U~_north + U~_south, U~_north - U~_south), the even/odd-l combinations the
// transposed Legendre sum consumes.
//
// Transform: Stockham autosort passes of radix 16 (a last pass of radix 8, 4 or 2 when
// log2 N is not a multiple of 4).  Every thread owns 16 elements of one transform
// (T = N / 16 threads per transform): it loads them, applies the inter-pass twiddles
// and a radix-R butterfly in registers (16 / R butterflies), and stores them; one
// block-wide sync separates loads from stores.  Shared-memory index i is padded to
// i + i / 16 to spread the strided stores over the banks.  A CTA of 512 threads holds
// 8192 / N transforms (two ring pairs at N = 4096, 70 KB of shared memory), so that two
// CTAs share an SM and one's global loads and stores overlap the other's passes.  The
// synthesis transform's last pass writes the rings and the analysis transform's first
// pass reads them straight from global memory; the E/O rows read by the synthesis and
// the U~ rows written by the analysis are shared with neighbouring CTAs at 32-byte-sector
// granularity, which L2 merges.
#include "modal_internal.cuh"

namespace modal {

constexpr int FFT_THREADS = 512;
constexpr int FFT_ELEMS = 8192;                  // complex elements per CTA (all transforms)
constexpr int FFT_LB = 4;                        // loads batched per thread

__host__ __device__ inline int fft_rings_per_block(int N) { return FFT_ELEMS / N; }
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// The same sums as packed FP32 pairs (one instruction each; a - b as b * (-1) + a, which
// rounds exactly as the subtraction does).
__device__ __forceinline__ float2 cadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
// Butterfly sums of a transform of sign SIGN: the analysis transform (SIGN = -1) runs them
// packed (r2c at l_max = 2000, 32 maps: 11.3 -> 10.3 ms); in the synthesis transform the
// packed form measured slower (c2r 20.4 -> 20.5 ms for two launches), so it keeps scalar sums.
template <int SIGN>
__device__ __forceinline__ float2 bfly_add(float2 a, float2 b) { return SIGN < 0 ? cadd2(a, b) : cadd(a, b); }
template <int SIGN>
__device__ __forceinline__ float2 bfly_sub(float2 a, float2 b) { return SIGN < 0 ? csub2(a, b) : csub(a, b); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// cos and sin of k pi / 8, k = 0..15 (exact values of the 16th roots of unity).
__constant__ float c_cos16[16] = {1.f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                                  0.f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                                  -1.f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                                  0.f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
__constant__ float c_sin16[16] = {0.f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
                                  1.f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                                  0.f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                                  -1.f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f};

// e^{SIGN 2 pi i k / 16}
template <int SIGN>
__device__ __forceinline__ float2 w16(int k) {
    return make_float2(c_cos16[k & 15], SIGN * c_sin16[k & 15]);
}

// In-register DFTs: X_k = sum_n x_n e^{SIGN 2 pi i n k / R}, in place (x[k] <- X_k).
template <int SIGN>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
    const float2 a0 = bfly_add<SIGN>(x0, x2), a1 = bfly_sub<SIGN>(x0, x2), a2 = bfly_add<SIGN>(x1, x3),
                 d = bfly_sub<SIGN>(x1, x3);
    x0 = bfly_add<SIGN>(a0, a2);
    x2 = bfly_sub<SIGN>(a0, a2);
    // x1, x3 = a1 +- SIGN i d: the swap of d's parts is a choice of registers (scalar form)
    if (SIGN > 0) {
        x1 = make_float2(a1.x - d.y, a1.y + d.x);
        x3 = make_float2(a1.x + d.y, a1.y - d.x);
    } else {
        x1 = make_float2(a1.x + d.y, a1.y - d.x);
        x3 = make_float2(a1.x - d.y, a1.y + d.x);
    }
}

template <int SIGN, int R>
__device__ __forceinline__ void dft(float2* x) {
    if (R == 2) {
        const float2 a = x[0], b = x[1];
        x[0] = bfly_add<SIGN>(a, b);
        x[1] = bfly_sub<SIGN>(a, b);
    } else if (R == 4) {
        dft4<SIGN>(x[0], x[1], x[2], x[3]);
    } else if (R == 8) {
        // n = 2 n1 + n2, k = k1 + 4 k2: DFT4 over n1, twiddle W8^(n2 k1), DFT2 over n2
        float2 y[8];
#pragma unroll
        for (int n2 = 0; n2 < 2; ++n2) {
            float2 a = x[n2], b = x[2 + n2], c = x[4 + n2], d = x[6 + n2];
            dft4<SIGN>(a, b, c, d);
            y[n2 * 4 + 0] = a;
            y[n2 * 4 + 1] = (n2 == 0) ? b : cmul(b, w16<SIGN>(2));
            y[n2 * 4 + 2] = (n2 == 0) ? c : cmul(c, w16<SIGN>(4));
            y[n2 * 4 + 3] = (n2 == 0) ? d : cmul(d, w16<SIGN>(6));
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            x[k1] = bfly_add<SIGN>(y[k1], y[4 + k1]);
            x[k1 + 4] = bfly_sub<SIGN>(y[k1], y[4 + k1]);
        }
    } else {
        // R = 16: n = 4 n1 + n2, k = k1 + 4 k2: DFT4 over n1, twiddle W16^(n2 k1), DFT4 over n2
        float2 y[16];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            float2 a = x[n2], b = x[4 + n2], c = x[8 + n2], d = x[12 + n2];
            dft4<SIGN>(a, b, c, d);
            y[n2 * 4 + 0] = a;
            y[n2 * 4 + 1] = (n2 == 0) ? b : cmul(b, w16<SIGN>(n2));
            y[n2 * 4 + 2] = (n2 == 0) ? c : cmul(c, w16<SIGN>(2 * n2));
            y[n2 * 4 + 3] = (n2 == 0) ? d : cmul(d, w16<SIGN>(3 * n2));
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 a = y[k1], b = y[4 + k1], c = y[8 + k1], d = y[12 + k1];
            dft4<SIGN>(a, b, c, d);
            x[k1] = a;
            x[k1 + 4] = b;
            x[k1 + 8] = c;
            x[k1 + 12] = d;
        }
    }
}

// Twiddles e^{SIGN 2 pi i r k / (R NS)}, r = 1..R-1, of one butterfly of a pass.  The
// table holds, per pass with NS > 1 and per k, w_1, w_2, w_3, w_4, w_8 and w_12 (three
// 16-byte blocks of NS entries each, so a warp's loads are contiguous); w_r for r = a + 4 b
// is w_a w_4b, one complex product of two correctly rounded values.
template <int SIGN, int R>
struct PassTwiddles {
    float2 w1, w2, w3, w4, w8, w12;
    __device__ __forceinline__ void load(const float4* __restrict__ tw, int NS, int k) {
        const float4 a = __ldg(&tw[k]);
        w1 = make_float2(a.x, SIGN * a.y);
        w2 = make_float2(a.z, SIGN * a.w);
        if (R > 2) {
            const float4 b = __ldg(&tw[NS + k]);
            w3 = make_float2(b.x, SIGN * b.y);
            w4 = make_float2(b.z, SIGN * b.w);
        }
        if (R > 8) {
            const float4 c = __ldg(&tw[2 * NS + k]);
            w8 = make_float2(c.x, SIGN * c.y);
            w12 = make_float2(c.z, SIGN * c.w);
        }
    }
    // r is a compile-time constant after unrolling, so the selections fold away
    __device__ __forceinline__ float2 get(int r) const {
        const int a = r & 3, b = r >> 2;
        const float2 wa = (a == 1) ? w1 : (a == 2) ? w2 : w3;
        const float2 wb = (b == 1) ? w4 : (b == 2) ? w8 : w12;
        if (a == 0) return wb;
        if (b == 0) return wa;
        return cmul(wa, wb);
    }
};

// Padded shared-memory index of element base + r * STRIDE.  When STRIDE is a multiple of
// 16 the padding of the r-th element is that of `base` plus r * STRIDE / 16, so every
// access of a pass is a per-thread base plus a compile-time offset.
template <int STRIDE>
__device__ __forceinline__ int pad_at(int base, int r) {
    if constexpr (STRIDE % 16 == 0) return pad16(base) + r * (STRIDE + STRIDE / 16);
    else return pad16(base + r * STRIDE);
}

// One Stockham pass of radix R at sub-transform length NS of an N-point transform at
// `buf` (padded indices).  Thread tl (0 <= tl < T = N / 16) handles butterflies
// j = tl + T u, u < 16 / R: it reads elements j + r N / R, applies the twiddles
// e^{SIGN 2 pi i r k / (R NS)} (k = j mod NS), transforms, and writes element r of
// butterfly j to R (j - k) + k + r NS.
template <int SIGN, int R, int N, int NS>
__device__ __forceinline__ void stockham_pass(float2* buf, int tl, const float4* __restrict__ tw) {
    constexpr int NB = 16 / R;                   // butterflies per thread
    constexpr int T = N / 16;
    constexpr int NR = N / R;
    static_assert(NS == 1 ? R == 16 : NS % 16 == 0, "pass shapes of a radix-16-first Stockham FFT");
    float2 v[16];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int j = tl + T * u;
        const int k = j & (NS - 1);
        PassTwiddles<SIGN, R> w;
        if (NS > 1) w.load(tw, NS, k);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 x = buf[pad_at<NR>(j, r)];
            if (r > 0 && NS > 1) x = cmul(x, w.get(r));
            v[u * R + r] = x;
        }
        dft<SIGN, R>(v + u * R);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int j = tl + T * u;
        const int k = j & (NS - 1);
        const int d = R * (j - k) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if constexpr (NS == 1) buf[pad16(d) + r] = v[u * R + r];   // d = 16 j: one padded group
            else buf[pad_at<NS>(d, r)] = v[u * R + r];
        }
    }
    __syncthreads();
}

// Passes: radix 16 while at least 16 remain, then the remainder (8, 4 or 2).  The twiddle
// table holds 3 NS float4 per pass with NS > 1, in pass order (PassTwiddles).
template <int SIGN, int N, int NS>
__device__ __forceinline__ void fft_passes(float2* buf, int tl, const float4* __restrict__ tw) {
    if constexpr (NS < N) {
        constexpr int R = (N / NS >= 16) ? 16 : N / NS;
        stockham_pass<SIGN, R, N, NS>(buf, tl, tw);
        fft_passes<SIGN, N, NS * R>(buf, tl, tw + (NS > 1 ? 3 * NS : 0));
    }
}

// The last pass of an N-point transform (NS = N / R) with its outputs handed to
// store(index, value) instead of shared memory: thread tl holds elements j + r NS of
// butterflies j = tl + T u, so the threads of a warp store consecutive indices.
template <int SIGN, int N, int NS, class Store>
__device__ __forceinline__ void fft_passes_out(float2* buf, int tl, const float4* __restrict__ tw, Store store) {
    constexpr int R = (N / NS >= 16) ? 16 : N / NS;
    if constexpr (NS * R < N) {
        stockham_pass<SIGN, R, N, NS>(buf, tl, tw);
        fft_passes_out<SIGN, N, NS * R>(buf, tl, tw + (NS > 1 ? 3 * NS : 0), store);
    } else {
        constexpr int NB = 16 / R;
        constexpr int T = N / 16;
        float2 v[16];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int j = tl + T * u;
            const int k = j & (NS - 1);
            PassTwiddles<SIGN, R> w;
            if (NS > 1) w.load(tw, NS, k);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 x = buf[pad_at<NS>(j, r)];
                if (r > 0 && NS > 1) x = cmul(x, w.get(r));
                v[u * R + r] = x;
            }
            dft<SIGN, R>(v + u * R);
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int j = tl + T * u;
            const int k = j & (NS - 1);
            const int d = R * (j - k) + k;
#pragma unroll
            for (int r = 0; r < R; ++r) store(d + r * NS, v[u * R + r]);
        }
    }
}

// The first pass (radix 16, NS = 1) with its inputs taken from load(index) instead of
// shared memory (thread tl reads elements tl + r N / 16: consecutive across a warp), then
// the remaining passes in shared memory.
template <int SIGN, int N, class Load>
__device__ __forceinline__ void fft_passes_in(float2* buf, int tl, const float4* __restrict__ tw, Load load) {
    constexpr int T = N / 16;
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = load(tl + r * T);
    dft<SIGN, 16>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[pad16(16 * tl) + r] = v[r];
    __syncthreads();
    fft_passes<SIGN, N, 16>(buf, tl, tw);
}

// Padded transform stride in float2: N + N/16 for the in-transform padding, + 4 so that
// the transforms of one CTA start 8 banks apart (the (m, ring pair) loads and the
// U~ reads, where the ring pair varies fastest, are then free of bank conflicts).
__host__ __device__ constexpr int fft_stride(int N) { return N + (N >> 4) + 4; }

// grid: (ceil(R_half / RPB), nmp); nmp = number of (map, p) rows.
// delta layout [nmp][L+1][2][RH]: even (E) and odd (O) Legendre sums per ring pair;
// north = E + O, south = E - O.
template <int LOG2N>
__global__ void __launch_bounds__(FFT_THREADS, 2)
k_ring_c2r(int L, int R, int R_half, int RH, const float2* __restrict__ delta, const float4* __restrict__ tw,
           float* __restrict__ maps) {
    constexpr int N = 1 << LOG2N;
    constexpr int lgR = 13 - LOG2N;                      // RPB = 2^lgR transforms per CTA
    constexpr int RPB = 1 << lgR;
    constexpr int NP = fft_stride(N);
    constexpr int T = N / 16;
    extern __shared__ float2 buf[];
    const int mp = blockIdx.y;
    const int j0 = blockIdx.x * RPB;
    const int ntr = min(RPB, R_half - j0);
    const int nzero = N - 2 * L - 1;                     // entries L+1 .. N-L-1 stay zero
    for (int i = threadIdx.x; i < RPB * nzero; i += FFT_THREADS) {
        const int q = i / nzero, k = L + 1 + i % nzero;
        buf[q * NP + pad16(k)] = make_float2(0.f, 0.f);
    }
    const float2* d = delta + (int64_t)mp * (L + 1) * 2 * RH + j0;
    // FFT_LB items (m, ring pair) per thread are loaded before any is stored, so that
    // 2 FFT_LB loads per thread are in flight.
    const int nitem = (L + 1) << lgR;
    for (int i0 = threadIdx.x; i0 < nitem; i0 += FFT_LB * FFT_THREADS) {
        float2 e[FFT_LB], o[FFT_LB];
#pragma unroll
        for (int u = 0; u < FFT_LB; ++u) {
            const int i = i0 + u * FFT_THREADS;
            const int m = i >> lgR, q = i & (RPB - 1);
            e[u] = make_float2(0.f, 0.f);
            o[u] = e[u];
            if (i < nitem && q < ntr) {
                const float2* dm = d + (int64_t)m * 2 * RH + q;
                e[u] = dm[0];
                o[u] = dm[RH];
            }
        }
#pragma unroll
        for (int u = 0; u < FFT_LB; ++u) {
            const int i = i0 + u * FFT_THREADS;
            if (i >= nitem) break;
            const int m = i >> lgR, q = i & (RPB - 1);
            const float2 dn = cadd(e[u], o[u]), ds = csub(e[u], o[u]);
            float2* b = buf + q * NP;
            if (m == 0) {
                b[0] = make_float2(dn.x, ds.x);
            } else {
                b[pad16(m)] = make_float2(dn.x - ds.y, dn.y + ds.x);       // X_n + i X_s
                b[pad16(N - m)] = make_float2(dn.x + ds.y, ds.x - dn.y);   // conj(X_n) + i conj(X_s)
            }
        }
    }
    __syncthreads();
    const int q = threadIdx.x / T, tl = threadIdx.x % T;
    // the last pass stores the north (Re) and south (Im) rings straight to global memory
    const int jn = j0 + q, js = R - 1 - jn;
    const bool valid = q < ntr, south = valid && js != jn;
    float* on = maps + ((int64_t)mp * R + (valid ? jn : 0)) * N;
    float* os = maps + ((int64_t)mp * R + (south ? js : 0)) * N;
    fft_passes_out<+1, N, 1>(buf + q * NP, tl, tw, [&](int k, float2 z) {
        if (valid) on[k] = z.x;
        if (south) os[k] = z.y;
    });
}

// grid: (ceil(R_half / RPB), nmp).  ut layout [nmp][L+1][2][RH].  If amax is not null,
// amax[row / P] is raised (atomicMax on the float bits) to the largest |Re| or |Im| this
// CTA writes: with amax cleared beforehand, it ends up as each map's max over all rows.
template <int LOG2N>
__global__ void __launch_bounds__(FFT_THREADS, 2)
k_ring_r2c(int L, int R, int R_half, int RH, int P, const float* __restrict__ maps,
           const float* __restrict__ ring_weight, const float4* __restrict__ tw, float2* __restrict__ ut,
           unsigned* __restrict__ amax) {
    constexpr int N = 1 << LOG2N;
    constexpr int lgR = 13 - LOG2N;
    constexpr int RPB = 1 << lgR;
    constexpr int NP = fft_stride(N);
    constexpr int T = N / 16;
    extern __shared__ float2 buf[];
    const int mp = blockIdx.y;
    const int j0 = blockIdx.x * RPB;
    const int ntr = min(RPB, R_half - j0);
    const int q = threadIdx.x / T, tl = threadIdx.x % T;
    {
        // the first pass reads the two rings of its pair straight from global memory,
        // packed as north + i south and scaled by the ring weights
        const int jn = j0 + q, js = R - 1 - jn;
        const bool valid = q < ntr, south = valid && js != jn;
        const float* in_n = maps + ((int64_t)mp * R + (valid ? jn : 0)) * N;
        const float* in_s = maps + ((int64_t)mp * R + (south ? js : 0)) * N;
        const float wn = (ring_weight && valid) ? ring_weight[jn] : 1.f;
        const float ws = (ring_weight && south) ? ring_weight[js] : 1.f;
        fft_passes_in<-1, N>(buf + q * NP, tl, tw, [&](int k) {
            return make_float2(valid ? wn * __ldg(in_n + k) : 0.f, south ? ws * __ldg(in_s + k) : 0.f);
        });
    }
    float2* o = ut + (int64_t)mp * (L + 1) * 2 * RH + j0;
    const int nout = (L + 1) << lgR;
    float vmax = 0.f;
    for (int i = threadIdx.x; i < nout; i += FFT_THREADS) {
        const int m = i >> lgR, qq = i & (RPB - 1);
        if (qq >= ntr) continue;
        const float2* b = buf + qq * NP;
        const float2 zm = b[pad16(m)];
        const float2 zc = b[pad16((N - m) & (N - 1))];
        // U~_n = (Z_m + conj Z_{N-m}) / 2 ; U~_s = (Z_m - conj Z_{N-m}) / 2i
        const float2 un = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
        const float2 us = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
        const float2 e = cadd2(un, us), od = csub2(un, us);
        o[((int64_t)m * 2 + 0) * RH + qq] = e;
        o[((int64_t)m * 2 + 1) * RH + qq] = od;
        vmax = fmaxf(vmax, fmaxf(fmaxf(fabsf(e.x), fabsf(e.y)), fmaxf(fabsf(od.x), fabsf(od.y))));
    }
    if (amax) {
        for (int off = 16; off > 0; off >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
        if ((threadIdx.x & 31) == 0 && vmax > 0.f) atomicMax(&amax[mp / P], __float_as_uint(vmax));
    }
}

static int ilog2(int n) {
    int r = 0;
    while ((1 << r) < n) ++r;
    return r;
}

static size_t fft_smem(int N) { return (size_t)fft_rings_per_block(N) * fft_stride(N) * sizeof(float2); }

template <int LOG2N>
static cudaError_t c2r_n(const Plan& pl, const float2* delta, int nmp, float* maps, cudaStream_t st) {
    constexpr int N = 1 << LOG2N;
    const size_t smem = fft_smem(N);
    cudaError_t e = cudaFuncSetAttribute(k_ring_c2r<LOG2N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int RPB = fft_rings_per_block(N);
    dim3 grid((pl.R_half + RPB - 1) / RPB, nmp);
    k_ring_c2r<LOG2N><<<grid, FFT_THREADS, smem, st>>>(pl.lmax, pl.nrings, pl.R_half, pl.RH, delta, pl.twiddle, maps);
    note_launch(pl);
    return cudaGetLastError();
}

template <int LOG2N>
static cudaError_t r2c_n(const Plan& pl, const float* maps, int nmp, const float* ring_weight, float2* ut,
                         unsigned* amax, cudaStream_t st) {
    constexpr int N = 1 << LOG2N;
    const size_t smem = fft_smem(N);
    cudaError_t e = cudaFuncSetAttribute(k_ring_r2c<LOG2N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int RPB = fft_rings_per_block(N);
    dim3 grid((pl.R_half + RPB - 1) / RPB, nmp);
    k_ring_r2c<LOG2N><<<grid, FFT_THREADS, smem, st>>>(pl.lmax, pl.nrings, pl.R_half, pl.RH, pl.P, maps,
                                                        ring_weight, pl.twiddle, ut, amax);
    note_launch(pl);
    return cudaGetLastError();
}

cudaError_t launch_ring_c2r(const Plan& pl, const float2* delta, int nmp, float* maps, cudaStream_t st) {
    if (nmp == 0) return cudaSuccess;
    switch (ilog2(pl.nphi)) {
        case 4: return c2r_n<4>(pl, delta, nmp, maps, st);
        case 5: return c2r_n<5>(pl, delta, nmp, maps, st);
        case 6: return c2r_n<6>(pl, delta, nmp, maps, st);
        case 7: return c2r_n<7>(pl, delta, nmp, maps, st);
        case 8: return c2r_n<8>(pl, delta, nmp, maps, st);
        case 9: return c2r_n<9>(pl, delta, nmp, maps, st);
        case 10: return c2r_n<10>(pl, delta, nmp, maps, st);
        case 11: return c2r_n<11>(pl, delta, nmp, maps, st);
        case 12: return c2r_n<12>(pl, delta, nmp, maps, st);
        case 13: return c2r_n<13>(pl, delta, nmp, maps, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ring_r2c(const Plan& pl, const float* maps, int nmp, const float* ring_weight, float2* ut,
                            unsigned* amax, cudaStream_t st) {
    if (nmp == 0) return cudaSuccess;
    switch (ilog2(pl.nphi)) {
        case 4: return r2c_n<4>(pl, maps, nmp, ring_weight, ut, amax, st);
        case 5: return r2c_n<5>(pl, maps, nmp, ring_weight, ut, amax, st);
        case 6: return r2c_n<6>(pl, maps, nmp, ring_weight, ut, amax, st);
        case 7: return r2c_n<7>(pl, maps, nmp, ring_weight, ut, amax, st);
        case 8: return r2c_n<8>(pl, maps, nmp, ring_weight, ut, amax, st);
        case 9: return r2c_n<9>(pl, maps, nmp, ring_weight, ut, amax, st);
        case 10: return r2c_n<10>(pl, maps, nmp, ring_weight, ut, amax, st);
        case 11: return r2c_n<11>(pl, maps, nmp, ring_weight, ut, amax, st);
        case 12: return r2c_n<12>(pl, maps, nmp, ring_weight, ut, amax, st);
        case 13: return r2c_n<13>(pl, maps, nmp, ring_weight, ut, amax, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace modal
