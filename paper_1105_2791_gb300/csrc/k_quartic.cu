// Trispectrum modal coefficients (Sec. IV: the B term of the quartic estimator with the
// four-harmonic Gaunt integral, separable R_n = q_p q_r q_s q_u, v_l = 1):
//
//   T_prsu   = sum_x W_x M_p M_r M_s M_u                               (p <= r <= s <= u)
//   tau_prsu = T_prsu - sum_6 H[(ab), (cd)] + K_prsu
//   H[(ab), (cd)] = sum_x W_x <ab>_x M_c M_d        (the six single pairs of the quadruple)
//   K_prsu   = sum_x W_x (<pr><su> + <ps><ru> + <pu><rs>)  (the three pair splits)
//
// with <ab>_x the Monte Carlo pair means of the linear term.  T is a GEMM of the
// weighted pair-product panel U_(pr) = W M_p M_r against the pair-product panel
// Q_(su) = M_s M_u restricted to r <= s, both built in shared memory tile by tile.
// H is a GEMM of the pair-mean panel against Q: per ring when the means are kept per
// ring (H = sum_j W_j <ab>_j RQ_(cd)(j) with the ring sums RQ of the pair products), or
// over all pixels (k_quartic_hpix, FP32 SIMT) when they are kept per pixel.
#include "modal_internal.cuh"

#include <algorithm>
#include <vector>

namespace modal {

// ---------------------------------------------------------------- quartic term
// Warp roles as in the cubic kernel: QT_TX fill threads (one pixel each, values
// prefetched two tiles ahead) build U (colex pairs, row layout [half][pair group][4]) and
// Q (lexicographic pairs over PM modes, row layout [quad][4]); compute threads hold one
// register tile of 8 U pairs x 4 Q pairs and one of `nl` pixel lanes.  Tiles whose pairs
// all have r > s are absent from the tile list.
constexpr int QT_TX = 64;
constexpr int QT_MAXCOMP = 320;
constexpr int QT_THREADS = QT_MAXCOMP + QT_TX;

__device__ __forceinline__ void qt_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void qt_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }

template <int PM>
__global__ void __launch_bounds__(QT_THREADS, 1)
k_quartic(int P, int n_pg, int n_sq, int ntiles, int nl, int ncomp, const int* __restrict__ tiles,
          const int* __restrict__ qidx, int64_t npix, int64_t px_per_cta, const float* __restrict__ maps,
          const float* __restrict__ W, double* __restrict__ partial, int n_quad) {
    extern __shared__ __align__(16) float smem[];
    const int SU = 8 * n_pg + 4, SQ = 4 * n_sq + 4;
    const int stage_floats = QT_TX * (SU + SQ);
    const int b = blockIdx.y;
    const int tid = threadIdx.x;
    const int nthr = ncomp + QT_TX;
    const int64_t x_begin = (int64_t)blockIdx.x * px_per_cta;
    const int64_t x_end = min(npix, x_begin + px_per_cta);
    const int nch = (x_end > x_begin) ? (int)((x_end - x_begin + QT_TX - 1) / QT_TX) : 0;
    const float* mb = maps + (int64_t)b * P * npix;

    // Per-stage FP32 sums are added to acc with a compensation term (Kahan): the quartic
    // sum is a small difference of large Monte Carlo terms once they are subtracted, so
    // the running sum over a CTA's pixels must not drift by more than a few ulp.
    float acc[32], comp[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) acc[e] = comp[e] = 0.f;
    const int tile = tid % ntiles, lane = tid / ntiles;
    auto kahan = [&](int e, float v) {
        const float y = v - comp[e];
        const float t = acc[e] + y;
        comp[e] = (t - acc[e]) - y;
        acc[e] = t;
    };

    if (tid >= ncomp) {
        // ------------------------------------------------ fill warps
        const int xl = tid - ncomp;
        float cur[PM + 1], n1[PM + 1], n2[PM + 1];
        auto load = [&](float* v, int k) {
            const int64_t x = x_begin + (int64_t)k * QT_TX + xl;
            const bool in = k < nch && x < x_end;
#pragma unroll
            for (int p = 0; p < PM; ++p) v[p] = (in && p < P) ? mb[(int64_t)p * npix + x] : 0.f;
            v[PM] = in ? W[x] : 0.f;
        };
        load(cur, 0);
        load(n1, 1);
        const int hoff = 4 * n_pg;
        constexpr int NPR = PM * (PM + 1) / 2;
        for (int k = 0; k < nch; ++k) {
            load(n2, k + 2);
            const int s = k & 1;
            if (k >= 2) qt_sync(3 + s, nthr);
            float* sU = smem + s * stage_floats + xl * SU;
            float* sQ = smem + s * stage_floats + QT_TX * SU + xl * SQ;
            float wm[PM];
#pragma unroll
            for (int p = 0; p < PM; ++p) wm[p] = cur[PM] * cur[p];
            float st[4];
            // U: colex pairs c = r (r + 1) / 2 + p
#pragma unroll
            for (int r = 0; r < PM; ++r)
#pragma unroll
                for (int p = 0; p <= r; ++p) {
                    const int c = r * (r + 1) / 2 + p;
                    st[c & 3] = wm[p] * cur[r];
                    if ((c & 3) == 3 && c < 8 * n_pg) {
                        const int k4 = c >> 2;
                        *reinterpret_cast<float4*>(sU + (k4 & 1) * hoff + (k4 >> 1) * 4) =
                            make_float4(st[0], st[1], st[2], st[3]);
                    }
                }
            if ((NPR & 3) != 0) {
                const int c0 = NPR & ~3;
#pragma unroll
                for (int i = (NPR & 3); i < 4; ++i) st[i] = 0.f;
                if (c0 < 8 * n_pg) {
                    const int k4 = c0 >> 2;
                    *reinterpret_cast<float4*>(sU + (k4 & 1) * hoff + (k4 >> 1) * 4) =
                        make_float4(st[0], st[1], st[2], st[3]);
                }
            }
            for (int c0 = (NPR + 3) & ~3; c0 < 8 * n_pg; c0 += 4) {
                const int k4 = c0 >> 2;
                *reinterpret_cast<float4*>(sU + (k4 & 1) * hoff + (k4 >> 1) * 4) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            // Q: lexicographic pairs d = s PM - s (s - 1) / 2 + (u - s)
#pragma unroll
            for (int s2 = 0; s2 < PM; ++s2)
#pragma unroll
                for (int u = s2; u < PM; ++u) {
                    const int d = s2 * PM - (s2 * (s2 - 1)) / 2 + (u - s2);
                    st[d & 3] = cur[s2] * cur[u];
                    if ((d & 3) == 3) *reinterpret_cast<float4*>(sQ + (d >> 2) * 4) = make_float4(st[0], st[1], st[2], st[3]);
                }
            if ((NPR & 3) != 0) {
#pragma unroll
                for (int i = (NPR & 3); i < 4; ++i) st[i] = 0.f;
                *reinterpret_cast<float4*>(sQ + (NPR >> 2) * 4) = make_float4(st[0], st[1], st[2], st[3]);
            }
            qt_arrive(1 + s, nthr);
#pragma unroll
            for (int p = 0; p <= PM; ++p) {
                cur[p] = n1[p];
                n1[p] = n2[p];
            }
        }
    } else {
        // ------------------------------------------------ compute warps
        const bool computes = lane < nl;
        const int tpk = computes ? tiles[tile] : 0;
        const int pg = tpk & 0xff, sq = tpk >> 8;
        const int hoff = 4 * n_pg;
        for (int k = 0; k < nch; ++k) {
            const int s = k & 1;
            qt_sync(1 + s, nthr);
            if (computes) {
                const float* sU = smem + s * stage_floats;
                const float* sQ = sU + QT_TX * SU;
                float2 tmp2[4][4];
#pragma unroll
                for (int ip = 0; ip < 4; ++ip)
#pragma unroll
                    for (int q = 0; q < 4; ++q) tmp2[ip][q] = make_float2(0.f, 0.f);
#pragma unroll 2
                for (int xi = lane; xi < QT_TX; xi += nl) {
                    const float4 u0 = *reinterpret_cast<const float4*>(sU + xi * SU + pg * 4);
                    const float4 u1 = *reinterpret_cast<const float4*>(sU + xi * SU + hoff + pg * 4);
                    const float4 qv = *reinterpret_cast<const float4*>(sQ + xi * SQ + sq * 4);
                    const float2 u2[4] = {make_float2(u0.x, u0.y), make_float2(u0.z, u0.w), make_float2(u1.x, u1.y),
                                          make_float2(u1.z, u1.w)};
                    const float2 q2[4] = {make_float2(qv.x, qv.x), make_float2(qv.y, qv.y), make_float2(qv.z, qv.z),
                                          make_float2(qv.w, qv.w)};
#pragma unroll
                    for (int ip = 0; ip < 4; ++ip)
#pragma unroll
                        for (int q = 0; q < 4; ++q) tmp2[ip][q] = __ffma2_rn(u2[ip], q2[q], tmp2[ip][q]);
                }
#pragma unroll
                for (int ip = 0; ip < 4; ++ip)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        kahan((2 * ip) * 4 + q, tmp2[ip][q].x);
                        kahan((2 * ip + 1) * 4 + q, tmp2[ip][q].y);
                    }
            }
            if (k + 2 < nch) qt_arrive(3 + s, nthr);
        }
    }
    __syncthreads();
    float* red = smem;   // [nl][ntiles][32]
    if (tid < ncomp && lane < nl) {
#pragma unroll
        for (int e = 0; e < 32; ++e) red[(lane * ntiles + tile) * 32 + e] = acc[e];
    }
    __syncthreads();
    for (int i = tid; i < ntiles * 32; i += nthr) {
        const int t = i / 32, e = i % 32;
        float v = 0.f;
        for (int ln = 0; ln < nl; ++ln) v += red[(ln * ntiles + t) * 32 + e];
        const int tp = tiles[t];
        const int c = (tp & 0xff) * 8 + e / 4, d = (tp >> 8) * 4 + e % 4;
        const int n = qidx[c * 4 * n_sq + d];
        if (n >= 0) partial[((int64_t)b * gridDim.x + blockIdx.x) * n_quad + n] = (double)v;
    }
}

static int quartic_pm(int P) { return P <= 4 ? 4 : (P <= 8 ? 8 : 16); }
static int quartic_lanes(const Plan& pl) { return std::max(1, std::min(8, QT_MAXCOMP / pl.qt.ntiles)); }

static size_t quartic_smem(const Plan& pl) {
    const size_t SU = 8 * (size_t)pl.n_pg + 4, SQ = 4 * (size_t)pl.qt.n_sq + 4;
    const size_t tilebuf = 2 * (size_t)QT_TX * (SU + SQ) * 4;
    const size_t redbuf = (size_t)quartic_lanes(pl) * pl.qt.ntiles * 32 * 4;
    return std::max(tilebuf, redbuf);
}

template <int PM>
static cudaError_t launch_quartic_pm(Plan& pl, const float* maps, int B, double* partial, cudaStream_t st) {
    const int nl = quartic_lanes(pl);
    const int ncomp = ((pl.qt.ntiles * nl + 31) / 32) * 32;
    const size_t smem = quartic_smem(pl);
    cudaError_t e = cudaFuncSetAttribute(k_quartic<PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t ppc = ((pl.npix + pl.cubic_ctas - 1) / pl.cubic_ctas + QT_TX - 1) / QT_TX * QT_TX;
    dim3 grid(pl.cubic_ctas, B);
    k_quartic<PM><<<grid, ncomp + QT_TX, smem, st>>>(pl.P, pl.n_pg, pl.qt.n_sq, pl.qt.ntiles, nl, ncomp, pl.qt.tiles,
                                                     pl.qt.idx, pl.npix, ppc, maps, pl.W, partial, pl.qt.n_quad);
    note_launch(pl);
    return cudaGetLastError();
}

cudaError_t launch_quartic(Plan& pl, const float* maps, int B, double* partial, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    if (pl.qt.ntiles > QT_MAXCOMP) return cudaErrorInvalidValue;
    switch (quartic_pm(pl.P)) {
        case 4: return launch_quartic_pm<4>(pl, maps, B, partial, st);
        case 8: return launch_quartic_pm<8>(pl, maps, B, partial, st);
        default: return launch_quartic_pm<16>(pl, maps, B, partial, st);
    }
}

// Host tables: quadruples (lexicographic), the register tiles and the map from
// (colex pair c, lexicographic PM-pair d) to the quadruple index (or -1).
cudaError_t quartic_tables(Plan& pl) {
    const int P = pl.P, PM = quartic_pm(P);
    const int npr = PM * (PM + 1) / 2;
    pl.qt.n_sq = (npr + 3) / 4;
    std::vector<int> quads;
    std::vector<int> qnum(P * P * P * P, -1);
    int n = 0;
    for (int p = 0; p < P; ++p)
        for (int r = p; r < P; ++r)
            for (int s = r; s < P; ++s)
                for (int u = s; u < P; ++u) {
                    quads.insert(quads.end(), {p, r, s, u});
                    qnum[((p * P + r) * P + s) * P + u] = n++;
                }
    pl.qt.n_quad = n;
    const int rows = 8 * pl.n_pg, cols = 4 * pl.qt.n_sq;
    std::vector<int> cp(rows, -1), cr(rows, -1), ds(cols, -1), du(cols, -1);
    for (int r = 0; r < PM; ++r)
        for (int p = 0; p <= r; ++p) {
            const int c = r * (r + 1) / 2 + p;
            if (c < rows && r < P) { cp[c] = p; cr[c] = r; }
        }
    for (int s = 0; s < PM; ++s)
        for (int u = s; u < PM; ++u) {
            const int d = s * PM - (s * (s - 1)) / 2 + (u - s);
            if (u < P) { ds[d] = s; du[d] = u; }
        }
    std::vector<int> idx((size_t)rows * cols, -1);
    for (int c = 0; c < rows; ++c)
        for (int d = 0; d < cols; ++d)
            if (cp[c] >= 0 && ds[d] >= 0 && cr[c] <= ds[d])
                idx[(size_t)c * cols + d] = qnum[((cp[c] * P + cr[c]) * P + ds[d]) * P + du[d]];
    std::vector<int> tiles;
    for (int g = 0; g < pl.n_pg; ++g)
        for (int q = 0; q < pl.qt.n_sq; ++q) {
            bool any = false;
            for (int e = 0; e < 32 && !any; ++e) any = idx[(size_t)(g * 8 + e / 4) * cols + q * 4 + e % 4] >= 0;
            if (any) tiles.push_back(g | (q << 8));
        }
    pl.qt.ntiles = (int)tiles.size();
    std::vector<int> pa, pb;
    for (int a = 0; a < P; ++a)
        for (int b = a; b < P; ++b) { pa.push_back(a); pb.push_back(b); }
    auto upload = [&](int** dst, const std::vector<int>& v) -> cudaError_t {
        cudaError_t e = cudaMalloc(dst, v.size() * sizeof(int));
        if (e != cudaSuccess) return e;
        pl.device_bytes += v.size() * sizeof(int);
        return cudaMemcpy(*dst, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice);
    };
    cudaError_t e;
    if ((e = upload(&pl.qt.tiles, tiles)) != cudaSuccess) return e;
    if ((e = upload(&pl.qt.idx, idx)) != cudaSuccess) return e;
    if ((e = upload(&pl.qt.modes, quads)) != cudaSuccess) return e;
    if ((e = upload(&pl.qt.pa, pa)) != cudaSuccess) return e;
    return upload(&pl.qt.pb, pb);
}

// ---------------------------------------------------------------- single-pair term
__device__ __forceinline__ int qt_pair_lex(int p, int r, int P) { return p * P - (p * (p - 1)) / 2 + (r - p); }

// Ring sums of the pair products of each map: rq[b][(ab)][j] = sum_k M_a M_b (j, k).
// One CTA per (ring, map); FP32 per-thread sums over the ring's longitudes, then one warp
// per pair reduces them by a fixed shuffle tree; stored in FP64.
constexpr int QR_THREADS = 128;

template <int PM>
__global__ void __launch_bounds__(QR_THREADS)
k_pair_ring_maps(int P, int nphi, int64_t npix, int nrings, int n_pair, const float* __restrict__ maps,
                 double* __restrict__ rq) {
    constexpr int NPM = PM * (PM + 1) / 2;
    extern __shared__ __align__(16) float qr_red[];          // [NPM][QR_THREADS + 4]
    const int j = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    float acc[NPM];
#pragma unroll
    for (int c = 0; c < NPM; ++c) acc[c] = 0.f;
    const float* mb = maps + (int64_t)b * P * npix + (int64_t)j * nphi;
    for (int k = tid; k < nphi; k += QR_THREADS) {
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
#pragma unroll
    for (int c = 0; c < NPM; ++c) qr_red[c * (QR_THREADS + 4) + tid] = acc[c];
    __syncthreads();
    // one warp per pair row: four partial sums per lane, then a shuffle tree (FP32, fixed
    // order), stored in FP64
    const int warp = tid / 32, lane = tid % 32;
    for (int c = warp; c < NPM; c += QR_THREADS / 32) {
        const float4 v = *reinterpret_cast<const float4*>(qr_red + c * (QR_THREADS + 4) + 4 * lane);
        float t = (v.x + v.y) + (v.z + v.w);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane != 0) continue;
        int p = 0, cc = c;
        while (cc >= PM - p) { cc -= PM - p; ++p; }
        const int r = p + cc;
        if (r >= P) continue;
        const double s = (double)t;
        rq[((int64_t)b * n_pair + qt_pair_lex(p, r, P)) * nrings + j] = s;
    }
}

// h[b][(ab)][(cd)] = sum_j W_j <ab>_j rq[b][(cd)][j].  CTA: 8 rows (ab) x all (cd) of
// one map; ring chunks of 32 staged in shared memory.
constexpr int QH_ROWS = 8, QH_J = 32;

__global__ void __launch_bounds__(256)
k_quartic_hring(int n_pair, int nrings, int nphi, const double* __restrict__ rq, const double* __restrict__ mean,
                const float* __restrict__ W, double* __restrict__ h) {
    __shared__ double s_rq[QH_J][137];
    __shared__ double s_m[QH_ROWS][QH_J];
    const int b = blockIdx.y, a0 = blockIdx.x * QH_ROWS, tid = threadIdx.x;
    double acc[QH_ROWS];
#pragma unroll
    for (int i = 0; i < QH_ROWS; ++i) acc[i] = 0.0;
    const double* rb = rq + (int64_t)b * n_pair * nrings;
    for (int j0 = 0; j0 < nrings; j0 += QH_J) {
        for (int i = tid; i < n_pair * QH_J; i += blockDim.x) {
            const int cd = i / QH_J, jj = i % QH_J;
            s_rq[jj][cd] = (j0 + jj < nrings) ? rb[(int64_t)cd * nrings + j0 + jj] : 0.0;
        }
        for (int i = tid; i < QH_ROWS * QH_J; i += blockDim.x) {
            const int r = i / QH_J, jj = i % QH_J;
            const int ab = a0 + r, j = j0 + jj;
            s_m[r][jj] = (ab < n_pair && j < nrings) ? (double)W[(int64_t)j * nphi] * mean[(int64_t)ab * nrings + j] : 0.0;
        }
        __syncthreads();
        if (tid < n_pair) {
            for (int jj = 0; jj < QH_J; ++jj) {
                const double x = s_rq[jj][tid];
#pragma unroll
                for (int r = 0; r < QH_ROWS; ++r) acc[r] = fma(s_m[r][jj], x, acc[r]);
            }
        }
        __syncthreads();
    }
    if (tid < n_pair)
        for (int r = 0; r < QH_ROWS; ++r)
            if (a0 + r < n_pair) h[((int64_t)b * n_pair + a0 + r) * n_pair + tid] = acc[r];
}

// Per-pixel means: out[z][(ab)][b n_pair + (cd)] = sum_{x in split z} W_x <ab>_x M_c M_d,
// a 64 x 64-tiled FP32 GEMM whose B tile is formed from the maps as it is staged; with
// bpanel given, the B rows are bpanel's rows instead (the two-pair term's W <ab> <cd>).
constexpr int QP_TM = 64, QP_TN = 64, QP_TK = 32;

__global__ void __launch_bounds__(256)
k_quartic_hpix(int P, int n_pair, int ncols, int64_t npix, int64_t kchunk, const float* __restrict__ panel,
               const float* __restrict__ W, const float* __restrict__ maps, const int* __restrict__ pa,
               const int* __restrict__ pb, const float* __restrict__ bpanel, double* __restrict__ out) {
    __shared__ __align__(16) float sA[QP_TK][QP_TM + 4];
    __shared__ __align__(16) float sB[QP_TK][QP_TN + 4];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int r0 = blockIdx.x * QP_TM, c0 = blockIdx.y * QP_TN;
    const int64_t k_begin = (int64_t)blockIdx.z * kchunk;
    const int64_t k_end = min(npix, k_begin + kchunk);
    // FP32 sums over 8 K tiles (256 pixels), then FP64
    float acc[4][4] = {};
    double acc64[4][4] = {};
    int tiles_in = 0;
    for (int64_t k0 = k_begin; k0 < k_end; k0 += QP_TK) {
        for (int i = tid; i < QP_TM * QP_TK; i += 256) {
            const int r = i / QP_TK, k = i % QP_TK;
            const int64_t x = k0 + k;
            sA[k][r] = (r0 + r < n_pair && x < k_end) ? panel[(int64_t)(r0 + r) * npix + x] * W[x] : 0.f;
        }
        for (int i = tid; i < QP_TN * QP_TK; i += 256) {
            const int c = i / QP_TK, k = i % QP_TK;
            const int64_t x = k0 + k;
            float v = 0.f;
            if (c0 + c < ncols && x < k_end) {
                if (bpanel) {
                    v = bpanel[(int64_t)(c0 + c) * npix + x];
                } else {
                    const int bm = (c0 + c) / n_pair, cd = (c0 + c) % n_pair;
                    const float* m = maps + (int64_t)bm * P * npix;
                    v = m[(int64_t)pa[cd] * npix + x] * m[(int64_t)pb[cd] * npix + x];
                }
            }
            sB[k][c] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < QP_TK; ++k) {
            const float4 a = *reinterpret_cast<const float4*>(&sA[k][ty * 4]);
            const float4 bb = *reinterpret_cast<const float4*>(&sB[k][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
        if (++tiles_in == 8) {
            tiles_in = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc64[i][j] += (double)acc[i][j];
                    acc[i][j] = 0.f;
                }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + ty * 4 + i, c = c0 + tx * 4 + j;
            if (r < n_pair && c < ncols) out[((int64_t)blockIdx.z * n_pair + r) * ncols + c] = acc64[i][j] + (double)acc[i][j];
        }
}

// Two-pair term.  kmat[z][(ab)][(cd)] = sum_x W_x <ab>_x <cd>_x: per ring
// (sum_j nphi W_j <ab>_j <cd>_j, FP64, one split) or per pixel (k_quartic_hpix against the
// mean panel, one block per K split); then k3[q] = sum_z sum of the three pair splits.
__global__ void k_quartic_kring(int n_pair, int nrings, int nphi, const double* __restrict__ mean,
                                const float* __restrict__ W, double* __restrict__ kmat) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pair * n_pair) return;
    const int ab = i / n_pair, cd = i % n_pair;
    double acc = 0.0;
    for (int j = 0; j < nrings; ++j)
        acc = fma((double)nphi * W[(int64_t)j * nphi] * mean[(int64_t)ab * nrings + j], mean[(int64_t)cd * nrings + j], acc);
    kmat[i] = acc;
}

__global__ void k_quartic_k3(int P, int n_quad, int n_pair, int nsplit, const int* __restrict__ modes,
                             const double* __restrict__ kmat, double* __restrict__ k3) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_quad) return;
    const int p = modes[4 * q], r = modes[4 * q + 1], s = modes[4 * q + 2], u = modes[4 * q + 3];
    const int m[3][2] = {{qt_pair_lex(p, r, P), qt_pair_lex(s, u, P)},
                         {qt_pair_lex(p, s, P), qt_pair_lex(r, u, P)},
                         {qt_pair_lex(p, u, P), qt_pair_lex(r, s, P)}};
    double acc = 0.0;
    for (int z = 0; z < nsplit; ++z)
        for (int i = 0; i < 3; ++i) acc += kmat[((int64_t)z * n_pair + m[i][0]) * n_pair + m[i][1]];
    k3[q] = acc;
}

// tau[b][q] = sum_cta partial - (six H terms) + k3[q].  h layout: [splits][n_pair][hcols]
// with column b hstride + (cd) (ring: hcols = n_pair, hstride = 0 and a per-map block
// of n_pair^2; pixel: hcols = B n_pair, hstride = n_pair).
__global__ void k_quartic_finalize(int P, int n_quad, int B, int nctas, int use_linear, int n_pair, int hsplits,
                                   int64_t hmap, int hcols, int hstride, const int* __restrict__ modes,
                                   const double* __restrict__ partial, const double* __restrict__ h,
                                   const double* __restrict__ k3, double* __restrict__ tau) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * n_quad) return;
    const int b = i / n_quad, q = i % n_quad;
    double v = 0.0;
    for (int c = 0; c < nctas; ++c) v += partial[((int64_t)b * nctas + c) * n_quad + q];
    if (use_linear) {
        const int id[4] = {modes[4 * q], modes[4 * q + 1], modes[4 * q + 2], modes[4 * q + 3]};
        const int sp[6][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}, {1, 2, 0, 3}, {1, 3, 0, 2}, {2, 3, 0, 1}};
        double l = 0.0;
        for (int z = 0; z < hsplits; ++z) {
            const double* hz = h + (int64_t)z * n_pair * hcols + (int64_t)b * hmap;
            for (int t = 0; t < 6; ++t) {
                const int ab = qt_pair_lex(id[sp[t][0]], id[sp[t][1]], P);
                const int cd = qt_pair_lex(id[sp[t][2]], id[sp[t][3]], P);
                l += hz[(int64_t)ab * hcols + b * hstride + cd];
            }
        }
        v += k3[q] - l;
    }
    tau[(int64_t)b * n_quad + q] = v;
}

cudaError_t launch_quartic_linear(Plan& pl, const float* maps, int B, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    const int np = pl.n_pair;
    if (pl.lin_mode == MODAL_LINEAR_RING) {
        const int PM = quartic_pm(pl.P);
        const int npm = PM * (PM + 1) / 2;
        const size_t smem = (size_t)npm * (QR_THREADS + 4) * sizeof(float);
        dim3 grid(pl.nrings, B);
        cudaError_t e;
        if (PM == 4) {
            k_pair_ring_maps<4><<<grid, QR_THREADS, smem, st>>>(pl.P, pl.nphi, pl.npix, pl.nrings, np, maps, pl.qt.rq);
        } else if (PM == 8) {
            k_pair_ring_maps<8><<<grid, QR_THREADS, smem, st>>>(pl.P, pl.nphi, pl.npix, pl.nrings, np, maps, pl.qt.rq);
        } else {
            if ((e = cudaFuncSetAttribute(k_pair_ring_maps<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
                return e;
            k_pair_ring_maps<16><<<grid, QR_THREADS, smem, st>>>(pl.P, pl.nphi, pl.npix, pl.nrings, np, maps, pl.qt.rq);
        }
        note_launch(pl);
        k_quartic_hring<<<dim3((np + QH_ROWS - 1) / QH_ROWS, B), 256, 0, st>>>(np, pl.nrings, pl.nphi, pl.qt.rq,
                                                                               pl.ring_mean, pl.W, pl.qt.h);
        note_launch(pl);
    } else {
        const int ncols = B * np;
        const int64_t kchunk = ((pl.npix + pl.lin_ksplit - 1) / pl.lin_ksplit + QP_TK - 1) / QP_TK * QP_TK;
        dim3 grid((np + QP_TM - 1) / QP_TM, (ncols + QP_TN - 1) / QP_TN, pl.lin_ksplit);
        k_quartic_hpix<<<grid, 256, 0, st>>>(pl.P, np, ncols, pl.npix, kchunk, pl.pair_mean, pl.W, maps, pl.qt.pa,
                                             pl.qt.pb, nullptr, pl.qt.h);
        note_launch(pl);
    }
    return cudaGetLastError();
}

cudaError_t launch_quartic_k3(Plan& pl, cudaStream_t st) {
    const int np = pl.n_pair;
    int nsplit = 1;
    if (pl.lin_mode == MODAL_LINEAR_RING) {
        k_quartic_kring<<<(np * np + 255) / 256, 256, 0, st>>>(np, pl.nrings, pl.nphi, pl.ring_mean, pl.W, pl.qt.kmat);
    } else {
        nsplit = pl.lin_ksplit;
        const int64_t kchunk = ((pl.npix + nsplit - 1) / nsplit + QP_TK - 1) / QP_TK * QP_TK;
        dim3 grid((np + QP_TM - 1) / QP_TM, (np + QP_TN - 1) / QP_TN, nsplit);
        k_quartic_hpix<<<grid, 256, 0, st>>>(pl.P, np, np, pl.npix, kchunk, pl.pair_mean, pl.W, nullptr, nullptr,
                                             nullptr, pl.pair_mean, pl.qt.kmat);
    }
    note_launch(pl);
    k_quartic_k3<<<(pl.qt.n_quad + 255) / 256, 256, 0, st>>>(pl.P, pl.qt.n_quad, np, nsplit, pl.qt.modes, pl.qt.kmat,
                                                             pl.qt.k3);
    note_launch(pl);
    return cudaGetLastError();
}

cudaError_t launch_quartic_finalize(Plan& pl, int B, int use_linear, double* tau, cudaStream_t st) {
    const bool ring = pl.lin_mode == MODAL_LINEAR_RING;
    const int np = pl.n_pair;
    const int hsplits = ring ? 1 : pl.lin_ksplit;
    const int64_t hmap = ring ? (int64_t)np * np : 0;
    const int hcols = ring ? np : B * np;
    const int hstride = ring ? 0 : np;
    const int n = B * pl.qt.n_quad;
    k_quartic_finalize<<<(n + 255) / 256, 256, 0, st>>>(pl.P, pl.qt.n_quad, B, pl.cubic_ctas, use_linear, np, hsplits,
                                                        hmap, hcols, hstride, pl.qt.modes, pl.qt.partial, pl.qt.h,
                                                        pl.qt.k3, tau);
    note_launch(pl);
    return cudaGetLastError();
}

}  // namespace modal
