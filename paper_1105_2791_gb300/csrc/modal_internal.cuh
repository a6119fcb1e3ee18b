// Internal declarations shared by the translation units of the modal library.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/modal.h"

#define MODAL_MAXP 16
#define MODAL_MAX_TILES 40

// Device-side error word bits (set by kernels, read by modal_sync).
#define MODAL_DEVERR_TIMEOUT 1
#define MODAL_DEVERR_NOTPD 2

namespace modal {

inline int64_t alm_index(int64_t l, int64_t m, int64_t lmax) { return m * (2 * lmax + 3 - m) / 2 + (l - m); }
__host__ __device__ inline int64_t d_alm_index(int64_t l, int64_t m, int64_t lmax) {
    return m * (2 * lmax + 3 - m) / 2 + (l - m);
}

// Tensor-core operand tiles: 128 ring pairs x 32 l values of one parity per tile.
constexpr int TC_BM = 128;

// Layout of the pre-split tensor-core Legendre tables (hi and lo parts).
struct TcTable {
    void* hi = nullptr;                 // element type per precision (fp32 for tf32, 16-bit otherwise)
    void* lo = nullptr;
    int elem_bytes = 4;
    int bk = 32;                        // l values per K block (one 128-byte swizzle row)
    int n_rt = 0;                       // ring tiles of TC_BM ring pairs
    std::vector<int64_t> kb_off;        // per (m, parity): first K block index (prefix sums)
    int64_t n_kb = 0;                   // total K blocks over all (m, parity)
    int64_t* d_kb_off = nullptr;        // device copy of kb_off ([2 (lmax+1)])
    int64_t* d_bkb_off = nullptr;       // first B stage block of (m, parity) ([2 (lmax+1)])
    int64_t total_bkb = 0;              // B stage blocks per group of 8 maps
    void* bops = nullptr;               // B stage blocks of the current chunk (workspace)
    unsigned* d_amax = nullptr;         // per-map scale bounds (float bits), [4096]
    float* d_fmax = nullptr;            // max_p |f_p(l)|, [lmax+1]
    size_t bytes = 0;
};

// Transposed pre-split Legendre table and operand workspace of the tensor-core adjoint.
struct TcAdjTable {
    void* table = nullptr;              // blocks (m, parity, l tile, ring-pair block): [hi][lo]
    int64_t* d_blk_base = nullptr;      // [2 (lmax+1)] first block of (m, parity)
    int64_t* d_item_base = nullptr;     // [2 (lmax+1) + 1] prefix sums of l tiles
    int64_t n_lt_total = 0;             // l tiles over all (m, parity)
    int nkb = 0;                        // ring-pair blocks per l tile
    void* bops = nullptr;               // U operand blocks of the current chunk (workspace)
    size_t bytes = 0;
};

// Trispectrum (quartic) modes: tables built and buffers sized on first use.
struct QuarticState {
    int n_quad = 0, ntiles = 0, n_sq = 0;
    int* tiles = nullptr;         // [ntiles] packed (colex pair group | lexicographic pair quad << 8)
    int* idx = nullptr;           // [8 n_pg][4 n_sq] quadruple index or -1
    int* modes = nullptr;         // [n_quad][4] (p, r, s, u)
    int* pa = nullptr;            // [n_pair] lexicographic pair -> a
    int* pb = nullptr;            // [n_pair] lexicographic pair -> b
    double* partial = nullptr;    // [chunk][cubic_ctas][n_quad]
    double* rq = nullptr;         // [chunk][n_pair][nrings] ring sums of pair products
    double* h = nullptr;          // single-pair term: ring [chunk][n_pair][n_pair] or pixel [ksplit][n_pair][chunk n_pair]
    double* kmat = nullptr;       // two-pair sums [ksplit or 1][n_pair][n_pair]
    double* k3 = nullptr;         // [n_quad] two-pair term
    int chunk = 0;                // maps the buffers were sized for
    int ctas = 0;                 // cubic_ctas the partial sums were sized for
};

struct Plan {
    int lmax = 0, P = 0, nrings = 0, nphi = 0, prec = 0, dev = 0;
    int R_half = 0;          // ring pairs (north rings incl. the equator)
    int RH = 0;              // R_half padded to a multiple of 32 (SIMT table stride)
    int n_alm = 0, n_max = 0, n_pair = 0;
    int64_t npix = 0;
    int chunk = 0;           // maps per internal pass
    std::vector<double> mu, w;            // host ring nodes/weights (north first, all rings)
    std::vector<double> basis, cl;        // host copies of the inputs
    std::vector<int> mode_p, mode_r, mode_s;

    // device tables
    float* lam = nullptr;        // [n_alm][RH] lambda_lm(theta_j), j < R_half
    float* filt = nullptr;       // [P][lmax+1]
    float* W = nullptr;          // [nrings*nphi] pixel weights with mask
    float* wring = nullptr;      // [nrings] w_j 2 pi / nphi (no mask)
    float4* twiddle = nullptr;   // ring-FFT twiddles: 3 Ns float4 per Stockham pass with Ns > 1
    int* modeidx = nullptr;      // [n_pair_colex_pad][16] -> mode index or -1 (cubic tiles)
    int* tiles = nullptr;        // [n_tiles] packed (pair group, s quad)
    int n_tiles = 0, n_pg = 0, n_sq = 0;
    int cubic_nslots = 0;        // compute items (half-warps) of the cubic kernel, stored after the tile codes
    int* pair_ab = nullptr;      // colex pair c -> (p | r << 8), padded entries = -1
    TcTable tc;
    TcAdjTable tca;

    // Monte Carlo accumulators
    double* pair_sum = nullptr;  // [n_pair][npix]
    float* pair_mean = nullptr;  // [n_pair][npix]
    long long n_lin = 0;
    int lin_final = 0;
    double* S1 = nullptr;        // [n_max]
    double* S2 = nullptr;        // [n_max][n_max]
    long long n_cov = 0;

    // workspace (sized by chunk)
    float2* delta = nullptr;     // [chunk][P][lmax+1][2][RH]: even/odd Legendre sums per ring pair
    float* maps = nullptr;       // [chunk][P][npix]
    float2* ut = nullptr;        // [chunk][P][lmax+1][2][RH] (adjoint)
    double* partial = nullptr;   // cubic / linear partial sums
    size_t partial_elems = 0;
    int cubic_ctas = 0;          // CTAs per map in the cubic and quartic kernels (tunable)
    int lin_ksplit = 0;          // K splits in the linear-term GEMM (SIMT)
    int tc_maps = 8;             // maps per work item of the tensor-core Legendre kernel (tunable)
    int nsm = 0;                 // SMs of the plan's device
    // maps of the last modal_cubic call kept in `maps` for modal_backward_retained
    int retain_maps = 0;
    const void* kept_alm = nullptr;   // a_lm they were synthesised from (nullptr: none kept)
    int kept_B = 0;
    float* hk = nullptr;         // [chunk][P][n_pair] adjoint weights
    char* adj_gops = nullptr;    // [chunk] tf32 hi/lo G operands of the tensor-core adjoint pixel weights
    float* adj_pmk = nullptr;    // per chunk: K of the adjoint's pair-mean part or S of the harmonic linear term
    float2* adj_pm = nullptr;    // [n_pair][n_alm] (l-major) adjoint transform of each weighted pair-mean row
    int adj_pm_ready = 0;        // adj_pm holds the current pair means
    int* adj_pm_blk = nullptr;   // blocks of the pair-mean gradient kernel: l << 8 | m block, largest l first
    int adj_pm_nblk = 0;
    // ring-only linear term (modal_set_linear_mode)
    int lin_mode = 0;            // MODAL_LINEAR_PIXEL or MODAL_LINEAR_RING
    int has_pix_mask = 0;        // W varies along rings: ring mode refused
    double* ring_sum = nullptr;  // [n_pair][nrings]
    double* ring_mean = nullptr; // [n_pair][nrings]
    float* vring = nullptr;      // [chunk][P][nrings] adjoint pair-mean term
    double* solve_ws = nullptr;  // [n_max][n_max] + vectors
    int* d_err = nullptr;        // device error words: [0] data path, [1] FP64 solve (Cholesky)
    size_t device_bytes = 0;
    size_t workspace_bytes = 0;
    std::vector<int> cubic_pair_ab_host, cubic_tiles_host;

    // profiling: per-stage event pairs and launch counters
    int prof = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double stage_ms[MODAL_NSTAGES] = {};
    long long stage_launches[MODAL_NSTAGES] = {};
    mutable long long launch_count = 0;   // kernels launched by this plan (note_launch)
    // Bumped by every change that alters what a modal_cubic call launches or which buffers it
    // touches (workspace reallocation, linear-term mode, map retention, reset, state load,
    // first allocation of the linear-term buffers): a captured batch graph is replayed only
    // while the generations of its plans are unchanged.
    unsigned long long generation = 0;
    QuarticState qt;
};

enum Stage {
    ST_LEGENDRE = 0, ST_C2R = 1, ST_CUBIC = 2, ST_LINEAR = 3, ST_BETA = 4, ST_PAIRS = 5,
    ST_COV = 6, ST_SOLVE = 7, ST_ADJ_PIXEL = 8, ST_R2C = 9, ST_LEGENDRE_ADJ = 10, ST_OTHER = 11,
    ST_LEGENDRE_PREP = 12, ST_LEGENDRE_ADJ_PREP = 13, ST_QUARTIC = 14
};

// ---- error reporting (modal_api.cu) ----
modal_status set_error(modal_status s, const std::string& msg);
modal_status cuda_check(cudaError_t e, const char* what);

// ---- kernels launchers ----
// k_tables.cu
cudaError_t launch_lambda_table(const Plan& pl, const double* d_mu_north, const double* d_log2c,
                                const double* d_a, const double* d_b, cudaStream_t st);
cudaError_t build_tc_tables(Plan& pl, cudaStream_t st);      // allocates pl.tc
size_t tc_table_bytes(const Plan& pl);                       // bytes build_tc_tables allocates for the table
bool tc_maps_valid(int P, int G);                            // G maps per forward Legendre item: 2 P G % 16 == 0, <= 256
size_t tc_adj_table_bytes(const Plan& pl);                   // the same for build_tc_adj_tables
size_t tc_b_workspace_bytes(const Plan& pl, int chunk);
// k_legendre_tc_adj.cu
cudaError_t build_tc_adj_tables(Plan& pl, cudaStream_t st);
void free_tc_adj_tables(Plan& pl);
size_t tc_adj_workspace_bytes(const Plan& pl, int chunk);
// amax_ready: pl.tc.d_amax already holds each map's max |U~| (from k_ring_r2c).
cudaError_t launch_legendre_adjoint_tc(const Plan& pl, const float2* ut, int B, float2* grad, bool amax_ready,
                                       int part, cudaStream_t st);
void free_tc_tables(Plan& pl);
// k_legendre_simt.cu
cudaError_t launch_legendre_simt(const Plan& pl, const float2* alm, int B, float2* delta, cudaStream_t st);
cudaError_t launch_legendre_adjoint_simt(const Plan& pl, const float2* ut, int B, const float* rowfilt,
                                         int nfilt, float2* out, cudaStream_t st);
// k_legendre_tc.cu
// Every kernel launch of the hot path is counted on its plan.
inline void note_launch(const Plan& pl) { ++pl.launch_count; }

// part: 1 = operand preparation (per-map scale, split B blocks), 2 = the contraction, 3 = both.
cudaError_t launch_legendre_tc(const Plan& pl, const float2* alm, int B, float2* delta, int part, cudaStream_t st);
// k_fft.cu
cudaError_t launch_ring_c2r(const Plan& pl, const float2* delta, int nmaps_p, float* maps, cudaStream_t st);
cudaError_t launch_ring_r2c(const Plan& pl, const float* maps, int nmaps_p, const float* ring_weight,
                            float2* ut, unsigned* amax, cudaStream_t st);
// k_cubic.cu
cudaError_t launch_cubic(Plan& pl, const float* maps, int B, double* partial, cudaStream_t st);
// The cubic sums of B[i] maps (one chunk, at maps[i], partial sums into plan i's partial
// buffer) of n plans with the same P as one persistent launch; counter: device int.
constexpr int CUBIC_MAX_JOBS = 8;
cudaError_t launch_cubic_multi(Plan* const* plans, const float* const* maps, const int* B, int n, int* counter,
                               cudaStream_t st);
cudaError_t launch_linear_gemm(Plan& pl, const float* maps, int B, double* partial, cudaStream_t st);
// lin_splits: K splits summed from lin_partial ([lin_splits][n_pair][B P])
cudaError_t launch_beta_finalize(Plan& pl, int B, int use_linear, const double* cub_partial,
                                 const double* lin_partial, int lin_splits, double* beta, cudaStream_t st);
cudaError_t launch_pair_accumulate(Plan& pl, const float* maps, int B, cudaStream_t st);
cudaError_t launch_pair_finalize(Plan& pl, cudaStream_t st);
cudaError_t launch_adjoint_weights(Plan& pl, const double* g, int B, float* hk, cudaStream_t st);
// pair-mean term: per pixel from pl.pair_mean (use_linear, pixel mode) or per ring from
// vring [B][P][nrings] (ring mode, use_linear = 0); neither when both are off.
cudaError_t launch_adjoint_u(Plan& pl, const float* maps, int B, const float* hk, int use_linear,
                             float* u, cudaStream_t st);
// k_adjoint_tc.cu: the same pixel weights as a tcgen05 product (split plans); in place on maps
// k_adjoint_v.cu: the map part of the pixel weights (in place over the maps).
size_t adjoint_v_workspace_bytes(const Plan& pl, int chunk);
cudaError_t launch_adjoint_v(Plan& pl, int B, const float* hk, float* maps, cudaStream_t st);
// k_pm_harmonic.cu: the pair means in harmonic space (split plans, per-pixel means): the table
// of adjoint-transformed weighted pair-mean rows (after each finalised mean), the linear term
// from a_lm, and the adjoint's pair-mean part applied to the gradient.
size_t adjoint_pm_workspace_bytes(const Plan& pl, int chunk);
cudaError_t build_pm_table(Plan& pl, cudaStream_t st);
cudaError_t launch_linear_harmonic(Plan& pl, const float2* alm, int B, double* lin, cudaStream_t st);
cudaError_t launch_adjoint_pm(Plan& pl, int B, const float* hk, float2* grad, float2* scratch, cudaStream_t st);
// k_ring_linear.cu
cudaError_t launch_pair_ring(Plan& pl, const float* maps, int B, cudaStream_t st);
cudaError_t launch_ring_finalize(Plan& pl, cudaStream_t st);
cudaError_t launch_linear_ring(Plan& pl, int B, double* lin, cudaStream_t st);
cudaError_t launch_vring(Plan& pl, const float* hk, int B, float* vring, cudaStream_t st);
// subtract nphi W_j V(j) from the m = 0 analysis coefficients of every ring (ring mode)
cudaError_t launch_vring_correct(Plan& pl, const float* vring, int nrows, float2* ut, unsigned* amax, cudaStream_t st);
cudaError_t launch_ring_mean_float(Plan& pl, float* out, cudaStream_t st);
// k_solve.cu
cudaError_t launch_cov_accumulate(Plan& pl, const double* beta, int B, cudaStream_t st);
cudaError_t launch_zeta(Plan& pl, double* zeta, cudaStream_t st);
cudaError_t launch_cholesky(Plan& pl, double* A, int n, cudaStream_t st);
cudaError_t launch_solve_rhs(Plan& pl, const double* Lc, int n, double* rhs, int nrhs, cudaStream_t st);
cudaError_t launch_estimates(Plan& pl, const double* rhs, int n, int B, double* out, cudaStream_t st);
// v = alpha' (forward-solved) -> w = L^-T alpha' / norm[0] (dev norm = |alpha'|^2)
cudaError_t launch_fnl_weights(Plan& pl, const double* Lc, int n, double* v, const double* norm, double* w,
                               cudaStream_t st);
cudaError_t launch_wait_selftest(int* d_err, int spin_limit, cudaStream_t st);
// trispectrum modes (k_quartic.cu)
cudaError_t quartic_tables(Plan& pl);
cudaError_t launch_quartic(Plan& pl, const float* maps, int B, double* partial, cudaStream_t st);
cudaError_t launch_quartic_linear(Plan& pl, const float* maps, int B, cudaStream_t st);
cudaError_t launch_quartic_k3(Plan& pl, cudaStream_t st);
cudaError_t launch_quartic_finalize(Plan& pl, int B, int use_linear, double* tau, cudaStream_t st);
// bivector form of the covariance (k_solve.cu)
cudaError_t launch_transpose(Plan& pl, int n, const double* in, double* out, cudaStream_t st);
cudaError_t launch_power_step(Plan& pl, int n, const double* Z, double* v, double* w, double* stat, cudaStream_t st);
cudaError_t launch_bivector_estimates(Plan& pl, const double* rhs, int n, int B, const double* bt, double* out,
                                      cudaStream_t st);
cudaError_t launch_bivector_rotate(Plan& pl, int n, int B, const double* bt, double* x, cudaStream_t st);

}  // namespace modal
