// C ABI of the modal bispectrum library: plan construction, dispatch of the
// per-map stages in chunks of maps, Monte Carlo accumulators, estimator solve,
// checkpointing.  Argument meaning and error behaviour are documented in modal.h.
#include "modal_internal.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

using namespace modal;

struct modal_plan : public Plan {};

// Offsets inside the small integer table `modeidx` (one allocation).
static constexpr int MI_MODEIDX = 0;      // [256][16]  colex pair c, s -> mode or -1
static constexpr int MI_MP = 4096;        // [1024] mode -> p
static constexpr int MI_MR = 5120;        // [1024] mode -> r
static constexpr int MI_MS = 6144;        // [1024] mode -> s
static constexpr int MI_MODEOF = 7168;    // [P][P][P] sorted triple -> mode
static constexpr int MI_TOTAL = 11264;

namespace modal {

static thread_local std::string g_last_error;

modal_status set_error(modal_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

modal_status cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return MODAL_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(MODAL_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    return set_error(MODAL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace modal

#define CK(expr, what)                                        \
    do {                                                      \
        modal_status _s = cuda_check((expr), (what));         \
        if (_s != MODAL_OK) return _s;                        \
    } while (0)

template <typename T>
static cudaError_t dalloc(modal_plan* pl, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e == cudaSuccess) pl->device_bytes += count * sizeof(T);
    return e;
}

static void dfree(void* p) {
    if (p) cudaFree(p);
}

// ------------------------------------------------------------------ host math
// Gauss-Legendre nodes (north first) and weights by Newton's method on P_n.
static void gauss_legendre(int n, std::vector<double>& mu, std::vector<double>& w) {
    mu.assign(n, 0.0);
    w.assign(n, 0.0);
    const int half = (n + 1) / 2;
    for (int j = 0; j < half; ++j) {
        double x = std::cos(M_PI * (j + 0.75) / (n + 0.5));
        double p = 0, pm1 = 0, dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            p = (n == 0) ? 1.0 : p1;
            pm1 = (n == 1) ? 1.0 : p0;
            if (n == 1) { p = x; pm1 = 1.0; }
            dp = n * (x * p - pm1) / (x * x - 1.0);
            const double dx = p / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            p = p1;
            pm1 = (n == 1) ? 1.0 : p0;
            dp = n * (x * p - pm1) / (x * x - 1.0);
        }
        if ((n & 1) && j == half - 1) x = 0.0;
        mu[j] = x;
        w[j] = 2.0 / ((1.0 - x * x) * dp * dp);
        mu[n - 1 - j] = -x;
        w[n - 1 - j] = w[j];
    }
}

static int n_modes_of(int P) { return P * (P + 1) * (P + 2) / 6; }

static void build_mode_tables(modal_plan* pl, std::vector<int>& mi) {
    const int P = pl->P;
    mi.assign(MI_TOTAL, -1);
    pl->mode_p.clear(); pl->mode_r.clear(); pl->mode_s.clear();
    std::vector<int> mode_of(P * P * P, -1);
    int n = 0;
    for (int p = 0; p < P; ++p)
        for (int r = p; r < P; ++r)
            for (int s = r; s < P; ++s) {
                pl->mode_p.push_back(p); pl->mode_r.push_back(r); pl->mode_s.push_back(s);
                mi[MI_MP + n] = p; mi[MI_MR + n] = r; mi[MI_MS + n] = s;
                mode_of[(p * P + r) * P + s] = n;
                mi[MI_MODEOF + (p * P + r) * P + s] = n;
                ++n;
            }
    // colex pairs (sorted by r then p), padded to a multiple of 8
    std::vector<std::pair<int, int>> colex;
    for (int r = 0; r < P; ++r)
        for (int p = 0; p <= r; ++p) colex.push_back({p, r});
    pl->n_pg = ((int)colex.size() + 7) / 8;
    pl->n_sq = (P + 3) / 4;
    std::vector<int> pair_ab(pl->n_pg * 8, -1);
    for (size_t c = 0; c < colex.size(); ++c) pair_ab[c] = colex[c].first | (colex[c].second << 8);
    for (size_t c = 0; c < colex.size(); ++c)
        for (int s = 0; s < P; ++s)
            if (s >= colex[c].second)
                mi[MI_MODEIDX + c * 16 + s] = mode_of[(colex[c].first * P + colex[c].second) * P + s];
    std::vector<int> tiles;
    for (int pg = 0; pg < pl->n_pg; ++pg)
        for (int sq = 0; sq < pl->n_sq; ++sq) {
            bool any = false;
            for (int c = pg * 8; c < pg * 8 + 8 && c < (int)colex.size(); ++c)
                for (int s = sq * 4; s < sq * 4 + 4 && s < P; ++s)
                    if (s >= colex[c].second) any = true;
            if (any) tiles.push_back(pg | (sq << 8));
        }
    pl->n_tiles = (int)tiles.size();
    // compute items of the cubic kernel: two tiles of one pair group (two quads), else two
    // pair groups of one quad, else a tile alone; items of the first kind first, each kind
    // padded to an even count with idle slots so that the two half-warps of a warp run the
    // same path.  Appended after the tile codes (from an even offset) as (tile a, tile b).
    {
        std::vector<std::vector<int>> by_pg(pl->n_pg);
        for (int t = 0; t < pl->n_tiles; ++t) by_pg[tiles[t] & 0xff].push_back(t);
        std::vector<std::pair<int, int>> kind_a, kind_b;
        std::vector<std::vector<int>> pool(pl->n_sq);
        for (int pg = 0; pg < pl->n_pg; ++pg) {
            const std::vector<int>& ts = by_pg[pg];            // quads ascending
            size_t i = 0;
            for (; i + 1 < ts.size(); i += 2) kind_a.push_back({ts[i], ts[i + 1]});
            if (i < ts.size()) pool[tiles[ts[i]] >> 8].push_back(ts[i]);
        }
        for (int sq = 0; sq < pl->n_sq; ++sq) {
            size_t i = 0;
            for (; i + 1 < pool[sq].size(); i += 2) kind_b.push_back({pool[sq][i], pool[sq][i + 1]});
            if (i < pool[sq].size()) kind_a.push_back({pool[sq][i], -1});
        }
        if (kind_a.size() % 2) kind_a.push_back({-1, -1});
        if (kind_b.size() % 2) kind_b.push_back({-1, -1});
        if (tiles.size() % 2) tiles.push_back(0);
        for (const auto& it : kind_a) { tiles.push_back(it.first); tiles.push_back(it.second); }
        for (const auto& it : kind_b) { tiles.push_back(it.first); tiles.push_back(it.second); }
        pl->cubic_nslots = (int)(kind_a.size() + kind_b.size());
    }
    pl->cubic_pair_ab_host = pair_ab;
    pl->cubic_tiles_host = tiles;
}

// ------------------------------------------------------------------ workspace
static size_t per_map_workspace(const modal_plan* pl) {
    const size_t L1 = pl->lmax + 1;
    const size_t delta = (size_t)pl->P * L1 * 2 * pl->RH * sizeof(float2);
    const size_t maps = (size_t)pl->P * pl->npix * sizeof(float);
    const size_t ut = (size_t)pl->P * L1 * 2 * pl->RH * sizeof(float2);
    return delta + maps + ut + tc_b_workspace_bytes(*pl, 8) / 8 + tc_adj_workspace_bytes(*pl, 8) / 8 +
           adjoint_v_workspace_bytes(*pl, 1) + adjoint_pm_workspace_bytes(*pl, 1);
}

static void free_workspace(modal_plan* pl) {
    ++pl->generation;
    dfree(pl->delta); pl->delta = nullptr;
    dfree(pl->maps); pl->maps = nullptr;
    dfree(pl->ut); pl->ut = nullptr;
    dfree(pl->partial); pl->partial = nullptr;
    dfree(pl->hk); pl->hk = nullptr;
    dfree(pl->adj_gops); pl->adj_gops = nullptr;
    dfree(pl->adj_pmk); pl->adj_pmk = nullptr;
    dfree(pl->vring); pl->vring = nullptr;
    dfree(pl->tc.bops); pl->tc.bops = nullptr;
    dfree(pl->tca.bops); pl->tca.bops = nullptr;
    pl->device_bytes -= pl->workspace_bytes;
    pl->workspace_bytes = 0;
}

static modal_status alloc_workspace_buffers(modal_plan* pl, int chunk) {
    const size_t L1 = pl->lmax + 1;
    CK(dalloc(pl, &pl->delta, (size_t)chunk * pl->P * L1 * 2 * pl->RH), "workspace delta");
    CK(dalloc(pl, &pl->maps, (size_t)chunk * pl->P * pl->npix), "workspace maps");
    CK(dalloc(pl, &pl->ut, (size_t)chunk * pl->P * L1 * 2 * pl->RH), "workspace ut");
    CK(dalloc(pl, &pl->hk, (size_t)chunk * pl->P * pl->n_pair), "workspace hk");
    CK(dalloc(pl, &pl->adj_gops, adjoint_v_workspace_bytes(*pl, chunk)), "workspace adjoint operands");
    CK(dalloc(pl, &pl->adj_pmk, adjoint_pm_workspace_bytes(*pl, chunk) / sizeof(float)), "workspace adjoint pair-mean weights");
    CK(dalloc(pl, &pl->vring, (size_t)chunk * pl->P * pl->nrings), "workspace vring");
    // cubic partials: [chunk][cubic_ctas][n_max]; linear partials: [ksplit][n_pair][chunk*P]
    const size_t cub = (size_t)chunk * pl->cubic_ctas * pl->n_max;
    const size_t lin = (size_t)std::max(pl->lin_ksplit, 1) * pl->n_pair * chunk * pl->P;
    pl->partial_elems = cub + lin;
    CK(dalloc(pl, &pl->partial, pl->partial_elems), "workspace partial");
    {
        const size_t bb = tc_b_workspace_bytes(*pl, chunk);
        char* p = nullptr;
        CK(dalloc(pl, &p, bb), "workspace tensor-core operands");
        pl->tc.bops = p;
        char* q = nullptr;
        CK(dalloc(pl, &q, tc_adj_workspace_bytes(*pl, chunk)), "workspace tensor-core adjoint operands");
        pl->tca.bops = q;
    }
    return MODAL_OK;
}

// The per-pass buffers for `chunk` maps.  On failure the buffers allocated so far stay
// attached (and counted) until the next free_workspace.
static modal_status alloc_workspace(modal_plan* pl, int chunk) {
    free_workspace(pl);
    pl->chunk = chunk;
    pl->kept_alm = nullptr;
    const size_t before = pl->device_bytes;
    const modal_status s = alloc_workspace_buffers(pl, chunk);
    pl->workspace_bytes = pl->device_bytes - before;
    return s;
}

// Calls that run maps through the plan need its workspace; a failed modal_set_chunk that
// could not restore the previous one leaves none (chunk 0).
static modal_status check_workspace(modal_h h) {
    if (h->chunk >= 1) return MODAL_OK;
    return set_error(MODAL_ESTATE, "the plan has no workspace (a modal_set_chunk failed); call modal_set_chunk");
}

static modal_status ensure_pair_buffers(modal_plan* pl) {
    if (pl->pair_sum) return MODAL_OK;
    ++pl->generation;
    const size_t n = (size_t)pl->n_pair * pl->npix;
    CK(dalloc(pl, &pl->pair_sum, n), "pair sums");
    CK(dalloc(pl, &pl->pair_mean, n), "pair mean");
    CK(cudaMemset(pl->pair_sum, 0, n * sizeof(double)), "pair sums clear");
    CK(cudaMemset(pl->pair_mean, 0, n * sizeof(float)), "pair mean clear");
    return MODAL_OK;
}

static modal_status ensure_ring_buffers(modal_plan* pl) {
    if (pl->ring_sum) return MODAL_OK;
    ++pl->generation;
    const size_t n = (size_t)pl->n_pair * pl->nrings;
    CK(dalloc(pl, &pl->ring_sum, n), "ring pair sums");
    CK(dalloc(pl, &pl->ring_mean, n), "ring pair means");
    CK(cudaMemset(pl->ring_sum, 0, n * sizeof(double)), "ring pair sums clear");
    CK(cudaMemset(pl->ring_mean, 0, n * sizeof(double)), "ring pair means clear");
    return MODAL_OK;
}

static void destroy_plan(modal_plan* pl) {
    if (!pl) return;
    cudaDeviceSynchronize();
    free_workspace(pl);
    dfree(pl->lam); dfree(pl->filt); dfree(pl->W); dfree(pl->wring); dfree(pl->twiddle);
    dfree(pl->modeidx); dfree(pl->tiles); dfree(pl->pair_ab);
    dfree(pl->pair_sum); dfree(pl->pair_mean); dfree(pl->S1); dfree(pl->S2);
    dfree(pl->ring_sum); dfree(pl->ring_mean);
    dfree(pl->solve_ws); dfree(pl->d_err); dfree(pl->adj_pm); dfree(pl->adj_pm_blk);
    dfree(pl->qt.tiles); dfree(pl->qt.idx); dfree(pl->qt.modes); dfree(pl->qt.pa); dfree(pl->qt.pb);
    dfree(pl->qt.partial); dfree(pl->qt.rq); dfree(pl->qt.h); dfree(pl->qt.k3); dfree(pl->qt.kmat);
    free_tc_tables(*pl);
    free_tc_adj_tables(*pl);
    for (auto& pe : pl->prof_pending) { cudaEventDestroy(pe.second.first); cudaEventDestroy(pe.second.second); }
    for (auto e : pl->prof_pool) cudaEventDestroy(e);
    delete pl;
}

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static modal_status check_plan(modal_h h) {
    if (!h) return set_error(MODAL_EINVAL, "null plan");
    return MODAL_OK;
}

static cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Brackets the launches of one stage: counts the kernels they launch under `stage` and,
// with profiling on, records CUDA events before and after them on the launching stream.
struct StageScope {
    modal_plan* pl;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    long long k0;                          // plan's kernel count when the scope opened
    static cudaEvent_t take(modal_plan* p) {
        if (!p->prof_pool.empty()) {
            cudaEvent_t e = p->prof_pool.back();
            p->prof_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    StageScope(modal_plan* p, int s, cudaStream_t stream) : pl(p), stage(s), st(stream), k0(p->launch_count) {
        if (pl->prof) {
            a = take(pl);
            cudaEventRecord(a, st);
        }
    }
    ~StageScope() {
        pl->stage_launches[stage] += pl->launch_count - k0;
        if (pl->prof && a) {
            cudaEvent_t b = take(pl);
            cudaEventRecord(b, st);
            pl->prof_pending.push_back({stage, {a, b}});
        }
    }
};
#define STAGE(pl, id, st) StageScope _scope_##id((pl), (id), (st))

// Legendre stage for one chunk: alm -> delta (tensor-core path: operand preparation and
// the contraction are timed as separate stages).
static cudaError_t legendre_forward(modal_plan* pl, const float2* alm, int B, cudaStream_t st) {
    if (pl->prec == MODAL_FP32) {
        STAGE(pl, ST_LEGENDRE, st);
        return launch_legendre_simt(*pl, alm, B, pl->delta, st);
    }
    {
        STAGE(pl, ST_LEGENDRE_PREP, st);
        cudaError_t e = launch_legendre_tc(*pl, alm, B, pl->delta, 1, st);
        if (e != cudaSuccess) return e;
    }
    STAGE(pl, ST_LEGENDRE, st);
    return launch_legendre_tc(*pl, alm, B, pl->delta, 2, st);
}

static cudaError_t synth_chunk(modal_plan* pl, const float2* alm, int B, float* maps_out, cudaStream_t st) {
    if (maps_out == pl->maps) pl->kept_alm = nullptr;
    {
        cudaError_t e = legendre_forward(pl, alm, B, st);
        if (e != cudaSuccess) return e;
    }
    STAGE(pl, ST_C2R, st);
    return launch_ring_c2r(*pl, pl->delta, B * pl->P, maps_out, st);
}

extern "C" {

const char* modal_last_error(void) { return g_last_error.c_str(); }

modal_status modal_init(int lmax, int P, const double* basis, const double* C_l, const modal_grid* grid, int prec,
                        modal_h* out) {
    if (!out) return set_error(MODAL_EINVAL, "out is NULL");
    *out = nullptr;
    if (lmax < 2 || lmax > 4000) return set_error(MODAL_EINVAL, "lmax must be in [2, 4000]");
    if (P < 1 || P > MODAL_MAXP) return set_error(MODAL_EINVAL, "P must be in [1, 16]");
    if (!basis || !C_l || !grid) return set_error(MODAL_EINVAL, "basis, C_l and grid are required");
    if (grid->nrings < lmax + 1) return set_error(MODAL_EINVAL, "nrings must be >= lmax + 1");
    if (!is_pow2(grid->nphi) || grid->nphi < 2 * lmax + 2 || grid->nphi < 16 || grid->nphi > 8192)
        return set_error(MODAL_EINVAL, "nphi must be a power of two in [max(16, 2 lmax + 2), 8192]");
    if (prec < MODAL_FP32 || prec > MODAL_FP16X3) return set_error(MODAL_EINVAL, "unknown precision");
    for (int l = 0; l <= lmax; ++l)
        if (!std::isfinite(C_l[l])) return set_error(MODAL_EINVAL, "C_l must be finite");
    for (int i = 0; i < P * (lmax + 1); ++i)
        if (!std::isfinite(basis[i])) return set_error(MODAL_EINVAL, "basis must be finite");

    modal_plan* pl = new modal_plan();
    int dev = 0;
    cudaGetDevice(&dev);
    pl->dev = dev;
    pl->lmax = lmax; pl->P = P; pl->nrings = grid->nrings; pl->nphi = grid->nphi; pl->prec = prec;
    pl->has_pix_mask = grid->pix_mask ? 1 : 0;
    pl->R_half = (grid->nrings + 1) / 2;
    pl->RH = (pl->R_half + 31) / 32 * 32;
    pl->n_alm = (lmax + 1) * (lmax + 2) / 2;
    pl->n_max = n_modes_of(P);
    pl->n_pair = P * (P + 1) / 2;
    pl->npix = (int64_t)grid->nrings * grid->nphi;
    pl->basis.assign(basis, basis + (size_t)P * (lmax + 1));
    pl->cl.assign(C_l, C_l + lmax + 1);
    gauss_legendre(grid->nrings, pl->mu, pl->w);

    // kernel geometry
    {
        cudaDeviceGetAttribute(&pl->nsm, cudaDevAttrMultiProcessorCount, pl->dev);
        pl->nsm = std::max(pl->nsm, 1);
        // pixel ranges of the cubic and quartic sums per map: one per 8192 pixels, at most one
        // per SM (a 32-map launch at l_max = 2000 then runs 4864 CTAs: 18.09 ms, against 18.53
        // with 512 ranges per map, whose per-CTA reductions and partial sums cost more)
        int64_t ctas = pl->npix / 8192;
        pl->cubic_ctas = (int)std::max<int64_t>(1, std::min<int64_t>(ctas, pl->nsm));
        int64_t ks = pl->npix / 16384;
        pl->lin_ksplit = (int)std::max<int64_t>(1, std::min<int64_t>(ks, 128));
        pl->tc_maps = 8;                                   // N = 16 P columns per Legendre item
    }

    auto fail = [&](modal_status s) { destroy_plan(pl); return s; };
    // Refuse a plan whose resident tables and a one-map workspace exceed the device's free
    // memory before allocating any of it (the tables grow as lmax^3: about 25 GB at lmax =
    // 2000 for the tensor-core precisions, near 200 GB at 4000).
    {
        const size_t tables = (size_t)pl->n_alm * pl->RH * sizeof(float) + tc_table_bytes(*pl) +
                              tc_adj_table_bytes(*pl) + (size_t)pl->npix * sizeof(float);
        const size_t one_map = per_map_workspace(pl) +
                               ((size_t)pl->cubic_ctas * pl->n_max +
                                (size_t)std::max(pl->lin_ksplit, pl->nsm) * pl->n_pair * pl->P) * sizeof(double);
        const size_t margin = (size_t)256 << 20;          // small tables, the context's own use
        size_t free_b = 0, total_b = 0;
        const cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
        if (e != cudaSuccess) return fail(cuda_check(e, "cudaMemGetInfo"));
        if (tables + one_map + margin > free_b) {
            char msg[256];
            std::snprintf(msg, sizeof msg,
                          "plan needs %.2f GB of device memory (tables %.2f GB, workspace for one map %.2f GB); "
                          "%.2f GB free",
                          (tables + one_map + margin) / 1e9, tables / 1e9, one_map / 1e9, free_b / 1e9);
            return fail(set_error(MODAL_ENOMEM, msg));
        }
    }
#define CKI(expr, what)                                        \
    do {                                                       \
        modal_status _s = cuda_check((expr), (what));          \
        if (_s != MODAL_OK) return fail(_s);                   \
    } while (0)

    // Legendre table (FP64 recurrence on the GPU)
    {
        std::vector<double> log2c(lmax + 1), ca(pl->n_alm, 0.0), cb(pl->n_alm, 0.0);
        double lp = 0.0;
        for (int m = 0; m <= lmax; ++m) {
            if (m > 0) lp += std::log2((2.0 * m - 1.0) / (2.0 * m));
            log2c[m] = 0.5 * (std::log2((2.0 * m + 1.0) / (4.0 * M_PI)) + lp);
            for (int l = m + 1; l <= lmax; ++l) {
                const int64_t i = alm_index(l, m, lmax);
                const double L = l, M = m;
                ca[i] = std::sqrt((4.0 * L * L - 1.0) / (L * L - M * M));
                cb[i] = std::sqrt(((L - 1.0) * (L - 1.0) - M * M) / (4.0 * (L - 1.0) * (L - 1.0) - 1.0));
            }
        }
        double *d_mu = nullptr, *d_log2c = nullptr, *d_a = nullptr, *d_b = nullptr;
        CKI(cudaMalloc(&d_mu, pl->R_half * sizeof(double)), "table mu");
        cudaMalloc(&d_log2c, (lmax + 1) * sizeof(double));
        cudaMalloc(&d_a, pl->n_alm * sizeof(double));
        cudaMalloc(&d_b, pl->n_alm * sizeof(double));
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(d_mu, pl->mu.data(), pl->R_half * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_log2c, log2c.data(), (lmax + 1) * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_a, ca.data(), pl->n_alm * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_b, cb.data(), pl->n_alm * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = dalloc(pl, &pl->lam, (size_t)pl->n_alm * pl->RH);
        if (e == cudaSuccess) e = launch_lambda_table(*pl, d_mu, d_log2c, d_a, d_b, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(d_mu); cudaFree(d_log2c); cudaFree(d_a); cudaFree(d_b);
        CKI(e, "legendre table");
    }
    // filter f_p(l) = q_p(l)/sqrt(C_l), zero where C_l <= 0
    {
        std::vector<float> f((size_t)P * (lmax + 1));
        for (int p = 0; p < P; ++p)
            for (int l = 0; l <= lmax; ++l)
                f[(size_t)p * (lmax + 1) + l] =
                    C_l[l] > 0 ? (float)(basis[(size_t)p * (lmax + 1) + l] / std::sqrt(C_l[l])) : 0.f;
        CKI(dalloc(pl, &pl->filt, f.size()), "filter");
        CKI(cudaMemcpy(pl->filt, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice), "filter copy");
    }
    // pixel weights W_x = w_j (2 pi / nphi) mask_x, ring weights, twiddles
    {
        std::vector<float> W((size_t)pl->npix), wr(pl->nrings);
        for (int j = 0; j < pl->nrings; ++j) {
            const double base = pl->w[j] * 2.0 * M_PI / pl->nphi;
            wr[j] = (float)base;
            const double rm = grid->ring_mask ? grid->ring_mask[j] : 1.0;
            for (int k = 0; k < pl->nphi; ++k) {
                const double pm = grid->pix_mask ? grid->pix_mask[(size_t)j * pl->nphi + k] : 1.0;
                W[(size_t)j * pl->nphi + k] = (float)(base * rm * pm);
            }
        }
        CKI(dalloc(pl, &pl->W, W.size()), "weights");
        CKI(cudaMemcpy(pl->W, W.data(), W.size() * sizeof(float), cudaMemcpyHostToDevice), "weights copy");
        CKI(dalloc(pl, &pl->wring, wr.size()), "ring weights");
        CKI(cudaMemcpy(pl->wring, wr.data(), wr.size() * sizeof(float), cudaMemcpyHostToDevice), "ring weights copy");
        // per-pass twiddles of the ring FFT (radix-16 passes, then one of radix 8, 4 or 2):
        // for each pass (R, Ns) with Ns > 1, three blocks of Ns float4 holding
        // (w_1, w_2), (w_3, w_4), (w_8, w_12) at k, w_r = e^{2 pi i r k / (R Ns)}
        std::vector<float4> tw;
        {
            int lg = 0;
            while ((1 << lg) < pl->nphi) ++lg;
            auto w = [](int r, int k, int R, int Ns) {
                const double a = 2.0 * M_PI * (double)((long long)r * k) / (double)((long long)R * Ns);
                return make_float2((float)std::cos(a), (float)std::sin(a));
            };
            for (int Ns = 1, left = lg; left > 0;) {
                const int lr = left >= 4 ? 4 : left;
                const int R = 1 << lr;
                if (Ns > 1) {
                    const int pairs[3][2] = {{1, 2}, {3, 4}, {8, 12}};
                    for (int blk = 0; blk < 3; ++blk)
                        for (int k = 0; k < Ns; ++k) {
                            const float2 x = w(pairs[blk][0], k, R, Ns), y = w(pairs[blk][1], k, R, Ns);
                            tw.push_back(make_float4(x.x, x.y, y.x, y.y));
                        }
                }
                Ns *= R;
                left -= lr;
            }
            if (tw.empty()) tw.push_back(make_float4(1.f, 0.f, 1.f, 0.f));
        }
        CKI(dalloc(pl, &pl->twiddle, tw.size()), "twiddles");
        CKI(cudaMemcpy(pl->twiddle, tw.data(), tw.size() * sizeof(float4), cudaMemcpyHostToDevice), "twiddles copy");
    }
    // mode / pair / tile tables
    {
        std::vector<int> mi;
        build_mode_tables(pl, mi);
        CKI(dalloc(pl, &pl->modeidx, mi.size()), "mode tables");
        CKI(cudaMemcpy(pl->modeidx, mi.data(), mi.size() * sizeof(int), cudaMemcpyHostToDevice), "mode tables copy");
        CKI(dalloc(pl, &pl->tiles, pl->cubic_tiles_host.size()), "tiles");
        CKI(cudaMemcpy(pl->tiles, pl->cubic_tiles_host.data(), pl->cubic_tiles_host.size() * sizeof(int),
                       cudaMemcpyHostToDevice), "tiles copy");
        CKI(dalloc(pl, &pl->pair_ab, pl->cubic_pair_ab_host.size()), "pairs");
        CKI(cudaMemcpy(pl->pair_ab, pl->cubic_pair_ab_host.data(), pl->cubic_pair_ab_host.size() * sizeof(int),
                       cudaMemcpyHostToDevice), "pairs copy");
    }
    // accumulators and solve workspace
    CKI(dalloc(pl, &pl->S1, (size_t)pl->n_max), "S1");
    CKI(dalloc(pl, &pl->S2, (size_t)pl->n_max * pl->n_max), "S2");
    CKI(cudaMemset(pl->S1, 0, pl->n_max * sizeof(double)), "S1 clear");
    CKI(cudaMemset(pl->S2, 0, (size_t)pl->n_max * pl->n_max * sizeof(double)), "S2 clear");
    CKI(dalloc(pl, &pl->d_err, 2), "error words");
    CKI(cudaMemset(pl->d_err, 0, 2 * sizeof(int)), "error words clear");
    // tensor-core tables
    if (prec != MODAL_FP32) CKI(build_tc_tables(*pl, 0), "tensor-core tables");
    if (prec != MODAL_FP32) CKI(build_tc_adj_tables(*pl, 0), "tensor-core adjoint tables");
    // workspace: as many maps per pass as fit a 24 GB budget (at least 1, at most 64)
    {
        const size_t per = per_map_workspace(pl);
        int chunk = (int)std::max<size_t>(1, std::min<size_t>(64, (size_t)24e9 / std::max<size_t>(per, 1)));
        modal_status s = alloc_workspace(pl, chunk);
        if (s != MODAL_OK) return fail(s);
    }
    CKI(cudaDeviceSynchronize(), "init");
#undef CKI
    *out = pl;
    return MODAL_OK;
}

void modal_destroy(modal_h h) { destroy_plan(h); }

modal_status modal_set_linear_mode(modal_h h, int mode) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (mode != MODAL_LINEAR_PIXEL && mode != MODAL_LINEAR_RING) return set_error(MODAL_EINVAL, "unknown linear-term mode");
    if (mode == MODAL_LINEAR_RING && h->has_pix_mask)
        return set_error(MODAL_EINVAL, "ring-only linear term needs weights that depend on the ring alone (no pixel mask)");
    const modal_status r = modal_reset(h, 1);
    if (r != MODAL_OK) return r;
    h->lin_mode = mode;
    ++h->generation;
    return MODAL_OK;
}

modal_status modal_set_chunk(modal_h h, int chunk) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (chunk < 1 || chunk > 4096) return set_error(MODAL_EINVAL, "chunk must be in [1, 4096]");
    CK(cudaDeviceSynchronize(), "set_chunk sync");
    const int old = h->chunk;
    const modal_status s = alloc_workspace(h, chunk);
    if (s == MODAL_OK) return MODAL_OK;
    const std::string why = modal_last_error();
    if (old >= 1 && alloc_workspace(h, old) == MODAL_OK) return set_error(s, why + " (the previous chunk is kept)");
    free_workspace(h);
    h->chunk = 0;
    return set_error(s, why + " (the plan has no workspace until modal_set_chunk succeeds)");
}

modal_status modal_get_tuning(modal_h h, modal_tuning* t) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!t) return set_error(MODAL_EINVAL, "t is NULL");
    t->chunk = h->chunk;
    t->legendre_maps = h->tc_maps;
    t->cubic_ctas = h->cubic_ctas;
    t->ms = 0.f;
    return MODAL_OK;
}

modal_status modal_set_tuning(modal_h h, const modal_tuning* t) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!t) return set_error(MODAL_EINVAL, "t is NULL");
    if (t->chunk < 1 || t->chunk > 4096) return set_error(MODAL_EINVAL, "chunk must be in [1, 4096]");
    if (!tc_maps_valid(h->P, t->legendre_maps))
        return set_error(MODAL_EINVAL, "legendre_maps: 2 P legendre_maps must be a multiple of 16 and at most 256");
    const int64_t max_ctas = std::max<int64_t>(1, h->npix / 128);
    if (t->cubic_ctas < 1 || t->cubic_ctas > max_ctas)
        return set_error(MODAL_EINVAL, "cubic_ctas must be in [1, max(1, npix / 128)]");
    CK(cudaDeviceSynchronize(), "set_tuning sync");
    const int old_chunk = h->chunk, old_maps = h->tc_maps, old_ctas = h->cubic_ctas;
    h->tc_maps = t->legendre_maps;
    h->cubic_ctas = t->cubic_ctas;
    const modal_status s = alloc_workspace(h, t->chunk);
    if (s == MODAL_OK) return MODAL_OK;
    const std::string why = modal_last_error();
    h->tc_maps = old_maps;
    h->cubic_ctas = old_ctas;
    if (old_chunk >= 1 && alloc_workspace(h, old_chunk) == MODAL_OK)
        return set_error(s, why + " (the previous tuning is kept)");
    free_workspace(h);
    h->chunk = 0;
    return set_error(s, why + " (the plan has no workspace until modal_set_chunk or modal_set_tuning succeeds)");
}

modal_status modal_autotune(modal_h h, const void* alm, int B, int use_linear, modal_tuning* best, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (check_workspace(h)) return MODAL_ESTATE;
    if (!alm || !best || B < 1) return set_error(MODAL_EINVAL, "alm, best and B >= 1 are required");
    if (use_linear && !h->lin_final) return set_error(MODAL_ESTATE, "linear term requested before modal_linear_term(finalize)");
    cudaStream_t st = as_stream(stream);
    double* beta = nullptr;
    CK(cudaMalloc(&beta, (size_t)B * h->n_max * sizeof(double)), "autotune beta");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // one warm-up call, then the better of two timed calls
    auto time_pass = [&](float* ms) -> modal_status {
        float bestv = 3.4e38f;
        for (int r = 0; r < 3; ++r) {
            CK(cudaEventRecord(e0, st), "autotune event");
            const modal_status s = modal_cubic(h, alm, B, use_linear, beta, stream);
            if (s != MODAL_OK) return s;
            CK(cudaEventRecord(e1, st), "autotune event");
            CK(cudaEventSynchronize(e1), "autotune sync");
            float v = 0.f;
            CK(cudaEventElapsedTime(&v, e0, e1), "autotune time");
            if (r > 0) bestv = std::min(bestv, v);
        }
        *ms = bestv;
        return MODAL_OK;
    };
    modal_tuning cur;
    modal_get_tuning(h, &cur);
    float cur_ms = 0.f;
    modal_status s = time_pass(&cur_ms);
    // a candidate replaces the incumbent only if it is at least 1 % faster; one that cannot
    // be set (its workspace does not fit) is skipped
    auto consider = [&](modal_tuning cand) -> modal_status {
        if (cand.chunk == cur.chunk && cand.legendre_maps == cur.legendre_maps && cand.cubic_ctas == cur.cubic_ctas)
            return MODAL_OK;
        if (modal_set_tuning(h, &cand) != MODAL_OK) return modal_set_tuning(h, &cur);
        float ms = 0.f;
        const modal_status r = time_pass(&ms);
        if (r != MODAL_OK) return r;
        if (ms < 0.99f * cur_ms) {
            cur = cand;
            cur_ms = ms;
            return MODAL_OK;
        }
        return modal_set_tuning(h, &cur);
    };
    const int nsm = h->nsm;
    if (s == MODAL_OK && h->prec != MODAL_FP32) {
        const int gs[] = {32, 28, 24, 20, 16, 14, 12, 10, 8, 6, 4, 2};
        int tried = 0;
        for (int g : gs) {
            if (s != MODAL_OK || tried >= 6) break;
            if (!tc_maps_valid(h->P, g) || g > std::max(8, B)) continue;
            modal_tuning c = cur;
            c.legendre_maps = g;
            s = consider(c);
            ++tried;
        }
    }
    if (s == MODAL_OK) {
        const int64_t max_ctas = std::max<int64_t>(1, h->npix / 128);
        const int cs[] = {std::max(1, nsm / 4), std::max(1, nsm / 2), nsm, 2 * nsm, 4 * nsm, 8 * nsm};
        for (int c : cs) {
            if (s != MODAL_OK) break;
            if (c > max_ctas) continue;
            modal_tuning t = cur;
            t.cubic_ctas = c;
            s = consider(t);
        }
    }
    if (s == MODAL_OK) {
        const int ks[] = {8, 16, 32, 64, 128};
        for (int k : ks) {
            if (s != MODAL_OK) break;
            if (k > B) continue;
            modal_tuning t = cur;
            t.chunk = k;
            s = consider(t);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(beta);
    if (s != MODAL_OK) return s;
    cur.ms = cur_ms;
    *best = cur;
    return MODAL_OK;
}

modal_status modal_synthesize(modal_h h, const void* alm, int B, float* maps, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (check_workspace(h)) return MODAL_ESTATE;
    if (B < 0) return set_error(MODAL_EINVAL, "B < 0");
    if (B > 0 && (!alm || !maps)) return set_error(MODAL_EINVAL, "null pointer");
    cudaStream_t st = as_stream(stream);
    const float2* a = static_cast<const float2*>(alm);
    for (int b0 = 0; b0 < B; b0 += h->chunk) {
        const int nb = std::min(h->chunk, B - b0);
        CK(synth_chunk(h, a + (size_t)b0 * h->n_alm, nb, maps + (size_t)b0 * h->P * h->npix, st), "synthesize");
    }
    return MODAL_OK;
}

modal_status modal_analyze(modal_h h, const float* maps, int B, void* alm, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (check_workspace(h)) return MODAL_ESTATE;
    if (B < 0) return set_error(MODAL_EINVAL, "B < 0");
    if (B > 0 && (!alm || !maps)) return set_error(MODAL_EINVAL, "null pointer");
    cudaStream_t st = as_stream(stream);
    float2* out = static_cast<float2*>(alm);
    const int step = h->chunk * h->P;   // ut holds chunk*P channels
    for (int b0 = 0; b0 < B; b0 += step) {
        const int nb = std::min(step, B - b0);
        { STAGE(h, ST_R2C, st); CK(launch_ring_r2c(*h, maps + (size_t)b0 * h->npix, nb, h->wring, h->ut, nullptr, st), "analyze r2c"); }
        { STAGE(h, ST_LEGENDRE_ADJ, st); CK(launch_legendre_adjoint_simt(*h, h->ut, nb, nullptr, 1, out + (size_t)b0 * h->n_alm, st), "analyze legendre"); }
    }
    return MODAL_OK;
}

// Split plans with per-pixel means take the linear term and the adjoint's pair-mean part in
// harmonic space, from the adjoint transforms of the weighted pair-mean rows; rebuilt whenever
// the per-pixel mean is finalised.
static modal_status refresh_pm_table(modal_plan* h, cudaStream_t st) {
    h->adj_pm_ready = 0;
    if (h->prec == MODAL_FP32 || h->lin_mode == MODAL_LINEAR_RING) return MODAL_OK;
    CK(build_pm_table(*h, st), "pair-mean harmonic table");
    return MODAL_OK;
}

modal_status modal_linear_term(modal_h h, const void* alm_sims, int B, int finalize, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (check_workspace(h)) return MODAL_ESTATE;
    if (B < 0) return set_error(MODAL_EINVAL, "B < 0");
    if (B > 0 && !alm_sims) return set_error(MODAL_EINVAL, "null pointer");
    const bool ring = h->lin_mode == MODAL_LINEAR_RING;
    modal_status s = ring ? ensure_ring_buffers(h) : ensure_pair_buffers(h);
    if (s != MODAL_OK) return s;
    cudaStream_t st = as_stream(stream);
    const float2* a = static_cast<const float2*>(alm_sims);
    for (int b0 = 0; b0 < B; b0 += h->chunk) {
        const int nb = std::min(h->chunk, B - b0);
        CK(synth_chunk(h, a + (size_t)b0 * h->n_alm, nb, h->maps, st), "linear-term synthesis");
        STAGE(h, ST_PAIRS, st);
        if (ring) CK(launch_pair_ring(*h, h->maps, nb, st), "ring pair sums");
        else CK(launch_pair_accumulate(*h, h->maps, nb, st), "pair accumulate");
    }
    h->n_lin += B;
    if (h->retain_maps && B > 0 && B <= h->chunk) {      // the whole batch is in the map workspace
        h->kept_alm = alm_sims;
        h->kept_B = B;
    }
    if (finalize) {
        if (h->n_lin < 1) return set_error(MODAL_ESTATE, "finalize with no linear-term simulations");
        STAGE(h, ST_PAIRS, st);
        if (ring) CK(launch_ring_finalize(*h, st), "ring pair means");
        else CK(launch_pair_finalize(*h, st), "pair finalize");
        const modal_status ps = refresh_pm_table(h, st);
        if (ps != MODAL_OK) return ps;
        h->lin_final = 1;
    }
    return MODAL_OK;
}

// The coefficient pass of B maps; kept: the maps (and, for the ring-mode linear term, their
// Legendre sums) are already in the plan's workspace from an earlier call on the same a_lm.
// The linear-term partial sums of one chunk of nb maps (a: their a_lm, maps: their maps, the
// m = 0 Legendre sums of the same synthesis in h->delta) into lin; returns through *splits
// the number of partial-sum slices beta's finalisation adds.
static modal_status linear_chunk(modal_h h, const float2* a, const float* maps, int nb, double* lin, int* splits,
                                 cudaStream_t st) {
    STAGE(h, ST_LINEAR, st);
    *splits = h->lin_ksplit;
    if (h->lin_mode == MODAL_LINEAR_RING) {
        // ring sums of the maps from the m = 0 Legendre sums still in h->delta
        CK(launch_linear_ring(*h, nb, lin, st), "linear term (ring)");
        *splits = 1;
    } else if (h->prec == MODAL_FP32) {
        CK(launch_linear_gemm(*h, maps, nb, lin, st), "linear gemm");
    } else {
        // from the a_lm and the harmonic pair-mean table (the same finite sums)
        CK(launch_linear_harmonic(*h, a, nb, lin, st), "linear term (harmonic)");
        *splits = 1;
    }
    return MODAL_OK;
}

static double* linear_partial(modal_h h) { return h->partial + (size_t)h->chunk * h->cubic_ctas * h->n_max; }

// After the cubic sums of one chunk of nb maps (a: their a_lm, beta: their rows): the linear
// term (if asked) and beta.
static modal_status cubic_chunk_tail(modal_h h, const float2* a, int nb, int use_linear, double* beta, cudaStream_t st) {
    double* lin = linear_partial(h);
    int splits = h->lin_ksplit;
    if (use_linear) {
        const modal_status r = linear_chunk(h, a, h->maps, nb, lin, &splits, st);
        if (r != MODAL_OK) return r;
    }
    { STAGE(h, ST_BETA, st); CK(launch_beta_finalize(*h, nb, use_linear, h->partial, lin, splits, beta, st), "beta finalize"); }
    return MODAL_OK;
}

static void keep_maps_if_whole(modal_h h, const void* alm, int B) {
    if (h->retain_maps && B > 0 && B <= h->chunk) {      // the whole batch is in the map workspace
        h->kept_alm = alm;
        h->kept_B = B;
    }
}

static modal_status cubic_impl(modal_h h, const void* alm, int B, int use_linear, double* beta, cudaStream_t st,
                               bool kept) {
    const float2* a = static_cast<const float2*>(alm);
    for (int b0 = 0; b0 < B; b0 += h->chunk) {
        const int nb = std::min(h->chunk, B - b0);
        if (!kept) CK(synth_chunk(h, a + (size_t)b0 * h->n_alm, nb, h->maps, st), "cubic synthesis");
        { STAGE(h, ST_CUBIC, st); CK(launch_cubic(*h, h->maps, nb, h->partial, st), "cubic"); }
        const modal_status r = cubic_chunk_tail(h, a + (size_t)b0 * h->n_alm, nb, use_linear, beta + (size_t)b0 * h->n_max, st);
        if (r != MODAL_OK) return r;
    }
    keep_maps_if_whole(h, alm, B);
    return MODAL_OK;
}

modal_status modal_cubic(modal_h h, const void* alm, int B, int use_linear, double* beta, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (check_workspace(h)) return MODAL_ESTATE;
    if (B < 0) return set_error(MODAL_EINVAL, "B < 0");
    if (B > 0 && (!alm || !beta)) return set_error(MODAL_EINVAL, "null pointer");
    if (use_linear && !h->lin_final) return set_error(MODAL_ESTATE, "linear term requested before modal_linear_term(finalize)");
    return cubic_impl(h, alm, B, use_linear, beta, as_stream(stream), false);
}

modal_status modal_cubic_retained(modal_h h, const void* alm, int B, int use_linear, double* beta, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (check_workspace(h)) return MODAL_ESTATE;
    if (B < 0) return set_error(MODAL_EINVAL, "B < 0");
    if (B == 0) return MODAL_OK;
    if (!alm || !beta) return set_error(MODAL_EINVAL, "null pointer");
    if (use_linear && !h->lin_final) return set_error(MODAL_ESTATE, "linear term requested before modal_linear_term(finalize)");
    if (!h->kept_alm || h->kept_alm != alm || h->kept_B != B)
        return set_error(MODAL_ESTATE, "no maps kept for this a_lm and batch (modal_set_retain_maps, B <= chunk, "
                                       "no synthesis or adjoint since the call that kept them)");
    return cubic_impl(h, alm, B, use_linear, beta, as_stream(stream), true);
}

modal_status modal_set_retain_maps(modal_h h, int on) {
    if (check_plan(h)) return MODAL_EINVAL;
    h->retain_maps = on ? 1 : 0;
    if (!on) h->kept_alm = nullptr;
    ++h->generation;
    return MODAL_OK;
}

// Quartic tables once per plan; partial sums, ring sums and the single-pair term sized
// for the current chunk (the pixel-mode single-pair term holds every K split).
static modal_status ensure_quartic(modal_plan* h) {
    if (!h->qt.tiles) {
        CK(quartic_tables(*h), "quartic tables");
        CK(dalloc(h, &h->qt.k3, (size_t)h->qt.n_quad), "quartic two-pair term");
        CK(dalloc(h, &h->qt.kmat, (size_t)std::max(h->lin_ksplit, 1) * h->n_pair * h->n_pair), "quartic two-pair sums");
    }
    if (h->qt.chunk == h->chunk && h->qt.ctas == h->cubic_ctas) return MODAL_OK;
    dfree(h->qt.partial); dfree(h->qt.rq); dfree(h->qt.h);
    h->qt.partial = h->qt.rq = h->qt.h = nullptr;
    h->qt.chunk = 0;
    const size_t np = h->n_pair, ch = h->chunk;
    const size_t hring = ch * np * np, hpix = (size_t)h->lin_ksplit * np * ch * np;
    CK(dalloc(h, &h->qt.partial, ch * h->cubic_ctas * h->qt.n_quad), "quartic partial sums");
    CK(dalloc(h, &h->qt.rq, ch * np * h->nrings), "quartic ring sums");
    CK(dalloc(h, &h->qt.h, std::max(hring, hpix)), "quartic single-pair term");
    h->qt.chunk = h->chunk;
    h->qt.ctas = h->cubic_ctas;
    return MODAL_OK;
}

modal_status modal_quartic(modal_h h, const void* alm, int B, int use_linear, double* tau, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (check_workspace(h)) return MODAL_ESTATE;
    if (B < 0) return set_error(MODAL_EINVAL, "B < 0");
    if (B > 0 && (!alm || !tau)) return set_error(MODAL_EINVAL, "null pointer");
    if (use_linear && !h->lin_final) return set_error(MODAL_ESTATE, "Monte Carlo terms requested before modal_linear_term(finalize)");
    if (B == 0) return MODAL_OK;
    modal_status s = ensure_quartic(h);
    if (s != MODAL_OK) return s;
    cudaStream_t st = as_stream(stream);
    const float2* a = static_cast<const float2*>(alm);
    if (use_linear) { STAGE(h, ST_LINEAR, st); CK(launch_quartic_k3(*h, st), "quartic two-pair term"); }
    for (int b0 = 0; b0 < B; b0 += h->chunk) {
        const int nb = std::min(h->chunk, B - b0);
        CK(synth_chunk(h, a + (size_t)b0 * h->n_alm, nb, h->maps, st), "quartic synthesis");
        { STAGE(h, ST_QUARTIC, st); CK(launch_quartic(*h, h->maps, nb, h->qt.partial, st), "quartic"); }
        if (use_linear) { STAGE(h, ST_LINEAR, st); CK(launch_quartic_linear(*h, h->maps, nb, st), "quartic single-pair term"); }
        { STAGE(h, ST_BETA, st); CK(launch_quartic_finalize(*h, nb, use_linear, tau + (size_t)b0 * h->qt.n_quad, st), "quartic finalize"); }
    }
    return MODAL_OK;
}

modal_status modal_cov_accumulate(modal_h h, const double* beta, int B, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (B < 0) return set_error(MODAL_EINVAL, "B < 0");
    if (B > 0 && !beta) return set_error(MODAL_EINVAL, "null pointer");
    { STAGE(h, ST_COV, as_stream(stream)); CK(launch_cov_accumulate(*h, beta, B, as_stream(stream)), "cov accumulate"); }
    h->n_cov += B;
    return MODAL_OK;
}

// word: the data path's error word (h->d_err) or the FP64 solve's (h->d_err + 1), so that a
// solve running on another stream beside the data path never reads the other's errors.
static modal_status read_device_error(modal_h h, cudaStream_t st, int* word) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, word, sizeof(int), cudaMemcpyDeviceToHost, st), "error word read");
    CK(cudaStreamSynchronize(st), "sync");
    if (e) {
        CK(cudaMemsetAsync(word, 0, sizeof(int), st), "error word clear");
        CK(cudaStreamSynchronize(st), "sync");
        if (e & MODAL_DEVERR_NOTPD) return set_error(MODAL_ENOTPD, "zeta is not positive definite");
        if (e & MODAL_DEVERR_TIMEOUT) return set_error(MODAL_ETIMEOUT, "a device-side wait hit its spin limit");
    }
    return MODAL_OK;
}

modal_status modal_fnl_weights(modal_h h, const double* alpha, double* w, double* sigma, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!alpha || !w) return set_error(MODAL_EINVAL, "alpha and w are required");
    if (h->n_cov < 2) return set_error(MODAL_ESTATE, "need at least 2 covariance simulations");
    cudaStream_t st = as_stream(stream);
    const int n = h->n_max;
    double* ws = nullptr;
    CK(cudaMallocAsync(&ws, ((size_t)n * n + n + 1) * sizeof(double), st), "weights workspace");
    double* A = ws;
    double* v = ws + (size_t)n * n;
    double* norm = v + n;
    auto run = [&]() -> modal_status {
        { STAGE(h, ST_SOLVE, st); CK(launch_zeta(*h, A, st), "zeta"); }
        { STAGE(h, ST_SOLVE, st); CK(launch_cholesky(*h, A, n, st), "cholesky"); }
        CK(cudaMemcpyAsync(v, alpha, n * sizeof(double), cudaMemcpyHostToDevice, st), "alpha copy");
        modal_status es = read_device_error(h, st, h->d_err + 1);
        if (es != MODAL_OK) return es;
        { STAGE(h, ST_SOLVE, st); CK(launch_solve_rhs(*h, A, n, v, 1, st), "triangular solve"); }
        { STAGE(h, ST_SOLVE, st); CK(launch_estimates(*h, v, n, 0, norm, st), "alpha norm"); }
        { STAGE(h, ST_SOLVE, st); CK(launch_fnl_weights(*h, A, n, v, norm, w, st), "back substitution"); }
        double nrm = 0.0;
        CK(cudaMemcpyAsync(&nrm, norm, sizeof(double), cudaMemcpyDeviceToHost, st), "norm copy");
        CK(cudaStreamSynchronize(st), "weights sync");
        if (!(nrm > 0.0)) return set_error(MODAL_ENOTPD, "alpha^T zeta^-1 alpha is not positive");
        if (sigma) *sigma = std::sqrt(6.0 / nrm);
        return MODAL_OK;
    };
    const modal_status s = run();
    cudaFreeAsync(ws, st);
    cudaStreamSynchronize(st);
    return s;
}

modal_status modal_solve(modal_h h, const double* alpha, const double* beta, int B, double* fnl, double* sigma,
                         void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!alpha || B < 0 || (B > 0 && (!beta || !fnl))) return set_error(MODAL_EINVAL, "bad arguments");
    if (h->n_cov < 2) return set_error(MODAL_ESTATE, "need at least 2 covariance simulations");
    cudaStream_t st = as_stream(stream);
    const int n = h->n_max;
    double* ws = nullptr;
    CK(cudaMallocAsync(&ws, ((size_t)n * n + (size_t)(B + 1) * n + (B + 1)) * sizeof(double), st), "solve workspace");
    double* A = ws;
    double* rhs = ws + (size_t)n * n;
    double* est = rhs + (size_t)(B + 1) * n;
    modal_status s = MODAL_OK;
    auto run = [&]() -> modal_status {
        { STAGE(h, ST_SOLVE, st); CK(launch_zeta(*h, A, st), "zeta"); }
        { STAGE(h, ST_SOLVE, st); CK(launch_cholesky(*h, A, n, st), "cholesky"); }
        CK(cudaMemcpyAsync(rhs, alpha, n * sizeof(double), cudaMemcpyHostToDevice, st), "alpha copy");
        if (B > 0) CK(cudaMemcpyAsync(rhs + n, beta, (size_t)B * n * sizeof(double), cudaMemcpyDeviceToDevice, st), "beta copy");
        modal_status es = read_device_error(h, st, h->d_err + 1);
        if (es != MODAL_OK) return es;
        { STAGE(h, ST_SOLVE, st); CK(launch_solve_rhs(*h, A, n, rhs, B + 1, st), "triangular solve"); }
        { STAGE(h, ST_SOLVE, st); CK(launch_estimates(*h, rhs, n, B, est, st), "estimates"); }
        std::vector<double> out(B + 1);
        CK(cudaMemcpyAsync(out.data(), est, (B + 1) * sizeof(double), cudaMemcpyDeviceToHost, st), "estimates copy");
        CK(cudaStreamSynchronize(st), "solve sync");
        if (!(out[0] > 0.0)) return set_error(MODAL_ENOTPD, "alpha^T zeta^-1 alpha is not positive");
        if (sigma) *sigma = std::sqrt(6.0 / out[0]);
        for (int b = 0; b < B; ++b) fnl[b] = out[1 + b];
        return MODAL_OK;
    };
    s = run();
    cudaFreeAsync(ws, st);
    cudaStreamSynchronize(st);
    return s;
}

// Power iteration of the bivector fit: stop when |Z v - lam v| <= kPowerTol |lam|, checked
// every kPowerCheck steps (the error of v is about that residual over the eigenvalue gap).
constexpr int kPowerMaxIters = 20000, kPowerCheck = 16;
constexpr double kPowerTol = 1e-12;

// Copies the host zeta0 into A and factors it in place (lower triangle = L0).
static modal_status factor_zeta0(modal_h h, const double* zeta0, double* A, cudaStream_t st) {
    const int n = h->n_max;
    CK(cudaMemcpyAsync(A, zeta0, (size_t)n * n * sizeof(double), cudaMemcpyHostToDevice, st), "zeta0 copy");
    { STAGE(h, ST_SOLVE, st); CK(launch_cholesky(*h, A, n, st), "cholesky of zeta0"); }
    modal_status es = read_device_error(h, st, h->d_err + 1);
    if (es == MODAL_ENOTPD) return set_error(MODAL_ENOTPD, "zeta0 is not positive definite");
    return es;
}

modal_status modal_bivector_fit(modal_h h, const double* zeta0, double* bt, double* lambda1, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!zeta0 || !bt) return set_error(MODAL_EINVAL, "null pointer");
    if (h->n_cov < 2) return set_error(MODAL_ESTATE, "need at least 2 covariance simulations");
    cudaStream_t st = as_stream(stream);
    const int n = h->n_max;
    double* ws = nullptr;
    CK(cudaMallocAsync(&ws, ((size_t)3 * n * n + 2 * (size_t)n + 2) * sizeof(double), st), "fit workspace");
    double* L0 = ws;
    double* Z = L0 + (size_t)n * n;
    double* T = Z + (size_t)n * n;
    double* v = T + (size_t)n * n;
    double* w = v + n;
    double* stat = w + n;
    auto run = [&]() -> modal_status {
        modal_status s = factor_zeta0(h, zeta0, L0, st);
        if (s != MODAL_OK) return s;
        {
            // whitened Z = L0^-1 zeta L0^-T: the rows of zeta (= its columns) are solved
            // against L0, giving (L0^-1 zeta)^T; its transpose's rows are solved again.
            STAGE(h, ST_SOLVE, st);
            CK(launch_zeta(*h, Z, st), "zeta");
            CK(launch_solve_rhs(*h, L0, n, Z, n, st), "whitening solve");
            CK(launch_transpose(*h, n, Z, T, st), "transpose");
            CK(launch_solve_rhs(*h, L0, n, T, n, st), "whitening solve");
        }
        std::vector<double> hv(n, 1.0 / std::sqrt((double)n));
        CK(cudaMemcpyAsync(v, hv.data(), n * sizeof(double), cudaMemcpyHostToDevice, st), "start vector");
        double hs[2] = {0.0, 0.0};
        bool converged = false;
        for (int it = 0; it < kPowerMaxIters && !converged; it += kPowerCheck) {
            {
                STAGE(h, ST_SOLVE, st);
                for (int k = 0; k < kPowerCheck; ++k) CK(launch_power_step(*h, n, T, v, w, stat, st), "power step");
            }
            CK(cudaMemcpyAsync(hs, stat, sizeof(hs), cudaMemcpyDeviceToHost, st), "eigenvalue read");
            CK(cudaStreamSynchronize(st), "sync");
            if (!std::isfinite(hs[0])) return set_error(MODAL_ENOTPD, "power iteration produced a non-finite value");
            converged = hs[1] <= kPowerTol * std::fabs(hs[0]);
        }
        if (!converged) return set_error(MODAL_ENOCONV, "power iteration for the bivector did not converge");
        // v was renormalised after the last residual: |Z v_old| v = Z v_old, the same direction
        CK(cudaMemcpyAsync(hv.data(), v, n * sizeof(double), cudaMemcpyDeviceToHost, st), "eigenvector read");
        CK(cudaStreamSynchronize(st), "sync");
        const double l1 = hs[0] - 1.0;
        double sum = 0.0;
        for (int i = 0; i < n; ++i) sum += hv[i];
        const double scale = std::sqrt(std::max(l1, 0.0)) * (sum < 0.0 ? -1.0 : 1.0);
        for (int i = 0; i < n; ++i) bt[i] = scale * hv[i];
        if (lambda1) *lambda1 = l1;
        return MODAL_OK;
    };
    modal_status s = run();
    cudaFreeAsync(ws, st);
    cudaStreamSynchronize(st);
    return s;
}

modal_status modal_solve_bivector(modal_h h, const double* zeta0, const double* bt, const double* alpha,
                                  const double* beta, int B, double* fnl, double* sigma, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!zeta0 || !bt || !alpha || B < 0 || (B > 0 && (!beta || !fnl))) return set_error(MODAL_EINVAL, "bad arguments");
    cudaStream_t st = as_stream(stream);
    const int n = h->n_max;
    double* ws = nullptr;
    CK(cudaMallocAsync(&ws, ((size_t)n * n + (size_t)(B + 2) * n + (B + 1)) * sizeof(double), st), "solve workspace");
    double* L0 = ws;
    double* rhs = L0 + (size_t)n * n;
    double* dbt = rhs + (size_t)(B + 1) * n;
    double* est = dbt + n;
    auto run = [&]() -> modal_status {
        modal_status s = factor_zeta0(h, zeta0, L0, st);
        if (s != MODAL_OK) return s;
        CK(cudaMemcpyAsync(rhs, alpha, n * sizeof(double), cudaMemcpyHostToDevice, st), "alpha copy");
        if (B > 0) CK(cudaMemcpyAsync(rhs + n, beta, (size_t)B * n * sizeof(double), cudaMemcpyDeviceToDevice, st), "beta copy");
        CK(cudaMemcpyAsync(dbt, bt, n * sizeof(double), cudaMemcpyHostToDevice, st), "bt copy");
        {
            STAGE(h, ST_SOLVE, st);
            CK(launch_solve_rhs(*h, L0, n, rhs, B + 1, st), "triangular solve");
            CK(launch_bivector_estimates(*h, rhs, n, B, dbt, est, st), "bivector estimates");
        }
        std::vector<double> out(B + 1);
        CK(cudaMemcpyAsync(out.data(), est, (B + 1) * sizeof(double), cudaMemcpyDeviceToHost, st), "estimates copy");
        CK(cudaStreamSynchronize(st), "solve sync");
        if (!(out[0] > 0.0)) return set_error(MODAL_ENOTPD, "alpha'^T (I + bt bt^T)^-1 alpha' is not positive");
        if (sigma) *sigma = std::sqrt(6.0 / out[0]);
        for (int b = 0; b < B; ++b) fnl[b] = out[1 + b];
        return MODAL_OK;
    };
    modal_status s = run();
    cudaFreeAsync(ws, st);
    cudaStreamSynchronize(st);
    return s;
}

modal_status modal_bivector_rotate(modal_h h, const double* zeta0, const double* bt, const double* x, int B,
                                   double* out, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!zeta0 || !bt || B < 0 || (B > 0 && (!x || !out))) return set_error(MODAL_EINVAL, "bad arguments");
    cudaStream_t st = as_stream(stream);
    const int n = h->n_max;
    double* ws = nullptr;
    CK(cudaMallocAsync(&ws, ((size_t)n * n + n) * sizeof(double), st), "rotate workspace");
    double* L0 = ws;
    double* dbt = L0 + (size_t)n * n;
    auto run = [&]() -> modal_status {
        modal_status s = factor_zeta0(h, zeta0, L0, st);
        if (s != MODAL_OK) return s;
        CK(cudaMemcpyAsync(dbt, bt, n * sizeof(double), cudaMemcpyHostToDevice, st), "bt copy");
        if (B > 0 && out != x)
            CK(cudaMemcpyAsync(out, x, (size_t)B * n * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy");
        STAGE(h, ST_SOLVE, st);
        CK(launch_solve_rhs(*h, L0, n, out, B, st), "triangular solve");
        CK(launch_bivector_rotate(*h, n, B, dbt, out, st), "bivector rotation");
        return MODAL_OK;
    };
    modal_status s = run();
    cudaFreeAsync(ws, st);
    CK(cudaStreamSynchronize(st), "rotate sync");
    return s;
}

// kept: the maps of a (one chunk) are already in h->maps (modal_backward_retained)
static modal_status backward_impl(modal_h h, const void* alm, int B, const double* g, int use_linear, void* grad_alm,
                                  cudaStream_t st, bool kept) {
    const float2* a = static_cast<const float2*>(alm);
    float2* out = static_cast<float2*>(grad_alm);
    // ring mode: the pair-mean term is constant on each ring and enters only through m = 0
    const bool ring = use_linear && h->lin_mode == MODAL_LINEAR_RING;
    // split plans, per-pixel means: the pair-mean term enters after the transposed Legendre
    // sums, through the adjoint transform of each weighted pair-mean row (built once per mean)
    const bool pm_late = use_linear && !ring && h->prec != MODAL_FP32;
    if (pm_late && !h->adj_pm_ready) {
        STAGE(h, ST_OTHER, st);
        CK(build_pm_table(*h, st), "pair-mean harmonic table");
    }
    for (int b0 = 0; b0 < B; b0 += h->chunk) {
        const int nb = std::min(h->chunk, B - b0);
        if (!kept) CK(synth_chunk(h, a + (size_t)b0 * h->n_alm, nb, h->maps, st), "backward synthesis");
        h->kept_alm = nullptr;                              // U overwrites the maps
        { STAGE(h, ST_ADJ_PIXEL, st); CK(launch_adjoint_weights(*h, g + (size_t)b0 * h->n_max, nb, h->hk, st), "adjoint weights"); }
        {
            STAGE(h, ST_ADJ_PIXEL, st);
            if (ring) CK(launch_vring(*h, h->hk, nb, h->vring, st), "adjoint ring term");
            if (h->prec == MODAL_FP32)
                CK(launch_adjoint_u(*h, h->maps, nb, h->hk, use_linear && !ring, h->maps, st), "adjoint pixel");
            else
                CK(launch_adjoint_v(*h, nb, h->hk, h->maps, st), "adjoint pixel");
        }
        {
            // split precisions: the r2c kernel also records each map's max |U~| for the operand scale
            STAGE(h, ST_R2C, st);
            unsigned* amax = (h->prec == MODAL_FP32) ? nullptr : h->tc.d_amax;
            if (amax) CK(cudaMemsetAsync(amax, 0, nb * sizeof(unsigned), st), "adjoint scale clear");
            CK(launch_ring_r2c(*h, h->maps, nb * h->P, nullptr, h->ut, amax, st), "adjoint r2c");
            if (ring) CK(launch_vring_correct(*h, h->vring, nb * h->P, h->ut, amax, st), "adjoint ring term");
        }
        if (h->prec == MODAL_FP32) {
            STAGE(h, ST_LEGENDRE_ADJ, st);
            CK(launch_legendre_adjoint_simt(*h, h->ut, nb, h->filt, h->P, out + (size_t)b0 * h->n_alm, st), "adjoint legendre");
        } else {
            { STAGE(h, ST_LEGENDRE_ADJ_PREP, st); CK(launch_legendre_adjoint_tc(*h, h->ut, nb, out + (size_t)b0 * h->n_alm, true, 1, st), "adjoint legendre prep"); }
            { STAGE(h, ST_LEGENDRE_ADJ, st); CK(launch_legendre_adjoint_tc(*h, h->ut, nb, out + (size_t)b0 * h->n_alm, true, 2, st), "adjoint legendre"); }
        }
        if (pm_late) {
            STAGE(h, ST_ADJ_PIXEL, st);
            // the Legendre sums' workspace is free once the transposed sums are done
            CK(launch_adjoint_pm(*h, nb, h->hk, out + (size_t)b0 * h->n_alm, h->delta, st), "adjoint pair-mean term");
        }
    }
    return MODAL_OK;
}

modal_status modal_backward(modal_h h, const void* alm, int B, const double* g, int use_linear, void* grad_alm,
                            void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (check_workspace(h)) return MODAL_ESTATE;
    if (B < 0) return set_error(MODAL_EINVAL, "B < 0");
    if (B > 0 && (!alm || !g || !grad_alm)) return set_error(MODAL_EINVAL, "null pointer");
    if (use_linear && !h->lin_final) return set_error(MODAL_ESTATE, "linear term requested before modal_linear_term(finalize)");
    return backward_impl(h, alm, B, g, use_linear, grad_alm, as_stream(stream), false);
}

modal_status modal_backward_retained(modal_h h, const void* alm, int B, const double* g, int use_linear,
                                     void* grad_alm, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (check_workspace(h)) return MODAL_ESTATE;
    if (B < 0) return set_error(MODAL_EINVAL, "B < 0");
    if (B == 0) return MODAL_OK;
    if (!alm || !g || !grad_alm) return set_error(MODAL_EINVAL, "null pointer");
    if (use_linear && !h->lin_final) return set_error(MODAL_ESTATE, "linear term requested before modal_linear_term(finalize)");
    if (!h->kept_alm || h->kept_alm != alm || h->kept_B != B)
        return set_error(MODAL_ESTATE, "no maps kept for this a_lm and batch (modal_set_retain_maps, B <= chunk, "
                                       "no synthesis or adjoint since the modal_cubic call)");
    return backward_impl(h, alm, B, g, use_linear, grad_alm, as_stream(stream), true);
}

modal_status modal_alpha_local(modal_h h, const double* C_signal, double* alpha) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!alpha) return set_error(MODAL_EINVAL, "alpha is NULL");
    const int L = h->lmax, P = h->P;
    const double* cs = C_signal ? C_signal : h->cl.data();
    std::vector<double> x, wx;
    gauss_legendre(3 * L / 2 + 2, x, wx);
    const int nx = (int)x.size();
    // A_p(x) = sum_l (2l+1)/4pi C_l f_p(l) P_l(x), D_p(x) = sum_l (2l+1)/4pi f_p(l) P_l(x)
    std::vector<double> A((size_t)P * nx, 0.0), D((size_t)P * nx, 0.0);
    for (int i = 0; i < nx; ++i) {
        double p0 = 1.0, p1 = x[i];
        for (int l = 0; l <= L; ++l) {
            double pl;
            if (l == 0) pl = 1.0;
            else if (l == 1) pl = x[i];
            else {
                pl = ((2.0 * l - 1.0) * x[i] * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = pl;
            }
            if (h->cl[l] <= 0) continue;
            const double c = (2.0 * l + 1.0) / (4.0 * M_PI) * pl / std::sqrt(h->cl[l]);
            for (int p = 0; p < P; ++p) {
                const double f = h->basis[(size_t)p * (L + 1) + l] * c;
                D[(size_t)p * nx + i] += f;
                A[(size_t)p * nx + i] += f * cs[l];
            }
        }
    }
    for (int n = 0; n < h->n_max; ++n) {
        const int p = h->mode_p[n], r = h->mode_r[n], s = h->mode_s[n];
        double acc = 0.0;
        for (int i = 0; i < nx; ++i) {
            const double* a = A.data();
            const double* d = D.data();
            acc += wx[i] * (a[p * nx + i] * a[r * nx + i] * d[s * nx + i] + a[p * nx + i] * d[r * nx + i] * a[s * nx + i]
                            + d[p * nx + i] * a[r * nx + i] * a[s * nx + i]);
        }
        alpha[n] = 16.0 * M_PI * M_PI * acc;
    }
    return MODAL_OK;
}

modal_status modal_get_info(modal_h h, modal_info* info) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!info) return set_error(MODAL_EINVAL, "info is NULL");
    info->lmax = h->lmax; info->P = h->P; info->nrings = h->nrings; info->nphi = h->nphi; info->prec = h->prec;
    info->n_alm = h->n_alm; info->n_max = h->n_max; info->n_pair = h->n_pair; info->npix = h->npix;
    info->n_lin = h->n_lin; info->n_cov = h->n_cov; info->lin_final = h->lin_final; info->chunk = h->chunk;
    info->device_bytes = h->device_bytes;
    info->n_quad = h->P * (h->P + 1) * (h->P + 2) * (h->P + 3) / 24;
    return MODAL_OK;
}

modal_status modal_get_rings(modal_h h, double* mu, double* w) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (mu) std::memcpy(mu, h->mu.data(), h->nrings * sizeof(double));
    if (w) std::memcpy(w, h->w.data(), h->nrings * sizeof(double));
    return MODAL_OK;
}

modal_status modal_get_pair_mean(modal_h h, float* out, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!out) return set_error(MODAL_EINVAL, "out is NULL");
    if (!h->lin_final) return set_error(MODAL_ESTATE, "pair mean not finalised");
    if (h->lin_mode == MODAL_LINEAR_RING) {
        CK(launch_ring_mean_float(*h, out, as_stream(stream)), "ring pair means copy");
        return MODAL_OK;
    }
    CK(cudaMemcpyAsync(out, h->pair_mean, (size_t)h->n_pair * h->npix * sizeof(float), cudaMemcpyDeviceToDevice,
                       as_stream(stream)), "pair mean copy");
    return MODAL_OK;
}

modal_status modal_get_zeta(modal_h h, double* zeta) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!zeta) return set_error(MODAL_EINVAL, "zeta is NULL");
    if (h->n_cov < 2) return set_error(MODAL_ESTATE, "need at least 2 covariance simulations");
    double* d = nullptr;
    const size_t nn = (size_t)h->n_max * h->n_max;
    CK(cudaMalloc(&d, nn * sizeof(double)), "zeta workspace");
    cudaError_t e = launch_zeta(*h, d, 0);
    if (e == cudaSuccess) e = cudaMemcpy(zeta, d, nn * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    CK(e, "zeta");
    return MODAL_OK;
}

modal_status modal_reset(modal_h h, int what) {
    if (check_plan(h)) return MODAL_EINVAL;
    CK(cudaDeviceSynchronize(), "reset sync");
    ++h->generation;
    if (what & 1) {
        if (h->pair_sum) CK(cudaMemset(h->pair_sum, 0, (size_t)h->n_pair * h->npix * sizeof(double)), "reset pair sums");
        if (h->ring_sum) CK(cudaMemset(h->ring_sum, 0, (size_t)h->n_pair * h->nrings * sizeof(double)), "reset ring sums");
        h->n_lin = 0;
        h->lin_final = 0;
        h->adj_pm_ready = 0;
    }
    if (what & 2) {
        CK(cudaMemset(h->S1, 0, h->n_max * sizeof(double)), "reset S1");
        CK(cudaMemset(h->S2, 0, (size_t)h->n_max * h->n_max * sizeof(double)), "reset S2");
        h->n_cov = 0;
    }
    return MODAL_OK;
}

modal_status modal_sync(modal_h h, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    cudaStream_t st = as_stream(stream);
    CK(cudaStreamSynchronize(st), "sync");
    CK(cudaGetLastError(), "sync");
    return read_device_error(h, st, h->d_err);
}

modal_status modal_selftest_wait(modal_h h, int spin_limit, void* stream) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (spin_limit < 1) return set_error(MODAL_EINVAL, "spin_limit must be >= 1");
    { STAGE(h, ST_OTHER, as_stream(stream)); CK(launch_wait_selftest(h->d_err, spin_limit, as_stream(stream)), "wait selftest"); }
    return MODAL_OK;
}

// State file: magic, sizes, n_lin, lin_final, n_cov, then pair sums (if present), S1, S2.
struct StateHeader {
    char magic[8];
    int32_t lmax, P, nrings, nphi;
    int64_t n_lin, n_cov;
    int32_t lin_final, has_pairs;
};

modal_status modal_save_state(modal_h h, const char* path) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!path) return set_error(MODAL_EINVAL, "path is NULL");
    CK(cudaDeviceSynchronize(), "save sync");
    FILE* f = std::fopen(path, "wb");
    if (!f) return set_error(MODAL_EINVAL, std::string("cannot open ") + path);
    StateHeader hd{};
    std::memcpy(hd.magic, "MODALST1", 8);
    hd.lmax = h->lmax; hd.P = h->P; hd.nrings = h->nrings; hd.nphi = h->nphi;
    hd.n_lin = h->n_lin; hd.n_cov = h->n_cov; hd.lin_final = h->lin_final;
    hd.has_pairs = (h->lin_mode == MODAL_LINEAR_RING) ? (h->ring_sum ? 2 : 0) : (h->pair_sum ? 1 : 0);
    bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
    auto dump = [&](const double* d, size_t n) {
        std::vector<double> buf(std::min<size_t>(n, (size_t)1 << 24));
        for (size_t off = 0; ok && off < n; off += buf.size()) {
            const size_t m = std::min(buf.size(), n - off);
            if (cudaMemcpy(buf.data(), d + off, m * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
            else ok = std::fwrite(buf.data(), sizeof(double), m, f) == m;
        }
    };
    if (hd.has_pairs == 1) dump(h->pair_sum, (size_t)h->n_pair * h->npix);
    if (hd.has_pairs == 2) dump(h->ring_sum, (size_t)h->n_pair * h->nrings);
    dump(h->S1, h->n_max);
    dump(h->S2, (size_t)h->n_max * h->n_max);
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return set_error(MODAL_ECUDA, "state write failed");
    return MODAL_OK;
}

modal_status modal_load_state(modal_h h, const char* path) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (!path) return set_error(MODAL_EINVAL, "path is NULL");
    FILE* f = std::fopen(path, "rb");
    if (!f) return set_error(MODAL_EINVAL, std::string("cannot open ") + path);
    StateHeader hd{};
    bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1 && std::memcmp(hd.magic, "MODALST1", 8) == 0 &&
              hd.lmax == h->lmax && hd.P == h->P && hd.nrings == h->nrings && hd.nphi == h->nphi;
    if (!ok) {
        std::fclose(f);
        return set_error(MODAL_EINVAL, "state file does not match this plan");
    }
    CK(cudaDeviceSynchronize(), "load sync");
    ++h->generation;
    if (hd.has_pairs && (hd.has_pairs == 2) != (h->lin_mode == MODAL_LINEAR_RING)) {
        std::fclose(f);
        return set_error(MODAL_EINVAL, "state file holds the other linear-term mode");
    }
    if (hd.has_pairs) {
        modal_status s = (hd.has_pairs == 2) ? ensure_ring_buffers(h) : ensure_pair_buffers(h);
        if (s != MODAL_OK) { std::fclose(f); return s; }
    }
    auto load = [&](double* d, size_t n) {
        std::vector<double> buf(std::min<size_t>(n, (size_t)1 << 24));
        for (size_t off = 0; ok && off < n; off += buf.size()) {
            const size_t m = std::min(buf.size(), n - off);
            ok = std::fread(buf.data(), sizeof(double), m, f) == m &&
                 cudaMemcpy(d + off, buf.data(), m * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
        }
    };
    if (hd.has_pairs == 1) load(h->pair_sum, (size_t)h->n_pair * h->npix);
    if (hd.has_pairs == 2) load(h->ring_sum, (size_t)h->n_pair * h->nrings);
    load(h->S1, h->n_max);
    load(h->S2, (size_t)h->n_max * h->n_max);
    std::fclose(f);
    if (!ok) return set_error(MODAL_EINVAL, "state file truncated");
    h->n_lin = hd.n_lin;
    h->n_cov = hd.n_cov;
    h->lin_final = 0;
    h->adj_pm_ready = 0;
    if (hd.has_pairs && hd.lin_final && h->n_lin > 0) {
        if (hd.has_pairs == 2) CK(launch_ring_finalize(*h, 0), "ring pair means");
        else CK(launch_pair_finalize(*h, 0), "pair finalize");
        const modal_status ps = refresh_pm_table(h, 0);
        if (ps != MODAL_OK) return ps;
        CK(cudaDeviceSynchronize(), "load sync");
        h->lin_final = 1;
    }
    return MODAL_OK;
}

static const char* kStageNames[MODAL_NSTAGES] = {
    "legendre", "ring_c2r", "cubic", "linear_term", "beta_finalize", "pair_means",
    "cov_accumulate", "solve", "adjoint_pixel", "ring_r2c", "legendre_adjoint", "other",
    "legendre_prep", "legendre_adjoint_prep", "quartic"};

const char* modal_stage_name(int stage) {
    return (stage >= 0 && stage < MODAL_NSTAGES) ? kStageNames[stage] : "";
}

modal_status modal_set_profiling(modal_h h, int enable) {
    if (check_plan(h)) return MODAL_EINVAL;
    h->prof = enable ? 1 : 0;
    return MODAL_OK;
}

modal_status modal_get_profile(modal_h h, double* stage_ms, long long* launches, int nstages) {
    if (check_plan(h)) return MODAL_EINVAL;
    if (nstages < 0 || nstages > MODAL_NSTAGES) return set_error(MODAL_EINVAL, "nstages out of range");
    CK(cudaDeviceSynchronize(), "profile sync");
    for (auto& pe : h->prof_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) h->stage_ms[pe.first] += ms;
        h->prof_pool.push_back(pe.second.first);
        h->prof_pool.push_back(pe.second.second);
    }
    h->prof_pending.clear();
    for (int s = 0; s < nstages; ++s) {
        if (stage_ms) stage_ms[s] = h->stage_ms[s];
        if (launches) launches[s] = h->stage_launches[s];
    }
    for (int s = 0; s < MODAL_NSTAGES; ++s) {
        h->stage_ms[s] = 0.0;
        h->stage_launches[s] = 0;
    }
    return MODAL_OK;
}

// ------------------------------------------------------------------ mixed-l_max batches
}  // extern "C"

struct modal_batch {
    std::vector<modal_h> plans;
    cudaStream_t main = nullptr;                  // the batch's own (capturable) stream
    std::vector<cudaStream_t> side;               // one per plan
    std::vector<cudaEvent_t> done;                // one per plan
    cudaEvent_t fork = nullptr, in = nullptr, out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // arguments the captured graph was made with
    std::vector<const void*> key_alm;
    std::vector<int> key_B;
    std::vector<double*> key_beta;
    std::vector<unsigned long long> key_gen;      // the plans' generations at capture
    int key_linear = -1;
    int schedule = MODAL_BATCH_STREAMS;
    cudaEvent_t cubic_done = nullptr;             // the shared cubic launch of one chunk pass
    int* counter = nullptr;                       // its work-queue counter (device)
};

static void batch_drop_graph(modal_batch* bh) {
    if (bh->exec) cudaGraphExecDestroy(bh->exec);
    if (bh->graph) cudaGraphDestroy(bh->graph);
    bh->exec = nullptr;
    bh->graph = nullptr;
    bh->key_linear = -1;
}

// True if the plans' cubic sums can share one launch: the same P (so the same mode tables
// and kernel instance) and at most CUBIC_MAX_JOBS plans with maps in the call.
static bool batch_shares_cubic(const modal_batch* bh, const int* B) {
    if (bh->schedule != MODAL_BATCH_SHARED_CUBIC) return false;
    int n = 0;
    const modal_plan* p0 = nullptr;
    for (size_t i = 0; i < bh->plans.size(); ++i) {
        if (B[i] == 0) continue;
        const modal_plan* p = bh->plans[i];
        if (!p0) p0 = p;
        if (p->P != p0->P || p->n_max != p0->n_max || p->n_tiles != p0->n_tiles || p->cubic_nslots != p0->cubic_nslots)
            return false;
        ++n;
    }
    return n >= 2 && n <= CUBIC_MAX_JOBS;
}

// Chunk passes over the plans with maps in the call.  Pass k: each plan synthesizes its k-th
// chunk on its own stream; one persistent cubic launch on bh->main takes the (plan, map,
// pixel range) items of every plan's chunk k from a work queue, plans with the longest pixel
// ranges first; then each plan's linear term and beta follow on its stream, and its next
// synthesis after them.  Every item is the one the plan's own launch computes, so beta is
// identical to modal_cubic's.
static modal_status batch_run_shared(modal_batch* bh, const void* const* alm, const int* B, int use_linear,
                                     double* const* beta) {
    const size_t n = bh->plans.size();
    std::vector<size_t> order;
    int passes = 0;
    for (size_t i = 0; i < n; ++i)
        if (B[i] > 0) {
            order.push_back(i);
            passes = std::max(passes, (B[i] + bh->plans[i]->chunk - 1) / bh->plans[i]->chunk);
        }
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        const modal_plan *px = bh->plans[x], *py = bh->plans[y];
        return (px->npix + px->cubic_ctas - 1) / px->cubic_ctas > (py->npix + py->cubic_ctas - 1) / py->cubic_ctas;
    });
    CK(cudaEventRecord(bh->fork, bh->main), "batch fork");
    for (size_t i : order) CK(cudaStreamWaitEvent(bh->side[i], bh->fork, 0), "batch fork wait");
    for (int k = 0; k < passes; ++k) {
        std::vector<Plan*> pl;
        std::vector<const float*> mp;
        std::vector<int> nb;
        for (size_t i : order) {
            modal_plan* h = bh->plans[i];
            const int b0 = k * h->chunk;
            if (b0 >= B[i]) continue;
            pl.push_back(h);
            mp.push_back(h->maps);
            nb.push_back(std::min(h->chunk, B[i] - b0));
            const float2* a = static_cast<const float2*>(alm[i]) + (size_t)b0 * h->n_alm;
            CK(synth_chunk(h, a, nb.back(), h->maps, bh->side[i]), "cubic synthesis");
            CK(cudaEventRecord(bh->done[i], bh->side[i]), "batch pass join");
            CK(cudaStreamWaitEvent(bh->main, bh->done[i], 0), "batch pass join wait");
        }
        {
            STAGE(static_cast<modal_plan*>(pl[0]), ST_CUBIC, bh->main);
            CK(launch_cubic_multi(pl.data(), mp.data(), nb.data(), (int)pl.size(), bh->counter, bh->main), "shared cubic");
        }
        CK(cudaEventRecord(bh->cubic_done, bh->main), "batch pass fork");
        for (size_t i : order) {
            modal_plan* h = bh->plans[i];
            const int b0 = k * h->chunk;
            if (b0 >= B[i]) continue;
            CK(cudaStreamWaitEvent(bh->side[i], bh->cubic_done, 0), "batch pass fork wait");
            const float2* a = static_cast<const float2*>(alm[i]) + (size_t)b0 * h->n_alm;
            const modal_status r = cubic_chunk_tail(h, a, std::min(h->chunk, B[i] - b0), use_linear,
                                                    beta[i] + (size_t)b0 * h->n_max, bh->side[i]);
            if (r != MODAL_OK) return r;
        }
    }
    for (size_t i : order) {
        keep_maps_if_whole(bh->plans[i], alm[i], B[i]);
        CK(cudaEventRecord(bh->done[i], bh->side[i]), "batch join");
        CK(cudaStreamWaitEvent(bh->main, bh->done[i], 0), "batch join wait");
    }
    return MODAL_OK;
}

// Fork to the plans' streams, run every plan's coefficient pass, join back on bh->main.
static modal_status batch_run(modal_batch* bh, const void* const* alm, const int* B, int use_linear,
                              double* const* beta) {
    if (batch_shares_cubic(bh, B)) return batch_run_shared(bh, alm, B, use_linear, beta);
    CK(cudaEventRecord(bh->fork, bh->main), "batch fork");
    for (size_t i = 0; i < bh->plans.size(); ++i) {
        CK(cudaStreamWaitEvent(bh->side[i], bh->fork, 0), "batch fork wait");
        const modal_status r = modal_cubic(bh->plans[i], alm[i], B[i], use_linear, beta[i], bh->side[i]);
        if (r != MODAL_OK) return r;
        CK(cudaEventRecord(bh->done[i], bh->side[i]), "batch join");
        CK(cudaStreamWaitEvent(bh->main, bh->done[i], 0), "batch join wait");
    }
    return MODAL_OK;
}

extern "C" {

modal_status modal_batch_create(const modal_h* plans, int nplans, modal_batch_h* out) {
    if (!out || !plans || nplans < 1) return set_error(MODAL_EINVAL, "batch needs at least one plan");
    *out = nullptr;
    for (int i = 0; i < nplans; ++i) {
        if (!plans[i]) return set_error(MODAL_EINVAL, "null plan in batch");
        if (plans[i]->dev != plans[0]->dev) return set_error(MODAL_EINVAL, "batch plans on different devices");
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return set_error(MODAL_EINVAL, "plan repeated in batch");
    }
    CK(cudaSetDevice(plans[0]->dev), "set device");
    auto* bh = new modal_batch();
    bh->plans.assign(plans, plans + nplans);
    bool ok = cudaStreamCreateWithFlags(&bh->main, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&bh->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&bh->in, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&bh->out, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&bh->cubic_done, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&bh->counter, sizeof(int)) == cudaSuccess;
    for (int i = 0; ok && i < nplans; ++i) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (s) bh->side.push_back(s);
        if (e) bh->done.push_back(e);
    }
    if (!ok) {
        modal_batch_destroy(bh);
        return set_error(MODAL_ECUDA, std::string("batch streams/events: ") + cudaGetErrorString(cudaGetLastError()));
    }
    *out = bh;
    return MODAL_OK;
}

modal_status modal_batch_cubic(modal_batch_h bh, const void* const* alm, const int* B, int use_linear,
                               double* const* beta, int use_graph, void* stream) {
    if (!bh || !alm || !B || !beta) return set_error(MODAL_EINVAL, "null batch argument");
    const size_t n = bh->plans.size();
    for (size_t i = 0; i < n; ++i) {
        if (B[i] < 0) return set_error(MODAL_EINVAL, "B < 0");
        if (B[i] > 0 && (!alm[i] || !beta[i])) return set_error(MODAL_EINVAL, "null pointer");
        if (use_linear && !bh->plans[i]->lin_final)
            return set_error(MODAL_ESTATE, "linear term requested before modal_linear_term(finalize)");
        if (check_workspace(bh->plans[i])) return MODAL_ESTATE;
    }
    CK(cudaSetDevice(bh->plans[0]->dev), "set device");
    const cudaStream_t st = as_stream(stream);
    CK(cudaEventRecord(bh->in, st), "batch in");
    CK(cudaStreamWaitEvent(bh->main, bh->in, 0), "batch in wait");
    if (!use_graph) {
        const modal_status r = batch_run(bh, alm, B, use_linear, beta);
        if (r != MODAL_OK) return r;
    } else {
        std::vector<unsigned long long> gen(n);
        for (size_t i = 0; i < n; ++i) gen[i] = bh->plans[i]->generation;
        const bool same = bh->exec && bh->key_linear == (use_linear ? 1 : 0) && bh->key_gen == gen &&
                          std::equal(bh->key_alm.begin(), bh->key_alm.end(), alm) &&
                          std::equal(bh->key_B.begin(), bh->key_B.end(), B) &&
                          std::equal(bh->key_beta.begin(), bh->key_beta.end(), beta);
        if (!same) {
            batch_drop_graph(bh);
            std::vector<int> prof(n);
            for (size_t i = 0; i < n; ++i) {
                prof[i] = bh->plans[i]->prof;
                bh->plans[i]->prof = 0;                  // no timing events inside a graph
            }
            CK(cudaStreamBeginCapture(bh->main, cudaStreamCaptureModeThreadLocal), "begin capture");
            const modal_status r = batch_run(bh, alm, B, use_linear, beta);
            cudaGraph_t g = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(bh->main, &g);
            for (size_t i = 0; i < n; ++i) bh->plans[i]->prof = prof[i];
            if (r != MODAL_OK) {
                if (g) cudaGraphDestroy(g);
                return r;
            }
            if (ce != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return set_error(MODAL_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
            }
            bh->graph = g;
            const cudaError_t ie = cudaGraphInstantiate(&bh->exec, bh->graph, 0);
            if (ie != cudaSuccess) {
                batch_drop_graph(bh);
                return set_error(MODAL_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
            }
            bh->key_alm.assign(alm, alm + n);
            bh->key_B.assign(B, B + n);
            bh->key_beta.assign(beta, beta + n);
            bh->key_gen = gen;
            bh->key_linear = use_linear ? 1 : 0;
        }
        CK(cudaGraphLaunch(bh->exec, bh->main), "graph launch");
    }
    CK(cudaEventRecord(bh->out, bh->main), "batch out");
    CK(cudaStreamWaitEvent(st, bh->out, 0), "batch out wait");
    return MODAL_OK;
}

modal_status modal_batch_set_schedule(modal_batch_h bh, int schedule) {
    if (!bh) return set_error(MODAL_EINVAL, "null batch");
    if (schedule != MODAL_BATCH_STREAMS && schedule != MODAL_BATCH_SHARED_CUBIC)
        return set_error(MODAL_EINVAL, "unknown batch schedule");
    if (schedule != bh->schedule) batch_drop_graph(bh);
    bh->schedule = schedule;
    return MODAL_OK;
}

void modal_batch_destroy(modal_batch_h bh) {
    if (!bh) return;
    if (bh->main) cudaStreamSynchronize(bh->main);
    batch_drop_graph(bh);
    for (cudaStream_t s : bh->side) cudaStreamDestroy(s);
    for (cudaEvent_t e : bh->done) cudaEventDestroy(e);
    if (bh->fork) cudaEventDestroy(bh->fork);
    if (bh->in) cudaEventDestroy(bh->in);
    if (bh->out) cudaEventDestroy(bh->out);
    if (bh->cubic_done) cudaEventDestroy(bh->cubic_done);
    if (bh->counter) cudaFree(bh->counter);
    if (bh->main) cudaStreamDestroy(bh->main);
    delete bh;
}

}  // extern "C"
