/*
 * modal.h -- C ABI of the GB300 (sm_103a) modal bispectrum library.
 *
 * The library computes the data-parallel hot path of the optimal modal
 * bispectrum estimator of Fergusson & Shellard, "Optimal Polyspectra
 * Estimation" (arXiv:1105.2791):
 *
 *   filtered maps   M_p(x) = sum_lm q_p(l) a_lm / sqrt(C_l) Y_lm(x)
 *                   (whitening of Eq. legoestimator, separable isotropic basis
 *                   of Eq. isobasisbi with v_l = 1, Sec. III.A);
 *   modal coeffs    beta_prs = sum_x W_x [M_p M_r M_s - (<M_p M_r>_x M_s
 *                   + <M_p M_s>_x M_r + <M_r M_s>_x M_p)],  p <= r <= s
 *                   (Eq. bbispect with the linear term of Eq. bispectrumest);
 *   covariance      zeta = <beta beta^T> / 6          (Eq. linearterm, Sec. II);
 *   estimator       fNL = alpha^T zeta^-1 beta / alpha^T zeta^-1 alpha,
 *                   sigma^2 = 6 / alpha^T zeta^-1 alpha
 *                   (Eq. modalest, Eq. modalvariance, via Eq. Cholrot).
 *
 * Conventions
 *  - Sums over the sphere are quadratures on a Gauss-Legendre grid of
 *    `nrings` rings (north first) x `nphi` equally spaced longitudes;
 *    W_x = w_j (2 pi / nphi) mask_x.
 *  - a_lm: complex64 (interleaved float re, im), m >= 0 only, m-major:
 *    idx(l, m) = m (2 lmax + 3 - m) / 2 + (l - m); n_alm = (lmax+1)(lmax+2)/2.
 *    Real field: a_{l,-m} = (-1)^m conj(a_lm); Im a_l0 is ignored.
 *  - Maps: float32 [B][P][nrings][nphi].
 *  - Modes n <-> (p, r, s), p <= r <= s, lexicographic; n_max = C(P+2, 3).
 *    Pairs (p, r), p <= r, lexicographic; n_pair = P (P + 1) / 2.
 *  - beta and the covariance sums are float64.
 *  - Every data pointer is caller-owned.  "dev" pointers are device memory of
 *    the current device, "host" pointers are host memory.  The plan owns its
 *    tables, workspace and Monte Carlo accumulators.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on that stream except modal_init, modal_solve, modal_sync,
 *    the getters and state I/O, which synchronise.
 *  - A plan is not thread-safe; calls on one plan whose work overlaps on the
 *    GPU (different streams) race, with one exception: the FP64 solve family
 *    (modal_solve, modal_fnl_weights) reads only the covariance sums and its
 *    arguments and writes only its own stream-ordered workspace and its own
 *    device error word, so it may run on a second stream beside modal_backward
 *    or modal_backward_retained of the same plan, issued from the same host
 *    thread, once the covariance sums it reads are complete on its stream (an
 *    event).  With profiling on, the stage times of such overlapping calls
 *    include each other's work.
 *  - Errors are returned as status codes and never abort; modal_last_error()
 *    gives a message for the calling thread's last failure.  Kernel faults
 *    surface as MODAL_ECUDA at the next synchronising call; a bounded device
 *    wait that gave up surfaces as MODAL_ETIMEOUT at modal_sync.
 */
#ifndef MODAL_H
#define MODAL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct modal_plan* modal_h;

typedef enum {
    MODAL_OK = 0,
    MODAL_EINVAL = 1,    /* bad argument (size, pointer, unsupported option) */
    MODAL_ENOMEM = 2,    /* device or host allocation failed */
    MODAL_ECUDA = 3,     /* CUDA runtime error (launch or asynchronous fault) */
    MODAL_ENOTPD = 4,    /* zeta is not positive definite (Cholesky pivot <= 0) */
    MODAL_ETIMEOUT = 5,  /* a bounded device-side wait hit its limit */
    MODAL_ESTATE = 6,    /* call out of order (e.g. solve before 2 covariance sims) */
    MODAL_ENOCONV = 7    /* an iteration (the bivector power iteration) did not converge */
} modal_status;

/* Arithmetic of the Legendre contraction (the dominant step).  FP32 is the plain
 * SIMT path; the others run on tcgen05 tensor cores with FP32 accumulation:
 * 3XTF32 and FP16X3 split each operand into two parts and sum three products,
 * BF16X3 does the same with bf16 parts, BF16 uses one bf16 product. */
typedef enum {
    MODAL_FP32 = 0,
    MODAL_3XTF32 = 1,
    MODAL_BF16X3 = 2,
    MODAL_BF16 = 3,
    MODAL_FP16X3 = 4
} modal_prec;

typedef struct {
    int nrings;              /* Gauss-Legendre rings, >= lmax + 1                          */
    int nphi;                /* longitudes: a power of two, >= max(16, 2 lmax + 2), <= 8192 */
    const float* ring_mask;  /* host [nrings] multiplying W_x, or NULL (all ones)           */
    const float* pix_mask;   /* host [nrings*nphi] multiplying W_x, or NULL (all ones)      */
} modal_grid;

typedef struct {
    int lmax, P, nrings, nphi, prec;
    int n_alm, n_max, n_pair;
    long long npix;
    long long n_lin;         /* simulations accumulated into <M_p M_r>_x      */
    long long n_cov;         /* beta vectors accumulated into the covariance  */
    int lin_final;           /* 1 once the linear-term mean has been formed   */
    int chunk;               /* maps per internal pass                        */
    size_t device_bytes;     /* device memory held by the plan                */
    int n_quad;              /* trispectrum modes C(P+3, 4) (modal_quartic)   */
} modal_info;

/* Build a plan: Gauss-Legendre nodes and weights (FP64 Newton on the host), the
 * normalised associated Legendre table lambda_lm(theta_j) (FP64 recurrence with
 * exponent rescaling on the GPU, stored FP32; plus the pre-split tensor-core
 * tables for the tensor-core precisions), the filter q_p(l)/sqrt(C_l) (zero where
 * C_l <= 0) and the pixel weights.  Sec. III.A (basis), Eq. legoestimator (filter).
 *   basis: host [P][lmax+1];  C_l: host [lmax+1];  1 <= P <= 16;  2 <= lmax <= 4000.
 * The tables stay resident (they grow as lmax^3: about 25 GB at lmax = 2000 for the
 * tensor-core precisions); when they and the workspace of one map exceed the device's
 * free memory, returns MODAL_ENOMEM before allocating anything, with the sizes in
 * modal_last_error().  Synchronises.  On failure *out is NULL. */
modal_status modal_init(int lmax, int P, const double* basis, const double* C_l,
                        const modal_grid* grid, int prec, modal_h* out);

/* Filtered maps M_p for B maps: dev alm [B][n_alm] -> dev maps [B][P][nrings][nphi]. */
modal_status modal_synthesize(modal_h h, const void* alm, int B, float* maps, void* stream);

/* Quadrature analysis a_lm = sum_x w_j (2 pi / nphi) T(x) conj(Y_lm(x)) of B maps
 * (no mask, no filter): dev maps [B][nrings][nphi] -> dev alm [B][n_alm] (complex64).
 * The inverse of synthesis with a unit filter for band-limited maps. */
modal_status modal_analyze(modal_h h, const float* maps, int B, void* alm, void* stream);

/* Linear-term simulations (Sec. II: the mean <M_p M_r>_x "calculated from Monte Carlo
 * simulations of Gaussian maps"): synthesise B sims, add M_p M_r of each to the FP64
 * pair sums.  finalize != 0 then forms <M_p M_r>_x = sums / n_lin (used by modal_cubic
 * and modal_backward with use_linear != 0); later simulations change the sums but not
 * this mean until the next finalize.  B may be 0 with finalize set. */
modal_status modal_linear_term(modal_h h, const void* alm_sims, int B, int finalize, void* stream);

/* Modal coefficients (Eq. bbispect): dev alm [B][n_alm] -> dev beta [B][n_max] (float64).
 * use_linear != 0 subtracts the linear term (needs a finalised mean, else MODAL_ESTATE). */
modal_status modal_cubic(modal_h h, const void* alm, int B, int use_linear, double* beta,
                         void* stream);

/* Trispectrum modal coefficients (Sec. IV: the B term of the quartic estimator with the
 * four-harmonic Gaunt integral, separable modes q_p q_r q_s q_u, v_l = 1), on the plan's
 * grid:  tau_prsu = sum_x W_x [M_p M_r M_s M_u - sum over the 6 single pairs <ab> M_c M_d
 *                              + sum over the 3 pair splits <ab> <cd>]
 * for p <= r <= s <= u (lexicographic, n_quad = C(P+3, 4) of them); the -6 C a a and +3 C C
 * terms of Sec. IV symmetrised over the ordered quadruple, with the Monte Carlo pair means
 * <ab> of modal_linear_term (per pixel, or per ring in MODAL_LINEAR_RING mode).
 * use_linear = 0 gives the quartic sum alone; otherwise the means must be finalised
 * (MODAL_ESTATE).  dev alm [B][n_alm] complex64; dev tau [B][n_quad] float64.  The first
 * call allocates the quartic tables and buffers (about chunk x 0.5 MB x cubic CTAs). */
modal_status modal_quartic(modal_h h, const void* alm, int B, int use_linear, double* tau, void* stream);

/* Covariance sums over simulations (Eq. linearterm): S1 += sum_b beta_b,
 * S2 += sum_b beta_b beta_b^T (FP64).  dev beta [B][n_max]. */
modal_status modal_cov_accumulate(modal_h h, const double* beta, int B, void* stream);

/* Estimator (Eq. modalest, Eq. modalvariance, Eq. Cholrot): zeta = sample covariance
 * of the accumulated beta / 6; FP64 Cholesky zeta = L L^T on the GPU;
 * alpha' = L^-1 alpha, beta'_b = L^-1 beta_b; fnl[b] = alpha'.beta'_b / |alpha'|^2,
 * sigma = sqrt(6 / |alpha'|^2).  alpha: host [n_max]; beta: dev [B][n_max] (B >= 0);
 * fnl: host [B] (may be NULL when B == 0); sigma: host [1] or NULL.
 * MODAL_ESTATE if fewer than 2 covariance sims; MODAL_ENOTPD if a pivot is <= 0.
 * Synchronises. */
modal_status modal_solve(modal_h h, const double* alpha, const double* beta, int B,
                         double* fnl, double* sigma, void* stream);

/* Derivative of the estimate with respect to the modal coefficients (Eq. modalest):
 * fNL = alpha^T zeta^-1 beta / alpha^T zeta^-1 alpha is linear in beta, so
 *   d fNL / d beta = w = zeta^-1 alpha / (alpha^T zeta^-1 alpha),
 * formed on the GPU from the accumulated covariance (FP64 Cholesky zeta = L L^T, forward
 * and back substitution).  w passed as g to modal_backward gives d fNL / d a_lm.
 * alpha: host [n_max]; w: dev out [n_max] float64; sigma: host out (may be NULL).
 * MODAL_ESTATE with fewer than 2 covariance sims; MODAL_ENOTPD if zeta is not positive
 * definite.  Synchronises. */
modal_status modal_fnl_weights(modal_h h, const double* alpha, double* w, double* sigma, void* stream);

/* Bivector form of the covariance (Sec. III.B, Eqs. ic_bivector, ic_bivectorinv,
 * bivecvariance).  Given an ideal covariance zeta0 = L0 L0^T (e.g. full sky with
 * homogeneous noise, where it is cheap to know), the Monte Carlo zeta is modelled as
 * L0 (I + bt bt^T) L0^T: bt = sqrt(max(l1, 0)) u1 from the largest eigenpair (l1, u1) of
 * the whitened L0^-1 zeta L0^-T - I, found by FP64 power iteration on the GPU (sign:
 * sum(bt) >= 0).
 *   zeta0: host [n_max][n_max] float64, symmetric positive definite (read only);
 *   bt: host out [n_max] (whitened basis); lambda1: host out l1 (may be NULL).
 * Errors: MODAL_ESTATE with fewer than 2 covariance sims; MODAL_ENOTPD if zeta0 is not
 * positive definite; MODAL_ENOCONV if the residual has not fallen below 1e-12 |1 + l1|
 * within 20000 steps (a near-degenerate top eigenvalue).  Synchronises. */
modal_status modal_bivector_fit(modal_h h, const double* zeta0, double* bt, double* lambda1, void* stream);

/* Eq. modalest with zeta = L0 (I + bt bt^T) L0^T: alpha' = L0^-1 alpha, beta'_b = L0^-1
 * beta_b, the inverse (I + bt bt^T)^-1 = I - bt bt^T / (1 + |bt|^2) (Eq. ic_bivectorinv),
 * fnl_b = alpha'^T (I + bt bt^T)^-1 beta'_b / N, N = alpha'^T (I + bt bt^T)^-1 alpha',
 * sigma = sqrt(6 / N) (Eq. bivecvariance with zeta = <beta beta^T>/6).  Needs no
 * covariance sims.  zeta0: host [n_max][n_max]; bt: host [n_max] (from
 * modal_bivector_fit); alpha: host [n_max]; beta: dev [B][n_max] float64; fnl: host [B];
 * sigma: host (may be NULL).  MODAL_ENOTPD if zeta0 or N is not positive.  Synchronises. */
modal_status modal_solve_bivector(modal_h h, const double* zeta0, const double* bt, const double* alpha,
                                  const double* beta, int B, double* fnl, double* sigma, void* stream);

/* Rotation into the orthonormal frame of the bivector model (Sec. III.B, analytic Cholesky):
 * out_b = Lt^-1 L0^-1 x_b, where zeta0 = L0 L0^T and Lt is the closed-form lower Cholesky
 * factor of I + bt bt^T (diagonal sqrt(S_i/S_{i-1}), below it b_i b_k / sqrt(S_{k-1} S_k),
 * S_i = 1 + sum_{j<=i} b_j^2), applied in O(n_max) per vector.  In that frame the
 * estimator is alpha''.beta'' / |alpha''|^2.  zeta0: host [n_max][n_max]; bt: host [n_max];
 * x, out: dev [B][n_max] float64 (out may equal x).  MODAL_ENOTPD if zeta0 is not
 * positive definite.  Synchronises. */
modal_status modal_bivector_rotate(modal_h h, const double* zeta0, const double* bt, const double* x, int B,
                                   double* out, void* stream);

/* Adjoint (not in the paper): for L = sum_n g_n beta_n, grad_lm = dL/dRe a_lm
 * + i dL/dIm a_lm for the stored m >= 0 entries (Im part of m = 0 is zero).
 * Maps are recomputed, not stored.  dev alm [B][n_alm]; dev g [B][n_max] (float64);
 * dev grad_alm [B][n_alm] complex64. */
modal_status modal_backward(modal_h h, const void* alm, int B, const double* g, int use_linear,
                            void* grad_alm, void* stream);

/* Keep the filtered maps of each modal_linear_term or modal_cubic call whose batch fits one
 * chunk (B <= chunk; no extra memory: they stay in the plan's map workspace), so that
 * modal_cubic_retained and modal_backward_retained can use them without synthesising them
 * again.  on: 0 (default) or 1. */
modal_status modal_set_retain_maps(modal_h h, int on);

/* modal_cubic (Eq. bbispect with the linear term of Eq. bispectrumest) at the a_lm of the
 * plan's last modal_linear_term or modal_cubic call, from the maps that call kept (and, for
 * the per-ring linear term, the Legendre sums still beside them): the same result as
 * modal_cubic(h, alm, B, use_linear, beta) without the synthesis, so that a batch that is
 * both a linear-term sample and a coefficient input is synthesised once.  alm and B must
 * be the pointer and count given to that call (checked; the caller must not have changed
 * the a_lm since), and this call must be ordered after it on the device.  The maps stay
 * kept.  B = 0 does nothing; MODAL_ESTATE if no maps are kept for (alm, B). */
modal_status modal_cubic_retained(modal_h h, const void* alm, int B, int use_linear, double* beta, void* stream);

/* modal_backward at the a_lm of the plan's last modal_linear_term or modal_cubic call, from
 * the maps that call kept: the same result as modal_backward(h, alm, B, g, use_linear, grad_alm) without the
 * synthesis.  alm and B must be the pointer and count given to that call (checked; the
 * caller must not have changed the a_lm since), and the call must be ordered after it on
 * the device (same stream, or an event).  B = 0 does nothing.  MODAL_ESTATE if no maps are
 * kept for (alm, B): retention off, B > chunk, or a later call reused the map workspace
 * (the synthesis of modal_linear_term, modal_cubic, modal_quartic or modal_backward;
 * modal_set_chunk).  The adjoint overwrites the kept maps: a second call returns
 * MODAL_ESTATE. */
modal_status modal_backward_retained(modal_h h, const void* alm, int B, const double* g, int use_linear,
                                     void* grad_alm, void* stream);

/* alpha_prs per unit fNL for the local shape b = 2 (C1 C2 + C2 C3 + C3 C1) (Eq. abispect
 * with the first-order bispectrum of T = G + f (G^2 - <G^2>)), by exact Gauss-Legendre
 * integration of Legendre series (FP64, host).  C_signal: host [lmax+1] (the signal
 * part of C_l; NULL = the C_l given to modal_init); alpha: host [n_max]. */
modal_status modal_alpha_local(modal_h h, const double* C_signal, double* alpha);

modal_status modal_get_info(modal_h h, modal_info* info);
/* Ring nodes mu_j = cos(theta_j) and weights w_j: host [nrings] each (either may be NULL). */
modal_status modal_get_rings(modal_h h, double* mu, double* w);
/* Copy <M_p M_r>_x (after finalize) to dev out [n_pair][nrings*nphi] float32; in ring mode
 * (modal_set_linear_mode) the ring means, dev out [n_pair][nrings] float32. */
modal_status modal_get_pair_mean(modal_h h, float* out, void* stream);

/* Linear-term mode (a refinement the paper's axisymmetric noise and mask allow, not part of
 * its method as printed).  MODAL_LINEAR_PIXEL (default): the Monte Carlo pair means are kept
 * per pixel, [n_pair][npix].  MODAL_LINEAR_RING: per ring, [n_pair][nrings], the mean over
 * the simulations and over the longitudes of each ring,
 *   <M_a M_b>_j = (1 / (N_lin nphi)) sum_sims sum_k M_a M_b (theta_j, phi_k),
 * which equals the pixel mean in expectation when the weights, noise and mask depend on the
 * ring alone; the linear term of modal_cubic and the adjoint then use it for every pixel of
 * the ring.  Refused (MODAL_EINVAL) for a plan built with a pixel mask.  Setting a mode
 * clears the linear-term sums (n_lin = 0, not finalised).  Checkpoints record the mode's
 * sums and load only into a plan in the same mode. */
#define MODAL_LINEAR_PIXEL 0
#define MODAL_LINEAR_RING 1
modal_status modal_set_linear_mode(modal_h h, int mode);
/* zeta = covariance / 6 of the accumulated beta: host [n_max][n_max]. Synchronises. */
modal_status modal_get_zeta(modal_h h, double* zeta);
/* Clear accumulators: what & 1 -> linear-term sums, what & 2 -> covariance sums. */
modal_status modal_reset(modal_h h, int what);
/* Maps per internal pass (workspace is sized by it); reallocates.  Synchronises.
 * chunk in [1, 4096], else MODAL_EINVAL.  If the new workspace cannot be allocated the
 * call returns MODAL_ENOMEM with the previous chunk restored; if even that fails, the
 * plan has no workspace and the calls that run maps through it return MODAL_ESTATE
 * until a modal_set_chunk succeeds. */
modal_status modal_set_chunk(modal_h h, int chunk);

/* Launch shapes of a plan's kernels (not part of the method; every setting gives the same
 * results up to the order of FP32/FP64 partial sums).
 *   chunk          maps per internal pass (as modal_set_chunk), [1, 4096]
 *   legendre_maps  maps per work item of the tensor-core Legendre contraction: the MMA
 *                  tile is 128 ring pairs x N = 2 P legendre_maps columns, N a multiple of
 *                  16 and at most 256, legendre_maps <= 32 (default 8; kept but unused by
 *                  the FP32 plan)
 *   cubic_ctas     CTAs per map of the cubic and quartic sums (split-K over pixels),
 *                  [1, max(1, npix / 128)]
 *   ms             output of modal_autotune: the winning coefficient-pass time (ignored
 *                  by modal_set_tuning) */
typedef struct modal_tuning {
    int chunk, legendre_maps, cubic_ctas;
    float ms;
} modal_tuning;
modal_status modal_get_tuning(modal_h h, modal_tuning* t);
/* Validates every field (MODAL_EINVAL, nothing changed) and reallocates the workspace
 * (synchronises).  If that allocation fails: MODAL_ENOMEM with the previous tuning
 * restored, or, if even that fails, no workspace (as modal_set_chunk). */
modal_status modal_set_tuning(modal_h h, const modal_tuning* t);
/* Autotuner: times modal_cubic(h, alm, B, use_linear, ...) (the coefficient pass: synthesis,
 * cubic sums and the linear term) on the caller's maps for candidate settings of each
 * field in turn (legendre_maps, cubic_ctas, chunk), CUDA events on
 * `stream`, one warm-up and the better of two timed calls per candidate, and keeps a
 * candidate only if it is at least 1 % faster than the best so far.  Leaves the plan on
 * the winning tuning and writes it to *best (best->ms = its time).  alm: dev [B][n_alm],
 * B >= 1; a candidate whose workspace does not fit is skipped.  Synchronises; takes about
 * 50 coefficient passes. */
modal_status modal_autotune(modal_h h, const void* alm, int B, int use_linear, modal_tuning* best, void* stream);
/* Synchronise `stream`, then report asynchronous faults (MODAL_ECUDA) or a device
 * wait that gave up (MODAL_ETIMEOUT, with the flag cleared). */
modal_status modal_sync(modal_h h, void* stream);

/* Checkpoint / resume of the Monte Carlo accumulators (pair sums, n_lin, S1, S2,
 * n_cov) in a binary file tagged with the plan's sizes.  Synchronise. */
modal_status modal_save_state(modal_h h, const char* path);
modal_status modal_load_state(modal_h h, const char* path);

/* Device wait self-test: one thread waits on a device flag that nothing sets, giving
 * up after `spin_limit` polls; the next modal_sync returns MODAL_ETIMEOUT.  Exercises
 * the bounded-wait error path without faulting the GPU. */
modal_status modal_selftest_wait(modal_h h, int spin_limit, void* stream);

/* Allocation-free cubic coefficients, for callers that cannot call cudaMalloc (device
 * memory owned by another allocator, or loops where an allocation's implicit device
 * synchronisation is not acceptable).  The paper has no counterpart: it is the cubic
 * reduction of modal_cubic without the linear term, on maps the caller already holds:
 *   beta[b][n] = sum_x W[x] M_p M_r M_s,  n <-> (p <= r <= s) lexicographic.
 * maps: dev float [B][P][npix]; W: dev float [npix]; beta: dev double [B][n_max].
 * Needs no plan and allocates nothing: per-block partial sums go to one static device
 * array of 4 Mi doubles (32 MiB, held by every GPU that loads the library until exit),
 * so B * n_max must not exceed 4 Mi (and B <= 65535), else MODAL_EINVAL.  Every call
 * shares that array and overwrites what it reads, so nothing needs clearing, but calls
 * that overlap on the GPU race on it.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any stream capture. */
modal_status modal_cubic_static(const float* maps, const float* W, long long npix, int P, int B,
                                double* beta, void* stream);

/* Throughput probes for roofline denominators (not part of the estimator): kind 0 = FP32
 * SIMT (packed f32x2 FMA), 1 = FP64 SIMT, 2 = tcgen05 tf32, 3 = tcgen05 f16 (M = 128,
 * N = 256, FP32 accumulate, operands in shared memory), 4 = tcgen05 tf32 at N = 16 (the
 * shape of the adjoint's pixel-weight product).  Runs a fixed amount of independent
 * work on every SM of the current device (a few ms) and writes the rate in TFLOP/s
 * (a multiply-add counts 2).  MODAL_EINVAL for another kind; MODAL_ETIMEOUT if the
 * tensor-core wait gave up.  Synchronises `stream`. */
modal_status modal_peak_probe(int kind, double* tflops, void* stream);

/* Per-stage timing.  With profiling enabled every kernel launch of the plan is
 * bracketed by CUDA events recorded on the launching stream.  modal_get_profile
 * synchronises, writes for each stage s < nstages the summed event time in ms
 * (stage_ms, may be NULL) and the number of kernel launches (launches, may be NULL;
 * counted whether or not profiling is on) since the previous call, then resets both.
 * Stages are numbered 0 .. MODAL_NSTAGES-1; modal_stage_name gives their names. */
#define MODAL_NSTAGES 15
modal_status modal_set_profiling(modal_h h, int enable);
modal_status modal_get_profile(modal_h h, double* stage_ms, long long* launches, int nstages);
const char* modal_stage_name(int stage);

/* Mixed-l_max batches.  A batch groups plans (typically one per l_max, each with its own
 * tables and workspace) so that one call runs the coefficient pass (modal_cubic) of all of
 * them.  Each plan runs on a stream of the batch's own; the caller's stream waits for all
 * of them before its next work.
 *   modal_batch_create: plans = host array of nplans >= 1 distinct handles on one device;
 *     the batch keeps the handles (destroy the batch before any of its plans).  Errors:
 *     MODAL_EINVAL (null, repeated or mixed-device plans), MODAL_ECUDA.
 *   modal_batch_cubic: for plan i, alm[i] = dev complex64 [B[i]][n_alm_i] and
 *     beta[i] = dev double [B[i]][n_max_i] exactly as modal_cubic; alm, B and beta are
 *     host arrays of nplans entries.  With use_graph != 0 the launches are captured into
 *     one CUDA graph on the first call and the graph is replayed by later calls with the
 *     same pointers, counts and use_linear (new contents of the same buffers are read)
 *     while no member plan has changed state since the capture; a different argument, or
 *     a plan changed by modal_set_chunk, modal_set_linear_mode, modal_set_retain_maps,
 *     modal_reset, modal_load_state or the first allocation of its linear-term buffers,
 *     re-captures it.  Kernels replayed from a graph are not counted by
 *     modal_get_profile, and plan profiling is suspended while a graph is captured.
 *     Errors: as modal_cubic for each plan (MODAL_ESTATE for a plan without workspace);
 *     MODAL_ECUDA if capture or replay fails. */
typedef struct modal_batch* modal_batch_h;
modal_status modal_batch_create(const modal_h* plans, int nplans, modal_batch_h* out);
modal_status modal_batch_cubic(modal_batch_h bh, const void* const* alm, const int* B, int use_linear,
                               double* const* beta, int use_graph, void* stream);

/* How modal_batch_cubic schedules its plans (Sec. 4's cubic sums, Eq. 41, for every plan):
 *   MODAL_BATCH_STREAMS (default): each plan's whole pass (synthesis, cubic sums, linear
 *     term, beta) runs chunk by chunk on its own stream, the streams concurrently.
 *   MODAL_BATCH_SHARED_CUBIC: the plans' chunks go in lockstep passes; in pass k every plan
 *     synthesizes its k-th chunk on its stream, then ONE persistent launch computes the
 *     cubic sums of all of them from a work queue of (plan, map, pixel range) items, plans
 *     with the longest pixel ranges first, before each plan's linear term and beta.  It
 *     applies to calls whose plans with maps share one P (at most 8 of them, at least 2);
 *     other calls run as MODAL_BATCH_STREAMS.  Every item is the one the plan's own launch
 *     computes, so beta is bit-identical under either schedule.
 * A change of schedule re-captures the batch graph.  Errors: MODAL_EINVAL (null batch,
 * unknown schedule). */
#define MODAL_BATCH_STREAMS 0
#define MODAL_BATCH_SHARED_CUBIC 1
modal_status modal_batch_set_schedule(modal_batch_h bh, int schedule);
void modal_batch_destroy(modal_batch_h bh);

void modal_destroy(modal_h h);
const char* modal_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MODAL_H */
