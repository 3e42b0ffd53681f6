/*
 * fpt.h -- C ABI of the GB300 first-passage-time library (libfpt.so).
 *
 * Stochastic-delta-N sampler of arXiv:2410.13683 ("Stochastic inflation
 * beyond slow roll: noise modelling and importance sampling"): many
 * independent (phi, pi) Langevin trajectories in e-fold time N, stepped by
 * Euler-Maruyama (Eq. 4.1) with field-dependent 1-D noise (Eq. 4.6) read from
 * phi-indexed tables (Sec. 5), an optional importance-sampling drift bias and
 * its log-likelihood-ratio weight (Eqs. 4.4-4.10), until first passage through
 * the end surface; then the weighted histogram of first-passage times that
 * estimates P(delta N) (Sec. 2.3, Sec. 4.1).
 *
 * Conventions for every call:
 *   - Status codes are returned; nothing throws across the ABI. Codes >= 100
 *     are warnings: results are valid. fpt_last_error() gives a message.
 *   - The context owns all device memory it allocates and its private CUDA
 *     stream; the caller owns every buffer it passes in.
 *   - Pointers documented as "host or device" may be either (unified virtual
 *     addressing decides); host buffers may be pageable or pinned.
 *   - `cuda_stream` arguments are cudaStream_t handles; NULL selects the
 *     context's private stream (cudaStreamLegacy selects the legacy default
 *     stream).
 *   - Calls on one context are not thread-safe: use one context per thread.
 *   - Results depend only on (seed, trajectory id, run id) and the inputs,
 *     never on launch shape, refill granularity or the number of calls that a
 *     trajectory range is split into.
 */
#ifndef FPT_H
#define FPT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fpt_ctx fpt_ctx;

typedef enum {
    FPT_OK = 0,
    FPT_E_INVALID = 1,   /* bad argument; nothing was launched              */
    FPT_E_CUDA = 2,      /* a CUDA runtime call failed                      */
    FPT_E_NOMEM = 3,     /* device or pinned-host allocation failed         */
    FPT_E_TIMEOUT = 4,   /* the kernel deadline passed; in-flight
                            trajectories carry status FPT_TRAJ_ABORTED      */
    FPT_E_STATE = 5,     /* call order violated (e.g. no table for a model) */
    FPT_W_CAPPED = 100   /* some trajectories hit max_steps (censored)      */
} fpt_status;

/* Potential families. */
enum {
    /* V = V0 [1 + a_plus (phi - phi_star)] for phi >= phi_star and
     * V = V0 [1 + a_minus (phi - phi_star)] below: Eq. (4.11) with the slopes
     * divided by V0. a_plus == a_minus is the linear potential V0 (1 + A phi)
     * (phi_star = 0). */
    FPT_POT_PWLINEAR = 0,
    /* V = V0 exp(mu phi): V'/V = mu, exact attractor pi = -mu (test model). */
    FPT_POT_EXP = 1,
    /* Gaussian bump, Eq. (4.12):
     * V = V0 phi^2/(bump_m^2 + phi^2) [1 + bump_K exp(-(phi - bump_phi0)^2 / (2 bump_width^2))].
     * With the transition rule, N_T is the onset of ultra-slow roll (the
     * first time eps2 = 2 pi'/pi reaches -3 on the background). */
    FPT_POT_BUMP = 2
};

/* Noise-table kinds (fpt_noise_table). */
enum {
    FPT_TABLE_DESITTER = 0,  /* S = H/2pi on phi only, Eq. (3.3), H on the
                                attractor pi = -V'/V                        */
    FPT_TABLE_BESSEL = 1,    /* semi-analytical Bessel-matched growing mode,
                                Eqs. (3.10)-(3.13); needs the transition rule */
    FPT_TABLE_USER = 2,      /* caller-supplied S(phi_j), S_pi(phi_j)        */
    /* N-indexed tables: the paper's production setting (Sec. 4.1), noise
     * precomputed along the classical background as a function of the time
     * N = n dN since the start and switched off outside the window: steps n
     * with ceil(N_lo/dN - 1e-9) <= n <= floor(N_hi/dN + 1e-9) draw noise from
     * the table (linear interpolation in N), all other steps are classical.
     * For these kinds phi_lo / phi_hi carry N_lo / N_hi (required). */
    FPT_TABLE_BESSEL_N = 3,  /* Bessel-matched noise of the mode crossing sigma a H
                                at background time N_in + N                   */
    FPT_TABLE_USER_N = 4,    /* caller-supplied S(N_j), S_pi(N_j)            */
    /* Full-rank (2-D) tables (fpt_noise_table2), phi-indexed: */
    FPT_TABLE_NUMERIC = 5,   /* numerical matching, Eq. (3.9): Xi of the full
                                mode at k = sigma a H, S = sqrt(Xi) (symmetric) */
    FPT_TABLE_USER2 = 6      /* caller-supplied symmetric S(phi_j)           */
};

/* Bias kinds (fpt_run_desc.bias_kind). */
enum {
    FPT_BIAS_NONE = 0,   /* direct sampling                                 */
    FPT_BIAS_CONST = 1,  /* diffusion-based bias of Eq. (4.10): amplitude A  */
    FPT_BIAS_MLP = 2     /* learned amplitude alpha = MLP(x, pi, N)          */
};

/* Per-trajectory status (fpt_traj_out.status). */
enum { FPT_TRAJ_PASSED = 0, FPT_TRAJ_CAPPED = 1, FPT_TRAJ_ABORTED = 2 };

/*
 * One model: potential, start point and end surface (Sec. 4.1: the system
 * starts at (phi_init, pi_init) and runs until the end surface is crossed).
 *
 * Start/end are either explicit (phi_in, pi_in, phi_end; pi_in = NaN means
 * the attractor value -V'/V(phi_in)), or -- when n_in is not NaN -- resolved
 * from the classical background (Eq. 2.21 without noise) that starts at
 * bg_phi0 on the slow-roll attractor: phi_in, pi_in are the background values
 * n_in e-folds after the transition time N_T (phi = phi_star; for the bump
 * the onset of ultra-slow roll) and phi_end the background field n_end
 * e-folds after N_T (the paper starts after the transition and sets the
 * start/end by the mode range, Secs. 4.1-4.3).
 * Passage is the first step n >= 1 with phi_n <= phi_end; N = n dN.
 */
typedef struct {
    int32_t kind;          /* FPT_POT_*                                      */
    int32_t pad;
    double V0;             /* potential scale (> 0)                          */
    double a_plus;         /* relative slope above phi_star                  */
    double a_minus;        /* relative slope below phi_star                  */
    double phi_star;       /* transition field value                         */
    double mu;             /* FPT_POT_EXP slope                              */
    double phi_in;         /* explicit start (ignored when n_in is set)      */
    double pi_in;          /* explicit momentum, NaN = attractor             */
    double phi_end;        /* explicit end surface                           */
    double bg_phi0;        /* transition rule: background start on attractor */
    double n_in;           /* transition rule: start, e-folds after N_T; NaN = explicit */
    double n_end;          /* transition rule: end, e-folds after N_T        */
    double dN;             /* e-fold step (> 0)                              */
    int64_t max_steps;     /* step cap per trajectory (>= 1, < 2^31)         */
    double bump_K;         /* FPT_POT_BUMP: bump height                      */
    double bump_m;         /* FPT_POT_BUMP: mass scale of the plateau        */
    double bump_width;     /* FPT_POT_BUMP: Gaussian width (> 0)             */
    double bump_phi0;      /* FPT_POT_BUMP: bump position                    */
} fpt_model;

/* Resolved start/end of a model (FP64, from the background solve). */
typedef struct {
    double phi_in, pi_in, phi_end;
    double N_T;            /* transition time of the background, NaN if none */
} fpt_model_info;

/*
 * Create a context on CUDA device `device` holding n_models models (1..64).
 * Resolves every model's start/end (host FP64 background solve). On error
 * *ctx is NULL and the status says why.
 */
fpt_status fpt_init_model(fpt_ctx **ctx, const fpt_model *models, int32_t n_models,
                          int32_t device);

/* Resolved start/end of model `model`. */
fpt_status fpt_model_get_info(const fpt_ctx *ctx, int32_t model, fpt_model_info *out);

/*
 * Build (or accept) model `model`'s noise table and upload it to the device.
 *
 * Grid: phi_j = phi_lo + j h, h = (phi_hi - phi_lo)/(n_points - 1),
 * j = 0 .. n_points-1 (2 <= n_points <= 8192). phi_lo/phi_hi = NaN select the
 * model's [phi_end, phi_in]. The stepper interpolates linearly in phi and
 * holds the end values outside [phi_lo, phi_hi].
 *
 * kind FPT_TABLE_BESSEL: for each phi_j the background time N_j with
 *   phi_bg(N_j) = phi_j, k_j = sigma a(N_j) H(N_j); the mode of Eq. (2.4)
 *   from its Bunch-Davies state (Eq. 2.5) at N_j - ln(100/sigma) through the
 *   kink to N_j; Bessel matching at -k eta = sigma with nu from Eq. (3.13);
 *   S = sqrt(Xi_phiphi) of Eq. (3.12) and S_pi = (nu - 3/2) S.
 *   Requires the transition rule (n_in set) and 0 < sigma <= 10.
 * kind FPT_TABLE_DESITTER: S = H/2pi with H^2 = V/(3 - pi_att^2/2), S_pi = 0.
 * kind FPT_TABLE_USER: user_S / user_Spi (host, n_points doubles each, S >= 0).
 *
 * kind FPT_TABLE_BESSEL_N / FPT_TABLE_USER_N: as BESSEL / USER on the grid
 *   N_j = N_lo + j h of times since the start (see the enum); learned-proposal
 *   runs need a phi-indexed table.
 *
 * out_S, out_Spi: optional host buffers of n_points doubles receiving the FP64
 * table. Blocks the calling thread until the upload finished.
 */
fpt_status fpt_noise_table(fpt_ctx *ctx, int32_t model, int32_t kind, int32_t n_points,
                           double sigma, double phi_lo, double phi_hi,
                           const double *user_S, const double *user_Spi,
                           double *out_S, double *out_Spi);

/*
 * Full-rank (2-D) noise table of model `model` (Sec. 3.3): the noise of the
 * Langevin system Eq. (2.24) is S xi sqrt(dN) with two independent normals
 * xi = (xi_1, xi_2) per step and the symmetric 2x2 matrix
 * S = [[S_phiphi, S_phipi], [S_phipi, S_pipi]], covariance Xi = S^2.
 * Grid and interpolation as fpt_noise_table (phi-indexed, end values held).
 *
 * kind FPT_TABLE_NUMERIC: for each phi_j the mode of k_j = sigma a H at N_j
 *   (phi_bg(N_j) = phi_j), from its Bunch-Davies state at N_j - ln(100/sigma)
 *   through the kink; Xi = k^3/(2 pi^2) (|dphi|^2, Re(dphi dpi*), |dpi|^2),
 *   dpi = d(dphi)/dN; S = sqrt(Xi). Requires the transition rule and
 *   0 < sigma <= 10. The paper uses sigma << 1 for this matching.
 * kind FPT_TABLE_USER2: user_S (host) holds 3 n_points doubles, the planes
 *   S_phiphi[n_points], S_phipi[n_points], S_pipi[n_points] (finite).
 * out_S: optional host buffer of 3 n_points doubles (same planes).
 * A model holds one table: this call replaces a 1-D table and vice versa.
 * Runs on a 2-D table use the 2-D stepper (see fpt_run_desc). Blocks until
 * the upload finished.
 */
fpt_status fpt_noise_table2(fpt_ctx *ctx, int32_t model, int32_t kind, int32_t n_points,
                            double sigma, double phi_lo, double phi_hi, const double *user_S,
                            double *out_S);

/*
 * Host-only helpers (no context, no GPU): the same FP64 model resolution and
 * table construction that fpt_init_model / fpt_noise_table(2) use.
 * fpt_table_build2 builds FPT_TABLE_NUMERIC only (out_S: 3 n_points doubles).
 */
fpt_status fpt_resolve_model(const fpt_model *model, fpt_model_info *out);
fpt_status fpt_table_build(const fpt_model *model, int32_t kind, int32_t n_points,
                           double sigma, double phi_lo, double phi_hi,
                           double *out_S, double *out_Spi);
fpt_status fpt_table_build2(const fpt_model *model, int32_t kind, int32_t n_points,
                            double sigma, double phi_lo, double phi_hi, double *out_S);

/*
 * ---- Classical delta N (Sec. 2.2), host only, FP64 ----
 * The comparison the paper draws between the stochastic P(delta N) and the
 * classical delta-N formalism: the linear power spectrum of Eq. (2.8),
 * P_R = k^3/(2 pi^2) |delta phi_k|^2 / (2 eps1), from the mode of Eq. (2.4)
 * (Bunch-Davies start, Eq. 2.5, at k/(aH) = 100/sigma, kink jump as for the
 * tables); its variance over the simulated mode range, Eq. (2.18); and the
 * constant-eps2 PDF of Eq. (2.20). Models need the transition rule.
 */

/* P_R of the modes k = sigma a H at background times N_s[j] (n entries, host),
 * read at N_eval (NaN: N_end + 4, outside the Hubble radius). */
fpt_status fpt_power_spectrum(const fpt_model *model, double sigma, int32_t n, const double *N_s,
                              double N_eval, double *out_PR);

typedef struct {
    double sigma_R2;       /* int P_R d ln k over the modes reaching sigma a H in
                              [N_in, N_end] (composite Simpson, n_k points)   */
    double eps2_in;        /* eps2 = 2 pi'/pi of the background at N_in       */
    double eps2_end;       /* ... and at N_end                               */
    double N_in, N_end;    /* background times of phi_in and phi_end          */
} fpt_classical;

/* n_k odd in [3, 4097]; N_eval as fpt_power_spectrum. */
fpt_status fpt_classical_dn(const fpt_model *model, double sigma, int32_t n_k, double N_eval,
                            fpt_classical *out);

/* Eq. (2.20) at dN[i] (host, n entries): P(dN) = exp[-(2/(sigma_R2 eps2^2))
 * (1 - e^{-eps2 dN/2})^2 - eps2 dN/2] / sqrt(2 pi sigma_R2); eps2 = 0 gives
 * the Gaussian of variance sigma_R2. */
fpt_status fpt_classical_pdf(const double *dN, int64_t n, double sigma_R2, double eps2, double *out);

/* Least-squares eps2 of Eq. (2.20) to a measured P(dN): minimises
 * sum_b ((ln pdf_b - ln P(dN_b))/(se_b/pdf_b))^2 over bins with pdf, se > 0
 * by golden-section search on [eps2_lo, eps2_hi] (the paper's fitted curves,
 * Sec. 4.3). chi2_out, bins_used nullable. All arrays host, n_bins entries. */
fpt_status fpt_fit_eps2(const double *dN, const double *pdf, const double *se, int32_t n_bins,
                        double sigma_R2, double eps2_lo, double eps2_hi, double *eps2_out,
                        double *chi2_out, int32_t *bins_used);

/*
 * One run: a set of trajectories of one model with one bias.
 *
 * The noise of step i of trajectory t is drawn from Philox4x32-10 with key
 * (seed_lo, seed_hi) and counter (i >> 2, traj_offset + t, run_id, 0): words
 * r_k -> u_k = ((r_k >> 9) + 0.5) 2^-23 -> Box-Muller pairs (u0,u1), (u2,u3);
 * step i uses normal number i & 3 of its block. All runs of one fpt_run call
 * must share `seed`; they are told apart by run_id.
 *
 * Bias (Eqs. 4.7-4.10): B = alpha S (1, tan theta_n), weight increment
 * dA = alpha (alpha dN/2 + xi sqrt(dN)), w = exp(-sum dA). alpha = A for
 * FPT_BIAS_CONST (A > 0 pushes phi up, towards longer first-passage times).
 * FPT_BIAS_MLP: alpha = clamp((o1 + t o2)/sqrt(1 + t^2), +-alpha_max) with
 * (o1, o2) = MLP((x - shift) * scale), x = (phi - phi_end, pi, n dN),
 * t = tan(theta_n) at the segment start, held fixed for `mlp_segment` steps
 * (steps n = 0, mlp_segment, 2 mlp_segment, ... start a segment). All MLP runs
 * of one call share mlp_segment, and a call with MLP runs refills finished
 * trajectories every mlp_segment steps. Each MLP run may carry its own network
 * (blob), shift, scale, alpha_max and flags: when they differ the stepper
 * evaluates each run's network from global memory (one evaluation per run
 * present in a warp), otherwise the shared network is staged in shared
 * memory. Runs with different networks need 1-D phi-indexed tables and the
 * piecewise-linear or exponential potential (FPT_E_INVALID otherwise).
 */
typedef struct {
    int32_t model;          /* model index                                   */
    int32_t bias_kind;      /* FPT_BIAS_*                                    */
    double A;               /* FPT_BIAS_CONST amplitude                      */
    int64_t n_traj;         /* trajectories (>= 0)                           */
    int64_t traj_offset;    /* first trajectory id (ids < 2^32)              */
    uint64_t seed;          /* Philox key                                    */
    uint32_t run_id;        /* Philox counter word 2                         */
    int32_t mlp_segment;    /* FPT_BIAS_MLP: steps per alpha (multiple of 4) */
    const void *mlp;        /* FPT_BIAS_MLP: device pointer, packed bf16     */
    float mlp_shift[3];     /* FPT_BIAS_MLP: input shift                     */
    float mlp_scale[3];     /* FPT_BIAS_MLP: input scale                     */
    float alpha_max;        /* FPT_BIAS_MLP: |alpha| clamp (> 0)             */
    int32_t mlp_flags;      /* FPT_BIAS_MLP: FPT_MLP_LOG_X = first input is
                               ln(max(phi - phi_end, mlp_x_floor)) instead of
                               phi - phi_end                                 */
    double A2;              /* FPT_BIAS_CONST on 2-D tables: beta_2          */
    float mlp_x_floor;      /* FPT_MLP_LOG_X: floor of phi - phi_end under the
                               log (<= 0: 1e-30). The log amplifies the field's
                               rounding error by 1/x near the end surface; a
                               floor a few orders below x_in keeps the input
                               well conditioned there                        */
    int32_t pad_;           /* reserved, 0                                   */
} fpt_run_desc;

enum { FPT_MLP_LOG_X = 1 };

/* Per-trajectory results of one run; each pointer host or device, nullable.
 * Arrays hold n_traj entries in trajectory order. */
typedef struct {
    double *N;          /* first-passage time n dN                            */
    double *logw;       /* ln w (0 for direct sampling)                       */
    int32_t *nsteps;    /* steps taken                                        */
    uint8_t *status;    /* FPT_TRAJ_*                                         */
} fpt_traj_out;

/* Launch shape. Zero fields take the context defaults (or the autotuned
 * choice). */
typedef struct {
    int32_t block;          /* threads per block: 128, 192, 256, 384 or 512
                               (default 512; learned-proposal launches use at
                               most 384)                                      */
    int32_t blocks_per_sm;  /* resident blocks per SM (persistent grid)        */
    int32_t check_steps;    /* steps between refill points (multiple of 4)     */
    int32_t use_graph;      /* 1: replay a captured CUDA graph per shape; a
                               replay runs with the call's seed and the
                               model's current tables, like a plain launch   */
    double deadline_s;      /* > 0: abort the kernel after this many seconds  */
} fpt_launch;

fpt_status fpt_set_launch(fpt_ctx *ctx, const fpt_launch *launch);
fpt_status fpt_get_launch(const fpt_ctx *ctx, fpt_launch *launch);

/*
 * Autotuner: runs `runs` (each n_traj scaled by `fraction`, 0 < fraction <= 1,
 * at least 32 trajectories) under every candidate shape -- block in
 * {128, 256, 384, 512} x check_steps in {8, 32, 128}, resident blocks at maximum
 * occupancy -- times each with CUDA events after one warm-up, and keeps the
 * fastest in the context (graph replay and deadline settings are kept).
 * Results of later runs do not depend on the choice. `chosen` (nullable)
 * receives it. Synchronous; overwrites the context's last-run results.
 */
fpt_status fpt_autotune(fpt_ctx *ctx, const fpt_run_desc *runs, int32_t n_runs, double fraction,
                        fpt_launch *chosen);

/*
 * Run n_runs runs (1..128) in one persistent launch: one trajectory per
 * thread, warp-level refill of finished trajectories every check_steps steps.
 * Results stay in the context for fpt_histogram; out (n_runs entries,
 * nullable) receives copies. Asynchronous on cuda_stream (NULL = the
 * context's stream) unless an `out` buffer is pageable host memory; returns
 * FPT_W_CAPPED / FPT_E_TIMEOUT only after synchronising (see fpt_sync).
 */
fpt_status fpt_run(fpt_ctx *ctx, const fpt_run_desc *runs, int32_t n_runs,
                   fpt_traj_out *out, void *cuda_stream);

/* Wait for the context's work and return the deferred run status
 * (FPT_OK, FPT_W_CAPPED or FPT_E_TIMEOUT). */
fpt_status fpt_sync(fpt_ctx *ctx);

/*
 * Weighted histogram of run `run` of the last fpt_run (Sec. 4.1).
 * Bins b = floor((N - N_lo)/db), db = (N_hi - N_lo)/n_bins, N = n dN, over
 * passed trajectories; n = all trajectories of the run (capped included).
 *   pdf    = sum_b w / (n db)                       (importance sampling)
 *   se_w   = its standard error (sample variance of w 1_b / db)
 *   pdf_ln, se_ln: lognormal-mean estimator (n_b/n) exp(m + s^2/2)/db with
 *            Cox's error on the log combined with the binomial error
 *   se_jk  = delete-one-block jackknife error, 32 blocks of trajectory index
 * log_sum_w / log_sum_w2 are ln(sum w) and ln(sum w^2) per bin (-inf empty).
 * The tail set T = {passed, N >= N_tail} gives ess_tail = (sum_T w)^2 /
 * sum_T w^2 and p_tail = sum_T w / n (N_tail = NaN: none).
 * Array outputs are host buffers of n_bins entries, each nullable.
 * 1 <= n_bins <= 4096, N_lo < N_hi. Blocks until the results are on the host.
 */
typedef struct {
    int64_t *count;
    double *log_sum_w, *log_sum_w2, *sum_lw, *sum_lw2;
    double *pdf, *se_w, *pdf_ln, *se_ln, *se_jk;
    int64_t n_total, n_passed, n_under, n_over, n_capped, n_tail;
    double N_mean;         /* mean N of passed trajectories                   */
    double N_mean_w;       /* self-normalised sum w N / sum w                 */
    double ess_tail, p_tail;
    double log_max_w;      /* max ln w over passed trajectories               */
} fpt_hist;

fpt_status fpt_histogram(fpt_ctx *ctx, int32_t run, double N_lo, double N_hi,
                         int32_t n_bins, double N_tail, fpt_hist *out, void *cuda_stream);

/*
 * The same weighted histogram over caller-supplied per-trajectory arrays
 * (n entries each, host or device; status as FPT_TRAJ_*), e.g. the merged
 * results of several fpt_run calls. Trajectories are numbered 0..n-1 for the
 * jackknife blocks. Blocks until the results are on the host.
 */
fpt_status fpt_histogram_data(fpt_ctx *ctx, const int32_t *nsteps, const double *logw,
                              const uint8_t *status, int64_t n, double dN, double N_lo,
                              double N_hi, int32_t n_bins, double N_tail, fpt_hist *out,
                              void *cuda_stream);

/*
 * ---- Learned importance-sampling proposal (FPT_BIAS_MLP) ----
 * The paper leaves the optimal bias in the 2-D phase space open (Sec. 5); the
 * learned proposal replaces the constant amplitude A of Eq. (4.10) by
 * alpha(x, pi, N) from a 3 -> 64 -> 64 -> 2 SiLU network with bf16 weights
 * and fp32 accumulation (see fpt_run_desc). Canonical fp32 parameter vector,
 * FPT_MLP_PARAMS floats, row-major (out, in): W1[64][3], b1[64], W2[64][64],
 * b2[64], W3[2][64], b3[2].
 */
#define FPT_MLP_PARAMS 4546
#define FPT_MLP_BLOB_BYTES 11808

/* Pack fp32 parameters (host or device, FPT_MLP_PARAMS floats) into the bf16
 * weight blob the stepper reads (device, FPT_MLP_BLOB_BYTES, 16-byte aligned,
 * caller-owned). Asynchronous on cuda_stream. */
fpt_status fpt_mlp_pack(fpt_ctx *ctx, const float *params, void *blob, void *cuda_stream);

/* alpha of the network at normalised inputs s (n x 3) and tan(theta_n) t (n),
 * with the stepper's own device code; o (n x 2, nullable) receives the raw
 * outputs. Buffers host or device; blocks until done. */
fpt_status fpt_mlp_eval(fpt_ctx *ctx, const void *blob, const float *s, const float *tan_t,
                        int64_t n, float alpha_max, float *alpha, float *o, void *cuda_stream);

/* grad = sum_r dalpha_r d alpha(s_r, t_r) / d theta over n records (the
 * backward kernel of training, bf16 tensor-core tiles, fp32 accumulation);
 * zero where |raw alpha| >= alpha_max. params fp32 (host or device); grad
 * FPT_MLP_PARAMS floats, overwritten. Blocks until done. */
fpt_status fpt_mlp_grad(fpt_ctx *ctx, const float *params, const float *s, const float *tan_t,
                        const float *dalpha, int64_t n, float alpha_max, float *grad,
                        void *cuda_stream);

/* Full-rank (2-D) counterpart: grad = sum_r dbeta_r . dbeta(s_r)/dtheta with
 * beta = (clamp(o1), clamp(o2)) (each to +-alpha_max, zero gradient on a
 * clamped component); dbeta n x 2 (host or device). Blocks until done. */
fpt_status fpt_mlp_grad2(fpt_ctx *ctx, const float *params, const float *s, const float *dbeta, int64_t n,
                         float alpha_max, float *grad, void *cuda_stream);

typedef struct {
    float lr, beta1, beta2, eps;
    float clip;            /* > 0: clamp each gradient component first        */
    int32_t step;          /* Adam step counter (1-based, bias correction)    */
} fpt_adam;

typedef struct {
    double loss;           /* Var(Y), Y = ln w + lambda min(N, N_cut)          */
    double mean_Y;
    double mean_N;         /* mean first-passage time of the round            */
    int64_t n_traj;
    int64_t n_records;     /* segments used for the gradient                  */
    int64_t n_capped;
    double grad_norm;      /* L2 norm of the gradient before clipping         */
} fpt_train_stats;

/*
 * One training round of the proposal: the run `run` (one FPT_BIAS_MLP run,
 * run->mlp == blob) is generated in chunks of `chunk` trajectories, recording
 * every held-alpha segment; then the gradient of the log-variance loss
 * L = Var[ln w + lambda min(N, N_cut)] at the sampling parameters,
 *   dL/dtheta = (2/n) sum_j (Y_j - mean_chunk Y) d ln w_j / dtheta,
 *   d ln w_j / dtheta = -sum_s sqrt(dN) (sum of xi over segment s) d alpha_s / dtheta,
 * (on a 2-D table: -sum_s sqrt(dN) sum_k (sum of xi_k over s) d beta_{s,k} / dtheta)
 * is accumulated, one Adam step updates params / adam_m / adam_v (device,
 * FPT_MLP_PARAMS floats each) and the blob is re-packed. Returns
 * FPT_E_NOMEM if a chunk's segment records exceed the record buffer (use a
 * smaller chunk). Blocks until done; the last chunk stays in the context as
 * the last run.
 */
fpt_status fpt_mlp_train_round(fpt_ctx *ctx, const fpt_run_desc *run, int64_t chunk,
                               double lambda, double N_cut, const fpt_adam *adam, float *params,
                               float *adam_m, float *adam_v, void *blob,
                               fpt_train_stats *stats, void *cuda_stream);

/*
 * One training round of n_runs proposals at once, each run (an FPT_BIAS_MLP run
 * on any model, 1-D phi-indexed table) with its own network: run k must use
 * blob k (blobs + k FPT_MLP_BLOB_BYTES, device) and its parameters and Adam
 * moments are params / adam_m / adam_v + k FPT_MLP_PARAMS (device floats). All
 * runs are generated in one launch with segment records (the runs share
 * mlp_segment); each run's records, in (trajectory, segment) order, give the
 * gradient of its own log-variance loss Var[ln w + lambda min(N, N_cut[k])]
 * over its own paths (as fpt_mlp_train_round with one chunk), then one Adam step
 * and a re-pack per network. stats (n_runs entries, nullable): loss, mean_Y,
 * mean_N, n_traj, n_records, n_capped per run (grad_norm NaN). FPT_E_NOMEM if
 * the records exceed 2^29. Blocks until done.
 */
fpt_status fpt_mlp_train_batch(fpt_ctx *ctx, const fpt_run_desc *runs, int32_t n_runs, double lambda,
                               const double *N_cut, const fpt_adam *adam, float *params, float *adam_m,
                               float *adam_v, void *blobs, fpt_train_stats *stats, void *cuda_stream);

/*
 * The held-alpha segments of one learned-proposal run (Sec. 5's open bias made
 * concrete: what the proposal did along each path), for analysis and tests:
 * the run (one FPT_BIAS_MLP run, 1-D table) is generated in record mode, the
 * same trajectories as fpt_run gives, and up to `cap` records are copied to
 * `records` (host or device, 8 floats each): the three normalised network
 * inputs, tan(theta_n), the unclamped alpha, the sum of xi over the segment,
 * the launch unit (trajectory index within the run, as uint32 bits) and the
 * segment's first step (int32 bits). Records come in the order the stepper
 * wrote them; sort by (unit, first step) for a path's sequence.
 * *n_records = all records of the run (possibly more than cap). Blocks.
 */
fpt_status fpt_run_records(fpt_ctx *ctx, const fpt_run_desc *run, int64_t cap, float *records,
                           int64_t *n_records, void *cuda_stream);

/*
 * The weighted histogram of fpt_histogram_data for callers that cannot
 * allocate device memory: code that runs where cudaMalloc is not allowed or
 * not wanted -- inside another library's allocation-free region, on a stream
 * being captured by an application that forbids allocation, or under an
 * allocator that owns all device memory. The paper has no counterpart; this is
 * an interface variant, not a step of the method.
 *
 * No context, no allocation: the scratch (per-bin maxima, jackknife moments,
 * scalars; about 1.3 MB) is a fixed array inside the library that every GPU
 * loading the library holds until the process exits. The call runs in the
 * CUDA context current on the calling thread (with none current, the current
 * device's primary context). The array's device address is valid only in
 * that context, so the first call in each context looks it up and caches it
 * by the context's id: the first call in the primary context of a device, in
 * a context pushed by another library, or after cudaDeviceReset (which makes
 * a new context). Make that first call in a context before any stream
 * capture. The array is cleared at the start of every call, and all calls
 * share it: calls whose work overlaps on the GPU (different streams, or
 * different threads without ordering) race and give wrong results.
 *
 * Inputs: nsteps, logw, status (device, n entries; status as FPT_TRAJ_*),
 * dN, bins as in fpt_histogram (1 <= n_bins <= FPT_NOALLOC_MAX_BINS), N_tail.
 * Output: `out`, device, FPT_HIST_OUT_DOUBLES(n_bins) doubles: ten arrays of
 * n_bins, then 16 scalars. Per bin b (empty bins in brackets):
 *   [0] count (0), [1] log_sum_w (-inf), [2] log_sum_w2 (-inf), [3] sum_lw (0),
 *   [4] sum_lw2 (0), [5] pdf (0), [6] se_w (0), [7] pdf_ln and [8] se_ln
 *   (NaN unless the bin holds at least 2 trajectories), [9] se_jk (0).
 * Scalars at 10 n_bins + k (value when no trajectory passed in brackets):
 *   0 n_total, 1 n_passed, 2 n_under, 3 n_over, 4 n_capped, 5 n_tail,
 *   6 N_mean (NaN), 7 N_mean_w (NaN), 8 ess_tail (0; also 0 with an empty
 *   tail set or N_tail = NaN), 9 p_tail (0 likewise), 10 log_max_w (-inf),
 *   11..15 reserved, written as 0.
 * Asynchronous on cuda_stream (NULL: the legacy default stream). Errors:
 * FPT_E_INVALID for bad sizes (message in fpt_last_error(NULL)), FPT_E_CUDA
 * for launch errors or a failed address lookup.
 */
#define FPT_NOALLOC_MAX_BINS 1024
#define FPT_HIST_OUT_DOUBLES(n_bins) (10 * (n_bins) + 16)
fpt_status fpt_histogram_noalloc(const int32_t *nsteps, const double *logw, const uint8_t *status,
                                 int64_t n, double dN, double N_lo, double N_hi, int32_t n_bins,
                                 double N_tail, double *out, void *cuda_stream);

/* Capped allocator: the device memory the context allocates (trajectory
 * outputs, tables, histogram, record and training scratch) is counted, and
 * from this call on an allocation that would take the count past max_bytes
 * fails as an out-of-memory cudaMalloc does: the call that needed it returns
 * FPT_E_NOMEM (fpt_last_error names the limit, the bytes in use and the bytes
 * requested), and the context stays usable -- a later call with a smaller
 * request, or after the limit is raised, succeeds. Memory already held is
 * kept. max_bytes = 0 removes the limit (the default); negative values are
 * FPT_E_INVALID. Serves memory budgeting beside other users of the GPU and
 * the injection of allocation failures.
 */
fpt_status fpt_set_memory_limit(fpt_ctx *ctx, int64_t max_bytes);

/* Device bytes the context holds now (*in_use) and its limit (*max_bytes,
 * 0 = none); either pointer may be NULL. */
fpt_status fpt_memory_in_use(const fpt_ctx *ctx, int64_t *in_use, int64_t *max_bytes);

/* Release everything the context owns. NULL is allowed. */
void fpt_destroy(fpt_ctx *ctx);

/* Message of the last error on this context (or of the last failed
 * fpt_init_model when ctx is NULL). Never NULL. */
const char *fpt_last_error(const fpt_ctx *ctx);

/* Library version string. */
const char *fpt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FPT_H */
