/*
 * fpt_oracle.c -- plain FP64 CPU oracle for the stochastic-delta-N
 * first-passage sampler of arXiv:2410.13683.
 *
 * TEST INFRASTRUCTURE ONLY. The product library never calls, links or loads
 * this file; only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg do. It shares no code, header, table or constant generator with
 * the CUDA path: everything here is restated from the paper and from the
 * published definition of the Philox generator.
 *
 * What it computes, step by step, in double precision:
 *   - Euler-Maruyama steps (Eq. 4.1) of the 1-D-noise Langevin system
 *     (Eq. 4.6) with the importance-sampling bias of Eq. (4.7); the momentum
 *     drift carries the minus sign of Eqs. (2.21) and (4.1) (Eq. 4.7 drops it,
 *     read here as a typo);
 *   - the bias lies along the noise vector (1, tan theta_n): B = alpha S (1, t).
 *     The per-dimension weights of Eq. (4.8) agree exactly when
 *     B_pi = tan(theta_n) B_phi (Eq. 4.9 prints the inverse relation);
 *   - per-step weight increment dA = alpha (alpha dN / 2 + xi sqrt(dN)), the
 *     one-dimensional form of Eq. (4.5); w = exp(-sum dA), Eq. (4.4);
 *   - first passage: the first step n >= 1 with phi_n <= phi_end, N = n dN
 *     (Sec. 4.1);
 *   - the noise S(phi) and S_pi(phi) = tan(theta_n) S(phi) come from a
 *     phi-indexed table by linear interpolation (the phi-indexing proposed in
 *     Sec. 5); outside the table the end values are held.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 * (seed_lo, seed_hi), counter = (step >> 2, trajectory id, run id, 0); the four
 * 32-bit words become uniforms u_k = ((r_k >> 9) + 0.5) 2^-23 and two
 * Box-Muller pairs (z0, z1) <- (u0, u1), (z2, z3) <- (u2, u3); step i uses
 * z[i & 3].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from its published definition.                    */
/* ------------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* Weyl key bumps    */
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(M0, c0, &hi0, &lo0);
        mulhilo32(M1, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Four standard normals for steps 4*block .. 4*block+3 of one trajectory. */
void oracle_normals4(uint64_t seed, uint32_t run_id, uint32_t traj,
                     uint32_t block, double z[4])
{
    uint32_t ctr[4] = {block, traj, run_id, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    oracle_philox4x32_10(ctr, key, r);
    double u[4];
    for (int k = 0; k < 4; ++k)
        u[k] = ((double)(r[k] >> 9) + 0.5) * (1.0 / 8388608.0);
    for (int p = 0; p < 2; ++p) {
        double rad = sqrt(-2.0 * log(u[2 * p]));
        double ang = 2.0 * OR_PI * u[2 * p + 1];
        z[2 * p] = rad * cos(ang);
        z[2 * p + 1] = rad * sin(ang);
    }
}

/* ------------------------------------------------------------------------ */
/* Model, table and bias descriptions.                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t kind;        /* 0: piecewise-linear, relative slopes; 1: V0 exp(mu phi);
                            2: Gaussian bump V0 phi^2/(m^2+phi^2) [1 + K exp(-(phi-phi0)^2/(2 w^2))] */
    int32_t pad;
    double V0, a_plus, a_minus, phi_star, mu;
    double phi_in, pi_in, phi_end, dN;
    int64_t max_steps;
    double bump_K, bump_m, bump_w, bump_phi0;
} oracle_model;

typedef struct {
    int64_t n_points;    /* M >= 2 */
    double phi_lo, h;    /* grid phi_j = phi_lo + j h (N-indexed: N_j = phi_lo + j h) */
    const double *S;     /* S_phiphi at the grid points              */
    const double *T;     /* S_piphi = tan(theta_n) S at the grid points */
    int32_t n_indexed;   /* 1: indexed by the time N = n dN since the start, with
                            zero noise outside [N_0, N_{M-1}] (the noise window) */
    int32_t pad;
} oracle_table;

typedef struct {
    int32_t kind;        /* 0: none, 1: constant amplitude, 2: MLP */
    int32_t hidden;      /* MLP width (64) */
    double A;            /* constant amplitude */
    int64_t segment;     /* MLP: alpha recomputed every `segment` steps */
    double alpha_max;    /* MLP: |alpha| clamp */
    int32_t round_bf16;  /* MLP: bfloat16 network -- inputs and hidden activations rounded
                            to bfloat16 here; the weights W1..W3 come already rounded
                            (oracle/stepper.py MLPBias), the biases as given */
    int32_t log_x;       /* MLP: first input ln(max(phi - phi_end, x_floor)) */
    const double *W1, *b1, *W2, *b2, *W3, *b3;   /* row-major (out, in) */
    double in_shift[3], in_scale[3];             /* input = (s - shift) * scale */
    double x_floor;      /* MLP, log_x: floor of x under the log (<= 0: 1e-30) */
} oracle_bias;

/* The log-field network input ln max(x, floor): below the floor the input is
 * held, so that it stays well conditioned as x -> 0 at the end surface. */
static double log_input(const oracle_bias *b, double x)
{
    const double fl = b->x_floor > 0.0 ? b->x_floor : 1e-30;
    return log(x > fl ? x : fl);
}

/* Slope term V'(phi)/V(phi) of the potential families. The Gaussian bump of
 * Sec. 4.3, V = V0 f (1 + g) with f = phi^2/(m^2 + phi^2) and
 * g = K exp(-(phi - phi0)^2/(2 w^2)), has V'/V = f'/f + g'/(1 + g),
 * f'/f = 2 m^2 / (phi (m^2 + phi^2)), g' = -g (phi - phi0)/w^2. */
static double dlnV(const oracle_model *m, double phi)
{
    if (m->kind == 1)
        return m->mu;
    if (m->kind == 2) {
        double m2 = m->bump_m * m->bump_m, d = phi - m->bump_phi0, w2 = m->bump_w * m->bump_w;
        double g = m->bump_K * exp(-0.5 * d * d / w2);
        return 2.0 * m2 / (phi * (m2 + phi * phi)) - g * d / (w2 * (1.0 + g));
    }
    double d = phi - m->phi_star;
    double a = (phi >= m->phi_star) ? m->a_plus : m->a_minus;
    return a / (1.0 + a * d);
}

/* Linear interpolation of the noise table. phi-indexed tables hold their end
 * values outside the grid; N-indexed tables (the paper's production setting,
 * Sec. 4.1: noise precomputed along the classical background in global time
 * and switched off after a window) give zero noise outside it. */
static void table_lookup(const oracle_table *t, double phi, double *S, double *T)
{
    double M1 = (double)(t->n_points - 1);
    double u = (phi - t->phi_lo) / t->h;
    if (u < 0.0) u = 0.0;
    if (u > M1) u = M1;
    int64_t i = (int64_t)floor(u);
    if (i > t->n_points - 2) i = t->n_points - 2;
    double f = u - (double)i;
    *S = t->S[i] + f * (t->S[i + 1] - t->S[i]);
    *T = t->T[i] + f * (t->T[i + 1] - t->T[i]);
}

/* Round a double to the nearest bfloat16 value (ties to even). */
static double to_bf16(double v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return v;  /* inf / nan */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double silu(double v) { return v / (1.0 + exp(-v)); }

/* MLP outputs (o1, o2) for state (x, pi, N); x = phi - phi_end. */
void oracle_mlp_forward(const oracle_bias *b, const double s[3], double o[2])
{
    int H = b->hidden;
    double in[3], h1[256], h2[256];
    for (int k = 0; k < 3; ++k) {
        in[k] = (s[k] - b->in_shift[k]) * b->in_scale[k];
        if (b->round_bf16) in[k] = to_bf16(in[k]);
    }
    for (int j = 0; j < H; ++j) {
        double a = b->b1[j];
        for (int k = 0; k < 3; ++k) a += b->W1[j * 3 + k] * in[k];
        h1[j] = silu(a);
        if (b->round_bf16) h1[j] = to_bf16(h1[j]);
    }
    for (int j = 0; j < H; ++j) {
        double a = b->b2[j];
        for (int k = 0; k < H; ++k) a += b->W2[j * H + k] * h1[k];
        h2[j] = silu(a);
        if (b->round_bf16) h2[j] = to_bf16(h2[j]);
    }
    for (int j = 0; j < 2; ++j) {
        double a = b->b3[j];
        for (int k = 0; k < H; ++k) a += b->W3[j * H + k] * h2[k];
        o[j] = a;
    }
}

/* Bias amplitude from the MLP: projection of (o1, o2) on the noise direction
 * (1, t)/sqrt(1 + t^2), clamped to |alpha| <= alpha_max. */
static double mlp_alpha(const oracle_bias *b, const oracle_model *m,
                        double phi, double pi, int64_t n, double t)
{
    double x = phi - m->phi_end;
    if (b->log_x) x = log_input(b, x);
    double s[3] = {x, pi, (double)n * m->dN};
    double o[2];
    oracle_mlp_forward(b, s, o);
    double a = (o[0] + t * o[1]) / sqrt(1.0 + t * t);
    if (a > b->alpha_max) a = b->alpha_max;
    if (a < -b->alpha_max) a = -b->alpha_max;
    return a;
}

typedef struct {
    int64_t *nsteps;
    double *logw;
    uint8_t *status;     /* 0: passed, 1: capped at max_steps */
    double *phi_final;
    double *pi_final;
    double *xmin_pre;    /* min of phi_n - phi_end over steps 1..n-1 (inf if none) */
} oracle_out;

/* Optional per-segment record for the learned-bias gradient. */
typedef struct {
    int64_t cap;         /* capacity in segments */
    int64_t *n_seg;      /* out: segments recorded */
    double *state;       /* [cap][3] (x, pi, N) at the segment start */
    double *tan_theta;   /* [cap] t at the segment start */
    double *alpha;       /* [cap] alpha used */
    double *sum_xi;      /* [cap] sum of xi over the steps of the segment */
} oracle_segments;

/* One trajectory, plain FP64 Euler-Maruyama. */
static void one_trajectory(const oracle_model *m, const oracle_table *tab,
                           const oracle_bias *b, uint64_t seed, uint32_t run_id,
                           uint32_t traj, int64_t *nsteps, double *logw,
                           uint8_t *status, double *phi_f, double *pi_f,
                           double *xmin, oracle_segments *seg)
{
    const double dN = m->dN, sdN = sqrt(m->dN);
    double phi = m->phi_in, pi = m->pi_in, lw = 0.0, xm = INFINITY;
    /* N-indexed tables: the window is the integer step range whose times n dN
     * lie in [N_0, N_{M-1}] (with a 1e-9 allowance for the division) */
    int64_t win_lo = 0, win_hi = -1;
    if (tab->n_indexed) {
        win_lo = (int64_t)ceil(tab->phi_lo / dN - 1e-9);
        win_hi = (int64_t)floor((tab->phi_lo + tab->h * (double)(tab->n_points - 1)) / dN + 1e-9);
    }
    double z[4];
    double alpha = (b->kind == 1) ? b->A : 0.0;
    int64_t n = 0, ns = 0;
    int passed = 0;
    while (n < m->max_steps) {
        if ((n & 3) == 0)
            oracle_normals4(seed, run_id, traj, (uint32_t)(n >> 2), z);
        double xi = z[n & 3];
        double S = 0.0, T = 0.0;
        int noisy = 1;
        if (!tab->n_indexed)
            table_lookup(tab, phi, &S, &T);
        else if (n >= win_lo && n <= win_hi)   /* step inside the noise window */
            table_lookup(tab, (double)n * dN, &S, &T);
        else
            noisy = 0;                         /* classical step: no noise, no bias, no weight */
        if (b->kind == 2 && (n % b->segment) == 0) {
            double t = (S != 0.0) ? T / S : 0.0;
            alpha = mlp_alpha(b, m, phi, pi, n, t);
            if (seg && ns < seg->cap) {
                double x = phi - m->phi_end;
                if (b->log_x) x = log_input(b, x);
                seg->state[3 * ns + 0] = x;
                seg->state[3 * ns + 1] = pi;
                seg->state[3 * ns + 2] = (double)n * dN;
                seg->tan_theta[ns] = t;
                seg->alpha[ns] = alpha;
                seg->sum_xi[ns] = 0.0;
            }
            ++ns;
        }
        if (b->kind == 2 && seg && ns - 1 < seg->cap)
            seg->sum_xi[ns - 1] += xi;
        const double a = noisy ? alpha : 0.0;
        double drift_pi = -(3.0 - 0.5 * pi * pi) * (pi + dlnV(m, phi));
        double phi_new = phi + pi * dN + a * S * dN + S * xi * sdN;
        double pi_new = pi + drift_pi * dN + a * T * dN + T * xi * sdN;
        lw -= a * (0.5 * a * dN + xi * sdN);
        phi = phi_new;
        pi = pi_new;
        ++n;
        if (phi <= m->phi_end) { passed = 1; break; }
        double x = phi - m->phi_end;
        if (x < xm) xm = x;
    }
    *nsteps = n;
    *logw = lw;
    *status = passed ? 0 : 1;
    *phi_f = phi;
    *pi_f = pi;
    *xmin = xm;
    if (seg) *seg->n_seg = ns < seg->cap ? ns : seg->cap;
}

/* ------------------------------------------------------------------------ */
/* Full-rank (2-D) noise: Euler-Maruyama of Eq. (2.24) with the symmetric     */
/* square root S of the covariance Xi of Eq. (3.9); two normals per step      */
/* (step i uses normals 2(i & 1) and 2(i & 1) + 1 of Philox block i >> 1).    */
/* The bias is written in standardised form, B = S beta, so that Eq. (4.5)    */
/* gives dA = (S beta dN/2 + S xi sqrt(dN))^T Xi^-1 S beta                    */
/*          = beta . (beta dN/2 + xi sqrt(dN))   (S^T Xi^-1 S = 1).           */
/* beta = (A, A2) for a constant bias; for the learned proposal               */
/* beta = (clamp(o1), clamp(o2)), the two MLP outputs, each clamped to        */
/* +-alpha_max and held for `segment` steps.                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n_points;
    double phi_lo, h;
    const double *Spp, *Spq, *Sqq;   /* S_phiphi, S_phipi = S_piphi, S_pipi */
} oracle_table2;

static void table2_lookup(const oracle_table2 *t, double phi, double *a, double *b, double *c)
{
    double M1 = (double)(t->n_points - 1);
    double u = (phi - t->phi_lo) / t->h;
    if (u < 0.0) u = 0.0;
    if (u > M1) u = M1;
    int64_t i = (int64_t)floor(u);
    if (i > t->n_points - 2) i = t->n_points - 2;
    double f = u - (double)i;
    *a = t->Spp[i] + f * (t->Spp[i + 1] - t->Spp[i]);
    *b = t->Spq[i] + f * (t->Spq[i + 1] - t->Spq[i]);
    *c = t->Sqq[i] + f * (t->Sqq[i + 1] - t->Sqq[i]);
}

static double clampd(double v, double lim)
{
    return v > lim ? lim : (v < -lim ? -lim : v);
}

/* Optional per-segment record of the learned 2-D bias. */
typedef struct {
    int64_t cap;
    int64_t *n_seg;
    double *state;       /* [cap][3] (x or ln x, pi, N) at the segment start */
    double *beta;        /* [cap][2] beta used */
    double *sum_xi;      /* [cap][2] sums of xi_1, xi_2 over the segment */
} oracle_segments2;

static void one_trajectory2(const oracle_model *m, const oracle_table2 *tab, const oracle_bias *bias,
                            double A2, uint64_t seed, uint32_t run_id, uint32_t traj,
                            int64_t *nsteps, double *logw, uint8_t *status, double *phi_f,
                            double *pi_f, double *xmin, oracle_segments2 *seg)
{
    int64_t ns = 0;
    const double dN = m->dN, sdN = sqrt(m->dN);
    double phi = m->phi_in, pi = m->pi_in, lw = 0.0, xm = INFINITY;
    double beta1 = 0.0, beta2 = 0.0;
    if (bias->kind == 1) { beta1 = bias->A; beta2 = A2; }
    double z[4];
    int64_t n = 0;
    int passed = 0;
    while (n < m->max_steps) {
        if ((n & 1) == 0)
            oracle_normals4(seed, run_id, traj, (uint32_t)(n >> 1), z);
        double xi1 = z[2 * (n & 1)], xi2 = z[2 * (n & 1) + 1];
        double a, b, c;
        table2_lookup(tab, phi, &a, &b, &c);
        if (bias->kind == 2 && (n % bias->segment) == 0) {
            double x = phi - m->phi_end;
            if (bias->log_x) x = log_input(bias, x);
            double s[3] = {x, pi, (double)n * dN}, o[2];
            oracle_mlp_forward(bias, s, o);
            beta1 = clampd(o[0], bias->alpha_max);
            beta2 = clampd(o[1], bias->alpha_max);
            if (seg && ns < seg->cap) {
                for (int k = 0; k < 3; ++k) seg->state[3 * ns + k] = s[k];
                seg->beta[2 * ns] = beta1;
                seg->beta[2 * ns + 1] = beta2;
                seg->sum_xi[2 * ns] = seg->sum_xi[2 * ns + 1] = 0.0;
            }
            ++ns;
        }
        if (bias->kind == 2 && seg && ns - 1 < seg->cap) {
            seg->sum_xi[2 * (ns - 1)] += xi1;
            seg->sum_xi[2 * (ns - 1) + 1] += xi2;
        }
        double B_phi = a * beta1 + b * beta2, B_pi = b * beta1 + c * beta2;   /* B = S beta */
        double drift_pi = -(3.0 - 0.5 * pi * pi) * (pi + dlnV(m, phi));
        double phi_new = phi + pi * dN + B_phi * dN + (a * xi1 + b * xi2) * sdN;
        double pi_new = pi + drift_pi * dN + B_pi * dN + (b * xi1 + c * xi2) * sdN;
        lw -= beta1 * (0.5 * beta1 * dN + xi1 * sdN) + beta2 * (0.5 * beta2 * dN + xi2 * sdN);
        phi = phi_new;
        pi = pi_new;
        ++n;
        if (phi <= m->phi_end) { passed = 1; break; }
        double x = phi - m->phi_end;
        if (x < xm) xm = x;
    }
    *nsteps = n;
    *logw = lw;
    *status = passed ? 0 : 1;
    *phi_f = phi;
    *pi_f = pi;
    *xmin = xm;
    if (seg) *seg->n_seg = ns < seg->cap ? ns : seg->cap;
}

/* One learned-bias 2-D trajectory with its per-segment records. */
int oracle_run2_segments(const oracle_model *m, const oracle_table2 *tab, const oracle_bias *bias,
                         uint64_t seed, uint32_t run_id, uint32_t traj, int64_t *nsteps, double *logw,
                         uint8_t *status, oracle_segments2 *seg)
{
    if (!m || !tab || !bias || !seg || bias->kind != 2 || bias->segment < 1) return 1;
    double phi_f, pi_f, xm;
    one_trajectory2(m, tab, bias, 0.0, seed, run_id, traj, nsteps, logw, status, &phi_f, &pi_f, &xm, seg);
    return 0;
}

int oracle_run2(const oracle_model *m, const oracle_table2 *tab, const oracle_bias *bias, double A2,
                uint64_t seed, uint32_t run_id, int64_t traj0, int64_t n, int threads, oracle_out *out)
{
    if (!m || !tab || !bias || !out || n < 0 || tab->n_points < 2) return 1;
    if (traj0 < 0 || traj0 + n > 4294967296LL) return 1;
    if (bias->kind == 2 && bias->segment < 1) return 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < n; ++i) {
        one_trajectory2(m, tab, bias, A2, seed, run_id, (uint32_t)(traj0 + i), &out->nsteps[i],
                        &out->logw[i], &out->status[i], &out->phi_final[i], &out->pi_final[i],
                        &out->xmin_pre[i], NULL);
    }
    return 0;
}

/* Run trajectories traj0 .. traj0+n-1 of one run. Returns 0 on success. */
int oracle_run(const oracle_model *m, const oracle_table *tab,
               const oracle_bias *b, uint64_t seed, uint32_t run_id,
               int64_t traj0, int64_t n, int threads, oracle_out *out)
{
    if (!m || !tab || !b || !out || n < 0 || tab->n_points < 2) return 1;
    if (traj0 < 0 || traj0 + n > 4294967296LL) return 1;
    if (b->kind == 2 && (b->segment <= 0 || b->hidden <= 0 || b->hidden > 256)) return 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < n; ++i) {
        one_trajectory(m, tab, b, seed, run_id, (uint32_t)(traj0 + i),
                       &out->nsteps[i], &out->logw[i], &out->status[i],
                       &out->phi_final[i], &out->pi_final[i], &out->xmin_pre[i],
                       NULL);
    }
    return 0;
}

/* One trajectory with its segment records (learned-bias gradient checks). */
int oracle_run_segments(const oracle_model *m, const oracle_table *tab,
                        const oracle_bias *b, uint64_t seed, uint32_t run_id,
                        int64_t traj, int64_t *nsteps, double *logw,
                        uint8_t *status, oracle_segments *seg)
{
    if (!m || !tab || !b || !seg || b->kind != 2) return 1;
    double pf, pif, xm;
    one_trajectory(m, tab, b, seed, run_id, (uint32_t)traj, nsteps, logw, status,
                   &pf, &pif, &xm, seg);
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
