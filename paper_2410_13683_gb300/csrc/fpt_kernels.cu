// fpt_kernels.cu -- sm_103a kernels of the first-passage sampler.
//
//   em_kernel      persistent Euler-Maruyama stepper: one trajectory per
//                  thread, Philox4x32-10 noise, phi-indexed noise table in
//                  shared memory, importance-sampling bias and Kahan-summed
//                  log-weight, warp-ballot refill of finished trajectories.
//   hist_*         weighted histogram of first-passage times (per-bin max,
//                  shifted sums in shared memory, FP64 flush) and the FP64
//                  finalisation of P(delta N) and its errors.
//
// Method (arXiv:2410.13683): Euler-Maruyama steps, Eq. (4.1), of the 1-D-noise
// system, Eq. (4.6), with the bias of Eq. (4.7) along the noise vector
// (1, tan theta_n) (the direction for which the weights of Eq. (4.8) agree) and
// the diffusion-based amplitude of Eq. (4.10); weight increment
// dA = A (A dN/2 + xi sqrt(dN)) (Eq. 4.5 in one dimension), w = exp(-sum dA)
// (Eq. 4.4); first passage at the first step n >= 1 with phi_n <= phi_end,
// N = n dN (Sec. 4.1).
#include "fpt_internal.h"
#include "fpt_mlp.cuh"

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

namespace fpt_dev {

// Device bounds checks of FPT_CHECKS builds: a failed check sets its bit
// (kCheck*) in the error word and redirects the access to a valid index; the
// kernel carries on (warp-synchronous code cannot leave early), and the host
// reads and clears the word after each run or histogram (checks_take) and
// turns it into FPT_E_STATE. Other builds compile the checks away.
#ifdef FPT_CHECKS
__device__ int g_check_word;
#define CHECK_INDEX(idx, n, bit)                        \
    do {                                                \
        if ((idx) < 0 || (idx) >= (n)) {                \
            atomicOr(&g_check_word, (bit));             \
            (idx) = 0;                                  \
        }                                               \
    } while (0)
#else
#define CHECK_INDEX(idx, n, bit) do {} while (0)
#endif

cudaError_t checks_take(int *word)
{
    *word = 0;
#ifdef FPT_CHECKS
    cudaError_t e = cudaMemcpyFromSymbol(word, g_check_word, sizeof(int));
    if (e != cudaSuccess) return e;
    const int zero = 0;
    return cudaMemcpyToSymbol(g_check_word, &zero, sizeof(int));
#else
    return cudaSuccess;
#endif
}

// ---------------------------------------------------------------------------
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// ---------------------------------------------------------------------------
// The key schedule (k0 + r W0, k1 + r W1 for rounds r = 0..9) is the same for
// every call of a launch: it comes precomputed in the kernel parameters
// (rk[2r], rk[2r+1]), so each round is two wide multiplies and two
// three-input XORs with constant-bank operands.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const uint32_t (&rk)[20])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = 0xD2511F53ull * (unsigned long long)c.x;
        const unsigned long long p1 = 0xCD9E8D57ull * (unsigned long long)c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
    }
    return c;
}

__device__ __forceinline__ float rcp_approx(float v)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ float sqrt_approx(float v)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Two standard normals from two Philox words: 23-bit uniforms
// u = ((r >> 9) + 0.5) 2^-23, built from the mantissa bits (1 + (r >> 9) 2^-23
// minus (1 - 2^-24), exact by Sterbenz), then Box-Muller
// z0 = rho cos(2 pi u1), z1 = rho sin(2 pi u1), rho = sqrt(-2 ln u0); the
// angle is evaluated as 2 pi u1 - pi, inside the accurate range of the
// hardware sine/cosine, and the signs restored.
__device__ __forceinline__ float uniform23(uint32_t r)
{
    return __int_as_float(0x3f800000u | (r >> 9)) - 0.99999994039535522f;   // 1 - 2^-24
}

// The normals are products (rho cos, rho sin): the record mode's sums of
// normals are explicit __fadd_rn, which the compiler never fuses with the
// product into an FMA. A contracted sum would round differently wherever the
// compiler chose to fuse, and the speculative and guarded paths (and the
// recomputation of a group's normals after a passage) would no longer give the
// same sums.
__device__ __forceinline__ void box_muller(uint32_t r0, uint32_t r1, float &z0, float &z1)
{
    const float u0 = uniform23(r0);
    const float u1 = uniform23(r1);
    const float rho = sqrt_approx(fmaxf(-1.38629436111989061f * __log2f(u0), 0.0f));   // -2 ln u0
    float sn, cs;
    __sincosf(fmaf(u1, 6.28318530717958648f, -3.14159265358979324f), &sn, &cs);
    z0 = -rho * cs;
    z1 = -rho * sn;
}

// Compensated (Kahan) accumulation of v into the pair (hi, lo), whose value
// is hi - lo: lo holds the amount by which hi overshoots the exact sum.
__device__ __forceinline__ void kahan_add(float &hi, float &lo, float v)
{
    const float y = __fsub_rn(v, lo);
    const float t = __fadd_rn(hi, y);
    lo = __fsub_rn(__fsub_rn(t, hi), y);
    hi = t;
}

// ---------------------------------------------------------------------------
// K1: persistent Euler-Maruyama stepper
// ---------------------------------------------------------------------------
struct RunSm {               // per-run constants staged in shared memory
    long long unit_begin;
    long long traj_offset;
    float cb, half_cb2, cb_b;
    uint32_t run_id;
    int32_t model;
    int32_t is_mlp;
    float sqrt_dN, dN;
};

struct Lane {                // per-thread trajectory state and its constants
    float x, x_c;            // shifted field phi - phi_end as a Kahan pair: x - x_c
    float p, p_c;            // momentum; p_c compensates it (Kahan) in the variants with pi-noise
    float lw_hi, lw_lo;      // ln w as a Kahan pair
    float lw_grp;            // increments of the current 4-step group, added to the pair per group
    int n;
    int nmax;
    uint32_t traj, run_id;
    float cb, half_cb2, dN, sqrt_dN;
    float cb_b;              // 2-D noise: beta_2 sqrt(dN) (cb = beta_1 sqrt(dN))
    union {                  // drift constants of the lane's potential
        struct { float x_star, x_star_lo, inv_a_plus, inv_a_minus, c; } pw;   // piecewise-linear / exponential
        struct { float scale, umax; int dtab, model; } bump;              // Gaussian bump: cubic V'/V table
    } dc;
    float u_scale, u_shift, u_max;
    int tbase;
    int M;                   // noise-table points of the lane's model (bounds checks)
    bool mlp;
    bool nidx;               // noise table indexed by the step count
    int win_lo, win_hi;      // noise window in steps (nidx)
    int run;                 // index of the lane's run in the launch
    long long unit;
};

struct SegRec {              // open segment of the record variant
    float in0, in1, in2, tan_t, raw, sum_xi;
    float sum_xi2;           // 2-D noise: sum of xi_2 (sum_xi holds xi_1)
    int n0;
    bool open;
};

__device__ __forceinline__ void lane_load(Lane &L, long long unit, const RunSm *s_run,
                                          const ModelDev *s_model, int n_runs)
{
    // last run whose first unit is <= unit (runs are contiguous in unit order)
    int lo = 0, hi = n_runs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_run[mid].unit_begin <= unit) lo = mid; else hi = mid - 1;
    }
    const RunSm &r = s_run[lo];
    const ModelDev &m = s_model[r.model];
    L.run = lo;
    L.unit = unit;
    L.traj = (uint32_t)(r.traj_offset + (unit - r.unit_begin));
    L.run_id = r.run_id;
    L.cb = r.cb;
    L.half_cb2 = r.half_cb2;
    L.cb_b = r.cb_b;
    L.mlp = r.is_mlp != 0;
    L.dN = m.dN;
    L.sqrt_dN = r.sqrt_dN;
    if (m.dtab >= 0) {
        L.dc.bump.scale = m.d_scale;
        L.dc.bump.umax = m.d_umax;
        L.dc.bump.dtab = m.dtab;
        L.dc.bump.model = r.model;
    } else {
        L.dc.pw.x_star = m.x_star;
        L.dc.pw.x_star_lo = m.x_star_lo;
        L.dc.pw.inv_a_plus = m.inv_a_plus;
        L.dc.pw.inv_a_minus = m.inv_a_minus;
        L.dc.pw.c = m.drift_c;
    }
    L.u_scale = m.u_scale;
    L.u_shift = m.u_shift;
    L.u_max = m.u_umax;
    L.tbase = m.table_offset;
    L.M = m.M;
    L.nidx = m.nidx != 0;
    L.win_lo = m.win_lo;
    L.win_hi = m.win_hi;
    L.nmax = m.max_steps;
    L.x = m.x_in;
    L.x_c = 0.0f;
    L.p = m.pi_in;
    L.p_c = 0.0f;
    L.lw_hi = 0.0f;
    L.lw_lo = 0.0f;
    L.lw_grp = 0.0f;
    L.n = 0;
}

// Table entry and interpolation weight at the lane's field. The 1-D tables
// hold, per interval k, the midpoint values (v_k + v_{k+1})/2 and the slopes
// v_{k+1} - v_k of (S', T') (times sqrt(dN)); with u' = (phi - phi_lo)/h - 1/2
// clamped to [-1/2, M - 3/2], k = round(u') comes from adding 1.5 2^23 (round
// to nearest in the mantissa, no float/int conversion) and f' = u' - k lies in
// [-1/2, 1/2]: v(u) = mid_k + f' slope_k. The last entry repeats v_{M-1} with
// zero slope, so every reachable k (0 .. M-1) is a valid entry.
template <bool SMEM, bool NIDX = false>
__device__ __forceinline__ float4 table_at(const Lane &L, const float4 *__restrict__ tab, float &f,
                                           const ModelDev &M0)
{
    const float kMagic = 12582912.0f;                        // 1.5 * 2^23
    // N-indexed tables: coordinate from the exact step count (n < 2^24 is exact in FP32)
    const float coord = (NIDX && L.nidx) ? __int2float_rn(L.n) : L.x;
    float u = fmaf(coord, SMEM ? M0.u_scale : L.u_scale, SMEM ? M0.u_shift : L.u_shift);
    u = fminf(fmaxf(u, -0.5f), SMEM ? M0.u_umax : L.u_max);
    const float t = u + kMagic;
    int i = __float_as_int(t) - 0x4b400000;
    f = u - (t - kMagic);
    CHECK_INDEX(i, SMEM ? M0.M : L.M, kCheckTable);
    return SMEM ? tab[i] : __ldg(tab + L.tbase + i);
}

// V'/V at the lane's field. Piecewise-linear (relative slopes) and
// exponential potentials: a / (1 + b (x - x_star)), branch by side.
// Gaussian bump (DTAB): near its inflection point V'/V is the small
// difference of two terms of size ~0.05, which FP32 cannot resolve, so it is
// read from a cubic (Hermite) table of the FP64 values on a uniform x grid
// (coefficients c0..c3 of s in [0, 1] per interval; one padding entry), and
// evaluated from the closed form in FP32 only above the table.
template <bool DTAB, bool SMEM>
__device__ __forceinline__ float drift_vpv(const Lane &L, const float4 *__restrict__ tab,
                                           const ModelDev *s_model, const ModelDev &M0)
{
    if (!DTAB) {
        // side of the kink from the compensated field and kink position:
        // x - x_c >= x_star + x_star_lo (x - x_star is exact near the kink), so
        // the branch follows the field itself, not the rounding of its FP32 head.
        // V'/V = a / (1 + a d) = 1 / (1/a + d) on each side (c = 1; the
        // exponential potential has c = 0 and V'/V = 1/(1/mu)).
        const float d = L.x - (SMEM ? M0.x_star : L.dc.pw.x_star);
        const bool up = d >= L.x_c + (SMEM ? M0.x_star_lo : L.dc.pw.x_star_lo);
        const float ia = up ? (SMEM ? M0.inv_a_plus : L.dc.pw.inv_a_plus)
                            : (SMEM ? M0.inv_a_minus : L.dc.pw.inv_a_minus);
        return rcp_approx(fmaf(SMEM ? M0.drift_c : L.dc.pw.c, d, ia));
    }
    const float u = fmaxf(L.x * (SMEM ? M0.d_scale : L.dc.bump.scale), 0.0f);
    if (u <= (SMEM ? M0.d_umax : L.dc.bump.umax)) {
        const float kMagic = 12582912.0f;                    // 1.5 * 2^23
        const float t = (u - 0.5f) + kMagic;
        int i = __float_as_int(t) - 0x4b400000;
        const float sv = u - (t - kMagic);
        CHECK_INDEX(i, (int)(SMEM ? M0.d_umax : L.dc.bump.umax) + 1, kCheckDriftTable);
        const float4 c = SMEM ? tab[M0.dtab + i] : __ldg(tab + L.tbase + L.dc.bump.dtab + i);
        return fmaf(sv, fmaf(sv, fmaf(sv, c.w, c.z), c.y), c.x);
    }
    const ModelDev &md = SMEM ? M0 : s_model[L.dc.bump.model];
    const float phi = L.x + md.bump_phi_end;
    const float d = L.x + md.bump_dphi0;                     // phi - phi0
    const float g = md.bump_K * __expf(-0.5f * d * d * md.bump_inv_w2);
    return __fdividef(2.0f * md.bump_m2, phi * fmaf(phi, phi, md.bump_m2)) -
           __fdividef(g * d * md.bump_inv_w2, 1.0f + g);
}

// Passage test on the compensated field: the pair's value x - x_c is <= 0
// exactly when x <= x_c (without flush-to-zero the rounded difference of two
// floats is zero or negative only when the exact one is), so the test needs
// no subtraction.
__device__ __forceinline__ bool passed(const Lane &L)
{
    return L.x <= L.x_c;
}

// Steps outside the noise window of an N-indexed table (step count below
// win_lo or above win_hi) are classical.
template <bool NIDX>
__device__ __forceinline__ bool outside_window(const Lane &L, int n)
{
    return NIDX && L.nidx && (n < L.win_lo || n > L.win_hi);
}

// (pi^2/2 - 3) dN, the momentum drift's factor, as (0.5 dN pi) pi - 3 dN with
// the FP32 constants 0.5 dN and -3 dN (single-model launches read them from
// the model descriptor, the others form the same products from dN).
template <bool SMEM>
__device__ __forceinline__ float hh_dN(const Lane &L, const ModelDev &M0)
{
    const float h = SMEM ? M0.half_dN : 0.5f * L.dN;
    const float m3 = SMEM ? M0.m3dN : -3.0f * L.dN;
    return fmaf(h * L.p, L.p, m3);
}

// One Euler-Maruyama step of Eq. (4.7) with bias amplitude L.cb / sqrt(dN).
// The field increment (drift + bias + noise) is formed first and added to the
// compensated field pair: a plain FP32 field would add the same drift
// increment to a value on its own grid every step, a rounding error with a
// fixed sign. Returns true when the trajectory has finished (passage or cap).
template <bool WEIGHTED, bool SMEM, bool NIDX = false, bool DTAB = false>
__device__ __forceinline__ bool em_step(Lane &L, float z, const float4 *__restrict__ tab,
                                        const ModelDev *s_model, const ModelDev &M0)
{
    // noise table: linear interpolation in x (or in time), end values held outside
    float f;
    const float4 e = table_at<SMEM, NIDX>(L, tab, f, M0);
    const float dN = SMEM ? M0.dN : L.dN;
    float S = fmaf(f, e.y, e.x);               // S_phiphi sqrt(dN)
    float T = fmaf(f, e.w, e.z);               // tan(theta_n) S_phiphi sqrt(dN)
    float cb = L.cb, half_cb2 = L.half_cb2;
    if (outside_window<NIDX>(L, L.n)) {
        // outside the noise window the step is classical: no noise, no bias, no weight
        S = 0.0f;
        T = 0.0f;
        cb = 0.0f;
        half_cb2 = 0.0f;
    }
    const float vpv = drift_vpv<DTAB, SMEM>(L, tab, s_model, M0);
    const float hdN = hh_dN<SMEM>(L, M0);               // (pi^2/2 - 3) dN
    const float zb = z + cb;                             // xi + alpha sqrt(dN)
    const float dx = fmaf(S, zb, L.p * dN);             // (pi + alpha S) dN + S xi sqrt(dN)
    if (DTAB) {
        // correlated pi-noise (tan theta_n ~ 0.3): the momentum is a compensated
        // pair, or its rounding performs a random walk that the field integrates
        kahan_add(L.p, L.p_c, fmaf(T, zb, hdN * (L.p + vpv)));
    } else {
        L.p = fmaf(T, zb, fmaf(hdN, L.p + vpv, L.p));
    }
    if (WEIGHTED) L.lw_grp -= fmaf(cb, z, half_cb2);   // the step's ln w increment (see group_lw)
    kahan_add(L.x, L.x_c, dx);
    ++L.n;
    return passed(L) | (L.n >= (SMEM ? M0.max_steps : L.nmax));
}

// ln w increments of the first k + 1 steps of a group that starts at step
// n0, summed as em_step sums them (same operands, same order).
template <bool NIDX>
__device__ __forceinline__ float group_lw(const Lane &L, const float (&z)[4], int n0, int k)
{
    float lw = 0.0f;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (s > k) break;
        const bool off = outside_window<NIDX>(L, n0 + s);
        lw -= fmaf(off ? 0.0f : L.cb, z[s], off ? 0.0f : L.half_cb2);
    }
    return lw;
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Learned proposal at a segment start: alpha from the warp's MLP evaluation
// at the current state; every lane of the warp takes part.
template <bool SMEM, bool REC>
__device__ __forceinline__ void mlp_segment_start(Lane &L, bool live, SegRec &sg, const float4 *tab,
                                                  const uint2 *tiles, const float *bias, const RunDev &pr,
                                                  const ModelDev &M0)
{
    const float dN = SMEM ? M0.dN : L.dN, sqrt_dN = SMEM ? M0.sqrt_dN : L.sqrt_dN;
    float in0 = 0.0f, in1 = 0.0f, in2 = 0.0f, tan_t = 0.0f;
    if (live) {
        const float xv = __fsub_rn(L.x, L.x_c);
        in0 = ((pr.mlp_flags & FPT_MLP_LOG_X) ? __logf(fmaxf(xv, pr.x_floor)) : xv);
        in0 = (in0 - pr.shift[0]) * pr.scale[0];
        in1 = (L.p - pr.shift[1]) * pr.scale[1];
        in2 = ((float)L.n * dN - pr.shift[2]) * pr.scale[2];
        float f;
        const float4 e = table_at<SMEM>(L, tab, f, M0);
        const float S = fmaf(f, e.y, e.x), T = fmaf(f, e.w, e.z);
        tan_t = S > 0.0f ? __fdividef(T, S) : 0.0f;
    }
    float o1, o2;
    mlp_forward_warp(tiles, bias, in0, in1, in2, o1, o2);
    if (live) {
        float raw;
        const float al = mlp_alpha_of(o1, o2, tan_t, pr.alpha_max, raw);
        L.cb = al * sqrt_dN;
        L.half_cb2 = 0.5f * al * al * dN;
        if (REC) {
            sg.in0 = in0; sg.in1 = in1; sg.in2 = in2; sg.tan_t = tan_t; sg.raw = raw;
            sg.sum_xi = 0.0f;
            sg.n0 = L.n;
            sg.open = true;
        }
    }
}

// Learned proposal with one network per run (the runs of a launch may carry
// different networks, input normalisations and clamps; they share the
// segment length): the warp evaluates the network of each run among its live
// lanes in turn -- runs are contiguous in unit order, so a warp mostly holds
// one run -- reading that run's packed weights through L1.
template <bool SMEM, bool REC>
__device__ __forceinline__ void mlp_segment_start_multi(Lane &L, bool live, SegRec &sg, const float4 *tab,
                                                        const RunDev *runs, const ModelDev &M0)
{
    const unsigned FULL = 0xffffffffu;
    const float dN = SMEM ? M0.dN : L.dN, sqrt_dN = SMEM ? M0.sqrt_dN : L.sqrt_dN;
    unsigned pend = __ballot_sync(FULL, live);
    while (pend) {
        const int run = __shfl_sync(FULL, L.run, __ffs(pend) - 1);
        const bool mine = live && L.run == run;
        pend &= ~__ballot_sync(FULL, mine);
        const RunDev &pr = runs[run];
        float in0 = 0.0f, in1 = 0.0f, in2 = 0.0f, tan_t = 0.0f;
        if (mine) {
            const float xv = __fsub_rn(L.x, L.x_c);
            in0 = ((pr.mlp_flags & FPT_MLP_LOG_X) ? __logf(fmaxf(xv, pr.x_floor)) : xv);
            in0 = (in0 - pr.shift[0]) * pr.scale[0];
            in1 = (L.p - pr.shift[1]) * pr.scale[1];
            in2 = ((float)L.n * dN - pr.shift[2]) * pr.scale[2];
            float f;
            const float4 e = table_at<SMEM>(L, tab, f, M0);
            const float S = fmaf(f, e.y, e.x), T = fmaf(f, e.w, e.z);
            tan_t = S > 0.0f ? __fdividef(T, S) : 0.0f;
        }
        const uint2 *tiles = reinterpret_cast<const uint2 *>(pr.mlp);
        const float *bias = reinterpret_cast<const float *>(tiles + kMlpTiles * 32);
        float o1, o2;
        mlp_forward_warp(tiles, bias, in0, in1, in2, o1, o2);
        if (mine) {
            float raw;
            const float al = mlp_alpha_of(o1, o2, tan_t, pr.alpha_max, raw);
            L.cb = al * sqrt_dN;
            L.half_cb2 = 0.5f * al * al * dN;
            if (REC) {
                sg.in0 = in0; sg.in1 = in1; sg.in2 = in2; sg.tan_t = tan_t; sg.raw = raw;
                sg.sum_xi = 0.0f;
                sg.n0 = L.n;
                sg.open = true;
            }
        }
    }
}

// Dynamic shared memory of a stepper launch: the table (SMEM variants), the
// staged proposal blob (single-network learned variants), then the launch's
// run constants and model descriptors, each as many as the launch has.
__device__ __forceinline__ RunSm *smem_runs(float4 *s_dyn, int table_entries, bool staged_blob)
{
    unsigned char *p = reinterpret_cast<unsigned char *>(s_dyn + table_entries);
    return reinterpret_cast<RunSm *>(p + (staged_blob ? kMlpBlobBytes : 0));
}

__device__ __forceinline__ ModelDev *smem_models(RunSm *s_run, int n_runs)
{
    const size_t b = ((sizeof(RunSm) * (size_t)n_runs + 15) / 16) * 16;
    return reinterpret_cast<ModelDev *>(reinterpret_cast<unsigned char *>(s_run) + b);
}

size_t em_smem_bytes(EmVariant v, int table_entries, int n_runs, int n_models)
{
    return sizeof(float4) * (size_t)table_entries + ((v.mlp && !v.mnet) ? (size_t)kMlpBlobBytes : 0) +
           ((sizeof(RunSm) * (size_t)n_runs + 15) / 16) * 16 + sizeof(ModelDev) * (size_t)n_models;
}

// Launch prologue shared by the steppers: clock origin, per-run and per-model
// constants, the table (SMEM variants) and the proposal blob (MLP variants)
// staged in shared memory. `table_entries` float4 entries are staged.
template <bool SMEM, bool MLP>
__device__ __forceinline__ void stage_launch(const EmParams &P, float4 *s_tab, RunSm *s_run,
                                             ModelDev *s_model, unsigned long long &s_t0,
                                             uint2 *s_tiles)
{
    if (P.budget_ns && threadIdx.x == 0) {
        // the launch's clock origin: the first block to start sets it
        const unsigned long long now = globaltimer();
        const unsigned long long prev = atomicCAS(P.t0, 0ull, now);
        s_t0 = prev ? prev : now;
    }
    for (int i = threadIdx.x; i < P.n_runs; i += blockDim.x) {
        const RunDev &r = P.runs[i];
        s_run[i].unit_begin = r.unit_begin;
        s_run[i].traj_offset = r.traj_offset;
        s_run[i].cb = r.cb;
        s_run[i].half_cb2 = r.half_cb2;
        s_run[i].cb_b = r.cb_b;
        s_run[i].run_id = r.run_id;
        s_run[i].model = r.model;
        s_run[i].is_mlp = r.bias_kind == FPT_BIAS_MLP;
        s_run[i].sqrt_dN = r.sqrt_dN;
        s_run[i].dN = r.dN;
    }
    for (int i = threadIdx.x; i < P.n_models; i += blockDim.x) s_model[i] = P.models[i];
    if (SMEM) {
        const float4 *src = P.tables + P.smem_table_offset;
        for (int i = threadIdx.x; i < P.smem_table_points; i += blockDim.x) s_tab[i] = src[i];
    }
    if (MLP) {
        const float4 *src = reinterpret_cast<const float4 *>(P.runs[P.mlp_run].mlp);
        float4 *dst = reinterpret_cast<float4 *>(s_tiles);
        for (int i = threadIdx.x; i < kMlpBlobBytes / 16; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
}

// Refill point: write the warp's finished trajectories and fetch new units
// with one warp-aggregated atomic on the work cursor.
__device__ __forceinline__ void refill_point(const EmParams &P, Lane &L, bool &active, bool &done,
                                             const RunSm *s_run, const ModelDev *s_model)
{
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const bool fin_me = active && done;
    const unsigned fin = __ballot_sync(FULL, fin_me);
    if (!fin) return;
    if (fin_me) {
        const bool pas = passed(L);
        CHECK_INDEX(L.unit, P.total_units, kCheckUnit);
        P.nsteps[L.unit] = L.n;
        P.logw[L.unit] = (double)L.lw_hi - (double)L.lw_lo;     // the pair holds hi - lo
        P.status[L.unit] = pas ? (uint8_t)FPT_TRAJ_PASSED : (uint8_t)FPT_TRAJ_CAPPED;
        if (!pas) atomicAdd(P.flags + 1, 1);
    }
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(P.cursor, (unsigned long long)__popc(fin));
    base = __shfl_sync(FULL, base, 0);
    if (fin_me) {
        const long long unit = (long long)(base + __popc(fin & ((1u << lane) - 1u)));
        done = false;
        active = unit < P.total_units;
        if (active) lane_load(L, unit, s_run, s_model, P.n_runs);
    }
}

// First units of a warp.
__device__ __forceinline__ void first_units(const EmParams &P, Lane &L, bool &active,
                                            const RunSm *s_run, const ModelDev *s_model)
{
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(P.cursor, 32ull);
    base = __shfl_sync(FULL, base, 0);
    const long long unit = (long long)(base + lane);
    active = unit < P.total_units;
    if (active) lane_load(L, unit, s_run, s_model, P.n_runs);
    else L.n = 0, L.traj = 0, L.run_id = 0, L.mlp = false, L.nidx = false, L.run = 0;
}

// Deadline: true when the launch should stop (lane 0 reads the device clock).
__device__ __forceinline__ bool past_deadline(const EmParams &P, unsigned long long t0)
{
    int stop = 0;
    if ((threadIdx.x & 31u) == 0) {
        if (globaltimer() - t0 > P.budget_ns) atomicExch(P.flags, 1);
        stop = *(volatile int *)P.flags;
    }
    return __shfl_sync(0xffffffffu, stop, 0) != 0;
}

// Close the warp's open segments at a refill point: record r holds
// q0 = (inputs, slot 3) and q1 = (slot 4, slot 5, unit, first step of the
// segment), appended with one warp-aggregated atomic on the record cursor;
// records past the buffer raise flag 3 instead of being written.
__device__ __forceinline__ void write_records(const EmParams &P, const Lane &L, SegRec &sg, bool active,
                                              float4 q0, float s4, float s5)
{
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const bool wr = active && sg.open;
    const unsigned m = __ballot_sync(FULL, wr);
    if (m) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(P.rec_cursor, (unsigned long long)__popc(m));
        base = __shfl_sync(FULL, base, 0);
        if (wr) {
            const long long idx = (long long)(base + __popc(m & ((1u << lane) - 1u)));
            if (idx < P.rec_cap) {
                float4 *q = reinterpret_cast<float4 *>(P.records + 8 * idx);
                q[0] = q0;
                q[1] = make_float4(s4, s5, __uint_as_float((uint32_t)L.unit), __int_as_float(sg.n0));
            } else {
                atomicExch(P.flags + 3, 1);
            }
        }
    }
    sg.open = false;
}

// Register budgets: the plain stepper keeps three 512-thread blocks per SM
// (48 warps, 40 registers); the noise-window and bump steppers two 512-thread
// blocks; the learned-proposal steppers at most 384 threads per block and two
// blocks, 80 registers: the network's fragments fit without spilling (a
// 64-register build ran 512-thread blocks but executed ~7% more instructions
// per step, and the autotuner chose 384 threads for it anyway).
template <bool WEIGHTED, bool SMEM, bool MLP, bool REC, bool NIDX, bool DTAB, bool MNET = false>
__global__ void __launch_bounds__(MLP ? kMlpMaxBlock : 512, (MLP || NIDX || DTAB) ? 2 : 3)
    em_kernel(const EmParams P)
{
    extern __shared__ __align__(16) float4 s_tab[];
    __shared__ unsigned long long s_t0;

    // single-network MLP variants: the proposal's fragment blob follows the
    // table in shared memory; then the run constants and model descriptors
    const int tab_entries = SMEM ? P.smem_table_points : 0;
    uint2 *s_tiles = reinterpret_cast<uint2 *>(s_tab + tab_entries);
    float *s_bias = reinterpret_cast<float *>(s_tiles + kMlpTiles * 32);
    RunSm *s_run = smem_runs(s_tab, tab_entries, MLP && !MNET);
    ModelDev *s_model = smem_models(s_run, P.n_runs);
    const RunDev &prun = P.runs[MLP ? P.mlp_run : 0];
    stage_launch<SMEM, MLP && !MNET>(P, s_tab, s_run, s_model, s_t0, s_tiles);

    const float4 *tab = SMEM ? s_tab : P.tables;
    const unsigned FULL = 0xffffffffu;

    Lane L;
    SegRec sg;
    sg.open = false;
    bool active = false, done = false;
    first_units(P, L, active, s_run, s_model);

    for (;;) {
        if (MLP && __any_sync(FULL, active && L.mlp)) {
            if (MNET) mlp_segment_start_multi<SMEM, REC>(L, active && L.mlp, sg, tab, P.runs, P.m0);
            else mlp_segment_start<SMEM, REC>(L, active && L.mlp, sg, tab, s_tiles, s_bias, prun, P.m0);
        }

        // Speculative groups (single-model launches): when every lane of the
        // warp is live and the whole interval stays below the cap, the four steps
        // of a group run without the per-step branch, each lane noting after
        // which steps its field was at or below the end surface. A lane that
        // passed at step k of the group then takes the state the guarded path
        // would have left: k + 1 steps counted, the ln w increments of those
        // steps summed again from the same operands, its field marked passed
        // (the later steps' field and momentum are discarded: the trajectory has
        // ended, and only its step count, weight and status are kept), and the
        // warp's remaining groups of the interval run guarded. Results do not
        // depend on which path ran.
        bool spec = SMEM && __all_sync(FULL, active && !done &&
                                                 L.n + 4 * P.groups_per_check < P.m0.max_steps);
        for (int g = 0; g < P.groups_per_check; ++g) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)L.n >> 2, L.traj, L.run_id, 0u), P.rk);
            float z[4];
            box_muller(r.x, r.y, z[0], z[1]);
            box_muller(r.z, r.w, z[2], z[3]);
            if (spec) {
                const float sx0 = REC ? sg.sum_xi : 0.0f;
                bool h[4];
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    if (REC) sg.sum_xi = __fadd_rn(sg.sum_xi, z[s]);
                    em_step<WEIGHTED, SMEM, NIDX, DTAB>(L, z[s], tab, s_model, P.m0);
                    h[s] = passed(L);
                }
                const bool hit = h[0] | h[1] | h[2] | h[3];
                if (__any_sync(FULL, hit)) spec = false;
                if (hit) {
                    const int k = h[0] ? 0 : h[1] ? 1 : h[2] ? 2 : 3;
                    const int n0 = L.n - 4;
                    // the group's normals again (not kept live through the steps)
                    const uint4 q = philox4x32_10(make_uint4((uint32_t)n0 >> 2, L.traj, L.run_id, 0u), P.rk);
                    float zz[4];
                    box_muller(q.x, q.y, zz[0], zz[1]);
                    box_muller(q.z, q.w, zz[2], zz[3]);
                    L.n = n0 + k + 1;
                    if (WEIGHTED) L.lw_grp = group_lw<NIDX>(L, zz, n0, k);
                    if (REC) {
                        float sx = sx0;
#pragma unroll
                        for (int s = 0; s < 4; ++s)
                            if (s <= k) sx = __fadd_rn(sx, zz[s]);
                        sg.sum_xi = sx;
                    }
                    L.x = -1.0f;
                    L.x_c = 0.0f;
                    done = true;
                }
            } else {
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    if (active && !done) {
                        if (REC) sg.sum_xi = __fadd_rn(sg.sum_xi, z[s]);
                        done = em_step<WEIGHTED, SMEM, NIDX, DTAB>(L, z[s], tab, s_model, P.m0);
                    }
            }
            // the group's weight increments (at most 4, so a plain FP32 sum) into the
            // pair; a lane that took no step in the group adds nothing (re-adding zero
            // would re-round the pair, and how often depends on the launch shape)
            if (WEIGHTED && L.lw_grp != 0.0f) {
                kahan_add(L.lw_hi, L.lw_lo, L.lw_grp);
                L.lw_grp = 0.0f;
            }
        }

        if (REC) {
            // close the segments of this interval: (inputs, tan, raw alpha, sum xi, unit, steps)
            write_records(P, L, sg, active, make_float4(sg.in0, sg.in1, sg.in2, sg.tan_t), sg.raw, sg.sum_xi);
        }

        // refill point: write finished trajectories, fetch new work
        refill_point(P, L, active, done, s_run, s_model);
        if (!__any_sync(FULL, active)) break;
        // trajectories in flight keep the ABORTED status set before launch
        if (P.budget_ns && past_deadline(P, s_t0)) break;
    }
}

// ---------------------------------------------------------------------------
// K1b: full-rank (2-D) noise stepper
// ---------------------------------------------------------------------------
// Euler-Maruyama of Eq. (2.24) with the symmetric noise matrix S = sqrt(Xi)
// (Eq. 3.9): two normals per step, step n using normals 2(n & 1), 2(n & 1) + 1
// of Philox block n >> 1. Bias in standardised form B = S beta, so that
// Eq. (4.5) reduces to dA = beta . (beta dN/2 + xi sqrt(dN)) (S^T Xi^-1 S = 1).
// Table: M + 1 float4 entries (S_phiphi, S_phipi, S_pipi, 0) sqrt(dN) at the
// grid points, entry M repeating entry M - 1; linear interpolation reads
// entries k and k + 1.
template <bool SMEM>
__device__ __forceinline__ void table2_at(const Lane &L, const float4 *__restrict__ tab, float &a,
                                          float &b, float &c, const ModelDev &M0)
{
    const float kMagic = 12582912.0f;                        // 1.5 * 2^23
    float u = fmaf(L.x, SMEM ? M0.u_scale : L.u_scale, SMEM ? M0.u_shift : L.u_shift);
    u = fminf(fmaxf(u, 0.0f), SMEM ? M0.u_umax : L.u_max);
    const float t = (u - 0.5f) + kMagic;
    int i = __float_as_int(t) - 0x4b400000;
    const float f = u - (t - kMagic);
    CHECK_INDEX(i, SMEM ? M0.M : L.M, kCheckTable);          // entries i, i + 1 of M + 1
    const float4 e0 = SMEM ? tab[i] : __ldg(tab + L.tbase + i);
    const float4 e1 = SMEM ? tab[i + 1] : __ldg(tab + L.tbase + i + 1);
    a = fmaf(f, e1.x - e0.x, e0.x);
    b = fmaf(f, e1.y - e0.y, e0.y);
    c = fmaf(f, e1.z - e0.z, e0.z);
}

template <bool WEIGHTED, bool SMEM, bool DTAB>
__device__ __forceinline__ bool em2_step(Lane &L, float z1, float z2, const float4 *__restrict__ tab,
                                         const ModelDev *s_model, const ModelDev &M0)
{
    float a, b, c;                                       // S sqrt(dN), interpolated in x
    table2_at<SMEM>(L, tab, a, b, c, M0);
    const float vpv = drift_vpv<DTAB, SMEM>(L, tab, s_model, M0);
    const float dN = SMEM ? M0.dN : L.dN;
    const float hdN = hh_dN<SMEM>(L, M0);               // (pi^2/2 - 3) dN
    const float e1 = z1 + L.cb, e2 = z2 + L.cb_b;       // xi + beta sqrt(dN)
    // (phi, pi) += D dN + S beta dN + S xi sqrt(dN) = D dN + (S sqrt(dN)) e
    const float dx = fmaf(a, e1, fmaf(b, e2, L.p * dN));
    // full-rank noise drives pi directly: compensated momentum (see em_step)
    kahan_add(L.p, L.p_c, fmaf(b, e1, fmaf(c, e2, hdN * (L.p + vpv))));
    if (WEIGHTED) L.lw_grp -= fmaf(L.cb, z1, fmaf(L.cb_b, z2, L.half_cb2));
    kahan_add(L.x, L.x_c, dx);
    ++L.n;
    return passed(L) | (L.n >= (SMEM ? M0.max_steps : L.nmax));
}

// Learned proposal in 2-D: beta = (clamp(o1), clamp(o2)) at the segment start.
template <bool SMEM, bool REC>
__device__ __forceinline__ void mlp2_segment_start(Lane &L, bool live, SegRec &sg, const uint2 *tiles,
                                                   const float *bias, const RunDev &pr, const ModelDev &M0)
{
    const float dN = SMEM ? M0.dN : L.dN, sqrt_dN = SMEM ? M0.sqrt_dN : L.sqrt_dN;
    float in0 = 0.0f, in1 = 0.0f, in2 = 0.0f;
    if (live) {
        const float xv = __fsub_rn(L.x, L.x_c);
        in0 = ((pr.mlp_flags & FPT_MLP_LOG_X) ? __logf(fmaxf(xv, pr.x_floor)) : xv);
        in0 = (in0 - pr.shift[0]) * pr.scale[0];
        in1 = (L.p - pr.shift[1]) * pr.scale[1];
        in2 = ((float)L.n * dN - pr.shift[2]) * pr.scale[2];
    }
    float o1, o2;
    mlp_forward_warp(tiles, bias, in0, in1, in2, o1, o2);
    if (live) {
        const float b1 = fminf(fmaxf(o1, -pr.alpha_max), pr.alpha_max);
        const float b2 = fminf(fmaxf(o2, -pr.alpha_max), pr.alpha_max);
        L.cb = b1 * sqrt_dN;
        L.cb_b = b2 * sqrt_dN;
        L.half_cb2 = 0.5f * fmaf(b1, b1, b2 * b2) * dN;
        if (REC) {
            sg.in0 = in0; sg.in1 = in1; sg.in2 = in2;
            sg.sum_xi = 0.0f;
            sg.sum_xi2 = 0.0f;
            sg.n0 = L.n;
            sg.open = true;
        }
    }
}

template <bool WEIGHTED, bool SMEM, bool MLP, bool DTAB, bool REC = false>
__global__ void __launch_bounds__(MLP ? kMlpMaxBlock : 512, 2) em2_kernel(const EmParams P)
{
    extern __shared__ __align__(16) float4 s_tab[];
    __shared__ unsigned long long s_t0;

    const int tab_entries = SMEM ? P.smem_table_points : 0;
    uint2 *s_tiles = reinterpret_cast<uint2 *>(s_tab + tab_entries);
    float *s_bias = reinterpret_cast<float *>(s_tiles + kMlpTiles * 32);
    RunSm *s_run = smem_runs(s_tab, tab_entries, MLP);
    ModelDev *s_model = smem_models(s_run, P.n_runs);
    const RunDev &prun = P.runs[MLP ? P.mlp_run : 0];
    stage_launch<SMEM, MLP>(P, s_tab, s_run, s_model, s_t0, s_tiles);

    const float4 *tab = SMEM ? s_tab : P.tables;
    const unsigned FULL = 0xffffffffu;
    Lane L;
    SegRec sg;
    sg.open = false;
    bool active = false, done = false;
    first_units(P, L, active, s_run, s_model);

    for (;;) {
        if (MLP && __any_sync(FULL, active && L.mlp))
            mlp2_segment_start<SMEM, REC>(L, active && L.mlp, sg, s_tiles, s_bias, prun, P.m0);

        // speculative groups as in em_kernel, the precondition checked once per interval
        bool spec = SMEM && __all_sync(FULL, active && !done &&
                                                 L.n + 4 * P.groups_per_check < P.m0.max_steps);
        for (int g = 0; g < P.groups_per_check; ++g) {
            // four steps per group, two per Philox block: L.n is even at each block
            // (a lane that finished keeps its count and ignores the normals).
            // Speculative group as in em_kernel: when every lane is live and the
            // interval stays below the cap, the steps run without the per-step
            // branch and a lane that passed at step k of the group is set back to
            // the guarded path's state (k + 1 steps, the weight and noise sums of
            // those steps formed again from the same normals, field marked passed).
            if (spec) {
                const float sx0 = REC ? sg.sum_xi : 0.0f, sy0 = REC ? sg.sum_xi2 : 0.0f;
                bool hit[4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint4 r = philox4x32_10(make_uint4((uint32_t)L.n >> 1, L.traj, L.run_id, 0u), P.rk);
                    float z[4];
                    box_muller(r.x, r.y, z[0], z[1]);
                    box_muller(r.z, r.w, z[2], z[3]);
                    if (REC) { sg.sum_xi = __fadd_rn(sg.sum_xi, z[0]); sg.sum_xi2 = __fadd_rn(sg.sum_xi2, z[1]); }
                    em2_step<WEIGHTED, SMEM, DTAB>(L, z[0], z[1], tab, s_model, P.m0);
                    hit[2 * h] = passed(L);
                    if (REC) { sg.sum_xi = __fadd_rn(sg.sum_xi, z[2]); sg.sum_xi2 = __fadd_rn(sg.sum_xi2, z[3]); }
                    em2_step<WEIGHTED, SMEM, DTAB>(L, z[2], z[3], tab, s_model, P.m0);
                    hit[2 * h + 1] = passed(L);
                }
                const bool any_hit = hit[0] | hit[1] | hit[2] | hit[3];
                if (__any_sync(FULL, any_hit)) spec = false;
                if (any_hit) {
                    const int k = hit[0] ? 0 : hit[1] ? 1 : hit[2] ? 2 : 3;
                    const int n0 = L.n - 4;
                    float zz[8];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint4 r = philox4x32_10(make_uint4(((uint32_t)n0 >> 1) + h, L.traj, L.run_id, 0u),
                                                      P.rk);
                        box_muller(r.x, r.y, zz[4 * h], zz[4 * h + 1]);
                        box_muller(r.z, r.w, zz[4 * h + 2], zz[4 * h + 3]);
                    }
                    float lw = 0.0f, sx = sx0, sy = sy0;
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        if (s > k) break;
                        lw -= fmaf(L.cb, zz[2 * s], fmaf(L.cb_b, zz[2 * s + 1], L.half_cb2));   // as em2_step
                        sx = __fadd_rn(sx, zz[2 * s]);
                        sy = __fadd_rn(sy, zz[2 * s + 1]);
                    }
                    L.n = n0 + k + 1;
                    if (WEIGHTED) L.lw_grp = lw;
                    if (REC) { sg.sum_xi = sx; sg.sum_xi2 = sy; }
                    L.x = -1.0f;
                    L.x_c = 0.0f;
                    done = true;
                }
            } else {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint4 r = philox4x32_10(make_uint4((uint32_t)L.n >> 1, L.traj, L.run_id, 0u), P.rk);
                    float z[4];
                    box_muller(r.x, r.y, z[0], z[1]);
                    box_muller(r.z, r.w, z[2], z[3]);
                    if (active && !done) {
                        if (REC) { sg.sum_xi = __fadd_rn(sg.sum_xi, z[0]); sg.sum_xi2 = __fadd_rn(sg.sum_xi2, z[1]); }
                        done = em2_step<WEIGHTED, SMEM, DTAB>(L, z[0], z[1], tab, s_model, P.m0);
                    }
                    if (active && !done) {
                        if (REC) { sg.sum_xi = __fadd_rn(sg.sum_xi, z[2]); sg.sum_xi2 = __fadd_rn(sg.sum_xi2, z[3]); }
                        done = em2_step<WEIGHTED, SMEM, DTAB>(L, z[2], z[3], tab, s_model, P.m0);
                    }
                }
            }
            if (WEIGHTED && L.lw_grp != 0.0f) {
                kahan_add(L.lw_hi, L.lw_lo, L.lw_grp);
                L.lw_grp = 0.0f;
            }
        }
        // 2-D records: (inputs, sum xi_2), (0, sum xi_1, unit, steps)
        if (REC) write_records(P, L, sg, active, make_float4(sg.in0, sg.in1, sg.in2, sg.sum_xi2), 0.0f, sg.sum_xi);
        refill_point(P, L, active, done, s_run, s_model);
        if (!__any_sync(FULL, active)) break;
        if (P.budget_ns && past_deadline(P, s_t0)) break;
    }
}

template <bool DTAB>
static const void *em_fn_t(EmVariant v)
{
    if (v.rank2) {
        if (v.rec) return v.smem ? (const void *)em2_kernel<true, true, true, DTAB, true>
                                 : (const void *)em2_kernel<true, false, true, DTAB, true>;
        if (v.mlp) return v.smem ? (const void *)em2_kernel<true, true, true, DTAB>
                                 : (const void *)em2_kernel<true, false, true, DTAB>;
        if (v.weighted) return v.smem ? (const void *)em2_kernel<true, true, false, DTAB>
                                      : (const void *)em2_kernel<true, false, false, DTAB>;
        return v.smem ? (const void *)em2_kernel<false, true, false, DTAB>
                      : (const void *)em2_kernel<false, false, false, DTAB>;
    }
    if (v.rec) return v.smem ? (const void *)em_kernel<true, true, true, true, false, DTAB>
                             : (const void *)em_kernel<true, false, true, true, false, DTAB>;
    if (v.mlp) return v.smem ? (const void *)em_kernel<true, true, true, false, false, DTAB>
                             : (const void *)em_kernel<true, false, true, false, false, DTAB>;
    if (v.weighted) return v.smem ? (const void *)em_kernel<true, true, false, false, false, DTAB>
                                  : (const void *)em_kernel<true, false, false, false, false, DTAB>;
    return v.smem ? (const void *)em_kernel<false, true, false, false, false, DTAB>
                  : (const void *)em_kernel<false, false, false, false, false, DTAB>;
}

static const void *em_fn(EmVariant v)
{
    if (v.mnet) {   // one network per run: 1-D, phi-indexed tables
        if (v.rec) return v.smem ? (const void *)em_kernel<true, true, true, true, false, false, true>
                                 : (const void *)em_kernel<true, false, true, true, false, false, true>;
        return v.smem ? (const void *)em_kernel<true, true, true, false, false, false, true>
                      : (const void *)em_kernel<true, false, true, false, false, false, true>;
    }
    if (v.dtab) return em_fn_t<true>(v);
    if (v.nidx && !v.rank2 && !v.mlp) {
        if (v.weighted) return v.smem ? (const void *)em_kernel<true, true, false, false, true, false>
                                      : (const void *)em_kernel<true, false, false, false, true, false>;
        return v.smem ? (const void *)em_kernel<false, true, false, false, true, false>
                      : (const void *)em_kernel<false, false, false, false, true, false>;
    }
    return em_fn_t<false>(v);
}

// Opt in to the dynamic shared memory the table (and proposal) need, outside
// any stream capture, then report resident blocks per SM for this shape.
int em_occupancy(EmVariant v, int block, size_t smem_bytes)
{
    const void *f = em_fn(v);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, block, smem_bytes) != cudaSuccess) return 0;
    return nb;
}

// Launch only (safe inside stream capture): em_occupancy() must have been
// called for this shape first.
cudaError_t em_launch(const EmParams &p, EmVariant v, int grid, int block, size_t smem_bytes, cudaStream_t s)
{
    void *args[] = {const_cast<EmParams *>(&p)};
    return cudaLaunchKernel(em_fn(v), dim3(grid), dim3(block), args, smem_bytes, s);
}

// ---------------------------------------------------------------------------
// K2: weighted histogram
// ---------------------------------------------------------------------------
// Order-preserving map of doubles onto unsigned 64-bit keys (0 = empty).
__device__ __forceinline__ unsigned long long dkey(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k)
{
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// Bin of a passed trajectory: q = (n dN - N_lo)/db in IEEE double without
// contraction, the same operations as the FP64 definition.
__device__ __forceinline__ double bin_coord(int32_t n, double dN, double N_lo, double db, double &N)
{
    N = __dmul_rn((double)n, dN);
    return __ddiv_rn(__dsub_rn(N, N_lo), db);
}

// Jackknife block g covers trajectories [ceil(g n / G), ceil((g+1) n / G)).
__device__ __forceinline__ long long jk_begin(long long g, long long n)
{
    return (g * n + kJackknife - 1) / kJackknife;
}

__global__ void hist_max_kernel(const HistParams P)
{
    extern __shared__ unsigned long long s_max[];
    const int nb = P.n_bins;
    for (int i = threadIdx.x; i < nb + 2; i += blockDim.x) s_max[i] = 0ull;
    __syncthreads();
    const bool has_tail = !isnan(P.N_tail);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P.n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long u = P.unit_begin + i;
        if (P.status[u] != FPT_TRAJ_PASSED) continue;
        const double lw = P.logw[u];
        double N;
        const double q = bin_coord(P.nsteps[u], P.dN, P.N_lo, P.db, N);
        const unsigned long long k = dkey(lw);
        if (q >= 0.0 && q < (double)nb) {
            int b = (int)floor(q);
            CHECK_INDEX(b, nb, kCheckBin);
            atomicMax(&s_max[b], k);
        }
        atomicMax(&s_max[nb], k);
        if (has_tail && N >= P.N_tail) atomicMax(&s_max[nb + 1], k);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb + 2; i += blockDim.x)
        if (s_max[i]) atomicMax(&P.maxkey[i], s_max[i]);
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) t += red[i];
    return t;  // valid in thread 0
}

// grid = (chunks, kJackknife): CTA (c, g) bins trajectories of jackknife
// block g, chunk c.
__global__ void hist_sum_kernel(const HistParams P)
{
    extern __shared__ double s_dyn[];
    __shared__ double s_red[32];
    const int nb = P.n_bins;
    double *s_mom = s_dyn;                         // [nb][4]: S1, S2, Slw, Slw2
    double *s_M = s_dyn + 4 * nb;                  // [nb] per-bin max ln w
    unsigned *s_cnt = (unsigned *)(s_dyn + 5 * nb);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        s_mom[4 * i] = s_mom[4 * i + 1] = s_mom[4 * i + 2] = s_mom[4 * i + 3] = 0.0;
        s_cnt[i] = 0u;
        s_M[i] = P.maxkey[i] ? dkey_inv(P.maxkey[i]) : 0.0;
    }
    __syncthreads();
    const double Mg = P.maxkey[nb] ? dkey_inv(P.maxkey[nb]) : 0.0;
    const double MT = P.maxkey[nb + 1] ? dkey_inv(P.maxkey[nb + 1]) : 0.0;
    const bool has_tail = !isnan(P.N_tail);

    const long long g = blockIdx.y;
    const long long b0 = jk_begin(g, P.n), b1 = jk_begin(g + 1, P.n);
    const long long c0 = b0 + (long long)blockIdx.x * P.chunk;
    const long long c1 = min(b1, c0 + (long long)P.chunk);

    double sc[kScCount];
#pragma unroll
    for (int k = 0; k < kScCount; ++k) sc[k] = 0.0;
    for (long long i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        const long long u = P.unit_begin + i;
        sc[kScN] += 1.0;
        const uint8_t st = P.status[u];
        if (st == FPT_TRAJ_CAPPED) { sc[kScCapped] += 1.0; continue; }
        if (st != FPT_TRAJ_PASSED) continue;
        const double lw = P.logw[u];
        double N;
        const double q = bin_coord(P.nsteps[u], P.dN, P.N_lo, P.db, N);
        sc[kScPassed] += 1.0;
        sc[kScSumN] += N;
        const double wg = exp(lw - Mg);
        sc[kScSumW] += wg;
        sc[kScSumWN] += wg * N;
        if (has_tail && N >= P.N_tail) {
            const double wt = exp(lw - MT);
            sc[kScTailW] += wt;
            sc[kScTailW2] += wt * wt;
            sc[kScTailN] += 1.0;
        }
        if (q < 0.0) { sc[kScUnder] += 1.0; continue; }
        if (!(q < (double)nb)) { sc[kScOver] += 1.0; continue; }
        int b = (int)floor(q);
        CHECK_INDEX(b, nb, kCheckBin);
        const double e = exp(lw - s_M[b]);
        atomicAdd(&s_cnt[b], 1u);
        atomicAdd(&s_mom[4 * b], e);
        atomicAdd(&s_mom[4 * b + 1], e * e);
        atomicAdd(&s_mom[4 * b + 2], lw);
        atomicAdd(&s_mom[4 * b + 3], lw * lw);
    }
    for (int k = 0; k < kScCount; ++k) {
        const double t = block_sum(sc[k], s_red);
        if (threadIdx.x == 0 && t != 0.0) atomicAdd(&P.scal[g * 16 + k], t);
    }
    __syncthreads();
    double *gm = P.mom + (size_t)g * nb * 5;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        if (!s_cnt[i]) continue;
        atomicAdd(&gm[5 * i], (double)s_cnt[i]);
        atomicAdd(&gm[5 * i + 1], s_mom[4 * i]);
        atomicAdd(&gm[5 * i + 2], s_mom[4 * i + 1]);
        atomicAdd(&gm[5 * i + 3], s_mom[4 * i + 2]);
        atomicAdd(&gm[5 * i + 4], s_mom[4 * i + 3]);
    }
}

// Output layout (doubles): 10 arrays of n_bins (count, log_sum_w, log_sum_w2,
// sum_lw, sum_lw2, pdf, se_w, pdf_ln, se_ln, se_jk) then 16 scalars.
__global__ void __launch_bounds__(128) hist_finalize_kernel(const HistParams P, double *out)
{
    const int nb = P.n_bins;
    const double n = (double)P.n;
    const double ninf = -INFINITY;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        double cnt = 0, S1 = 0, S2 = 0, Slw = 0, Slw2 = 0;
        for (int g = 0; g < kJackknife; ++g) {
            const double *m = P.mom + ((size_t)g * nb + b) * 5;
            cnt += m[0]; S1 += m[1]; S2 += m[2]; Slw += m[3]; Slw2 += m[4];
        }
        const double M = P.maxkey[b] ? dkey_inv(P.maxkey[b]) : 0.0;
        const bool any = cnt > 0;
        const double lsw = any ? M + log(S1) : ninf;
        const double lsw2 = any ? 2.0 * M + log(S2) : ninf;
        out[0 * nb + b] = cnt;
        out[1 * nb + b] = lsw;
        out[2 * nb + b] = lsw2;
        out[3 * nb + b] = Slw;
        out[4 * nb + b] = Slw2;
        // weighted estimator and its error
        out[5 * nb + b] = any ? exp(lsw - log(n * P.db)) : 0.0;
        const double var = fmax(S2 - S1 * S1 / n, 0.0) / ((n - 1.0) * n);
        out[6 * nb + b] = any ? exp(M) * sqrt(var) / P.db : 0.0;
        // lognormal-mean estimator (n_b >= 2)
        double pl = NAN, sl = NAN;
        if (cnt >= 2.0) {
            const double m = Slw / cnt;
            const double s2 = fmax((Slw2 - cnt * m * m) / (cnt - 1.0), 0.0);
            pl = (cnt / n) * exp(m + 0.5 * s2) / P.db;
            const double cox = sqrt(s2 / cnt + s2 * s2 / (2.0 * (cnt - 1.0)));
            const double binom = sqrt(fmax(1.0 - cnt / n, 0.0) / cnt);
            sl = pl * sqrt(cox * cox + binom * binom);
        }
        out[7 * nb + b] = pl;
        out[8 * nb + b] = sl;
        // delete-one-block jackknife of the weighted estimator
        double q[kJackknife], qm = 0.0;
        for (int g = 0; g < kJackknife; ++g) {
            const double ng = (double)(jk_begin(g + 1, P.n) - jk_begin(g, P.n));
            const double *m = P.mom + ((size_t)g * nb + b) * 5;
            q[g] = (S1 - m[1]) / (n - ng);
            qm += q[g];
        }
        qm /= kJackknife;
        double ss = 0.0;
        for (int g = 0; g < kJackknife; ++g) ss += (q[g] - qm) * (q[g] - qm);
        out[9 * nb + b] = any ? exp(M) * sqrt((kJackknife - 1.0) / kJackknife * ss) / P.db : 0.0;
    }
    if (threadIdx.x == 0) {
        double s[kScCount];
        for (int k = 0; k < kScCount; ++k) {
            s[k] = 0.0;
            for (int g = 0; g < kJackknife; ++g) s[k] += P.scal[g * 16 + k];
        }
        const double Mg = P.maxkey[nb] ? dkey_inv(P.maxkey[nb]) : -INFINITY;
        const double MT = P.maxkey[nb + 1] ? dkey_inv(P.maxkey[nb + 1]) : 0.0;
        double *o = out + 10 * nb;
        o[0] = s[kScN];
        o[1] = s[kScPassed];
        o[2] = s[kScUnder];
        o[3] = s[kScOver];
        o[4] = s[kScCapped];
        o[5] = s[kScTailN];
        o[6] = s[kScPassed] > 0 ? s[kScSumN] / s[kScPassed] : NAN;
        o[7] = s[kScSumW] > 0 ? s[kScSumWN] / s[kScSumW] : NAN;
        o[8] = s[kScTailW2] > 0 ? s[kScTailW] * s[kScTailW] / s[kScTailW2] : 0.0;
        o[9] = s[kScTailW] > 0 ? exp(MT + log(s[kScTailW]) - log(n)) : 0.0;
        o[10] = Mg;
        for (int k = 11; k < 16; ++k) o[k] = 0.0;     // reserved
    }
}

cudaError_t hist_launch(const HistParams &p, double *out, cudaStream_t s)
{
    const int nb = p.n_bins;
    cudaError_t e;
    if ((e = cudaMemsetAsync(p.maxkey, 0, sizeof(unsigned long long) * (nb + 2), s))) return e;
    if ((e = cudaMemsetAsync(p.mom, 0, sizeof(double) * (size_t)kJackknife * nb * 5, s))) return e;
    if ((e = cudaMemsetAsync(p.scal, 0, sizeof(double) * kJackknife * 16, s))) return e;
    const size_t smax = sizeof(unsigned long long) * (nb + 2);
    const int grid1 = (int)min(4096LL, max(1LL, (p.n + 255) / 256));
    if ((e = cudaFuncSetAttribute(hist_max_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax))) return e;
    hist_max_kernel<<<grid1, 256, smax, s>>>(p);
    if ((e = cudaGetLastError())) return e;
    const size_t ssum = sizeof(double) * 5 * nb + sizeof(unsigned) * nb;
    if ((e = cudaFuncSetAttribute(hist_sum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssum))) return e;
    const long long per_block = (p.n + kJackknife - 1) / kJackknife;
    const int chunks = (int)max(1LL, (per_block + p.chunk - 1) / p.chunk);
    hist_sum_kernel<<<dim3(chunks, kJackknife), 256, ssum, s>>>(p);
    if ((e = cudaGetLastError())) return e;
    hist_finalize_kernel<<<1, 128, 0, s>>>(p, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Histogram without allocation: the scratch lives in a file-scope device array
// ---------------------------------------------------------------------------
// Layout of the array: per-bin maxima (n_bins + 2 keys), then the jackknife
// moments (kJackknife x n_bins x 5 doubles), then the scalars (kJackknife x 16).
constexpr size_t kNoAllocKeyBytes = ((sizeof(unsigned long long) * (kNoAllocMaxBins + 2) + 255) / 256) * 256;
constexpr size_t kNoAllocMomBytes = sizeof(double) * (size_t)kJackknife * kNoAllocMaxBins * 5;
constexpr size_t kNoAllocScalBytes = sizeof(double) * kJackknife * 16;
constexpr size_t kNoAllocBytes = kNoAllocKeyBytes + kNoAllocMomBytes + kNoAllocScalBytes;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_hist_scratch[kNoAllocBytes];

size_t hist_noalloc_scratch_bytes() { return kNoAllocBytes; }

// Device address of the array. A device address is valid only in the context
// it was looked up in, so the cache is keyed by the id of the calling thread's
// current context (cuCtxGetId: unique for the life of the process, so a
// context created after cudaDeviceReset, or a non-primary context pushed by
// another library, looks the address up again). The first call in a context
// does the lookup; host code must not use the symbol itself as an address.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
struct NoAllocEntry {
    unsigned long long ctx_id;
    unsigned char *ptr;
};
static std::mutex g_noalloc_mu;
static NoAllocEntry g_noalloc_cache[64];
static int g_noalloc_n = 0;
static CtxGetCurrentFn g_ctx_get_current = nullptr;
static CtxGetIdFn g_ctx_get_id = nullptr;

// Id of the current context; 0 when no context is current.
static cudaError_t current_ctx_id(unsigned long long *id)
{
    *id = 0;
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorNotSupported;
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext c = nullptr;
    if (g_ctx_get_current(&c) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
    if (!c) return cudaSuccess;
    if (g_ctx_get_id(c, id) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
    return cudaSuccess;
}

static cudaError_t noalloc_scratch(unsigned char **out)
{
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    unsigned long long id = 0;
    cudaError_t e = current_ctx_id(&id);
    if (e != cudaSuccess) return e;
    for (int i = 0; id && i < g_noalloc_n; ++i)
        if (g_noalloc_cache[i].ctx_id == id) {
            *out = g_noalloc_cache[i].ptr;
            return cudaSuccess;
        }
    // no cached address for this context: look it up (with no context
    // current, this initialises the current device's primary context first)
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_hist_scratch);
    if (e != cudaSuccess) return e;
    if (!id && (e = current_ctx_id(&id)) != cudaSuccess) return e;
    if (id && g_noalloc_n < 64) g_noalloc_cache[g_noalloc_n++] = NoAllocEntry{id, static_cast<unsigned char *>(p)};
    *out = static_cast<unsigned char *>(p);
    return cudaSuccess;
}

cudaError_t hist_noalloc_launch(HistParams p, double *out, cudaStream_t s)
{
    if (p.n_bins < 1 || p.n_bins > kNoAllocMaxBins) return cudaErrorInvalidValue;
    unsigned char *base = nullptr;
    cudaError_t e = noalloc_scratch(&base);
    if (e != cudaSuccess) return e;
    p.maxkey = reinterpret_cast<unsigned long long *>(base);
    p.mom = reinterpret_cast<double *>(base + kNoAllocKeyBytes);
    p.scal = reinterpret_cast<double *>(base + kNoAllocKeyBytes + kNoAllocMomBytes);
    // hist_launch clears the maxima, moments and scalars before it bins
    return hist_launch(p, out, s);
}

__global__ void n_of_steps_kernel(const int32_t *nsteps, long long n, double dN, double *N)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        N[i] = __dmul_rn((double)nsteps[i], dN);
}

cudaError_t n_of_steps_launch(const int32_t *nsteps, long long n, double dN, double *N,
                              cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int grid = (int)min(4096LL, (n + 255) / 256);
    n_of_steps_kernel<<<grid, 256, 0, s>>>(nsteps, n, dN, N);
    return cudaGetLastError();
}

}  // namespace fpt_dev
