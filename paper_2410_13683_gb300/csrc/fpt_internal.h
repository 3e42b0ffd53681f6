// fpt_internal.h -- declarations shared by the C ABI (fpt_abi.cu), the
// kernels (fpt_kernels.cu) and the host table builder (fpt_tables.cpp).
// Not part of the public interface.
#pragma once

#include "fpt.h"

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace fpt_host {
std::string validate_model(const fpt_model &m);
fpt_model_info resolve(const fpt_model &m);
void build_table(const fpt_model &m, int kind, int n_points, double sigma, double phi_lo,
                 double phi_hi, std::vector<double> &S, std::vector<double> &Spi,
                 double &lo_out, double &h_out);
void build_table2(const fpt_model &m, int kind, int n_points, double sigma, double phi_lo,
                  double phi_hi, std::vector<double> &Spp, std::vector<double> &Spq,
                  std::vector<double> &Sqq, double &lo_out, double &h_out);
void power_spectrum(const fpt_model &m, double sigma, int n, const double *Ns, double N_eval, double *out);
void classical_dn(const fpt_model &m, double sigma, int n_k, double N_eval, double &s2,
                  double &eps2_in, double &eps2_end, double &N_in, double &N_end);
double dlnV(const fpt_model &m, double phi, int branch);
double d2V_over_V(const fpt_model &m, double phi);
double Vof(const fpt_model &m, double phi, int branch);
double hubble(const fpt_model &m, double phi, double pi, int branch);
}  // namespace fpt_host

namespace fpt_dev {

constexpr int kMaxRuns = 128;
constexpr int kMaxModels = 64;
constexpr int kMaxTablePoints = 8192;
constexpr int kJackknife = 32;       // jackknife blocks of the histogram
constexpr int kMaxBins = 4096;
constexpr int kNoAllocMaxBins = 1024;   // fpt_histogram_noalloc
constexpr int kMlpHidden = 64;
constexpr int kMlpMaxBlock = 384;       // block-size cap of the learned-proposal steppers

// Flag words of a stepper launch (64 bytes of device memory, zeroed before
// the launch; the first kFlagWords ints are read back after it).
constexpr int kFlagAbort = 0;        // the deadline passed
constexpr int kFlagCapped = 1;       // trajectories that hit max_steps
constexpr int kFlagRecOverflow = 3;  // segment records past the record buffer
constexpr int kFlagChecks = 4;       // FPT_CHECKS builds: failed bounds checks (kCheck* bits)
constexpr int kFlagWords = 5;
constexpr int kFlagT0 = 8;           // ints 8-9: the launch's clock origin (64-bit)

// Bits of the FPT_CHECKS error word.
constexpr int kCheckTable = 1;       // noise-table entry index
constexpr int kCheckDriftTable = 2;  // drift-table entry index
constexpr int kCheckUnit = 4;        // trajectory (output) index from the work cursor
constexpr int kCheckBin = 8;         // histogram bin


// Model constants in the shifted coordinate x = phi - phi_end (FP32).
struct ModelDev {
    float x_star;              // phi_star - phi_end (FP32 head)
    float x_star_lo;           // phi_star - phi_end - x_star (FP32 tail)
    float inv_a_plus, inv_a_minus;   // V'/V = 1 / (1/a + c (x - x_star)), side by sign
    float drift_c;             // 1: piecewise linear (relative slopes); 0: exponential (V'/V = mu)
    float x_in, pi_in;
    float u_scale, u_shift;    // table coordinate u = x * u_scale + u_shift (1-D tables: minus 1/2)
    float u_umax;              // upper clamp of u: M - 3/2 (1-D tables), M - 1 (2-D tables)
    float dN;
    float sqrt_dN;
    int32_t M;                 // table points
    int32_t max_steps;
    int32_t table_offset;      // first float4 entry of this model's table
    int32_t nidx;              // 1: table indexed by the step count (noise window)
    int32_t rank2;             // 1: full-rank 2-D noise table (M + 1 entries)
    // Gaussian bump: cubic V'/V table after the noise entries (dtab >= 0) and
    // the closed form's constants for fields above it
    int32_t dtab;              // first drift entry, relative to the model's table; -1: none
    float d_scale;             // drift-table coordinate u = x * d_scale
    float d_umax;              // intervals of the drift table
    float bump_m2, bump_phi_end, bump_dphi0, bump_inv_w2, bump_K;
    int32_t win_lo, win_hi;    // noise window [win_lo, win_hi] in steps (nidx)
    float half_dN, m3dN;       // 0.5 dN and -3 dN in FP32 (momentum drift)
};

// One run of a launch (FP32 constants; 64-bit unit bookkeeping).
struct RunDev {
    int32_t model;
    int32_t bias_kind;
    float cb;                  // A sqrt(dN) (2-D noise: beta_1 sqrt(dN))
    float half_cb2;            // A^2 dN / 2 (2-D noise: |beta|^2 dN / 2)
    float cb_b;                // 2-D noise: beta_2 sqrt(dN)
    long long n_traj;
    long long traj_offset;
    long long unit_begin;      // first launch unit of this run
    uint32_t run_id;
    int32_t segment;           // MLP: steps per alpha
    const void *mlp;           // MLP: packed bf16 weights (device)
    float shift[3], scale[3];
    float alpha_max;
    float sqrt_dN;
    float dN;
    int32_t mlp_flags;
    float x_floor;             // MLP with log-field input: floor of x under the log
};

struct EmParams {
    const ModelDev *models;
    const RunDev *runs;
    int n_models;
    int n_runs;
    const float4 *tables;      // packed (S', dS', T', dT') entries, S' = S sqrt(dN)
    // the launch's model when all runs share one (SMEM variants): the steppers
    // read its constants from the kernel parameters instead of lane registers
    ModelDev m0;
    int smem_table_offset;     // SMEM mode: first entry of the staged table
    int smem_table_points;     // SMEM mode: entries staged
    long long total_units;
    unsigned long long *cursor;
    int *flags;                // flag words (kFlag*)
    int32_t *nsteps;
    double *logw;
    uint8_t *status;
    uint32_t rk[20];           // Philox round keys: rk[2r] = key_lo + r W0, rk[2r+1] = key_hi + r W1
    int groups_per_check;      // refill every 4 * groups_per_check steps
    unsigned long long budget_ns;    // > 0: abort after this long (device clock)
    unsigned long long *t0;          // first %globaltimer reading of the launch (0 before)
    // learned proposal (MLP variants): launch-wide proposal, from the first MLP run
    int mlp_run;               // index of a run carrying the proposal parameters
    // segment records (record variant)
    float *records;            // [rec_cap][8]
    unsigned long long *rec_cursor;
    long long rec_cap;
};

struct HistParams {
    const int32_t *nsteps;
    const double *logw;
    const uint8_t *status;
    long long unit_begin;
    long long n;               // trajectories of the run
    double dN;
    double N_lo, db, N_tail;   // N_tail NaN: no tail set
    int n_bins;
    int chunk;                 // units per CTA
    unsigned long long *maxkey;   // [n_bins + 2]: per-bin, global, tail max of ln w
    double *mom;               // [kJackknife][n_bins][5]: count, S1, S2, Slw, Slw2
    double *scal;              // [kJackknife][16] scalars
};

// Scalar slots of HistParams::scal (per jackknife block).
enum {
    kScN = 0, kScPassed, kScUnder, kScOver, kScCapped, kScSumN, kScSumWN, kScSumW,
    kScTailW, kScTailW2, kScTailN, kScCount
};

// Stepper variants: weighted (any bias), table in shared memory, learned
// proposal, segment records.
struct EmVariant {
    bool weighted, smem, mlp, rec, nidx;
    bool rank2;              // full-rank 2-D noise stepper
    bool dtab;               // V'/V from the bump's cubic table
    bool mnet;               // learned proposal with one network per run
};

// Host wrappers implemented in fpt_kernels.cu.
int em_occupancy(EmVariant v, int block, size_t smem_bytes);
size_t em_smem_bytes(EmVariant v, int table_entries, int n_runs, int n_models);
// FPT_CHECKS builds: read and clear the device error word of the bounds checks
// (kCheck* bits; synchronous). Other builds return 0.
cudaError_t checks_take(int *word);
cudaError_t em_launch(const EmParams &p, EmVariant v, int grid, int block, size_t smem_bytes,
                      cudaStream_t s);

// Host wrappers implemented in fpt_mlp.cu.
cudaError_t mlp_pack_launch(const float *params, void *blob, cudaStream_t s);
cudaError_t mlp_eval_launch(const void *blob, const float *s, const float *tan_t, long long n, float amax,
                            float *alpha, float *o, cudaStream_t st);
cudaError_t mlp_coef_launch(const int32_t *nsteps, const double *logw, long long n, double dN, double lambda,
                            double N_cut, double scale, double *Y, double *acc, float *coef, cudaStream_t s);
cudaError_t mlp_bwd_launch(const float *params, const float *rec, long long n_rec, const float *coef, float dN,
                           float amax, const float *dalpha_direct, float *grad, int sm_count, cudaStream_t s,
                           const uint32_t *perm, float *partial, int rank2 = 0, long long rec_bound = 0);
int mlp_bwd_max_blocks(int sm_count);
size_t mlp_coef_scratch_doubles();
cudaError_t rec_order_launch(const float *rec, long long n_rec, long long n_units, int segment, int *cnt,
                             long long *off, uint32_t *perm, int *err, cudaStream_t s);
cudaError_t mlp_adam_launch(float *P, const float *G, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, int step, float clip, cudaStream_t s);
size_t mlp_bwd_smem();
cudaError_t hist_launch(const HistParams &p, double *out, cudaStream_t s);
cudaError_t hist_noalloc_launch(HistParams p, double *out, cudaStream_t s);
size_t hist_noalloc_scratch_bytes();
cudaError_t n_of_steps_launch(const int32_t *nsteps, long long n, double dN, double *N,
                              cudaStream_t s);

}  // namespace fpt_dev
