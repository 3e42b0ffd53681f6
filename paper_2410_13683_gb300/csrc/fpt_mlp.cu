// fpt_mlp.cu -- kernels of the learned importance-sampling proposal.
//
//   mlp_pack_kernel     fp32 canonical parameters -> bf16 fragment blob
//   mlp_eval_kernel     alpha for given states (the stepper's device forward)
//   mlp_coef_kernel     per-trajectory coefficient of the log-variance loss
//   mlp_bwd_kernel      gradient of sum_r dalpha_r alpha(s_r) over segment
//                       records, bf16 mma.sync with fp32 accumulation
//   mlp_adam_kernel     Adam update of the fp32 master parameters
//
// Loss (log-variance towards the exponentially tilted target, held-alpha
// segments): L = Var_Q[ln w + lambda min(N, N_cut)], evaluated at the sampling
// parameters; with Y_j = ln w_j + lambda min(N_j, N_cut),
//   dL/dtheta = (2/n) sum_j (Y_j - b) d ln w_j / dtheta,
//   d ln w_j / dtheta = -sum_s sqrt(dN) (sum of xi over segment s) d alpha_s / dtheta,
// for any baseline b (the score of the sampling law has zero mean).
#include "fpt_internal.h"
#include "fpt_mlp.cuh"

#include <cuda_runtime.h>
#include <math.h>

namespace fpt_dev {

// ---------------------------------------------------------------------------
// packing
// ---------------------------------------------------------------------------
__device__ __forceinline__ float w_kn(const float *P, int layer, int k, int n)
{
    // B[k][n] = W[n][k] of the layer, zero outside the real shape
    if (layer == 0) return (k < kMlpIn && n < kMlpH) ? P[kOffW1 + n * kMlpIn + k] : 0.0f;
    if (layer == 1) return P[kOffW2 + n * kMlpH + k];
    return (n < kMlpOut) ? P[kOffW3 + n * kMlpH + k] : 0.0f;
}

__global__ void mlp_pack_kernel(const float *__restrict__ P, uint2 *__restrict__ tiles, float *__restrict__ bias)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id < kMlpTiles * 32) {
        const int tile = id >> 5, lane = id & 31, g = lane >> 2, t = lane & 3;
        int layer, nt, kt;
        if (tile < kTilesL1) { layer = 0; nt = tile; kt = 0; }
        else if (tile < kTilesL1 + kTilesL2) { layer = 1; nt = (tile - kTilesL1) >> 2; kt = (tile - kTilesL1) & 3; }
        else { layer = 2; nt = 0; kt = tile - kTilesL1 - kTilesL2; }
        const int n = 8 * nt + g, k = 16 * kt + 2 * t;
        uint2 v;
        v.x = pack_bf16x2(w_kn(P, layer, k, n), w_kn(P, layer, k + 1, n));
        v.y = pack_bf16x2(w_kn(P, layer, k + 8, n), w_kn(P, layer, k + 9, n));
        tiles[id] = v;
    }
    if (id < kMlpBiasFloats) {
        float b;
        if (id < kMlpH) b = P[kOffB1 + id];
        else if (id < 2 * kMlpH) b = P[kOffB2 + id - kMlpH];
        else b = (id - 2 * kMlpH < kMlpOut) ? P[kOffB3 + id - 2 * kMlpH] : 0.0f;
        bias[id] = b;
    }
}

cudaError_t mlp_pack_launch(const float *params, void *blob, cudaStream_t s)
{
    uint2 *tiles = reinterpret_cast<uint2 *>(blob);
    float *bias = reinterpret_cast<float *>(tiles + kMlpTiles * 32);
    mlp_pack_kernel<<<(kMlpTiles * 32 + 255) / 256, 256, 0, s>>>(params, tiles, bias);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// evaluation: states s (n x 3, already normalised), t (n) -> alpha, (o1, o2)
// ---------------------------------------------------------------------------
__global__ void mlp_eval_kernel(const uint2 *__restrict__ tiles, const float *__restrict__ bias,
                                const float *__restrict__ s, const float *__restrict__ tan_t, long long n,
                                float amax, float *__restrict__ alpha, float *__restrict__ o)
{
    const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long w = warp0; w * 32 < n; w += nwarps) {
        const long long i = w * 32 + lane;
        const bool ok = i < n;
        const float in0 = ok ? s[3 * i] : 0.0f, in1 = ok ? s[3 * i + 1] : 0.0f, in2 = ok ? s[3 * i + 2] : 0.0f;
        float o1, o2;
        mlp_forward_warp(tiles, bias, in0, in1, in2, o1, o2);
        if (ok) {
            float raw;
            alpha[i] = mlp_alpha_of(o1, o2, tan_t[i], amax, raw);
            if (o) { o[2 * i] = o1; o[2 * i + 1] = o2; }
        }
    }
}

cudaError_t mlp_eval_launch(const void *blob, const float *s, const float *tan_t, long long n, float amax,
                            float *alpha, float *o, cudaStream_t st)
{
    const uint2 *tiles = reinterpret_cast<const uint2 *>(blob);
    const float *bias = reinterpret_cast<const float *>(tiles + kMlpTiles * 32);
    const long long warps = (n + 31) / 32;
    const int grid = (int)std::min<long long>(4096, (warps + 3) / 4);
    mlp_eval_kernel<<<grid, 128, 0, st>>>(tiles, bias, s, tan_t, n, amax, alpha, o);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// loss coefficients: c_j = (2/n)(Y_j - b), Y_j = ln w_j + lambda min(N_j, N_cut),
// with b = mean Y over the run; also writes sum Y and sum Y^2 (loss monitor).
// The sums are deterministic: each block reduces its grid-stride share in a
// fixed order into its own partial, and one thread adds the partials in block
// order (no floating-point atomics, so the result does not depend on timing).
// ---------------------------------------------------------------------------
constexpr int kYBlocks = 1024;

__global__ void __launch_bounds__(256) mlp_y_kernel(const int32_t *__restrict__ nsteps,
                                                    const double *__restrict__ logw, long long n, double dN,
                                                    double lambda, double N_cut, double *__restrict__ Y,
                                                    double *__restrict__ part)
{
    __shared__ double r1[8], r2[8];
    double s1 = 0.0, s2 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double N = (double)nsteps[i] * dN;
        const double y = logw[i] + lambda * fmin(N, N_cut);
        Y[i] = y;
        s1 += y;
        s2 += y * y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = s1;
        r2[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t1 += r1[w]; t2 += r2[w]; }
        part[2 * blockIdx.x] = t1;
        part[2 * blockIdx.x + 1] = t2;
    }
}

__global__ void sum_partials_kernel(const double *__restrict__ part, int nb, double *__restrict__ acc)
{
    double t1 = 0.0, t2 = 0.0;
    for (int b = 0; b < nb; ++b) { t1 += part[2 * b]; t2 += part[2 * b + 1]; }
    acc[0] = t1;
    acc[1] = t2;
}

__global__ void mlp_coef_kernel(const double *__restrict__ Y, long long n, const double *__restrict__ acc,
                                double scale, float *__restrict__ coef)
{
    const double mean = acc[0] / (double)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        coef[i] = (float)(scale * (Y[i] - mean));
}

size_t mlp_coef_scratch_doubles() { return 2 * kYBlocks + 2; }

// coef_j = scale (Y_j - mean Y); scale = 2/n of the whole round. acc holds
// 2 kYBlocks + 2 doubles: the block partials, then (sum Y, sum Y^2).
cudaError_t mlp_coef_launch(const int32_t *nsteps, const double *logw, long long n, double dN, double lambda,
                            double N_cut, double scale, double *Y, double *acc, float *coef, cudaStream_t s)
{
    const int grid = (int)std::min<long long>(kYBlocks, std::max<long long>(1, (n + 255) / 256));
    double *part = acc + 2;
    mlp_y_kernel<<<grid, 256, 0, s>>>(nsteps, logw, n, dN, lambda, N_cut, Y, part);
    sum_partials_kernel<<<1, 1, 0, s>>>(part, grid, acc);
    mlp_coef_kernel<<<grid, 256, 0, s>>>(Y, n, acc, scale, coef);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// record order
// ---------------------------------------------------------------------------
// The stepper appends segment records with an atomic cursor, so their order
// in the buffer depends on warp timing. The backward sums over records in
// tiles, and floating-point sums depend on the order, so the records are put
// in a fixed order first: by trajectory (launch unit), then by segment. A
// trajectory's segments start at multiples of the segment length (the lane
// that runs it was loaded at a refill point, and refill points are segment
// starts), so segment k of unit u goes to position off[u] + k, off the
// exclusive prefix sum of the per-unit counts: a permutation built by integer
// counting and a scan, exact and independent of timing.
__global__ void rec_count_kernel(const float *__restrict__ rec, long long n_rec, long long n_units,
                                 int *__restrict__ cnt, int *__restrict__ err)
{
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n_rec;
         r += (long long)gridDim.x * blockDim.x) {
        const uint32_t u = __float_as_uint(rec[8 * r + 6]);
        if ((long long)u < n_units) atomicAdd(cnt + u, 1);
        else atomicOr(err, 1);
    }
}

// Exclusive scan of cnt[0 .. n) into off (one block of 1024 threads: each
// thread scans a contiguous slice, the slice totals are scanned in shared
// memory, then each slice is written with its base).
__global__ void __launch_bounds__(1024) rec_scan_kernel(const int *__restrict__ cnt, long long n,
                                                        long long *__restrict__ off)
{
    __shared__ long long tot[1024];
    const long long per = (n + blockDim.x - 1) / blockDim.x;
    const long long b = threadIdx.x * per, e = min(n, b + per);
    long long t = 0;
    for (long long i = b; i < e; ++i) t += cnt[i];
    tot[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            const long long v = tot[k];
            tot[k] = run;
            run += v;
        }
    }
    __syncthreads();
    long long run = tot[threadIdx.x];
    for (long long i = b; i < e; ++i) {
        off[i] = run;
        run += cnt[i];
    }
}

__global__ void rec_perm_kernel(const float *__restrict__ rec, long long n_rec, long long n_units, int segment,
                                const int *__restrict__ cnt, const long long *__restrict__ off,
                                uint32_t *__restrict__ perm, int *__restrict__ err)
{
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n_rec;
         r += (long long)gridDim.x * blockDim.x) {
        const uint32_t u = __float_as_uint(rec[8 * r + 6]);
        const int n0 = __float_as_int(rec[8 * r + 7]);
        if ((long long)u >= n_units || n0 < 0 || (n0 % segment) != 0) { atomicOr(err, 2); continue; }
        const int k = n0 / segment;
        if (k >= cnt[u]) { atomicOr(err, 4); continue; }
        // slots start at 0xffffffff: a slot taken twice means two records of one segment
        if (atomicExch(perm + off[u] + k, (uint32_t)r) != 0xffffffffu) atomicOr(err, 8);
    }
}

cudaError_t rec_order_launch(const float *rec, long long n_rec, long long n_units, int segment, int *cnt,
                             long long *off, uint32_t *perm, int *err, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n_units, s))) return e;
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), s))) return e;
    if (n_rec <= 0) return cudaSuccess;
    if ((e = cudaMemsetAsync(perm, 0xff, sizeof(uint32_t) * (size_t)n_rec, s))) return e;
    const int grid = (int)std::min<long long>(4096, (n_rec + 255) / 256);
    rec_count_kernel<<<grid, 256, 0, s>>>(rec, n_rec, n_units, cnt, err);
    rec_scan_kernel<<<1, 1024, 0, s>>>(cnt, n_units, off);
    rec_perm_kernel<<<grid, 256, 0, s>>>(rec, n_rec, n_units, segment, cnt, off, perm, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// backward over segment records
// ---------------------------------------------------------------------------
// Record layout (8 x 32-bit): in0, in1, in2, tan_t, raw alpha, sum_xi, unit,
// first step of the segment.
// dalpha = coef[unit] * (-sqrt(dN) * sum_xi), zero where |raw alpha| >= amax.
// Full-rank (2-D) records: in0, in1, in2, sum_xi2, 0, sum_xi1, unit, first step; the
// output gradient is coef[unit] (-sqrt(dN)) (sum_xi1, sum_xi2), each component
// zero where that output is clamped (beta_k = clamp(o_k)).
constexpr int kBwdWarps = 4;
constexpr int kBwdRows = 16 * kBwdWarps;     // records per tile
constexpr int kSX = 24;                      // row strides (bf16 elements), chosen
constexpr int kSA = 72;                      // so that 8 consecutive rows of a
constexpr int kSH = 88;                      // ldmatrix hit distinct banks

struct BwdSmem {
    uint2 tiles[kMlpTiles * 32];
    float bias[kMlpBiasFloats];
    uint32_t w2t[kMlpH * kSA / 2];           // W2 transposed [in][out], bf16
    float w3[kMlpOut * kMlpH];
    __nv_bfloat16 x[kBwdRows * kSX];         // inputs, column 3 = 1 (bias gradient)
    __nv_bfloat16 h1[kBwdRows * kSH];        // silu(a1), column 64 = 1
    __nv_bfloat16 h2[kBwdRows * kSH];        // silu(a2), column 64 = 1
    __nv_bfloat16 da1[kBwdRows * kSA];
    __nv_bfloat16 da2[kBwdRows * kSA];
    __nv_bfloat16 dout[kBwdRows * kSX];      // d alpha / d(o1, o2) scaled by dalpha
    float tt[kBwdRows], dal[kBwdRows];
};

__device__ __forceinline__ void ldsm_x4_trans(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3,
                                              const void *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(a));
}

__device__ __forceinline__ float sigmoid_f(float v) { return __fdividef(1.0f, 1.0f + __expf(-v)); }

__device__ __forceinline__ float dsilu_f(float v)
{
    const float s = sigmoid_f(v);
    return s * fmaf(v, 1.0f - s, 1.0f);
}

// A fragment (16 x 16, m x k) of M^T where M is stored row-major [k][m]
// (row stride ld elements), rows k0.., columns m0..
__device__ __forceinline__ void ldA_trans(uint32_t a[4], const __nv_bfloat16 *M, int ld, int k0, int m0)
{
    const int lane = threadIdx.x & 31, j = lane >> 3, i = lane & 7;
    // matrices: (m 0-7, k 0-7), (m 8-15, k 0-7), (m 0-7, k 8-15), (m 8-15, k 8-15)
    const __nv_bfloat16 *p = M + (size_t)(k0 + i + 8 * (j >> 1)) * ld + m0 + 8 * (j & 1);
    ldsm_x4_trans(a[0], a[1], a[2], a[3], p);
}

// B fragments (k 16 x n 8) for two adjacent n tiles, B stored row-major [k][n]
__device__ __forceinline__ void ldB2_trans(uint2 &b0, uint2 &b1, const __nv_bfloat16 *M, int ld, int k0, int n0)
{
    const int lane = threadIdx.x & 31, j = lane >> 3, i = lane & 7;
    // matrices: (k 0-7, n0), (k 8-15, n0), (k 0-7, n0+8), (k 8-15, n0+8)
    const __nv_bfloat16 *p = M + (size_t)(k0 + i + 8 * (j & 1)) * ld + n0 + 8 * (j >> 1);
    ldsm_x4_trans(b0.x, b0.y, b1.x, b1.y, p);
}

__device__ __forceinline__ void st_bf16x2(__nv_bfloat16 *p, float lo, float hi)
{
    *reinterpret_cast<uint32_t *>(p) = pack_bf16x2(lo, hi);
}

__global__ void __launch_bounds__(kBwdWarps * 32)
mlp_bwd_kernel(const float *__restrict__ P, const float *__restrict__ rec, long long n_rec, long long rec_bound,
               const float *__restrict__ coef, float neg_sqrt_dN, float amax,
               const float *__restrict__ dalpha_direct, const uint32_t *__restrict__ perm,
               float *__restrict__ partial, int rank2)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem &S = *reinterpret_cast<BwdSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
    const unsigned FULL = 0xffffffffu;

    // stage the weights: forward blob, W2^T (bf16), W3 (fp32)
    for (int id = tid; id < kMlpTiles * 32; id += blockDim.x) {
        const int tile = id >> 5, ln = id & 31, gg = ln >> 2, tq = ln & 3;
        int layer, nt, kt;
        if (tile < kTilesL1) { layer = 0; nt = tile; kt = 0; }
        else if (tile < kTilesL1 + kTilesL2) { layer = 1; nt = (tile - kTilesL1) >> 2; kt = (tile - kTilesL1) & 3; }
        else { layer = 2; nt = 0; kt = tile - kTilesL1 - kTilesL2; }
        const int nn = 8 * nt + gg, kk = 16 * kt + 2 * tq;
        uint2 v;
        v.x = pack_bf16x2(w_kn(P, layer, kk, nn), w_kn(P, layer, kk + 1, nn));
        v.y = pack_bf16x2(w_kn(P, layer, kk + 8, nn), w_kn(P, layer, kk + 9, nn));
        S.tiles[id] = v;
    }
    for (int id = tid; id < kMlpBiasFloats; id += blockDim.x) {
        float b;
        if (id < kMlpH) b = P[kOffB1 + id];
        else if (id < 2 * kMlpH) b = P[kOffB2 + id - kMlpH];
        else b = (id - 2 * kMlpH < kMlpOut) ? P[kOffB3 + id - 2 * kMlpH] : 0.0f;
        S.bias[id] = b;
    }
    for (int id = tid; id < kMlpH * kMlpH / 2; id += blockDim.x) {
        const int in = id / (kMlpH / 2), op = 2 * (id % (kMlpH / 2));   // W2T[in][op], W2T[in][op+1]
        S.w2t[in * (kSA / 2) + op / 2] = pack_bf16x2(P[kOffW2 + op * kMlpH + in], P[kOffW2 + (op + 1) * kMlpH + in]);
    }
    for (int id = tid; id < kMlpOut * kMlpH; id += blockDim.x) S.w3[id] = P[kOffW3 + id];
    // constant columns: zero the padded operand rows once, ones for the bias gradients
    for (int id = tid; id < kBwdRows * kSX; id += blockDim.x) {
        S.x[id] = __float2bfloat16_rn((id % kSX) == 3 ? 1.0f : 0.0f);
        S.dout[id] = __float2bfloat16_rn(0.0f);
    }
    for (int id = tid; id < kBwdRows * kSH; id += blockDim.x) {
        const int c = id % kSH;
        const float v = (c == kMlpH) ? 1.0f : 0.0f;
        S.h1[id] = __float2bfloat16_rn(v);
        S.h2[id] = __float2bfloat16_rn(v);
    }
    __syncthreads();

    // persistent gradient accumulators of this warp
    float gW2[9][4], gW1[2][4], gW3[3][4];
#pragma unroll
    for (int i = 0; i < 9; ++i) gW2[i][0] = gW2[i][1] = gW2[i][2] = gW2[i][3] = 0.0f;
#pragma unroll
    for (int i = 0; i < 2; ++i) gW1[i][0] = gW1[i][1] = gW1[i][2] = gW1[i][3] = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) gW3[i][0] = gW3[i][1] = gW3[i][2] = gW3[i][3] = 0.0f;

    const long long n_tiles = (n_rec + kBwdRows - 1) / kBwdRows;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // ---- load records of this tile
        if (tid < kBwdRows) {
            const long long slot = tile * kBwdRows + tid;
            // records in a fixed order; a slot the ordering left unfilled (it
            // reports that as an error) reads as an empty row
            const long long r = slot < n_rec ? (perm ? (long long)perm[slot] : slot) : rec_bound;
            float in0 = 0, in1 = 0, in2 = 0, tq = 0, da = 0;
            if (r < rec_bound) {
                const float *q = rec + 8 * r;
                in0 = q[0]; in1 = q[1]; in2 = q[2]; tq = q[3];
                if (rank2) {
                    // (tt, dal) = output gradients of o2 and o1 (direct: dalpha_direct[2r], [2r + 1])
                    if (dalpha_direct) { da = dalpha_direct[2 * r]; tq = dalpha_direct[2 * r + 1]; }
                    else {
                        const float c = coef[__float_as_uint(q[6])] * neg_sqrt_dN;
                        da = c * q[5];
                        tq = c * q[3];
                    }
                } else if (dalpha_direct) {
                    da = dalpha_direct[r];
                } else {
                    da = coef[__float_as_uint(q[6])] * (neg_sqrt_dN * q[5]);
                }
            }
            __nv_bfloat16 *xr = S.x + tid * kSX;
            st_bf16x2(xr, in0, in1);
            xr[2] = __float2bfloat16_rn(in2);
            S.tt[tid] = tq;
            S.dal[tid] = da;
        }
        __syncthreads();

        // ---- per-warp forward (rows 16 warp + g, + 8) and backward to da1, da2
        const int r0 = 16 * warp + g, r1 = r0 + 8;
        const __nv_bfloat16 *x0p = S.x + r0 * kSX, *x1p = S.x + r1 * kSX;
        const uint32_t a0 = *reinterpret_cast<const uint32_t *>(x0p + 2 * t);
        const uint32_t a1 = *reinterpret_cast<const uint32_t *>(x1p + 2 * t);
        const uint32_t a2 = *reinterpret_cast<const uint32_t *>(x0p + 2 * t + 8);
        const uint32_t a3 = *reinterpret_cast<const uint32_t *>(x1p + 2 * t + 8);
        float d1[8][4], d2[8][4];
        uint32_t A2[4][4], A3[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float2 c = *reinterpret_cast<const float2 *>(S.bias + 8 * nt + 2 * t);
            d1[nt][0] = c.x; d1[nt][1] = c.y; d1[nt][2] = c.x; d1[nt][3] = c.y;
            mma_bf16_16816(d1[nt], a0, a1, a2, a3, S.tiles[nt * 32 + lane]);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float h00 = silu_f(d1[nt][0]), h01 = silu_f(d1[nt][1]);
            const float h10 = silu_f(d1[nt][2]), h11 = silu_f(d1[nt][3]);
            st_bf16x2(S.h1 + r0 * kSH + 8 * nt + 2 * t, h00, h01);
            st_bf16x2(S.h1 + r1 * kSH + 8 * nt + 2 * t, h10, h11);
            const int kt = nt >> 1, hi = nt & 1;
            A2[kt][0 + 2 * hi] = pack_bf16x2(h00, h01);
            A2[kt][1 + 2 * hi] = pack_bf16x2(h10, h11);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float2 c = *reinterpret_cast<const float2 *>(S.bias + kMlpH + 8 * nt + 2 * t);
            d2[nt][0] = c.x; d2[nt][1] = c.y; d2[nt][2] = c.x; d2[nt][3] = c.y;
#pragma unroll
            for (int kt = 0; kt < 4; ++kt)
                mma_bf16_16816(d2[nt], A2[kt][0], A2[kt][1], A2[kt][2], A2[kt][3],
                               S.tiles[(kTilesL1 + nt * 4 + kt) * 32 + lane]);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float h00 = silu_f(d2[nt][0]), h01 = silu_f(d2[nt][1]);
            const float h10 = silu_f(d2[nt][2]), h11 = silu_f(d2[nt][3]);
            st_bf16x2(S.h2 + r0 * kSH + 8 * nt + 2 * t, h00, h01);
            st_bf16x2(S.h2 + r1 * kSH + 8 * nt + 2 * t, h10, h11);
            const int kt = nt >> 1, hi = nt & 1;
            A3[kt][0 + 2 * hi] = pack_bf16x2(h00, h01);
            A3[kt][1 + 2 * hi] = pack_bf16x2(h10, h11);
        }
        float d3[4];
        {
            const float2 c = *reinterpret_cast<const float2 *>(S.bias + 2 * kMlpH + 2 * t);
            d3[0] = c.x; d3[1] = c.y; d3[2] = c.x; d3[3] = c.y;
#pragma unroll
            for (int kt = 0; kt < 4; ++kt)
                mma_bf16_16816(d3, A3[kt][0], A3[kt][1], A3[kt][2], A3[kt][3],
                               S.tiles[(kTilesL1 + kTilesL2 + kt) * 32 + lane]);
        }
        // d alpha / d o on rows r0, r1 (computed by the t == 0 lanes, shared in the quad)
        float do0a = 0.f, do1a = 0.f, do0b = 0.f, do1b = 0.f;
        if (t == 0) {
            if (rank2) {
                // beta_k = clamp(o_k): each output passes its own gradient unless clamped
                do0a = fabsf(d3[0]) < amax ? S.dal[r0] : 0.0f;
                do1a = fabsf(d3[1]) < amax ? S.tt[r0] : 0.0f;
                do0b = fabsf(d3[2]) < amax ? S.dal[r1] : 0.0f;
                do1b = fabsf(d3[3]) < amax ? S.tt[r1] : 0.0f;
            } else {
                const float ta = S.tt[r0], tb = S.tt[r1];
                const float ia = rsqrtf(fmaf(ta, ta, 1.0f)), ib = rsqrtf(fmaf(tb, tb, 1.0f));
                const float rawa = (d3[0] + ta * d3[1]) * ia, rawb = (d3[2] + tb * d3[3]) * ib;
                const float ca = fabsf(rawa) < amax ? S.dal[r0] * ia : 0.0f;
                const float cb = fabsf(rawb) < amax ? S.dal[r1] * ib : 0.0f;
                do0a = ca; do1a = ca * ta; do0b = cb; do1b = cb * tb;
            }
            st_bf16x2(S.dout + r0 * kSX, do0a, do1a);
            st_bf16x2(S.dout + r1 * kSX, do0b, do1b);
        }
        const int q0 = lane & ~3;
        do0a = __shfl_sync(FULL, do0a, q0); do1a = __shfl_sync(FULL, do1a, q0);
        do0b = __shfl_sync(FULL, do0b, q0); do1b = __shfl_sync(FULL, do1b, q0);
        // da2 = (do W3) * silu'(a2), stored and re-packed as the A operand of dh1 = da2 W2
        uint32_t D2[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int u = 8 * nt + 2 * t;
            const float w00 = S.w3[u], w01 = S.w3[u + 1], w10 = S.w3[kMlpH + u], w11 = S.w3[kMlpH + u + 1];
            const float e00 = fmaf(do0a, w00, do1a * w10) * dsilu_f(d2[nt][0]);
            const float e01 = fmaf(do0a, w01, do1a * w11) * dsilu_f(d2[nt][1]);
            const float e10 = fmaf(do0b, w00, do1b * w10) * dsilu_f(d2[nt][2]);
            const float e11 = fmaf(do0b, w01, do1b * w11) * dsilu_f(d2[nt][3]);
            st_bf16x2(S.da2 + r0 * kSA + u, e00, e01);
            st_bf16x2(S.da2 + r1 * kSA + u, e10, e11);
            const int kt = nt >> 1, hi = nt & 1;
            D2[kt][0 + 2 * hi] = pack_bf16x2(e00, e01);
            D2[kt][1 + 2 * hi] = pack_bf16x2(e10, e11);
        }
        // dh1 = da2 W2: B[k = out][n = in] = W2[out][in] = W2T[in][out]
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float e[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                const uint32_t *row = S.w2t + (8 * nt + g) * (kSA / 2);
                uint2 b;
                b.x = row[8 * kt + t];
                b.y = row[8 * kt + 4 + t];
                mma_bf16_16816(e, D2[kt][0], D2[kt][1], D2[kt][2], D2[kt][3], b);
            }
            const int u = 8 * nt + 2 * t;
            st_bf16x2(S.da1 + r0 * kSA + u, e[0] * dsilu_f(d1[nt][0]), e[1] * dsilu_f(d1[nt][1]));
            st_bf16x2(S.da1 + r1 * kSA + u, e[2] * dsilu_f(d1[nt][2]), e[3] * dsilu_f(d1[nt][3]));
        }
        __syncthreads();

        // ---- weight gradients: contractions over the kBwdRows records of the tile
        const int m0 = 16 * warp;
#pragma unroll
        for (int ks = 0; ks < kBwdRows / 16; ++ks) {
            uint32_t a[4];
            ldA_trans(a, S.da2, kSA, 16 * ks, m0);              // dW2 rows: outputs m0..m0+15
#pragma unroll
            for (int np = 0; np < 4; ++np) {
                uint2 b0, b1;
                ldB2_trans(b0, b1, S.h1, kSH, 16 * ks, 16 * np);
                mma_bf16_16816(gW2[2 * np], a[0], a[1], a[2], a[3], b0);
                mma_bf16_16816(gW2[2 * np + 1], a[0], a[1], a[2], a[3], b1);
            }
            {
                uint2 b0, b1;                                      // n tile 8: column 64 = ones (db2)
                ldB2_trans(b0, b1, S.h1, kSH, 16 * ks, 64);
                mma_bf16_16816(gW2[8], a[0], a[1], a[2], a[3], b0);
            }
            ldA_trans(a, S.da1, kSA, 16 * ks, m0);              // dW1 rows, inputs (col 3 = db1)
            {
                uint2 b0, b1;
                ldB2_trans(b0, b1, S.x, kSX, 16 * ks, 0);
                mma_bf16_16816(gW1[0], a[0], a[1], a[2], a[3], b0);
                mma_bf16_16816(gW1[1], a[0], a[1], a[2], a[3], b1);
            }
            ldA_trans(a, S.dout, kSX, 16 * ks, 0);              // dW3: outputs 0, 1 (rows of the tile)
            {
                uint2 b0, b1;
                ldB2_trans(b0, b1, S.h2, kSH, 16 * ks, 16 * warp);   // n tiles 2 warp, 2 warp + 1
                mma_bf16_16816(gW3[0], a[0], a[1], a[2], a[3], b0);
                mma_bf16_16816(gW3[1], a[0], a[1], a[2], a[3], b1);
                if (warp == 0) {
                    ldB2_trans(b0, b1, S.h2, kSH, 16 * ks, 64);      // n tile 8 (db3)
                    mma_bf16_16816(gW3[2], a[0], a[1], a[2], a[3], b0);
                }
            }
        }
        __syncthreads();
    }

    // ---- flush: accumulator element (row g / g + 8, column 2t / 2t + 1 of each n tile)
    // into this block's partial gradient; every parameter has exactly one
    // writer in the block (warps own disjoint output rows of W1, W2 and disjoint
    // column tiles of W3), so plain stores fill the whole row and the partials
    // are summed later in block order
    const int m0 = 16 * warp;
    float *grad = partial + (size_t)blockIdx.x * kMlpParams;
#pragma unroll
    for (int nt = 0; nt < 9; ++nt) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int o = m0 + g + 8 * (e >> 1), c = 8 * nt + 2 * t + (e & 1);
            if (c < kMlpH) grad[kOffW2 + o * kMlpH + c] = gW2[nt][e];
            else if (c == kMlpH) grad[kOffB2 + o] = gW2[nt][e];
        }
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int o = m0 + g + 8 * (e >> 1), c = 8 * nt + 2 * t + (e & 1);
            if (c < kMlpIn) grad[kOffW1 + o * kMlpIn + c] = gW1[nt][e];
            else if (c == kMlpIn) grad[kOffB1 + o] = gW1[nt][e];
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j == 2 && warp != 0) break;
        const int nt = (j < 2) ? 2 * warp + j : 8;
#pragma unroll
        for (int e = 0; e < 2; ++e) {                           // rows g only (outputs 0, 1)
            const int o = g, c = 8 * nt + 2 * t + e;
            if (o >= kMlpOut) continue;
            if (c < kMlpH) grad[kOffW3 + o * kMlpH + c] = gW3[j][e];
            else if (c == kMlpH) grad[kOffB3 + o] = gW3[j][e];
        }
    }
}

size_t mlp_bwd_smem() { return sizeof(BwdSmem); }

// grad[i] += sum over blocks b = 0, 1, ... of partial[b][i], in block order.
__global__ void mlp_grad_reduce_kernel(const float *__restrict__ partial, int nb, float *__restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    float t = 0.0f;
    for (int b = 0; b < nb; ++b) t += partial[(size_t)b * kMlpParams + i];
    grad[i] += t;
}

int mlp_bwd_max_blocks(int sm_count) { return 3 * sm_count; }

// The gradient of a call is deterministic: records in the order perm gives
// (nullptr: buffer order), tiles statically assigned to blocks, per-block
// partials (partial: mlp_bwd_max_blocks(sm_count) x kMlpParams floats) added
// in block order. grad accumulates (+=). n_rec records are used (perm[0 ..
// n_rec) when perm is given); rec_bound is the number of records in the buffer,
// the bound of a valid perm entry (0: n_rec).
cudaError_t mlp_bwd_launch(const float *params, const float *rec, long long n_rec, const float *coef, float dN,
                           float amax, const float *dalpha_direct, float *grad, int sm_count, cudaStream_t s,
                           const uint32_t *perm, float *partial, int rank2, long long rec_bound)
{
    if (rec_bound <= 0) rec_bound = n_rec;
    const size_t smem = sizeof(BwdSmem);
    cudaError_t e = cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (n_rec <= 0) return cudaSuccess;
    // one wave: as many blocks as are resident at once (registers allow two per
    // SM), so no block waits for a second wave; the tile partition, and with it
    // the gradient, is fixed for a given device
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_bwd_kernel, kBwdWarps * 32, smem)))
        return e;
    per_sm = std::max(1, std::min(per_sm, 3));
    const long long tiles = (n_rec + kBwdRows - 1) / kBwdRows;
    const int grid = (int)std::min<long long>(tiles, (long long)per_sm * sm_count);
    mlp_bwd_kernel<<<grid, kBwdWarps * 32, smem, s>>>(params, rec, n_rec, rec_bound, coef, -sqrtf(dN), amax,
                                                      dalpha_direct, perm, partial, rank2);
    if ((e = cudaGetLastError())) return e;
    mlp_grad_reduce_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(partial, grid, grad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba) on the fp32 master parameters
// ---------------------------------------------------------------------------
__global__ void mlp_adam_kernel(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ m,
                                float *__restrict__ v, int n, float lr, float b1, float b2, float eps,
                                float bc1, float bc2, float clip)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float g = G[i];
    if (clip > 0.0f) g = fminf(fmaxf(g, -clip), clip);
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

cudaError_t mlp_adam_launch(float *P, const float *G, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, int step, float clip, cudaStream_t s)
{
    const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
    mlp_adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(P, G, m, v, n, lr, b1, b2, eps, bc1, bc2, clip);
    return cudaGetLastError();
}

}  // namespace fpt_dev
