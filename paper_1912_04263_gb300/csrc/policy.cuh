// rho adaptation on the device: the residual-ratio rule (paper Section 3.4,
// applied every rho_every iterations as in Section 5.3.3) and the learned
// policy, a 4-64-64-2 MLP with BF16 operands and FP32 accumulation that
// proposes rho as a log correction to the ratio rule's proposal (and
// optionally a log factor on the PCG tolerance weight lambda of Section
// 5.3.4).  The learned policy is not part of the paper; a zero output
// reproduces the ratio rule, and it falls back to the ratio rule whenever
// progress stalls.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace gb {

// Parameter vector layout (floats).
constexpr int kPolIn = 4, kPolHid = 64, kPolOut = 2;
constexpr int kOffMean = 0;                       // feature means (4)
constexpr int kOffStd = kOffMean + kPolIn;        // feature std devs (4)
constexpr int kOffW1 = kOffStd + kPolIn;          // 64 x 4, row major
constexpr int kOffB1 = kOffW1 + kPolHid * kPolIn;  // 64
constexpr int kOffW2 = kOffB1 + kPolHid;          // 64 x 64
constexpr int kOffB2 = kOffW2 + kPolHid * kPolHid;  // 64
constexpr int kOffW3 = kOffB2 + kPolHid;          // 2 x 64
constexpr int kOffB3 = kOffW3 + kPolOut * kPolHid;  // 2
constexpr int kOffExtra = kOffB3 + kPolOut;       // clamp, lambda_min, lambda_max, use_lambda
constexpr int kPolTotal = kOffExtra + 4;
static_assert(kPolTotal == GBOSQP_POLICY_PARAMS, "policy parameter layout");

struct PolicyDev {
    const float *params = nullptr;
};

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Residual-ratio rule (reading S2): rho * sqrt((||r_p|| / max(||Ax||, ||z||)) /
// (||r_d|| / max(||Px||, ||A'y||, ||q||))) on scaled quantities, clamped;
// a zero normaliser or dual residual leaves rho unchanged.
__host__ __device__ __forceinline__ double rho_ratio(const Status *st) {
    const double prim_norm = fmax(st->ax_s, st->z_s);
    const double dual_norm = fmax(fmax(st->px_s, st->aty_s), st->qnorm_s);
    if (!(prim_norm > 0.0) || !(dual_norm > 0.0) || !(st->rd_s > 0.0)) return st->rho;
    const double ratio = (st->rp_s / prim_norm) / (st->rd_s / dual_norm);
    if (!isfinite(ratio)) return st->rho;
    return fmin(fmax(st->rho * sqrt(ratio), st->rho_min), st->rho_max);
}

// Policy features: log ||r_prim||, log ||r_dual|| (scaled problem), log rho,
// log(1 + PCG steps since the last decision).
__device__ __forceinline__ void policy_features(const Status *st, float f[kPolIn]) {
    f[0] = (float)log(fmax(st->rp_s, 1e-30));
    f[1] = (float)log(fmax(st->rd_s, 1e-30));
    f[2] = (float)log(st->rho);
    f[3] = (float)log1p((double)st->cg_since_update);
}

// Forward pass by one CTA (>= 64 threads).  x: normalised features in
// shared memory; h1, h2: 64 floats of shared scratch; out: 2 floats.
// Operands are rounded to BF16, products accumulated in FP32.
__device__ __forceinline__ void policy_forward(const float *P, const float *x, float *h1, float *h2, float *out) {
    const int t = threadIdx.x;
    if (t < kPolHid) {
        float a = P[kOffB1 + t];
#pragma unroll
        for (int k = 0; k < kPolIn; ++k) a = fmaf(bf16r(P[kOffW1 + t * kPolIn + k]), x[k], a);
        h1[t] = bf16r(fmaxf(a, 0.f));
    }
    __syncthreads();
    if (t < kPolHid) {
        float a = P[kOffB2 + t];
        for (int k = 0; k < kPolHid; ++k) a = fmaf(bf16r(P[kOffW2 + t * kPolHid + k]), h1[k], a);
        h2[t] = bf16r(fmaxf(a, 0.f));
    }
    __syncthreads();
    if (t < kPolOut) {
        float a = P[kOffB3 + t];
        for (int k = 0; k < kPolHid; ++k) a = fmaf(bf16r(P[kOffW3 + t * kPolHid + k]), h2[k], a);
        out[t] = a;
    }
    __syncthreads();
}

// One rho decision with the learned policy, by the whole CTA.  Stall rule
// (reading S12): if the merit max(r_prim/eps_prim, r_dual/eps_dual) has not
// fallen by 10% since the previous decision, or the network output is not
// finite, the ratio rule decides for the next 50 iterations; after 3 stalls
// the ratio rule decides for the rest of the solve.
__device__ __forceinline__ void policy_decide(const PolicyDev &pol, Status *st, double *new_rho) {
    __shared__ float x[kPolIn], h1[kPolHid], h2[kPolHid], out[kPolOut];
    __shared__ int use;
    const float *P = pol.params;
    if (threadIdx.x == 0) {
        const double merit = fmax(st->r_prim / st->eps_prim, st->r_dual / st->eps_dual);
        int u = (!st->policy_disabled && st->stall_left <= 0) ? 1 : 0;
        if (st->stall_left > 0) st->stall_left -= st->rho_every;
        if (u && st->prev_merit > 0.0 && !(merit <= 0.9 * st->prev_merit)) {
            st->stall_count += 1;
            if (st->stall_count >= 3) st->policy_disabled = 1;
            else st->stall_left = 50;
            u = 0;
        }
        st->prev_merit = merit;
        float f[kPolIn];
        policy_features(st, f);
        for (int k = 0; k < kPolIn; ++k) x[k] = bf16r((f[k] - P[kOffMean + k]) / P[kOffStd + k]);
        use = u;
    }
    __syncthreads();
    if (use) policy_forward(P, x, h1, h2, out);
    if (threadIdx.x == 0) {
        double nr;
        if (use && isfinite(out[0]) && isfinite(out[1])) {
            const float cl = P[kOffExtra + 0];
            const float lm = fminf(fmaxf(out[0], -cl), cl);
            nr = fmin(fmax(rho_ratio(st) * exp((double)lm), st->rho_min), st->rho_max);
            if (P[kOffExtra + 3] != 0.f) {
                const double lam = 0.15 * exp((double)out[1]);
                st->lambda = fmin(fmax(lam, (double)P[kOffExtra + 1]), (double)P[kOffExtra + 2]);
            }
        } else {
            if (use) {  // non-finite output counts as a stall
                st->stall_count += 1;
                if (st->stall_count >= 3) st->policy_disabled = 1;
                else st->stall_left = 50;
            }
            nr = rho_ratio(st);
            st->fallbacks += 1;
        }
        *new_rho = nr;
    }
    __syncthreads();
}

}  // namespace gb
