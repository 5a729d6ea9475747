// Solve engine: ADMM (Algorithm 1) with the reduced KKT system eq.
// (kkt_red_sc) solved by warm-started Jacobi-PCG (Algorithm 3,
// Section 5.3), on the equilibrated problem, in working precision T
// (float: FP32 matrices and vectors with FP64 dot products and FP64
// termination reductions; double: everything FP64).
//
// Data layout in device memory (T unless noted):
//   A      m x n CSR          PAt = [P A'] n x (n+m) CSR, pend splits P | A'
//   xy  = [x ; y]    (n+m)    ADMM primal x and dual y, contiguous so that
//                             one gather over PAt reads P x and A' y
//   xt  = [x~ ; t0]  (n+m)    PCG iterate x~ (the warm start) and
//                             t0 = rho (A x~ - z) + y for the next PCG init
//   pt  = [p ; t]    (n+m)    PCG direction p and t = rho A p
//   dxy = [dx ; dy]  (n+m)    x^k - x^(k-1) and y^k - y^(k-1) (scaled)
//   z, zt (= A x~), l, u (m); q, minv, diagP, colsq, kp (K p), r (n);
//   ypc = (yv, pc) pairs (n): yv = M^{-1} r and pc = the previous p,
//   interleaved so that one load gathers both; D, E and their reciprocals
//   (double) for unscaling.
//
// Kernels of one ADMM iteration (each row-block kernel streams one matrix):
//   pcg_init   PAt: r = P x~ + sigma (x~ - x) + q + A' t0  (= K x~ - b),
//              yv = M^{-1} r, r'yv, ||r||_inf          [Alg. 3 initialize]
//   pcg_p_t    A:   p = -yv + beta p_prev, t = rho A p [Alg. 3 direction;
//                                                        K-apply, part 1]
//   pcg_kp     PAt: Kp = P p + sigma p + A' t, p'Kp    [K-apply, part 2]
//   pcg_update n:   x~ += a p, r += a Kp, yv = M^{-1} r, r'yv, ||r||_inf,
//                   beta, stop test ||r||_inf <= eps  [Alg. 3 loop body]
//   admm_update A:  z~ = A x~; x, z (projection), y (dual), t0, and the
//                   iterate differences dx, dy     [Alg. 1 steps 5-7]
// every check_every iterations:
//   check_a    A:   ||A x - z||, ||A x||, ||z|| (FP64 accumulation)
//   inf_a      A:   A dx against the bounds, dy clipped to the cone of
//                   finite support, ||dy||, support  [Section 3.1]
//   inf_b      PAt: ||P dx||, ||A'dy||, q'dx, ||dx|| [Section 3.1]
//   check_b    PAt: ||P x + q + A'y||, ||P x||, ||A'y||, objective; then
//              eq. (termination), the infeasibility tests, the PCG
//              tolerance of Section 5.3.4 and the rho update (Section 3.4 /
//              5.3.3 or the learned policy)
//   rho_apply  n, m: M^{-1} and t0 for a changed rho
#include <math.h>

#include <algorithm>
#include <cstddef>
#include <initializer_list>
#include <cstring>
#include <future>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <utility>

#include "common.cuh"
#include "engine.cuh"
#include "spmv.cuh"
#include "policy.cuh"

namespace gb {

namespace {

// (M^{-1} r, previous direction) pairs, stored interleaved so that the
// direction kernel's gather of p = -M^{-1} r + beta p_prev is one load
template <class T>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
};
template <>
struct Pair<double> {
    using type = double2;
};
template <class T>
using pair_t = typename Pair<T>::type;

// Single-reduction PCG state of one variable: r, w = K M^-1 r, s = K p and
// the Jacobi factor M^-1, kept together so that the direction kernel's
// gather of y = M^-1 r of the next step is one load.
template <class T>
struct __align__(4 * sizeof(T)) SrVec {
    T r, w, s, m;
};

// Rounded arithmetic with the operation order fixed (no contraction left to
// the compiler), so that a value formed at a gathered column is bitwise the
// one formed by the thread that owns that column.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Where the plan of k_pcg_kp keeps the rows it cut between warps: the
// split-row index of every row (-1 when whole), the split rows and their
// parts' sums, which k_pcg_update adds into Kp.
struct KpParts {
    const int *split_of;
    const SplitRow *split;
    const double *split_part;
};

template <class T>
struct Vecs {
    T *xy, *xt, *pt, *dxy;
    T *z, *zt, *l, *u;
    T *q, *minv, *diagp, *colsq, *kp, *r;
    pair_t<T> *ypc;  // (yv = M^{-1} r, pc = previous p) per variable
    SrVec<T> *sr0, *sr1;  // single-reduction PCG state, two buffers used in turn (nullptr: classic PCG)
    T *srp;               // single-reduction PCG direction p
    const T *rs;  // R = rho diag(rs), eq. (rho_vec): 1e3 on rows with l = u, else 1;
                  // nullptr for R = rho I (Section 5.3)
    const double *D, *E, *Dinv, *Einv;
    double *x_out, *y_out, *z_out;
    int n, m;
};

// doubles of the per-CTA record of a grid reduction (sums then maxima) that
// the partials buffer holds for every CTA of the largest grid
constexpr int kPartialRecord = 16;

// resident CTAs per SM requested for the row-block kernels of the PCG loop
// (bounds registers so that enough loads are in flight per SM)
#ifndef GB_MIN_BLOCKS
#define GB_MIN_BLOCKS 4
#endif
constexpr int kMinBlocks = GB_MIN_BLOCKS;
// steps of 32 nonzeros per batch of the warp-stream SpMV (see spmv.cuh)
constexpr int kU = 4;
// plan cost of a row of the group path, in nonzeros (measured on GB300 on
// the Lasso [P A']: at a weight of 24, the warps holding its 101000 rows of
// two nonzeros finished their share in under a third of the time the warps
// of its long rows took)
#ifndef GB_GROUP_ROW
#define GB_GROUP_ROW 8
#endif
// rows longer than this go to CTA bundles in the warp-stream plan
#ifndef GB_BUNDLE_MIN
#define GB_BUNDLE_MIN 4096
#endif
constexpr int kBundleMin = GB_BUNDLE_MIN;

template <class T>
__device__ __forceinline__ T clampv(T v, T lo, T hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

// rho_j / rho of row j (1 when R = rho I)
template <class T>
__device__ __forceinline__ T rscale(const Vecs<T> &v, int j) {
    return v.rs ? v.rs[j] : T(1);
}

// |v| as a double, the conversion of a float done on the integer pipe
template <class T>
__device__ __forceinline__ double absd(T v) {
    return to_acc<double>(v < T(0) ? -v : v);
}

// ------------------------------------------------------------ gathers

template <class T, class Acc>
struct GatherVec {
    const T *v;
    __device__ __forceinline__ Acc operator()(int c) const { return Acc(__ldg(v + c)); }
};

// x and dx at column c together (the SpMV core sums both products)
template <class T>
struct GatherDual {
    static constexpr bool kDual = true;
    const T *v, *w;
    __device__ __forceinline__ T operator()(int c) const { return __ldg(v + c); }
    __device__ __forceinline__ T second(int c) const { return __ldg(w + c); }
};

template <class T>
struct GatherDir {  // p = -yv + beta * p_prev
    const pair_t<T> *ypc;
    T beta;
    __device__ __forceinline__ T operator()(int c) const {
        const pair_t<T> w = __ldg(ypc + c);
        return -w.x + beta * w.y;
    }
};

// ------------------------------------------------------------ kernels

template <class T>
__global__ void __launch_bounds__(kThreads) k_reset(Vecs<T> v, Status *st, cudaGraphConditionalHandle hA,
                                                    int use_h) {
    const int n = v.n, m = v.m;
    const bool warm = st->warm != 0;
    const double rho = warm ? st->rho : st->rho0;
    const double sigma = st->sigma;
    const long long N = n > m ? n : m;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        if (i < n) {
            if (!warm) {
                v.xy[i] = T(0);
                v.xt[i] = T(0);
            }
            v.minv[i] = T(1.0 / ((double)v.diagp[i] + sigma + rho * (double)v.colsq[i]));
            v.ypc[i].y = T(0);
        }
        if (i < m && !warm) {
            v.xy[n + i] = T(0);
            v.xt[n + i] = T(0);
            v.z[i] = T(0);
            v.zt[i] = T(0);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->rho = rho;
        st->k = 0;
        st->cg_total = 0;
        st->status = 0;
        if (st->warm != 2) {
            st->eps_pcg = st->eps0;
            st->lambda = st->lambda0;
        }
        st->rho_updates = 0;
        st->rho_changed = 0;
        st->fallbacks = 0;
        st->stall_count = 0;
        st->stall_left = 0;
        st->policy_disabled = 0;
        st->last_merit = -1.0;
        st->prev_merit = -1.0;
        st->cg_since_update = 0;
        st->admm_continue = st->max_iter > 0 ? 1 : 0;
        if (use_h) cudaGraphSetConditional(hA, st->admm_continue);
    }
}

// r = K x~ - b = P x~ + sigma (x~ - x) + q + A' t0,  yv = M^{-1} r
template <class T>
struct EpiInit {
    Vecs<T> v;
    T sigma;
    __device__ __forceinline__ void row(int i, T s1, T, Red<1, 1> &red) {
        const T r = s1 + sigma * (v.xt[i] - v.xy[i]) + v.q[i];
        const T y = v.minv[i] * r;
        v.r[i] = r;
        v.ypc[i] = pair_t<T>{y, T(0)};
        if (v.sr0) {  // single reduction: w = 0, s = 0, p = 0 before the first step
            v.sr0[i] = SrVec<T>{r, T(0), T(0), v.minv[i]};
            v.srp[i] = T(0);
        }
        red.s[0] += (double)r * (double)y;
        red.m[0] = amax(red.m[0], absd(r));
    }
};

template <class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : 2) k_pcg_init(CsrW<T> PAt, Vecs<T> v, Status *st, double *partials,
                                                       cudaGraphConditionalHandle hP, int use_h) {
    EpiInit<T> epi{v, T(st->sigma)};
    Red<1, 1> red;
    red.zero();
    warp_rows<kU, T, false, false, true>(PAt, GatherVec<T, T>{v.xt}, epi, red);
    auto fin = [&](const Red<1, 1> &t) {
        if (threadIdx.x != 0) return;
        st->ry = t.s[0];
        st->rnorm = t.m[0];
        st->beta = 0.0;
        st->cg_it = 0;
        st->breakdown = 0;
        if (v.sr0) {  // the first single-reduction pair applies no step (alpha = 0)
            st->ry_prev = t.s[0];
            st->alpha_cg = 0.0;
            st->sr_par = 0;
            st->sr_pair = 0;
        }
        const int cont = (!st->device_error && isfinite(t.m[0]) && t.m[0] > st->eps_pcg && st->max_cg > 0) ? 1 : 0;
        st->pcg_continue = cont;
        if (use_h) cudaGraphSetConditional(hP, cont);
    };
    grid_finish_w<1, 1>(red, PAt, partials, &st->tickets[kTkI1], fin);
}

// p = -yv + beta p_prev (stored in pt[0..n)), t = rho A p (pt[n..n+m))
template <class T>
struct EpiDir {
    T *t;
    const T *rs;
    T rho;
    __device__ __forceinline__ void row(int j, T s1, T, Red<0, 0> &) { t[j] = (rs ? rho * rs[j] : rho) * s1; }
};

template <class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : 2) k_pcg_p_t(CsrW<T> A, Vecs<T> v, const Status *st) {
    const T beta = T(st->beta);
    const int n = v.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const pair_t<T> w = v.ypc[i];
        v.pt[i] = -w.x + beta * w.y;
    }
    EpiDir<T> epi{v.pt + n, v.rs, T(st->rho)};
    Red<0, 0> red;
    warp_rows<kU, T, false, true>(A, GatherDir<T>{v.ypc, beta}, epi, red);
}

// Kp = P p + sigma p + A' t;  p'Kp.  A row cut between warps contributes
// by parts: p_i (part sum) to p'Kp from each part and p_i sigma p_i from
// the part holding the row's start; its Kp entry is formed from the parts
// by k_pcg_update, the one reader of Kp.  So no warp waits on the others'
// parts and the kernel's end is not held up by a chain of combining warps.
template <class T>
struct EpiKp {
    static constexpr bool kSplitParts = true;
    Vecs<T> v;
    T sigma;
    __device__ __forceinline__ void row(int i, T s1, T, Red<1, 0> &red) {
        const T p = v.pt[i];
        const T kp = s1 + sigma * p;
        v.kp[i] = kp;
        red.s[0] += (double)p * (double)kp;
    }
    __device__ __forceinline__ void part(int i, bool first, T s1, T, Red<1, 0> &red) {
        const T p = v.pt[i];
        red.s[0] += (double)p * (double)s1;
        if (first) red.s[0] += (double)p * (double)(sigma * p);
    }
};

template <class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : 2) k_pcg_kp(CsrW<T> PAt, Vecs<T> v, Status *st, double *partials) {
    EpiKp<T> epi{v, T(st->sigma)};
    Red<1, 0> red;
    red.zero();
    warp_rows<kU, T, false>(PAt, GatherVec<T, T>{v.pt}, epi, red);
    auto fin = [&](const Red<1, 0> &t) {
        if (threadIdx.x != 0) return;
        const double pkp = t.s[0];
        st->pkp = pkp;
        if (pkp > 0.0 && isfinite(pkp)) {
            st->alpha_cg = st->ry / pkp;  // step length alpha = r'y / p'Kp
        } else {
            st->alpha_cg = 0.0;
            st->breakdown = 1;
        }
    };
    grid_finish_w<1, 0, false>(red, PAt, partials, &st->tickets[kTkK2], fin);
}

// x~ += a p; r += a Kp; yv = M^{-1} r; p_prev = p; r'yv; ||r||_inf; beta.
// The vector updates run in the working precision; r'yv accumulates the
// exact products in FP64.
// Kp_i of a row that k_pcg_kp's plan cut between warps: its parts' sums
// (FP64, slot order) rounded to T, plus sigma p_i, as EpiKp::row forms it.
template <class T>
__device__ __forceinline__ T kp_from_parts(const SplitRow &S, const double *split_part, T sigma, T p) {
    constexpr int kLd = 8;
    double s = 0.0;
    for (int k0 = 0; k0 < S.nparts; k0 += kLd) {
        double v[kLd];
#pragma unroll
        for (int u = 0; u < kLd; ++u) v[u] = k0 + u < S.nparts ? __ldcg(split_part + 2 * (size_t)(S.slot0 + k0 + u)) : 0.0;
#pragma unroll
        for (int u = 0; u < kLd; ++u)
            if (k0 + u < S.nparts) s += v[u];
    }
    return T(s) + sigma * p;
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_pcg_update(Vecs<T> v, Status *st, double *partials, KpParts kpp,
                                                         cudaGraphConditionalHandle hP, int use_h) {
    const T a = T(st->alpha_cg);
    const T sigma = T(st->sigma);
    const int n = v.n;
    Red<1, 1> red;
    red.zero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const T p = v.pt[i];
        const T x = v.xt[i] + a * p;
        T kp;
        const int l = kpp.split_of[i];
        if (l < 0) {
            kp = v.kp[i];
        } else {
            kp = kp_from_parts<T>(kpp.split[l], kpp.split_part, sigma, p);
            v.kp[i] = kp;
        }
        const T r = v.r[i] + a * kp;
        const T y = v.minv[i] * r;
        v.xt[i] = x;
        v.r[i] = r;
        v.ypc[i] = pair_t<T>{y, p};
        red.s[0] += (double)r * (double)y;
        red.m[0] = amax(red.m[0], absd(r));
    }
    auto fin = [&](const Red<1, 1> &t) {
        if (threadIdx.x != 0) return;
        const double ry_new = t.s[0];
        st->beta = st->ry != 0.0 ? ry_new / st->ry : 0.0;
        st->ry = ry_new;
        st->rnorm = t.m[0];
        st->cg_it += 1;
        st->cg_total += 1;
        const int cont = (!st->device_error && !st->breakdown && isfinite(t.m[0]) && t.m[0] > st->eps_pcg &&
                          st->cg_it < st->max_cg) ? 1 : 0;
        st->pcg_continue = cont;
        if (use_h) cudaGraphSetConditional(hP, cont);
    };
    grid_finish<1, 1>(red, partials, &st->tickets[kTkK3], fin);
}

// ---- single-reduction PCG (Chronopoulos-Gear rearrangement of Algorithm 3)
//
// A step i has two kernels.  sr_direction (SpMV A): with alpha_i, beta_i from
// the previous sr_kapply, every variable forms p_i = -y_i + beta_i p_(i-1),
// s_i = -w_i + beta_i s_(i-1), x_(i+1) = x_i + alpha_i p_i, r_(i+1) = r_i +
// alpha_i s_i, y_(i+1) = M^-1 r_(i+1), and the kernel reduces r'y and
// ||r||_inf of the new r and takes the stopping test; the A SpMV forms
// t = rho A y_(i+1), forming y_(i+1) at each gathered column from the old
// state (r, w, s, M^-1 of step i in one SrVec).  The new state goes to the
// other SrVec buffer, since other CTAs still gather the old one.
// sr_kapply (SpMV [P A']): w_(i+1) = K y_(i+1) = P y + sigma y + A' t, w'y,
// and the coefficients alpha_(i+1), beta_(i+1) (Chronopoulos and Gear, 1989).
// The first pair of a PCG solve runs with alpha = beta = 0 (no step) and
// yields w_0 = K y_0 and alpha_0 = r'y / w'y; the solve's stopping test is
// the one of Section 5.3.4 on each new r.

template <class T>
struct GatherSr {  // y_(i+1) at column c, formed as the owner of c forms it
    const SrVec<T> *S;
    T a, b;
    __device__ __forceinline__ T operator()(int c) const {
        const SrVec<T> g = S[c];
        const T sn = fma_rn(b, g.s, -g.w);
        return mul_rn(g.m, fma_rn(a, sn, g.r));
    }
};

template <class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : 2)
    k_sr_direction(CsrW<T> A, Vecs<T> v, Status *st, double *partials, cudaGraphConditionalHandle hP, int use_h) {
    const T a = T(st->alpha_cg), b = T(st->beta);
    const int par = st->sr_par;
    const SrVec<T> *S = par ? v.sr1 : v.sr0;
    SrVec<T> *Sn = par ? v.sr0 : v.sr1;
    const int n = v.n;
    Red<1, 1> red;
    red.zero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const SrVec<T> g = S[i];
        const T sn = fma_rn(b, g.s, -g.w);
        const T rn = fma_rn(a, sn, g.r);
        const T yn = mul_rn(g.m, rn);
        const T p = fma_rn(b, v.srp[i], -mul_rn(g.m, g.r));
        v.xt[i] = fma_rn(a, p, v.xt[i]);
        v.srp[i] = p;
        Sn[i] = SrVec<T>{rn, T(0), sn, g.m};
        v.pt[i] = yn;
        red.s[0] += (double)rn * (double)yn;
        red.m[0] = amax(red.m[0], absd(rn));
    }
    EpiDir<T> epi{v.pt + n, v.rs, T(st->rho)};
    Red<0, 0> none;
    warp_rows<kU, T, false, true>(A, GatherSr<T>{S, a, b}, epi, none);
    auto fin = [&](const Red<1, 1> &t) {
        if (threadIdx.x != 0) return;
        st->ry_prev = st->ry;
        st->ry = t.s[0];
        st->rnorm = t.m[0];
        if (st->sr_pair > 0) {  // a step was taken
            st->cg_it += 1;
            st->cg_total += 1;
        }
        const int cont = (!st->device_error && !st->breakdown && isfinite(t.m[0]) && t.m[0] > st->eps_pcg &&
                          st->cg_it < st->max_cg) ? 1 : 0;
        st->pcg_continue = cont;
        if (use_h) cudaGraphSetConditional(hP, cont);
    };
    // the sums come from the vector loop only (not from split rows of A)
    grid_finish<1, 1>(red, partials, &st->tickets[kTkSr1], fin);
}

template <class T>
struct EpiSrW {
    Vecs<T> v;
    SrVec<T> *Sn;
    T sigma;
    __device__ __forceinline__ void row(int i, T s1, T, Red<1, 0> &red) {
        const T y = v.pt[i];
        const T w = s1 + sigma * y;
        Sn[i].w = w;
        red.s[0] += (double)w * (double)y;
    }
};

template <class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : 2)
    k_sr_kapply(CsrW<T> PAt, Vecs<T> v, Status *st, double *partials) {
    if (!st->pcg_continue) return;  // the solve stopped at this pair's direction kernel
    const int par = st->sr_par;
    EpiSrW<T> epi{v, par ? v.sr0 : v.sr1, T(st->sigma)};
    Red<1, 0> red;
    red.zero();
    warp_rows<kU, T, false>(PAt, GatherVec<T, T>{v.pt}, epi, red);
    auto fin = [&](const Red<1, 0> &t) {
        if (threadIdx.x != 0) return;
        const double delta = t.s[0], gamma = st->ry;
        double beta = 0.0, den = delta;
        if (st->sr_pair > 0) {
            beta = st->ry_prev != 0.0 ? gamma / st->ry_prev : 0.0;
            den = delta - beta * gamma / st->alpha_cg;
        }
        st->pkp = delta;
        if (den > 0.0 && isfinite(den) && isfinite(beta)) {
            st->alpha_cg = gamma / den;
            st->beta = beta;
        } else {
            st->alpha_cg = 0.0;
            st->beta = 0.0;
            st->breakdown = 1;
        }
        st->sr_pair += 1;
        st->sr_par = par ^ 1;
    };
    grid_finish_w<1, 0>(red, PAt, partials, &st->tickets[kTkSr2], fin);
}

// z~ = A x~;  relaxation, projection, dual update (Algorithm 1 steps 5-7);
// t0 = rho (z~ - z) + y for the next PCG initialisation
template <class T>
struct EpiAdmm {
    Vecs<T> v;
    T alpha, rho, rho_inv;
    __device__ __forceinline__ void row(int j, T s1, T, Red<0, 0> &) {
        const int n = v.n;
        const T zt = s1;
        const T zr = alpha * zt + (T(1) - alpha) * v.z[j];
        const T y = v.xy[n + j];
        T rj = rho, rij = rho_inv;
        if (v.rs) {
            const T sc = v.rs[j];
            rj = rho * sc;
            rij = rho_inv / sc;
        }
        const T zn = clampv(zr + y * rij, v.l[j], v.u[j]);
        const T dy = rj * (zr - zn);
        const T yn = y + dy;
        v.z[j] = zn;
        v.zt[j] = zt;
        v.xy[n + j] = yn;
        v.dxy[n + j] = dy;
        v.xt[n + j] = rj * (zt - zn) + yn;
    }
};

template <class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : 2) k_admm_update(CsrW<T> A, Vecs<T> v, Status *st) {
    const T alpha = T(st->alpha);
    const T rho = T(st->rho);
    const int n = v.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const T x = v.xy[i];
        const T xn = alpha * v.xt[i] + (T(1) - alpha) * x;
        v.xy[i] = xn;
        v.dxy[i] = xn - x;
    }
    EpiAdmm<T> epi{v, alpha, rho, T(1.0 / st->rho)};
    Red<0, 0> red;
    warp_rows<kU, T, false, true>(A, GatherVec<T, T>{v.xt}, epi, red);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->k += 1;
        st->cg_since_update += st->cg_it;
    }
}

// Termination check, part A (rows of A): r_prim = A x - z, FP64 sums.
template <class T>
struct EpiCheckA {
    Vecs<T> v;
    // the six maxima of row j into red.m[M0 .. M0 + 6)
    template <int M0, class R>
    __device__ __forceinline__ void check(int j, double s1, R &red) const {
        const double z = to_acc<double>(v.z[j]);
        const double rp = fabs(s1 - z);
        const double ax = fabs(s1), az = fabs(z);
        const double ei = v.Einv[j];
        red.m[M0 + 0] = amax(red.m[M0 + 0], rp);
        red.m[M0 + 1] = amax(red.m[M0 + 1], ax);
        red.m[M0 + 2] = amax(red.m[M0 + 2], az);
        red.m[M0 + 3] = amax(red.m[M0 + 3], rp * ei);
        red.m[M0 + 4] = amax(red.m[M0 + 4], ax * ei);
        red.m[M0 + 5] = amax(red.m[M0 + 5], az * ei);
    }
    __device__ __forceinline__ void row(int j, double s1, double, Red<0, 6> &red) { check<0>(j, s1, red); }
};

template <class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2) k_check_a(CsrW<T> A, Vecs<T> v, Status *st, double *partials) {
    EpiCheckA<T> epi{v};
    Red<0, 6> red;
    red.zero();
    warp_rows<kU, double, false, true>(A, GatherVec<T, T>{v.xy}, epi, red);
    auto fin = [&](const Red<0, 6> &t) {
        if (threadIdx.x == 0)
            for (int i = 0; i < 6; ++i) st->c1[i] = t.m[i];
    };
    grid_finish_w<0, 6>(red, A, partials, &st->tickets[kTkC1], fin);
}

// Infeasibility detection (Section 3.1), part A (rows of A), on the
// differences of the last iteration: (A dx)_j = E_j^{-1} (A_bar dx_bar)_j
// against the finite bounds; dy_bar clipped to the cone where the support
// function of [l, u] is finite (a component that faces an infinite bound is
// set to zero) and written back for part B; ||dy|| (times c) and the
// support l_bar'(dy_bar)_- + u_bar'(dy_bar)_+ (times c).  Sums in the
// working precision: the tests compare with a relative 1e-4.
template <class T>
struct EpiInfA {
    Vecs<T> v;
    // row j's three maxima into red.m[M0 .. M0 + 3), the support into red.s[0]
    template <int M0, class R>
    __device__ __forceinline__ void detect(int j, T s1, R &red) const {
        const int n = v.n;
        const double ad = to_acc<double>(s1) * v.Einv[j];
        const T l = v.l[j], u = v.u[j];
        const bool lfin = l > -T(INFINITY), ufin = u < T(INFINITY);
        if (ufin) red.m[M0 + 0] = amax(red.m[M0 + 0], ad);    // keeps max(0, ...)
        if (lfin) red.m[M0 + 1] = amax(red.m[M0 + 1], -ad);
        T dy = v.dxy[n + j];
        if (!ufin && dy > T(0)) dy = T(0);
        if (!lfin && dy < T(0)) dy = T(0);
        v.dxy[n + j] = dy;
        red.m[M0 + 2] = amax(red.m[M0 + 2], absd(dy) * v.E[j]);
        if (dy > T(0)) red.s[0] += to_acc<double>(u) * to_acc<double>(dy);
        else if (dy < T(0)) red.s[0] += to_acc<double>(l) * to_acc<double>(dy);
    }
};

#ifndef GB_CHECK_INF_BLOCKS
#define GB_CHECK_INF_BLOCKS 2
#endif

// With detection on, the rows of A of the termination check and of the
// detection in one pass over A that gathers x and dx together: (A x)_j
// summed as k_check_a sums it, (A dx)_j in the working precision as a
// detection pass of its own would sum it (so both results are bitwise
// those of the two separate passes), and A's values and columns read once.
// dx holds the variables' differences only (columns < n); the rows write
// the clipped dy at n + j.
template <class T>
struct EpiCheckInfA {
    Vecs<T> v;
    __device__ __forceinline__ void row(int j, double ax, double adx, Red<1, 9> &red) {
        EpiCheckA<T>{v}.template check<0>(j, ax, red);
        EpiInfA<T>{v}.template detect<6>(j, T(adx), red);
    }
};

template <class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? GB_CHECK_INF_BLOCKS : 2) k_check_inf_a(CsrW<T> A, Vecs<T> v, Status *st, double *partials) {
    static_assert(1 + 9 <= kPartialRecord, "record wider than the partials buffer holds");
    EpiCheckInfA<T> epi{v};
    Red<1, 9> red;
    red.zero();
    warp_rows<kU, double, false, true>(A, GatherDual<T>{v.xy, v.dxy}, epi, red);
    auto fin = [&](const Red<1, 9> &t) {
        if (threadIdx.x != 0) return;
        for (int i = 0; i < 6; ++i) st->c1[i] = t.m[i];
        st->inf_a[0] = t.m[6];
        st->inf_a[1] = t.m[7];
        st->inf_a[2] = t.m[8];
        st->inf_a[3] = t.s[0];
    };
    grid_finish_w<1, 9>(red, A, partials, &st->tickets[kTkC1], fin);
}

// Part B (rows of [P A']): ||D^-1 P_bar dx_bar|| and ||D^-1 A_bar' dy_bar||
// (c times the unscaled ||P dx|| and ||A'dy||), q_bar'dx_bar (c q'dx) and
// ||D dx_bar|| = ||dx||.
template <class T>
struct EpiInfB {
    Vecs<T> v;
    __device__ __forceinline__ void row(int i, T pdx, T atdy, Red<1, 3> &red) {
        const double di = v.Dinv[i];
        const T dx = v.dxy[i];
        red.m[0] = amax(red.m[0], absd(pdx) * di);
        red.m[1] = amax(red.m[1], absd(atdy) * di);
        red.m[2] = amax(red.m[2], absd(dx) * v.D[i]);
        red.s[0] += to_acc<double>(v.q[i]) * to_acc<double>(dx);
    }
};

template <class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2) k_inf_b(CsrW<T> PAt, Vecs<T> v, Status *st, double *partials) {
    EpiInfB<T> epi{v};
    Red<1, 3> red;
    red.zero();
    warp_rows<kU, T, true>(PAt, GatherVec<T, T>{v.dxy}, epi, red);
    auto fin = [&](const Red<1, 3> &t) {
        if (threadIdx.x != 0) return;
        st->inf_b[0] = t.m[0];
        st->inf_b[1] = t.m[1];
        st->inf_b[2] = t.s[0];
        st->inf_b[3] = t.m[2];
    };
    grid_finish_w<1, 3>(red, PAt, partials, &st->tickets[kTkInfB], fin);
}

// The approximate certificate tests of Section 3.1 on the normalised
// differences (the margins of the strict certificate inequalities on the
// safe side, -eps): primal when ||A'dy|| <= eps ||dy|| and support < -eps
// ||dy||; dual when ||P dx|| <= eps ||dx||, q'dx < -eps ||dx|| and A dx
// within eps ||dx|| of the recession cone of [l, u].  Unscaled, dy = E
// dy_bar / c, A'dy = D^-1 A_bar' dy_bar / c and the support carry 1/c, which
// cancels in the primal test; dx = D dx_bar and A dx = E^-1 A_bar dx_bar
// carry none while P dx = D^-1 P_bar dx_bar / c and q'dx = q_bar'dx_bar / c
// do, so the dual test applies 1/c to those two.
__device__ __forceinline__ int infeasibility_status(const Status *st) {
    if (!st->inf_on) return 0;
    const double ndy = st->inf_a[2];
    if (st->eps_pinf > 0.0 && ndy > 0.0 && isfinite(ndy) && st->inf_a[3] < -st->eps_pinf * ndy &&
        st->inf_b[1] <= st->eps_pinf * ndy)
        return GBOSQP_PRIMAL_INFEASIBLE;
    const double ndx = st->inf_b[3];
    const double tol = st->eps_dinf * ndx;
    if (st->eps_dinf > 0.0 && ndx > 0.0 && isfinite(ndx) && st->inf_b[2] * st->cinv < -tol &&
        st->inf_b[0] * st->cinv <= tol && st->inf_a[0] <= tol && st->inf_a[1] <= tol)
        return GBOSQP_DUAL_INFEASIBLE;
    return 0;
}

// Part B (rows of [P A']): r_dual = P x + q + A'y, FP64 sums; objective.
template <class T>
struct EpiCheckB {
    Vecs<T> v;
    __device__ __forceinline__ void row(int i, double px, double aty, Red<1, 6> &red) {
        const double q = to_acc<double>(v.q[i]);
        const double rd = fabs(px + q + aty);
        const double apx = fabs(px), aaty = fabs(aty);
        const double di = v.Dinv[i];
        red.m[0] = amax(red.m[0], rd);
        red.m[1] = amax(red.m[1], apx);
        red.m[2] = amax(red.m[2], aaty);
        red.m[3] = amax(red.m[3], rd * di);
        red.m[4] = amax(red.m[4], apx * di);
        red.m[5] = amax(red.m[5], aaty * di);
        red.s[0] += to_acc<double>(v.xy[i]) * (0.5 * px + q);
    }
};

template <class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2) k_check_b(CsrW<T> PAt, Vecs<T> v, Status *st, double *partials,
                                                      PolicyDev pol, cudaGraphConditionalHandle hA, int use_h) {
    __shared__ double new_rho_sh;
    __shared__ int decide_sh;
    EpiCheckB<T> epi{v};
    Red<1, 6> red;
    red.zero();
    warp_rows<kU, double, true>(PAt, GatherVec<T, T>{v.xy}, epi, red);
    auto fin = [&](const Red<1, 6> &t) {
        if (threadIdx.x == 0) {
            const double cinv = st->cinv;
            st->r_prim = st->c1[kC1RpU];
            st->r_dual = t.m[3] * cinv;
            st->eps_prim = st->eps_abs + st->eps_rel * fmax(st->c1[kC1AxU], st->c1[kC1ZU]);
            st->eps_dual = st->eps_abs + st->eps_rel * cinv * fmax(fmax(t.m[4], t.m[5]), st->qnorm_u);
            st->rp_s = st->c1[kC1RpS];
            st->ax_s = st->c1[kC1AxS];
            st->z_s = st->c1[kC1ZS];
            st->rd_s = t.m[0];
            st->px_s = t.m[1];
            st->aty_s = t.m[2];
            st->obj = t.s[0] * cinv;
            st->rho_changed = 0;
            const bool finite = isfinite(st->r_prim) && isfinite(st->r_dual) && isfinite(st->rp_s) && isfinite(st->rd_s);
            const bool conv = finite && st->r_prim <= st->eps_prim && st->r_dual <= st->eps_dual;
            int status = 0;
            if (!finite || st->device_error) status = GBOSQP_NONFINITE;
            else if (conv) status = GBOSQP_SOLVED;
            else if ((status = infeasibility_status(st)) != 0) {
                st->obj = status == GBOSQP_PRIMAL_INFEASIBLE ? INFINITY : -INFINITY;
            } else if (st->k >= st->max_iter) status = GBOSQP_MAX_ITER;
            st->status = status;
            if (status == 0) {
                st->eps_pcg = fmax(st->lambda * sqrt(st->rp_s * st->rd_s), st->eps_min);
            }
            decide_sh = (status == 0 && st->policy != GBOSQP_RHO_FIXED && st->rho_every > 0 &&
                         st->k % st->rho_every == 0) ? 1 : 0;
            new_rho_sh = st->rho;
        }
        __syncthreads();
        if (decide_sh) {
            if (st->policy == GBOSQP_RHO_LEARNED && pol.params != nullptr) {
                policy_decide(pol, st, &new_rho_sh);  // whole CTA; falls back to the ratio rule
            } else if (threadIdx.x == 0) {
                new_rho_sh = rho_ratio(st);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (decide_sh) {
                const double nr = new_rho_sh;
                if (nr != st->rho && isfinite(nr) && nr > 0.0) {
                    st->rho = nr;
                    st->rho_changed = 1;
                    st->rho_updates += 1;
                }
                st->cg_since_update = 0;
            }
            st->admm_continue = st->status == 0 ? 1 : 0;
            if (use_h) cudaGraphSetConditional(hA, st->admm_continue);
        }
    };
    grid_finish_w<1, 6>(red, PAt, partials, &st->tickets[kTkC2], fin);
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_rho_apply(Vecs<T> v, const Status *st) {
    if (!st->rho_changed) return;
    const double rho = st->rho, sigma = st->sigma;
    const int n = v.n, m = v.m;
    const long long N = n > m ? n : m;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        if (i < n) v.minv[i] = T(1.0 / ((double)v.diagp[i] + sigma + rho * (double)v.colsq[i]));
        if (i < m) v.xt[n + i] = T(rho) * rscale(v, (int)i) * (v.zt[i] - v.z[i]) + v.xy[n + i];
    }
}

// Unscaled output: x = D x_bar, z = z_bar / E, y = E y_bar / c.  For an
// infeasible problem the certificate of unit inf-norm takes the place of y
// (primal: E dy_bar / ||E dy_bar||) or of x (dual: D dx_bar / ||D dx_bar||)
// and the other outputs are NaN.
template <class T>
__global__ void __launch_bounds__(kThreads) k_output(Vecs<T> v, Status *st) {
    const int n = v.n, m = v.m;
    const double cinv = st->cinv;
    const int status = st->status;
    const bool pinf = status == GBOSQP_PRIMAL_INFEASIBLE, dinf = status == GBOSQP_DUAL_INFEASIBLE;
    const double sy = pinf ? 1.0 / st->inf_a[2] : 0.0, sx = dinf ? 1.0 / st->inf_b[3] : 0.0;
    const long long N = n > m ? n : m;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        if (i < n)
            v.x_out[i] = pinf ? (double)NAN : (dinf ? v.D[i] * (double)v.dxy[i] * sx : v.D[i] * (double)v.xy[i]);
        if (i < m) {
            v.z_out[i] = (pinf || dinf) ? (double)NAN : (double)v.z[i] * v.Einv[i];
            v.y_out[i] = dinf ? (double)NAN : (pinf ? v.E[i] * (double)v.dxy[n + i] * sy : v.E[i] * (double)v.xy[n + i] * cinv);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->warm = st->keep_warm;
}

// Generic y = alpha M x (test hook and set-up helpers).
template <class T, class Acc>
struct EpiStore {
    T *y;
    Acc alpha;
    __device__ __forceinline__ void row(int r, Acc s1, Acc s2, Red<0, 0> &) { y[r] = T(alpha * (s1 + s2)); }
};

template <class T, class Acc>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kMinBlocks : 2) k_spmv(CsrW<T> M, const T *x, T *y, Acc alpha) {
    EpiStore<T, Acc> epi{y, alpha};
    Red<0, 0> red;
    warp_rows<kU, Acc, false>(M, GatherVec<T, Acc>{x}, epi, red);
}

template <class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2) k_spmv_dbl(CsrW<T> M, const T *x, double *y) {
    EpiStore<double, double> epi{y, 1.0};
    Red<0, 0> red;
    warp_rows<kU, double, false>(M, GatherVec<T, T>{x}, epi, red);
}

// t0 = rho (zt - z) + y
template <class T>
__global__ void k_t0(Vecs<T> v, double rho) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < v.m) v.xt[v.n + j] = T(rho) * rscale(v, j) * (v.zt[j] - v.z[j]) + v.xy[v.n + j];
}

// Parametric updates: q_bar = c D q, and |q_bar|, |q_bar| / D maxima (on
// the bit patterns of the non-negative values) for the tolerances; a
// non-finite entry sets flag.
__global__ void k_scale_q(double *q, const double *D, double c, int n, unsigned long long *norms, int *flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = q[i];
    if (!isfinite(v)) atomicOr(flag, 1);
    const double s = c * D[i] * v;
    q[i] = s;
    const double a = fabs(s);
    atomicMax(norms, (unsigned long long)__double_as_longlong(a));
    atomicMax(norms + 1, (unsigned long long)__double_as_longlong(a / D[i]));
}

// l_bar = E l, u_bar = E u with |v| >= 1e20 taken as infinite; a missing
// side (nullptr) keeps its current scaled value.  NaN, l > u, l = +inf or
// u = -inf set flag.
template <class T>
__global__ void k_scale_bounds(const double *l, const double *u, const double *E, int m, const T *lcur, const T *ucur,
                               double *lo, double *uo, int *flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double a, b;
    if (l) {
        a = l[i];
        if (a != a) atomicOr(flag, 1);
        a = a <= -kInf ? -INFINITY : (a >= kInf ? INFINITY : a * E[i]);
    } else {
        a = (double)lcur[i];
    }
    if (u) {
        b = u[i];
        if (b != b) atomicOr(flag, 1);
        b = b >= kInf ? INFINITY : (b <= -kInf ? -INFINITY : b * E[i]);
    } else {
        b = (double)ucur[i];
    }
    if (a > b || a == INFINITY || b == -INFINITY) atomicOr(flag, 1);
    lo[i] = a;
    uo[i] = b;
}

// eq. (rho_vec): rs_j = 1e3 where l_j = u_j (scaled bounds), else 1
template <class T>
__global__ void k_rho_scale(const T *l, const T *u, int m, T *rs) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) rs[j] = l[j] == u[j] ? T(1e3) : T(1);
}

// colsq_i = sum_j rs_j A_ji^2 over the A' part of row i of [P A'] (one
// warp per row, FP64 sums): the diagonal of A'RA / rho for the Jacobi
// preconditioner with a rho vector
template <class T>
__global__ void k_colsq_weighted(const int *rowptr, const int *col, const int *pend, const T *val, const T *rs,
                                 int n, T *colsq) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= n) return;
    double acc = 0.0;
    for (int k = pend[w] + lane; k < rowptr[w + 1]; k += 32) {
        const double a = (double)val[k];
        acc += a * a * (double)rs[col[k] - n];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) colsq[w] = T(acc);
}

__global__ void k_recip(const double *in, double *out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = 1.0 / in[i];
}

template <class T>
__global__ void k_minv(Vecs<T> v, double rho, double sigma) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < v.n) v.minv[i] = T(1.0 / ((double)v.diagp[i] + sigma + rho * (double)v.colsq[i]));
}

template <class T>
__global__ void k_from_double(const double *in, T *out, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = T(in[i]);
}

template <class T>
__global__ void k_to_double(const T *in, double *out, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

template <class T>
__global__ void k_neg(T *v, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = -v[i];
}

// Warm start: x_bar = x / D, y_bar = c y / E, z_bar = proj(A_bar x_bar).
template <class T>
__global__ void k_warm(Vecs<T> v, const double *x, const double *y, double c) {
    const int n = v.n, m = v.m;
    const long long N = n > m ? n : m;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        if (i < n) {
            const T xb = x ? T(x[i] / v.D[i]) : T(0);
            v.xy[i] = xb;
            v.xt[i] = xb;
        }
        if (i < m) v.xy[n + i] = y ? T(c * y[i] / v.E[i]) : T(0);
    }
}

template <class T>
__global__ void k_proj_z(Vecs<T> v) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < v.m) v.z[j] = clampv(v.zt[j], v.l[j], v.u[j]);
}

// ----------------------------------------------------- graph construction

template <class... KArgs, class... Args>
cudaGraphNode_t add_kernel_smem(cudaGraph_t g, const cudaGraphNode_t *dep, void (*kern)(KArgs...), int grid,
                                size_t smem, Args &&...args) {
    std::tuple<KArgs...> vals(std::forward<Args>(args)...);
    void *ptrs[sizeof...(KArgs)];
    std::apply([&](auto &...e) {
        int i = 0;
        ((ptrs[i++] = (void *)&e), ...);
    }, vals);
    cudaKernelNodeParams p;
    std::memset(&p, 0, sizeof(p));
    p.func = (void *)kern;
    p.gridDim = dim3(grid > 0 ? grid : 1);
    p.blockDim = dim3(kThreads);
    p.sharedMemBytes = (unsigned)smem;
    p.kernelParams = ptrs;
    cudaGraphNode_t node;
    GB_CUDA(cudaGraphAddKernelNode(&node, g, dep, dep ? 1 : 0, &p));
    return node;
}

template <class... KArgs, class... Args>
cudaGraphNode_t add_kernel(cudaGraph_t g, const cudaGraphNode_t *dep, void (*kern)(KArgs...), int grid,
                           Args &&...args) {
    return add_kernel_smem(g, dep, kern, grid, 0, std::forward<Args>(args)...);
}

cudaGraphNode_t add_while(cudaGraph_t g, const cudaGraphNode_t *dep, cudaGraphConditionalHandle h,
                          cudaGraph_t *body) {
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    GB_CUDA(cudaGraphAddNode(&node, g, dep, nullptr, dep ? 1 : 0, &cp));
    *body = cp.conditional.phGraph_out[0];
    return node;
}

// ------------------------------------------------------- launch geometry

// CTAs of a warp-stream kernel over a matrix with row pointer rp: as many
// as fit at once, fewer for small matrices (about 512 nonzeros per warp).
int grid_for_rows(const std::vector<int> &rp, const void *kernel) {
    int per_sm = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
    const long long work = (rp.empty() ? 0LL : (long long)rp.back()) + 16LL * (long long)(rp.size() - 1);
    const long long want = (work + (long long)kWWarps * 512 - 1) / ((long long)kWWarps * 512);
    return (int)std::max(1LL, std::min<long long>(want, (long long)device_sm_count() * std::max(per_sm, 1)));
}

// The grids of every matrix kernel of a handle in precision T.
struct Grids {
    int pt = 1, admm = 1, ca = 1, ia = 1, spA = 1, sr1 = 1;  // over A
    int kp = 1, init = 1, cb = 1, ib = 1, spP = 1, sr2 = 1;  // over [P A']
    std::vector<int> over_A(bool sr) const {
        std::vector<int> g{pt, admm, ca, ia, spA};
        if (sr) g.push_back(sr1);
        return g;
    }
    std::vector<int> over_PAt(bool sr) const {
        std::vector<int> g{kp, init, cb, ib, spP};
        if (sr) g.push_back(sr2);
        return g;
    }
};

template <class T>
Grids solve_grids(const std::vector<int> &rpA, const std::vector<int> &rpP, bool sr) {
    Grids g;
    g.pt = grid_for_rows(rpA, (const void *)k_pcg_p_t<T>);
    g.admm = grid_for_rows(rpA, (const void *)k_admm_update<T>);
    g.ca = grid_for_rows(rpA, (const void *)k_check_a<T>);
    g.ia = grid_for_rows(rpA, (const void *)k_check_inf_a<T>);
    g.spA = grid_for_rows(rpA, (const void *)k_spmv<T, T>);
    g.kp = grid_for_rows(rpP, (const void *)k_pcg_kp<T>);
    g.init = grid_for_rows(rpP, (const void *)k_pcg_init<T>);
    g.cb = grid_for_rows(rpP, (const void *)k_check_b<T>);
    g.ib = grid_for_rows(rpP, (const void *)k_inf_b<T>);
    g.spP = grid_for_rows(rpP, (const void *)k_spmv<T, T>);
    if (sr) {
        g.sr1 = grid_for_rows(rpA, (const void *)k_sr_direction<T>);
        g.sr2 = grid_for_rows(rpP, (const void *)k_sr_kapply<T>);
    }
    return g;
}

// Host plan of the warp-stream SpMV over a matrix for one grid.
WPlanHost host_plan(const std::vector<int> &rp, int grid) {
    WPlanCost cost;
    cost.bundle_min = kBundleMin;
    cost.group_row = GB_GROUP_ROW;
    return build_wplan(rp, grid * kWWarps, cost);
}

}  // namespace

// Plans started on host threads during set-up (see engine.cuh).
struct PlanPrefetch {
    std::vector<int> rpA, rpP;
    std::vector<std::pair<int, int>> keys;  // (0: A, 1: [P A'], grid)
    std::vector<std::future<WPlanHost>> fut;
    std::vector<WPlanHost> plans;
    void wait() {
        for (auto &f : fut) plans.push_back(f.get());
        fut.clear();
    }
    const WPlanHost *find(int mat, int grid) const {
        for (size_t i = 0; i < plans.size(); ++i)
            if (keys[i] == std::make_pair(mat, grid)) return &plans[i];
        return nullptr;
    }
};

std::shared_ptr<PlanPrefetch> start_plans(const gbosqp_settings &s, std::vector<int> &&A_rp,
                                          std::vector<int> &&PAt_rp) {
    auto pf = std::make_shared<PlanPrefetch>();
    pf->rpA = std::move(A_rp);
    pf->rpP = std::move(PAt_rp);
    const bool sr = s.pcg_variant == GBOSQP_PCG_SINGLE_REDUCTION;
    const Grids g = s.precision == GBOSQP_FP64 ? solve_grids<double>(pf->rpA, pf->rpP, sr)
                                               : solve_grids<float>(pf->rpA, pf->rpP, sr);
    for (int mat = 0; mat < 2; ++mat) {
        const std::vector<int> &rp = mat == 0 ? pf->rpA : pf->rpP;
        for (int grid : (mat == 0 ? g.over_A(sr) : g.over_PAt(sr))) {
            if (std::find(pf->keys.begin(), pf->keys.end(), std::make_pair(mat, grid)) != pf->keys.end()) continue;
            pf->keys.emplace_back(mat, grid);
            pf->fut.push_back(std::async(std::launch::async, host_plan, std::cref(rp), grid));
        }
    }
    return pf;
}

namespace {

// ------------------------------------------------------------------ engine

template <class T>
class Engine final : public EngineBase {
public:
    Engine(SetupData &&sd, const gbosqp_settings &s, cudaStream_t stream, PlanPrefetch *pre) : s_(s), stream_(stream) {
        n = sd.n;
        m = sd.m;
        nnzA = sd.nnzA;
        nnzPAt = sd.nnzPAt;
        nnzP = sd.nnzP;
        c_ = sd.c;
        // matrices in working precision
        A_rowptr_ = std::move(sd.A_rowptr);
        A_col_ = std::move(sd.A_col);
        PAt_rowptr_ = std::move(sd.PAt_rowptr);
        PAt_col_ = std::move(sd.PAt_col);
        PAt_pend_ = std::move(sd.PAt_pend);
        A_val_ = convert(std::move(sd.A_val), nnzA);
        PAt_val_ = convert(std::move(sd.PAt_val), nnzPAt);
        D_ = std::move(sd.D);
        E_ = std::move(sd.E);
        // host row pointers of the work plans (from the plans started during
        // set-up, when there are some)
        matA_.rp = pre ? std::move(pre->rpA) : std::move(sd.A_rowptr_host);
        matPAt_.rp = pre ? std::move(pre->rpP) : std::move(sd.PAt_rowptr_host);
        // vectors
        const size_t nm = (size_t)n + m;
        xy_.alloc(sizeof(T) * std::max<size_t>(nm, 1));
        dxy_.alloc(sizeof(T) * std::max<size_t>(nm, 1));
        xt_.alloc(sizeof(T) * std::max<size_t>(nm, 1));
        pt_.alloc(sizeof(T) * std::max<size_t>(nm, 1));
        for (DevBuf *b : {&z_, &zt_}) b->alloc(sizeof(T) * std::max(m, 1));
        l_ = convert(std::move(sd.l), m);
        u_ = convert(std::move(sd.u), m);
        q_ = convert(std::move(sd.q), n);
        diagp_ = convert(std::move(sd.diagP), n);
        colsq_ = convert(std::move(sd.colsq), n);
        for (DevBuf *b : {&minv_, &kp_, &r_, &tmp_n_}) b->alloc(sizeof(T) * std::max(n, 1));
        ypc_.alloc(sizeof(pair_t<T>) * std::max(n, 1));
        sr_ = s.pcg_variant == GBOSQP_PCG_SINGLE_REDUCTION;
        if (sr_) {
            for (DevBuf *b : {&sr0_, &sr1_}) b->alloc(sizeof(SrVec<T>) * std::max(n, 1));
            srp_.alloc(sizeof(T) * std::max(n, 1));
        }
        tmp_nm_.alloc(sizeof(T) * std::max<size_t>(nm, 1));
        x_out_.alloc(sizeof(double) * std::max(n, 1));
        y_out_.alloc(sizeof(double) * std::max(m, 1));
        z_out_.alloc(sizeof(double) * std::max(m, 1));
        GB_CUDA(cudaMemsetAsync(xy_.p, 0, xy_.bytes, stream_));
        GB_CUDA(cudaMemsetAsync(dxy_.p, 0, dxy_.bytes, stream_));
        Dinv_.alloc(sizeof(double) * std::max(n, 1));
        Einv_.alloc(sizeof(double) * std::max(m, 1));
        if (n) launch(k_recip, ceil_div(n, 256), 256, stream_, D_.as<double>(), Dinv_.as<double>(), (long long)n);
        if (m) launch(k_recip, ceil_div(m, 256), 256, stream_, E_.as<double>(), Einv_.as<double>(), (long long)m);
        GB_CUDA(cudaMemsetAsync(xt_.p, 0, xt_.bytes, stream_));
        GB_CUDA(cudaMemsetAsync(z_.p, 0, z_.bytes, stream_));
        GB_CUDA(cudaMemsetAsync(zt_.p, 0, zt_.bytes, stream_));
        GB_CUDA(cudaMemsetAsync(x_out_.p, 0, x_out_.bytes, stream_));
        GB_CUDA(cudaMemsetAsync(y_out_.p, 0, y_out_.bytes, stream_));
        GB_CUDA(cudaMemsetAsync(z_out_.p, 0, z_out_.bytes, stream_));
        // launch geometry and reduction scratch: each matrix kernel's grid
        // is the CTAs that fit at once, fewer for small matrices
        const Grids G = solve_grids<T>(matA_.rp, matPAt_.rp, sr_);
        gPt_ = G.pt;
        gAdmm_ = G.admm;
        gCa_ = G.ca;
        gIa_ = G.ia;
        gKp_ = G.kp;
        gInit_ = G.init;
        gCb_ = G.cb;
        gIb_ = G.ib;
        if (sr_) {
            gSr1_ = G.sr1;
            gSr2_ = G.sr2;
        }
        // vector kernels: about 4 elements per thread
        const int cap = device_sm_count() * 8;
        gridVec_ = std::max(1, std::min(grid_for_n(n, kThreads), cap));
        gridN_ = std::max(1, std::min(grid_for_n(std::max(n, m), kThreads * 4), cap));
        const int maxgrid = std::max({gPt_, gAdmm_, gCa_, gKp_, gInit_, gCb_, gIa_, gIb_, gridN_, gridVec_, gSr1_, gSr2_});
        build_plans(G.over_A(sr_), G.over_PAt(sr_), pre);
        partials_.alloc(sizeof(double) * (size_t)maxgrid * kPartialRecord);
        // status block
        Status h;
        std::memset(&h, 0, sizeof(h));
        h.sigma = s.sigma;
        h.alpha = s.alpha;
        h.eps_abs = s.eps_abs;
        h.eps_rel = s.eps_rel;
        h.lambda = s.pcg_lambda;
        h.lambda0 = s.pcg_lambda;
        h.eps_min = s.pcg_eps_min;
        h.rho_min = s.rho_min;
        h.rho_max = s.rho_max;
        h.rho0 = s.rho0;
        h.rho = s.rho0;
        h.c = c_;
        h.cinv = 1.0 / c_;
        h.qnorm_s = sd.qnorm_s;
        h.qnorm_u = sd.qnorm_u;
        h.eps0 = std::max(s.pcg_lambda * sd.qnorm_s, s.pcg_eps_min);
        h.eps_pcg = h.eps0;
        h.n = n;
        h.m = m;
        const int ce = s.check_every;
        h.max_iter = ((s.max_iter + ce - 1) / ce) * ce;
        h.max_cg = s.max_cg_iter;
        h.check_every = ce;
        h.rho_every = s.rho_every;
        h.policy = s.rho_policy;
        h.eps_pinf = s.eps_prim_inf;
        h.eps_dinf = s.eps_dual_inf;
        h.inf_on = (s.eps_prim_inf > 0.0 || s.eps_dual_inf > 0.0) ? 1 : 0;
        h.keep_warm = s.warm_start ? 1 : 0;
        inf_on_ = h.inf_on != 0;
        st_.alloc(sizeof(Status));
        st2_.alloc(sizeof(Status));
        GB_CUDA(cudaMemcpyAsync(st_.p, &h, sizeof(h), cudaMemcpyHostToDevice, stream_));
        // learned policy parameters
        if (s.rho_policy == GBOSQP_RHO_LEARNED && s.policy_params) {
            policy_.alloc(sizeof(float) * GBOSQP_POLICY_PARAMS);
            GB_CUDA(cudaMemcpyAsync(policy_.p, s.policy_params, sizeof(float) * GBOSQP_POLICY_PARAMS,
                                    cudaMemcpyHostToDevice, stream_));
        }
        if (s.rho_vector) {
            rs_.alloc(sizeof(T) * std::max(m, 1));
            rho_vector_setup();
        }
        GB_CUDA(cudaStreamSynchronize(stream_));
        if (s.loop_mode == GBOSQP_LOOP_GRAPH) build_graph();
    }

    ~Engine() override {
        if (exec_) cudaGraphExecDestroy(exec_);
        if (graph_) cudaGraphDestroy(graph_);
    }

    // ---------------------------------------------------------- solve
    int solve() override {
        cudaEvent_t e0, e1;
        GB_CUDA(cudaEventCreate(&e0));
        GB_CUDA(cudaEventCreate(&e1));
        GB_CUDA(cudaEventRecord(e0, stream_));
        const long long before = g_launches;
        if (exec_) {
            GB_CUDA(cudaGraphLaunch(exec_, stream_));
        } else {
            host_solve();
        }
        GB_CUDA(cudaEventRecord(e1, stream_));
        GB_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        GB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        solve_ms_ = ms;
        Status h = read_status();
        last_ = h;
        if (h.device_error) fail(GBOSQP_ERR_DEVICE_TIMEOUT, "a bounded device wait gave up");
        solve_launches = g_launches - before;
        if (exec_) {
            // kernels executed by the graph: reset, output, per iteration
            // pcg_init and admm_update, per PCG step three kernels, per
            // check three kernels (four with infeasibility detection: the
            // pass over A takes the detection's rows too, and the
            // detection's pass over [P A'] is added)
            const long long checks = s_.check_every > 0 ? h.k / s_.check_every : 0;
            // single reduction: a pair of kernels per step plus the first pair of each PCG solve
            const long long pcg = sr_ ? 2LL * (h.cg_total + h.k) : 3LL * h.cg_total;
            solve_launches += 2 + 2LL * h.k + pcg + (inf_on_ ? 4LL : 3LL) * checks;
        }
        return h.status;
    }

    void update_rho(double rho) override {
        // the next solve starts from rho; the preconditioner is rebuilt now
        GB_CUDA(cudaMemcpyAsync((char *)st_.p + offsetof(Status, rho0), &rho, sizeof(double), cudaMemcpyHostToDevice,
                                stream_));
        GB_CUDA(cudaMemcpyAsync((char *)st_.p + offsetof(Status, rho), &rho, sizeof(double), cudaMemcpyHostToDevice,
                                stream_));
        launch(k_minv<T>, ceil_div(std::max(n, 1), 256), 256, stream_, vecs(), rho, s_.sigma);
        GB_CUDA(cudaGetLastError());
        GB_CUDA(cudaStreamSynchronize(stream_));
    }

    void warm_start(const double *x, const double *y) override {
        DevBuf xd, yd;
        if (x) {
            xd.alloc(sizeof(double) * std::max(n, 1));
            GB_CUDA(cudaMemcpyAsync(xd.p, x, sizeof(double) * n, cudaMemcpyHostToDevice, stream_));
        }
        if (y) {
            yd.alloc(sizeof(double) * std::max(m, 1));
            GB_CUDA(cudaMemcpyAsync(yd.p, y, sizeof(double) * m, cudaMemcpyHostToDevice, stream_));
        }
        Status h = read_status();
        Vecs<T> v = vecs();
        launch(k_warm<T>, gridN_, kThreads, stream_, v, xd.as<double>(), yd.as<double>(), c_);
        spmv_dev(matA_, A_val_.as<T>(), v.xt, v.zt, T(1));
        launch(k_proj_z<T>, ceil_div(std::max(m, 1), 256), 256, stream_, v);
        launch(k_t0<T>, ceil_div(std::max(m, 1), 256), 256, stream_, v, h.rho0);
        const int one = 1;
        GB_CUDA(cudaMemcpyAsync((char *)st_.p + offsetof(Status, warm), &one, sizeof(int), cudaMemcpyHostToDevice,
                                stream_));
        GB_CUDA(cudaMemcpyAsync((char *)st_.p + offsetof(Status, rho), &h.rho0, sizeof(double), cudaMemcpyHostToDevice,
                                stream_));
        GB_CUDA(cudaGetLastError());
        GB_CUDA(cudaStreamSynchronize(stream_));
    }

    void update_lin_cost(const double *q) override {
        DevBuf qd(sizeof(double) * std::max(n, 1)), norms(2 * sizeof(unsigned long long)), flag(sizeof(int));
        const cudaMemcpyKind kind = s_.input_location == GBOSQP_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (n) GB_CUDA(cudaMemcpyAsync(qd.p, q, sizeof(double) * n, kind, stream_));
        GB_CUDA(cudaMemsetAsync(norms.p, 0, norms.bytes, stream_));
        GB_CUDA(cudaMemsetAsync(flag.p, 0, flag.bytes, stream_));
        if (n) launch(k_scale_q, ceil_div(n, 256), 256, stream_, qd.as<double>(), D_.as<double>(), c_, n,
                      norms.as<unsigned long long>(), flag.as<int>());
        int bad = 0;
        double qn[2] = {0.0, 0.0};
        GB_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, stream_));
        GB_CUDA(cudaMemcpyAsync(qn, norms.p, sizeof(qn), cudaMemcpyDeviceToHost, stream_));
        GB_CUDA(cudaStreamSynchronize(stream_));
        if (bad) fail(GBOSQP_ERR_NONFINITE, "q holds a NaN or an infinite value");
        if (n) launch(k_from_double<T>, ceil_div(n, 256), 256, stream_, qd.as<double>(), q_.as<T>(), (long long)n);
        const double eps0 = std::max(s_.pcg_lambda * qn[0], s_.pcg_eps_min);
        GB_CUDA(cudaMemcpyAsync((char *)st_.p + offsetof(Status, qnorm_s), &qn[0], sizeof(double), cudaMemcpyHostToDevice, stream_));
        GB_CUDA(cudaMemcpyAsync((char *)st_.p + offsetof(Status, qnorm_u), &qn[1], sizeof(double), cudaMemcpyHostToDevice, stream_));
        GB_CUDA(cudaMemcpyAsync((char *)st_.p + offsetof(Status, eps0), &eps0, sizeof(double), cudaMemcpyHostToDevice, stream_));
        GB_CUDA(cudaGetLastError());
        GB_CUDA(cudaStreamSynchronize(stream_));
    }

    void update_bounds(const double *l, const double *u) override {
        if (!m || (!l && !u)) return;
        const cudaMemcpyKind kind = s_.input_location == GBOSQP_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        DevBuf li, ui, lo(sizeof(double) * m), uo(sizeof(double) * m), flag(sizeof(int));
        if (l) {
            li.alloc(sizeof(double) * m);
            GB_CUDA(cudaMemcpyAsync(li.p, l, sizeof(double) * m, kind, stream_));
        }
        if (u) {
            ui.alloc(sizeof(double) * m);
            GB_CUDA(cudaMemcpyAsync(ui.p, u, sizeof(double) * m, kind, stream_));
        }
        GB_CUDA(cudaMemsetAsync(flag.p, 0, flag.bytes, stream_));
        launch(k_scale_bounds<T>, ceil_div(m, 256), 256, stream_, (const double *)li.as<double>(),
               (const double *)ui.as<double>(), E_.as<double>(), m, (const T *)l_.as<T>(), (const T *)u_.as<T>(),
               lo.as<double>(), uo.as<double>(), flag.as<int>());
        int bad = 0;
        GB_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, stream_));
        GB_CUDA(cudaStreamSynchronize(stream_));
        if (bad) fail(GBOSQP_ERR_BOUNDS, "bounds hold a NaN, l > u, l = +inf or u = -inf");
        launch(k_from_double<T>, ceil_div(m, 256), 256, stream_, lo.as<double>(), l_.as<T>(), (long long)m);
        launch(k_from_double<T>, ceil_div(m, 256), 256, stream_, uo.as<double>(), u_.as<T>(), (long long)m);
        if (s_.rho_vector) rho_vector_setup();  // the equality rows may have changed
        GB_CUDA(cudaGetLastError());
        GB_CUDA(cudaStreamSynchronize(stream_));
    }

    void get_solution(double *x, double *y, double *z, bool device) override {
        const cudaMemcpyKind k = device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (x && n) GB_CUDA(cudaMemcpyAsync(x, x_out_.p, sizeof(double) * n, k, stream_));
        if (y && m) GB_CUDA(cudaMemcpyAsync(y, y_out_.p, sizeof(double) * m, k, stream_));
        if (z && m) GB_CUDA(cudaMemcpyAsync(z, z_out_.p, sizeof(double) * m, k, stream_));
        GB_CUDA(cudaStreamSynchronize(stream_));
    }

    void fill_info(gbosqp_info &info) override {
        const Status &h = last_;
        info.status = h.status;
        info.iters = h.k;
        info.pcg_iters = h.cg_total;
        info.obj = h.obj;
        info.r_prim = h.r_prim;
        info.r_dual = h.r_dual;
        info.eps_prim = h.eps_prim;
        info.eps_dual = h.eps_dual;
        info.rho = h.rho;
        info.pcg_eps = h.eps_pcg;
        info.solve_ms = solve_ms_;
        info.rho_updates = h.rho_updates;
        info.policy_fallbacks = h.fallbacks;
        info.nnz_P = nnzP;
        info.nnz_A = nnzA;
    }

    // ------------------------------------------------ inspection / steps
    void get_scaling(double *D, double *E, double *c) override {
        if (D && n) GB_CUDA(cudaMemcpyAsync(D, D_.p, sizeof(double) * n, cudaMemcpyDeviceToHost, stream_));
        if (E && m) GB_CUDA(cudaMemcpyAsync(E, E_.p, sizeof(double) * m, cudaMemcpyDeviceToHost, stream_));
        GB_CUDA(cudaStreamSynchronize(stream_));
        if (c) *c = c_;
    }

    void get_scaled_csr(int which, int64_t *rowptr, int32_t *col, double *val) override {
        const bool isA = which == GBOSQP_MAT_A;
        const int nr = isA ? m : n;
        const long long nnz = isA ? nnzA : nnzPAt;
        const DevBuf &rp = isA ? A_rowptr_ : PAt_rowptr_;
        const DevBuf &cl = isA ? A_col_ : PAt_col_;
        const DevBuf &vl = isA ? A_val_ : PAt_val_;
        if (rowptr) {
            std::vector<int> tmp(nr + 1);
            GB_CUDA(cudaMemcpyAsync(tmp.data(), rp.p, sizeof(int) * (nr + 1), cudaMemcpyDeviceToHost, stream_));
            GB_CUDA(cudaStreamSynchronize(stream_));
            for (int i = 0; i <= nr; ++i) rowptr[i] = tmp[i];
        }
        if (col && nnz) GB_CUDA(cudaMemcpyAsync(col, cl.p, sizeof(int) * nnz, cudaMemcpyDeviceToHost, stream_));
        if (val && nnz) {
            DevBuf d(sizeof(double) * nnz);
            launch(k_to_double<T>, ceil_div(nnz, 256), 256, stream_, vl.as<T>(), d.as<double>(), nnz);
            GB_CUDA(cudaMemcpyAsync(val, d.p, sizeof(double) * nnz, cudaMemcpyDeviceToHost, stream_));
            GB_CUDA(cudaStreamSynchronize(stream_));
        }
        GB_CUDA(cudaStreamSynchronize(stream_));
    }

    void spmv(int which, const double *x, double *y, bool fp64acc) override {
        const bool isA = which == GBOSQP_MAT_A;
        const int nin = isA ? n : n + m;
        const int nout = isA ? m : n;
        DevBuf xd(sizeof(double) * std::max(nin, 1)), xT(sizeof(T) * std::max(nin, 1)), yT(sizeof(T) * std::max(nout, 1)),
            yd(sizeof(double) * std::max(nout, 1));
        if (nin) GB_CUDA(cudaMemcpyAsync(xd.p, x, sizeof(double) * nin, cudaMemcpyHostToDevice, stream_));
        launch(k_from_double<T>, ceil_div(std::max(nin, 1), 256), 256, stream_, xd.as<double>(), xT.as<T>(), nin);
        const MatPlans &pl = isA ? matA_ : matPAt_;
        const T *val = isA ? A_val_.as<T>() : PAt_val_.as<T>();
        if (fp64acc) {
            // FP64 output through a double staging vector
            DevBuf yy(sizeof(double) * std::max(nout, 1));
            const int g = grid_for_rows(pl.rp, (const void *)k_spmv_dbl<T>);
            CsrW<T> M = csr(pl, val, g);
            k_spmv_d(M, xT.as<T>(), yy.as<double>(), g);
            GB_CUDA(cudaMemcpyAsync(y, yy.p, sizeof(double) * nout, cudaMemcpyDeviceToHost, stream_));
        } else {
            spmv_dev(pl, val, xT.as<T>(), yT.as<T>(), T(1));
            launch(k_to_double<T>, ceil_div(std::max(nout, 1), 256), 256, stream_, yT.as<T>(), yd.as<double>(), nout);
            GB_CUDA(cudaMemcpyAsync(y, yd.p, sizeof(double) * nout, cudaMemcpyDeviceToHost, stream_));
        }
        GB_CUDA(cudaGetLastError());
        GB_CUDA(cudaStreamSynchronize(stream_));
    }

    void pcg(double rho, const double *b, const double *x0, double eps, int max_iter, double *x, int *iters,
             double *rnorm) override {
        // r0 = K x0 - b is formed by the PCG-init kernel with x = 0, q = -b,
        // t0 = rho A x0, on private copies of the vectors it reads.
        Vecs<T> v = vecs();
        DevBuf xy(sizeof(T) * std::max(n + m, 1)), xt(sizeof(T) * std::max(n + m, 1)), q(sizeof(T) * std::max(n, 1)),
            minv(sizeof(T) * std::max(n, 1)), bd(sizeof(double) * std::max(n, 1)), zt(sizeof(T) * std::max(m, 1)),
            zz(sizeof(T) * std::max(m, 1));
        GB_CUDA(cudaMemsetAsync(xy.p, 0, xy.bytes, stream_));
        GB_CUDA(cudaMemsetAsync(zz.p, 0, zz.bytes, stream_));
        GB_CUDA(cudaMemcpyAsync(bd.p, b, sizeof(double) * n, cudaMemcpyHostToDevice, stream_));
        launch(k_from_double<T>, ceil_div(std::max(n, 1), 256), 256, stream_, bd.as<double>(), q.as<T>(), n);
        launch(k_neg<T>, ceil_div(std::max(n, 1), 256), 256, stream_, q.as<T>(), n);
        GB_CUDA(cudaMemcpyAsync(bd.p, x0, sizeof(double) * n, cudaMemcpyHostToDevice, stream_));
        launch(k_from_double<T>, ceil_div(std::max(n, 1), 256), 256, stream_, bd.as<double>(), xt.as<T>(), n);
        v.xy = xy.as<T>();
        v.xt = xt.as<T>();
        v.q = q.as<T>();
        v.minv = minv.as<T>();
        v.zt = zt.as<T>();
        v.z = zz.as<T>();
        spmv_dev(matA_, A_val_.as<T>(), v.xt, v.zt, T(1));
        launch(k_t0<T>, ceil_div(std::max(m, 1), 256), 256, stream_, v, rho);
        launch(k_minv<T>, ceil_div(std::max(n, 1), 256), 256, stream_, v, rho, s_.sigma);
        // private status: parameters of the main one, with rho and eps set
        Status h = read_status();
        h.rho = rho;
        h.eps_pcg = eps;
        h.max_cg = max_iter;
        std::memset(h.tickets, 0, sizeof(h.tickets));
        GB_CUDA(cudaMemcpyAsync(st2_.p, &h, sizeof(h), cudaMemcpyHostToDevice, stream_));
        Status *st = st2_.as<Status>();
        launch_init(v, st, 0, 0);
        int it = 0;
        while (read_int(st2_, offsetof(Status, pcg_continue))) {
            launch_step(v, st, 0, 0);
            ++it;
        }
        Status r = read_status(st2_);
        if (iters) *iters = r.cg_it;
        if (rnorm) *rnorm = r.rnorm;
        launch(k_to_double<T>, ceil_div(std::max(n, 1), 256), 256, stream_, v.xt, bd.as<double>(), n);
        GB_CUDA(cudaMemcpyAsync(x, bd.p, sizeof(double) * n, cudaMemcpyDeviceToHost, stream_));
        GB_CUDA(cudaStreamSynchronize(stream_));
        (void)it;
    }

    void set_iterates(const double *x, const double *z, const double *y, const double *xt, double rho) override {
        Vecs<T> v = vecs();
        upload(x, v.xy, n);
        upload(y, v.xy + n, m);
        upload(z, v.z, m);
        upload(xt, v.xt, n);
        spmv_dev(matA_, A_val_.as<T>(), v.xt, v.zt, T(1));
        launch(k_t0<T>, ceil_div(std::max(m, 1), 256), 256, stream_, v, rho);
        launch(k_minv<T>, ceil_div(std::max(n, 1), 256), 256, stream_, v, rho, s_.sigma);
        Status h = read_status();
        h.rho = rho;
        h.k = 0;
        h.cg_total = 0;
        h.status = 0;
        h.rho_changed = 0;
        h.cg_since_update = 0;
        std::memset(h.tickets, 0, sizeof(h.tickets));
        GB_CUDA(cudaMemcpyAsync(st_.p, &h, sizeof(h), cudaMemcpyHostToDevice, stream_));
        GB_CUDA(cudaGetLastError());
        GB_CUDA(cudaStreamSynchronize(stream_));
    }

    void get_iterates(double *x, double *z, double *y, double *xt, double *rho) override {
        Vecs<T> v = vecs();
        download(v.xy, x, n);
        download(v.xy + n, y, m);
        download(v.z, z, m);
        download(v.xt, xt, n);
        if (rho) *rho = read_status().rho;
    }

    int admm_iterations(int k, int *pcg_per_iter) override {
        Vecs<T> v = vecs();
        Status *st = st_.as<Status>();
        int status = 0;
        for (int it = 0; it < k; ++it) {
            launch_init(v, st, 0, 0);
            while (read_int(st_, offsetof(Status, pcg_continue))) launch_step(v, st, 0, 0);
            // PCG steps taken (the single-reduction PCG runs one more kernel pair than steps)
            if (pcg_per_iter) pcg_per_iter[it] = read_int(st_, offsetof(Status, cg_it));
            launch_admm(v, st);
            const int kk = read_int(st_, offsetof(Status, k));
            if (kk % s_.check_every == 0) {
                launch_check(v, st, 0, 0);
                launch_rho(v, st);
                status = read_int(st_, offsetof(Status, status));
                if (status != 0) break;
            }
        }
        GB_CUDA(cudaStreamSynchronize(stream_));
        last_ = read_status();
        return status;
    }

    void check(double *out) override {
        // evaluate on a private copy of the status so the solve state is kept
        Status h = read_status();
        h.policy = GBOSQP_RHO_FIXED;
        std::memset(h.tickets, 0, sizeof(h.tickets));
        GB_CUDA(cudaMemcpyAsync(st2_.p, &h, sizeof(h), cudaMemcpyHostToDevice, stream_));
        Vecs<T> v = vecs();
        launch_check(v, st2_.as<Status>(), 0, 0);
        Status r = read_status(st2_);
        const double vals[GBOSQP_CHECK_FIELDS] = {r.r_prim, r.r_dual, r.eps_prim, r.eps_dual, r.rp_s, r.rd_s,
                                                  r.ax_s,   r.z_s,    r.px_s,     r.aty_s,    r.qnorm_s, r.obj,
                                                  rho_ratio(&r), h.lambda, (double)h.stall_count,
                                                  (double)h.fallbacks};
        std::memcpy(out, vals, sizeof(vals));
    }

    double bench_kernel(int kernel, int reps) override {
        Status h = read_status();
        std::memset(h.tickets, 0, sizeof(h.tickets));
        h.policy = GBOSQP_RHO_FIXED;
        h.pcg_continue = 1;  // the single-reduction K-apply runs only inside a PCG solve
        GB_CUDA(cudaMemcpyAsync(st2_.p, &h, sizeof(h), cudaMemcpyHostToDevice, stream_));
        Status *st = st2_.as<Status>();
        Vecs<T> v = vecs();
        // the timed kernels read and write the solve's vectors; keep a copy
        // of the state they modify and restore it afterwards
        DevBuf save_xy(xy_.bytes), save_xt(xt_.bytes), save_z(z_.bytes), save_zt(zt_.bytes), save_dxy(dxy_.bytes);
        GB_CUDA(cudaMemcpyAsync(save_dxy.p, dxy_.p, dxy_.bytes, cudaMemcpyDeviceToDevice, stream_));
        GB_CUDA(cudaMemcpyAsync(save_xy.p, xy_.p, xy_.bytes, cudaMemcpyDeviceToDevice, stream_));
        GB_CUDA(cudaMemcpyAsync(save_xt.p, xt_.p, xt_.bytes, cudaMemcpyDeviceToDevice, stream_));
        GB_CUDA(cudaMemcpyAsync(save_z.p, z_.p, z_.bytes, cudaMemcpyDeviceToDevice, stream_));
        GB_CUDA(cudaMemcpyAsync(save_zt.p, zt_.p, zt_.bytes, cudaMemcpyDeviceToDevice, stream_));
        auto one = [&]() {
            switch (kernel) {
                case GBOSQP_K_PCG_DIRECTION: launch_smem(k_pcg_p_t<T>, gPt_, kThreads, kSmemT, stream_, csrA(gPt_), v, (const Status *)st); break;
                case GBOSQP_K_PCG_KAPPLY: launch_smem(k_pcg_kp<T>, gKp_, kThreads, kSmemT, stream_, csrPAt(gKp_), v, st, partials_.as<double>()); break;
                case GBOSQP_K_PCG_UPDATE: launch(k_pcg_update<T>, gridVec_, kThreads, stream_, v, st, partials_.as<double>(), kp_parts(), (cudaGraphConditionalHandle)0, 0); break;
                case GBOSQP_K_PCG_INIT: launch_smem(k_pcg_init<T>, gInit_, kThreads, kSmemT, stream_, csrPAt(gInit_), v, st, partials_.as<double>(), (cudaGraphConditionalHandle)0, 0); break;
                case GBOSQP_K_ADMM_UPDATE: launch_smem(k_admm_update<T>, gAdmm_, kThreads, kSmemT, stream_, csrA(gAdmm_), v, st); break;
                case GBOSQP_K_CHECK_A: launch_smem(k_check_a<T>, gCa_, kThreads, kSmemD, stream_, csrA(gCa_), v, st, partials_.as<double>()); break;
                case GBOSQP_K_CHECK_B: launch_smem(k_check_b<T>, gCb_, kThreads, kSmemDS, stream_, csrPAt(gCb_), v, st, partials_.as<double>(), policy(), (cudaGraphConditionalHandle)0, 0); break;
                case GBOSQP_K_INF_A: launch_smem(k_check_inf_a<T>, gIa_, kThreads, kSmemD, stream_, csrA(gIa_), v, st, partials_.as<double>()); break;
                case GBOSQP_K_INF_B: launch_smem(k_inf_b<T>, gIb_, kThreads, kSmemT, stream_, csrPAt(gIb_), v, st, partials_.as<double>()); break;
                case GBOSQP_K_PCG_SR_DIRECTION:
                    if (!sr_) fail(GBOSQP_ERR_INVALID_ARG, "the handle does not use the single-reduction PCG");
                    launch(k_sr_direction<T>, gSr1_, kThreads, stream_, csrA(gSr1_), v, st, partials_.as<double>(), (cudaGraphConditionalHandle)0, 0);
                    break;
                case GBOSQP_K_PCG_SR_KAPPLY:
                    if (!sr_) fail(GBOSQP_ERR_INVALID_ARG, "the handle does not use the single-reduction PCG");
                    launch(k_sr_kapply<T>, gSr2_, kThreads, stream_, csrPAt(gSr2_), v, st, partials_.as<double>());
                    break;
                default: fail(GBOSQP_ERR_INVALID_ARG, "unknown kernel selector");
            }
        };
        one();  // warm-up
        GB_CUDA(cudaStreamSynchronize(stream_));
        // L2 is flushed before every timed launch (a write of twice the L2
        // size): graph A = reps x [flush, kernel], graph B = reps x [flush];
        // the kernel time is (A - B) / reps, host launch cost excluded
        int dev = 0, l2 = 0;
        GB_CUDA(cudaGetDevice(&dev));
        GB_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
        const size_t fbytes = 2 * (size_t)std::max(l2, 1 << 20);
        DevBuf flush(fbytes);
        auto time_graph = [&](bool with_kernel) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            GB_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
            for (int i = 0; i < reps; ++i) {
                GB_CUDA(cudaMemsetAsync(flush.p, i & 0xff, fbytes, stream_));
                if (with_kernel) one();
            }
            GB_CUDA(cudaStreamEndCapture(stream_, &g));
            GB_CUDA(cudaGraphInstantiate(&ge, g, 0));
            GB_CUDA(cudaGraphLaunch(ge, stream_));
            cudaEvent_t e0, e1;
            GB_CUDA(cudaEventCreate(&e0));
            GB_CUDA(cudaEventCreate(&e1));
            GB_CUDA(cudaEventRecord(e0, stream_));
            GB_CUDA(cudaGraphLaunch(ge, stream_));
            GB_CUDA(cudaEventRecord(e1, stream_));
            GB_CUDA(cudaEventSynchronize(e1));
            float t = 0.f;
            GB_CUDA(cudaEventElapsedTime(&t, e0, e1));
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cudaGraphExecDestroy(ge);
            cudaGraphDestroy(g);
            return t;
        };
        const float ms = std::max(0.f, time_graph(true) - time_graph(false));
        GB_CUDA(cudaMemcpyAsync(xy_.p, save_xy.p, xy_.bytes, cudaMemcpyDeviceToDevice, stream_));
        GB_CUDA(cudaMemcpyAsync(dxy_.p, save_dxy.p, dxy_.bytes, cudaMemcpyDeviceToDevice, stream_));
        GB_CUDA(cudaMemcpyAsync(xt_.p, save_xt.p, xt_.bytes, cudaMemcpyDeviceToDevice, stream_));
        GB_CUDA(cudaMemcpyAsync(z_.p, save_z.p, z_.bytes, cudaMemcpyDeviceToDevice, stream_));
        GB_CUDA(cudaMemcpyAsync(zt_.p, save_zt.p, zt_.bytes, cudaMemcpyDeviceToDevice, stream_));
        GB_CUDA(cudaStreamSynchronize(stream_));
        return reps > 0 ? ms / reps : 0.0;
    }

    void resume() override {
        const int two = 2;
        GB_CUDA(cudaMemcpyAsync((char *)st_.p + offsetof(Status, warm), &two, sizeof(int), cudaMemcpyHostToDevice,
                                stream_));
        GB_CUDA(cudaStreamSynchronize(stream_));
    }

    void set_lambda(double lambda, double eps) override {
        GB_CUDA(cudaMemcpyAsync((char *)st_.p + offsetof(Status, lambda), &lambda, sizeof(double),
                                cudaMemcpyHostToDevice, stream_));
        GB_CUDA(cudaMemcpyAsync((char *)st_.p + offsetof(Status, eps_pcg), &eps, sizeof(double),
                                cudaMemcpyHostToDevice, stream_));
        GB_CUDA(cudaStreamSynchronize(stream_));
    }

    void spmv_noalloc(int which, const void *x, void *y, unsigned char *scratch, size_t scratch_bytes) override {
        const bool isA = which == GBOSQP_MAT_A;
        const MatPlans &mp = isA ? matA_ : matPAt_;
        const int g = grid_for_rows(mp.rp, (const void *)k_spmv<T, T>);
        // the plan for this grid was built at set-up; a missing one is an
        // internal error here (building it would allocate)
        auto it = mp.by_grid.find(g);
        if (it == mp.by_grid.end()) fail(GBOSQP_ERR_CUDA, "internal: no SpMV plan for the allocation-free grid");
        const WDev &pd = it->second;
        if (pd.scratch_bytes > scratch_bytes)
            fail(GBOSQP_ERR_UNSUPPORTED, "the matrix's SpMV plan needs " + std::to_string(pd.scratch_bytes) +
                                             " bytes of scratch; the allocation-free SpMV holds " +
                                             std::to_string(scratch_bytes));
        CsrW<T> M = csr(mp, isA ? A_val_.as<T>() : PAt_val_.as<T>(), g);
        // the same layout as the plan's own scratch, in the caller's memory
        M.split_count = reinterpret_cast<int *>(scratch);
        M.split_part = reinterpret_cast<double *>(scratch + pd.off_part);
        M.split_red = reinterpret_cast<double *>(scratch + pd.off_red);
        GB_CUDA(cudaMemsetAsync(scratch, 0, pd.off_part, stream_));  // the tickets start at zero
        launch(k_spmv<T, T>, g, kThreads, stream_, M, static_cast<const T *>(x), static_cast<T *>(y), T(1));
    }

private:
    // Warp-stream plan of one matrix for one grid size: the immutable
    // tables (items, per-warp ranges and split rows) and the zeroed scratch
    // of the split rows (tickets, partial sums, epilogue sums).
    struct WDev {
        DevBuf meta, scratch;
        int nwarps = 0, nsplit = 0;
        size_t off_wpart = 0, off_wsplit = 0, off_split = 0, off_split_of = 0;  // in meta
        size_t off_part = 0, off_red = 0, scratch_bytes = 0;  // in scratch
    };
    struct MatPlans {
        std::vector<int> rp;                     // host row pointers
        mutable std::map<int, WDev> by_grid;     // plans by grid size
    };

    DevBuf convert(DevBuf &&src, long long count) {
        if (sizeof(T) == sizeof(double)) return std::move(src);
        DevBuf out(sizeof(T) * (count + kSlack));  // zeroed slack past the last element, like the set-up arrays
        GB_CUDA(cudaMemsetAsync(out.as<T>() + count, 0, sizeof(T) * kSlack, stream_));
        if (count) launch(k_from_double<T>, ceil_div(count, 256), 256, stream_, src.as<double>(), out.as<T>(), count);
        GB_CUDA(cudaGetLastError());
        return out;  // src is released after the conversion in stream order
    }

    // The plan of matrix mp for a launch of `grid` CTAs (built once per
    // grid size; kernels with the same grid share it).

    // Build the host plans of all the given grids of both matrices on host
    // threads at once, then upload them (the device calls stay on this thread).
    void build_plans(const std::vector<int> &gA, const std::vector<int> &gP, const PlanPrefetch *pre = nullptr) {
        std::vector<std::pair<const MatPlans *, int>> todo;
        for (int g : gA)
            if (!matA_.by_grid.count(g) && std::find(todo.begin(), todo.end(), std::make_pair((const MatPlans *)&matA_, g)) == todo.end())
                todo.emplace_back(&matA_, g);
        for (int g : gP)
            if (!matPAt_.by_grid.count(g) && std::find(todo.begin(), todo.end(), std::make_pair((const MatPlans *)&matPAt_, g)) == todo.end())
                todo.emplace_back(&matPAt_, g);
        std::vector<std::future<WPlanHost>> fut(todo.size());
        std::vector<const WPlanHost *> ready(todo.size(), nullptr);
        for (size_t i = 0; i < todo.size(); ++i) {
            if (pre) ready[i] = pre->find(todo[i].first == &matA_ ? 0 : 1, todo[i].second);
            if (!ready[i]) fut[i] = std::async(std::launch::async, host_plan, std::cref(todo[i].first->rp), todo[i].second);
        }
        for (size_t i = 0; i < todo.size(); ++i) {
            if (ready[i]) {
                plan_for(*todo[i].first, todo[i].second, ready[i]);
            } else {
                WPlanHost hp = fut[i].get();
                plan_for(*todo[i].first, todo[i].second, &hp);
            }
        }
    }

    const WDev &plan_for(const MatPlans &mp, int grid, const WPlanHost *prebuilt = nullptr) const {
        auto it = mp.by_grid.find(grid);
        if (it != mp.by_grid.end()) return it->second;
        const WPlanHost hp = prebuilt ? *prebuilt : host_plan(mp.rp, grid);
        WDev d;
        d.nwarps = hp.nwarps;
        d.nsplit = (int)hp.split.size();
        auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
        d.off_wpart = up16(sizeof(WItem) * hp.items.size());
        d.off_wsplit = d.off_wpart + up16(sizeof(int) * hp.wpart.size());
        d.off_split = d.off_wsplit + up16(sizeof(WSplit) * hp.wsplit.size());
        d.off_split_of = d.off_split + up16(sizeof(SplitRow) * hp.split.size());
        const int nrows = (int)mp.rp.size() - 1;
        const size_t meta_bytes = d.off_split_of + up16(sizeof(int) * std::max(nrows, 1));
        std::vector<unsigned char> h(meta_bytes, 0);
        if (!hp.items.empty()) std::memcpy(h.data(), hp.items.data(), sizeof(WItem) * hp.items.size());
        std::memcpy(h.data() + d.off_wpart, hp.wpart.data(), sizeof(int) * hp.wpart.size());
        std::memcpy(h.data() + d.off_wsplit, hp.wsplit.data(), sizeof(WSplit) * hp.wsplit.size());
        if (!hp.split.empty()) std::memcpy(h.data() + d.off_split, hp.split.data(), sizeof(SplitRow) * hp.split.size());
        {
            int *so = reinterpret_cast<int *>(h.data() + d.off_split_of);
            std::fill(so, so + std::max(nrows, 1), -1);
            for (size_t l = 0; l < hp.split.size(); ++l) so[hp.split[l].row] = (int)l;
        }
        d.meta.alloc(meta_bytes);
        // pageable source: the copy is staged before the call returns
        GB_CUDA(cudaMemcpyAsync(d.meta.p, h.data(), meta_bytes, cudaMemcpyHostToDevice, stream_));
        d.off_part = up16(sizeof(int) * hp.split.size());
        d.off_red = d.off_part + up16(2 * sizeof(double) * (size_t)hp.nslots);
        d.scratch_bytes = d.off_red + up16(kMaxSplitSums * sizeof(double) * hp.split.size());
        d.scratch.alloc(d.scratch_bytes);
        GB_CUDA(cudaMemsetAsync(d.scratch.p, 0, d.scratch.bytes, stream_));
        return mp.by_grid.emplace(grid, std::move(d)).first->second;
    }

    CsrW<T> csr(const MatPlans &mp, const T *val, int grid) const {
        const bool isA = &mp == &matA_;
        const WDev &pd = plan_for(mp, grid);
        const unsigned char *meta = pd.meta.template as<unsigned char>();
        unsigned char *scr = pd.scratch.template as<unsigned char>();
        CsrW<T> M;
        M.nrows = (int)mp.rp.size() - 1;
        M.ncols = isA ? n : n + m;
        M.rowptr = (isA ? A_rowptr_ : PAt_rowptr_).template as<int>();
        M.col = (isA ? A_col_ : PAt_col_).template as<int>();
        M.val = val;
        M.pend = isA ? nullptr : PAt_pend_.template as<int>();
        M.items = reinterpret_cast<const WItem *>(meta);
        M.wpart = reinterpret_cast<const int *>(meta + pd.off_wpart);
        M.wsplit = reinterpret_cast<const WSplit *>(meta + pd.off_wsplit);
        M.split = reinterpret_cast<const SplitRow *>(meta + pd.off_split);
        M.nsplit = pd.nsplit;
        M.split_count = reinterpret_cast<int *>(scr);
        M.split_part = reinterpret_cast<double *>(scr + pd.off_part);
        M.split_red = reinterpret_cast<double *>(scr + pd.off_red);
        M.split_of = reinterpret_cast<const int *>(meta + pd.off_split_of);
        return M;
    }
    // CTAs of a warp-stream kernel: as many as fit at once, fewer when the
    // matrix is small (at least about 512 nonzeros per warp)
    // rs from the scaled bounds, and the weighted column sums it implies
    void rho_vector_setup() {
        if (m) launch(k_rho_scale<T>, ceil_div(m, 256), 256, stream_, (const T *)l_.as<T>(), (const T *)u_.as<T>(), m,
                      rs_.as<T>());
        if (n) launch(k_colsq_weighted<T>, ceil_div((long long)n * 32, 256), 256, stream_, PAt_rowptr_.as<int>(),
                      PAt_col_.as<int>(), PAt_pend_.as<int>(), (const T *)PAt_val_.as<T>(), (const T *)rs_.as<T>(), n,
                      colsq_.as<T>());
        GB_CUDA(cudaGetLastError());
    }

    CsrW<T> csrA(int grid) const { return csr(matA_, A_val_.as<T>(), grid); }
    CsrW<T> csrPAt(int grid) const { return csr(matPAt_, PAt_val_.as<T>(), grid); }
    KpParts kp_parts() const {
        const CsrW<T> M = csrPAt(gKp_);
        return KpParts{M.split_of, M.split, M.split_part};
    }

    Vecs<T> vecs() const {
        Vecs<T> v;
        v.xy = xy_.as<T>();
        v.dxy = dxy_.as<T>();
        v.xt = xt_.as<T>();
        v.pt = pt_.as<T>();
        v.z = z_.as<T>();
        v.zt = zt_.as<T>();
        v.l = l_.as<T>();
        v.u = u_.as<T>();
        v.q = q_.as<T>();
        v.minv = minv_.as<T>();
        v.diagp = diagp_.as<T>();
        v.colsq = colsq_.as<T>();
        v.rs = s_.rho_vector ? rs_.as<T>() : nullptr;
        v.ypc = ypc_.as<pair_t<T>>();
        v.sr0 = sr_ ? sr0_.as<SrVec<T>>() : nullptr;
        v.sr1 = sr_ ? sr1_.as<SrVec<T>>() : nullptr;
        v.srp = sr_ ? srp_.as<T>() : nullptr;
        v.kp = kp_.as<T>();
        v.r = r_.as<T>();
        v.D = D_.as<double>();
        v.E = E_.as<double>();
        v.Dinv = Dinv_.as<double>();
        v.Einv = Einv_.as<double>();
        v.x_out = x_out_.as<double>();
        v.y_out = y_out_.as<double>();
        v.z_out = z_out_.as<double>();
        v.n = n;
        v.m = m;
        return v;
    }

    PolicyDev policy() const {
        PolicyDev p;
        p.params = policy_.as<float>();
        return p;
    }

    void spmv_dev(const MatPlans &pl, const T *val, const T *x, T *y, T alpha) {
        const int g = grid_for_rows(pl.rp, (const void *)k_spmv<T, T>);
        launch_smem(k_spmv<T, T>, g, kThreads, kSmemT, stream_, csr(pl, val, g), x, y, alpha);
        GB_CUDA(cudaGetLastError());
    }
    void k_spmv_d(CsrW<T> M, const T *x, double *y, int g) {
        launch_smem(k_spmv_dbl<T>, g, kThreads, kSmemD, stream_, M, x, y);
        GB_CUDA(cudaGetLastError());
    }

    // ---- host-driven launches (same kernels as the graph)
    void launch_init(const Vecs<T> &v, Status *st, cudaGraphConditionalHandle h, int use_h) {
        launch_smem(k_pcg_init<T>, gInit_, kThreads, kSmemT, stream_, csrPAt(gInit_), v, st, partials_.as<double>(), h, use_h);
        GB_CUDA(cudaGetLastError());
    }
    void launch_step(const Vecs<T> &v, Status *st, cudaGraphConditionalHandle h, int use_h) {
        if (sr_) {
            launch(k_sr_direction<T>, gSr1_, kThreads, stream_, csrA(gSr1_), v, st, partials_.as<double>(), h, use_h);
            launch(k_sr_kapply<T>, gSr2_, kThreads, stream_, csrPAt(gSr2_), v, st, partials_.as<double>());
            GB_CUDA(cudaGetLastError());
            return;
        }
        launch_smem(k_pcg_p_t<T>, gPt_, kThreads, kSmemT, stream_, csrA(gPt_), v, st);
        launch_smem(k_pcg_kp<T>, gKp_, kThreads, kSmemT, stream_, csrPAt(gKp_), v, st, partials_.as<double>());
        launch(k_pcg_update<T>, gridVec_, kThreads, stream_, v, st, partials_.as<double>(), kp_parts(), h, use_h);
        GB_CUDA(cudaGetLastError());
    }
    void launch_admm(const Vecs<T> &v, Status *st) {
        launch_smem(k_admm_update<T>, gAdmm_, kThreads, kSmemT, stream_, csrA(gAdmm_), v, st);
        GB_CUDA(cudaGetLastError());
    }
    void launch_check(const Vecs<T> &v, Status *st, cudaGraphConditionalHandle h, int use_h) {
        if (inf_on_) {  // the check's and the detection's rows of A in one pass
            launch_smem(k_check_inf_a<T>, gIa_, kThreads, kSmemD, stream_, csrA(gIa_), v, st, partials_.as<double>());
            launch_smem(k_inf_b<T>, gIb_, kThreads, kSmemT, stream_, csrPAt(gIb_), v, st, partials_.as<double>());
        } else {
            launch_smem(k_check_a<T>, gCa_, kThreads, kSmemD, stream_, csrA(gCa_), v, st, partials_.as<double>());
        }
        launch_smem(k_check_b<T>, gCb_, kThreads, kSmemDS, stream_, csrPAt(gCb_), v, st, partials_.as<double>(), policy(), h, use_h);
        GB_CUDA(cudaGetLastError());
    }
    void launch_rho(const Vecs<T> &v, Status *st) {
        launch(k_rho_apply<T>, gridN_, kThreads, stream_, v, st);
        GB_CUDA(cudaGetLastError());
    }

    void host_solve() {
        Vecs<T> v = vecs();
        Status *st = st_.as<Status>();
        launch(k_reset<T>, gridN_, kThreads, stream_, v, st, 0, 0);
        GB_CUDA(cudaGetLastError());
        while (read_int(st_, offsetof(Status, admm_continue))) {
            for (int s = 0; s < s_.check_every; ++s) {
                launch_init(v, st, 0, 0);
                while (read_int(st_, offsetof(Status, pcg_continue))) launch_step(v, st, 0, 0);
                launch_admm(v, st);
            }
            launch_check(v, st, 0, 0);
            launch_rho(v, st);
        }
        launch(k_output<T>, gridN_, kThreads, stream_, v, st);
        GB_CUDA(cudaGetLastError());
    }

    // Whole solve as one graph:
    //   reset -> WHILE(admm) { check_every x [pcg_init -> WHILE(pcg)
    //   { p_t -> kp -> update } -> admm_update] -> check_a [-> inf_a ->
    //   inf_b] -> check_b -> rho_apply } -> output
    void build_graph() {
        Vecs<T> v = vecs();
        Status *st = st_.as<Status>();
        double *part = partials_.as<double>();

        GB_CUDA(cudaGraphCreate(&graph_, 0));
        cudaGraphConditionalHandle hA;
        GB_CUDA(cudaGraphConditionalHandleCreate(&hA, graph_, 1, cudaGraphCondAssignDefault));
        cudaGraphNode_t n_reset = add_kernel(graph_, nullptr, k_reset<T>, gridN_, v, st, hA, 1);
        cudaGraph_t body;
        cudaGraphNode_t n_while = add_while(graph_, &n_reset, hA, &body);
        add_kernel(graph_, &n_while, k_output<T>, gridN_, v, st);
        cudaGraphNode_t prev = nullptr;
        for (int s = 0; s < s_.check_every; ++s) {
            cudaGraphConditionalHandle hP;
            GB_CUDA(cudaGraphConditionalHandleCreate(&hP, body, 0, 0));
            cudaGraphNode_t ni = add_kernel_smem(body, prev ? &prev : nullptr, k_pcg_init<T>, gInit_, kSmemT, csrPAt(gInit_), v, st, part, hP, 1);
            cudaGraph_t pbody;
            cudaGraphNode_t nw = add_while(body, &ni, hP, &pbody);
            if (sr_) {
                cudaGraphNode_t a = add_kernel(pbody, nullptr, k_sr_direction<T>, gSr1_, csrA(gSr1_), v, st, part, hP, 1);
                add_kernel(pbody, &a, k_sr_kapply<T>, gSr2_, csrPAt(gSr2_), v, st, part);
            } else {
                cudaGraphNode_t a = add_kernel_smem(pbody, nullptr, k_pcg_p_t<T>, gPt_, kSmemT, csrA(gPt_), v, (const Status *)st);
                cudaGraphNode_t b = add_kernel_smem(pbody, &a, k_pcg_kp<T>, gKp_, kSmemT, csrPAt(gKp_), v, st, part);
                add_kernel(pbody, &b, k_pcg_update<T>, gridVec_, v, st, part, kp_parts(), hP, 1);
            }
            prev = add_kernel_smem(body, &nw, k_admm_update<T>, gAdmm_, kSmemT, csrA(gAdmm_), v, st);
        }
        cudaGraphNode_t ca;
        if (inf_on_) {  // the check's and the detection's rows of A in one pass
            ca = add_kernel_smem(body, &prev, k_check_inf_a<T>, gIa_, kSmemD, csrA(gIa_), v, st, part);
            ca = add_kernel_smem(body, &ca, k_inf_b<T>, gIb_, kSmemT, csrPAt(gIb_), v, st, part);
        } else {
            ca = add_kernel_smem(body, &prev, k_check_a<T>, gCa_, kSmemD, csrA(gCa_), v, st, part);
        }
        cudaGraphNode_t cb = add_kernel_smem(body, &ca, k_check_b<T>, gCb_, kSmemDS, csrPAt(gCb_), v, st, part, policy(), hA, 1);
        add_kernel(body, &cb, k_rho_apply<T>, gridN_, v, (const Status *)st);
        GB_CUDA(cudaGraphInstantiate(&exec_, graph_, 0));
    }

    // ---- small host helpers
    Status read_status() { return read_status(st_); }
    Status read_status(const DevBuf &b) {
        Status h;
        GB_CUDA(cudaMemcpyAsync(&h, b.p, sizeof(h), cudaMemcpyDeviceToHost, stream_));
        GB_CUDA(cudaStreamSynchronize(stream_));
        return h;
    }
    int read_int(const DevBuf &b, size_t off) {
        int v = 0;
        GB_CUDA(cudaMemcpyAsync(&v, (const char *)b.p + off, sizeof(int), cudaMemcpyDeviceToHost, stream_));
        GB_CUDA(cudaStreamSynchronize(stream_));
        return v;
    }
    void upload(const double *src, T *dst, int count) {
        if (!src || count <= 0) return;
        DevBuf d(sizeof(double) * count);
        GB_CUDA(cudaMemcpyAsync(d.p, src, sizeof(double) * count, cudaMemcpyHostToDevice, stream_));
        launch(k_from_double<T>, ceil_div(count, 256), 256, stream_, d.as<double>(), dst, count);
        GB_CUDA(cudaStreamSynchronize(stream_));
    }
    void download(const T *src, double *dst, int count) {
        if (!dst || count <= 0) return;
        DevBuf d(sizeof(double) * count);
        launch(k_to_double<T>, ceil_div(count, 256), 256, stream_, src, d.as<double>(), count);
        GB_CUDA(cudaMemcpyAsync(dst, d.p, sizeof(double) * count, cudaMemcpyDeviceToHost, stream_));
        GB_CUDA(cudaStreamSynchronize(stream_));
    }

    gbosqp_settings s_;
    cudaStream_t stream_;
    double c_ = 1.0;
    DevBuf A_rowptr_, A_col_, A_val_, PAt_rowptr_, PAt_col_, PAt_val_, PAt_pend_;
    DevBuf D_, E_, Dinv_, Einv_;
    DevBuf dxy_, rs_;
    DevBuf xy_, xt_, pt_, z_, zt_, l_, u_, q_, minv_, diagp_, colsq_, kp_, r_, ypc_, tmp_n_, tmp_nm_;
    DevBuf x_out_, y_out_, z_out_;
    DevBuf partials_, st_, st2_, policy_;
    MatPlans matA_, matPAt_;
    int gPt_ = 1, gAdmm_ = 1, gCa_ = 1, gKp_ = 1, gInit_ = 1, gCb_ = 1, gIa_ = 1, gIb_ = 1, gridN_ = 1, gridVec_ = 1;
    int gSr1_ = 1, gSr2_ = 1;
    bool sr_ = false;          // single-reduction PCG
    DevBuf sr0_, sr1_, srp_;
    bool inf_on_ = false;
    // the warp-stream kernels use no dynamic shared memory
    static constexpr size_t kSmemT = 0, kSmemD = 0, kSmemDS = 0;
    cudaGraph_t graph_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
    float solve_ms_ = 0.f;
    Status last_{};
};

}  // namespace

std::unique_ptr<EngineBase> make_engine(SetupData &&sd, const gbosqp_settings &s, cudaStream_t stream,
                                        std::shared_ptr<PlanPrefetch> pre) {
    if (pre) pre->wait();  // every host thread done before the row pointers move
    if (s.precision == GBOSQP_FP64)
        return std::unique_ptr<EngineBase>(new Engine<double>(std::move(sd), s, stream, pre.get()));
    return std::unique_ptr<EngineBase>(new Engine<float>(std::move(sd), s, stream, pre.get()));
}

}  // namespace gb
