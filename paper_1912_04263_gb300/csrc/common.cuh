// Shared device and host machinery of the gbosqp library.
//
// * Error handling: host code throws GbError; every extern "C" entry point
//   catches it and returns the code.
// * DevBuf: owning device allocation.
// * Status: the device-resident scalar block of a solve (rho, PCG scalars,
//   check results, flags), so that the iteration loop needs no host
//   round trip: every decision of Algorithm 1 is taken on the device.
// * The CSR SpMV core itself (warp-stream kernels and their plan) is in
//   spmv.cuh; this file keeps the reductions it uses.
// * Block reductions with a last-block finalize: per-CTA partials are summed
//   in CTA order by the last CTA to finish (FP64 sums, NaN-propagating max).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/gbosqp.h"

namespace gb {

// ------------------------------------------------------------------ errors

struct GbError {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg);
void check_cuda(cudaError_t e, const char *what, const char *file, int line);
#define GB_CUDA(call) ::gb::check_cuda((call), #call, __FILE__, __LINE__)

// ----------------------------------------------------------------- buffers

// Device buffer.  Inside a PoolScope (osqp_setup) it comes from the
// device's stream-ordered memory pool on the scope's stream and is returned
// to the pool on that stream (no device-wide synchronisation, memory reused
// by the next set-up); elsewhere it is a plain cudaMalloc allocation.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t pool_stream = nullptr;  // set when the buffer came from the pool
    bool pooled = false;
    DevBuf() = default;
    explicit DevBuf(size_t nbytes) { alloc(nbytes); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes), pool_stream(o.pool_stream), pooled(o.pooled) {
        o.p = nullptr;
        o.bytes = 0;
        o.pooled = false;
    }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            bytes = o.bytes;
            pool_stream = o.pool_stream;
            pooled = o.pooled;
            o.p = nullptr;
            o.bytes = 0;
            o.pooled = false;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t nbytes);
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Makes the DevBuf allocations of this host thread stream-ordered on s
// while it lives (nested scopes restore the previous stream).  The stream
// must outlive the buffers allocated in the scope.
struct PoolScope {
    cudaStream_t prev;
    explicit PoolScope(cudaStream_t s);
    ~PoolScope();
};

// -------------------------------------------------------------- constants

constexpr int kThreads = 256;             // CTA size of every kernel of the solve
constexpr int kWarps = kThreads / 32;
constexpr double kInf = 1e20;             // |bound| >= kInf is infinite
// Zeroed elements after the last nonzero of every matrix array the SpMV
// kernels read: a warp loads whole batches of 4 steps of 32 elements, so it
// may load up to 127 elements past its range (those products are
// discarded), and a zero column index keeps the discarded lanes' gathers in
// bounds.
constexpr int kSlack = 128;

// ------------------------------------------------------------ status block

enum StatusSlot { kC1RpS = 0, kC1AxS, kC1ZS, kC1RpU, kC1AxU, kC1ZU, kC1N };

struct Status {
    // problem constants
    double sigma, alpha, eps_abs, eps_rel, lambda, eps_min, rho_min, rho_max;
    double rho0, c, cinv, eps0, qnorm_s, qnorm_u;
    int n, m, max_iter, max_cg, check_every, rho_every, policy;
    int warm;  // 0: cold start; 1: start from the iterates (warm start, rho kept);
               // 2: resume (also keep the PCG tolerance and lambda)
    // evolving
    double rho, eps_pcg;
    double ry, pkp, alpha_cg, beta, rnorm;
    double ry_prev;       // single-reduction PCG: r'y of the previous step
    int sr_par, sr_pair;  // single-reduction PCG: current state buffer, steps begun in this solve
    int cg_it, breakdown, pcg_continue, admm_continue;
    long long cg_total;
    int k, rho_changed, rho_updates, status;
    // termination check
    double c1[kC1N];
    double r_prim, r_dual, eps_prim, eps_dual;
    double rp_s, rd_s, ax_s, z_s, px_s, aty_s, obj;
    // learned policy
    int fallbacks, stall_count, stall_left, policy_disabled;
    double last_merit, prev_merit;
    int cg_since_update, device_error;
    // infeasibility detection (Section 3.1): tolerances, whether the tests
    // run, and the reductions of the two detection kernels
    double eps_pinf, eps_dinf;
    double inf_a[4];  // rows of A: max (A dx)_j [u_j finite], max -(A dx)_j
                      // [l_j finite] (unscaled), ||E dy_bar||, support of dy_bar
    double inf_b[4];  // rows of [P A']: ||D^-1 P_bar dx_bar||, ||D^-1 A_bar' dy_bar||,
                      // q_bar'dx_bar, ||D dx_bar||
    int inf_on;
    int keep_warm;  // 1: each solve starts from the previous solve's iterates
    double lambda0; // the settings' PCG tolerance weight (a solve starts with it)
    // last-block tickets, one per kernel kind
    unsigned int tickets[16];
};

enum Ticket { kTkI1 = 0, kTkK2, kTkK3, kTkC1, kTkC2, kTkSetupA, kTkSetupB, kTkSetupC, kTkMisc, kTkInfA, kTkInfB,
              kTkSr1, kTkSr2 };

// ------------------------------------------------------------- reductions

// Maximum of two values that are >= 0 (or NaN with a clear sign bit) on
// their encodings: for such values the IEEE-754 order is the integer order
// of the bit patterns, and NaN encodings lie above +inf, so a NaN wins (a
// non-finite norm is never hidden).  Runs on the integer pipe (the FP64 pipe
// is narrow on this GPU).
// With one operand >= 0 the result is max(that operand, other) whenever the
// other is >= 0, and that operand when the other is negative.
__device__ __forceinline__ double amax(double a, double b) {
    const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
    return __longlong_as_double(x > y ? x : y);
}

template <int NS, int NM>
struct Red {
    static constexpr int kNS = NS, kNM = NM;
    double s[NS > 0 ? NS : 1];
    double m[NM > 0 ? NM : 1];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < (NS > 0 ? NS : 1); ++i) s[i] = 0.0;
#pragma unroll
        for (int i = 0; i < (NM > 0 ? NM : 1); ++i) m[i] = 0.0;
    }
};

// Reduce red over the CTA; thread 0 returns the CTA total in red.
template <int NS, int NM>
__device__ __forceinline__ void block_reduce(Red<NS, NM> &red) {
    constexpr int NR = NS + NM;
    __shared__ double sred[kWarps][NR > 0 ? NR : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        double v = red.s[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sred[warp][i] = v;
    }
#pragma unroll
    for (int i = 0; i < NM; ++i) {
        double v = red.m[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = amax(v, __shfl_down_sync(0xffffffffu, v, o));
        if (lane == 0) sred[warp][NS + i] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            double a = 0.0;
            for (int w = 0; w < kWarps; ++w) a += sred[w][i];
            red.s[i] = a;
        }
#pragma unroll
        for (int i = 0; i < NM; ++i) {
            double a = 0.0;
            for (int w = 0; w < kWarps; ++w) a = amax(a, sred[w][NS + i]);
            red.m[i] = a;
        }
    }
    __syncthreads();
}

// Adds records b = threadIdx.x, threadIdx.x + blockDim.x, ... (b < count)
// of a table of FP64 records (stride doubles apart; RS sums then RM maxima
// each) into acc, in that order.  The loads of kLd records are issued
// before their sums, so the last CTA of a grid reduction waits for about
// one L2 round trip per kLd records instead of one per record.
template <int NS, int NM, int RS, int RM>
__device__ __forceinline__ void add_records(Red<NS, NM> &acc, const double *tab, int stride, int count) {
    static_assert(RS <= NS && RM <= NM, "record wider than the reduction");
    constexpr int kLd = 4, RR = RS + RM > 0 ? RS + RM : 1;
    for (int b0 = threadIdx.x; b0 < count; b0 += kLd * blockDim.x) {
        double v[kLd][RR];
#pragma unroll
        for (int u = 0; u < kLd; ++u) {
            const int b = b0 + u * (int)blockDim.x;
#pragma unroll
            for (int i = 0; i < RS + RM; ++i) v[u][i] = b < count ? __ldcg(tab + (size_t)b * stride + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kLd; ++u) {
#pragma unroll
            for (int i = 0; i < RS; ++i) acc.s[i] += v[u][i];
#pragma unroll
            for (int i = 0; i < RM; ++i) acc.m[i] = amax(acc.m[i], v[u][RS + i]);
        }
    }
}

// Arrival at a grid-wide ticket, with release and acquire semantics at GPU
// scope: the writes this thread made before (and those other threads of its
// CTA made before a CTA barrier that precedes the call) are visible to every
// thread that arrives later, and the writes published by earlier arrivals
// are visible to this thread and, after a CTA barrier, to its whole CTA.
// Returns the ticket's value before the arrival.  (A full fence before a
// relaxed atomic, and another after it, order the same accesses at more
// cost.)
#ifndef GB_ACQREL
#define GB_ACQREL 1
#endif
__device__ __forceinline__ unsigned int ticket_arrive(unsigned int *t) {
#if GB_ACQREL
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(t) : "memory");
    return old;
#else
    __threadfence();
    const unsigned int old = atomicAdd(t, 1u);
    __threadfence();
    return old;
#endif
}

// Per-CTA partials -> the last CTA to arrive sums them in CTA order and
// calls fin(total) with every thread of that CTA (thread 0 holds nothing
// special; the total is broadcast through shared memory).
template <int NS, int NM, class Fin>
__device__ __forceinline__ void grid_finish(Red<NS, NM> &red, double *partials, unsigned int *ticket,
                                            Fin &fin) {
    constexpr int NR = NS + NM;
    __shared__ bool am_last;
    __shared__ double total[NR > 0 ? NR : 1];
    block_reduce<NS, NM>(red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NS; ++i) partials[(size_t)blockIdx.x * NR + i] = red.s[i];
#pragma unroll
        for (int i = 0; i < NM; ++i) partials[(size_t)blockIdx.x * NR + NS + i] = red.m[i];
        const unsigned int t = ticket_arrive(ticket);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    Red<NS, NM> acc;
    acc.zero();
    add_records<NS, NM, NS, NM>(acc, partials, NR, (int)gridDim.x);
    block_reduce<NS, NM>(acc);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NS; ++i) total[i] = acc.s[i];
#pragma unroll
        for (int i = 0; i < NM; ++i) total[NS + i] = acc.m[i];
        *ticket = 0u;
    }
    __syncthreads();
    Red<NS, NM> tot;
#pragma unroll
    for (int i = 0; i < NS; ++i) tot.s[i] = total[i];
#pragma unroll
    for (int i = 0; i < NM; ++i) tot.m[i] = total[NS + i];
    fin(tot);
}

// ------------------------------------------------------- SpMV arithmetic

// Exact float -> double by rebuilding the IEEE-754 fields (sign, exponent
// rebiased from 127 to 1023, 23-bit significand shifted into the 52-bit
// one) with integer operations; zero, subnormal, inf and NaN inputs take
// the ordinary conversion.  Keeps the conversion off the FP64 pipe, which
// is narrow on this GPU, in the FP64-accumulating SpMVs.
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ex = (u >> 23) & 0xffu;
    if (ex == 0u || ex == 0xffu) return (double)f;
    const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(ex + (1023u - 127u)) << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

template <class Acc, class T>
__device__ __forceinline__ Acc to_acc(T v) { return Acc(v); }
template <>
__device__ __forceinline__ double to_acc<double, float>(float v) { return f2d_exact(v); }

// Per-lane running sum of products of type T in the accumulation type Acc.
// For FP32 products summed in FP64 (the termination checks) a lane keeps a
// compensated FP32 pair instead: Knuth's error-free TwoSum turns each
// addition into a rounded sum and its exact rounding error, the errors are
// summed separately, and the pair is converted to FP64 once (the summation
// of Ogita, Rump and Oishi, "Accurate sum and dot product", 2005: as
// accurate as summing in twice the working precision).  GB300's FP64 pipe is
// narrow; this moves the per-product additions to the FP32 pipe while the
// lane sums are still combined in FP64.
template <class Acc, class T>
struct LaneSum {
    Acc s = Acc(0);
    __device__ __forceinline__ void add(T x) { s += to_acc<Acc>(x); }
    __device__ __forceinline__ Acc value() const { return s; }
};
template <>
struct LaneSum<double, float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = __fadd_rn(s, x);
        const float xp = __fsub_rn(t, s);
        const float sp = __fsub_rn(t, xp);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, sp), __fsub_rn(x, xp)));
        s = t;
    }
    __device__ __forceinline__ double value() const { return f2d_exact(s) + f2d_exact(c); }
};

// ------------------------------------------------------------- utilities

// Kernel launches issued by this host thread (for the launch count the
// library reports; CUDA graph executions are counted from the solve's
// iteration counters instead).
extern thread_local long long g_launches;

// Launch kern<<<grid, block, smem, stream>>>(args...) and count it.
template <class... KArgs, class... Args>
inline void launch_smem(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t stream,
                        Args &&...args) {
    std::tuple<KArgs...> vals(std::forward<Args>(args)...);
    void *ptrs[sizeof...(KArgs) > 0 ? sizeof...(KArgs) : 1];
    std::apply([&](auto &...e) {
        int i = 0;
        ((ptrs[i++] = (void *)&e), ...);
    }, vals);
    ++g_launches;
    GB_CUDA(cudaLaunchKernel((const void *)kern, dim3(grid > 0 ? grid : 1), dim3(block), ptrs, smem, stream));
}

template <class... KArgs, class... Args>
inline void launch(void (*kern)(KArgs...), int grid, int block, cudaStream_t stream, Args &&...args) {
    launch_smem(kern, grid, block, 0, stream, std::forward<Args>(args)...);
}

__host__ __device__ __forceinline__ int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

int device_sm_count();
int grid_for_n(long long n, int threads = kThreads);

}  // namespace gb
