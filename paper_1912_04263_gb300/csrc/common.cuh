// Shared device and host machinery of the gbosqp library.
//
// * Error handling: host code throws GbError; every extern "C" entry point
//   catches it and returns the code.
// * DevBuf: owning device allocation.
// * Status: the device-resident scalar block of a solve (rho, PCG scalars,
//   check results, flags), so that the iteration loop needs no host
//   round trip: every decision of Algorithm 1 is taken on the device.
// * Row-block CSR SpMV: the rows of a CSR matrix are cut at set-up into work
//   items of at most kCap nonzeros (consecutive short rows), and rows longer
//   than kCap are cut into pieces whose partial sums are combined in a fixed
//   order by the last piece to finish.  A CTA streams an item's contiguous
//   value/column range with coalesced loads, multiplies by the gathered
//   vector into shared memory, then reduces each row with a lane group sized
//   to the item's mean row length.  Results are bitwise reproducible.
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

constexpr int kThreads = 256;             // CTA size of every row-block kernel
constexpr int kWarps = kThreads / 32;
#ifndef GB_CAP
#define GB_CAP 2048
#endif
constexpr int kCap = GB_CAP;              // max nonzeros per work item
// Fixed cost of a work item in nonzero-equivalents (descriptor, barriers,
// epilogue latency), used to give every CTA an equal share of the work.
// Measured on GB300 an item costs about the same whatever its nonzero
// count (items of 512 and of 2048 nonzeros take about equally long), so the
// fixed part dominates: CTAs get equal item counts, nonzeros break ties.
#ifndef GB_ITEM_COST
#define GB_ITEM_COST (1 << 20)
#endif
constexpr long long kItemCost = GB_ITEM_COST;
constexpr int kPerThread = kCap / kThreads;
constexpr double kInf = 1e20;             // |bound| >= kInf is infinite

// ------------------------------------------------------------ SpMV items

struct Item {
    int r0;  // first row (block) or the long row (piece)
    int r1;  // one past the last row (block, >= 0) or -(long-row id + 1)
    int k0;  // first nonzero
    int k1;  // one past the last nonzero
};

struct LongRow {
    int first_item;
    int npieces;
};

// Host-side plan of one matrix: items and the long-row table.
struct HostPlan {
    std::vector<Item> items;
    std::vector<LongRow> longrows;
};
HostPlan build_plan(const std::vector<int> &rowptr);

// Assignment of the items to `grid` CTAs: CTA b takes the contiguous range
// [part[b], part[b+1]); every CTA gets at least one item (grid <= items) and
// the ranges have about equal cost (nonzeros + kItemCost per item).
// lr_cta[l] holds the first and last CTA with a piece of long row l.
struct HostPartition {
    std::vector<int> part;
    std::vector<int2> lr_cta;
};
HostPartition partition_items(const HostPlan &hp, int grid);

// Device view of a CSR matrix with its plan.  pend (optional) splits each
// row into two segments [rowptr[r], pend[r]) and [pend[r], rowptr[r+1]).
template <class T>
struct CsrDev {
    int nrows = 0, ncols = 0;
    const int *rowptr = nullptr;
    const int *col = nullptr;
    const T *val = nullptr;
    const int *pend = nullptr;
    const Item *items = nullptr;
    int nitems = 0;
    const LongRow *longrows = nullptr;
    int *lr_count = nullptr;     // one ticket counter per long row (zeroed)
    double *lr_part = nullptr;   // 2 partial sums per item
    const int *part = nullptr;   // grid + 1 item boundaries (see partition_items)
    const int2 *lr_cta = nullptr;  // first and last CTA of each long row
    int *err = nullptr;          // device error flag (no kernel waits today; kept for bounded waits)
};

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

enum Ticket { kTkI1 = 0, kTkK2, kTkK3, kTkC1, kTkC2, kTkSetupA, kTkSetupB, kTkSetupC, kTkMisc, kTkInfA, kTkInfB };

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
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    Red<NS, NM> acc;
    acc.zero();
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int i = 0; i < NS; ++i) acc.s[i] += __ldcg(partials + (size_t)b * NR + i);
#pragma unroll
        for (int i = 0; i < NM; ++i) acc.m[i] = amax(acc.m[i], __ldcg(partials + (size_t)b * NR + NS + i));
    }
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

// ------------------------------------------------------ row-block SpMV core

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

// Row reduction of one block item with lane groups of G threads.  sprod
// holds the item's products; epi.row(r, s1, s2, red) consumes each row.
// With G = 1 every thread sums and finishes its own rows.  With G > 1 the
// groups leave their row sums in rsum and the rows are then finished one
// per thread, so that the epilogue (a chain of dependent loads, and in the
// FP64 checks the expensive arithmetic) runs on all lanes instead of on one
// lane per group; rows are taken in chunks of kThreads.  For FP64 sums the
// G lane partials of a row go through shared memory (over the products,
// once they are read) and one thread adds them in lane order: one FP64 add
// per partial instead of log2(G) shuffle rounds on every lane, the FP64
// pipe being narrow on this GPU.
template <int G, bool SPLIT, class Acc, class T, class Epi, class RedT>
__device__ __forceinline__ void reduce_rows(const CsrDev<T> &M, const Item &it, T *sprod, Epi &epi,
                                            RedT &red, Acc (*rsum)[kThreads]) {
    const int lane_g = threadIdx.x & (G - 1);
    const int grp = threadIdx.x / G;
    constexpr int ngrp = kThreads / G;
    constexpr int kParts = SPLIT ? 2 : 1;
    const int R = it.r1 - it.r0;
    // transposed FP64 reduction when every partial of the item fits over the
    // products (kCap * sizeof(T) bytes)
    constexpr bool kFp64 = sizeof(Acc) == 8 && G > 1;
    constexpr int kRounds = kFp64 ? 4 : 1;  // lane-group rounds kept in registers
    const int nb = (R + ngrp - 1) / ngrp;
    const bool transposed =
        kFp64 && nb <= kRounds && R * G * kParts * (int)sizeof(Acc) <= kCap * (int)sizeof(T);
    if (transposed) {
        LaneSum<Acc, T> p1[kRounds], p2[kRounds];
#pragma unroll
        for (int b = 0; b < kRounds; ++b) {
            const int lr = b * ngrp + grp;
            if (b < nb && lr < R) {
                const int r = it.r0 + lr;
                const int a = __ldg(M.rowptr + r) - it.k0;
                const int e1 = __ldg(M.rowptr + r + 1) - it.k0;
                if (SPLIT) {
                    const int sp = __ldg(M.pend + r) - it.k0;
                    for (int e = a + lane_g; e < e1; e += G) {
                        if (e < sp) p1[b].add(sprod[e]); else p2[b].add(sprod[e]);
                    }
                } else {
                    for (int e = a + lane_g; e < e1; e += G) p1[b].add(sprod[e]);
                }
            }
        }
        __syncthreads();  // every product read: the buffer takes the partials
        Acc *lp = reinterpret_cast<Acc *>(sprod);
#pragma unroll
        for (int b = 0; b < kRounds; ++b) {
            const int lr = b * ngrp + grp;
            if (b < nb && lr < R) {
                lp[lr * G + lane_g] = p1[b].value();
                if (SPLIT) lp[R * G + lr * G + lane_g] = p2[b].value();
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < R; t += kThreads) {
            Acc s1 = Acc(0), s2 = Acc(0);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                s1 += lp[t * G + g];
                if (SPLIT) s2 += lp[R * G + t * G + g];
            }
            epi.row(it.r0 + t, s1, s2, red);
        }
        return;
    }
    for (int c0 = 0; c0 < R; c0 += (G > 1 ? kThreads : R)) {
        const int cn = G > 1 ? min(kThreads, R - c0) : R;
        for (int base = 0; base < cn; base += ngrp) {
            const int lr = base + grp;
            const int r = it.r0 + c0 + lr;
            const bool active = lr < cn;
            Acc s1 = Acc(0), s2 = Acc(0);
            if (active) {
                const int a = __ldg(M.rowptr + r) - it.k0;
                const int b = __ldg(M.rowptr + r + 1) - it.k0;
                if (SPLIT) {
                    const int sp = __ldg(M.pend + r) - it.k0;
                    for (int e = a + lane_g; e < b; e += G) {
                        if (e < sp) s1 += to_acc<Acc>(sprod[e]); else s2 += to_acc<Acc>(sprod[e]);
                    }
                } else {
                    for (int e = a + lane_g; e < b; e += G) s1 += to_acc<Acc>(sprod[e]);
                }
            }
            if (G > 1) {
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) {
                    s1 += __shfl_down_sync(0xffffffffu, s1, o, G);
                    if (SPLIT) s2 += __shfl_down_sync(0xffffffffu, s2, o, G);
                }
                if (active && lane_g == 0) {
                    rsum[0][lr] = s1;
                    if (SPLIT) rsum[1][lr] = s2;
                }
            } else if (active) {
                epi.row(r, s1, s2, red);
            }
        }
        if (G > 1) {
            __syncthreads();
            if ((int)threadIdx.x < cn)
                epi.row(it.r0 + c0 + threadIdx.x, rsum[0][threadIdx.x], SPLIT ? rsum[1][threadIdx.x] : Acc(0), red);
            if (c0 + kThreads < R) __syncthreads();  // rsum is refilled by the next chunk
        }
    }
}

// Whether a row-block kernel double-buffers its products and row sums (no
// closing barrier per item).  Not for FP64 sums of split rows, whose row-sum
// buffers are the largest and where the extra shared memory measured slower.
template <class Acc, bool SPLIT>
constexpr bool rowblock_double_buffered() {
    return !(SPLIT && sizeof(Acc) == 8);
}

// Dynamic shared memory of a row-block kernel: the products of one item
// (two when double-buffered), kept in the working precision; rows
// accumulate them in Acc.
template <class T, class Acc, bool SPLIT = false>
constexpr size_t rowblock_smem() {
    return (rowblock_double_buffered<Acc, SPLIT>() ? 2 : 1) * (size_t)kCap * sizeof(T);
}

// Load the value/column range of an item into registers (streaming loads:
// evict-first, so that L1 keeps the gathered vector).
template <class T>
__device__ __forceinline__ void load_item(const CsrDev<T> &M, const Item &it, T (&v)[kPerThread], int (&c)[kPerThread]) {
    const int nnz = it.k1 - it.k0;
#pragma unroll
    for (int u = 0; u < kPerThread; ++u) {
        const int e = u * kThreads + threadIdx.x;
        if (e < nnz) {
            v[u] = __ldcs(M.val + it.k0 + e);
            c[u] = __ldcs(M.col + it.k0 + e);
        }
    }
}

// Long-row ends pending in a CTA before they are finished together.
constexpr int kRowBatch = 32;

// Finish the pending long-row ends of a CTA, one per thread: add the warp
// partials in warp order, then either consume the row (all its pieces in
// this CTA) or publish this CTA's partial and, if this CTA is the last of
// the row's CTAs to arrive, add every CTA's partial in CTA order and
// consume the row.  Called by every thread of the CTA (it synchronises).
template <class Acc, class T, class Epi, class RedT>
__device__ __forceinline__ void finish_long_rows(const CsrDev<T> &M, int i0, int nq, const int *qlr,
                                                 Acc (*qsum)[2][kWarps], Epi &epi, RedT &red) {
    __syncthreads();
    if ((int)threadIdx.x < nq) {
        const int q = threadIdx.x;
        double a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < kWarps; ++w) {
            a1 += (double)qsum[q][0][w];
            a2 += (double)qsum[q][1][w];
        }
        const int lr = qlr[q];
        const LongRow L = M.longrows[lr];
        const int row = M.items[L.first_item].r0;
        const int first = L.first_item;
        const int2 cr = M.lr_cta[lr];  // CTAs holding pieces of the row
        if (cr.x == cr.y) {
            epi.row(row, Acc(a1), Acc(a2), red);
        } else {
            const int slot = max(first, i0);  // this CTA's first piece of the row
            M.lr_part[2 * (size_t)slot] = a1;
            M.lr_part[2 * (size_t)slot + 1] = a2;
            __threadfence();
            const int t = atomicAdd(M.lr_count + lr, 1);
            if (t == cr.y - cr.x) {
                __threadfence();
                double t1 = 0.0, t2 = 0.0;
                for (int cc = cr.x; cc <= cr.y; ++cc) {
                    const int sl = max(first, M.part[cc]);
                    t1 += __ldcg(M.lr_part + 2 * (size_t)sl);
                    t2 += __ldcg(M.lr_part + 2 * (size_t)sl + 1);
                }
                M.lr_count[lr] = 0;
                epi.row(row, Acc(t1), Acc(t2), red);
            }
        }
    }
    __syncthreads();
}

// Process the contiguous range of items assigned to this CTA.  Each step
// prefetches the next item's values and columns into registers, then
// multiplies the current item by the gathered vector in the working
// precision (into shared memory) and reduces its rows with lane groups sized
// to the mean row length, accumulating in Acc (FP64 for the termination
// check: FP32 products summed in FP64).
// Consecutive pieces of a long row accumulate per thread; at the row's end
// (in this CTA) the warps leave their partials in shared memory and up to
// kRowBatch such row ends are finished together (finish_long_rows); a long
// row that crosses a CTA boundary is combined by the last of its
// contributors, in CTA order.  gather(c) returns the vector entry for
// column c in the accumulation type; epi.row(r, s1, s2, red) consumes rows.
template <class Acc, bool SPLIT, class T, class Gather, class Epi, class RedT>
__device__ __forceinline__ bool run_items(const CsrDev<T> &M, const Gather &gather, Epi &epi, RedT &red) {
    // Products and row sums are double-buffered by item parity: item i+1
    // writes the other buffers while slow threads may still read item i's, and
    // the barrier after item i+1's products orders item i's reads before item
    // i+2 reuses them, so an item needs no closing barrier.  Single-buffered
    // kernels close every item with a barrier instead.
    constexpr bool kDB = rowblock_double_buffered<Acc, SPLIT>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sprod_buf = reinterpret_cast<T *>(smem_raw);
    __shared__ Acc rsum_buf[kDB ? 2 : 1][SPLIT ? 2 : 1][kThreads];
    __shared__ Acc qsum[kRowBatch][2][kWarps];
    __shared__ int qlr[kRowBatch];
    const int i0 = M.part[blockIdx.x];
    const int i1 = M.part[blockIdx.x + 1];
    T va[kPerThread], vb[kPerThread];
    int ca[kPerThread], cb[kPerThread];
    // descriptors run one item ahead of the value/column registers
    Item cur, nx;
    if (i0 < i1) {
        cur = M.items[i0];
        load_item(M, cur, va, ca);
    }
    if (i0 + 1 < i1) nx = M.items[i0 + 1];
    LaneSum<Acc, T> ps1, ps2;  // running sums of a long row's pieces
    int nq = 0;                      // pending long-row ends (uniform in the CTA)
    for (int itx = i0; itx < i1; ++itx) {
        const Item it = cur;
        const bool has_next = itx + 1 < i1;
        Item nx2;
        if (has_next) {
            load_item(M, nx, vb, cb);
            if (itx + 2 < i1) nx2 = M.items[itx + 2];
        }
        const int nnz = it.k1 - it.k0;
        if (it.r1 >= 0) {
            const int buf = kDB ? ((itx - i0) & 1) : 0;
            T *sprod = sprod_buf + buf * kCap;
            Acc(*rsum)[kThreads] = rsum_buf[buf];
#pragma unroll
            for (int u = 0; u < kPerThread; ++u) {
                const int e = u * kThreads + threadIdx.x;
                if (e < nnz) sprod[e] = va[u] * gather(ca[u]);
            }
            __syncthreads();
            const int R = it.r1 - it.r0;
            const int avg = R > 0 ? nnz / R : 0;
            if (avg >= 24) reduce_rows<32, SPLIT, Acc>(M, it, sprod, epi, red, rsum);
            else if (avg >= 12) reduce_rows<16, SPLIT, Acc>(M, it, sprod, epi, red, rsum);
            else if (avg >= 6) reduce_rows<8, SPLIT, Acc>(M, it, sprod, epi, red, rsum);
            else if (avg >= 3) reduce_rows<4, SPLIT, Acc>(M, it, sprod, epi, red, rsum);
            else reduce_rows<1, SPLIT, Acc>(M, it, sprod, epi, red, rsum);
            if (!kDB) __syncthreads();
        } else {
            const int row = it.r0;
            const int sp = SPLIT ? __ldg(M.pend + row) - it.k0 : 0x7fffffff;
#pragma unroll
            for (int u = 0; u < kPerThread; ++u) {
                const int e = u * kThreads + threadIdx.x;
                if (e < nnz) {
                    const T pr = va[u] * gather(ca[u]);
                    if (!SPLIT || e < sp) ps1.add(pr); else ps2.add(pr);
                }
            }
            const bool row_end = !has_next || nx.r1 != it.r1;
            if (row_end) {
                Acc s1 = ps1.value(), s2 = ps2.value();
                ps1 = LaneSum<Acc, T>();
                ps2 = LaneSum<Acc, T>();
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    s1 += __shfl_down_sync(0xffffffffu, s1, o);
                    s2 += __shfl_down_sync(0xffffffffu, s2, o);
                }
                const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
                if (lane == 0) {
                    qsum[nq][0][warp] = s1;
                    qsum[nq][1][warp] = s2;
                }
                if (threadIdx.x == 0) qlr[nq] = -(it.r1 + 1);
                if (++nq == kRowBatch) {
                    finish_long_rows<Acc>(M, i0, nq, qlr, qsum, epi, red);
                    nq = 0;
                }
            }
        }
        if (has_next) {
#pragma unroll
            for (int u = 0; u < kPerThread; ++u) {
                va[u] = vb[u];
                ca[u] = cb[u];
            }
            cur = nx;
            nx = nx2;
        }
    }
    if (nq > 0) finish_long_rows<Acc>(M, i0, nq, qlr, qsum, epi, red);
    return true;
}

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
int grid_for_items(int nitems, const void *kernel, int smem_dynamic = 0);
int grid_for_n(long long n, int threads = kThreads);

}  // namespace gb
