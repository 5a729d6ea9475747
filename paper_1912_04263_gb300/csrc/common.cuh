// Shared device and host machinery of the gbosqp library.
//
// * Error handling: host code throws GbError; every extern "C" entry point
//   catches it and returns the code.
// * DevBuf: owning device allocation.
// * Status: the device-resident scalar block of a solve (rho, PCG scalars,
//   check results, flags), so that the iteration loop needs no host
//   round trip (north of Algorithm 1: every decision is taken on the device).
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

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    explicit DevBuf(size_t nbytes) { alloc(nbytes); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t nbytes);
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// -------------------------------------------------------------- constants

constexpr int kThreads = 256;             // CTA size of every row-block kernel
constexpr int kWarps = kThreads / 32;
#ifndef GB_CAP
#define GB_CAP 2048
#endif
constexpr int kCap = GB_CAP;              // max nonzeros per work item
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
    int *err = nullptr;          // set to 1 if a bulk copy wait timed out
};

// ------------------------------------------------------------ status block

enum StatusSlot { kC1RpS = 0, kC1AxS, kC1ZS, kC1RpU, kC1AxU, kC1ZU, kC1N };

struct Status {
    // problem constants
    double sigma, alpha, eps_abs, eps_rel, lambda, eps_min, rho_min, rho_max;
    double rho0, c, cinv, eps0, qnorm_s, qnorm_u;
    int n, m, max_iter, max_cg, check_every, rho_every, policy, warm;
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
    // last-block tickets, one per kernel kind
    unsigned int tickets[16];
};

enum Ticket { kTkI1 = 0, kTkK2, kTkK3, kTkC1, kTkC2, kTkSetupA, kTkSetupB, kTkSetupC, kTkMisc, kTkInfA, kTkInfB };

// ------------------------------------------------------------- reductions

__device__ __forceinline__ double nanmax(double a, double b) {
    return (a != a) ? a : ((b != b) ? b : (a > b ? a : b));
}

// Maximum of two values that are >= 0 (or NaN with a clear sign bit) on
// their encodings: for such values the IEEE-754 order is the integer order
// of the bit patterns, and NaN encodings lie above +inf, so a NaN wins as in
// nanmax.  Runs on the integer pipe (the FP64 pipe is narrow on this GPU).
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

// Row reduction of one block item with lane groups of G threads.  sprod
// holds the item's products; epi.row(r, s1, s2, red) consumes each row.
// With G = 1 every thread sums and finishes its own rows.  With G > 1 the
// groups leave their row sums in rsum and the rows are then finished one
// per thread, so that the epilogue (a chain of dependent loads, and in the
// FP64 checks the expensive arithmetic) runs on all lanes instead of on one
// lane per group; rows are taken in chunks of kThreads.
template <int G, bool SPLIT, class Acc, class T, class Epi, class RedT>
__device__ __forceinline__ void reduce_rows(const CsrDev<T> &M, const Item &it, const T *sprod, Epi &epi,
                                            RedT &red, Acc (*rsum)[kThreads]) {
    const int lane_g = threadIdx.x & (G - 1);
    const int grp = threadIdx.x / G;
    constexpr int ngrp = kThreads / G;
    const int R = it.r1 - it.r0;
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

// Dynamic shared memory of a row-block kernel (the products of one item,
// kept in the working precision; rows accumulate them in Acc).
template <class T, class Acc>
constexpr size_t rowblock_smem() {
    return (size_t)kCap * sizeof(T);
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

// Process the contiguous range of items assigned to this CTA.  Each step
// prefetches the next item's values and columns into registers, then
// multiplies the current item by the gathered vector in the working
// precision (into shared memory) and reduces its rows with lane groups sized
// to the mean row length, accumulating in Acc (FP64 for the termination
// check: FP32 products summed in FP64).
// Consecutive pieces of a long row accumulate per thread and are reduced
// once; a long row that crosses a CTA boundary is combined by the last of
// its contributors, in CTA order.  gather(c) returns the vector entry for
// column c in the accumulation type; epi.row(r, s1, s2, red) consumes rows.
template <class Acc, bool SPLIT, class T, class Gather, class Epi, class RedT>
__device__ __forceinline__ bool run_items(const CsrDev<T> &M, const Gather &gather, Epi &epi, RedT &red) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sprod = reinterpret_cast<T *>(smem_raw);
    __shared__ Acc wsum[2][kWarps];
    __shared__ Acc rsum[SPLIT ? 2 : 1][kThreads];
    const int Q = (M.nitems + (int)gridDim.x - 1) / (int)gridDim.x;
    const int i0 = (int)blockIdx.x * Q;
    const int i1 = min(M.nitems, i0 + Q);
    T va[kPerThread], vb[kPerThread];
    int ca[kPerThread], cb[kPerThread];
    // descriptors run one item ahead of the value/column registers
    Item cur, nx;
    if (i0 < i1) {
        cur = M.items[i0];
        load_item(M, cur, va, ca);
    }
    if (i0 + 1 < i1) nx = M.items[i0 + 1];
    Acc ps1 = Acc(0), ps2 = Acc(0);  // running sums of a long row's pieces
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
            __syncthreads();
        } else {
            const int row = it.r0;
            const int sp = SPLIT ? __ldg(M.pend + row) - it.k0 : 0x7fffffff;
#pragma unroll
            for (int u = 0; u < kPerThread; ++u) {
                const int e = u * kThreads + threadIdx.x;
                if (e < nnz) {
                    const Acc pr = to_acc<Acc>(va[u] * gather(ca[u]));
                    if (!SPLIT || e < sp) ps1 += pr; else ps2 += pr;
                }
            }
            const bool row_end = !has_next || nx.r1 != it.r1;
            if (row_end) {
                Acc s1 = ps1, s2 = ps2;
                ps1 = Acc(0);
                ps2 = Acc(0);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    s1 += __shfl_down_sync(0xffffffffu, s1, o);
                    s2 += __shfl_down_sync(0xffffffffu, s2, o);
                }
                const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
                if (lane == 0) { wsum[0][warp] = s1; wsum[1][warp] = s2; }
                __syncthreads();
                if (threadIdx.x == 0) {
                    double a1 = 0.0, a2 = 0.0;
                    for (int w = 0; w < kWarps; ++w) { a1 += (double)wsum[0][w]; a2 += (double)wsum[1][w]; }
                    const int lr = -(it.r1 + 1);
                    const LongRow L = M.longrows[lr];
                    const int first = L.first_item, last = L.first_item + L.npieces - 1;
                    const int c0 = first / Q, c1 = last / Q;  // CTA ranges covering the row
                    if (c0 == c1) {
                        epi.row(row, Acc(a1), Acc(a2), red);
                    } else {
                        const int slot = max(first, i0);  // this CTA's first piece of the row
                        M.lr_part[2 * (size_t)slot] = a1;
                        M.lr_part[2 * (size_t)slot + 1] = a2;
                        __threadfence();
                        const int t = atomicAdd(M.lr_count + lr, 1);
                        if (t == c1 - c0) {
                            __threadfence();
                            double t1 = 0.0, t2 = 0.0;
                            for (int cc = c0; cc <= c1; ++cc) {
                                const int sl = max(first, cc * Q);
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
