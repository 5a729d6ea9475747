// Device set-up of a QP (paper Section 5.2 "Representation of Matrices" and
// Section 5.4 "Matrix Equilibration"):
//   1. validation of the CSR inputs and bounds (device kernels, one flag word)
//   2. A' in CSR by a stable LSD radix sort of A's nonzeros by column
//      (so every row of A' is sorted; its row pointer comes from the sorted
//      keys), and the full P from its upper triangle as U'(strictly lower
//      part) followed by U, row by row
//   3. Ruiz equilibration, Algorithm 2, in FP64: column inf-norms of
//      M_bar = [[P_bar, A_bar'], [A_bar, 0]] as row norms of P, A' and A (a
//      segmented max over CSR rows, Section 5.4.1) with the scaling so far
//      applied on the fly (P_bar = c D P D, A_bar = E A D), the scaling
//      delta = 1/sqrt(norm) accumulated into D and E, and the cost scaling
//      gamma accumulated into c; the pre- and post-multiplication of P, A
//      and A' by the diagonal matrices (Sections 5.4.2-5.4.3) is done once,
//      after the last pass, instead of once per pass
//   4. the concatenated [P_bar A_bar'] (row i: row i of P_bar, then row i
//      of A_bar' with columns offset by n), diag(P_bar) and the squared
//      column norms of A_bar for the Jacobi preconditioner (Section 5.3.1)
// Everything after the input copy stays on the device; the host reads one
// validation word and the row pointers used to build the SpMV work plans.
#include <math.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "engine.cuh"

namespace gb {

namespace {

constexpr int kScanBlock = 1024;
constexpr int kRsWarps = 8;
constexpr int kRsPerLane = 32;
constexpr int kRsTile = 32 * kRsPerLane;

enum Flag {
    kFlagRowptr = 1,
    kFlagColRange = 2,
    kFlagColOrder = 4,
    kFlagValue = 8,
    kFlagLower = 16,
    kFlagQ = 32,
    kFlagBounds = 64,
};

// Stream-ordered temporary allocation.
struct Tmp {
    void *p = nullptr;
    cudaStream_t s;
    Tmp(size_t bytes, cudaStream_t st) : s(st) {
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMallocAsync(&p, bytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(GBOSQP_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
        }
    }
    ~Tmp() {
        if (p) cudaFreeAsync(p, s);
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// A second stream that runs beside st: fork() makes it wait for st's work
// so far and returns it; join() makes st wait for what was queued on it.
struct SideStream {
    cudaStream_t st, side = nullptr;
    cudaEvent_t forked = nullptr, joined = nullptr;
    explicit SideStream(cudaStream_t s) : st(s) {
        GB_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        GB_CUDA(cudaEventCreateWithFlags(&forked, cudaEventDisableTiming));
        GB_CUDA(cudaEventCreateWithFlags(&joined, cudaEventDisableTiming));
    }
    ~SideStream() {
        if (joined) cudaEventDestroy(joined);
        if (forked) cudaEventDestroy(forked);
        if (side) cudaStreamDestroy(side);
    }
    SideStream(const SideStream &) = delete;
    SideStream &operator=(const SideStream &) = delete;
    cudaStream_t fork() {
        GB_CUDA(cudaEventRecord(forked, st));
        GB_CUDA(cudaStreamWaitEvent(side, forked, 0));
        return side;
    }
    void join() {
        GB_CUDA(cudaEventRecord(joined, side));
        GB_CUDA(cudaStreamWaitEvent(st, joined, 0));
    }
};

inline int blocks_for(long long n, int threads) { return (int)std::max(1LL, (n + threads - 1) / threads); }
inline int warp_blocks(long long rows) { return (int)std::max(1LL, (rows + kWarps - 1) / kWarps); }

// ------------------------------------------------------------ validation

__global__ void k_check_rowptr(const int64_t *rp, int nrows, long long nnz, int *flags) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0 && (rp[0] != 0 || rp[nrows] != nnz)) atomicOr(flags, kFlagRowptr);
    if (r < nrows && rp[r + 1] < rp[r]) atomicOr(flags, kFlagRowptr);
}

__global__ void k_rowptr_i32(const int64_t *in, int n1, int *out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) out[i] = (int)in[i];
}

// One warp per row: columns in range, strictly increasing, finite values,
// and (upper) no entry below the diagonal.
__global__ void k_check_rows(const int *rp, const int *col, const double *val, int nrows, int ncols,
                             int upper, int *flags) {
    const int row = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= nrows) return;
    int bad = 0;
    for (int k = rp[row] + lane; k < rp[row + 1]; k += 32) {
        const int c = col[k];
        if (c < 0 || c >= ncols) bad |= kFlagColRange;
        if (k > rp[row] && col[k - 1] >= c) bad |= kFlagColOrder;
        if (!isfinite(val[k])) bad |= kFlagValue;
        if (upper && c < row) bad |= kFlagLower;
    }
    if (bad) atomicOr(flags, bad);
}

// Infinite-bound convention: |v| >= 1e20 is +-inf.
__global__ void k_check_vectors(const double *q, int n, const double *l, const double *u, int m, double *qd,
                                double *ld, double *ud, int *flags) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double v = q[i];
        if (!isfinite(v)) atomicOr(flags, kFlagQ);
        qd[i] = v;
    }
    if (i < m) {
        double a = l[i], b = u[i];
        if (a != a || b != b || a > b) atomicOr(flags, kFlagBounds);
        if (a <= -kInf) a = -INFINITY;
        if (a >= kInf) a = INFINITY;
        if (b >= kInf) b = INFINITY;
        if (b <= -kInf) b = -INFINITY;
        if (a == INFINITY || b == -INFINITY) atomicOr(flags, kFlagBounds);
        ld[i] = a;
        ud[i] = b;
    }
}

// ------------------------------------------------------------ row tiers
// The row-wise set-up passes share the rows out by length (counted over the
// one or two matrices a pass reads): a thread to each row of at most
// kThreadRow nonzeros, a warp to each row of at most kLongRow, and a CTA to
// each longer row.  The warp and CTA rows are listed once per matrix, so
// that neither the many short rows (one or two nonzeros in the Lasso's
// [P A']) nor a few very long ones (its columns of D, as rows of A') leave
// the GPU running a handful of busy lanes.  Maxima and elementwise passes
// give the same results on every tier; sums are added in a fixed order.
constexpr int kThreadRow = 16;
constexpr int kLongRow = 2048;
enum Tier { kTierThread = 0, kTierWarp = 1, kTierCta = 2 };

struct LongRows {
    DevBuf flag;           // per row: its Tier
    DevBuf list, count;    // the CTA rows, in no particular order, and how many
    DevBuf wlist, wcount;  // the warp rows
    int grid = 1;          // CTAs of the CTA-row kernels
};

__global__ void k_long_rows(const int *rp1, const int *rp2, int nrows, int *flag, int *list, int *count, int *wlist,
                            int *wcount) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    int len = rp1[i + 1] - rp1[i];
    if (rp2) len += rp2[i + 1] - rp2[i];
    const int f = len > kLongRow ? kTierCta : len > kThreadRow ? kTierWarp : kTierThread;
    flag[i] = f;
    if (f == kTierCta) list[atomicAdd(count, 1)] = i;
    if (f == kTierWarp) wlist[atomicAdd(wcount, 1)] = i;
}

LongRows long_rows(const int *rp1, const int *rp2, int nrows, long long nnz, cudaStream_t st) {
    LongRows L;
    L.flag.alloc(sizeof(int) * (size_t)std::max(nrows, 1));
    L.list.alloc(sizeof(int) * (size_t)std::max(nrows, 1));
    L.wlist.alloc(sizeof(int) * (size_t)std::max(nrows, 1));
    L.count.alloc(sizeof(int));
    L.wcount.alloc(sizeof(int));
    GB_CUDA(cudaMemsetAsync(L.count.p, 0, sizeof(int), st));
    GB_CUDA(cudaMemsetAsync(L.wcount.p, 0, sizeof(int), st));
    GB_CUDA(cudaMemsetAsync(L.flag.p, 0, L.flag.bytes, st));
    if (nrows > 0) launch(k_long_rows, blocks_for(nrows, 256), 256, st, rp1, rp2, nrows, L.flag.as<int>(),
                          L.list.as<int>(), L.count.as<int>(), L.wlist.as<int>(), L.wcount.as<int>());
    // at most nnz / kLongRow rows are long
    L.grid = (int)std::max(1LL, std::min<long long>(nnz / kLongRow + 1, (long long)device_sm_count() * 8));
    return L;
}

// CTAs of a warp-row kernel: as many as fit on the GPU at once, and no more
// than one warp per row.
int resident_grid(const void *kernel, long long nrows) {
    int per_sm = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
    const long long cap = (long long)device_sm_count() * std::max(per_sm, 1);
    return (int)std::max(1LL, std::min<long long>((nrows + kWarps - 1) / kWarps, cap));
}

// Maximum of non-negative doubles on their bit patterns (integer pipe).
__device__ __forceinline__ double nmax(double a, double b) {
    const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
    return __longlong_as_double(x > y ? x : y);
}

// max_k |val[k]| sc[col[k]] over k in [k0, k1) taken by the thread t of a
// group of S threads (k = k0 + t, k0 + t + S, ...), with kLd entries
// loaded before their products are taken.  The CTA-row kernels take kLd =
// 4 so that 8 CTAs fit on an SM and every long row of a pass runs at once.
template <int kLd = 8>
__device__ __forceinline__ double strided_scaled_max(const int *col, const double *val, const double *sc, int k0,
                                                     int k1, int t, int S) {
    double mx = 0.0;
    for (int k = k0 + t; k < k1; k += kLd * S) {
        double v[kLd];
        int c[kLd];
#pragma unroll
        for (int u = 0; u < kLd; ++u) {
            const int e = k + u * S;
            v[u] = e < k1 ? val[e] : 0.0;
            c[u] = e < k1 ? col[e] : -1;
        }
        double g[kLd];
#pragma unroll
        for (int u = 0; u < kLd; ++u) g[u] = c[u] >= 0 ? sc[c[u]] : 0.0;
#pragma unroll
        for (int u = 0; u < kLd; ++u) mx = nmax(mx, fabs(v[u]) * g[u]);
    }
    return mx;
}

// Maxima of non-negative doubles and sums over a CTA, in a fixed order;
// every thread gets the result.
__device__ double block_max(double v) {
    __shared__ double sh[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = nmax(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = sh[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r = nmax(r, sh[k]);
    return r;
}
__device__ double block_sum(double v) {
    __shared__ double sh[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = sh[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    return r;
}

// ----------------------------------------------------------------- scan

__global__ void k_scan_block(const int *in, int n, int *out, int *bsum) {
    __shared__ int wsum[32];
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = i < n ? in[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    const int incl = x + (w > 0 ? wsum[w - 1] : 0);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = incl;
}

__global__ void k_scan_add(int *out, int n, const int *boff) {
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) out[i] += boff[blockIdx.x];
}

__global__ void k_copy_int(int *dst, const int *src) { *dst = *src; }
__global__ void k_zero_int(int *dst) { *dst = 0; }

// out[0..n) = exclusive prefix sums of in, out[n] = total.
void exclusive_scan(const int *in, int n, int *out, cudaStream_t st) {
    if (n <= 0) {
        launch(k_zero_int, 1, 1, st, out);
        return;
    }
    const int nb = ceil_div(n, kScanBlock);
    Tmp bsum((size_t)nb * sizeof(int), st);
    launch(k_scan_block, nb, kScanBlock, st, in, n, out, bsum.as<int>());
    if (nb == 1) {
        launch(k_copy_int, 1, 1, st, out + n, bsum.as<int>());
    } else {
        Tmp boff((size_t)(nb + 1) * sizeof(int), st);
        exclusive_scan(bsum.as<int>(), nb, boff.as<int>(), st);
        launch(k_scan_add, nb, kScanBlock, st, out, n, boff.as<int>());
        launch(k_copy_int, 1, 1, st, out + n, boff.as<int>() + nb);
    }
    GB_CUDA(cudaGetLastError());
}

// ------------------------------------------------------ radix sort by key

__global__ void k_iota(int *v, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int)i;
}

// Digits of up to kRsMaxBits bits: the key bits are split into as few
// passes as that allows, of about equal width (17-bit column indices: two
// passes of 9 and 8 bits instead of three of 8).
constexpr int kRsMaxBits = 9;
constexpr int kRsMaxDigits = 1 << kRsMaxBits;

__global__ void k_radix_hist(const int *keys, long long nnz, int shift, int bits, int ntiles, int *H) {
    __shared__ int hist[kRsWarps][kRsMaxDigits];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kRsWarps + w;
    const int nd = 1 << bits, mask = nd - 1;
    for (int d = lane; d < nd; d += 32) hist[w][d] = 0;
    __syncwarp();
    if (tile >= ntiles) return;
    const long long base = (long long)tile * kRsTile;
    for (int it = 0; it < kRsPerLane; ++it) {
        const long long k = base + it * 32 + lane;
        if (k < nnz) atomicAdd(&hist[w][(keys[k] >> shift) & mask], 1);
    }
    __syncwarp();
    for (int d = lane; d < nd; d += 32) H[(size_t)d * ntiles + tile] = hist[w][d];
}

// Stable scatter: each warp walks its tile in order; equal digits within a
// 32-key step are ranked by lane, and a per-warp running count per digit
// carries the order across steps.
__global__ void k_radix_scatter(const int *kin, const int *vin, long long nnz, int shift, int bits, int ntiles,
                                const int *offs, int *kout, int *vout) {
    __shared__ int cnt[kRsWarps][kRsMaxDigits];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kRsWarps + w;
    const int nd = 1 << bits, mask = nd - 1;
    for (int d = lane; d < nd; d += 32) cnt[w][d] = 0;
    __syncwarp();
    if (tile >= ntiles) return;
    const long long base = (long long)tile * kRsTile;
    for (int it = 0; it < kRsPerLane; ++it) {
        const long long k = base + it * 32 + lane;
        const bool valid = k < nnz;
        int key = 0, val = 0, d = 0;
        if (valid) {
            key = kin[k];
            val = vin[k];
            d = (key >> shift) & mask;
        }
        const unsigned act = __ballot_sync(0xffffffffu, valid);
        unsigned peers = 0;
        if (valid) {
            peers = __match_any_sync(act, d);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            const int pos = offs[(size_t)d * ntiles + tile] + cnt[w][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) cnt[w][d] += __popc(peers);
        __syncwarp();
    }
}

// Stable sort of (key, index) pairs by key (0 <= key <= max_key); returns
// in perm the original positions in key order and, if sorted is not null,
// the keys in order.
void stable_sort_by_key(const int *keys, long long nnz, int max_key, int *perm, cudaStream_t st,
                        int *sorted = nullptr) {
    if (nnz == 0) return;
    Tmp ka(nnz * sizeof(int), st), kb(nnz * sizeof(int), st), va(nnz * sizeof(int), st),
        vb(nnz * sizeof(int), st);
    GB_CUDA(cudaMemcpyAsync(ka.p, keys, nnz * sizeof(int), cudaMemcpyDeviceToDevice, st));
    launch(k_iota, blocks_for(nnz, 256), 256, st, va.as<int>(), nnz);
    int key_bits = 1;
    while (key_bits < 31 && (max_key >> key_bits) > 0) ++key_bits;
    const int passes = (key_bits + kRsMaxBits - 1) / kRsMaxBits;
    const int width = (key_bits + passes - 1) / passes;
    const int ntiles = ceil_div(nnz, kRsTile);
    const long long hsz = (long long)(1 << width) * ntiles;
    Tmp H(hsz * sizeof(int), st), offs((hsz + 1) * sizeof(int), st);
    int *kin = ka.as<int>(), *kout = kb.as<int>(), *vin = va.as<int>(), *vout = vb.as<int>();
    for (int pass = 0, shift = 0; pass < passes; ++pass, shift += width) {
        const int bits = std::min(width, key_bits - shift);
        const long long hn = (long long)(1 << bits) * ntiles;
        const int grid = ceil_div(ntiles, kRsWarps);
        launch(k_radix_hist, grid, kRsWarps * 32, st, kin, nnz, shift, bits, ntiles, H.as<int>());
        exclusive_scan(H.as<int>(), (int)hn, offs.as<int>(), st);
        launch(k_radix_scatter, grid, kRsWarps * 32, st, kin, vin, nnz, shift, bits, ntiles, offs.as<int>(), kout,
               vout);
        GB_CUDA(cudaGetLastError());
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    GB_CUDA(cudaMemcpyAsync(perm, vin, nnz * sizeof(int), cudaMemcpyDeviceToDevice, st));
    if (sorted) GB_CUDA(cudaMemcpyAsync(sorted, kin, nnz * sizeof(int), cudaMemcpyDeviceToDevice, st));
}

// --------------------------------------------------------------- transpose

__global__ void k_expand_rows(const int *rp, int nrows, int *rowidx) {
    const int row = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= nrows) return;
    for (int k = rp[row] + lane; k < rp[row + 1]; k += 32) rowidx[k] = row;
}

// Row pointer of the transpose from the sorted column keys: position k is
// where every column strictly after key[k-1] and up to key[k] starts
// (key[-1] = -1, key[nnz] = ncols).
__global__ void k_col_bounds(const int *key, long long nnz, int ncols, int *rp) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nnz) return;
    const int c_prev = k == 0 ? -1 : key[k - 1];
    const int c_cur = k == nnz ? ncols : key[k];
    for (int c = c_prev + 1; c <= c_cur; ++c) rp[c] = (int)k;
}

__global__ void k_gather_t(const int *perm, const int *rowidx, const double *val, long long nnz, int *tcol,
                           double *tval) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnz) {
        const int s = perm[i];
        tcol[i] = rowidx[s];
        tval[i] = val[s];
    }
}

struct Csr {
    int nrows = 0, ncols = 0;
    long long nnz = 0;
    DevBuf rp, col, val;  // int, int, double
};

// CSR of M' (sorted rows) from the CSR of M (Section 4.3.3: the CSC of M
// read as the CSR of M').
Csr transpose(const int *rp, const int *col, const double *val, int nrows, int ncols, long long nnz,
              cudaStream_t st) {
    Csr T;
    T.nrows = ncols;
    T.ncols = nrows;
    T.nnz = nnz;
    T.rp.alloc((size_t)(ncols + 1) * sizeof(int));
    T.col.alloc(std::max<long long>(nnz, 1) * sizeof(int));
    T.val.alloc(std::max<long long>(nnz, 1) * sizeof(double));
    if (nnz == 0) GB_CUDA(cudaMemsetAsync(T.rp.p, 0, (size_t)(ncols + 1) * sizeof(int), st));
    if (nnz > 0) {
        Tmp rowidx(nnz * sizeof(int), st), perm(nnz * sizeof(int), st), skey(nnz * sizeof(int), st);
        launch(k_expand_rows, warp_blocks(nrows), kThreads, st, rp, nrows, rowidx.as<int>());
        stable_sort_by_key(col, nnz, std::max(ncols - 1, 0), perm.as<int>(), st, skey.as<int>());
        launch(k_col_bounds, blocks_for(nnz + 1, 256), 256, st, (const int *)skey.as<int>(), nnz, ncols, T.rp.as<int>());
        launch(k_gather_t, blocks_for(nnz, 256), 256, st, perm.as<int>(), rowidx.as<int>(), val, nnz,
                                                         T.col.as<int>(), T.val.as<double>());
    }
    GB_CUDA(cudaGetLastError());
    return T;
}

// ----------------------------------------------------------- full P from U

__global__ void k_fullp_len(const int *urp, const int *utrp, const int *utcol, int n, int *len) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int lt = utrp[i + 1] - utrp[i];
    const int dg = (lt > 0 && utcol[utrp[i + 1] - 1] == i) ? 1 : 0;
    len[i] = (urp[i + 1] - urp[i]) + lt - dg;
}

__global__ void k_fullp_fill(const int *urp, const int *ucol, const double *uval, const int *utrp,
                             const int *utcol, const double *utval, int n, const int *frp, int *fcol,
                             double *fval) {
    const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int t0 = utrp[i], t1 = utrp[i + 1];
    const int dg = (t1 > t0 && utcol[t1 - 1] == i) ? 1 : 0;
    const int nl = t1 - t0 - dg;
    int out = frp[i];
    for (int k = lane; k < nl; k += 32) {
        fcol[out + k] = utcol[t0 + k];
        fval[out + k] = utval[t0 + k];
    }
    out += nl;
    const int u0 = urp[i], nu = urp[i + 1] - u0;
    for (int k = lane; k < nu; k += 32) {
        fcol[out + k] = ucol[u0 + k];
        fval[out + k] = uval[u0 + k];
    }
}

// ------------------------------------------------------------------ Ruiz

__device__ __forceinline__ double limit_scaling(double v) {
    // norms below 1e-4 are taken as 1, norms above 1e4 as 1e4
    return v < 1e-4 ? 1.0 : (v > 1e4 ? 1e4 : v);
}

// Norms of the equilibrated matrices from the unscaled ones and the scaling
// so far (the matrices are scaled once, after the last pass).

// Columns j < n of [[P_bar, A_bar'], [A_bar, 0]]: out[j] = D_j max(c max_k
// |P_jk| D_k, max_i |A'_ji| E_i), one warp per j (rows of P and of A').
__global__ void k_norm_x(const int *prp, const int *pcol, const double *pval, const int *arp, const int *acol,
                         const double *aval, int n, const double *D, const double *E, const double *scal,
                         double *out, const int *tier) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;  // thread rows
    if (j >= n || tier[j] != kTierThread) return;
    double mp = 0.0, ma = 0.0;
    for (int k = prp[j]; k < prp[j + 1]; ++k) mp = nmax(mp, fabs(pval[k]) * D[pcol[k]]);
    for (int k = arp[j]; k < arp[j + 1]; ++k) ma = nmax(ma, fabs(aval[k]) * E[acol[k]]);
    out[j] = D[j] * nmax(scal[0] * mp, ma);
}
__global__ void k_norm_x_warp(const int *prp, const int *pcol, const double *pval, const int *arp, const int *acol,
                              const double *aval, const int *wlist, const int *wcount, const double *D,
                              const double *E, const double *scal, double *out) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * kWarps;
    for (int l = blockIdx.x * kWarps + (threadIdx.x >> 5); l < *wcount; l += nw) {
        const int j = wlist[l];
        double mp = strided_scaled_max(pcol, pval, D, prp[j], prp[j + 1], lane, 32);
        double ma = strided_scaled_max(acol, aval, E, arp[j], arp[j + 1], lane, 32);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mp = nmax(mp, __shfl_down_sync(0xffffffffu, mp, o));
            ma = nmax(ma, __shfl_down_sync(0xffffffffu, ma, o));
        }
        if (lane == 0) out[j] = D[j] * nmax(scal[0] * mp, ma);
    }
}
__global__ void __launch_bounds__(kThreads, 8) k_norm_x_long(const int *prp, const int *pcol, const double *pval, const int *arp, const int *acol,
                              const double *aval, const int *list, const int *count, const double *D,
                              const double *E, const double *scal, double *out) {
    for (int l = blockIdx.x; l < *count; l += gridDim.x) {
        const int j = list[l];
        double mp = 0.0, ma = 0.0;
        mp = strided_scaled_max<4>(pcol, pval, D, prp[j], prp[j + 1], threadIdx.x, blockDim.x);
        ma = strided_scaled_max<4>(acol, aval, E, arp[j], arp[j + 1], threadIdx.x, blockDim.x);
        mp = block_max(mp);
        ma = block_max(ma);
        if (threadIdx.x == 0) out[j] = D[j] * nmax(scal[0] * mp, ma);
    }
}

// Columns n + i (rows of A_bar): out[i] = E_i max_j |A_ij| D_j.
__global__ void k_norm_z(const int *rp, const int *col, const double *val, int m, const double *D, const double *E,
                         double *out, const int *tier) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // thread rows
    if (i >= m || tier[i] != kTierThread) return;
    double mx = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) mx = nmax(mx, fabs(val[k]) * D[col[k]]);
    out[i] = E[i] * mx;
}
__global__ void k_norm_z_warp(const int *rp, const int *col, const double *val, const int *wlist, const int *wcount,
                              const double *D, const double *E, double *out) {
    // a half-warp per row: two rows per warp in flight
    const int lane = threadIdx.x & 31, hl = lane & 15;
    const int nh = gridDim.x * kWarps * 2;
    const int cnt = *wcount;
    for (int l = (blockIdx.x * kWarps + (threadIdx.x >> 5)) * 2 + (lane >> 4); l - (lane >> 4) < cnt; l += nh) {
        double mx = 0.0;
        int i = -1;
        if (l < cnt) {
            i = wlist[l];
            mx = strided_scaled_max(col, val, D, rp[i], rp[i + 1], hl, 16);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) mx = nmax(mx, __shfl_down_sync(0xffffffffu, mx, o, 16));
        if (hl == 0 && i >= 0) out[i] = E[i] * mx;
    }
}
__global__ void __launch_bounds__(kThreads, 8) k_norm_z_long(const int *rp, const int *col, const double *val, const int *list, const int *count,
                              const double *D, const double *E, double *out) {
    for (int l = blockIdx.x; l < *count; l += gridDim.x) {
        const int i = list[l];
        double mx = 0.0;
        mx = strided_scaled_max<4>(col, val, D, rp[i], rp[i + 1], threadIdx.x, blockDim.x);
        mx = block_max(mx);
        if (threadIdx.x == 0) out[i] = E[i] * mx;
    }
}

// delta = 1/sqrt(limit(norm)); accumulated scaling *= delta.
__global__ void k_delta(const double *norm, int n, double *delta, double *acc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double d = 1.0 / sqrt(limit_scaling(norm[i]));
    delta[i] = d;
    acc[i] *= d;
}

// M <- g diag(rs) M diag(cs), one warp per row: v = (v * (g rs[r])) * cs[c]
// (g = *gp, or 1 when gp is null).
__global__ void k_scale_csr(const int *rp, const int *col, double *val, int nrows, const double *rs,
                            const double *cs, const double *gp, const int *skip) {
    const int r = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= nrows || skip[r] == kTierCta) return;
    const double a = (gp ? *gp : 1.0) * rs[r];
    for (int k = rp[r] + lane; k < rp[r + 1]; k += 32) val[k] = (val[k] * a) * cs[col[k]];
}
__global__ void k_scale_csr_long(const int *rp, const int *col, double *val, const int *list, const int *count,
                                 const double *rs, const double *cs, const double *gp) {
    for (int l = blockIdx.x; l < *count; l += gridDim.x) {
        const int r = list[l];
        const double a = (gp ? *gp : 1.0) * rs[r];
        for (int k = rp[r] + threadIdx.x; k < rp[r + 1]; k += blockDim.x) val[k] = (val[k] * a) * cs[col[k]];
    }
}

// q_bar = c D q
__global__ void k_scale_q_final(double *q, const double *D, const double *scal, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = (scal[0] * D[i]) * q[i];
}

// Cost scaling: gamma = 1 / limit(max(mean_j ||P_bar_j||_inf, ||q_bar||_inf))
// with P_bar = c D P D and q_bar = c D q after this pass's D; c *= gamma.
// scal[0] = c, scal[1] = gamma.  Partial sums per CTA, last CTA finishes.
__global__ void k_cost_scale(const int *prp, const int *pcol, const double *pval, int n, const double *q,
                             const double *D, double *partials, unsigned int *ticket, double *scal) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double c = scal[0];
    double sum = 0.0, qmax = 0.0;
    // rows of at most kThreadRow entries: a thread each
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int a = prp[r], b = prp[r + 1];
        if (b - a <= kThreadRow) {
            double mx = 0.0;
            for (int k = a; k < b; ++k) mx = nmax(mx, fabs(pval[k]) * D[pcol[k]]);
            sum += c * D[r] * mx;
        }
        qmax = nmax(qmax, fabs(c * D[r] * q[r]));
    }
    // longer rows: a warp each
    const int nwarps_grid = gridDim.x * kWarps;
    for (int r = blockIdx.x * kWarps + warp; r < n; r += nwarps_grid) {
        const int a = prp[r], b = prp[r + 1];
        if (b - a <= kThreadRow) continue;
        double mx = strided_scaled_max(pcol, pval, D, a, b, lane, 32);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = nmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        if (lane == 0) sum += c * D[r] * mx;
    }
    Red<1, 1> red;
    red.s[0] = sum;
    red.m[0] = qmax;
    auto fin = [&](const Red<1, 1> &t) {
        if (threadIdx.x == 0) {
            const double mean = n > 0 ? t.s[0] / n : 0.0;
            const double g = 1.0 / limit_scaling(fmax(mean, t.m[0]));
            scal[1] = g;
            scal[0] *= g;
        }
    };
    grid_finish<1, 1>(red, partials, ticket, fin);
}

__global__ void k_fill(double *v, long long n, double a) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = a;
}

__global__ void k_scale_bounds(double *l, double *u, const double *E, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    if (isfinite(l[i])) l[i] = E[i] * l[i];
    if (isfinite(u[i])) u[i] = E[i] * u[i];
}

// ----------------------------------------------------------- [P A'] build

__global__ void k_pat_rowptr(const int *prp, const int *atrp, int n, int *patrp, int *pend) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    patrp[i] = prp[i] + atrp[i];
    if (i < n) pend[i] = prp[i] + atrp[i] + (prp[i + 1] - prp[i]);
}

__global__ void k_pat_fill(const int *prp, const int *pcol, const double *pval, const int *atrp,
                           const int *atcol, const double *atval, int n, const int *patrp, int *patcol,
                           double *patval, const int *skip) {
    const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n || skip[i] == kTierCta) return;
    int out = patrp[i];
    const int p0 = prp[i], np = prp[i + 1] - p0;
    for (int k = lane; k < np; k += 32) {
        patcol[out + k] = pcol[p0 + k];
        patval[out + k] = pval[p0 + k];
    }
    out += np;
    const int a0 = atrp[i], na = atrp[i + 1] - a0;
    for (int k = lane; k < na; k += 32) {
        patcol[out + k] = atcol[a0 + k] + n;
        patval[out + k] = atval[a0 + k];
    }
}
__global__ void k_pat_fill_long(const int *prp, const int *pcol, const double *pval, const int *atrp,
                                const int *atcol, const double *atval, int n, const int *list, const int *count,
                                const int *patrp, int *patcol, double *patval) {
    for (int l = blockIdx.x; l < *count; l += gridDim.x) {
        const int i = list[l];
        int out = patrp[i];
        const int p0 = prp[i], np = prp[i + 1] - p0;
        for (int k = threadIdx.x; k < np; k += blockDim.x) {
            patcol[out + k] = pcol[p0 + k];
            patval[out + k] = pval[p0 + k];
        }
        out += np;
        const int a0 = atrp[i], na = atrp[i + 1] - a0;
        for (int k = threadIdx.x; k < na; k += blockDim.x) {
            patcol[out + k] = atcol[a0 + k] + n;
            patval[out + k] = atval[a0 + k];
        }
    }
}

// diag(P_bar) and ||A_bar column i||_2^2 (row i of A_bar'), one warp per i.
__global__ void k_diag_colsq(const int *prp, const int *pcol, const double *pval, const int *atrp,
                             const double *atval, int n, double *diagP, double *colsq, const int *skip) {
    const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n || skip[i] == kTierCta) return;
    double d = 0.0, s = 0.0;
    for (int k = prp[i] + lane; k < prp[i + 1]; k += 32)
        if (pcol[k] == i) d = pval[k];
    for (int k = atrp[i] + lane; k < atrp[i + 1]; k += 32) s += atval[k] * atval[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d += __shfl_down_sync(0xffffffffu, d, o);
        s += __shfl_down_sync(0xffffffffu, s, o);
    }
    if (lane == 0) {
        diagP[i] = d;
        colsq[i] = s;
    }
}
__global__ void k_diag_colsq_long(const int *prp, const int *pcol, const double *pval, const int *atrp,
                                  const double *atval, const int *list, const int *count, double *diagP,
                                  double *colsq) {
    for (int l = blockIdx.x; l < *count; l += gridDim.x) {
        const int i = list[l];
        double d = 0.0, s = 0.0;
        for (int k = prp[i] + threadIdx.x; k < prp[i + 1]; k += blockDim.x)
            if (pcol[k] == i) d = pval[k];
        for (int k = atrp[i] + threadIdx.x; k < atrp[i + 1]; k += blockDim.x) s += atval[k] * atval[k];
        d = block_sum(d);
        s = block_sum(s);
        if (threadIdx.x == 0) {
            diagP[i] = d;
            colsq[i] = s;
        }
    }
}

__global__ void k_qnorms(const double *q, const double *D, int n, unsigned long long *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0, b = 0.0;
    if (i < n) {
        a = fabs(q[i]);
        b = a / D[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = nmax(a, __shfl_down_sync(0xffffffffu, a, o));
        b = nmax(b, __shfl_down_sync(0xffffffffu, b, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(a));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(b));
    }
}

// ------------------------------------------------------------ host pieces

struct Input {
    const int64_t *rp64 = nullptr;
    const int32_t *col = nullptr;
    const double *val = nullptr;
    DevBuf rp64_dev, col_dev, val_dev;  // used when the input is on the host
};

void stage(const gbosqp_csr &M, bool host, Input &in, cudaStream_t st) {
    if (!host) {
        in.rp64 = M.rowptr;
        in.col = M.colind;
        in.val = M.val;
        return;
    }
    in.rp64_dev.alloc((size_t)(M.nrows + 1) * sizeof(int64_t));
    in.col_dev.alloc(std::max<int64_t>(M.nnz, 1) * sizeof(int32_t));
    in.val_dev.alloc(std::max<int64_t>(M.nnz, 1) * sizeof(double));
    GB_CUDA(cudaMemcpyAsync(in.rp64_dev.p, M.rowptr, (M.nrows + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (M.nnz > 0) {
        GB_CUDA(cudaMemcpyAsync(in.col_dev.p, M.colind, M.nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        GB_CUDA(cudaMemcpyAsync(in.val_dev.p, M.val, M.nnz * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    in.rp64 = in.rp64_dev.as<int64_t>();
    in.col = in.col_dev.as<int32_t>();
    in.val = in.val_dev.as<double>();
}

// Own FP64 copy of a validated input matrix with int32 row pointers.
Csr own_copy(const gbosqp_csr &M, const Input &in, cudaStream_t st) {
    Csr C;
    C.nrows = M.nrows;
    C.ncols = M.ncols;
    C.nnz = M.nnz;
    C.rp.alloc((size_t)(M.nrows + 1) * sizeof(int));
    // kSlack zeroed elements past the last nonzero (the SpMV's edge steps load past a warp's range)
    C.col.alloc((M.nnz + kSlack) * sizeof(int));
    C.val.alloc((M.nnz + kSlack) * sizeof(double));
    GB_CUDA(cudaMemsetAsync(C.col.as<int>() + M.nnz, 0, kSlack * sizeof(int), st));
    GB_CUDA(cudaMemsetAsync(C.val.as<double>() + M.nnz, 0, kSlack * sizeof(double), st));
    launch(k_rowptr_i32, blocks_for(M.nrows + 1, 256), 256, st, in.rp64, M.nrows + 1, C.rp.as<int>());
    if (M.nnz > 0) {
        GB_CUDA(cudaMemcpyAsync(C.col.p, in.col, M.nnz * sizeof(int), cudaMemcpyDeviceToDevice, st));
        GB_CUDA(cudaMemcpyAsync(C.val.p, in.val, M.nnz * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    return C;
}

std::string flag_text(int f) {
    std::string s;
    if (f & kFlagRowptr) s += "row pointers not monotone or not [0..nnz]; ";
    if (f & kFlagColRange) s += "column index out of range; ";
    if (f & kFlagColOrder) s += "columns not strictly increasing within a row (unsorted or duplicate); ";
    if (f & kFlagValue) s += "non-finite matrix value; ";
    if (f & kFlagLower) s += "entry below the diagonal in upper-triangular P; ";
    if (f & kFlagQ) s += "non-finite q; ";
    if (f & kFlagBounds) s += "l > u, NaN bound, or l = +inf / u = -inf; ";
    return s;
}

int flag_code(int f) {
    if (f & (kFlagRowptr | kFlagColRange | kFlagColOrder | kFlagLower)) return GBOSQP_ERR_CSR;
    if (f & kFlagBounds) return GBOSQP_ERR_BOUNDS;
    return GBOSQP_ERR_NONFINITE;
}

}  // namespace

SetupData device_setup(const gbosqp_csr &P, const gbosqp_csr &A, const double *q, const double *l,
                       const double *u, const gbosqp_settings &s, cudaStream_t st, const RowptrHook &hook) {
    const int n = P.nrows, m = A.nrows;
    const bool host = s.input_location == GBOSQP_HOST;
    SetupData sd;
    sd.n = n;
    sd.m = m;
    sd.nnzA = A.nnz;

    // ---- 1. stage and validate
    Input inP, inA;
    stage(P, host, inP, st);
    stage(A, host, inA, st);
    DevBuf qv, lv, uv;
    const double *qd = q, *ld = l, *ud = u;
    if (host) {
        qv.alloc((size_t)std::max(n, 1) * sizeof(double));
        lv.alloc((size_t)std::max(m, 1) * sizeof(double));
        uv.alloc((size_t)std::max(m, 1) * sizeof(double));
        if (n) GB_CUDA(cudaMemcpyAsync(qv.p, q, n * sizeof(double), cudaMemcpyHostToDevice, st));
        if (m) GB_CUDA(cudaMemcpyAsync(lv.p, l, m * sizeof(double), cudaMemcpyHostToDevice, st));
        if (m) GB_CUDA(cudaMemcpyAsync(uv.p, u, m * sizeof(double), cudaMemcpyHostToDevice, st));
        qd = qv.as<double>();
        ld = lv.as<double>();
        ud = uv.as<double>();
    }
    sd.q.alloc((size_t)std::max(n, 1) * sizeof(double));
    sd.l.alloc((size_t)std::max(m, 1) * sizeof(double));
    sd.u.alloc((size_t)std::max(m, 1) * sizeof(double));
    DevBuf flags(sizeof(int));
    GB_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(int), st));
    launch(k_check_rowptr, blocks_for(n + 1, 256), 256, st, inP.rp64, n, P.nnz, flags.as<int>());
    launch(k_check_rowptr, blocks_for(m + 1, 256), 256, st, inA.rp64, m, A.nnz, flags.as<int>());
    launch(k_check_vectors, blocks_for(std::max(n, m), 256), 256, st, 
        qd, n, ld, ud, m, sd.q.as<double>(), sd.l.as<double>(), sd.u.as<double>(), flags.as<int>());
    GB_CUDA(cudaGetLastError());
    int hflags = 0;
    GB_CUDA(cudaMemcpyAsync(&hflags, flags.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (hflags & kFlagRowptr) fail(GBOSQP_ERR_CSR, "invalid CSR: " + flag_text(hflags));
    Csr Pin = own_copy(P, inP, st);
    Csr Ain = own_copy(A, inA, st);
    launch(k_check_rows, warp_blocks(n), kThreads, st, Pin.rp.as<int>(), Pin.col.as<int>(), Pin.val.as<double>(), n,
                                                      n, s.P_is_upper ? 1 : 0, flags.as<int>());
    launch(k_check_rows, warp_blocks(m), kThreads, st, Ain.rp.as<int>(), Ain.col.as<int>(), Ain.val.as<double>(), m,
                                                      A.ncols, 0, flags.as<int>());
    GB_CUDA(cudaGetLastError());
    GB_CUDA(cudaMemcpyAsync(&hflags, flags.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (hflags) fail(flag_code(hflags), "invalid problem data: " + flag_text(hflags));
    inP = Input();
    inA = Input();
    qv.release();
    lv.release();
    uv.release();

    // ---- 2. full P and A'
    Csr Pf;
    if (s.P_is_upper) {
        Csr Ut = transpose(Pin.rp.as<int>(), Pin.col.as<int>(), Pin.val.as<double>(), n, n, Pin.nnz, st);
        Tmp len((size_t)std::max(n, 1) * sizeof(int), st);
        launch(k_fullp_len, blocks_for(n, 256), 256, st, Pin.rp.as<int>(), Ut.rp.as<int>(), Ut.col.as<int>(), n,
                                                         len.as<int>());
        Pf.nrows = Pf.ncols = n;
        Pf.rp.alloc((size_t)(n + 1) * sizeof(int));
        exclusive_scan(len.as<int>(), n, Pf.rp.as<int>(), st);
        int total = 0;
        GB_CUDA(cudaMemcpyAsync(&total, Pf.rp.as<int>() + n, sizeof(int), cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaStreamSynchronize(st));
        Pf.nnz = total;
        Pf.col.alloc(std::max(total, 1) * sizeof(int));
        Pf.val.alloc(std::max(total, 1) * sizeof(double));
        launch(k_fullp_fill, warp_blocks(n), kThreads, st, Pin.rp.as<int>(), Pin.col.as<int>(), Pin.val.as<double>(),
                                                          Ut.rp.as<int>(), Ut.col.as<int>(), Ut.val.as<double>(), n,
                                                          Pf.rp.as<int>(), Pf.col.as<int>(), Pf.val.as<double>());
        GB_CUDA(cudaGetLastError());
        GB_CUDA(cudaStreamSynchronize(st));
    } else {
        Pf = std::move(Pin);
    }
    Pin = Csr();
    Csr At = transpose(Ain.rp.as<int>(), Ain.col.as<int>(), Ain.val.as<double>(), m, n, Ain.nnz, st);
    sd.nnzP = Pf.nnz;
    // rows of [P A'] and of A that the row-wise passes give a CTA each
    const LongRows LP = long_rows(Pf.rp.as<int>(), At.rp.as<int>(), n, Pf.nnz + At.nnz, st);
    const LongRows LA = long_rows(Ain.rp.as<int>(), nullptr, m, Ain.nnz, st);
    // the row pointer of [P A'] (structure only), and both row pointers on
    // the host: with a hook the SpMV plans are built from them on host
    // threads while the device runs the equilibration below
    sd.nnzPAt = Pf.nnz + At.nnz;
    if (sd.nnzPAt >= (1LL << 31) - 256 || A.nnz >= (1LL << 31) - 256)
        fail(GBOSQP_ERR_UNSUPPORTED, "2^31 - 256 or more nonzeros in A or [P A']");
    sd.PAt_rowptr.alloc((size_t)(n + 1) * sizeof(int));
    sd.PAt_pend.alloc((size_t)std::max(n, 1) * sizeof(int));
    launch(k_pat_rowptr, blocks_for(n + 1, 256), 256, st, Pf.rp.as<int>(), At.rp.as<int>(), n,
                                                          sd.PAt_rowptr.as<int>(), sd.PAt_pend.as<int>());
    sd.A_rowptr_host.resize(m + 1);
    sd.PAt_rowptr_host.resize(n + 1);
    GB_CUDA(cudaMemcpyAsync(sd.A_rowptr_host.data(), Ain.rp.p, (m + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(sd.PAt_rowptr_host.data(), sd.PAt_rowptr.p, (n + 1) * sizeof(int),
                            cudaMemcpyDeviceToHost, st));
    if (hook) {
        GB_CUDA(cudaStreamSynchronize(st));
        hook(std::move(sd.A_rowptr_host), std::move(sd.PAt_rowptr_host));
        sd.A_rowptr_host.clear();
        sd.PAt_rowptr_host.clear();
    }

    // ---- 3. Ruiz equilibration (Algorithm 2)
    sd.D.alloc((size_t)std::max(n, 1) * sizeof(double));
    sd.E.alloc((size_t)std::max(m, 1) * sizeof(double));
    Tmp nx((size_t)std::max(n, 1) * sizeof(double), st), nz((size_t)std::max(m, 1) * sizeof(double), st);
    Tmp dx((size_t)std::max(n, 1) * sizeof(double), st), dz((size_t)std::max(m, 1) * sizeof(double), st);
    Tmp scal(2 * sizeof(double), st);
    const int cs_grid = std::max(1, std::min(ceil_div(std::max(n, 1), kWarps), device_sm_count() * 4));
    Tmp partials((size_t)cs_grid * 2 * sizeof(double), st), ticket(sizeof(unsigned int), st);
    GB_CUDA(cudaMemsetAsync(ticket.p, 0, sizeof(unsigned int), st));
    launch(k_fill, blocks_for(n, 256), 256, st, sd.D.as<double>(), n, 1.0);
    launch(k_fill, blocks_for(m, 256), 256, st, sd.E.as<double>(), m, 1.0);
    launch(k_fill, 1, 32, st, scal.as<double>(), 1, 1.0);
    const int gxw = resident_grid((const void *)k_norm_x_warp, n), gzw = resident_grid((const void *)k_norm_z_warp, m);
    // the norms of the columns j < n and of the columns n + i run side by
    // side: those of x on a second stream, joined by events
    SideStream side(st);
    for (int pass = 0; pass < s.scaling_iters; ++pass) {
        // column inf-norms of [[P_bar, A_bar'], [A_bar, 0]] from the unscaled
        // matrices and the scaling so far: columns j < n are rows of P and
        // A'; columns n + i are rows of A
        const cudaStream_t sx = side.fork();
        if (n) launch(k_norm_x_warp, gxw, kThreads, sx, Pf.rp.as<int>(), Pf.col.as<int>(), Pf.val.as<double>(),
                      At.rp.as<int>(), At.col.as<int>(), At.val.as<double>(), LP.wlist.as<int>(), LP.wcount.as<int>(),
                      sd.D.as<double>(), sd.E.as<double>(), scal.as<double>(), nx.as<double>());
        if (n) launch(k_norm_x, blocks_for(n, kThreads), kThreads, sx, Pf.rp.as<int>(), Pf.col.as<int>(), Pf.val.as<double>(),
                                                            At.rp.as<int>(), At.col.as<int>(), At.val.as<double>(), n,
                                                            sd.D.as<double>(), sd.E.as<double>(), scal.as<double>(),
                                                            nx.as<double>(), LP.flag.as<int>());
        if (n) launch(k_norm_x_long, LP.grid, kThreads, sx, Pf.rp.as<int>(), Pf.col.as<int>(), Pf.val.as<double>(),
                      At.rp.as<int>(), At.col.as<int>(), At.val.as<double>(), LP.list.as<int>(), LP.count.as<int>(),
                      sd.D.as<double>(), sd.E.as<double>(), scal.as<double>(), nx.as<double>());
        if (m) launch(k_norm_z_warp, gzw, kThreads, st, Ain.rp.as<int>(), Ain.col.as<int>(), Ain.val.as<double>(),
                      LA.wlist.as<int>(), LA.wcount.as<int>(), sd.D.as<double>(), sd.E.as<double>(), nz.as<double>());
        if (m) launch(k_norm_z, blocks_for(m, kThreads), kThreads, st, Ain.rp.as<int>(), Ain.col.as<int>(), Ain.val.as<double>(),
                                                            m, sd.D.as<double>(), sd.E.as<double>(), nz.as<double>(),
                                                            LA.flag.as<int>());
        if (m) launch(k_norm_z_long, LA.grid, kThreads, st, Ain.rp.as<int>(), Ain.col.as<int>(), Ain.val.as<double>(),
                      LA.list.as<int>(), LA.count.as<int>(), sd.D.as<double>(), sd.E.as<double>(), nz.as<double>());
        side.join();  // both sides read D and E; the deltas below rewrite them
        if (n) launch(k_delta, blocks_for(n, 256), 256, st, nx.as<double>(), n, dx.as<double>(), sd.D.as<double>());
        if (m) launch(k_delta, blocks_for(m, 256), 256, st, nz.as<double>(), m, dz.as<double>(), sd.E.as<double>());
        // cost scaling on P_bar = c D P D, q_bar = c D q with the new D
        launch(k_cost_scale, cs_grid, kThreads, st, Pf.rp.as<int>(), Pf.col.as<int>(), Pf.val.as<double>(), n,
                                                   sd.q.as<double>(), sd.D.as<double>(), partials.as<double>(),
                                                   ticket.as<unsigned int>(), scal.as<double>());
        GB_CUDA(cudaGetLastError());
    }
    // the scaled problem: P <- c D P D, A <- E A D, A' <- D A' E, q <- c D q
    auto scale = [&](const Csr &M, int nrows, const LongRows &L, const double *rs, const double *cs, const double *g) {
        if (!nrows) return;
        launch(k_scale_csr, warp_blocks(nrows), kThreads, st, M.rp.as<int>(), M.col.as<int>(), M.val.as<double>(), nrows,
               rs, cs, g, L.flag.as<int>());
        launch(k_scale_csr_long, L.grid, kThreads, st, M.rp.as<int>(), M.col.as<int>(), M.val.as<double>(),
               L.list.as<int>(), L.count.as<int>(), rs, cs, g);
    };
    scale(Pf, n, LP, sd.D.as<double>(), sd.D.as<double>(), (const double *)scal.as<double>());
    scale(Ain, m, LA, sd.E.as<double>(), sd.D.as<double>(), (const double *)nullptr);
    scale(At, n, LP, sd.D.as<double>(), sd.E.as<double>(), (const double *)nullptr);
    if (n) launch(k_scale_q_final, blocks_for(n, 256), 256, st, sd.q.as<double>(), (const double *)sd.D.as<double>(),
                                                               (const double *)scal.as<double>(), n);
    if (m) launch(k_scale_bounds, blocks_for(m, 256), 256, st, sd.l.as<double>(), sd.u.as<double>(), sd.E.as<double>(), m);
    GB_CUDA(cudaMemcpyAsync(&sd.c, scal.p, sizeof(double), cudaMemcpyDeviceToHost, st));

    // ---- 4. [P A'], Jacobi data, q norms
    // kSlack zeroed elements past the last nonzero, as in the copy of A
    sd.PAt_col.alloc((sd.nnzPAt + kSlack) * sizeof(int));
    sd.PAt_val.alloc((sd.nnzPAt + kSlack) * sizeof(double));
    GB_CUDA(cudaMemsetAsync(sd.PAt_col.as<int>() + sd.nnzPAt, 0, kSlack * sizeof(int), st));
    GB_CUDA(cudaMemsetAsync(sd.PAt_val.as<double>() + sd.nnzPAt, 0, kSlack * sizeof(double), st));
    if (n) launch(k_pat_fill, warp_blocks(n), kThreads, st, Pf.rp.as<int>(), Pf.col.as<int>(), Pf.val.as<double>(),
                                                          At.rp.as<int>(), At.col.as<int>(), At.val.as<double>(), n,
                                                          sd.PAt_rowptr.as<int>(), sd.PAt_col.as<int>(),
                                                          sd.PAt_val.as<double>(), LP.flag.as<int>());
    if (n) launch(k_pat_fill_long, LP.grid, kThreads, st, Pf.rp.as<int>(), Pf.col.as<int>(), Pf.val.as<double>(),
                  At.rp.as<int>(), At.col.as<int>(), At.val.as<double>(), n, LP.list.as<int>(), LP.count.as<int>(),
                  sd.PAt_rowptr.as<int>(), sd.PAt_col.as<int>(), sd.PAt_val.as<double>());
    sd.diagP.alloc((size_t)std::max(n, 1) * sizeof(double));
    sd.colsq.alloc((size_t)std::max(n, 1) * sizeof(double));
    if (n) launch(k_diag_colsq, warp_blocks(n), kThreads, st, Pf.rp.as<int>(), Pf.col.as<int>(), Pf.val.as<double>(),
                                                            At.rp.as<int>(), At.val.as<double>(), n,
                                                            sd.diagP.as<double>(), sd.colsq.as<double>(),
                                                            LP.flag.as<int>());
    if (n) launch(k_diag_colsq_long, LP.grid, kThreads, st, Pf.rp.as<int>(), Pf.col.as<int>(), Pf.val.as<double>(),
                  At.rp.as<int>(), At.val.as<double>(), LP.list.as<int>(), LP.count.as<int>(), sd.diagP.as<double>(),
                  sd.colsq.as<double>());
    Tmp qn(2 * sizeof(unsigned long long), st);
    GB_CUDA(cudaMemsetAsync(qn.p, 0, 2 * sizeof(unsigned long long), st));
    if (n) launch(k_qnorms, blocks_for(n, 256), 256, st, sd.q.as<double>(), sd.D.as<double>(), n,
                                                        qn.as<unsigned long long>());
    double qnh[2] = {0.0, 0.0};
    GB_CUDA(cudaMemcpyAsync(qnh, qn.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaGetLastError());
    // A keeps its own copy; host row pointers for the work plans
    sd.A_rowptr = std::move(Ain.rp);
    sd.A_col = std::move(Ain.col);
    sd.A_val = std::move(Ain.val);
    GB_CUDA(cudaStreamSynchronize(st));
    sd.qnorm_s = qnh[0];
    sd.qnorm_u = qnh[1];
    return sd;
}

}  // namespace gb
