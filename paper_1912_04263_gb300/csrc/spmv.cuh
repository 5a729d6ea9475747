// Warp-stream CSR SpMV core.
//
// The rows of a CSR matrix are divided among the warps of a persistent grid
// in contiguous ranges of about equal cost (nonzeros plus a fixed cost per
// row).  A cut between two warps may fall inside a long row; the parts of
// such a split row are summed by the last of its warps to finish, in warp
// order (or, for epilogues that take a split row by parts, stored in fixed
// slots for a later kernel), so every result is bitwise reproducible.
//
// Inside its range a warp walks items of two kinds:
// * stream items: consecutive rows of more than 32 nonzeros (and the parts
//   of split rows).  The warp streams the item's value/column range in
//   aligned 32-element steps, U steps per batch, with the next batch's loads
//   in flight while the current one is gathered and summed.  Because every
//   row inside the item holds more than 32 nonzeros, at most one row ends
//   inside a step: lanes before the end add to the current row, lanes after
//   it to the next, and the finished row is reduced across the warp with
//   shuffles.  Up to 32 finished rows wait in registers (one per lane) and
//   their epilogues then run together, one per lane.
// * group items: consecutive rows of at most 32 nonzeros with the same lane
//   group width G (len <= 2 G): a group of G lanes sums a row, 32 / G rows
//   per round, R rounds loaded together.
//
// The epilogue functor's row(r, s1, s2, red) consumes a row's sums (s1 over
// the first segment [rowptr[r], pend[r]), s2 over the rest, when a split
// point pend is given; with a gather of two vectors, s2 is the row's sum
// with the second; otherwise s2 = 0) and adds to the warp's reduction.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace gb {

constexpr int kWThreads = 256;               // CTA size of every warp-stream kernel
constexpr int kWWarps = kWThreads / 32;
constexpr int kGroupMaxLen = 32;             // rows up to this length take the group path
constexpr int kMaxSplitSums = 2;             // epilogue sums a kernel may accumulate per split row

// One item of a warp's range.
struct WItem {
    int r0;  // first row
    int r1;  // one past the last row touched
    int k0;  // stream item: first nonzero (inside row r0 for a split row); group item: -G
    int k1;  // stream item: one past the last nonzero (inside row r1 - 1 for a split row)
};

// A row cut between warps: its nparts parts (one per warp holding elements
// of it, in warp order) publish their sums to slots slot0 .. slot0 + nparts - 1.
struct SplitRow {
    int row;
    int slot0;
    int nparts;
    int pad;
};

// Per warp: the split rows at the head and the tail of its range and the
// warp's slot in each (-1: none).
struct WSplit {
    int head, head_slot, tail, tail_slot;
};

template <class T>
struct CsrW {
    int nrows = 0, ncols = 0;
    const int *rowptr = nullptr;
    const int *col = nullptr;
    const T *val = nullptr;
    const int *pend = nullptr;        // optional split of each row
    const WItem *items = nullptr;
    const int *wpart = nullptr;       // items of warp w: [wpart[w], wpart[w+1])
    const WSplit *wsplit = nullptr;
    const SplitRow *split = nullptr;
    int nsplit = 0;
    int *split_count = nullptr;       // one ticket per split row, zero between launches
    double *split_part = nullptr;     // 2 sums per slot
    double *split_red = nullptr;      // kMaxSplitSums epilogue sums per split row
    const int *split_of = nullptr;    // per row: its index in split, or -1
};

// ------------------------------------------------------------ host plan

struct WPlanHost {
    int nwarps = 0;
    std::vector<WItem> items;
    std::vector<int> wpart;
    std::vector<WSplit> wsplit;
    std::vector<SplitRow> split;
    int nslots = 0;
};

// Cost weights of the warp partition (in nonzero equivalents).
struct WPlanCost {
    int stream_row = 8;    // per row of the stream path (reduction, epilogue)
    int group_row = 24;    // per row of the group path (a chain of dependent loads per round)
    int split_min = 256;   // rows longer than this may be cut between warps
    int bundle_min = 0;    // rows longer than this go to bundles (0: none)
};

WPlanHost build_wplan(const std::vector<int> &rowptr, int nwarps, const WPlanCost &cost = WPlanCost());

// Lane-group width of a row of the group path: the smallest power of two
// G with 2 G >= len.
__host__ __device__ __forceinline__ int group_width_of(int len) {
    return len <= 2 ? 1 : len <= 4 ? 2 : len <= 8 ? 4 : len <= 16 ? 8 : 16;
}

// ---------------------------------------------------------- device core

namespace wdetail {

constexpr unsigned kFull = 0xffffffffu;

template <class Acc>
__device__ __forceinline__ Acc warp_allsum(Acc v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Entry idx (0..63) of the two-window row table (lane k of win holds entry k).
__device__ __forceinline__ int win_get(int win, int nwin, int idx) {
    const int a = __shfl_sync(kFull, win, idx & 31);
    const int b = __shfl_sync(kFull, nwin, idx & 31);
    return idx < 32 ? a : b;
}

// Publish one warp's part of split row l (lane 0) and, in the last warp of
// the row to arrive, sum the parts in slot order and run the row's
// epilogue; its sums go to split_red[l] so that the grid total adds them in
// a fixed order.
template <class Acc, bool HOIST = false, class T, class Epi, class RedT>
__device__ __forceinline__ void publish_part(const CsrW<T> &M, int l, int slot, int row, Acc t1, Acc t2, Epi &epi,
                                             RedT &red) {
    const int lane = threadIdx.x & 31;
    int last = 0;
    if (lane == 0) {
        M.split_part[2 * (size_t)slot] = (double)t1;
        M.split_part[2 * (size_t)slot + 1] = (double)t2;
        const SplitRow S = M.split[l];
        const int t = (int)ticket_arrive(reinterpret_cast<unsigned int *>(M.split_count + l));
        last = t == S.nparts - 1;
        if (last) {
            double s1 = 0.0, s2 = 0.0;
            if constexpr (HOIST) {
                // the parts' loads issued kLd at a time, then added in slot order
                constexpr int kLd = 4;
                for (int k0 = 0; k0 < S.nparts; k0 += kLd) {
                    double a[kLd], b[kLd];
#pragma unroll
                    for (int u = 0; u < kLd; ++u) {
                        const bool in = k0 + u < S.nparts;
                        a[u] = in ? __ldcg(M.split_part + 2 * (size_t)(S.slot0 + k0 + u)) : 0.0;
                        b[u] = in ? __ldcg(M.split_part + 2 * (size_t)(S.slot0 + k0 + u) + 1) : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < kLd; ++u)
                        if (k0 + u < S.nparts) {
                            s1 += a[u];
                            s2 += b[u];
                        }
                }
            } else {
                for (int k = 0; k < S.nparts; ++k) {
                    s1 += __ldcg(M.split_part + 2 * (size_t)(S.slot0 + k));
                    s2 += __ldcg(M.split_part + 2 * (size_t)(S.slot0 + k) + 1);
                }
            }
            M.split_count[l] = 0;
            RedT tmp;
            tmp.zero();
            epi.row(row, Acc(s1), Acc(s2), tmp);
            constexpr int NS = RedT::kNS, NM = RedT::kNM;
            static_assert(NS <= kMaxSplitSums, "more epilogue sums than the split-row slots hold");
#pragma unroll
            for (int i = 0; i < NM; ++i) red.m[i] = amax(red.m[i], tmp.m[i]);
#pragma unroll
            for (int i = 0; i < NS; ++i) M.split_red[(size_t)l * kMaxSplitSums + i] = tmp.s[i];
            // seen by the grid total through the CTA barrier before thread 0 arrives at its ticket
        }
    }
    (void)last;
}

// An epilogue whose split rows contribute linearly (Epi::kSplitParts) takes
// each part of a split row by itself: the core stores the part's sums in
// its slot, and epi.part(row, first, s1, s2, red) adds what the part
// contributes to the warp's reduction (first: the part holding the row's
// start); a later kernel forms the row's value from the slots, in slot
// order.  Such a kernel needs no ticket, fence or combining warp.
template <class E, class = void>
struct SplitParts : std::false_type {};
template <class E>
struct SplitParts<E, std::void_t<decltype(E::kSplitParts)>> : std::integral_constant<bool, E::kSplitParts> {};

// A gather with a second vector (Gather::kDual, Gather::second(c)): the core
// also sums the products with the second vector, in the working precision T
// as a kernel over that vector alone would, and hands each row's second sum
// to the epilogue as s2 (exactly, as Acc).  Only for kernels without a row
// split point (SPLIT = false), whose s2 is otherwise zero; a row cut between
// warps carries it through the same slot.
template <class G, class = void>
struct DualGather : std::false_type {};
template <class G>
struct DualGather<G, std::void_t<decltype(G::kDual)>> : std::integral_constant<bool, G::kDual> {};

// One warp's part of split row l, in slot `slot`.
template <class Acc, bool HOIST = false, class T, class Epi, class RedT>
__device__ __forceinline__ void split_part(const CsrW<T> &M, int l, int slot, int row, Acc t1, Acc t2, Epi &epi,
                                           RedT &red) {
    if constexpr (SplitParts<Epi>::value) {
        if ((threadIdx.x & 31) == 0) {
            M.split_part[2 * (size_t)slot] = (double)t1;
            M.split_part[2 * (size_t)slot + 1] = (double)t2;
            epi.part(row, slot == M.split[l].slot0, t1, t2, red);
        }
    } else {
        publish_part<Acc, HOIST>(M, l, slot, row, t1, t2, epi, red);
    }
}

}  // namespace wdetail

// Stream item: rows [it.r0, it.r1), nonzeros [it.k0, it.k1), each row
// longer than 32 nonzeros except parts of split rows at the ends.  The warp
// walks aligned 32-element steps from it.k0 rounded down to 32; the loads
// of the first and last steps may reach up to 31 elements outside the
// item (the matrix arrays carry kSlack zeroed elements past the last
// nonzero), and those lanes' products are discarded.  The next batch of U
// steps is loaded while the current one is summed.
template <int U, class Acc, bool SPLIT, bool EDGE, bool HOIST, class T, class Gather, class Epi, class RedT>
__device__ __forceinline__ void stream_item(const CsrW<T> &M, const WItem &it, const WSplit &ws,
                                            const Gather &gather, Epi &epi, RedT &red) {
    using namespace wdetail;
    const int lane = threadIdx.x & 31;
    const int kbeg = it.k0, kend = it.k1;
    const int base = kbeg & ~31;
    const int nsteps = (kend - base + 31) >> 5;
    // row table: lane k of rwin holds the end of row wbase + k, of pwin the
    // split point of row wbase + k; nrwin / npwin the next 32 rows
    int wbase = it.r0;
    auto load_win = [&](int b, int &rw, int &pw) {
        const int r = b + lane;
        rw = r < it.r1 ? __ldg(M.rowptr + r + 1) : 0x7fffffff;
        if (SPLIT) pw = r < it.r1 ? __ldg(M.pend + r) : 0x7fffffff;
    };
    int rwin, pwin = 0, nrwin, npwin = 0;
    load_win(wbase, rwin, pwin);
    load_win(wbase + 32, nrwin, npwin);
    int row = it.r0;
    int rend = min(__shfl_sync(kFull, rwin, 0), kend);
    // step holding the first element of the next row (none when the row ends with the item)
    int cross = rend < kend ? (rend - base) >> 5 : 0x7fffffff;
    int pcur = SPLIT ? __shfl_sync(kFull, pwin, 0) : 0;
    const int head_row = ws.head >= 0 ? M.split[ws.head].row : -1;
    const int tail_row = ws.tail >= 0 ? M.split[ws.tail].row : -1;
    const int wid = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);

    constexpr bool DUAL = DualGather<Gather>::value;
    static_assert(!(DUAL && SPLIT), "a second vector's sums take the place of the split point's");
    LaneSum<Acc, T> a1, a2, b1, b2;
    LaneSum<T, T> q1, q2;  // DUAL: the second vector's sums of the current and the next row
    // finished rows waiting for their epilogue, one per lane
    int prow = -1, npend = 0;
    Acc p1 = Acc(0), p2 = Acc(0);

    auto flush = [&]() {
        if (lane < npend) epi.row(prow, p1, p2, red);
        npend = 0;
    };
    auto finish_row = [&](int r, Acc t1, Acc t2) {
        if (r == head_row || r == tail_row) {
            const WSplit w2 = M.wsplit[wid];  // reloaded: keeps the split ids out of the loop's registers
            if (r == head_row) split_part<Acc, HOIST>(M, w2.head, w2.head_slot, r, t1, t2, epi, red);
            else split_part<Acc, HOIST>(M, w2.tail, w2.tail_slot, r, t1, t2, epi, red);
        } else {
            if (lane == npend) {
                prow = r;
                p1 = t1;
                p2 = t2;
            }
            if (++npend == 32) flush();
        }
    };

    const T *pv = M.val + base + lane;
    const int *pc = M.col + base + lane;
    T va[U], vb[U];
    int ca[U], cb[U];
#if GB_PREDICATED_LOADS
    // steps at or past nsteps are not loaded (their lanes gather entry 0 and
    // are never summed): only the item's own steps, which reach at most 31
    // elements past it, touch the matrix arrays
    auto load = [&](int s0, T(&v)[U], int(&c)[U]) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (s0 + u < nsteps) {
                v[u] = __ldcs(pv + ((s0 + u) << 5));
                c[u] = __ldcs(pc + ((s0 + u) << 5));
            } else {
                v[u] = T(0);
                c[u] = 0;
            }
        }
    };
#else
    // a batch that starts inside the item is loaded whole: its last step may
    // end up to 32 U - 1 elements past the item, inside the arrays' zeroed
    // slack (kSlack >= 32 U) or other rows' nonzeros, so every loaded column
    // is a valid index; steps past nsteps are never summed
    static_assert(32 * U <= kSlack, "the matrix arrays' slack must hold a whole batch");
    auto load = [&](int s0, T(&v)[U], int(&c)[U]) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            v[u] = __ldcs(pv + ((s0 + u) << 5));
            c[u] = __ldcs(pc + ((s0 + u) << 5));
        }
    };
#endif
    // add the products of the U steps from s0 to their rows
    auto sum_batch = [&](int s0, T(&pr)[U], T(&pq)[U]) {
        // EDGE (see warp_rows): only the first and the last batch hold steps
        // that reach outside the item or past its last step, so the others
        // skip those masks
        const bool edge = !EDGE || s0 == 0 || s0 + U >= nsteps;
        if (EDGE && edge) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int s = s0 + u;
                const int e = base + (s << 5) + lane;
                if (s < nsteps && (s == 0 || s == nsteps - 1) && (e < kbeg || e >= kend)) {
                    pr[u] = T(0);
                    if (DUAL) pq[u] = T(0);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int s = s0 + u;
            if (edge && s >= nsteps) break;
            const int e = base + (s << 5) + lane;
            if (!EDGE && (s == 0 || s == nsteps - 1) && (e < kbeg || e >= kend)) {
                pr[u] = T(0);
                if (DUAL) pq[u] = T(0);
            }
            if (s != cross) {
                if (!SPLIT || e < pcur) a1.add(pr[u]); else a2.add(pr[u]);
                if (DUAL) q1.add(pq[u]);
            } else {
                // row `row` ends at rend inside this step; the next row is in the item
                const int pnext = SPLIT ? win_get(pwin, npwin, row + 1 - wbase) : 0;
                if (e < rend) {
                    if (!SPLIT || e < pcur) a1.add(pr[u]); else a2.add(pr[u]);
                    if (DUAL) q1.add(pq[u]);
                } else {
                    if (!SPLIT || e < pnext) b1.add(pr[u]); else b2.add(pr[u]);
                    if (DUAL) q2.add(pq[u]);
                }
                const Acc t1 = warp_allsum(a1.value());
                const Acc t2 = SPLIT ? warp_allsum(a2.value()) : DUAL ? to_acc<Acc>(warp_allsum(q1.value())) : Acc(0);
                finish_row(row, t1, t2);
                a1 = b1;
                a2 = b2;
                b1 = LaneSum<Acc, T>();
                b2 = LaneSum<Acc, T>();
                if (DUAL) {
                    q1 = q2;
                    q2 = LaneSum<T, T>();
                }
                ++row;
                if (row - wbase == 32) {
                    wbase += 32;
                    rwin = nrwin;
                    pwin = npwin;
                    load_win(wbase + 32, nrwin, npwin);
                }
                rend = min(win_get(rwin, nrwin, row - wbase), kend);
                cross = rend < kend ? (rend - base) >> 5 : 0x7fffffff;
                pcur = pnext;
            }
        }
    };
    auto process = [&](int s0, const T(&v)[U], const int(&c)[U]) {
        T pr[U], pq[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            pr[u] = v[u] * gather(c[u]);
            if constexpr (DUAL) pq[u] = v[u] * gather.second(c[u]);
        }
        sum_batch(s0, pr, pq);
    };
    load(0, va, ca);
    for (int s0 = 0; s0 < nsteps; s0 += 2 * U) {
        if (s0 + U < nsteps) load(s0 + U, vb, cb);
        process(s0, va, ca);
        if (s0 + U >= nsteps) break;
        if (s0 + 2 * U < nsteps) load(s0 + 2 * U, va, ca);
        process(s0 + U, vb, cb);
    }
    // the last row ends with the item
    const Acc t1 = warp_allsum(a1.value());
    const Acc t2 = SPLIT ? warp_allsum(a2.value()) : DUAL ? to_acc<Acc>(warp_allsum(q1.value())) : Acc(0);
    finish_row(row, t1, t2);
    flush();
}

// Group item: rows [r0, r1), each of at most 2 G nonzeros; a group of G
// lanes sums one row, 32 / G rows per round, R rounds in flight together.
template <int G, int R, class Acc, bool SPLIT, class T, class Gather, class Epi, class RedT>
__device__ __forceinline__ void group_item(const CsrW<T> &M, int r0, int r1, const Gather &gather, Epi &epi,
                                           RedT &red) {
    constexpr bool DUAL = wdetail::DualGather<Gather>::value;
    static_assert(!(DUAL && SPLIT), "a second vector's sums take the place of the split point's");
    constexpr int kRows = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gi = lane / G, gl = lane % G;
    for (int base = r0; base < r1; base += R * kRows) {
        int a[R], b[R], sp[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int r = base + k * kRows + gi;
            a[k] = 0;
            b[k] = 0;
            sp[k] = 0;
            if (r < r1) {
                a[k] = __ldg(M.rowptr + r);
                b[k] = __ldg(M.rowptr + r + 1);
                if (SPLIT) sp[k] = __ldg(M.pend + r);
            }
        }
        T v[R][2];
        int c[R][2];
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int e = a[k] + gl + u * G;
                if (e < b[k]) {
                    v[k][u] = __ldcs(M.val + e);
                    c[k][u] = __ldcs(M.col + e);
                } else {
                    v[k][u] = T(0);
                    c[k][u] = -1;
                }
            }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            LaneSum<Acc, T> s1, s2;
            LaneSum<T, T> sq;  // DUAL: the second vector's sum
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (c[k][u] >= 0) {
                    const T pr = v[k][u] * gather(c[k][u]);
                    const int e = a[k] + gl + u * G;
                    if (!SPLIT || e < sp[k]) s1.add(pr); else s2.add(pr);
                    if constexpr (DUAL) sq.add(v[k][u] * gather.second(c[k][u]));
                }
            }
            Acc t1 = s1.value(), t2 = s2.value();
            T tq = sq.value();
            if (G > 1) {
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) {
                    t1 += __shfl_down_sync(wdetail::kFull, t1, o, G);
                    if (SPLIT) t2 += __shfl_down_sync(wdetail::kFull, t2, o, G);
                    if (DUAL) tq += __shfl_down_sync(wdetail::kFull, tq, o, G);
                }
            }
            if (DUAL) t2 = to_acc<Acc>(tq);
            const int r = base + k * kRows + gi;
            if (gl == 0 && r < r1) epi.row(r, t1, t2, red);
        }
    }
}

// The whole range of this warp.  HOIST: the last warp of a row cut between
// warps loads the parts together (measured: the PCG initialisation gains,
// kernels with heavier register use lose).  EDGE: the stream path tests a batch once
// for reaching past its item instead of testing every step (measured: the
// kernels over A, with rows of about 150 nonzeros, gain; the [P A'] kernels,
// whose long parts run in few large batches, lose to the extra code).
template <int U, class Acc, bool SPLIT, bool EDGE = false, bool HOIST = false, class T, class Gather, class Epi,
          class RedT>
__device__ __forceinline__ void warp_rows(const CsrW<T> &M, const Gather &gather, Epi &epi, RedT &red) {
    const int w = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int i0 = M.wpart[w], i1 = M.wpart[w + 1];
    if (i0 >= i1) return;
    const WSplit ws = M.wsplit[w];
    for (int i = i0; i < i1; ++i) {
        const WItem it = M.items[i];
        if (it.k0 >= 0) {
            stream_item<U, Acc, SPLIT, EDGE, HOIST>(M, it, ws, gather, epi, red);
        } else {
            switch (-it.k0) {
#ifndef GB_GROUP_R
#define GB_GROUP_R 4
#endif
                case 1: group_item<1, GB_GROUP_R, Acc, SPLIT>(M, it.r0, it.r1, gather, epi, red); break;
                case 2: group_item<2, GB_GROUP_R, Acc, SPLIT>(M, it.r0, it.r1, gather, epi, red); break;
                case 4: group_item<4, (GB_GROUP_R > 1 ? GB_GROUP_R / 2 : 1), Acc, SPLIT>(M, it.r0, it.r1, gather, epi, red); break;
                case 8: group_item<8, (GB_GROUP_R > 1 ? GB_GROUP_R / 2 : 1), Acc, SPLIT>(M, it.r0, it.r1, gather, epi, red); break;
                default: group_item<16, (GB_GROUP_R > 1 ? GB_GROUP_R / 2 : 1), Acc, SPLIT>(M, it.r0, it.r1, gather, epi, red); break;
            }
        }
    }
}

// Grid total of a warp-stream kernel's reduction: per-CTA partials and (but
// for kernels whose split rows contribute by parts, SplitRed = false) the
// split rows' epilogue sums, added in a fixed order by the last CTA to
// arrive, which then calls fin(total) with every thread.
template <int NS, int NM, bool SplitRed = true, class T, class Fin>
__device__ __forceinline__ void grid_finish_w(Red<NS, NM> &red, const CsrW<T> &M, double *partials,
                                              unsigned int *ticket, Fin &fin) {
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
    static_assert(NS <= kMaxSplitSums, "more sums than the split-row slots hold");
    if (NS > 0 && SplitRed) add_records<NS, NM, NS, 0>(acc, M.split_red, kMaxSplitSums, M.nsplit);
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

}  // namespace gb
