// Host plan of the warp-stream SpMV (spmv.cuh): the cut of a CSR matrix's
// rows into per-warp ranges of about equal cost, the items of each range,
// and the table of rows cut between warps.
//
// Rows longer than bundle_min (when set) are taken out of the contiguous
// cut and put into bundles of kWWarps consecutive long rows.  The bundles
// share a run of CTAs in proportion to their longest rows, continuously: CTA
// c takes the same weight range [B_c, B_(c+1)) of the bundles' total, which
// may end inside one bundle and go on into the next, and warp j of the CTA
// takes, of row j of every bundle its range touches, the part that range
// covers.  The warps of a CTA then sweep the same column window of their
// rows side by side, which for rows with similarly spread columns keeps the
// gathered entries shared in the CTA's L1, and every CTA gets the same
// amount of work.  The other rows are cut contiguously over the remaining
// warps.
#include <algorithm>
#include <vector>

#include "spmv.cuh"

namespace gb {

namespace {

struct Cut {
    int r;  // row
    int k;  // first nonzero: rowptr[r] (a row start) or inside row r
};

bool before(const Cut &a, const Cut &b) { return a.r < b.r || (a.r == b.r && a.k < b.k); }

}  // namespace

WPlanHost build_wplan(const std::vector<int> &rp, int nwarps, const WPlanCost &cost) {
    WPlanHost P;
    const int ncta = std::max((nwarps + kWWarps - 1) / kWWarps, 1);
    nwarps = ncta * kWWarps;
    P.nwarps = nwarps;
    const int nrows = (int)rp.size() - 1;
    const int nnz = nrows > 0 ? rp[nrows] : 0;
    auto len_of = [&](int r) { return rp[r + 1] - rp[r]; };
    auto row_cost = [&](int len) { return (long long)len + (len > kGroupMaxLen ? cost.stream_row : cost.group_row); };

    // bundled rows and their share of the CTAs; prefix of the costs of the
    // other rows (one pass)
    std::vector<int> brows;
    std::vector<long long> pre(nrows + 1, 0);
    long long cost_all = 0, cost_b = 0;
    for (int r = 0; r < nrows; ++r) {
        const int len = len_of(r);
        const long long c = row_cost(len);
        cost_all += c;
        if (cost.bundle_min > 0 && len > cost.bundle_min) {
            brows.push_back(r);
            cost_b += c;
            pre[r + 1] = pre[r];
        } else {
            pre[r + 1] = pre[r] + c;
        }
    }
    int cta_b = 0;
    {
        const int nbundles = (int)(brows.size() + kWWarps - 1) / kWWarps;
        if (nbundles > 0) {
            cta_b = (int)((double)ncta * cost_b / std::max(cost_all, 1LL) + 0.5);
            if (cost_b < cost_all) cta_b = std::min(cta_b, ncta - 1);  // keep a CTA for the other rows
            if (cta_b < nbundles) {                                    // too few CTAs: no bundles
                brows.clear();
                cta_b = 0;
                for (int r = 0; r < nrows; ++r) pre[r + 1] = pre[r] + row_cost(len_of(r));
            }
        }
    }
    const int nb = (int)(brows.size() + kWWarps - 1) / kWWarps;
    std::vector<char> bundled(nrows > 0 ? nrows : 1, 0);
    for (int r : brows) bundled[r] = 1;
    // weight of bundle b: its longest row; prefix wpre, CTA c's range
    // [bound(c), bound(c + 1)) of the total
    std::vector<long long> wpre(nb + 1, 0);
    for (int b = 0; b < nb; ++b) {
        long long mx = 0;
        for (int j = 0; j < kWWarps && b * kWWarps + j < (int)brows.size(); ++j)
            mx = std::max(mx, row_cost(len_of(brows[b * kWWarps + j])));
        wpre[b + 1] = wpre[b] + std::max(mx, 1LL);
    }
    auto bound = [&](int c) -> long long { return cta_b > 0 ? wpre[nb] * c / cta_b : 0; };

    // contiguous cut of the other rows over warps [wb, nwarps); a cut may
    // fall inside a row longer than split_min, at a nonzero index rounded to
    // a multiple of 32 (aligned loads)
    const int wb = cta_b * kWWarps;
    const int nw = nwarps - wb;
    const long long total = pre[nrows];
    std::vector<Cut> cut(nw + 1);
    cut[0] = Cut{0, 0};
    cut[nw] = Cut{nrows, nnz};
    int rw = 0;  // the targets grow with w: the row holding target t is found by walking forward
    for (int w = 1; w < nw; ++w) {
        Cut c{nrows, nnz};
        if (nrows > 0 && total > 0) {
            const long long t = (long long)((double)total * w / nw);
            while (rw < nrows - 1 && pre[rw + 1] <= t) ++rw;  // the last row r with pre[r] <= t
            const int r = rw;
            const int len = len_of(r);
            if (len > cost.split_min) {
                long long o = t - pre[r] - cost.stream_row;
                o = std::min<long long>(std::max<long long>(o, 0), len);
                long long k = rp[r] + o;
                k = ((k + 16) / 32) * 32;
                if (k <= rp[r]) c = Cut{r, rp[r]};
                else if (k >= rp[r + 1]) c = Cut{r + 1, rp[r + 1]};
                else c = Cut{r, (int)k};
            } else {
                c = 2 * (t - pre[r]) < pre[r + 1] - pre[r] ? Cut{r, rp[r]} : Cut{r + 1, rp[r + 1]};
            }
        }
        if (before(c, cut[w - 1])) c = cut[w - 1];
        cut[w] = c;
    }
    auto interior = [&](const Cut &c) { return c.r < nrows && c.k > rp[c.r]; };

    // the element of row r of bundle b at weight B: the same rounding for
    // the two CTAs that share a boundary, so the parts tile the row
    auto cutp = [&](int r, int b, long long B) -> int {
        if (B <= wpre[b]) return rp[r];
        if (B >= wpre[b + 1]) return rp[r + 1];
        long long e = rp[r] + (long long)len_of(r) * (B - wpre[b]) / (wpre[b + 1] - wpre[b]);
        e = ((e + 16) / 32) * 32;
        return (int)std::min<long long>(std::max<long long>(e, rp[r]), rp[r + 1]);
    };
    // the non-empty parts of bundle warp w, in row order: (row, lo, hi)
    struct Part {
        int r, lo, hi;
    };
    auto bparts = [&](int w, std::vector<Part> &out) {
        out.clear();
        const int c = w / kWWarps, j = w % kWWarps;
        const long long B0 = bound(c), B1 = bound(c + 1);
        if (B0 >= B1) return;
        int b = (int)(std::upper_bound(wpre.begin(), wpre.end(), B0) - wpre.begin()) - 1;
        for (; b < nb && wpre[b] < B1; ++b) {
            if (b * kWWarps + j >= (int)brows.size()) continue;
            const int r = brows[b * kWWarps + j];
            const int lo = cutp(r, b, B0), hi = cutp(r, b, B1);
            if (lo < hi) out.push_back(Part{r, lo, hi});
        }
    };
    std::vector<Part> parts;
    std::vector<int> npieces(nrows > 0 ? nrows : 1, 0);
    for (int w = 0; w < cta_b * kWWarps; ++w) {
        bparts(w, parts);
        for (const Part &q : parts) ++npieces[q.r];
    }

    // rows cut between warps, in row order
    std::vector<int> split_rows;
    for (int w = 1; w < nw; ++w)
        if (interior(cut[w]) && (split_rows.empty() || split_rows.back() != cut[w].r)) split_rows.push_back(cut[w].r);
    for (int r : brows)
        if (npieces[r] >= 2) split_rows.push_back(r);
    std::sort(split_rows.begin(), split_rows.end());
    std::vector<int> sid(nrows > 0 ? nrows : 1, -1);
    for (size_t l = 0; l < split_rows.size(); ++l) sid[split_rows[l]] = (int)l;
    auto id_of = [&](int r) -> int { return sid[r]; };

    P.wpart.assign(nwarps + 1, 0);
    P.wsplit.assign(nwarps, WSplit{-1, -1, -1, -1});
    std::vector<int> nparts(split_rows.size(), 0);
    for (int w = 0; w < wb; ++w) {
        P.wpart[w] = (int)P.items.size();
        bparts(w, parts);
        for (const Part &q : parts) {
            const int h = id_of(q.r);
            if (h >= 0) {  // at most two: a part of a bundle inside the range is not split
                if (P.wsplit[w].head < 0) P.wsplit[w].head = h;
                else P.wsplit[w].tail = h;
                ++nparts[h];
            }
            P.items.push_back(WItem{q.r, q.r + 1, q.lo, q.hi});
        }
    }
    for (int v = 0; v < nw; ++v) {
        const int w = wb + v;
        P.wpart[w] = (int)P.items.size();
        const Cut a = cut[v], b = cut[v + 1];
        if (!before(a, b)) continue;  // empty range
        const int r_end = interior(b) ? b.r + 1 : b.r;  // one past the last row touched
        // split rows at the ends of the range
        const int h = bundled[a.r] ? -1 : id_of(a.r);
        const int t = (r_end - 1 != a.r && !bundled[r_end - 1]) ? id_of(r_end - 1) : -1;
        if (h >= 0) P.wsplit[w].head = h, ++nparts[h];
        if (t >= 0) P.wsplit[w].tail = t, ++nparts[t];
        int r = a.r;
        while (r < r_end) {
            if (bundled[r]) {
                ++r;
                continue;
            }
            const bool part = id_of(r) >= 0;
            const int len = len_of(r);
            if (len > kGroupMaxLen || part) {
                const int r0 = r;
                const int k0 = r == a.r ? a.k : rp[r];
                while (r < r_end && !bundled[r] && (len_of(r) > kGroupMaxLen || id_of(r) >= 0)) ++r;
                const int k1 = (r == r_end && interior(b)) ? b.k : rp[r];
                P.items.push_back(WItem{r0, r, k0, k1});
            } else {
                const int G = group_width_of(len);
                const int r0 = r;
                while (r < r_end && !bundled[r] && len_of(r) <= kGroupMaxLen && id_of(r) < 0 &&
                       group_width_of(len_of(r)) == G)
                    ++r;
                P.items.push_back(WItem{r0, r, -G, 0});
            }
        }
    }
    P.wpart[nwarps] = (int)P.items.size();
    // slots of the split rows' parts, in warp order
    P.split.resize(split_rows.size());
    int slot = 0;
    for (size_t l = 0; l < split_rows.size(); ++l) {
        P.split[l] = SplitRow{split_rows[l], slot, nparts[l], 0};
        slot += nparts[l];
    }
    P.nslots = slot;
    std::vector<int> next(split_rows.size(), 0);
    for (int w = 0; w < nwarps; ++w) {
        WSplit &s = P.wsplit[w];
        if (s.head >= 0) s.head_slot = P.split[s.head].slot0 + next[s.head]++;
        if (s.tail >= 0) s.tail_slot = P.split[s.tail].slot0 + next[s.tail]++;
    }
    return P;
}

}  // namespace gb
