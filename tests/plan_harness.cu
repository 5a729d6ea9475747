// Host-only check of the warp-stream SpMV plan (build_wplan) on seeded
// random row-length profiles: the host replays the device's walk of every
// warp's items (stream items in aligned 32-element steps, group items in
// rounds of lane groups, split rows' parts published to their slots) and
// checks that every nonzero is visited once, every row is finished once
// (whole, or from all of its parts in warp order), that at most one row
// ends inside a 32-element step of a stream item, and that group rows fit
// their lane groups.  Prints "ok" or the first violated invariant.  Built
// and run by tests/test_host_plan.py (no GPU needed).  With --time it times
// the plans of the 100000 x 1000 Lasso workload's A and [P A'] instead.
#include <chrono>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../paper_1912_04263_gb300/csrc/spmv.cuh"

using namespace gb;

#define REQUIRE(c, ...)                          \
    do {                                         \
        if (!(c)) {                              \
            printf(__VA_ARGS__);                 \
            printf("\n");                        \
            return 1;                            \
        }                                        \
    } while (0)

template <class F>
static double mean_ms(F f, int reps) {
    const auto t0 = std::chrono::steady_clock::now();
    for (int k = 0; k < reps; ++k) f();
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() / reps;
}

// Row lengths of the Lasso workload: A has 100000 rows of 1 + Binomial(1000,
// 0.15) nonzeros and 2000 rows of 2; [P A'] has 1000 rows of 2 +
// Binomial(100000, 0.15), then 101000 rows of 2.
static int time_lasso_plans() {
    std::mt19937 rng(1);
    std::binomial_distribution<int> row(1000, 0.15), col(100000, 0.15);
    std::vector<int> rpA(1, 0), rpP(1, 0);
    for (int r = 0; r < 100000; ++r) rpA.push_back(rpA.back() + row(rng) + 1);
    for (int r = 0; r < 2000; ++r) rpA.push_back(rpA.back() + 2);
    for (int r = 0; r < 1000; ++r) rpP.push_back(rpP.back() + col(rng) + 2);
    for (int r = 0; r < 101000; ++r) rpP.push_back(rpP.back() + 2);
    const char *names[2] = {"A", "[P A']"};
    const std::vector<int> *rps[2] = {&rpA, &rpP};
    for (int i = 0; i < 2; ++i) {
        WPlanCost cost;
        cost.bundle_min = 4096;
        WPlanHost p = build_wplan(*rps[i], 152 * 4 * kWWarps, cost);
        const double t = mean_ms([&] { p = build_wplan(*rps[i], 152 * 4 * kWWarps, cost); }, 100);
        printf("%s: %zu items, %zu split rows for %d warps; build_wplan %.3f ms\n", names[i], p.items.size(),
               p.split.size(), p.nwarps, t);
    }
    return 0;
}

// Replay the device walk of plan P over row pointer rp.
static int replay(const std::vector<int> &rp, const WPlanHost &P) {
    const int nrows = (int)rp.size() - 1;
    const int nnz = rp[nrows];
    std::vector<int> seen(nnz, 0), finished(nrows, 0), parts(P.split.size(), 0);
    std::vector<int> slot_used(P.nslots, 0);
    REQUIRE((int)P.wpart.size() == P.nwarps + 1 && P.wpart[0] == 0 && P.wpart[P.nwarps] == (int)P.items.size(),
            "wpart bounds");
    for (size_t l = 0; l < P.split.size(); ++l) {
        REQUIRE(P.split[l].nparts >= 2, "split row %zu has %d parts", l, P.split[l].nparts);
        REQUIRE(l == 0 || P.split[l].row > P.split[l - 1].row, "split rows not in row order");
        REQUIRE(P.split[l].slot0 >= 0 && P.split[l].slot0 + P.split[l].nparts <= P.nslots, "slot range");
    }
    for (int w = 0; w < P.nwarps; ++w) {
        REQUIRE(P.wpart[w] <= P.wpart[w + 1], "wpart not monotone at warp %d", w);
        const WSplit ws = P.wsplit[w];
        const int head_row = ws.head >= 0 ? P.split[ws.head].row : -1;
        const int tail_row = ws.tail >= 0 ? P.split[ws.tail].row : -1;
        REQUIRE(ws.head < 0 || ws.tail < 0 || head_row < tail_row, "warp %d head/tail order", w);
        auto finish = [&](int r) -> int {
            if (r == head_row || r == tail_row) {
                const int l = r == head_row ? ws.head : ws.tail;
                const int slot = r == head_row ? ws.head_slot : ws.tail_slot;
                REQUIRE(slot >= P.split[l].slot0 && slot < P.split[l].slot0 + P.split[l].nparts, "slot of warp %d", w);
                REQUIRE(slot_used[slot]++ == 0, "slot %d used twice", slot);
                if (++parts[l] == P.split[l].nparts) ++finished[r];
            } else {
                ++finished[r];
            }
            return 0;
        };
        for (int i = P.wpart[w]; i < P.wpart[w + 1]; ++i) {
            const WItem it = P.items[i];
            REQUIRE(it.r0 >= 0 && it.r0 < it.r1 && it.r1 <= nrows, "item %d rows [%d, %d)", i, it.r0, it.r1);
            if (it.k0 >= 0) {
                REQUIRE(it.k0 >= rp[it.r0] && it.k0 < rp[it.r0 + 1], "stream item %d start", i);
                REQUIRE(it.k1 > rp[it.r1 - 1] && it.k1 <= rp[it.r1], "stream item %d end", i);
                for (int r = it.r0; r < it.r1; ++r) {
                    const bool part = r == head_row || r == tail_row;
                    REQUIRE(part || rp[r + 1] - rp[r] > kGroupMaxLen, "short row %d in a stream item", r);
                    REQUIRE(!part || r == it.r0 || r == it.r1 - 1, "split row %d inside an item", r);
                }
                // walk in aligned steps: at most one row end strictly inside the item per step
                const int base = it.k0 & ~31;
                const int nsteps = (it.k1 - base + 31) >> 5;
                // the device loads whole batches of 4 steps: inside the arrays and their zeroed slack
                const long long loaded = 32LL * 4 * ((nsteps + 3) / 4);
                REQUIRE(base >= 0 && (long long)base + loaded <= (long long)nnz + kSlack,
                        "item %d loads [%d, %lld) outside the %d nonzeros and their slack", i, base, base + loaded, nnz);
                int row = it.r0;
                for (int s = base; s < it.k1; s += 32) {
                    int ends = 0;
                    for (int e = std::max(s, it.k0); e < std::min(s + 32, it.k1); ++e) {
                        while (e >= rp[row + 1]) {
                            if (finish(row)) return 1;
                            ++row;
                            ++ends;
                        }
                        ++seen[e];
                    }
                    REQUIRE(ends <= 1, "item %d: %d row ends in one step", i, ends);
                }
                REQUIRE(row == it.r1 - 1, "item %d walk ended at row %d", i, row);
                if (finish(row)) return 1;
            } else {
                const int G = -it.k0;
                REQUIRE(G == 1 || G == 2 || G == 4 || G == 8 || G == 16, "group width %d", G);
                for (int r = it.r0; r < it.r1; ++r) {
                    const int len = rp[r + 1] - rp[r];
                    REQUIRE(len <= 2 * G && group_width_of(len) == G, "row %d of length %d in a group of %d", r, len,
                            G);
                    REQUIRE(r != head_row && r != tail_row, "split row %d in a group item", r);
                    for (int e = rp[r]; e < rp[r + 1]; ++e) ++seen[e];
                    ++finished[r];
                }
            }
        }
    }
    for (int e = 0; e < nnz; ++e) REQUIRE(seen[e] == 1, "nonzero %d visited %d times", e, seen[e]);
    for (int r = 0; r < nrows; ++r) REQUIRE(finished[r] == 1, "row %d finished %d times", r, finished[r]);
    for (int s = 0; s < P.nslots; ++s) REQUIRE(slot_used[s] == 1, "slot %d unused", s);
    return 0;
}

int main(int argc, char **argv) {
    if (argc > 1 && std::strcmp(argv[1], "--time") == 0) return time_lasso_plans();
    std::mt19937 rng(12345);
    for (int trial = 0; trial < 600; ++trial) {
        const int nrows = (int)(rng() % 3000);
        std::vector<int> rp(nrows + 1, 0);
        const int mode = trial % 4;
        for (int r = 0; r < nrows; ++r) {
            const int k = (int)(rng() % 10);
            int len;
            if (mode == 0) len = k < 4 ? (int)(rng() % 4) : k < 7 ? (int)(rng() % 200) : k < 9 ? (int)(rng() % 3000) : (int)(rng() % 20000);
            else if (mode == 1) len = (int)(rng() % 40);          // around the group / stream boundary
            else if (mode == 2) len = k == 0 ? (int)(rng() % 50000) : (int)(rng() % 3);  // few long rows
            else len = 33 + (int)(rng() % 300);                     // stream rows only
            rp[r + 1] = rp[r] + len;
        }
        const int nwarps = 1 + (int)(rng() % 5000);
        WPlanCost cost;
        if (trial % 3 == 1) cost.split_min = 33 + (int)(rng() % 400);
        if (trial % 5 == 2) cost.group_row = (int)(rng() % 64);
        if (trial % 2 == 1) cost.bundle_min = 33 + (int)(rng() % 3000);
        const WPlanHost P = build_wplan(rp, nwarps, cost);
        if (replay(rp, P)) {
            printf("trial %d (rows %d, warps %d)\n", trial, nrows, nwarps);
            return 1;
        }
    }
    printf("ok\n");
    return 0;
}
