// Host-only check of the SpMV work plan (build_plan) and of the CTA
// partition (partition_items) on seeded random row-length profiles; prints
// "ok" or the first violated invariant.  Built and run by
// tests/test_host_plan.py (no GPU needed).  With --time it instead times
// both on the row-length profiles of the 100000 x 1000 Lasso workload's A and
// [P A'] (the per-set-up host cost of the plans).
#include <chrono>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../paper_1912_04263_gb300/csrc/common.cuh"

using namespace gb;

static int group_width_of(long long avg) {
    return avg >= 24 ? 32 : avg >= 12 ? 16 : avg >= 6 ? 8 : avg >= 3 ? 4 : 1;
}

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
        HostPlan hp = build_plan(*rps[i]);
        const double b = mean_ms([&] { hp = build_plan(*rps[i]); }, 200);
        const double p608 = mean_ms([&] { volatile size_t n = partition_items(hp, 608).part.size(); (void)n; }, 200);
        const double p456 = mean_ms([&] { volatile size_t n = partition_items(hp, 456).part.size(); (void)n; }, 200);
        printf("%s: %zu items, %zu long rows; build_plan %.3f ms, partition(608) %.3f ms, partition(456) %.3f ms\n",
               names[i], hp.items.size(), hp.longrows.size(), b, p608, p456);
    }
    return 0;
}

int main(int argc, char **argv) {
    if (argc > 1 && std::strcmp(argv[1], "--time") == 0) return time_lasso_plans();
    std::mt19937 rng(12345);
    for (int trial = 0; trial < 400; ++trial) {
        const int nrows = 1 + (int)(rng() % 4000);
        std::vector<int> rp(nrows + 1, 0);
        for (int r = 0; r < nrows; ++r) {
            const int k = (int)(rng() % 10);
            const int len = k < 4 ? (int)(rng() % 4) : k < 7 ? (int)(rng() % 200)
                            : k < 9 ? (int)(rng() % 5000) : (int)(rng() % 30000);
            rp[r + 1] = rp[r] + len;
        }
        const HostPlan hp = build_plan(rp);
        // items tile the nonzeros in order; rows are covered once
        long long next_k = 0;
        int next_row = 0;
        size_t lr_seen = 0;
        for (size_t i = 0; i < hp.items.size(); ++i) {
            const Item &it = hp.items[i];
            if (it.k0 != next_k || it.k1 < it.k0) { printf("gap or overlap at item %zu\n", i); return 1; }
            if (it.k1 - it.k0 > kCap) { printf("item %zu over the cap\n", i); return 1; }
            if (it.r1 >= 0) {  // run of short rows
                if (it.r0 != next_row || it.r1 <= it.r0) { printf("row order at item %zu\n", i); return 1; }
                if (rp[it.r0] != it.k0 || rp[it.r1] != it.k1) { printf("row bounds at item %zu\n", i); return 1; }
                const int rows = it.r1 - it.r0;
                const int gw = group_width_of((long long)(it.k1 - it.k0) / rows);
                if (rows > 1 && rows * gw > (gw <= 4 ? 1 : 2) * kThreads) { printf("rounds at item %zu\n", i); return 1; }
                next_row = it.r1;
            } else {  // piece of a long row
                const int lr = -(it.r1 + 1);
                if (lr < 0 || (size_t)lr >= hp.longrows.size()) { printf("long-row id at item %zu\n", i); return 1; }
                const LongRow &L = hp.longrows[lr];
                const int len = rp[it.r0 + 1] - rp[it.r0];
                if (len <= kCap) { printf("short row cut into pieces at item %zu\n", i); return 1; }
                const int piece = (int)i - L.first_item;
                if (piece < 0 || piece >= L.npieces) { printf("piece index at item %zu\n", i); return 1; }
                const int np = L.npieces;
                if (np != (len + kCap - 1) / kCap) { printf("piece count of long row %d\n", lr); return 1; }
                const int plen = it.k1 - it.k0;
                if (plen < len / np - 1 || plen > len / np + 1) { printf("uneven piece at item %zu\n", i); return 1; }
                if (piece == 0) {
                    if (it.r0 != next_row || it.k0 != rp[it.r0]) { printf("long row start at item %zu\n", i); return 1; }
                    if ((size_t)lr != lr_seen++) { printf("long-row ids out of order\n"); return 1; }
                }
                if (piece == np - 1) {
                    if (it.k1 != rp[it.r0 + 1]) { printf("long row end at item %zu\n", i); return 1; }
                    next_row = it.r0 + 1;
                }
            }
            next_k = it.k1;
        }
        // trailing empty rows form short items too; everything is covered
        if (next_k != rp[nrows] || next_row != nrows) { printf("rows not covered (trial %d)\n", trial); return 1; }
        const int n = (int)hp.items.size();
        for (int grid : {1, 2, 7, 152, 608, 1000, 4000}) {
            if (grid > n) continue;
            const HostPartition P = partition_items(hp, grid);
            if ((int)P.part.size() != grid + 1 || P.part[0] != 0 || P.part[grid] != n) { printf("partition ends\n"); return 1; }
            for (int b = 0; b < grid; ++b)
                if (P.part[b + 1] <= P.part[b]) { printf("empty CTA %d of %d\n", b, grid); return 1; }
            for (size_t l = 0; l < hp.longrows.size(); ++l) {
                const int f = hp.longrows[l].first_item, e = f + hp.longrows[l].npieces - 1;
                const int c0 = P.lr_cta[l].x, c1 = P.lr_cta[l].y;
                if (!(P.part[c0] <= f && f < P.part[c0 + 1] && P.part[c1] <= e && e < P.part[c1 + 1])) {
                    printf("CTA range of long row %zu\n", l);
                    return 1;
                }
            }
        }
    }
    printf("ok\n");
    return 0;
}
