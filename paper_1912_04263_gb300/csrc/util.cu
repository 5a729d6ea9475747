// Host utilities: errors, device buffers, launch geometry, and the
// row-block work plan of the CSR SpMV kernels.
#include <algorithm>
#include <string>

#include "common.cuh"

namespace gb {

thread_local long long g_launches = 0;

void fail(int code, const std::string &msg) { throw GbError{code, msg}; }

void check_cuda(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    cudaGetLastError();
    const int code = (e == cudaErrorMemoryAllocation) ? GBOSQP_ERR_OOM : GBOSQP_ERR_CUDA;
    throw GbError{code, std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" + std::to_string(line) + ")"};
}

namespace {
thread_local cudaStream_t g_pool_stream = nullptr;
thread_local bool g_pool_on = false;
}  // namespace

PoolScope::PoolScope(cudaStream_t s) : prev(g_pool_stream) {
    g_pool_stream = s;
    g_pool_on = true;
}
PoolScope::~PoolScope() {
    g_pool_stream = prev;
    g_pool_on = prev != nullptr;
}

void DevBuf::alloc(size_t nbytes) {
    release();
    if (nbytes == 0) nbytes = 16;
    cudaError_t e;
    if (g_pool_on) {
        e = cudaMallocAsync(&p, nbytes, g_pool_stream);
        pooled = e == cudaSuccess;
        pool_stream = g_pool_stream;
    } else {
        e = cudaMalloc(&p, nbytes);
        pooled = false;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        pooled = false;
        fail(GBOSQP_ERR_OOM, "device allocation of " + std::to_string(nbytes) + " bytes failed: " +
                                 cudaGetErrorString(e));
    }
    bytes = nbytes;
}

void DevBuf::release() {
    if (p) {
        if (pooled) cudaFreeAsync(p, pool_stream);
        else cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
    pooled = false;
}

int device_sm_count() {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(sms, 1);
}

int grid_for_items(int nitems, const void *kernel, int smem_dynamic) {
    int per_sm = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem_dynamic));
    per_sm = std::max(per_sm, 1);
    return std::max(1, std::min(nitems, device_sm_count() * per_sm));
}

int grid_for_n(long long n, int threads) { return (int)std::max(1LL, (n + threads - 1) / threads); }

// Lane-group width the kernels use for an item with mean row length avg
// (must match the choice in run_items).
static int group_width(long long avg) {
    return avg >= 24 ? 32 : avg >= 12 ? 16 : avg >= 6 ? 8 : avg >= 3 ? 4 : 1;
}

// Cut the rows into work items: runs of consecutive rows with at most kCap
// nonzeros and few enough rows that the CTA's lane groups reduce them in one
// round when rows are short (group width <= 4: the cost is each row's
// epilogue, a chain of dependent memory accesses) and in two rounds
// otherwise (the cost is summing the row), so that items cost about the
// same; a row longer than kCap becomes ceil(len / kCap) pieces of nearly
// equal length.
HostPlan build_plan(const std::vector<int> &rp) {
    HostPlan hp;
    const int nrows = (int)rp.size() - 1;
    int r = 0;
    while (r < nrows) {
        const long long len = (long long)rp[r + 1] - rp[r];
        if (len > kCap) {
            const int np = (int)((len + kCap - 1) / kCap);
            const int id = (int)hp.longrows.size();
            hp.longrows.push_back(LongRow{(int)hp.items.size(), np});
            for (int p = 0; p < np; ++p) {
                const int k0 = rp[r] + (int)(len * p / np);
                const int k1 = rp[r] + (int)(len * (p + 1) / np);
                hp.items.push_back(Item{r, -(id + 1), k0, k1});
            }
            ++r;
            continue;
        }
        const int r0 = r;
        long long tot = 0;
        while (r < nrows) {
            const long long l = (long long)rp[r + 1] - rp[r];
            if (l > kCap || tot + l > kCap) break;
            const long long rows = r - r0 + 1;
            const int gw = group_width((tot + l) / rows);
            const long long rounds = gw <= 4 ? 1 : 2;  // short rows: one epilogue per thread
            if (rows > 1 && rows * gw > rounds * kThreads) break;
            tot += l;
            ++r;
        }
        hp.items.push_back(Item{r0, r, rp[r0], rp[r]});
    }
    return hp;
}

HostPartition partition_items(const HostPlan &hp, int grid) {
    HostPartition out;
    const int n = (int)hp.items.size();
    grid = std::max(1, std::min(grid, std::max(n, 1)));
    std::vector<long long> prefix(n + 1, 0);
    for (int i = 0; i < n; ++i)
        prefix[i + 1] = prefix[i] + (long long)(hp.items[i].k1 - hp.items[i].k0) + kItemCost;
    out.part.assign(grid + 1, 0);
    out.part[grid] = n;
    for (int b = 1; b < grid; ++b) {
        const long long target = (long long)((double)prefix[n] * b / grid);
        int j = (int)(std::lower_bound(prefix.begin(), prefix.end(), target) - prefix.begin());
        if (j > 0 && target - prefix[j - 1] < prefix[j] - target) --j;  // nearer boundary
        // strictly increasing, leaving one item for each remaining CTA
        j = std::max(j, out.part[b - 1] + 1);
        j = std::min(j, n - (grid - b));
        out.part[b] = j;
    }
    out.lr_cta.resize(hp.longrows.size());
    auto cta_of = [&](int item) {
        return (int)(std::upper_bound(out.part.begin(), out.part.end(), item) - out.part.begin()) - 1;
    };
    for (size_t l = 0; l < hp.longrows.size(); ++l) {
        const LongRow &L = hp.longrows[l];
        out.lr_cta[l] = make_int2(cta_of(L.first_item), cta_of(L.first_item + L.npieces - 1));
    }
    return out;
}

}  // namespace gb
