// Allocation-free SpMV entry point (gbosqp_spmv_noalloc, include/gbosqp.h).
//
// Some callers cannot let the library allocate device memory while they
// run: a real-time or control loop that must not take the allocator's
// latency (cudaMalloc and cudaFree can take milliseconds and cudaFree waits
// for the whole device), code that is recording a CUDA stream capture (a
// device-wide synchronisation there invalidates the capture), and hosts
// whose device memory is owned by another allocator (a framework's caching
// allocator may leave nothing free, so an allocation could fail mid-loop).
// For them the SpMV's scratch (the partial sums and ticket counters that
// combine the pieces of long rows) lives in a fixed file-scope device array
// that comes with the library's module and stays resident until the process
// exits, instead of being allocated.
#include <mutex>
#include <string>

#include "common.cuh"
#include "engine.cuh"
#include "handle.cuh"

namespace {

// Capacity: work items and long rows of one matrix plan.
constexpr long long kMaxItems = 1LL << 17;     // 131072 items (2 MiB of partial sums)
constexpr long long kMaxLongRows = 1LL << 17;  // 131072 long rows (512 KiB of counters)
constexpr size_t kPartBytes = 2 * sizeof(double) * (size_t)kMaxItems;
constexpr size_t kCountBytes = sizeof(int) * (size_t)kMaxLongRows;

}  // namespace

// The scratch.  In host code this name is a host-side stand-in, not a device
// address: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_spmv_scratch[kPartBytes + kCountBytes];

namespace {

std::mutex g_mu;
void *g_scratch_addr[256] = {};  // device address of g_spmv_scratch, per device ordinal

// Device address of the scratch on the current device (set up on the first
// call for each device, with that device current).
void *scratch_address(int device) {
    if (device < 0 || device >= 256) gb::fail(GBOSQP_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_spmv_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            gb::fail(GBOSQP_ERR_CUDA, std::string("cudaGetSymbolAddress of the SpMV scratch failed: ") +
                                          cudaGetErrorString(e));
        }
        g_scratch_addr[device] = p;
    }
    return g_scratch_addr[device];
}

}  // namespace

extern "C" int gbosqp_spmv_noalloc(gbosqp_handle *h, int which, const void *x, void *y) {
    if (!h || !h->eng || !x || !y) return GBOSQP_ERR_INVALID_ARG;
    if (which != GBOSQP_MAT_A && which != GBOSQP_MAT_PAT) {
        h->err = "bad matrix selector";
        return GBOSQP_ERR_INVALID_ARG;
    }
    try {
        GB_CUDA(cudaSetDevice(h->s.device));
        char *base = static_cast<char *>(scratch_address(h->s.device));
        h->eng->spmv_noalloc(which, x, y, reinterpret_cast<double *>(base), reinterpret_cast<int *>(base + kPartBytes),
                             kMaxItems, kMaxLongRows);
        return GBOSQP_OK;
    } catch (const gb::GbError &e) {
        h->err = e.msg;
        return e.code;
    } catch (const std::exception &e) {
        h->err = e.what();
        return GBOSQP_ERR_CUDA;
    }
}
