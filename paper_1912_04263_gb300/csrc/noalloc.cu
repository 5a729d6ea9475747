// Allocation-free SpMV entry point (gbosqp_spmv_noalloc, include/gbosqp.h).
//
// Some callers cannot let the library allocate device memory while they
// run: a real-time or control loop that must not take the allocator's
// latency (cudaMalloc and cudaFree can take milliseconds and cudaFree waits
// for the whole device), code that is recording a CUDA stream capture (a
// device-wide synchronisation there invalidates the capture), and hosts
// whose device memory is owned by another allocator (a framework's caching
// allocator may leave nothing free, so an allocation could fail mid-loop).
// For them the SpMV's scratch (the tickets and partial sums that combine the
// parts of rows cut between warps) lives in a fixed file-scope device array
// that comes with the library's module and stays resident until the process
// exits, instead of being allocated.
#include <mutex>
#include <string>

#include "common.cuh"
#include "engine.cuh"
#include "handle.cuh"

namespace {

// Capacity.  A plan needs at most 4 + 2 * 16 + 16 = 52 bytes per warp of the
// launch (one split row and two partial-sum slots per warp at most), so
// 1 MiB serves grids of up to about 20000 warps (a full GB300 runs 9728).
constexpr size_t kScratchBytes = (size_t)1 << 20;

}  // namespace

// The scratch.  In host code this name is a host-side stand-in, not a device
// address: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_spmv_scratch[kScratchBytes];

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
        unsigned char *base = static_cast<unsigned char *>(scratch_address(h->s.device));
        h->eng->spmv_noalloc(which, x, y, base, kScratchBytes);
        return GBOSQP_OK;
    } catch (const gb::GbError &e) {
        h->err = e.msg;
        return e.code;
    } catch (const std::exception &e) {
        h->err = e.what();
        return GBOSQP_ERR_CUDA;
    }
}
