// Host utilities: errors, device buffers, launch geometry.
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

int grid_for_n(long long n, int threads) { return (int)std::max(1LL, (n + threads - 1) / threads); }

}  // namespace gb
