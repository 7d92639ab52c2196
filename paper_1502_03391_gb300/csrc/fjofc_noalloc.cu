// fjofc_embed_noalloc: the in-sample embedding with all of its device scratch in one
// fixed, file-scope device array instead of memory obtained at call time.
//
// Some callers cannot allocate device memory while they run: real-time or embedded loops
// that must not touch the allocator (or any framework's caching allocator) after
// start-up, processes whose device memory is carved up once at launch by another
// component, and code that must not fail part-way for lack of memory.  For them this
// entry point takes the same arguments as fjofc_embed and uses only the caller's buffers
// plus the array below.  It launches kernels and synchronises the caller's stream like
// fjofc_embed, so it is called from ordinary host code.
//
// The array (kNoallocScratchBytes) lives in this translation unit's device module, so
// every GPU on which that module is loaded keeps it until the process exits.  Its
// device address is looked up once per device with cudaGetSymbolAddress (host code
// cannot use the array's name as a device address: on the host that name refers to a
// host-side shadow).  Under lazy module loading that first lookup, and the first launch
// of each kernel, load device code, which allocates: callers make one call per device at
// start-up.  Calls share the array, which keeps whatever the previous call left there;
// the kernels clear everything that must start at zero (status block, work ticket,
// barrier counter, centring means, walk offsets) at the start of every call, and every
// partial is written before it is read.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "fjofc_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(FJOFC_NOALLOC_SCRATCH_BYTES);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        fjofc::set_message("no usable current CUDA device");
        return FJOFC_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
            cudaGetLastError();
            fjofc::set_message(msg);
            return FJOFC_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return FJOFC_OK;
}

}  // namespace

extern "C" int fjofc_embed_noalloc(int32_t m, int64_t n, int32_t d, const void* const* delta, int64_t ld,
                                   int32_t delta_dtype, const float* delta_scale, const double* weights, float* X,
                                   const fjofc_opts* opts, fjofc_result* res, void* cuda_stream) {
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc == FJOFC_OK) {
        const fjofc::ExtScratch ext{base, kNoallocScratchBytes};
        rc = fjofc::run_insample(m, n, d, delta, ld, delta_dtype, delta_scale, weights, X, opts, res,
                                 static_cast<cudaStream_t>(cuda_stream), false, nullptr, &ext);
    }
    if (res) res->status = rc;
    return rc;
}
