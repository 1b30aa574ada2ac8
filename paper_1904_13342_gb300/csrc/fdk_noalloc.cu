// pyro_fdk_noalloc: FDK for callers that cannot allocate device memory.
//
// pyro_fdk needs a caller-provided workspace for the weighted, filtered
// sinogram.  Some callers cannot provide one: code that only ever receives
// the input and output buffers (for example a reconstruction stage plugged
// into an acquisition pipeline, or a host application whose own allocator
// owns all device memory and forbids allocations while it runs) has no way
// to call cudaMalloc or to hand out extra device memory.  This entry point
// takes its scratch from a fixed, file-scope device array instead and then
// runs exactly the pyro_fdk kernels.
//
// Rules of use:
//  * The array holds PYRO_FDK_NOALLOC_SCRATCH_BYTES (64 MiB); problems whose
//    filtered sinogram (4 * batch * n_views * nv * nu bytes) is larger are
//    rejected with PYRO_EWORKSPACE before anything is enqueued.
//  * The array belongs to the loaded library: every GPU that loads this
//    module keeps it allocated until the process exits.
//  * The first call on a device looks up the array's device address (with
//    that device current) and caches it, keyed by the device and its current
//    CUDA context: a context created anew on that device (after a
//    cudaDeviceReset, say) reloads the module, so its first call looks the
//    address up again.  Make the first call in a context before any stream
//    capture on that device.
//  * Every call on a device shares the one array and it keeps the contents
//    of the last call.  The filter stage overwrites every scratch element it
//    reads back, so nothing needs clearing; but calls whose work overlaps on
//    the GPU (different streams, or different host threads, without
//    ordering between them) race on the array and corrupt each other.
//  * It calls no cudaMalloc, cudaFree or other allocating routine.
#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_fdk_scratch[PYRO_FDK_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
// (device ordinal, current context) -> device address of g_fdk_scratch
std::map<std::pair<int, CUcontext>, void *> g_scratch_addr;

using CtxGetCurrentFn = CUresult (*)(CUcontext *);

// the calling thread's current context (the runtime's primary context once
// any runtime call has run on the device); NULL when the CUDA driver entry point
// is unavailable, which then keys by the device alone
CUcontext current_context()
{
    static CtxGetCurrentFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return (CtxGetCurrentFn)f;
    }();
    CUcontext c = nullptr;
    if (fn == nullptr || fn(&c) != CUDA_SUCCESS) c = nullptr;
    return c;
}

}  // namespace

extern "C" PYRO_API int pyro_fdk_noalloc(const void *sino, void *vol, int batch, const pyro_geom3d *g,
                                         pyro_filter kind, const float *custom_K, pyro_redund redund,
                                         pyro_dtype dtype, void *stream)
{
    const size_t need = pyro_fdk_workspace_bytes(g, batch);
    if (g == nullptr || batch < 0) return pyro_fdk(sino, vol, batch, g, kind, custom_K, redund, nullptr, 0, dtype, stream);
    if (need > (size_t)PYRO_FDK_NOALLOC_SCRATCH_BYTES) {
        pyro::set_last_error("pyro_fdk_noalloc: this problem needs %zu bytes of scratch but the static scratch holds "
                             "%zu bytes (64 MiB); use pyro_fdk with a caller workspace",
                             need, (size_t)PYRO_FDK_NOALLOC_SCRATCH_BYTES);
        return PYRO_EWORKSPACE;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        pyro::set_last_error("pyro_fdk_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
        return PYRO_ECUDA;
    }
    // make the device's context current (a no-op when it already is), so
    // that the key names the context the kernels will run in
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) {
        pyro::set_last_error("pyro_fdk_noalloc: cudaSetDevice: %s", cudaGetErrorString(e));
        return PYRO_ECUDA;
    }
    const std::pair<int, CUcontext> key(dev, current_context());
    void *ptr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_scratch_addr.find(key);
        if (it != g_scratch_addr.end()) {
            ptr = it->second;
        } else {
            e = cudaGetSymbolAddress(&ptr, g_fdk_scratch);
            if (e != cudaSuccess || ptr == nullptr) {
                pyro::set_last_error("pyro_fdk_noalloc: cudaGetSymbolAddress of the static scratch failed: %s",
                                     cudaGetErrorString(e));
                return PYRO_ECUDA;
            }
            g_scratch_addr[key] = ptr;
        }
    }
    return pyro_fdk(sino, vol, batch, g, kind, custom_K, redund, ptr, (size_t)PYRO_FDK_NOALLOC_SCRATCH_BYTES, dtype,
                    stream);
}
