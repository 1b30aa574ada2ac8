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
//    that device current) and caches it; make that first call before any
//    stream capture on that device.
//  * Every call on a device shares the one array and it keeps the contents
//    of the last call.  The filter stage overwrites every scratch element it
//    reads back, so nothing needs clearing; but calls whose work overlaps on
//    the GPU (different streams, or different host threads, without
//    ordering between them) race on the array and corrupt each other.
//  * It calls no cudaMalloc, cudaFree or other allocating routine.
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_fdk_scratch[PYRO_FDK_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
std::map<int, void *> g_scratch_addr;  // device ordinal -> device address of g_fdk_scratch

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
    void *ptr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_scratch_addr.find(dev);
        if (it != g_scratch_addr.end()) {
            ptr = it->second;
        } else {
            e = cudaGetSymbolAddress(&ptr, g_fdk_scratch);
            if (e != cudaSuccess || ptr == nullptr) {
                pyro::set_last_error("pyro_fdk_noalloc: cudaGetSymbolAddress of the static scratch failed: %s",
                                     cudaGetErrorString(e));
                return PYRO_ECUDA;
            }
            g_scratch_addr[dev] = ptr;
        }
    }
    return pyro_fdk(sino, vol, batch, g, kind, custom_K, redund, ptr, (size_t)PYRO_FDK_NOALLOC_SCRATCH_BYTES, dtype,
                    stream);
}
