// Total variation and the vector steps of the TV-regularised iterative
// reconstruction (Eq. 7: min |A x - p|^2 + lambda TV(x), x initialised with 0).
//
// TV(x) = sum over the three axes and every voxel with a forward neighbour of
// phi(x_{i+e} - x_i), phi(d) = sqrt(d^2 + eps^2) - eps (the smoothed form of
// the anisotropic TV).  Its gradient at voxel i collects phi'(x_i - x_{i-e})
// from the backward neighbour and -phi'(x_{i+e} - x_i) from the forward one.
// One thread per voxel; reductions are FP32 per block, then FP32 atomics.
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace pyro {

namespace {

__device__ __forceinline__ float phi(float d, float eps)
{
    return sqrtf(fmaf(d, d, eps * eps)) - eps;
}

__device__ __forceinline__ float dphi(float d, float eps)
{
    return d / sqrtf(fmaf(d, d, eps * eps));
}

__device__ __forceinline__ float block_sum(float v)
{
    __shared__ float warp_sums[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_sums[w] = v;
    __syncthreads();
    float r = 0.0f;
    if (w == 0) {
        r = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    return r;  // valid in thread 0
}

constexpr int kTVThreads = 256;

__global__ void __launch_bounds__(kTVThreads) tv_kernel(const float *__restrict__ x, float *__restrict__ grad,
                                                        const float *__restrict__ base, float alpha, float lambda,
                                                        float *__restrict__ value, int nz, int ny, int nx, float eps)
{
    const long nvox = (long)nx * ny * nz;
    const int b = blockIdx.y;
    const float *xb = x + b * nvox;
    float tv_part = 0.0f;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nvox; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e % nx);
        const long r = e / nx;
        const int j = (int)(r % ny);
        const int k = (int)(r / ny);
        const float c = xb[e];
        float gsum = 0.0f;
        if (i + 1 < nx) {
            const float d = xb[e + 1] - c;
            tv_part += phi(d, eps);
            gsum -= dphi(d, eps);
        }
        if (i > 0) gsum += dphi(c - xb[e - 1], eps);
        if (j + 1 < ny) {
            const float d = xb[e + nx] - c;
            tv_part += phi(d, eps);
            gsum -= dphi(d, eps);
        }
        if (j > 0) gsum += dphi(c - xb[e - nx], eps);
        if (k + 1 < nz) {
            const float d = xb[e + (long)nx * ny] - c;
            tv_part += phi(d, eps);
            gsum -= dphi(d, eps);
        }
        if (k > 0) gsum += dphi(c - xb[e - (long)nx * ny], eps);
        if (grad) {
            const float bse = base ? alpha * base[b * nvox + e] : 0.0f;
            grad[b * nvox + e] = fmaf(lambda, gsum, bse);
        }
    }
    if (value) {
        const float s = block_sum(tv_part);
        if (threadIdx.x == 0) atomicAdd(value + b, s);
    }
}

__global__ void axpby_kernel(const float *__restrict__ x, float *__restrict__ y, long n, float a, float b)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        y[e] = fmaf(a, x[e], b * y[e]);
}

__global__ void __launch_bounds__(kTVThreads) dot_kernel(const float *__restrict__ a, const float *__restrict__ b,
                                                         long n, float *__restrict__ out)
{
    float s = 0.0f;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        s = fmaf(a[e], b[e], s);
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

// |x - x_prev|^2 and (x - x_prev).(g - g_prev) in one pass: the two scalars
// of a Barzilai-Borwein step, without forming the differences
__global__ void __launch_bounds__(kTVThreads) bb_dots_kernel(const float *__restrict__ x,
                                                             const float *__restrict__ xp,
                                                             const float *__restrict__ g,
                                                             const float *__restrict__ gp, long n,
                                                             float *__restrict__ dots)
{
    float ss = 0.0f, sy = 0.0f;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const float s = x[e] - xp[e];
        ss = fmaf(s, s, ss);
        sy = fmaf(s, g[e] - gp[e], sy);
    }
    ss = block_sum(ss);
    __syncthreads();  // block_sum's shared array is reused
    sy = block_sum(sy);
    if (threadIdx.x == 0) {
        atomicAdd(dots, ss);
        atomicAdd(dots + 1, sy);
    }
}

// alpha = first ? alpha0 : clamp(ss / sy, 0, alpha_max) (alpha0 when sy <= 0);
// x_prev = x, g_prev = g, x -= alpha g
__global__ void bb_update_kernel(float *__restrict__ x, float *__restrict__ xp, const float *__restrict__ g,
                                 float *__restrict__ gp, long n, const float *__restrict__ dots, float alpha0,
                                 float alpha_max, int first, float *__restrict__ alpha_out)
{
    float alpha = alpha0;
    if (!first) {
        const float ss = dots[0], sy = dots[1];
        alpha = sy > 0.0f ? fminf(fmaxf(ss / sy, 0.0f), alpha_max) : alpha0;
    }
    if (alpha_out && blockIdx.x == 0 && threadIdx.x == 0) *alpha_out = alpha;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const float xe = x[e], ge = g[e];
        xp[e] = xe;
        gp[e] = ge;
        x[e] = fmaf(-alpha, ge, xe);
    }
}

// Gather-bandwidth probe: every thread reads `loads` 16-byte chunks at
// pseudo-random positions of a buffer of n16 chunks (a linear congruential
// walk scaled to the buffer by a high multiply: three integer instructions
// per load) and folds them into one word, written once so that no load is
// dead.
__global__ void __launch_bounds__(256) gather_probe_kernel(const uint4 *__restrict__ buf, unsigned n16, int loads,
                                                           unsigned *__restrict__ sink)
{
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned h = tid * 2654435761u + 12345u;
    unsigned acc = 0u;
#pragma unroll 8
    for (int i = 0; i < loads; ++i) {
        h = h * 1664525u + 1013904223u;
        const uint4 v = __ldg(buf + __umulhi(h, n16));  // h / 2^32 scaled to [0, n16): one instruction
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x9e3779b9u) sink[tid & 1023] = acc;  // practically never: keeps the loads alive
}

}  // namespace

cudaError_t launch_gather_probe(const void *buf, unsigned n16, int loads, unsigned *sink, long threads,
                                cudaStream_t s)
{
    gather_probe_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>((const uint4 *)buf, n16, loads, sink);
    return cudaGetLastError();
}

cudaError_t launch_bb_dots(const float *x, const float *xp, const float *g, const float *gp, long n, float *dots,
                           cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(dots, 0, 2 * sizeof(float), s);
    if (e != cudaSuccess) return e;
    const long blocks = std::min<long>((n + kTVThreads - 1) / kTVThreads, (long)device_sm_count() * 8);
    bb_dots_kernel<<<(unsigned)std::max<long>(blocks, 1), kTVThreads, 0, s>>>(x, xp, g, gp, n, dots);
    return cudaGetLastError();
}

cudaError_t launch_bb_update(float *x, float *xp, const float *g, float *gp, long n, const float *dots, float alpha0,
                             float alpha_max, int first, float *alpha_out, cudaStream_t s)
{
    const long blocks = std::min<long>((n + 255) / 256, (long)device_sm_count() * 16);
    bb_update_kernel<<<(unsigned)std::max<long>(blocks, 1), 256, 0, s>>>(x, xp, g, gp, n, dots, alpha0, alpha_max,
                                                                         first, alpha_out);
    return cudaGetLastError();
}

cudaError_t launch_tv(const float *x, float *grad, const float *base, float alpha, float lambda, float *value,
                      int batch, int nz, int ny, int nx, float eps, cudaStream_t s)
{
    if (value) {
        cudaError_t e = cudaMemsetAsync(value, 0, sizeof(float) * batch, s);
        if (e != cudaSuccess) return e;
    }
    const long nvox = (long)nx * ny * nz;
    const long blocks = std::min<long>((nvox + kTVThreads - 1) / kTVThreads, (long)device_sm_count() * 8);
    tv_kernel<<<dim3((unsigned)blocks, batch), kTVThreads, 0, s>>>(x, grad, base, alpha, lambda, value, nz, ny, nx,
                                                                   eps);
    return cudaGetLastError();
}

cudaError_t launch_axpby(const float *x, float *y, long n, float a, float b, cudaStream_t s)
{
    const long blocks = std::min<long>((n + 255) / 256, (long)device_sm_count() * 16);
    axpby_kernel<<<(unsigned)std::max<long>(blocks, 1), 256, 0, s>>>(x, y, n, a, b);
    return cudaGetLastError();
}

cudaError_t launch_dot(const float *a, const float *b, long n, float *out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    const long blocks = std::min<long>((n + kTVThreads - 1) / kTVThreads, (long)device_sm_count() * 8);
    dot_kernel<<<(unsigned)std::max<long>(blocks, 1), kTVThreads, 0, s>>>(a, b, n, out);
    return cudaGetLastError();
}

}  // namespace pyro
