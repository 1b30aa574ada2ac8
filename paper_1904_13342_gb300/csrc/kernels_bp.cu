// Voxel-driven back-projection and its transpose
// (paper, Section "The Operator as a Layer": one thread per pixel / voxel
// projects its centre onto every view and accumulates the interpolated
// detector value; the cone-beam form follows Scherl et al. with projection
// matrices).
//
// Per view the host supplies a voxel-index -> detector map divided by SID
// (so w = L / SID and the FDK weight (SID/L)^2 is just 1/w^2) whose first
// rows are centred on the detector.  Each cone-beam thread owns one (x, y)
// column and ZB consecutive z; for circular trajectories the u coordinate
// and the weight do not depend on z and are computed once per view.
#include "device_common.cuh"
#include "internal.h"

namespace pyro {

namespace {

__device__ __forceinline__ float weight_of(float rw, int wexp)
{
    return wexp == 0 ? 1.0f : (wexp == 1 ? rw : rw * rw);
}

template <typename TS, typename TV, bool PAR>
__global__ void __launch_bounds__(256) bp2d_kernel(const TS *__restrict__ sino, TV *__restrict__ vol,
                                                   const __grid_constant__ BP2DParams p, int accumulate)
{
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int b = blockIdx.z;
    if (i >= p.nx || j >= p.ny) return;
    const float fi = (float)i, fj = (float)j;
    const TS *S = sino + ((size_t)b * p.views_total + p.view0) * p.nu;
    float acc = 0.0f;
    for (int v = 0; v < p.n_views; ++v) {
        const float *m = p.m[v];
        const float x = fmaf(m[0], fi, fmaf(m[1], fj, m[2]));
        float k, om;
        if (PAR) {
            k = x + p.cu;
            om = 1.0f;
        } else {
            const float w = fmaf(m[3], fi, fmaf(m[4], fj, m[5]));
            const float rw = 1.0f / w;
            k = fmaf(x, rw, p.cu);
            om = weight_of(rw, p.wexp);
        }
        acc = fmaf(om, lerp_zero(S + (size_t)v * p.nu, p.nu, k), acc);
    }
    const size_t o = ((size_t)b * p.ny + j) * p.nx + i;
    float out = p.scale * acc;
    if (accumulate) out += to_float<TV>(vol[o]);
    vol[o] = to_storage<TV>(out);
}

__global__ void __launch_bounds__(256) bp2d_transpose_kernel(const float *__restrict__ vol, float *__restrict__ sino,
                                                             const __grid_constant__ BP2DParams p)
{
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int b = blockIdx.z;
    if (i >= p.nx || j >= p.ny) return;
    const float g = p.scale * vol[((size_t)b * p.ny + j) * p.nx + i];
    if (g == 0.0f) return;
    const float fi = (float)i, fj = (float)j;
    float *S = sino + ((size_t)b * p.views_total + p.view0) * p.nu;
    for (int v = 0; v < p.n_views; ++v) {
        const float *m = p.m[v];
        const float x = fmaf(m[0], fi, fmaf(m[1], fj, m[2]));
        float k, om;
        if (p.parallel) {
            k = x + p.cu;
            om = 1.0f;
        } else {
            const float w = fmaf(m[3], fi, fmaf(m[4], fj, m[5]));
            const float rw = 1.0f / w;
            k = fmaf(x, rw, p.cu);
            om = weight_of(rw, p.wexp);
        }
        const Axis a = axis_taps(k, p.nu);
        float *row = S + (size_t)v * p.nu;
        const float gw = g * om;
        if (a.w0 != 0.0f) atomicAdd(row + a.i0, gw * a.w0);
        if (a.w1 != 0.0f) atomicAdd(row + a.i1, gw * a.w1);
    }
}

constexpr int kBPX = 32, kBPY = 8, kBPZ = 8;

// The 32 x 8 voxel tile of a block is cut into 8 x 4 tiles per warp (not 32 x 1
// rows): a warp's voxels then project onto ~16 detector columns instead of
// ~40, one cache line per detector row.
template <typename TS, typename TV, bool ZINV>
__global__ void __launch_bounds__(kBPX *kBPY) bp3d_kernel(const TS *__restrict__ sino, TV *__restrict__ vol,
                                                          const __grid_constant__ BP3DParams p)
{
    const int t = threadIdx.y * kBPX + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int i = blockIdx.x * kBPX + (warp & 3) * 8 + (lane & 7);
    const int j = blockIdx.y * kBPY + (warp >> 2) * 4 + (lane >> 3);
    const int zblocks = (p.nz + kBPZ - 1) / kBPZ;
    const int b = blockIdx.z / zblocks;
    const int z0 = (blockIdx.z % zblocks) * kBPZ;
    if (i >= p.nx || j >= p.ny) return;
    const float fi = (float)i, fj = (float)j;
    const size_t vstride = (size_t)p.nu * p.nv;
    const TS *S0 = sino + ((size_t)b * p.views_total + p.view0) * vstride;
    float acc[kBPZ];
#pragma unroll
    for (int zz = 0; zz < kBPZ; ++zz) acc[zz] = 0.0f;

    for (int v = 0; v < p.n_views; ++v) {
        const float *P = p.P[v];
        const TS *S = S0 + (size_t)v * vstride;
        const float xb = fmaf(P[0], fi, fmaf(P[1], fj, P[3]));
        const float yb = fmaf(P[4], fi, fmaf(P[5], fj, P[7]));
        const float wb = fmaf(P[8], fi, fmaf(P[9], fj, P[11]));
        if (ZINV) {
            const float rw = 1.0f / wb;
            const float om = weight_of(rw, p.wexp);
            const float fu = fmaf(xb, rw, p.cu);
            const float dl = P[6] * rw;
            const float l0 = fmaf(yb, rw, p.cv);
            const float la = fmaf((float)z0, dl, l0), lb = fmaf((float)(z0 + kBPZ - 1), dl, l0);
            const float hu = (float)(p.nu - 1) - 1e-3f, hv = (float)(p.nv - 1) - 1e-3f;
            if (fu >= 1e-3f && fu <= hu && fminf(la, lb) >= 1e-3f && fmaxf(la, lb) <= hv) {
                // every tap of the ZB voxels lies inside the detector: no masking
                const float fu0 = floorf(fu);
                const float au = fu - fu0;
                const float w1 = om * au, w0 = om - w1;
                const TS *Sk = S + (int)fu0;
#pragma unroll
                for (int zz = 0; zz < kBPZ; ++zz) {
                    const float ll = fmaf((float)(z0 + zz), dl, l0);
                    const float tl = floor_magic(ll);
                    const float av = ll - magic_to_float(tl);
                    const TS *r0 = Sk + magic_to_int(tl) * p.nu;
                    const float t0 = fmaf(w0, ld(r0), w1 * ld(r0 + 1));
                    const float t1 = fmaf(w0, ld(r0 + p.nu), w1 * ld(r0 + p.nu + 1));
                    acc[zz] += lerpf(t0, t1, av);
                }
                continue;
            }
            const Axis au = axis_taps(fu, p.nu);
            const float w0 = om * au.w0, w1 = om * au.w1;
#pragma unroll
            for (int zz = 0; zz < kBPZ; ++zz) {
                const Axis av = axis_taps(fmaf((float)(z0 + zz), dl, l0), p.nv);
                const TS *r0 = S + (size_t)av.i0 * p.nu;
                const TS *r1 = S + (size_t)av.i1 * p.nu;
                const float t0 = fmaf(w0, ld(r0 + au.i0), w1 * ld(r0 + au.i1));
                const float t1 = fmaf(w0, ld(r1 + au.i0), w1 * ld(r1 + au.i1));
                acc[zz] = fmaf(av.w0, t0, fmaf(av.w1, t1, acc[zz]));
            }
        } else {
#pragma unroll
            for (int zz = 0; zz < kBPZ; ++zz) {
                const float fz = (float)(z0 + zz);
                const float x = fmaf(P[2], fz, xb);
                const float y = fmaf(P[6], fz, yb);
                const float w = fmaf(P[10], fz, wb);
                const float rw = 1.0f / w;
                const float om = weight_of(rw, p.wexp);
                acc[zz] = fmaf(om, bilerp_zero(S, p.nu, p.nv, fmaf(x, rw, p.cu), fmaf(y, rw, p.cv)), acc[zz]);
            }
        }
    }
    const size_t sxy = (size_t)p.nx * p.ny;
    TV *out = vol + (size_t)b * sxy * p.nz + (size_t)j * p.nx + i;
#pragma unroll
    for (int zz = 0; zz < kBPZ; ++zz) {
        const int z = z0 + zz;
        if (z < p.nz) {
            float r = p.scale * acc[zz];
            if (p.accumulate) r += to_float<TV>(out[z * sxy]);
            out[z * sxy] = to_storage<TV>(r);
        }
    }
}

// ---- texture-mode cone BP (the paper's fast BP mode) ----------------------
// The sinogram sits in a layered 2D CUDA array (one layer per view), read with
// hardware bilinear filtering and a zero border: one fetch per voxel and view
// replaces four taps and three lerps, with fixed-point interpolation weights
// (8 fractional bits).  Same voxel-to-detector map, weights and tiling as
// bp3d_kernel; texel k's centre is at coordinate k + 0.5.
template <typename TV>
__global__ void __launch_bounds__(kBPX *kBPY) bp3d_tex_kernel(cudaTextureObject_t tex, TV *__restrict__ vol,
                                                              const __grid_constant__ BP3DParams p)
{
    const int t = threadIdx.y * kBPX + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int i = blockIdx.x * kBPX + (warp & 3) * 8 + (lane & 7);
    const int j = blockIdx.y * kBPY + (warp >> 2) * 4 + (lane >> 3);
    const int z0 = blockIdx.z * kBPZ;
    if (i >= p.nx || j >= p.ny) return;
    const float fi = (float)i, fj = (float)j;
    const float cu = p.cu + 0.5f, cv = p.cv + 0.5f;
    float acc[kBPZ];
#pragma unroll
    for (int zz = 0; zz < kBPZ; ++zz) acc[zz] = 0.0f;
    for (int v = 0; v < p.n_views; ++v) {
        const float *P = p.P[v];
        const int layer = p.view0 + v;
        const float xb = fmaf(P[0], fi, fmaf(P[1], fj, P[3]));
        const float yb = fmaf(P[4], fi, fmaf(P[5], fj, P[7]));
        const float wb = fmaf(P[8], fi, fmaf(P[9], fj, P[11]));
        if (p.z_invariant) {
            const float rw = 1.0f / wb;
            const float om = weight_of(rw, p.wexp);
            const float fu = fmaf(xb, rw, cu);
            const float dl = P[6] * rw;
            const float l0 = fmaf(yb, rw, cv);
#pragma unroll
            for (int zz = 0; zz < kBPZ; ++zz)
                acc[zz] = fmaf(om, tex2DLayered<float>(tex, fu, fmaf((float)(z0 + zz), dl, l0), layer), acc[zz]);
        } else {
#pragma unroll
            for (int zz = 0; zz < kBPZ; ++zz) {
                const float fz = (float)(z0 + zz);
                const float rw = 1.0f / fmaf(P[10], fz, wb);
                const float om = weight_of(rw, p.wexp);
                const float val = tex2DLayered<float>(tex, fmaf(fmaf(P[2], fz, xb), rw, cu),
                                                      fmaf(fmaf(P[6], fz, yb), rw, cv), layer);
                acc[zz] = fmaf(om, val, acc[zz]);
            }
        }
    }
    const size_t sxy = (size_t)p.nx * p.ny;
    TV *out = vol + (size_t)j * p.nx + i;
#pragma unroll
    for (int zz = 0; zz < kBPZ; ++zz) {
        const int z = z0 + zz;
        if (z < p.nz) {
            float r = p.scale * acc[zz];
            if (p.accumulate) r += to_float<TV>(out[z * sxy]);
            out[z * sxy] = to_storage<TV>(r);
        }
    }
}

// ---- TMA-staged cone BP (circular-type trajectories, FP32 sinogram) ------
// Per view a block's 32 x 8 x ZB voxel tile projects onto a small detector
// box; one thread copies the boxes of the next views into a ring of shared
// memory stages with cp.async.bulk.tensor (completion counted on an
// mbarrier), and every thread reads its four taps per voxel from shared
// memory.  Out-of-range parts of a box are zero-filled by the copy, which is
// the zero extension of the detector, so no tap needs masking.  Box sizes are
// a host-computed bound; shared-memory indices are clamped to the stage.
constexpr int kTmaStages = 3;

__device__ int g_status;  // set to 1 by a wait that gave up (read by pyro_sync_status)

// Self-test of the wait-and-report path: one warp waits on an mbarrier that
// nothing arrives at, gives up after limit_ns and sets the status word.
__global__ void wait_timeout_probe_kernel(unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (!mbar_wait(&bar, 0, limit_ns) && threadIdx.x == 0) atomicExch(&g_status, 1);
}

__device__ __forceinline__ void tma_load_3d(float *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

template <typename TV>
__global__ void __launch_bounds__(kBPX *kBPY) bp3d_tma_kernel(const __grid_constant__ CUtensorMap map,
                                                              TV *__restrict__ vol,
                                                              const __grid_constant__ BP3DParams p, int bu, int bv,
                                                              int stage_floats)
{
    extern __shared__ __align__(128) float stages[];
    __shared__ __align__(8) uint64_t full[kTmaStages];
    __shared__ int2 origin[kTmaStages];
    __shared__ int gave_up;
    const int t = threadIdx.y * kBPX + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int i0 = blockIdx.x * kBPX, j0 = blockIdx.y * kBPY;
    const int i = i0 + (warp & 3) * 8 + (lane & 7);
    const int j = j0 + (warp >> 2) * 4 + (lane >> 3);
    const int zblocks = (p.nz + kBPZ - 1) / kBPZ;
    const int b = blockIdx.z / zblocks;
    const int z0 = (blockIdx.z % zblocks) * kBPZ;
    const int i1 = min(i0 + kBPX - 1, p.nx - 1), j1 = min(j0 + kBPY - 1, p.ny - 1), z1 = min(z0 + kBPZ - 1, p.nz - 1);
    const int vbase = b * p.views_total + p.view0;
    const bool active = i < p.nx && j < p.ny;  // the others still take part in the barriers
    const unsigned stage_bytes = (unsigned)(bu * bv * sizeof(float));
    if (t == 0) {
        for (int s = 0; s < kTmaStages; ++s) mbar_init(&full[s], 1);
        gave_up = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // thread 0: the box of view v from the tile's eight corners (the
    // projection is linear-fractional with a positive depth, so the corners
    // bound it), then the copy into stage v % kTmaStages
    auto issue = [&](int v) {
        const int s = v % kTmaStages;
        const float *P = p.P[v];
        float umin = 3.0e38f, umax = -3.0e38f, lmin = 3.0e38f;
        for (int c = 0; c < 4; ++c) {
            const float fi = (float)((c & 1) ? i1 : i0), fj = (float)((c & 2) ? j1 : j0);
            const float xb = fmaf(P[0], fi, fmaf(P[1], fj, P[3]));
            const float yb = fmaf(P[4], fi, fmaf(P[5], fj, P[7]));
            const float wb = fmaf(P[8], fi, fmaf(P[9], fj, P[11]));
            const float rw = 1.0f / wb;
            const float fu = fmaf(xb, rw, p.cu);
            const float dl = P[6] * rw;
            const float l0 = fmaf(yb, rw, p.cv);
            umin = fminf(umin, fu);
            umax = fmaxf(umax, fu);
            lmin = fminf(lmin, fminf(fmaf((float)z0, dl, l0), fmaf((float)z1, dl, l0)));
        }
        // x of a tensor copy must be a multiple of 4 floats (16 bytes)
        const int ux = ((int)floorf(fmaxf(umin, -1.0e8f) - 0.01f)) & ~3;
        const int ly = (int)floorf(fmaxf(lmin, -1.0e8f) - 0.01f);
        origin[s] = make_int2(ux, ly);
        mbar_expect_tx(&full[s], stage_bytes);
        tma_load_3d(stages + s * stage_floats, &map, ux, ly, vbase + v, &full[s]);
    };
    if (t == 0)
        for (int v = 0; v < min(kTmaStages, p.n_views); ++v) issue(v);

    float acc[kBPZ];
#pragma unroll
    for (int zz = 0; zz < kBPZ; ++zz) acc[zz] = 0.0f;
    const float fi = (float)i, fj = (float)j;
    const int last = stage_floats - bu - 2;  // highest first tap index of a 2 x 2 patch
    int v = 0;
    for (; v < p.n_views; ++v) {
        const int s = v % kTmaStages;
        if (!mbar_wait(&full[s], (unsigned)(v / kTmaStages) & 1u)) atomicExch(&gave_up, 1);
        if (active) {
            const float *S = stages + s * stage_floats;
            const int2 o = origin[s];
            const float *P = p.P[v];
            const float xb = fmaf(P[0], fi, fmaf(P[1], fj, P[3]));
            const float yb = fmaf(P[4], fi, fmaf(P[5], fj, P[7]));
            const float wb = fmaf(P[8], fi, fmaf(P[9], fj, P[11]));
            const float rw = 1.0f / wb;
            const float om = weight_of(rw, p.wexp);
            const float fu = fmaf(xb, rw, p.cu);
            const float dl = P[6] * rw;
            const float l0 = fmaf(yb, rw, p.cv);
            const float tu = floor_magic(fu);
            const float au = fu - magic_to_float(tu);
            const float w1 = om * au, w0 = om - w1;
            const int col = magic_to_int(tu) - o.x;
#pragma unroll
            for (int zz = 0; zz < kBPZ; ++zz) {
                const float ll = fmaf((float)(z0 + zz), dl, l0);
                const float tl = floor_magic(ll);
                const float av = ll - magic_to_float(tl);
                const int e = min(max((magic_to_int(tl) - o.y) * bu + col, 0), last);
                const float t0 = fmaf(w0, S[e], w1 * S[e + 1]);
                const float t1 = fmaf(w0, S[e + bu], w1 * S[e + bu + 1]);
                acc[zz] += lerpf(t0, t1, av);
            }
        }
        __syncthreads();  // stage s is free again; gave_up is visible
        if (gave_up) break;
        if (t == 0 && v + kTmaStages < p.n_views) issue(v + kTmaStages);
    }
    if (gave_up) {
        // let the copies still in flight land (bounded) before the block ends
        if (t == 0) {
            atomicExch(&g_status, 1);
            for (int w = v; w < min(v + kTmaStages, p.n_views); ++w)
                mbar_wait(&full[w % kTmaStages], (unsigned)(w / kTmaStages) & 1u);
        }
        return;
    }
    if (!active) return;
    const size_t sxy = (size_t)p.nx * p.ny;
    TV *out = vol + (size_t)b * sxy * p.nz + (size_t)j * p.nx + i;
#pragma unroll
    for (int zz = 0; zz < kBPZ; ++zz) {
        const int z = z0 + zz;
        if (z < p.nz) {
            float r = p.scale * acc[zz];
            if (p.accumulate) r += to_float<TV>(out[z * sxy]);
            out[z * sxy] = to_storage<TV>(r);
        }
    }
}

__global__ void __launch_bounds__(kBPX *kBPY) bp3d_transpose_kernel(const float *__restrict__ vol,
                                                                    float *__restrict__ sino,
                                                                    const __grid_constant__ BP3DParams p)
{
    const int i = blockIdx.x * kBPX + threadIdx.x;
    const int j = blockIdx.y * kBPY + threadIdx.y;
    const int b = blockIdx.z / p.nz;
    const int z = blockIdx.z % p.nz;
    if (i >= p.nx || j >= p.ny) return;
    const float g = p.scale * vol[(((size_t)b * p.nz + z) * p.ny + j) * p.nx + i];
    if (g == 0.0f) return;
    const float fi = (float)i, fj = (float)j, fz = (float)z;
    const size_t vstride = (size_t)p.nu * p.nv;
    float *S0 = sino + ((size_t)b * p.views_total + p.view0) * vstride;
    for (int v = 0; v < p.n_views; ++v) {
        const float *P = p.P[v];
        const float x = fmaf(P[0], fi, fmaf(P[1], fj, fmaf(P[2], fz, P[3])));
        const float y = fmaf(P[4], fi, fmaf(P[5], fj, fmaf(P[6], fz, P[7])));
        const float w = fmaf(P[8], fi, fmaf(P[9], fj, fmaf(P[10], fz, P[11])));
        const float rw = 1.0f / w;
        const float gw = g * weight_of(rw, p.wexp);
        const Axis au = axis_taps(fmaf(x, rw, p.cu), p.nu);
        const Axis av = axis_taps(fmaf(y, rw, p.cv), p.nv);
        float *S = S0 + (size_t)v * vstride;
        float *r0 = S + (size_t)av.i0 * p.nu;
        float *r1 = S + (size_t)av.i1 * p.nu;
        const float g0 = gw * av.w0, g1 = gw * av.w1;
        if (g0 * au.w0 != 0.0f) atomicAdd(r0 + au.i0, g0 * au.w0);
        if (g0 * au.w1 != 0.0f) atomicAdd(r0 + au.i1, g0 * au.w1);
        if (g1 * au.w0 != 0.0f) atomicAdd(r1 + au.i0, g1 * au.w0);
        if (g1 * au.w1 != 0.0f) atomicAdd(r1 + au.i1, g1 * au.w1);
    }
}

template <typename TS, typename TV>
cudaError_t bp2d_dispatch(const void *sino, void *vol, int batch, const BP2DParams &p, int accumulate, cudaStream_t s)
{
    dim3 block(32, 8);
    dim3 grid((p.nx + 31) / 32, (p.ny + 7) / 8, batch);
    if (p.parallel)
        bp2d_kernel<TS, TV, true><<<grid, block, 0, s>>>((const TS *)sino, (TV *)vol, p, accumulate);
    else
        bp2d_kernel<TS, TV, false><<<grid, block, 0, s>>>((const TS *)sino, (TV *)vol, p, accumulate);
    return cudaGetLastError();
}

template <typename TS, typename TV>
cudaError_t bp3d_dispatch(const void *sino, void *vol, int batch, const BP3DParams &p, cudaStream_t s)
{
    dim3 block(kBPX, kBPY);
    const int zblocks = (p.nz + kBPZ - 1) / kBPZ;
    dim3 grid((p.nx + kBPX - 1) / kBPX, (p.ny + kBPY - 1) / kBPY, (unsigned)(zblocks * batch));
    if (p.z_invariant)
        bp3d_kernel<TS, TV, true><<<grid, block, 0, s>>>((const TS *)sino, (TV *)vol, p);
    else
        bp3d_kernel<TS, TV, false><<<grid, block, 0, s>>>((const TS *)sino, (TV *)vol, p);
    return cudaGetLastError();
}

template <typename TS>
cudaError_t bp2d_by_vol(const void *sino, void *vol, int batch, const BP2DParams &p, pyro_dtype vol_dt, int acc,
                        cudaStream_t s)
{
    switch (vol_dt) {
    case PYRO_F32: return bp2d_dispatch<TS, float>(sino, vol, batch, p, acc, s);
    case PYRO_F16: return bp2d_dispatch<TS, __half>(sino, vol, batch, p, acc, s);
    case PYRO_BF16: return bp2d_dispatch<TS, __nv_bfloat16>(sino, vol, batch, p, acc, s);
    }
    return cudaErrorInvalidValue;
}

template <typename TS>
cudaError_t bp3d_by_vol(const void *sino, void *vol, int batch, const BP3DParams &p, pyro_dtype vol_dt,
                        cudaStream_t s)
{
    switch (vol_dt) {
    case PYRO_F32: return bp3d_dispatch<TS, float>(sino, vol, batch, p, s);
    case PYRO_F16: return bp3d_dispatch<TS, __half>(sino, vol, batch, p, s);
    case PYRO_BF16: return bp3d_dispatch<TS, __nv_bfloat16>(sino, vol, batch, p, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_bp2d(const void *sino, void *vol, int batch, const BP2DParams &p, pyro_dtype sino_dt,
                        pyro_dtype vol_dt, int accumulate, cudaStream_t s)
{
    switch (sino_dt) {
    case PYRO_F32: return bp2d_by_vol<float>(sino, vol, batch, p, vol_dt, accumulate, s);
    case PYRO_F16: return bp2d_by_vol<__half>(sino, vol, batch, p, vol_dt, accumulate, s);
    case PYRO_BF16: return bp2d_by_vol<__nv_bfloat16>(sino, vol, batch, p, vol_dt, accumulate, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_bp2d_transpose(const void *vol, void *sino, int batch, const BP2DParams &p, cudaStream_t s)
{
    dim3 block(32, 8);
    dim3 grid((p.nx + 31) / 32, (p.ny + 7) / 8, batch);
    bp2d_transpose_kernel<<<grid, block, 0, s>>>((const float *)vol, (float *)sino, p);
    return cudaGetLastError();
}

cudaError_t launch_bp3d(const void *sino, void *vol, int batch, const BP3DParams &p, pyro_dtype sino_dt,
                        pyro_dtype vol_dt, cudaStream_t s)
{
    switch (sino_dt) {
    case PYRO_F32: return bp3d_by_vol<float>(sino, vol, batch, p, vol_dt, s);
    case PYRO_F16: return bp3d_by_vol<__half>(sino, vol, batch, p, vol_dt, s);
    case PYRO_BF16: return bp3d_by_vol<__nv_bfloat16>(sino, vol, batch, p, vol_dt, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_bp3d_tex(cudaTextureObject_t tex, void *vol, const BP3DParams &p, pyro_dtype vol_dt, cudaStream_t s)
{
    dim3 block(kBPX, kBPY);
    dim3 grid((p.nx + kBPX - 1) / kBPX, (p.ny + kBPY - 1) / kBPY, (unsigned)((p.nz + kBPZ - 1) / kBPZ));
    switch (vol_dt) {
    case PYRO_F32:
        bp3d_tex_kernel<float><<<grid, block, 0, s>>>(tex, (float *)vol, p);
        break;
    case PYRO_F16:
        bp3d_tex_kernel<__half><<<grid, block, 0, s>>>(tex, (__half *)vol, p);
        break;
    case PYRO_BF16:
        bp3d_tex_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(tex, (__nv_bfloat16 *)vol, p);
        break;
    }
    return cudaGetLastError();
}

int tma_stage_floats(int bu, int bv)
{
    return (bu * bv + 31) / 32 * 32;  // stages start on 128-byte boundaries
}

cudaError_t launch_bp3d_tma(const CUtensorMap &map, void *vol, int batch, const BP3DParams &p, int bu, int bv,
                            pyro_dtype vol_dt, cudaStream_t s)
{
    const int sf = tma_stage_floats(bu, bv);
    const size_t smem = (size_t)kTmaStages * sf * sizeof(float);
    dim3 block(kBPX, kBPY);
    const int zblocks = (p.nz + kBPZ - 1) / kBPZ;
    dim3 grid((p.nx + kBPX - 1) / kBPX, (p.ny + kBPY - 1) / kBPY, (unsigned)(zblocks * batch));
    switch (vol_dt) {
    case PYRO_F32:
        bp3d_tma_kernel<float><<<grid, block, smem, s>>>(map, (float *)vol, p, bu, bv, sf);
        break;
    case PYRO_F16:
        bp3d_tma_kernel<__half><<<grid, block, smem, s>>>(map, (__half *)vol, p, bu, bv, sf);
        break;
    case PYRO_BF16:
        bp3d_tma_kernel<__nv_bfloat16><<<grid, block, smem, s>>>(map, (__nv_bfloat16 *)vol, p, bu, bv, sf);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_wait_timeout_probe(unsigned long long limit_ns, cudaStream_t s)
{
    wait_timeout_probe_kernel<<<1, 32, 0, s>>>(limit_ns);
    return cudaGetLastError();
}

cudaError_t status_word(int **ptr)
{
    return cudaGetSymbolAddress((void **)ptr, g_status);
}

cudaError_t launch_bp3d_transpose(const void *vol, void *sino, int batch, const BP3DParams &p, cudaStream_t s)
{
    dim3 block(kBPX, kBPY);
    dim3 grid((p.nx + kBPX - 1) / kBPX, (p.ny + kBPY - 1) / kBPY, (unsigned)(p.nz * batch));
    bp3d_transpose_kernel<<<grid, block, 0, s>>>((const float *)vol, (float *)sino, p);
    return cudaGetLastError();
}

}  // namespace pyro
