// Ray-driven forward projection A and its exact adjoint A^T
// (paper, Section "The Operator as a Layer": one thread per detector pixel
// casts its ray and accumulates interpolated samples; the cone-beam rays
// come from projection matrices, after Galigekere et al.).
//
// Every ray is sampled at t_c + m * dt, m = -M..M, t_c the closest approach
// of the line to the iso-centre; only the m whose sample can touch the
// support (-1, N) of the zero-extended interpolant are visited (the others
// contribute exactly zero).  Arithmetic is FP32, accumulation along the ray
// is FP32; storage is FP32, FP16 or BF16.
#include "device_common.cuh"
#include "internal.h"

namespace pyro {

namespace {

// ---- 2D ray set-up: sample position p0 + m q in pixel-index units --------
struct Ray2 {
    float px, py, qx, qy;
};

__device__ __forceinline__ Ray2 ray2d(const FP2DParams &p, int v, int k)
{
    const float2 c = p.dir[v];
    const float u = ((float)k - p.cu) * p.su;
    float bx, by, dx, dy;
    if (p.fan) {
        const float L2 = fmaf(p.sdd, p.sdd, u * u);
        const float f = p.sid * u / L2;
        // e_u = (-c.y, c.x); B = f (SDD e_u - u c)
        bx = f * fmaf(-p.sdd, c.y, -u * c.x);
        by = f * fmaf(p.sdd, c.x, -u * c.y);
        const float rL = 1.0f / sqrtf(L2);
        dx = fmaf(p.sdd, c.x, -u * c.y) * rL;
        dy = fmaf(p.sdd, c.y, u * c.x) * rL;
    } else {
        bx = -u * c.y;
        by = u * c.x;
        dx = c.x;
        dy = c.y;
    }
    Ray2 r;
    r.px = fmaf(bx, p.inv_sx, p.cx);
    r.py = fmaf(by, p.inv_sy, p.cy);
    r.qx = dx * p.dt * p.inv_sx;
    r.qy = dy * p.dt * p.inv_sy;
    return r;
}

__device__ __forceinline__ void range2d(const Ray2 &r, const FP2DParams &p, int &m0, int &m1)
{
    float lo = -(float)p.M, hi = (float)p.M;
    clip_axis(r.px, r.qx, p.nx, lo, hi);
    clip_axis(r.py, r.qy, p.ny, lo, hi);
    m0 = max(-p.M, (int)floorf(lo));
    m1 = min(p.M, (int)ceilf(hi));
}

template <typename T>
__global__ void __launch_bounds__(128) fp2d_kernel(const T *__restrict__ vol, T *__restrict__ sino,
                                                   const __grid_constant__ FP2DParams p)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    const int b = blockIdx.z;
    if (k >= p.nu) return;
    const Ray2 r = ray2d(p, v, k);
    int m0, m1;
    range2d(r, p, m0, m1);
    const T *img = vol + (size_t)b * p.nx * p.ny;
    float acc = 0.0f;
    for (int m = m0; m <= m1; ++m) {
        const float fm = (float)m;
        acc += bilerp_zero(img, p.nx, p.ny, fmaf(fm, r.qx, r.px), fmaf(fm, r.qy, r.py));
    }
    sino[((size_t)b * p.views_total + p.view0 + v) * p.nu + k] = to_storage<T>(p.dt * acc);
}

__global__ void __launch_bounds__(128) fp2d_adjoint_kernel(const float *__restrict__ sino, float *__restrict__ vol,
                                                           const __grid_constant__ FP2DParams p)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    const int b = blockIdx.z;
    if (k >= p.nu) return;
    const float y = p.dt * sino[((size_t)b * p.views_total + p.view0 + v) * p.nu + k];
    if (y == 0.0f) return;
    const Ray2 r = ray2d(p, v, k);
    int m0, m1;
    range2d(r, p, m0, m1);
    float *img = vol + (size_t)b * p.nx * p.ny;
    for (int m = m0; m <= m1; ++m) {
        const float fm = (float)m;
        const Axis ax = axis_taps(fmaf(fm, r.qx, r.px), p.nx);
        const Axis ay = axis_taps(fmaf(fm, r.qy, r.py), p.ny);
        float *r0 = img + (size_t)ay.i0 * p.nx;
        float *r1 = img + (size_t)ay.i1 * p.nx;
        const float y0 = y * ay.w0, y1 = y * ay.w1;
        if (y0 * ax.w0 != 0.0f) atomicAdd(r0 + ax.i0, y0 * ax.w0);
        if (y0 * ax.w1 != 0.0f) atomicAdd(r0 + ax.i1, y0 * ax.w1);
        if (y1 * ax.w0 != 0.0f) atomicAdd(r1 + ax.i0, y1 * ax.w0);
        if (y1 * ax.w1 != 0.0f) atomicAdd(r1 + ax.i1, y1 * ax.w1);
    }
}

// ---- 3D cone ray set-up --------------------------------------------------
struct Ray3 {
    float px, py, pz, qx, qy, qz;
};

__device__ __forceinline__ Ray3 ray3d(const FP3DParams &p, int v, int k, int l)
{
    const ConeFPView &V = p.v[v];
    const float fk = (float)k, fl = (float)l;
    const float qx = fmaf(V.a0, fk, fmaf(V.a1, fl, V.a2));
    const float qy = fmaf(V.b0, fl, V.b2);
    const float q2 = fmaf(qx, qx, qy * qy);
    const float n2 = q2 + 1.0f;
    const float rn2 = 1.0f / n2;
    const float sq = fmaf(V.s1, qx, V.s2 * qy);  // s_perp . q
    const float g = (sq + V.s3) * rn2;
    // closest approach in camera coordinates
    const float c0 = fmaf(-g, qx, V.s1);
    const float c1 = fmaf(-g, qy, V.s2);
    const float c2 = fmaf(V.s3, q2, -sq) * rn2;
    const float rn = 1.0f / sqrtf(n2);
    const float *W = V.W;
    Ray3 r;
    r.px = fmaf(W[0], c0, fmaf(W[1], c1, fmaf(W[2], c2, p.cx)));
    r.py = fmaf(W[3], c0, fmaf(W[4], c1, fmaf(W[5], c2, p.cy)));
    r.pz = fmaf(W[6], c0, fmaf(W[7], c1, fmaf(W[8], c2, p.cz)));
    const float s = p.dt * rn;
    r.qx = s * fmaf(W[0], qx, fmaf(W[1], qy, W[2]));
    r.qy = s * fmaf(W[3], qx, fmaf(W[4], qy, W[5]));
    r.qz = s * fmaf(W[6], qx, fmaf(W[7], qy, W[8]));
    return r;
}

__device__ __forceinline__ void range3d(const Ray3 &r, const FP3DParams &p, int &m0, int &m1)
{
    float lo = -(float)p.M, hi = (float)p.M;
    clip_axis(r.px, r.qx, p.nx, lo, hi);
    clip_axis(r.py, r.qy, p.ny, lo, hi);
    clip_axis(r.pz, r.qz, p.nz, lo, hi);
    m0 = max(-p.M, (int)floorf(lo));
    m1 = min(p.M, (int)ceilf(hi));
}

// Sum of the samples m0..m1 of one ray through a volume with element strides
// (stx, sty, stz).  Samples strictly inside the array take the unmasked
// interior path; the few near the faces take the zero-extended path.  The
// sample positions are the same FMA p + m q on both paths.
template <typename T>
__device__ __forceinline__ float march3d(const T *vol, const FP3DParams &p, int stx, int sty, int stz, const Ray3 &r,
                                         int m0, int m1)
{
    float lo = (float)m0, hi = (float)m1;
    clip_axis_interior(r.px, r.qx, p.nx, lo, hi);
    clip_axis_interior(r.py, r.qy, p.ny, lo, hi);
    clip_axis_interior(r.pz, r.qz, p.nz, lo, hi);
    int i0 = max(m0, (int)ceilf(lo)), i1 = min(m1, (int)floorf(hi));
    if (i0 > i1) {  // no interior sample
        i0 = m1 + 1;
        i1 = m1;
    }
    float acc = 0.0f;
    for (int m = m0; m < i0; ++m) {
        const float fm = (float)m;
        acc += trilerp_zero_strided(vol, p.nx, p.ny, p.nz, (size_t)stx, (size_t)sty, (size_t)stz, fmaf(fm, r.qx, r.px),
                                    fmaf(fm, r.qy, r.py), fmaf(fm, r.qz, r.pz));
    }
    for (int m = i0; m <= i1; ++m) {
        const float fm = (float)m;
        acc += trilerp_interior(vol, stx, sty, stz, fmaf(fm, r.qx, r.px), fmaf(fm, r.qy, r.py), fmaf(fm, r.qz, r.pz));
    }
    for (int m = max(i1 + 1, i0); m <= m1; ++m) {
        const float fm = (float)m;
        acc += trilerp_zero_strided(vol, p.nx, p.ny, p.nz, (size_t)stx, (size_t)sty, (size_t)stz, fmaf(fm, r.qx, r.px),
                                    fmaf(fm, r.qy, r.py), fmaf(fm, r.qz, r.pz));
    }
    return acc;
}

constexpr int kFP3DBlockX = 32, kFP3DBlockY = 4;

template <typename T>
__global__ void __launch_bounds__(kFP3DBlockX *kFP3DBlockY) fp3d_kernel(const T *__restrict__ vol,
                                                                        T *__restrict__ sino,
                                                                        const __grid_constant__ FP3DParams p)
{
    const int k = blockIdx.x * kFP3DBlockX + threadIdx.x;
    const int l = blockIdx.y * kFP3DBlockY + threadIdx.y;
    const int v = blockIdx.z % p.n_views;
    const int b = blockIdx.z / p.n_views;
    if (k >= p.nu || l >= p.nv) return;
    const Ray3 r = ray3d(p, v, k, l);
    int m0, m1;
    range3d(r, p, m0, m1);
    const T *V = vol + (size_t)b * p.nx * p.ny * p.nz;
    const float acc = march3d(V, p, 1, p.nx, p.nx * p.ny, r, m0, m1);
    sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k] = to_storage<T>(p.dt * acc);
}

// Staged forward projection: the volume has been re-laid out z-fastest
// ([y][x][z]) and each warp's 32 lanes take 32 consecutive detector rows l of
// one column k.  Those rays differ only in elevation, so at every sample
// the warp's taps lie in one or two short contiguous runs along z: one or two
// cache lines per tap load, whatever the view angle.
constexpr int kFPZLanes = 32, kFPZWarps = 4;

template <typename T>
__global__ void __launch_bounds__(kFPZLanes *kFPZWarps) fp3d_zmajor_kernel(const T *__restrict__ vz,
                                                                          T *__restrict__ sino,
                                                                          const __grid_constant__ FP3DParams p,
                                                                          int b)
{
    const int l = blockIdx.x * kFPZLanes + threadIdx.x;
    const int k = blockIdx.y * kFPZWarps + threadIdx.y;
    const int v = blockIdx.z;
    if (k >= p.nu || l >= p.nv) return;
    const Ray3 r = ray3d(p, v, k, l);
    int m0, m1;
    range3d(r, p, m0, m1);
    const float acc = march3d(vz, p, p.nz, p.nz * p.nx, 1, r, m0, m1);
    sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k] = to_storage<T>(p.dt * acc);
}

// [z][y][x] -> [y][x][z]: 32 x 32 tiles of one y-plane through shared memory
template <typename T>
__global__ void __launch_bounds__(256) relayout_zmajor_kernel(const T *__restrict__ vol, T *__restrict__ vz, int nx,
                                                              int ny, int nz)
{
    __shared__ T tile[32][33];
    const int x0 = blockIdx.x * 32, z0 = blockIdx.y * 32, y = blockIdx.z;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int z = z0 + i, x = x0 + threadIdx.x;
        if (z < nz && x < nx) tile[i][threadIdx.x] = vol[((size_t)z * ny + y) * nx + x];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int x = x0 + i, z = z0 + threadIdx.x;
        if (z < nz && x < nx) vz[((size_t)y * nx + x) * nz + z] = tile[threadIdx.x][i];
    }
}

__global__ void __launch_bounds__(kFP3DBlockX *kFP3DBlockY) fp3d_adjoint_kernel(const float *__restrict__ sino,
                                                                                float *__restrict__ vol,
                                                                                const __grid_constant__ FP3DParams p)
{
    const int k = blockIdx.x * kFP3DBlockX + threadIdx.x;
    const int l = blockIdx.y * kFP3DBlockY + threadIdx.y;
    const int v = blockIdx.z % p.n_views;
    const int b = blockIdx.z / p.n_views;
    if (k >= p.nu || l >= p.nv) return;
    const float y = p.dt * sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k];
    if (y == 0.0f) return;
    const Ray3 r = ray3d(p, v, k, l);
    int m0, m1;
    range3d(r, p, m0, m1);
    float *V = vol + (size_t)b * p.nx * p.ny * p.nz;
    const size_t sxy = (size_t)p.nx * p.ny;
    for (int m = m0; m <= m1; ++m) {
        const float fm = (float)m;
        const Axis ax = axis_taps(fmaf(fm, r.qx, r.px), p.nx);
        const Axis ay = axis_taps(fmaf(fm, r.qy, r.py), p.ny);
        const Axis az = axis_taps(fmaf(fm, r.qz, r.pz), p.nz);
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
            const float wz = y * (dz ? az.w1 : az.w0);
            if (wz == 0.0f) continue;
            const size_t oz = (dz ? az.i1 : az.i0) * sxy;
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const float wzy = wz * (dy ? ay.w1 : ay.w0);
                if (wzy == 0.0f) continue;
                float *row = V + oz + (size_t)(dy ? ay.i1 : ay.i0) * p.nx;
                if (ax.w0 != 0.0f) atomicAdd(row + ax.i0, wzy * ax.w0);
                if (ax.w1 != 0.0f) atomicAdd(row + ax.i1, wzy * ax.w1);
            }
        }
    }
}

}  // namespace

cudaError_t launch_fp2d(const void *vol, void *sino, int batch, const FP2DParams &p, pyro_dtype dt, cudaStream_t s)
{
    dim3 block(128);
    dim3 grid((p.nu + 127) / 128, p.n_views, batch);
    switch (dt) {
    case PYRO_F32:
        fp2d_kernel<float><<<grid, block, 0, s>>>((const float *)vol, (float *)sino, p);
        break;
    case PYRO_F16:
        fp2d_kernel<__half><<<grid, block, 0, s>>>((const __half *)vol, (__half *)sino, p);
        break;
    case PYRO_BF16:
        fp2d_kernel<__nv_bfloat16><<<grid, block, 0, s>>>((const __nv_bfloat16 *)vol, (__nv_bfloat16 *)sino, p);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_fp2d_adjoint(const void *sino, void *vol, int batch, const FP2DParams &p, cudaStream_t s)
{
    dim3 block(128);
    dim3 grid((p.nu + 127) / 128, p.n_views, batch);
    fp2d_adjoint_kernel<<<grid, block, 0, s>>>((const float *)sino, (float *)vol, p);
    return cudaGetLastError();
}

cudaError_t launch_fp3d(const void *vol, void *sino, int batch, const FP3DParams &p, pyro_dtype dt, cudaStream_t s)
{
    dim3 block(kFP3DBlockX, kFP3DBlockY);
    dim3 grid((p.nu + kFP3DBlockX - 1) / kFP3DBlockX, (p.nv + kFP3DBlockY - 1) / kFP3DBlockY,
              (unsigned)(p.n_views * batch));
    switch (dt) {
    case PYRO_F32:
        fp3d_kernel<float><<<grid, block, 0, s>>>((const float *)vol, (float *)sino, p);
        break;
    case PYRO_F16:
        fp3d_kernel<__half><<<grid, block, 0, s>>>((const __half *)vol, (__half *)sino, p);
        break;
    case PYRO_BF16:
        fp3d_kernel<__nv_bfloat16><<<grid, block, 0, s>>>((const __nv_bfloat16 *)vol, (__nv_bfloat16 *)sino, p);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_relayout_zmajor(const void *vol, void *vz, int nx, int ny, int nz, pyro_dtype dt, cudaStream_t s)
{
    dim3 block(32, 8), grid((nx + 31) / 32, (nz + 31) / 32, ny);
    switch (dt) {
    case PYRO_F32:
        relayout_zmajor_kernel<float><<<grid, block, 0, s>>>((const float *)vol, (float *)vz, nx, ny, nz);
        break;
    case PYRO_F16:
        relayout_zmajor_kernel<__half><<<grid, block, 0, s>>>((const __half *)vol, (__half *)vz, nx, ny, nz);
        break;
    case PYRO_BF16:
        relayout_zmajor_kernel<__nv_bfloat16>
            <<<grid, block, 0, s>>>((const __nv_bfloat16 *)vol, (__nv_bfloat16 *)vz, nx, ny, nz);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_fp3d_zmajor(const void *vz, void *sino, int b, const FP3DParams &p, pyro_dtype dt, cudaStream_t s)
{
    dim3 block(kFPZLanes, kFPZWarps);
    dim3 grid((p.nv + kFPZLanes - 1) / kFPZLanes, (p.nu + kFPZWarps - 1) / kFPZWarps, (unsigned)p.n_views);
    switch (dt) {
    case PYRO_F32:
        fp3d_zmajor_kernel<float><<<grid, block, 0, s>>>((const float *)vz, (float *)sino, p, b);
        break;
    case PYRO_F16:
        fp3d_zmajor_kernel<__half><<<grid, block, 0, s>>>((const __half *)vz, (__half *)sino, p, b);
        break;
    case PYRO_BF16:
        fp3d_zmajor_kernel<__nv_bfloat16><<<grid, block, 0, s>>>((const __nv_bfloat16 *)vz, (__nv_bfloat16 *)sino,
                                                                   p, b);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_fp3d_adjoint(const void *sino, void *vol, int batch, const FP3DParams &p, cudaStream_t s)
{
    dim3 block(kFP3DBlockX, kFP3DBlockY);
    dim3 grid((p.nu + kFP3DBlockX - 1) / kFP3DBlockX, (p.nv + kFP3DBlockY - 1) / kFP3DBlockY,
              (unsigned)(p.n_views * batch));
    fp3d_adjoint_kernel<<<grid, block, 0, s>>>((const float *)sino, (float *)vol, p);
    return cudaGetLastError();
}

}  // namespace pyro
