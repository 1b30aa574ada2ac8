// Ray-driven forward projection A and its exact adjoint A^T
// (paper, Section "The Operator as a Layer": one thread per detector pixel
// casts its ray and accumulates interpolated samples; the cone-beam rays
// come from projection matrices, after Galigekere et al.).
//
// Every ray X(w) = a + w g (g with unit depth along the view's principal
// axis) is sampled on the depth planes w_m = w0 + m dt, m = -M..M, w0 the
// depth of the iso-centre, and p = dt |g| sum_m f(X(w_m)).  Only the m whose
// sample can touch the support (-1, N) of the zero-extended interpolant are
// visited (the others contribute exactly zero).  Rays of one detector column
// lie in one plane through the source, so on a given depth plane they share
// their (x, y) point: the warps below put consecutive detector rows on
// consecutive lanes.  Arithmetic and accumulation are FP32; storage is FP32,
// FP16 or BF16.
#include "device_common.cuh"
#include "internal.h"

namespace pyro {

namespace {

// ---- 2D ray set-up: sample position p0 + m q in pixel-index units --------
struct Ray2 {
    float px, py, qx, qy, w;  // sample m at (px + m qx, py + m qy); weight w = dt |g|
};

// parallel beam: a = u e_u, g = c, w0 = 0; fan beam: g = c + (u / SDD) e_u and
// the sample on the iso-centre's depth plane is a + SID g = (SID u / SDD) e_u
__device__ __forceinline__ Ray2 ray2d(const FP2DParams &p, int v, int k)
{
    const float2 c = p.dir[v];
    const float u = ((float)k - p.cu) * p.su;
    float bx, by, gx, gy, w;
    if (p.fan) {
        const float t = u / p.sdd;
        const float f = p.sid * t;
        bx = -f * c.y;  // e_u = (-c.y, c.x)
        by = f * c.x;
        gx = fmaf(-t, c.y, c.x);
        gy = fmaf(t, c.x, c.y);
        w = p.dt * sqrtf(fmaf(t, t, 1.0f));
    } else {
        bx = -u * c.y;
        by = u * c.x;
        gx = c.x;
        gy = c.y;
        w = p.dt;
    }
    Ray2 r;
    r.px = fmaf(bx, p.inv_sx, p.cx);
    r.py = fmaf(by, p.inv_sy, p.cy);
    r.qx = gx * p.dt * p.inv_sx;
    r.qy = gy * p.dt * p.inv_sy;
    r.w = w;
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
    sino[((size_t)b * p.views_total + p.view0 + v) * p.nu + k] = to_storage<T>(r.w * acc);
}

__global__ void __launch_bounds__(128) fp2d_adjoint_kernel(const float *__restrict__ sino, float *__restrict__ vol,
                                                           const __grid_constant__ FP2DParams p)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    const int b = blockIdx.z;
    if (k >= p.nu) return;
    const float y0s = sino[((size_t)b * p.views_total + p.view0 + v) * p.nu + k];
    if (y0s == 0.0f) return;
    const Ray2 r = ray2d(p, v, k);
    const float y = r.w * y0s;
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
    float px, py, pz, qx, qy, qz, w;  // sample m at p + m q (voxel-index units); weight w = dt |g|
};

// In camera coordinates the ray of pixel (k, l) is S + w q, q = K^-1 (k, l, 1)
// = (q_x, q_y, 1) (unit depth).  Its sample on the iso-centre's depth plane
// (w0 = -s3) is (s1 - s3 q_x, s2 - s3 q_y, 0): no FP32 cancellation.
__device__ __forceinline__ Ray3 ray3d(const FP3DParams &p, int v, int k, int l)
{
    const ConeFPView &V = p.v[v];
    const float fk = (float)k, fl = (float)l;
    const float qx = fmaf(V.a0, fk, fmaf(V.a1, fl, V.a2));
    const float qy = fmaf(V.b0, fl, V.b2);
    const float c0 = fmaf(-V.s3, qx, V.s1);
    const float c1 = fmaf(-V.s3, qy, V.s2);
    const float *W = V.W;
    Ray3 r;
    r.px = fmaf(W[0], c0, fmaf(W[1], c1, p.cx));
    r.py = fmaf(W[3], c0, fmaf(W[4], c1, p.cy));
    r.pz = fmaf(W[6], c0, fmaf(W[7], c1, p.cz));
    r.qx = p.dt * fmaf(W[0], qx, fmaf(W[1], qy, W[2]));
    r.qy = p.dt * fmaf(W[3], qx, fmaf(W[4], qy, W[5]));
    r.qz = p.dt * fmaf(W[6], qx, fmaf(W[7], qy, W[8]));
    r.w = p.dt * sqrtf(fmaf(qx, qx, fmaf(qy, qy, 1.0f)));
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
    sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k] = to_storage<T>(r.w * acc);
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
    // samples strictly inside the volume take the unmasked path; the rest the zero-extended one
    float lo = (float)m0, hi = (float)m1;
    clip_axis_interior(r.px, r.qx, p.nx, lo, hi);
    clip_axis_interior(r.py, r.qy, p.ny, lo, hi);
    clip_axis_interior(r.pz, r.qz, p.nz, lo, hi);
    int i0 = max(m0, (int)ceilf(lo)), i1 = min(m1, (int)floorf(hi));
    if (i0 > i1) {
        i0 = m1 + 1;
        i1 = m1;
    }
    const size_t sx = (size_t)p.nz, sy = (size_t)p.nz * p.nx;
    float acc = 0.0f;
    for (int m = m0; m < i0; ++m) {
        const float fm = (float)m;
        acc += trilerp_zero_strided(vz, p.nx, p.ny, p.nz, sx, sy, (size_t)1, fmaf(fm, r.qx, r.px), fmaf(fm, r.qy, r.py),
                                    fmaf(fm, r.qz, r.pz));
    }
    // interior: consecutive samples are half a voxel apart and the warp's rays
    // (consecutive detector rows) sit at one (x, y) point on every depth plane,
    // so the 8 taps of the current cell stay in registers until the cell changes
    const int stx = p.nz, sty = p.nz * p.nx;
    int cur = -1;
    float c000 = 0.f, c001 = 0.f, c010 = 0.f, c011 = 0.f, c100 = 0.f, c101 = 0.f, c110 = 0.f, c111 = 0.f;
    for (int m = i0; m <= i1; ++m) {
        const float fm = (float)m;
        const float fx = fmaf(fm, r.qx, r.px), fy = fmaf(fm, r.qy, r.py), fz = fmaf(fm, r.qz, r.pz);
        const float x0 = floorf(fx), y0 = floorf(fy), z0 = floorf(fz);
        const int cell = (int)x0 * stx + (int)y0 * sty + (int)z0;
        if (cell != cur) {
            const T *q = vz + cell;
            c000 = ld(q);
            c001 = ld(q + 1);
            c010 = ld(q + sty);
            c011 = ld(q + sty + 1);
            c100 = ld(q + stx);
            c101 = ld(q + stx + 1);
            c110 = ld(q + stx + sty);
            c111 = ld(q + stx + sty + 1);
            cur = cell;
        }
        const float ax = fx - x0, ay = fy - y0, az = fz - z0;
        const float v00 = lerpf(c000, c001, az), v01 = lerpf(c010, c011, az);
        const float v10 = lerpf(c100, c101, az), v11 = lerpf(c110, c111, az);
        acc += lerpf(lerpf(v00, v01, ay), lerpf(v10, v11, ay), ax);
    }
    for (int m = max(i1 + 1, i0); m <= m1; ++m) {
        const float fm = (float)m;
        acc += trilerp_zero_strided(vz, p.nx, p.ny, p.nz, sx, sy, (size_t)1, fmaf(fm, r.qx, r.px), fmaf(fm, r.qy, r.py),
                                    fmaf(fm, r.qz, r.pz));
    }
    sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k] = to_storage<T>(r.w * acc);
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
    const float y0s = sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k];
    if (y0s == 0.0f) return;
    const Ray3 r = ray3d(p, v, k, l);
    const float y = r.w * y0s;
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
