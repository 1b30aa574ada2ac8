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

// volT (may be NULL): the batch transposed, [b][x][y].  The lanes of a warp
// take consecutive detector bins, which for a given sample lie along e_u:
// when the rays run closer to x than to y (|c_x| > |c_y|) the bins spread
// along y, so their taps are contiguous in the transposed copy; the kernel
// then reads that copy with the roles of x and y swapped.
template <typename T>
__global__ void __launch_bounds__(128) fp2d_kernel(const T *__restrict__ vol, const T *__restrict__ volT,
                                                   T *__restrict__ sino, const __grid_constant__ FP2DParams p)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    const int b = blockIdx.z;
    if (k >= p.nu) return;
    Ray2 r = ray2d(p, v, k);
    int m0, m1;
    range2d(r, p, m0, m1);
    const T *img = vol + (size_t)b * p.nx * p.ny;
    int nx = p.nx, ny = p.ny;
    if (volT && fabsf(p.dir[v].x) > fabsf(p.dir[v].y)) {  // the whole block: one view
        img = volT + (size_t)b * p.nx * p.ny;
        nx = p.ny;
        ny = p.nx;
        const float t0 = r.px, t1 = r.qx;
        r.px = r.py;
        r.qx = r.qy;
        r.py = t0;
        r.qy = t1;
    }
    // samples whose four taps are all inside the image take the unmasked path
    float lo = (float)m0, hi = (float)m1;
    clip_axis_interior(r.px, r.qx, nx, lo, hi);
    clip_axis_interior(r.py, r.qy, ny, lo, hi);
    int i0 = max(m0, (int)ceilf(lo)), i1 = min(m1, (int)floorf(hi));
    if (i0 > i1) {  // no interior sample
        i0 = m1 + 1;
        i1 = m1;
    }
    float acc = 0.0f;
    for (int m = m0; m < i0; ++m) {
        const float fm = (float)m;
        acc += bilerp_zero(img, nx, ny, fmaf(fm, r.qx, r.px), fmaf(fm, r.qy, r.py));
    }
    // two samples per iteration with separate partial sums (unrolled twice
    // more by the compiler), so that several samples' loads are in flight
    float acc2 = 0.0f;
    int m = i0;
#pragma unroll 2
    for (; m + 1 <= i1; m += 2) {
        const float fa = (float)m, fb = (float)(m + 1);
        acc += bilerp_interior(img, 1, nx, fmaf(fa, r.qx, r.px), fmaf(fa, r.qy, r.py));
        acc2 += bilerp_interior(img, 1, nx, fmaf(fb, r.qx, r.px), fmaf(fb, r.qy, r.py));
    }
    if (m <= i1) acc += bilerp_interior(img, 1, nx, fmaf((float)m, r.qx, r.px), fmaf((float)m, r.qy, r.py));
    acc += acc2;
    for (int m = max(i1 + 1, i0); m <= m1; ++m) {
        const float fm = (float)m;
        acc += bilerp_zero(img, nx, ny, fmaf(fm, r.qx, r.px), fmaf(fm, r.qy, r.py));
    }
    sino[((size_t)b * p.views_total + p.view0 + v) * p.nu + k] = to_storage<T>(r.w * acc);
}

// volT (may be NULL): a zeroed transposed accumulator [b][x][y] that takes
// the views whose rays run closer to x than to y (their detector bins spread
// along y, so the warp's atomics are contiguous there); the caller adds it
// back, transposed, into vol.
__global__ void __launch_bounds__(128) fp2d_adjoint_kernel(const float *__restrict__ sino, float *__restrict__ vol,
                                                           float *__restrict__ volT,
                                                           const __grid_constant__ FP2DParams p)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    const int b = blockIdx.z;
    if (k >= p.nu) return;
    const float y0s = sino[((size_t)b * p.views_total + p.view0 + v) * p.nu + k];
    if (y0s == 0.0f) return;
    Ray2 r = ray2d(p, v, k);
    const float y = r.w * y0s;
    int m0, m1;
    range2d(r, p, m0, m1);
    float *img = vol + (size_t)b * p.nx * p.ny;
    int nx = p.nx, ny = p.ny;
    if (volT && fabsf(p.dir[v].x) > fabsf(p.dir[v].y)) {  // the whole block: one view
        img = volT + (size_t)b * p.nx * p.ny;
        nx = p.ny;
        ny = p.nx;
        const float t0 = r.px, t1 = r.qx;
        r.px = r.py;
        r.qx = r.qy;
        r.py = t0;
        r.qy = t1;
    }
    for (int m = m0; m <= m1; ++m) {
        const float fm = (float)m;
        const Axis ax = axis_taps(fmaf(fm, r.qx, r.px), nx);
        const Axis ay = axis_taps(fmaf(fm, r.qy, r.py), ny);
        float *r0 = img + (size_t)ay.i0 * nx;
        float *r1 = img + (size_t)ay.i1 * nx;
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

// Texture-mode forward projection, the paper's fast mode (Section "The
// Operator as a Layer"): the volume sits in a 3D CUDA array, read through a
// texture object with hardware trilinear filtering and a zero border (the
// zero extension of the software path), so one fetch replaces eight taps and
// seven lerps.  The price is the second copy of the volume and the hardware's
// fixed-point interpolation weights (8 fractional bits), which put the result
// about 1e-4 .. 1e-3 from the FP32 software path.  Same rays, sample grid and
// clipping as fp3d_kernel.  A warp covers 8 detector columns x 4 rows, a
// compact footprint for the texture cache.
constexpr int kFPTexX = 8, kFPTexY = 16;

template <typename T>
__global__ void __launch_bounds__(kFPTexX *kFPTexY) fp3d_tex_kernel(cudaTextureObject_t tex, T *__restrict__ sino,
                                                                    const __grid_constant__ FP3DParams p)
{
    const int k = blockIdx.x * kFPTexX + threadIdx.x;
    const int l = blockIdx.y * kFPTexY + threadIdx.y;
    const int v = blockIdx.z;
    if (k >= p.nu || l >= p.nv) return;
    const Ray3 r = ray3d(p, v, k, l);
    int m0, m1;
    range3d(r, p, m0, m1);
    // texel i's centre is at texture coordinate i + 0.5
    const float px = r.px + 0.5f, py = r.py + 0.5f, pz = r.pz + 0.5f;
    float acc0 = 0.0f, acc1 = 0.0f;
    int m = m0;
    for (; m + 1 <= m1; m += 2) {
        const float f0 = (float)m, f1 = (float)(m + 1);
        acc0 += tex3D<float>(tex, fmaf(f0, r.qx, px), fmaf(f0, r.qy, py), fmaf(f0, r.qz, pz));
        acc1 += tex3D<float>(tex, fmaf(f1, r.qx, px), fmaf(f1, r.qy, py), fmaf(f1, r.qz, pz));
    }
    if (m <= m1) {
        const float f0 = (float)m;
        acc0 += tex3D<float>(tex, fmaf(f0, r.qx, px), fmaf(f0, r.qy, py), fmaf(f0, r.qz, pz));
    }
    sino[((size_t)(p.view0 + v) * p.nv + l) * p.nu + k] = to_storage<T>(r.w * (acc0 + acc1));
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

// Column-shared projection.  When the detector's v axis maps onto the
// volume's z axis (circular and helical-free trajectories: no skew, camera y
// axis = z), all rays of one detector column k share their (x, y) point on
// every depth plane; only z differs, and it grows monotonically with the row
// l.  A warp takes column k and R windows of 32 consecutive rows.  On each
// depth plane it computes the (x, y) cell and its bilinear weights once; in
// each window every lane loads the four (x, y) columns at one z of the
// window's 32-voxel run (one coalesced 128-byte load per column) and
// combines them in x and y, and each lane then takes the two z taps of its
// own ray from the lanes holding them (two shuffles).  The host checks that
// 31 row steps stay below 29.5 voxels in z, so a window's taps always fall in
// its 32-voxel run.  The volume copy is [ny+2][nx+2][nz+2] with a zero voxel
// on every face: loads need no bounds test, and the zero-extended
// interpolant comes out of the padding.
constexpr int kFPCWarps = 4;

struct ColumnWindow {
    float pz, qz;    // this lane's ray: z(m) = pz + m qz
    float pzb, qzb;  // the window's lowest row
    float w;         // ray weight dt |g|
    float acc;       // forward: the ray sum; adjoint: w times the ray's datum
    int ma, mb;      // samples of the window's rows that can touch the volume
};

// (x, y) cell of depth plane m shared by the column's rays: bilinear weights
// and the padded element index of (x0, y0, z = 0)
struct PlaneXY {
    float w00, w10, w01, w11;
    int col;
};

__device__ __forceinline__ PlaneXY plane_xy(float fm, const Ray3 &rc, int sxp, int syp)
{
    const float fx = fmaf(fm, rc.qx, rc.px), fy = fmaf(fm, rc.qy, rc.py);
    const float tx = floor_magic(fx), ty = floor_magic(fy);
    const float ax = fx - magic_to_float(tx), ay = fy - magic_to_float(ty);
    const float bx = 1.0f - ax, by = 1.0f - ay;
    PlaneXY q;
    q.w00 = bx * by;
    q.w10 = ax * by;
    q.w01 = bx * ay;
    q.w11 = ax * ay;
    q.col = (magic_to_int(ty) + 1) * syp + (magic_to_int(tx) + 1) * sxp + 1;
    return q;
}

// One depth plane of one window: the lane's x/y-interpolated value at
// z = zb + lane, then its own ray's z interpolation from two lanes.
template <typename T>
__device__ __forceinline__ void column_step(ColumnWindow &W, float fm, int lane, int nz, const T *const (&c)[4],
                                            const PlaneXY &q)
{
    const float tzb = floor_magic(fmaf(fm, W.qzb, W.pzb));
    const int zi = min(max(magic_to_int(tzb) + lane, -1), nz);
    const float g = q.w00 * ld(c[0] + zi) + q.w10 * ld(c[1] + zi) + q.w01 * ld(c[2] + zi) + q.w11 * ld(c[3] + zi);
    const float fz = fmaf(fm, W.qz, W.pz);
    const float tz = floor_magic(fz);
    const int j = __float_as_int(tz) - __float_as_int(tzb);  // own cell relative to the window's run
    const float g0 = __shfl_sync(0xffffffffu, g, j), g1 = __shfl_sync(0xffffffffu, g, j + 1);
    W.acc += fmaf(fz - magic_to_float(tz), g1 - g0, g0);
}

// Transpose of column_step: the lane's ray datum y is split between the two
// z cells of its sample in the window's run (a shared-memory array of 32
// sums), then each lane spreads the sum of its cell over the four (x, y)
// columns with global atomics: four atomics per 32 samples.  Only the taps
// with z in [zs0, zs1) are written (the host passes the whole volume:
// accumulating a volume larger than L2 slab by slab, each slab a launch,
// was measured slower, 2.7 s against 1.7 s at 512^3, because windows that
// straddle a slab boundary repeat their work).
__device__ __forceinline__ void column_step_adjoint(const ColumnWindow &W, float fm, int lane, int zs0, int zs1,
                                                    float *const (&c)[4], const PlaneXY &q, float *run)
{
    const float tzb = floor_magic(fmaf(fm, W.qzb, W.pzb));
    const int zi = magic_to_int(tzb) + lane;
    const float fz = fmaf(fm, W.qz, W.pz);
    const float tz = floor_magic(fz);
    // 0..30 for every real row (host-checked); clamped so that no shared
    // access leaves the run
    const int j = min(max(__float_as_int(tz) - __float_as_int(tzb), 0), 30);
    const float az = fz - magic_to_float(tz);
    const float y = W.acc;
    if (y != 0.0f) {
        atomicAdd(run + j, fmaf(-az, y, y));
        atomicAdd(run + j + 1, az * y);
    }
    __syncwarp();
    const float d = run[lane];
    run[lane] = 0.0f;
    __syncwarp();
    // only this launch's slab: the taps of the other z belong to other launches
    if (d != 0.0f && zi >= zs0 && zi < zs1) {
        atomicAdd(c[0] + zi, q.w00 * d);
        atomicAdd(c[1] + zi, q.w10 * d);
        atomicAdd(c[2] + zi, q.w01 * d);
        atomicAdd(c[3] + zi, q.w11 * d);
    }
}

// Depth planes m0..m1 of all R windows.  CHECK skips the windows whose rows
// cannot touch the volume on a plane (outside the planes every window
// reaches; elsewhere the skipped terms would be exact zeros anyway: the
// forward reads the zero padding, the adjoint writes into it).
template <typename T, int R, bool CHECK, bool ADJ>
__device__ __forceinline__ void column_planes(ColumnWindow (&W)[R], int m0, int m1, const Ray3 &rc, int lane, T *vp,
                                              int nz, int sxp, int syp, float *runs, int zs0, int zs1)
{
    // unrolled by 4 on the forward path (measured 1 % faster than 2, while
    // 1, 6 and 8 were slower) and by 2 on the adjoint's
    constexpr int kUnroll = ADJ ? 2 : 4;
    float fm = (float)m0;
#pragma unroll kUnroll
    for (int m = m0; m <= m1; ++m, fm += 1.0f) {
        const PlaneXY q = plane_xy(fm, rc, sxp, syp);
        T *const c[4] = {vp + q.col, vp + q.col + sxp, vp + q.col + syp, vp + q.col + sxp + syp};
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (CHECK && (m < W[r].ma || m > W[r].mb)) continue;  // whole warp
            if constexpr (ADJ) {
                column_step_adjoint(W[r], fm, lane, zs0, zs1, c, q, runs + 32 * r);
            } else {
                const T *const cr[4] = {c[0], c[1], c[2], c[3]};
                column_step(W[r], fm, lane, nz, cr, q);
            }
        }
    }
}

// Set-up shared by the forward and adjoint column kernels: the column's
// (x, y) track rc, the windows' rays and ranges; returns the union [mlo, mhi]
// of the windows' ranges and the planes [clo, chi] every window reaches.
// Restrict m of p0 + m q to the open interval (a, b) (rounded outwards).
__device__ __forceinline__ void clip_open(float p0, float q, float a, float b, float &lo, float &hi)
{
    if (fabsf(q) > 1e-30f) {
        const float t1 = (a - p0) / q, t2 = (b - p0) / q;
        lo = fmaxf(lo, fminf(t1, t2));
        hi = fminf(hi, fmaxf(t1, t2));
    } else if (!(p0 > a && p0 < b)) {
        lo = 1.0f;
        hi = -1.0f;
    }
}

// zlo, zhi: the open z interval whose samples matter (the volume's (-1, nz),
// or a slab's (zs0 - 1, zs1) for the slab-blocked adjoint)
template <int R>
__device__ __forceinline__ void column_setup(const FP3DParams &p, int v, int k, int row0, int lane, Ray3 &rc,
                                             ColumnWindow (&W)[R], int &mlo, int &mhi, int &clo, int &chi,
                                             float zlo, float zhi)
{
    const unsigned full = 0xffffffffu;
    rc = ray3d(p, v, k, row0);  // (x, y) track of the column, common to all its rows
    float lo = -(float)p.M, hi = (float)p.M;
    clip_axis(rc.px, rc.qx, p.nx, lo, hi);
    clip_axis(rc.py, rc.qy, p.ny, lo, hi);
    int m0 = max(-p.M, (int)floorf(lo)), m1 = min(p.M, (int)ceilf(hi));
    // keep the samples whose cell (x0, y0) lies in [-1, n-1]^2; the clip above
    // is rounded outwards by at most one sample
    auto inside = [&](int m) {
        const float fx = fmaf((float)m, rc.qx, rc.px), fy = fmaf((float)m, rc.qy, rc.py);
        return fx >= -1.0f && fx < (float)p.nx && fy >= -1.0f && fy < (float)p.ny;
    };
    while (m0 <= m1 && !inside(m0)) ++m0;
    while (m1 >= m0 && !inside(m1)) --m1;
    mlo = INT_MAX;
    mhi = INT_MIN;
    clo = INT_MIN;
    chi = INT_MAX;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int l = row0 + 32 * r + lane;
        const Ray3 rr = ray3d(p, v, k, l);
        W[r].pz = rr.pz;
        W[r].qz = rr.qz;
        W[r].w = rr.w;
        W[r].acc = 0.0f;
        // the window's lowest z is at its first or its last row (depth > 0)
        const float z_first = __shfl_sync(full, rr.pz, 0), z_last = __shfl_sync(full, rr.pz, 31);
        const int src = z_last >= z_first ? 0 : 31;
        W[r].pzb = __shfl_sync(full, rr.pz, src);
        W[r].qzb = __shfl_sync(full, rr.qz, src);
        float zl = (float)m0, zh = (float)m1;
        clip_open(rr.pz, rr.qz, zlo, zhi, zl, zh);
        int a = max(m0, (int)floorf(zl)), e = min(m1, (int)ceilf(zh));
        if (l >= p.nv || a > e) {  // no sample of this row touches the volume
            a = INT_MAX;
            e = INT_MIN;
        }
        W[r].ma = __reduce_min_sync(full, a);
        W[r].mb = __reduce_max_sync(full, e);
        if (W[r].ma <= W[r].mb) {
            mlo = min(mlo, W[r].ma);
            mhi = max(mhi, W[r].mb);
            clo = max(clo, W[r].ma);
            chi = min(chi, W[r].mb);
        }
    }
    if (mlo <= mhi && clo > chi) {  // no plane common to all windows
        clo = mhi + 1;
        chi = mhi;
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(32 * kFPCWarps) fp3d_column_kernel(const T *__restrict__ vp,
                                                                     T *__restrict__ sino,
                                                                     const __grid_constant__ FP3DParams p, int b)
{
    const int lane = threadIdx.x;
    const int k = blockIdx.y * kFPCWarps + threadIdx.y;
    const int v = blockIdx.x;
    if (k >= p.nu) return;  // whole warp
    const int row0 = blockIdx.z * (32 * R);
    Ray3 rc;
    ColumnWindow W[R];
    int mlo, mhi, clo, chi;
    column_setup<R>(p, v, k, row0, lane, rc, W, mlo, mhi, clo, chi, -1.0f, (float)p.nz);
    const int sxp = p.nz + 2, syp = (p.nx + 2) * (p.nz + 2);
    if (mlo <= mhi) {
        T *vq = const_cast<T *>(vp);  // read only on the forward path
        column_planes<T, R, true, false>(W, mlo, clo - 1, rc, lane, vq, p.nz, sxp, syp, nullptr, 0, 0);
        column_planes<T, R, false, false>(W, clo, chi, rc, lane, vq, p.nz, sxp, syp, nullptr, 0, 0);
        column_planes<T, R, true, false>(W, max(chi + 1, clo), mhi, rc, lane, vq, p.nz, sxp, syp, nullptr, 0, 0);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int l = row0 + 32 * r + lane;
        if (l < p.nv)
            sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k] = to_storage<T>(W[r].w * W[r].acc);
    }
}

// Exact adjoint of fp3d_column_kernel, accumulated into a zeroed padded
// z-major FP32 volume (the padding collects the terms of samples outside the
// volume and is discarded afterwards).
template <int R>
__global__ void __launch_bounds__(32 * kFPCWarps) fp3d_column_adjoint_kernel(const float *__restrict__ sino,
                                                                             float *__restrict__ vp,
                                                                             const __grid_constant__ FP3DParams p,
                                                                             int b)
{
    __shared__ float runs[kFPCWarps][R * 32];
    const int lane = threadIdx.x;
    const int k = blockIdx.y * kFPCWarps + threadIdx.y;
    const int v = blockIdx.x;
    if (k >= p.nu) return;  // whole warp
    float *run = runs[threadIdx.y];
#pragma unroll
    for (int r = 0; r < R; ++r) run[32 * r + lane] = 0.0f;
    __syncwarp();
    const int row0 = blockIdx.z * (32 * R);
    Ray3 rc;
    ColumnWindow W[R];
    int mlo, mhi, clo, chi;
    column_setup<R>(p, v, k, row0, lane, rc, W, mlo, mhi, clo, chi, (float)(p.zs0 - 1), (float)p.zs1);
    if (mlo > mhi) return;  // whole warp: no sample of its rays touches the slab
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int l = row0 + 32 * r + lane;
        W[r].acc = l < p.nv ? W[r].w * sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k] : 0.0f;
    }
    const int sxp = p.nz + 2, syp = (p.nx + 2) * (p.nz + 2);
    {
        column_planes<float, R, true, true>(W, mlo, clo - 1, rc, lane, vp, p.nz, sxp, syp, run, p.zs0, p.zs1);
        column_planes<float, R, false, true>(W, clo, chi, rc, lane, vp, p.nz, sxp, syp, run, p.zs0, p.zs1);
        column_planes<float, R, true, true>(W, max(chi + 1, clo), mhi, rc, lane, vp, p.nz, sxp, syp, run, p.zs0,
                                            p.zs1);
    }
}

// ---- two rays per lane: windows of up to 64 rows on one 32-voxel run -----
// When a row step moves a ray by less than about 0.76 voxel in z, 32 rows
// use only part of their window's 32-voxel run.  These kernels give each
// lane two rays, rows row0 + lane and row0 + 32 + lane of a window of WR
// rows (WR = pair_rows <= 64, chosen on the host so that WR - 1 row steps
// stay below 29.5 voxels; the lanes past WR - 32 have no second ray), and
// both rays take their taps from the same run: one set of loads and x/y
// combinations for up to twice the rays.  The arithmetic of every ray is
// that of fp3d_column_kernel.
struct PairRowsWindow {
    float pz[2], qz[2];  // the lane's two rays: z(m) = pz + m qz
    float pzb, qzb;      // the window's lowest row
    float acc[2];        // forward: the ray sums; adjoint: w times the rays' data
    int ma, mb;          // samples of the window's rows that can touch the volume
};

template <int R>
__device__ __forceinline__ void pair_rows_setup(const FP3DParams &p, int v, int k, int row0, int lane, Ray3 &rc,
                                                PairRowsWindow (&W)[R], int &mlo, int &mhi, int &clo, int &chi,
                                                float zlo, float zhi)
{
    const unsigned full = 0xffffffffu;
    const int WR = p.pair_rows;
    rc = ray3d(p, v, k, row0);
    float lo = -(float)p.M, hi = (float)p.M;
    clip_axis(rc.px, rc.qx, p.nx, lo, hi);
    clip_axis(rc.py, rc.qy, p.ny, lo, hi);
    int m0 = max(-p.M, (int)floorf(lo)), m1 = min(p.M, (int)ceilf(hi));
    auto inside = [&](int m) {
        const float fx = fmaf((float)m, rc.qx, rc.px), fy = fmaf((float)m, rc.qy, rc.py);
        return fx >= -1.0f && fx < (float)p.nx && fy >= -1.0f && fy < (float)p.ny;
    };
    while (m0 <= m1 && !inside(m0)) ++m0;
    while (m1 >= m0 && !inside(m1)) --m1;
    mlo = INT_MAX;
    mhi = INT_MIN;
    clo = INT_MIN;
    chi = INT_MAX;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int a = INT_MAX, e = INT_MIN;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = row0 + r * WR + 32 * h + lane;
            const Ray3 rr = ray3d(p, v, k, l);
            W[r].pz[h] = rr.pz;
            W[r].qz[h] = rr.qz;
            W[r].acc[h] = 0.0f;
            const bool real = l < p.nv && 32 * h + lane < WR;
            float zl = (float)m0, zh = (float)m1;
            clip_open(rr.pz, rr.qz, zlo, zhi, zl, zh);
            const int aa = max(m0, (int)floorf(zl)), ee = min(m1, (int)ceilf(zh));
            if (real && aa <= ee) {
                a = min(a, aa);
                e = max(e, ee);
            }
        }
        // the window's lowest z is at its first row (lane 0's first ray) or its
        // last (lane WR - 33's second ray): depth > 0
        const float zf = __shfl_sync(full, W[r].pz[0], 0), zq = __shfl_sync(full, W[r].qz[0], 0);
        const float zl = __shfl_sync(full, W[r].pz[1], WR - 33), zlq = __shfl_sync(full, W[r].qz[1], WR - 33);
        W[r].pzb = zl >= zf ? zf : zl;
        W[r].qzb = zl >= zf ? zq : zlq;
        W[r].ma = __reduce_min_sync(full, a);
        W[r].mb = __reduce_max_sync(full, e);
        if (W[r].ma <= W[r].mb) {
            mlo = min(mlo, W[r].ma);
            mhi = max(mhi, W[r].mb);
            clo = max(clo, W[r].ma);
            chi = min(chi, W[r].mb);
        }
    }
    if (mlo <= mhi && clo > chi) {
        clo = mhi + 1;
        chi = mhi;
    }
}


// one depth plane of one window: the run as in column_step, then both rays'
// z interpolations from it
template <typename T>
__device__ __forceinline__ void pair_rows_step(PairRowsWindow &W, float fm, int lane, int nz, const T *const (&c)[4],
                                               const PlaneXY &q)
{
    const float tzb = floor_magic(fmaf(fm, W.qzb, W.pzb));
    const int zi = min(max(magic_to_int(tzb) + lane, -1), nz);
    const float g = q.w00 * ld(c[0] + zi) + q.w10 * ld(c[1] + zi) + q.w01 * ld(c[2] + zi) + q.w11 * ld(c[3] + zi);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float fz = fmaf(fm, W.qz[h], W.pz[h]);
        const float tz = floor_magic(fz);
        const int j = __float_as_int(tz) - __float_as_int(tzb);
        const float g0 = __shfl_sync(0xffffffffu, g, j), g1 = __shfl_sync(0xffffffffu, g, j + 1);
        W.acc[h] += fmaf(fz - magic_to_float(tz), g1 - g0, g0);
    }
}

// transpose of pair_rows_step: both rays' data go into the run's cells, then
// each lane spreads its cell over the four (x, y) columns (as
// column_step_adjoint)
__device__ __forceinline__ void pair_rows_step_adjoint(const PairRowsWindow &W, float fm, int lane, int zs0, int zs1,
                                                       float *const (&c)[4], const PlaneXY &q, float *run)
{
    const float tzb = floor_magic(fmaf(fm, W.qzb, W.pzb));
    const int zi = magic_to_int(tzb) + lane;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float fz = fmaf(fm, W.qz[h], W.pz[h]);
        const float tz = floor_magic(fz);
        const int j = min(max(__float_as_int(tz) - __float_as_int(tzb), 0), 30);
        const float az = fz - magic_to_float(tz);
        const float y = W.acc[h];
        if (y != 0.0f) {
            atomicAdd(run + j, fmaf(-az, y, y));
            atomicAdd(run + j + 1, az * y);
        }
    }
    __syncwarp();
    const float d = run[lane];
    run[lane] = 0.0f;
    __syncwarp();
    if (d != 0.0f && zi >= zs0 && zi < zs1) {
        atomicAdd(c[0] + zi, q.w00 * d);
        atomicAdd(c[1] + zi, q.w10 * d);
        atomicAdd(c[2] + zi, q.w01 * d);
        atomicAdd(c[3] + zi, q.w11 * d);
    }
}

template <typename T, int R, bool CHECK, bool ADJ>
__device__ __forceinline__ void pair_rows_planes(PairRowsWindow (&W)[R], int m0, int m1, const Ray3 &rc, int lane,
                                                 T *vp, int nz, int sxp, int syp, float *runs, int zs0, int zs1)
{
    constexpr int kUnroll = ADJ ? 2 : 4;
    float fm = (float)m0;
#pragma unroll kUnroll
    for (int m = m0; m <= m1; ++m, fm += 1.0f) {
        const PlaneXY q = plane_xy(fm, rc, sxp, syp);
        T *const c[4] = {vp + q.col, vp + q.col + sxp, vp + q.col + syp, vp + q.col + sxp + syp};
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (CHECK && (m < W[r].ma || m > W[r].mb)) continue;  // whole warp
            if constexpr (ADJ) {
                pair_rows_step_adjoint(W[r], fm, lane, zs0, zs1, c, q, runs + 32 * r);
            } else {
                const T *const cr[4] = {c[0], c[1], c[2], c[3]};
                pair_rows_step(W[r], fm, lane, nz, cr, q);
            }
        }
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(32 * kFPCWarps) fp3d_pair_rows_kernel(const T *__restrict__ vp,
                                                                        T *__restrict__ sino,
                                                                        const __grid_constant__ FP3DParams p, int b)
{
    const int lane = threadIdx.x;
    const int k = blockIdx.y * kFPCWarps + threadIdx.y;
    const int v = blockIdx.x;
    if (k >= p.nu) return;  // whole warp
    const int WR = p.pair_rows;
    const int row0 = blockIdx.z * (R * WR);
    Ray3 rc;
    PairRowsWindow W[R];
    int mlo, mhi, clo, chi;
    pair_rows_setup<R>(p, v, k, row0, lane, rc, W, mlo, mhi, clo, chi, -1.0f, (float)p.nz);
    const int sxp = p.nz + 2, syp = (p.nx + 2) * (p.nz + 2);
    if (mlo <= mhi) {
        T *vq = const_cast<T *>(vp);  // read only on the forward path
        pair_rows_planes<T, R, true, false>(W, mlo, clo - 1, rc, lane, vq, p.nz, sxp, syp, nullptr, 0, 0);
        pair_rows_planes<T, R, false, false>(W, clo, chi, rc, lane, vq, p.nz, sxp, syp, nullptr, 0, 0);
        pair_rows_planes<T, R, true, false>(W, max(chi + 1, clo), mhi, rc, lane, vq, p.nz, sxp, syp, nullptr, 0, 0);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = row0 + r * WR + 32 * h + lane;
            if (l < p.nv && 32 * h + lane < WR)
                sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k] =
                    to_storage<T>(ray3d(p, v, k, l).w * W[r].acc[h]);
        }
}

template <int R>
__global__ void __launch_bounds__(32 * kFPCWarps) fp3d_pair_rows_adjoint_kernel(const float *__restrict__ sino,
                                                                                float *__restrict__ vp,
                                                                                const __grid_constant__ FP3DParams p,
                                                                                int b)
{
    __shared__ float runs[kFPCWarps][R * 32];
    const int lane = threadIdx.x;
    const int k = blockIdx.y * kFPCWarps + threadIdx.y;
    const int v = blockIdx.x;
    if (k >= p.nu) return;  // whole warp
    float *run = runs[threadIdx.y];
#pragma unroll
    for (int r = 0; r < R; ++r) run[32 * r + lane] = 0.0f;
    __syncwarp();
    const int WR = p.pair_rows;
    const int row0 = blockIdx.z * (R * WR);
    Ray3 rc;
    PairRowsWindow W[R];
    int mlo, mhi, clo, chi;
    pair_rows_setup<R>(p, v, k, row0, lane, rc, W, mlo, mhi, clo, chi, (float)(p.zs0 - 1), (float)p.zs1);
    if (mlo > mhi) return;  // whole warp: no sample of its rays touches the slab
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = row0 + r * WR + 32 * h + lane;
            W[r].acc[h] = (l < p.nv && 32 * h + lane < WR)
                              ? ray3d(p, v, k, l).w * sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k]
                              : 0.0f;
        }
    const int sxp = p.nz + 2, syp = (p.nx + 2) * (p.nz + 2);
    pair_rows_planes<float, R, true, true>(W, mlo, clo - 1, rc, lane, vp, p.nz, sxp, syp, run, p.zs0, p.zs1);
    pair_rows_planes<float, R, false, true>(W, clo, chi, rc, lane, vp, p.nz, sxp, syp, run, p.zs0, p.zs1);
    pair_rows_planes<float, R, true, true>(W, max(chi + 1, clo), mhi, rc, lane, vp, p.nz, sxp, syp, run, p.zs0,
                                           p.zs1);
}


// interior of the padded z-major array -> [z][y][x]
__global__ void __launch_bounds__(256) relayout_unpad_kernel(const float *__restrict__ vp, float *__restrict__ vol,
                                                             int nx, int ny, int nz)
{
    __shared__ float tile[32][33];
    const int nxp = nx + 2, nzp = nz + 2;
    const int x0 = blockIdx.x * 32, z0 = blockIdx.y * 32, y = blockIdx.z;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int x = x0 + i, z = z0 + threadIdx.x;
        if (x < nx && z < nz) tile[i][threadIdx.x] = vp[((size_t)(y + 1) * nxp + x + 1) * nzp + z + 1];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int z = z0 + i, x = x0 + threadIdx.x;
        if (x < nx && z < nz) vol[((size_t)z * ny + y) * nx + x] = tile[threadIdx.x][i];
    }
}

// [z][y][x] -> [y+1][x+1][z+1] of a zero-padded (ny+2)(nx+2)(nz+2) array:
// every padded element is written once (source voxel or 0)
template <typename T>
__global__ void __launch_bounds__(256) relayout_padded_kernel(const T *__restrict__ vol, T *__restrict__ vp, int nx,
                                                              int ny, int nz)
{
    __shared__ T tile[32][33];
    const int nxp = nx + 2, nzp = nz + 2;
    const int x0 = blockIdx.x * 32, z0 = blockIdx.y * 32, yp = blockIdx.z;
    const int y = yp - 1;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int z = z0 + i - 1, x = x0 + threadIdx.x - 1;
        const bool in = y >= 0 && y < ny && z >= 0 && z < nz && x >= 0 && x < nx;
        tile[i][threadIdx.x] = in ? vol[((size_t)z * ny + y) * nx + x] : to_storage<T>(0.0f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int xp = x0 + i, zp = z0 + threadIdx.x;
        if (zp < nzp && xp < nxp) vp[((size_t)yp * nxp + xp) * nzp + zp] = tile[threadIdx.x][i];
    }
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

cudaError_t launch_fp2d(const void *vol, const void *volT, void *sino, int batch, const FP2DParams &p, pyro_dtype dt,
                        cudaStream_t s)
{
    dim3 block(128);
    dim3 grid((p.nu + 127) / 128, p.n_views, batch);
    switch (dt) {
    case PYRO_F32:
        fp2d_kernel<float><<<grid, block, 0, s>>>((const float *)vol, (const float *)volT, (float *)sino, p);
        break;
    case PYRO_F16:
        fp2d_kernel<__half><<<grid, block, 0, s>>>((const __half *)vol, (const __half *)volT, (__half *)sino, p);
        break;
    case PYRO_BF16:
        fp2d_kernel<__nv_bfloat16><<<grid, block, 0, s>>>((const __nv_bfloat16 *)vol, (const __nv_bfloat16 *)volT,
                                                          (__nv_bfloat16 *)sino, p);
        break;
    }
    return cudaGetLastError();
}

// [b][y][x] -> [b][x][y], 32 x 32 tiles through shared memory
template <typename T>
__global__ void __launch_bounds__(256) transpose2d_kernel(const T *__restrict__ in, T *__restrict__ out, int nx, int ny)
{
    __shared__ T tile[32][33];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const size_t off = (size_t)blockIdx.z * nx * ny;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int y = y0 + i, x = x0 + threadIdx.x;
        if (y < ny && x < nx) tile[i][threadIdx.x] = in[off + (size_t)y * nx + x];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int x = x0 + i, y = y0 + threadIdx.x;
        if (y < ny && x < nx) out[off + (size_t)x * ny + y] = tile[threadIdx.x][i];
    }
}

cudaError_t launch_transpose2d(const void *in, void *out, int batch, int nx, int ny, pyro_dtype dt, cudaStream_t s)
{
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 31) / 32, batch);
    switch (dt) {
    case PYRO_F32:
        transpose2d_kernel<float><<<grid, block, 0, s>>>((const float *)in, (float *)out, nx, ny);
        break;
    case PYRO_F16:
        transpose2d_kernel<__half><<<grid, block, 0, s>>>((const __half *)in, (__half *)out, nx, ny);
        break;
    case PYRO_BF16:
        transpose2d_kernel<__nv_bfloat16>
            <<<grid, block, 0, s>>>((const __nv_bfloat16 *)in, (__nv_bfloat16 *)out, nx, ny);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_fp2d_adjoint(const void *sino, void *vol, void *volT, int batch, const FP2DParams &p,
                                cudaStream_t s)
{
    dim3 block(128);
    dim3 grid((p.nu + 127) / 128, p.n_views, batch);
    fp2d_adjoint_kernel<<<grid, block, 0, s>>>((const float *)sino, (float *)vol, (float *)volT, p);
    return cudaGetLastError();
}

// vol[b][y][x] += accT[b][x][y], 32 x 32 tiles through shared memory
__global__ void __launch_bounds__(256) add_transposed_kernel(const float *__restrict__ accT, float *__restrict__ vol,
                                                             int nx, int ny)
{
    __shared__ float tile[32][33];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const size_t off = (size_t)blockIdx.z * nx * ny;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int x = x0 + i, y = y0 + threadIdx.x;
        if (x < nx && y < ny) tile[i][threadIdx.x] = accT[off + (size_t)x * ny + y];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int y = y0 + i, x = x0 + threadIdx.x;
        if (x < nx && y < ny) vol[off + (size_t)y * nx + x] += tile[threadIdx.x][i];
    }
}

cudaError_t launch_add_transposed(const void *accT, void *vol, int batch, int nx, int ny, cudaStream_t s)
{
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 31) / 32, batch);
    add_transposed_kernel<<<grid, block, 0, s>>>((const float *)accT, (float *)vol, nx, ny);
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

cudaError_t launch_relayout_padded(const void *vol, void *vp, int nx, int ny, int nz, pyro_dtype dt, cudaStream_t s)
{
    dim3 block(32, 8), grid((nx + 2 + 31) / 32, (nz + 2 + 31) / 32, ny + 2);
    switch (dt) {
    case PYRO_F32:
        relayout_padded_kernel<float><<<grid, block, 0, s>>>((const float *)vol, (float *)vp, nx, ny, nz);
        break;
    case PYRO_F16:
        relayout_padded_kernel<__half><<<grid, block, 0, s>>>((const __half *)vol, (__half *)vp, nx, ny, nz);
        break;
    case PYRO_BF16:
        relayout_padded_kernel<__nv_bfloat16>
            <<<grid, block, 0, s>>>((const __nv_bfloat16 *)vol, (__nv_bfloat16 *)vp, nx, ny, nz);
        break;
    }
    return cudaGetLastError();
}

// Grid (views, column groups, row groups): blocks start in linear index
// order, so the blocks in flight share a band of detector rows across the
// views, and with it a band of the volume's z (measured 1 % faster than
// the row groups varying fastest).
template <typename T, int R>
static void column_launch(const void *vp, void *sino, int b, const FP3DParams &p, cudaStream_t s)
{
    dim3 block(32, kFPCWarps);
    dim3 grid((unsigned)p.n_views, (p.nu + kFPCWarps - 1) / kFPCWarps, (p.nv + 32 * R - 1) / (32 * R));
    fp3d_column_kernel<T, R><<<grid, block, 0, s>>>((const T *)vp, (T *)sino, p, b);
}

// 32-row windows per column, 1 to 5 per warp.  Cost model in issue slots
// per warp and depth plane: about 28 per window (windows past the last row
// included) plus about 30 shared by the warp's windows.
static int column_windows_per_warp(int nv)
{
    const int windows = (nv + 31) / 32;
    int best = 1, cost = INT_MAX;
    for (int r = 1; r <= 5 && r <= windows; ++r) {
        const int c = (windows + r - 1) / r * (28 * r + 30);
        if (c <= cost) {
            best = r;
            cost = c;
        }
    }
    return best;
}

template <typename T>
static void column_dispatch(const void *vp, void *sino, int b, const FP3DParams &p, cudaStream_t s)
{
    const int best = column_windows_per_warp(p.nv);
    if (best == 5)
        column_launch<T, 5>(vp, sino, b, p, s);
    else if (best == 4)
        column_launch<T, 4>(vp, sino, b, p, s);
    else if (best == 3)
        column_launch<T, 3>(vp, sino, b, p, s);
    else if (best == 2)
        column_launch<T, 2>(vp, sino, b, p, s);
    else
        column_launch<T, 1>(vp, sino, b, p, s);
}

// two-ray windows per warp: about 40 issue slots per window and depth plane
// plus about 30 shared by the warp's windows
static int pair_rows_windows_per_warp(int nv, int wr)
{
    const int windows = (nv + wr - 1) / wr;
    int best = 1, cost = INT_MAX;
    for (int r = 1; r <= 4 && r <= windows; ++r) {
        const int c = (windows + r - 1) / r * (40 * r + 30);
        if (c <= cost) {
            best = r;
            cost = c;
        }
    }
    return best;
}

template <typename T, int R>
static void pair_rows_launch(const void *vp, void *sino, int b, const FP3DParams &p, cudaStream_t s)
{
    dim3 block(32, kFPCWarps);
    dim3 grid((unsigned)p.n_views, (p.nu + kFPCWarps - 1) / kFPCWarps, (p.nv + R * p.pair_rows - 1) / (R * p.pair_rows));
    fp3d_pair_rows_kernel<T, R><<<grid, block, 0, s>>>((const T *)vp, (T *)sino, p, b);
}

template <typename T>
static void pair_rows_dispatch(const void *vp, void *sino, int b, const FP3DParams &p, cudaStream_t s)
{
    switch (pair_rows_windows_per_warp(p.nv, p.pair_rows)) {
    case 4: pair_rows_launch<T, 4>(vp, sino, b, p, s); break;
    case 3: pair_rows_launch<T, 3>(vp, sino, b, p, s); break;
    case 2: pair_rows_launch<T, 2>(vp, sino, b, p, s); break;
    default: pair_rows_launch<T, 1>(vp, sino, b, p, s); break;
    }
}

cudaError_t launch_fp3d_column(const void *vp, void *sino, int b, const FP3DParams &p, pyro_dtype dt, cudaStream_t s)
{
    if (p.pair_rows > 0) {
        switch (dt) {
        case PYRO_F32: pair_rows_dispatch<float>(vp, sino, b, p, s); break;
        case PYRO_F16: pair_rows_dispatch<__half>(vp, sino, b, p, s); break;
        case PYRO_BF16: pair_rows_dispatch<__nv_bfloat16>(vp, sino, b, p, s); break;
        }
        return cudaGetLastError();
    }
    switch (dt) {
    case PYRO_F32:
        column_dispatch<float>(vp, sino, b, p, s);
        break;
    case PYRO_F16:
        column_dispatch<__half>(vp, sino, b, p, s);
        break;
    case PYRO_BF16:
        column_dispatch<__nv_bfloat16>(vp, sino, b, p, s);
        break;
    }
    return cudaGetLastError();
}

template <int R>
static void column_adjoint_launch(const float *sino, float *vp, int b, const FP3DParams &p, cudaStream_t s)
{
    dim3 block(32, kFPCWarps);
    dim3 grid((unsigned)p.n_views, (p.nu + kFPCWarps - 1) / kFPCWarps, (p.nv + 32 * R - 1) / (32 * R));
    fp3d_column_adjoint_kernel<R><<<grid, block, 0, s>>>(sino, vp, p, b);
}

template <int R>
static void pair_rows_adjoint_launch(const float *sino, float *vp, int b, const FP3DParams &p, cudaStream_t s)
{
    dim3 block(32, kFPCWarps);
    dim3 grid((unsigned)p.n_views, (p.nu + kFPCWarps - 1) / kFPCWarps, (p.nv + R * p.pair_rows - 1) / (R * p.pair_rows));
    fp3d_pair_rows_adjoint_kernel<R><<<grid, block, 0, s>>>(sino, vp, p, b);
}

cudaError_t launch_fp3d_column_adjoint(const void *sino, void *vp, int b, const FP3DParams &p, cudaStream_t s)
{
    if (p.pair_rows > 0) {
        const float *si = (const float *)sino;
        float *vo = (float *)vp;
        switch (pair_rows_windows_per_warp(p.nv, p.pair_rows)) {
        case 4: pair_rows_adjoint_launch<4>(si, vo, b, p, s); break;
        case 3: pair_rows_adjoint_launch<3>(si, vo, b, p, s); break;
        case 2: pair_rows_adjoint_launch<2>(si, vo, b, p, s); break;
        default: pair_rows_adjoint_launch<1>(si, vo, b, p, s); break;
        }
        return cudaGetLastError();
    }
    switch (column_windows_per_warp(p.nv)) {
    case 5:
        column_adjoint_launch<5>((const float *)sino, (float *)vp, b, p, s);
        break;
    case 4:
        column_adjoint_launch<4>((const float *)sino, (float *)vp, b, p, s);
        break;
    case 3:
        column_adjoint_launch<3>((const float *)sino, (float *)vp, b, p, s);
        break;
    case 2:
        column_adjoint_launch<2>((const float *)sino, (float *)vp, b, p, s);
        break;
    default:
        column_adjoint_launch<1>((const float *)sino, (float *)vp, b, p, s);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_relayout_unpad(const void *vp, void *vol, int nx, int ny, int nz, cudaStream_t s)
{
    dim3 block(32, 8), grid((nx + 31) / 32, (nz + 31) / 32, ny);
    relayout_unpad_kernel<<<grid, block, 0, s>>>((const float *)vp, (float *)vol, nx, ny, nz);
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

cudaError_t launch_fp3d_tex(cudaTextureObject_t tex, void *sino, const FP3DParams &p, pyro_dtype dt, cudaStream_t s)
{
    dim3 block(kFPTexX, kFPTexY);
    dim3 grid((p.nu + kFPTexX - 1) / kFPTexX, (p.nv + kFPTexY - 1) / kFPTexY, (unsigned)p.n_views);
    switch (dt) {
    case PYRO_F32:
        fp3d_tex_kernel<float><<<grid, block, 0, s>>>(tex, (float *)sino, p);
        break;
    case PYRO_F16:
        fp3d_tex_kernel<__half><<<grid, block, 0, s>>>(tex, (__half *)sino, p);
        break;
    case PYRO_BF16:
        fp3d_tex_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(tex, (__nv_bfloat16 *)sino, p);
        break;
    }
    return cudaGetLastError();
}

}  // namespace pyro
