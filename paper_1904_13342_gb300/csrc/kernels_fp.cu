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
//
// Sample positions.  A sample's voxel-index coordinate is p + m q per axis;
// written as one FP32 number it carries half an ulp of its size (~3e-5 voxel
// near index 500), which noise data turns into ~2e-5 relative error.  So p
// and q are evaluated in float-float arithmetic from the host's FP64 set-up
// (passed as hi/lo pairs), and every kFPSegment samples the position is
// re-anchored: an integer cell plus an FP32 fraction per axis (a Seg); the
// samples of the segment step in FP32 from the fraction, so their
// coordinates stay within ~1e-6 voxel of the exact ones.
#include "device_common.cuh"
#include "internal.h"

namespace pyro {

namespace {

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_neg(ff a)
{
    return {-a.h, -a.l};
}

// one axis of a ray's samples near segment start ms: the coordinate of
// sample m is i + f + (m - ms) q, i an integer, f in [0, 1)
struct Seg {
    int i;
    float f, q;
};

__device__ __forceinline__ Seg seg_at(ff p, ff q, int ms)
{
    Seg s;
    ff_split(ff_add(p, ff_mul_f(q, (float)ms)), 0.0f, s.i, s.f);
    s.q = q.h;
    return s;
}

// cell and fraction of sample ms + dm on one axis
struct Tap {
    int i;
    float a;
};

__device__ __forceinline__ Tap seg_tap(const Seg &s, float dm)
{
    const float x = fmaf(dm, s.q, s.f);
    const float t = floor_magic(x);
    return {s.i + magic_to_int(t), x - magic_to_float(t)};
}

// zero-extended linear interpolation weights of a tap on an axis of n cells:
// taps i (weight 1 - a) and i + 1 (weight a), a weight zeroed outside, the
// indices clamped for addressing
__device__ __forceinline__ Axis tap_axis(Tap t, int n)
{
    Axis r;
    r.w0 = ((unsigned)t.i < (unsigned)n) ? 1.0f - t.a : 0.0f;
    r.w1 = ((unsigned)(t.i + 1) < (unsigned)n) ? t.a : 0.0f;
    r.i0 = min(max(t.i, 0), n - 1);
    r.i1 = min(max(t.i + 1, 0), n - 1);
    return r;
}

// ---- 2D rays: sample m at p + m q in pixel-index units (float-float) ----
struct Ray2 {
    ff px, py, qx, qy;
    float w;  // dt |g|
};

__device__ __forceinline__ Ray2 ray2d(const FP2DParams &p, int v, int k)
{
    const FP2DLine &H = p.ln[v], &L = p.lnlo[v];
    const float fk = (float)k;
    Ray2 r;
    r.px = ff_add({H.p0x, L.p0x}, ff_mul_f({H.pkx, L.pkx}, fk));
    r.py = ff_add({H.p0y, L.p0y}, ff_mul_f({H.pky, L.pky}, fk));
    r.qx = ff_add({H.q0x, L.q0x}, ff_mul_f({H.qkx, L.qkx}, fk));
    r.qy = ff_add({H.q0y, L.q0y}, ff_mul_f({H.qky, L.qky}, fk));
    if (p.fan) {
        const float t = ((float)k - p.cu) * p.su / p.sdd;
        r.w = p.dt * sqrtf(fmaf(t, t, 1.0f));
    } else {
        r.w = p.dt;
    }
    return r;
}

__device__ __forceinline__ void range2d(const Ray2 &r, const FP2DParams &p, int nx, int ny, int &m0, int &m1)
{
    float lo = -(float)p.M, hi = (float)p.M;
    clip_axis(r.px.h, r.qx.h, nx, lo, hi);
    clip_axis(r.py.h, r.qy.h, ny, lo, hi);
    m0 = max(-p.M, (int)floorf(lo));
    m1 = min(p.M, (int)ceilf(hi));
}

// the views whose rays run closer to x than to y read (or scatter into) the
// transposed image: swap the roles of x and y
__device__ __forceinline__ void swap_xy(Ray2 &r)
{
    const ff t0 = r.px, t1 = r.qx;
    r.px = r.py;
    r.qx = r.qy;
    r.py = t0;
    r.qy = t1;
}

template <typename T>
__device__ __forceinline__ float bilerp_taps_zero(const T *img, int nx, int ny, Tap tx, Tap ty)
{
    const Axis ax = tap_axis(tx, nx), ay = tap_axis(ty, ny);
    const T *r0 = img + (size_t)ay.i0 * nx;
    const T *r1 = img + (size_t)ay.i1 * nx;
    const float v0 = ax.w0 * ld(r0 + ax.i0) + ax.w1 * ld(r0 + ax.i1);
    const float v1 = ax.w0 * ld(r1 + ax.i0) + ax.w1 * ld(r1 + ax.i1);
    return ay.w0 * v0 + ay.w1 * v1;
}

// all four taps inside the image (0 <= i < n - 1 on both axes)
template <typename T>
__device__ __forceinline__ float bilerp_taps_interior(const T *img, int nx, Tap tx, Tap ty)
{
    const T *b = img + (tx.i + ty.i * nx);
    return lerpf(lerpf(ld(b), ld(b + 1), tx.a), lerpf(ld(b + nx), ld(b + nx + 1), tx.a), ty.a);
}

// samples m0..m1 of a 2D ray split into a first zero-extended part, an
// interior part [i0, i1] (rounded inwards by clip_axis_interior's margin, so
// that the anchored positions of its samples are interior too) and a last
// zero-extended part
__device__ __forceinline__ void interior2d(const Ray2 &r, int nx, int ny, int m0, int m1, int &i0, int &i1)
{
    float lo = (float)m0, hi = (float)m1;
    clip_axis_interior(r.px.h, r.qx.h, nx, lo, hi);
    clip_axis_interior(r.py.h, r.qy.h, ny, lo, hi);
    i0 = max(m0, (int)ceilf(lo));
    i1 = min(m1, (int)floorf(hi));
    if (i0 > i1) {  // no interior sample
        i0 = m1 + 1;
        i1 = m1;
    }
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
    const T *img = vol + (size_t)b * p.nx * p.ny;
    int nx = p.nx, ny = p.ny;
    if (volT && fabsf(p.dir[v].x) > fabsf(p.dir[v].y)) {  // the whole block: one view
        img = volT + (size_t)b * p.nx * p.ny;
        nx = p.ny;
        ny = p.nx;
        swap_xy(r);
    }
    int m0, m1, i0, i1;
    range2d(r, p, nx, ny, m0, m1);
    interior2d(r, nx, ny, m0, m1, i0, i1);
    float acc = 0.0f, acc2 = 0.0f;
    for (int ms = m0; ms <= m1; ms += kFPSegment) {
        const int me = min(ms + kFPSegment - 1, m1);
        const Seg X = seg_at(r.px, r.qx, ms), Y = seg_at(r.py, r.qy, ms);
        for (int m = ms; m <= min(me, i0 - 1); ++m) {
            const float dm = (float)(m - ms);
            acc += bilerp_taps_zero(img, nx, ny, seg_tap(X, dm), seg_tap(Y, dm));
        }
        // two samples per iteration with separate partial sums, so that
        // several samples' loads are in flight
        int m = max(ms, i0);
        const int ie = min(me, i1);
#pragma unroll 2
        for (; m + 1 <= ie; m += 2) {
            const float da = (float)(m - ms), db = da + 1.0f;
            acc += bilerp_taps_interior(img, nx, seg_tap(X, da), seg_tap(Y, da));
            acc2 += bilerp_taps_interior(img, nx, seg_tap(X, db), seg_tap(Y, db));
        }
        if (m <= ie) {
            const float dm = (float)(m - ms);
            acc += bilerp_taps_interior(img, nx, seg_tap(X, dm), seg_tap(Y, dm));
        }
        for (m = max(ms, i1 + 1); m <= me; ++m) {
            const float dm = (float)(m - ms);
            acc += bilerp_taps_zero(img, nx, ny, seg_tap(X, dm), seg_tap(Y, dm));
        }
    }
    sino[((size_t)b * p.views_total + p.view0 + v) * p.nu + k] = to_storage<T>(r.w * (acc + acc2));
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
    float *img = vol + (size_t)b * p.nx * p.ny;
    int nx = p.nx, ny = p.ny;
    if (volT && fabsf(p.dir[v].x) > fabsf(p.dir[v].y)) {  // the whole block: one view
        img = volT + (size_t)b * p.nx * p.ny;
        nx = p.ny;
        ny = p.nx;
        swap_xy(r);
    }
    int m0, m1;
    range2d(r, p, nx, ny, m0, m1);
    for (int ms = m0; ms <= m1; ms += kFPSegment) {
        const int me = min(ms + kFPSegment - 1, m1);
        const Seg X = seg_at(r.px, r.qx, ms), Y = seg_at(r.py, r.qy, ms);
        for (int m = ms; m <= me; ++m) {
            const float dm = (float)(m - ms);
            const Axis ax = tap_axis(seg_tap(X, dm), nx);
            const Axis ay = tap_axis(seg_tap(Y, dm), ny);
            float *r0 = img + (size_t)ay.i0 * nx;
            float *r1 = img + (size_t)ay.i1 * nx;
            const float y0 = y * ay.w0, y1 = y * ay.w1;
            if (y0 * ax.w0 != 0.0f) atomicAdd(r0 + ax.i0, y0 * ax.w0);
            if (y0 * ax.w1 != 0.0f) atomicAdd(r0 + ax.i1, y0 * ax.w1);
            if (y1 * ax.w0 != 0.0f) atomicAdd(r1 + ax.i0, y1 * ax.w0);
            if (y1 * ax.w1 != 0.0f) atomicAdd(r1 + ax.i1, y1 * ax.w1);
        }
    }
}

// ---- 3D cone rays --------------------------------------------------------
// In camera coordinates the ray of pixel (k, l) is S + w q, q = K^-1 (k, l, 1)
// = (q_x, q_y, 1) (unit depth).  Its sample on the iso-centre's depth plane
// (w0 = -s3) is (s1 - s3 q_x, s2 - s3 q_y, 0): no FP32 cancellation.
struct Ray3 {
    float px, py, pz, qx, qy, qz, w;  // FP32: sample m near p + m q (voxel-index units); weight w = dt |g|
};

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

// the same ray in float-float: axis a (0, 1, 2) of the sample position p + m q
struct RayFF {
    ff p[3], q[3];
};

__device__ __forceinline__ RayFF ray3d_ff(const FP3DParams &p, int v, int k, int l, int axes = 7)
{
    const ConeFPView &H = p.v[v], &L = p.vlo[v];
    const float fk = (float)k, fl = (float)l;
    const ff qx = ff_add(ff_add({H.a2, L.a2}, ff_mul_f({H.a0, L.a0}, fk)), ff_mul_f({H.a1, L.a1}, fl));
    const ff qy = ff_add({H.b2, L.b2}, ff_mul_f({H.b0, L.b0}, fl));
    const ff s3 = {H.s3, L.s3};
    const ff c0 = ff_add({H.s1, L.s1}, ff_neg(ff_mul(s3, qx)));
    const ff c1 = ff_add({H.s2, L.s2}, ff_neg(ff_mul(s3, qy)));
    const ff dt = {p.dt, p.dt_lo};
    const float cen[3] = {p.cx, p.cy, p.cz};
    RayFF r;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!(axes & (1 << a))) continue;
        const ff w0 = {H.W[3 * a], L.W[3 * a]}, w1 = {H.W[3 * a + 1], L.W[3 * a + 1]};
        const ff w2 = {H.W[3 * a + 2], L.W[3 * a + 2]};
        r.p[a] = ff_add(ff_add(ff_mul(w0, c0), ff_mul(w1, c1)), {cen[a], 0.0f});
        r.q[a] = ff_mul(dt, ff_add(ff_add(ff_mul(w0, qx), ff_mul(w1, qy)), w2));
    }
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

// the samples of m0..m1 strictly inside the array on every axis (rounded
// inwards by clip_axis_interior's margin, far above the difference between
// these FP32 positions and the anchored ones)
__device__ __forceinline__ void interior3d(const Ray3 &r, const FP3DParams &p, int m0, int m1, int &i0, int &i1)
{
    float lo = (float)m0, hi = (float)m1;
    clip_axis_interior(r.px, r.qx, p.nx, lo, hi);
    clip_axis_interior(r.py, r.qy, p.ny, lo, hi);
    clip_axis_interior(r.pz, r.qz, p.nz, lo, hi);
    i0 = max(m0, (int)ceilf(lo));
    i1 = min(m1, (int)floorf(hi));
    if (i0 > i1) {  // no interior sample
        i0 = m1 + 1;
        i1 = m1;
    }
}

// trilinear interpolation at anchored taps of a volume with element strides
// (stx, sty, stz): zero-extended, and the unmasked interior form
template <typename T>
__device__ __forceinline__ float trilerp_taps_zero(const T *vol, const FP3DParams &p, size_t stx, size_t sty,
                                                   size_t stz, Tap tx, Tap ty, Tap tz)
{
    const Axis ax = tap_axis(tx, p.nx), ay = tap_axis(ty, p.ny), az = tap_axis(tz, p.nz);
    const T *p00 = vol + ax.i0 * stx + ay.i0 * sty;
    const T *p01 = vol + ax.i0 * stx + ay.i1 * sty;
    const T *p10 = vol + ax.i1 * stx + ay.i0 * sty;
    const T *p11 = vol + ax.i1 * stx + ay.i1 * sty;
    const size_t z0 = az.i0 * stz, z1 = az.i1 * stz;
    const float v00 = az.w0 * ld(p00 + z0) + az.w1 * ld(p00 + z1);
    const float v01 = az.w0 * ld(p01 + z0) + az.w1 * ld(p01 + z1);
    const float v10 = az.w0 * ld(p10 + z0) + az.w1 * ld(p10 + z1);
    const float v11 = az.w0 * ld(p11 + z0) + az.w1 * ld(p11 + z1);
    return ax.w0 * (ay.w0 * v00 + ay.w1 * v01) + ax.w1 * (ay.w0 * v10 + ay.w1 * v11);
}

template <typename T>
__device__ __forceinline__ float trilerp_taps_interior(const T *vol, int stx, int sty, int stz, Tap tx, Tap ty,
                                                       Tap tz)
{
    const T *b = vol + (tx.i * stx + ty.i * sty + tz.i * stz);
    const float v00 = lerpf(ld(b), ld(b + stz), tz.a);
    const float v01 = lerpf(ld(b + sty), ld(b + sty + stz), tz.a);
    const float v10 = lerpf(ld(b + stx), ld(b + stx + stz), tz.a);
    const float v11 = lerpf(ld(b + stx + sty), ld(b + stx + sty + stz), tz.a);
    return lerpf(lerpf(v00, v01, ty.a), lerpf(v10, v11, ty.a), tx.a);
}

// Sum of the samples m0..m1 of one ray through a volume with element strides
// (stx, sty, stz): segment by segment, the interior samples unmasked, the
// few near the faces zero-extended.
template <typename T>
__device__ __forceinline__ float march3d(const T *vol, const FP3DParams &p, int stx, int sty, int stz,
                                         const RayFF &rf, const Ray3 &r, int m0, int m1)
{
    int i0, i1;
    interior3d(r, p, m0, m1, i0, i1);
    float acc = 0.0f;
    for (int ms = m0; ms <= m1; ms += kFPSegment) {
        const int me = min(ms + kFPSegment - 1, m1);
        const Seg X = seg_at(rf.p[0], rf.q[0], ms), Y = seg_at(rf.p[1], rf.q[1], ms), Z = seg_at(rf.p[2], rf.q[2], ms);
        int m = ms;
        for (; m <= min(me, i0 - 1); ++m) {
            const float dm = (float)(m - ms);
            acc += trilerp_taps_zero(vol, p, (size_t)stx, (size_t)sty, (size_t)stz, seg_tap(X, dm), seg_tap(Y, dm),
                                     seg_tap(Z, dm));
        }
        for (m = max(ms, i0); m <= min(me, i1); ++m) {
            const float dm = (float)(m - ms);
            acc += trilerp_taps_interior(vol, stx, sty, stz, seg_tap(X, dm), seg_tap(Y, dm), seg_tap(Z, dm));
        }
        for (m = max(ms, i1 + 1); m <= me; ++m) {
            const float dm = (float)(m - ms);
            acc += trilerp_taps_zero(vol, p, (size_t)stx, (size_t)sty, (size_t)stz, seg_tap(X, dm), seg_tap(Y, dm),
                                     seg_tap(Z, dm));
        }
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
    float acc = 0.0f;
    if (m0 <= m1) acc = march3d(V, p, 1, p.nx, p.nx * p.ny, ray3d_ff(p, v, k, l), r, m0, m1);
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
    float acc = 0.0f;
    if (m0 <= m1) {
        const RayFF rf = ray3d_ff(p, v, k, l);
        int i0, i1;
        interior3d(r, p, m0, m1, i0, i1);
        const size_t sx = (size_t)p.nz, sy = (size_t)p.nz * p.nx;
        // interior: consecutive samples are half a voxel apart and the warp's
        // rays (consecutive detector rows) sit at one (x, y) point on every
        // depth plane, so the 8 taps of the current cell stay in registers
        // until the cell changes
        const int stx = p.nz, sty = p.nz * p.nx;
        int cur = -1;
        float c000 = 0.f, c001 = 0.f, c010 = 0.f, c011 = 0.f, c100 = 0.f, c101 = 0.f, c110 = 0.f, c111 = 0.f;
        for (int ms = m0; ms <= m1; ms += kFPSegment) {
            const int me = min(ms + kFPSegment - 1, m1);
            const Seg X = seg_at(rf.p[0], rf.q[0], ms), Y = seg_at(rf.p[1], rf.q[1], ms);
            const Seg Z = seg_at(rf.p[2], rf.q[2], ms);
            int m = ms;
            for (; m <= min(me, i0 - 1); ++m) {
                const float dm = (float)(m - ms);
                acc += trilerp_taps_zero(vz, p, sx, sy, (size_t)1, seg_tap(X, dm), seg_tap(Y, dm), seg_tap(Z, dm));
            }
            for (m = max(ms, i0); m <= min(me, i1); ++m) {
                const float dm = (float)(m - ms);
                const Tap tx = seg_tap(X, dm), ty = seg_tap(Y, dm), tz = seg_tap(Z, dm);
                const int cell = tx.i * stx + ty.i * sty + tz.i;
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
                const float v00 = lerpf(c000, c001, tz.a), v01 = lerpf(c010, c011, tz.a);
                const float v10 = lerpf(c100, c101, tz.a), v11 = lerpf(c110, c111, tz.a);
                acc += lerpf(lerpf(v00, v01, ty.a), lerpf(v10, v11, ty.a), tx.a);
            }
            for (m = max(ms, i1 + 1); m <= me; ++m) {
                const float dm = (float)(m - ms);
                acc += trilerp_taps_zero(vz, p, sx, sy, (size_t)1, seg_tap(X, dm), seg_tap(Y, dm), seg_tap(Z, dm));
            }
        }
    }
    sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k] = to_storage<T>(r.w * acc);
}

// Column-shared projection.  When the detector's v axis maps onto the
// volume's z axis (circular and helical-free trajectories: no skew, camera y
// axis = z), all rays of one detector column k share their (x, y) point on
// every depth plane; only z differs, and it grows monotonically with the row
// l.  A warp takes column k and R windows of 32 consecutive rows.  The (x, y)
// cell and bilinear weights of each depth plane are computed once per warp
// (32 planes at a time, one per lane, handed over through shared memory); in
// each window every lane loads the four (x, y) columns at one z of the
// window's 32-voxel run and combines them in x and y, and each lane then
// takes the two z taps of its own ray from the lanes holding them (two
// shuffles).  The host checks that 31 row steps stay below 29.5 voxels in z,
// so a window's taps always fall in its 32-voxel run.  The volume copy is a
// quad copy: cell (x, y, z) of [ny+4][nx+4][nz+2] holds the four columns
// (x, y), (x + 1, y), (x, y + 1), (x + 1, y + 1) at z, so one 16-byte load
// per lane (coalesced along z) brings the four taps of a plane; zero voxels
// around the data (two in x and y, one in z) mean no load needs a bounds
// test, and the zero-extended interpolant comes out of the padding.
//
// Positions: the column's (x, y) track is anchored (float-float) at the
// start of every kFPSegment planes; each ray's z once, at the middle plane of
// the warp's range, since the rays' z moves by at most a few tens of voxels
// over a whole ray (|q_z| stays near 0.1 voxel per plane for these
// trajectories), which keeps the FP32 steps from the anchor within ~2e-6
// voxel.
//
// Warps (detector columns) per block: 8 for the one-ray kernel, 16 for the
// two-ray kernel; the adjacent columns of a block follow nearby tracks, so
// larger blocks share more cells in L1 (256^3 workload: 18.15 ms with 4,
// 17.85 with 8 and the pair loop unrolled by 4; 512^3 TV geometry: 464 ms
// with 4, 454 with 8, 440 with 16)
constexpr int kFPCWarps = 8;
constexpr int kFPPWarps = 16;

struct ColumnWindow {
    float acc;  // the ray sum
    int ma, mb; // samples of the window's rows that can touch the volume
};

// the window's lowest z and the lane's z, anchored on the lowest row's
// integer cell ib at plane mz: zb = ib + fb + dz qb, z = ib + f + dz q, dz =
// m - mz (f holds the lane's offset from the lowest row, below 32)
struct ZSeg {
    float f, q;
    float fb, qb;
    int zbase;  // ib + 1 + lane - 0x4B400000: the lane's cell in the padded column minus the magic bits
};

__device__ __forceinline__ ZSeg zseg(const float4 &zr, int src, int lane, int mz)
{
    const Seg Z = seg_at({zr.x, zr.y}, {zr.z, zr.w}, mz);
    const unsigned full = 0xffffffffu;
    ZSeg s;
    const int ib = __shfl_sync(full, Z.i, src);
    s.fb = __shfl_sync(full, Z.f, src);
    s.qb = __shfl_sync(full, Z.q, src);
    s.f = Z.f + (float)(Z.i - ib);
    s.q = Z.q;
    s.zbase = ib + 1 + lane - 0x4B400000;
    return s;
}

// the track anchored at plane ms: x = X.i + X.f + dx X.q, and the index of
// the padded column (X.i, Y.i) (its cell 0 is the zero below z = 0) minus
// the magic bits of the in-segment floors (mod 2^32)
struct TrackSeg {
    float xf, xq, yf, yq;
    int col0;
};

__device__ __forceinline__ TrackSeg track_seg(const float4 *t, int ms, int sxp, int syp)
{
    const float4 a = t[0], b = t[1];  // (px, py) and (qx, qy) as hi/lo pairs
    const Seg X = seg_at({a.x, a.y}, {b.x, b.y}, ms), Y = seg_at({a.z, a.w}, {b.z, b.w}, ms);
    TrackSeg s;
    s.xf = X.f;
    s.xq = X.q;
    s.yf = Y.f;
    s.yq = Y.q;
    s.col0 = (int)((unsigned)(Y.i + kFPPadXY - 0x4B400000) * (unsigned)syp +
                   (unsigned)(X.i + kFPPadXY - 0x4B400000) * (unsigned)sxp);
    return s;
}

// (x, y) cell of a depth plane shared by the column's rays: its bilinear
// weights as the pairs (w00, w10) and (w01, w11), matching the two halves of
// a quad-copy cell, and the index of the padded column (x0, y0)
struct PlaneXY {
    f32x2 wa, wb;
    int col;
};

__device__ __forceinline__ PlaneXY plane_xy(const TrackSeg &s, float dx, int sxp, int syp)
{
    const float fx = fmaf(dx, s.xq, s.xf), fy = fmaf(dx, s.yq, s.yf);
    const float tx = floor_magic(fx), ty = floor_magic(fy);
    const float ax = fx - magic_to_float(tx), ay = fy - magic_to_float(ty);
    const float bx = 1.0f - ax, by = 1.0f - ay;
    PlaneXY q;
    q.wa = pk2(bx * by, ax * by);
    q.wb = pk2(bx * ay, ax * ay);
    q.col = (int)((unsigned)s.col0 + (unsigned)__float_as_int(ty) * (unsigned)syp +
                  (unsigned)__float_as_int(tx) * (unsigned)sxp);  // mod 2^32: the magic bits cancel
    return q;
}

// a quad-copy cell's bilinear value: (w00 v00 + w01 v01) + (w10 v10 + w11 v11)
__device__ __forceinline__ float bilerp_quad(f32x2 wa, f32x2 wb, float4 v)
{
    float a, b;
    upk2(fma2(wb, pk2(v.z, v.w), mul2(wa, pk2(v.x, v.y))), a, b);
    return a + b;
}

// the lane's cell in the padded column: run start zbase + tb (tb the magic
// floor of the lowest row's z) clamped to the column's cells 0 .. nz + 1,
// whose ends are zeros; one add-min-relu
__device__ __forceinline__ unsigned run_cell(int zbase, float tb, int nz1)
{
    return (unsigned)__viaddmin_s32_relu(zbase, __float_as_int(tb), nz1);
}

// the four (x, y) columns of a cell at one z from the quad copy: (x, y),
// (x + 1, y), (x, y + 1), (x + 1, y + 1), one 16-byte (FP32) or 8-byte load
template <typename T>
__device__ __forceinline__ float4 ldq(const T *p);
template <>
__device__ __forceinline__ float4 ldq<float>(const float *p)
{
    return __ldg(reinterpret_cast<const float4 *>(p));
}
template <>
__device__ __forceinline__ float4 ldq<__half>(const __half *p)
{
    const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ float4 ldq<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// One depth plane of one window: the lane's x/y-interpolated value at
// z = zb + lane, then its own ray's z interpolation from two lanes.
template <typename T>
__device__ __forceinline__ void column_step(ColumnWindow &W, const ZSeg &z, float dz, int nz1, const T *cq,
                                            const PlaneXY &q)
{
    const float tzb = floor_magic(fmaf(dz, z.qb, z.fb));
    const float g = bilerp_quad(q.wa, q.wb, ldq(cq + 4 * run_cell(z.zbase, tzb, nz1)));
    const float fz = fmaf(dz, z.q, z.f);
    const float tz = floor_magic(fz);
    const int j = __float_as_int(tz) - __float_as_int(tzb);  // own cell relative to the window's run
    const float g0 = __shfl_sync(0xffffffffu, g, j), g1 = __shfl_sync(0xffffffffu, g, j + 1);
    W.acc += fmaf(fz - magic_to_float(tz), g1 - g0, g0);
}

// Two consecutive depth planes: each plane's weights as in plane_xy, the
// columns' pointers, and whether both planes lie in the same (x, y) cell.
template <typename T>
struct PlanePair {
    f32x2 wa0, wb0, wa1, wb1;
    const T *c0, *c1;
    bool same;
};

// One window on two consecutive planes: as column_step for each plane, the
// z arithmetic in f32x2 pairs (plane m in the low half, m + 1 in the high).
// When both planes read the same cells (same (x, y) cell and run start,
// about half the pairs) the second load is skipped: the kernel is bound by
// the L1 data pipe (256^3 workload: 16.83 -> 16.61 ms).
template <typename T>
__device__ __forceinline__ void column_step_pair(f32x2 &acc, const ZSeg &z, float dz, int nz1, const PlanePair<T> &q)
{
    const f32x2 MAGIC = pk2(kFloorMagic, kFloorMagic);
    const f32x2 D = pk2(dz, dz + 1.0f);
    const f32x2 TB = add2_rm(fma2(D, pk2(z.qb, z.qb), pk2(z.fb, z.fb)), MAGIC);
    float tb0, tb1;
    upk2(TB, tb0, tb1);
    const float4 v0 = ldq(q.c0 + 4 * run_cell(z.zbase, tb0, nz1));
    float4 v1 = v0;
    if (!q.same || tb1 != tb0) v1 = ldq(q.c1 + 4 * run_cell(z.zbase, tb1, nz1));  // whole warp
    const float g0 = bilerp_quad(q.wa0, q.wb0, v0), g1 = bilerp_quad(q.wa1, q.wb1, v1);
    const f32x2 FZ = fma2(D, pk2(z.q, z.q), pk2(z.f, z.f));
    const f32x2 TZ = add2_rm(FZ, MAGIC);
    float tz0, tz1;
    upk2(TZ, tz0, tz1);
    const int j0 = __float_as_int(tz0) - __float_as_int(tb0), j1 = __float_as_int(tz1) - __float_as_int(tb1);
    const unsigned full = 0xffffffffu;
    const f32x2 G0 = pk2(__shfl_sync(full, g0, j0), __shfl_sync(full, g1, j1));
    const f32x2 G1 = pk2(__shfl_sync(full, g0, j0 + 1), __shfl_sync(full, g1, j1 + 1));
    acc = add2(acc, fma2(sub2(FZ, sub2(TZ, MAGIC)), sub2(G1, G0), G0));
}

// planes mb .. mb + 31 of the segment anchored at ms: lane i computes plane
// mb + i and stores its weights and column for the whole warp
__device__ __forceinline__ void plane_batch(const TrackSeg &ts, int mb, int ms, int lane, int sxp, int syp, float4 *pw,
                                            int *pc)
{
    const PlaneXY q = plane_xy(ts, (float)(mb - ms + lane), sxp, syp);  // lanes past the segment: unused
    float a0, a1, b0, b1;
    upk2(q.wa, a0, a1);
    upk2(q.wb, b0, b1);
    __syncwarp();  // the previous batch is no longer read
    pw[lane] = make_float4(a0, a1, b0, b1);
    pc[lane] = q.col;
    __syncwarp();
}

__device__ __forceinline__ PlaneXY plane_from_batch(const float4 *pw, const int *pc, int i)
{
    const float4 w = pw[i];
    PlaneXY q;
    q.wa = pk2(w.x, w.y);
    q.wb = pk2(w.z, w.w);
    q.col = pc[i];
    return q;
}

// the main phase of the forward: every window active, planes in pairs.
// The (x, y) cell and weights of 32 planes at a time are computed one plane
// per lane and handed to the warp through shared memory (pw, pc: 32 entries
// of the warp's own), so that each plane's set-up costs a lane 1/32 of its
// arithmetic plus two broadcast loads; the values are those of plane_xy.
template <typename T, int R>
__device__ __forceinline__ void column_planes_paired(ColumnWindow (&W)[R], const ZSeg (&zs)[R], const float4 *track,
                                                     int mz, int m0, int m1, const T *vp, const FP3DParams &p,
                                                     int sxp, int syp, float4 *pw, int *pc, int lane)
{
    f32x2 acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = pk2(0.0f, 0.0f);
    for (int ms = m0; ms <= m1; ms += kFPSegment) {
        const int me = min(ms + kFPSegment - 1, m1);
        const TrackSeg ts = track_seg(track, ms, sxp, syp);
        for (int mb = ms; mb <= me; mb += 32) {
            const int n = min(32, me - mb + 1);
            plane_batch(ts, mb, ms, lane, sxp, syp, pw, pc);
            float dz = (float)(mb - mz);
            int i = 0;
#pragma unroll 4
            for (; i + 1 < n; i += 2, dz += 2.0f) {
                const float4 w0 = pw[i], w1 = pw[i + 1];
                const int2 c = *reinterpret_cast<const int2 *>(pc + i);  // i even: 8-byte aligned
                PlanePair<T> q;
                q.wa0 = pk2(w0.x, w0.y);
                q.wb0 = pk2(w0.z, w0.w);
                q.wa1 = pk2(w1.x, w1.y);
                q.wb1 = pk2(w1.z, w1.w);
                q.c0 = vp + 4 * (size_t)c.x;
                q.c1 = vp + 4 * (size_t)c.y;
                q.same = c.x == c.y;
#pragma unroll
                for (int r = 0; r < R; ++r) column_step_pair(acc[r], zs[r], dz, p.nz + 1, q);
            }
            if (i < n) {  // an odd plane left in the segment
                const PlaneXY q = plane_from_batch(pw, pc, i);
                const T *cq = vp + 4 * (size_t)q.col;
#pragma unroll
                for (int r = 0; r < R; ++r) column_step(W[r], zs[r], dz, p.nz + 1, cq, q);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float a0, a1;
        upk2(acc[r], a0, a1);
        W[r].acc += a0 + a1;
    }
}

// Depth planes m0..m1 of all R windows, the track re-anchored every
// kFPSegment planes and the planes' set-up shared through 32-plane batches.
// Skips the windows whose rows cannot touch the volume on a plane (the
// planes outside those every window reaches; elsewhere the skipped terms
// would be exact zeros anyway: the taps read the zero padding).
template <typename T, int R>
__device__ __forceinline__ void column_planes(ColumnWindow (&W)[R], const ZSeg (&zs)[R], const float4 *track, int mz,
                                              int m0, int m1, const T *vp, const FP3DParams &p, int sxp, int syp,
                                              float4 *pw, int *pc, int lane)
{
    for (int ms = m0; ms <= m1; ms += kFPSegment) {
        const int me = min(ms + kFPSegment - 1, m1);
        const TrackSeg ts = track_seg(track, ms, sxp, syp);
        for (int mb = ms; mb <= me; mb += 32) {
            const int n = min(32, me - mb + 1);
            plane_batch(ts, mb, ms, lane, sxp, syp, pw, pc);
            float dz = (float)(mb - mz);
#pragma unroll 4
            for (int i = 0; i < n; ++i, dz += 1.0f) {
                const int m = mb + i;
                const PlaneXY q = plane_from_batch(pw, pc, i);
                const T *cq = vp + 4 * (size_t)q.col;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (m < W[r].ma || m > W[r].mb) continue;  // whole warp
                    column_step(W[r], zs[r], dz, p.nz + 1, cq, q);
                }
            }
        }
    }
}

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

// the planes whose (x, y) cell lies in [-1, n-1]^2 by the FP32 track (an
// anchored cell may differ by one; the second padding voxel covers it)
__device__ __forceinline__ void track_range(const FP3DParams &p, const Ray3 &rc, int &m0, int &m1)
{
    float lo = -(float)p.M, hi = (float)p.M;
    clip_axis(rc.px, rc.qx, p.nx, lo, hi);
    clip_axis(rc.py, rc.qy, p.ny, lo, hi);
    m0 = max(-p.M, (int)floorf(lo));
    m1 = min(p.M, (int)ceilf(hi));
    // the clip above is rounded outwards by at most one sample
    auto inside = [&](int m) {
        const float fx = fmaf((float)m, rc.qx, rc.px), fy = fmaf((float)m, rc.qy, rc.py);
        return fx >= -1.0f && fx < (float)p.nx && fy >= -1.0f && fy < (float)p.ny;
    };
    while (m0 <= m1 && !inside(m0)) ++m0;
    while (m1 >= m0 && !inside(m1)) --m1;
}

// the column's track (float-float, uniform over the warp) into `track`
__device__ __forceinline__ void store_track(const FP3DParams &p, int v, int k, int row0, int lane, float4 *track)
{
    if (lane == 0) {
        const RayFF tf = ray3d_ff(p, v, k, row0, 3);
        track[0] = make_float4(tf.p[0].h, tf.p[0].l, tf.p[1].h, tf.p[1].l);
        track[1] = make_float4(tf.q[0].h, tf.q[0].l, tf.q[1].h, tf.q[1].l);
    }
}

// Set-up of the column kernel: the column's (x, y) track (float-float, into
// `track`), the windows' rays and ranges (each lane's z in float-float into
// `zray`); returns the union [mlo, mhi] of the windows' ranges and the
// planes [clo, chi] every window reaches.  last_low: bit r set when window
// r's lowest row is its last (lane 31).  zlo, zhi: the open z interval whose
// samples matter (the volume's (-1, nz)).
template <int R>
__device__ __forceinline__ void column_setup(const FP3DParams &p, int v, int k, int row0, int lane, float4 *track,
                                             ColumnWindow (&W)[R], float4 *zray, int &last_low, int &mlo, int &mhi,
                                             int &clo, int &chi, float zlo, float zhi)
{
    const unsigned full = 0xffffffffu;
    last_low = 0;
    store_track(p, v, k, row0, lane, track);
    int m0, m1;
    track_range(p, ray3d(p, v, k, row0), m0, m1);
    mlo = INT_MAX;
    mhi = INT_MIN;
    clo = INT_MIN;
    chi = INT_MAX;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int l = row0 + 32 * r + lane;
        const Ray3 rr = ray3d(p, v, k, l);
        const RayFF zf = ray3d_ff(p, v, k, l, 4);
        zray[32 * r + lane] = make_float4(zf.p[2].h, zf.p[2].l, zf.q[2].h, zf.q[2].l);
        W[r].acc = 0.0f;
        // the window's lowest z is at its first or its last row (depth > 0)
        const float z_first = __shfl_sync(full, rr.pz, 0), z_last = __shfl_sync(full, rr.pz, 31);
        if (z_last < z_first) last_low |= 1 << r;
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
    __syncwarp();
}

// all planes mlo..mhi: the rays' z anchored at the middle plane, then the
// planes split by window coverage ([clo, chi] without window checks, in
// plane pairs)
template <typename T, int R>
__device__ __forceinline__ void column_march(ColumnWindow (&W)[R], const float4 *track, const float4 *zray,
                                             int last_low, int mlo, int mhi, int clo, int chi, int lane, const T *vp,
                                             const FP3DParams &p, float4 *pw, int *pc)
{
    const int sxp = p.nz + 2, syp = (p.nx + 2 * kFPPadXY) * (p.nz + 2);
    const int mz = mlo + (mhi - mlo) / 2;
    ZSeg zs[R];
#pragma unroll
    for (int r = 0; r < R; ++r) zs[r] = zseg(zray[32 * r + lane], (last_low >> r & 1) ? 31 : 0, lane, mz);
    column_planes<T, R>(W, zs, track, mz, mlo, clo - 1, vp, p, sxp, syp, pw, pc, lane);
    column_planes_paired<T, R>(W, zs, track, mz, clo, chi, vp, p, sxp, syp, pw, pc, lane);
    column_planes<T, R>(W, zs, track, mz, max(chi + 1, clo), mhi, vp, p, sxp, syp, pw, pc, lane);
}

template <typename T, typename TO, int R>
__global__ void __launch_bounds__(32 * kFPCWarps, 4) fp3d_column_kernel(const T *__restrict__ vp,
                                                                     TO *__restrict__ sino,
                                                                     const __grid_constant__ FP3DParams p, int b)
{
    __shared__ float4 zrays[kFPCWarps][R * 32];
    __shared__ float4 tracks[kFPCWarps][2];
    __shared__ float4 pws[kFPCWarps][32];
    __shared__ int pcs[kFPCWarps][32];
    const int lane = threadIdx.x;
    const int k = blockIdx.y * kFPCWarps + threadIdx.y;
    const int v = blockIdx.x;
    if (k >= p.nu) return;  // whole warp
    const int row0 = blockIdx.z * (32 * R);
    ColumnWindow W[R];
    int last_low, mlo, mhi, clo, chi;
    column_setup<R>(p, v, k, row0, lane, tracks[threadIdx.y], W, zrays[threadIdx.y], last_low, mlo, mhi, clo, chi,
                    -1.0f, (float)p.nz);
    if (mlo <= mhi)
        column_march<T, R>(W, tracks[threadIdx.y], zrays[threadIdx.y], last_low, mlo, mhi, clo, chi, lane, vp, p,
                           pws[threadIdx.y], pcs[threadIdx.y]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int l = row0 + 32 * r + lane;
        if (l < p.nv)
            sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k] =
                to_storage<TO>(ray3d(p, v, k, l).w * W[r].acc);
    }
}

// ---- two rays per lane: windows of up to 64 rows on one 32-voxel run -----
// When a row step moves a ray by less than about 0.76 voxel in z, 32 rows
// use only part of their window's 32-voxel run.  These kernels give each
// lane two rays, rows row0 + lane and row0 + 32 + lane of a window of WR
// rows (WR = pair_rows <= 64, chosen on the host so that WR - 1 row steps
// stay below 29.5 voxels; the lanes past WR - 32 have no second ray), and
// both rays take their taps from the same run: one set of loads and x/y
// combinations for up to twice the rays.  The arithmetic and the anchoring
// of every ray are those of fp3d_column_kernel.
struct PairRowsWindow {
    float acc[2];  // the rays' sums
    int ma, mb;    // samples of the window's rows that can touch the volume
};

// as ZSeg, for the lane's two rays
struct ZSeg2 {
    float f[2], q[2];
    float fb, qb;
    int zbase;
};

// src, src_h: the lane and the ray (0: first, 1: second) of the window's lowest row
__device__ __forceinline__ ZSeg2 zseg2(const float4 &z0, const float4 &z1, int src, int src_h, int lane, int mz)
{
    const Seg A = seg_at({z0.x, z0.y}, {z0.z, z0.w}, mz), B = seg_at({z1.x, z1.y}, {z1.z, z1.w}, mz);
    const unsigned full = 0xffffffffu;
    const int ib = __shfl_sync(full, src_h ? B.i : A.i, src);
    ZSeg2 s;
    s.fb = __shfl_sync(full, src_h ? B.f : A.f, src);
    s.qb = __shfl_sync(full, src_h ? B.q : A.q, src);
    s.f[0] = A.f + (float)(A.i - ib);
    s.q[0] = A.q;
    s.f[1] = B.f + (float)(B.i - ib);
    s.q[1] = B.q;
    s.zbase = ib + 1 + lane - 0x4B400000;
    return s;
}

// last_low: bit r set when window r's lowest row is its last (lane WR - 33's second ray)
template <int R>
__device__ __forceinline__ void pair_rows_setup(const FP3DParams &p, int v, int k, int row0, int lane, float4 *track,
                                                PairRowsWindow (&W)[R], float4 *zray, int &last_low, int &mlo,
                                                int &mhi, int &clo, int &chi, float zlo, float zhi)
{
    const unsigned full = 0xffffffffu;
    const int WR = p.pair_rows;
    last_low = 0;
    store_track(p, v, k, row0, lane, track);
    int m0, m1;
    track_range(p, ray3d(p, v, k, row0), m0, m1);
    mlo = INT_MAX;
    mhi = INT_MIN;
    clo = INT_MIN;
    chi = INT_MAX;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int a = INT_MAX, e = INT_MIN;
        float pz[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = row0 + r * WR + 32 * h + lane;
            const Ray3 rr = ray3d(p, v, k, l);
            const RayFF zf = ray3d_ff(p, v, k, l, 4);
            zray[(2 * r + h) * 32 + lane] = make_float4(zf.p[2].h, zf.p[2].l, zf.q[2].h, zf.q[2].l);
            pz[h] = rr.pz;
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
        const float zf0 = __shfl_sync(full, pz[0], 0), zl1 = __shfl_sync(full, pz[1], WR - 33);
        if (zl1 < zf0) last_low |= 1 << r;
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
    __syncwarp();
}

// one depth plane of one window: the run as in column_step, then both rays'
// z interpolations from it
template <typename T>
__device__ __forceinline__ void pair_rows_step(PairRowsWindow &W, const ZSeg2 &z, float dz, int nz1, const T *cq,
                                               const PlaneXY &q)
{
    const float tzb = floor_magic(fmaf(dz, z.qb, z.fb));
    const float g = bilerp_quad(q.wa, q.wb, ldq(cq + 4 * run_cell(z.zbase, tzb, nz1)));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float fz = fmaf(dz, z.q[h], z.f[h]);
        const float tz = floor_magic(fz);
        const int j = __float_as_int(tz) - __float_as_int(tzb);
        const float g0 = __shfl_sync(0xffffffffu, g, j), g1 = __shfl_sync(0xffffffffu, g, j + 1);
        W.acc[h] += fmaf(fz - magic_to_float(tz), g1 - g0, g0);
    }
}

// planes m0..m1 with the planes' set-up shared through 32-plane batches, as
// in column_planes; CHECK skips the windows whose rows cannot touch the
// volume on a plane (outside the planes every window reaches)
template <typename T, int R, bool CHECK>
__device__ __forceinline__ void pair_rows_planes(PairRowsWindow (&W)[R], const ZSeg2 (&zs)[R],
                                                         const float4 *track, int mz, int m0, int m1, const T *vp,
                                                         const FP3DParams &p, int sxp, int syp, float4 *pw, int *pc,
                                                         int lane)
{
    for (int ms = m0; ms <= m1; ms += kFPSegment) {
        const int me = min(ms + kFPSegment - 1, m1);
        const TrackSeg ts = track_seg(track, ms, sxp, syp);
        for (int mb = ms; mb <= me; mb += 32) {
            const int n = min(32, me - mb + 1);
            plane_batch(ts, mb, ms, lane, sxp, syp, pw, pc);
            float dz = (float)(mb - mz);
#pragma unroll 4
            for (int i = 0; i < n; ++i, dz += 1.0f) {
                const int m = mb + i;
                const PlaneXY q = plane_from_batch(pw, pc, i);
                const T *cq = vp + 4 * (size_t)q.col;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (CHECK && (m < W[r].ma || m > W[r].mb)) continue;  // whole warp
                    pair_rows_step(W[r], zs[r], dz, p.nz + 1, cq, q);
                }
            }
        }
    }
}

template <typename T, int R>
__device__ __forceinline__ void pair_rows_march(PairRowsWindow (&W)[R], const float4 *track, const float4 *zray,
                                                int last_low, int mlo, int mhi, int clo, int chi, int lane, const T *vp,
                                                const FP3DParams &p, float4 *pw, int *pc)
{
    const int sxp = p.nz + 2, syp = (p.nx + 2 * kFPPadXY) * (p.nz + 2);
    const int mz = mlo + (mhi - mlo) / 2;
    ZSeg2 zs[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool hi = last_low >> r & 1;
        zs[r] = zseg2(zray[(2 * r) * 32 + lane], zray[(2 * r + 1) * 32 + lane], hi ? p.pair_rows - 33 : 0, hi, lane, mz);
    }
    pair_rows_planes<T, R, true>(W, zs, track, mz, mlo, clo - 1, vp, p, sxp, syp, pw, pc, lane);
    pair_rows_planes<T, R, false>(W, zs, track, mz, clo, chi, vp, p, sxp, syp, pw, pc, lane);
    pair_rows_planes<T, R, true>(W, zs, track, mz, max(chi + 1, clo), mhi, vp, p, sxp, syp, pw, pc, lane);
}

template <typename T, typename TO, int R>
__global__ void __launch_bounds__(32 * kFPPWarps) fp3d_pair_rows_kernel(const T *__restrict__ vp,
                                                                        TO *__restrict__ sino,
                                                                        const __grid_constant__ FP3DParams p, int b)
{
    __shared__ float4 zrays[kFPPWarps][2 * R * 32];
    __shared__ float4 tracks[kFPPWarps][2];
    __shared__ float4 pws[kFPPWarps][32];
    __shared__ int pcs[kFPPWarps][32];
    const int lane = threadIdx.x;
    const int k = blockIdx.y * kFPPWarps + threadIdx.y;
    const int v = blockIdx.x;
    if (k >= p.nu) return;  // whole warp
    const int WR = p.pair_rows;
    const int row0 = blockIdx.z * (R * WR);
    PairRowsWindow W[R];
    int last_low, mlo, mhi, clo, chi;
    pair_rows_setup<R>(p, v, k, row0, lane, tracks[threadIdx.y], W, zrays[threadIdx.y], last_low, mlo, mhi, clo, chi,
                       -1.0f, (float)p.nz);
    if (mlo <= mhi)
        pair_rows_march<T, R>(W, tracks[threadIdx.y], zrays[threadIdx.y], last_low, mlo, mhi, clo, chi, lane, vp, p,
                              pws[threadIdx.y], pcs[threadIdx.y]);
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = row0 + r * WR + 32 * h + lane;
            if (l < p.nv && 32 * h + lane < WR)
                sino[(((size_t)b * p.views_total + p.view0 + v) * p.nv + l) * p.nu + k] =
                    to_storage<TO>(ray3d(p, v, k, l).w * W[r].acc[h]);
        }
}

// [z][y][x] -> the quad copy: cell (x + P, y + P, z + 1) of the zero-padded
// (ny + 2P)(nx + 2P)(nz + 2) array (P = kFPPadXY) holds the voxels (x, y),
// (x + 1, y), (x, y + 1), (x + 1, y + 1) at z, zero outside the volume; every
// cell is written once, converted from the volume's type TI to the copy's T.
// A block stages two y rows of a 32 (z) x 33 (x) tile in shared memory
// (loads coalesced along x) and writes 32 x 32 cells (coalesced along z).
template <typename T>
__device__ __forceinline__ void store_quad(T *p, float a, float b, float c, float d);
template <>
__device__ __forceinline__ void store_quad<float>(float *p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
template <>
__device__ __forceinline__ void store_quad<__half>(__half *p, float a, float b, float c, float d)
{
    const __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
    *reinterpret_cast<uint2 *>(p) =
        make_uint2(*reinterpret_cast<const unsigned *>(&lo), *reinterpret_cast<const unsigned *>(&hi));
}
template <>
__device__ __forceinline__ void store_quad<__nv_bfloat16>(__nv_bfloat16 *p, float a, float b, float c, float d)
{
    const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    *reinterpret_cast<uint2 *>(p) =
        make_uint2(*reinterpret_cast<const unsigned *>(&lo), *reinterpret_cast<const unsigned *>(&hi));
}

template <typename TI, typename T>
__global__ void __launch_bounds__(256) relayout_quad_kernel(const TI *__restrict__ vol, T *__restrict__ vq, int nx,
                                                            int ny, int nz)
{
    __shared__ float tile[2][32][33];  // [y, y + 1][z][x .. x + 32]
    const int nxp = nx + 2 * kFPPadXY, nzp = nz + 2;
    const int x0 = blockIdx.x * 32, z0 = blockIdx.y * 32, yp = blockIdx.z;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int y = yp - kFPPadXY + r;
        for (int i = threadIdx.y; i < 32; i += 8) {
            const int z = z0 + i - 1;
            for (int j = threadIdx.x; j < 33; j += 32) {
                const int x = x0 + j - kFPPadXY;
                const bool in = y >= 0 && y < ny && z >= 0 && z < nz && x >= 0 && x < nx;
                // the copy's rounding happens once, on the stored values
                tile[r][i][j] = in ? to_float<T>(to_storage<T>(to_float<TI>(vol[((size_t)z * ny + y) * nx + x])))
                                   : 0.0f;
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int xp = x0 + i, zp = z0 + threadIdx.x;
        if (zp < nzp && xp < nxp)
            store_quad<T>(vq + 4 * (((size_t)yp * nxp + xp) * nzp + zp), tile[0][threadIdx.x][i],
                          tile[0][threadIdx.x][i + 1], tile[1][threadIdx.x][i], tile[1][threadIdx.x][i + 1]);
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
    if (m0 > m1) return;
    const RayFF rf = ray3d_ff(p, v, k, l);
    float *V = vol + (size_t)b * p.nx * p.ny * p.nz;
    const size_t sxy = (size_t)p.nx * p.ny;
    for (int ms = m0; ms <= m1; ms += kFPSegment) {
        const int me = min(ms + kFPSegment - 1, m1);
        const Seg X = seg_at(rf.p[0], rf.q[0], ms), Y = seg_at(rf.p[1], rf.q[1], ms), Z = seg_at(rf.p[2], rf.q[2], ms);
        for (int m = ms; m <= me; ++m) {
            const float dm = (float)(m - ms);
            const Axis ax = tap_axis(seg_tap(X, dm), p.nx);
            const Axis ay = tap_axis(seg_tap(Y, dm), p.ny);
            const Axis az = tap_axis(seg_tap(Z, dm), p.nz);
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

// the volume's type and the copy's: the same type, or FP32 into FP16 / BF16
cudaError_t launch_relayout_quad(const void *vol, void *vp, int nx, int ny, int nz, pyro_dtype dt,
                                   pyro_dtype storage, cudaStream_t s)
{
    dim3 block(32, 8), grid((nx + 2 * kFPPadXY + 31) / 32, (nz + 2 + 31) / 32, ny + 2 * kFPPadXY);
    if (dt == PYRO_F32 && storage == PYRO_F32)
        relayout_quad_kernel<float, float><<<grid, block, 0, s>>>((const float *)vol, (float *)vp, nx, ny, nz);
    else if (dt == PYRO_F32 && storage == PYRO_F16)
        relayout_quad_kernel<float, __half><<<grid, block, 0, s>>>((const float *)vol, (__half *)vp, nx, ny, nz);
    else if (dt == PYRO_F32 && storage == PYRO_BF16)
        relayout_quad_kernel<float, __nv_bfloat16>
            <<<grid, block, 0, s>>>((const float *)vol, (__nv_bfloat16 *)vp, nx, ny, nz);
    else if (dt == PYRO_F16 && storage == PYRO_F16)
        relayout_quad_kernel<__half, __half><<<grid, block, 0, s>>>((const __half *)vol, (__half *)vp, nx, ny, nz);
    else if (dt == PYRO_BF16 && storage == PYRO_BF16)
        relayout_quad_kernel<__nv_bfloat16, __nv_bfloat16>
            <<<grid, block, 0, s>>>((const __nv_bfloat16 *)vol, (__nv_bfloat16 *)vp, nx, ny, nz);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// Grid (views, column groups, row groups): blocks start in linear index
// order, so the blocks in flight share a band of detector rows across the
// views, and with it a band of the volume's z (measured 1 % faster than
// the row groups varying fastest).
template <typename T, typename TO, int R>
static void column_launch(const void *vp, void *sino, int b, const FP3DParams &p, cudaStream_t s)
{
    dim3 block(32, kFPCWarps);
    dim3 grid((unsigned)p.n_views, (p.nu + kFPCWarps - 1) / kFPCWarps, (p.nv + 32 * R - 1) / (32 * R));
    fp3d_column_kernel<T, TO, R><<<grid, block, 0, s>>>((const T *)vp, (TO *)sino, p, b);
}

// 32-row windows per column, 1 to rmax per warp.  Cost model in issue slots
// per warp and depth plane: about 28 per window (windows past the last row
// included) plus about 30 shared by the warp's windows.  With the quad copy
// (16-byte loads) the forward takes at most 2: more windows hold more
// registers, and the fewer resident warps then hide the loads' latency
// worse (256^3 workload: 18.2 ms with at most 2, 19.6 with 3, 21.6 with 4).
static int column_windows_per_warp(int nv, int rmax = 2)
{
    const int windows = (nv + 31) / 32;
    int best = 1, cost = INT_MAX;
    for (int r = 1; r <= rmax && r <= windows; ++r) {
        const int c = (windows + r - 1) / r * (28 * r + 30);
        if (c <= cost) {
            best = r;
            cost = c;
        }
    }
    return best;
}

template <typename T, typename TO>
static void column_dispatch(const void *vp, void *sino, int b, const FP3DParams &p, cudaStream_t s)
{
    if (column_windows_per_warp(p.nv) == 2)
        column_launch<T, TO, 2>(vp, sino, b, p, s);
    else
        column_launch<T, TO, 1>(vp, sino, b, p, s);
}

// two-ray windows per warp: about 40 issue slots per window and depth plane
// plus about 30 shared by the warp's windows; at most 2, as for the one-ray
// kernel (512^3 TV workload: 490 ms with at most 2 or 3, 575 with 4)
static int pair_rows_windows_per_warp(int nv, int wr)
{
    const int windows = (nv + wr - 1) / wr;
    int best = 1, cost = INT_MAX;
    for (int r = 1; r <= 2 && r <= windows; ++r) {
        const int c = (windows + r - 1) / r * (40 * r + 30);
        if (c <= cost) {
            best = r;
            cost = c;
        }
    }
    return best;
}

template <typename T, typename TO, int R>
static void pair_rows_launch(const void *vp, void *sino, int b, const FP3DParams &p, cudaStream_t s)
{
    dim3 block(32, kFPPWarps);
    dim3 grid((unsigned)p.n_views, (p.nu + kFPPWarps - 1) / kFPPWarps, (p.nv + R * p.pair_rows - 1) / (R * p.pair_rows));
    fp3d_pair_rows_kernel<T, TO, R><<<grid, block, 0, s>>>((const T *)vp, (TO *)sino, p, b);
}

template <typename T, typename TO>
static void pair_rows_dispatch(const void *vp, void *sino, int b, const FP3DParams &p, cudaStream_t s)
{
    if (pair_rows_windows_per_warp(p.nv, p.pair_rows) == 2)
        pair_rows_launch<T, TO, 2>(vp, sino, b, p, s);
    else
        pair_rows_launch<T, TO, 1>(vp, sino, b, p, s);
}

template <typename T, typename TO>
static void column_any(const void *vp, void *sino, int b, const FP3DParams &p, cudaStream_t s)
{
    if (p.pair_rows > 0)
        pair_rows_dispatch<T, TO>(vp, sino, b, p, s);
    else
        column_dispatch<T, TO>(vp, sino, b, p, s);
}

// the copy's storage type and the sinogram's: the same type, or an FP16 /
// BF16 copy of an FP32 volume projected into an FP32 sinogram
cudaError_t launch_fp3d_column(const void *vp, void *sino, int b, const FP3DParams &p, pyro_dtype storage,
                               pyro_dtype sino_dt, cudaStream_t s)
{
    if (storage == PYRO_F32 && sino_dt == PYRO_F32)
        column_any<float, float>(vp, sino, b, p, s);
    else if (storage == PYRO_F16 && sino_dt == PYRO_F32)
        column_any<__half, float>(vp, sino, b, p, s);
    else if (storage == PYRO_BF16 && sino_dt == PYRO_F32)
        column_any<__nv_bfloat16, float>(vp, sino, b, p, s);
    else if (storage == PYRO_F16 && sino_dt == PYRO_F16)
        column_any<__half, __half>(vp, sino, b, p, s);
    else if (storage == PYRO_BF16 && sino_dt == PYRO_BF16)
        column_any<__nv_bfloat16, __nv_bfloat16>(vp, sino, b, p, s);
    else
        return cudaErrorInvalidValue;
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
