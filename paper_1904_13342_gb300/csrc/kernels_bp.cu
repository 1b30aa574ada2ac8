// Voxel-driven back-projection and its transpose
// (paper, Section "The Operator as a Layer": one thread per pixel / voxel
// projects its centre onto every view and accumulates the interpolated
// detector value; the cone-beam form follows Scherl et al. with projection
// matrices).
//
// Per view the host supplies a voxel-index -> detector map divided by SID
// (so w = L / SID and the FDK weight (SID/L)^2 is just 1/w^2) whose first
// rows are centred on the detector, as FP32 hi/lo pairs of the FP64 map.
// Every block first evaluates, for each view, the map at the centre of its
// voxel tile in float-float arithmetic (the anchor: an integer detector cell
// plus an FP32 fraction) together with the local slopes, into a shared-memory
// table; its voxels then add small FP32 offsets to the anchor.  An absolute
// FP32 detector coordinate near pixel 300 carries ~2e-5 pixel of rounding,
// which back-projected noise turns into ~2e-5 relative error; the anchored
// coordinate keeps ~1e-6.  Each cone-beam thread owns one (x, y) column and
// ZB consecutive z; for circular trajectories the u coordinate and the
// weight do not depend on z and are computed once per view.
#include "device_common.cuh"
#include "internal.h"

namespace pyro {

namespace {

__device__ __forceinline__ float weight_of(float rw, int wexp)
{
    return wexp == 0 ? 1.0f : (wexp == 1 ? rw : rw * rw);
}

// ---- anchors ---------------------------------------------------------------
__device__ __forceinline__ BP2DAnchor bp2d_anchor(const BP2DParams &p, int v, float ia, float ja)
{
    const float *m = p.m[v], *ml = p.mlo[v];
    const float hx[4] = {m[0], m[1], 0.0f, m[2]}, lx[4] = {ml[0], ml[1], 0.0f, ml[2]};
    const float hw[4] = {m[3], m[4], 0.0f, m[5]}, lw[4] = {ml[3], ml[4], 0.0f, ml[5]};
    const ff x = ff_dot4(hx, lx, ia, ja, 0.0f);
    const ff w = p.parallel ? ff{1.0f, 0.0f} : ff_dot4(hw, lw, ia, ja, 0.0f);
    const ff u = p.parallel ? x : ff_div(x, w);  // centred detector coordinate
    BP2DAnchor a;
    ff_split(u, p.cu, a.cu, a.fu);
    a.wa = w.h;
    a.w0 = p.parallel ? 0.0f : m[3];
    a.w1 = p.parallel ? 0.0f : m[4];
    a.a0 = fmaf(-u.h, a.w0, m[0]);
    a.a1 = fmaf(-u.h, a.w1, m[1]);
    a.pad = 0.0f;
    return a;
}

__device__ __forceinline__ BP3DAnchor bp3d_anchor(const BP3DParams &p, int v, float ia, float ja, float za)
{
    const float *P = p.P[v], *L = p.Plo[v];
    const ff x = ff_dot4(P, L, ia, ja, za);
    const ff y = ff_dot4(P + 4, L + 4, ia, ja, za);
    const ff w = ff_dot4(P + 8, L + 8, ia, ja, za);
    const ff u = ff_div(x, w), l = ff_div(y, w);  // centred detector coordinates
    BP3DAnchor a;
    ff_split(u, p.cu, a.cu, a.fu);
    ff_split(l, p.cv, a.cl, a.fl);
    a.wa = w.h;
    a.w0 = P[8];
    a.w1 = P[9];
    a.w2 = P[10];
    a.au0 = fmaf(-u.h, P[8], P[0]);
    a.au1 = fmaf(-u.h, P[9], P[1]);
    a.au2 = fmaf(-u.h, P[10], P[2]);
    a.al0 = fmaf(-l.h, P[8], P[4]);
    a.al1 = fmaf(-l.h, P[9], P[5]);
    a.al2 = fmaf(-l.h, P[10], P[6]);
    a.bx = 0;
    a.by = 0;
    return a;
}

// detector position of voxel anchor + d, relative to the anchor's cell
struct DetPos {
    float u, l, rw;  // u - cu, l - cl, 1 / w
};

__device__ __forceinline__ DetPos det_pos(const BP3DAnchor &a, float di, float dj, float dz)
{
    DetPos r;
    r.rw = 1.0f / fmaf(a.w0, di, fmaf(a.w1, dj, fmaf(a.w2, dz, a.wa)));
    r.u = fmaf(fmaf(a.au0, di, fmaf(a.au1, dj, a.au2 * dz)), r.rw, a.fu);
    r.l = fmaf(fmaf(a.al0, di, fmaf(a.al1, dj, a.al2 * dz)), r.rw, a.fl);
    return r;
}

// the TMA box of a tile: bounds of its corners' taps (the projection is
// linear-fractional with a positive depth, so the corners bound it), less a
// rounding margin, the column rounded down to `align` elements; cu, cl are
// made relative to the box
__device__ __forceinline__ void bp3d_box(BP3DAnchor &a, float d0i, float d1i, float d0j, float d1j, float d0z,
                                         float d1z, int align)
{
    float umin = 3.0e38f, lmin = 3.0e38f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const DetPos q = det_pos(a, (c & 1) ? d1i : d0i, (c & 2) ? d1j : d0j, (c & 4) ? d1z : d0z);
        umin = fminf(umin, q.u);
        lmin = fminf(lmin, q.l);
    }
    const int bx = (a.cu + (int)floorf(fmaxf(umin, -1.0e8f)) - 1) & ~(align - 1);
    const int by = a.cl + (int)floorf(fmaxf(lmin, -1.0e8f)) - 1;
    a.cu -= bx;
    a.cl -= by;
    a.bx = bx;
    a.by = by;
}

// shared-memory bytes of a per-view anchor table, rounded to 128
__host__ __device__ constexpr size_t table_bytes(int n_views, size_t entry)
{
    return ((size_t)n_views * entry + 127) / 128 * 128;
}

template <typename T>
__device__ __forceinline__ float lds(const T *p)
{
    return to_float<T>(*p);
}

// ---- 2D -----------------------------------------------------------------
template <typename TS, typename TV, bool PAR>
__global__ void __launch_bounds__(256) bp2d_kernel(const TS *__restrict__ sino, TV *__restrict__ vol,
                                                   const __grid_constant__ BP2DParams p, int accumulate)
{
    extern __shared__ __align__(16) unsigned char bp2_smem[];
    BP2DAnchor *tab = reinterpret_cast<BP2DAnchor *>(bp2_smem);
    const int t = threadIdx.y * 32 + threadIdx.x;
    const float ia = blockIdx.x * 32 + 15.5f, ja = blockIdx.y * 8 + 3.5f;
    for (int v = t; v < p.n_views; v += 256) tab[v] = bp2d_anchor(p, v, ia, ja);
    __syncthreads();
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int b = blockIdx.z;
    if (i >= p.nx || j >= p.ny) return;
    const float di = (float)i - ia, dj = (float)j - ja;
    const TS *S = sino + ((size_t)b * p.views_total + p.view0) * p.nu;
    float acc = 0.0f;
    for (int v = 0; v < p.n_views; ++v) {
        const BP2DAnchor a = tab[v];
        float rw = 1.0f, om = 1.0f;
        if (!PAR) {
            rw = 1.0f / fmaf(a.w0, di, fmaf(a.w1, dj, a.wa));
            om = weight_of(rw, p.wexp);
        }
        const float tu = fmaf(fmaf(a.a0, di, a.a1 * dj), rw, a.fu);
        const float mu = floor_magic(tu);
        const float f = tu - magic_to_float(mu);
        const int k = a.cu + magic_to_int(mu);
        const TS *row = S + (size_t)v * p.nu;
        const float w0 = ((unsigned)k < (unsigned)p.nu) ? 1.0f - f : 0.0f;
        const float w1 = ((unsigned)(k + 1) < (unsigned)p.nu) ? f : 0.0f;
        const int k0 = min(max(k, 0), p.nu - 1), k1 = min(max(k + 1, 0), p.nu - 1);
        acc = fmaf(om, fmaf(w0, ld(row + k0), w1 * ld(row + k1)), acc);
    }
    const size_t o = ((size_t)b * p.ny + j) * p.nx + i;
    float out = p.scale * acc;
    if (accumulate) out += to_float<TV>(vol[o]);
    vol[o] = to_storage<TV>(out);
}

__global__ void __launch_bounds__(256) bp2d_transpose_kernel(const float *__restrict__ vol, float *__restrict__ sino,
                                                             const __grid_constant__ BP2DParams p)
{
    extern __shared__ __align__(16) unsigned char bp2_smem[];
    BP2DAnchor *tab = reinterpret_cast<BP2DAnchor *>(bp2_smem);
    const int t = threadIdx.y * 32 + threadIdx.x;
    const float ia = blockIdx.x * 32 + 15.5f, ja = blockIdx.y * 8 + 3.5f;
    for (int v = t; v < p.n_views; v += 256) tab[v] = bp2d_anchor(p, v, ia, ja);
    __syncthreads();
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int b = blockIdx.z;
    if (i >= p.nx || j >= p.ny) return;
    const float g = p.scale * vol[((size_t)b * p.ny + j) * p.nx + i];
    if (g == 0.0f) return;
    const float di = (float)i - ia, dj = (float)j - ja;
    float *S = sino + ((size_t)b * p.views_total + p.view0) * p.nu;
    for (int v = 0; v < p.n_views; ++v) {
        const BP2DAnchor a = tab[v];
        float rw = 1.0f, om = 1.0f;
        if (!p.parallel) {
            rw = 1.0f / fmaf(a.w0, di, fmaf(a.w1, dj, a.wa));
            om = weight_of(rw, p.wexp);
        }
        const float tu = fmaf(fmaf(a.a0, di, a.a1 * dj), rw, a.fu);
        const float mu = floor_magic(tu);
        const float f = tu - magic_to_float(mu);
        const int k = a.cu + magic_to_int(mu);
        float *row = S + (size_t)v * p.nu;
        const float gw = g * om;
        if ((unsigned)k < (unsigned)p.nu && f != 1.0f) atomicAdd(row + k, gw * (1.0f - f));
        if ((unsigned)(k + 1) < (unsigned)p.nu && f != 0.0f) atomicAdd(row + k + 1, gw * f);
    }
}

constexpr int kBPX = 32, kBPY = 8, kBPZ = 8;

// ---- cone beam, L1 gathers ---------------------------------------------------
// The 32 x 8 voxel tile of a block is cut into 8 x 4 tiles per warp (not 32 x 1
// rows): a warp's voxels then project onto ~16 detector columns instead of
// ~40, one cache line per detector row.
template <typename TS, typename TV, bool ZINV>
__global__ void __launch_bounds__(kBPX *kBPY) bp3d_kernel(const TS *__restrict__ sino, TV *__restrict__ vol,
                                                          const __grid_constant__ BP3DParams p)
{
    extern __shared__ __align__(16) unsigned char bp3_smem[];
    BP3DAnchor *tab = reinterpret_cast<BP3DAnchor *>(bp3_smem);
    const int t = threadIdx.y * kBPX + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int i = blockIdx.x * kBPX + (warp & 3) * 8 + (lane & 7);
    const int j = blockIdx.y * kBPY + (warp >> 2) * 4 + (lane >> 3);
    const int zblocks = (p.nz + kBPZ - 1) / kBPZ;
    const int b = blockIdx.z / zblocks;
    const int z0 = (blockIdx.z % zblocks) * kBPZ;
    const float ia = blockIdx.x * kBPX + 15.5f, ja = blockIdx.y * kBPY + 3.5f, za = z0 + 3.5f;
    for (int v = t; v < p.n_views; v += kBPX * kBPY) tab[v] = bp3d_anchor(p, v, ia, ja, za);
    __syncthreads();
    if (i >= p.nx || j >= p.ny) return;
    const float di = (float)i - ia, dj = (float)j - ja, dz0 = (float)z0 - za;
    const size_t vstride = (size_t)p.nu * p.nv;
    const TS *S0 = sino + ((size_t)b * p.views_total + p.view0) * vstride;
    float acc[kBPZ];
#pragma unroll
    for (int zz = 0; zz < kBPZ; ++zz) acc[zz] = 0.0f;

    for (int v = 0; v < p.n_views; ++v) {
        const BP3DAnchor a = tab[v];
        const TS *S = S0 + (size_t)v * vstride;
        if (ZINV) {
            const DetPos q = det_pos(a, di, dj, dz0);
            const float om = weight_of(q.rw, p.wexp);
            const float dl = a.al2 * q.rw;
            const float mu = floor_magic(q.u);
            const float au = q.u - magic_to_float(mu);
            const int k = a.cu + magic_to_int(mu);
            const float la = q.l, lb = fmaf((float)(kBPZ - 1), dl, q.l);
            const int ra = a.cl + (int)floorf(fminf(la, lb)), rb = a.cl + (int)floorf(fmaxf(la, lb));
            if (k >= 0 && k + 1 < p.nu && ra >= 0 && rb + 1 < p.nv) {
                // every tap of the ZB voxels lies inside the detector: no masking
                const float w1 = om * au, w0 = om - w1;
                const TS *Sk = S + k + (long)a.cl * p.nu;  // row a.cl + floor(ll) >= 0 by the test above
#pragma unroll
                for (int zz = 0; zz < kBPZ; ++zz) {
                    const float ll = fmaf((float)zz, dl, q.l);
                    const float tl = floor_magic(ll);
                    const float av = ll - magic_to_float(tl);
                    const TS *r0 = Sk + magic_to_int(tl) * p.nu;
                    const float t0 = fmaf(w0, ld(r0), w1 * ld(r0 + 1));
                    const float t1 = fmaf(w0, ld(r0 + p.nu), w1 * ld(r0 + p.nu + 1));
                    acc[zz] += lerpf(t0, t1, av);
                }
                continue;
            }
            const float wu0 = ((unsigned)k < (unsigned)p.nu) ? om * (1.0f - au) : 0.0f;
            const float wu1 = ((unsigned)(k + 1) < (unsigned)p.nu) ? om * au : 0.0f;
            const int k0 = min(max(k, 0), p.nu - 1), k1 = min(max(k + 1, 0), p.nu - 1);
#pragma unroll
            for (int zz = 0; zz < kBPZ; ++zz) {
                const float ll = fmaf((float)zz, dl, q.l);
                const float tl = floor_magic(ll);
                const float av = ll - magic_to_float(tl);
                const int r = a.cl + magic_to_int(tl);
                const float wv0 = ((unsigned)r < (unsigned)p.nv) ? 1.0f - av : 0.0f;
                const float wv1 = ((unsigned)(r + 1) < (unsigned)p.nv) ? av : 0.0f;
                const TS *r0 = S + (size_t)min(max(r, 0), p.nv - 1) * p.nu;
                const TS *r1 = S + (size_t)min(max(r + 1, 0), p.nv - 1) * p.nu;
                const float t0 = fmaf(wu0, ld(r0 + k0), wu1 * ld(r0 + k1));
                const float t1 = fmaf(wu0, ld(r1 + k0), wu1 * ld(r1 + k1));
                acc[zz] = fmaf(wv0, t0, fmaf(wv1, t1, acc[zz]));
            }
        } else {
#pragma unroll
            for (int zz = 0; zz < kBPZ; ++zz) {
                const DetPos q = det_pos(a, di, dj, dz0 + (float)zz);
                const float om = weight_of(q.rw, p.wexp);
                const float mu = floor_magic(q.u), ml = floor_magic(q.l);
                const float au = q.u - magic_to_float(mu), av = q.l - magic_to_float(ml);
                const int k = a.cu + magic_to_int(mu), r = a.cl + magic_to_int(ml);
                const float wu0 = ((unsigned)k < (unsigned)p.nu) ? 1.0f - au : 0.0f;
                const float wu1 = ((unsigned)(k + 1) < (unsigned)p.nu) ? au : 0.0f;
                const float wv0 = ((unsigned)r < (unsigned)p.nv) ? 1.0f - av : 0.0f;
                const float wv1 = ((unsigned)(r + 1) < (unsigned)p.nv) ? av : 0.0f;
                const int k0 = min(max(k, 0), p.nu - 1), k1 = min(max(k + 1, 0), p.nu - 1);
                const TS *r0 = S + (size_t)min(max(r, 0), p.nv - 1) * p.nu;
                const TS *r1 = S + (size_t)min(max(r + 1, 0), p.nv - 1) * p.nu;
                const float v0 = fmaf(wu0, ld(r0 + k0), wu1 * ld(r0 + k1));
                const float v1 = fmaf(wu0, ld(r1 + k0), wu1 * ld(r1 + k1));
                acc[zz] = fmaf(om, fmaf(wv0, v0, wv1 * v1), acc[zz]);
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

// ---- TMA-staged cone BP (circular-type trajectories) --------------------
// Per view a block's 32 x 8 x kTZ voxel tile (kTZ = 8 or 16 z voxels per
// thread) projects onto a small detector box.  The boxes of G consecutive
// views form one stage of a ring of kBPTmaStages stages; threads 0..G-1 each
// copy one box with cp.async.bulk.tensor (completion counted on the stage's
// mbarrier), and every thread reads its four taps per voxel from shared
// memory.  One block barrier per stage (G views) frees the stage for the copy
// of the stage kBPTmaStages ahead.  Out-of-range parts of a box are
// zero-filled by the copy, which is the zero extension of the detector, so no
// tap needs masking.  Box sizes are a host-computed bound (the host also
// picks kTZ and G); every load stays inside its box (bp_view_box).  The
// sinogram is FP32, FP16 or BF16 (the taps are converted to FP32 on load).
constexpr int kTmaStages = kBPTmaStages;

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

template <typename TS>
__device__ __forceinline__ void tma_load_3d(TS *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One view of one thread's 8 voxels from a box in shared memory: the z
// voxels go in pairs through the packed f32x2 instructions; the box row pitch
// PITCH is a compile-time constant, so each voxel's four taps are one IMAD
// and four loads with immediate offsets.  The thread's rows are monotone in
// z, so checking the first and the last keeps every load inside the box; a
// thread whose rows would leave it (the host's box bound rules this out)
// takes the clamped scalar loop instead.
template <typename TS, int PITCH, int kTZ>
__device__ __forceinline__ void bp_view_box(const TS *S, int bv, const BP3DAnchor &a, float di, float dj, float dz0,
                                            int wexp, f32x2 (&acc)[kTZ / 2])
{
    const float rw = 1.0f / fmaf(a.w0, di, fmaf(a.w1, dj, a.wa));
    const float qu = fmaf(fmaf(a.au0, di, a.au1 * dj), rw, a.fu);
    const float ql = fmaf(fmaf(a.al0, di, fmaf(a.al1, dj, a.al2 * dz0)), rw, a.fl);
    const float om = weight_of(rw, wexp);
    const float mu = floor_magic(qu);
    const float au = qu - magic_to_float(mu);
    const float w1 = om * au, w0 = om - w1;
    const int col = a.cu + magic_to_int(mu);
    const float dl = a.al2 * rw;
    const float l7 = fmaf((float)(kTZ - 1), dl, ql);
    const int r0 = a.cl + magic_to_int(floor_magic(ql)), r7 = a.cl + magic_to_int(floor_magic(l7));
    if (col >= 0 && col + 1 < PITCH && min(r0, r7) >= 0 && max(r0, r7) + 1 < bv) {
        // element index of voxel zz's first tap: bits(floor_magic(l_zz)) * PITCH + off (mod 2^32)
        const unsigned off = (unsigned)(a.cl * PITCH + col) - 0x4B400000u * (unsigned)PITCH;
        const f32x2 W0 = pk2(w0, w0), W1 = pk2(w1, w1), L = pk2(ql, ql), DL = pk2(dl, dl);
        const f32x2 MAGIC = pk2(kFloorMagic, kFloorMagic);
#pragma unroll
        for (int pp = 0; pp < kTZ / 2; ++pp) {
            const f32x2 LL = fma2(pk2((float)(2 * pp), (float)(2 * pp + 1)), DL, L);
            const f32x2 TL = add2_rm(LL, MAGIC);
            const f32x2 AV = sub2(LL, sub2(TL, MAGIC));
            float t0, t1;
            upk2(TL, t0, t1);
            const TS *p0 = S + (__float_as_uint(t0) * (unsigned)PITCH + off);
            const TS *p1 = S + (__float_as_uint(t1) * (unsigned)PITCH + off);
            const f32x2 A = pk2(lds(p0), lds(p1)), B = pk2(lds(p0 + 1), lds(p1 + 1));
            const f32x2 C = pk2(lds(p0 + PITCH), lds(p1 + PITCH)), D = pk2(lds(p0 + PITCH + 1), lds(p1 + PITCH + 1));
            const f32x2 T0 = fma2(W0, A, mul2(W1, B)), T1 = fma2(W0, C, mul2(W1, D));
            acc[pp] = add2(acc[pp], fma2(AV, sub2(T1, T0), T0));
        }
        return;
    }
    const int last = PITCH * bv - PITCH - 2;
#pragma unroll
    for (int zz = 0; zz < kTZ; ++zz) {
        const float ll = fmaf((float)zz, dl, ql);
        const float tl = floor_magic(ll);
        const float av = ll - magic_to_float(tl);
        const int e = min(max((a.cl + magic_to_int(tl)) * PITCH + col, 0), last);
        const float s0 = fmaf(w0, lds(S + e), w1 * lds(S + e + 1));
        const float s1 = fmaf(w0, lds(S + e + PITCH), w1 * lds(S + e + PITCH + 1));
        float x, y;
        upk2(acc[zz / 2], x, y);
        if (zz & 1) y += lerpf(s0, s1, av);
        else x += lerpf(s0, s1, av);
        acc[zz / 2] = pk2(x, y);
    }
}

template <typename TS, typename TV, int G, int PITCH, int kTZ>
__global__ void __launch_bounds__(kBPX *kBPY, 4) bp3d_tma_kernel(const __grid_constant__ CUtensorMap map,
                                                              TV *__restrict__ vol,
                                                              const __grid_constant__ BP3DParams p, int bv,
                                                              int box_elems)
{
    extern __shared__ __align__(128) unsigned char tma_smem[];
    BP3DAnchor *tab = reinterpret_cast<BP3DAnchor *>(tma_smem);
    TS *stages = reinterpret_cast<TS *>(tma_smem + table_bytes(p.n_views, sizeof(BP3DAnchor)));
    __shared__ __align__(8) uint64_t full[kTmaStages];
    __shared__ int gave_up;
    const int t = threadIdx.y * kBPX + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int i0 = blockIdx.x * kBPX, j0 = blockIdx.y * kBPY;
    const int i = i0 + (warp & 3) * 8 + (lane & 7);
    const int j = j0 + (warp >> 2) * 4 + (lane >> 3);
    const int zblocks = (p.nz + kTZ - 1) / kTZ;
    const int b = blockIdx.z / zblocks;
    const int z0 = (blockIdx.z % zblocks) * kTZ;
    const int i1 = min(i0 + kBPX - 1, p.nx - 1), j1 = min(j0 + kBPY - 1, p.ny - 1), z1 = min(z0 + kTZ - 1, p.nz - 1);
    const float ia = i0 + 15.5f, ja = j0 + 3.5f, za = z0 + 0.5f * (kTZ - 1);
    const int vbase = b * p.views_total + p.view0;
    const bool active = i < p.nx && j < p.ny;  // the others still take part in the barriers
    const unsigned box_bytes = (unsigned)(PITCH * bv * sizeof(TS));
    constexpr int align = 16 / (int)sizeof(TS);  // x of a tensor copy: a multiple of 16 bytes
    for (int v = t; v < p.n_views; v += kBPX * kBPY) {
        BP3DAnchor a = bp3d_anchor(p, v, ia, ja, za);
        bp3d_box(a, (float)i0 - ia, (float)i1 - ia, (float)j0 - ja, (float)j1 - ja, (float)z0 - za, (float)z1 - za,
                 align);
        tab[v] = a;
    }
    if (t == 0) {
        for (int s = 0; s < kTmaStages; ++s) mbar_init(&full[s], G);
        gave_up = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int n_st = (p.n_views + G - 1) / G;
    // thread t < G: the box of view s G + t into stage s (a plain arrive for
    // the views past the end, so that the stage's G arrivals complete)
    auto issue = [&](int s) {
        const int slot = s % kTmaStages, v = s * G + t;
        if (v < p.n_views) {
            mbar_expect_tx(&full[slot], box_bytes);
            tma_load_3d(stages + (slot * G + t) * box_elems, &map, tab[v].bx, tab[v].by, vbase + v, &full[slot]);
        } else {
            mbar_arrive(&full[slot]);
        }
    };
    if (t < G)
        for (int s = 0; s < min(kTmaStages, n_st); ++s) issue(s);

    f32x2 acc[kTZ / 2];
#pragma unroll
    for (int pp = 0; pp < kTZ / 2; ++pp) acc[pp] = pk2(0.0f, 0.0f);
    const float di = (float)i - ia, dj = (float)j - ja, dz0 = (float)z0 - za;
    int s = 0;
    for (; s < n_st; ++s) {
        const int slot = s % kTmaStages;
        if (!mbar_wait(&full[slot], (unsigned)(s / kTmaStages) & 1u)) atomicExch(&gave_up, 1);
        if (active) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int v = s * G + g;
                if (v >= p.n_views) break;  // block-uniform
                bp_view_box<TS, PITCH, kTZ>(stages + (slot * G + g) * box_elems, bv, tab[v], di, dj, dz0, p.wexp, acc);
            }
        }
        __syncthreads();  // stage `slot` is free again; gave_up is visible
        if (gave_up) break;
        if (t < G && s + kTmaStages < n_st) issue(s + kTmaStages);
    }
    if (gave_up) {
        // let the copies still in flight land (bounded) before the block ends
        if (t == 0) {
            atomicExch(&g_status, 1);
            for (int w = s; w < min(s + kTmaStages, n_st); ++w)
                mbar_wait(&full[w % kTmaStages], (unsigned)(w / kTmaStages) & 1u);
        }
        return;
    }
    if (!active) return;
    const size_t sxy = (size_t)p.nx * p.ny;
    TV *out = vol + (size_t)b * sxy * p.nz + (size_t)j * p.nx + i;
#pragma unroll
    for (int zz = 0; zz < kTZ; ++zz) {
        const int z = z0 + zz;
        float x, y;
        upk2(acc[zz / 2], x, y);
        if (z < p.nz) {
            float r = p.scale * ((zz & 1) ? y : x);
            if (p.accumulate) r += to_float<TV>(out[z * sxy]);
            out[z * sxy] = to_storage<TV>(r);
        }
    }
}

__global__ void __launch_bounds__(kBPX *kBPY) bp3d_transpose_kernel(const float *__restrict__ vol,
                                                                    float *__restrict__ sino,
                                                                    const __grid_constant__ BP3DParams p)
{
    extern __shared__ __align__(16) unsigned char bp3_smem[];
    BP3DAnchor *tab = reinterpret_cast<BP3DAnchor *>(bp3_smem);
    const int b = blockIdx.z / p.nz;
    const int z = blockIdx.z % p.nz;
    const float ia = blockIdx.x * kBPX + 15.5f, ja = blockIdx.y * kBPY + 3.5f, za = (float)z;
    const int t = threadIdx.y * kBPX + threadIdx.x;
    for (int v = t; v < p.n_views; v += kBPX * kBPY) tab[v] = bp3d_anchor(p, v, ia, ja, za);
    __syncthreads();
    const int i = blockIdx.x * kBPX + threadIdx.x;
    const int j = blockIdx.y * kBPY + threadIdx.y;
    if (i >= p.nx || j >= p.ny) return;
    const float g = p.scale * vol[(((size_t)b * p.nz + z) * p.ny + j) * p.nx + i];
    if (g == 0.0f) return;
    const float di = (float)i - ia, dj = (float)j - ja;
    const size_t vstride = (size_t)p.nu * p.nv;
    float *S0 = sino + ((size_t)b * p.views_total + p.view0) * vstride;
    for (int v = 0; v < p.n_views; ++v) {
        const BP3DAnchor a = tab[v];
        const DetPos q = det_pos(a, di, dj, 0.0f);
        const float gw = g * weight_of(q.rw, p.wexp);
        const float mu = floor_magic(q.u), ml = floor_magic(q.l);
        const float au = q.u - magic_to_float(mu), av = q.l - magic_to_float(ml);
        const int k = a.cu + magic_to_int(mu), r = a.cl + magic_to_int(ml);
        float *S = S0 + (size_t)v * vstride;
        const float g0 = gw * (1.0f - av), g1 = gw * av;
        const bool k0 = (unsigned)k < (unsigned)p.nu, k1 = (unsigned)(k + 1) < (unsigned)p.nu;
        if ((unsigned)r < (unsigned)p.nv) {
            float *row = S + (size_t)r * p.nu;
            if (k0 && g0 * (1.0f - au) != 0.0f) atomicAdd(row + k, g0 * (1.0f - au));
            if (k1 && g0 * au != 0.0f) atomicAdd(row + k + 1, g0 * au);
        }
        if ((unsigned)(r + 1) < (unsigned)p.nv) {
            float *row = S + (size_t)(r + 1) * p.nu;
            if (k0 && g1 * (1.0f - au) != 0.0f) atomicAdd(row + k, g1 * (1.0f - au));
            if (k1 && g1 * au != 0.0f) atomicAdd(row + k + 1, g1 * au);
        }
    }
}

template <typename TS, typename TV>
cudaError_t bp2d_dispatch(const void *sino, void *vol, int batch, const BP2DParams &p, int accumulate, cudaStream_t s)
{
    dim3 block(32, 8);
    dim3 grid((p.nx + 31) / 32, (p.ny + 7) / 8, batch);
    const size_t smem = table_bytes(p.n_views, sizeof(BP2DAnchor));
    if (p.parallel)
        bp2d_kernel<TS, TV, true><<<grid, block, smem, s>>>((const TS *)sino, (TV *)vol, p, accumulate);
    else
        bp2d_kernel<TS, TV, false><<<grid, block, smem, s>>>((const TS *)sino, (TV *)vol, p, accumulate);
    return cudaGetLastError();
}

template <typename TS, typename TV>
cudaError_t bp3d_dispatch(const void *sino, void *vol, int batch, const BP3DParams &p, cudaStream_t s)
{
    dim3 block(kBPX, kBPY);
    const int zblocks = (p.nz + kBPZ - 1) / kBPZ;
    dim3 grid((p.nx + kBPX - 1) / kBPX, (p.ny + kBPY - 1) / kBPY, (unsigned)(zblocks * batch));
    const size_t smem = table_bytes(p.n_views, sizeof(BP3DAnchor));
    if (p.z_invariant)
        bp3d_kernel<TS, TV, true><<<grid, block, smem, s>>>((const TS *)sino, (TV *)vol, p);
    else
        bp3d_kernel<TS, TV, false><<<grid, block, smem, s>>>((const TS *)sino, (TV *)vol, p);
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

template <typename TS, typename TV, int G, int PITCH, int kTZ>
cudaError_t tma_launch(const CUtensorMap &map, void *vol, int batch, const BP3DParams &p, int bv, cudaStream_t s)
{
    const int be = tma_box_elems(PITCH, bv, sizeof(TS));
    const size_t smem = bp3d_tma_smem_bytes(p.n_views, PITCH, bv, sizeof(TS), G);
    auto kern = bp3d_tma_kernel<TS, TV, G, PITCH, kTZ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 block(kBPX, kBPY);
    const int zblocks = (p.nz + kTZ - 1) / kTZ;
    dim3 grid((p.nx + kBPX - 1) / kBPX, (p.ny + kBPY - 1) / kBPY, (unsigned)(zblocks * batch));
    kern<<<grid, block, smem, s>>>(map, (TV *)vol, p, bv, be);
    return cudaGetLastError();
}

template <typename TS, typename TV, int PITCH>
cudaError_t tma_by_stage(const CUtensorMap &map, void *vol, int batch, const BP3DParams &p, const BPTmaPlan &pl,
                         cudaStream_t s)
{
    if (pl.per_stage == 1 && pl.tile_z == 16) return tma_launch<TS, TV, 1, PITCH, 16>(map, vol, batch, p, pl.bv, s);
    if (pl.per_stage == 2 && pl.tile_z == 16) return tma_launch<TS, TV, 2, PITCH, 16>(map, vol, batch, p, pl.bv, s);
    if (pl.per_stage == 1 && pl.tile_z == 8) return tma_launch<TS, TV, 1, PITCH, 8>(map, vol, batch, p, pl.bv, s);
    if (pl.per_stage == 2 && pl.tile_z == 8) return tma_launch<TS, TV, 2, PITCH, 8>(map, vol, batch, p, pl.bv, s);
    return cudaErrorInvalidValue;
}

// bu: the box width, which is also the row pitch of a box in shared memory:
// 16 words modulo the 32 banks (80 or 144 floats, 96 or 160 halves), so that
// the taps of one column in adjacent rows, which a warp's lanes often read
// together, fall 16 banks apart
template <typename TS, typename TV>
cudaError_t tma_by_pitch(const CUtensorMap &map, void *vol, int batch, const BP3DParams &p, const BPTmaPlan &pl,
                         cudaStream_t s)
{
    constexpr int P0 = sizeof(TS) == 4 ? 80 : 96, P1 = sizeof(TS) == 4 ? 144 : 160;
    if (pl.bu == P0) return tma_by_stage<TS, TV, P0>(map, vol, batch, p, pl, s);
    if (pl.bu == P1) return tma_by_stage<TS, TV, P1>(map, vol, batch, p, pl, s);
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
    bp2d_transpose_kernel<<<grid, block, table_bytes(p.n_views, sizeof(BP2DAnchor)), s>>>((const float *)vol,
                                                                                        (float *)sino, p);
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

int tma_box_elems(int bu, int bv, size_t elem)
{
    const size_t per = 128 / elem;  // boxes start on 128-byte boundaries
    return (int)(((size_t)bu * bv + per - 1) / per * per);
}

size_t bp3d_tma_smem_bytes(int n_views, int bu, int bv, size_t elem, int per_stage)
{
    return table_bytes(n_views, sizeof(BP3DAnchor)) +
           (size_t)kTmaStages * per_stage * tma_box_elems(bu, bv, elem) * elem;
}

// the sinogram's type and the volume's: FP32 into any storage type (FDK
// reads its FP32 workspace), FP16 and BF16 into their own type
cudaError_t launch_bp3d_tma(const CUtensorMap &map, void *vol, int batch, const BP3DParams &p, const BPTmaPlan &pl,
                            pyro_dtype sino_dt, pyro_dtype vol_dt, cudaStream_t s)
{
    if (sino_dt == PYRO_F32) {
        switch (vol_dt) {
        case PYRO_F32: return tma_by_pitch<float, float>(map, vol, batch, p, pl, s);
        case PYRO_F16: return tma_by_pitch<float, __half>(map, vol, batch, p, pl, s);
        case PYRO_BF16: return tma_by_pitch<float, __nv_bfloat16>(map, vol, batch, p, pl, s);
        }
    }
    if (sino_dt == PYRO_F16 && vol_dt == PYRO_F16) return tma_by_pitch<__half, __half>(map, vol, batch, p, pl, s);
    if (sino_dt == PYRO_BF16 && vol_dt == PYRO_BF16)
        return tma_by_pitch<__nv_bfloat16, __nv_bfloat16>(map, vol, batch, p, pl, s);
    return cudaErrorInvalidValue;
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
    bp3d_transpose_kernel<<<grid, block, table_bytes(p.n_views, sizeof(BP3DAnchor)), s>>>((const float *)vol,
                                                                                        (float *)sino, p);
    return cudaGetLastError();
}

}  // namespace pyro
