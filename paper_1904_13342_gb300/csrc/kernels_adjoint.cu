// Exact adjoint A^T of the cone-beam ray-driven projector, gathered voxel by
// voxel (the gradient of the FP layer; paper, Section "The Known Operator":
// the gradient of A is A^T).
//
// For circular-type trajectories (the detector's v axis along the volume's z
// axis) the samples of detector column k on depth plane m share their (x, y)
// point P(k, m) = p(k) + m q(k), and row l samples z_l(m) = A + B l +
// m (C + D l) there: one affine map per plane, the same for every column.
// The adjoint at voxel (i, j, z) is then
//   sum over views, planes m and columns k of
//     t_xy(P(k, m) - (i, j)) * Z_km(z),   Z_km(z) = sum_l w_kl y_kl t(z - z_l(m)),
// t the linear tent (the interpolation weight), w_kl = dt |g_kl| the ray's
// step.  A block owns a T x T tile of voxel columns and kGW x 32 z
// voxels (one per lane).  Per view it tabulates the points (k, m) whose
// tents reach the tile (cell and bilinear weights), and every warp stages
// the rows its 32 z voxels can reach, for every column of the view that
// crosses the tile.  Planes are taken in groups of up to G: a lane's tent
// weights for a plane depend on the plane only, so they are computed once
// per group, and the rows of one column that the group's planes reach fit
// one window of W rows, read once per column with 128-bit loads.  The
// sums Z_km(z) then go to the tile columns the point's cell reaches,
// accumulated in registers.  Each output voxel is summed by one lane in a
// fixed order (views, column chunks, plane groups, columns, planes): the
// result is the same bit for bit from run to run, with no atomics on data.
// The weighted sinogram w y is read from a transposed copy [view][k][l], so
// that a column's rows are contiguous.
//
// Positions: the points' (x, y) and each warp's z anchor are evaluated in
// float-float from the host's FP64 maps (hi/lo pairs) and split into an
// integer cell and an FP32 fraction, as in the forward projector.
#include "device_common.cuh"
#include "internal.h"

namespace pyro {

namespace {

constexpr int kGW = kGatherWarps;  // warps per block, 32 z voxels each
constexpr int kGZ = 32 * kGW;

__device__ __forceinline__ ff ffv(const float (&a)[2])
{
    return {a[0], a[1]};
}

__device__ __forceinline__ ff ff_neg(ff a)
{
    return {-a.h, -a.l};
}

// a warp's z anchor on one depth plane
struct __align__(16) GPlane {
    int lc;          // the row whose z is at or below the warp's first z
    int n;           // rows a tent can reach: floor(2 / |beta|) + 1
    float f;         // warp's first z - z_lc(m)
    float beta;      // z step per row
    float ib;        // 1 / beta
    float pad[3];
};

// first row whose tent can reach z, as an offset from lc (d0 = z - z_lc):
// the rows with |d0 - beta j| < 1 are j in ((d0 - 1) / beta, (d0 + 1) / beta)
__device__ __forceinline__ int first_row(float d0, float ib)
{
    return (int)floorf(fminf((d0 - 1.0f) * ib, (d0 + 1.0f) * ib)) + 1;
}

// weighted transpose: yT[v][k][l] = dt |g_kl| y[b][v][l][k] for the views of a chunk
__global__ void __launch_bounds__(256) weighted_transpose_kernel(const float *__restrict__ sino,
                                                                 float *__restrict__ yT,
                                                                 const __grid_constant__ FP3DParams p, int b)
{
    __shared__ float tile[32][33];
    const int v = blockIdx.z;
    const int k0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
    const float *S = sino + (((size_t)b * p.views_total + p.view0 + v) * p.nv) * p.nu;
    const ConeFPView &V = p.v[v];
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int l = l0 + i, k = k0 + threadIdx.x;
        float y = 0.0f;
        if (l < p.nv && k < p.nu) {
            const float qx = fmaf(V.a0, (float)k, fmaf(V.a1, (float)l, V.a2));
            const float qy = fmaf(V.b0, (float)l, V.b2);
            y = p.dt * sqrtf(fmaf(qx, qx, fmaf(qy, qy, 1.0f))) * S[(size_t)l * p.nu + k];
        }
        tile[i][threadIdx.x] = y;
    }
    __syncthreads();
    float *T = yT + ((size_t)(p.view0 + v) * p.nu) * p.nv;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int k = k0 + i, l = l0 + threadIdx.x;
        if (k < p.nu && l < p.nv) T[(size_t)k * p.nv + l] = tile[threadIdx.x][i];
    }
}

// shared-memory layout of the gather kernel (bytes from the dynamic base)
struct GatherSmem {
    size_t rec, cell, pmask, prange, planes, stage, acc, total;
};

__host__ __device__ inline size_t align16(size_t o)
{
    return (o + 15) / 16 * 16;
}

__host__ __device__ inline GatherSmem gather_smem(const GatherParams &g)
{
    // every region starts on a 16-byte boundary (128-bit loads and stores)
    GatherSmem s;
    const size_t pts = (size_t)g.plmax * g.kmax;
    size_t o = 0;
    s.rec = o;  // float4 [plmax][kmax]: bilinear weights of the cell's corners
    o = align16(o + 16 * pts);
    s.cell = o;  // int [plmax][kmax]: accumulator offset of the first corner + 4096, + 65536 * corner mask
    o = align16(o + 4 * pts);
    s.pmask = o;  // u32 [ceil(plmax / 32)][kmax]: planes with a point, per column
    o = align16(o + 4 * (size_t)((g.plmax + 31) / 32) * g.kmax);
    s.prange = o;  // int2 [plmax]: first and last column with a point, per plane
    o = align16(o + 8 * (size_t)g.plmax);
    s.planes = o;  // GPlane [kGW][plmax]
    o = align16(o + sizeof(GPlane) * (size_t)kGW * g.plmax);
    s.stage = o;  // float [kGW][sc]
    o = align16(o + 4 * (size_t)kGW * g.sc);
    s.acc = o;  // float [kGW][tile * tile][32]
    o = align16(o + 4 * (size_t)kGW * g.tile * g.tile * 32);
    s.total = o;
    return s;
}

// add a point's four corner terms w Z to the warp's accumulators (tile side
// T): c packs the offset of corner (0, 0) plus 4096 and, times 65536, the
// mask of the corners inside the tile
template <int T>
__device__ __forceinline__ void corner_update(float *acc, int c, float4 w, float Z)
{
    const int mk = c >> 16;
    float *a = acc + ((c & 0xffff) - 4096);
    if (mk & 1) a[0] = fmaf(w.x, Z, a[0]);
    if (mk & 2) a[32] = fmaf(w.y, Z, a[32]);
    if (mk & 4) a[32 * T] = fmaf(w.z, Z, a[32 * T]);
    if (mk & 8) a[32 * T + 32] = fmaf(w.w, Z, a[32 * T + 32]);
}

template <int W, int G, int T>
__global__ void __launch_bounds__(32 * kGW, 4) fp3d_gather_adjoint_kernel(const float *__restrict__ yT,
                                                                          float *__restrict__ vol,
                                                                          const __grid_constant__ GatherParams g,
                                                                          int *status)
{
    static_assert(W % 4 == 0 && W >= 4 && W <= 32 && G >= 1 && G <= 4, "the window is whole float4s");
    extern __shared__ __align__(16) unsigned char gsm[];
    const GatherSmem L = gather_smem(g);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float4 *rec = reinterpret_cast<float4 *>(gsm + L.rec);
    int *cell = reinterpret_cast<int *>(gsm + L.cell);
    float *acc = reinterpret_cast<float *>(gsm + L.acc) + (size_t)warp * T * T * 32 + lane;
    unsigned *pmask = reinterpret_cast<unsigned *>(gsm + L.pmask);
    int2 *prange = reinterpret_cast<int2 *>(gsm + L.prange);
    GPlane *zpl = reinterpret_cast<GPlane *>(gsm + L.planes) + (size_t)warp * g.plmax;
    float *stage = reinterpret_cast<float *>(gsm + L.stage) + (size_t)warp * g.sc;
    __shared__ int s_bad;
    const unsigned full = 0xffffffffu;
    const int i0 = blockIdx.x * T, j0 = blockIdx.y * T;
    const int zw0 = blockIdx.z * kGZ + 32 * warp;  // the warp's first z
    // the support of the tile's tents: P in [i0 - 1, i0 + T) x [j0 - 1, j0 + T)
    const float bx0 = (float)(i0 - 1), bx1 = (float)(i0 + T), by0 = (float)(j0 - 1), by1 = (float)(j0 + T);
#pragma unroll
    for (int c = 0; c < T * T; ++c) acc[32 * c] = 0.0f;
    if (t == 0) s_bad = 0;

    for (int v = 0; v < g.n_views; ++v) {
        const GatherView &V = g.v[v];
        __syncthreads();  // the previous view's tables are no longer read
        // columns and depth planes that can reach the support: its corners
        // projected (every thread alike, so the branches below are uniform)
        float umn = 3.0e38f, umx = -3.0e38f, mmn = 3.0e38f, mmx = -3.0e38f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float x = (c & 1) ? bx1 : bx0, y = (c & 2) ? by1 : by0;
            const float u = fmaf(V.ui, x, fmaf(V.uj, y, V.u0)) / fmaf(V.wi, x, fmaf(V.wj, y, V.w0));
            const float m = fmaf(V.mi, x, fmaf(V.mj, y, V.mc));
            umn = fminf(umn, u);
            umx = fmaxf(umx, u);
            mmn = fminf(mmn, m);
            mmx = fmaxf(mmx, m);
        }
        const int klo = max(0, (int)ceilf(umn - 1e-3f)), khi = min(g.nu - 1, (int)floorf(umx + 1e-3f));
        const int mlo = max(-g.M, (int)ceilf(mmn - 1e-3f)), mhi = min(g.M, (int)floorf(mmx + 1e-3f));
        int K = khi - klo + 1, NP = mhi - mlo + 1;
        if (K <= 0 || NP <= 0) continue;
        if (K > g.kmax || NP > g.plmax) {
            if (t == 0) s_bad = 1;
            K = min(K, g.kmax);
            NP = min(NP, g.plmax);
        }
        const int NW = (NP + 31) >> 5;
        for (int e = t; e < NW * K; e += 32 * kGW) pmask[e] = 0u;
        for (int e = t; e < NP; e += 32 * kGW) prange[e] = make_int2(INT_MAX, -1);
        __syncthreads();
        // the points: (x, y) relative to the support's corner, from a
        // float-float anchor at the middle point of the tables and exact
        // bilinear increments in FP32 (X is bilinear in k and m:
        // X = X_a + (pxk + m_a qxk) dk + (qx0 + k_a qxk) dm + qxk dk dm)
        const int ka = klo + K / 2, ma = mlo + NP / 2;
        float xa, ya, bxk, bxm, byk, bym;
        {
            const float fk = (float)ka, fm = (float)ma;
            const ff X = ff_add(ff_add(ffv(V.px0), ff_mul_f(ffv(V.pxk), fk)),
                                ff_mul_f(ff_add(ffv(V.qx0), ff_mul_f(ffv(V.qxk), fk)), fm));
            const ff Y = ff_add(ff_add(ffv(V.py0), ff_mul_f(ffv(V.pyk), fk)),
                                ff_mul_f(ff_add(ffv(V.qy0), ff_mul_f(ffv(V.qyk), fk)), fm));
            const ff Xr = ff_add(X, {-bx0, 0.0f}), Yr = ff_add(Y, {-by0, 0.0f});
            xa = Xr.h + Xr.l;
            ya = Yr.h + Yr.l;
            bxk = fmaf(V.qxk[0], fm, V.pxk[0]);
            bxm = fmaf(V.qxk[0], fk, V.qx0[0]);
            byk = fmaf(V.qyk[0], fm, V.pyk[0]);
            bym = fmaf(V.qyk[0], fk, V.qy0[0]);
        }
        for (int p = warp; p < NP; p += kGW) {
            const float dm = (float)(mlo + p - ma);
            const float xm = fmaf(bxm, dm, xa), ym = fmaf(bym, dm, ya);
            const float sxk = fmaf(V.qxk[0], dm, bxk), syk = fmaf(V.qyk[0], dm, byk);
            for (int kk = lane; kk < K; kk += 32) {
                const float dk = (float)(klo + kk - ka);
                const float X = fmaf(sxk, dk, xm), Y = fmaf(syk, dk, ym);
                const float fx = floorf(X), fy = floorf(Y);
                const int cx = (int)fx, cy = (int)fy;
                const float ax = X - fx, ay = Y - fy;
                const bool in = cx >= 0 && cx <= T && cy >= 0 && cy <= T;
                const int e = p * K + kk;
                rec[e] = make_float4((1.0f - ax) * (1.0f - ay), ax * (1.0f - ay), (1.0f - ax) * ay, ax * ay);
                const int tx = cx - 1, ty = cy - 1;
                const int mk = (tx >= 0 && ty >= 0 ? 1 : 0) | (tx + 1 < T && ty >= 0 ? 2 : 0) |
                               (tx >= 0 && ty + 1 < T ? 4 : 0) | (tx + 1 < T && ty + 1 < T ? 8 : 0);
                cell[e] = in ? (ty * T + tx) * 32 + 4096 + 65536 * mk : 0;
                if (in) {  // integer OR / min / max: the same result in any order
                    atomicOr(&pmask[(p >> 5) * K + kk], 1u << (p & 31));
                    atomicMin(&prange[p].x, kk);
                    atomicMax(&prange[p].y, kk);
                }
            }
        }
        // the warp's z anchor on every plane, and the rows its lanes reach:
        // z_l(m) = alpha + beta l, alpha = A + m C, beta = B + m D
        int rlo = INT_MAX, rtop = INT_MIN;
        for (int p = lane; p < NP; p += 32) {
            const float fm = (float)(mlo + p);
            const ff alpha = ff_add(ffv(V.A), ff_mul_f(ffv(V.C), fm));
            const ff beta = ff_add(ffv(V.B), ff_mul_f(ffv(V.D), fm));
            const float z0 = (float)zw0;
            const ff x = ff_div(ff_add({z0, 0.0f}, ff_neg(alpha)), beta);  // row at the warp's first z
            const int lc = (int)floorf(x.h);
            const ff zl = ff_add(alpha, ff_mul_f(beta, (float)lc));
            GPlane pl;
            pl.lc = lc;
            pl.f = ff_add({z0, 0.0f}, ff_neg(zl)).h;
            pl.beta = beta.h;
            pl.ib = 1.0f / beta.h;
            pl.n = (int)floorf(2.0f * fabsf(pl.ib) + 1e-4f) + 1;
            pl.pad[0] = pl.pad[1] = pl.pad[2] = 0.0f;
            zpl[p] = pl;
            const int ja = first_row(pl.f, pl.ib), jb = first_row(pl.f + 31.0f, pl.ib);  // monotone in z
            rlo = min(rlo, lc + min(ja, jb));
            rtop = max(rtop, lc + max(ja, jb));
        }
        rlo = __reduce_min_sync(full, rlo);
        rtop = __reduce_max_sync(full, rtop);
        const int rlo4 = rlo & ~3;                      // floor to a multiple of 4
        const int RP = (rtop + W - rlo4 + 3) & ~3;      // staged rows per column
        __syncthreads();                                // points and z anchors ready
        const int KC = min(K, g.sc / RP);               // columns per stage fill
        if (KC < 1) {
            if (lane == 0) s_bad = 1;
            continue;
        }
        const float *Tv = yT + (size_t)(g.view0 + v) * g.nu * g.nv;
        for (int c0 = 0; c0 < K; c0 += KC) {
            const int nc = min(KC, K - c0);
            __syncwarp();  // the previous fill is no longer read
            const bool vec = (g.nv & 3) == 0;  // rows of a column start 16-byte aligned
            for (int kk = 0; kk < nc; ++kk) {
                const float *col = Tv + (size_t)(klo + c0 + kk) * g.nv;
                float4 *dst = reinterpret_cast<float4 *>(stage + kk * RP);
                for (int r4 = lane; r4 < RP / 4; r4 += 32) {
                    const int l = rlo4 + 4 * r4;
                    float4 x;
                    if (vec && l >= 0 && l + 3 < g.nv) {
                        x = __ldg(reinterpret_cast<const float4 *>(col + l));
                    } else {
                        x.x = (l >= 0 && l < g.nv) ? __ldg(col + l) : 0.0f;
                        x.y = (l + 1 >= 0 && l + 1 < g.nv) ? __ldg(col + l + 1) : 0.0f;
                        x.z = (l + 2 >= 0 && l + 2 < g.nv) ? __ldg(col + l + 2) : 0.0f;
                        x.w = (l + 3 >= 0 && l + 3 < g.nv) ? __ldg(col + l + 3) : 0.0f;
                    }
                    dst[r4] = x;
                }
            }
            __syncwarp();
            for (int p0 = 0; p0 < NP;) {
                // the group: consecutive planes (one mask word) whose rows fit
                // one W-row window starting at a multiple of 4, for every lane
                int lo = INT_MAX, hi = INT_MIN, gs = 0;
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    if (gs == q && p0 + q < NP && ((p0 + q) >> 5) == (p0 >> 5)) {
                        const GPlane pl = zpl[p0 + q];
                        const int js = pl.lc + first_row(pl.f + (float)lane, pl.ib);
                        const int nlo = min(lo, js), nhi = max(hi, js + pl.n);
                        if (__all_sync(full, nhi - (nlo & ~3) <= W)) {
                            lo = nlo;
                            hi = nhi;
                            gs = q + 1;
                        }
                    }
                }
                if (gs == 0) {  // a single plane always fits (W >= n + 3 on the host)
                    if (lane == 0) s_bad = 1;
                    const GPlane pl = zpl[p0];
                    lo = pl.lc + first_row(pl.f + (float)lane, pl.ib);
                    gs = 1;
                }
                const int ws = lo & ~3;
                const int soff = min(max(ws - rlo4, 0), RP - W);  // in range by construction
                // tent weights of rows ws + r, as pairs of rows (r even, r + 1)
                f32x2 wt[G][W / 2];
                int kf = INT_MAX, kl = -1;
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    if (q < gs) {  // uniform
                        const GPlane pl = zpl[p0 + q];
                        const int2 pr = prange[p0 + q];
                        kf = min(kf, pr.x);
                        kl = max(kl, pr.y);
                        const float d0 = pl.f + (float)lane;
                        const int o = ws - pl.lc;
#pragma unroll
                        for (int r = 0; r < W; r += 2)
                            wt[q][r / 2] = pk2(fmaxf(0.0f, 1.0f - fabsf(fmaf(-pl.beta, (float)(o + r), d0))),
                                               fmaxf(0.0f, 1.0f - fabsf(fmaf(-pl.beta, (float)(o + r + 1), d0))));
                    } else {
#pragma unroll
                        for (int r = 0; r < W / 2; ++r) wt[q][r] = 0ull;  // planes past the group: no point
                    }
                }
                const unsigned gmask = (1u << gs) - 1u;
                const unsigned *pm = pmask + (p0 >> 5) * K;
                const int sh = p0 & 31;
                const int kb = max(kf, c0), ke = min(kl, c0 + nc - 1);
                for (int k = kb; k <= ke; ++k) {
                    const unsigned bits = (pm[k] >> sh) & gmask;
                    if (!bits) continue;  // warp-uniform
                    const int e0 = p0 * K + k;
                    int cq[G];  // accumulator offsets and corner masks, fetched ahead of the sums
#pragma unroll
                    for (int q = 0; q < G; ++q) cq[q] = cell[e0 + min(q, gs - 1) * K];
                    const ulonglong2 *sp = reinterpret_cast<const ulonglong2 *>(stage + (k - c0) * RP + soff);
                    f32x2 sv[W / 2];
#pragma unroll
                    for (int q = 0; q < W / 4; ++q) {
                        const ulonglong2 a = sp[q];
                        sv[2 * q] = a.x;
                        sv[2 * q + 1] = a.y;
                    }
                    // the group's sums as independent chains of row pairs (a
                    // plane without a point here has zero weights or is skipped)
                    f32x2 Zp[G];
#pragma unroll
                    for (int q = 0; q < G; ++q) Zp[q] = 0ull;
#pragma unroll
                    for (int r = 0; r < W / 2; ++r) {
#pragma unroll
                        for (int q = 0; q < G; ++q) Zp[q] = fma2(wt[q][r], sv[r], Zp[q]);
                    }
#pragma unroll
                    for (int q = 0; q < G; ++q) {
                        if ((bits >> q) & 1u) {  // uniform
                            float za, zb;
                            upk2(Zp[q], za, zb);
                            corner_update<T>(acc, cq[q], rec[e0 + q * K], za + zb);
                        }
                    }
                }
                p0 += gs;
            }
        }
    }
    __syncthreads();
    if (t == 0 && s_bad) atomicOr(status, 2);
    // the tile's voxels: lane z of every column
    const int z = zw0 + lane;
    if (z < g.nz) {
        float *out = vol + (size_t)z * g.ny * g.nx;
#pragma unroll
        for (int c = 0; c < T * T; ++c) {
            const int x = i0 + c % T, y = j0 + c / T;
            if (x < g.nx && y < g.ny) {
                float *o = out + (size_t)y * g.nx + x;
                *o = g.accumulate ? *o + acc[32 * c] : acc[32 * c];
            }
        }
    }
}

}  // namespace

size_t gather_smem_bytes(const GatherParams &g)
{
    return gather_smem(g).total;
}

cudaError_t launch_weighted_transpose(const void *sino, void *yT, int b, const FP3DParams &p, cudaStream_t s)
{
    dim3 block(32, 8), grid((p.nu + 31) / 32, (p.nv + 31) / 32, p.n_views);
    weighted_transpose_kernel<<<grid, block, 0, s>>>((const float *)sino, (float *)yT, p, b);
    return cudaGetLastError();
}

template <int W, int G, int T>
static cudaError_t gather_launch(const void *yT, void *vol, const GatherParams &g, int *status, cudaStream_t s)
{
    if (g.sc % 4 != 0 || g.sc < W || g.kmax < 1 || g.plmax < 1 || g.tile != T) return cudaErrorInvalidValue;
    const size_t smem = gather_smem_bytes(g);
    cudaError_t e = cudaFuncSetAttribute(fp3d_gather_adjoint_kernel<W, G, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.nx + T - 1) / T, (g.ny + T - 1) / T, (g.nz + kGZ - 1) / kGZ);
    fp3d_gather_adjoint_kernel<W, G, T><<<grid, 32 * kGW, smem, s>>>((const float *)yT, (float *)vol, g, status);
    return cudaGetLastError();
}

template <int T>
static cudaError_t gather_by_window(const void *yT, void *vol, const GatherParams &g, int *status, cudaStream_t s)
{
    // planes per group: their tent weights stay in registers (G W / 2 pairs)
    switch (g.wrows) {
    case 4:
        return gather_launch<4, 4, T>(yT, vol, g, status, s);
    case 8:
        return gather_launch<8, 4, T>(yT, vol, g, status, s);
    case 12:
        return gather_launch<12, 4, T>(yT, vol, g, status, s);
    case 16:
        return gather_launch<16, 3, T>(yT, vol, g, status, s);
    case 20:
        return gather_launch<20, 2, T>(yT, vol, g, status, s);
    case 24:
        return gather_launch<24, 2, T>(yT, vol, g, status, s);
    case 28:
        return gather_launch<28, 1, T>(yT, vol, g, status, s);
    case 32:
        return gather_launch<32, 1, T>(yT, vol, g, status, s);
    default:
        return cudaErrorInvalidValue;
    }
}

// one batch item: yT holds its transposed, weighted views
cudaError_t launch_gather_adjoint(const void *yT, void *vol, const GatherParams &g, int *status, cudaStream_t s)
{
    switch (g.tile) {
    case 4:
        return gather_by_window<4>(yT, vol, g, status, s);
    case 6:
        return gather_by_window<6>(yT, vol, g, status, s);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace pyro
