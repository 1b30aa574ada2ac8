// Residual 3D CNN kernels (BF16 storage, FP32 accumulation): the learned
// initialiser placed in front of the TV iteration.  The paper has no such
// network; it is the "learned parts" extension of the reconstruction path.
//
// Activations are channels-last [B][D][H][W][C] bf16.  Weights are
// [27][Cout][Cin] bf16 (tap = (dz*3 + dy)*3 + dx, taps of a 3x3x3 window,
// stride 1, zero padding 1); master weights and gradients are FP32.
//
// conv3d_tc_kernel: implicit GEMM on the 5th-generation tensor cores
// (tcgen05.mma, bf16 in, FP32 accumulate in tensor memory); a block computes
// 128 output voxels (a TX x TY x TZ box) x Cout.  The same kernel computes the
// data gradient with the spatially flipped, channel-transposed weights.
// conv3d_wgrad_tc_kernel: dW[tap][co][ci] = sum_v dY[v][co] X[v+tap][ci] as a
// GEMM on tcgen05 with M = (tap, ci) rows, N = Cout, K = voxels.
#include <cuda_bf16.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace pyro {

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ unsigned pack_bf16(bf16 lo, bf16 hi)
{
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}


// 128 output voxels per block: TX x TY x TZ (x fastest)
struct Tile {
    int TX, TY, TZ;
};

__host__ __device__ inline Tile conv_tile(int W, int H)
{
    Tile t;
    t.TX = W >= 64 ? 64 : W;
    t.TY = min(H, 128 / t.TX);
    t.TZ = 128 / (t.TX * t.TY);
    return t;
}

// ---- conv3d_tc_kernel: the same implicit GEMM on the 5th-generation tensor
// cores.  A block of 128 threads owns 128 output voxels (row m = thread m)
// and a [128 x Cout] FP32 accumulator in tensor memory.  Per tap of the 3x3x3
// window every thread gathers its voxel's shifted input row (Cin bf16, 16-byte
// loads; zero outside the volume) and the block gathers the tap's [Cout x Cin]
// weights, both into a double-buffered shared-memory stage in the canonical
// K-major layout of the MMA (8 x 8 core matrices of 128 contiguous bytes);
// one thread issues Cin / 16 tcgen05.mma (M = 128, N = Cout, K = 16) and
// commits them to the stage's mbarrier, so the gather of tap t + 1 overlaps
// the MMAs of tap t.  The epilogue reads the accumulator with tcgen05.ld and
// adds the bias and the ReLU.  Waits are time-bounded.  A block whose wait
// gives up stops at once (every thread leaves the tap loop together: no
// further stage writes or MMAs), drains the last commit with another bounded
// wait, writes nothing, sets the status word and then frees its tensor
// memory.
__device__ __forceinline__ uint64_t umma_desc(const void *smem, unsigned lbo, unsigned sbo)
{
    uint64_t d = (uint64_t)((smem_addr(smem) >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;  // next core matrix along K
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;  // next group of 8 rows
    d |= (uint64_t)1 << 46;                      // descriptor version; no swizzle, base offset 0
    return d;
}

// COUTR <= COUT output channels are real: the weights are [27][COUTR][Cin],
// the MMA's other rows of B are zero, and only COUTR channels are stored
// (a layer with one output channel runs as N = 16).
template <int CIN, int COUT, int COUTR = COUT>
__global__ void __launch_bounds__(128) conv3d_tc_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ Wt,
                                                        const float *__restrict__ bias, bf16 *__restrict__ Y, int D,
                                                        int H, int Wd, int relu, int *status)
{
    static_assert(COUTR >= 1 && COUTR <= COUT && (COUTR == COUT || COUTR < 16), "real output channels");
    constexpr int KCH = CIN / 8;  // 16-byte chunks of a row
    constexpr int A_EL = 128 * CIN, B_EL = COUT * CIN;
    constexpr unsigned TCOLS = COUT < 32 ? 32 : COUT;  // tensor-memory columns (a power of two >= 32)
    extern __shared__ __align__(128) unsigned char conv_smem[];
    bf16 *sA = reinterpret_cast<bf16 *>(conv_smem);  // [2][128 x Cin]
    bf16 *sB = sA + 2 * A_EL;                         // [2][Cout x Cin]
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ unsigned tmem_slot;
    const int t = threadIdx.x, warp = t >> 5;
    const Tile tl = conv_tile(Wd, H);
    const int TX = tl.TX, TY = tl.TY;
    const int tiles_x = Wd / TX, tiles_y = H / TY, tiles_z = D / tl.TZ;
    int blk = blockIdx.x;
    const int tx0 = (blk % tiles_x) * TX;
    blk /= tiles_x;
    const int ty0 = (blk % tiles_y) * TY;
    blk /= tiles_y;
    const int tz0 = (blk % tiles_z) * tl.TZ;
    const int b = blk / tiles_z;
    const int vz = tz0 + t / (TX * TY), vy = ty0 + (t / TX) % TY, vx = tx0 + t % TX;
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    if constexpr (COUTR < COUT) {  // rows of B past the real channels: zero in both stages
        for (int q = t; q < 2 * B_EL / 8; q += 128) reinterpret_cast<uint4 *>(sB)[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_slot;
    // f32 accumulate, bf16 A and B, both K-major, N = Cout, M = 128
    constexpr unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(COUT >> 3) << 17) | (8u << 24);
    bool ok = true;
    int last = -1;  // the last tap whose MMAs were committed
    for (int tap = 0; tap < 27; ++tap) {
        const int buf = tap & 1;
        // the MMAs of tap - 2 read this stage; after a wait gives up the
        // block writes no stage and issues no MMA any more
        if (tap >= 2) {
            if (!mbar_wait(&bar[buf], (unsigned)((tap - 2) >> 1) & 1u)) ok = false;
            if (!__syncthreads_and(ok ? 1 : 0)) break;
        }
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        const int gz = vz + dz - 1, gy = vy + dy - 1, gx = vx + dx - 1;
        const bool in = gz >= 0 && gz < D && gy >= 0 && gy < H && gx >= 0 && gx < Wd;
        const uint4 *src = reinterpret_cast<const uint4 *>(X + ((((size_t)b * D + gz) * H + gy) * Wd + gx) * CIN);
        bf16 *A = sA + buf * A_EL;
#pragma unroll
        for (int c = 0; c < KCH; ++c) {
            const uint4 v = in ? __ldg(src + c) : make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(A + ((t >> 3) * KCH + c) * 64 + (t & 7) * 8) = v;
        }
        bf16 *Bs = sB + buf * B_EL;
        const uint4 *wsrc = reinterpret_cast<const uint4 *>(Wt + (size_t)tap * COUTR * CIN);
        for (int q = t; q < COUTR * KCH; q += 128) {
            const int n = q / KCH, c = q - n * KCH;
            *reinterpret_cast<uint4 *>(Bs + ((n >> 3) * KCH + c) * 64 + (n & 7) * 8) = __ldg(wsrc + q);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int kk = 0; kk < CIN / 16; ++kk) {
                const uint64_t ad = umma_desc(A + kk * 128, 128, CIN * 16);
                const uint64_t bd = umma_desc(Bs + kk * 128, 128, CIN * 16);
                const unsigned accumulate = (tap > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n"
                    " .reg .pred p;\n"
                    " setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
                    "}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&bar[buf]))
                         : "memory");
        }
        last = tap;
    }
    // the last commit tracks every MMA issued before it: drain it (bounded)
    // before the accumulator is read or the tensor memory released
    if (last >= 0 && !mbar_wait(&bar[last & 1], (unsigned)(last >> 1) & 1u)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int all_ok = __syncthreads_and(ok && last == 26 ? 1 : 0);
    if (all_ok && COUTR < 16) {  // the first COUTR columns only
        unsigned r[16];
        const unsigned addr = tmem + ((unsigned)(32 * warp) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        bf16 *out = Y + ((((size_t)b * D + vz) * H + vy) * Wd + vx) * COUTR;
#pragma unroll
        for (int c = 0; c < COUTR; ++c) {
            float a = __uint_as_float(r[c]);
            if (bias) a += bias[c];
            if (relu) a = fmaxf(a, 0.0f);
            out[c] = __float2bfloat16(a);
        }
    } else if (all_ok) {
        bf16 *out = Y + ((((size_t)b * D + vz) * H + vy) * Wd + vx) * COUT;
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 16) {
            unsigned r[16];
            const unsigned addr = tmem + ((unsigned)(32 * warp) << 16) + (unsigned)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            unsigned pk[8];
#pragma unroll
            for (int c = 0; c < 16; c += 2) {
                float a = __uint_as_float(r[c]), d = __uint_as_float(r[c + 1]);
                if (bias) {
                    a += bias[c0 + c];
                    d += bias[c0 + c + 1];
                }
                if (relu) {
                    a = fmaxf(a, 0.0f);
                    d = fmaxf(d, 0.0f);
                }
                pk[c / 2] = pack_bf16(__float2bfloat16(a), __float2bfloat16(d));
            }
            uint4 *o = reinterpret_cast<uint4 *>(out + c0);
            o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
    } else if (t == 0) {
        atomicExch(status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

// ---- conv3d_tc_k27_kernel: one input channel (the first layer).  The 27
// taps are the GEMM's K (padded to 32 with zeros): every thread gathers its
// voxel's 27 neighbours into one row of A, the block stages B = the [Cout x
// 32] tap weights once, and two tcgen05.mma (K = 16 each) make the whole
// convolution; epilogue as conv3d_tc_kernel.
template <int COUT>
__global__ void __launch_bounds__(128) conv3d_tc_k27_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ Wt,
                                                            const float *__restrict__ bias, bf16 *__restrict__ Y,
                                                            int D, int H, int Wd, int relu, int *status)
{
    constexpr int KCH = 4;  // 32 bf16 of K in 16-byte chunks
    constexpr unsigned TCOLS = COUT < 32 ? 32 : COUT;
    __shared__ __align__(128) bf16 sA[128 * 32];
    __shared__ __align__(128) bf16 sB[COUT * 32];
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned tmem_slot;
    const int t = threadIdx.x, warp = t >> 5;
    const Tile tl = conv_tile(Wd, H);
    const int TX = tl.TX, TY = tl.TY;
    const int tiles_x = Wd / TX, tiles_y = H / TY, tiles_z = D / tl.TZ;
    int blk = blockIdx.x;
    const int tx0 = (blk % tiles_x) * TX;
    blk /= tiles_x;
    const int ty0 = (blk % tiles_y) * TY;
    blk /= tiles_y;
    const int tz0 = (blk % tiles_z) * tl.TZ;
    const int b = blk / tiles_z;
    const int vz = tz0 + t / (TX * TY), vy = ty0 + (t / TX) % TY, vx = tx0 + t % TX;
    if (t == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    // the block's voxels with a one-voxel halo (zero outside the volume):
    // at most 3 x 4 x 66 values (TX TY TZ = 128, TX <= 64)
    __shared__ bf16 sX[1024];
    const bf16 zero = __float2bfloat16(0.0f);
    const int HX = TX + 2, HY = TY + 2, HZ = tl.TZ + 2;
    for (int q = t; q < HX * HY * HZ; q += 128) {
        const int hx = q % HX, hy = (q / HX) % HY, hz = q / (HX * HY);
        const int gz = tz0 + hz - 1, gy = ty0 + hy - 1, gx = tx0 + hx - 1;
        const bool in = gz >= 0 && gz < D && gy >= 0 && gy < H && gx >= 0 && gx < Wd;
        sX[q] = in ? X[(((size_t)b * D + gz) * H + gy) * Wd + gx] : zero;
    }
    __syncthreads();
    // A: row t = the 27 neighbours of voxel t, then 5 zeros
    const int lz = vz - tz0, ly = vy - ty0, lx = vx - tx0;
    bf16 v[32];
#pragma unroll
    for (int tap = 0; tap < 27; ++tap)
        v[tap] = sX[((lz + tap / 9) * HY + ly + (tap / 3) % 3) * HX + lx + tap % 3];
#pragma unroll
    for (int k = 27; k < 32; ++k) v[k] = zero;
#pragma unroll
    for (int c = 0; c < KCH; ++c) {
        uint4 u;
        u.x = pack_bf16(v[8 * c], v[8 * c + 1]);
        u.y = pack_bf16(v[8 * c + 2], v[8 * c + 3]);
        u.z = pack_bf16(v[8 * c + 4], v[8 * c + 5]);
        u.w = pack_bf16(v[8 * c + 6], v[8 * c + 7]);
        *reinterpret_cast<uint4 *>(sA + ((t >> 3) * KCH + c) * 64 + (t & 7) * 8) = u;
    }
    // B[n][k] = W[tap = k][n] (weights [27][Cout][1]), zero for k >= 27
    for (int q = t; q < COUT * 32; q += 128) {
        const int n = q >> 5, k = q & 31;
        sB[((n >> 3) * KCH + (k >> 3)) * 64 + (n & 7) * 8 + (k & 7)] = k < 27 ? Wt[k * COUT + n] : zero;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_slot;
    constexpr unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(COUT >> 3) << 17) | (8u << 24);
    if (t == 0) {
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const uint64_t ad = umma_desc(sA + kk * 128, 128, 32 * 16);
            const uint64_t bd = umma_desc(sB + kk * 128, 128, 32 * 16);
            const unsigned accumulate = kk > 0 ? 1u : 0u;
            asm volatile(
                "{\n"
                " .reg .pred p;\n"
                " setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
                "}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&bar))
                     : "memory");
    }
    bool ok = mbar_wait(&bar, 0u);
    // after a give-up, drain the commit (bounded) before the accumulator is
    // dropped and the tensor memory freed
    if (!ok) mbar_wait(&bar, 0u);
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int all_ok = __syncthreads_and(ok ? 1 : 0);
    if (all_ok) {
        bf16 *out = Y + ((((size_t)b * D + vz) * H + vy) * Wd + vx) * COUT;
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 16) {
            unsigned r[16];
            const unsigned addr = tmem + ((unsigned)(32 * warp) << 16) + (unsigned)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            unsigned pk[8];
#pragma unroll
            for (int c = 0; c < 16; c += 2) {
                float a = __uint_as_float(r[c]), d = __uint_as_float(r[c + 1]);
                if (bias) {
                    a += bias[c0 + c];
                    d += bias[c0 + c + 1];
                }
                if (relu) {
                    a = fmaxf(a, 0.0f);
                    d = fmaxf(d, 0.0f);
                }
                pk[c / 2] = pack_bf16(__float2bfloat16(a), __float2bfloat16(d));
            }
            uint4 *o = reinterpret_cast<uint4 *>(out + c0);
            o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
    } else if (t == 0) {
        atomicExch(status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

// ---- conv3d_tc_rows_kernel: rows of 128 output voxels along x (W a
// multiple of 128: the full-resolution 16-channel layers), walked along z.
// A block owns output rows (b, z, y, x0 .. x0 + 127) for kRowsZ consecutive
// z.  It keeps the input lines it needs in a ring of four z slots of three
// lines (dy = -1, 0, 1), each line x0 - 1 .. x0 + 128 stored as Cin / 8
// planes of 130 contiguous 16-byte rows, so that tap (dz, dy, dx) of row z
// is the line (z + dz - 1, dy) read from row dx on: a K-major operand whose
// 8-row groups sit 128 bytes apart and whose K chunks one plane apart.  Per
// row only the three lines of z + 2 are new: they are fetched with cp.async
// (zero-filled outside the volume) while the MMAs of the current row run,
// and the accumulator is double-buffered in tensor memory, so the epilogue
// of row z - 1 overlaps them too.  The 27 taps' weights are staged once per
// block.  Waits are time-bounded; after a give-up the block stops issuing,
// drains its last commit (bounded), writes nothing more, sets the status
// word and frees its tensor memory.
constexpr int kRowsZ = 16;

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool in)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(in ? 16 : 0)
                 : "memory");
}

template <int CIN, int COUT, int COUTR>
__device__ __forceinline__ void rows_epilogue(unsigned tmem_acc, int warp, bf16 *out, const float *bias, int relu)
{
    unsigned r[16];
#pragma unroll
    for (int c0 = 0; c0 < COUT; c0 += 16) {
        if (c0 >= COUTR) break;
        const unsigned addr = tmem_acc + ((unsigned)(32 * warp) << 16) + (unsigned)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if constexpr (COUTR < 16) {
#pragma unroll
            for (int c = 0; c < COUTR; ++c) {
                float a = __uint_as_float(r[c]);
                if (bias) a += bias[c];
                if (relu) a = fmaxf(a, 0.0f);
                out[c] = __float2bfloat16(a);
            }
        } else {
            unsigned pk[8];
#pragma unroll
            for (int c = 0; c < 16; c += 2) {
                float a = __uint_as_float(r[c]), d = __uint_as_float(r[c + 1]);
                if (bias) {
                    a += bias[c0 + c];
                    d += bias[c0 + c + 1];
                }
                if (relu) {
                    a = fmaxf(a, 0.0f);
                    d = fmaxf(d, 0.0f);
                }
                pk[c / 2] = pack_bf16(__float2bfloat16(a), __float2bfloat16(d));
            }
            uint4 *o = reinterpret_cast<uint4 *>(out + c0);
            o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
    }
}

template <int CIN, int COUT, int COUTR = COUT>
__global__ void __launch_bounds__(128) conv3d_tc_rows_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ Wt,
                                                             const float *__restrict__ bias, bf16 *__restrict__ Y,
                                                             int D, int H, int Wd, int relu, int *status)
{
    static_assert(COUTR >= 1 && COUTR <= COUT && (COUTR == COUT || COUTR < 16), "real output channels");
    constexpr int KCH = CIN / 8;
    constexpr int ROWS = 130;          // input x0 - 1 .. x0 + 128
    constexpr int P = ROWS * 16;       // bytes of one K-chunk plane of a line
    constexpr int LINE = KCH * P;      // bytes of one staged line
    constexpr int SET = 3 * LINE;      // the three lines (dy) of one input z
    constexpr int B_TAP = COUT * CIN;  // bf16 of one tap's B
    constexpr unsigned TCOLS = 2 * COUT < 32 ? 32 : 2 * COUT;  // two accumulators
    extern __shared__ __align__(128) unsigned char rows_smem[];
    unsigned char *ring = rows_smem;                              // [4 slots][3 lines][KCH][130][16 B]
    bf16 *sB = reinterpret_cast<bf16 *>(rows_smem + 4 * SET);    // [27][COUT x CIN] canonical
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ unsigned tmem_slot;
    const int t = threadIdx.x, warp = t >> 5;
    const int lines_x = Wd / 128, zchunks = (D + kRowsZ - 1) / kRowsZ;
    int blk = blockIdx.x;
    const int x0 = (blk % lines_x) * 128;
    blk /= lines_x;
    const int y = blk % H;
    blk /= H;
    const int z0 = (blk % zchunks) * kRowsZ;
    const int b = blk / zchunks;
    const int nrows = min(z0 + kRowsZ, D) - z0;
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    // every tap's weights (rows past the real channels zero)
    if constexpr (COUTR < COUT) {
        for (int q = t; q < 27 * B_TAP / 8; q += 128) reinterpret_cast<uint4 *>(sB)[q] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
    }
    for (int q = t; q < 27 * COUTR * KCH; q += 128) {
        const int tap = q / (COUTR * KCH), rem = q - tap * (COUTR * KCH);
        const int n = rem / KCH, c = rem - n * KCH;
        *reinterpret_cast<uint4 *>(sB + tap * B_TAP + ((n >> 3) * KCH + c) * 64 + (n & 7) * 8) =
            __ldg(reinterpret_cast<const uint4 *>(Wt) + q);
    }
    // the three lines of input z zi into ring slot zi mod 4 (zero outside the volume)
    auto fetch = [&](int zi) {
        unsigned char *dst = ring + (zi & 3) * SET;
        for (int q = t; q < 3 * ROWS * KCH; q += 128) {
            const int L = q / (ROWS * KCH), rem = q - L * (ROWS * KCH);
            const int r = rem / KCH, c = rem - r * KCH;
            const int gy = y + L - 1, gx = x0 - 1 + r;
            const bool in = zi >= 0 && zi < D && gy >= 0 && gy < H && gx >= 0 && gx < Wd;
            const bf16 *src = in ? X + ((((size_t)b * D + zi) * H + gy) * Wd + gx) * CIN + 8 * c : X;
            cp_async16(dst + L * LINE + c * P + r * 16, src, in);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    fetch(z0 - 1);
    fetch(z0);
    fetch(z0 + 1);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_slot;
    constexpr unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(COUT >> 3) << 17) | (8u << 24);
    bool ok = true;
    int issued = -1;  // the last row whose MMAs were committed
    for (int i = 0; i < nrows; ++i) {
        const int z = z0 + i;
        if (i >= 1) {  // row z - 1 done: its lines' slot is refilled below, its accumulator read
            if (!mbar_wait(&bar[(i - 1) & 1], (unsigned)((i - 1) >> 1) & 1u)) ok = false;
            if (!__syncthreads_and(ok ? 1 : 0)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
        }
        const bool more = i + 1 < nrows;
        if (more) fetch(z + 2);  // slot (z + 2) mod 4 held the lines of z - 2, last read by row z - 1
        // the lines of z - 1 .. z + 1 in place; the group just issued may stay in flight
        if (more)
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        else
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const unsigned d = tmem + (unsigned)((i & 1) * COUT);
            for (int tap = 0; tap < 27; ++tap) {
                const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                const unsigned char *Ab = ring + ((z + dz - 1) & 3) * SET + dy * LINE + dx * 16;
#pragma unroll
                for (int kk = 0; kk < CIN / 16; ++kk) {
                    const uint64_t ad = umma_desc(Ab + kk * 2 * P, P, 128);
                    const uint64_t bd = umma_desc(sB + tap * B_TAP + kk * 128, 128, CIN * 16);
                    const unsigned accumulate = (tap > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n"
                        " .reg .pred p;\n"
                        " setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
                        "}\n" ::"r"(d),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&bar[i & 1]))
                         : "memory");
        }
        issued = i;
        // row z - 1 out of the other accumulator while the MMAs of row z run;
        // its reads precede the next row's MMAs into it (barrier at the loop top)
        if (i >= 1)
            rows_epilogue<CIN, COUT, COUTR>(tmem + (unsigned)(((i - 1) & 1) * COUT), warp,
                                            Y + ((((size_t)b * D + z - 1) * H + y) * Wd + x0 + t) * COUTR, bias,
                                            relu);
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    // the last commit tracks every MMA issued before it: drain it (bounded)
    // before the accumulator is read or the tensor memory released
    if (issued >= 0 && !mbar_wait(&bar[issued & 1], (unsigned)(issued >> 1) & 1u)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int all_ok = __syncthreads_and(ok && issued == nrows - 1 ? 1 : 0);
    if (all_ok)
        rows_epilogue<CIN, COUT, COUTR>(tmem + (unsigned)((issued & 1) * COUT), warp,
                                        Y + ((((size_t)b * D + z0 + issued) * H + y) * Wd + x0 + t) * COUTR, bias,
                                        relu);
    else if (t == 0)
        atomicExch(status, 1);
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy into shared memory outlives the block
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

// ---- conv3d_wgrad_tc_kernel: the weight gradient on tcgen05.  As a GEMM,
// dW^T[(tap, ci)][co] = sum_v X[v + tap][ci] dY[v][co]: M = 128 rows of
// (tap, ci) pairs (128 / Cin taps per block), N = Cout, K = voxels.  Both
// operands come straight from the channels-last tensors, so they are staged
// MN-major: for each voxel the 128 (tap, ci) values, resp. the Cout values,
// are contiguous, in core matrices of 8 voxels x 8 channels (16 bytes per
// voxel).  For this layout the descriptor's leading offset is the step
// between core matrices along K (voxels) and its stride offset the 128-byte
// step along M or N (checked on a single-tile probe against a CPU GEMM).  A
// block takes 64-voxel chunks (four K = 16 MMAs) in a strided loop with two
// shared-memory stages, so the gather of one chunk overlaps the MMAs of the
// previous one; the [128 x Cout] FP32 accumulator lives in tensor memory and
// every thread finally adds its row to dW with FP32 atomics.  Waits are
// time-bounded; a block whose wait gives up stops issuing (as the forward
// kernel), drains its last commit with a bounded wait, adds nothing and sets
// the status word.  The voxel count must be a multiple of 64.
constexpr int kWgChunk = 64;

template <int CIN, int COUT>
__global__ void __launch_bounds__(128) conv3d_wgrad_tc_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ dY,
                                                              float *__restrict__ dW, long nvox, int D, int H, int Wd,
                                                              int lw, int lh, int ld, int *status)
{
    constexpr int TPB = 128 / CIN;  // taps per block
    constexpr int CA = CIN / 8, CB = COUT / 8;
    constexpr int A_EL = kWgChunk * 128, B_EL = kWgChunk * COUT;
    constexpr unsigned TCOLS = COUT < 32 ? 32 : COUT;
    extern __shared__ __align__(128) unsigned char wg_smem[];
    bf16 *sA = reinterpret_cast<bf16 *>(wg_smem);  // [2][64 voxels x 128 rows], MN-major
    bf16 *sB = sA + 2 * A_EL;                       // [2][64 voxels x Cout], MN-major
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ unsigned tmem_slot;
    const int t = threadIdx.x, warp = t >> 5;
    const int tap0 = blockIdx.y * TPB;
    const long n_chunks = nvox / kWgChunk;
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_slot;
    // f32 accumulate, bf16 A and B, A and B MN-major, N = Cout, M = 128
    constexpr unsigned idesc =
        (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((unsigned)(COUT >> 3) << 17) | (8u << 24);
    bool ok = true;
    int it = 0;
    for (long c = blockIdx.x; c < n_chunks; c += gridDim.x, ++it) {
        const int buf = it & 1;
        // the MMAs of chunk it - 2 read this stage; after a wait gives up the
        // block writes no stage and issues no MMA any more
        if (it >= 2) {
            if (!mbar_wait(&bar[buf], (unsigned)((it - 2) >> 1) & 1u)) ok = false;
            if (!__syncthreads_and(ok ? 1 : 0)) break;
        }
        bf16 *A = sA + buf * A_EL;
        bf16 *Bs = sB + buf * B_EL;
        const long v0 = c * kWgChunk;
        // A: 16-byte items (voxel k, tap tp, channel chunk cc), k mod 8 fastest
        // so that a warp's stores fill whole core matrices
#pragma unroll
        for (int j = 0; j < A_EL / 8 / 128; ++j) {
            const int i = t + 128 * j;
            const int klo = i & 7, r = i >> 3;
            const int cc = r % CA, r2 = r / CA;
            const int tp = r2 % TPB, khi = r2 / TPB;
            const int tap = tap0 + tp;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (tap < 27) {
                const long v = v0 + khi * 8 + klo;
                // (x, y, z) by shifts when W, H and D are powers of two (lw, lh, ld >= 0)
                int x, y, z;
                if (lw >= 0 && lh >= 0 && ld >= 0) {
                    x = (int)v & (Wd - 1);
                    y = (int)(v >> lw) & (H - 1);
                    z = (int)(v >> (lw + lh)) & (D - 1);
                } else {
                    x = (int)(v % Wd);
                    const long q = v / Wd;
                    y = (int)(q % H);
                    z = (int)((q / H) % D);
                }
                const int gx = x + tap % 3 - 1, gy = y + (tap / 3) % 3 - 1, gz = z + tap / 9 - 1;
                // the shifted voxel's offset from v, when it lies inside the volume
                if ((unsigned)gx < (unsigned)Wd && (unsigned)gy < (unsigned)H && (unsigned)gz < (unsigned)D)
                    val = __ldg(reinterpret_cast<const uint4 *>(
                                    X + (v + ((long)(gz - z) * H + (gy - y)) * Wd + (gx - x)) * CIN) +
                                cc);
            }
            *reinterpret_cast<uint4 *>(A + (khi * 16 + tp * CA + cc) * 64 + klo * 8) = val;
        }
        // B: (voxel k, channel chunk cc) of dY
        for (int i = t; i < B_EL / 8; i += 128) {
            const int klo = i & 7, r = i >> 3;
            const int cc = r % CB, khi = r / CB;
            const long v = v0 + khi * 8 + klo;
            *reinterpret_cast<uint4 *>(Bs + (khi * CB + cc) * 64 + klo * 8) =
                __ldg(reinterpret_cast<const uint4 *>(dY + v * COUT) + cc);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int kk = 0; kk < kWgChunk / 16; ++kk) {
                const uint64_t ad = umma_desc(A + kk * 2 * 16 * 64, 128 * 16, 128);
                const uint64_t bd = umma_desc(Bs + kk * 2 * CB * 64, COUT * 16, 128);
                const unsigned accumulate = (it > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n"
                    " .reg .pred p;\n"
                    " setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
                    "}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&bar[buf]))
                         : "memory");
        }
    }
    // the last commit tracks every MMA issued before it: drain it (bounded)
    // before the accumulator is read or the tensor memory released (after a
    // break, `it` is the chunk that issued nothing, so it - 1 is the last commit)
    if (it > 0 && !mbar_wait(&bar[(it - 1) & 1], (unsigned)((it - 1) >> 1) & 1u)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int all_ok = __syncthreads_and(ok ? 1 : 0);
    const int tap = tap0 + t / CIN, ci = t % CIN;
    if (all_ok && it > 0) {
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 16) {
            unsigned r[16];
            const unsigned addr = tmem + ((unsigned)(32 * warp) << 16) + (unsigned)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (tap < 27) {
                float *w = dW + ((size_t)tap * COUT + c0) * CIN + ci;
#pragma unroll
                for (int c = 0; c < 16; ++c) atomicAdd(w + (size_t)c * CIN, __uint_as_float(r[c]));
            }
        }
    } else if (!all_ok && t == 0) {
        atomicExch(status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

// dW for the narrow layers: one block per (tap, co, ci) triple range, FP32 sums
__global__ void conv3d_wgrad_direct_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ dY,
                                           float *__restrict__ dW, int cin, int cout, long nvox, int D, int H,
                                           int Wd)
{
    // blockIdx.y = tap, blockIdx.z = co * cin + ci; blockIdx.x strides over voxels
    const int tap = blockIdx.y, co = blockIdx.z / cin, ci = blockIdx.z % cin;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    float s = 0.0f;
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvox; v += (long)gridDim.x * blockDim.x) {
        const int x = (int)(v % Wd);
        long r = v / Wd;
        const int y = (int)(r % H);
        r /= H;
        const int z = (int)(r % D);
        const long b = r / D;
        const int gx = x + dx, gy = y + dy, gz = z + dz;
        if ((unsigned)gx < (unsigned)Wd && (unsigned)gy < (unsigned)H && (unsigned)gz < (unsigned)D)
            s = fmaf(__bfloat162float(dY[v * cout + co]),
                     __bfloat162float(X[((((size_t)b * D + gz) * H + gy) * Wd + gx) * cin + ci]), s);
    }
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(dW + ((size_t)tap * cout + co) * cin + ci, s);
    }
}

// W'[t][ci][co] = W[26 - t][co][ci]: the weights of the data-gradient convolution
__global__ void weight_flip_kernel(const bf16 *__restrict__ W, bf16 *__restrict__ Wf, int cin, int cout)
{
    const int n = 27 * cin * cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int t = i / (cin * cout), r = i - t * cin * cout;
        const int ci = r / cout, co = r - ci * cout;
        Wf[i] = W[((size_t)(26 - t) * cout + co) * cin + ci];
    }
}

// ---- elementwise / reduction helpers of the network (channels-last) -------
__global__ void relu_bwd_kernel(bf16 *__restrict__ dy, const bf16 *__restrict__ y, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        if (!(__bfloat162float(y[i]) > 0.0f)) dy[i] = __float2bfloat16_rn(0.0f);
}

// 2x2x2 average pooling: [B][D][H][W][C] -> [B][D/2][H/2][W/2][C]
__global__ void avgpool2_kernel(const bf16 *__restrict__ x, bf16 *__restrict__ y, long n_out, int D, int H, int W,
                                int C)
{
    const int Dh = D / 2, Hh = H / 2, Wh = W / 2;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n_out; i += (long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long r = i / C;
        const int xo = (int)(r % Wh);
        r /= Wh;
        const int yo = (int)(r % Hh);
        r /= Hh;
        const int zo = (int)(r % Dh);
        const long b = r / Dh;
        float s = 0.0f;
        for (int d = 0; d < 8; ++d) {
            const int zz = 2 * zo + (d >> 2), yy = 2 * yo + ((d >> 1) & 1), xx = 2 * xo + (d & 1);
            s += __bfloat162float(x[((((size_t)b * D + zz) * H + yy) * W + xx) * C + c]);
        }
        y[i] = __float2bfloat16_rn(0.125f * s);
    }
}

// its transpose: dx[v] = dy[v / 2] / 8
__global__ void avgpool2_bwd_kernel(const bf16 *__restrict__ dy, bf16 *__restrict__ dx, long n_in, int D, int H, int W,
                                    int C)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n_in; i += (long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long r = i / C;
        const int xx = (int)(r % W);
        r /= W;
        const int yy = (int)(r % H);
        r /= H;
        const int zz = (int)(r % D);
        const long b = r / D;
        const size_t o = ((((size_t)b * (D / 2) + zz / 2) * (H / 2) + yy / 2) * (W / 2) + xx / 2) * C + c;
        dx[i] = __float2bfloat16_rn(0.125f * __bfloat162float(dy[o]));
    }
}

// nearest 2x upsampling [B][D][H][W][C] -> [B][2D][2H][2W][C], optionally adding `skip`
__global__ void upsample2_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ skip, bf16 *__restrict__ y,
                                 long n_out, int D, int H, int W, int C)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n_out; i += (long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long r = i / C;
        const int xx = (int)(r % (2 * W));
        r /= 2 * W;
        const int yy = (int)(r % (2 * H));
        r /= 2 * H;
        const int zz = (int)(r % (2 * D));
        const long b = r / (2 * D);
        float v = __bfloat162float(x[((((size_t)b * D + zz / 2) * H + yy / 2) * W + xx / 2) * C + c]);
        if (skip) v += __bfloat162float(skip[i]);
        y[i] = __float2bfloat16_rn(v);
    }
}

// its transpose: dx[u] = sum of the 8 children of u
__global__ void upsample2_bwd_kernel(const bf16 *__restrict__ dy, bf16 *__restrict__ dx, long n_in, int D, int H,
                                     int W, int C)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n_in; i += (long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long r = i / C;
        const int xo = (int)(r % W);
        r /= W;
        const int yo = (int)(r % H);
        r /= H;
        const int zo = (int)(r % D);
        const long b = r / D;
        float s = 0.0f;
        for (int d = 0; d < 8; ++d) {
            const int zz = 2 * zo + (d >> 2), yy = 2 * yo + ((d >> 1) & 1), xx = 2 * xo + (d & 1);
            s += __bfloat162float(dy[((((size_t)b * 2 * D + zz) * 2 * H + yy) * 2 * W + xx) * C + c]);
        }
        dx[i] = __float2bfloat16_rn(s);
    }
}

// ---- the same four maps on 8 channels (16 bytes) per thread, for C a
// multiple of 8 and fewer than 2^31 chunks (32-bit index arithmetic);
// sums in FP32, one rounding to bf16, as the scalar kernels above
__device__ __forceinline__ void bf8_to_f(const uint4 &u, float (&f)[8])
{
    const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 p = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[k]));
        f[2 * k] = p.x;
        f[2 * k + 1] = p.y;
    }
}

__device__ __forceinline__ uint4 f_to_bf8(const float (&f)[8])
{
    unsigned w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const __nv_bfloat162 p = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
        w[k] = *reinterpret_cast<const unsigned *>(&p);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// chunk i of an output of [B][Do][Ho][Wo][C8 chunks] -> (b, z, y, x, c)
struct Chunk {
    int b, z, y, x, c;
};

__device__ __forceinline__ Chunk chunk_of(unsigned i, int C8, int Wo, int Ho, int Do)
{
    Chunk k;
    k.c = (int)(i % (unsigned)C8);
    unsigned r = i / (unsigned)C8;
    k.x = (int)(r % (unsigned)Wo);
    r /= (unsigned)Wo;
    k.y = (int)(r % (unsigned)Ho);
    r /= (unsigned)Ho;
    k.z = (int)(r % (unsigned)Do);
    k.b = (int)(r / (unsigned)Do);
    return k;
}

__global__ void avgpool2_v8_kernel(const uint4 *__restrict__ x, uint4 *__restrict__ y, unsigned n, int D, int H, int W,
                                   int C8)
{
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Chunk k = chunk_of(i, C8, W / 2, H / 2, D / 2);
        float s[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int zz = 2 * k.z + (d >> 2), yy = 2 * k.y + ((d >> 1) & 1), xx = 2 * k.x + (d & 1);
            float f[8];
            bf8_to_f(x[((((size_t)k.b * D + zz) * H + yy) * W + xx) * C8 + k.c], f);
#pragma unroll
            for (int e = 0; e < 8; ++e) s[e] += f[e];
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) s[e] *= 0.125f;
        y[i] = f_to_bf8(s);
    }
}

__global__ void avgpool2_bwd_v8_kernel(const uint4 *__restrict__ dy, uint4 *__restrict__ dx, unsigned n, int D, int H,
                                       int W, int C8)
{
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Chunk k = chunk_of(i, C8, W, H, D);
        float f[8];
        bf8_to_f(dy[((((size_t)k.b * (D / 2) + k.z / 2) * (H / 2) + k.y / 2) * (W / 2) + k.x / 2) * C8 + k.c], f);
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] *= 0.125f;
        dx[i] = f_to_bf8(f);
    }
}

__global__ void upsample2_v8_kernel(const uint4 *__restrict__ x, const uint4 *__restrict__ skip, uint4 *__restrict__ y,
                                    unsigned n, int D, int H, int W, int C8)
{
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Chunk k = chunk_of(i, C8, 2 * W, 2 * H, 2 * D);
        const uint4 v = x[((((size_t)k.b * D + k.z / 2) * H + k.y / 2) * W + k.x / 2) * C8 + k.c];
        if (skip) {
            float f[8], g[8];
            bf8_to_f(v, f);
            bf8_to_f(skip[i], g);
#pragma unroll
            for (int e = 0; e < 8; ++e) f[e] += g[e];
            y[i] = f_to_bf8(f);
        } else {
            y[i] = v;
        }
    }
}

__global__ void upsample2_bwd_v8_kernel(const uint4 *__restrict__ dy, uint4 *__restrict__ dx, unsigned n, int D,
                                        int H, int W, int C8)
{
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Chunk k = chunk_of(i, C8, W, H, D);
        float s[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int zz = 2 * k.z + (d >> 2), yy = 2 * k.y + ((d >> 1) & 1), xx = 2 * k.x + (d & 1);
            float f[8];
            bf8_to_f(dy[((((size_t)k.b * 2 * D + zz) * 2 * H + yy) * 2 * W + xx) * C8 + k.c], f);
#pragma unroll
            for (int e = 0; e < 8; ++e) s[e] += f[e];
        }
        dx[i] = f_to_bf8(s);
    }
}

__global__ void add_bf16_kernel(const bf16 *__restrict__ a, const bf16 *__restrict__ b, bf16 *__restrict__ y, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

// mode 0: f32 -> bf16, 1: bf16 -> f32, 2: y(f32) = a(f32) + x(bf16) (the residual output)
__global__ void cast_kernel(const void *__restrict__ x, void *__restrict__ y, const float *__restrict__ a, long n,
                            int mode)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        if (mode == 0)
            ((bf16 *)y)[i] = __float2bfloat16_rn(((const float *)x)[i]);
        else if (mode == 1)
            ((float *)y)[i] = __bfloat162float(((const bf16 *)x)[i]);
        else
            ((float *)y)[i] = a[i] + __bfloat162float(((const bf16 *)x)[i]);
    }
}

// db[c] = sum over voxels of dy[v][c]
__global__ void bias_grad_kernel(const bf16 *__restrict__ dy, float *__restrict__ db, long nvox, int C)
{
    const int c = blockIdx.y;
    float s = 0.0f;
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvox; v += (long)gridDim.x * blockDim.x)
        s += __bfloat162float(dy[v * C + c]);
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(db + c, s);
    }
}

// mean squared error of out against target; grad = 2 (out - target) / n as bf16,
// loss[0] += sum (out - target)^2 / n
__global__ void mse_kernel(const float *__restrict__ out, const float *__restrict__ target, bf16 *__restrict__ grad,
                           float *__restrict__ loss, long n)
{
    const float inv = 1.0f / (float)n;
    float s = 0.0f;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float d = out[i] - target[i];
        s = fmaf(d * inv, d, s);
        if (grad) grad[i] = __float2bfloat16_rn(2.0f * d * inv);
    }
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(loss, s);
    }
}

// Adam on FP32 master parameters; refreshes their bf16 copy (may be NULL)
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, bf16 *__restrict__ p16, long n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        p[i] = pi;
        if (p16) p16[i] = __float2bfloat16_rn(pi);
    }
}

long grid_for(long n)
{
    return std::max<long>(1, std::min<long>((n + 255) / 256, (long)device_sm_count() * 16));
}

template <int CIN, int COUT, int COUTR = COUT>
cudaError_t conv_tc_launch(const bf16 *X, const bf16 *W, const float *bias, bf16 *Y, int B, int D, int H, int Wd,
                           int relu, cudaStream_t s)
{
    const Tile tl = conv_tile(Wd, H);
    const size_t smem = (size_t)2 * (128 * CIN + COUT * CIN) * sizeof(bf16);
    auto k = conv3d_tc_kernel<CIN, COUT, COUTR>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int *status = nullptr;
    e = status_word(&status);
    if (e != cudaSuccess) return e;
    const long blocks = (long)B * (D / tl.TZ) * (H / tl.TY) * (Wd / tl.TX);
    k<<<(unsigned)blocks, 128, smem, s>>>(X, W, bias, Y, D, H, Wd, relu, status);
    return cudaGetLastError();
}

template <int CIN, int COUT, int COUTR = COUT>
cudaError_t conv_rows_launch(const bf16 *X, const bf16 *W, const float *bias, bf16 *Y, int B, int D, int H, int Wd,
                             int relu, cudaStream_t s)
{
    const size_t smem = (size_t)4 * 3 * (CIN / 8) * 130 * 16 + (size_t)27 * COUT * CIN * sizeof(bf16);
    auto k = conv3d_tc_rows_kernel<CIN, COUT, COUTR>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int *status = nullptr;
    e = status_word(&status);
    if (e != cudaSuccess) return e;
    const long blocks = (long)B * ((D + kRowsZ - 1) / kRowsZ) * H * (Wd / 128);
    k<<<(unsigned)blocks, 128, smem, s>>>(X, W, bias, Y, D, H, Wd, relu, status);
    return cudaGetLastError();
}

template <int COUT>
cudaError_t conv_k27_launch(const bf16 *X, const bf16 *W, const float *bias, bf16 *Y, int B, int D, int H, int Wd,
                            int relu, cudaStream_t s)
{
    const Tile tl = conv_tile(Wd, H);
    int *status = nullptr;
    cudaError_t e = status_word(&status);
    if (e != cudaSuccess) return e;
    const long blocks = (long)B * (D / tl.TZ) * (H / tl.TY) * (Wd / tl.TX);
    conv3d_tc_k27_kernel<COUT><<<(unsigned)blocks, 128, 0, s>>>(X, W, bias, Y, D, H, Wd, relu, status);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t wgrad_tc_launch(const bf16 *X, const bf16 *dY, float *dW, int B, int D, int H, int Wd, cudaStream_t s)
{
    const size_t smem = (size_t)2 * kWgChunk * (128 + COUT) * sizeof(bf16);
    auto k = conv3d_wgrad_tc_kernel<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int *status = nullptr;
    e = status_word(&status);
    if (e != cudaSuccess) return e;
    const long nvox = (long)B * D * H * Wd;
    constexpr int groups = (27 + 128 / CIN - 1) / (128 / CIN);
    const long chunks = nvox / kWgChunk;
    const long per_group = std::max<long>(1, std::min<long>(chunks, (long)device_sm_count() * 4 / groups));
    auto log2_or_minus1 = [](int n) {
        int l = 0;
        while ((1 << l) < n) ++l;
        return (1 << l) == n ? l : -1;
    };
    k<<<dim3((unsigned)per_group, groups), 128, smem, s>>>(X, dY, dW, nvox, D, H, Wd, log2_or_minus1(Wd),
                                                           log2_or_minus1(H), log2_or_minus1(D), status);
    return cudaGetLastError();
}

}  // namespace

bool conv_supported(int cin, int cout)
{
    auto mma_ok = [](int c) { return c == 16 || c == 32 || c == 64; };
    if (mma_ok(cin) && mma_ok(cout)) return true;
    return (cin == 1 && cout == 16) || (cin == 16 && cout == 1);
}

cudaError_t launch_conv3d(const void *X, const void *W, const float *bias, void *Y, int B, int D, int H, int Wd,
                          int cin, int cout, int relu, cudaStream_t s)
{
    const bf16 *x = (const bf16 *)X, *w = (const bf16 *)W;
    bf16 *y = (bf16 *)Y;
    // 16 input channels on rows of 128 voxels: the row-pipelined kernel
    if (cin == 16 && Wd % 128 == 0) {
        if (cout == 16) return conv_rows_launch<16, 16>(x, w, bias, y, B, D, H, Wd, relu, s);
        if (cout == 32) return conv_rows_launch<16, 32>(x, w, bias, y, B, D, H, Wd, relu, s);
        if (cout == 1) return conv_rows_launch<16, 16, 1>(x, w, bias, y, B, D, H, Wd, relu, s);
    }
#define PYRO_CONV_CASE(ci, co)                                                      \
    if (cin == ci && cout == co) return conv_tc_launch<ci, co>(x, w, bias, y, B, D, H, Wd, relu, s);
    PYRO_CONV_CASE(16, 16)
    PYRO_CONV_CASE(16, 32)
    PYRO_CONV_CASE(16, 64)
    PYRO_CONV_CASE(32, 16)
    PYRO_CONV_CASE(32, 32)
    PYRO_CONV_CASE(32, 64)
    PYRO_CONV_CASE(64, 16)
    PYRO_CONV_CASE(64, 32)
    PYRO_CONV_CASE(64, 64)
#undef PYRO_CONV_CASE
    // the narrow layers on the tensor cores too: one input channel as a
    // K = 27 tap GEMM, one output channel as N = 16 with 15 zero rows
    if (cin == 1 && cout == 16) return conv_k27_launch<16>(x, w, bias, y, B, D, H, Wd, relu, s);
    if (cin == 16 && cout == 1) return conv_tc_launch<16, 16, 1>(x, w, bias, y, B, D, H, Wd, relu, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_conv3d_wgrad(const void *X, const void *dY, float *dW, int B, int D, int H, int Wd, int cin,
                                int cout, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(dW, 0, sizeof(float) * 27 * cin * cout, s);
    if (e != cudaSuccess) return e;
    const bf16 *x = (const bf16 *)X, *dy = (const bf16 *)dY;
    // the tensor-core kernel takes 64-voxel chunks (the shapes the convolutions
    // accept are multiples of 128 voxels); anything else runs on the CUDA cores
    const bool tc = ((long)B * D * H * Wd) % kWgChunk == 0;
#define PYRO_WG_CASE(ci, co) \
    if (tc && cin == ci && cout == co) return wgrad_tc_launch<ci, co>(x, dy, dW, B, D, H, Wd, s);
    PYRO_WG_CASE(16, 16)
    PYRO_WG_CASE(16, 32)
    PYRO_WG_CASE(16, 64)
    PYRO_WG_CASE(32, 16)
    PYRO_WG_CASE(32, 32)
    PYRO_WG_CASE(32, 64)
    PYRO_WG_CASE(64, 16)
    PYRO_WG_CASE(64, 32)
    PYRO_WG_CASE(64, 64)
#undef PYRO_WG_CASE
    const long nvox = (long)B * D * H * Wd;
    const long per = std::max<long>(1, std::min<long>((nvox + 255) / 256, 64));
    dim3 grid((unsigned)per, 27, cin * cout);
    conv3d_wgrad_direct_kernel<<<grid, 256, 0, s>>>(x, dy, dW, cin, cout, nvox, D, H, Wd);
    return cudaGetLastError();
}

cudaError_t launch_weight_flip(const void *W, void *Wf, int cin, int cout, cudaStream_t s)
{
    weight_flip_kernel<<<(27 * cin * cout + 255) / 256, 256, 0, s>>>((const bf16 *)W, (bf16 *)Wf, cin, cout);
    return cudaGetLastError();
}

cudaError_t launch_cnn_elementwise(int op, const void *a, const void *b, void *y, const float *f, long n, int D,
                                   int H, int W, int C, cudaStream_t s)
{
    const unsigned g = (unsigned)grid_for(n);
    const bool a16 = (((uintptr_t)a | (uintptr_t)b | (uintptr_t)y) & 15) == 0;
    if (op >= 1 && op <= 4 && C % 8 == 0 && n / 8 < (1L << 31) && a16) {  // 8 channels per thread
        const unsigned n8 = (unsigned)(n / 8), g8 = (unsigned)grid_for(n / 8);
        const int C8 = C / 8;
        switch (op) {
        case 1: avgpool2_v8_kernel<<<g8, 256, 0, s>>>((const uint4 *)a, (uint4 *)y, n8, D, H, W, C8); break;
        case 2: avgpool2_bwd_v8_kernel<<<g8, 256, 0, s>>>((const uint4 *)a, (uint4 *)y, n8, D, H, W, C8); break;
        case 3:
            upsample2_v8_kernel<<<g8, 256, 0, s>>>((const uint4 *)a, (const uint4 *)b, (uint4 *)y, n8, D, H, W, C8);
            break;
        default: upsample2_bwd_v8_kernel<<<g8, 256, 0, s>>>((const uint4 *)a, (uint4 *)y, n8, D, H, W, C8); break;
        }
        return cudaGetLastError();
    }
    switch (op) {
    case 0: relu_bwd_kernel<<<g, 256, 0, s>>>((bf16 *)y, (const bf16 *)a, n); break;
    case 1: avgpool2_kernel<<<g, 256, 0, s>>>((const bf16 *)a, (bf16 *)y, n, D, H, W, C); break;
    case 2: avgpool2_bwd_kernel<<<g, 256, 0, s>>>((const bf16 *)a, (bf16 *)y, n, D, H, W, C); break;
    case 3: upsample2_kernel<<<g, 256, 0, s>>>((const bf16 *)a, (const bf16 *)b, (bf16 *)y, n, D, H, W, C); break;
    case 4: upsample2_bwd_kernel<<<g, 256, 0, s>>>((const bf16 *)a, (bf16 *)y, n, D, H, W, C); break;
    case 5: add_bf16_kernel<<<g, 256, 0, s>>>((const bf16 *)a, (const bf16 *)b, (bf16 *)y, n); break;
    case 6: cast_kernel<<<g, 256, 0, s>>>(a, y, nullptr, n, 0); break;
    case 7: cast_kernel<<<g, 256, 0, s>>>(a, y, nullptr, n, 1); break;
    case 8: cast_kernel<<<g, 256, 0, s>>>(a, y, f, n, 2); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_bias_grad(const void *dy, float *db, long nvox, int C, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(db, 0, sizeof(float) * C, s);
    if (e != cudaSuccess) return e;
    const long per = std::max<long>(1, std::min<long>((nvox + 255) / 256, 128));
    bias_grad_kernel<<<dim3((unsigned)per, C), 256, 0, s>>>((const bf16 *)dy, db, nvox, C);
    return cudaGetLastError();
}

cudaError_t launch_mse(const float *out, const float *target, void *grad, float *loss, long n, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    mse_kernel<<<(unsigned)grid_for(n), 256, 0, s>>>(out, target, (bf16 *)grad, loss, n);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, void *p16, long n, float lr, float b1, float b2,
                        float eps, int step, cudaStream_t s)
{
    const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<(unsigned)grid_for(n), 256, 0, s>>>(p, g, m, v, (bf16 *)p16, n, lr, b1, b2, eps, bc1, bc2);
    return cudaGetLastError();
}

}  // namespace pyro
