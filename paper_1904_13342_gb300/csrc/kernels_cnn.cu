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
// conv3d_wgrad_mma_kernel: dW[tap][co][ci] = sum_v dY[v][co] X[v+tap][ci] as a
// GEMM with M = Cout, N = taps x Cin, K = voxels on mma.sync.m16n8k16: a
// block owns a group of taps, walks a strided set of voxel tiles accumulating
// in registers, and adds its partial sums to dW with FP32 atomics at the end.
#include <cuda_bf16.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace pyro {

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_bf16(bf16 lo, bf16 hi)
{
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

constexpr int kConvThreads = 256;

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
// adds the bias and the ReLU.  Waits are time-bounded; a block whose wait
// gives up writes nothing and sets the status word.
__device__ __forceinline__ uint64_t umma_desc(const void *smem, unsigned lbo, unsigned sbo)
{
    uint64_t d = (uint64_t)((smem_addr(smem) >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;  // next core matrix along K
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;  // next group of 8 rows
    d |= (uint64_t)1 << 46;                      // descriptor version; no swizzle, base offset 0
    return d;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(128) conv3d_tc_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ Wt,
                                                        const float *__restrict__ bias, bf16 *__restrict__ Y, int D,
                                                        int H, int Wd, int relu, int *status)
{
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
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_slot;
    // f32 accumulate, bf16 A and B, both K-major, N = Cout, M = 128
    constexpr unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(COUT >> 3) << 17) | (8u << 24);
    bool ok = true;
    for (int tap = 0; tap < 27; ++tap) {
        const int buf = tap & 1;
        // the MMAs of tap - 2 read this stage
        if (tap >= 2 && !mbar_wait(&bar[buf], (unsigned)((tap - 2) >> 1) & 1u)) ok = false;
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
        const uint4 *wsrc = reinterpret_cast<const uint4 *>(Wt + (size_t)tap * COUT * CIN);
        for (int q = t; q < COUT * KCH; q += 128) {
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
    }
    // the last commit tracks every MMA issued before it
    if (!mbar_wait(&bar[26 & 1], (26 >> 1) & 1u)) ok = false;
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

// taps per wgrad block: enough to keep COUT x CIN x TP accumulators <= 64 per thread
__host__ __device__ constexpr int wgrad_taps(int cin, int cout)
{
    return cin * cout * 27 <= 64 * kConvThreads ? 27 : (cin * cout * 9 <= 64 * kConvThreads ? 9 : 3);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) conv3d_wgrad_mma_kernel(const bf16 *__restrict__ X,
                                                                        const bf16 *__restrict__ dY,
                                                                        float *__restrict__ dW, int B, int D, int H,
                                                                        int Wd)
{
    constexpr int TP = wgrad_taps(CIN, COUT);
    constexpr int MT = COUT / 16;                 // m tiles (output channels)
    constexpr int NT = TP * CIN / 8;              // n tiles (tap, 8 input channels)
    constexpr int PER_WARP = (MT * NT + 7) / 8;   // mma tiles per warp
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Tile tl = conv_tile(Wd, H);
    const int TX = tl.TX, TY = tl.TY, TZ = tl.TZ, HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
    constexpr int DYP = 128 + 8;                  // padded voxel stride of the transposed dY tile
    bf16 *dyt = reinterpret_cast<bf16 *>(smem_raw);                 // [COUT][DYP]
    bf16 *halo = dyt + COUT * DYP;                                  // [3*HY*HX][CIN + 8]
    constexpr int CP = CIN + 8;
    const int tap0 = blockIdx.y * TP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
    float acc[PER_WARP][4];
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0f;
    const int tiles_x = Wd / TX, tiles_y = H / TY, tiles_z = D / TZ;
    const long n_tiles = (long)B * tiles_z * tiles_y * tiles_x;
    for (long t0 = blockIdx.x; t0 < n_tiles; t0 += gridDim.x) {
        long t = t0;
        const int tx0 = (int)(t % tiles_x) * TX;
        t /= tiles_x;
        const int ty0 = (int)(t % tiles_y) * TY;
        t /= tiles_y;
        const int tz0 = (int)(t % tiles_z) * TZ;
        const int b = (int)(t / tiles_z);
        // dY tile transposed: dyt[co][m], m = (lz * TY + ly) * TX + lx
        for (int e = threadIdx.x; e < 128 * COUT; e += kConvThreads) {
            const int m = e / COUT, co = e - m * COUT;
            const int lz = m / (TX * TY), ly = (m / TX) % TY, lx = m % TX;
            dyt[co * DYP + m] = dY[((((size_t)b * D + tz0 + lz) * H + ty0 + ly) * Wd + tx0 + lx) * COUT + co];
        }
        constexpr int CH = CIN / 8;
        const int nvox = HZ * HY * HX;
        for (int e = threadIdx.x; e < nvox * CH; e += kConvThreads) {
            const int vox = e / CH, ch = e - vox * CH;
            const int hx = vox % HX, r = vox / HX;
            const int hy = r % HY, hz = r / HY;
            const int gx = tx0 + hx - 1, gy = ty0 + hy - 1, gz = tz0 + hz - 1;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if ((unsigned)gx < (unsigned)Wd && (unsigned)gy < (unsigned)H && (unsigned)gz < (unsigned)D)
                val = __ldg(reinterpret_cast<const uint4 *>(X + ((((size_t)b * D + gz) * H + gy) * Wd + gx) * CIN) +
                            ch);
            *reinterpret_cast<uint4 *>(halo + (size_t)vox * CP + ch * 8) = val;
        }
        __syncthreads();
#pragma unroll
        for (int kc = 0; kc < 8; ++kc) {  // K = 128 voxels in steps of 16
            const int v0 = kc * 16 + 2 * tg;  // voxels v0, v0+1 and v0+8, v0+9 of this thread's fragments
            const int lzA = v0 / (TX * TY), lyA = (v0 / TX) % TY, lxA = v0 % TX;
            const int lzB = (v0 + 8) / (TX * TY), lyB = ((v0 + 8) / TX) % TY, lxB = (v0 + 8) % TX;
#pragma unroll
            for (int i = 0; i < PER_WARP; ++i) {
                const int tile = warp + 8 * i;
                if (tile >= MT * NT) break;
                const int mt = tile / NT, nt = tile - mt * NT;
                const int co = mt * 16 + g;
                const unsigned a0 = *reinterpret_cast<const unsigned *>(dyt + co * DYP + v0);
                const unsigned a1 = *reinterpret_cast<const unsigned *>(dyt + (co + 8) * DYP + v0);
                const unsigned a2 = *reinterpret_cast<const unsigned *>(dyt + co * DYP + v0 + 8);
                const unsigned a3 = *reinterpret_cast<const unsigned *>(dyt + (co + 8) * DYP + v0 + 8);
                const int tap = tap0 + nt / (CIN / 8);
                const int ci = (nt % (CIN / 8)) * 8 + g;
                const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                // B[k = voxel][n = ci] = X[voxel + tap][ci]: voxels v0, v0+1 (same row) and v0+8, v0+9
                const bf16 *hA = halo + (((lzA + dz) * HY + lyA + dy) * HX + lxA + dx) * CP + ci;
                const bf16 *hB = halo + (((lzB + dz) * HY + lyB + dy) * HX + lxB + dx) * CP + ci;
                const unsigned b0 = pack_bf16(hA[0], hA[CP]);
                const unsigned b1 = pack_bf16(hB[0], hB[CP]);
                mma_bf16(acc[i], a0, a1, a2, a3, b0, b1);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i) {
        const int tile = warp + 8 * i;
        if (tile >= MT * NT) break;
        const int mt = tile / NT, nt = tile - mt * NT;
        const int tap = tap0 + nt / (CIN / 8);
        const int ci = (nt % (CIN / 8)) * 8 + 2 * tg;
        const int co = mt * 16 + g;
        float *w = dW + (size_t)tap * COUT * CIN;
        atomicAdd(w + (size_t)co * CIN + ci, acc[i][0]);
        atomicAdd(w + (size_t)co * CIN + ci + 1, acc[i][1]);
        atomicAdd(w + (size_t)(co + 8) * CIN + ci, acc[i][2]);
        atomicAdd(w + (size_t)(co + 8) * CIN + ci + 1, acc[i][3]);
    }
}

// Direct convolution on the CUDA cores for the narrow layers (Cin or Cout
// below 16): one thread per output voxel, all output channels.
template <int CIN, int COUT>
__global__ void conv3d_direct_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ Wt,
                                     const float *__restrict__ bias, bf16 *__restrict__ Y, long nvox, int D, int H,
                                     int Wd, int relu)
{
    __shared__ float w[27 * COUT * CIN];
    for (int i = threadIdx.x; i < 27 * COUT * CIN; i += blockDim.x) w[i] = __bfloat162float(Wt[i]);
    __syncthreads();
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvox; v += (long)gridDim.x * blockDim.x) {
        const int x = (int)(v % Wd);
        long r = v / Wd;
        const int y = (int)(r % H);
        r /= H;
        const int z = (int)(r % D);
        const long b = r / D;
        float acc[COUT];
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = bias ? bias[co] : 0.0f;
        for (int dz = 0; dz < 3; ++dz) {
            const int gz = z + dz - 1;
            if ((unsigned)gz >= (unsigned)D) continue;
            for (int dy = 0; dy < 3; ++dy) {
                const int gy = y + dy - 1;
                if ((unsigned)gy >= (unsigned)H) continue;
                for (int dx = 0; dx < 3; ++dx) {
                    const int gx = x + dx - 1;
                    if ((unsigned)gx >= (unsigned)Wd) continue;
                    const int tap = (dz * 3 + dy) * 3 + dx;
                    const bf16 *xp = X + ((((size_t)b * D + gz) * H + gy) * Wd + gx) * CIN;
#pragma unroll
                    for (int ci = 0; ci < CIN; ++ci) {
                        const float xv = __bfloat162float(xp[ci]);
#pragma unroll
                        for (int co = 0; co < COUT; ++co) acc[co] = fmaf(w[(tap * COUT + co) * CIN + ci], xv, acc[co]);
                    }
                }
            }
        }
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
            const float o = relu ? fmaxf(acc[co], 0.0f) : acc[co];
            Y[v * COUT + co] = __float2bfloat16_rn(o);
        }
    }
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

template <int CIN, int COUT>
cudaError_t conv_tc_launch(const bf16 *X, const bf16 *W, const float *bias, bf16 *Y, int B, int D, int H, int Wd,
                           int relu, cudaStream_t s)
{
    const Tile tl = conv_tile(Wd, H);
    const size_t smem = (size_t)2 * (128 * CIN + COUT * CIN) * sizeof(bf16);
    auto k = conv3d_tc_kernel<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int *status = nullptr;
    e = status_word(&status);
    if (e != cudaSuccess) return e;
    const long blocks = (long)B * (D / tl.TZ) * (H / tl.TY) * (Wd / tl.TX);
    k<<<(unsigned)blocks, 128, smem, s>>>(X, W, bias, Y, D, H, Wd, relu, status);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t wgrad_mma_launch(const bf16 *X, const bf16 *dY, float *dW, int B, int D, int H, int Wd, cudaStream_t s)
{
    const Tile tl = conv_tile(Wd, H);
    constexpr int TP = wgrad_taps(CIN, COUT);
    const size_t smem =
        ((size_t)COUT * (128 + 8) + (size_t)(tl.TZ + 2) * (tl.TY + 2) * (tl.TX + 2) * (CIN + 8)) * sizeof(bf16);
    auto k = conv3d_wgrad_mma_kernel<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long n_tiles = (long)B * (D / tl.TZ) * (H / tl.TY) * (Wd / tl.TX);
    const long per_group = std::max<long>(1, std::min<long>(n_tiles, (long)device_sm_count() * 4 / (27 / TP) + 1));
    dim3 grid((unsigned)per_group, 27 / TP);
    k<<<grid, kConvThreads, smem, s>>>(X, dY, dW, B, D, H, Wd);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t direct_launch(const bf16 *X, const bf16 *W, const float *bias, bf16 *Y, int B, int D, int H, int Wd,
                          int relu, cudaStream_t s)
{
    const long nvox = (long)B * D * H * Wd;
    const long blocks = std::min<long>((nvox + 255) / 256, (long)device_sm_count() * 16);
    conv3d_direct_kernel<CIN, COUT><<<(unsigned)blocks, 256, 0, s>>>(X, W, bias, Y, nvox, D, H, Wd, relu);
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
    if (cin == 1 && cout == 16) return direct_launch<1, 16>(x, w, bias, y, B, D, H, Wd, relu, s);
    if (cin == 16 && cout == 1) return direct_launch<16, 1>(x, w, bias, y, B, D, H, Wd, relu, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_conv3d_wgrad(const void *X, const void *dY, float *dW, int B, int D, int H, int Wd, int cin,
                                int cout, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(dW, 0, sizeof(float) * 27 * cin * cout, s);
    if (e != cudaSuccess) return e;
    const bf16 *x = (const bf16 *)X, *dy = (const bf16 *)dY;
#define PYRO_WG_CASE(ci, co) \
    if (cin == ci && cout == co) return wgrad_mma_launch<ci, co>(x, dy, dW, B, D, H, Wd, s);
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
