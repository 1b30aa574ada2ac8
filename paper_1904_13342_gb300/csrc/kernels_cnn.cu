// Residual 3D CNN kernels (BF16 storage, FP32 accumulation): the learned
// initialiser placed in front of the TV iteration.  The paper has no such
// network; it is the "learned parts" extension of the reconstruction path.
//
// Activations are channels-last [B][D][H][W][C] bf16.  Weights are
// [27][Cout][Cin] bf16 (tap = (dz*3 + dy)*3 + dx, taps of a 3x3x3 window,
// stride 1, zero padding 1); master weights and gradients are FP32.
//
// conv3d_mma_kernel: implicit GEMM on the tensor cores with
// mma.sync.m16n8k16 (bf16 in, fp32 accumulate).  A block computes 128 output
// voxels (a TX x TY x TZ box) x Cout; its input halo ((TZ+2) x (TY+2) x
// (TX+2) voxels x Cin) is staged in shared memory with each voxel's channel
// vector padded by 8 so that the A-fragment loads of the 8 row groups fall
// in distinct banks.  The same kernel computes the data gradient with the
// spatially flipped, channel-transposed weights.
// conv3d_wgrad_mma_kernel: dW[tap][co][ci] = sum_v dY[v][co] X[v+tap][ci] as a
// GEMM with M = Cout, N = taps x Cin, K = voxels: a block owns a group of
// taps, walks a strided set of voxel tiles accumulating in registers, and
// adds its partial sums to dW with FP32 atomics once at the end.
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

template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) conv3d_mma_kernel(const bf16 *__restrict__ X,
                                                                  const bf16 *__restrict__ Wt,
                                                                  const float *__restrict__ bias,
                                                                  bf16 *__restrict__ Y, int D, int H, int Wd,
                                                                  int relu)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *halo = reinterpret_cast<bf16 *>(smem_raw);
    constexpr int CP = CIN + 8;
    const Tile tl = conv_tile(Wd, H);
    const int TX = tl.TX, TY = tl.TY, TZ = tl.TZ, HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
    const int tiles_x = Wd / TX, tiles_y = H / TY, tiles_z = D / TZ;
    int t = blockIdx.x;
    const int tx0 = (t % tiles_x) * TX;
    t /= tiles_x;
    const int ty0 = (t % tiles_y) * TY;
    t /= tiles_y;
    const int tz0 = (t % tiles_z) * TZ;
    const int b = t / tiles_z;
    constexpr int CH = CIN / 8;  // 16-byte chunks per voxel
    const int nvox = HZ * HY * HX;
    for (int e = threadIdx.x; e < nvox * CH; e += kConvThreads) {
        const int vox = e / CH, ch = e - vox * CH;
        const int hx = vox % HX, r = vox / HX;
        const int hy = r % HY, hz = r / HY;
        const int gx = tx0 + hx - 1, gy = ty0 + hy - 1, gz = tz0 + hz - 1;
        uint4 val = make_uint4(0u, 0u, 0u, 0u);
        if ((unsigned)gx < (unsigned)Wd && (unsigned)gy < (unsigned)H && (unsigned)gz < (unsigned)D)
            val = __ldg(reinterpret_cast<const uint4 *>(X + ((((size_t)b * D + gz) * H + gy) * Wd + gx) * CIN) + ch);
        *reinterpret_cast<uint4 *>(halo + (size_t)vox * CP + ch * 8) = val;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
    const int m0 = warp * 16 + g, m1 = m0 + 8;  // the two output voxels (rows) of this thread
    const int lz0 = m0 / (TX * TY), lz1 = m1 / (TX * TY);
    const int ly0 = (m0 / TX) % TY, lx0 = m0 % TX, ly1 = (m1 / TX) % TY, lx1 = m1 % TX;
    float acc[COUT / 8][4];
#pragma unroll
    for (int n = 0; n < COUT / 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.0f;
    for (int dz = 0; dz < 3; ++dz)
        for (int dy = 0; dy < 3; ++dy)
            for (int dx = 0; dx < 3; ++dx) {
                const int tap = (dz * 3 + dy) * 3 + dx;
                const bf16 *r0 = halo + (((lz0 + dz) * HY + ly0 + dy) * HX + lx0 + dx) * CP;
                const bf16 *r1 = halo + (((lz1 + dz) * HY + ly1 + dy) * HX + lx1 + dx) * CP;
                const bf16 *wt = Wt + (size_t)tap * COUT * CIN;
#pragma unroll
                for (int kc = 0; kc < CIN / 16; ++kc) {
                    const int c0 = kc * 16 + 2 * tg;
                    const unsigned a0 = *reinterpret_cast<const unsigned *>(r0 + c0);
                    const unsigned a1 = *reinterpret_cast<const unsigned *>(r1 + c0);
                    const unsigned a2 = *reinterpret_cast<const unsigned *>(r0 + c0 + 8);
                    const unsigned a3 = *reinterpret_cast<const unsigned *>(r1 + c0 + 8);
#pragma unroll
                    for (int n = 0; n < COUT / 8; ++n) {
                        const bf16 *wr = wt + (size_t)(n * 8 + g) * CIN + c0;
                        const unsigned b0 = __ldg(reinterpret_cast<const unsigned *>(wr));
                        const unsigned b1 = __ldg(reinterpret_cast<const unsigned *>(wr + 8));
                        mma_bf16(acc[n], a0, a1, a2, a3, b0, b1);
                    }
                }
            }
    const size_t o0 = ((((size_t)b * D + tz0 + lz0) * H + ty0 + ly0) * Wd + tx0 + lx0) * COUT;
    const size_t o1 = ((((size_t)b * D + tz0 + lz1) * H + ty0 + ly1) * Wd + tx0 + lx1) * COUT;
#pragma unroll
    for (int n = 0; n < COUT / 8; ++n) {
        const int co = n * 8 + 2 * tg;
        const float b0 = bias ? bias[co] : 0.0f, b1 = bias ? bias[co + 1] : 0.0f;
        float v0 = acc[n][0] + b0, v1 = acc[n][1] + b1, v2 = acc[n][2] + b0, v3 = acc[n][3] + b1;
        if (relu) {
            v0 = fmaxf(v0, 0.0f);
            v1 = fmaxf(v1, 0.0f);
            v2 = fmaxf(v2, 0.0f);
            v3 = fmaxf(v3, 0.0f);
        }
        *reinterpret_cast<unsigned *>(Y + o0 + co) = pack_bf16(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
        *reinterpret_cast<unsigned *>(Y + o1 + co) = pack_bf16(__float2bfloat16_rn(v2), __float2bfloat16_rn(v3));
    }
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
cudaError_t conv_mma_launch(const bf16 *X, const bf16 *W, const float *bias, bf16 *Y, int B, int D, int H, int Wd,
                            int relu, cudaStream_t s)
{
    const Tile tl = conv_tile(Wd, H);
    const size_t smem = (size_t)(tl.TZ + 2) * (tl.TY + 2) * (tl.TX + 2) * (CIN + 8) * sizeof(bf16);
    auto k = conv3d_mma_kernel<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long blocks = (long)B * (D / tl.TZ) * (H / tl.TY) * (Wd / tl.TX);
    k<<<(unsigned)blocks, kConvThreads, smem, s>>>(X, W, bias, Y, D, H, Wd, relu);
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
    if (cin == ci && cout == co) return conv_mma_launch<ci, co>(x, w, bias, y, B, D, H, Wd, relu, s);
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
