// Cosine / Parker weighting and ramp-type row filtering F^H K F (Eq. 4, Eq. 5).
//
// The filter runs two detector rows per complex FFT: z = p_1 + i p_2 is
// zero-padded to pn, transformed (decimation in frequency, so the spectrum
// comes out in bit-reversed order), multiplied by the real even K, and
// transformed back (decimation in time, bit-reversed in, natural out).
// Because K is real and even, the real part of the result is the filtered
// row 1 and the imaginary part row 2; no permutation pass is needed.  A
// persistent grid of CTAs walks over row pairs; all of one pair's FFT state
// lives in shared memory.  FP32 throughout, twiddles from sincospif.
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace pyro {

namespace {

__device__ __forceinline__ float cosine_weight(const WeightParams &w, float u, float v)
{
    return w.sdd / sqrtf(fmaf(w.sdd, w.sdd, fmaf(u, u, v * v)));
}

// Parker short-scan weight: beta from the first view, gamma the fan angle of
// the bin, delta the half fan angle (regions of the short scan pi + 2 delta).
__device__ __forceinline__ float parker_weight(float beta, float gamma, float delta)
{
    const float pi = 3.14159265358979323846f;
    if (beta < 0.0f) return 0.0f;
    if (beta <= 2.0f * (delta - gamma)) {
        const float s = sinpif(0.25f * beta / (delta - gamma));
        return s * s;
    }
    if (beta <= pi - 2.0f * gamma) return 1.0f;
    if (beta <= pi + 2.0f * delta) {
        const float s = sinpif(0.25f * (pi + 2.0f * delta - beta) / (delta + gamma));
        return s * s;
    }
    return 0.0f;
}

__device__ __forceinline__ float total_weight(const WeightParams &w, const BetaTable &bt, int view, int l, int k)
{
    const float u = ((float)k - w.cu) * w.su;
    const float v = ((float)l - w.cv) * w.sv;
    float r = w.cosine ? cosine_weight(w, u, v) : 1.0f;
    if (w.redund == PYRO_REDUND_FULL) r *= 0.5f;
    if (w.redund == PYRO_REDUND_PARKER) r *= parker_weight(bt.beta[view], atanf(u / w.sdd), w.delta);
    return r;
}

template <typename T>
__global__ void weights_kernel(T *__restrict__ sino, long n, const __grid_constant__ WeightParams w,
                               const __grid_constant__ BetaTable bt)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const int k = (int)(e % w.nu);
        const long r = e / w.nu;
        const int l = (int)(r % w.nv);
        const int view = (int)((r / w.nv) % w.n_views);
        sino[e] = to_storage<T>(to_float<T>(sino[e]) * total_weight(w, bt, view, l, k));
    }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b)  // a * conj(b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// Forward DIF FFT of length pn in shared memory: natural order in,
// bit-reversed order out.  tw[t] = exp(-2 pi i t / pn), t < pn/2.
__device__ void fft_dif(float2 *z, const float2 *tw, int pn, int log2pn)
{
    const int half_n = pn >> 1;
    for (int s = log2pn; s >= 1; --s) {
        const int half = 1 << (s - 1);
        const int tstride = pn >> s;  // twiddle index step for this length
        for (int i = threadIdx.x; i < half_n; i += blockDim.x) {
            const int pos = i & (half - 1);
            const int a = ((i >> (s - 1)) << s) + pos;
            const int b = a + half;
            const float2 x = z[a], y = z[b];
            z[a] = make_float2(x.x + y.x, x.y + y.y);
            z[b] = cmul(make_float2(x.x - y.x, x.y - y.y), tw[pos * tstride]);
        }
        __syncthreads();
    }
}

// Inverse DIT FFT (unnormalised): bit-reversed order in, natural order out.
__device__ void ifft_dit(float2 *z, const float2 *tw, int pn, int log2pn)
{
    const int half_n = pn >> 1;
    for (int s = 1; s <= log2pn; ++s) {
        const int half = 1 << (s - 1);
        const int tstride = pn >> s;
        for (int i = threadIdx.x; i < half_n; i += blockDim.x) {
            const int pos = i & (half - 1);
            const int a = ((i >> (s - 1)) << s) + pos;
            const int b = a + half;
            const float2 x = z[a];
            const float2 t = cmul_conj(z[b], tw[pos * tstride]);
            z[a] = make_float2(x.x + t.x, x.y + t.y);
            z[b] = make_float2(x.x - t.x, x.y - t.y);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int bitrev(int x, int bits)
{
    return (int)(__brev((unsigned)x) >> (32 - bits));
}

__device__ void init_twiddles(float2 *tw, int pn)
{
    for (int t = threadIdx.x; t < pn / 2; t += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)t / (float)pn, &s, &c);
        tw[t] = make_float2(c, -s);
    }
}

constexpr int kFilterThreads = 256;

template <typename TI, typename TO>
__global__ void __launch_bounds__(kFilterThreads) filter_kernel(const TI *__restrict__ in, TO *__restrict__ out,
                                                                const __grid_constant__ FilterParams p,
                                                                const __grid_constant__ BetaTable bt,
                                                                const float *__restrict__ customK)
{
    extern __shared__ float2 smem[];
    const int pn = p.pn, nu = p.nu;
    float2 *z = smem;
    float2 *tw = smem + pn;
    float *Kb = reinterpret_cast<float *>(tw + pn / 2);  // K in bit-reversed order, pn entries
    init_twiddles(tw, pn);
    for (int t = threadIdx.x; t < pn; t += blockDim.x) {
        const int m = bitrev(t, p.log2pn);
        const int mm = m <= pn / 2 ? m : pn - m;
        Kb[t] = customK ? customK[mm] : p.K[mm];
    }
    __syncthreads();
    const float inv_pn = 1.0f / (float)pn;
    const long n_pairs = (p.n_rows + 1) / 2;
    for (long pr = blockIdx.x; pr < n_pairs; pr += gridDim.x) {
        const long r0 = 2 * pr, r1 = r0 + 1;
        const bool has1 = r1 < p.n_rows;
        int view0 = 0, l0 = 0, view1 = 0, l1 = 0;
        if (p.apply_weights) {
            view0 = (int)((r0 / p.rows_per_view) % p.n_views);
            l0 = (int)(r0 % p.rows_per_view);
            view1 = (int)((r1 / p.rows_per_view) % p.n_views);
            l1 = (int)(r1 % p.rows_per_view);
        }
        for (int n = threadIdx.x; n < pn; n += blockDim.x) {
            float a = 0.0f, c = 0.0f;
            if (n < nu) {
                a = ld(in + r0 * nu + n);
                if (has1) c = ld(in + r1 * nu + n);
                if (p.apply_weights) {
                    a *= total_weight(p.w, bt, view0, l0, n);
                    if (has1) c *= total_weight(p.w, bt, view1, l1, n);
                }
            }
            z[n] = make_float2(a, c);
        }
        __syncthreads();
        fft_dif(z, tw, pn, p.log2pn);
        for (int t = threadIdx.x; t < pn; t += blockDim.x) {
            const float k = Kb[t] * inv_pn;
            z[t] = make_float2(z[t].x * k, z[t].y * k);
        }
        __syncthreads();
        ifft_dit(z, tw, pn, p.log2pn);
        for (int n = threadIdx.x; n < nu; n += blockDim.x) {
            out[r0 * nu + n] = to_storage<TO>(z[n].x);
            if (has1) out[r1 * nu + n] = to_storage<TO>(z[n].y);
        }
        __syncthreads();
    }
}

// dK[m] += c_m / pn * sum over row pairs of 1/2 Re(Z_m conj(Y_m) + Z_{-m} conj(Y_{-m})),
// Z = FFT(p_1 + i p_2), Y = FFT(g_1 + i g_2): the per-row sums
// Re(P_r[m] conj(G_r[m])) of both rows of the pair.
__global__ void __launch_bounds__(kFilterThreads) filter_grad_K_kernel(const float *__restrict__ p,
                                                                       const float *__restrict__ g,
                                                                       float *__restrict__ dK, long n_rows, int nu,
                                                                       int pn, int log2pn)
{
    extern __shared__ float2 smem[];
    float2 *z = smem;
    float2 *y = smem + pn;
    float2 *tw = y + pn;
    float *acc = reinterpret_cast<float *>(tw + pn / 2);  // pn/2 + 1
    init_twiddles(tw, pn);
    for (int m = threadIdx.x; m <= pn / 2; m += blockDim.x) acc[m] = 0.0f;
    __syncthreads();
    const long n_pairs = (n_rows + 1) / 2;
    for (long pr = blockIdx.x; pr < n_pairs; pr += gridDim.x) {
        const long r0 = 2 * pr, r1 = r0 + 1;
        const bool has1 = r1 < n_rows;
        for (int n = threadIdx.x; n < pn; n += blockDim.x) {
            float a = 0, b = 0, c = 0, d = 0;
            if (n < nu) {
                a = p[r0 * nu + n];
                c = g[r0 * nu + n];
                if (has1) {
                    b = p[r1 * nu + n];
                    d = g[r1 * nu + n];
                }
            }
            z[n] = make_float2(a, b);
            y[n] = make_float2(c, d);
        }
        __syncthreads();
        fft_dif(z, tw, pn, log2pn);
        fft_dif(y, tw, pn, log2pn);
        for (int m = threadIdx.x; m <= pn / 2; m += blockDim.x) {
            const int tm = bitrev(m, log2pn);
            const int tn = bitrev((pn - m) & (pn - 1), log2pn);
            const float2 s = cmul_conj(z[tm], y[tm]);
            const float2 t = cmul_conj(z[tn], y[tn]);
            acc[m] += 0.5f * (s.x + t.x);
        }
        __syncthreads();
    }
    for (int m = threadIdx.x; m <= pn / 2; m += blockDim.x) {
        const float c = (m == 0 || m == pn / 2) ? 1.0f : 2.0f;
        atomicAdd(dK + m, c / (float)pn * acc[m]);
    }
}

template <typename TI, typename TO>
cudaError_t filter_dispatch(const void *in, void *out, const FilterParams &p, const BetaTable &bt,
                            const float *customK, cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (size_t)p.pn * 3 / 2 + sizeof(float) * (size_t)p.pn;
    cudaError_t e = cudaFuncSetAttribute(filter_kernel<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, filter_kernel<TI, TO>, kFilterThreads, smem);
    if (e != cudaSuccess) return e;
    const long pairs = (p.n_rows + 1) / 2;
    const long grid = std::min<long>(pairs, (long)device_sm_count() * std::max(per_sm, 1));
    filter_kernel<TI, TO><<<(unsigned)grid, kFilterThreads, smem, s>>>((const TI *)in, (TO *)out, p, bt, customK);
    return cudaGetLastError();
}

template <typename TI>
cudaError_t filter_by_out(const void *in, void *out, const FilterParams &p, const BetaTable &bt, const float *K,
                          pyro_dtype out_dt, cudaStream_t s)
{
    switch (out_dt) {
    case PYRO_F32: return filter_dispatch<TI, float>(in, out, p, bt, K, s);
    case PYRO_F16: return filter_dispatch<TI, __half>(in, out, p, bt, K, s);
    case PYRO_BF16: return filter_dispatch<TI, __nv_bfloat16>(in, out, p, bt, K, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_weights(void *sino, int batch, const WeightParams &w, const BetaTable &beta, pyro_dtype dt,
                           cudaStream_t s)
{
    const long n = (long)batch * w.n_views * w.nv * w.nu;
    const long blocks = std::min<long>((n + 255) / 256, (long)device_sm_count() * 16);
    switch (dt) {
    case PYRO_F32:
        weights_kernel<float><<<(unsigned)blocks, 256, 0, s>>>((float *)sino, n, w, beta);
        break;
    case PYRO_F16:
        weights_kernel<__half><<<(unsigned)blocks, 256, 0, s>>>((__half *)sino, n, w, beta);
        break;
    case PYRO_BF16:
        weights_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, s>>>((__nv_bfloat16 *)sino, n, w, beta);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_filter(const void *in, void *out, const FilterParams &p, const BetaTable *beta,
                          const float *custom_K, pyro_dtype in_dt, pyro_dtype out_dt, cudaStream_t s)
{
    static const BetaTable zero_beta = {};
    const BetaTable &bt = beta ? *beta : zero_beta;
    switch (in_dt) {
    case PYRO_F32: return filter_by_out<float>(in, out, p, bt, custom_K, out_dt, s);
    case PYRO_F16: return filter_by_out<__half>(in, out, p, bt, custom_K, out_dt, s);
    case PYRO_BF16: return filter_by_out<__nv_bfloat16>(in, out, p, bt, custom_K, out_dt, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_filter_grad_K(const float *p, const float *g, float *dK, long n_rows, int nu, int pn, int log2pn,
                                 cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(dK, 0, sizeof(float) * (size_t)(pn / 2 + 1), s);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(float2) * (size_t)pn * 5 / 2 + sizeof(float) * (size_t)(pn / 2 + 1);
    e = cudaFuncSetAttribute(filter_grad_K_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, filter_grad_K_kernel, kFilterThreads, smem);
    if (e != cudaSuccess) return e;
    const long pairs = (n_rows + 1) / 2;
    const long grid = std::min<long>(pairs, (long)device_sm_count() * std::max(per_sm, 1));
    filter_grad_K_kernel<<<(unsigned)grid, kFilterThreads, smem, s>>>(p, g, dK, n_rows, nu, pn, log2pn);
    return cudaGetLastError();
}

}  // namespace pyro
