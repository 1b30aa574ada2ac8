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
// A scan over any range R <= 2 pi takes the same form with delta = (R - pi) / 2:
// the overlap at the start, beta <= R - pi - 2 gamma, holds exactly the rays
// whose line is measured again before R, and the overlap at the end their
// partners; every other ray is measured once (weight 1).  For those delta the
// start overlap can be empty (delta <= gamma), hence the first guard.
__device__ __forceinline__ float parker_weight(float beta, float gamma, float delta)
{
    const float pi = 3.14159265358979323846f;
    if (beta < 0.0f) return 0.0f;
    if (delta - gamma > 0.0f && beta <= 2.0f * (delta - gamma)) {
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
    if (w.redund == PYRO_REDUND_PARKER || w.redund == PYRO_REDUND_SCAN)
        r *= parker_weight(bt.beta[view], atanf(u / w.sdd), w.delta);
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

// Cosine weight times a redundancy table W_red[view][k] (learnable weights,
// one value per view and detector column), in place.
template <typename T>
__global__ void weights_table_kernel(T *__restrict__ sino, long n, const __grid_constant__ WeightParams w,
                                     const float *__restrict__ table)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const int k = (int)(e % w.nu);
        const long r = e / w.nu;
        const int l = (int)(r % w.nv);
        const int view = (int)((r / w.nv) % w.n_views);
        float f = table[(size_t)view * w.nu + k];
        if (w.cosine) f *= cosine_weight(w, ((float)k - w.cu) * w.su, ((float)l - w.cv) * w.sv);
        sino[e] = to_storage<T>(to_float<T>(sino[e]) * f);
    }
}

// out[view][k] = sum over the batch and the rows l of a[b][view][l][k] g[b][view][l][k]:
// one thread per (view, k), reading rows along k (coalesced)
__global__ void __launch_bounds__(256) redundancy_grad_kernel(const float *__restrict__ a,
                                                              const float *__restrict__ g, float *__restrict__ out,
                                                              int batch, int n_views, int nv, int nu)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int view = blockIdx.y;
    if (k >= nu) return;
    float s0 = 0.0f, s1 = 0.0f;
    for (int b = 0; b < batch; ++b) {
        const size_t base = (((size_t)b * n_views + view) * nv) * nu + k;
        int l = 0;
        for (; l + 1 < nv; l += 2) {
            s0 = fmaf(a[base + (size_t)l * nu], g[base + (size_t)l * nu], s0);
            s1 = fmaf(a[base + (size_t)(l + 1) * nu], g[base + (size_t)(l + 1) * nu], s1);
        }
        if (l < nv) s0 = fmaf(a[base + (size_t)l * nu], g[base + (size_t)l * nu], s0);
    }
    out[(size_t)view * nu + k] = s0 + s1;
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

// ---- Stockham autosort FFT (natural order in and out), radix 8 passes in
// registers, a final radix-4 or radix-2 pass when log2(pn) is not a
// multiple of 3.  Pass i reads element j + r*pn/R of buffer `src`, applies
// the twiddles w^(r k), w = exp(-2 pi i / (Ns R)), k = j mod Ns, runs an
// R-point DFT and writes X[r] to (j / Ns) Ns R + k + r Ns of `dst`.
// Pass i (0-based) of a length-2^L transform: radix 8 with Ns = 8^i, except
// the last pass which has radix 2^(L - 3 (P-1)); its twiddle table (Ns
// entries) starts at (8^i - 1) / 7.
__host__ __device__ inline int n_passes(int log2pn)
{
    return (log2pn + 2) / 3;
}

__host__ __device__ inline int twiddle_total(int log2pn)
{
    const int P = n_passes(log2pn);
    return ((1 << (3 * P)) - 1) / 7;  // sum of 8^i, i < P (bounds the last pass's Ns too)
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul_negi(float2 a) { return make_float2(a.y, -a.x); }  // a * (-i)

// R-point DFTs X[k] = sum v[n] exp(-2 pi i n k / R), natural order out
__device__ __forceinline__ void dft4(float2 *v)
{
    const float2 e0 = cadd(v[0], v[2]), e1 = cadd(v[1], v[3]);
    const float2 o0 = csub(v[0], v[2]), o1 = mul_negi(csub(v[1], v[3]));
    v[0] = cadd(e0, e1);
    v[2] = csub(e0, e1);
    v[1] = cadd(o0, o1);
    v[3] = csub(o0, o1);
}

__device__ __forceinline__ void dft8(float2 *v)
{
    const float h = 0.70710678118654752440f;
    float2 a[4], c[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        a[n] = cadd(v[n], v[n + 4]);
        c[n] = csub(v[n], v[n + 4]);
    }
    // c[n] *= exp(-2 pi i n / 8)
    c[1] = make_float2(h * (c[1].x + c[1].y), h * (c[1].y - c[1].x));
    c[2] = mul_negi(c[2]);
    c[3] = make_float2(h * (c[3].y - c[3].x), -h * (c[3].x + c[3].y));
    dft4(a);
    dft4(c);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = a[k];
        v[2 * k + 1] = c[k];
    }
}

// Shared-memory index with one pad slot per 8 complex values: spreads the
// strided Stockham stores over all banks.
__device__ __forceinline__ int sp(int i)
{
    return i + (i >> 3);
}

// One pass over `groups` independent transforms of length pn stored back to back.
template <int R>
__device__ __forceinline__ void stockham_pass(const float2 *src, float2 *dst, const float2 *tw, int pn, int ns,
                                              int groups)
{
    const int nb = pn / R;
    for (int b = threadIdx.x; b < groups * nb; b += blockDim.x) {
        const int g = b / nb, j = b - g * nb;
        const float2 *s = src + g * sp(pn);
        float2 *d = dst + g * sp(pn);
        const int k = j & (ns - 1);
        float2 v[R];
        if (ns == 1) {  // the first pass: every twiddle is 1
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = s[sp(j + r * nb)];
        } else {
            const float2 w1 = tw[k];
            float2 w = w1;
            v[0] = s[sp(j)];
#pragma unroll
            for (int r = 1; r < R; ++r) {
                v[r] = cmul(s[sp(j + r * nb)], w);
                if (r + 1 < R) w = cmul(w, w1);
            }
        }
        if (R == 8) dft8(v);
        if (R == 4) dft4(v);
        if (R == 2) {
            const float2 t = v[0];
            v[0] = cadd(t, v[1]);
            v[1] = csub(t, v[1]);
        }
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[sp(base + r * ns)] = v[r];
    }
}

// Full forward transform of `groups` rows; returns the buffer holding the
// result.  LOG2 > 0 fixes log2(pn) at compile time (the passes unrolled,
// their strides constants); 0 takes it from log2pn.
template <int LOG2>
__device__ __forceinline__ float2 *stockham_fft(float2 *a, float2 *b, const float2 *tw, int log2pn, int pn, int groups)
{
    if (LOG2 > 0) {
        log2pn = LOG2;
        pn = 1 << LOG2;
    }
    const int P = n_passes(log2pn);
#pragma unroll
    for (int i = 0; i < (LOG2 > 0 ? (LOG2 + 2) / 3 : P); ++i) {
        const int ns = 1 << (3 * i);
        const float2 *t = tw + (ns - 1) / 7;
        const int rb = i < P - 1 ? 3 : log2pn - 3 * (P - 1);
        if (rb == 3) stockham_pass<8>(a, b, t, pn, ns, groups);
        else if (rb == 2) stockham_pass<4>(a, b, t, pn, ns, groups);
        else stockham_pass<2>(a, b, t, pn, ns, groups);
        __syncthreads();
        float2 *tmp = a;
        a = b;
        b = tmp;
    }
    return a;
}

__device__ void init_stockham_twiddles(float2 *tw, int log2pn)
{
    const int P = n_passes(log2pn);
    for (int i = 0; i < P; ++i) {
        const int ns = 1 << (3 * i);
        const int rb = i < P - 1 ? 3 : log2pn - 3 * (P - 1);
        const int nr = ns << rb;
        for (int k = threadIdx.x; k < ns; k += blockDim.x) {
            float s, c;
            sincospif(2.0f * (float)k / (float)nr, &s, &c);
            tw[(ns - 1) / 7 + k] = make_float2(c, -s);
        }
    }
}

// rows per CTA pass: enough pairs to fill a 2048-point buffer
__host__ __device__ inline int pairs_per_cta(int pn)
{
    return pn >= 2048 ? 1 : 2048 / pn;
}

// LOG2 > 0: the kernel for pn = 2^LOG2 only (the FFT's strides and loop
// counts constants); 0: any pn.
template <typename TI, typename TO, int LOG2>
__global__ void __launch_bounds__(kFilterThreads) filter_stockham_kernel(const TI *__restrict__ in,
                                                                         TO *__restrict__ out,
                                                                         const __grid_constant__ FilterParams p,
                                                                         const __grid_constant__ BetaTable bt,
                                                                         const float *__restrict__ customK)
{
    extern __shared__ float2 smem[];
    const int pn = LOG2 > 0 ? 1 << LOG2 : p.pn, nu = p.nu;
    const int log2pn = LOG2 > 0 ? LOG2 : p.log2pn;
    const int ppc = pairs_per_cta(pn);
    const int stride = sp(pn);  // padded length of one transform
    float2 *A = smem;
    float2 *Bf = A + (size_t)ppc * stride;
    float2 *tw = Bf + (size_t)ppc * stride;
    float *Kh = reinterpret_cast<float *>(tw + twiddle_total(log2pn));  // K[0..pn/2] / pn
    float *wrow = Kh + pn / 2 + 1;                                          // W_red of the current view, nu
    int cached_view = -1;
    init_stockham_twiddles(tw, log2pn);
    const float inv_pn = 1.0f / (float)pn;
    for (int m = threadIdx.x; m <= pn / 2; m += blockDim.x) Kh[m] = (customK ? customK[m] : p.K[m]) * inv_pn;
    __syncthreads();
    // each CTA takes a contiguous run of pairs, so consecutive pairs share a view
    const long n_pairs = (p.n_rows + 1) / 2;
    const long per_cta = (n_pairs + gridDim.x - 1) / gridDim.x;
    const long first = (long)blockIdx.x * per_cta, last = min(n_pairs, first + per_cta);
    for (long pr0 = first; pr0 < last; pr0 += ppc) {
        const int groups = (int)min((long)ppc, last - pr0);
        if (p.apply_weights && (p.w.redund == PYRO_REDUND_PARKER || p.w.redund == PYRO_REDUND_SCAN)) {
            // the scan weight depends on (view, u) only: one row per view, cached
            const int view = (int)(((2 * pr0) / p.rows_per_view) % p.n_views);
            const int view_end = (int)(((2 * (pr0 + groups) - 1) / p.rows_per_view) % p.n_views);
            if (view == view_end && view != cached_view) {
                for (int k = threadIdx.x; k < nu; k += blockDim.x) {
                    const float u = ((float)k - p.w.cu) * p.w.su;
                    wrow[k] = parker_weight(bt.beta[view], atanf(u / p.w.sdd), p.w.delta);
                }
                cached_view = view;
                __syncthreads();
            } else if (view != view_end) {
                cached_view = -1;
            }
        }
        // load: two weighted rows per complex sequence, zero-padded to pn
        for (int g = 0; g < groups; ++g) {
            const long r0 = 2 * (pr0 + g), r1 = r0 + 1;
            const bool has1 = r1 < p.n_rows;
            const int l0 = (int)(r0 % p.rows_per_view), l1 = (int)(r1 % p.rows_per_view);
            const int view0 = (int)((r0 / p.rows_per_view) % p.n_views), view1 = (int)((r1 / p.rows_per_view) % p.n_views);
            const float v0 = ((float)l0 - p.w.cv) * p.w.sv, v1 = ((float)l1 - p.w.cv) * p.w.sv;
            const TI *in0 = in + r0 * nu, *in1 = in + r1 * nu;
            float2 *dst = A + g * stride;
            for (int n = threadIdx.x; n < pn; n += blockDim.x) {
                float a = 0.0f, c = 0.0f;
                if (n < nu) {
                    a = ld(in0 + n);
                    if (has1) c = ld(in1 + n);
                    if (p.apply_weights) {
                        if (cached_view >= 0) {
                            // W_cos (and the cached Parker row)
                            const float u = ((float)n - p.w.cu) * p.w.su;
                            const float wr = wrow[n];
                            a *= wr * cosine_weight(p.w, u, v0);
                            c *= wr * cosine_weight(p.w, u, v1);
                        } else {
                            a *= total_weight(p.w, bt, view0, l0, n);
                            if (has1) c *= total_weight(p.w, bt, view1, l1, n);
                        }
                    }
                }
                dst[sp(n)] = make_float2(a, c);
            }
        }
        __syncthreads();
        float2 *X = stockham_fft<LOG2>(A, Bf, tw, log2pn, pn, groups);
        float2 *Y = X == A ? Bf : A;
        // conj(K X): the inverse transform as conj(FFT(conj(.)))
        for (int g = 0; g < groups; ++g)
            for (int m = threadIdx.x; m < pn; m += blockDim.x) {
                const float k = Kh[m <= pn / 2 ? m : pn - m];
                const int q = g * stride + sp(m);
                X[q] = make_float2(X[q].x * k, -X[q].y * k);
            }
        __syncthreads();
        float2 *Z = stockham_fft<LOG2>(X, Y, tw, log2pn, pn, groups);
        for (int g = 0; g < groups; ++g) {
            const long r0 = 2 * (pr0 + g), r1 = r0 + 1;
            const bool has1 = r1 < p.n_rows;
            for (int n = threadIdx.x; n < nu; n += blockDim.x) {
                const float2 z = Z[g * stride + sp(n)];
                out[r0 * nu + n] = to_storage<TO>(z.x);
                if (has1) out[r1 * nu + n] = to_storage<TO>(-z.y);
            }
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

template <typename TI, typename TO, int LOG2>
cudaError_t filter_launch(const void *in, void *out, const FilterParams &p, const BetaTable &bt,
                          const float *customK, cudaStream_t s)
{
    const int ppc = pairs_per_cta(p.pn);
    const size_t padded = (size_t)p.pn + (p.pn >> 3);
    const size_t smem = sizeof(float2) * (2 * ppc * padded + twiddle_total(p.log2pn)) +
                        sizeof(float) * ((size_t)(p.pn / 2 + 1) + p.nu);
    auto kern = filter_stockham_kernel<TI, TO, LOG2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFilterThreads, smem);
    if (e != cudaSuccess) return e;
    const long pairs = (p.n_rows + 1) / 2;
    const long ctas = (pairs + ppc - 1) / ppc;
    const long grid = std::min<long>(ctas, (long)device_sm_count() * std::max(per_sm, 1));
    kern<<<(unsigned)grid, kFilterThreads, smem, s>>>((const TI *)in, (TO *)out, p, bt, customK);
    return cudaGetLastError();
}

// the detector widths 513..1024 and 1025..2048 (pn 2048, 4096) take kernels
// specialised to their pn
template <typename TI, typename TO>
cudaError_t filter_dispatch(const void *in, void *out, const FilterParams &p, const BetaTable &bt,
                            const float *customK, cudaStream_t s)
{
    switch (p.log2pn) {
    case 11: return filter_launch<TI, TO, 11>(in, out, p, bt, customK, s);
    case 12: return filter_launch<TI, TO, 12>(in, out, p, bt, customK, s);
    default: return filter_launch<TI, TO, 0>(in, out, p, bt, customK, s);
    }
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

cudaError_t launch_weights_table(void *sino, int batch, const WeightParams &w, const float *table, pyro_dtype dt,
                                 cudaStream_t s)
{
    const long n = (long)batch * w.n_views * w.nv * w.nu;
    const long blocks = std::min<long>((n + 255) / 256, (long)device_sm_count() * 16);
    switch (dt) {
    case PYRO_F32:
        weights_table_kernel<float><<<(unsigned)blocks, 256, 0, s>>>((float *)sino, n, w, table);
        break;
    case PYRO_F16:
        weights_table_kernel<__half><<<(unsigned)blocks, 256, 0, s>>>((__half *)sino, n, w, table);
        break;
    case PYRO_BF16:
        weights_table_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, s>>>((__nv_bfloat16 *)sino, n, w, table);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_redundancy_grad(const float *a, const float *g, float *out, int batch, int n_views, int nv, int nu,
                                   cudaStream_t s)
{
    dim3 grid((nu + 255) / 256, n_views);
    redundancy_grad_kernel<<<grid, 256, 0, s>>>(a, g, out, batch, n_views, nv, nu);
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
