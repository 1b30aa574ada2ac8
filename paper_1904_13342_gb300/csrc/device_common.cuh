// Device helpers shared by the projector, back-projector and filter kernels:
// storage-type loads/stores (FP32 arithmetic for every storage type) and the
// zero-extended linear / bilinear / trilinear interpolation of the paper's
// "kernel interpolation" mode, done in software so that the FP32 result
// stays within ~1e-6 of the exact interpolant (hardware texture filtering
// quantises the weights to 8 fractional bits).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace pyro {

template <typename T>
__device__ __forceinline__ float ld(const T *p);
template <>
__device__ __forceinline__ float ld<float>(const float *p)
{
    return __ldg(p);
}
template <>
__device__ __forceinline__ float ld<__half>(const __half *p)
{
    return __half2float(__ldg(p));
}
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}

template <typename T>
__device__ __forceinline__ T to_storage(float v);
template <>
__device__ __forceinline__ float to_storage<float>(float v)
{
    return v;
}
template <>
__device__ __forceinline__ __half to_storage<__half>(float v)
{
    return __float2half_rn(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 to_storage<__nv_bfloat16>(float v)
{
    return __float2bfloat16_rn(v);
}

template <typename T>
__device__ __forceinline__ float to_float(T v);
template <>
__device__ __forceinline__ float to_float<float>(float v)
{
    return v;
}
template <>
__device__ __forceinline__ float to_float<__half>(__half v)
{
    return __half2float(v);
}
template <>
__device__ __forceinline__ float to_float<__nv_bfloat16>(__nv_bfloat16 v)
{
    return __bfloat162float(v);
}

// One axis of a zero-extended linear interpolation at index position f:
// the two taps i0 (weight w0) and i1 = i0 + 1 (weight w1), clamped into
// [0, n-1] for addressing, with the weight of a tap outside the array zeroed.
struct Axis {
    int i0, i1;
    float w0, w1;
};

__device__ __forceinline__ Axis axis_taps(float f, int n)
{
    const float f0 = floorf(f);
    const float a = f - f0;
    const int i = (int)f0;
    Axis r;
    r.w0 = ((unsigned)i < (unsigned)n) ? 1.0f - a : 0.0f;
    r.w1 = ((unsigned)(i + 1) < (unsigned)n) ? a : 0.0f;
    r.i0 = min(max(i, 0), n - 1);
    r.i1 = min(max(i + 1, 0), n - 1);
    return r;
}

template <typename T>
__device__ __forceinline__ float lerp_zero(const T *row, int n, float f)
{
    const Axis a = axis_taps(f, n);
    return a.w0 * ld(row + a.i0) + a.w1 * ld(row + a.i1);
}

template <typename T>
__device__ __forceinline__ float bilerp_zero(const T *img, int nx, int ny, float fx, float fy)
{
    const Axis ax = axis_taps(fx, nx);
    const Axis ay = axis_taps(fy, ny);
    const T *r0 = img + (size_t)ay.i0 * nx;
    const T *r1 = img + (size_t)ay.i1 * nx;
    const float v0 = ax.w0 * ld(r0 + ax.i0) + ax.w1 * ld(r0 + ax.i1);
    const float v1 = ax.w0 * ld(r1 + ax.i0) + ax.w1 * ld(r1 + ax.i1);
    return ay.w0 * v0 + ay.w1 * v1;
}

template <typename T>
__device__ __forceinline__ float trilerp_zero(const T *vol, int nx, int ny, int nz, float fx, float fy, float fz)
{
    const Axis ax = axis_taps(fx, nx);
    const Axis ay = axis_taps(fy, ny);
    const Axis az = axis_taps(fz, nz);
    const size_t sxy = (size_t)nx * ny;
    const T *p00 = vol + az.i0 * sxy + (size_t)ay.i0 * nx;
    const T *p01 = vol + az.i0 * sxy + (size_t)ay.i1 * nx;
    const T *p10 = vol + az.i1 * sxy + (size_t)ay.i0 * nx;
    const T *p11 = vol + az.i1 * sxy + (size_t)ay.i1 * nx;
    const float v00 = ax.w0 * ld(p00 + ax.i0) + ax.w1 * ld(p00 + ax.i1);
    const float v01 = ax.w0 * ld(p01 + ax.i0) + ax.w1 * ld(p01 + ax.i1);
    const float v10 = ax.w0 * ld(p10 + ax.i0) + ax.w1 * ld(p10 + ax.i1);
    const float v11 = ax.w0 * ld(p11 + ax.i0) + ax.w1 * ld(p11 + ax.i1);
    return az.w0 * (ay.w0 * v00 + ay.w1 * v01) + az.w1 * (ay.w0 * v10 + ay.w1 * v11);
}

// Trilinear interpolation of a zero-extended volume stored with arbitrary
// strides (elements) per axis: x-fastest [z][y][x] or the z-major copy
// [y][x][z] used by the staged forward projector.
template <typename T>
__device__ __forceinline__ float trilerp_zero_strided(const T *vol, int nx, int ny, int nz, size_t stx, size_t sty,
                                                      size_t stz, float fx, float fy, float fz)
{
    const Axis ax = axis_taps(fx, nx);
    const Axis ay = axis_taps(fy, ny);
    const Axis az = axis_taps(fz, nz);
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

__device__ __forceinline__ float lerpf(float a, float b, float t)
{
    return fmaf(t, b - a, a);
}

// Trilinear interpolation at a position known to be strictly inside the
// array on every axis (0 <= f < n-1): no tap is outside, so no clamping or
// weight masking is needed; 32-bit element offsets (arrays < 2^31 elements).
template <typename T>
__device__ __forceinline__ float trilerp_interior(const T *vol, int stx, int sty, int stz, float fx, float fy, float fz)
{
    const float x0 = floorf(fx), y0 = floorf(fy), z0 = floorf(fz);
    const float ax = fx - x0, ay = fy - y0, az = fz - z0;
    const T *b = vol + ((int)x0 * stx + (int)y0 * sty + (int)z0 * stz);
    const float v00 = lerpf(ld(b), ld(b + stz), az);
    const float v01 = lerpf(ld(b + sty), ld(b + sty + stz), az);
    const float v10 = lerpf(ld(b + stx), ld(b + stx + stz), az);
    const float v11 = lerpf(ld(b + stx + sty), ld(b + stx + sty + stz), az);
    return lerpf(lerpf(v00, v01, ay), lerpf(v10, v11, ay), ax);
}

// ---- mbarrier waits with a time limit (shared by the TMA and tcgen05 kernels)
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // a wait gives up after one second

__device__ __forceinline__ unsigned smem_addr(const void *ptr)
{
    return (unsigned)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    unsigned ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait: false when it gave up after limit_ns
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned phase, unsigned long long limit_ns = kWaitLimitNs)
{
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int n = 0; n < 64; ++n)
            if (mbar_try_wait(bar, phase)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// floor(x) for |x| < 2^22 on the FMA pipe: x + 1.5 * 2^23 rounded toward
// -inf is exactly 1.5 * 2^23 + floor(x) (unit spacing there), so the float
// floor and the integer floor (low bits of the sum) both follow without a
// conversion instruction.
constexpr float kFloorMagic = 12582912.0f;  // 1.5 * 2^23, bit pattern 0x4B400000
__device__ __forceinline__ float floor_magic(float x) { return __fadd_rd(x, kFloorMagic); }
__device__ __forceinline__ float magic_to_float(float t) { return t - kFloorMagic; }
__device__ __forceinline__ int magic_to_int(float t) { return __float_as_int(t) - 0x4B400000; }

// Bilinear interpolation at a point whose four taps are all inside the
// image (no masking); strides in elements.
template <typename T>
__device__ __forceinline__ float bilerp_interior(const T *img, int stx, int sty, float fx, float fy)
{
    const float x0 = floorf(fx), y0 = floorf(fy);
    const float ax = fx - x0, ay = fy - y0;
    const T *b = img + ((int)x0 * stx + (int)y0 * sty);
    return lerpf(lerpf(ld(b), ld(b + stx), ax), lerpf(ld(b + sty), ld(b + sty + stx), ax), ay);
}

// Restrict m to samples strictly inside [margin, n-1-margin] on one axis
// (rounded inwards), the interior where trilerp_interior applies.
__device__ __forceinline__ void clip_axis_interior(float p0, float q, int n, float &lo, float &hi)
{
    const float a = 1e-3f, b = (float)(n - 1) - 1e-3f;
    if (fabsf(q) > 1e-30f) {
        const float t1 = (a - p0) / q;
        const float t2 = (b - p0) / q;
        lo = fmaxf(lo, fminf(t1, t2));
        hi = fminf(hi, fmaxf(t1, t2));
    } else if (!(p0 >= a && p0 <= b)) {
        lo = 1.0f;
        hi = -1.0f;
    }
}

// Restrict the sample index m of p(m) = p0 + m q to the open support
// (-1, n) of the zero-extended interpolant on one axis.  Rounded outwards:
// a sample just outside contributes an exact 0 through axis_taps.
__device__ __forceinline__ void clip_axis(float p0, float q, int n, float &lo, float &hi)
{
    if (fabsf(q) > 1e-30f) {
        const float t1 = (-1.0f - p0) / q;
        const float t2 = ((float)n - p0) / q;
        lo = fmaxf(lo, fminf(t1, t2));
        hi = fminf(hi, fmaxf(t1, t2));
    } else if (!(p0 > -1.0f && p0 < (float)n)) {
        lo = 1.0f;
        hi = -1.0f;
    }
}

}  // namespace pyro

// ---- float-float arithmetic (an unevaluated sum hi + lo of two floats,
// about 44 significant bits) from the error-free transformations of Knuth
// (TwoSum), Dekker (FastTwoSum) and the FMA form of TwoProduct.  The
// intrinsics are the round-to-nearest operations that the compiler never
// contracts or reorders, which these transformations rely on.
namespace pyro {

struct ff {
    float h, l;
};

__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b)  // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const ff s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    const float p = __fmul_rn(a.h, b);
    const float e = __fmaf_rn(a.h, b, -p);
    return fast_two_sum(p, __fmaf_rn(a.l, b, e));
}

__device__ __forceinline__ ff ff_div(ff a, ff b)
{
    const float q1 = __fdiv_rn(a.h, b.h);
    const ff r = ff_add(a, ff_mul_f(b, -q1));
    return fast_two_sum(q1, __fdiv_rn(r.h, b.h));
}

// r . (x, y, z, 1) with the row as hi/lo pairs and x, y, z exact floats
__device__ __forceinline__ ff ff_dot4(const float *hi, const float *lo, float x, float y, float z)
{
    ff s = {hi[3], lo[3]};
    s = ff_add(s, ff_mul_f({hi[0], lo[0]}, x));
    s = ff_add(s, ff_mul_f({hi[1], lo[1]}, y));
    s = ff_add(s, ff_mul_f({hi[2], lo[2]}, z));
    return s;
}

// c + v split into an integer and a fraction in [0, 1) (FP32), for |c + v| < 2^22
__device__ __forceinline__ void ff_split(ff v, float c, int &n, float &f)
{
    const ff s = ff_add(v, {c, 0.0f});
    const float fl = floorf(s.h);
    float r = __fadd_rn(__fsub_rn(s.h, fl), s.l);  // s.h - fl is exact
    int k = (int)fl;
    if (r < 0.0f) {
        r = __fadd_rn(r, 1.0f);
        k -= 1;
    }
    if (r >= 1.0f) {
        r = __fsub_rn(r, 1.0f);
        k += 1;
    }
    n = k;
    f = fminf(fmaxf(r, 0.0f), 0.99999994f);
}

}  // namespace pyro

// ---- packed FP32 pairs: the sm_100-family f32x2 instructions (one issue
// slot for two IEEE FP32 operations, each rounded as its scalar form) ----
namespace pyro {

typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float a, float b)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void upk2(f32x2 r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)  // a * b + c
{
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// a + b rounded toward -inf (floor_magic on a pair)
__device__ __forceinline__ f32x2 add2_rm(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

}  // namespace pyro
