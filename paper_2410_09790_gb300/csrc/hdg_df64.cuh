// Double-FP32 ("pair") arithmetic for FP64-accurate kernels on the FP32 pipes.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so an FP64 kernel with a few FP64 operations per byte
// is bound by the FP64 pipe, not by HBM. A value is carried here as an unevaluated pair hi + lo of
// FP32 numbers (48 significant bits); sums of products use the error-free transformations of
// Dekker (1971) and Knuth: TwoProduct by one FMA (a*b - fl(a*b) is exact in FP32) and TwoSum (six
// additions), the accumulated errors kept in the lo word, as in the compensated dot product Dot2 of
// Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005). A sum of n products is then accurate to
// about n * 2^-48 of the sum of the terms' magnitudes (FP64: n * 2^-53), at roughly ten FP32
// operations per FP64 multiply-add. The _rn intrinsics keep the compiler from contracting products
// into sums, which would break the transformations.
#pragma once
#include <cuda_runtime.h>

namespace hdg {

struct f2 {
    float h, l;
};

__device__ __forceinline__ f2 f2_of(double x) {
    const float h = __double2float_rn(x);
    return f2{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ f2 f2_of(float2 v) { return f2{v.x, v.y}; }

// an FP32 number widened to FP64 by assembling the FP64 bit pattern on the integer pipes (exact
// for normal numbers; zeros and subnormals give a signed zero, an error below 2^-126): keeps the
// conversion off GB300's narrow FP64 pipe
__device__ __forceinline__ double f32_widen(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xFFu, s = b & 0x80000000u, m = b & 0x7FFFFFu;
    if (e == 0u) return __hiloint2double((int)s, 0);
    const unsigned ed = e == 0xFFu ? 0x7FFu : e + 896u;         // (inf / NaN keep their class)
    return __hiloint2double((int)(s | (ed << 20) | (m >> 3)), (int)(m << 29));
}

// the pair as one FP64 number: both words widened exactly, one FP64 addition
__device__ __forceinline__ double f2_dbl(f2 a) { return f32_widen(a.h) + f32_widen(a.l); }

// s + t = a + b exactly (TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__device__ __forceinline__ f2 f2_norm(float h, float l) {
    float s, t;
    two_sum(h, l, s, t);
    return f2{s, t};
}

__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    float s, t;
    two_sum(a.h, b.h, s, t);
    return f2_norm(s, __fadd_rn(t, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ f2 f2_neg(f2 a) { return f2{-a.h, -a.l}; }

__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) { return f2_add(a, f2_neg(b)); }

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    const float p = __fmul_rn(a.h, b.h);
    const float e = fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)));
    return f2_norm(p, e);
}

// a running sum of products as a pair
struct acc2 {
    float h = 0.f, l = 0.f;
    __device__ __forceinline__ void fma(f2 a, f2 b) {
        const float p = __fmul_rn(a.h, b.h);
        const float e = fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)));
        float s, t;
        two_sum(h, p, s, t);
        h = s;
        l = __fadd_rn(l, __fadd_rn(t, e));
    }
    __device__ __forceinline__ void add(f2 a) {
        float s, t;
        two_sum(h, a.h, s, t);
        h = s;
        l = __fadd_rn(l, __fadd_rn(t, a.l));
    }
    __device__ __forceinline__ f2 get() const { return f2_norm(h, l); }
};

}  // namespace hdg
