// Device code shared by the cost and centre kernels: the contract's FP32 reciprocal and the FP64 projection
// of FTV_PRECISION_FP64 contexts.
#pragma once

#include <cuda_runtime.h>

namespace ftv {

// The contract's r = 1/w is the IEEE round-to-nearest reciprocal. On devices where an exhaustive
// start-up comparison found it equal, for every float w in [2^-126, 2^126), to one Newton-Raphson step
// on the hardware estimate r0 ~ 1/w, namely r = r0 + r0 (1 - w r0) with both steps fused multiply-adds
// (Markstein's method), the kernels use that step:
//   rcp_newton: exact for w in [2^-126, 2^126);
//   rcp_scaled: any w. Positive subnormal w (and w <= 0) are first scaled by 2^64, which is exact,
//               and the result scaled back; 1/w = 2^64 / (2^64 w) and power-of-two scaling commutes
//               with round-to-nearest, including the overflow to infinity of 1/w for w < 2^-128. For
//               w <= 0 or NaN the result is non-positive or NaN, which the in-view test rejects, as it
//               rejects the IEEE reciprocal of such w.
// w >= 2^126 cannot occur: the host bounds |h| <= 2^100, so |Wz| < 2^117.
__device__ __forceinline__ float rcp_newton(float w) {
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(w));
    return __fmaf_rn(r0, __fmaf_rn(-w, r0, 1.0f), r0);
}

__device__ __forceinline__ float rcp_scaled(float w) {
    const bool small = w < 0x1p-126f;
    const float r = rcp_newton(small ? w * 0x1p64f : w);
    return small ? r * 0x1p64f : r;
}

template <bool FAST>
__device__ __forceinline__ float contract_rcp(float w) {
    return FAST ? rcp_scaled(w) : __frcp_rn(w);
}

// The same reciprocal for w known to lie in [2^-126, 2^126) (kIn and kFront entries: w > 2^-92).
template <bool FAST>
__device__ __forceinline__ float contract_rcp_normal(float w) {
    return FAST ? rcp_newton(w) : __frcp_rn(w);
}

// Operation by operation as the contract writes it: IEEE double, each product, sum and the quotient
// rounded on its own, the sums left to right, (ui, vi) = (floor(X / Wz + 0.5), floor(Y / Wz + 0.5)) and the
// view's range test. Out of line: in the cost kernel it runs only for evaluations near a rounding
// boundary and for entries without an error bound.
static __device__ __noinline__ bool project_fp64(const double* __restrict__ h, int x, int y, int wv, int hv, int* ui,
                                                 int* vi) {
    const double dx = (double)x, dy = (double)y;
    const double X = __dadd_rn(__dadd_rn(__dmul_rn(__ldg(&h[0]), dx), __dmul_rn(__ldg(&h[1]), dy)), __ldg(&h[2]));
    const double Y = __dadd_rn(__dadd_rn(__dmul_rn(__ldg(&h[3]), dx), __dmul_rn(__ldg(&h[4]), dy)), __ldg(&h[5]));
    const double Wz = __dadd_rn(__dadd_rn(__dmul_rn(__ldg(&h[6]), dx), __dmul_rn(__ldg(&h[7]), dy)), __ldg(&h[8]));
    if (!(Wz > 0.0)) return false;
    const double fu = floor(__dadd_rn(__ddiv_rn(X, Wz), 0.5));
    const double fv = floor(__dadd_rn(__ddiv_rn(Y, Wz), 0.5));
    if (!(fu >= 0.0 && fu <= (double)(wv - 1) && fv >= 0.0 && fv <= (double)(hv - 1))) return false;
    *ui = (int)fu;
    *vi = (int)fv;
    return true;
}

// The same projection with its result returned by value, (vi << 32) | ui when in view and -1 when out, so
// that a caller needs no addressable locals (which would live on the stack) around the call.
static __device__ __noinline__ long long project_fp64_packed(const double* __restrict__ h, int x, int y, int wv,
                                                             int hv) {
    const double dx = (double)x, dy = (double)y;
    const double X = __dadd_rn(__dadd_rn(__dmul_rn(__ldg(&h[0]), dx), __dmul_rn(__ldg(&h[1]), dy)), __ldg(&h[2]));
    const double Y = __dadd_rn(__dadd_rn(__dmul_rn(__ldg(&h[3]), dx), __dmul_rn(__ldg(&h[4]), dy)), __ldg(&h[5]));
    const double Wz = __dadd_rn(__dadd_rn(__dmul_rn(__ldg(&h[6]), dx), __dmul_rn(__ldg(&h[7]), dy)), __ldg(&h[8]));
    if (!(Wz > 0.0)) return -1;
    const double fu = floor(__dadd_rn(__ddiv_rn(X, Wz), 0.5));
    const double fv = floor(__dadd_rn(__ddiv_rn(Y, Wz), 0.5));
    if (!(fu >= 0.0 && fu <= (double)(wv - 1) && fv >= 0.0 && fv <= (double)(hv - 1))) return -1;
    return ((long long)(int)fv << 32) | (unsigned)(int)fu;
}

}  // namespace ftv
