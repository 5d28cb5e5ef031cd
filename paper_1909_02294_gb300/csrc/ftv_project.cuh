// The FP64 projection of FTV_PRECISION_FP64 contexts (device code shared by the cost and centre kernels).
#pragma once

#include <cuda_runtime.h>

namespace ftv {

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

}  // namespace ftv
