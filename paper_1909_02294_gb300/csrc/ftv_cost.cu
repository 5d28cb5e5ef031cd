// Segment x depth-label matching-cost volume: the persistent cost kernel.
//
// Paper: Eq. 4 (L1 distance of Y, Cb, Cr between a reference point and its transform T[.] into a
// neighbouring view for the considered depth), Eq. 1 (costs of the neighbouring views c' in D are
// combined for every segment of every view), Sec. III-A (segments are the units; depth per segment).
// Here every pixel of a segment is a sample point (window of one pixel), the per-pixel costs of the
// neighbours are combined by min or sum, and the segment's cost is the int32 sum over its pixels.
//
// Work decomposition (GB300 design, not the paper's CPU threading of Sec. IV-A): a work item is one
// tile of kTile consecutive pixels of the listed segments (segments in list order, each segment's
// pixels contiguous) times one block of LB consecutive labels of one (job, reference) unit. Resident
// CTAs take items from a global counter in increasing order, so CTAs that run together work on
// neighbouring tiles and label blocks and share their neighbour-view footprints in L2. Per item:
//   - the N x LB homographies and the neighbour geometry are staged in shared memory;
//   - each thread owns kPPT pixels (x, y and the reference samples in registers);
//   - for each label, for each neighbour: FP32 projection, one packed-texel gather, |dY|+|dCb|+|dCr|,
//     running min/sum per pixel in registers;
//   - per label, warp reductions over runs of equal segment collapse the per-pixel costs, one shared
//     atomic per run, and at the end of the item each segment's row slice is written: plain stores
//     for segments wholly inside the tile, global atomics for segments cut by a tile boundary.
// All arithmetic that decides a sample position is explicit round-to-nearest FP32 (no contraction
// freedom is left to the compiler), so the result is bit-identical to any implementation of the same
// sequence; costs are integers, so summation order does not matter.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "ftv_internal.h"
#include "ftv_project.cuh"

namespace ftv {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSentinel = INT_MAX;
// Segments of a tile whose listed-pixel offsets are cached in shared memory (more: binary search in
// global memory). Together with kSegAcc this keeps a CTA near 30 KB of shared memory, so that four CTAs
// leave about half of the SM's 256 KB L1 to the neighbour-view gathers (prefer_l1).
constexpr int kLocCache = 257;

// cost(): |dY| + |dCb| + |dCr| as a chain of __sad (|x - y| + z, unsigned accumulate; exact here, as every
// term and the sum are below 2^18), which measured 12.5 % fewer instructions per evaluation than separate
// subtractions, absolute values and adds (1920x1080 8-view rig: 30.9 -> 29.4 ms).
template <int FMT>
struct TexelOps;

template <>
struct TexelOps<FMT_U8X4> {
    static __device__ __forceinline__ void unpack_ref(const void* base, int64_t i, int& a, int& b, int& c) {
        const uint32_t t = __ldg(static_cast<const uint32_t*>(base) + i);
        a = t & 0xff;
        b = (t >> 8) & 0xff;
        c = t >> 16;
    }
    static __device__ __forceinline__ int cost(const void* base, int i, int a, int b, int c) {
        const uint32_t t = __ldg(static_cast<const uint32_t*>(base) + i);
        return (int)__sad((int)(t & 0xff), a, __sad((int)((t >> 8) & 0xff), b, __sad((int)(t >> 16), c, 0u)));
    }
};

template <>
struct TexelOps<FMT_P10> {
    static __device__ __forceinline__ void unpack_ref(const void* base, int64_t i, int& a, int& b, int& c) {
        const uint32_t t = __ldg(static_cast<const uint32_t*>(base) + i);
        a = t & 0x3ff;
        b = (t >> 10) & 0x3ff;
        c = t >> 20;
    }
    static __device__ __forceinline__ int cost(const void* base, int i, int a, int b, int c) {
        const uint32_t t = __ldg(static_cast<const uint32_t*>(base) + i);
        return (int)__sad((int)(t & 0x3ff), a, __sad((int)((t >> 10) & 0x3ff), b, __sad((int)(t >> 20), c, 0u)));
    }
};

template <>
struct TexelOps<FMT_U16X4> {
    static __device__ __forceinline__ void unpack_ref(const void* base, int64_t i, int& a, int& b, int& c) {
        const uint2 t = __ldg(static_cast<const uint2*>(base) + i);
        a = t.x & 0xffff;
        b = t.x >> 16;
        c = t.y;
    }
    static __device__ __forceinline__ int cost(const void* base, int i, int a, int b, int c) {
        const uint2 t = __ldg(static_cast<const uint2*>(base) + i);
        return (int)__sad((int)(t.x & 0xffff), a, __sad((int)(t.x >> 16), b, __sad((int)t.y, c, 0u)));
    }
};

// Staged per-(neighbour, label) entry: the FP32 homography and the neighbour's geometry, 48 bytes so
// that a thread fetches it with three 128-bit shared loads. `pm` holds the row pitch (low 28 bits)
// and the entry's evaluation mode (high bits):
//   kGeneral  projective homography, evaluated as written in the contract;
//   kAffine   h6 == h7 == 0: Wz = fma(h6, x, fma(h7, y, h8)) is exactly h8 for every pixel, so
//             r = 1/h8 is computed once at staging time and stored in place of h6;
//   kUnit     affine with r == 1: u = X * 1 is exactly X, the multiplications are skipped;
//   kRect     unit with h0 = 1, h1 = 0, h3 = 0, h4 = 1, |h5| < 0.25 (rectified rigs: the row is kept):
//             X = fma(1, x, fma(0, y, h2)) is x + h2 rounded once, and Y = y + h5 rounded once lies
//             within 0.25 + 2^-9 of the integer y < 2^15, so floor(Y + 0.5) is exactly y;
//   kShift    rectified, and the column is x + D for every x < 2^15 with D = floor(h2 + 0.5) (FP64-precision
//             units: see shift_fp64; the FP32 contract: s = x + h2
//             rounded is within 2^-24 (|x| + |h2|) of x + h2; when h2 + 0.5 lies more than twice that
//             from every integer (checked at staging with |x| < 2^15, |h2| < 2^20), s + 0.5 lies more than
//             2^-24 from every integer, where rounding s + 0.5 cannot cross one (below 1 in magnitude its
//             rounding error is at most 2^-24; above, s + 0.5 is exact or only crosses into a binade
//             whose lower end is the integer below it), so floor((s + 0.5) rounded) = x + D. Used when the
//             view's pitch is the reference width and its height at least the reference height: the
//             sample's index is then the pixel's y * W + x plus D, the row needs no test, and the column
//             test is -D <= x < w - D, staged as floats (h[6], h[7]) with D in h[8];
//   kOut      affine with 1/h8 not finite and positive, or no pixel of the item's tile can reach the view
//             (box_class): every sample is out of view;
//   kIn       projective, and at every pixel of the item's tile Wz > 2^-92 and the sample rounds into the
//             view (box_class): r = 1/Wz is a normal reciprocal (no subnormal scaling) and neither the
//             finite-reciprocal test nor a range test can fail, so none is made;
//   kFront    projective, Wz > 2^-92 at every pixel of the tile (box_class): the reciprocal needs no
//             subnormal scaling and is finite and positive; the range tests remain.
// All of them give bit-identical results to the general sequence; they only skip work whose result
// is known exactly.
struct __align__(16) HEntry {
    float h[9];
    uint32_t w, h_, pm;
};
enum : uint32_t { kGeneral = 0, kAffine = 1, kUnit = 2, kOut = 3, kRect = 4, kSlow = 5, kShift = 6, kIn = 7, kFront = 8 };

// FP64-projection entries (kKindPrecise) stage local-frame coefficients in HEntry::h (stage_precise) and
// this alongside: the integer column u0 and row v0 the frame is shifted by, and the tie-test thresholds.
struct __align__(16) PEntry {
    int32_t u0, v0;
    float thr_u, thr_v;
};
constexpr uint32_t kPitchMask = (1u << 28) - 1u;

__device__ __forceinline__ bool finite_positive(float r) {
    return (unsigned)(__float_as_int(r) - 1) < 0x7f7fffffu;
}

// Position of one sample: reference pixel (x, y) through homography e.h into one neighbour view.
// Returns whether it is in view and its texel index. Equivalent to the contract's float test (Wz > 0,
// 0 <= floor(u + 0.5) <= W - 1, ...): the host guarantees |h| <= 2^100, so X and Y are finite;
// r = 1/Wz is then finite and positive exactly when Wz > 0 and 1/Wz does not overflow (if it does, u
// is +-inf or NaN and the contract says "out"); with finite positive r, u + 0.5 is finite or +-inf,
// and floor-to-int with saturation followed by an unsigned range test decides "in view" exactly as
// the float compares do.
template <bool FAST_RCP>
__device__ __forceinline__ bool pos_general(const float4& a, const float4& b, const float4& c, int pitch, float x,
                                            float y, int& idx) {
    const float X = __fmaf_rn(a.x, x, __fmaf_rn(a.y, y, a.z));
    const float Yh = __fmaf_rn(a.w, x, __fmaf_rn(b.x, y, b.y));
    const float Wz = __fmaf_rn(b.z, x, __fmaf_rn(b.w, y, c.x));
    const float r = contract_rcp<FAST_RCP>(Wz);
    const int ui = __float2int_rd(__fadd_rn(__fmul_rn(X, r), 0.5f));
    const int vi = __float2int_rd(__fadd_rn(__fmul_rn(Yh, r), 0.5f));
    idx = vi * pitch + ui;
    return finite_positive(r) & ((unsigned)ui < __float_as_uint(c.y)) & ((unsigned)vi < __float_as_uint(c.z));
}

// Affine entries: r (finite, positive) was hoisted out of the pixel loop; UNIT means r == 1.
template <bool UNIT>
__device__ __forceinline__ bool pos_affine(const float4& a, const float4& b, const float4& c, float r, int pitch,
                                           float x, float y, int& idx) {
    const float X = __fmaf_rn(a.x, x, __fmaf_rn(a.y, y, a.z));
    const float Yh = __fmaf_rn(a.w, x, __fmaf_rn(b.x, y, b.y));
    const float u = UNIT ? X : __fmul_rn(X, r);
    const float v = UNIT ? Yh : __fmul_rn(Yh, r);
    const int ui = __float2int_rd(__fadd_rn(u, 0.5f));
    const int vi = __float2int_rd(__fadd_rn(v, 0.5f));
    idx = vi * pitch + ui;
    return ((unsigned)ui < __float_as_uint(c.y)) & ((unsigned)vi < __float_as_uint(c.z));
}

// Rectified entries (kRect): u = x + h2, the sample row is the reference row y.
__device__ __forceinline__ bool pos_rect(float h2, uint32_t wv, uint32_t hv, int pitch, float x, int iy, int& idx) {
    const int ui = __float2int_rd(__fadd_rn(__fadd_rn(x, h2), 0.5f));
    idx = iy * pitch + ui;
    return ((unsigned)ui < wv) & ((unsigned)iy < hv);
}

// Folds one sample into the pixel's running combination over views (min or sum). With the kernel's PF
// (min only, the penalty at least the largest possible sample cost) the running minimum starts at the
// penalty, which an out-of-view sample cannot lower; the projective path then lets only in-view
// samples update it (PF here), which pays off where many samples fall outside (wide convergent
// baselines), while the rectified and affine paths keep the select form, measured faster there. Both
// forms give the minimum over in-view costs and penalties of the contract.
//
// Checked builds (FTV_CHECKED): every gather is first tested against the neighbour view's texel count lim;
// an index outside it is recorded in the launch's plan (ST_CHECKED) and the sample is skipped, so a path
// whose in-view claim were wrong shows up as a status instead of an out-of-bounds read. Regular builds drop
// the test (lim and status are unused).
__device__ __forceinline__ bool checked_gather(bool ok, int idx, unsigned lim, uint32_t* status) {
#ifdef FTV_CHECKED
    if (ok && (unsigned)idx >= lim) {
        atomicOr(status, ST_CHECKED);
        return false;
    }
#else
    (void)idx;
    (void)lim;
    (void)status;
#endif
    return ok;
}

template <int FMT, int COMB, bool PF>
__device__ __forceinline__ void accumulate(int& m, bool ok, const void* tex, int idx, int a, int b, int c,
                                           int penalty, unsigned lim, uint32_t* status) {
    ok = checked_gather(ok, idx, lim, status);
    if (COMB == FTV_COMBINE_MIN && PF) {
        if (ok) m = min(m, TexelOps<FMT>::cost(tex, idx, a, b, c));
    } else {
        int cst = penalty;
        if (ok) cst = TexelOps<FMT>::cost(tex, idx, a, b, c);
        m = COMB == FTV_COMBINE_MIN ? min(m, cst) : m + cst;
    }
}

// Classifies a projective entry for the pixel box [x0, x1] x [y0, y1] (x, y >= 0) under the FP32 contract,
// from the homography evaluated at the box's four corners:
//   kOut     no pixel can sample the wv x hv view. At every corner the point lies left of u = -1 (X + Wz < 0),
//            right of u = wv (X - wv Wz > 0), above v = -1 or below v = hv (the same with Y), or behind the
//            camera (Wz < 0);
//   kIn      at every pixel Wz > 2^-92 and the sample rounds into the view. At every corner Wz is positive
//            (and above 2^-90), X and Y are positive, and (wv - 1) Wz - X and (hv - 1) Wz - Y are positive;
//   kFront   at every pixel Wz > 2^-92 (the corners as for kIn, Wz only);
//   kGeneral otherwise.
// Each corner condition carries a margin of 2^-20 times the magnitude of its terms (sx = |h0| x + |h1| y +
// |h2|, likewise sy, sz). Why the conclusions hold at every pixel: the contract's two fused multiply-adds
// put X, Y and Wz within 2^-23 of those magnitudes of their exact values, at any pixel and at the corners.
// With the margin, each corner condition implies, in exact arithmetic, a condition linear (convex, for
// kOut) in the pixel position with half the margin (for Wz: Wz - 2^-22 sz - 2^-92 > 0), which therefore
// holds at every pixel of the box, and there the FP32 value keeps the sign the conclusion needs:
//   Wz_f32 > 2^-92, so r = 1/Wz is finite, positive and the reciprocal of a normal float;
//   X_f32 >= 0, so u = X r >= 0 and floor(u + 0.5) >= 0;
//   X_f32 <= (wv - 1) Wz_f32, so u <= (wv - 1)(1 + 2^-23) < wv - 1 + 2^-7 (wv <= 2^15), u + 0.5 rounds
//   below wv and floor(u + 0.5) <= wv - 1 (the same for rows);
//   for kOut as before: a point left of u = -1 has u + 0.5 < 0 after rounding, one right of u = wv rounds to
//   a column of at least wv, one behind the camera has Wz <= 0.
// |h| <= 2^100 keeps every term finite; an overflow or a NaN fails the comparisons and gives kGeneral.
__device__ __forceinline__ uint32_t box_class(const float* h, float x0, float x1, float y0, float y1, float wv,
                                              float hv) {
    const float m = 0x1p-20f;
    const float wv1 = wv - 1.0f, hv1 = hv - 1.0f;
    bool left = true, right = true, top = true, bottom = true, behind = true;
    bool front = true, inside = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float x = (k & 1) ? x1 : x0, y = (k & 2) ? y1 : y0;  // x, y >= 0
        const float X = __fmaf_rn(h[0], x, __fmaf_rn(h[1], y, h[2]));
        const float Y = __fmaf_rn(h[3], x, __fmaf_rn(h[4], y, h[5]));
        const float Z = __fmaf_rn(h[6], x, __fmaf_rn(h[7], y, h[8]));
        const float sx = __fmaf_rn(fabsf(h[0]), x, __fmaf_rn(fabsf(h[1]), y, fabsf(h[2])));
        const float sy = __fmaf_rn(fabsf(h[3]), x, __fmaf_rn(fabsf(h[4]), y, fabsf(h[5])));
        const float sz = __fmaf_rn(fabsf(h[6]), x, __fmaf_rn(fabsf(h[7]), y, fabsf(h[8])));
        const float tl = __fadd_rn(X, Z), tr = __fmaf_rn(-wv, Z, X);
        const float tt = __fadd_rn(Y, Z), tb = __fmaf_rn(-hv, Z, Y);
        left = left && tl < -m * (sx + sz + fabsf(tl));
        right = right && tr > m * (sx + wv * sz + fabsf(tr));
        top = top && tt < -m * (sy + sz + fabsf(tt));
        bottom = bottom && tb > m * (sy + hv * sz + fabsf(tb));
        behind = behind && Z < -m * (sz + fabsf(Z));
        front = front && Z > fmaxf(m * (sz + fabsf(Z)), 0x1p-90f);
        const float ir = __fmaf_rn(wv1, Z, -X), ib = __fmaf_rn(hv1, Z, -Y);
        inside = inside && X > m * (sx + fabsf(X)) && Y > m * (sy + fabsf(Y)) &&
                 ir > m * (sx + wv1 * sz + fabsf(ir)) && ib > m * (sy + hv1 * sz + fabsf(ib));
    }
    if (left || right || top || bottom || behind) return kOut;
    if (front) return inside ? kIn : kFront;
    return kGeneral;
}

// Integer-shift entries of the FP64 projection (linear rigs with parallel axes): the unrounded homography
// is exactly [[1, 0, h2], [0, 1, h5], [0, 0, 1]] with |h5| < 0.49 and |h2| < 2^20. The FP64 projection then
// computes X = x + h2 (one rounding; 1 * x and 0 * y are exact), Wz = 1 and X / Wz = X exactly, and
// floor(X + 0.5) rounded once more; likewise the row from y + h5. g = h2 + 0.5 is exact (|h2| < 2^20), and
// with D = floor(g):
//   g an integer: x + h2 = x + D - 0.5 and x + D are exact, so the column is x + D;
//   otherwise the two roundings move x + h2 + 0.5 by less than 2^-31 (|x + h2 + 0.5| < 2^21, unit roundoff
//   2^-53), so when g lies more than 2^-30 from every integer the column is floor(x + g) = x + D.
// The row is y: y + h5 + 0.5 lies in (y + 0.01, y + 0.99) and moves by less than 2^-35.
// Then every pixel's sample is (x + D, y), in view exactly when 0 <= x + D < wv (the view being at least as
// tall as the reference). Returns whether the entry has this form, with D.
__device__ __forceinline__ bool shift_fp64(const double* __restrict__ hg, int& D) {
    const double h0 = __ldg(&hg[0]), h1 = __ldg(&hg[1]), h2 = __ldg(&hg[2]), h3 = __ldg(&hg[3]), h4 = __ldg(&hg[4]),
                 h5 = __ldg(&hg[5]), h6 = __ldg(&hg[6]), h7 = __ldg(&hg[7]), h8 = __ldg(&hg[8]);
    if (!(h0 == 1.0 && h1 == 0.0 && h3 == 0.0 && h4 == 1.0 && h6 == 0.0 && h7 == 0.0 && h8 == 1.0 && fabs(h5) < 0.49 &&
          fabs(h2) < 0x1p20))
        return false;
    const double g = h2 + 0.5, f = floor(g), r = g - f;
    if (!(r == 0.0 || fmin(r, 1.0 - r) > 0x1p-30)) return false;
    D = (int)f;
    return true;
}

// Stages one (neighbour, label) entry of an FP64-precision unit for a tile whose pixels lie in the box
// x0 + [-rx, rx] x y0 + [-ry, ry]. In the local frame x' = x - x0, y' = y - y0 the projection is
//   u = U0 + X'/W, v = V0 + Y'/W,  X' = X - U0 W = a0 x' + a1 y' + a2,  Y' = Y - V0 W = b0 x' + b1 y' + b2,
//   W = c0 x' + c1 y' + c2,
// with (U0, V0) the integer position nearest the box centre's projection. The coefficients are formed in
// FP64 (that is where the cancellation of X - U0 W happens) and rounded to FP32 into h[]; u' = X'/W then
// stays within a few pixels, so the FP32 evaluation is accurate to about 2^-24 of the tile's extent
// instead of 2^-24 of the image coordinates. The bound delta covers, at every pixel of the box:
//   the FP32 rounding of the coefficients and of the two fused multiply-adds (3 * 2^-24 of the magnitude
//   M = |a0| rx + |a1| ry + |a2|), the FP64 rounding of the coefficients (2^-50 of the global magnitudes),
//   the quotient of those errors ((e_X + |u'| e_W) / W), the rounded reciprocal, product and + 0.5
//   (2^-23 |u'| + 2^-24 (|u'| + 1)), and the FP64 projection's own error against exact arithmetic
//   (3 * 2^-53 (A_X + |u| A_W) / W + 2 * 2^-53 (|u| + 1)),
// doubled. Where t = u' + 0.5 computed in FP32 lies farther than delta from every integer, floor(t) + U0
// is the FP64 projection's column (both floors see the same side of the same integer); otherwise the
// evaluation is redone in FP64. Returns kGeneral (that test applies), kRect (the same, rectified: below),
// kOut (the FP64 projection puts no
// pixel of the box in view: behind the camera, or wholly beyond one image edge by more than the bound) or
// kSlow (no bound: W may come near zero in the box, or delta is large; every evaluation in FP64).
__device__ uint32_t stage_precise(const double* __restrict__ hg, int x0, int y0, int rx, int ry, int wv, int hv,
                                  float* h, PEntry& P) {
    double H[9];
#pragma unroll
    for (int f = 0; f < 9; ++f) H[f] = __ldg(&hg[f]);
    const double u = 0x1p-53;
    const double dx0 = (double)x0, dy0 = (double)y0, drx = (double)rx, dry = (double)ry;
    const double ax = fabs(dx0) + drx, ay = fabs(dy0) + dry;
    const double AX = fabs(H[0]) * ax + fabs(H[1]) * ay + fabs(H[2]);
    const double AY = fabs(H[3]) * ax + fabs(H[4]) * ay + fabs(H[5]);
    const double AW = fabs(H[6]) * ax + fabs(H[7]) * ay + fabs(H[8]);
    const double X0 = fma(H[0], dx0, fma(H[1], dy0, H[2]));
    const double Y0 = fma(H[3], dx0, fma(H[4], dy0, H[5]));
    const double W0 = fma(H[6], dx0, fma(H[7], dy0, H[8]));
    const double gW = fabs(H[6]) * drx + fabs(H[7]) * dry + 0x1p-48 * AW;
    if (W0 + gW < 0.0) return kOut;  // W < 0 at every pixel of the box
    const double Wlo = W0 - gW;      // the exact W is at least this at every pixel of the box
    if (!(Wlo > 0x1p-60)) return kSlow;
    const double U0 = rint(fmin(fmax((double)__fdiv_rn((float)X0, (float)W0), -0x1p24), 0x1p24));
    const double V0 = rint(fmin(fmax((double)__fdiv_rn((float)Y0, (float)W0), -0x1p24), 0x1p24));
    h[0] = __double2float_rn(fma(-U0, H[6], H[0]));
    h[1] = __double2float_rn(fma(-U0, H[7], H[1]));
    h[2] = __double2float_rn(fma(-U0, W0, X0));
    h[3] = __double2float_rn(fma(-V0, H[6], H[3]));
    h[4] = __double2float_rn(fma(-V0, H[7], H[4]));
    h[5] = __double2float_rn(fma(-V0, W0, Y0));
    h[6] = __double2float_rn(H[6]);
    h[7] = __double2float_rn(H[7]);
    h[8] = __double2float_rn(W0);
    const double Ma = fabs((double)h[0]) * drx + fabs((double)h[1]) * dry + fabs((double)h[2]);
    const double Mb = fabs((double)h[3]) * drx + fabs((double)h[4]) * dry + fabs((double)h[5]);
    const double Mc = fabs((double)h[6]) * drx + fabs((double)h[7]) * dry + fabs((double)h[8]);
    const double eX = 0x1.82p-23 * Ma + 0x1p-50 * (Ma + AX + fabs(U0) * AW) + 0x1p-130;
    const double eY = 0x1.82p-23 * Mb + 0x1p-50 * (Mb + AY + fabs(V0) * AW) + 0x1p-130;
    const double eW = 0x1.82p-23 * Mc + 0x1p-50 * (Mc + AW) + 0x1p-130;
    if (!(Wlo > 2.0 * eW)) return kSlow;
    const double Wl = Wlo - eW;  // lower bound of the FP32 W and of the FP64 projection's W
    const double Ub = (Ma * (1.0 + 0x1p-20) + 2.0 * eX) / Wl;
    const double Vb = (Mb * (1.0 + 0x1p-20) + 2.0 * eY) / Wl;
    const double qu = (eX + Ub * eW) / Wl, qv = (eY + Vb * eW) / Wl;
    const double du = 2.0 * (qu + 0x1.01p-23 * Ub + 0x1.01p-24 * (Ub + 1.0) +
                             3.0 * u * (AX + (fabs(U0) + Ub) * AW) / Wl + 2.01 * u * (fabs(U0) + Ub + 1.0)) + 0x1p-30;
    const double dv = 2.0 * (qv + 0x1.01p-23 * Vb + 0x1.01p-24 * (Vb + 1.0) +
                             3.0 * u * (AY + (fabs(V0) + Vb) * AW) / Wl + 2.01 * u * (fabs(V0) + Vb + 1.0)) + 0x1p-30;
    // every pixel of the box has its column (row) beyond one edge by more than the bound
    if (U0 + Ub + 0.5 + du < 0.0 || U0 - Ub + 0.5 - du >= (double)wv || V0 + Vb + 0.5 + dv < 0.0 ||
        V0 - Vb + 0.5 - dv >= (double)hv)
        return kOut;
    if (!(du < 0.25 && dv < 0.25 && Ub < 0x1p21 && Vb < 0x1p21)) return kSlow;
    P.u0 = (int)U0;
    P.v0 = (int)V0;
    // near a tie when |frac(t) - 0.5| >= thr; 2^-22 more covers the FP32 rounding of that test itself
    P.thr_u = __double2float_rd(0.5 - du - 0x1p-22);
    P.thr_v = __double2float_rd(0.5 - dv - 0x1p-22);
    // Rectified local frame (linear rigs with parallel axes): with a0 = b1 = c2 = 1 and a1 = b0 = c0 = c1 = 0
    // the general evaluation computes exactly t_u = (x' + a2) + 0.5 (both rounded) and W = r = 1, so the
    // bound above holds for that shorter sequence; and when |b2| + delta_v < 0.5 every pixel's row decision
    // is floor(y' + b2 + 0.5 +- delta_v) = y', i.e. the row is y' + V0 with no test.
    if (h[0] == 1.0f && h[1] == 0.0f && h[3] == 0.0f && h[4] == 1.0f && h[6] == 0.0f && h[7] == 0.0f &&
        h[8] == 1.0f && fabs((double)h[5]) + dv < 0.49)
        return kRect;
    return kGeneral;
}

// First item of chunk k when n items are split into K nearly equal consecutive chunks (32-bit, no overflow).
__device__ __forceinline__ int chunk_begin(int n, int k, int K) {
    const int q = n / K, r = n - q * K;
    return k * q + min(k, r);
}

__device__ __forceinline__ int find_job(const RefJob* __restrict__ jobs, int n_jobs, int item) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&jobs[mid].item_base) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Largest k in [lo, hi) with a[k] <= w (a nondecreasing, a[lo] <= w).
__device__ __forceinline__ int upper_index(const int32_t* a, int lo, int hi, int w) {
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= w) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Warp-cooperative version (all 32 lanes call it): 32 probes per round narrow the range ~33-fold, so a
// search over n entries takes about log33(n) dependent loads instead of log2(n).
__device__ __forceinline__ int warp_upper_index(const int32_t* a, int lo, int hi, int w) {
    const int lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        const int64_t span = hi - lo;
        const bool le = a[lo + (int)(span * (lane + 1) / 33)] <= w;
        const int cnt = __popc(__ballot_sync(0xffffffffu, le));  // the true probes are a prefix
        const int nlo = cnt ? lo + (int)(span * cnt / 33) : lo;
        const int nhi = cnt < 32 ? lo + (int)(span * (cnt + 1) / 33) : hi;
        lo = nlo;
        hi = nhi;
    }
    const int p = lo + lane;
    const unsigned m = __ballot_sync(0xffffffffu, p < hi && a[p] <= w);
    return lo + 31 - __clz(m);
}

template <int FMT, int COMB, bool FAST_RCP, bool PF, int KIND>
__global__ void __launch_bounds__(kThreads, kMinBlocks) cost_kernel(const RefJob* __restrict__ jobs,
                                                                    Plan* __restrict__ plan, int chunk, int chunks) {
    __shared__ HEntry sH[kHEntries];
    __shared__ const void* sBase[FTV_MAX_NBRS];
    __shared__ int sAcc[kSegAcc * kMaxLB];
    __shared__ int sWoffs[kLocCache + 1];
    __shared__ int s_item, s_k0, s_k1, s_culled;
    __shared__ int s_box[4];  // the tile's pixel box: x min, x max, y min, y max
    __shared__ PEntry sP[precise_kind(KIND) ? kHEntries : 1];
    __shared__ uint8_t sOrd[KIND == kKindProjective ? kHEntries : 1];  // per label: neighbours to visit
    __shared__ int sCnt[KIND == kKindProjective ? kMaxLB : 1];         // per label: kIn | kFront << 8 | kGeneral << 16
    unsigned n_recomputed = 0;  // FP64-precision evaluations computed in double precision by this thread
    uint32_t* const ck = &plan->checked;  // out-of-view gathers of checked builds

    const int tid = threadIdx.x, lane = tid & 31;
    // this launch's items: [chunk_begin(chunk), chunk_begin(chunk + 1)); only thread 0 needs the first (it
    // recomputes it from the plan when it fetches an item, which keeps it out of every thread's registers)
    const int total = chunk_begin(*reinterpret_cast<volatile int*>(&plan->total_items), chunk + 1, chunks);
    const int n_jobs = *reinterpret_cast<volatile int*>(&plan->n_jobs);
    for (int i = tid; i < kSegAcc * kMaxLB; i += kThreads) sAcc[i] = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0)
            s_item = chunk_begin(*reinterpret_cast<volatile int*>(&plan->total_items), chunk, chunks) +
                     atomicAdd(&plan->counter[chunk], 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;

        const RefJob* Jp = &jobs[find_job(jobs, n_jobs, item)];
        const int q = item - Jp->item_base;
        const int nLB = Jp->nLB, L = Jp->L, N = Jp->N, W = Jp->W, penalty = Jp->penalty;
        const int tile = q / nLB, lb = q - tile * nLB;
        const int d0 = lb * Jp->LB;
        const int LBa = min(Jp->LB, L - d0);
        const int n_rec = Jp->n_rec, n_work = Jp->n_work;
        const int32_t* __restrict__ woffs = Jp->woffs;
        const int32_t* __restrict__ list = Jp->list;
        const int32_t* __restrict__ offs = Jp->offs;
        const uint32_t* __restrict__ pix = Jp->pix;
        const void* ref_tex = Jp->ref_texels;
        int32_t* __restrict__ cost = Jp->cost;
        const int w0 = tile * kTile;
        const int w1 = min(w0 + kTile, n_rec);

        // stage homographies and neighbour geometry: entry (n, l) for n < N, l < LBa
        const float* __restrict__ Hg = Jp->H;
        const NbrView* __restrict__ nbrs = Jp->nbrs;
        const int nh = N * LBa;
        for (int e = tid; e < (precise_kind(KIND) ? 0 : nh); e += kThreads) {
            const int n = e / LBa, l = e - n * LBa;
            const float* src = &Hg[((int64_t)n * L + d0 + l) * 9];
            HEntry& E = sH[e];
#pragma unroll
            for (int f = 0; f < 9; ++f) E.h[f] = __ldg(&src[f]);
            uint32_t mode = kGeneral;
            if (E.h[6] == 0.0f && E.h[7] == 0.0f) {
                const float r = __frcp_rn(E.h[8]);
                mode = !finite_positive(r) ? kOut : (r == 1.0f ? kUnit : kAffine);
                if (mode == kUnit && E.h[0] == 1.0f && E.h[1] == 0.0f && E.h[3] == 0.0f && E.h[4] == 1.0f &&
                    fabsf(E.h[5]) < 0.25f)
                    mode = kRect;
                E.h[6] = r;
                E.h[8] = E.h[2];  // Wz is not needed any more; a rectified entry then reads one float4
                if (mode == kRect && nbrs[n].pitch == W && nbrs[n].h >= Jp->Href) {
                    const double h2 = (double)E.h[2];
                    const double D = floor(h2 + 0.5), g = h2 + 0.5 - D;
                    if (fabs(h2) < 0x1p20 && fmin(g, 1.0 - g) > 0x1p-23 * (32768.0 + fabs(h2))) {
                        mode = kShift;
                        E.h[6] = (float)(-D);
                        E.h[7] = (float)((double)nbrs[n].w - D);
                        E.h[8] = __int_as_float((int)D);
                    }
                }
            }
            E.w = (uint32_t)nbrs[n].w;
            E.h_ = (uint32_t)nbrs[n].h;
            E.pm = (uint32_t)nbrs[n].pitch | (mode << 28);
        }
        for (int i = tid; i < N; i += kThreads) sBase[i] = nbrs[i].texels;
        if (tid == 0) {
            s_box[0] = s_box[2] = INT_MAX;
            s_box[1] = s_box[3] = INT_MIN;
            s_culled = 0;
        }
        if (tid < 32) {
            const int k = warp_upper_index(woffs, 0, n_work + 1, w0);
            if (lane == 0) s_k0 = k;
        } else if (tid < 64) {
            const int k = warp_upper_index(woffs, 0, n_work + 1, w1 - 1);
            if (lane == 0) s_k1 = k;
        }
        __syncthreads();
        const int k0 = s_k0, k1 = s_k1;
        const int nk = k1 - k0 + 1;
        const bool cached = nk + 1 <= kLocCache;
        if (cached)
            for (int i = tid; i <= nk; i += kThreads) sWoffs[i] = woffs[k0 + i];
        __syncthreads();

        // this thread's pixels
        float px[kPPT], py[kPPT];
        int ra[kPPT], rb[kPPT], rc[kPPT], key[kPPT], iy[kPPT];
        int rowx[kPPT];  // y * W + x (kShift entries of the mixed kernel)
        // The float row: kept in registers except in the mixed kernel, which needs registers for rowx and,
        // on the rigs it serves, rarely takes the general or affine paths that read it (exact conversion).
        auto row_f = [&](int j) { return KIND == kKindMixed ? (float)iy[j] : py[j]; };
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
            const int w = w0 + j * kThreads + tid;
            key[j] = kSentinel;
            iy[j] = 0;
            rowx[j] = 0;
            px[j] = py[j] = 0.0f;
            ra[j] = rb[j] = rc[j] = 0;
            if (w < w1) {
                int k;
                if (cached) k = k0 + upper_index(sWoffs, 0, nk + 1, w);
                else k = upper_index(woffs, k0, k1 + 1, w);
                const int s = list ? list[k] : k;
                const int base = cached ? sWoffs[k - k0] : woffs[k];
                const uint32_t xy = pix[offs[s] + (w - base)];
                const int x = xy & 0xffff, y = xy >> 16;
                px[j] = (float)x;
                py[j] = (float)y;
                iy[j] = y;
                rowx[j] = y * W + x;
                TexelOps<FMT>::unpack_ref(ref_tex, (int64_t)y * W + x, ra[j], rb[j], rc[j]);
                key[j] = k - k0;
            }
        }

        // An entry whose neighbour view no pixel of the tile can reach (box_class, on the staged coefficients)
        // takes the penalty for every pixel, without sampling: it becomes an all-out entry, which the pixel
        // loop does not visit. box_class also marks the entries whose samples all land in view (kIn) or in
        // front of the camera (kFront), which skip the tests they cannot fail. Only the projective-only
        // instantiation does this: on a rectified rig an out-of-view sample is
        // already cheap, and there the test cost more than it saved (1920x1080 linear 8-view rig: 7.8 % of
        // the evaluations culled, 31.1 against 30.9 ms).
        // FP64-precision units stage their entries here, once the box is known (stage_precise), and move the
        // pixels into the box's local frame.
        int fx0 = 0, fy0 = 0;  // local-frame origin (kKindPrecise)
        if constexpr (KIND == kKindProjective || precise_kind(KIND)) {  // uniform way through the barriers
            int bx0 = INT_MAX, bx1 = INT_MIN, by0 = INT_MAX, by1 = INT_MIN;
#pragma unroll
            for (int j = 0; j < kPPT; ++j)
                if (key[j] != kSentinel) {
                    bx0 = min(bx0, (int)px[j]);
                    bx1 = max(bx1, (int)px[j]);
                    by0 = min(by0, iy[j]);
                    by1 = max(by1, iy[j]);
                }
            bx0 = __reduce_min_sync(kFull, bx0);
            bx1 = __reduce_max_sync(kFull, bx1);
            by0 = __reduce_min_sync(kFull, by0);
            by1 = __reduce_max_sync(kFull, by1);
            if (lane == 0) {
                atomicMin(&s_box[0], bx0);
                atomicMax(&s_box[1], bx1);
                atomicMin(&s_box[2], by0);
                atomicMax(&s_box[3], by1);
            }
            __syncthreads();
            if constexpr (KIND == kKindProjective) {
                if (s_box[0] <= s_box[1]) {
                    const float bx0f = (float)s_box[0], bx1f = (float)s_box[1], by0f = (float)s_box[2],
                                by1f = (float)s_box[3];
                    // Slots past the end of the unit's last tile hold no pixel (their result is discarded);
                    // they take the box's first corner, so that every slot lies in the box and the kIn
                    // path's unchecked gathers stay inside the view for them too.
#pragma unroll
                    for (int j = 0; j < kPPT; ++j)
                        if (key[j] == kSentinel) {
                            px[j] = bx0f;
                            py[j] = by0f;
                        }
                    for (int e = tid; e < nh; e += kThreads) {
                        HEntry& E = sH[e];
                        if ((E.pm >> 28) == kGeneral) {
                            const uint32_t cls = box_class(E.h, bx0f, bx1f, by0f, by1f, (float)E.w, (float)E.h_);
                            E.pm = (E.pm & kPitchMask) | (cls << 28);
                            if (cls == kOut) atomicAdd(&s_culled, 1);
                        }
                    }
                }
            } else {
                const bool any = s_box[0] <= s_box[1];  // a tile always holds a pixel; kept for safety
                fx0 = any ? (s_box[0] + s_box[1]) >> 1 : 0;
                fy0 = any ? (s_box[2] + s_box[3]) >> 1 : 0;
                const int rx = any ? max(fx0 - s_box[0], s_box[1] - fx0) : 0;
                const int ry = any ? max(fy0 - s_box[2], s_box[3] - fy0) : 0;
                for (int e = tid; e < nh; e += kThreads) {
                    const int n = e / LBa, l = e - n * LBa;
                    HEntry& E = sH[e];
                    const int wv = nbrs[n].w, hv = nbrs[n].h;
                    const double* hg = &Jp->H64[((int64_t)n * L + d0 + l) * 9];
                    int D = 0;
                    uint32_t mode;
                    if (KIND == kKindPreciseMixed && nbrs[n].pitch == W && hv >= Jp->Href && shift_fp64(hg, D)) {
                        // every pixel's FP64 column is x + D and its row y: bounds on the local x' = x - fx0
                        mode = kShift;
                        E.h[6] = (float)(-D - fx0);
                        E.h[7] = (float)(wv - D - fx0);
                        E.h[8] = __int_as_float(D);
                    } else {
                        mode = stage_precise(hg, fx0, fy0, rx, ry, wv, hv, E.h, sP[e]);
                    }
                    E.w = (uint32_t)wv;
                    E.h_ = (uint32_t)hv;
                    E.pm = (uint32_t)nbrs[n].pitch | (mode << 28);
                    if (mode == kOut) atomicAdd(&s_culled, 1);
                }
                // every slot into the local frame; an empty slot (past the end of the unit's last tile, its
                // result discarded) takes the box's centre pixel, row and row index, so that every slot lies
                // in the box the entries were staged for and its local coordinates, row index and FP64
                // projection arguments name the same reference pixel
#pragma unroll
                for (int j = 0; j < kPPT; ++j) {
                    if (key[j] == kSentinel) {
                        px[j] = (float)fx0;
                        iy[j] = fy0;
                        rowx[j] = fy0 * W + fx0;
                    }
                    px[j] = (float)((int)px[j] - fx0);
                    py[j] = (float)(iy[j] - fy0);
                }
            }
            __syncthreads();
            if (tid == 0 && s_culled > 0) atomicAdd(&plan->culled, (unsigned long long)s_culled * (unsigned)(w1 - w0));
            if constexpr (KIND == kKindProjective) {
                // per label, the neighbours to visit grouped by class (kIn, then kFront, then kGeneral; kOut
                // entries are left out): one warp per label, N <= 32
                for (int l = tid >> 5; l < LBa; l += kThreads / 32) {
                    const uint32_t mode = lane < N ? (sH[lane * LBa + l].pm >> 28) : (uint32_t)kOut;
                    const unsigned mi = __ballot_sync(kFull, mode == kIn);
                    const unsigned mf = __ballot_sync(kFull, mode == kFront);
                    const unsigned mg = __ballot_sync(kFull, mode == kGeneral);
                    const unsigned lt = (1u << lane) - 1u;
                    const int ci = __popc(mi), cf = __popc(mf);
                    int pos = -1;
                    if (mode == kIn) pos = __popc(mi & lt);
                    else if (mode == kFront) pos = ci + __popc(mf & lt);
                    else if (mode == kGeneral) pos = ci + cf + __popc(mg & lt);
                    if (pos >= 0) sOrd[l * N + pos] = (uint8_t)lane;
                    if (lane == 0) sCnt[l] = ci | (cf << 8) | (__popc(mg) << 16);
                }
                __syncthreads();
            }
        }

        // Per pixel slot, whether the warp's 32 pixels belong to one segment (uni: one reduction, lane 0's key)
        // or to none (none: nothing to add); decided once per item instead of once per label.
        unsigned uni = 0, none = 0;
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
            const int kf = __shfl_sync(kFull, key[j], 0), kl = __shfl_sync(kFull, key[j], 31);
            if (kf == kl) {
                if (kf != kSentinel) uni |= 1u << j;
                else none |= 1u << j;
            }
        }
        for (int l = 0; l < LBa; ++l) {
            int m[kPPT];
#pragma unroll
            for (int j = 0; j < kPPT; ++j)
                m[j] = (COMB == FTV_COMBINE_MIN && N > 0) ? (PF ? penalty : INT_MAX) : 0;
            if constexpr (KIND == kKindProjective) {
                const int cnt = sCnt[l];
                const int ci = cnt & 0xff, cf = ci + ((cnt >> 8) & 0xff), cg = cf + (cnt >> 16);
                const uint8_t* ord = &sOrd[l * N];
#pragma unroll 2  // two entries in flight: measured 2 % faster on the 4K rig together with the uniform mask
                for (int k = 0; k < ci; ++k) {  // every pixel's sample is in view
                    const int n = ord[k];
                    const float4* e4 = reinterpret_cast<const float4*>(&sH[n * LBa + l]);
                    const float4 ha = e4[0], hb = e4[1], hc = e4[2];
                    const void* tex = sBase[n];
                    const int pitch = (int)(__float_as_uint(hc.w) & kPitchMask);
                    const unsigned lim = (unsigned)pitch * __float_as_uint(hc.z);  // texels of the view
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        const float X = __fmaf_rn(ha.x, px[j], __fmaf_rn(ha.y, py[j], ha.z));
                        const float Yh = __fmaf_rn(ha.w, px[j], __fmaf_rn(hb.x, py[j], hb.y));
                        const float Wz = __fmaf_rn(hb.z, px[j], __fmaf_rn(hb.w, py[j], hc.x));
                        const float r = contract_rcp_normal<FAST_RCP>(Wz);
                        const int ui = __float2int_rd(__fadd_rn(__fmul_rn(X, r), 0.5f));
                        const int vi = __float2int_rd(__fadd_rn(__fmul_rn(Yh, r), 0.5f));
#ifdef FTV_CHECKED
                        accumulate<FMT, COMB, false>(m[j], true, tex, vi * pitch + ui, ra[j], rb[j], rc[j], penalty, lim,
                                                     ck);
#else
                        const int cst = TexelOps<FMT>::cost(tex, vi * pitch + ui, ra[j], rb[j], rc[j]);
                        m[j] = COMB == FTV_COMBINE_MIN ? min(m[j], cst) : m[j] + cst;
#endif
                    }
                }
                for (int k = ci; k < cf; ++k) {  // Wz proven positive and normal: range tests only
                    const int n = ord[k];
                    const float4* e4 = reinterpret_cast<const float4*>(&sH[n * LBa + l]);
                    const float4 ha = e4[0], hb = e4[1], hc = e4[2];
                    const void* tex = sBase[n];
                    const int pitch = (int)(__float_as_uint(hc.w) & kPitchMask);
                    const unsigned lim = (unsigned)pitch * __float_as_uint(hc.z);  // texels of the view
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        const float X = __fmaf_rn(ha.x, px[j], __fmaf_rn(ha.y, py[j], ha.z));
                        const float Yh = __fmaf_rn(ha.w, px[j], __fmaf_rn(hb.x, py[j], hb.y));
                        const float Wz = __fmaf_rn(hb.z, px[j], __fmaf_rn(hb.w, py[j], hc.x));
                        const float r = contract_rcp_normal<FAST_RCP>(Wz);
                        const int ui = __float2int_rd(__fadd_rn(__fmul_rn(X, r), 0.5f));
                        const int vi = __float2int_rd(__fadd_rn(__fmul_rn(Yh, r), 0.5f));
                        const bool ok = ((unsigned)ui < __float_as_uint(hc.y)) & ((unsigned)vi < __float_as_uint(hc.z));
                        accumulate<FMT, COMB, PF>(m[j], ok, tex, vi * pitch + ui, ra[j], rb[j], rc[j], penalty, lim, ck);
                    }
                }
                for (int k = cf; k < cg; ++k) {  // the contract's sequence as written
                    const int n = ord[k];
                    const float4* e4 = reinterpret_cast<const float4*>(&sH[n * LBa + l]);
                    const float4 ha = e4[0], hb = e4[1], hc = e4[2];
                    const void* tex = sBase[n];
                    const int pitch = (int)(__float_as_uint(hc.w) & kPitchMask);
                    const unsigned lim = (unsigned)pitch * __float_as_uint(hc.z);  // texels of the view
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        int idx;
                        const bool ok = pos_general<FAST_RCP>(ha, hb, hc, pitch, px[j], py[j], idx);
                        accumulate<FMT, COMB, PF>(m[j], ok, tex, idx, ra[j], rb[j], rc[j], penalty, lim, ck);
                    }
                }
                if (!(COMB == FTV_COMBINE_MIN && PF) && cg < N) {  // entries out of view: the penalty each
#pragma unroll
                    for (int j = 0; j < kPPT; ++j)
                        m[j] = (COMB == FTV_COMBINE_MIN) ? min(m[j], penalty) : m[j] + (N - cg) * penalty;
                }
            }
            for (int n = 0; n < (KIND == kKindProjective ? 0 : N); ++n) {
                const float4* e4 = reinterpret_cast<const float4*>(&sH[n * LBa + l]);
                const float4 hc = e4[2];
                const void* tex = sBase[n];
                const uint32_t pm = __float_as_uint(hc.w);
                const uint32_t mode = pm >> 28;
                const int pitch = (int)(pm & kPitchMask);
                const unsigned lim = (unsigned)pitch * __float_as_uint(hc.z);  // texels of the view
                // a projective-only launch (no entry with h6 = h7 = 0) keeps the general path alone; a
                // rectified-only instantiation measured slower than this mixed loop, so there is none
                if (precise_kind(KIND)) {
                    const double* h64 = &Jp->H64[((int64_t)n * L + d0 + l) * 9];
                    const int wv = __float_as_int(hc.y), hv = __float_as_int(hc.z);
                    if (mode == kOut) {
                        if (!(COMB == FTV_COMBINE_MIN && PF)) {
#pragma unroll
                            for (int j = 0; j < kPPT; ++j)
                                m[j] = (COMB == FTV_COMBINE_MIN) ? min(m[j], penalty) : m[j] + penalty;
                        }
                    } else if (mode == kSlow) {
#pragma unroll
                        for (int j = 0; j < kPPT; ++j) {
                            const long long q = project_fp64_packed(h64, (int)px[j] + fx0, iy[j], wv, hv);
                            n_recomputed += key[j] != kSentinel;
                            const int idx = (int)(q >> 32) * pitch + (int)(unsigned)q;
                            accumulate<FMT, COMB, PF>(m[j], q >= 0, tex, idx, ra[j], rb[j], rc[j], penalty, lim, ck);
                        }
                    } else if (KIND == kKindPreciseMixed && mode == kShift) {
                        const float4 hb = e4[1];  // (h4, h5, lower and upper bound of x')
                        const int D = __float_as_int(hc.x);
#pragma unroll
                        for (int j = 0; j < kPPT; ++j) {
                            const bool ok = (px[j] >= hb.z) & (px[j] < hb.w);
                            accumulate<FMT, COMB, PF>(m[j], ok, tex, rowx[j] + D, ra[j], rb[j], rc[j], penalty, lim, ck);
                        }
                    } else if (KIND == kKindPreciseMixed && mode == kRect) {
                        const float a2 = e4[0].z;
                        const float4 pe = reinterpret_cast<const float4*>(sP)[n * LBa + l];
                        const int u0 = __float_as_int(pe.x), dv0 = __float_as_int(pe.y) - fy0;
#pragma unroll
                        for (int j = 0; j < kPPT; ++j) {
                            const float tu = __fadd_rn(__fadd_rn(px[j], a2), 0.5f);
                            const float fu = floorf(tu);
                            int ui = __float2int_rz(fu) + u0, vi = iy[j] + dv0;
                            bool ok;
                            if (fabsf(__fsub_rn(__fsub_rn(tu, fu), 0.5f)) >= pe.z) {
                                const long long q = project_fp64_packed(h64, (int)px[j] + fx0, iy[j], wv, hv);
                                ok = q >= 0;
                                ui = (int)(unsigned)q;
                                vi = (int)(q >> 32);
                                n_recomputed += key[j] != kSentinel;
                            } else {
                                ok = ((unsigned)ui < (unsigned)wv) & ((unsigned)vi < (unsigned)hv);
                            }
                            accumulate<FMT, COMB, PF>(m[j], ok, tex, vi * pitch + ui, ra[j], rb[j], rc[j], penalty, lim, ck);
                        }
                    } else {
                        const float4 ha = e4[0], hb = e4[1];
                        const float4 pe = reinterpret_cast<const float4*>(sP)[n * LBa + l];
                        const int u0 = __float_as_int(pe.x), v0 = __float_as_int(pe.y);
#pragma unroll
                        for (int j = 0; j < kPPT; ++j) {
                            const float X = __fmaf_rn(ha.x, px[j], __fmaf_rn(ha.y, py[j], ha.z));
                            const float Yh = __fmaf_rn(ha.w, px[j], __fmaf_rn(hb.x, py[j], hb.y));
                            const float Wz = __fmaf_rn(hb.z, px[j], __fmaf_rn(hb.w, py[j], hc.x));
                            const float r = contract_rcp<FAST_RCP>(Wz);
                            const float tu = __fadd_rn(__fmul_rn(X, r), 0.5f);
                            const float tv = __fadd_rn(__fmul_rn(Yh, r), 0.5f);
                            const float fu = floorf(tu), fv = floorf(tv);
                            const bool near = fabsf(__fsub_rn(__fsub_rn(tu, fu), 0.5f)) >= pe.z ||
                                              fabsf(__fsub_rn(__fsub_rn(tv, fv), 0.5f)) >= pe.w;
                            int ui = __float2int_rz(fu) + u0, vi = __float2int_rz(fv) + v0;
                            bool ok;
                            if (near) {
                                const long long q = project_fp64_packed(h64, (int)px[j] + fx0, iy[j], wv, hv);
                                ok = q >= 0;
                                ui = (int)(unsigned)q;
                                vi = (int)(q >> 32);
                                n_recomputed += key[j] != kSentinel;
                            } else {
                                ok = ((unsigned)ui < (unsigned)wv) & ((unsigned)vi < (unsigned)hv);
                            }
                            accumulate<FMT, COMB, PF>(m[j], ok, tex, vi * pitch + ui, ra[j], rb[j], rc[j], penalty, lim, ck);
                        }
                    }
                } else if (KIND == kKindMixed && mode == kShift) {
                    const float4 hb = e4[1];  // (h4, h5, -D, w - D)
                    const int D = __float_as_int(hc.x);
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        const bool ok = (px[j] >= hb.z) & (px[j] < hb.w);
                        accumulate<FMT, COMB, false>(m[j], ok, tex, rowx[j] + D, ra[j], rb[j], rc[j], penalty, lim, ck);
                    }
                } else if (KIND == kKindMixed && mode == kRect) {
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        int idx;
                        const bool ok = pos_rect(hc.x, __float_as_uint(hc.y), __float_as_uint(hc.z), pitch, px[j], iy[j],
                                                 idx);
                        accumulate<FMT, COMB, false>(m[j], ok, tex, idx, ra[j], rb[j], rc[j], penalty, lim, ck);
                    }
                } else if (KIND == kKindMixed && mode == kGeneral) {
                    const float4 ha = e4[0], hb = e4[1];
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        int idx;
                        const bool ok = pos_general<FAST_RCP>(ha, hb, hc, pitch, px[j], row_f(j), idx);
                        accumulate<FMT, COMB, PF>(m[j], ok, tex, idx, ra[j], rb[j], rc[j], penalty, lim, ck);
                    }
                } else if (KIND == kKindMixed && mode == kUnit) {
                    const float4 ha = e4[0], hb = e4[1];
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        int idx;
                        const bool ok = pos_affine<true>(ha, hb, hc, 1.0f, pitch, px[j], row_f(j), idx);
                        accumulate<FMT, COMB, false>(m[j], ok, tex, idx, ra[j], rb[j], rc[j], penalty, lim, ck);
                    }
                } else if (KIND == kKindMixed && mode == kAffine) {
                    const float4 ha = e4[0], hb = e4[1];
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        int idx;
                        const bool ok = pos_affine<false>(ha, hb, hc, hb.z, pitch, px[j], row_f(j), idx);
                        accumulate<FMT, COMB, false>(m[j], ok, tex, idx, ra[j], rb[j], rc[j], penalty, lim, ck);
                    }
                } else if (KIND == kKindMixed && !(COMB == FTV_COMBINE_MIN && PF)) {
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) m[j] = (COMB == FTV_COMBINE_MIN) ? min(m[j], penalty) : m[j] + penalty;
                }
            }
            // segmented warp reduction: keys are nondecreasing along the lanes
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                const int v = key[j] != kSentinel ? m[j] : 0;
                const int kfirst = key[j];  // lane 0's key is the warp's when uni
                if ((uni | none) >> j & 1u) {
                    if (uni >> j & 1u) {
                        const int sum = __reduce_add_sync(kFull, v);
                        if (lane == 0) {
                            if (kfirst < kSegAcc) atomicAdd(&sAcc[kfirst * kMaxLB + l], sum);
                            else {
                                const int s = list ? list[k0 + kfirst] : k0 + kfirst;
                                atomicAdd(&cost[(int64_t)s * L + d0 + l], sum);
                            }
                        }
                    }
                } else {
                    unsigned rem = kFull;
                    while (rem) {
                        const int leader = __ffs(rem) - 1;
                        const int kk = __shfl_sync(kFull, key[j], leader);
                        const unsigned grp = __ballot_sync(kFull, key[j] == kk);
                        const int sum = __reduce_add_sync(kFull, key[j] == kk ? v : 0);
                        if (lane == leader && kk != kSentinel) {
                            if (kk < kSegAcc) atomicAdd(&sAcc[kk * kMaxLB + l], sum);
                            else {
                                const int s = list ? list[k0 + kk] : k0 + kk;
                                atomicAdd(&cost[(int64_t)s * L + d0 + l], sum);
                            }
                        }
                        rem &= ~grp;
                    }
                }
            }
        }
        __syncthreads();

        // write the row slices of this tile's segments
        const int nacc = min(nk, kSegAcc);
        for (int i = tid; i < nacc * LBa; i += kThreads) {
            const int loc = i / LBa, l = i - loc * LBa;
            const int k = k0 + loc;
            const int s = list ? list[k] : k;
            const int v = sAcc[loc * kMaxLB + l];
            sAcc[loc * kMaxLB + l] = 0;
            if ((unsigned)s >= (unsigned)Jp->S) continue;  // an invalid list entry owns no pixels
            const int a = cached ? sWoffs[loc] : woffs[k];
            const int b = cached ? sWoffs[loc + 1] : woffs[k + 1];
            int32_t* dst = &cost[(int64_t)s * L + d0 + l];
            if (a >= w0 && b <= w0 + kTile) *dst = v;
            else atomicAdd(dst, v);
        }
    }
    if constexpr (precise_kind(KIND)) {
        const unsigned n = __reduce_add_sync(kFull, n_recomputed);
        if (lane == 0 && n) atomicAdd(&plan->recomputed, (unsigned long long)n);
    }
}

template <int FMT, int COMB, bool FAST>
int blocks_per_sm_for() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cost_kernel<FMT, COMB, FAST, COMB == FTV_COMBINE_MIN, kKindMixed>,
                                                      kThreads, 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

// Exhaustive comparison with the IEEE reciprocal over every positive float below 2^126: subnormals go
// through rcp_scaled's scaling, normals through rcp_newton directly.
__global__ void reciprocal_check_kernel(unsigned long long* mismatches) {
    const uint32_t lo = 0x00000001u, hi = 0x7e800000u;
    unsigned long long bad = 0;
    for (uint64_t i = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const float w = __uint_as_float((uint32_t)i);
        bad += __float_as_uint(rcp_scaled(w)) != __float_as_uint(__frcp_rn(w));
    }
    bad = __reduce_add_sync(0xffffffffu, (unsigned)bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(mismatches, bad);
}

std::mutex g_rcp_mutex;
int8_t g_rcp_state[64] = {};  // per device: 0 unknown, 1 exact, -1 not exact

}  // namespace

int64_t reciprocal_mismatches() {
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) return -1;
    unsigned long long h = 0;
    int n_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMemset(d, 0, sizeof(h));
    if (e == cudaSuccess) {
        reciprocal_check_kernel<<<std::max(1, n_sm) * 8, 256>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? (int64_t)h : -1;
}

bool fast_reciprocal_exact() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lock(g_rcp_mutex);
    if (g_rcp_state[dev] == 0) g_rcp_state[dev] = reciprocal_mismatches() == 0 ? 1 : -1;
    return g_rcp_state[dev] == 1;
}

int cost_blocks_per_sm(int fmt, int combine, bool fast) {
#define FTV_OCC(F, C) (fast ? blocks_per_sm_for<F, C, true>() : blocks_per_sm_for<F, C, false>())
    if (fmt == FMT_U8X4) return combine == FTV_COMBINE_MIN ? FTV_OCC(FMT_U8X4, FTV_COMBINE_MIN)
                                                           : FTV_OCC(FMT_U8X4, FTV_COMBINE_SUM);
    if (fmt == FMT_P10) return combine == FTV_COMBINE_MIN ? FTV_OCC(FMT_P10, FTV_COMBINE_MIN)
                                                          : FTV_OCC(FMT_P10, FTV_COMBINE_SUM);
    return combine == FTV_COMBINE_MIN ? FTV_OCC(FMT_U16X4, FTV_COMBINE_MIN) : FTV_OCC(FMT_U16X4, FTV_COMBINE_SUM);
#undef FTV_OCC
}

namespace {

// Shared-memory carveout hint: the smallest split that still holds kMinBlocks CTAs of this kernel, so
// that the rest of the SM's L1 caches the neighbour-view gathers. Once per instantiation and process.
template <typename Kernel>
bool prefer_l1(Kernel kernel) {
    cudaFuncAttributes a{};
    int dev = 0, smem_sm = 0;
    if (cudaFuncGetAttributes(&a, kernel) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        smem_sm > 0) {
        const size_t need = (size_t)kMinBlocks * (a.sharedSizeBytes + 1024);
        const int pct = (int)std::min<size_t>(100, (need * 100 + smem_sm - 1) / smem_sm);
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    }
    cudaGetLastError();  // a hint only
    return true;
}

template <int FMT, int COMB, bool FAST, bool PF, int KIND>
void launch_one(const RefJob* jobs, Plan* p, int ck, int nck, int grid, cudaStream_t s) {
    static const bool hinted = prefer_l1(cost_kernel<FMT, COMB, FAST, PF, KIND>);
    (void)hinted;
    cost_kernel<FMT, COMB, FAST, PF, KIND><<<grid, kThreads, 0, s>>>(jobs, p, ck, nck);
}

template <int FMT, int COMB, bool FAST, bool PF>
void launch_kind(const RefJob* jobs, Plan* p, int kind, int ck, int nck, int grid, cudaStream_t s) {
    if (kind == kKindPrecise) launch_one<FMT, COMB, FAST, PF, kKindPrecise>(jobs, p, ck, nck, grid, s);
    else if (kind == kKindPreciseMixed) launch_one<FMT, COMB, FAST, PF, kKindPreciseMixed>(jobs, p, ck, nck, grid, s);
    else if (kind == kKindProjective) launch_one<FMT, COMB, FAST, PF, kKindProjective>(jobs, p, ck, nck, grid, s);
    else launch_one<FMT, COMB, FAST, PF, kKindMixed>(jobs, p, ck, nck, grid, s);
}

template <int FMT, int COMB>
void launch_fast_pf(const RefJob* jobs, Plan* p, bool fast, bool pf, int kind, int ck, int nck, int grid,
                    cudaStream_t s) {
    const bool use_pf = COMB == FTV_COMBINE_MIN && pf;
    if (fast) {
        if (use_pf) launch_kind<FMT, COMB, true, true>(jobs, p, kind, ck, nck, grid, s);
        else launch_kind<FMT, COMB, true, false>(jobs, p, kind, ck, nck, grid, s);
    } else {
        if (use_pf) launch_kind<FMT, COMB, false, true>(jobs, p, kind, ck, nck, grid, s);
        else launch_kind<FMT, COMB, false, false>(jobs, p, kind, ck, nck, grid, s);
    }
}

template <int FMT>
void launch_comb(const RefJob* jobs, Plan* p, int combine, bool fast, bool pf, int kind, int ck, int nck, int grid,
                 cudaStream_t s) {
    if (combine == FTV_COMBINE_MIN) launch_fast_pf<FMT, FTV_COMBINE_MIN>(jobs, p, fast, pf, kind, ck, nck, grid, s);
    else launch_fast_pf<FMT, FTV_COMBINE_SUM>(jobs, p, fast, pf, kind, ck, nck, grid, s);
}

}  // namespace

cudaError_t launch_cost(const RefJob* jobs, const Plan* plan, int fmt, int combine, bool fast, bool pf, int kind,
                        int chunk, int chunks, int grid, cudaStream_t s) {
    if (chunks < 1 || chunks > kMaxChunks || chunk < 0 || chunk >= chunks) return cudaErrorInvalidValue;
    Plan* p = const_cast<Plan*>(plan);
    if (fmt == FMT_U8X4) launch_comb<FMT_U8X4>(jobs, p, combine, fast, pf, kind, chunk, chunks, grid, s);
    else if (fmt == FMT_P10) launch_comb<FMT_P10>(jobs, p, combine, fast, pf, kind, chunk, chunks, grid, s);
    else launch_comb<FMT_U16X4>(jobs, p, combine, fast, pf, kind, chunk, chunks, grid, s);
    return cudaGetLastError();
}

}  // namespace ftv
