// Centre table: Eq. 4 evaluated the way the paper states it, on a window around each segment's centre,
// together with the segment s' of the neighbouring view that the centre maps to (the correspondence
// Eq. 5 needs to form M = min{0, m - K} when d_s = d_s').
//
// Paper, Sec. III-C: m_{s,s'}(d_s) = 1/size(W) * sum_{w in W} || YCbCr(mu_s + w) - YCbCr(T[mu_s] + w) ||_1
// with mu_s the centre of segment s and T[.] the transform into the neighbouring view for depth d_s;
// the matching is done "only for centers of segments". Here:
//   mu_s  = integer centroid floor((2 sum x + n) / (2 n)) of the segment's n pixels (the paper does not
//           define the centre);
//   T     = the same projection as the cost volume: the FP32 homography and rounding, or the FP64
//           projection for FP64-precision contexts;
//   m     = the raw window sum (the consumer divides by size(W)); a window pair with a position outside
//           its image, or a centre that projects out of view, costs the out-of-view penalty;
//   s'    = the neighbour view's label at T[mu_s] (-1 when out of view or no label map is given).
// Work: one thread per (segment, label, neighbour); this is not the volume's hot loop (one window per
// segment instead of every pixel), so the contract's sequence is written out literally.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "ftv_internal.h"
#include "ftv_project.cuh"

namespace ftv {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void texel(const void* base, int fmt, int64_t i, int* v) {
    if (fmt == FMT_U16X4) {
        const uint2 t = static_cast<const uint2*>(base)[i];
        v[0] = t.x & 0xffff;
        v[1] = t.x >> 16;
        v[2] = t.y;
    } else {
        const uint32_t t = static_cast<const uint32_t*>(base)[i];
        const int sh = fmt == FMT_P10 ? 10 : 8;
        const uint32_t m = (1u << sh) - 1u;
        v[0] = t & m;
        v[1] = (t >> sh) & m;
        v[2] = t >> (2 * sh);
    }
}

// One warp per segment: rounded mean of its pixel coordinates from the segment index. (-1, -1) marks
// an empty segment.
__global__ void centroid_kernel(const int32_t* __restrict__ offs, const uint32_t* __restrict__ pix, int S,
                                int2* __restrict__ centre) {
    const int lane = threadIdx.x & 31;
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += (gridDim.x * blockDim.x) >> 5) {
        const int b = offs[s], e = offs[s + 1];
        long long sx = 0, sy = 0;
        for (int i = b + lane; i < e; i += 32) {
            const uint32_t xy = pix[i];
            sx += xy & 0xffff;
            sy += xy >> 16;
        }
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(kFull, sx, o);
            sy += __shfl_xor_sync(kFull, sy, o);
        }
        if (lane == 0) {
            const long long n = e - b;
            centre[s] = n > 0 ? make_int2((int)((2 * sx + n) / (2 * n)), (int)((2 * sy + n) / (2 * n))) : make_int2(-1, -1);
        }
    }
}

struct CentreArgs {
    const int2* centre;
    const float* H;         // [N][L][9]
    const double* H64;      // [N][L][9] unrounded table, FP64-precision contexts (else nullptr)
    const void* ref_tex;    // packed reference view
    const NbrView* nbrs;    // [N]
    const int32_t* const* labels_v;  // [N] neighbour label maps (entries may be null)
    int32_t* m;             // [S][L][N]
    int32_t* sp;            // [S][L][N]
    int32_t S, L, N, W, H_, window, penalty, fmt;
    uint32_t l_magic;       // ceil(2^32 / L) for L > 1: j / L = umulhi(j, l_magic) for j < 2^20
};

constexpr int kCentreThreads = 256;
constexpr int kMaxWindow = 15;

// One CTA per segment (grid-stride): the segment's reference window is unpacked once into shared memory
// (-1 marks a pixel outside the reference image), then the CTA's threads take the segment's (label,
// neighbour) entries, label fastest: a warp then works on consecutive labels of one neighbour, whose
// windows lie a few pixels apart in that view and share its cache lines. Any odd window up to 15; the
// paper's 3x3 takes centre_table3_kernel.
__global__ void __launch_bounds__(kCentreThreads) centre_table_kernel(CentreArgs a) {
    __shared__ int sref[kMaxWindow * kMaxWindow][3];
    __shared__ NbrView snb[FTV_MAX_NBRS];
    __shared__ const int32_t* slab[FTV_MAX_NBRS];
    const int tid = threadIdx.x;
    for (int k = tid; k < a.N; k += kCentreThreads) {
        snb[k] = a.nbrs[k];
        slab[k] = a.labels_v[k];
    }
    const int win = a.window;
    const int half = win / 2, ww = win * win, nent = a.L * a.N;
    for (int s = blockIdx.x; s < a.S; s += gridDim.x) {
        const int2 c = a.centre[s];
        __syncthreads();  // the previous segment's window is no longer read
        for (int i = tid; i < ww; i += kCentreThreads) {
            const int iy = i / win;  // per segment only
            const int rx = c.x - half + (i - iy * win), ry = c.y - half + iy;
            if (c.x >= 0 && rx >= 0 && rx < a.W && ry >= 0 && ry < a.H_) {
                int v[3];
                texel(a.ref_tex, a.fmt, (int64_t)ry * a.W + rx, v);
                sref[i][0] = v[0];
                sref[i][1] = v[1];
                sref[i][2] = v[2];
            } else {
                sref[i][0] = -1;
            }
        }
        __syncthreads();
        int32_t* mrow = a.m + (int64_t)s * nent;
        int32_t* srow = a.sp + (int64_t)s * nent;
        for (int j = tid; j < nent; j += kCentreThreads) {
            const int k = a.L == 1 ? j : (int)__umulhi((uint32_t)j, a.l_magic), d = j - k * a.L;
            const int64_t out = (int64_t)d * a.N + k;
            const NbrView& nv = snb[k];
            const float* h = a.H + ((int64_t)k * a.L + d) * 9;
            bool in = c.x >= 0;
            int ui = 0, vi = 0;
            if (in && a.H64) {
                in = project_fp64(a.H64 + ((int64_t)k * a.L + d) * 9, c.x, c.y, nv.w, nv.h, &ui, &vi);
            } else if (in) {
                const float x = (float)c.x, y = (float)c.y;
                const float X = __fmaf_rn(__ldg(&h[0]), x, __fmaf_rn(__ldg(&h[1]), y, __ldg(&h[2])));
                const float Yh = __fmaf_rn(__ldg(&h[3]), x, __fmaf_rn(__ldg(&h[4]), y, __ldg(&h[5])));
                const float Wz = __fmaf_rn(__ldg(&h[6]), x, __fmaf_rn(__ldg(&h[7]), y, __ldg(&h[8])));
                in = Wz > 0.0f;
                if (in) {
                    const float r = __frcp_rn(Wz);
                    const float fu = floorf(__fadd_rn(__fmul_rn(X, r), 0.5f));
                    const float fv = floorf(__fadd_rn(__fmul_rn(Yh, r), 0.5f));
                    in = fu >= 0.0f && fu <= (float)(nv.w - 1) && fv >= 0.0f && fv <= (float)(nv.h - 1);
                    if (in) {
                        ui = (int)fu;
                        vi = (int)fv;
                    }
                }
            }
            int m = 0;
            if (!in) {
                m = ww * a.penalty;
            } else {
                const bool inside = ui >= half && ui + half < nv.w && vi >= half && vi + half < nv.h;
                for (int wy = 0; wy < win; ++wy) {
                    const int qy = vi - half + wy;
                    const int64_t qrow = (int64_t)qy * nv.pitch;
                    for (int wx = 0; wx < win; ++wx) {
                        const int i = wy * win + wx, qx = ui - half + wx;
                        if (sref[i][0] < 0 || (!inside && (qx < 0 || qx >= nv.w || qy < 0 || qy >= nv.h))) {
                            m += a.penalty;
                            continue;
                        }
                        int q[3];
                        texel(nv.texels, a.fmt, qrow + qx, q);
                        m += (int)__sad(sref[i][0], q[0], __sad(sref[i][1], q[1], __sad(sref[i][2], q[2], 0u)));
                    }
                }
            }
            mrow[out] = m;
            const int32_t* lv = slab[k];
            srow[out] = (in && lv) ? lv[(int64_t)vi * nv.w + ui] : -1;
        }
    }
}

// Texel of a packed view with the format fixed at compile time.
template <int FMT>
__device__ __forceinline__ void texel_t(const void* base, int64_t i, int& p, int& q, int& r) {
    if (FMT == FMT_U16X4) {
        const uint2 t = __ldg(static_cast<const uint2*>(base) + i);
        p = t.x & 0xffff;
        q = t.x >> 16;
        r = t.y;
    } else {
        const uint32_t t = __ldg(static_cast<const uint32_t*>(base) + i);
        constexpr int sh = FMT == FMT_P10 ? 10 : 8;
        constexpr uint32_t mk = (1u << sh) - 1u;
        p = t & mk;
        q = (t >> sh) & mk;
        r = t >> (2 * sh);
    }
}

// The paper's 3x3 window (FMT at compile time). Same results as centre_table_kernel; per segment the 27
// reference samples move from shared memory into registers (every entry of the segment reads them), and
// an entry whose two windows lie inside both images, the common case, sums its nine pixel pairs with no
// per-pixel test. Entry j of a segment is (neighbour k, label d) with j = k L + d, so its homography is
// the table's entry j. Four CTAs per SM (64 registers): the kernel is latency-bound (each entry is a
// dependent chain of loads), and the fourth CTA measured 5 % faster than three at 80 registers; unrolling
// two entries per iteration measured slower.
template <int FMT>
__global__ void __launch_bounds__(kCentreThreads, 4) centre_table3_kernel(CentreArgs a) {
    __shared__ int sref[9][3];
    __shared__ NbrView snb[FTV_MAX_NBRS];
    __shared__ const int32_t* slab[FTV_MAX_NBRS];
    const int tid = threadIdx.x;
    for (int k = tid; k < a.N; k += kCentreThreads) {
        snb[k] = a.nbrs[k];
        slab[k] = a.labels_v[k];
    }
    const int nent = a.L * a.N;
    for (int s = blockIdx.x; s < a.S; s += gridDim.x) {
        const int2 c = a.centre[s];
        __syncthreads();  // the previous segment's window is no longer read
        if (tid < 9) {
            const int rx = c.x - 1 + tid % 3, ry = c.y - 1 + tid / 3;
            if (c.x >= 0 && rx >= 0 && rx < a.W && ry >= 0 && ry < a.H_) {
                texel_t<FMT>(a.ref_tex, (int64_t)ry * a.W + rx, sref[tid][0], sref[tid][1], sref[tid][2]);
            } else {
                sref[tid][0] = -1;
            }
        }
        __syncthreads();
        int rv[9][3];
        bool ref_in = true;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            rv[i][0] = sref[i][0];
            rv[i][1] = sref[i][1];
            rv[i][2] = sref[i][2];
            ref_in = ref_in && rv[i][0] >= 0;
        }
        int32_t* mrow = a.m + (int64_t)s * nent;
        int32_t* srow = a.sp + (int64_t)s * nent;
        for (int j = tid; j < nent; j += kCentreThreads) {
            const int k = a.L == 1 ? j : (int)__umulhi((uint32_t)j, a.l_magic), d = j - k * a.L;
            const int64_t out = (int64_t)d * a.N + k;
            const NbrView nv = snb[k];
            bool in = c.x >= 0;
            int ui = 0, vi = 0;
            if (in && a.H64) {
                in = project_fp64(a.H64 + (int64_t)j * 9, c.x, c.y, nv.w, nv.h, &ui, &vi);
            } else if (in) {
                const float* h = a.H + (int64_t)j * 9;
                const float x = (float)c.x, y = (float)c.y;
                const float X = __fmaf_rn(__ldg(&h[0]), x, __fmaf_rn(__ldg(&h[1]), y, __ldg(&h[2])));
                const float Yh = __fmaf_rn(__ldg(&h[3]), x, __fmaf_rn(__ldg(&h[4]), y, __ldg(&h[5])));
                const float Wz = __fmaf_rn(__ldg(&h[6]), x, __fmaf_rn(__ldg(&h[7]), y, __ldg(&h[8])));
                in = Wz > 0.0f;
                if (in) {
                    const float r = __frcp_rn(Wz);
                    const float fu = floorf(__fadd_rn(__fmul_rn(X, r), 0.5f));
                    const float fv = floorf(__fadd_rn(__fmul_rn(Yh, r), 0.5f));
                    in = fu >= 0.0f && fu <= (float)(nv.w - 1) && fv >= 0.0f && fv <= (float)(nv.h - 1);
                    if (in) {
                        ui = (int)fu;
                        vi = (int)fv;
                    }
                }
            }
            int m = 0;
            if (!in) {
                m = 9 * a.penalty;
            } else if (ref_in && ui >= 1 && ui + 1 < nv.w && vi >= 1 && vi + 1 < nv.h) {
                const int64_t base = (int64_t)(vi - 1) * nv.pitch + (ui - 1);
#pragma unroll
                for (int wy = 0; wy < 3; ++wy)
#pragma unroll
                    for (int wx = 0; wx < 3; ++wx) {
                        int p, q, r;
                        texel_t<FMT>(nv.texels, base + (int64_t)wy * nv.pitch + wx, p, q, r);
                        const int i = wy * 3 + wx;
                        m += (int)__sad(rv[i][0], p, __sad(rv[i][1], q, __sad(rv[i][2], r, 0u)));
                    }
            } else {
#pragma unroll
                for (int wy = 0; wy < 3; ++wy)
#pragma unroll
                    for (int wx = 0; wx < 3; ++wx) {
                        const int i = wy * 3 + wx, qx = ui - 1 + wx, qy = vi - 1 + wy;
                        if (rv[i][0] < 0 || qx < 0 || qx >= nv.w || qy < 0 || qy >= nv.h) {
                            m += a.penalty;
                            continue;
                        }
                        int p, q, r;
                        texel_t<FMT>(nv.texels, (int64_t)qy * nv.pitch + qx, p, q, r);
                        m += (int)__sad(rv[i][0], p, __sad(rv[i][1], q, __sad(rv[i][2], r, 0u)));
                    }
            }
            mrow[out] = m;
            const int32_t* lv = slab[k];
            srow[out] = (in && lv) ? lv[(int64_t)vi * nv.w + ui] : -1;
        }
    }
}

// One 3x3 window pair's sum for 4-byte texels: t[i] the neighbour's packed texels (Y | Cb << sh | Cr << 2 sh),
// ref[i] the reference's samples (Y, Cb, Cr, unused), read from shared memory (one broadcast load each).
// Each window row accumulates in its own chain (three independent chains of nine absolute differences
// instead of one of 27), which shortens the dependent path of an entry.
template <int FMT>
__device__ __forceinline__ int window_sum(const uint32_t* t, const int4* ref) {
    constexpr int sh = FMT == FMT_P10 ? 10 : 8;
    constexpr uint32_t mk = (1u << sh) - 1u;
    unsigned m[3] = {0u, 0u, 0u};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int4 r = ref[i];
        unsigned& a = m[i / 3];
        a = __sad(t[i] & mk, (unsigned)r.x, __sad((t[i] >> sh) & mk, (unsigned)r.y, __sad(t[i] >> (2 * sh), (unsigned)r.z, a)));
    }
    return (int)(m[0] + m[1] + m[2]);
}

// The paper's 3x3 window for 4-byte texels (8- and 10-bit samples) in FP32-contract contexts: the results
// of centre_table_kernel, with the roles of entries and segments exchanged. A work item is (a chunk of 256
// consecutive entries, a group of kGroup consecutive segments); each thread owns one entry of the chunk
// (neighbour k, label d) and holds its homography and the neighbour view's geometry in registers, so the
// per-(segment, entry) chain starts at the projection instead of at nine homography loads. The CTA stages
// the group's centres and reference windows in shared memory; the next item's stage is loaded into
// registers while the current group is worked on and stored to the other buffer afterwards (one barrier
// per item). Within a group each thread software-pipelines its segments: the next segment's projection is
// computed while the current window's nine gathers are in flight. Windows that touch an image border take
// the checked loop. The reciprocal is the Newton-Raphson step where the start-up check found it exact.
constexpr int kGroup = 16;
static_assert(9 * kGroup <= kCentreThreads, "one stage sample per thread");

struct CentreStage {
    int4 ref[kGroup * 9];  // reference samples (Y, Cb, Cr, 0), segment-major
    int2 c[kGroup];        // centres; (-1, -1) for an empty segment
    int inside[kGroup];    // the segment's 3x3 window lies inside the reference image
};

// One thread's share of a group's stage: thread t < 9 kGroup loads sample t % 9 of segment t / 9.
struct StageLoad {
    int2 c;
    uint32_t w;
    bool valid;
};

template <int FMT>
__device__ __forceinline__ StageLoad load_stage(const CentreArgs& a, int group, int tid) {
    StageLoad r{make_int2(-1, -1), 0u, false};
    const int g = tid / 9, i = tid - 9 * g, s = group * kGroup + g;
    if (tid < 9 * kGroup && s < a.S) {
        r.valid = true;
        r.c = __ldg(a.centre + s);
        const int rx = r.c.x - 1 + i % 3, ry = r.c.y - 1 + i / 3;
        if (r.c.x >= 0 && rx >= 0 && rx < a.W && ry >= 0 && ry < a.H_)
            r.w = __ldg(static_cast<const uint32_t*>(a.ref_tex) + (int64_t)ry * a.W + rx);
    }
    return r;
}

template <int FMT>
__device__ __forceinline__ void store_stage(const CentreArgs& a, CentreStage& st, const StageLoad& r, int tid) {
    constexpr int sh = FMT == FMT_P10 ? 10 : 8;
    constexpr uint32_t mk = (1u << sh) - 1u;
    if (!r.valid) return;
    const int g = tid / 9;
    st.ref[tid] = make_int4((int)(r.w & mk), (int)((r.w >> sh) & mk), (int)(r.w >> (2 * sh)), 0);
    if (tid - 9 * g == 0) {
        st.c[g] = r.c;
        st.inside[g] = r.c.x >= 1 && r.c.x + 1 < a.W && r.c.y >= 1 && r.c.y + 1 < a.H_;
    }
}

// The projection of a segment centre through one entry (the contract's FP32 sequence) and the fast-path test.
struct CentreProj {
    int2 c;
    int ui, vi;
    bool in, fast;
};

template <bool FAST>
__device__ __forceinline__ CentreProj project_entry(const float (&h)[9], const CentreStage& st, int g, int w,
                                                    int hgt) {
    CentreProj p{st.c[g], 0, 0, false, false};
    if (p.c.x < 0) return p;
    const float x = (float)p.c.x, y = (float)p.c.y;
    const float X = __fmaf_rn(h[0], x, __fmaf_rn(h[1], y, h[2]));
    const float Yh = __fmaf_rn(h[3], x, __fmaf_rn(h[4], y, h[5]));
    const float Wz = __fmaf_rn(h[6], x, __fmaf_rn(h[7], y, h[8]));
    if (!(Wz > 0.0f)) return p;
    const float r = contract_rcp<FAST>(Wz);
    const float fu = floorf(__fadd_rn(__fmul_rn(X, r), 0.5f));
    const float fv = floorf(__fadd_rn(__fmul_rn(Yh, r), 0.5f));
    if (!(fu >= 0.0f && fu <= (float)(w - 1) && fv >= 0.0f && fv <= (float)(hgt - 1))) return p;
    p.ui = (int)fu;
    p.vi = (int)fv;
    p.in = true;
    p.fast = st.inside[g] && p.ui >= 1 && p.ui + 1 < w && p.vi >= 1 && p.vi + 1 < hgt;
    return p;
}

template <int FMT, bool FAST>
__global__ void __launch_bounds__(kCentreThreads, 4) centre_table3t_kernel(CentreArgs a, int chunks, int groups) {
    __shared__ CentreStage st[2];
    constexpr int sh = FMT == FMT_P10 ? 10 : 8;
    constexpr uint32_t mk = (1u << sh) - 1u;
    const int tid = threadIdx.x;
    const int nent = a.L * a.N;
    const int64_t items = (int64_t)chunks * groups;
    int64_t item = blockIdx.x;
    int buf = 0;
    if (item < items) store_stage<FMT>(a, st[0], load_stage<FMT>(a, (int)(item / chunks), tid), tid);
    for (; item < items; item += gridDim.x, buf ^= 1) {
        __syncthreads();  // st[buf] holds this item's group; st[buf ^ 1] is no longer read
        const int64_t next = item + gridDim.x;
        const StageLoad pre = next < items ? load_stage<FMT>(a, (int)(next / chunks), tid) : StageLoad{};
        const int group = (int)(item / chunks), j = (int)(item - (int64_t)group * chunks) * kCentreThreads + tid;
        if (j < nent) {
            // this thread's entry: neighbour k, label d (j = k L + d), its homography and the neighbour view
            const int k = a.L == 1 ? j : (int)__umulhi((uint32_t)j, a.l_magic), d = j - k * a.L;
            float h[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) h[i] = __ldg(a.H + (int64_t)j * 9 + i);
            const NbrView nv = a.nbrs[k];
            const int32_t* lv = a.labels_v[k];
            const uint32_t* tex = static_cast<const uint32_t*>(nv.texels);
            const CentreStage& cs = st[buf];
            const int s0 = group * kGroup, n = min(kGroup, a.S - s0);
            int32_t* mp = a.m + (int64_t)s0 * nent + (int64_t)d * a.N + k;
            int32_t* spp = a.sp + (int64_t)s0 * nent + (int64_t)d * a.N + k;
            CentreProj cur = project_entry<FAST>(h, cs, 0, nv.w, nv.h);
            for (int g = 0; g < n; ++g) {
                uint32_t t[9];
                if (cur.fast) {
                    const uint32_t* base = tex + ((int64_t)(cur.vi - 1) * nv.pitch + (cur.ui - 1));
#pragma unroll
                    for (int wy = 0; wy < 3; ++wy)
#pragma unroll
                        for (int wx = 0; wx < 3; ++wx) t[wy * 3 + wx] = __ldg(base + (int64_t)wy * nv.pitch + wx);
                }
                const int spv = (cur.in && lv) ? __ldg(lv + (int64_t)cur.vi * nv.w + cur.ui) : -1;
                CentreProj nxt{};
                if (g + 1 < n) nxt = project_entry<FAST>(h, cs, g + 1, nv.w, nv.h);
                int m;
                if (cur.fast) {
                    m = window_sum<FMT>(t, cs.ref + 9 * g);
                } else if (!cur.in) {
                    m = 9 * a.penalty;
                } else {
                    m = 0;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const int qx = cur.ui - 1 + i % 3, qy = cur.vi - 1 + i / 3;
                        const int rx = cur.c.x - 1 + i % 3, ry = cur.c.y - 1 + i / 3;
                        const bool rin = rx >= 0 && rx < a.W && ry >= 0 && ry < a.H_;
                        if (!rin || qx < 0 || qx >= nv.w || qy < 0 || qy >= nv.h) {
                            m += a.penalty;
                            continue;
                        }
                        const uint32_t q = __ldg(tex + (int64_t)qy * nv.pitch + qx);
                        const int4 r = cs.ref[9 * g + i];
                        m += (int)__sad(q & mk, (unsigned)r.x, __sad((q >> sh) & mk, (unsigned)r.y,
                                                                      __sad(q >> (2 * sh), (unsigned)r.z, 0u)));
                    }
                }
                *mp = m;
                *spp = spv;
                mp += nent;
                spp += nent;
                cur = nxt;
            }
        }
        if (next < items) store_stage<FMT>(a, st[buf ^ 1], pre, tid);
    }
}

}  // namespace
}  // namespace ftv

using namespace ftv;

extern "C" ftv_status ftv_centre_table(ftv_ctx* ctx, const void* const* d_planes, const int64_t* pitch_bytes,
                                       const int32_t* const* d_labels_views, const int32_t* n_segments,
                                       int32_t window, int32_t* const* d_m, int32_t* const* d_sprime,
                                       ftv_stream stream) {
    if (!ctx || !d_planes || !pitch_bytes || !d_labels_views || !n_segments || !d_m || !d_sprime)
        return FTV_ERR_INVALID_ARG;
    if (window < 1 || window > 15 || (window & 1) == 0) return FTV_ERR_INVALID_ARG;
    if (ctx->n_refs > kMaxUnits) return FTV_ERR_INVALID_ARG;
    for (int i = 0; i < ctx->n_refs; ++i) {
        const RefState& r = ctx->refs[i];
        if (!d_labels_views[r.view] || !d_m[i] || !d_sprime[i]) return FTV_ERR_INVALID_ARG;
        if (n_segments[i] < 0 || n_segments[i] > ctx->max_segments) return FTV_ERR_INVALID_ARG;
    }
    for (int v = 0; v < ctx->n_views; ++v)
        for (int c = 0; c < 3; ++c)
            if (!d_planes[3 * v + c] || pitch_bytes[3 * v + c] < (int64_t)ctx->cams[v].width * ctx->sample_bytes)
                return FTV_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    NvtxRange range("ftv_centre_table");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < ctx->n_views && e == cudaSuccess; ++v) {
        e = launch_pack(d_planes + 3 * v, pitch_bytes + 3 * v, ctx->sample_bytes, ctx->bit_depth, ctx->fmt,
                        ctx->cams[v].width, ctx->cams[v].height,
                        static_cast<char*>(ctx->d_packed) + ctx->view_offset_bytes[v], ctx->d_status, s);
        ctx->launches++;
    }
    for (int i = 0; i < ctx->n_refs && e == cudaSuccess; ++i) {
        RefState& r = ctx->refs[i];
        const int S = n_segments[i];
        // same int32 bound as ftv_cost_volume, since the index is cached for later volume calls
        const int64_t one = std::max<int64_t>(ctx->penalty, 3LL * ((1LL << ctx->bit_depth) - 1));
        const int64_t mpc = ctx->combine == FTV_COMBINE_MIN ? one : one * std::max(1, r.n_nbrs);
        e = launch_segment_index(d_labels_views[r.view], r.W, r.H, S, mpc, r.d_offs, r.d_cursor, r.d_pix, ctx->d_status,
                                 s, &ctx->launches);
        r.S_indexed = S;
        if (e != cudaSuccess) break;
        centroid_kernel<<<std::max(1, std::min(65535, (S + 7) / 8)), 256, 0, s>>>(r.d_offs, r.d_pix, S, r.d_centre);
        ctx->launches++;
        std::vector<const int32_t*> lv(r.n_nbrs);
        for (int k = 0; k < r.n_nbrs; ++k) lv[k] = d_labels_views[r.nbrs[k]];
        // the table of label-map pointers is copied into the reference's scratch, ordered on the stream
        e = cudaMemcpyAsync(r.d_nbr_labels, lv.data(), sizeof(const int32_t*) * std::max(1, r.n_nbrs),
                            cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        CentreArgs a{};
        a.centre = r.d_centre;
        a.H = r.d_H;
        a.H64 = r.d_H64;
        a.ref_tex = static_cast<char*>(ctx->d_packed) + ctx->view_offset_bytes[r.view];
        a.nbrs = r.d_nbrs;
        a.labels_v = r.d_nbr_labels;
        a.m = d_m[i];
        a.sp = d_sprime[i];
        a.S = S;
        a.L = ctx->L;
        a.N = r.n_nbrs;
        a.W = r.W;
        a.H_ = r.H;
        a.window = window;
        a.penalty = ctx->penalty;
        a.fmt = ctx->fmt;
        a.l_magic = ctx->L > 1 ? (uint32_t)((0x100000000ull + (uint64_t)ctx->L - 1) / (uint64_t)ctx->L) : 0u;
        const int64_t total = (int64_t)S * ctx->L * r.n_nbrs;
        const int blocks = std::max(1, std::min(S, ctx->n_sm * 8));
        // centre_table3t_kernel: (entry chunk, segment group) items over four resident CTAs per SM
        const int chunks = (ctx->L * r.n_nbrs + kCentreThreads - 1) / kCentreThreads, groups = (S + kGroup - 1) / kGroup;
        const int tblocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)chunks * groups, ctx->n_sm * 4));
        if (total > 0) {
            const bool fast = ctx->fast_rcp, fp32 = ctx->precision == FTV_PRECISION_FP32;
            if (window == 3 && !fp32 && ctx->fmt == FMT_P10) centre_table3_kernel<FMT_P10><<<blocks, kCentreThreads, 0, s>>>(a);
            else if (window == 3 && !fp32 && ctx->fmt == FMT_U8X4)
                centre_table3_kernel<FMT_U8X4><<<blocks, kCentreThreads, 0, s>>>(a);
            else if (window == 3 && ctx->fmt == FMT_P10 && fast)
                centre_table3t_kernel<FMT_P10, true><<<tblocks, kCentreThreads, 0, s>>>(a, chunks, groups);
            else if (window == 3 && ctx->fmt == FMT_P10)
                centre_table3t_kernel<FMT_P10, false><<<tblocks, kCentreThreads, 0, s>>>(a, chunks, groups);
            else if (window == 3 && ctx->fmt == FMT_U8X4 && fast)
                centre_table3t_kernel<FMT_U8X4, true><<<tblocks, kCentreThreads, 0, s>>>(a, chunks, groups);
            else if (window == 3 && ctx->fmt == FMT_U8X4)
                centre_table3t_kernel<FMT_U8X4, false><<<tblocks, kCentreThreads, 0, s>>>(a, chunks, groups);
            else if (window == 3) centre_table3_kernel<FMT_U16X4><<<blocks, kCentreThreads, 0, s>>>(a);
            else centre_table_kernel<<<blocks, kCentreThreads, 0, s>>>(a);
            ctx->launches++;
        }
        e = cudaGetLastError();
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return e == cudaSuccess ? FTV_OK : FTV_ERR_CUDA;
}
