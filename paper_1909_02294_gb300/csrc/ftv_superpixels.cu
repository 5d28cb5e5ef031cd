// Superpixel segmentation (Sec. IV-C): the label maps the method consumes, as SNIC-like superpixels in
// (Y, Cb, Cr) with compactness factor m and 8-connected segments.
//
// SNIC grows every cluster from its seed through a single priority queue, which is sequential. This is
// its data-parallel reformulation (the clustering SNIC itself derives from), with SNIC's seeds, distance
// and connectivity:
//   - seeds on an S x S grid: cell (i, j) of width w and height h has label j * ceil(W/S) + i and seed
//     (iS + (w-1)/2, jS + (h-1)/2);
//   - D = S^2 ||c_p - c_k||^2 + m^2 ||x_p - x_k||^2 on the 8-bit colour scale (the spatial weight times
//     4^(bd-8) above 8 bits, the colour weight times 4^(8-bd) below), evaluated exactly in 64-bit
//     integers on 16 * (pixel value) - (cluster mean in 1/16 units);
//   - assignment passes: a pixel of cell (i, j) joins the least-D cluster among cells (i+a, j+b),
//     a, b in {-1, 0, 1} (smallest label on ties); between passes every cluster mean becomes
//     floor((32 sum + n) / (2 n)) of its pixels (an empty cluster keeps its mean);
//   - connectivity: components are the 8-connected sets of equally labelled pixels (named by their first
//     pixel); a label's largest component (earliest on ties) is anchored with that label; the other
//     components merge in rounds, each unanchored group joining the 8-adjacent group of nearest mean
//     colour (L1 of the rounded 1/16 means; on ties the group of smallest name, a group's name being its
//     smallest component name), all picks of a round at once, until every group is anchored.
// The result is unique (integer arithmetic, order-free rules), so it equals the CPU definition exactly.
//
// Kernels: seeds; per pass a tiled assignment (128 x 8 pixels per CTA, 4 adjacent pixels per thread; the
// CTA's candidate centres staged in shared memory; D in 32-bit integers when the weights reduced by their
// gcd provably keep it below 2^32, else in 64-bit; runs of equal labels summed in registers, then into
// per-tile shared accumulators, then one global add per cluster and field) and an update; union-find
// components over the pixels (atomicMin linking, so a root is its component's first pixel): every pixel
// points at its row run's start (one warp ballot), and only runs are linked; component sums and the main
// component per label; then per round a pick (round 0 over every pixel, later rounds over the pixels of
// unanchored groups that still touched another group, a list that shrinks every round), a link, a merge
// that moves group sums and anchors, and a finish that forms the means and counts the unanchored groups
// (every round kernel returns at once when the count is zero); a final relabel.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "ftv_internal.h"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;
constexpr int kTileW = 32, kTileH = 8;           // component tiles: one pixel per thread, one warp per row
constexpr int kPX = 4;                           // assignment: adjacent pixels per thread
constexpr int kATileW = 32 * kPX, kATileH = 8;   // assignment tile
constexpr int kLoopCap = 1 << 26;                // bound of every union-find walk (parents strictly decrease)
constexpr unsigned long long kNone = ~0ull;

enum : uint32_t { SP_LOOP_CAP = 1u, SP_ROUND_CAP = 2u };
enum : int { DIST_DOT32 = 0, DIST_NARROW = 1, DIST_WIDE = 2, DIST_WIDE_COLOUR = 3 };

struct SegImage {
    const void* plane[3];
    int64_t pitch[3];
    int32_t* out;
    int32_t W, H, gw, gh;
    int32_t pix_base, seg_base, K, pad;
};

struct alignas(32) Centre {
    int x, y, c0, c1, c2, p0, p1, p2;
};

struct alignas(32) Sums {
    uint32_t n, x, y, c0, c1, c2, p0, p1;
};

struct alignas(32) GSum {
    unsigned long long n, c0, c1, c2;
};

// counters: [0] components, [1 + r] unanchored groups at the start of round r (r = 0..rounds), which
// is also the length of the round's list uroots, [2 + rounds + r] length of round r's pick list,
// [3 + 2 rounds] main components
struct Scratch {
    const SegImage* img;
    Centre* cen;
    Sums* sums;
    unsigned long long* mainkey;  // [K]: (size << 32) | ~name of the label's largest component
    int32_t* lab;                 // [P] global segment id of each pixel
    int32_t* par;                 // [P] union-find over pixels, then the component name
    ulonglong2* csum;             // [P] per component name: (n << 40) + sum Y, (sum Cb << 32) + sum Cr
                                  // (a component lies in one cluster: n < 2^24, each sum < 2^32)
    int32_t* gpar;                // [P] union-find over component names (groups)
    int32_t* glab;                // [P] anchored label of a group (-1 unanchored)
    GSum* gsum;                   // [P] group sums (valid at group roots)
    int4* gmean;                  // [P] group mean colour in 1/16 units
    unsigned long long* best;     // [P] (distance << 32) | name picked by an unanchored group
    int32_t* comps;               // [P] list of component names
    int32_t* uroots[2];           // [P] unanchored group roots at the start of a round, alternating
    int32_t* mains;               // [P] the main components (anchored group roots; they stay roots)
    int32_t* gname;               // [P] name of a group (its smallest component name), at its root
    uint8_t* dirty;               // [P] an anchored root gained members in the current merge round
    int2* orph[2];                // [P] pick lists of (pixel, image), alternating between rounds
    int32_t* cnt;
    uint32_t* status;
    int32_t S, sb, rounds, max_cells;
    unsigned long long wc, ws;    // distance weights
    uint32_t wcn, wsn;            // the weights divided by their gcd (32-bit distance)
};

__device__ __forceinline__ int sample(const SegImage& im, int c, int x, int y, int sb) {
    const char* row = static_cast<const char*>(im.plane[c]) + (int64_t)y * im.pitch[c];
    return sb == 1 ? (int)reinterpret_cast<const uint8_t*>(row)[x] : (int)reinterpret_cast<const uint16_t*>(row)[x];
}

__device__ __forceinline__ int seed_coord(int n, int S, int i) {
    const int w = min(S, n - i * S);
    return i * S + (w - 1) / 2;
}

// round(16 * s / n), halves up: floor((32 s + n) / (2 n)); 32-bit division when it fits
__device__ __forceinline__ int mean16(unsigned long long s, unsigned long long n) {
    const unsigned long long num = 32ull * s + n, den = 2ull * n;
    if ((num >> 32) == 0 && (den >> 32) == 0) return (int)((uint32_t)num / (uint32_t)den);
    return (int)(num / den);
}

// Walk to the root. Reads may be stale while other threads link (a stale parent is still an ancestor),
// so a walk always ends at a node that is or was a root; unite() then corrects itself through the atomic.
// CG: read parents from L2 (ld.global.cg), for walks that run while other SMs link.
template <bool CG = false>
__device__ int find_root(const int32_t* par, int32_t x, uint32_t* status) {
    for (int it = 0; it < kLoopCap; ++it) {
        const int32_t p = CG ? __ldcg(&par[x]) : par[x];
        if (p == x) return x;
        x = p;
    }
    atomicOr(status, SP_LOOP_CAP);
    return x;
}

// Link the sets of a and b; the smaller root becomes the parent (so a root is its set's smallest name).
__device__ void unite(int32_t* par, int32_t a, int32_t b, uint32_t* status) {
    for (int it = 0; it < kLoopCap; ++it) {
        a = find_root<true>(par, a, status);
        b = find_root<true>(par, b, status);
        if (a == b) return;
        if (a > b) {
            const int32_t t = a;
            a = b;
            b = t;
        }
        const int32_t old = atomicMin(&par[b], a);
        if (old == b) return;  // b was a root and now hangs under a
        b = old;               // b was linked meanwhile: join a with b's new parent instead
    }
    atomicOr(status, SP_LOOP_CAP);
}

// Append the threads with keep set to list[*counter...], one atomic per CTA. Every thread of the CTA
// (kThreads, any shape) must call it.
template <class T>
__device__ __forceinline__ void block_append(bool keep, const T& v, T* list, int32_t* counter) {
    __shared__ int s_off[kThreads / 32 + 1];
    const int t = threadIdx.y * blockDim.x + threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned m = __ballot_sync(kFull, keep);
    if (lane == 0) s_off[warp] = __popc(m);
    __syncthreads();
    if (t == 0) {
        int tot = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            const int c = s_off[w];
            s_off[w] = tot;
            tot += c;
        }
        s_off[kThreads / 32] = tot ? atomicAdd(counter, tot) : 0;
    }
    __syncthreads();
    if (keep) list[s_off[kThreads / 32] + s_off[warp] + __popc(m & ((1u << lane) - 1u))] = v;
    __syncthreads();
}

// ---------------------------------------------------------------------------------------- clustering

__global__ void seed_kernel(Scratch s) {
    const SegImage im = s.img[blockIdx.y];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= im.K) return;
    const int i = k % im.gw, j = k / im.gw;
    const int x = seed_coord(im.W, s.S, i), y = seed_coord(im.H, s.S, j);
    Centre c{};
    c.x = 16 * x;
    c.y = 16 * y;
    c.c0 = 16 * sample(im, 0, x, y, s.sb);
    c.c1 = 16 * sample(im, 1, x, y, s.sb);
    c.c2 = 16 * sample(im, 2, x, y, s.sb);
    s.cen[im.seg_base + k] = c;
    s.sums[im.seg_base + k] = Sums{};
    s.mainkey[im.seg_base + k] = 0;
}

// D of one candidate, from the staged cell (a, b). Direct forms (a = x, y, Y, Cb of the mean; b.x = Cr):
// NARROW uses the gcd-reduced weights in 32 bits (the host has shown that D stays below 2^32); WIDE
// 32-bit squares and a 64-bit weighted sum; WIDE_COLOUR 64-bit colour squares (bit depth > 11).
// DOT32 drops the pixel's own squares, common to all candidates: with tile-relative positions,
// D - wc' |v|^2 - ws' |p|^2 = K - 2 (wc' <v, c> + ws' <p, x>) where K = wc' |c|^2 + ws' |x|^2, so
// a = (K, -2 ws' x, -2 ws' y, -2 wc' Y), b = (-2 wc' Cb, -2 wc' Cr): five multiply-adds in 32 bits
// (the host has shown that every partial sum stays below 2^31 in magnitude).
template <int DM>
struct Dist {
    using T = unsigned long long;
};
template <>
struct Dist<DIST_NARROW> {
    using T = uint32_t;
};
template <>
struct Dist<DIST_DOT32> {
    using T = int;
};

template <int DM>
__device__ __forceinline__ typename Dist<DM>::T distance(const int4 a, const int4 b, int vx, int vy, int w0, int w1,
                                                         int w2, const Scratch& s) {
    if (DM == DIST_DOT32) {
        int d = a.x;
        d += vx * a.y;
        d += vy * a.z;
        d += w0 * a.w;
        d += w1 * b.x;
        d += w2 * b.y;
        return d;
    }
    const int dx = vx - a.x, dy = vy - a.y;
    const uint32_t dsp = (uint32_t)dx * (uint32_t)dx + (uint32_t)dy * (uint32_t)dy;
    const int d0 = w0 - a.z, d1 = w1 - a.w, d2 = w2 - b.x;
    if (DM == DIST_NARROW) {
        const uint32_t dcol = (uint32_t)d0 * (uint32_t)d0 + (uint32_t)d1 * (uint32_t)d1 + (uint32_t)d2 * (uint32_t)d2;
        return (typename Dist<DM>::T)(s.wcn * dcol + s.wsn * dsp);
    } else if (DM == DIST_WIDE) {
        const uint32_t dcol = (uint32_t)d0 * (uint32_t)d0 + (uint32_t)d1 * (uint32_t)d1 + (uint32_t)d2 * (uint32_t)d2;
        return (typename Dist<DM>::T)(s.wc * dcol + s.ws * dsp);
    } else {
        const unsigned long long dcol = (unsigned long long)((long long)d0 * d0) +
                                        (unsigned long long)((long long)d1 * d1) +
                                        (unsigned long long)((long long)d2 * d2);
        return (typename Dist<DM>::T)(s.wc * dcol + s.ws * dsp);
    }
}

// One assignment pass over a 128 x 8 tile (4 adjacent pixels per thread). accumulate: add every pixel to
// its cluster's sums for the next update. last: also start the component search (par = self).
// The 3 x 3 candidates are visited unrolled in increasing label order; a candidate outside the grid is
// replaced by the nearest existing cell, a repeat of a label already visited with the same D, which the
// strict comparison ignores.
template <int DM>
__global__ void __launch_bounds__(kThreads) assign_kernel(Scratch s, int accumulate, int last) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SegImage im = s.img[blockIdx.z];
    const int x0 = blockIdx.x * kATileW, y0 = blockIdx.y * kATileH;
    if (x0 >= im.W || y0 >= im.H) return;  // uniform over the CTA
    const int S = s.S, MC = s.max_cells;
    const int cx0 = max(0, x0 / S - 1), cx1 = min(im.gw - 1, min(im.W - 1, x0 + kATileW - 1) / S + 1);
    const int cy0 = max(0, y0 / S - 1), cy1 = min(im.gh - 1, min(im.H - 1, y0 + kATileH - 1) / S + 1);
    const int ncx = cx1 - cx0 + 1, ncells = ncx * (cy1 - cy0 + 1);
    int4* sA = reinterpret_cast<int4*>(smem);
    int4* sB = sA + MC;
    uint32_t* acc = reinterpret_cast<uint32_t*>(sB + MC);  // [6][MC]: n, x, y, Y, Cb, Cr
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int e = tid; e < ncells; e += kThreads) {
        const int j = cy0 + e / ncx, i = cx0 + e % ncx;
        const Centre c = s.cen[im.seg_base + j * im.gw + i];
        if (DM == DIST_DOT32) {
            const int xr = c.x - 16 * x0, yr = c.y - 16 * y0;
            const long long K = (long long)s.wcn * ((long long)c.c0 * c.c0 + (long long)c.c1 * c.c1 +
                                                    (long long)c.c2 * c.c2) +
                                (long long)s.wsn * ((long long)xr * xr + (long long)yr * yr);
            const int wc2 = 2 * (int)s.wcn, ws2 = 2 * (int)s.wsn;
            sA[e] = make_int4((int)K, -ws2 * xr, -ws2 * yr, -wc2 * c.c0);
            sB[e] = make_int4(-wc2 * c.c1, -wc2 * c.c2, 0, 0);
        } else {
            sA[e] = make_int4(c.x, c.y, c.c0, c.c1);
            sB[e] = make_int4(c.c2, 0, 0, 0);
        }
        if (accumulate)
            for (int f = 0; f < 6; ++f) acc[f * MC + e] = 0;
    }
    __syncthreads();

    const int y = y0 + threadIdx.y;
    int rk = -1;
    uint32_t rn = 0, rx = 0, ry = 0, r0 = 0, r1 = 0, r2 = 0;
    if (y < im.H) {
        const int cj = y / S;
        const int jv[3] = {max(cj - 1, 0), cj, min(cj + 1, im.gh - 1)};
        const int ro[3] = {(jv[0] - cy0) * ncx - cx0, (jv[1] - cy0) * ncx - cx0, (jv[2] - cy0) * ncx - cx0};
        const int vy = DM == DIST_DOT32 ? 16 * (y - y0) : 16 * y;
        const int64_t row = (int64_t)im.pix_base + (int64_t)y * im.W;
        const int xs = x0 + kPX * threadIdx.x;
        int ci = xs / S, rem = xs - ci * S;  // cell column of the current pixel, and x within the cell
#pragma unroll 1
        for (int q = 0; q < kPX; ++q, ++rem) {
            const int x = xs + q;
            if (x >= im.W) break;
            if (rem == S) {
                ++ci;
                rem = 0;
            }
            const int v0 = sample(im, 0, x, y, s.sb), v1 = sample(im, 1, x, y, s.sb), v2 = sample(im, 2, x, y, s.sb);
            const int co[3] = {max(ci - 1, 0), ci, min(ci + 1, im.gw - 1)};
            const int vx = DM == DIST_DOT32 ? 16 * (x - x0) : 16 * x;
            const int w0 = 16 * v0, w1 = 16 * v1, w2 = 16 * v2;
            int be = ro[0] + co[0], bc = 0;
            typename Dist<DM>::T bd = distance<DM>(sA[be], sB[be], vx, vy, w0, w1, w2, s);
#pragma unroll
            for (int c = 1; c < 9; ++c) {
                const int e = ro[c / 3] + co[c % 3];
                const typename Dist<DM>::T D = distance<DM>(sA[e], sB[e], vx, vy, w0, w1, w2, s);
                if (D < bd) {
                    be = e;
                    bc = c;
                    bd = D;
                }
            }
            const int bj = bc < 3 ? jv[0] : (bc < 6 ? jv[1] : jv[2]);
            const int bm = bc - 3 * (bc < 3 ? 0 : (bc < 6 ? 1 : 2));
            const int bi = bm == 0 ? co[0] : (bm == 1 ? co[1] : co[2]);
            const int64_t gp = row + x;
            s.lab[gp] = im.seg_base + bj * im.gw + bi;
            if (last) {
                s.par[gp] = (int32_t)gp;
                s.csum[gp] = make_ulonglong2(0, 0);
            }
            if (accumulate) {
                if (be != rk) {
                    if (rk >= 0) {
                        atomicAdd(&acc[0 * MC + rk], rn);
                        atomicAdd(&acc[1 * MC + rk], rx);
                        atomicAdd(&acc[2 * MC + rk], ry);
                        atomicAdd(&acc[3 * MC + rk], r0);
                        atomicAdd(&acc[4 * MC + rk], r1);
                        atomicAdd(&acc[5 * MC + rk], r2);
                    }
                    rk = be;
                    rn = rx = ry = r0 = r1 = r2 = 0;
                }
                rn += 1;
                rx += x;
                ry += y;
                r0 += v0;
                r1 += v1;
                r2 += v2;
            }
        }
    }
    if (!accumulate) return;
    if (rk >= 0) {
        atomicAdd(&acc[0 * MC + rk], rn);
        atomicAdd(&acc[1 * MC + rk], rx);
        atomicAdd(&acc[2 * MC + rk], ry);
        atomicAdd(&acc[3 * MC + rk], r0);
        atomicAdd(&acc[4 * MC + rk], r1);
        atomicAdd(&acc[5 * MC + rk], r2);
    }
    __syncthreads();
    for (int e = tid; e < ncells; e += kThreads) {
        const uint32_t n = acc[e];
        if (n == 0) continue;
        const int j = cy0 + e / ncx, i = cx0 + e % ncx;
        Sums* t = &s.sums[im.seg_base + j * im.gw + i];
        atomicAdd(&t->n, n);
        atomicAdd(&t->x, acc[1 * MC + e]);
        atomicAdd(&t->y, acc[2 * MC + e]);
        atomicAdd(&t->c0, acc[3 * MC + e]);
        atomicAdd(&t->c1, acc[4 * MC + e]);
        atomicAdd(&t->c2, acc[5 * MC + e]);
    }
}

__global__ void update_kernel(Scratch s) {
    const SegImage im = s.img[blockIdx.y];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= im.K) return;
    Sums& t = s.sums[im.seg_base + k];
    const unsigned long long n = t.n;
    if (n > 0) {
        Centre& c = s.cen[im.seg_base + k];
        c.x = mean16(t.x, n);
        c.y = mean16(t.y, n);
        c.c0 = mean16(t.c0, n);
        c.c1 = mean16(t.c1, n);
        c.c2 = mean16(t.c2, n);
    }
    t = Sums{};
}

// ------------------------------------------------------------------------------------- connectivity

// 8-connected components of equal labels, built from row runs. A warp holds 32 pixels of a row: a ballot
// finds each pixel's run start inside the warp's segment, and every pixel points there.
__global__ void __launch_bounds__(kThreads) runs_kernel(Scratch s) {
    const SegImage im = s.img[blockIdx.z];
    const int x = blockIdx.x * kTileW + threadIdx.x, y = blockIdx.y * kTileH + threadIdx.y;
    const bool valid = x < im.W && y < im.H;
    const int32_t gp = valid ? im.pix_base + y * im.W + x : -1;
    const int l = valid ? s.lab[gp] : -1;
    const int lane = threadIdx.x;
    const int left = __shfl_up_sync(kFull, l, 1);
    const unsigned cont = __ballot_sync(kFull, valid && lane > 0 && left == l);  // continues the run on its left
    const unsigned upto = lane == 31 ? kFull : ((2u << lane) - 1u);
    const int start = 31 - __clz(~cont & upto);
    if (valid) s.par[gp] = gp - (lane - start);
}

// Links between runs: a run continuing across a warp segment; a run and the run above it where they
// overlap (issued once, from the later of the two run starts) or touch diagonally (from the run's first
// and last pixel). Runs here are the segment-local ones, so a few links are issued twice.
__global__ void __launch_bounds__(kThreads) links_kernel(Scratch s) {
    const SegImage im = s.img[blockIdx.z];
    const int x = blockIdx.x * kTileW + threadIdx.x, y = blockIdx.y * kTileH + threadIdx.y;
    const bool valid = x < im.W && y < im.H;
    const int32_t gp = valid ? im.pix_base + y * im.W + x : -1;
    const int l = valid ? s.lab[gp] : -1;
    const int lane = threadIdx.x;
    const int left = __shfl_up_sync(kFull, l, 1), right = __shfl_down_sync(kFull, l, 1);
    if (!valid) return;
    // run starts and ends from the labels (parents change under the links being made)
    const bool is_start = lane == 0 || left != l;
    const bool is_end = lane == 31 || x + 1 >= im.W || right != l;
    if (lane == 0 && x > 0 && s.lab[gp - 1] == l) unite(s.par, gp, gp - 1, s.status);
    if (y == 0) return;
    const int32_t up = gp - im.W;
    if (s.lab[up] == l && (is_start || s.lab[up - 1] != l)) unite(s.par, gp, up, s.status);
    if (is_start && x > 0 && s.lab[up - 1] == l) unite(s.par, gp, up - 1, s.status);
    if (is_end && x + 1 < im.W && s.lab[up + 1] == l) unite(s.par, gp, up + 1, s.status);
}

// Component name of every pixel, and the component's pixel count and colour sums: one walk per row run
// (its first lane), broadcast to the run; each run's sums reduced over its lanes.
__global__ void __launch_bounds__(kThreads) flatten_kernel(Scratch s) {
    const SegImage im = s.img[blockIdx.z];
    const int x = blockIdx.x * kTileW + threadIdx.x, y = blockIdx.y * kTileH + threadIdx.y;
    const bool valid = x < im.W && y < im.H;
    const int32_t gp = valid ? im.pix_base + y * im.W + x : -1;
    const int l = valid ? s.lab[gp] : -1;
    const int lane = threadIdx.x;
    const int left = __shfl_up_sync(kFull, l, 1);
    const unsigned cont = __ballot_sync(kFull, valid && lane > 0 && left == l);
    const int start = 31 - __clz(~cont & (lane == 31 ? kFull : ((2u << lane) - 1u)));
    const unsigned above = ~cont & (start == 31 ? 0u : ~((2u << start) - 1u));  // run breaks after start
    const int end = above ? __ffs(above) - 2 : 31;
    const unsigned run = (end == 31 ? kFull : ((2u << end) - 1u)) & ~((1u << start) - 1u);
    int32_t r = -1;
    if (valid && lane == start) r = find_root(s.par, gp, s.status);
    r = __shfl_sync(kFull, r, start);
    int v0 = 0, v1 = 0, v2 = 0;
    if (valid) {
        s.par[gp] = r;
        v0 = sample(im, 0, x, y, s.sb);
        v1 = sample(im, 1, x, y, s.sb);
        v2 = sample(im, 2, x, y, s.sb);
    }
    // lanes of one run share the mask; disjoint runs reduce side by side
    const uint32_t s0 = __reduce_add_sync(run, (uint32_t)v0);
    const uint32_t s1 = __reduce_add_sync(run, (uint32_t)v1);
    const uint32_t s2 = __reduce_add_sync(run, (uint32_t)v2);
    if (valid && lane == start) {
        ulonglong2* t = &s.csum[r];
        atomicAdd(&t->x, ((unsigned long long)__popc(run) << 40) + s0);
        atomicAdd(&t->y, ((unsigned long long)s1 << 32) + s2);
    }
}

// Every component offers itself as its label's main component: the largest, the earliest named on ties.
__global__ void __launch_bounds__(kThreads) main_kernel(Scratch s) {
    const SegImage im = s.img[blockIdx.z];
    const int x = blockIdx.x * kTileW + threadIdx.x, y = blockIdx.y * kTileH + threadIdx.y;
    const bool valid = x < im.W && y < im.H;
    const int32_t gp = valid ? im.pix_base + y * im.W + x : -1;
    const bool root = valid && s.par[gp] == gp;
    if (root) {
        const unsigned long long key = ((s.csum[gp].x >> 40) << 32) | (unsigned long long)(~(uint32_t)gp);
        atomicMax(&s.mainkey[s.lab[gp]], key);
    }
    block_append(root, gp, s.comps, &s.cnt[0]);
}

// Groups start as single components; main components are anchored with their label. The unanchored
// ones form round 0's list.
__global__ void __launch_bounds__(kThreads) group_init_kernel(Scratch s) {
    const int n = s.cnt[0];
    for (int base = blockIdx.x * kThreads; base < n; base += gridDim.x * kThreads) {
        const int i = base + threadIdx.x;
        bool is_main = false;
        int32_t c = 0;
        if (i < n) {
            c = s.comps[i];
            const int32_t k = s.lab[c];
            is_main = (uint32_t)(~s.mainkey[k]) == (uint32_t)c;
            s.gpar[c] = c;
            s.gname[c] = c;
            s.glab[c] = is_main ? k : -1;
            const ulonglong2 t = s.csum[c];
            const unsigned long long n = t.x >> 40, sy = t.x & ((1ull << 40) - 1), scb = t.y >> 32,
                                     scr = t.y & 0xffffffffull;
            s.gsum[c] = GSum{n, sy, scb, scr};
            s.gmean[c] = make_int4(mean16(sy, n), mean16(scb, n), mean16(scr, n), 0);
            s.best[c] = kNone;
            s.dirty[c] = 0;
        }
        block_append(i < n && !is_main, c, s.uroots[0], &s.cnt[1]);
        block_append(is_main, c, s.mains, &s.cnt[3 + 2 * s.rounds]);
    }
}

// The pick of one pixel p (component pc) of group a (unanchored): the neighbouring group of least
// (distance, name). The lookups run in stages over all eight neighbours at once (components, one step
// up the group forest, the rest of the walk where one is left, then means and names), so that each
// stage's independent loads are in flight together; neighbours in p's own component are skipped.
__device__ __forceinline__ bool pick_pixel(const Scratch& s, const SegImage& im, int32_t p, int32_t pc, int32_t a) {
    const int local = p - im.pix_base;
    const int x = local % im.W, y = local / im.W;
    int32_t g[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int dx = k < 3 ? k - 1 : (k == 3 ? -1 : (k == 4 ? 1 : k - 6));
        const int dy = k < 3 ? -1 : (k < 5 ? 0 : 1);
        const int qx = x + dx, qy = y + dy;
        g[k] = (qx >= 0 && qx < im.W && qy >= 0 && qy < im.H) ? s.par[p + dy * im.W + dx] : -1;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) g[k] = (g[k] < 0 || g[k] == pc) ? -1 : s.gpar[g[k]];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (g[k] >= 0) {
            const int32_t up = s.gpar[g[k]];
            if (up != g[k]) g[k] = find_root(s.gpar, up, s.status);
        }
    const int4 ma = s.gmean[a];
    unsigned long long best = kNone;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (g[k] >= 0 && g[k] != a) {
            const int4 mb = s.gmean[g[k]];
            const unsigned long long d = (unsigned long long)(abs(ma.x - mb.x) + abs(ma.y - mb.y) + abs(ma.z - mb.z));
            best = min(best, (d << 32) | (unsigned long long)(uint32_t)s.gname[g[k]]);
        }
    if (best == kNone) return false;
    atomicMin(&s.best[a], best);
    return true;
}

// Round r's pick: every unanchored group takes the 8-adjacent group of nearest mean colour. A pixel whose
// group is anchored, or whose neighbours all lie in its own group, can never matter again (anchors are
// kept and groups only merge): only the others enter round r + 1's list. Round 0 visits every pixel.
__global__ void __launch_bounds__(kThreads) pick0_kernel(Scratch s) {
    if (s.cnt[1] == 0) return;
    const SegImage im = s.img[blockIdx.z];
    const int x0 = blockIdx.x * kTileW, y0 = blockIdx.y * kTileH;
    if (x0 >= im.W || y0 >= im.H) return;  // uniform over the CTA
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    bool keep = false;
    int32_t gp = -1;
    if (x < im.W && y < im.H) {
        gp = im.pix_base + y * im.W + x;
        const int32_t pc = s.par[gp];
        const int32_t a = find_root(s.gpar, pc, s.status);
        keep = s.glab[a] < 0 && pick_pixel(s, im, gp, pc, a);
    }
    block_append(keep, make_int2(gp, (int)blockIdx.z), s.orph[1], &s.cnt[2 + s.rounds + 1]);
}

__global__ void __launch_bounds__(kThreads) pick_kernel(Scratch s, int r) {
    if (s.cnt[1 + r] == 0) return;
    const int n = s.cnt[2 + s.rounds + r];
    const int2* in = s.orph[r & 1];
    int2* next = s.orph[(r + 1) & 1];
    int32_t* next_n = &s.cnt[2 + s.rounds + r + 1];
    for (int base = blockIdx.x * kThreads; base < n; base += gridDim.x * kThreads) {
        const int i = base + threadIdx.x;
        bool keep = false;
        int2 o = make_int2(0, 0);
        if (i < n) {
            o = in[i];
            const int32_t pc = s.par[o.x];
            const int32_t a = find_root(s.gpar, pc, s.status);
            keep = s.glab[a] < 0 && pick_pixel(s, s.img[o.y], o.x, pc, a);
        }
        block_append(keep, o, next, next_n);
    }
}

// Group links order roots anchored first, then by smaller name, and hang the later root under the earlier
// one (compare-and-swap on a root): an anchored root therefore never gets a parent, and the order is total,
// so no cycle can form. Anchored status does not change while links are made.
__device__ void unite_groups(Scratch& s, int32_t a, int32_t b) {
    for (int it = 0; it < kLoopCap; ++it) {
        a = find_root<true>(s.gpar, a, s.status);
        b = find_root<true>(s.gpar, b, s.status);
        if (a == b) return;
        const bool aa = s.glab[a] >= 0, ab = s.glab[b] >= 0;
        if (ab > aa || (ab == aa && b < a)) {
            const int32_t t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(&s.gpar[b], b, a) == b) return;
    }
    atomicOr(s.status, SP_LOOP_CAP);
}

// Round r, link: all picks at once (the round's unanchored roots with the groups they picked, found from
// the picked group's name, which is one of its components).
__global__ void link_kernel(Scratch s, int r) {
    const int n = s.cnt[1 + r];
    const int32_t* u = s.uroots[r & 1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t c = u[i];
        const unsigned long long b = s.best[c];
        if (b != kNone) unite_groups(s, c, (int32_t)(uint32_t)b);
    }
}

// Round r, merge: every unanchored root that now hangs under another root moves its sums and its name
// there (only the round's unanchored roots can have gained a parent).
__global__ void merge_kernel(Scratch s, int r) {
    const int n = s.cnt[1 + r];
    const int32_t* u = s.uroots[r & 1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t c = u[i];
        const int32_t t = find_root(s.gpar, c, s.status);
        if (t == c) continue;
        const GSum g = s.gsum[c];
        GSum* d = &s.gsum[t];
        atomicAdd(&d->n, g.n);
        atomicAdd(&d->c0, g.c0);
        atomicAdd(&d->c1, g.c1);
        atomicAdd(&d->c2, g.c2);
        atomicMin(&s.gname[t], s.gname[c]);
        if (s.glab[t] >= 0) s.dirty[t] = 1;
    }
}

// Round r, finish: the round's roots point at their new roots; those still unanchored (then still roots)
// get their mean and form round r + 1's list; anchored roots that gained members get their mean.
__global__ void __launch_bounds__(kThreads) finish_kernel(Scratch s, int r) {
    if (s.cnt[1 + r] == 0) return;
    const int n = s.cnt[1 + r];
    const int32_t* u = s.uroots[r & 1];
    int32_t* next = s.uroots[(r + 1) & 1];
    for (int base = blockIdx.x * kThreads; base < n; base += gridDim.x * kThreads) {
        const int i = base + threadIdx.x;
        bool keep = false;
        int32_t c = 0;
        if (i < n) {
            c = u[i];
            s.best[c] = kNone;
            const int32_t t = find_root(s.gpar, c, s.status);
            s.gpar[c] = t;
            if (t == c) {
                const GSum g = s.gsum[c];
                s.gmean[c] = make_int4(mean16(g.c0, g.n), mean16(g.c1, g.n), mean16(g.c2, g.n), 0);
                keep = true;
            }
        }
        block_append(keep, c, next, &s.cnt[2 + r]);
    }
    const int nm = s.cnt[3 + 2 * s.rounds];
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < nm; i += gridDim.x * kThreads) {
        const int32_t t = s.mains[i];
        if (!s.dirty[t]) continue;
        s.dirty[t] = 0;
        const GSum g = s.gsum[t];
        s.gmean[t] = make_int4(mean16(g.c0, g.n), mean16(g.c1, g.n), mean16(g.c2, g.n), 0);
    }
}

// Every component points straight at its group's root.
__global__ void final_flatten_kernel(Scratch s) {
    const int n = s.cnt[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t c = s.comps[i];
        s.gpar[c] = find_root(s.gpar, c, s.status);
    }
}

__global__ void __launch_bounds__(kThreads) relabel_kernel(Scratch s) {
    const SegImage im = s.img[blockIdx.z];
    const int x = blockIdx.x * kTileW + threadIdx.x, y = blockIdx.y * kTileH + threadIdx.y;
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0 &&
        s.cnt[1 + s.rounds] != 0)
        atomicOr(s.status, SP_ROUND_CAP);
    if (x >= im.W || y >= im.H) return;
    const int32_t gp = im.pix_base + y * im.W + x;
    const int32_t g = s.gpar[s.par[gp]];
    const int32_t k = s.glab[g];
    im.out[(int64_t)y * im.W + x] = (k >= 0 ? k : s.lab[gp]) - im.seg_base;
}

}  // namespace

struct ftv_segmenter {
    int device = 0;
    int n_images = 0, sb = 1, bd = 8, S = 1, m = 0, T = 1;
    std::vector<SegImage> h_meta;  // sizes and bases (pointers filled per call)
    int64_t P = 0;
    int32_t K = 0;
    int max_W = 0, max_H = 0, max_K = 0, rounds = 0, dist_mode = 0;
    size_t assign_smem = 0;
    unsigned long long wc = 0, ws = 0;
    SegImage* h_img = nullptr;  // pinned staging of the per-call descriptors
    SegImage* d_img = nullptr;
    Scratch sc{};
    std::vector<void*> blocks;  // every device allocation, freed at destroy
    cudaEvent_t staged = nullptr;
    int64_t launches = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> ev;  // profiling: call begin, call end, then a pair per assignment pass
    bool timed = false;
};

namespace {

template <class T>
bool dalloc(ftv_segmenter* g, T** p, size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, sizeof(T) * std::max<size_t>(n, 1)) != cudaSuccess) return false;
    g->blocks.push_back(q);
    *p = static_cast<T*>(q);
    return true;
}

void release(ftv_segmenter* g) {
    for (void* q : g->blocks) cudaFree(q);
    g->blocks.clear();
    if (g->h_img) cudaFreeHost(g->h_img);
    if (g->staged) cudaEventDestroy(g->staged);
    for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
    delete g;
}

}  // namespace

extern "C" ftv_status ftv_segmenter_init(const ftv_segmenter_config* cfg, ftv_segmenter** out) {
    if (!cfg || !out) return FTV_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->n_images < 1 || cfg->n_images > FTV_SEG_MAX_IMAGES || !cfg->widths || !cfg->heights)
        return FTV_ERR_INVALID_ARG;
    if (cfg->sample_bytes != 1 && cfg->sample_bytes != 2) return FTV_ERR_INVALID_ARG;
    if (cfg->bit_depth < 1 || cfg->bit_depth > 8 * cfg->sample_bytes) return FTV_ERR_INVALID_ARG;
    if (cfg->grid_step < 1 || cfg->grid_step > FTV_SEG_MAX_STEP) return FTV_ERR_INVALID_ARG;
    if (cfg->compactness < 0 || cfg->compactness > 255) return FTV_ERR_INVALID_ARG;
    if (cfg->iterations < 1 || cfg->iterations > 64) return FTV_ERR_INVALID_ARG;
    auto* g = new ftv_segmenter();
    g->n_images = cfg->n_images;
    g->sb = cfg->sample_bytes;
    g->bd = cfg->bit_depth;
    g->S = cfg->grid_step;
    g->m = cfg->compactness;
    g->T = cfg->iterations;
    int64_t P = 0, K = 0;
    for (int i = 0; i < g->n_images; ++i) {
        const int W = cfg->widths[i], H = cfg->heights[i];
        if (W < 1 || H < 1 || W > FTV_MAX_DIM || H > FTV_MAX_DIM) {
            delete g;
            return FTV_ERR_INVALID_ARG;
        }
        SegImage m{};
        m.W = W;
        m.H = H;
        m.gw = (W + g->S - 1) / g->S;
        m.gh = (H + g->S - 1) / g->S;
        m.K = m.gw * m.gh;
        m.pix_base = (int32_t)std::min<int64_t>(P, INT32_MAX);
        m.seg_base = (int32_t)std::min<int64_t>(K, INT32_MAX);
        P += (int64_t)W * H;
        K += m.K;
        g->max_W = std::max(g->max_W, W);
        g->max_H = std::max(g->max_H, H);
        g->max_K = std::max(g->max_K, m.K);
        g->h_meta.push_back(m);
    }
    // global pixel names must fit 31 bits (component names are packed into 32-bit key halves)
    if (P >= INT32_MAX || K >= INT32_MAX) {
        delete g;
        return FTV_ERR_INVALID_ARG;
    }
    g->P = P;
    g->K = (int32_t)K;
    g->wc = (unsigned long long)g->S * g->S;
    g->ws = (unsigned long long)g->m * g->m;
    if (g->bd > 8) g->ws <<= 2 * (g->bd - 8);
    if (g->bd < 8) g->wc <<= 2 * (8 - g->bd);
    // unanchored groups at least halve every round
    int64_t maxP = 0;
    for (const auto& m : g->h_meta) maxP = std::max<int64_t>(maxP, (int64_t)m.W * m.H);
    int rounds = 1;
    while ((1LL << (rounds - 1)) < maxP) ++rounds;
    g->rounds = rounds + 1;
    cudaGetDevice(&g->device);

    Scratch& s = g->sc;
    bool ok = cudaMallocHost(reinterpret_cast<void**>(&g->h_img), sizeof(SegImage) * g->n_images) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&g->staged, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && dalloc(g, &g->d_img, g->n_images);
    ok = ok && dalloc(g, &s.cen, K) && dalloc(g, &s.sums, K) && dalloc(g, &s.mainkey, K);
    ok = ok && dalloc(g, &s.lab, P) && dalloc(g, &s.par, P) && dalloc(g, &s.csum, P) && dalloc(g, &s.gpar, P);
    ok = ok && dalloc(g, &s.glab, P) && dalloc(g, &s.gsum, P) && dalloc(g, &s.gmean, P);
    ok = ok && dalloc(g, &s.best, P) && dalloc(g, &s.comps, P) && dalloc(g, &s.orph[0], P) &&
         dalloc(g, &s.orph[1], P);
    ok = ok && dalloc(g, &s.uroots[0], P) && dalloc(g, &s.uroots[1], P) && dalloc(g, &s.mains, P) &&
         dalloc(g, &s.gname, P) && dalloc(g, &s.dirty, P);
    ok = ok && dalloc(g, &s.cnt, 2 * g->rounds + 4) && dalloc(g, &s.status, 1);
    ok = ok && cudaMemset(s.status, 0, sizeof(uint32_t)) == cudaSuccess;
    if (!ok) {
        release(g);
        cudaGetLastError();
        return FTV_ERR_OUT_OF_MEMORY;
    }
    s.img = g->d_img;
    s.S = g->S;
    s.sb = g->sb;
    s.rounds = g->rounds;
    s.wc = g->wc;
    s.ws = g->ws;
    // Distance arithmetic. |x - X| < 3S in pixels for every candidate (a candidate's pixels, hence its
    // mean, lie within one cell of the candidate's cell), so in 1/16 units dsp < 2 (48 S)^2, and
    // dcol <= 3 (16 (2^bd - 1))^2 for samples within the bit depth. In the DOT32 form positions are
    // relative to the tile, |position| <= 16 (127 + 3S) = R, and every partial sum is bounded by
    // wc' 3 vmax^2 + ws' 6 R^2.
    {
        const unsigned long long gcd = std::gcd(g->wc, g->ws);
        const unsigned long long wcn = g->wc / gcd, wsn = g->ws / gcd;
        const unsigned long long vmax = 16ull * ((1ull << g->bd) - 1), dmax = 48ull * g->S;
        const unsigned long long R = 16ull * (kATileW - 1 + 3ull * g->S);
        const unsigned long long direct = wcn * 3ull * vmax * vmax + wsn * 2ull * dmax * dmax;
        const unsigned long long dot = wcn * 3ull * vmax * vmax + wsn * 6ull * R * R;
        g->dist_mode = dot < (1ull << 31) ? DIST_DOT32
                       : direct < (1ull << 32) ? DIST_NARROW
                       : (g->bd <= 11 ? DIST_WIDE : DIST_WIDE_COLOUR);
        s.wcn = (uint32_t)(g->dist_mode <= DIST_NARROW ? wcn : 0);
        s.wsn = (uint32_t)(g->dist_mode <= DIST_NARROW ? wsn : 0);
    }
    // shared memory of an assignment tile: the cells it can see, 44 bytes each
    {
        const int ncx = (kATileW - 1 + g->S - 1) / g->S + 3, ncy = (kATileH - 1 + g->S - 1) / g->S + 3;
        s.max_cells = ncx * ncy;
        g->assign_smem = (size_t)s.max_cells * (2 * sizeof(int4) + 6 * sizeof(uint32_t));
        cudaError_t e = cudaSuccess;
        const int smem_bytes = (int)g->assign_smem;
        switch (g->dist_mode) {
            case DIST_DOT32:
                e = cudaFuncSetAttribute(assign_kernel<DIST_DOT32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes);
                break;
            case DIST_NARROW:
                e = cudaFuncSetAttribute(assign_kernel<DIST_NARROW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes);
                break;
            case DIST_WIDE:
                e = cudaFuncSetAttribute(assign_kernel<DIST_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes);
                break;
            default:
                e = cudaFuncSetAttribute(assign_kernel<DIST_WIDE_COLOUR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes);
        }
        if (e != cudaSuccess) {
            release(g);
            return FTV_ERR_CUDA;
        }
    }
    *out = g;
    return FTV_OK;
}

extern "C" ftv_status ftv_segmenter_segments(const ftv_segmenter* g, int32_t* n_segments) {
    if (!g || !n_segments) return FTV_ERR_INVALID_ARG;
    for (int i = 0; i < g->n_images; ++i) n_segments[i] = g->h_meta[i].K;
    return FTV_OK;
}

extern "C" ftv_status ftv_superpixels(ftv_segmenter* g, const void* const* d_planes, const int64_t* pitch_bytes,
                                      int32_t* const* d_labels, ftv_stream stream) {
    if (!g || !d_planes || !pitch_bytes || !d_labels) return FTV_ERR_INVALID_ARG;
    for (int i = 0; i < g->n_images; ++i) {
        if (!d_labels[i]) return FTV_ERR_INVALID_ARG;
        for (int c = 0; c < 3; ++c)
            if (!d_planes[3 * i + c] || pitch_bytes[3 * i + c] < (int64_t)g->h_meta[i].W * g->sb)
                return FTV_ERR_INVALID_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->device) cudaSetDevice(g->device);
    ftv::NvtxRange range("ftv_superpixels");
    cudaStream_t st = (cudaStream_t)stream;
    // the staging copy of the previous call must have left before it is rewritten
    if (cudaEventSynchronize(g->staged) != cudaSuccess) {
        if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
        return FTV_ERR_CUDA;
    }
    for (int i = 0; i < g->n_images; ++i) {
        SegImage m = g->h_meta[i];
        for (int c = 0; c < 3; ++c) {
            m.plane[c] = d_planes[3 * i + c];
            m.pitch[c] = pitch_bytes[3 * i + c];
        }
        m.out = d_labels[i];
        g->h_img[i] = m;
    }
    Scratch& s = g->sc;
    cudaError_t e = cudaMemcpyAsync(g->d_img, g->h_img, sizeof(SegImage) * g->n_images, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(g->staged, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.cnt, 0, sizeof(int32_t) * (2 * g->rounds + 4), st);
    if (e != cudaSuccess) {
        if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
        return FTV_ERR_CUDA;
    }
    const dim3 kgrid((g->max_K + kThreads - 1) / kThreads, g->n_images);
    const dim3 tgrid((g->max_W + kTileW - 1) / kTileW, (g->max_H + kTileH - 1) / kTileH, g->n_images);
    const dim3 agrid((g->max_W + kATileW - 1) / kATileW, (g->max_H + kATileH - 1) / kATileH, g->n_images);
    const dim3 tblock(kTileW, kTileH);
    int sm = 0;
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, g->device);
    const int lgrid = std::max(1, std::min<int>((int)((g->P + kThreads - 1) / kThreads), sm * 8));
    int64_t n = 0;
    const bool prof = g->profiling;
    if (prof) cudaEventRecord(g->ev[0], st);
    seed_kernel<<<kgrid, kThreads, 0, st>>>(s);
    ++n;
    for (int it = 0; it < g->T; ++it) {
        const int acc = it + 1 < g->T, last = it + 1 == g->T;
        if (prof) cudaEventRecord(g->ev[2 + 2 * it], st);
        const size_t sm_bytes = g->assign_smem;
        switch (g->dist_mode) {
            case DIST_DOT32: assign_kernel<DIST_DOT32><<<agrid, tblock, sm_bytes, st>>>(s, acc, last); break;
            case DIST_NARROW: assign_kernel<DIST_NARROW><<<agrid, tblock, sm_bytes, st>>>(s, acc, last); break;
            case DIST_WIDE: assign_kernel<DIST_WIDE><<<agrid, tblock, sm_bytes, st>>>(s, acc, last); break;
            default: assign_kernel<DIST_WIDE_COLOUR><<<agrid, tblock, sm_bytes, st>>>(s, acc, last);
        }
        if (prof) cudaEventRecord(g->ev[3 + 2 * it], st);
        ++n;
        if (acc) {
            update_kernel<<<kgrid, kThreads, 0, st>>>(s);
            ++n;
        }
    }
    runs_kernel<<<tgrid, tblock, 0, st>>>(s);
    links_kernel<<<tgrid, tblock, 0, st>>>(s);
    flatten_kernel<<<tgrid, tblock, 0, st>>>(s);
    main_kernel<<<tgrid, tblock, 0, st>>>(s);
    group_init_kernel<<<lgrid, kThreads, 0, st>>>(s);
    n += 5;
    for (int r = 0; r < g->rounds; ++r) {
        if (r == 0) pick0_kernel<<<tgrid, tblock, 0, st>>>(s);
        else pick_kernel<<<lgrid, kThreads, 0, st>>>(s, r);
        link_kernel<<<lgrid, kThreads, 0, st>>>(s, r);
        merge_kernel<<<lgrid, kThreads, 0, st>>>(s, r);
        finish_kernel<<<lgrid, kThreads, 0, st>>>(s, r);
        n += 4;
    }
    final_flatten_kernel<<<lgrid, kThreads, 0, st>>>(s);
    relabel_kernel<<<tgrid, tblock, 0, st>>>(s);
    n += 2;
    if (prof) cudaEventRecord(g->ev[1], st);
    g->timed = g->timed || prof;
    g->launches += n;
    e = cudaGetLastError();
    if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    return e == cudaSuccess ? FTV_OK : FTV_ERR_CUDA;
}

extern "C" ftv_status ftv_segmenter_check(ftv_segmenter* g, ftv_stream stream) {
    if (!g) return FTV_ERR_INVALID_ARG;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return FTV_ERR_CUDA;
    uint32_t st = 0;
    if (cudaMemcpy(&st, g->sc.status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return FTV_ERR_CUDA;
    if (st && cudaMemset(g->sc.status, 0, sizeof(st)) != cudaSuccess) return FTV_ERR_CUDA;
    return st ? FTV_ERR_TIMEOUT : FTV_OK;
}

extern "C" int64_t ftv_segmenter_launch_count(const ftv_segmenter* g) { return g ? g->launches : 0; }

extern "C" ftv_status ftv_segmenter_set_profiling(ftv_segmenter* g, int32_t enable) {
    if (!g) return FTV_ERR_INVALID_ARG;
    if (enable && g->ev.empty()) {
        g->ev.resize(2 + 2 * g->T, nullptr);
        for (auto& e : g->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return FTV_ERR_CUDA;
    }
    g->profiling = enable != 0;
    return FTV_OK;
}

extern "C" ftv_status ftv_segmenter_kernel_ms(ftv_segmenter* g, float* assign_ms, float* total_ms) {
    if (!g || (!assign_ms && !total_ms)) return FTV_ERR_INVALID_ARG;
    if (!g->timed) return FTV_ERR_STATE;
    if (cudaEventSynchronize(g->ev[1]) != cudaSuccess) return FTV_ERR_CUDA;
    float ms = 0.f, sum = 0.f;
    for (int it = 0; it < g->T; ++it) {
        if (cudaEventElapsedTime(&ms, g->ev[2 + 2 * it], g->ev[3 + 2 * it]) != cudaSuccess) return FTV_ERR_CUDA;
        sum += ms;
    }
    if (assign_ms) *assign_ms = sum / g->T;
    if (total_ms) {
        if (cudaEventElapsedTime(&ms, g->ev[0], g->ev[1]) != cudaSuccess) return FTV_ERR_CUDA;
        *total_ms = ms;
    }
    return FTV_OK;
}

extern "C" ftv_status ftv_segmenter_destroy(ftv_segmenter* g) {
    if (!g) return FTV_ERR_INVALID_ARG;
    cudaEventSynchronize(g->staged);
    release(g);
    return FTV_OK;
}
