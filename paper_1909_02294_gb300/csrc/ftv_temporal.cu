// Temporal consistency test, winner-take-all readout and per-pixel depth maps.
//
// Paper, Sec. III-E: a segment is left out of the new estimate when every component of its mean
// (Y, Cb, Cr) vector changed by less than T_P against the collocated segment of the previous P frame,
// or by less than T_I against the I frame; it then adopts that frame's depth. With the segment's
// pixel set fixed by the current label map, n pixels and channel sums S, "mean changed by less than
// T" is |S_cur - S_ref| < T * n, which the kernels below evaluate exactly in 64-bit integers.
// The winner-take-all readout stands in for the paper's graph-cut optimisation (Sec. IV-B), which is
// not part of this library: it returns the label of least cost per segment.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>

#include "ftv_internal.h"

namespace ftv {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int SB>
__device__ __forceinline__ int load_sample(const char* p) {
    if (SB == 1) return __ldg(reinterpret_cast<const uint8_t*>(p));
    return __ldg(reinterpret_cast<const uint16_t*>(p));
}

__device__ __forceinline__ void add64(int64_t* dst, int v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)(long long)v);
}

// Per-segment sums over a tile of kAccCols x kAccGroups kAccRows pixels per CTA of 256 threads: each thread
// walks one column of kAccRows pixels and sums the vertical runs of equal labels in registers (a segment's
// pixels are contiguous, so a column meets few runs). A finished run is added to the CTA's bins in shared
// memory, indexed by label - (the tile's least label); labels beyond kBins of it go to global memory
// directly. At the end each non-empty bin is added to the segment's 64-bit sums, once per tile. All sums are
// exact integers, so the order of the additions does not change the result. Tile bins are 32-bit: a tile
// has at most 2048 pixels of differences below 2^16.
constexpr int kAccCols = 128;   // pixels per tile row, one thread each
constexpr int kAccRows = 8;     // rows per thread
constexpr int kAccGroups = 2;   // row groups per CTA
constexpr int kAccThreads = kAccCols * kAccGroups;
constexpr int kBins = 512;
static_assert(kAccThreads == 256, "one CTA of 256 threads per tile");

// The references of one launch (kernel parameters, read in place).
struct TemporalRefs {
    TemporalRef r[kMaxTemporalRefs];
};

template <int SB, int NCH, bool HAS_I>
__global__ void __launch_bounds__(kAccThreads) temporal_accumulate_kernel(const __grid_constant__ TemporalRefs p,
                                                                          uint32_t* status) {
    constexpr int Q = 1 + NCH * (HAS_I ? 2 : 1);  // per segment: n, dP[NCH], dI[NCH]
    constexpr int TR = kAccGroups * kAccRows;     // tile rows
    __shared__ __align__(16) int bins[Q][kBins];
    __shared__ int s_base, s_top;
    const TemporalRef& f = p.r[blockIdx.z];  // blockIdx.z: the reference
    const int W = f.W, H = f.H, S = f.S;
    if ((int)blockIdx.x * kAccCols >= W || (int)blockIdx.y * TR >= H) return;  // past this view
    int64_t* __restrict__ stats = f.stats;
    const int tid = threadIdx.x;
    const int x = blockIdx.x * kAccCols + tid % kAccCols;
    const int y0 = blockIdx.y * TR + (tid / kAccCols) * kAccRows;
    // Every load of the column is issued before any is used: positions past the view's edge are clamped into
    // it (the block starts inside the view), so the loads need no branch, and those pixels are then dropped
    // through their label. Each plane's row pointer steps down the column (no per-row multiplication) and
    // stays on the last row of the view once it is reached.
    const int xc = min(x, W - 1), yc0 = min(y0, H - 1);
    const int32_t* pl = f.labels + (int64_t)yc0 * W + xc;
    const char* pa[NCH];
    const char* pb[NCH];
    const char* pe[HAS_I ? NCH : 1];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        pa[c] = static_cast<const char*>(f.cur[c]) + (int64_t)yc0 * f.pc[c] + (int64_t)xc * SB;
        pb[c] = static_cast<const char*>(f.prev[c]) + (int64_t)yc0 * f.pp[c] + (int64_t)xc * SB;
        if (HAS_I) pe[c] = static_cast<const char*>(f.ifr[c]) + (int64_t)yc0 * f.pi[c] + (int64_t)xc * SB;
    }
    int lab[kAccRows];
    int a[kAccRows][NCH], b[kAccRows][NCH], e[kAccRows][HAS_I ? NCH : 1];
#pragma unroll
    for (int r = 0; r < kAccRows; ++r) {
        lab[r] = __ldg(pl);
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            a[r][c] = load_sample<SB>(pa[c]);
            b[r][c] = load_sample<SB>(pb[c]);
            if (HAS_I) e[r][c] = load_sample<SB>(pe[c]);
        }
        if (r + 1 < kAccRows && y0 + r + 1 < H) {  // next row, unless it lies past the view
            pl += W;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                pa[c] += f.pc[c];
                pb[c] += f.pp[c];
                if (HAS_I) pe[c] += f.pi[c];
            }
        }
    }
    int lmin = INT_MAX, lmax = -1;
    bool bad = false;
#pragma unroll
    for (int r = 0; r < kAccRows; ++r) {
        const bool in = x < W && y0 + r < H;
        if (in && (unsigned)lab[r] < (unsigned)S) {
            lmin = min(lmin, lab[r]);
            lmax = max(lmax, lab[r]);
        } else {
            bad = bad || in;
            lab[r] = -1;
        }
    }
    if (bad) atomicOr(status, ST_BAD_LABEL);
    for (int i = tid; i < Q * kBins / 4; i += kAccThreads) reinterpret_cast<int4*>(&bins[0][0])[i] = make_int4(0, 0, 0, 0);
    if (tid == 0) {
        s_base = INT_MAX;
        s_top = -1;
    }
    __syncthreads();
    lmin = __reduce_min_sync(kFull, lmin);
    lmax = __reduce_max_sync(kFull, lmax);
    if ((tid & 31) == 0 && lmax >= 0) {
        atomicMin(&s_base, lmin);
        atomicMax(&s_top, lmax);
    }
    __syncthreads();
    const int base = s_base;

    // word q of segment s: stats[q * ms + s] (q = 0: n, 1 + c: dP[c], 4 + c: dI[c])
    const int64_t ms = f.ms;
    {
        int cur = -1;
        int acc[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[q] = 0;
        auto flush = [&]() {
            const unsigned bi = (unsigned)(cur - base);
            if (bi < (unsigned)kBins) {
#pragma unroll
                for (int q = 0; q < Q; ++q)
                    if (q == 0 || acc[q] != 0) atomicAdd(&bins[q][bi], acc[q]);
            } else {
                add64(&stats[cur], acc[0]);
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    add64(&stats[(1 + c) * ms + cur], acc[1 + c]);
                    if (HAS_I) add64(&stats[(4 + c) * ms + cur], acc[1 + NCH + c]);
                }
            }
        };
#pragma unroll
        for (int r = 0; r < kAccRows; ++r) {
            const int l = lab[r];
            if (l != cur) {
                if (cur >= 0) flush();
                cur = l;
#pragma unroll
                for (int q = 0; q < Q; ++q) acc[q] = 0;
            }
            if (l >= 0) {
                acc[0] += 1;
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    acc[1 + c] += a[r][c] - b[r][c];
                    if (HAS_I) acc[1 + NCH + c] += a[r][c] - e[r][c];
                }
            }
        }
        if (cur >= 0) flush();
    }
    __syncthreads();
    // the bins in use: the tile's labels from base to s_top (those beyond kBins went to global memory)
    const int used = min(kBins, s_top - base + 1);
    for (int i = tid; i < used; i += kAccThreads) {
        const int n = bins[0][i];
        if (n == 0) continue;
        const int64_t sg = base + i;
        add64(&stats[sg], n);
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            if (bins[1 + c][i] != 0) add64(&stats[(1 + c) * ms + sg], bins[1 + c][i]);
            if (HAS_I && bins[1 + NCH + c][i] != 0) add64(&stats[(4 + c) * ms + sg], bins[1 + NCH + c][i]);
        }
    }
}

__device__ int block_exclusive_scan(int v, int* total) {
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += t;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const int base = warp > 0 ? warp_sums[warp - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + incl - v;
}

__device__ __forceinline__ int64_t abs64(int64_t v) { return v < 0 ? -v : v; }

// The masks and the ordered list of changed segments, in two passes over blocks of kChunk segments.
// decide: one thread per segment reads its sums (one word from each plane in use, coalesced over the block),
// sets its mask and clears those words, so that the next call needs no clearing pass; each block's count of
// changed segments goes to plane 7 at the block's index. compact: each block adds up the counts of the
// blocks before it, scans its own changed flags and writes their positions; the last block writes the total.
constexpr int kChunk = 256;

// blockIdx.y: the reference; blocks past its segments return.
template <int NCH, bool HAS_I>
__global__ void __launch_bounds__(kChunk) temporal_decide_kernel(const __grid_constant__ TemporalRefs p, int t_p,
                                                                 int t_i) {
    const TemporalRef& R = p.r[blockIdx.y];
    const int S = R.S;
    if ((int)blockIdx.x * kChunk >= S) return;
    int64_t* __restrict__ stats = R.stats;
    const int64_t ms = R.ms;
    const int s = blockIdx.x * kChunk + threadIdx.x;
    int m = FTV_MASK_CHANGED;
    if (s < S) {
        int64_t dp[NCH], di[HAS_I ? NCH : 1];
        const int64_t n = stats[s];
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            dp[c] = stats[(1 + c) * ms + s];
            if (HAS_I) di[c] = stats[(4 + c) * ms + s];
        }
        if (n > 0) {
            bool okp = true, oki = HAS_I;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                okp = okp && abs64(dp[c]) < (int64_t)t_p * n;
                if (HAS_I) oki = oki && abs64(di[c]) < (int64_t)t_i * n;
            }
            m = okp ? FTV_MASK_REUSE_P : (oki ? FTV_MASK_REUSE_I : FTV_MASK_CHANGED);
        }
        R.mask[s] = (uint8_t)m;
        // leave the sums zero for the next call
        stats[s] = 0;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            stats[(1 + c) * ms + s] = 0;
            if (HAS_I) stats[(4 + c) * ms + s] = 0;
        }
    }
    const int cnt = __syncthreads_count(s < S && m == FTV_MASK_CHANGED);
    if (threadIdx.x == 0) stats[7 * ms + blockIdx.x] = cnt;
}

// blockIdx.y: the reference; blocks past its chunks return (a reference without segments has one chunk).
__global__ void __launch_bounds__(kChunk) temporal_compact_kernel(const __grid_constant__ TemporalRefs p) {
    __shared__ int s_base;
    const TemporalRef& R = p.r[blockIdx.y];
    const int S = R.S, chunks = S > 0 ? (S + kChunk - 1) / kChunk : 1;
    if ((int)blockIdx.x >= chunks) return;
    const int64_t* __restrict__ counts = R.stats + 7 * (int64_t)R.ms;
    const uint8_t* __restrict__ mask = R.mask;
    int32_t* __restrict__ changed = R.changed;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    int before = 0;  // changed segments of the blocks before this one
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += kChunk) before += (int)counts[b];
    before = __reduce_add_sync(kFull, before);
    if ((threadIdx.x & 31) == 0 && before) atomicAdd(&s_base, before);
    __syncthreads();
    const int s = blockIdx.x * kChunk + threadIdx.x;
    const int flag = s < S && mask[s] == FTV_MASK_CHANGED;
    int total;
    const int pos = block_exclusive_scan(flag, &total);
    if (flag) changed[s_base + pos] = s;
    if ((int)blockIdx.x == chunks - 1 && threadIdx.x == 0) *R.n_changed = s_base + total;
}

// One warp per listed segment: least-cost label, smallest on ties; masked segments adopt.
__global__ void wta_kernel(const int32_t* __restrict__ cost, int S, int L, const uint8_t* __restrict__ mask,
                           const uint16_t* __restrict__ prev_label, const uint16_t* __restrict__ ifr_label,
                           const int32_t* __restrict__ list, const int32_t* __restrict__ n_listed,
                           uint16_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int n = list ? min(max(*n_listed, 0), S) : S;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
        const int s = list ? list[i] : i;
        if ((unsigned)s >= (unsigned)S) continue;
        const int m = mask ? mask[s] : FTV_MASK_CHANGED;
        if (m == FTV_MASK_REUSE_P && prev_label) {
            if (lane == 0) out[s] = prev_label[s];
            continue;
        }
        if (m == FTV_MASK_REUSE_I && ifr_label) {
            if (lane == 0) out[s] = ifr_label[s];
            continue;
        }
        // order key: signed cost mapped to unsigned in the high word, label in the low word
        unsigned long long best = ~0ull;
        const int32_t* row = cost + (int64_t)s * L;
        for (int d = lane; d < L; d += 32) {
            const unsigned long long k =
                ((unsigned long long)((uint32_t)row[d] ^ 0x80000000u) << 32) | (unsigned long long)d;
            best = k < best ? k : best;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(kFull, best, o);
            best = t < best ? t : best;
        }
        if (lane == 0) out[s] = (uint16_t)(best & 0xffffu);
    }
}

__global__ void depth_map_kernel(const int32_t* __restrict__ labels, int W, int S,
                                 const uint16_t* __restrict__ seg_label, const float* __restrict__ label_z, int L,
                                 float* __restrict__ depth, uint32_t* status) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const int64_t p = (int64_t)y * W + x;
    const int s = labels[p];
    float z = 0.0f;
    if ((unsigned)s < (unsigned)S) {
        const int d = seg_label[s];
        if (d < L) z = label_z[d];
        else atomicOr(status, ST_BAD_LABEL);
    } else {
        atomicOr(status, ST_BAD_LABEL);
    }
    depth[p] = z;
}

}  // namespace

cudaError_t launch_temporal_refs(const TemporalRef* refs, int n, int sample_bytes, int mode, bool has_i, int t_p,
                                 int t_i, uint32_t* status, cudaStream_t s, int64_t* launches) {
    if (n <= 0) return cudaSuccess;
    if (n > kMaxTemporalRefs) return cudaErrorInvalidValue;
    TemporalRefs p{};
    int tx = 0, ty = 0, chunks = 1;
    bool any_s = false;
    for (int k = 0; k < n; ++k) {
        p.r[k] = refs[k];
        tx = std::max(tx, (refs[k].W + kAccCols - 1) / kAccCols);
        ty = std::max(ty, (refs[k].H + kAccGroups * kAccRows - 1) / (kAccGroups * kAccRows));
        chunks = std::max(chunks, (refs[k].S + kChunk - 1) / kChunk);
        any_s = any_s || refs[k].S > 0;
    }
    const int nch = mode == FTV_TM_ALL_YUV ? 3 : 1;
    if (tx > 0 && ty > 0) {
        const dim3 block(kAccThreads), grid(tx, ty, n);
#define FTV_T(SB, NCH, HI) temporal_accumulate_kernel<SB, NCH, HI><<<grid, block, 0, s>>>(p, status)
        if (sample_bytes == 1) {
            if (nch == 1) { if (has_i) FTV_T(1, 1, true); else FTV_T(1, 1, false); }
            else { if (has_i) FTV_T(1, 3, true); else FTV_T(1, 3, false); }
        } else {
            if (nch == 1) { if (has_i) FTV_T(2, 1, true); else FTV_T(2, 1, false); }
            else { if (has_i) FTV_T(2, 3, true); else FTV_T(2, 3, false); }
        }
#undef FTV_T
        *launches += 1;
    }
    if (any_s) {
        const dim3 grid(chunks, n);
        if (nch == 1) {
            if (has_i) temporal_decide_kernel<1, true><<<grid, kChunk, 0, s>>>(p, t_p, t_i);
            else temporal_decide_kernel<1, false><<<grid, kChunk, 0, s>>>(p, t_p, t_i);
        } else {
            if (has_i) temporal_decide_kernel<3, true><<<grid, kChunk, 0, s>>>(p, t_p, t_i);
            else temporal_decide_kernel<3, false><<<grid, kChunk, 0, s>>>(p, t_p, t_i);
        }
        *launches += 1;
    }
    temporal_compact_kernel<<<dim3(chunks, n), kChunk, 0, s>>>(p);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_temporal(const void* const* cur, const int64_t* cur_pitch, const void* const* prev,
                            const int64_t* prev_pitch, const void* const* ifr, const int64_t* ifr_pitch,
                            int sample_bytes, const int32_t* labels, int W, int H, int S, int t_p, int t_i,
                            int mode, int64_t* stats, int ms, uint8_t* mask, int32_t* changed, int32_t* n_changed,
                            uint32_t* status, bool clear, cudaStream_t s, int64_t* launches) {
    if (clear) {  // planes 0 to 6 over the call's segments
        const cudaError_t e = cudaMemsetAsync(stats, 0, sizeof(int64_t) * (6 * (size_t)ms + (size_t)S), s);
        if (e != cudaSuccess) return e;
    }
    TemporalRef r{};
    for (int c = 0; c < 3; ++c) {
        r.cur[c] = cur[c];
        r.prev[c] = prev[c];
        r.ifr[c] = ifr ? ifr[c] : nullptr;
        r.pc[c] = cur_pitch[c];
        r.pp[c] = prev_pitch[c];
        r.pi[c] = ifr ? ifr_pitch[c] : 0;
    }
    r.labels = labels;
    r.stats = stats;
    r.mask = mask;
    r.changed = changed;
    r.n_changed = n_changed;
    r.W = W;
    r.H = H;
    r.S = S;
    r.ms = ms;
    return launch_temporal_refs(&r, 1, sample_bytes, mode, ifr != nullptr, t_p, t_i, status, s, launches);
}

cudaError_t launch_wta(const int32_t* cost, int S, int L, const uint8_t* mask, const uint16_t* prev_label,
                       const uint16_t* ifr_label, const int32_t* list, const int32_t* n_listed, uint16_t* out,
                       cudaStream_t s) {
    const int warps_per_block = 8;
    const int blocks = std::max(1, std::min(65535, (S + warps_per_block - 1) / warps_per_block));
    wta_kernel<<<blocks, warps_per_block * 32, 0, s>>>(cost, S, L, mask, prev_label, ifr_label, list, n_listed, out);
    return cudaGetLastError();
}

cudaError_t launch_depth_map(const int32_t* labels, int W, int H, int S, const uint16_t* seg_label,
                             const float* label_z, int L, float* depth, uint32_t* status, cudaStream_t s) {
    if (W <= 0 || H <= 0) return cudaSuccess;
    const dim3 block(256), grid((W + 255) / 256, H);
    depth_map_kernel<<<grid, block, 0, s>>>(labels, W, S, seg_label, label_z, L, depth, status);
    return cudaGetLastError();
}

}  // namespace ftv
