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

#include "ftv_internal.h"

namespace ftv {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStat = 8;  // per segment: n, dP[3], dI[3], pad

template <int SB>
__device__ __forceinline__ int sample(const void* plane, int64_t pitch, int x, int y) {
    const char* row = static_cast<const char*>(plane) + (int64_t)y * pitch;
    if (SB == 1) return reinterpret_cast<const uint8_t*>(row)[x];
    return reinterpret_cast<const uint16_t*>(row)[x];
}

struct Frames {
    const void* cur[3];
    const void* prev[3];
    const void* ifr[3];
    int64_t pc[3], pp[3], pi[3];
};

__device__ __forceinline__ void add64(int64_t* dst, int v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)(long long)v);
}

// One thread per pixel (blockIdx.y = row). Per-pixel differences cur - prev and cur - I are summed per
// segment; lanes with the same label are reduced in the warp first (one atomic per run and quantity).
template <int SB, int NCH, bool HAS_I>
__global__ void temporal_accumulate_kernel(Frames f, const int32_t* __restrict__ labels, int W, int S,
                                           int64_t* __restrict__ stats, uint32_t* status) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const bool in = x < W;
    const int l = in ? labels[(int64_t)y * W + x] : -1;
    const bool ok = in && (unsigned)l < (unsigned)S;
    if (in && !ok) atomicOr(status, ST_BAD_LABEL);
    int dp[3] = {0, 0, 0}, di[3] = {0, 0, 0};
    if (ok) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int a = sample<SB>(f.cur[c], f.pc[c], x, y);
            dp[c] = a - sample<SB>(f.prev[c], f.pp[c], x, y);
            if (HAS_I) di[c] = a - sample<SB>(f.ifr[c], f.pi[c], x, y);
        }
    }
    const int key = ok ? l : -1;
    unsigned rem = __ballot_sync(kFull, ok);
    while (rem) {
        const int leader = __ffs(rem) - 1;
        const int kk = __shfl_sync(kFull, key, leader);
        const bool mine = key == kk;
        const unsigned grp = __ballot_sync(kFull, mine);
        int sums[1 + 2 * NCH];
        sums[0] = __popc(grp);
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            sums[1 + c] = __reduce_add_sync(kFull, mine ? dp[c] : 0);
            sums[1 + NCH + c] = HAS_I ? __reduce_add_sync(kFull, mine ? di[c] : 0) : 0;
        }
        if (lane == leader) {
            int64_t* st = stats + (int64_t)kk * kStat;
            add64(&st[0], sums[0]);
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                add64(&st[1 + c], sums[1 + c]);
                if (HAS_I) add64(&st[4 + c], sums[1 + NCH + c]);
            }
        }
        rem &= ~grp;
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
// decide: one thread per segment sets its mask; each block's count of changed segments goes to the spare
// word (index 7) of the stats of its first segment. compact: each block adds up the counts of the blocks
// before it, scans its own changed flags and writes their positions; the last block writes the total.
constexpr int kChunk = 1024;

__device__ __forceinline__ int decide(const int64_t* st, int nch, bool has_i, int t_p, int t_i) {
    const int64_t n = st[0];
    int m = FTV_MASK_CHANGED;
    if (n > 0) {
        bool okp = true, oki = has_i;
        for (int c = 0; c < nch; ++c) {
            okp = okp && abs64(st[1 + c]) < (int64_t)t_p * n;
            oki = oki && abs64(st[4 + c]) < (int64_t)t_i * n;
        }
        m = okp ? FTV_MASK_REUSE_P : (oki ? FTV_MASK_REUSE_I : FTV_MASK_CHANGED);
    }
    return m;
}

__global__ void __launch_bounds__(kChunk) temporal_decide_kernel(int64_t* __restrict__ stats, int S, int nch, bool has_i,
                                                                 int t_p, int t_i, uint8_t* __restrict__ mask) {
    const int s = blockIdx.x * kChunk + threadIdx.x;
    int m = FTV_MASK_CHANGED;
    if (s < S) {
        m = decide(stats + (int64_t)s * kStat, nch, has_i, t_p, t_i);
        mask[s] = (uint8_t)m;
    }
    const int cnt = __syncthreads_count(s < S && m == FTV_MASK_CHANGED);
    if (threadIdx.x == 0) stats[(int64_t)blockIdx.x * kChunk * kStat + 7] = cnt;
}

__global__ void __launch_bounds__(kChunk) temporal_compact_kernel(const int64_t* __restrict__ stats, int S,
                                                                  const uint8_t* __restrict__ mask,
                                                                  int32_t* __restrict__ changed, int32_t* n_changed) {
    __shared__ int s_base;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    int before = 0;  // changed segments of the blocks before this one
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += kChunk) before += (int)stats[(int64_t)b * kChunk * kStat + 7];
    before = __reduce_add_sync(kFull, before);
    if ((threadIdx.x & 31) == 0 && before) atomicAdd(&s_base, before);
    __syncthreads();
    const int s = blockIdx.x * kChunk + threadIdx.x;
    const int flag = s < S && mask[s] == FTV_MASK_CHANGED;
    int total;
    const int pos = block_exclusive_scan(flag, &total);
    if (flag) changed[s_base + pos] = s;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *n_changed = s_base + total;
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

cudaError_t launch_temporal(const void* const* cur, const int64_t* cur_pitch, const void* const* prev,
                            const int64_t* prev_pitch, const void* const* ifr, const int64_t* ifr_pitch,
                            int sample_bytes, const int32_t* labels, int W, int H, int S, int t_p, int t_i,
                            int mode, int64_t* stats, uint8_t* mask, int32_t* changed, int32_t* n_changed,
                            uint32_t* status, cudaStream_t s, int64_t* launches) {
    cudaError_t e = cudaMemsetAsync(stats, 0, sizeof(int64_t) * kStat * (size_t)(S > 0 ? S : 1), s);
    if (e != cudaSuccess) return e;
    Frames f{};
    const int nch = mode == FTV_TM_ALL_YUV ? 3 : 1;
    for (int c = 0; c < 3; ++c) {
        f.cur[c] = cur[c];
        f.prev[c] = prev[c];
        f.ifr[c] = ifr ? ifr[c] : nullptr;
        f.pc[c] = cur_pitch[c];
        f.pp[c] = prev_pitch[c];
        f.pi[c] = ifr ? ifr_pitch[c] : 0;
    }
    const dim3 block(256), grid((W + 255) / 256, H);
    const bool hi = ifr != nullptr;
#define FTV_T(SB, NCH, HI) temporal_accumulate_kernel<SB, NCH, HI><<<grid, block, 0, s>>>(f, labels, W, S, stats, status)
    if (W > 0 && H > 0) {
        if (sample_bytes == 1) {
            if (nch == 1) { if (hi) FTV_T(1, 1, true); else FTV_T(1, 1, false); }
            else { if (hi) FTV_T(1, 3, true); else FTV_T(1, 3, false); }
        } else {
            if (nch == 1) { if (hi) FTV_T(2, 1, true); else FTV_T(2, 1, false); }
            else { if (hi) FTV_T(2, 3, true); else FTV_T(2, 3, false); }
        }
        *launches += 1;
    }
#undef FTV_T
    const int chunks = std::max(1, (S + kChunk - 1) / kChunk);
    if (S > 0) temporal_decide_kernel<<<chunks, kChunk, 0, s>>>(stats, S, nch, hi, t_p, t_i, mask);
    temporal_compact_kernel<<<chunks, kChunk, 0, s>>>(stats, S, mask, changed, n_changed);
    *launches += S > 0 ? 2 : 1;
    return cudaGetLastError();
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
