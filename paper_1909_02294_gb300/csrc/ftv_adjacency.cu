// Segment adjacency and adaptive smoothing weights (Sec. III-D, Eq. 2-3).
//
// Paper: the intra-view discontinuity cost V_{s,t} = beta |d_s - d_t| links every pair of adjacent
// segments s, t of a view, with beta = beta0 / || mean YCbCr_s - mean YCbCr_t ||_1 (Eq. 3). The graph
// cut that uses V is not part of this library; this builds its input: the sorted list of adjacent
// segment pairs s < t (pixels 4- or 8-connected) and beta per pair, in the frame's colours.
// The paper leaves a zero distance open: the distance is floored at min_diff. The distance is the exact
// rational sum_c |S_cs n_t - S_ct n_s| / (n_s n_t) (S channel sums, n pixel counts), and
// beta = beta0 * (n_s n_t) / numerator in double, rounded to float.
//
// Kernels: one warp per segment walks the segment's pixels (segment index), collects the labels t > s of
// their neighbours in a small shared hash, sorts them and sums the segment's colour; a scan turns the
// per-segment counts into edge offsets; one thread per segment writes its edges and weights.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ftv_internal.h"

namespace ftv {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kHash = 64;        // per-warp neighbour hash slots
constexpr int kMaxDeg = 32;      // neighbours t > s kept per segment (more sets ST_OVERFLOW)
constexpr int kWarps = 8;

__device__ __forceinline__ int plane_sample(const void* p, int64_t pitch, int sb, int x, int y) {
    const char* row = static_cast<const char*>(p) + (int64_t)y * pitch;
    return sb == 1 ? (int)reinterpret_cast<const uint8_t*>(row)[x] : (int)reinterpret_cast<const uint16_t*>(row)[x];
}

struct AdjArgs {
    const int32_t* offs;
    const uint32_t* pix;
    const int32_t* labels;
    const void* plane[3];
    int64_t pitch[3];
    int32_t W, H, S, sb, conn;
    int64_t* stats;   // [S][4]: n, sum Y, sum Cb, sum Cr
    int32_t* deg;     // [S]
    int32_t* slots;   // [S][kMaxDeg] sorted neighbours t > s
    uint32_t* status;
};

__global__ void __launch_bounds__(kWarps * 32) neighbours_kernel(AdjArgs a) {
    __shared__ int table[kWarps][kHash];
    __shared__ int list[kWarps][kHash];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int* tab = table[wib];
    int* lst = list[wib];
    static const int dxs[8] = {1, -1, 0, 0, 1, 1, -1, -1}, dys[8] = {0, 0, 1, -1, 1, -1, 1, -1};
    const int ndir = a.conn == 8 ? 8 : 4;
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < a.S; s += (gridDim.x * blockDim.x) >> 5) {
        tab[lane] = -1;
        tab[lane + 32] = -1;
        __syncwarp();
        const int b = a.offs[s], e = a.offs[s + 1];
        long long sy = 0, su = 0, sv = 0;
        bool full = false;
        for (int i = b + lane; i < e; i += 32) {
            const uint32_t xy = a.pix[i];
            const int x = xy & 0xffff, y = xy >> 16;
            sy += plane_sample(a.plane[0], a.pitch[0], a.sb, x, y);
            su += plane_sample(a.plane[1], a.pitch[1], a.sb, x, y);
            sv += plane_sample(a.plane[2], a.pitch[2], a.sb, x, y);
            for (int k = 0; k < ndir; ++k) {
                const int qx = x + dxs[k], qy = y + dys[k];
                if (qx < 0 || qx >= a.W || qy < 0 || qy >= a.H) continue;
                const int t = a.labels[(int64_t)qy * a.W + qx];
                if (t <= s || t >= a.S) continue;
                int h = (int)((unsigned)t * 2654435761u >> 26);  // top 6 bits: 0..63
                int probes = 0;
                for (; probes < kHash; ++probes) {
                    const int old = atomicCAS(&tab[h], -1, t);
                    if (old == -1 || old == t) break;
                    h = (h + 1) & (kHash - 1);
                }
                if (probes == kHash) full = true;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            sy += __shfl_xor_sync(kFull, sy, o);
            su += __shfl_xor_sync(kFull, su, o);
            sv += __shfl_xor_sync(kFull, sv, o);
        }
        __syncwarp();
        // compact the distinct neighbours, then rank them (each is compared with every other)
        const int v0 = tab[lane], v1 = tab[lane + 32];
        const unsigned m0 = __ballot_sync(kFull, v0 >= 0), m1 = __ballot_sync(kFull, v1 >= 0);
        const int n0 = __popc(m0), n = n0 + __popc(m1);
        if (v0 >= 0) lst[__popc(m0 & ((1u << lane) - 1u))] = v0;
        if (v1 >= 0) lst[n0 + __popc(m1 & ((1u << lane) - 1u))] = v1;
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            const int v = lst[j];
            int rank = 0;
            for (int q = 0; q < n; ++q) rank += lst[q] < v;
            if (rank < kMaxDeg) a.slots[(int64_t)s * kMaxDeg + rank] = v;
        }
        if (__any_sync(kFull, full) || n > kMaxDeg) {
            if (lane == 0) atomicOr(a.status, ST_OVERFLOW);
        }
        if (lane == 0) {
            a.deg[s] = min(n, kMaxDeg);
            int64_t* st = a.stats + (int64_t)s * 4;
            st[0] = e - b;
            st[1] = sy;
            st[2] = su;
            st[3] = sv;
        }
        __syncwarp();
    }
}

__device__ int block_scan_adj(int v, int* total) {
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
        int x = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += t;
        }
        warp_sums[lane] = x;
    }
    __syncthreads();
    const int base = warp > 0 ? warp_sums[warp - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + incl - v;
}

// One block of 1024 threads: edge offsets from the per-segment counts, and the edge count.
__global__ void edge_offsets_kernel(const int32_t* __restrict__ deg, int S, int32_t* __restrict__ offs,
                                    int32_t* n_edges) {
    const int per = (S + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(S, b + per);
    int sum = 0;
    for (int s = b; s < e; ++s) sum += deg[s];
    int total;
    int run = block_scan_adj(sum, &total);
    for (int s = b; s < e; ++s) {
        offs[s] = run;
        run += deg[s];
    }
    if (threadIdx.x == 0) *n_edges = total;
}

__global__ void edges_kernel(const int32_t* __restrict__ deg, const int32_t* __restrict__ slots,
                             const int32_t* __restrict__ offs, const int64_t* __restrict__ stats, int S, int cap,
                             double beta0, double min_diff, int32_t* __restrict__ es, int32_t* __restrict__ et,
                             float* __restrict__ beta) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        const int64_t* A = stats + (int64_t)s * 4;
        for (int j = 0; j < deg[s]; ++j) {
            const int e = offs[s] + j;
            if (e >= cap) break;
            const int t = slots[(int64_t)s * kMaxDeg + j];
            const int64_t* B = stats + (int64_t)t * 4;
            long long num = 0;
            for (int c = 1; c <= 3; ++c) {
                const long long d = A[c] * B[0] - B[c] * A[0];
                num += d < 0 ? -d : d;
            }
            const double den = (double)(A[0] * B[0]);
            const double dist = __ddiv_rn((double)num, den);
            const double bt = dist < min_diff ? __ddiv_rn(beta0, min_diff) : __ddiv_rn(__dmul_rn(beta0, den), (double)num);
            es[e] = s;
            et[e] = t;
            beta[e] = (float)bt;
        }
    }
}

}  // namespace
}  // namespace ftv

using namespace ftv;

extern "C" ftv_status ftv_adjacency(ftv_ctx* ctx, int32_t ref_index, const void* const* d_frame,
                                    const int64_t* frame_pitch, const int32_t* d_labels, int32_t n_segments,
                                    int32_t connectivity, double beta0, double min_diff, int32_t capacity,
                                    int32_t* d_edge_s, int32_t* d_edge_t, float* d_beta, int32_t* d_n_edges,
                                    ftv_stream stream) {
    if (!ctx || ref_index < 0 || ref_index >= ctx->n_refs || !d_frame || !frame_pitch || !d_labels) return FTV_ERR_INVALID_ARG;
    if (n_segments < 0 || n_segments > ctx->max_segments || (connectivity != 4 && connectivity != 8))
        return FTV_ERR_INVALID_ARG;
    if (capacity < 0 || (capacity > 0 && (!d_edge_s || !d_edge_t || !d_beta)) || !d_n_edges) return FTV_ERR_INVALID_ARG;
    if (!(min_diff > 0.0) || !(beta0 == beta0)) return FTV_ERR_INVALID_ARG;
    RefState& r = ctx->refs[ref_index];
    for (int c = 0; c < 3; ++c)
        if (!d_frame[c] || frame_pitch[c] < (int64_t)r.W * ctx->sample_bytes) return FTV_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    NvtxRange range("ftv_adjacency");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t one = std::max<int64_t>(ctx->penalty, 3LL * ((1LL << ctx->bit_depth) - 1));
    const int64_t mpc = ctx->combine == FTV_COMBINE_MIN ? one : one * std::max(1, r.n_nbrs);
    cudaError_t e = launch_segment_index(d_labels, r.W, r.H, n_segments, mpc, r.d_offs, r.d_cursor, r.d_pix,
                                         ctx->d_status, s, &ctx->launches);
    r.S_indexed = n_segments;
    if (e == cudaSuccess && n_segments > 0) {
        AdjArgs a{};
        a.offs = r.d_offs;
        a.pix = r.d_pix;
        a.labels = d_labels;
        for (int c = 0; c < 3; ++c) {
            a.plane[c] = d_frame[c];
            a.pitch[c] = frame_pitch[c];
        }
        a.W = r.W;
        a.H = r.H;
        a.S = n_segments;
        a.sb = ctx->sample_bytes;
        a.conn = connectivity;
        // scratch: this reference's slot of the temporal sums, which is then no longer known to be zero
        int64_t* const scratch = ctx->d_tstats + (size_t)ref_index * ctx->max_segments * 8;
        ctx->tstats_zero[ref_index] = 0;
        a.stats = scratch;
        a.deg = ctx->d_adj_deg;
        a.slots = ctx->d_adj_slots;
        a.status = ctx->d_status;
        const int blocks = std::max(1, std::min(65535, (n_segments + kWarps - 1) / kWarps));
        neighbours_kernel<<<blocks, kWarps * 32, 0, s>>>(a);
        edge_offsets_kernel<<<1, 1024, 0, s>>>(ctx->d_adj_deg, n_segments, ctx->d_adj_offs, d_n_edges);
        edges_kernel<<<std::max(1, std::min(65535, (n_segments + 255) / 256)), 256, 0, s>>>(
            ctx->d_adj_deg, ctx->d_adj_slots, ctx->d_adj_offs, scratch, n_segments, capacity, beta0, min_diff,
            d_edge_s, d_edge_t, d_beta);
        ctx->launches += 3;
        e = cudaGetLastError();
    } else if (e == cudaSuccess) {
        e = cudaMemsetAsync(d_n_edges, 0, sizeof(int32_t), s);
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return e == cudaSuccess ? FTV_OK : FTV_ERR_CUDA;
}
