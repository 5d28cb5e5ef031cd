// Batched and served forms: per-stream resident state and one launch sequence for many jobs.
//
// Paper: Sec. III-E keeps an I-type and the preceding P-type depth frame per view and re-estimates only
// segments whose colour changed. Here every camera stream keeps that state on the device (a ring of
// three packed frames: current, previous P, I; per-segment labels of the previous and the I frame), and
// a batch runs the whole hot path for many jobs (frames of different streams, shapes, view, segment and
// label counts) with one fixed sequence of launches:
//   H2D descriptor copy -> pack (all views of all jobs) -> temporal statistics -> masks -> changed lists
//   -> zero changed cost rows -> plan -> persistent cost kernel over the flat (job, reference, tile,
//   label block) queue -> winner-take-all with adoption and label-state update -> optional depth maps.
// Every kernel reads its work from the descriptor block and sizes its loop from it, with grids fixed
// at creation, so one captured CUDA graph of the sequence replays for any batch composition (the host
// rewrites the pinned descriptor block between replays).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <vector>

#include "ftv_internal.h"

using namespace ftv;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStat = 8;

struct PackTask {
    const void* planes[3];
    int64_t pitch[3];
    void* out;
    uint32_t* status;  // the job's status word
    int32_t W, H, sb, fmt;
    uint32_t maxv;
    int32_t row_base;  // first row of this task in the flattened row space
};

struct TempUnit {
    const void* cur;
    const void* prev;
    const void* ifr;
    const int32_t* labels;
    int64_t* stats;
    uint8_t* mask;
    int32_t* changed;
    int32_t* n_changed;
    uint32_t* status;              // the job's status word
    const uint32_t* stream_status; // errors of the stream's resident state (its label maps' index)
    int32_t W, H, S, t_p, t_i, nch, fmt, is_i;
    int32_t tile_base;  // temporal tiles of P-frame units, flattened (I-frame units have none)
    int32_t stat_base;  // stats words of P-frame units, flattened
    int32_t chunk_base; // decide/compact chunks of all units, flattened
    int32_t pad;
};

struct WtaUnit {
    const int32_t* cost;
    const uint8_t* mask;
    uint16_t* prev_label;
    uint16_t* i_label;
    uint16_t* out;
    const int32_t* labels;
    float* depth;
    const float* label_z;
    uint32_t* status;  // the job's status word
    int32_t S, L, W, H, is_i;
    int32_t seg_base;    // segments, flattened
    int32_t depth_base;  // rows of units with depth maps, flattened (units without depth own no rows)
};

struct Header {
    int32_t n_pack, n_units, fmt, combine;
    int32_t pack_rows, temp_tiles, temp_stats, wta_segs, depth_rows, temp_chunks, pad[2];
};

struct BatchLayout {
    size_t header, pack, temp, jobs, wta, total;
};

BatchLayout layout(int max_views, int max_units) {
    BatchLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 255) & ~(size_t)255;
        return at;
    };
    L.header = take(sizeof(Header));
    L.pack = take(sizeof(PackTask) * max_views);
    L.temp = take(sizeof(TempUnit) * max_units);
    L.jobs = take(sizeof(RefJob) * max_units);
    L.wta = take(sizeof(WtaUnit) * max_units);
    L.total = o;
    return L;
}

__device__ __forceinline__ int find_base(const int32_t* base_field_of, int stride_bytes, int n, int v) {
    // largest i in [0, n) with base(i) <= v, where base(i) is an int at byte offset i * stride
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int b = *reinterpret_cast<const int32_t*>(reinterpret_cast<const char*>(base_field_of) +
                                                         (size_t)mid * stride_bytes);
        if (b <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// --------------------------------------------------------------------------------------------- pack

__device__ __forceinline__ uint32_t load_plane(const void* plane, int64_t pitch, int sb, int x, int y) {
    const char* row = static_cast<const char*>(plane) + (int64_t)y * pitch;
    return sb == 1 ? (uint32_t)reinterpret_cast<const uint8_t*>(row)[x] : (uint32_t)reinterpret_cast<const uint16_t*>(row)[x];
}

__global__ void pack_multi_kernel(const Header* __restrict__ hdr, const PackTask* __restrict__ tasks) {
    const int rows = hdr->pack_rows, n = hdr->n_pack;
    for (int g = blockIdx.x; g < rows; g += gridDim.x) {
        const int t = find_base(&tasks[0].row_base, sizeof(PackTask), n, g);
        const PackTask& T = tasks[t];
        const int y = g - T.row_base;
        for (int x = threadIdx.x; x < T.W; x += blockDim.x) {
            uint32_t a = load_plane(T.planes[0], T.pitch[0], T.sb, x, y);
            uint32_t b = load_plane(T.planes[1], T.pitch[1], T.sb, x, y);
            uint32_t c = load_plane(T.planes[2], T.pitch[2], T.sb, x, y);
            if (a > T.maxv || b > T.maxv || c > T.maxv) {
                atomicOr(T.status, ST_BAD_SAMPLE);
                a = min(a, T.maxv);
                b = min(b, T.maxv);
                c = min(c, T.maxv);
            }
            const int64_t i = (int64_t)y * T.W + x;
            if (T.fmt == FMT_U8X4) static_cast<uint32_t*>(T.out)[i] = a | (b << 8) | (c << 16);
            else if (T.fmt == FMT_P10) static_cast<uint32_t*>(T.out)[i] = a | (b << 10) | (c << 20);
            else static_cast<uint2*>(T.out)[i] = make_uint2(a | (b << 16), c);
        }
    }
}

// ----------------------------------------------------------------------------------------- temporal

__device__ __forceinline__ void texel_fields(const void* base, int fmt, int64_t i, int* v) {
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

__global__ void temporal_zero_multi_kernel(const Header* __restrict__ hdr, const TempUnit* __restrict__ units) {
    const int total = hdr->temp_stats, n = hdr->n_units;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const int u = find_base(&units[0].stat_base, sizeof(TempUnit), n, g);
        units[u].stats[g - units[u].stat_base] = 0;
    }
}

// Per-segment sums of cur - prev and cur - I over the P-frame units' pixels, in tiles of kTTileW x kTTileH
// pixels flattened over the units (tile_base). Each thread walks one column of kTRows pixels of a tile and
// sums the vertical runs of equal labels in registers; finished runs go to the CTA's 32-bit bins in shared
// memory, indexed by label - (the tile's least label) (labels beyond kTBins of it go to global memory
// directly), and each non-empty bin is added to the segment's 64-bit sums once per tile. Every load of a
// column is issued before any is used (positions past the view's edge are clamped into it and dropped
// through their label). The sums are exact integers: the order of the additions does not matter.
constexpr int kTTileW = 128, kTRows = 8, kTTileH = 2 * kTRows, kTBins = 512;

__global__ void __launch_bounds__(256) temporal_accumulate_multi_kernel(const Header* __restrict__ hdr,
                                                                        const TempUnit* __restrict__ units) {
    __shared__ __align__(16) int bins[7][kTBins];  // n, dP[3], dI[3]
    __shared__ int s_base, s_top;
    const int tiles = hdr->temp_tiles, n_units = hdr->n_units;
    const int tid = threadIdx.x;
    for (int g = blockIdx.x; g < tiles; g += gridDim.x) {
        const TempUnit& T = units[find_base(&units[0].tile_base, sizeof(TempUnit), n_units, g)];
        const int W = T.W, H = T.H, S = T.S, nch = T.nch, fmt = T.fmt;
        const int tx = (W + kTTileW - 1) / kTTileW, t = g - T.tile_base;
        const int x = (t % tx) * kTTileW + (tid % kTTileW), y0 = (t / tx) * kTTileH + (tid / kTTileW) * kTRows;
        const int xc = min(x, W - 1);
        int lab[kTRows];
        int d[kTRows][6];  // dP[3], dI[3]
#pragma unroll
        for (int r = 0; r < kTRows; ++r) {
            const int64_t i = (int64_t)min(y0 + r, H - 1) * W + xc;
            lab[r] = __ldg(T.labels + i);
            int a[3], b[3], c[3];
            texel_fields(T.cur, fmt, i, a);
            texel_fields(T.prev, fmt, i, b);
            texel_fields(T.ifr, fmt, i, c);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                d[r][k] = k < nch ? a[k] - b[k] : 0;
                d[r][3 + k] = k < nch ? a[k] - c[k] : 0;
            }
        }
        int lmin = INT_MAX, lmax = -1;
        bool bad = false;
#pragma unroll
        for (int r = 0; r < kTRows; ++r) {
            const bool in = x < W && y0 + r < H;
            if (in && (unsigned)lab[r] < (unsigned)S) {
                lmin = min(lmin, lab[r]);
                lmax = max(lmax, lab[r]);
            } else {
                bad = bad || in;
                lab[r] = -1;
            }
        }
        if (bad) atomicOr(T.status, ST_BAD_LABEL);
        __syncthreads();  // the previous tile's bins are no longer read
        for (int i = tid; i < 7 * kTBins / 4; i += blockDim.x) reinterpret_cast<int4*>(&bins[0][0])[i] = make_int4(0, 0, 0, 0);
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
        int cur = -1, acc[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) acc[q] = 0;
        auto flush = [&]() {
            const unsigned bi = (unsigned)(cur - base);
            if (bi < (unsigned)kTBins) {
#pragma unroll
                for (int q = 0; q < 7; ++q)
                    if (q == 0 || acc[q] != 0) atomicAdd(&bins[q][bi], acc[q]);
            } else {
                unsigned long long* st = reinterpret_cast<unsigned long long*>(T.stats + (int64_t)cur * kStat);
#pragma unroll
                for (int q = 0; q < 7; ++q)
                    if (acc[q] != 0) atomicAdd(&st[q], (unsigned long long)(long long)acc[q]);
            }
        };
#pragma unroll
        for (int r = 0; r < kTRows; ++r) {
            const int l = lab[r];
            if (l != cur) {
                if (cur >= 0) flush();
                cur = l;
#pragma unroll
                for (int q = 0; q < 7; ++q) acc[q] = 0;
            }
            if (l >= 0) {
                acc[0] += 1;
#pragma unroll
                for (int q = 1; q < 7; ++q) acc[q] += d[r][q - 1];
            }
        }
        if (cur >= 0) flush();
        __syncthreads();
        const int used = min(kTBins, s_top - base + 1);
        for (int i = tid; i < used; i += blockDim.x) {
            if (bins[0][i] == 0) continue;
            unsigned long long* st = reinterpret_cast<unsigned long long*>(T.stats + (int64_t)(base + i) * kStat);
#pragma unroll
            for (int q = 0; q < 7; ++q)
                if (bins[q][i] != 0) atomicAdd(&st[q], (unsigned long long)(long long)bins[q][i]);
        }
    }
}

__device__ int block_scan_1024(int v, int* total) {
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
        int s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
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

__device__ __forceinline__ int64_t iabs64(int64_t v) { return v < 0 ? -v : v; }

// Masks and ordered changed lists of every unit, in two passes over chunks of kTChunk segments flattened over
// the units (chunk_base; a unit without segments has one chunk). decide: one thread per segment sets its mask
// (I-frame units list every segment: Sec. III-E estimates all segments of an I-type frame) and each chunk's
// count of changed segments goes to the spare word (index 7) of its first segment's sums; the unit's first
// chunk also reports errors found when the stream's resident state was built (a label outside [0, S), a
// segment too large for int32 sums), which every job of that stream carries. compact: each chunk adds the
// counts of the unit's chunks before it, scans its own flags and writes their positions; the unit's last
// chunk writes the total.
constexpr int kTChunk = 256;

__global__ void __launch_bounds__(kTChunk) temporal_decide_multi_kernel(const Header* __restrict__ hdr,
                                                                        const TempUnit* __restrict__ units) {
    const int chunks = hdr->temp_chunks, n_units = hdr->n_units;
    for (int g = blockIdx.x; g < chunks; g += gridDim.x) {
        const TempUnit& T = units[find_base(&units[0].chunk_base, sizeof(TempUnit), n_units, g)];
        const int c = g - T.chunk_base, S = T.S;
        if (c == 0 && threadIdx.x == 0 && T.stream_status) {
            const uint32_t e = *T.stream_status;
            if (e) atomicOr(T.status, e);
        }
        const int s = c * kTChunk + threadIdx.x;
        int m = FTV_MASK_CHANGED;
        if (s < S && !T.is_i) {
            const int64_t* st = T.stats + (int64_t)s * kStat;
            const int64_t n = st[0];
            if (n > 0) {
                bool okp = true, oki = true;
                for (int k = 0; k < T.nch; ++k) {
                    okp = okp && iabs64(st[1 + k]) < (int64_t)T.t_p * n;
                    oki = oki && iabs64(st[4 + k]) < (int64_t)T.t_i * n;
                }
                m = okp ? FTV_MASK_REUSE_P : (oki ? FTV_MASK_REUSE_I : FTV_MASK_CHANGED);
            }
        }
        if (s < S) T.mask[s] = (uint8_t)m;
        const int cnt = __syncthreads_count(s < S && m == FTV_MASK_CHANGED);
        if (threadIdx.x == 0 && S > 0) T.stats[(int64_t)c * kTChunk * kStat + 7] = cnt;
    }
}

__global__ void __launch_bounds__(kTChunk) temporal_compact_multi_kernel(const Header* __restrict__ hdr,
                                                                         const TempUnit* __restrict__ units) {
    __shared__ int s_before;
    const int chunks = hdr->temp_chunks, n_units = hdr->n_units;
    for (int g = blockIdx.x; g < chunks; g += gridDim.x) {
        const TempUnit& T = units[find_base(&units[0].chunk_base, sizeof(TempUnit), n_units, g)];
        const int c = g - T.chunk_base, S = T.S, nc = S > 0 ? (S + kTChunk - 1) / kTChunk : 1;
        if (threadIdx.x == 0) s_before = 0;
        __syncthreads();
        int before = 0;  // changed segments of the unit's chunks before this one
        for (int b = threadIdx.x; b < c; b += kTChunk) before += (int)T.stats[(int64_t)b * kTChunk * kStat + 7];
        before = __reduce_add_sync(kFull, before);
        if ((threadIdx.x & 31) == 0 && before) atomicAdd(&s_before, before);
        __syncthreads();
        const int s = c * kTChunk + threadIdx.x;
        const int flag = s < S && T.mask[s] == FTV_MASK_CHANGED;
        int total;
        const int pos = block_scan_1024(flag, &total);
        if (flag) T.changed[s_before + pos] = s;
        if (c == nc - 1 && threadIdx.x == 0) *T.n_changed = s_before + total;
        __syncthreads();  // s_before is reset for the next chunk only after every thread has used it
    }
}

// Zero the cost rows of each unit's changed segments (blockIdx.y = unit).
__global__ void zero_changed_rows_kernel(const Header* __restrict__ hdr, const RefJob* __restrict__ jobs) {
    for (int u = blockIdx.y; u < hdr->n_units; u += gridDim.y) {
        const RefJob& J = jobs[u];
        const int n = min(max(*J.n_listed, 0), J.S);
        const int64_t total = (int64_t)n * J.L;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
            const int k = (int)(i / J.L), d = (int)(i - (int64_t)k * J.L);
            const int s = J.list[k];
            if ((unsigned)s < (unsigned)J.S) J.cost[(int64_t)s * J.L + d] = 0;
        }
    }
}

// ------------------------------------------------------------------------------------------ WTA etc.

// One warp per segment over all units: argmin for changed segments (smallest label on ties), adoption
// for reused ones; the result updates the stream's label state and is copied to the caller's output.
__global__ void wta_multi_kernel(const Header* __restrict__ hdr, const WtaUnit* __restrict__ units) {
    const int lane = threadIdx.x & 31;
    const int total = hdr->wta_segs, n = hdr->n_units;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < total; g += (gridDim.x * blockDim.x) >> 5) {
        const int u = find_base(&units[0].seg_base, sizeof(WtaUnit), n, g);
        const WtaUnit& T = units[u];
        const int s = g - T.seg_base;
        const int m = T.mask[s];
        uint16_t label;
        if (m == FTV_MASK_REUSE_P) {
            label = T.prev_label[s];
        } else if (m == FTV_MASK_REUSE_I) {
            label = T.i_label[s];
        } else {
            unsigned long long best = ~0ull;
            const int32_t* row = T.cost + (int64_t)s * T.L;
            for (int d = lane; d < T.L; d += 32) {
                const unsigned long long k = ((unsigned long long)((uint32_t)row[d] ^ 0x80000000u) << 32) | (unsigned)d;
                best = k < best ? k : best;
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long t = __shfl_xor_sync(kFull, best, o);
                best = t < best ? t : best;
            }
            label = (uint16_t)(best & 0xffffu);
        }
        if (lane == 0) {
            T.prev_label[s] = label;
            if (T.is_i) T.i_label[s] = label;
            if (T.out) T.out[s] = label;
        }
    }
}

__global__ void depth_multi_kernel(const Header* __restrict__ hdr, const WtaUnit* __restrict__ units) {
    const int rows = hdr->depth_rows, n = hdr->n_units;
    for (int g = blockIdx.x; g < rows; g += gridDim.x) {
        const int u = find_base(&units[0].depth_base, sizeof(WtaUnit), n, g);
        const WtaUnit& T = units[u];
        const int y = g - T.depth_base;
        for (int x = threadIdx.x; x < T.W; x += blockDim.x) {
            const int64_t p = (int64_t)y * T.W + x;
            const int s = T.labels[p];
            float z = 0.0f;
            if ((unsigned)s < (unsigned)T.S && T.prev_label[s] < T.L) z = T.label_z[T.prev_label[s]];
            else atomicOr(T.status, ST_BAD_LABEL);
            T.depth[p] = z;
        }
    }
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1));
}

}  // namespace

// A job submitted with ftv_batch_submit and not yet launched: the caller's arrays copied.
struct QueuedJob {
    ftv_ctx* ctx = nullptr;
    int32_t frame_type = 0;
    std::vector<const void*> planes;
    std::vector<int64_t> pitch;
    std::vector<uint16_t*> label_out;
    std::vector<float*> depth_out;
    bool has_label_out = false, has_depth_out = false;
    int64_t footprint = 0;
};

constexpr int kTicketRing = 4096;  // completed tickets whose status ftv_batch_poll still reports

struct ftv_batch {
    int device = 0;
    int n_sm = 0;
    int temp_per_sm = 1;  // resident CTAs per SM of temporal_accumulate_multi_kernel
    int32_t max_jobs = 0, max_units = 0, max_views = 0;
    BatchLayout lay{};
    char* d_desc = nullptr;     // device descriptor block
    char* h_stage = nullptr;    // pinned staging copy
    ftv::Plan* d_plan = nullptr;
    uint32_t* d_job_status = nullptr;  // [max_jobs] one status word per job of a launch
    uint32_t* h_job_status = nullptr;  // pinned copy, written back by the launch's last step
    int32_t prepared_jobs = 0, launched_jobs = 0;
    // ticketed submission (ftv_batch_submit / ftv_batch_flush / ftv_batch_poll)
    std::vector<QueuedJob> queue;
    uint64_t next_ticket = 1;
    uint64_t launch_first = 0;          // tickets [launch_first, launch_first + launch_n) are in the last launch
    int32_t launch_n = 0;
    bool harvested = true;              // their statuses are in `ring`
    int64_t launch_footprint = 0;       // footprint of the jobs of the launch in flight
    int64_t budget = 0;                 // admission budget in device bytes (0: none)
    std::vector<int8_t> ring;           // status of ticket t at t % kTicketRing
    int32_t fmt = -1, combine = -1;
    bool fast_rcp = false;
    bool penalty_floor = false;
    int kind = 0;
    int chunks = 1;           // cost-kernel launches per batch launch
    int graph_chunks = 0;
    int32_t prepared_units = 0;
    int cost_grid = 0;
    cudaEvent_t done = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_fmt = -1, graph_combine = -1;
    bool graph_pf = false;
    int graph_kind = -1;
    int64_t launches = 0;
};

namespace ftv {

void free_stream_state(ftv_ctx* c) {
    StreamState& st = c->stream;
    for (auto& r : st.refs) {
        cudaFree(r.d_prev_label);
        cudaFree(r.d_i_label);
        cudaFree(r.d_mask);
        cudaFree(r.d_changed);
        cudaFree(r.d_n_changed);
        cudaFree(r.d_stats);
        cudaFree(r.d_cost);
        cudaFree(r.d_labels);
        for (auto* p : r.d_nbrs_ring) cudaFree(p);
    }
    st.refs.clear();
    for (auto& p : st.d_ring) {
        cudaFree(p);
        p = nullptr;
    }
    cudaFree(st.d_status);
    st.d_status = nullptr;
    st.ready = false;
}

}  // namespace ftv

namespace {

// A job's (or a batch's) device status bits as the ABI's status.
ftv_status status_of(uint32_t st) {
    if (st & ST_CHECKED) return FTV_ERR_CHECKED;
    if (st & ST_OVERFLOW) return FTV_ERR_OVERFLOW;
    if (st) return FTV_ERR_INVALID_ARG;
    return FTV_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Geometry of one reference for the footprint formulas.
struct RefDims {
    int64_t W, H, N, S;
};

// Checked builds: the last launch's out-of-view gathers (recorded in its plan), reported by all its jobs.
uint32_t checked_bits(const ftv_batch* b) {
#ifdef FTV_CHECKED
    uint32_t ck = 0;
    if (cudaMemcpy(&ck, &b->d_plan->checked, sizeof(ck), cudaMemcpyDeviceToHost) != cudaSuccess) return ST_CHECKED;
    return ck;
#else
    (void)b;
    return 0;
#endif
}

// Records the statuses of the last launch's tickets once it has completed; false while it runs.
bool harvest(ftv_batch* b) {
    if (b->harvested) return true;
    const cudaError_t e = cudaEventQuery(b->done);
    if (e == cudaErrorNotReady) return false;
    const uint32_t ck = e == cudaSuccess ? checked_bits(b) : 0;
    for (int k = 0; k < b->launch_n; ++k)
        b->ring[(b->launch_first + k) % kTicketRing] =
            (int8_t)(e == cudaSuccess ? status_of(b->h_job_status[k] | ck) : FTV_ERR_CUDA);
    if (e != cudaSuccess) cudaGetLastError();
    b->harvested = true;
    b->launch_footprint = 0;
    return true;
}


// Device bytes ftv_stream_init allocates: the status word, three packed frames, and per reference its
// labels of the previous and the I frame, mask, changed list and count, temporal sums, cost rows, label
// map copy and the neighbour geometry into each ring slot.
int64_t stream_bytes_of(size_t packed, const std::vector<RefDims>& refs, int64_t L) {
    int64_t b = sizeof(uint32_t) + 3 * (int64_t)packed;
    for (const RefDims& r : refs)
        b += r.S * (2 + 2 + 1 + 4 + 8 * kStat) + 4 + r.S * L * 4 + r.W * r.H * 4 + 3 * r.N * (int64_t)sizeof(NbrView);
    return b;
}

// Device bytes ftv_depth_init allocates (max_segments MS): packed views, status, unit descriptors, plan,
// temporal sums (one slot per reference) and adjacency scratch, label depths, and per reference its tables, neighbour geometry, segment
// index, centres and neighbour label pointers.
int64_t context_bytes_of(size_t packed, const std::vector<RefDims>& refs, int64_t L, int64_t MS, bool fp64) {
    int64_t b = (int64_t)packed + sizeof(uint32_t) + kMaxUnits * (int64_t)sizeof(RefJob) + sizeof(Plan);
    b += std::max<int64_t>(1, (int64_t)refs.size()) * MS * 8 * 8 + L * 4 + MS * 4 + MS * 32 * 4 + MS * 4;
    for (const RefDims& r : refs) {
        b += r.N * L * 9 * 4 + (fp64 ? r.N * L * 9 * 8 : 0) + r.N * (int64_t)sizeof(NbrView);
        b += 2 * (MS + 1) * 4 + MS * 4 + r.W * r.H * 4 + MS * 8 + std::max<int64_t>(1, r.N) * 8;
    }
    return b;
}

int64_t stream_bytes(const ftv_ctx* c, const int32_t* n_segments) {
    size_t packed = 0;
    for (int v = 0; v < c->n_views; ++v) packed += align256((size_t)c->cams[v].width * c->cams[v].height * c->texel_bytes);
    std::vector<RefDims> refs;
    for (int i = 0; i < c->n_refs; ++i)
        refs.push_back({c->refs[i].W, c->refs[i].H, c->refs[i].n_nbrs, n_segments[i]});
    return stream_bytes_of(packed, refs, c->L);
}

// A stream's whole footprint, as ftv_job_footprint states it: its context, its resident stream state and
// one frame of input planes.
int64_t job_bytes(const ftv_ctx* c) {
    size_t packed = 0;
    int64_t input = 0;
    for (int v = 0; v < c->n_views; ++v) {
        packed += align256((size_t)c->cams[v].width * c->cams[v].height * c->texel_bytes);
        input += 3 * (int64_t)c->cams[v].width * c->cams[v].height * c->sample_bytes;
    }
    std::vector<RefDims> refs;
    for (int i = 0; i < c->n_refs; ++i)
        refs.push_back({c->refs[i].W, c->refs[i].H, c->refs[i].n_nbrs,
                        c->stream.ready ? c->stream.refs[i].S : c->max_segments});
    return context_bytes_of(packed, refs, c->L, c->max_segments, c->precision == FTV_PRECISION_FP64) +
           stream_bytes_of(packed, refs, c->L) + input;
}

}  // namespace

extern "C" {

ftv_status ftv_stream_init(ftv_ctx* ctx, const int32_t* const* d_labels, const int32_t* n_segments, int32_t t_p,
                           int32_t t_i, int32_t mode, ftv_stream stream) {
    if (!ctx || !d_labels || !n_segments || t_p < 0 || t_i < 0) return FTV_ERR_INVALID_ARG;
    if (mode != FTV_TM_Y_ONLY && mode != FTV_TM_ALL_YUV) return FTV_ERR_INVALID_ARG;
    for (int i = 0; i < ctx->n_refs; ++i)
        if (!d_labels[i] || n_segments[i] < 0 || n_segments[i] > ctx->max_segments) return FTV_ERR_INVALID_ARG;
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != ctx->device) cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    free_stream_state(ctx);
    StreamState& st = ctx->stream;
    st.t_p = t_p;
    st.t_i = t_i;
    st.mode = mode;
    st.prev = st.iframe = -1;
    st.frames = 0;
    size_t packed = 0;
    for (int v = 0; v < ctx->n_views; ++v)
        packed += (((size_t)ctx->cams[v].width * ctx->cams[v].height * ctx->texel_bytes) + 255) & ~(size_t)255;
    bool ok = dalloc(&st.d_status, 1) == cudaSuccess && cudaMemsetAsync(st.d_status, 0, sizeof(uint32_t), s) == cudaSuccess;
    for (auto& p : st.d_ring) ok = ok && cudaMalloc(&p, packed) == cudaSuccess;
    st.refs.resize(ctx->n_refs);
    for (int i = 0; i < ctx->n_refs && ok; ++i) {
        StreamRef& R = st.refs[i];
        const RefState& r = ctx->refs[i];
        R.S = n_segments[i];
        const size_t S = (size_t)R.S;
        ok = ok && dalloc(&R.d_prev_label, S) == cudaSuccess && dalloc(&R.d_i_label, S) == cudaSuccess;
        ok = ok && dalloc(&R.d_mask, S) == cudaSuccess && dalloc(&R.d_changed, S) == cudaSuccess;
        ok = ok && dalloc(&R.d_n_changed, 1) == cudaSuccess && dalloc(&R.d_stats, S * kStat) == cudaSuccess;
        ok = ok && dalloc(&R.d_cost, S * ctx->L) == cudaSuccess;
        ok = ok && dalloc(&R.d_labels, (size_t)r.W * r.H) == cudaSuccess;
        for (int b = 0; b < 3 && ok; ++b) {
            ok = dalloc(&R.d_nbrs_ring[b], (size_t)r.n_nbrs) == cudaSuccess;
            std::vector<NbrView> nv(r.n_nbrs);
            for (int k = 0; k < r.n_nbrs; ++k) {
                const int v = r.nbrs[k];
                nv[k].texels = static_cast<char*>(st.d_ring[b]) + ctx->view_offset_bytes[v];
                nv[k].w = ctx->cams[v].width;
                nv[k].h = ctx->cams[v].height;
                nv[k].pitch = ctx->cams[v].width;
                nv[k].pad = 0;
            }
            if (ok && r.n_nbrs)
                ok = cudaMemcpy(R.d_nbrs_ring[b], nv.data(), sizeof(NbrView) * nv.size(), cudaMemcpyHostToDevice) ==
                     cudaSuccess;
        }
        if (ok) ok = cudaMemsetAsync(R.d_prev_label, 0, sizeof(uint16_t) * std::max<size_t>(S, 1), s) == cudaSuccess;
        if (ok) ok = cudaMemsetAsync(R.d_i_label, 0, sizeof(uint16_t) * std::max<size_t>(S, 1), s) == cudaSuccess;
        if (ok)
            ok = cudaMemcpyAsync(R.d_labels, d_labels[i], sizeof(int32_t) * (size_t)r.W * r.H, cudaMemcpyDeviceToDevice,
                                 s) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        free_stream_state(ctx);
        if (prev_dev >= 0 && prev_dev != ctx->device) cudaSetDevice(prev_dev);
        return FTV_ERR_OUT_OF_MEMORY;
    }
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < ctx->n_refs && e == cudaSuccess; ++i) {
        // the stream's label map is static: its segment index is built once here (with the same int32
        // overflow check as ftv_segment_index) and reused by every frame
        RefState& r = ctx->refs[i];
        const int64_t one = std::max<int64_t>(ctx->penalty, 3LL * ((1LL << ctx->bit_depth) - 1));
        const int64_t mpc = ctx->combine == FTV_COMBINE_MIN ? one : one * std::max(1, r.n_nbrs);
        e = launch_segment_index(st.refs[i].d_labels, r.W, r.H, n_segments[i], mpc, r.d_offs, r.d_cursor, r.d_pix,
                                 st.d_status, s, &ctx->launches);
        r.S_indexed = n_segments[i];
    }
    if (prev_dev >= 0 && prev_dev != ctx->device) cudaSetDevice(prev_dev);
    if (e != cudaSuccess) return FTV_ERR_CUDA;
    st.ready = true;
    return FTV_OK;
}

ftv_status ftv_stream_footprint(const ftv_ctx* ctx, const int32_t* n_segments, int64_t* bytes) {
    if (!ctx || !n_segments || !bytes) return FTV_ERR_INVALID_ARG;
    *bytes = stream_bytes(ctx, n_segments);
    return FTV_OK;
}

ftv_status ftv_stream_labels(const ftv_ctx* ctx, int32_t ref_index, const uint16_t** d_labels_out) {
    if (!ctx || !d_labels_out || !ctx->stream.ready || ref_index < 0 || ref_index >= ctx->n_refs)
        return FTV_ERR_INVALID_ARG;
    *d_labels_out = ctx->stream.refs[ref_index].d_prev_label;
    return FTV_OK;
}

ftv_status ftv_stream_mask(const ftv_ctx* ctx, int32_t ref_index, const uint8_t** d_mask, const int32_t** d_n_changed) {
    if (!ctx || !d_mask || !d_n_changed || !ctx->stream.ready || ref_index < 0 || ref_index >= ctx->n_refs)
        return FTV_ERR_INVALID_ARG;
    *d_mask = ctx->stream.refs[ref_index].d_mask;
    *d_n_changed = ctx->stream.refs[ref_index].d_n_changed;
    return FTV_OK;
}

namespace {

// Checkpoint layout of a stream's resident state: this header, the per-reference segment counts, then the
// previous P frame's packed views (if any), the I frame's packed views (if any and different), and per
// reference the previous and the I frame's per-segment labels (uint16 each).
struct StateHeader {
    char magic[4];        // "FTVS"
    int32_t version;      // 1
    int32_t n_refs, n_views, L, fmt;
    int32_t has_prev, has_i, i_is_prev, pad;
    int64_t packed_bytes, frames;
};

size_t packed_bytes_of(const ftv_ctx* c) {
    size_t packed = 0;
    for (int v = 0; v < c->n_views; ++v) packed += align256((size_t)c->cams[v].width * c->cams[v].height * c->texel_bytes);
    return packed;
}

int64_t state_bytes(const ftv_ctx* c) {
    const StreamState& st = c->stream;
    int64_t b = sizeof(StateHeader) + sizeof(int32_t) * c->n_refs;
    const bool has_prev = st.prev >= 0, has_i = st.iframe >= 0 && st.iframe != st.prev;
    b += (int64_t)packed_bytes_of(c) * ((has_prev ? 1 : 0) + (has_i ? 1 : 0));
    for (const StreamRef& r : st.refs) b += 2 * (int64_t)sizeof(uint16_t) * r.S;
    return b;
}

}  // namespace

ftv_status ftv_stream_state_bytes(const ftv_ctx* ctx, int64_t* bytes) {
    if (!ctx || !bytes || !ctx->stream.ready) return FTV_ERR_INVALID_ARG;
    *bytes = state_bytes(ctx);
    return FTV_OK;
}

ftv_status ftv_stream_state_save(const ftv_ctx* ctx, void* host_buf, int64_t bytes, ftv_stream stream) {
    if (!ctx || !host_buf || !ctx->stream.ready || bytes < state_bytes(ctx)) return FTV_ERR_INVALID_ARG;
    NvtxRange range("ftv_stream_state_save");
    const StreamState& st = ctx->stream;
    char* h = static_cast<char*>(host_buf);
    StateHeader hd{};
    std::memcpy(hd.magic, "FTVS", 4);
    hd.version = 1;
    hd.n_refs = ctx->n_refs;
    hd.n_views = ctx->n_views;
    hd.L = ctx->L;
    hd.fmt = ctx->fmt;
    hd.has_prev = st.prev >= 0;
    hd.i_is_prev = st.iframe >= 0 && st.iframe == st.prev;
    hd.has_i = st.iframe >= 0 && !hd.i_is_prev;
    hd.packed_bytes = (int64_t)packed_bytes_of(ctx);
    hd.frames = st.frames;
    std::memcpy(h, &hd, sizeof(hd));
    h += sizeof(hd);
    for (int i = 0; i < ctx->n_refs; ++i) {
        std::memcpy(h, &st.refs[i].S, sizeof(int32_t));
        h += sizeof(int32_t);
    }
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != ctx->device) cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (hd.has_prev) {
        e = cudaMemcpyAsync(h, st.d_ring[st.prev], hd.packed_bytes, cudaMemcpyDeviceToHost, s);
        h += hd.packed_bytes;
    }
    if (e == cudaSuccess && hd.has_i) {
        e = cudaMemcpyAsync(h, st.d_ring[st.iframe], hd.packed_bytes, cudaMemcpyDeviceToHost, s);
        h += hd.packed_bytes;
    }
    for (int i = 0; i < ctx->n_refs && e == cudaSuccess; ++i) {
        const StreamRef& r = st.refs[i];
        e = cudaMemcpyAsync(h, r.d_prev_label, sizeof(uint16_t) * r.S, cudaMemcpyDeviceToHost, s);
        h += sizeof(uint16_t) * r.S;
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, r.d_i_label, sizeof(uint16_t) * r.S, cudaMemcpyDeviceToHost, s);
        h += sizeof(uint16_t) * r.S;
    }
    if (prev_dev >= 0 && prev_dev != ctx->device) cudaSetDevice(prev_dev);
    return e == cudaSuccess ? FTV_OK : FTV_ERR_CUDA;
}

ftv_status ftv_stream_state_load(ftv_ctx* ctx, const void* host_buf, int64_t bytes, ftv_stream stream) {
    if (!ctx || !host_buf || !ctx->stream.ready || bytes < (int64_t)sizeof(StateHeader)) return FTV_ERR_INVALID_ARG;
    StreamState& st = ctx->stream;
    const char* h = static_cast<const char*>(host_buf);
    StateHeader hd;
    std::memcpy(&hd, h, sizeof(hd));
    h += sizeof(hd);
    // the checkpoint must come from a stream of the same shape (views, references, labels, texel format)
    if (std::memcmp(hd.magic, "FTVS", 4) != 0 || hd.version != 1 || hd.n_refs != ctx->n_refs ||
        hd.n_views != ctx->n_views || hd.L != ctx->L || hd.fmt != ctx->fmt ||
        hd.packed_bytes != (int64_t)packed_bytes_of(ctx) || (hd.i_is_prev && !hd.has_prev) ||
        (hd.has_i && !hd.has_prev))
        return FTV_ERR_INVALID_ARG;
    int64_t need = sizeof(StateHeader) + sizeof(int32_t) * ctx->n_refs +
                   hd.packed_bytes * ((hd.has_prev ? 1 : 0) + (hd.has_i ? 1 : 0));
    for (int i = 0; i < ctx->n_refs; ++i) {
        int32_t S;
        std::memcpy(&S, h + sizeof(int32_t) * i, sizeof(S));
        if (S != st.refs[i].S) return FTV_ERR_INVALID_ARG;
        need += 2 * (int64_t)sizeof(uint16_t) * S;
    }
    if (bytes < need) return FTV_ERR_INVALID_ARG;
    h += sizeof(int32_t) * ctx->n_refs;
    NvtxRange range("ftv_stream_state_load");
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != ctx->device) cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    // previous P frame into ring slot 0, a separate I frame into slot 1
    if (hd.has_prev) {
        e = cudaMemcpyAsync(st.d_ring[0], h, hd.packed_bytes, cudaMemcpyHostToDevice, s);
        h += hd.packed_bytes;
    }
    if (e == cudaSuccess && hd.has_i) {
        e = cudaMemcpyAsync(st.d_ring[1], h, hd.packed_bytes, cudaMemcpyHostToDevice, s);
        h += hd.packed_bytes;
    }
    for (int i = 0; i < ctx->n_refs && e == cudaSuccess; ++i) {
        StreamRef& r = st.refs[i];
        e = cudaMemcpyAsync(r.d_prev_label, h, sizeof(uint16_t) * r.S, cudaMemcpyHostToDevice, s);
        h += sizeof(uint16_t) * r.S;
        if (e == cudaSuccess) e = cudaMemcpyAsync(r.d_i_label, h, sizeof(uint16_t) * r.S, cudaMemcpyHostToDevice, s);
        h += sizeof(uint16_t) * r.S;
    }
    if (prev_dev >= 0 && prev_dev != ctx->device) cudaSetDevice(prev_dev);
    if (e != cudaSuccess) return FTV_ERR_CUDA;
    st.prev = hd.has_prev ? 0 : -1;
    st.iframe = hd.has_i ? 1 : (hd.i_is_prev ? 0 : -1);
    st.frames = hd.frames;
    return FTV_OK;
}

ftv_status ftv_stream_changed(const ftv_ctx* ctx, int32_t ref_index, const int32_t** d_changed) {
    if (!ctx || !d_changed || !ctx->stream.ready || ref_index < 0 || ref_index >= ctx->n_refs)
        return FTV_ERR_INVALID_ARG;
    *d_changed = ctx->stream.refs[ref_index].d_changed;
    return FTV_OK;
}

ftv_status ftv_batch_create(int32_t max_jobs, int32_t max_units, int32_t max_views, ftv_batch** out) {
    if (!out || max_jobs < 1 || max_units < 1 || max_views < 1 || max_units > kMaxUnits) return FTV_ERR_INVALID_ARG;
    *out = nullptr;
    ftv_batch* b = new (std::nothrow) ftv_batch();
    if (!b) return FTV_ERR_OUT_OF_MEMORY;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return FTV_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
    // the temporal accumulation strides over its tiles with as many CTAs as stay resident (a second wave
    // would only be a tail)
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->temp_per_sm, temporal_accumulate_multi_kernel, 256, 0) !=
            cudaSuccess ||
        b->temp_per_sm < 1)
        b->temp_per_sm = 1;
    b->fast_rcp = fast_reciprocal_exact();
    b->max_jobs = max_jobs;
    b->max_units = max_units;
    b->max_views = max_views;
    b->lay = layout(max_views, max_units);
    bool ok = cudaMalloc(reinterpret_cast<void**>(&b->d_desc), b->lay.total) == cudaSuccess;
    ok = ok && cudaMallocHost(reinterpret_cast<void**>(&b->h_stage), b->lay.total) == cudaSuccess;
    ok = ok && cudaMalloc(reinterpret_cast<void**>(&b->d_plan), sizeof(Plan)) == cudaSuccess;
    ok = ok && cudaMalloc(reinterpret_cast<void**>(&b->d_job_status), sizeof(uint32_t) * max_jobs) == cudaSuccess;
    ok = ok && cudaMemset(b->d_job_status, 0, sizeof(uint32_t) * max_jobs) == cudaSuccess;
    ok = ok && cudaMallocHost(reinterpret_cast<void**>(&b->h_job_status), sizeof(uint32_t) * max_jobs) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
        std::memset(b->h_stage, 0, b->lay.total);
        std::memset(b->h_job_status, 0, sizeof(uint32_t) * max_jobs);
        b->ring.assign(kTicketRing, (int8_t)FTV_OK);
        b->queue.reserve(max_jobs);
    }
    if (!ok) {
        cudaGetLastError();
        cudaFree(b->d_desc);
        cudaFreeHost(b->h_stage);
        cudaFree(b->d_plan);
        cudaFree(b->d_job_status);
        cudaFreeHost(b->h_job_status);
        if (b->done) cudaEventDestroy(b->done);
        delete b;
        return FTV_ERR_OUT_OF_MEMORY;
    }
    *out = b;
    return FTV_OK;
}

ftv_status ftv_batch_destroy(ftv_batch* b) {
    if (!b) return FTV_OK;
    cudaEventSynchronize(b->done);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_desc);
    cudaFreeHost(b->h_stage);
    cudaFree(b->d_plan);
    cudaFree(b->d_job_status);
    cudaFreeHost(b->h_job_status);
    cudaEventDestroy(b->done);
    delete b;
    return FTV_OK;
}

ftv_status ftv_batch_prepare(ftv_batch* b, const ftv_frame_job* jobs, int32_t n_jobs) {
    if (!b || (!jobs && n_jobs > 0) || n_jobs < 0 || n_jobs > b->max_jobs) return FTV_ERR_INVALID_ARG;
    // the staging block must not be rewritten while a launch that reads it is pending
    if (cudaEventQuery(b->done) == cudaErrorNotReady) return FTV_ERR_BUSY;
    cudaGetLastError();
    harvest(b);  // a completed ticketed launch keeps its jobs' statuses before this launch overwrites them
    NvtxRange range("ftv_batch_prepare");
    int n_views = 0, n_units = 0, fmt = -1, combine = -1;
    bool pf_all = true;
    int kind = kKindMixed;
    for (int j = 0; j < n_jobs; ++j) {
        const ftv_frame_job& J = jobs[j];
        if (!J.ctx || !J.ctx->stream.ready || !J.d_planes || !J.pitch_bytes) return FTV_ERR_INVALID_ARG;
        if (J.frame_type != FTV_FRAME_I && J.frame_type != FTV_FRAME_P) return FTV_ERR_INVALID_ARG;
        if (J.frame_type == FTV_FRAME_P && J.ctx->stream.prev < 0) return FTV_ERR_STATE;
        if (J.ctx->device != b->device) return FTV_ERR_INVALID_ARG;
        for (int k = 0; k < j; ++k)
            if (jobs[k].ctx == J.ctx) return FTV_ERR_INVALID_ARG;  // one frame per stream per batch
        if (fmt >= 0 && (J.ctx->fmt != fmt || J.ctx->combine != combine)) return FTV_ERR_INVALID_ARG;
        // one cost-kernel instantiation per launch: FP32- and FP64-precision streams do not share a batch
        if (j > 0 && J.ctx->precision != jobs[0].ctx->precision) return FTV_ERR_INVALID_ARG;
        fmt = J.ctx->fmt;
        combine = J.ctx->combine;
        pf_all = pf_all && J.ctx->penalty_floor;
        // contexts of one batch share a precision; differing entry classes take the mixed instantiation
        if (j == 0) kind = J.ctx->kind;
        else if (kind != J.ctx->kind) kind = precise_kind(kind) ? kKindPreciseMixed : kKindMixed;
        n_views += J.ctx->n_views;
        n_units += J.ctx->n_refs;
        for (int v = 0; v < J.ctx->n_views; ++v)
            for (int c = 0; c < 3; ++c) {
                if (!J.d_planes[3 * v + c]) return FTV_ERR_INVALID_ARG;
                if (J.pitch_bytes[3 * v + c] < (int64_t)J.ctx->cams[v].width * J.ctx->sample_bytes) return FTV_ERR_INVALID_ARG;
            }
    }
    if (n_views > b->max_views || n_units > b->max_units) return FTV_ERR_BUSY;

    char* h = b->h_stage;
    Header& H = *reinterpret_cast<Header*>(h + b->lay.header);
    PackTask* P = reinterpret_cast<PackTask*>(h + b->lay.pack);
    TempUnit* T = reinterpret_cast<TempUnit*>(h + b->lay.temp);
    RefJob* R = reinterpret_cast<RefJob*>(h + b->lay.jobs);
    WtaUnit* Wt = reinterpret_cast<WtaUnit*>(h + b->lay.wta);
    std::memset(&H, 0, sizeof(H));
    int pv = 0, pu = 0, pack_rows = 0, temp_tiles = 0, temp_stats = 0, temp_chunks = 0, wta_segs = 0, depth_rows = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const ftv_frame_job& J = jobs[j];
        ftv_ctx* c = J.ctx;
        StreamState& st = c->stream;
        const bool is_i = J.frame_type == FTV_FRAME_I;
        int cur = 0;
        while (cur == st.prev || (!is_i && cur == st.iframe)) ++cur;  // a ring slot that is neither prev nor I
        const int prev = is_i ? cur : st.prev;
        const int ifr = is_i ? cur : st.iframe;
        const uint32_t maxv = c->bit_depth >= 32 ? 0xffffffffu : ((1u << c->bit_depth) - 1u);
        for (int v = 0; v < c->n_views; ++v) {
            PackTask& t = P[pv++];
            for (int k = 0; k < 3; ++k) {
                t.planes[k] = J.d_planes[3 * v + k];
                t.pitch[k] = J.pitch_bytes[3 * v + k];
            }
            t.out = static_cast<char*>(st.d_ring[cur]) + c->view_offset_bytes[v];
            t.W = c->cams[v].width;
            t.H = c->cams[v].height;
            t.sb = c->sample_bytes;
            t.fmt = c->fmt;
            t.maxv = maxv;
            t.status = b->d_job_status + j;
            t.row_base = pack_rows;
            pack_rows += t.H;
        }
        for (int i = 0; i < c->n_refs; ++i) {
            const RefState& r = c->refs[i];
            StreamRef& S = st.refs[i];
            const size_t ref_off = c->view_offset_bytes[r.view];
            TempUnit& t = T[pu];
            t.cur = static_cast<char*>(st.d_ring[cur]) + ref_off;
            t.prev = static_cast<char*>(st.d_ring[prev]) + ref_off;
            t.ifr = static_cast<char*>(st.d_ring[ifr]) + ref_off;
            t.labels = S.d_labels;
            t.stats = S.d_stats;
            t.mask = S.d_mask;
            t.changed = S.d_changed;
            t.n_changed = S.d_n_changed;
            t.status = b->d_job_status + j;
            t.stream_status = st.d_status;
            t.W = r.W;
            t.H = is_i ? 0 : r.H;
            t.S = S.S;
            t.t_p = st.t_p;
            t.t_i = st.t_i;
            t.nch = st.mode == FTV_TM_ALL_YUV ? 3 : 1;
            t.fmt = c->fmt;
            t.is_i = is_i;
            t.tile_base = temp_tiles;
            t.stat_base = temp_stats;
            t.chunk_base = temp_chunks;
            t.pad = 0;
            if (!is_i) {
                temp_tiles += ((r.W + kTTileW - 1) / kTTileW) * ((r.H + kTTileH - 1) / kTTileH);
                temp_stats += S.S * kStat;
            }
            temp_chunks += S.S > 0 ? (S.S + kTChunk - 1) / kTChunk : 1;
            RefJob& q = R[pu];
            std::memset(&q, 0, sizeof(q));
            q.ref_texels = t.cur;
            q.pix = r.d_pix;
            q.offs = r.d_offs;
            q.list = S.d_changed;
            q.n_listed = S.d_n_changed;
            q.woffs = r.d_woffs;
            q.H = r.d_H;
            q.H64 = r.d_H64;
            q.nbrs = S.d_nbrs_ring[cur];
            q.cost = S.d_cost;
            q.W = r.W;
            q.Href = r.H;
            q.S = S.S;
            q.N = r.n_nbrs;
            q.L = c->L;
            q.LB = c->LB;
            q.nLB = c->nLB;
            q.penalty = c->penalty;
            q.fmt = c->fmt;
            WtaUnit& w = Wt[pu];
            w.cost = S.d_cost;
            w.mask = S.d_mask;
            w.prev_label = S.d_prev_label;
            w.i_label = S.d_i_label;
            w.out = J.d_label_out ? J.d_label_out[i] : nullptr;
            w.labels = S.d_labels;
            w.depth = J.d_depth_out ? J.d_depth_out[i] : nullptr;
            w.label_z = c->d_label_z;
            w.status = b->d_job_status + j;
            w.S = S.S;
            w.L = c->L;
            w.W = r.W;
            w.H = r.H;
            w.is_i = is_i;
            w.seg_base = wta_segs;
            wta_segs += S.S;
            ++pu;
        }
        st.prev = cur;
        if (is_i) st.iframe = cur;
        st.frames++;
    }
    // Depth rows flattened over the units that asked for depth maps. Units without one own no rows:
    // they share their base with the next unit, and find_base (largest index whose base is <= row)
    // always resolves a row to the unit that owns it. The temporal row/stat bases of I-frame units
    // and the segment bases of empty units follow the same rule.
    {
        int next = 0;
        for (int u = 0; u < pu; ++u) {
            Wt[u].depth_base = next;
            if (Wt[u].depth) next += Wt[u].H;
        }
        depth_rows = next;
    }
    H.n_pack = pv;
    H.n_units = pu;
    H.fmt = fmt;
    H.combine = combine;
    H.pack_rows = pack_rows;
    H.temp_tiles = temp_tiles;
    H.temp_chunks = temp_chunks;
    H.temp_stats = temp_stats;
    H.wta_segs = wta_segs;
    H.depth_rows = depth_rows;
    if (fmt >= 0 && (fmt != b->fmt || combine != b->combine))
        b->cost_grid = b->n_sm * cost_blocks_per_sm(fmt, combine, b->fast_rcp);
    if (fmt >= 0) {
        b->fmt = fmt;
        b->combine = combine;
        b->penalty_floor = pf_all;
        b->kind = kind;
    }
    b->prepared_units = pu;
    b->prepared_jobs = n_jobs;
    return FTV_OK;
}

static cudaError_t enqueue(ftv_batch* b, cudaStream_t s) {
    const Header* hdr = reinterpret_cast<const Header*>(b->d_desc + b->lay.header);
    const PackTask* pack = reinterpret_cast<const PackTask*>(b->d_desc + b->lay.pack);
    const TempUnit* temp = reinterpret_cast<const TempUnit*>(b->d_desc + b->lay.temp);
    RefJob* jobs = reinterpret_cast<RefJob*>(b->d_desc + b->lay.jobs);
    const WtaUnit* wta = reinterpret_cast<const WtaUnit*>(b->d_desc + b->lay.wta);
    const int g = b->n_sm * 4;
    cudaError_t e = cudaMemcpyAsync(b->d_desc, b->h_stage, b->lay.total, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_job_status, 0, sizeof(uint32_t) * b->max_jobs, s);
    if (e != cudaSuccess) return e;
    pack_multi_kernel<<<g, 256, 0, s>>>(hdr, pack);
    temporal_zero_multi_kernel<<<g, 256, 0, s>>>(hdr, temp);
    temporal_accumulate_multi_kernel<<<b->n_sm * b->temp_per_sm, 256, 0, s>>>(hdr, temp);
    temporal_decide_multi_kernel<<<g, kTChunk, 0, s>>>(hdr, temp);
    temporal_compact_multi_kernel<<<g, kTChunk, 0, s>>>(hdr, temp);
    zero_changed_rows_kernel<<<dim3(64, std::min(b->max_units, 65535)), 256, 0, s>>>(hdr, jobs);
    e = launch_plan_device(jobs, &hdr->n_units, b->d_plan, s);
    if (e != cudaSuccess) return e;
    // The cost items run in `chunks` persistent launches over consecutive item ranges: between two of
    // them the GPU can start other streams' work (of a higher priority first) instead of waiting for the
    // whole batch.
    for (int k = 0; k < b->chunks && e == cudaSuccess; ++k)
        e = launch_cost(jobs, b->d_plan, b->fmt, b->combine, b->fast_rcp, b->penalty_floor, b->kind, k, b->chunks,
                        b->cost_grid, s);
    if (e != cudaSuccess) return e;
    wta_multi_kernel<<<g, 256, 0, s>>>(hdr, wta);
    depth_multi_kernel<<<g, 256, 0, s>>>(hdr, wta);
    b->launches += 9 + b->chunks;
    e = cudaGetLastError();
    // every job's status word back to pinned host memory, read by ftv_batch_wait / ftv_batch_poll once the
    // launch's completion event has fired
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->h_job_status, b->d_job_status, sizeof(uint32_t) * b->max_jobs, cudaMemcpyDeviceToHost, s);
    return e;
}

ftv_status ftv_batch_launch(ftv_batch* b, ftv_stream stream) {
    if (!b || b->fmt < 0) return FTV_ERR_STATE;
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != b->device) cudaSetDevice(b->device);
    NvtxRange range("ftv_batch_launch");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = enqueue(b, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->done, s);
    if (e == cudaSuccess) b->launched_jobs = b->prepared_jobs;
    if (prev_dev >= 0 && prev_dev != b->device) cudaSetDevice(prev_dev);
    return e == cudaSuccess ? FTV_OK : FTV_ERR_CUDA;
}

ftv_status ftv_batch_replay(ftv_batch* b, ftv_stream stream) {
    if (!b || b->fmt < 0) return FTV_ERR_STATE;
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != b->device) cudaSetDevice(b->device);
    NvtxRange range("ftv_batch_replay");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!b->exec || b->graph_fmt != b->fmt || b->graph_combine != b->combine || b->graph_pf != b->penalty_floor ||
        b->graph_kind != b->kind || b->graph_chunks != b->chunks) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        cudaStream_t cap;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t e1 = enqueue(b, cap);
                b->launches -= 9 + b->chunks;
                e = cudaStreamEndCapture(cap, &b->graph);
                if (e1 != cudaSuccess) e = e1;
            }
            cudaStreamDestroy(cap);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e == cudaSuccess) {
            b->graph_fmt = b->fmt;
            b->graph_combine = b->combine;
            b->graph_pf = b->penalty_floor;
            b->graph_kind = b->kind;
            b->graph_chunks = b->chunks;
        }
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
    if (e == cudaSuccess) {
        b->launches += 9 + b->chunks;
        e = cudaEventRecord(b->done, s);
    }
    if (e == cudaSuccess) b->launched_jobs = b->prepared_jobs;
    if (prev_dev >= 0 && prev_dev != b->device) cudaSetDevice(prev_dev);
    return e == cudaSuccess ? FTV_OK : FTV_ERR_CUDA;
}

static_assert(FTV_MAX_BATCH_CHUNKS == kMaxChunks, "chunk limit of the ABI and of the plan");

ftv_status ftv_batch_set_chunks(ftv_batch* b, int32_t chunks) {
    if (!b || chunks < 1 || chunks > FTV_MAX_BATCH_CHUNKS) return FTV_ERR_INVALID_ARG;
    b->chunks = chunks;  // the next replay captures a new graph
    return FTV_OK;
}

ftv_status ftv_batch_query(ftv_batch* b) {
    if (!b) return FTV_ERR_INVALID_ARG;
    const cudaError_t e = cudaEventQuery(b->done);
    if (e == cudaErrorNotReady) return FTV_ERR_BUSY;
    return e == cudaSuccess ? FTV_OK : FTV_ERR_CUDA;
}

ftv_status ftv_batch_wait(ftv_batch* b) {
    if (!b) return FTV_ERR_INVALID_ARG;
    if (cudaEventSynchronize(b->done) != cudaSuccess) return FTV_ERR_CUDA;
    uint32_t st = checked_bits(b);
    for (int j = 0; j < b->launched_jobs; ++j) st |= b->h_job_status[j];
    return status_of(st);
}

int64_t ftv_batch_launch_count(const ftv_batch* b) { return b ? b->launches : 0; }

ftv_status ftv_job_footprint(const ftv_config* cfg, int32_t n_segments_max, int64_t* bytes) {
    if (!cfg || !bytes || n_segments_max < 0) return FTV_ERR_INVALID_ARG;
    if (cfg->n_views < 1 || cfg->n_views > FTV_MAX_VIEWS || !cfg->cams) return FTV_ERR_INVALID_ARG;
    if (cfg->n_refs < 1 || cfg->n_refs > cfg->n_views || !cfg->ref_views) return FTV_ERR_INVALID_ARG;
    if (cfg->n_labels < 1 || cfg->n_labels > FTV_MAX_LABELS || cfg->max_segments < 1) return FTV_ERR_INVALID_ARG;
    if (cfg->sample_bytes != 1 && cfg->sample_bytes != 2) return FTV_ERR_INVALID_ARG;
    if (cfg->bit_depth < 1 || cfg->bit_depth > 8 * cfg->sample_bytes) return FTV_ERR_INVALID_ARG;
    const size_t tb = (cfg->sample_bytes == 1 || cfg->bit_depth <= 10) ? 4 : 8;
    size_t packed = 0;
    int64_t input = 0;
    for (int v = 0; v < cfg->n_views; ++v) {
        const int64_t w = cfg->cams[v].width, h = cfg->cams[v].height;
        if (w < 1 || h < 1 || w > FTV_MAX_DIM || h > FTV_MAX_DIM) return FTV_ERR_INVALID_ARG;
        packed += align256((size_t)(w * h) * tb);
        input += 3 * w * h * cfg->sample_bytes;
    }
    const int64_t S = n_segments_max > 0 ? n_segments_max : cfg->max_segments;
    std::vector<RefDims> refs;
    for (int i = 0; i < cfg->n_refs; ++i) {
        const int r = cfg->ref_views[i];
        if (r < 0 || r >= cfg->n_views) return FTV_ERR_INVALID_ARG;
        int64_t N = cfg->n_views - 1;
        if (cfg->nbr_offsets) {
            N = cfg->nbr_offsets[i + 1] - cfg->nbr_offsets[i];
            if (N < 0 || N > FTV_MAX_NBRS) return FTV_ERR_INVALID_ARG;
        }
        refs.push_back({cfg->cams[r].width, cfg->cams[r].height, N, S});
    }
    *bytes = context_bytes_of(packed, refs, cfg->n_labels, cfg->max_segments, cfg->precision == FTV_PRECISION_FP64) +
             stream_bytes_of(packed, refs, cfg->n_labels) + input;
    return FTV_OK;
}

ftv_status ftv_batch_set_budget(ftv_batch* b, int64_t hbm_budget_bytes) {
    if (!b || hbm_budget_bytes < 0) return FTV_ERR_INVALID_ARG;
    b->budget = hbm_budget_bytes;
    return FTV_OK;
}


ftv_status ftv_batch_submit(ftv_batch* b, const ftv_frame_job* job, uint64_t* ticket) {
    if (!b || !job || !ticket) return FTV_ERR_INVALID_ARG;
    ftv_ctx* c = job->ctx;
    if (!c || !c->stream.ready || !job->d_planes || !job->pitch_bytes) return FTV_ERR_INVALID_ARG;
    const int64_t footprint_bytes = job_bytes(c);
    if (job->frame_type != FTV_FRAME_I && job->frame_type != FTV_FRAME_P) return FTV_ERR_INVALID_ARG;
    if (c->device != b->device) return FTV_ERR_INVALID_ARG;
    for (int v = 0; v < c->n_views; ++v)
        for (int k = 0; k < 3; ++k) {
            if (!job->d_planes[3 * v + k]) return FTV_ERR_INVALID_ARG;
            if (job->pitch_bytes[3 * v + k] < (int64_t)c->cams[v].width * c->sample_bytes) return FTV_ERR_INVALID_ARG;
        }
    if (b->budget > 0 && footprint_bytes > b->budget) return FTV_ERR_OUT_OF_MEMORY;  // can never be admitted
    // capacity, one frame per stream per launch, one precision, sample format and combination per launch
    int units = c->n_refs, views = c->n_views;
    int64_t queued = footprint_bytes;
    bool stream_has_i = c->stream.prev >= 0;
    for (const QueuedJob& q : b->queue) {
        if (q.ctx == c) return FTV_ERR_BUSY;
        if (q.ctx->precision != c->precision || q.ctx->fmt != c->fmt || q.ctx->combine != c->combine)
            return FTV_ERR_BUSY;
        units += q.ctx->n_refs;
        views += q.ctx->n_views;
        queued += q.footprint;
    }
    if (job->frame_type == FTV_FRAME_P && !stream_has_i) return FTV_ERR_STATE;
    if ((int)b->queue.size() >= b->max_jobs || units > b->max_units || views > b->max_views) return FTV_ERR_BUSY;
    harvest(b);
    if (b->budget > 0 && queued + b->launch_footprint > b->budget) return FTV_ERR_BUSY;  // admission by footprint
    QueuedJob q;
    q.ctx = c;
    q.frame_type = job->frame_type;
    q.planes.assign(job->d_planes, job->d_planes + 3 * c->n_views);
    q.pitch.assign(job->pitch_bytes, job->pitch_bytes + 3 * c->n_views);
    q.has_label_out = job->d_label_out != nullptr;
    q.has_depth_out = job->d_depth_out != nullptr;
    if (q.has_label_out) q.label_out.assign(job->d_label_out, job->d_label_out + c->n_refs);
    if (q.has_depth_out) q.depth_out.assign(job->d_depth_out, job->d_depth_out + c->n_refs);
    q.footprint = footprint_bytes;
    b->queue.push_back(std::move(q));
    *ticket = b->next_ticket++;
    return FTV_OK;
}

ftv_status ftv_batch_flush(ftv_batch* b, ftv_stream stream) {
    if (!b) return FTV_ERR_INVALID_ARG;
    NvtxRange range("ftv_batch_flush");
    if (b->queue.empty()) return FTV_OK;
    if (!harvest(b)) return FTV_ERR_BUSY;  // the previous launch still reads the staging block
    const int n = (int)b->queue.size();
    std::vector<ftv_frame_job> jobs(n);
    int64_t footprint = 0;
    for (int j = 0; j < n; ++j) {
        QueuedJob& q = b->queue[j];
        jobs[j].ctx = q.ctx;
        jobs[j].d_planes = q.planes.data();
        jobs[j].pitch_bytes = q.pitch.data();
        jobs[j].frame_type = q.frame_type;
        jobs[j].d_label_out = q.has_label_out ? q.label_out.data() : nullptr;
        jobs[j].d_depth_out = q.has_depth_out ? q.depth_out.data() : nullptr;
        footprint += q.footprint;
    }
    const uint64_t first = b->next_ticket - (uint64_t)n;
    ftv_status st = ftv_batch_prepare(b, jobs.data(), n);
    if (st == FTV_OK) st = ftv_batch_replay(b, stream);
    b->queue.clear();
    if (st != FTV_OK) {
        for (int k = 0; k < n; ++k) b->ring[(first + k) % kTicketRing] = (int8_t)st;
        return st;
    }
    b->launch_first = first;
    b->launch_n = n;
    b->harvested = false;
    b->launch_footprint = footprint;
    return FTV_OK;
}

ftv_status ftv_batch_poll(ftv_batch* b, uint64_t ticket, ftv_status* job_status) {
    if (!b || !job_status || ticket == 0 || ticket >= b->next_ticket) return FTV_ERR_INVALID_ARG;
    if (ticket + kTicketRing < b->next_ticket) return FTV_ERR_INVALID_ARG;  // no longer kept
    if (ticket > b->next_ticket - 1 - b->queue.size()) return FTV_ERR_BUSY;  // submitted, not yet flushed
    if (ticket >= b->launch_first && ticket < b->launch_first + (uint64_t)b->launch_n && !harvest(b))
        return FTV_ERR_BUSY;
    *job_status = (ftv_status)b->ring[ticket % kTicketRing];
    return FTV_OK;
}

}  // extern "C"
