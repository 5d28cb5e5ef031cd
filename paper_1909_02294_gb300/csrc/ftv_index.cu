// Data preparation kernels: texel packing, the per-reference segment index and the work plan of the
// persistent cost kernel.
//
// Paper: segments are the estimation units (Sec. III-A: "depth is estimated for segments"; Sec. IV-C:
// segments come from any superpixel method, one label map per view). The index groups each
// reference's pixels by segment so that a cost tile reads consecutive pixels of few segments.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ftv_internal.h"

namespace ftv {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------------------------------ packing

template <int SB>
__device__ __forceinline__ uint32_t load_sample(const void* plane, int64_t pitch, int x, int y) {
    const char* row = static_cast<const char*>(plane) + (int64_t)y * pitch;
    if (SB == 1) return reinterpret_cast<const uint8_t*>(row)[x];
    return reinterpret_cast<const uint16_t*>(row)[x];
}

// One thread per pixel of a row; blockIdx.y is the row. Samples above max_value are reported and
// clamped so that they cannot spill into a neighbouring packed field.
template <int SB, int FMT>
__global__ void pack_kernel(const void* Yp, const void* Up, const void* Vp, int64_t pY, int64_t pU, int64_t pV,
                            int W, uint32_t max_value, void* out, uint32_t* status) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    uint32_t a = load_sample<SB>(Yp, pY, x, y);
    uint32_t b = load_sample<SB>(Up, pU, x, y);
    uint32_t c = load_sample<SB>(Vp, pV, x, y);
    if (a > max_value || b > max_value || c > max_value) {
        atomicOr(status, ST_BAD_SAMPLE);
        a = min(a, max_value);
        b = min(b, max_value);
        c = min(c, max_value);
    }
    const int64_t i = (int64_t)y * W + x;
    if (FMT == FMT_U8X4) {
        static_cast<uint32_t*>(out)[i] = a | (b << 8) | (c << 16);
    } else if (FMT == FMT_P10) {
        static_cast<uint32_t*>(out)[i] = a | (b << 10) | (c << 20);
    } else {
        static_cast<uint2*>(out)[i] = make_uint2(a | (b << 16), c);
    }
}

// ------------------------------------------------------------------------------------ segment index

// Per-segment pixel counts. Lanes of a warp that hold the same label (a run along the row) add their
// count with one atomic.
__global__ void histogram_kernel(const int32_t* __restrict__ labels, int W, int S, int32_t* counts,
                                 uint32_t* status) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const bool in = x < W;
    const int l = in ? labels[(int64_t)y * W + x] : -1;
    const bool ok = in && (unsigned)l < (unsigned)S;
    if (in && !ok) atomicOr(status, ST_BAD_LABEL);
    const unsigned active = __ballot_sync(kFull, ok);
    if (ok) {
        const unsigned peers = __match_any_sync(active, l);
        const int lane = threadIdx.x & 31;
        if (lane == __ffs(peers) - 1) atomicAdd(&counts[l], __popc(peers));
    }
}

// Block-wide exclusive scan of one int per thread (blockDim.x == 1024). Returns the exclusive prefix;
// *total receives the block sum.
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
        warp_sums[lane] = s;  // inclusive prefix of warp sums
    }
    __syncthreads();
    const int base = warp > 0 ? warp_sums[warp - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + incl - v;
}

// Counts (in `cursor`) -> offsets[S + 1]; cursor[s] = offsets[s] for the scatter. One block of 1024.
// Also checks that no segment is large enough for its int32 cost sum to overflow.
__global__ void offsets_kernel(int S, int64_t max_pix_cost, int32_t* offs, int32_t* cursor, uint32_t* status) {
    const int per = (S + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(S, b + per);
    int sum = 0, mx = 0;
    for (int s = b; s < e; ++s) {
        const int c = cursor[s];
        sum += c;
        mx = max(mx, c);
    }
    int total;
    int run = block_exclusive_scan(sum, &total);
    for (int s = b; s < e; ++s) {
        const int c = cursor[s];
        offs[s] = run;
        cursor[s] = run;
        run += c;
    }
    if (threadIdx.x == 0) offs[S] = total;
    mx = __reduce_max_sync(kFull, mx);
    if ((threadIdx.x & 31) == 0 && (int64_t)mx * max_pix_cost > (int64_t)INT32_MAX) atomicOr(status, ST_OVERFLOW);
}

// Scatter (y << 16 | x) records into their segment's range. A warp's run of equal labels takes one
// atomic and keeps its left-to-right order.
__global__ void scatter_kernel(const int32_t* __restrict__ labels, int W, int S, int32_t* cursor,
                               uint32_t* __restrict__ pix) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const bool in = x < W;
    const int l = in ? labels[(int64_t)y * W + x] : -1;
    const bool ok = in && (unsigned)l < (unsigned)S;
    const unsigned active = __ballot_sync(kFull, ok);
    if (ok) {
        const unsigned peers = __match_any_sync(active, l);
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&cursor[l], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        pix[base + rank] = ((uint32_t)y << 16) | (uint32_t)x;
    }
}

// ---------------------------------------------------------------------------------------------- plan

template <int CAP>
struct PlanArgs {
    RefJob jobs[CAP];
};

// Completes the plan fields of one (job, reference) unit: the listed pixel prefix (woffs), the number
// of work items (tiles x label blocks) and the unit's first item. Called by all threads of one block
// of 1024 with the same unit; *base is the running item count in shared memory.
__device__ void plan_unit(const RefJob& J, RefJob* out, int* base) {
    int n_work = J.S;
    if (J.list != nullptr) n_work = min(max(*J.n_listed, 0), J.S);
    int n_rec;
    if (J.list == nullptr) {
        n_rec = J.offs[J.S];
    } else {
        const int per = (n_work + blockDim.x - 1) / blockDim.x;
        const int b = threadIdx.x * per, e = min(n_work, b + per);
        int sum = 0;
        for (int i = b; i < e; ++i) {
            const int s = J.list[i];
            if ((unsigned)s < (unsigned)J.S) sum += J.offs[s + 1] - J.offs[s];
        }
        int total;
        int run = block_exclusive_scan(sum, &total);
        for (int i = b; i < e; ++i) {
            J.woffs[i] = run;
            const int s = J.list[i];
            if ((unsigned)s < (unsigned)J.S) run += J.offs[s + 1] - J.offs[s];
        }
        if (threadIdx.x == 0) J.woffs[n_work] = total;
        n_rec = total;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int tiles = (n_rec + kTile - 1) / kTile;
        RefJob o = J;
        if (o.list == nullptr) o.woffs = const_cast<int32_t*>(o.offs);
        o.n_work = n_work;
        o.n_rec = n_rec;
        o.n_items = tiles * o.nLB;
        o.item_base = *base;
        *out = o;
        *base += o.n_items;
    }
    __syncthreads();
}

// One block of 1024 threads; descriptors arrive as kernel parameters and are written, completed, to `out`.
template <int CAP>
__global__ void plan_kernel(const __grid_constant__ PlanArgs<CAP> args, int n_jobs, RefJob* out, Plan* plan) {
    __shared__ int s_base;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int j = 0; j < n_jobs; ++j) plan_unit(args.jobs[j], &out[j], &s_base);
    if (threadIdx.x == 0) {
        plan->total_items = s_base;
        for (int k = 0; k < kMaxChunks; ++k) plan->counter[k] = 0;
        plan->n_jobs = n_jobs;
        plan->culled = 0;
        plan->recomputed = 0;
        plan->checked = 0;
    }
}

// One block of 1024 threads; descriptors already in device memory are completed in place.
__global__ void plan_device_kernel(RefJob* jobs, const int32_t* n_jobs_ptr, Plan* plan) {
    __shared__ int s_base;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    const int n_jobs = *n_jobs_ptr;
    for (int j = 0; j < n_jobs; ++j) {
        const RefJob J = jobs[j];
        __syncthreads();
        plan_unit(J, &jobs[j], &s_base);
    }
    if (threadIdx.x == 0) {
        plan->total_items = s_base;
        for (int k = 0; k < kMaxChunks; ++k) plan->counter[k] = 0;
        plan->n_jobs = n_jobs;
        plan->culled = 0;
        plan->recomputed = 0;
        plan->checked = 0;
    }
}

// Zero the cost rows of listed segments (grid-stride over list entries x labels).
__global__ void zero_rows_kernel(int32_t* cost, int L, int S, const int32_t* list, const int32_t* n_listed) {
    const int n = min(max(*n_listed, 0), S);
    const int64_t total = (int64_t)n * L;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / L), d = (int)(i - (int64_t)k * L);
        const int s = list[k];
        if ((unsigned)s < (unsigned)S) cost[(int64_t)s * L + d] = 0;
    }
}

}  // namespace

cudaError_t launch_pack(const void* const* planes, const int64_t* pitch, int sample_bytes, int bit_depth, int fmt,
                        int W, int H, void* out, uint32_t* status, cudaStream_t s) {
    if (W <= 0 || H <= 0) return cudaSuccess;
    const dim3 block(256), grid((W + 255) / 256, H);
    const uint32_t maxv = (bit_depth >= 32) ? 0xffffffffu : ((1u << bit_depth) - 1u);
    if (sample_bytes == 1) {
        pack_kernel<1, FMT_U8X4><<<grid, block, 0, s>>>(planes[0], planes[1], planes[2], pitch[0], pitch[1],
                                                       pitch[2], W, maxv, out, status);
    } else if (fmt == FMT_P10) {
        pack_kernel<2, FMT_P10><<<grid, block, 0, s>>>(planes[0], planes[1], planes[2], pitch[0], pitch[1],
                                                      pitch[2], W, maxv, out, status);
    } else {
        pack_kernel<2, FMT_U16X4><<<grid, block, 0, s>>>(planes[0], planes[1], planes[2], pitch[0], pitch[1],
                                                        pitch[2], W, maxv, out, status);
    }
    return cudaGetLastError();
}

cudaError_t launch_segment_index(const int32_t* labels, int W, int H, int S, int64_t max_pix_cost, int32_t* offs,
                                 int32_t* cursor, uint32_t* pix, uint32_t* status, cudaStream_t s, int64_t* launches) {
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)(S > 0 ? S : 1), s);
    if (e != cudaSuccess) return e;
    const dim3 block(256), grid((W + 255) / 256, H);
    histogram_kernel<<<grid, block, 0, s>>>(labels, W, S, cursor, status);
    offsets_kernel<<<1, 1024, 0, s>>>(S, max_pix_cost, offs, cursor, status);
    scatter_kernel<<<grid, block, 0, s>>>(labels, W, S, cursor, pix);
    *launches += 3;
    return cudaGetLastError();
}

template <int CAP>
static cudaError_t launch_plan_cap(const RefJob* host_jobs, int n_jobs, RefJob* d_jobs, Plan* plan, cudaStream_t s) {
    static_assert(sizeof(PlanArgs<CAP>) + 32 <= 32764, "kernel parameter space");
    PlanArgs<CAP> args;
    for (int j = 0; j < n_jobs; ++j) args.jobs[j] = host_jobs[j];
    plan_kernel<CAP><<<1, 1024, 0, s>>>(args, n_jobs, d_jobs, plan);
    return cudaGetLastError();
}

cudaError_t launch_plan_device(RefJob* d_jobs, const int32_t* n_jobs, Plan* plan, cudaStream_t s) {
    plan_device_kernel<<<1, 1024, 0, s>>>(d_jobs, n_jobs, plan);
    return cudaGetLastError();
}

cudaError_t launch_plan(const RefJob* host_jobs, int n_jobs, RefJob* d_jobs, Plan* plan, cudaStream_t s) {
    if (n_jobs < 0 || n_jobs > kMaxUnits) return cudaErrorInvalidValue;
    if (n_jobs <= 16) return launch_plan_cap<16>(host_jobs, n_jobs, d_jobs, plan, s);
    return launch_plan_cap<kMaxUnits>(host_jobs, n_jobs, d_jobs, plan, s);
}

cudaError_t launch_zero_rows(int32_t* cost, int L, int S, const int32_t* list, const int32_t* n_listed,
                             cudaStream_t s) {
    const int64_t total = (int64_t)S * L;
    const int blocks = (int)std::min<int64_t>(4096, (total + 255) / 256 + 1);
    zero_rows_kernel<<<blocks, 256, 0, s>>>(cost, L, S, list, n_listed);
    return cudaGetLastError();
}

}  // namespace ftv
