// Temporal consistency test for callers that cannot allocate device memory.
//
// ftv_temporal_mask needs an ftv_ctx, and creating one calls cudaMalloc. Some callers cannot do that:
// a process whose device memory is reserved in full at start-up (a fixed budget shared with other
// engines), or a latency-critical loop where cudaMalloc's implicit device-wide synchronisation would
// stall every other stream. ftv_temporal_mask_static runs the same kernels with its per-segment
// accumulators in a fixed, statically sized device array instead, and calls no allocator.
#include <cuda_runtime.h>

#include "ftv_internal.h"

namespace {

constexpr int kStatWords = 8;     // int64 accumulators per segment (eight planes of FTV_STATIC_MAX_SEGMENTS)
constexpr int kSpareWords = 32;   // tail of the array: the status word when the caller passes none

// Accumulators of ftv_temporal_mask_static: FTV_STATIC_MAX_SEGMENTS x 8 int64 (4 MiB for 65536
// segments) plus a spare tail. Every GPU that loads this library holds it until the process exits.
static __device__ __align__(256) int64_t g_tm_scratch[FTV_STATIC_MAX_SEGMENTS * kStatWords + kSpareWords];

// Device address of g_tm_scratch on the current device. In host code the symbol's name is only a
// host-side stand-in, so the address is looked up with the device current. The lookup runs on every call:
// it allocates nothing, and no address is kept that a device reset could leave stale.
ftv_status scratch_for_current_device(int64_t** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tm_scratch) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return FTV_ERR_CUDA;
    }
    *out = static_cast<int64_t*>(p);
    return FTV_OK;
}

// True when p is device memory of device `dev` (or managed memory): the kernels run on the current device
// with the current device's scratch, so an argument on another device, or in host memory, is refused
// before anything is launched.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" ftv_status ftv_temporal_mask_static(int32_t width, int32_t height, int32_t sample_bytes,
                                               const void* const* d_cur, const int64_t* cur_pitch,
                                               const void* const* d_prev, const int64_t* prev_pitch,
                                               const void* const* d_iframe, const int64_t* iframe_pitch,
                                               const int32_t* d_labels, int32_t n_segments, int32_t t_p, int32_t t_i,
                                               int32_t mode, uint8_t* d_mask, int32_t* d_changed_list,
                                               int32_t* d_n_changed, uint32_t* d_status, ftv_stream stream) {
    if (width < 1 || height < 1 || width > FTV_MAX_DIM || height > FTV_MAX_DIM) return FTV_ERR_INVALID_ARG;
    if (sample_bytes != 1 && sample_bytes != 2) return FTV_ERR_INVALID_ARG;
    if (!d_cur || !cur_pitch || !d_prev || !prev_pitch || !d_labels || !d_mask || !d_changed_list || !d_n_changed)
        return FTV_ERR_INVALID_ARG;
    if (n_segments < 0 || n_segments > FTV_STATIC_MAX_SEGMENTS) return FTV_ERR_INVALID_ARG;
    if (t_p < 0 || t_i < 0) return FTV_ERR_INVALID_ARG;
    if (mode != FTV_TM_Y_ONLY && mode != FTV_TM_ALL_YUV) return FTV_ERR_INVALID_ARG;
    if (d_iframe && !iframe_pitch) return FTV_ERR_INVALID_ARG;
    const int nch = mode == FTV_TM_ALL_YUV ? 3 : 1;
    const int64_t row = (int64_t)width * sample_bytes;
    for (int c = 0; c < nch; ++c) {
        if (!d_cur[c] || !d_prev[c] || cur_pitch[c] < row || prev_pitch[c] < row) return FTV_ERR_INVALID_ARG;
        if (d_iframe && (!d_iframe[c] || iframe_pitch[c] < row)) return FTV_ERR_INVALID_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FTV_ERR_CUDA;
    if (!on_device(d_labels, dev) || !on_device(d_mask, dev) || !on_device(d_changed_list, dev) ||
        !on_device(d_n_changed, dev) || (d_status && !on_device(d_status, dev)))
        return FTV_ERR_INVALID_ARG;
    for (int c = 0; c < nch; ++c)
        if (!on_device(d_cur[c], dev) || !on_device(d_prev[c], dev) || (d_iframe && !on_device(d_iframe[c], dev)))
            return FTV_ERR_INVALID_ARG;
    int64_t* scratch = nullptr;
    const ftv_status st = scratch_for_current_device(&scratch);
    if (st != FTV_OK) return st;
    uint32_t* status = d_status ? d_status
                                : reinterpret_cast<uint32_t*>(scratch + (size_t)FTV_STATIC_MAX_SEGMENTS * kStatWords);
    int64_t launches = 0;
    // the accumulators are cleared on `stream` before use, so the previous call's contents do not matter
    const cudaError_t e = ftv::launch_temporal(d_cur, cur_pitch, d_prev, prev_pitch, d_iframe, iframe_pitch,
                                               sample_bytes, d_labels, width, height, n_segments, t_p, t_i, mode,
                                               scratch, FTV_STATIC_MAX_SEGMENTS, d_mask, d_changed_list,
                                               d_n_changed, status, true,
                                               (cudaStream_t)stream, &launches);
    return e == cudaSuccess ? FTV_OK : FTV_ERR_CUDA;
}
