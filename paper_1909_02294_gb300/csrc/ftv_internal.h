// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ftv.h"

namespace ftv {

// A host-side NVTX range over one stage of an entry point ("ftv_cost_volume", "cost kernel", ...): a profiler
// that records NVTX ranges (Nsight Systems) shows the pipeline's stages and their launches; with no profiler
// attached the calls return at once.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Packed texel formats: one load fetches the three samples of a pixel.
enum TexelFormat : int32_t {
    FMT_U8X4 = 0,   // uint32: Y | Cb << 8 | Cr << 16          (8-bit samples)
    FMT_P10 = 1,    // uint32: Y | Cb << 10 | Cr << 20         (16-bit samples of at most 10 bits)
    FMT_U16X4 = 2,  // uint2 : (Y | Cb << 16, Cr)              (16-bit samples of 11 to 16 bits)
};

// Device status bits (OR-ed by kernels, read and cleared by ftv_check).
// ST_CHECKED: a checked build (FTV_CHECKED) found a gather index outside its view and skipped it.
enum StatusBits : uint32_t { ST_BAD_LABEL = 1u, ST_BAD_SAMPLE = 2u, ST_OVERFLOW = 4u, ST_CHECKED = 8u };

// Cost-kernel tiling: each work item is one tile of kTile consecutive segment pixels (in listed-segment
// order) times one block of consecutive labels. kThreads threads own kPPT pixels each.
#ifndef FTV_THREADS
#define FTV_THREADS 256
#endif
#ifndef FTV_PPT
#define FTV_PPT 4
#endif
#ifndef FTV_MINB
#define FTV_MINB 4
#endif
constexpr int kThreads = FTV_THREADS;
constexpr int kPPT = FTV_PPT;
constexpr int kMinBlocks = FTV_MINB;  // resident CTAs per SM the register budget is sized for
constexpr int kTile = kThreads * kPPT;
constexpr int kMaxLB = 64;          // labels per block
constexpr int kHEntries = 512;      // shared-memory capacity for N x LB staged homographies
constexpr int kSegAcc = 16;         // per-tile segment accumulators in shared memory (more: global atomics)

// Geometry of a neighbour view as the cost kernel sees it.
struct NbrView {
    const void* texels;  // packed view, row pitch `pitch` texels
    int32_t w, h, pitch, pad;
};

// One (job, reference) unit of the persistent cost kernel. Plan fields are written on the device.
struct RefJob {
    const void* ref_texels;    // packed reference view (row pitch = W texels)
    const uint32_t* pix;       // segment index records: (y << 16) | x, grouped by segment
    const int32_t* offs;       // segment index offsets [S + 1]
    const int32_t* list;       // listed segments or nullptr (all)
    const int32_t* n_listed;   // device length of `list` (nullptr with list == nullptr)
    int32_t* woffs;            // scratch [S + 1]: prefix of listed segment sizes (written by plan)
    const float* H;            // [N][L][9]
    const double* H64;         // [N][L][9] unrounded table (FP64-precision units; else nullptr)
    const NbrView* nbrs;       // [N]
    int32_t* cost;             // [S][L]
    int32_t W, S, N, L, LB, nLB, penalty, fmt;
    int32_t Href;              // reference height
    // plan outputs
    int32_t n_work;            // listed segments
    int32_t n_rec;             // listed pixels
    int32_t n_items;           // tiles * nLB
    int32_t item_base;         // first item of this unit in the launch
};

constexpr int kMaxChunks = 16;  // a launch's items may be split over this many cost-kernel launches
struct Plan {
    int32_t total_items;
    int32_t n_jobs;            // units in the launch
    unsigned long long culled; // evaluations decided without sampling: the tile is out of that view
    unsigned long long recomputed;  // FP64-precision evaluations computed in double precision
    uint32_t checked;          // checked builds: ST_CHECKED when a gather index fell outside its view
    int32_t counter[kMaxChunks];  // next item of each chunk, relative to the chunk's first (persistent CTAs)
};

struct RefState {
    int32_t view;              // camera index
    int32_t W, H;
    int32_t n_nbrs;
    std::vector<int32_t> nbrs;
    float* d_H = nullptr;      // [N][L][9]
    double* d_H64 = nullptr;   // [N][L][9] unrounded table (FP64-precision contexts only)
    NbrView* d_nbrs = nullptr; // [N]
    int32_t* d_offs = nullptr;   // [max_segments + 1]
    int32_t* d_cursor = nullptr; // [max_segments]
    int32_t* d_woffs = nullptr;  // [max_segments + 1]
    uint32_t* d_pix = nullptr;   // [W * H]
    int32_t S_indexed = -1;      // segment count of the cached index (-1: none)
    int2* d_centre = nullptr;    // [max_segments] segment centres (centre table)
    const int32_t** d_nbr_labels = nullptr;  // [N] neighbour label maps (centre table)
    std::vector<float> h_H;      // host copy of the table
    std::vector<double> h_H64;   // the table before its rounding to FP32
};

// Resident per-stream state of one reference view (ftv_stream_init).
struct StreamRef {
    uint16_t* d_prev_label = nullptr;  // [S] labels of the previous frame (updated in place)
    uint16_t* d_i_label = nullptr;     // [S] labels of the last I frame
    uint8_t* d_mask = nullptr;         // [S]
    int32_t* d_changed = nullptr;      // [S]
    int32_t* d_n_changed = nullptr;    // [1]
    int64_t* d_stats = nullptr;        // [S][8]
    int32_t* d_cost = nullptr;         // [S][L] cost scratch
    int32_t* d_labels = nullptr;       // [H][W] copy of the reference label map
    NbrView* d_nbrs_ring[3] = {nullptr, nullptr, nullptr};  // neighbour geometry into ring buffer b
    int32_t S = 0;
};

// Resident per-stream state: a ring of three packed frames (current, previous P, I) and per-reference
// label states, so that consecutive frames of one camera stream can skip unchanged segments.
struct StreamState {
    bool ready = false;
    uint32_t* d_status = nullptr;  // errors found building the resident state (reported by every job)
    int32_t t_p = 0, t_i = 0, mode = 0;
    void* d_ring[3] = {nullptr, nullptr, nullptr};
    int32_t prev = -1, iframe = -1;
    int64_t frames = 0;
    std::vector<StreamRef> refs;
};

}  // namespace ftv

struct ftv_ctx {
    int device = 0;
    int n_sm = 0;
    int cost_blocks_per_sm = 0;
    int32_t n_views = 0, n_refs = 0, L = 0, plane_mode = 0, centre = 0;
    int32_t sample_bytes = 1, bit_depth = 8, penalty = 0, combine = 0, max_segments = 0, fmt = 0;
    int32_t precision = 0;       // FTV_PRECISION_*
    bool fast_rcp = false;
    bool penalty_floor = false;  // penalty >= 3 (2^bit_depth - 1)
    int kind = 0;                // entry classification for the cost kernel (kKind*)
    int32_t LB = 0, nLB = 0;
    int32_t lb_max = 0;          // largest label block the kernel's stage holds for this context's neighbours
    int32_t ctas_per_sm = 0;     // cost-kernel CTAs per SM (0: the occupancy limit, cost_blocks_per_sm)
    double z_near = 0, z_far = 0;
    std::vector<ftv_camera> cams;
    std::vector<ftv::RefState> refs;
    std::vector<float> label_z;
    // device scratch
    void* d_packed = nullptr;                 // all views, packed texels
    std::vector<size_t> view_offset_bytes;    // byte offset of each packed view
    size_t texel_bytes = 4;
    uint32_t* d_status = nullptr;
    ftv::RefJob* d_jobs = nullptr;            // [n_refs]
    ftv::Plan* d_plan = nullptr;
    int64_t* d_tstats = nullptr;              // per reference: temporal sums, 8 planes of max_segments (adjacency scratch)
    std::vector<uint8_t> tstats_zero;         // per reference: its d_tstats slot holds zero sums
    float* d_label_z = nullptr;               // [L]
    int32_t* d_adj_deg = nullptr;             // [max_segments] adjacency: neighbours t > s per segment
    int32_t* d_adj_slots = nullptr;           // [max_segments][32]
    int32_t* d_adj_offs = nullptr;            // [max_segments]
    int64_t launches = 0;
    bool profiling = false;
    bool timed = false;
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
    ftv::StreamState stream;
};

namespace ftv {

// Stream state (ftv_batch.cu)
void free_stream_state(ftv_ctx* c);

// Host geometry (ftv_geometry.cpp)
bool label_inv_depths(int L, double z_near, double z_far, std::vector<double>& iz);
int plane_homography(const ftv_camera& cr, const ftv_camera& cv, const ftv_camera* cc, double iz, double H[9]);

// Launchers (ftv_index.cu)
cudaError_t launch_pack(const void* const* planes, const int64_t* pitch, int sample_bytes, int bit_depth, int fmt,
                        int W, int H, void* out, uint32_t* status, cudaStream_t s);
cudaError_t launch_segment_index(const int32_t* labels, int W, int H, int S, int64_t max_pix_cost, int32_t* offs,
                                 int32_t* cursor, uint32_t* pix, uint32_t* status, cudaStream_t s, int64_t* launches);
// Descriptors travel as kernel parameters (graph-capturable, no host staging buffer to race on).
constexpr int kMaxUnits = 240;  // (job, reference) units per launch
cudaError_t launch_plan(const RefJob* host_jobs, int n_jobs, RefJob* d_jobs, Plan* plan, cudaStream_t s);
// Same plan for descriptors already in device memory (completed in place); the unit count is read from
// *n_jobs on the device, so one captured launch serves any batch composition.
cudaError_t launch_plan_device(RefJob* d_jobs, const int32_t* n_jobs, Plan* plan, cudaStream_t s);
cudaError_t launch_zero_rows(int32_t* cost, int L, int S, const int32_t* list, const int32_t* n_listed,
                             cudaStream_t s);

// Cost kernel (ftv_cost.cu)
int cost_blocks_per_sm(int fmt, int combine, bool fast_rcp);
// pf: the penalty is at least the largest possible sample cost (lets the min combination skip
// out-of-view samples; see accumulate() in ftv_cost.cu).
// kind: kKindProjective when no homography entry of the launch is affine (h6 = h7 = 0), else kKindMixed;
// the projective instantiation of the cost kernel has the general path alone. kKindPrecise and
// kKindPreciseMixed: the units take their sample positions from the FP64 projection (FTV_PRECISION_FP64;
// every unit has H64); the mixed one adds the rectified local-frame path, for rigs with affine entries.
enum : int { kKindMixed = 0, kKindProjective = 1, kKindPrecise = 2, kKindPreciseMixed = 3 };
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr bool precise_kind(int kind) { return kind == kKindPrecise || kind == kKindPreciseMixed; }
// chunk, chunks: this launch takes items [total * chunk / chunks, total * (chunk + 1) / chunks) of the plan
// (chunks <= kMaxChunks; a whole launch is chunk 0 of 1).
cudaError_t launch_cost(const RefJob* jobs, const Plan* plan, int fmt, int combine, bool fast_rcp, bool pf, int kind,
                        int chunk, int chunks, int grid, cudaStream_t s);
// Whether the current device's one-step Newton-Raphson reciprocal equals the IEEE round-to-nearest
// reciprocal for every float in [2^-126, 2^126) (exhaustive check, run once per device and cached).
bool fast_reciprocal_exact();
// Run the exhaustive check on the current device; returns the number of mismatching inputs, or -1.
int64_t reciprocal_mismatches();

// Temporal / WTA (ftv_temporal.cu)
// One reference of a temporal-test launch sequence: its current, previous-P and I frames (plane pointers and
// pitches in bytes; ifr unused without an I frame), label map [H][W], per-segment sums and outputs. The sums
// are eight planes of ms int64 words (ms >= S): word q of segment s at stats[q * ms + s], q = 0 the pixel
// count, 1 + c and 4 + c the channel-c sums of cur - prev and cur - I, plane 7 the decide pass's per-block
// counts. Planes 0-6 are zero on entry and left zero on exit.
struct TemporalRef {
    const void* cur[3];
    const void* prev[3];
    const void* ifr[3];
    int64_t pc[3], pp[3], pi[3];
    const int32_t* labels;
    int64_t* stats;
    uint8_t* mask;
    int32_t* changed;
    int32_t* n_changed;
    int32_t W, H, S, ms;
};
constexpr int kMaxTemporalRefs = 16;  // references per launch sequence (they travel as kernel parameters)
// The temporal test of refs[0..n) (n <= kMaxTemporalRefs) in three launches: accumulate, decide, compact.
cudaError_t launch_temporal_refs(const TemporalRef* refs, int n, int sample_bytes, int mode, bool has_i, int t_p,
                                 int t_i, uint32_t* status, cudaStream_t s, int64_t* launches);
cudaError_t launch_temporal(const void* const* cur, const int64_t* cur_pitch, const void* const* prev,
                            const int64_t* prev_pitch, const void* const* ifr, const int64_t* ifr_pitch,
                            int sample_bytes, const int32_t* labels, int W, int H, int S, int t_p, int t_i,
                            int mode, int64_t* stats, int ms, uint8_t* mask, int32_t* changed, int32_t* n_changed,
                            uint32_t* status, bool clear, cudaStream_t s, int64_t* launches);
cudaError_t launch_wta(const int32_t* cost, int S, int L, const uint8_t* mask, const uint16_t* prev_label,
                       const uint16_t* ifr_label, const int32_t* list, const int32_t* n_listed, uint16_t* out,
                       cudaStream_t s);
cudaError_t launch_depth_map(const int32_t* labels, int W, int H, int S, const uint16_t* seg_label,
                             const float* label_z, int L, float* depth, uint32_t* status, cudaStream_t s);

}  // namespace ftv
