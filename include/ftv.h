/*
 * ftv.h - C ABI of a GB300 (sm_103a) library for the data-parallel hot path of the segment-based
 * multiview depth estimator of Mieloch, Stankiewicz and Domanski, "Depth Map Estimation for
 * Free-Viewpoint Television" (arXiv:1909.02294):
 *   - the segment x depth-label matching-cost volume (Eq. 4 summed over every segment pixel,
 *     combined over the neighbouring views of Eq. 1),
 *   - the per-segment temporal consistency test of Sec. III-E,
 *   - a winner-take-all readout of the volume (a stand-in for the paper's graph cut, Sec. IV-B),
 *   - a batched form that runs many such jobs in one persistent launch,
 *   - the superpixel segmentation that produces the label maps (Sec. IV-C).
 *
 * Conventions shared by every entry point
 *   - Pointers named d_* are CUDA device pointers owned by the caller; host_* / plain pointers are
 *     host memory owned by the caller. The library never frees caller memory. An ftv_ctx owns its
 *     own device scratch (homography table, segment index, packed views) for its lifetime.
 *   - ftv_stream is a cudaStream_t (NULL = the legacy default stream). Entry points that take a
 *     stream only enqueue work on it and return without waiting.
 *   - Argument errors are detected on the host before anything is enqueued and returned at once.
 *     Errors found by kernels (a label outside [0, S), a sample above 2^bit_depth - 1, a segment
 *     sum that could overflow int32) set a status word in the context; ftv_check() waits for the
 *     stream and returns and clears it. Kernels never trap.
 *   - An ftv_ctx may be used from one host thread and one stream at a time.
 *   - Arithmetic contract: the homographies are formed in FP64 on the host and rounded once to FP32;
 *     the projection, reciprocal and rounding on the device are the FP32 round-to-nearest sequence
 *     documented at ftv_cost_volume; all costs are exact integers, so results do not depend on the
 *     order of summation, tiling or batching.
 */
#ifndef FTV_H
#define FTV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FTV_API __attribute__((visibility("default")))
#else
#define FTV_API
#endif

typedef enum ftv_status {
    FTV_OK = 0,
    FTV_ERR_INVALID_ARG = 1,   /* bad argument, or a kernel found an invalid label or sample */
    FTV_ERR_OUT_OF_MEMORY = 2, /* device allocation failed */
    FTV_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    FTV_ERR_OVERFLOW = 4,      /* a segment is large enough that its int32 cost sum could overflow */
    FTV_ERR_TIMEOUT = 5,       /* reserved: a bounded device wait gave up */
    FTV_ERR_BUSY = 6,          /* batch admission refused: over the HBM budget or out of slots */
    FTV_ERR_STATE = 7,         /* call out of order (e.g. no segment index built yet) */
    FTV_ERR_CHECKED = 8        /* checked builds (FTV_CHECKED) only: a cost-kernel gather index fell outside
                                  its view and was skipped; regular builds never report it */
} ftv_status;

typedef void* ftv_stream; /* cudaStream_t */
typedef struct ftv_ctx ftv_ctx;

/* Pinhole camera: X_cam = R * X_world + t; K upper triangular with K[8] == 1 (row-major).
 * Pixel centres sit at integer coordinates. */
typedef struct ftv_camera {
    double K[9];
    double R[9];
    double t[3];
    int32_t width;
    int32_t height;
} ftv_camera;

enum { FTV_PLANES_REF = 0, FTV_PLANES_CENTRE = 1 };
enum { FTV_COMBINE_MIN = 0, FTV_COMBINE_SUM = 1 };
enum { FTV_TM_Y_ONLY = 0, FTV_TM_ALL_YUV = 1 };
enum { FTV_MASK_CHANGED = 0, FTV_MASK_REUSE_P = 1, FTV_MASK_REUSE_I = 2 };
enum { FTV_PRECISION_FP32 = 0, FTV_PRECISION_FP64 = 1 };

#define FTV_MAX_VIEWS 64
#define FTV_MAX_NBRS 32
#define FTV_MAX_LABELS 4096
#define FTV_MAX_DIM 32767

/*
 * Depth-estimation configuration (one rig, one set of candidate depths).
 *   n_views, cams        all cameras of the rig (cams[n_views], host memory, copied at init)
 *   n_refs, ref_views    views for which cost volumes are produced (Sec. III-A: all views at once)
 *   nbr_offsets/views    CSR neighbour lists per reference (nbr_offsets[n_refs+1]); NULL = every other
 *                        view. Sec. III-B's set D (nearest left and right view) is one such list.
 *   n_labels, z_near,    candidate depths uniform in 1/z, label 0 = z_far, label n_labels-1 = z_near
 *   z_far                (Sec. IV-A: depth levels are planes parallel to the camera plane)
 *   plane_mode           FTV_PLANES_REF: planes parallel to each reference camera; FTV_PLANES_CENTRE:
 *                        planes parallel to the centre camera `centre_view` and depth measured from it
 *                        (Sec. III-B, for non-parallel optical axes)
 *   sample_bytes         1 (uint8 samples) or 2 (uint16 samples)
 *   bit_depth            significant bits per sample (<= 8 for 1 byte, <= 16 for 2 bytes)
 *   oob_penalty          cost of a sample that falls outside a view; < 0 selects 3 * (2^bit_depth - 1)
 *   combine              per-pixel combination over neighbours: FTV_COMBINE_MIN or FTV_COMBINE_SUM
 *   max_segments         capacity: largest segment count any reference label map will use
 *   precision            how sample positions are computed (Eq. 4's T[.]; the paper fixes no precision):
 *                        FTV_PRECISION_FP32 (0, the default when the field is zero): the FP32 contract
 *                        of ftv_cost_volume; FTV_PRECISION_FP64: the FP64 projection (same entry),
 *                        which agrees with double-precision geometry wherever the FP32 contract rounds a
 *                        sample near a pixel boundary the other way.
 */
typedef struct ftv_config {
    int32_t n_views;
    const ftv_camera* cams;
    int32_t n_refs;
    const int32_t* ref_views;
    const int32_t* nbr_offsets;
    const int32_t* nbr_views;
    int32_t n_labels;
    double z_near;
    double z_far;
    int32_t plane_mode;
    int32_t centre_view;
    int32_t sample_bytes;
    int32_t bit_depth;
    int32_t oob_penalty;
    int32_t combine;
    int32_t max_segments;
    int32_t precision;
} ftv_config;

/*
 * Create a context: validates the configuration, forms every homography (below), allocates the
 * device scratch and uploads the table. Synchronous. On success *out receives the context.
 *
 * Candidate inverse depths (Sec. IV-A): a = 1/z_far, b = 1/z_near, step = (b - a)/(L - 1),
 * iz_d = a + d * step (FP64). Plane homography of Eq. 4's transform T[.] from reference r into view v
 * for candidate d, in FP64 and in this order:
 *   A = R_v R_r^T;  b = t_v - A t_r;
 *   reference planes: n = (0,0,1), w = iz_d;
 *   centre planes:    n = R_r R_c^T (0,0,1), delta = (1/iz_d - t_c[2]) + n . t_r, w = 1/delta;
 *   M = A + (b n^T) w;  H = K_v (M K_r^-1)  with the closed-form upper-triangular K_r^-1
 *   [[1/fx, -s/(fx fy), (s cy - cx fy)/(fx fy)], [0, 1/fy, -cy/fy], [0, 0, 1]];
 *   every 3-term dot product summed left to right; each entry rounded once to FP32.
 * Errors: FTV_ERR_INVALID_ARG (bad sizes, K not upper triangular, z range, a degenerate centre
 * plane), FTV_ERR_OUT_OF_MEMORY, FTV_ERR_CUDA.
 */
FTV_API ftv_status ftv_depth_init(const ftv_config* cfg, ftv_ctx** out);

/* Host-only: the FP32 homography table that ftv_depth_init would form for reference ref_index of cfg,
 * laid out [n_nbrs][n_labels][9] into host_out (same arithmetic, no device needed). */
FTV_API ftv_status ftv_compute_homographies(const ftv_config* cfg, int32_t ref_index, float* host_out);

/* Host-only: the same table before its rounding to FP32 (FP64 entries, [n_nbrs][n_labels][9]), i.e. the
 * homographies of the FTV_PRECISION_FP64 projection. */
FTV_API ftv_status ftv_compute_homographies_f64(const ftv_config* cfg, int32_t ref_index, double* host_out);

/* Release a context and its device scratch. Waits for the device. NULL is accepted. */
FTV_API ftv_status ftv_depth_destroy(ftv_ctx* ctx);

/* Copy the FP32 homography table of reference ref_index (0 <= ref_index < n_refs) into host_out,
 * laid out [n_nbrs][n_labels][9] row-major, neighbours in list order. */
FTV_API ftv_status ftv_get_homographies(const ftv_ctx* ctx, int32_t ref_index, float* host_out);

/* The same table before its rounding to FP32: FP64 entries [n_nbrs][n_labels][9] into host_out. It is the
 * homography of the FTV_PRECISION_FP64 projection (available in either precision). */
FTV_API ftv_status ftv_get_homographies_f64(const ftv_ctx* ctx, int32_t ref_index, double* host_out);

/* Number of neighbours of reference ref_index, and the views they are, in table order
 * (host_views may be NULL; else it receives n entries). */
FTV_API ftv_status ftv_get_neighbours(const ftv_ctx* ctx, int32_t ref_index, int32_t* n, int32_t* host_views);

/* Candidate depths z_d = 1/iz_d in FP64 rounded to FP32, host_out[n_labels]. */
FTV_API ftv_status ftv_get_label_depths(const ftv_ctx* ctx, float* host_out);

/*
 * Build and cache the segment index of reference ref_index from its label map: d_labels is int32
 * [height][width] of that reference camera (row pitch = width), values in [0, n_segments),
 * n_segments <= max_segments. Segments are the estimation units (Sec. III-A: depth per segment;
 * Sec. IV-C: any superpixel segmentation). A label outside the range sets FTV_ERR_INVALID_ARG in
 * the status word and that pixel is left out. A segment whose pixel count times the largest per-pixel
 * cost exceeds INT32_MAX sets FTV_ERR_OVERFLOW. Asynchronous on `stream`.
 */
FTV_API ftv_status ftv_segment_index(ftv_ctx* ctx, int32_t ref_index, const int32_t* d_labels,
                                     int32_t n_segments, ftv_stream stream);

/*
 * Segment x label matching-cost volumes of every reference (Eq. 4 per pixel, Eq. 1's combination over
 * neighbours, summed over each segment's pixels).
 *
 *   d_planes[3*v + c], pitch_bytes[3*v + c]  (host arrays of n_views*3 entries) sample plane c
 *       (0 = Y, 1 = Cb, 2 = Cr, 4:4:4) of view v, `sample_bytes` per sample, rows pitch_bytes apart.
 *   d_labels[r]   label map of reference r, or NULL to reuse the index cached by ftv_segment_index
 *                 (FTV_ERR_STATE if none); d_labels itself may be NULL (all cached).
 *   n_segments[r] segment count of reference r (ignored when the cached index is used).
 *   d_seg_list[r], d_n_listed[r]  optional device list of segments to evaluate and a device pointer to
 *                 its length (e.g. the changed list of ftv_temporal_mask); NULL = all segments.
 *                 Rows of segments that are not listed are left untouched.
 *   d_cost[r]     int32 [n_segments][n_labels] output of reference r (label-contiguous rows).
 *
 * For each listed segment s and label d: cost[s][d] = sum over pixels (x, y) of s of
 * comb over neighbours v of c_v(x, y, d), comb = min or sum, where with h = H[r][v][d] (FP32):
 *   X = fma(h0, x, fma(h1, y, h2)); Y = fma(h3, x, fma(h4, y, h5)); Wz = fma(h6, x, fma(h7, y, h8));
 *   out of view unless Wz > 0; r = 1/Wz; u = X * r; v = Y * r (all IEEE FP32 round-to-nearest);
 *   (ui, vi) = (floor(u + 0.5), floor(v + 0.5)) must satisfy 0 <= ui <= W_v - 1, 0 <= vi <= H_v - 1;
 *   c_v = |Y_r - Y_v| + |Cb_r - Cb_v| + |Cr_r - Cr_v| at (x, y) and (ui, vi) (integer samples), else the
 *   out-of-view penalty. Eq. 4's 1/size(W) factor is dropped (the sum is an argmin-preserving scale).
 * FTV_PRECISION_FP64 contexts replace the position by the FP64 projection: with h the unrounded FP64
 * homography (ftv_get_homographies_f64) and IEEE double arithmetic, each operation rounded on its own,
 *   X = (h0 * x + h1 * y) + h2; Y = (h3 * x + h4 * y) + h5; Wz = (h6 * x + h7 * y) + h8;
 *   out of view unless Wz > 0; (ui, vi) = (floor(X / Wz + 0.5), floor(Y / Wz + 0.5)), same range test.
 * (The kernel evaluates it in FP32 in a local frame around each tile of pixels, with a rigorous error
 * bound, and redoes in FP64 exactly the evaluations that lie within that bound of a rounding boundary:
 * ftv_fp64_recomputed.)
 * Asynchronous on `stream`.
 */
FTV_API ftv_status ftv_cost_volume(ftv_ctx* ctx, const void* const* d_planes, const int64_t* pitch_bytes,
                                   const int32_t* const* d_labels, const int32_t* n_segments,
                                   const int32_t* const* d_seg_list, const int32_t* const* d_n_listed,
                                   int32_t* const* d_cost, ftv_stream stream);

/*
 * Temporal consistency test of Sec. III-E for reference ref_index with the current label map d_labels
 * ([height][width] int32 of that camera, n_segments segments). d_cur/d_prev/d_iframe are 3-entry host
 * arrays of device plane pointers (Y, Cb, Cr; Cb/Cr may be NULL in FTV_TM_Y_ONLY mode) with
 * pitches in bytes; d_iframe may be NULL (no I-frame test). For each segment with n pixels and
 * per-channel sums S over its pixels, mask = FTV_MASK_REUSE_P when every compared channel has
 * |S_cur - S_prev| < t_p * n; else FTV_MASK_REUSE_I when an I frame is given and every channel has
 * |S_cur - S_I| < t_i * n; else FTV_MASK_CHANGED (also for empty segments). This is the paper's test
 * on segment means (mean change < T) in exact integers. d_mask[n_segments] receives the mask,
 * d_changed_list the changed segments in increasing order and *d_n_changed their count (device).
 * The paper's thresholds are T_P = 3 and T_I = 1 for 8-bit samples. Asynchronous. The per-segment sums live
 * in the context, one slot per reference (ftv_adjacency uses the same slot as scratch): calls for one
 * reference whose work overlaps on the GPU (different streams without ordering between them) race.
 * Device-found errors (a label outside [0, n_segments): the pixel is left out) are reported by ftv_check.
 */
FTV_API ftv_status ftv_temporal_mask(ftv_ctx* ctx, int32_t ref_index, const void* const* d_cur,
                                     const int64_t* cur_pitch, const void* const* d_prev, const int64_t* prev_pitch,
                                     const void* const* d_iframe, const int64_t* iframe_pitch,
                                     const int32_t* d_labels, int32_t n_segments, int32_t t_p, int32_t t_i,
                                     int32_t mode, uint8_t* d_mask, int32_t* d_changed_list,
                                     int32_t* d_n_changed, ftv_stream stream);

/*
 * ftv_temporal_mask_views - ftv_temporal_mask for n distinct references of one context in one launch
 * sequence (three kernel launches for up to 16 references), e.g. every view of a frame. Reference
 * ref_indices[k] (host array [n]) takes d_cur[3k..3k+2], d_prev[3k..3k+2] and, when d_iframe is not NULL,
 * d_iframe[3k..3k+2] (host arrays of device plane pointers, pitches in bytes alike; the I-frame test is
 * made for all or none), d_labels[k] with n_segments[k] segments, and writes d_mask[k], d_changed_list[k]
 * and *d_n_changed[k] (host arrays of device pointers). Each reference gets exactly the results of
 * ftv_temporal_mask. Arguments are checked before anything is launched (FTV_ERR_INVALID_ARG: a repeated or
 * out-of-range reference index, a NULL pointer, a short pitch, a segment count above max_segments).
 * Asynchronous on `stream`.
 */
FTV_API ftv_status ftv_temporal_mask_views(ftv_ctx* ctx, int32_t n, const int32_t* ref_indices,
                                           const void* const* d_cur, const int64_t* cur_pitch,
                                           const void* const* d_prev, const int64_t* prev_pitch,
                                           const void* const* d_iframe, const int64_t* iframe_pitch,
                                           const int32_t* const* d_labels, const int32_t* n_segments, int32_t t_p,
                                           int32_t t_i, int32_t mode, uint8_t* const* d_mask,
                                           int32_t* const* d_changed_list, int32_t* const* d_n_changed,
                                           ftv_stream stream);

/*
 * ftv_temporal_mask_static - the temporal test of ftv_temporal_mask without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that cannot call cudaMalloc,
 * e.g. a process whose device memory is fully reserved up front under a fixed budget, or a
 * latency-critical loop that must not take cudaMalloc's implicit device-wide synchronisation. It needs
 * no ftv_ctx (creating one allocates): the caller passes the geometry (width, height, sample_bytes of
 * the frames and label map) plus the same inputs and outputs as ftv_temporal_mask, and gets the same
 * results. Device-found errors (a label outside [0, n_segments)) are OR-ed into *d_status when
 * d_status (a caller-owned device word) is not NULL; such pixels are left out.
 *
 * Scratch: the per-segment accumulators live in one statically sized device array inside this library
 * (FTV_STATIC_MAX_SEGMENTS x 64 bytes = 4 MiB), which every GPU that loads the library holds until the
 * process exits. n_segments above FTV_STATIC_MAX_SEGMENTS is rejected with FTV_ERR_INVALID_ARG.
 * The work runs on the current device: every device pointer argument must be memory of that device, else
 * FTV_ERR_INVALID_ARG before anything is launched. Each call looks up the array's device address with the
 * current device (no address is cached, so a device reset leaves nothing stale); the first call on a
 * device also loads the library's device code there, so make it before any stream capture. Every call on
 * a device shares the same array and clears it on its stream before use: calls whose work overlaps on the
 * GPU (different streams without ordering between them) race and give wrong results. Asynchronous on
 * `stream`.
 */
#define FTV_STATIC_MAX_SEGMENTS 65536
FTV_API ftv_status ftv_temporal_mask_static(int32_t width, int32_t height, int32_t sample_bytes,
                                            const void* const* d_cur, const int64_t* cur_pitch,
                                            const void* const* d_prev, const int64_t* prev_pitch,
                                            const void* const* d_iframe, const int64_t* iframe_pitch,
                                            const int32_t* d_labels, int32_t n_segments, int32_t t_p, int32_t t_i,
                                            int32_t mode, uint8_t* d_mask, int32_t* d_changed_list,
                                            int32_t* d_n_changed, uint32_t* d_status, ftv_stream stream);

/*
 * Winner-take-all readout of one cost volume d_cost [n_segments][n_labels]: d_label_out[s] = the label
 * of least cost, the smallest such label on ties. With d_mask (from ftv_temporal_mask), segments
 * marked FTV_MASK_REUSE_P take d_prev_label[s] and FTV_MASK_REUSE_I take d_iframe_label[s]
 * (Sec. III-E adoption). With d_seg_list/d_n_listed only listed segments are written. With d_labels_pix
 * (the reference label map) and d_depth_map, also writes the per-pixel depth z of each pixel's segment
 * label (float [height][width]) for reference ref_index. Asynchronous.
 */
FTV_API ftv_status ftv_wta_depth(ftv_ctx* ctx, int32_t ref_index, const int32_t* d_cost, int32_t n_segments,
                                 const uint8_t* d_mask, const uint16_t* d_prev_label,
                                 const uint16_t* d_iframe_label, const int32_t* d_seg_list,
                                 const int32_t* d_n_listed, uint16_t* d_label_out, const int32_t* d_labels_pix,
                                 float* d_depth_map, ftv_stream stream);

/* ------------------------------------------------------------------ batched and served forms -----
 * A camera stream is one ftv_ctx with resident state (ftv_stream_init): its static label maps and
 * segment indexes, a ring of three packed frames (current, previous P, I) and per-segment labels of
 * the previous and the I frame (Sec. III-E: I-type and P-type depth frames). A batch runs one frame
 * of each of many streams (any mix of shapes, view, segment and label counts that share sample
 * format and combination rule) as one fixed launch sequence: pack, temporal test, one persistent cost
 * kernel over the flat (job, reference, tile, label block) queue, winner-take-all with adoption. */

enum { FTV_FRAME_I = 0, FTV_FRAME_P = 1 };
typedef struct ftv_batch ftv_batch;

/* One frame of one stream. d_planes/pitch_bytes as in ftv_cost_volume (3 entries per view, host
 * arrays of device pointers); frame_type FTV_FRAME_I (every segment is estimated; the frame becomes the
 * stream's I frame) or FTV_FRAME_P (only segments that fail the temporal test are estimated; the others
 * adopt the previous or the I frame's label). d_label_out[r] (optional, uint16 [S_r]) receives the
 * labels; d_depth_out[r] (optional, float [H][W]) the per-pixel depth; either array may be NULL. */
typedef struct ftv_frame_job {
    ftv_ctx* ctx;
    const void* const* d_planes;
    const int64_t* pitch_bytes;
    int32_t frame_type;
    uint16_t* const* d_label_out;
    float* const* d_depth_out;
} ftv_frame_job;

/* Make ctx a stream: copies the label maps d_labels[r] (int32 [H][W], n_segments[r] segments each, kept
 * for the stream's life), builds their segment indexes and allocates the resident state. t_p, t_i,
 * mode: the temporal test of ftv_temporal_mask. The first frame of a stream must be FTV_FRAME_I.
 * Asynchronous on `stream` apart from the allocations. */
FTV_API ftv_status ftv_stream_init(ftv_ctx* ctx, const int32_t* const* d_labels, const int32_t* n_segments,
                                   int32_t t_p, int32_t t_i, int32_t mode, ftv_stream stream);

/* Device bytes of a stream's resident state for segment counts n_segments[n_refs] (for admission by
 * HBM footprint; the context's own scratch is allocated at ftv_depth_init). */
FTV_API ftv_status ftv_stream_footprint(const ftv_ctx* ctx, const int32_t* n_segments, int64_t* bytes);

/* Device pointer to a stream's current per-segment labels of reference ref_index (uint16 [S]). */
FTV_API ftv_status ftv_stream_labels(const ftv_ctx* ctx, int32_t ref_index, const uint16_t** d_labels_out);

/* Device pointers to a stream's temporal mask of reference ref_index (uint8 [S]: FTV_MASK_*) and to the
 * count of segments its last frame re-estimated (int32 [1]); valid after that frame's batch completes. */
FTV_API ftv_status ftv_stream_mask(const ftv_ctx* ctx, int32_t ref_index, const uint8_t** d_mask,
                                   const int32_t** d_n_changed);

/*
 * Checkpoint and resume of a stream's resident temporal state (Sec. III-E: the previous P and the I depth
 * frame of every view, with the colours the temporal test compares against). The checkpoint holds the
 * previous frame's and the I frame's packed views and, per reference, the per-segment labels of both.
 * ftv_stream_state_bytes: size of the checkpoint of ctx's stream now (host only).
 * ftv_stream_state_save: copy it into host_buf (bytes at least that size; pinned memory keeps the copy
 * asynchronous) on `stream`; valid once the stream's work up to the call, and the copy, have completed.
 * ftv_stream_state_load: restore it into a stream made by ftv_stream_init with the same cameras, references,
 * label count, texel format and segment counts (the label maps themselves are ftv_stream_init's input);
 * the next frame may then be a P frame. FTV_ERR_INVALID_ARG for a checkpoint of another shape or a short
 * buffer. Asynchronous on `stream`; host_buf must stay valid until the copy completes.
 */
FTV_API ftv_status ftv_stream_state_bytes(const ftv_ctx* ctx, int64_t* bytes);
FTV_API ftv_status ftv_stream_state_save(const ftv_ctx* ctx, void* host_buf, int64_t bytes, ftv_stream stream);
FTV_API ftv_status ftv_stream_state_load(ftv_ctx* ctx, const void* host_buf, int64_t bytes, ftv_stream stream);

/* Device pointer to a stream's list of the segments its last frame of reference ref_index re-estimated
 * (int32, in increasing order, *d_n_changed entries as reported by ftv_stream_mask; every segment for an I
 * frame). Sec. III-E: only these segments' costs are computed. Valid after that frame's batch completes. */
FTV_API ftv_status ftv_stream_changed(const ftv_ctx* ctx, int32_t ref_index, const int32_t** d_changed);

/* A batch executor with room for max_jobs frames, max_units (job, reference) units (<= 240) and
 * max_views views in total; owns a device descriptor block and a pinned staging copy of it. */
FTV_API ftv_status ftv_batch_create(int32_t max_jobs, int32_t max_units, int32_t max_views, ftv_batch** out);
FTV_API ftv_status ftv_batch_destroy(ftv_batch* b);

/* Host side of one batch: validates the jobs (one frame per stream, same sample format and combination
 * rule, capacity), writes their descriptors into the pinned staging block and advances each stream's
 * ring. Must be followed by exactly one ftv_batch_launch or ftv_batch_replay. Returns FTV_ERR_BUSY
 * while the previous launch of this batch object is still pending (the staging block is in use).
 * A stream may have at most one frame in flight: submit its next frame after this batch completes. */
FTV_API ftv_status ftv_batch_prepare(ftv_batch* b, const ftv_frame_job* jobs, int32_t n_jobs);

/* Enqueue the prepared batch on `stream` (one H2D copy of the descriptor block + 9 kernels). */
FTV_API ftv_status ftv_batch_launch(ftv_batch* b, ftv_stream stream);

/* Same work as ftv_batch_launch through a CUDA graph of the launch sequence, captured on the first
 * call (and again if the sample format or combination rule changes) and replayed afterwards: the
 * descriptor block is re-read from the staging copy at every replay, so any batch composition
 * within capacity replays the same graph. */
FTV_API ftv_status ftv_batch_replay(ftv_batch* b, ftv_stream stream);

#define FTV_MAX_BATCH_CHUNKS 16

/* Split the batch's cost work over `chunks` (1..FTV_MAX_BATCH_CHUNKS, default 1) consecutive persistent
 * launches, each over an equal share of the (tile, label-block) items. The paper has no counterpart: this
 * is a scheduling aid for serving. One persistent launch holds every SM until the whole batch is done;
 * between chunks the GPU can start other streams' kernels, higher-priority streams first, so a large
 * batch launched on a low-priority stream delays a small one on a high-priority stream by at most about
 * one chunk. Results are identical for every chunk count. Applies from the next ftv_batch_launch, or the
 * next ftv_batch_replay, which captures a new graph. */
FTV_API ftv_status ftv_batch_set_chunks(ftv_batch* b, int32_t chunks);

/* Non-blocking completion test of the last launch: FTV_OK when done, FTV_ERR_BUSY while running. */
FTV_API ftv_status ftv_batch_query(ftv_batch* b);

/* Wait for the last launch; returns the device-found errors of its jobs (the OR of their statuses). */
FTV_API ftv_status ftv_batch_wait(ftv_batch* b);

/* Kernel launches this batch object has enqueued (for accounting). */
FTV_API int64_t ftv_batch_launch_count(const ftv_batch* b);

/*
 * Job-level boundary of the batched and served forms (the paper has no serving system; these calls carry
 * its per-view I/P depth frames of Sec. III-E for many camera streams at once).
 *
 * ftv_job_footprint: device bytes one camera stream of configuration cfg needs, with at most n_segments_max
 * segments per reference (0: cfg->max_segments): the context ftv_depth_init allocates (packed views,
 * homography tables, segment index, scratch), the resident state ftv_stream_init allocates (three packed
 * frames, per-segment labels, mask, list, sums, the cost rows) and one frame of input planes. Host only;
 * FTV_ERR_INVALID_ARG for an invalid configuration.
 *
 * ftv_batch_set_budget: admission budget of a batch object in device bytes (0, the default: none).
 *
 * ftv_batch_submit: queue one frame of one stream (job->ctx after ftv_stream_init) for the batch's next
 * launch and return its ticket (> 0). The job's arrays are copied; its device buffers must stay valid
 * until the ticket completes. Synchronous argument errors: FTV_ERR_INVALID_ARG (as ftv_batch_prepare),
 * FTV_ERR_STATE (a P frame before the stream's first I frame). Admission: FTV_ERR_BUSY when the stream
 * already has a queued frame, when the queued jobs would exceed the batch's capacity or differ in precision,
 * sample format or combination rule, or when the footprints (ftv_job_footprint of each job's stream) of the
 * queued jobs plus those of the launch in flight would exceed the budget: retry after a ticket completes.
 * FTV_ERR_OUT_OF_MEMORY when the job alone exceeds the budget.
 *
 * ftv_batch_flush: launch every queued job as one batch on `stream` (the captured graph of
 * ftv_batch_replay). FTV_OK with nothing queued; FTV_ERR_BUSY while the previous launch of this batch
 * object runs (the queue is kept: retry).
 *
 * ftv_batch_poll: non-blocking. FTV_ERR_BUSY while the ticket's job is queued or running; FTV_OK once it
 * has completed, with *job_status that job's own result: FTV_OK, FTV_ERR_INVALID_ARG (a sample above the
 * bit depth, or a label outside [0, S) in its stream's label maps), FTV_ERR_OVERFLOW (a segment too large
 * for int32 sums) or FTV_ERR_CUDA. Every job of a launch has its own device status word, so a failed job
 * does not fail the others. FTV_ERR_INVALID_ARG for a ticket never issued or older than the last 4096.
 * ftv_batch_wait after a flush waits for the launch and returns the OR of its jobs' statuses.
 */
FTV_API ftv_status ftv_job_footprint(const ftv_config* cfg, int32_t n_segments_max, int64_t* bytes);
FTV_API ftv_status ftv_batch_set_budget(ftv_batch* b, int64_t hbm_budget_bytes);
FTV_API ftv_status ftv_batch_submit(ftv_batch* b, const ftv_frame_job* job, uint64_t* ticket);
FTV_API ftv_status ftv_batch_flush(ftv_batch* b, ftv_stream stream);
FTV_API ftv_status ftv_batch_poll(ftv_batch* b, uint64_t ticket, ftv_status* job_status);

/*
 * Centre table (Sec. III-C as written): Eq. 4 on a window around each segment's centre and the
 * neighbour segment that the centre maps to, i.e. what a graph-cut consumer needs to form Eq. 5's
 * M = min{0, m - K} (K = 30 in the paper) when d_s = d_s'. For every reference r, segment s, label d
 * and neighbour k (table order of ftv_get_neighbours):
 *   mu_s  integer centroid (floor((2 sum x + n) / (2 n)), floor((2 sum y + n) / (2 n))) of s;
 *   m     sum over the window x window offsets w (odd, <= 15; the paper uses 3) of the L1 (Y, Cb, Cr)
 *         distance between mu_s + w in r and T[mu_s] + w in view k, T[.] being the volume's projection
 *         (FP32 contract, or the FP64 projection in FTV_PRECISION_FP64 contexts); pairs with a position
 *         outside its image, or a centre out of view, cost the
 *         penalty. Eq. 4's 1/size(W) is left to the consumer (m_paper = m / window^2);
 *   s'    d_labels_views[view k]'s label at T[mu_s], or -1 if out of view or that map is NULL.
 * d_labels_views: host array of n_views device label maps (int32 [H][W] per view; every reference's is
 * required, the others are optional). n_segments[r]: segment count of reference r. d_m[r], d_sprime[r]:
 * int32 [S_r][n_labels][n_nbrs_r]. Also (re)builds the references' cached segment indexes. Asynchronous.
 */
FTV_API ftv_status ftv_centre_table(ftv_ctx* ctx, const void* const* d_planes, const int64_t* pitch_bytes,
                                    const int32_t* const* d_labels_views, const int32_t* n_segments, int32_t window,
                                    int32_t* const* d_m, int32_t* const* d_sprime, ftv_stream stream);

/*
 * Segment adjacency and adaptive smoothing weights of Sec. III-D (Eq. 2-3) for reference ref_index:
 * the adjacent segment pairs s < t of label map d_labels (int32 [H][W], n_segments segments; pixels
 * 4-connected, or also diagonally with connectivity 8), in increasing (s, t) order, and for each pair
 * beta = beta0 / || mean YCbCr_s - mean YCbCr_t ||_1 in the colours of d_frame (3 device planes, pitches
 * in bytes). The paper leaves a zero distance open: distances below min_diff (> 0) count as min_diff.
 * The distance is the exact rational sum_c |S_cs n_t - S_ct n_s| / (n_s n_t) and beta is formed in
 * double as beta0 * (n_s n_t) / numerator, then rounded to float (exact for n_s n_t 3 (2^bd - 1) < 2^63).
 * Writes min(count, capacity) edges to d_edge_s, d_edge_t, d_beta and the full count to *d_n_edges
 * (device). A segment with more than 32 neighbours t > s sets FTV_ERR_OVERFLOW in the status word
 * (its list is truncated). Also (re)builds the reference's cached segment index. Asynchronous.
 */
FTV_API ftv_status ftv_adjacency(ftv_ctx* ctx, int32_t ref_index, const void* const* d_frame,
                                 const int64_t* frame_pitch, const int32_t* d_labels, int32_t n_segments,
                                 int32_t connectivity, double beta0, double min_diff, int32_t capacity,
                                 int32_t* d_edge_s, int32_t* d_edge_t, float* d_beta, int32_t* d_n_edges,
                                 ftv_stream stream);

/* ------------------------------------------------------------------------ superpixel segmentation -----
 *
 * Sec. IV-C: the label maps come from SNIC superpixels computed in (Y, Cb, Cr) with compactness factor
 * m (the paper uses m = 5) and 8-connected segments. SNIC's single priority queue is sequential; these
 * entry points compute its data-parallel reformulation, defined exactly as follows.
 *   - Seeds lie on an S x S grid (S = grid_step): cell (i, j) covers x in [iS, min(iS + S, W)) and
 *     y in [jS, min(jS + S, H)), has label j * ceil(W/S) + i and seed (iS + (w-1)/2, jS + (h-1)/2) for a
 *     cell w wide and h high. An image has ceil(W/S) * ceil(H/S) labels (some may end empty).
 *   - Distance of a pixel (position x, colour c) to a cluster (mean position X, mean colour C):
 *     D = S^2 ||c - C||^2 + m^2 ||x - X||^2 with colours on the 8-bit scale (for bit depth bd > 8 the
 *     spatial term is multiplied by 4^(bd - 8), for bd < 8 the colour term by 4^(8 - bd)). Means are
 *     held in 1/16 units, M = floor((32 sum + n) / (2 n)), and D is evaluated exactly in integers on
 *     16 * value - M.
 *   - `iterations` assignment passes: a pixel of cell (i, j) joins the cluster of least D among the cells
 *     (i + a, j + b), a, b in {-1, 0, 1} (smallest label on ties); between passes each cluster's mean
 *     becomes that of its pixels (a cluster without pixels keeps its mean). Clusters start at their
 *     seed pixel.
 *   - Connectivity: components are the 8-connected sets of equally labelled pixels, named by their first
 *     pixel in raster order. A label's largest component (earliest named on ties) keeps the label; every
 *     other component is merged in rounds: each group not yet holding a kept component joins the
 *     8-adjacent group whose mean colour (rounded to 1/16, L1 over the three channels) is nearest (the
 *     smallest name on ties), all joins of a round at once, until every group holds one. Every label is
 *     then one 8-connected set (or empty).
 * The result is unique, independent of tiling and scheduling.
 */
typedef struct ftv_segmenter ftv_segmenter;

#define FTV_SEG_MAX_IMAGES 4096
#define FTV_SEG_MAX_STEP 64

/*
 *   n_images            images segmented by one call (views of a rig, frames), 1..FTV_SEG_MAX_IMAGES
 *   widths, heights     [n_images] sizes, 1..FTV_MAX_DIM (host memory, copied); all pixels of all images
 *                       together must stay below 2^31 - 1
 *   sample_bytes        1 (uint8) or 2 (uint16) samples
 *   bit_depth           significant bits, <= 8 * sample_bytes; samples must not exceed 2^bit_depth - 1
 *   grid_step           S, 1..FTV_SEG_MAX_STEP
 *   compactness         m, 0..255
 *   iterations          assignment passes, 1..64
 */
typedef struct ftv_segmenter_config {
    int32_t n_images;
    const int32_t* widths;
    const int32_t* heights;
    int32_t sample_bytes;
    int32_t bit_depth;
    int32_t grid_step;
    int32_t compactness;
    int32_t iterations;
} ftv_segmenter_config;

/* Create a segmenter for a fixed set of image sizes on the current device; allocates its device scratch
 * (about 100 bytes per pixel) and a pinned staging block. Synchronous. FTV_ERR_INVALID_ARG,
 * FTV_ERR_OUT_OF_MEMORY. */
FTV_API ftv_status ftv_segmenter_init(const ftv_segmenter_config* cfg, ftv_segmenter** out);

/* Host: label count of every image, n_segments[n_images] = ceil(W/S) * ceil(H/S). */
FTV_API ftv_status ftv_segmenter_segments(const ftv_segmenter* sg, int32_t* n_segments);

/* Segment every image. d_planes[3 * n_images]: device Y, Cb, Cr planes of image i at 3i..3i+2, row pitches
 * in bytes in pitch_bytes[3 * n_images] (>= width * sample_bytes); d_labels[n_images]: device int32 [H][W]
 * outputs, dense rows. Asynchronous on `stream`, except that it first waits until the previous call's
 * descriptor upload has left the staging block. One stream at a time per segmenter. A device-side bound
 * that trips (it cannot on valid input) is reported by ftv_segmenter_check. */
FTV_API ftv_status ftv_superpixels(ftv_segmenter* sg, const void* const* d_planes, const int64_t* pitch_bytes,
                                   int32_t* const* d_labels, ftv_stream stream);

/* Wait for `stream`, then return and clear the segmenter's device status word (FTV_OK if clean,
 * FTV_ERR_TIMEOUT if a bounded loop gave up). */
FTV_API ftv_status ftv_segmenter_check(ftv_segmenter* sg, ftv_stream stream);

/* Kernel launches this segmenter has enqueued since creation. */
FTV_API int64_t ftv_segmenter_launch_count(const ftv_segmenter* sg);

/* Timing: with enable != 0 every ftv_superpixels call records CUDA events on its stream around the whole
 * call and around each assignment-pass launch (the events belong to the segmenter). */
FTV_API ftv_status ftv_segmenter_set_profiling(ftv_segmenter* sg, int32_t enable);

/* Of the most recent timed call: *assign_ms = mean duration of one assignment-pass launch, *total_ms =
 * device time of the whole call (either pointer may be NULL). Waits for the call's end event.
 * FTV_ERR_STATE if no call was timed. */
FTV_API ftv_status ftv_segmenter_kernel_ms(ftv_segmenter* sg, float* assign_ms, float* total_ms);

FTV_API ftv_status ftv_segmenter_destroy(ftv_segmenter* sg);

/* Wait for `stream`, then return and clear the context's device status word (FTV_OK if clean). Errors
 * found building a stream's resident state (ftv_stream_init: a label outside [0, S), a segment too large
 * for int32 sums) are included and not cleared: they hold for every frame of that stream. */
FTV_API ftv_status ftv_check(ftv_ctx* ctx, ftv_stream stream);

/* Wait for `stream`, then report in *culled how many pixel x label x neighbour evaluations of the context's
 * most recent ftv_cost_volume call were decided without sampling. The cost kernel bounds each tile of
 * pixels by its box and tests every (neighbour, label) homography against the neighbour view at the
 * box's corners, with a margin that covers the FP32 contract's rounding at every pixel of the box; when
 * no pixel can land inside the view, every one of those samples costs the out-of-view penalty, which is
 * what the kernel then applies (under the minimum with a penalty of at least 3 (2^bit_depth - 1), the
 * default, that changes nothing). Results are identical with and without this; the count is for
 * accounting (a roofline that charges only the samples taken). */
FTV_API ftv_status ftv_culled_evaluations(ftv_ctx* ctx, ftv_stream stream, int64_t* culled);

/* Wait for `stream`, then report in *recomputed how many evaluations of the context's most recent
 * ftv_cost_volume call (FTV_PRECISION_FP64 contexts) were computed in double precision: those whose
 * FP32 local-frame position lay within its error bound of a rounding boundary, plus every evaluation of
 * a (tile, neighbour, label) whose bound could not be established (Wz near zero inside the tile). 0 for
 * FP32 contexts. Results do not depend on it; the count is for accounting. */
FTV_API ftv_status ftv_fp64_recomputed(ftv_ctx* ctx, ftv_stream stream, int64_t* recomputed);

/* Timing of the dominant kernel: with enable != 0, every ftv_cost_volume call records a pair of CUDA
 * events on its stream immediately around its cost-kernel launch (the events belong to the context). */
FTV_API ftv_status ftv_set_profiling(ftv_ctx* ctx, int32_t enable);

/* Elapsed milliseconds between the events of the most recent timed cost-kernel launch; waits for the
 * stop event. FTV_ERR_STATE if no timed launch happened. */
FTV_API ftv_status ftv_last_kernel_ms(ftv_ctx* ctx, float* ms);

/*
 * Launch shape of the context's cost kernel (no paper counterpart: the GPU's work decomposition). A work
 * item is one tile of the kernel's compile-time pixel count times one block of consecutive labels;
 * label_block caps the labels per block (the labels are split into equal blocks of at most that many,
 * 1 <= label_block <= the stage's limit for the context's neighbour count), and ctas_per_sm sets the
 * persistent grid (1 up to the occupancy limit; 0 = the occupancy limit). Every shape gives the same
 * volume. Set between calls, not while a call of the context is being issued. The batch path
 * (ftv_batch_*) uses a context's label block and its own occupancy-sized grid.
 */
FTV_API ftv_status ftv_set_launch_shape(ftv_ctx* ctx, int32_t label_block, int32_t ctas_per_sm);

/* The effective shape (the label block in use, CTAs per SM in use) and the limits for this context. Any
 * output pointer may be NULL. */
FTV_API ftv_status ftv_get_launch_shape(const ftv_ctx* ctx, int32_t* label_block, int32_t* ctas_per_sm,
                                        int32_t* max_label_block, int32_t* max_ctas_per_sm);

/*
 * Autotuner: for every candidate shape (label_blocks[i], ctas[j]) runs ftv_cost_volume on the given
 * inputs `reps` times, times the cost kernel with the context's events (ftv_set_profiling), and keeps the
 * fastest shape on the context (best_* may be NULL). ms_out (host, may be NULL) receives the minimum
 * kernel milliseconds per candidate, [n_label_blocks][n_ctas]. The first run indexes d_labels (NULL:
 * the cached index); d_cost receives the volume (identical for every shape). Synchronous (waits for each
 * timed launch). Errors: FTV_ERR_INVALID_ARG for a candidate outside the limits of
 * ftv_get_launch_shape; any error of ftv_cost_volume, after which the previous shape is restored.
 */
FTV_API ftv_status ftv_autotune(ftv_ctx* ctx, const void* const* d_planes, const int64_t* pitch_bytes,
                                const int32_t* const* d_labels, const int32_t* n_segments, int32_t* const* d_cost,
                                const int32_t* label_blocks, int32_t n_label_blocks, const int32_t* ctas,
                                int32_t n_ctas, int32_t reps, ftv_stream stream, float* ms_out,
                                int32_t* best_label_block, int32_t* best_ctas_per_sm);

/* Kernel launches this context has enqueued since creation (for accounting). */
FTV_API int64_t ftv_launch_count(const ftv_ctx* ctx);

/* Self-check of the cost kernel's reciprocal on the current device. The contract's r = 1/Wz is the IEEE
 * round-to-nearest reciprocal. The kernel forms it as one Newton-Raphson step on the hardware estimate
 * (r = r0 + r0 (1 - Wz r0) with fused multiply-adds; Markstein's method), scaling positive subnormal
 * Wz by 2^64 first, but only on a device where this equals the IEEE reciprocal for every positive float
 * below 2^126 (|Wz| < 2^117 always): the first context created on a device runs that exhaustive
 * comparison (about 2.1e9 inputs, a few milliseconds) and otherwise keeps the IEEE routine.
 * *mismatches receives the count of disagreeing inputs, *fast_path_used (optional) whether the kernel
 * uses the Newton step. */
FTV_API ftv_status ftv_reciprocal_check(int64_t* mismatches, int32_t* fast_path_used);

/* Human-readable name of a status code (static storage). */
FTV_API const char* ftv_status_str(ftv_status s);

#ifdef __cplusplus
}
#endif
#endif /* FTV_H */
