// C ABI entry points: argument validation, context set-up and launch sequencing.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "ftv_internal.h"

using namespace ftv;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool valid_camera(const ftv_camera& c) {
    if (c.width < 1 || c.height < 1 || c.width > FTV_MAX_DIM || c.height > FTV_MAX_DIM) return false;
    if (c.K[3] != 0.0 || c.K[6] != 0.0 || c.K[7] != 0.0 || c.K[8] != 1.0 || c.K[0] == 0.0 || c.K[4] == 0.0) return false;
    for (double v : c.K) if (!(v == v)) return false;
    for (double v : c.R) if (!(v == v)) return false;
    for (double v : c.t) if (!(v == v)) return false;
    return true;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1));
}

void free_ctx(ftv_ctx* c) {
    if (!c) return;
    free_stream_state(c);
    for (auto& r : c->refs) {
        cudaFree(r.d_H);
        cudaFree(r.d_H64);
        cudaFree(r.d_nbrs);
        cudaFree(r.d_offs);
        cudaFree(r.d_cursor);
        cudaFree(r.d_woffs);
        cudaFree(r.d_pix);
        cudaFree(r.d_centre);
        cudaFree(r.d_nbr_labels);
    }
    cudaFree(c->d_packed);
    cudaFree(c->d_status);
    cudaFree(c->d_jobs);
    cudaFree(c->d_plan);
    cudaFree(c->d_tstats);
    cudaFree(c->d_label_z);
    cudaFree(c->d_adj_deg);
    cudaFree(c->d_adj_slots);
    cudaFree(c->d_adj_offs);
    if (c->ev_start) cudaEventDestroy(c->ev_start);
    if (c->ev_stop) cudaEventDestroy(c->ev_stop);
    delete c;
}

int64_t max_sample_cost(const ftv_ctx* c) { return 3LL * ((1LL << c->bit_depth) - 1); }

int64_t max_pixel_cost(const ftv_ctx* c, int n_nbrs) {
    const int64_t one = std::max<int64_t>(c->penalty, max_sample_cost(c));
    return c->combine == FTV_COMBINE_MIN ? one : one * std::max(1, n_nbrs);
}

}  // namespace

// The host-only tables of ftv_compute_homographies[_f64]: the same arithmetic as ftv_depth_init.
template <typename T>
static ftv_status compute_homographies(const ftv_config* cfg, int32_t ref_index, T* host_out) {
    if (!cfg || !host_out || !cfg->cams || !cfg->ref_views) return FTV_ERR_INVALID_ARG;
    if (cfg->n_views < 1 || cfg->n_views > FTV_MAX_VIEWS || ref_index < 0 || ref_index >= cfg->n_refs)
        return FTV_ERR_INVALID_ARG;
    if (cfg->plane_mode == FTV_PLANES_CENTRE && (cfg->centre_view < 0 || cfg->centre_view >= cfg->n_views))
        return FTV_ERR_INVALID_ARG;
    std::vector<double> iz;
    if (!label_inv_depths(cfg->n_labels, cfg->z_near, cfg->z_far, iz)) return FTV_ERR_INVALID_ARG;
    const int ref = cfg->ref_views[ref_index];
    if (ref < 0 || ref >= cfg->n_views) return FTV_ERR_INVALID_ARG;
    std::vector<int> nbrs;
    if (cfg->nbr_offsets) {
        for (int k = cfg->nbr_offsets[ref_index]; k < cfg->nbr_offsets[ref_index + 1]; ++k) nbrs.push_back(cfg->nbr_views[k]);
    } else {
        for (int v = 0; v < cfg->n_views; ++v)
            if (v != ref) nbrs.push_back(v);
    }
    const ftv_camera* cc = cfg->plane_mode == FTV_PLANES_CENTRE ? &cfg->cams[cfg->centre_view] : nullptr;
    for (size_t k = 0; k < nbrs.size(); ++k) {
        if (nbrs[k] < 0 || nbrs[k] >= cfg->n_views) return FTV_ERR_INVALID_ARG;
        for (int d = 0; d < cfg->n_labels; ++d) {
            double H[9];
            if (plane_homography(cfg->cams[ref], cfg->cams[nbrs[k]], cc, iz[d], H) != 0) return FTV_ERR_INVALID_ARG;
            for (int e = 0; e < 9; ++e) host_out[(k * cfg->n_labels + d) * 9 + e] = (T)H[e];
        }
    }
    return FTV_OK;
}

extern "C" {

const char* ftv_status_str(ftv_status s) {
    switch (s) {
        case FTV_OK: return "ok";
        case FTV_ERR_INVALID_ARG: return "invalid argument";
        case FTV_ERR_OUT_OF_MEMORY: return "out of device memory";
        case FTV_ERR_CUDA: return "CUDA error";
        case FTV_ERR_OVERFLOW: return "segment cost may overflow int32";
        case FTV_ERR_TIMEOUT: return "device wait timed out";
        case FTV_ERR_BUSY: return "busy: admission refused";
        case FTV_ERR_STATE: return "call out of order";
        case FTV_ERR_CHECKED: return "checked build: a gather index outside its view was skipped";
    }
    return "unknown status";
}

ftv_status ftv_depth_init(const ftv_config* cfg, ftv_ctx** out) {
    if (!cfg || !out) return FTV_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->n_views < 1 || cfg->n_views > FTV_MAX_VIEWS || !cfg->cams) return FTV_ERR_INVALID_ARG;
    if (cfg->n_refs < 1 || cfg->n_refs > cfg->n_views || !cfg->ref_views) return FTV_ERR_INVALID_ARG;
    if (cfg->n_labels < 1 || cfg->n_labels > FTV_MAX_LABELS) return FTV_ERR_INVALID_ARG;
    if (!(cfg->z_near > 0.0) || !(cfg->z_far > cfg->z_near)) return FTV_ERR_INVALID_ARG;
    if (cfg->plane_mode != FTV_PLANES_REF && cfg->plane_mode != FTV_PLANES_CENTRE) return FTV_ERR_INVALID_ARG;
    if (cfg->plane_mode == FTV_PLANES_CENTRE && (cfg->centre_view < 0 || cfg->centre_view >= cfg->n_views))
        return FTV_ERR_INVALID_ARG;
    if (cfg->sample_bytes != 1 && cfg->sample_bytes != 2) return FTV_ERR_INVALID_ARG;
    if (cfg->bit_depth < 1 || cfg->bit_depth > 8 * cfg->sample_bytes) return FTV_ERR_INVALID_ARG;
    if (cfg->combine != FTV_COMBINE_MIN && cfg->combine != FTV_COMBINE_SUM) return FTV_ERR_INVALID_ARG;
    if (cfg->max_segments < 1) return FTV_ERR_INVALID_ARG;
    if (cfg->precision != FTV_PRECISION_FP32 && cfg->precision != FTV_PRECISION_FP64) return FTV_ERR_INVALID_ARG;
    for (int v = 0; v < cfg->n_views; ++v)
        if (!valid_camera(cfg->cams[v])) return FTV_ERR_INVALID_ARG;

    ftv_ctx* c = new (std::nothrow) ftv_ctx();
    if (!c) return FTV_ERR_OUT_OF_MEMORY;
    c->n_views = cfg->n_views;
    c->n_refs = cfg->n_refs;
    c->L = cfg->n_labels;
    c->plane_mode = cfg->plane_mode;
    c->centre = cfg->centre_view;
    c->sample_bytes = cfg->sample_bytes;
    c->bit_depth = cfg->bit_depth;
    c->combine = cfg->combine;
    c->max_segments = cfg->max_segments;
    c->precision = cfg->precision;
    c->z_near = cfg->z_near;
    c->z_far = cfg->z_far;
    c->penalty = cfg->oob_penalty >= 0 ? cfg->oob_penalty : (int32_t)(3 * ((1LL << cfg->bit_depth) - 1));
    // 4-byte texels wherever the samples fit (one 32-bit gather per evaluation)
    c->fmt = cfg->sample_bytes == 1 ? FMT_U8X4 : (cfg->bit_depth <= 10 ? FMT_P10 : FMT_U16X4);
    c->texel_bytes = c->fmt == FMT_U16X4 ? 8 : 4;
    c->cams.assign(cfg->cams, cfg->cams + cfg->n_views);

    std::vector<double> iz;
    if (!label_inv_depths(c->L, c->z_near, c->z_far, iz)) { delete c; return FTV_ERR_INVALID_ARG; }
    c->label_z.resize(c->L);
    for (int d = 0; d < c->L; ++d) c->label_z[d] = (float)(1.0 / iz[d]);

    // references and their neighbour lists
    std::vector<char> seen(c->n_views, 0);
    int max_n = 0;
    c->refs.resize(c->n_refs);
    for (int i = 0; i < c->n_refs; ++i) {
        RefState& r = c->refs[i];
        r.view = cfg->ref_views[i];
        if (r.view < 0 || r.view >= c->n_views || seen[r.view]) { free_ctx(c); return FTV_ERR_INVALID_ARG; }
        seen[r.view] = 1;
        r.W = c->cams[r.view].width;
        r.H = c->cams[r.view].height;
        if (cfg->nbr_offsets) {
            const int b = cfg->nbr_offsets[i], e = cfg->nbr_offsets[i + 1];
            if (b < 0 || e < b || !cfg->nbr_views) { free_ctx(c); return FTV_ERR_INVALID_ARG; }
            for (int k = b; k < e; ++k) r.nbrs.push_back(cfg->nbr_views[k]);
        } else {
            for (int v = 0; v < c->n_views; ++v)
                if (v != r.view) r.nbrs.push_back(v);
        }
        r.n_nbrs = (int)r.nbrs.size();
        if (r.n_nbrs > FTV_MAX_NBRS) { free_ctx(c); return FTV_ERR_INVALID_ARG; }
        for (int v : r.nbrs)
            if (v < 0 || v >= c->n_views || v == r.view) { free_ctx(c); return FTV_ERR_INVALID_ARG; }
        max_n = std::max(max_n, r.n_nbrs);
    }

    // label blocking: N x LB x 9 homography floats must fit the kernel's shared-memory stage
    int lb_max = std::min(kMaxLB, kHEntries / std::max(1, max_n));
    lb_max = std::max(1, std::min(lb_max, c->L));
    c->lb_max = lb_max;
    c->nLB = (c->L + lb_max - 1) / lb_max;
    c->LB = (c->L + c->nLB - 1) / c->nLB;

    // homographies (FP64 -> FP32; the FP64 table is kept for the FP64 projection)
    const ftv_camera* cc = c->plane_mode == FTV_PLANES_CENTRE ? &c->cams[c->centre] : nullptr;
    for (auto& r : c->refs) {
        r.h_H.resize((size_t)r.n_nbrs * c->L * 9);
        r.h_H64.resize(r.h_H.size());
        for (int k = 0; k < r.n_nbrs; ++k)
            for (int d = 0; d < c->L; ++d) {
                double H[9];
                if (plane_homography(c->cams[r.view], c->cams[r.nbrs[k]], cc, iz[d], H) != 0) {
                    free_ctx(c);
                    return FTV_ERR_INVALID_ARG;
                }
                for (int e = 0; e < 9; ++e) {
                    const float f = (float)H[e];
                    // the device's exact in-view test relies on |h| <= 2^100 (finite projections)
                    if (!(std::fabs(f) <= 0x1p100f) || !(std::fabs(H[e]) <= 0x1p100)) {
                        free_ctx(c);
                        return FTV_ERR_INVALID_ARG;
                    }
                    r.h_H[((size_t)k * c->L + d) * 9 + e] = f;
                    r.h_H64[((size_t)k * c->L + d) * 9 + e] = H[e];
                }
            }
    }

    // Classify the entries the way the cost kernel's staging does: projective-only when no entry has
    // h6 = h7 = 0, so that no entry takes an affine or rectified path.
    {
        bool any_affine = false;
        for (const auto& r : c->refs)
            for (size_t e = 0; e < r.h_H.size(); e += 9) any_affine = any_affine || (r.h_H[e + 6] == 0.0f && r.h_H[e + 7] == 0.0f);
        c->kind = any_affine ? kKindMixed : kKindProjective;
        if (c->precision == FTV_PRECISION_FP64) c->kind = any_affine ? kKindPreciseMixed : kKindPrecise;
    }

    // device scratch (all host-side validation is done by now)
    if (cudaGetDevice(&c->device) != cudaSuccess) { free_ctx(c); return FTV_ERR_CUDA; }
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    size_t packed = 0;
    c->view_offset_bytes.resize(c->n_views);
    for (int v = 0; v < c->n_views; ++v) {
        c->view_offset_bytes[v] = packed;
        const size_t bytes = (size_t)c->cams[v].width * c->cams[v].height * c->texel_bytes;
        packed += (bytes + 255) & ~(size_t)255;
    }
    bool ok = dalloc(reinterpret_cast<char**>(&c->d_packed), packed) == cudaSuccess;
    ok = ok && dalloc(&c->d_status, 1) == cudaSuccess;
    ok = ok && dalloc(&c->d_jobs, kMaxUnits) == cudaSuccess;
    ok = ok && dalloc(&c->d_plan, 1) == cudaSuccess;
    ok = ok && dalloc(&c->d_tstats, (size_t)std::max(1, c->n_refs) * c->max_segments * 8) == cudaSuccess;
    c->tstats_zero.assign(c->n_refs, 0);
    ok = ok && dalloc(&c->d_label_z, (size_t)c->L) == cudaSuccess;
    ok = ok && dalloc(&c->d_adj_deg, (size_t)c->max_segments) == cudaSuccess;
    ok = ok && dalloc(&c->d_adj_slots, (size_t)c->max_segments * 32) == cudaSuccess;
    ok = ok && dalloc(&c->d_adj_offs, (size_t)c->max_segments) == cudaSuccess;
    for (auto& r : c->refs) {
        ok = ok && dalloc(&r.d_H, r.h_H.size()) == cudaSuccess;
        if (c->precision == FTV_PRECISION_FP64) ok = ok && dalloc(&r.d_H64, r.h_H64.size()) == cudaSuccess;
        ok = ok && dalloc(&r.d_nbrs, (size_t)r.n_nbrs) == cudaSuccess;
        ok = ok && dalloc(&r.d_offs, (size_t)c->max_segments + 1) == cudaSuccess;
        ok = ok && dalloc(&r.d_cursor, (size_t)c->max_segments) == cudaSuccess;
        ok = ok && dalloc(&r.d_woffs, (size_t)c->max_segments + 1) == cudaSuccess;
        ok = ok && dalloc(&r.d_pix, (size_t)r.W * r.H) == cudaSuccess;
        ok = ok && dalloc(&r.d_centre, (size_t)c->max_segments) == cudaSuccess;
        ok = ok && dalloc(&r.d_nbr_labels, (size_t)std::max(1, r.n_nbrs)) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        free_ctx(c);
        return FTV_ERR_OUT_OF_MEMORY;
    }
    ok = cudaMemset(c->d_status, 0, sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaMemcpy(c->d_label_z, c->label_z.data(), sizeof(float) * c->L, cudaMemcpyHostToDevice) == cudaSuccess;
    for (auto& r : c->refs) {
        std::vector<NbrView> nv(r.n_nbrs);
        for (int k = 0; k < r.n_nbrs; ++k) {
            const int v = r.nbrs[k];
            nv[k].texels = static_cast<char*>(c->d_packed) + c->view_offset_bytes[v];
            nv[k].w = c->cams[v].width;
            nv[k].h = c->cams[v].height;
            nv[k].pitch = c->cams[v].width;
            nv[k].pad = 0;
        }
        ok = ok && cudaMemcpy(r.d_H, r.h_H.data(), sizeof(float) * r.h_H.size(), cudaMemcpyHostToDevice) == cudaSuccess;
        if (r.d_H64)
            ok = ok && cudaMemcpy(r.d_H64, r.h_H64.data(), sizeof(double) * r.h_H64.size(), cudaMemcpyHostToDevice) ==
                           cudaSuccess;
        if (r.n_nbrs)
            ok = ok && cudaMemcpy(r.d_nbrs, nv.data(), sizeof(NbrView) * nv.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    c->fast_rcp = fast_reciprocal_exact();
    c->penalty_floor = (int64_t)c->penalty >= max_sample_cost(c);
    c->cost_blocks_per_sm = cost_blocks_per_sm(c->fmt, c->combine, c->fast_rcp);
    if (!ok) {
        free_ctx(c);
        return FTV_ERR_CUDA;
    }
    *out = c;
    return FTV_OK;
}

ftv_status ftv_compute_homographies(const ftv_config* cfg, int32_t ref_index, float* host_out) {
    return compute_homographies(cfg, ref_index, host_out);
}

ftv_status ftv_compute_homographies_f64(const ftv_config* cfg, int32_t ref_index, double* host_out) {
    return compute_homographies(cfg, ref_index, host_out);
}

ftv_status ftv_depth_destroy(ftv_ctx* ctx) {
    if (!ctx) return FTV_OK;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    free_ctx(ctx);
    return FTV_OK;
}

ftv_status ftv_get_homographies(const ftv_ctx* ctx, int32_t ref_index, float* host_out) {
    if (!ctx || !host_out || ref_index < 0 || ref_index >= ctx->n_refs) return FTV_ERR_INVALID_ARG;
    const auto& r = ctx->refs[ref_index];
    std::memcpy(host_out, r.h_H.data(), sizeof(float) * r.h_H.size());
    return FTV_OK;
}

ftv_status ftv_get_homographies_f64(const ftv_ctx* ctx, int32_t ref_index, double* host_out) {
    if (!ctx || !host_out || ref_index < 0 || ref_index >= ctx->n_refs) return FTV_ERR_INVALID_ARG;
    const auto& r = ctx->refs[ref_index];
    std::memcpy(host_out, r.h_H64.data(), sizeof(double) * r.h_H64.size());
    return FTV_OK;
}

ftv_status ftv_get_neighbours(const ftv_ctx* ctx, int32_t ref_index, int32_t* n, int32_t* host_views) {
    if (!ctx || !n || ref_index < 0 || ref_index >= ctx->n_refs) return FTV_ERR_INVALID_ARG;
    const auto& r = ctx->refs[ref_index];
    *n = r.n_nbrs;
    if (host_views) std::copy(r.nbrs.begin(), r.nbrs.end(), host_views);
    return FTV_OK;
}

ftv_status ftv_get_label_depths(const ftv_ctx* ctx, float* host_out) {
    if (!ctx || !host_out) return FTV_ERR_INVALID_ARG;
    std::copy(ctx->label_z.begin(), ctx->label_z.end(), host_out);
    return FTV_OK;
}

ftv_status ftv_segment_index(ftv_ctx* ctx, int32_t ref_index, const int32_t* d_labels, int32_t n_segments,
                             ftv_stream stream) {
    if (!ctx || !d_labels || ref_index < 0 || ref_index >= ctx->n_refs) return FTV_ERR_INVALID_ARG;
    if (n_segments < 0 || n_segments > ctx->max_segments) return FTV_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    RefState& r = ctx->refs[ref_index];
    const cudaError_t e = launch_segment_index(d_labels, r.W, r.H, n_segments, max_pixel_cost(ctx, r.n_nbrs), r.d_offs,
                                               r.d_cursor, r.d_pix, ctx->d_status, (cudaStream_t)stream,
                                               &ctx->launches);
    if (e != cudaSuccess) return FTV_ERR_CUDA;
    r.S_indexed = n_segments;
    return FTV_OK;
}

ftv_status ftv_cost_volume(ftv_ctx* ctx, const void* const* d_planes, const int64_t* pitch_bytes,
                           const int32_t* const* d_labels, const int32_t* n_segments,
                           const int32_t* const* d_seg_list, const int32_t* const* d_n_listed, int32_t* const* d_cost,
                           ftv_stream stream) {
    if (!ctx || !d_planes || !pitch_bytes || !d_cost) return FTV_ERR_INVALID_ARG;
    if (ctx->n_refs > kMaxUnits) return FTV_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // which views are read
    std::vector<char> used(ctx->n_views, 0);
    for (const auto& r : ctx->refs) {
        used[r.view] = 1;
        for (int v : r.nbrs) used[v] = 1;
    }
    for (int v = 0; v < ctx->n_views; ++v) {
        if (!used[v]) continue;
        for (int ch = 0; ch < 3; ++ch) {
            if (!d_planes[3 * v + ch]) return FTV_ERR_INVALID_ARG;
            if (pitch_bytes[3 * v + ch] < (int64_t)ctx->cams[v].width * ctx->sample_bytes) return FTV_ERR_INVALID_ARG;
        }
    }
    for (int i = 0; i < ctx->n_refs; ++i) {
        const RefState& r = ctx->refs[i];
        const bool fresh = d_labels && d_labels[i];
        if (fresh && (!n_segments || n_segments[i] < 0 || n_segments[i] > ctx->max_segments)) return FTV_ERR_INVALID_ARG;
        if (!fresh && r.S_indexed < 0) return FTV_ERR_STATE;
        if (!d_cost[i]) return FTV_ERR_INVALID_ARG;
        if (d_seg_list && d_seg_list[i] && (!d_n_listed || !d_n_listed[i])) return FTV_ERR_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    NvtxRange range("ftv_cost_volume");
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < ctx->n_views && e == cudaSuccess; ++v) {
        if (!used[v]) continue;
        NvtxRange stage("pack");
        e = launch_pack(d_planes + 3 * v, pitch_bytes + 3 * v, ctx->sample_bytes, ctx->bit_depth, ctx->fmt,
                        ctx->cams[v].width, ctx->cams[v].height,
                        static_cast<char*>(ctx->d_packed) + ctx->view_offset_bytes[v], ctx->d_status, s);
        ctx->launches++;
    }
    std::vector<RefJob> jobs(ctx->n_refs);
    for (int i = 0; i < ctx->n_refs && e == cudaSuccess; ++i) {
        RefState& r = ctx->refs[i];
        if (d_labels && d_labels[i]) {
            NvtxRange stage("segment index");
            e = launch_segment_index(d_labels[i], r.W, r.H, n_segments[i], max_pixel_cost(ctx, r.n_nbrs), r.d_offs,
                                     r.d_cursor, r.d_pix, ctx->d_status, s, &ctx->launches);
            r.S_indexed = n_segments[i];
        }
        const int S = r.S_indexed;
        const int32_t* list = d_seg_list ? d_seg_list[i] : nullptr;
        const int32_t* nl = list ? d_n_listed[i] : nullptr;
        if (e == cudaSuccess) {
            if (list) {
                e = launch_zero_rows(d_cost[i], ctx->L, S, list, nl, s);
                ctx->launches++;
            } else {
                e = cudaMemsetAsync(d_cost[i], 0, sizeof(int32_t) * (size_t)S * ctx->L, s);
            }
        }
        RefJob& J = jobs[i];
        std::memset(&J, 0, sizeof(J));
        J.ref_texels = static_cast<char*>(ctx->d_packed) + ctx->view_offset_bytes[r.view];
        J.pix = r.d_pix;
        J.offs = r.d_offs;
        J.list = list;
        J.n_listed = nl;
        J.woffs = r.d_woffs;
        J.H = r.d_H;
        J.H64 = r.d_H64;
        J.nbrs = r.d_nbrs;
        J.cost = d_cost[i];
        J.W = r.W;
        J.Href = r.H;
        J.S = S;
        J.N = r.n_nbrs;
        J.L = ctx->L;
        J.LB = ctx->LB;
        J.nLB = ctx->nLB;
        J.penalty = ctx->penalty;
        J.fmt = ctx->fmt;
    }
    if (e == cudaSuccess) {
        NvtxRange stage("plan");
        e = launch_plan(jobs.data(), ctx->n_refs, ctx->d_jobs, ctx->d_plan, s);
        ctx->launches++;
    }
    if (e == cudaSuccess && ctx->profiling) e = cudaEventRecord(ctx->ev_start, s);
    if (e == cudaSuccess) {
        NvtxRange stage("cost kernel");
        const int per_sm = ctx->ctas_per_sm > 0 ? ctx->ctas_per_sm : ctx->cost_blocks_per_sm;
        e = launch_cost(ctx->d_jobs, ctx->d_plan, ctx->fmt, ctx->combine, ctx->fast_rcp, ctx->penalty_floor, ctx->kind,
                        0, 1, ctx->n_sm * per_sm, s);
        ctx->launches++;
    }
    if (e == cudaSuccess && ctx->profiling) {
        e = cudaEventRecord(ctx->ev_stop, s);
        ctx->timed = e == cudaSuccess;
    }
    return e == cudaSuccess ? FTV_OK : FTV_ERR_CUDA;
}

// The temporal test of n references of a context (ftv_temporal_mask and ftv_temporal_mask_views): arguments
// checked, then one launch sequence per kMaxTemporalRefs references. Reference ref_indices[k] takes its own
// slot of the context's sums, cleared first when the slot is not known to be zero.
static ftv_status temporal_views(ftv_ctx* ctx, int32_t n, const int32_t* ref_indices, const void* const* d_cur,
                                 const int64_t* cur_pitch, const void* const* d_prev, const int64_t* prev_pitch,
                                 const void* const* d_iframe, const int64_t* iframe_pitch,
                                 const int32_t* const* d_labels, const int32_t* n_segments, int32_t t_p, int32_t t_i,
                                 int32_t mode, uint8_t* const* d_mask, int32_t* const* d_changed_list,
                                 int32_t* const* d_n_changed, ftv_stream stream) {
    if (!ctx || n < 0 || (n > 0 && (!ref_indices || !d_cur || !cur_pitch || !d_prev || !prev_pitch || !d_labels ||
                                    !n_segments || !d_mask || !d_changed_list || !d_n_changed)))
        return FTV_ERR_INVALID_ARG;
    if (t_p < 0 || t_i < 0 || (mode != FTV_TM_Y_ONLY && mode != FTV_TM_ALL_YUV)) return FTV_ERR_INVALID_ARG;
    if (d_iframe && !iframe_pitch) return FTV_ERR_INVALID_ARG;
    const int nch = mode == FTV_TM_ALL_YUV ? 3 : 1;
    std::vector<uint8_t> seen(ctx->n_refs, 0);
    for (int k = 0; k < n; ++k) {
        const int ri = ref_indices[k];
        if (ri < 0 || ri >= ctx->n_refs || seen[ri]) return FTV_ERR_INVALID_ARG;
        seen[ri] = 1;
        if (!d_labels[k] || !d_mask[k] || !d_changed_list[k] || !d_n_changed[k]) return FTV_ERR_INVALID_ARG;
        if (n_segments[k] < 0 || n_segments[k] > ctx->max_segments) return FTV_ERR_INVALID_ARG;
        const int64_t row = (int64_t)ctx->refs[ri].W * ctx->sample_bytes;
        for (int c = 0; c < nch; ++c) {
            const int i = 3 * k + c;
            if (!d_cur[i] || !d_prev[i] || cur_pitch[i] < row || prev_pitch[i] < row) return FTV_ERR_INVALID_ARG;
            if (d_iframe && (!d_iframe[i] || iframe_pitch[i] < row)) return FTV_ERR_INVALID_ARG;
        }
    }
    DeviceGuard g(ctx->device);
    NvtxRange range("ftv_temporal_mask");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t slot = (size_t)ctx->max_segments * 8;  // int64 words per reference
    cudaError_t e = cudaSuccess;
    for (int k0 = 0; k0 < n && e == cudaSuccess; k0 += kMaxTemporalRefs) {
        const int m = std::min(n - k0, kMaxTemporalRefs);
        TemporalRef refs[kMaxTemporalRefs];
        for (int j = 0; j < m && e == cudaSuccess; ++j) {
            const int k = k0 + j, ri = ref_indices[k];
            TemporalRef& r = refs[j];
            r = TemporalRef{};
            for (int c = 0; c < 3; ++c) {
                const bool used = c < nch;
                r.cur[c] = used ? d_cur[3 * k + c] : nullptr;
                r.prev[c] = used ? d_prev[3 * k + c] : nullptr;
                r.ifr[c] = used && d_iframe ? d_iframe[3 * k + c] : nullptr;
                r.pc[c] = used ? cur_pitch[3 * k + c] : 0;
                r.pp[c] = used ? prev_pitch[3 * k + c] : 0;
                r.pi[c] = used && d_iframe ? iframe_pitch[3 * k + c] : 0;
            }
            r.labels = d_labels[k];
            r.stats = ctx->d_tstats + ri * slot;
            r.mask = d_mask[k];
            r.changed = d_changed_list[k];
            r.n_changed = d_n_changed[k];
            r.W = ctx->refs[ri].W;
            r.H = ctx->refs[ri].H;
            r.S = n_segments[k];
            r.ms = ctx->max_segments;
            // the decide pass leaves the sums zero; a slot of unknown contents (first use, a failed launch,
            // adjacency scratch) is cleared whole
            if (!ctx->tstats_zero[ri] && slot > 0) e = cudaMemsetAsync(r.stats, 0, slot * sizeof(int64_t), s);
            ctx->tstats_zero[ri] = 0;
        }
        if (e == cudaSuccess)
            e = launch_temporal_refs(refs, m, ctx->sample_bytes, mode, d_iframe != nullptr, t_p, t_i, ctx->d_status, s,
                                     &ctx->launches);
        if (e == cudaSuccess)
            for (int j = 0; j < m; ++j) ctx->tstats_zero[ref_indices[k0 + j]] = 1;
    }
    return e == cudaSuccess ? FTV_OK : FTV_ERR_CUDA;
}

ftv_status ftv_temporal_mask(ftv_ctx* ctx, int32_t ref_index, const void* const* d_cur, const int64_t* cur_pitch,
                             const void* const* d_prev, const int64_t* prev_pitch, const void* const* d_iframe,
                             const int64_t* iframe_pitch, const int32_t* d_labels, int32_t n_segments, int32_t t_p,
                             int32_t t_i, int32_t mode, uint8_t* d_mask, int32_t* d_changed_list,
                             int32_t* d_n_changed, ftv_stream stream) {
    if (!ctx || !d_cur || !cur_pitch || !d_prev || !prev_pitch) return FTV_ERR_INVALID_ARG;
    return temporal_views(ctx, 1, &ref_index, d_cur, cur_pitch, d_prev, prev_pitch, d_iframe, iframe_pitch, &d_labels,
                          &n_segments, t_p, t_i, mode, &d_mask, &d_changed_list, &d_n_changed, stream);
}

ftv_status ftv_temporal_mask_views(ftv_ctx* ctx, int32_t n, const int32_t* ref_indices, const void* const* d_cur,
                                   const int64_t* cur_pitch, const void* const* d_prev, const int64_t* prev_pitch,
                                   const void* const* d_iframe, const int64_t* iframe_pitch,
                                   const int32_t* const* d_labels, const int32_t* n_segments, int32_t t_p,
                                   int32_t t_i, int32_t mode, uint8_t* const* d_mask, int32_t* const* d_changed_list,
                                   int32_t* const* d_n_changed, ftv_stream stream) {
    return temporal_views(ctx, n, ref_indices, d_cur, cur_pitch, d_prev, prev_pitch, d_iframe, iframe_pitch, d_labels,
                          n_segments, t_p, t_i, mode, d_mask, d_changed_list, d_n_changed, stream);
}

ftv_status ftv_wta_depth(ftv_ctx* ctx, int32_t ref_index, const int32_t* d_cost, int32_t n_segments,
                         const uint8_t* d_mask, const uint16_t* d_prev_label, const uint16_t* d_iframe_label,
                         const int32_t* d_seg_list, const int32_t* d_n_listed, uint16_t* d_label_out,
                         const int32_t* d_labels_pix, float* d_depth_map, ftv_stream stream) {
    if (!ctx || !d_cost || !d_label_out || n_segments < 0 || n_segments > ctx->max_segments) return FTV_ERR_INVALID_ARG;
    if (ref_index < 0 || ref_index >= ctx->n_refs) return FTV_ERR_INVALID_ARG;
    if (d_seg_list && !d_n_listed) return FTV_ERR_INVALID_ARG;
    if ((d_labels_pix == nullptr) != (d_depth_map == nullptr)) return FTV_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    NvtxRange range("ftv_wta_depth");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_wta(d_cost, n_segments, ctx->L, d_mask, d_prev_label, d_iframe_label, d_seg_list,
                               d_n_listed, d_label_out, s);
    ctx->launches++;
    if (e == cudaSuccess && d_depth_map) {
        const RefState& r = ctx->refs[ref_index];
        e = launch_depth_map(d_labels_pix, r.W, r.H, n_segments, d_label_out, ctx->d_label_z, ctx->L, d_depth_map,
                             ctx->d_status, s);
        ctx->launches++;
    }
    return e == cudaSuccess ? FTV_OK : FTV_ERR_CUDA;
}

ftv_status ftv_fp64_recomputed(ftv_ctx* ctx, ftv_stream stream, int64_t* recomputed) {
    if (!ctx || !recomputed) return FTV_ERR_INVALID_ARG;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return FTV_ERR_CUDA;
    unsigned long long v = 0;
    if (cudaMemcpy(&v, &ctx->d_plan->recomputed, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return FTV_ERR_CUDA;
    *recomputed = (int64_t)v;
    return FTV_OK;
}

ftv_status ftv_culled_evaluations(ftv_ctx* ctx, ftv_stream stream, int64_t* culled) {
    if (!ctx || !culled) return FTV_ERR_INVALID_ARG;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return FTV_ERR_CUDA;
    unsigned long long v = 0;
    if (cudaMemcpy(&v, &ctx->d_plan->culled, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return FTV_ERR_CUDA;
    *culled = (int64_t)v;
    return FTV_OK;
}

ftv_status ftv_check(ftv_ctx* ctx, ftv_stream stream) {
    if (!ctx) return FTV_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return FTV_ERR_CUDA;
    uint32_t st = 0;
    if (cudaMemcpy(&st, ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return FTV_ERR_CUDA;
    if (st && cudaMemset(ctx->d_status, 0, sizeof(st)) != cudaSuccess) return FTV_ERR_CUDA;
#ifdef FTV_CHECKED
    {  // the last cost-kernel launch's out-of-view gathers (checked builds)
        uint32_t ck = 0;
        if (cudaMemcpy(&ck, &ctx->d_plan->checked, sizeof(ck), cudaMemcpyDeviceToHost) != cudaSuccess) return FTV_ERR_CUDA;
        st |= ck;
    }
#endif
    // errors found building a stream's resident state stay with the stream (every job of it reports them)
    if (ctx->stream.d_status) {
        uint32_t ss = 0;
        if (cudaMemcpy(&ss, ctx->stream.d_status, sizeof(ss), cudaMemcpyDeviceToHost) != cudaSuccess) return FTV_ERR_CUDA;
        st |= ss;
    }
    if (cudaGetLastError() != cudaSuccess) return FTV_ERR_CUDA;
    if (st & ST_CHECKED) return FTV_ERR_CHECKED;
    if (st & (ST_BAD_LABEL | ST_BAD_SAMPLE)) return FTV_ERR_INVALID_ARG;
    if (st & ST_OVERFLOW) return FTV_ERR_OVERFLOW;
    return FTV_OK;
}

int64_t ftv_launch_count(const ftv_ctx* ctx) { return ctx ? ctx->launches : 0; }

ftv_status ftv_reciprocal_check(int64_t* mismatches, int32_t* fast_path_used) {
    if (!mismatches) return FTV_ERR_INVALID_ARG;
    *mismatches = reciprocal_mismatches();
    if (fast_path_used) *fast_path_used = fast_reciprocal_exact() ? 1 : 0;
    return *mismatches < 0 ? FTV_ERR_CUDA : FTV_OK;
}

ftv_status ftv_set_profiling(ftv_ctx* ctx, int32_t enable) {
    if (!ctx) return FTV_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (enable && !ctx->ev_start) {
        if (cudaEventCreate(&ctx->ev_start) != cudaSuccess || cudaEventCreate(&ctx->ev_stop) != cudaSuccess)
            return FTV_ERR_CUDA;
    }
    ctx->profiling = enable != 0;
    return FTV_OK;
}

ftv_status ftv_set_launch_shape(ftv_ctx* ctx, int32_t label_block, int32_t ctas_per_sm) {
    if (!ctx || label_block < 1 || label_block > ctx->lb_max) return FTV_ERR_INVALID_ARG;
    if (ctas_per_sm < 0 || ctas_per_sm > ctx->cost_blocks_per_sm) return FTV_ERR_INVALID_ARG;
    ctx->nLB = (ctx->L + label_block - 1) / label_block;
    ctx->LB = (ctx->L + ctx->nLB - 1) / ctx->nLB;  // equal blocks of at most label_block labels
    ctx->ctas_per_sm = ctas_per_sm;
    return FTV_OK;
}

ftv_status ftv_get_launch_shape(const ftv_ctx* ctx, int32_t* label_block, int32_t* ctas_per_sm,
                                int32_t* max_label_block, int32_t* max_ctas_per_sm) {
    if (!ctx) return FTV_ERR_INVALID_ARG;
    if (label_block) *label_block = ctx->LB;
    if (ctas_per_sm) *ctas_per_sm = ctx->ctas_per_sm > 0 ? ctx->ctas_per_sm : ctx->cost_blocks_per_sm;
    if (max_label_block) *max_label_block = ctx->lb_max;
    if (max_ctas_per_sm) *max_ctas_per_sm = ctx->cost_blocks_per_sm;
    return FTV_OK;
}

ftv_status ftv_autotune(ftv_ctx* ctx, const void* const* d_planes, const int64_t* pitch_bytes,
                        const int32_t* const* d_labels, const int32_t* n_segments, int32_t* const* d_cost,
                        const int32_t* label_blocks, int32_t n_label_blocks, const int32_t* ctas, int32_t n_ctas,
                        int32_t reps, ftv_stream stream, float* ms_out, int32_t* best_label_block,
                        int32_t* best_ctas_per_sm) {
    if (!ctx || !label_blocks || !ctas || n_label_blocks < 1 || n_ctas < 1 || reps < 1 || !d_cost)
        return FTV_ERR_INVALID_ARG;
    for (int i = 0; i < n_label_blocks; ++i)
        if (label_blocks[i] < 1 || label_blocks[i] > ctx->lb_max) return FTV_ERR_INVALID_ARG;
    for (int j = 0; j < n_ctas; ++j)
        if (ctas[j] < 0 || ctas[j] > ctx->cost_blocks_per_sm) return FTV_ERR_INVALID_ARG;
    const int32_t keep_lb = ctx->LB, keep_ctas = ctx->ctas_per_sm;
    const bool keep_profiling = ctx->profiling;
    ftv_status st = ftv_set_profiling(ctx, 1);
    float best = 0.0f;
    int bi = -1, bj = -1;
    for (int i = 0; i < n_label_blocks && st == FTV_OK; ++i)
        for (int j = 0; j < n_ctas && st == FTV_OK; ++j) {
            st = ftv_set_launch_shape(ctx, label_blocks[i], ctas[j]);
            float t_min = 0.0f;
            for (int r = 0; r < reps && st == FTV_OK; ++r) {
                // the first call indexes the label maps; later ones reuse the cached index
                st = ftv_cost_volume(ctx, d_planes, pitch_bytes, (i == 0 && j == 0 && r == 0) ? d_labels : nullptr,
                                     n_segments, nullptr, nullptr, d_cost, stream);
                float ms = 0.0f;
                if (st == FTV_OK) st = ftv_last_kernel_ms(ctx, &ms);
                if (st == FTV_OK && (r == 0 || ms < t_min)) t_min = ms;
            }
            if (st != FTV_OK) break;
            if (ms_out) ms_out[i * n_ctas + j] = t_min;
            if (bi < 0 || t_min < best) {
                best = t_min;
                bi = i;
                bj = j;
            }
        }
    ctx->profiling = keep_profiling;
    if (st != FTV_OK) {
        ftv_set_launch_shape(ctx, keep_lb, keep_ctas);
        return st;
    }
    st = ftv_set_launch_shape(ctx, label_blocks[bi], ctas[bj]);
    if (best_label_block) *best_label_block = label_blocks[bi];
    if (best_ctas_per_sm) *best_ctas_per_sm = ctas[bj];
    return st;
}

ftv_status ftv_last_kernel_ms(ftv_ctx* ctx, float* ms) {
    if (!ctx || !ms) return FTV_ERR_INVALID_ARG;
    if (!ctx->timed) return FTV_ERR_STATE;
    DeviceGuard g(ctx->device);
    if (cudaEventSynchronize(ctx->ev_stop) != cudaSuccess) return FTV_ERR_CUDA;
    if (cudaEventElapsedTime(ms, ctx->ev_start, ctx->ev_stop) != cudaSuccess) return FTV_ERR_CUDA;
    return FTV_OK;
}

}  // extern "C"
