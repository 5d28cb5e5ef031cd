/*
 * Plain CPU oracle for the segment x depth-label matching-cost volume, the per-segment temporal
 * consistency test, the winner-take-all readout and the superpixel segmentation of Mieloch,
 * Stankiewicz and Domanski, "Depth Map Estimation for Free-Viewpoint Television" (arXiv:1909.02294).
 *
 * TEST INFRASTRUCTURE ONLY. The library under test never links, loads or calls this file; only the
 * tests, the smoke check and the benchmark's CPU-baseline leg do. It shares no code, header, table
 * or constant with the CUDA library: it is written from the paper and from the arithmetic contract
 * stated below, and it is deliberately slow and direct (single thread, no blocking, no reordering).
 *
 * Arithmetic contract (the paper leaves the numerics open; this is the reading both sides follow):
 *  - Candidate depths are uniform in 1/z between z_far (label 0) and z_near (label L-1), on planes
 *    parallel to the reference camera's image plane (Sec. IV-A), or to the centre camera's image
 *    plane when depths are measured from the centre camera (Sec. III-B).
 *  - The transform T[.] of Eq. 4 for plane n^T X_r = delta is the plane homography
 *    H = K_v (R_v R_r^T + (t_v - R_v R_r^T t_r) n^T / delta) K_r^-1, formed in FP64 in a fixed
 *    operation order (or_homography_f64) and rounded once per entry to FP32.
 *  - A reference pixel (x, y) maps to X = fma(h0,x,fma(h1,y,h2)), Y = fma(h3,x,fma(h4,y,h5)),
 *    Wz = fma(h6,x,fma(h7,y,h8)) in FP32; it is out of the view unless Wz > 0; otherwise
 *    r = 1/Wz, u = X*r, v = Y*r (each IEEE FP32 round-to-nearest), and the nearest sample is
 *    (floor(u + 0.5), floor(v + 0.5)), which must lie inside the view.
 *  - FP64 projection mode: the same decision in IEEE double with the unrounded FP64 table
 *    (or_homography_table_f64): X = (h0*x + h1*y) + h2 etc., each operation rounded on its own,
 *    out unless Wz > 0, (floor(X/Wz + 0.5), floor(Y/Wz + 0.5)) (project_f64).
 *  - The sample cost is the L1 distance of the integer (Y, Cb, Cr) vectors (Eq. 4 with a one-pixel
 *    window and without the 1/size(W) scaling), or a fixed penalty when the sample is out of view.
 *  - Per pixel the costs of the neighbouring views are combined by their minimum (or their sum, the
 *    shape of the sum over c' in Eq. 1), and the segment's cost is the int32 sum over its pixels.
 *  - Temporal test (Sec. III-E): a segment keeps the previous P frame's depth when every compared
 *    component of its mean colour moved by less than T_P, else the I frame's depth when every
 *    component moved by less than T_I, else it is re-estimated. With n pixels and channel sums S,
 *    |S_cur - S_ref| < T * n is the same test on means, evaluated exactly in integers.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double K[9], R[9], t[3];
    int32_t width, height;
} or_camera;

typedef struct {
    const void* Y;
    const void* U;
    const void* V;
    int64_t pitch; /* row pitch in samples (same for the three planes) */
} or_image;

/* ------------------------------------------------------------------------------------ depths */

/* Candidate inverse depths, uniform in 1/z, label 0 = far (Sec. IV-A: planes parallel to the camera). */
int or_label_inv_depths(int L, double z_near, double z_far, double* iz) {
    if (L < 1 || !(z_near > 0) || !(z_far > z_near) || !iz) return 1;
    double a = 1.0 / z_far;
    double b = 1.0 / z_near;
    if (L == 1) {
        iz[0] = a;
        return 0;
    }
    double step = (b - a) / (double)(L - 1);
    for (int d = 0; d < L; d++) iz[d] = a + (double)d * step;
    return 0;
}

/* --------------------------------------------------------------------------------- geometry */

static int k_ok(const double* K) {
    return K[3] == 0.0 && K[6] == 0.0 && K[7] == 0.0 && K[8] == 1.0 && K[0] != 0.0 && K[4] != 0.0;
}

/* Inverse of an upper-triangular intrinsic matrix K = [[fx, s, cx], [0, fy, cy], [0, 0, 1]]. */
static void k_inverse(const double* K, double* Ki) {
    double fx = K[0], s = K[1], cx = K[2], fy = K[4], cy = K[5];
    double fxfy = fx * fy;
    Ki[0] = 1.0 / fx;
    Ki[1] = -s / fxfy;
    Ki[2] = (s * cy - cx * fy) / fxfy;
    Ki[3] = 0.0;
    Ki[4] = 1.0 / fy;
    Ki[5] = -cy / fy;
    Ki[6] = 0.0;
    Ki[7] = 0.0;
    Ki[8] = 1.0;
}

/* c = a * b for row-major 3x3, each entry summed left to right */
static void mat3_mul(const double* a, const double* b, double* c) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            c[i * 3 + j] = (a[i * 3 + 0] * b[0 * 3 + j] + a[i * 3 + 1] * b[1 * 3 + j]) + a[i * 3 + 2] * b[2 * 3 + j];
}

/*
 * FP64 plane homography of Eq. 4's transform T[.] from reference camera cr into view cv for the
 * candidate plane with inverse depth iz (Sec. IV-A). With cc == NULL the plane is parallel to the
 * reference image plane at depth 1/iz: n = (0,0,1), delta = 1/iz. With a centre camera cc
 * (Sec. III-B) the plane is parallel to cc's image plane at depth 1/iz from it, written in the
 * reference frame as n = R_r R_c^T (0,0,1), delta = (1/iz - t_c[2]) + n . t_r.
 * Operation order: A = R_v R_r^T; b = t_v - A t_r; M = A + (b n^T) w with w = iz or 1/delta;
 * H = K_v (M K_r^-1).
 */
int or_homography_f64(const or_camera* cr, const or_camera* cv, const or_camera* cc, double iz, double* H) {
    if (!cr || !cv || !H || !k_ok(cr->K) || !k_ok(cv->K)) return 1;
    double A[9], b[3], n[3], w, M[9], Ki[9], T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            A[i * 3 + j] = (cv->R[i * 3 + 0] * cr->R[j * 3 + 0] + cv->R[i * 3 + 1] * cr->R[j * 3 + 1]) +
                           cv->R[i * 3 + 2] * cr->R[j * 3 + 2];
    for (int i = 0; i < 3; i++)
        b[i] = cv->t[i] - ((A[i * 3 + 0] * cr->t[0] + A[i * 3 + 1] * cr->t[1]) + A[i * 3 + 2] * cr->t[2]);
    if (cc == NULL) {
        n[0] = 0.0;
        n[1] = 0.0;
        n[2] = 1.0;
        w = iz;
    } else {
        for (int j = 0; j < 3; j++)
            n[j] = (cr->R[j * 3 + 0] * cc->R[2 * 3 + 0] + cr->R[j * 3 + 1] * cc->R[2 * 3 + 1]) +
                   cr->R[j * 3 + 2] * cc->R[2 * 3 + 2];
        double z = 1.0 / iz;
        double delta = (z - cc->t[2]) + ((n[0] * cr->t[0] + n[1] * cr->t[1]) + n[2] * cr->t[2]);
        if (!(fabs(delta) > 1e-12)) return 2;
        w = 1.0 / delta;
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) M[i * 3 + j] = A[i * 3 + j] + (b[i] * n[j]) * w;
    k_inverse(cr->K, Ki);
    mat3_mul(M, Ki, T);
    mat3_mul(cv->K, T, H);
    return 0;
}

/* Table [n_nbrs][L][9] for one reference view, rounded to FP32 (out) or kept in FP64 (out64; exactly one
 * of the two is given). plane_mode 0 = reference planes, 1 = centre. */
static int homography_table(const or_camera* cams, int n_views, int ref, int n_nbrs, const int32_t* nbrs, int L,
                            double z_near, double z_far, int plane_mode, int centre, float* out, double* out64) {
    if (!cams || ref < 0 || ref >= n_views || n_nbrs < 0 || L < 1 || !out == !out64) return 1;
    if (plane_mode == 1 && (centre < 0 || centre >= n_views)) return 1;
    double* iz = (double*)malloc(sizeof(double) * (size_t)L);
    if (!iz) return 1;
    if (or_label_inv_depths(L, z_near, z_far, iz)) { free(iz); return 1; }
    for (int k = 0; k < n_nbrs; k++) {
        int v = nbrs[k];
        if (v < 0 || v >= n_views) { free(iz); return 1; }
        for (int d = 0; d < L; d++) {
            double H[9];
            int rc = or_homography_f64(&cams[ref], &cams[v], plane_mode == 1 ? &cams[centre] : NULL, iz[d], H);
            if (rc) { free(iz); return rc; }
            for (int e = 0; e < 9; e++) {
                if (out) out[((size_t)k * L + d) * 9 + e] = (float)H[e];
                else out64[((size_t)k * L + d) * 9 + e] = H[e];
            }
        }
    }
    free(iz);
    return 0;
}

int or_homography_table(const or_camera* cams, int n_views, int ref, int n_nbrs, const int32_t* nbrs, int L,
                        double z_near, double z_far, int plane_mode, int centre, float* out) {
    if (!out) return 1;
    return homography_table(cams, n_views, ref, n_nbrs, nbrs, L, z_near, z_far, plane_mode, centre, out, NULL);
}

int or_homography_table_f64(const or_camera* cams, int n_views, int ref, int n_nbrs, const int32_t* nbrs, int L,
                            double z_near, double z_far, int plane_mode, int centre, double* out) {
    if (!out) return 1;
    return homography_table(cams, n_views, ref, n_nbrs, nbrs, L, z_near, z_far, plane_mode, centre, NULL, out);
}

/* ------------------------------------------------------------------------------------ samples */

static int sample_at(const or_image* im, int sample_bytes, int c, int x, int y) {
    const void* p = c == 0 ? im->Y : (c == 1 ? im->U : im->V);
    size_t i = (size_t)y * (size_t)im->pitch + (size_t)x;
    return sample_bytes == 1 ? (int)((const uint8_t*)p)[i] : (int)((const uint16_t*)p)[i];
}

/* Nearest-sample position of reference pixel (x, y) in a view under FP32 homography h; returns 1 and
 * the integer position when the sample lies inside the Wv x Hv view, 0 when it is out of view. */
static int project_f32(const float* h, int x, int y, int Wv, int Hv, int* ui, int* vi) {
    float fx = (float)x, fy = (float)y;
    float X = fmaf(h[0], fx, fmaf(h[1], fy, h[2]));
    float Yh = fmaf(h[3], fx, fmaf(h[4], fy, h[5]));
    float Wz = fmaf(h[6], fx, fmaf(h[7], fy, h[8]));
    if (!(Wz > 0.0f)) return 0;
    float r = 1.0f / Wz;
    float u = X * r;
    float v = Yh * r;
    float fu = floorf(u + 0.5f);
    float fv = floorf(v + 0.5f);
    if (!(fu >= 0.0f && fu <= (float)(Wv - 1) && fv >= 0.0f && fv <= (float)(Hv - 1))) return 0;
    *ui = (int)fu;
    *vi = (int)fv;
    return 1;
}

/* The FP64 projection: the same decision in IEEE double arithmetic with the unrounded homography, each
 * operation rounded on its own, the sums taken left to right. It is the sample position of the FP64
 * precision mode, and the yardstick the FP32 contract's mismatch fraction is measured against. */
static int project_f64(const double* h, int x, int y, int Wv, int Hv, long* ui, long* vi) {
    double X = h[0] * x + h[1] * y + h[2];
    double Yh = h[3] * x + h[4] * y + h[5];
    double Wz = h[6] * x + h[7] * y + h[8];
    if (!(Wz > 0.0)) return 0;
    double fu = floor(X / Wz + 0.5), fv = floor(Yh / Wz + 0.5);
    if (!(fu >= 0.0 && fu <= (double)(Wv - 1) && fv >= 0.0 && fv <= (double)(Hv - 1))) return 0;
    *ui = (long)fu;
    *vi = (long)fv;
    return 1;
}

/* Eq. 4 with a one-pixel window: L1 distance of (Y, Cb, Cr) at reference pixel (x, y) and at the
 * corresponding sample of view v, or the out-of-view penalty. */
static int view_cost(const or_image* ref_im, const or_image* v_im, int sample_bytes, const float* h,
                     const double* h64, int x, int y, int Wv, int Hv, int penalty) {
    int ui, vi;
    if (h64) {
        long lu, lv;
        if (!project_f64(h64, x, y, Wv, Hv, &lu, &lv)) return penalty;
        ui = (int)lu;
        vi = (int)lv;
    } else if (!project_f32(h, x, y, Wv, Hv, &ui, &vi)) {
        return penalty;
    }
    int c = 0;
    for (int ch = 0; ch < 3; ch++) {
        int a = sample_at(ref_im, sample_bytes, ch, x, y);
        int b = sample_at(v_im, sample_bytes, ch, ui, vi);
        c += a > b ? a - b : b - a;
    }
    return c;
}

/* Per-pixel combination over the neighbouring views: minimum (combine 0) or sum (combine 1). Sample
 * positions come from the FP32 table H, or from the FP64 table H64 when that is given. */
static int pixel_cost(const or_camera* cams, const or_image* imgs, int sample_bytes, int ref, int n_nbrs,
                      const int32_t* nbrs, const float* H, const double* H64, int L, int d, int x, int y, int penalty,
                      int combine) {
    int acc = combine == 0 ? INT32_MAX : 0;
    for (int k = 0; k < n_nbrs; k++) {
        int v = nbrs[k];
        const size_t o = ((size_t)k * L + d) * 9;
        int c = view_cost(&imgs[ref], &imgs[v], sample_bytes, H64 ? NULL : H + o, H64 ? H64 + o : NULL, x, y,
                          cams[v].width, cams[v].height, penalty);
        if (combine == 0) acc = c < acc ? c : acc;
        else acc += c;
    }
    if (n_nbrs == 0) acc = 0;
    return acc;
}

/* Pixels of every segment in raster order: offsets[S+1], pix[n] (y * W + x). Labels outside [0, S)
 * make the call fail. */
static int segment_lists(const int32_t* labels, int W, int H, int S, int32_t** offs_out, int32_t** pix_out) {
    size_t P = (size_t)W * (size_t)H;
    int32_t* offs = (int32_t*)calloc((size_t)S + 1, sizeof(int32_t));
    int32_t* pix = (int32_t*)malloc(sizeof(int32_t) * (P ? P : 1));
    int32_t* fill = (int32_t*)calloc((size_t)S + 1, sizeof(int32_t));
    if (!offs || !pix || !fill) { free(offs); free(pix); free(fill); return 1; }
    for (size_t p = 0; p < P; p++) {
        int s = labels[p];
        if (s < 0 || s >= S) { free(offs); free(pix); free(fill); return 2; }
        offs[s + 1]++;
    }
    for (int s = 0; s < S; s++) offs[s + 1] += offs[s];
    for (size_t p = 0; p < P; p++) {
        int s = labels[p];
        pix[offs[s] + fill[s]++] = (int32_t)p;
    }
    free(fill);
    *offs_out = offs;
    *pix_out = pix;
    return 0;
}

/*
 * Cost volume of one reference view: cost[s][d] for every listed segment s (all segments when
 * seg_list is NULL) and every label d; rows of unlisted segments are not written. H is the
 * reference's FP32 table [n_nbrs][L][9] (or_homography_table), or, with H = NULL, H64 its FP64 table
 * (or_homography_table_f64) for the FP64 projection. Sums are exact int64 and the call fails with 3 if
 * one does not fit in int32.
 */
int or_cost_volume(const or_camera* cams, int n_views, const or_image* imgs, int sample_bytes, int ref, int n_nbrs,
                   const int32_t* nbrs, const float* H, const double* H64, int L, const int32_t* labels, int S,
                   int penalty, int combine, const int32_t* seg_list, int n_list, int32_t* cost) {
    if (!cams || !imgs || ref < 0 || ref >= n_views || L < 1 || S < 0 || !labels || !cost) return 1;
    if (!H == !H64) return 1;
    if (sample_bytes != 1 && sample_bytes != 2) return 1;
    int W = cams[ref].width, Hh = cams[ref].height;
    int32_t *offs, *pix;
    int rc = segment_lists(labels, W, Hh, S, &offs, &pix);
    if (rc) return rc;
    int n = seg_list ? n_list : S;
    for (int i = 0; i < n; i++) {
        int s = seg_list ? seg_list[i] : i;
        if (s < 0 || s >= S) { rc = 1; break; }
        for (int d = 0; d < L; d++) {
            int64_t sum = 0;
            for (int32_t q = offs[s]; q < offs[s + 1]; q++) {
                int x = pix[q] % W, y = pix[q] / W;
                sum += pixel_cost(cams, imgs, sample_bytes, ref, n_nbrs, nbrs, H, H64, L, d, x, y, penalty, combine);
            }
            if (sum > INT32_MAX) rc = 3;
            cost[(size_t)s * L + d] = (int32_t)sum;
        }
    }
    free(offs);
    free(pix);
    return rc;
}

/* Selected entries cost[seg[i]][lab[i]] of the same volume, each computed on its own. */
int or_cost_entries(const or_camera* cams, int n_views, const or_image* imgs, int sample_bytes, int ref, int n_nbrs,
                    const int32_t* nbrs, const float* H, const double* H64, int L, const int32_t* labels, int S,
                    int penalty, int combine, int n_entries, const int32_t* seg, const int32_t* lab, int32_t* out) {
    if (!cams || !imgs || ref < 0 || ref >= n_views || !labels || !out) return 1;
    if (!H == !H64) return 1;
    int W = cams[ref].width, Hh = cams[ref].height;
    int32_t *offs, *pix;
    int rc = segment_lists(labels, W, Hh, S, &offs, &pix);
    if (rc) return rc;
    for (int i = 0; i < n_entries; i++) {
        int s = seg[i], d = lab[i];
        if (s < 0 || s >= S || d < 0 || d >= L) { rc = 1; break; }
        int64_t sum = 0;
        for (int32_t q = offs[s]; q < offs[s + 1]; q++) {
            int x = pix[q] % W, y = pix[q] / W;
            sum += pixel_cost(cams, imgs, sample_bytes, ref, n_nbrs, nbrs, H, H64, L, d, x, y, penalty, combine);
        }
        if (sum > INT32_MAX) rc = 3;
        out[i] = (int32_t)sum;
    }
    free(offs);
    free(pix);
    return rc;
}

/*
 * Rounding-precision check: over the listed reference pixels (pix[i] = y * W + x, all pixels when
 * NULL), every label and every neighbour, count evaluations whose FP32 sample position or in/out
 * decision differs from the FP64 projection with the unrounded homography. Returns counts in
 * out[0] (mismatches) and out[1] (evaluations).
 */
int or_fp64_mismatch(const or_camera* cams, int n_views, int ref, int n_nbrs, const int32_t* nbrs, int L,
                     double z_near, double z_far, int plane_mode, int centre, int n_pix, const int32_t* pix,
                     int64_t* out) {
    if (!cams || ref < 0 || ref >= n_views || !out) return 1;
    double* iz = (double*)malloc(sizeof(double) * (size_t)L);
    if (!iz || or_label_inv_depths(L, z_near, z_far, iz)) { free(iz); return 1; }
    int W = cams[ref].width, Hh = cams[ref].height;
    int64_t n_eval = 0, n_bad = 0;
    int np = pix ? n_pix : W * Hh;
    for (int k = 0; k < n_nbrs; k++) {
        int v = nbrs[k];
        for (int d = 0; d < L; d++) {
            double Hd[9];
            float Hf[9];
            int rc = or_homography_f64(&cams[ref], &cams[v], plane_mode == 1 ? &cams[centre] : NULL, iz[d], Hd);
            if (rc) { free(iz); return rc; }
            for (int e = 0; e < 9; e++) Hf[e] = (float)Hd[e];
            for (int i = 0; i < np; i++) {
                int p = pix ? pix[i] : i;
                int x = p % W, y = p / W;
                int ui = 0, vi = 0;
                long uj = 0, vj = 0;
                int a = project_f32(Hf, x, y, cams[v].width, cams[v].height, &ui, &vi);
                int b = project_f64(Hd, x, y, cams[v].width, cams[v].height, &uj, &vj);
                n_eval++;
                if (a != b || (a && (ui != uj || vi != vj))) n_bad++;
            }
        }
    }
    free(iz);
    out[0] = n_bad;
    out[1] = n_eval;
    return 0;
}

/* -------------------------------------------------------------------------------- temporal */

/*
 * Temporal consistency test of Sec. III-E for one view with the current frame's label map: for every
 * segment, the per-channel sums of the current frame over the segment's pixels are compared with the
 * sums of the previous frame and of the I frame over the same pixels. mode 0 compares Y only, mode 1
 * compares Y, Cb and Cr. mask[s] = 1 (adopt previous depth) if every compared channel satisfies
 * |S_cur - S_prev| < t_p * n, else 2 (adopt I-frame depth) if iframe is given and every channel
 * satisfies |S_cur - S_I| < t_i * n, else 0 (estimate again). Empty segments are 0. changed_list
 * receives the segments with mask 0 in increasing order and *n_changed their count.
 */
int or_temporal_mask(int W, int Hh, const int32_t* labels, int S, const or_image* cur, const or_image* prev,
                     const or_image* iframe, int sample_bytes, int t_p, int t_i, int mode, uint8_t* mask,
                     int32_t* changed_list, int32_t* n_changed) {
    if (!labels || S < 0 || !cur || !prev || !mask) return 1;
    int nch = mode == 1 ? 3 : 1;
    int64_t* n = (int64_t*)calloc((size_t)S + 1, sizeof(int64_t));
    int64_t* dp = (int64_t*)calloc((size_t)S * 3 + 1, sizeof(int64_t));
    int64_t* di = (int64_t*)calloc((size_t)S * 3 + 1, sizeof(int64_t));
    if (!n || !dp || !di) { free(n); free(dp); free(di); return 1; }
    for (int y = 0; y < Hh; y++)
        for (int x = 0; x < W; x++) {
            int s = labels[(size_t)y * W + x];
            if (s < 0 || s >= S) { free(n); free(dp); free(di); return 2; }
            n[s]++;
            for (int c = 0; c < nch; c++) {
                int a = sample_at(cur, sample_bytes, c, x, y);
                dp[(size_t)s * 3 + c] += a - sample_at(prev, sample_bytes, c, x, y);
                if (iframe) di[(size_t)s * 3 + c] += a - sample_at(iframe, sample_bytes, c, x, y);
            }
        }
    int32_t cnt = 0;
    for (int s = 0; s < S; s++) {
        int m = 0;
        if (n[s] > 0) {
            int okp = 1, oki = iframe != NULL;
            for (int c = 0; c < nch; c++) {
                int64_t a = dp[(size_t)s * 3 + c], b = di[(size_t)s * 3 + c];
                if (!((a < 0 ? -a : a) < (int64_t)t_p * n[s])) okp = 0;
                if (!((b < 0 ? -b : b) < (int64_t)t_i * n[s])) oki = 0;
            }
            m = okp ? 1 : (oki ? 2 : 0);
        }
        mask[s] = (uint8_t)m;
        if (m == 0) {
            if (changed_list) changed_list[cnt] = s;
            cnt++;
        }
    }
    if (n_changed) *n_changed = cnt;
    free(n);
    free(dp);
    free(di);
    return 0;
}

/* ------------------------------------------------------------------------------------- WTA */

/*
 * Winner-take-all readout: for each listed segment (all when seg_list is NULL) out[s] is the label
 * with the smallest cost, the smallest label on ties; with a mask, segments marked 1 take
 * prev_label[s] and segments marked 2 take iframe_label[s] instead (Sec. III-E adoption).
 */
int or_wta(const int32_t* cost, int S, int L, const uint8_t* mask, const uint16_t* prev_label,
           const uint16_t* iframe_label, const int32_t* seg_list, int n_list, uint16_t* out) {
    if (!cost || S < 0 || L < 1 || !out) return 1;
    int n = seg_list ? n_list : S;
    for (int i = 0; i < n; i++) {
        int s = seg_list ? seg_list[i] : i;
        if (s < 0 || s >= S) return 1;
        int m = mask ? mask[s] : 0;
        if (m == 1 && prev_label) { out[s] = prev_label[s]; continue; }
        if (m == 2 && iframe_label) { out[s] = iframe_label[s]; continue; }
        int best = 0;
        for (int d = 1; d < L; d++)
            if (cost[(size_t)s * L + d] < cost[(size_t)s * L + best]) best = d;
        out[s] = (uint16_t)best;
    }
    return 0;
}

/* Per-pixel depth map from per-segment labels: depth[p] = z of label[labels[p]] (FP64 1/iz rounded). */
int or_depth_map(int W, int Hh, const int32_t* labels, int S, const uint16_t* seg_label, int L, double z_near,
                 double z_far, float* depth) {
    double* iz = (double*)malloc(sizeof(double) * (size_t)L);
    if (!iz || or_label_inv_depths(L, z_near, z_far, iz)) { free(iz); return 1; }
    for (size_t p = 0; p < (size_t)W * Hh; p++) {
        int s = labels[p];
        if (s < 0 || s >= S || seg_label[s] >= L) { free(iz); return 2; }
        depth[p] = (float)(1.0 / iz[seg_label[s]]);
    }
    free(iz);
    return 0;
}

/* ----------------------------------------------------------------------------- centre table */

/*
 * Eq. 4 at segment centres and the correspondence that Eq. 5 needs (Sec. III-C): for reference `ref`,
 * every segment s, label d and neighbour k (view nbrs[k]):
 *   mu_s      the integer centroid of s: (floor((2 sum x + n) / (2 n)), floor((2 sum y + n) / (2 n)))
 *             over its n pixels (the paper does not define the centre; this is the rounded mean);
 *   T[mu_s]   mu_s projected with H[k][d] by the same FP32 sequence as the cost volume (or, with
 *             H = NULL, with the FP64 table H64 by the FP64 projection);
 *   m         sum over the window offsets w (window x window, odd) of the L1 distance of (Y, Cb, Cr)
 *             at mu_s + w in the reference and at T[mu_s] + w in view nbrs[k]; a pair with either
 *             position outside its image (or T[mu_s] out of view) costs the penalty. The paper's
 *             1/size(W) factor is left to the consumer (m_paper = m / window^2);
 *   s'        the label of view nbrs[k]'s own segmentation at T[mu_s], or -1 when T[mu_s] is out of
 *             view or that view has no label map (labels_views[v] == NULL).
 * Empty segments: every pair is out (m = window^2 * penalty), s' = -1.
 * Outputs are int32 [S][L][n_nbrs].
 */
int or_centre_table(const or_camera* cams, int n_views, const or_image* imgs, int sample_bytes, int ref, int n_nbrs,
                    const int32_t* nbrs, const float* H, const double* H64, int L, const int32_t* const* labels_views,
                    int S, int window, int penalty, int32_t* out_m, int32_t* out_sp) {
    if (!cams || !imgs || ref < 0 || ref >= n_views || !labels_views || !labels_views[ref] || S < 0 || L < 1)
        return 1;
    if (!H == !H64) return 1;
    if (window < 1 || (window & 1) == 0 || !out_m || !out_sp) return 1;
    const int W = cams[ref].width, Hh = cams[ref].height, half = window / 2;
    const int32_t* lab = labels_views[ref];
    int64_t* sx = (int64_t*)calloc((size_t)S + 1, sizeof(int64_t));
    int64_t* sy = (int64_t*)calloc((size_t)S + 1, sizeof(int64_t));
    int64_t* cnt = (int64_t*)calloc((size_t)S + 1, sizeof(int64_t));
    if (!sx || !sy || !cnt) { free(sx); free(sy); free(cnt); return 1; }
    for (int y = 0; y < Hh; y++)
        for (int x = 0; x < W; x++) {
            int s = lab[(size_t)y * W + x];
            if (s < 0 || s >= S) { free(sx); free(sy); free(cnt); return 2; }
            sx[s] += x;
            sy[s] += y;
            cnt[s]++;
        }
    for (int s = 0; s < S; s++) {
        int mx = 0, my = 0;
        if (cnt[s] > 0) {
            mx = (int)((2 * sx[s] + cnt[s]) / (2 * cnt[s]));
            my = (int)((2 * sy[s] + cnt[s]) / (2 * cnt[s]));
        }
        for (int d = 0; d < L; d++)
            for (int k = 0; k < n_nbrs; k++) {
                int v = nbrs[k];
                const size_t ho = ((size_t)k * L + d) * 9;
                int ui = 0, vi = 0, in = 0;
                if (cnt[s] > 0 && H64) {
                    long lu = 0, lv = 0;
                    in = project_f64(H64 + ho, mx, my, cams[v].width, cams[v].height, &lu, &lv);
                    ui = (int)lu;
                    vi = (int)lv;
                } else if (cnt[s] > 0) {
                    in = project_f32(H + ho, mx, my, cams[v].width, cams[v].height, &ui, &vi);
                }
                int64_t m = 0;
                for (int dy = -half; dy <= half; dy++)
                    for (int dx = -half; dx <= half; dx++) {
                        int rx = mx + dx, ry = my + dy, qx = ui + dx, qy = vi + dy;
                        if (!in || rx < 0 || rx >= W || ry < 0 || ry >= Hh || qx < 0 || qx >= cams[v].width || qy < 0 ||
                            qy >= cams[v].height) {
                            m += penalty;
                            continue;
                        }
                        for (int ch = 0; ch < 3; ch++) {
                            int a = sample_at(&imgs[ref], sample_bytes, ch, rx, ry);
                            int b = sample_at(&imgs[v], sample_bytes, ch, qx, qy);
                            m += a > b ? a - b : b - a;
                        }
                    }
                size_t o = ((size_t)s * L + d) * n_nbrs + k;
                out_m[o] = (int32_t)m;
                out_sp[o] = (in && labels_views[v]) ? labels_views[v][(size_t)vi * cams[v].width + ui] : -1;
            }
    }
    free(sx);
    free(sy);
    free(cnt);
    return 0;
}

/* -------------------------------------------------------------------- adjacency and beta */

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/*
 * Intra-view discontinuity weights of Eq. 2-3 (Sec. III-D): the segments s < t that are adjacent (some
 * pixel of s and some pixel of t are neighbours: 4-connected, or 8-connected with connectivity 8),
 * listed in increasing (s, t) order, and for each edge beta = beta0 / || mean_s - mean_t ||_1, the
 * L1 distance of the segments' mean (Y, Cb, Cr) vectors in this frame. The paper leaves a zero
 * distance open: the distance is floored at min_diff (a distance below it counts as min_diff). With
 * per-channel sums S and counts n the distance is sum_c |S_cs n_t - S_ct n_s| / (n_s n_t), evaluated
 * as beta = beta0 * (n_s n_t) / num in double (num the exact int64 numerator), and rounded to float.
 * Returns the number of edges in *n_edges (at most cap are written).
 */
int or_adjacency(int W, int Hh, const int32_t* labels, int S, const or_image* frame, int sample_bytes,
                 int connectivity, double beta0, double min_diff, int cap, int32_t* edge_s, int32_t* edge_t,
                 float* beta, int32_t* n_edges) {
    if (!labels || S < 0 || !frame || (connectivity != 4 && connectivity != 8) || !n_edges) return 1;
    size_t P = (size_t)W * Hh, maxp = P * 4 + 1, np = 0;
    uint64_t* pairs = (uint64_t*)malloc(sizeof(uint64_t) * maxp);
    int64_t* sum = (int64_t*)calloc((size_t)S * 4 + 4, sizeof(int64_t));
    if (!pairs || !sum) { free(pairs); free(sum); return 1; }
    static const int dxs[4] = {1, 0, 1, -1}, dys[4] = {0, 1, 1, 1};
    int ndir = connectivity == 8 ? 4 : 2;
    for (int y = 0; y < Hh; y++)
        for (int x = 0; x < W; x++) {
            int s = labels[(size_t)y * W + x];
            if (s < 0 || s >= S) { free(pairs); free(sum); return 2; }
            sum[(size_t)s * 4 + 0]++;
            for (int c = 0; c < 3; c++) sum[(size_t)s * 4 + 1 + c] += sample_at(frame, sample_bytes, c, x, y);
            for (int k = 0; k < ndir; k++) {
                int qx = x + dxs[k], qy = y + dys[k];
                if (qx < 0 || qx >= W || qy < 0 || qy >= Hh) continue;
                int t = labels[(size_t)qy * W + qx];
                if (t < 0 || t >= S) { free(pairs); free(sum); return 2; }
                if (t == s) continue;
                uint64_t a = (uint64_t)(s < t ? s : t), b = (uint64_t)(s < t ? t : s);
                pairs[np++] = (a << 32) | b;
            }
        }
    qsort(pairs, np, sizeof(uint64_t), cmp_u64);
    int32_t e = 0;
    for (size_t i = 0; i < np; i++) {
        if (i > 0 && pairs[i] == pairs[i - 1]) continue;
        int s = (int)(pairs[i] >> 32), t = (int)(pairs[i] & 0xffffffffu);
        if (e < cap) {
            const int64_t* a = &sum[(size_t)s * 4];
            const int64_t* b = &sum[(size_t)t * 4];
            int64_t num = 0;
            for (int c = 1; c <= 3; c++) {
                int64_t d = a[c] * b[0] - b[c] * a[0];
                num += d < 0 ? -d : d;
            }
            double den = (double)(a[0] * b[0]);
            double dist = (double)num / den;
            double bt = dist < min_diff ? beta0 / min_diff : (beta0 * den) / (double)num;
            if (edge_s) edge_s[e] = s;
            if (edge_t) edge_t[e] = t;
            if (beta) beta[e] = (float)bt;
        }
        e++;
    }
    *n_edges = e;
    free(pairs);
    free(sum);
    return 0;
}

/* ------------------------------------------------------------------ superpixel segmentation */

/*
 * Segmentation (Sec. IV-C): the label maps the method consumes come from SNIC superpixels computed in
 * (Y, Cb, Cr) with compactness factor m = 5 and 8-connected segments. The paper gives no more; the
 * readings both functions below share are:
 *  - seeds lie on an S x S grid: cell (i, j) covers x in [iS, min(iS + S, W)) and y in
 *    [jS, min(jS + S, H)), has label j * ceil(W / S) + i, and its seed is the cell's middle pixel
 *    (iS + (w - 1) / 2, jS + (h - 1) / 2) with w, h the cell's width and height;
 *  - the distance of pixel p to a cluster with mean position x_k and mean colour c_k is SNIC's (and
 *    SLIC's) weighting of colour against space, squared and multiplied by S^2:
 *        D = S^2 * ||c_p - c_k||^2 + m^2 * ||x_p - x_k||^2,
 *    with colours on the 8-bit scale: for bit depth bd > 8 the spatial term is multiplied by
 *    4^(bd - 8) instead of dividing the colours, for bd < 8 the colour term by 4^(8 - bd).
 */
static void grid_dims(int W, int Hh, int S, int* gw, int* gh) {
    *gw = (W + S - 1) / S;
    *gh = (Hh + S - 1) / S;
}

static int seed_coord(int n, int S, int i) {
    int w = n - i * S < S ? n - i * S : S;
    return i * S + (w - 1) / 2;
}

static void dist_weights(int S, int m, int bd, uint64_t* wc, uint64_t* ws) {
    *wc = (uint64_t)S * (uint64_t)S;
    *ws = (uint64_t)m * (uint64_t)m;
    if (bd > 8) *ws <<= 2 * (bd - 8);
    if (bd < 8) *wc <<= 2 * (8 - bd);
}

/* --- sequential SNIC (the segmentation the paper uses), for quality comparison only --- */

typedef struct {
    double d;
    int64_t seq;
    int32_t x, y, k;
} snic_elem;

static int elem_less(const snic_elem* a, const snic_elem* b) {
    return a->d < b->d || (a->d == b->d && a->seq < b->seq);
}

static void heap_push(snic_elem* h, size_t* n, snic_elem e) {
    size_t i = (*n)++;
    h[i] = e;
    while (i > 0) {
        size_t p = (i - 1) / 2;
        if (!elem_less(&h[i], &h[p])) break;
        snic_elem t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static snic_elem heap_pop(snic_elem* h, size_t* n) {
    snic_elem top = h[0];
    h[0] = h[--(*n)];
    size_t i = 0;
    for (;;) {
        size_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < *n && elem_less(&h[l], &h[s])) s = l;
        if (r < *n && elem_less(&h[r], &h[s])) s = r;
        if (s == i) break;
        snic_elem t = h[i]; h[i] = h[s]; h[s] = t;
        i = s;
    }
    return top;
}

/*
 * SNIC (Achanta and Suesstrunk, CVPR 2017), as Sec. IV-C uses it: every seed enters a priority queue
 * with distance 0; repeatedly the element of least distance (earliest pushed on ties) is taken, and if
 * its pixel has no label yet the pixel joins the element's cluster, the cluster's running mean of
 * position and colour absorbs it, and each unlabelled 8-neighbour is pushed with its distance D (in
 * double, exact means) to that cluster. Labels are the grid labels; every pixel ends labelled.
 */
int or_snic(int W, int Hh, const or_image* img, int sample_bytes, int bit_depth, int S, int m, int32_t* labels) {
    if (W < 1 || Hh < 1 || !img || !labels || S < 1 || m < 0) return 1;
    int gw, gh;
    grid_dims(W, Hh, S, &gw, &gh);
    int K = gw * gh;
    uint64_t wc, ws;
    dist_weights(S, m, bit_depth, &wc, &ws);
    size_t P = (size_t)W * Hh, cap = 8 * P + (size_t)K + 1, n = 0;
    snic_elem* heap = (snic_elem*)malloc(sizeof(snic_elem) * cap);
    double* acc = (double*)calloc((size_t)K * 6, sizeof(double)); /* n, sx, sy, sY, sCb, sCr */
    if (!heap || !acc) { free(heap); free(acc); return 1; }
    for (size_t p = 0; p < P; p++) labels[p] = -1;
    int64_t seq = 0;
    for (int j = 0; j < gh; j++)
        for (int i = 0; i < gw; i++) {
            snic_elem e = {0.0, seq++, seed_coord(W, S, i), seed_coord(Hh, S, j), j * gw + i};
            heap_push(heap, &n, e);
        }
    while (n > 0) {
        snic_elem e = heap_pop(heap, &n);
        size_t p = (size_t)e.y * W + e.x;
        if (labels[p] >= 0) continue;
        labels[p] = e.k;
        double* a = &acc[(size_t)e.k * 6];
        a[0] += 1.0;
        a[1] += e.x;
        a[2] += e.y;
        for (int c = 0; c < 3; c++) a[3 + c] += sample_at(img, sample_bytes, c, e.x, e.y);
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int qx = e.x + dx, qy = e.y + dy;
                if ((dx == 0 && dy == 0) || qx < 0 || qx >= W || qy < 0 || qy >= Hh) continue;
                if (labels[(size_t)qy * W + qx] >= 0) continue;
                double ex = qx - a[1] / a[0], ey = qy - a[2] / a[0], dc = 0.0;
                for (int c = 0; c < 3; c++) {
                    double t = sample_at(img, sample_bytes, c, qx, qy) - a[3 + c] / a[0];
                    dc += t * t;
                }
                snic_elem q = {(double)wc * dc + (double)ws * (ex * ex + ey * ey), seq++, qx, qy, e.k};
                if (n < cap) heap_push(heap, &n, q);
            }
    }
    free(heap);
    free(acc);
    return 0;
}

/* --- the data-parallel reformulation the GPU computes --- */

/* union-find over component names: the root of a set is its smallest name */
static int32_t uf_find(int32_t* par, int32_t x) {
    while (par[x] != x) x = par[x];
    return x;
}

/*
 * Connectivity step: makes every label's pixel set 8-connected (Sec. IV-C asks for 8-connected
 * segments; SNIC's growth gives them by construction, a data-parallel clustering does not).
 *  - Components are the maximal 8-connected sets of equally labelled pixels, named by their first
 *    pixel in raster order.
 *  - A label's main component is its largest (the earliest named on ties). Main components are
 *    anchored groups that keep their label; every other component starts as an unanchored group.
 *  - A group's mean colour is M_c = floor((32 S_c + n) / (2 n)) per channel (n pixels, channel
 *    sums S_c), in 1/16 units.
 *  - In a round, every unanchored group g picks, among the groups with a pixel 8-adjacent to a pixel
 *    of g, the group h of least sum_c |M_c(g) - M_c(h)| (the smallest name on ties). All picked
 *    pairs are merged at once; a merged group is named by its smallest member name and, if it holds
 *    an anchored group (at most one: only unanchored groups pick), is anchored with that label.
 *  - Rounds repeat until every group is anchored (each round at least halves the unanchored groups);
 *    every pixel then takes its group's label.
 * Labels must lie in [0, K).
 */
int or_connectivity(int W, int Hh, int32_t* labels, int K, const or_image* img, int sample_bytes) {
    if (W < 1 || Hh < 1 || !labels || K < 1 || !img) return 1;
    size_t P = (size_t)W * Hh;
    for (size_t p = 0; p < P; p++)
        if (labels[p] < 0 || labels[p] >= K) return 2;
    int32_t* comp = (int32_t*)malloc(sizeof(int32_t) * P);
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * P);
    int32_t* size = (int32_t*)calloc(P, sizeof(int32_t));
    int32_t* main_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
    int32_t* grp = (int32_t*)malloc(sizeof(int32_t) * P);  /* group of each component name */
    int32_t* par = (int32_t*)malloc(sizeof(int32_t) * P);  /* union-find over group names */
    int32_t* glab = (int32_t*)malloc(sizeof(int32_t) * P); /* label of an anchored group, -1 if none */
    int64_t* gsum = (int64_t*)malloc(sizeof(int64_t) * P * 4);
    int64_t* best = (int64_t*)malloc(sizeof(int64_t) * P * 2); /* (distance, name) picked by a group */
    if (!comp || !stack || !size || !main_of || !grp || !par || !glab || !gsum || !best) {
        free(comp); free(stack); free(size); free(main_of); free(grp); free(par); free(glab); free(gsum); free(best);
        return 1;
    }
    for (size_t p = 0; p < P; p++) comp[p] = -1;
    /* flood fill in raster order: the seed pixel of each fill is its component's first pixel */
    for (size_t p0 = 0; p0 < P; p0++) {
        if (comp[p0] >= 0) continue;
        size_t top = 0;
        comp[p0] = (int32_t)p0;
        stack[top++] = (int32_t)p0;
        while (top > 0) {
            int32_t p = stack[--top];
            size[p0]++;
            int x = p % W, y = p / W;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int qx = x + dx, qy = y + dy;
                    if (qx < 0 || qx >= W || qy < 0 || qy >= Hh) continue;
                    size_t q = (size_t)qy * W + qx;
                    if (comp[q] >= 0 || labels[q] != labels[p0]) continue;
                    comp[q] = (int32_t)p0;
                    stack[top++] = (int32_t)q;
                }
        }
    }
    for (int k = 0; k < K; k++) main_of[k] = -1;
    for (size_t r = 0; r < P; r++) {
        if (comp[r] != (int32_t)r) continue;
        int k = labels[r];
        if (main_of[k] < 0 || size[r] > size[main_of[k]]) main_of[k] = (int32_t)r; /* raster order: earliest on ties */
    }
    for (size_t r = 0; r < P; r++) {
        grp[r] = comp[r] == (int32_t)r ? (int32_t)r : -1;
        glab[r] = (comp[r] == (int32_t)r && main_of[labels[r]] == (int32_t)r) ? labels[r] : -1;
    }
    int rc = 0;
    for (int round = 0;; round++) {
        int unanchored = 0;
        for (size_t r = 0; r < P; r++)
            if (grp[r] == (int32_t)r && glab[r] < 0) unanchored++;
        if (unanchored == 0) break;
        if (round > 64) { rc = 3; break; } /* cannot happen: each round at least halves the count */
        memset(gsum, 0, sizeof(int64_t) * P * 4);
        for (size_t p = 0; p < P; p++) {
            int64_t* g = &gsum[(size_t)grp[comp[p]] * 4];
            int x = (int)(p % W), y = (int)(p / W);
            g[0]++;
            for (int c = 0; c < 3; c++) g[1 + c] += sample_at(img, sample_bytes, c, x, y);
        }
        for (size_t r = 0; r < P; r++) best[2 * r] = -1;
        for (size_t p = 0; p < P; p++) {
            int32_t a = grp[comp[p]];
            if (glab[a] >= 0) continue;
            int x = (int)(p % W), y = (int)(p / W);
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int qx = x + dx, qy = y + dy;
                    if (qx < 0 || qx >= W || qy < 0 || qy >= Hh) continue;
                    int32_t b = grp[comp[(size_t)qy * W + qx]];
                    if (b == a) continue;
                    const int64_t* sa = &gsum[(size_t)a * 4];
                    const int64_t* sb = &gsum[(size_t)b * 4];
                    int64_t d = 0;
                    for (int c = 1; c <= 3; c++) {
                        int64_t ma = (32 * sa[c] + sa[0]) / (2 * sa[0]), mb = (32 * sb[c] + sb[0]) / (2 * sb[0]);
                        d += ma > mb ? ma - mb : mb - ma;
                    }
                    int64_t* bt = &best[2 * (size_t)a];
                    if (bt[0] < 0 || d < bt[0] || (d == bt[0] && b < bt[1])) { bt[0] = d; bt[1] = b; }
                }
        }
        /* merge every picked pair at once */
        for (size_t r = 0; r < P; r++) par[r] = (int32_t)r;
        for (size_t r = 0; r < P; r++) {
            if (grp[r] != (int32_t)r || glab[r] >= 0 || best[2 * r] < 0) continue;
            int32_t u = uf_find(par, (int32_t)r), v = uf_find(par, (int32_t)best[2 * r + 1]);
            if (u < v) par[v] = u;
            else if (v < u) par[u] = v;
        }
        for (size_t r = 0; r < P; r++) {
            if (grp[r] != (int32_t)r || glab[r] < 0) continue;
            int32_t t = uf_find(par, (int32_t)r);
            glab[t] = glab[r]; /* the merged group holds this anchored group only */
        }
        for (size_t r = 0; r < P; r++)
            if (grp[r] >= 0) grp[r] = uf_find(par, grp[r]);
    }
    if (rc == 0)
        for (size_t p = 0; p < P; p++) labels[p] = glab[grp[comp[p]]];
    free(comp); free(stack); free(size); free(main_of); free(grp); free(par); free(glab); free(gsum); free(best);
    return rc;
}

/*
 * Grid-seeded clustering with SNIC's distance, in passes that parallelise (the GPU's reformulation of
 * Sec. IV-C's segmentation; SNIC's single priority queue does not).
 *  - Cluster k starts at its seed pixel: mean position and colour are those of the pixel.
 *  - Means are kept in fixed point with 4 fractional bits: M = floor((32 * sum + n) / (2 n)), the
 *    nearest multiple of 1/16 (halves rounded up); D is then evaluated exactly in 64-bit integers on
 *    16 * (pixel value) - M.
 *  - Assignment pass: a pixel in grid cell (i, j) joins the cluster of least D among the cells
 *    (i + a, j + b), a, b in {-1, 0, 1}, that exist; ties go to the smallest label.
 *  - Update: each cluster's mean becomes that of its assigned pixels; a cluster with no pixel keeps it.
 *  - `iterations` assignment passes run with an update between consecutive passes; the last pass's
 *    assignment is the clustering, and `connect` then applies or_connectivity.
 */
int or_superpixels(int W, int Hh, const or_image* img, int sample_bytes, int bit_depth, int S, int m,
                   int iterations, int connect, int32_t* labels) {
    if (W < 1 || Hh < 1 || !img || !labels || S < 1 || m < 0 || iterations < 1) return 1;
    int gw, gh;
    grid_dims(W, Hh, S, &gw, &gh);
    int K = gw * gh;
    uint64_t wc, ws;
    dist_weights(S, m, bit_depth, &wc, &ws);
    int64_t* mean = (int64_t*)malloc(sizeof(int64_t) * (size_t)K * 5); /* 16x: x, y, Y, Cb, Cr */
    int64_t* sum = (int64_t*)malloc(sizeof(int64_t) * (size_t)K * 6);  /* n, x, y, Y, Cb, Cr */
    if (!mean || !sum) { free(mean); free(sum); return 1; }
    for (int j = 0; j < gh; j++)
        for (int i = 0; i < gw; i++) {
            int64_t* M = &mean[((size_t)j * gw + i) * 5];
            int sx = seed_coord(W, S, i), sy = seed_coord(Hh, S, j);
            M[0] = 16 * (int64_t)sx;
            M[1] = 16 * (int64_t)sy;
            for (int c = 0; c < 3; c++) M[2 + c] = 16 * (int64_t)sample_at(img, sample_bytes, c, sx, sy);
        }
    for (int it = 0; it < iterations; it++) {
        for (int y = 0; y < Hh; y++)
            for (int x = 0; x < W; x++) {
                int ci = x / S, cj = y / S, best = -1;
                uint64_t bestD = 0;
                int64_t v[5] = {16 * (int64_t)x, 16 * (int64_t)y, 0, 0, 0};
                for (int c = 0; c < 3; c++) v[2 + c] = 16 * (int64_t)sample_at(img, sample_bytes, c, x, y);
                for (int b = -1; b <= 1; b++)
                    for (int a = -1; a <= 1; a++) {
                        int i = ci + a, j = cj + b;
                        if (i < 0 || i >= gw || j < 0 || j >= gh) continue;
                        int k = j * gw + i;
                        const int64_t* M = &mean[(size_t)k * 5];
                        uint64_t dsp = 0, dcol = 0;
                        for (int t = 0; t < 2; t++) dsp += (uint64_t)((v[t] - M[t]) * (v[t] - M[t]));
                        for (int t = 2; t < 5; t++) dcol += (uint64_t)((v[t] - M[t]) * (v[t] - M[t]));
                        uint64_t D = wc * dcol + ws * dsp;
                        if (best < 0 || D < bestD) { best = k; bestD = D; } /* labels visited in increasing order */
                    }
                labels[(size_t)y * W + x] = best;
            }
        if (it + 1 == iterations) break;
        memset(sum, 0, sizeof(int64_t) * (size_t)K * 6);
        for (int y = 0; y < Hh; y++)
            for (int x = 0; x < W; x++) {
                int64_t* s = &sum[(size_t)labels[(size_t)y * W + x] * 6];
                s[0] += 1;
                s[1] += x;
                s[2] += y;
                for (int c = 0; c < 3; c++) s[3 + c] += sample_at(img, sample_bytes, c, x, y);
            }
        for (int k = 0; k < K; k++) {
            const int64_t* s = &sum[(size_t)k * 6];
            if (s[0] == 0) continue;
            for (int t = 0; t < 5; t++) mean[(size_t)k * 5 + t] = (32 * s[1 + t] + s[0]) / (2 * s[0]);
        }
    }
    free(mean);
    free(sum);
    return connect ? or_connectivity(W, Hh, labels, K, img, sample_bytes) : 0;
}
