/*
 * Seeded synthetic multiview scenes: a CPU ray-caster of textured planes.
 *
 * This is input generation only. It stands in for the multiview test sequences that the paper
 * measures on (Table I) and that are not available here. It holds none of the depth estimator's
 * arithmetic: it never forms a plane homography and never computes a matching cost. Both the CUDA
 * library and the CPU oracle consume the images it writes.
 *
 * Camera convention: X_cam = R * X_world + t; pixel centres sit at integer coordinates; the ray of
 * pixel (x, y) has camera-frame direction K^-1 (x, y, 1).
 *
 * Every random draw is a pure function of (seed, integer coordinates), so a pixel's colour does not
 * depend on the thread count or on which pixels are rendered.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double K[9], R[9], t[3];
    int32_t width, height;
} syn_camera;

typedef struct {
    double p0[3];          /* a point on the plane (world), centre of a bounded plane */
    double e1[3], e2[3];   /* orthonormal in-plane axes (world); normal = e1 x e2 */
    double half1, half2;   /* half extents along e1 / e2; <= 0 means unbounded */
    double texel;          /* world size of one texture cell (world-texture mode) */
    uint64_t seed;         /* texture seed */
    int32_t mode;          /* 0: world texture on the plane; 1: painted from the paint camera */
    int32_t pad;
} syn_plane;

typedef struct {
    const syn_camera* cam;
    const syn_camera* paint;
    int n_planes;
    const syn_plane* planes;
    const double* offsets; /* [n_planes][3] world translation of each plane for this frame, or NULL */
    int bit_depth;
    double noise_sigma;
    double specular_frac;
    uint64_t noise_seed;
    int chroma420;
    uint16_t *Y, *U, *V;
    float* depth;
    int32_t* plane_id;
    int row0, row1;
} syn_job;

static uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t hash4(uint64_t seed, int64_t a, int64_t b, int64_t c) {
    uint64_t h = mix64(seed ^ 0x5851f42d4c957f2dULL);
    h = mix64(h ^ (uint64_t)a);
    h = mix64(h ^ (uint64_t)b);
    h = mix64(h ^ (uint64_t)c);
    return h;
}

/* uniform double in [0, 1) from 53 hash bits */
static double unit(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

static void cam_centre(const syn_camera* c, double C[3]) {
    /* C = -R^T t */
    for (int i = 0; i < 3; i++)
        C[i] = -(c->R[0 * 3 + i] * c->t[0] + c->R[1 * 3 + i] * c->t[1] + c->R[2 * 3 + i] * c->t[2]);
}

/* Solve K d = (x, y, 1) for an upper-triangular K with K[8] == 1. */
static void back_dir(const syn_camera* c, double x, double y, double d[3]) {
    const double* K = c->K;
    double dy = (y - K[5]) / K[4];
    double dx = (x - K[2] - K[1] * dy) / K[0];
    d[0] = dx;
    d[1] = dy;
    d[2] = 1.0;
}

/* Project a world point; returns 0 when the point is not in front of the camera. */
static int project(const syn_camera* c, const double P[3], double* u, double* v) {
    double Xc[3];
    for (int i = 0; i < 3; i++)
        Xc[i] = c->R[i * 3 + 0] * P[0] + c->R[i * 3 + 1] * P[1] + c->R[i * 3 + 2] * P[2] + c->t[i];
    if (!(Xc[2] > 0)) return 0;
    const double* K = c->K;
    double xn = Xc[0] / Xc[2], yn = Xc[1] / Xc[2];
    *u = K[0] * xn + K[1] * yn + K[2];
    *v = K[4] * yn + K[5];
    return 1;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Colour of the nearest plane hit by the ray of pixel (x, y); returns the plane index or -1. */
static int shade(const syn_job* j, double x, double y, int px, int py, int vals[3], double* zc) {
    const syn_camera* cam = j->cam;
    double C[3], dc[3], dw[3];
    cam_centre(cam, C);
    back_dir(cam, x, y, dc);
    for (int i = 0; i < 3; i++)
        dw[i] = cam->R[0 * 3 + i] * dc[0] + cam->R[1 * 3 + i] * dc[1] + cam->R[2 * 3 + i] * dc[2];
    int best = -1;
    double best_l = INFINITY, bq[3] = {0, 0, 0};
    for (int k = 0; k < j->n_planes; k++) {
        const syn_plane* pl = &j->planes[k];
        double p0[3];
        for (int i = 0; i < 3; i++) p0[i] = pl->p0[i] + (j->offsets ? j->offsets[k * 3 + i] : 0.0);
        double n[3] = {pl->e1[1] * pl->e2[2] - pl->e1[2] * pl->e2[1],
                       pl->e1[2] * pl->e2[0] - pl->e1[0] * pl->e2[2],
                       pl->e1[0] * pl->e2[1] - pl->e1[1] * pl->e2[0]};
        double den = n[0] * dw[0] + n[1] * dw[1] + n[2] * dw[2];
        if (fabs(den) < 1e-15) continue;
        double num = n[0] * (p0[0] - C[0]) + n[1] * (p0[1] - C[1]) + n[2] * (p0[2] - C[2]);
        double lam = num / den;
        if (!(lam > 1e-9) || !(lam < best_l)) continue;
        double Q[3] = {C[0] + lam * dw[0], C[1] + lam * dw[1], C[2] + lam * dw[2]};
        double a = (Q[0] - p0[0]) * pl->e1[0] + (Q[1] - p0[1]) * pl->e1[1] + (Q[2] - p0[2]) * pl->e1[2];
        double b = (Q[0] - p0[0]) * pl->e2[0] + (Q[1] - p0[1]) * pl->e2[1] + (Q[2] - p0[2]) * pl->e2[2];
        if (pl->half1 > 0 && fabs(a) > pl->half1) continue;
        if (pl->half2 > 0 && fabs(b) > pl->half2) continue;
        best = k;
        best_l = lam;
        bq[0] = Q[0]; bq[1] = Q[1]; bq[2] = Q[2];
    }
    const int vmax = (1 << j->bit_depth) - 1;
    if (best < 0) {
        vals[0] = vals[1] = vals[2] = 0;
        *zc = 0.0;
        return -1;
    }
    *zc = best_l; /* dc[2] == 1, so the ray parameter is the camera-frame depth */
    const syn_plane* pl = &j->planes[best];
    int64_t ia, ib;
    if (pl->mode == 1 && j->paint) {
        double u, v;
        if (project(j->paint, bq, &u, &v)) {
            ia = (int64_t)floor(u + 0.5);
            ib = (int64_t)floor(v + 0.5);
        } else {
            ia = ib = INT64_MIN / 2;
        }
    } else {
        double p0[3];
        for (int i = 0; i < 3; i++) p0[i] = pl->p0[i] + (j->offsets ? j->offsets[best * 3 + i] : 0.0);
        double a = (bq[0] - p0[0]) * pl->e1[0] + (bq[1] - p0[1]) * pl->e1[1] + (bq[2] - p0[2]) * pl->e1[2];
        double b = (bq[0] - p0[0]) * pl->e2[0] + (bq[1] - p0[1]) * pl->e2[1] + (bq[2] - p0[2]) * pl->e2[2];
        ia = (int64_t)floor(a / pl->texel);
        ib = (int64_t)floor(b / pl->texel);
    }
    for (int c = 0; c < 3; c++) vals[c] = (int)(hash4(pl->seed, ia, ib, c) % (uint64_t)(vmax + 1));
    (void)px; (void)py;
    return best;
}

static void* render_rows(void* arg) {
    syn_job* j = (syn_job*)arg;
    const int W = j->cam->width, H = j->cam->height;
    const int vmax = (1 << j->bit_depth) - 1;
    for (int y = j->row0; y < j->row1; y++) {
        for (int x = 0; x < W; x++) {
            int vals[3];
            double zc;
            int pid = shade(j, (double)x, (double)y, x, y, vals, &zc);
            if (j->chroma420) {
                /* chroma of a 2x2 block is the chroma seen at its top-left pixel, replicated */
                int cx = x & ~1, cy = y & ~1;
                if (cx != x || cy != y) {
                    int cv[3];
                    double zz;
                    shade(j, (double)cx, (double)cy, cx, cy, cv, &zz);
                    vals[1] = cv[1];
                    vals[2] = cv[2];
                }
            }
            size_t p = (size_t)y * W + x;
            if (j->noise_sigma > 0) {
                for (int c = 0; c < 3; c++) {
                    uint64_t h1 = hash4(j->noise_seed, (int64_t)p, c, 1);
                    uint64_t h2 = hash4(j->noise_seed, (int64_t)p, c, 2);
                    double u1 = unit(h1), u2 = unit(h2);
                    if (u1 < 1e-300) u1 = 1e-300;
                    double g = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
                    vals[c] = clampi((int)floor(vals[c] + j->noise_sigma * g + 0.5), 0, vmax);
                }
            }
            if (j->specular_frac > 0) {
                uint64_t h = hash4(j->noise_seed, (int64_t)p, 7, 3);
                if (unit(h) < j->specular_frac) {
                    int lo = vmax - (vmax + 1) / 8;
                    uint64_t h2 = hash4(j->noise_seed, (int64_t)p, 7, 4);
                    vals[0] = lo + (int)(h2 % (uint64_t)(vmax - lo + 1));
                }
            }
            j->Y[p] = (uint16_t)vals[0];
            j->U[p] = (uint16_t)vals[1];
            j->V[p] = (uint16_t)vals[2];
            if (j->depth) j->depth[p] = (float)zc;
            if (j->plane_id) j->plane_id[p] = pid;
        }
    }
    return NULL;
}

/* Render one view. Returns 0 on success. */
int syn_render(const syn_camera* cam, const syn_camera* paint, int n_planes, const syn_plane* planes,
               const double* offsets, int bit_depth, double noise_sigma, double specular_frac,
               uint64_t noise_seed, int chroma420, uint16_t* Y, uint16_t* U, uint16_t* V, float* depth,
               int32_t* plane_id, int n_threads) {
    if (!cam || !Y || !U || !V || bit_depth < 1 || bit_depth > 16 || n_planes < 0) return 1;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    const int H = cam->height;
    if (n_threads > H) n_threads = H > 0 ? H : 1;
    syn_job jobs[256];
    pthread_t th[256];
    for (int i = 0; i < n_threads; i++) {
        syn_job* j = &jobs[i];
        j->cam = cam;
        j->paint = paint;
        j->n_planes = n_planes;
        j->planes = planes;
        j->offsets = offsets;
        j->bit_depth = bit_depth;
        j->noise_sigma = noise_sigma;
        j->specular_frac = specular_frac;
        j->noise_seed = noise_seed;
        j->chroma420 = chroma420;
        j->Y = Y;
        j->U = U;
        j->V = V;
        j->depth = depth;
        j->plane_id = plane_id;
        j->row0 = (int)((int64_t)H * i / n_threads);
        j->row1 = (int)((int64_t)H * (i + 1) / n_threads);
    }
    int started = 0;
    for (int i = 1; i < n_threads; i++) {
        if (pthread_create(&th[i], NULL, render_rows, &jobs[i]) != 0) break;
        started = i;
    }
    render_rows(&jobs[0]);
    for (int i = started + 1; i < n_threads; i++) render_rows(&jobs[i]);
    for (int i = 1; i <= started; i++) pthread_join(th[i], NULL);
    return 0;
}

/* Grid label map: cells of `cell` pixels whose row and column boundaries are each shifted by a seeded
 * integer in [-jitter, jitter]. Segment id = row * n_cols + col. Returns the segment count. */
int syn_grid_labels(int W, int H, int cell, int jitter, uint64_t seed, int32_t* labels) {
    if (W <= 0 || H <= 0 || cell <= 0 || jitter < 0 || 2 * jitter >= cell) return -1;
    int nc = (W + cell - 1) / cell, nr = (H + cell - 1) / cell;
    int* xb = (int*)malloc(sizeof(int) * (nc + 1));
    int* yb = (int*)malloc(sizeof(int) * (nr + 1));
    if (!xb || !yb) { free(xb); free(yb); return -1; }
    for (int k = 0; k <= nc; k++) {
        int j = (int)(hash4(seed, 0, k, 0) % (uint64_t)(2 * jitter + 1)) - jitter;
        xb[k] = (k == 0) ? 0 : (k == nc ? W : k * cell + j);
    }
    for (int k = 0; k <= nr; k++) {
        int j = (int)(hash4(seed, 1, k, 0) % (uint64_t)(2 * jitter + 1)) - jitter;
        yb[k] = (k == 0) ? 0 : (k == nr ? H : k * cell + j);
    }
    /* keep boundaries inside the image and strictly increasing */
    for (int k = 1; k < nc; k++) { if (xb[k] > W - 1) xb[k] = W - 1; if (xb[k] <= xb[k - 1]) xb[k] = xb[k - 1] + 1; }
    for (int k = 1; k < nr; k++) { if (yb[k] > H - 1) yb[k] = H - 1; if (yb[k] <= yb[k - 1]) yb[k] = yb[k - 1] + 1; }
    int r = 0;
    for (int y = 0; y < H; y++) {
        while (r + 1 < nr && y >= yb[r + 1]) r++;
        int c = 0;
        for (int x = 0; x < W; x++) {
            while (c + 1 < nc && x >= xb[c + 1]) c++;
            labels[(size_t)y * W + x] = r * nc + c;
        }
    }
    free(xb);
    free(yb);
    return nr * nc;
}
