// Host geometry: candidate depths and plane homographies in FP64 (the library's only FP64 step).
//
// Paper: Eq. 4's transform T[.] "obtained from intrinsic and extrinsic parameters" maps the centre of a
// segment into a neighbouring view for the considered depth; Sec. IV-A: depth levels are planes
// parallel to the camera plane; Sec. III-B: for non-parallel optical axes depth is measured from the
// plane of the centre camera. For a plane n^T X_r = delta in the reference frame the transform is the
// homography H = K_v (R_vr + t_vr n^T / delta) K_r^-1 with R_vr = R_v R_r^T, t_vr = t_v - R_vr t_r.
// The operation order below is fixed (and documented in ftv.h) so that the FP32 rounding of each
// entry is reproducible by any implementation that follows the same order.
#include <cmath>
#include <vector>

#include "ftv_internal.h"

namespace ftv {

bool label_inv_depths(int L, double z_near, double z_far, std::vector<double>& iz) {
    if (L < 1 || !(z_near > 0.0) || !(z_far > z_near)) return false;
    iz.assign(L, 0.0);
    const double a = 1.0 / z_far;
    const double b = 1.0 / z_near;
    if (L == 1) {
        iz[0] = a;
        return true;
    }
    const double step = (b - a) / static_cast<double>(L - 1);
    for (int d = 0; d < L; ++d) iz[d] = a + static_cast<double>(d) * step;
    return true;
}

namespace {

// 3-term dot product summed left to right.
inline double dot3(double a0, double b0, double a1, double b1, double a2, double b2) {
    return (a0 * b0 + a1 * b1) + a2 * b2;
}

// Row-major 3x3 product C = A * B.
void mul33(const double* A, const double* B, double* C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C[i * 3 + j] = dot3(A[i * 3 + 0], B[0 * 3 + j], A[i * 3 + 1], B[1 * 3 + j], A[i * 3 + 2], B[2 * 3 + j]);
}

// Closed-form inverse of K = [[fx, s, cx], [0, fy, cy], [0, 0, 1]].
void intrinsics_inverse(const double* K, double* Kinv) {
    const double fx = K[0], s = K[1], cx = K[2], fy = K[4], cy = K[5];
    const double fxfy = fx * fy;
    Kinv[0] = 1.0 / fx;
    Kinv[1] = -s / fxfy;
    Kinv[2] = (s * cy - cx * fy) / fxfy;
    Kinv[3] = 0.0;
    Kinv[4] = 1.0 / fy;
    Kinv[5] = -cy / fy;
    Kinv[6] = 0.0;
    Kinv[7] = 0.0;
    Kinv[8] = 1.0;
}

}  // namespace

// Returns 0 on success, 1 for a bad intrinsic matrix, 2 for a degenerate centre plane.
int plane_homography(const ftv_camera& cr, const ftv_camera& cv, const ftv_camera* cc, double iz, double H[9]) {
    for (const ftv_camera* c : {&cr, &cv}) {
        if (c->K[3] != 0.0 || c->K[6] != 0.0 || c->K[7] != 0.0 || c->K[8] != 1.0 || c->K[0] == 0.0 || c->K[4] == 0.0)
            return 1;
    }
    double Rvr[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Rvr[i * 3 + j] = dot3(cv.R[i * 3 + 0], cr.R[j * 3 + 0], cv.R[i * 3 + 1], cr.R[j * 3 + 1],
                                  cv.R[i * 3 + 2], cr.R[j * 3 + 2]);
    double tvr[3];
    for (int i = 0; i < 3; ++i)
        tvr[i] = cv.t[i] - dot3(Rvr[i * 3 + 0], cr.t[0], Rvr[i * 3 + 1], cr.t[1], Rvr[i * 3 + 2], cr.t[2]);
    double n[3];
    double w;
    if (cc == nullptr) {
        n[0] = 0.0;
        n[1] = 0.0;
        n[2] = 1.0;
        w = iz;
    } else {
        // normal of the centre camera's image plane, written in the reference frame: R_r R_c^T e3
        for (int j = 0; j < 3; ++j)
            n[j] = dot3(cr.R[j * 3 + 0], cc->R[6], cr.R[j * 3 + 1], cc->R[7], cr.R[j * 3 + 2], cc->R[8]);
        const double z = 1.0 / iz;
        const double delta = (z - cc->t[2]) + dot3(n[0], cr.t[0], n[1], cr.t[1], n[2], cr.t[2]);
        if (!(std::fabs(delta) > 1e-12)) return 2;
        w = 1.0 / delta;
    }
    double M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i * 3 + j] = Rvr[i * 3 + j] + (tvr[i] * n[j]) * w;
    double Kinv[9], T[9];
    intrinsics_inverse(cr.K, Kinv);
    mul33(M, Kinv, T);
    mul33(cv.K, T, H);
    return 0;
}

}  // namespace ftv
