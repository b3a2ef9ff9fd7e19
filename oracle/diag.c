/*
 * diag.c -- oracle of the shape and mesh diagnostics the paper reports beside
 * the Taylor deformation.  Test infrastructure only.
 *
 *   orc_tank_treading   -- angular velocity omega_i = dphi_i / dt of each node,
 *                          phi_i its angle about the capsule centroid projected
 *                          on the xz plane (Sec. III).  Reading: phi is measured
 *                          from +x toward +z and omega = -dphi/dt, so that the
 *                          rotation of simple shear u_x = gdot z (a stiff sphere
 *                          turns at gdot / 2) is positive; dphi is wrapped to
 *                          (-pi, pi].
 *   orc_ellipsoid_fit   -- the linear least-squares fit of Eq. (chisquare) to
 *                          the node positions relative to the centroid, the
 *                          matrix Q, its eigenvalues lambda, semiaxes
 *                          1/sqrt(lambda), D = (r_a - r_c)/(r_a + r_c) of the
 *                          largest and smallest, and the inclination of the
 *                          major axis in the xz plane (as in taylor.c).
 *                          Solved by Householder QR of the n x 4 design matrix.
 *   orc_face_area_stats -- mean and standard deviation (over faces, 1/N) of
 *                          the relative face area deviation dA/A0 of Fig.
 *                          degrade, and its largest magnitude.
 *
 * Pins (tests/test_oracle_diagnostics.py): rigid rotations of a sphere give
 * omega = angle / dt at every node; nodes on an exact ellipsoid, rotated about
 * y, give back its semiaxes, D and angle; a uniform stretch by s gives
 * dA/A0 = s^2 - 1 on every face.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

double orc_tank_treading(int n, const double *x0, const double *x1, const double c0[3],
                         const double c1[3], double dt, double *omega) {
    const double pi = 3.14159265358979323846;
    double sum = 0.0;
    int used = 0;
    for (int i = 0; i < n; ++i) {
        double a0 = atan2(x0[3 * i + 2] - c0[2], x0[3 * i] - c0[0]);
        double a1 = atan2(x1[3 * i + 2] - c1[2], x1[3 * i] - c1[0]);
        double d = a1 - a0;
        while (d > pi) d -= 2.0 * pi;
        while (d <= -pi) d += 2.0 * pi;
        double w = -d / dt;
        if (omega) omega[i] = w;
        sum += w;
        ++used;
    }
    return used ? sum / used : 0.0;
}

/* Least squares min |A z - b| by Householder reflections, A: m x 4 (row-major,
 * overwritten), b: m (overwritten). */
static int lsq4(int m, double *A, double *b, double z[4]) {
    for (int k = 0; k < 4; ++k) {
        double norm = 0.0;
        for (int i = k; i < m; ++i) norm += A[4 * i + k] * A[4 * i + k];
        norm = sqrt(norm);
        if (norm == 0.0) return -1;
        double alpha = A[4 * k + k] > 0 ? -norm : norm;
        /* v = a_k - alpha e_k, stored in place */
        A[4 * k + k] -= alpha;
        double vv = 0.0;
        for (int i = k; i < m; ++i) vv += A[4 * i + k] * A[4 * i + k];
        for (int j = k + 1; j < 4; ++j) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += A[4 * i + k] * A[4 * i + j];
            s = 2.0 * s / vv;
            for (int i = k; i < m; ++i) A[4 * i + j] -= s * A[4 * i + k];
        }
        double s = 0.0;
        for (int i = k; i < m; ++i) s += A[4 * i + k] * b[i];
        s = 2.0 * s / vv;
        for (int i = k; i < m; ++i) b[i] -= s * A[4 * i + k];
        A[4 * k + k] = alpha; /* R diagonal */
    }
    for (int k = 3; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < 4; ++j) s -= A[4 * k + j] * z[j];
        z[k] = s / A[4 * k + k];
    }
    return 0;
}

int orc_ellipsoid_fit(int n, const double *x, const double c[3], double out[9]) {
    if (n < 4) return -1;
    double *A = (double *)malloc(sizeof(double) * 4 * n), *b = (double *)malloc(sizeof(double) * n);
    if (!A || !b) {
        free(A); free(b);
        return -2;
    }
    for (int i = 0; i < n; ++i) {
        double px = x[3 * i] - c[0], py = x[3 * i + 1] - c[1], pz = x[3 * i + 2] - c[2];
        A[4 * i] = px * px;
        A[4 * i + 1] = py * py;
        A[4 * i + 2] = pz * pz;
        A[4 * i + 3] = -2.0 * px * pz;
        b[i] = 1.0;
    }
    double z[4];
    int rc = lsq4(n, A, b, z);
    free(A); free(b);
    if (rc) return rc;
    double Q[9] = {z[0], 0.0, -z[3], 0.0, z[1], 0.0, -z[3], 0.0, z[2]};
    double ev[3], V[9];
    orc_eig3(Q, ev, V);
    if (!(ev[0] > 0.0)) return -3;
    /* ascending eigenvalues: the largest semiaxis belongs to ev[0] */
    double ra = 1.0 / sqrt(ev[0]), rb = 1.0 / sqrt(ev[1]), rc_ = 1.0 / sqrt(ev[2]);
    double vx = V[0], vz = V[6];
    if (vx < 0) {
        vx = -vx;
        vz = -vz;
    }
    for (int k = 0; k < 4; ++k) out[k] = z[k];
    out[4] = ra;
    out[5] = rb;
    out[6] = rc_;
    out[7] = (ra - rc_) / (ra + rc_);
    out[8] = atan2(vz, vx);
    return 0;
}

static double tri_area(const double *p, const int *t) {
    double e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = p[3 * t[1] + k] - p[3 * t[0] + k];
        e2[k] = p[3 * t[2] + k] - p[3 * t[0] + k];
    }
    double cx = e1[1] * e2[2] - e1[2] * e2[1];
    double cy = e1[2] * e2[0] - e1[0] * e2[2];
    double cz = e1[0] * e2[1] - e1[1] * e2[0];
    return 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
}

/* two passes: the mean first, then the spread about it */
int orc_face_area_stats(int n_tri, const int *tri, const double *X0, const double *x, double out[3]) {
    if (n_tri < 1) return -1;
    double sum = 0.0, mx = 0.0;
    for (int f = 0; f < n_tri; ++f) {
        double a0 = tri_area(X0, tri + 3 * f), a = tri_area(x, tri + 3 * f);
        double r = (a - a0) / a0;
        sum += r;
        if (fabs(r) > mx) mx = fabs(r);
    }
    double mean = sum / n_tri, ss = 0.0;
    for (int f = 0; f < n_tri; ++f) {
        double a0 = tri_area(X0, tri + 3 * f), a = tri_area(x, tri + 3 * f);
        double r = (a - a0) / a0 - mean;
        ss += r * r;
    }
    out[0] = mean;
    out[1] = sqrt(ss / n_tri);
    out[2] = mx;
    return 0;
}
