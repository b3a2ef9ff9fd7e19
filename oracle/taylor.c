/*
 * taylor.c -- oracle of the capsule shape measures of Sec. III: volume,
 * surface area, the inertia tensor of Ramanujan and Pozrikidis as the paper
 * writes it, the equivalent unit-mass ellipsoid, the Taylor deformation
 * D = (r_a - r_c)/(r_a + r_c) and the inclination angle theta.  Test
 * infrastructure only.
 *
 * Readings (the paper leaves them open):
 *   - face area vector A n = (x2 - x1) x (x3 - x1) / 2 (outward for the
 *     counter-clockwise faces of the mesh);
 *   - volume V = 1/3 sum r_f . (A n)_f and centroid c = sum (r_f . A n) r_f
 *     / (4 V), face centroids r_f taken about the mean of the nodes (both are
 *     exact for a closed polyhedron of flat faces);
 *   - the inertia formula is evaluated about the centroid c and divided by V
 *     (unit mass);
 *   - eigenvalues J_a <= J_b <= J_c of that tensor give
 *     r_a^2 = 5/2 (J_b + J_c - J_a), r_b^2 = 5/2 (J_a + J_c - J_b),
 *     r_c^2 = 5/2 (J_a + J_b - J_c) (diagonal of the ellipsoid tensor in
 *     Sec. III);
 *   - theta = atan2(v_z, v_x) of the eigenvector v of J_a (the major axis),
 *     sign chosen with v_x >= 0: the angle in the xz shear plane measured
 *     from the flow direction +x toward the velocity-gradient direction +z
 *     (Fig. geometry draws the cross-section in the plane of the shear).
 *
 * Pins (tests/test_oracle_taylor.py): the eigen-solver against explicitly
 * rotated diagonal matrices; V and A of the icosphere against the polyhedron
 * formulas for the regular icosahedron and the sphere limit; D = 0 for the
 * icosphere (icosahedral symmetry); an icosphere stretched to an ellipsoid
 * with semi-axes (a, b, c) and rotated by theta0 about y gives
 * D -> (a - c)/(a + c) and theta -> theta0 under refinement.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

/* Cyclic Jacobi method for a symmetric matrix (Golub and Van Loan, symmetric
 * Schur decomposition): rotations zero one off-diagonal entry at a time until
 * the off-diagonal norm is negligible. */
void orc_eig3(const real Ain[9], real eval[3], real vec[9]) {
    real A[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A[i][j] = Ain[3 * i + j];
            V[i][j] = (i == j) ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 100; ++sweep) {
        real off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        real diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (RE(off) <= 1e-40 * RE(diag) || RE(off) == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (RE(A[p][q]) == 0.0) continue;
                real theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                real t = (RE(theta) >= 0.0 ? 1.0 : -1.0) /
                         (r_abs(theta) + r_sqrt(theta * theta + 1.0));
                real c = 1.0 / r_sqrt(t * t + 1.0), s = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < 3; ++k) {
                    real akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    real apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    real vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int order[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (RE(A[order[j]][order[j]]) < RE(A[order[i]][order[i]])) {
                int tmp = order[i];
                order[i] = order[j];
                order[j] = tmp;
            }
    for (int k = 0; k < 3; ++k) {
        eval[k] = A[order[k]][order[k]];
        for (int i = 0; i < 3; ++i) vec[3 * i + k] = V[i][order[k]];
    }
}

int orc_taylor(int n_nodes, const real *x, int n_tri, const int *tri,
               real out[16]) {
    if (n_nodes < 4 || n_tri < 4) return -1;
    real o[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n_nodes; ++i)
        for (int a = 0; a < 3; ++a) o[a] += x[3 * i + a];
    for (int a = 0; a < 3; ++a) o[a] /= n_nodes;

    real V = 0.0, A = 0.0, m1[3] = {0.0, 0.0, 0.0};
    for (int f = 0; f < n_tri; ++f) {
        const real *p1 = x + 3 * tri[3 * f], *p2 = x + 3 * tri[3 * f + 1],
                     *p3 = x + 3 * tri[3 * f + 2];
        real e1[3], e2[3], An[3], rc[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = p2[a] - p1[a];
            e2[a] = p3[a] - p1[a];
            rc[a] = (p1[a] + p2[a] + p3[a]) / 3.0 - o[a];
        }
        An[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
        An[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
        An[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
        real rn = rc[0] * An[0] + rc[1] * An[1] + rc[2] * An[2];
        V += rn / 3.0;
        A += r_sqrt(An[0] * An[0] + An[1] * An[1] + An[2] * An[2]);
        for (int a = 0; a < 3; ++a) m1[a] += rn * rc[a];
    }
    real c[3];
    for (int a = 0; a < 3; ++a) c[a] = o[a] + m1[a] / (4.0 * V);

    /* I_ab = 1/5 sum_faces A_i (r_i^2 delta_ab r_g - r_ia r_ib r_ig) n_ig */
    real I[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int f = 0; f < n_tri; ++f) {
        const real *p1 = x + 3 * tri[3 * f], *p2 = x + 3 * tri[3 * f + 1],
                     *p3 = x + 3 * tri[3 * f + 2];
        real e1[3], e2[3], An[3], r[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = p2[a] - p1[a];
            e2[a] = p3[a] - p1[a];
            r[a] = (p1[a] + p2[a] + p3[a]) / 3.0 - c[a];
        }
        An[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
        An[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
        An[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
        real r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        real rn = r[0] * An[0] + r[1] * An[1] + r[2] * An[2];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                I[a][b] += ((a == b ? r2 : 0.0) - r[a] * r[b]) * rn / 5.0;
    }
    real J[9], ev[3], vec[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) J[3 * a + b] = I[a][b] / V;
    orc_eig3(J, ev, vec);
    real ra = r_sqrt(2.5 * (ev[1] + ev[2] - ev[0]));
    real rb = r_sqrt(2.5 * (ev[0] + ev[2] - ev[1]));
    real rcc = r_sqrt(2.5 * (ev[0] + ev[1] - ev[2]));
    real vx = vec[0], vz = vec[6];
    if (RE(vx) < 0.0) {
        vx = -vx;
        vz = -vz;
    }
    out[0] = (ra - rcc) / (ra + rcc);
    out[1] = r_atan2(vz, vx);
    out[2] = ra;
    out[3] = rb;
    out[4] = rcc;
    out[5] = V;
    out[6] = A;
    out[7] = c[0];
    out[8] = c[1];
    out[9] = c[2];
    out[10] = I[0][0];
    out[11] = I[1][1];
    out[12] = I[2][2];
    out[13] = I[0][1];
    out[14] = I[0][2];
    out[15] = I[1][2];
    return 0;
}
