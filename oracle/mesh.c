/*
 * mesh.c -- oracle of the icosahedron-subdivision membrane mesh (Sec. II.D,
 * Fig. subdivision).  Test infrastructure only.
 *
 * The paper fixes the construction (regular icosahedron; each subdivision
 * halves every edge, connects the six nodes into four faces and pushes the new
 * nodes radially onto the circumsphere) but not an ordering.  The canonical
 * ordering taken here (and, written separately, by the CUDA library) is:
 *
 *   base node k = 4 g + j (g = 0, 1, 2; j = 0..3), s1 = +1 for even j else -1,
 *   s2 = +1 for j < 2 else -1, golden ratio t:
 *       g = 0: (0, s1, s2 t)   g = 1: (s1, s2 t, 0)   g = 2: (s2 t, 0, s1)
 *   scaled to radius r;
 *   base faces: every triple i < j < k of mutually adjacent base nodes, in
 *   lexicographic order, written (i, j, k) if (x_j - x_i) x (x_k - x_i)
 *   points outward, else (i, k, j);
 *   one subdivision: faces in order; for each face (a, b, c) the edges
 *   (a, b), (b, c), (c, a) get a midpoint node, appended at its first
 *   encounter, m = (x_a + x_b)/2 scaled by r/|m|; the face is replaced by the
 *   children (a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca);
 *   finally every node is translated by the centre.
 *
 * Pins (tests/test_oracle_mesh.py): N_f = 20 4^m and 2 N_n = N_f + 4 (Sec.
 * II.D); closed, consistently oriented, outward (positive volume); neighbour
 * counts 5 and 6 and the scatter of face area, edge length and angles of
 * Tab. mesh_quality; mean edge length at r = 5 quoted in Sec. IV.B.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define MAXNB 8

static int midpoint(int a, int b, double r, double *p, int *n_nodes, int *nb,
                    int *mid, int *cnt) {
    int lo = a < b ? a : b, hi = a < b ? b : a;
    for (int k = 0; k < cnt[lo]; ++k)
        if (nb[lo * MAXNB + k] == hi) return mid[lo * MAXNB + k];
    int m = (*n_nodes)++;
    double q[3];
    for (int d = 0; d < 3; ++d) q[d] = (p[3 * a + d] + p[3 * b + d]) * 0.5;
    double len = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    double s = r / len;
    for (int d = 0; d < 3; ++d) p[3 * m + d] = q[d] * s;
    nb[lo * MAXNB + cnt[lo]] = hi;
    mid[lo * MAXNB + cnt[lo]] = m;
    cnt[lo]++;
    return m;
}

int orc_icosphere(int m, double r, const double c[3], double *nodes, int *tri) {
    if (m < 0 || m > 8 || !(r > 0.0)) return -1;
    int nf_final = 20;
    for (int k = 0; k < m; ++k) nf_final *= 4;
    int nn_final = nf_final / 2 + 2;
    double *p = (double *)malloc(sizeof(double) * 3 * nn_final);
    int *fa = (int *)malloc(sizeof(int) * 3 * nf_final);
    int *fb = (int *)malloc(sizeof(int) * 3 * nf_final);
    int *nb = (int *)malloc(sizeof(int) * MAXNB * nn_final);
    int *mid = (int *)malloc(sizeof(int) * MAXNB * nn_final);
    int *cnt = (int *)malloc(sizeof(int) * nn_final);
    if (!p || !fa || !fb || !nb || !mid || !cnt) {
        free(p); free(fa); free(fb); free(nb); free(mid); free(cnt);
        return -2;
    }
    const double t = (1.0 + sqrt(5.0)) / 2.0;
    double v[12][3];
    for (int k = 0; k < 12; ++k) {
        int g = k / 4, j = k % 4;
        double s1 = (j % 2 == 0) ? 1.0 : -1.0;
        double s2 = (j < 2) ? 1.0 : -1.0;
        if (g == 0) { v[k][0] = 0.0; v[k][1] = s1; v[k][2] = s2 * t; }
        if (g == 1) { v[k][0] = s1; v[k][1] = s2 * t; v[k][2] = 0.0; }
        if (g == 2) { v[k][0] = s2 * t; v[k][1] = 0.0; v[k][2] = s1; }
    }
    /* base faces: mutually adjacent triples (edge length 2 before scaling) */
    int nf = 0;
    for (int i = 0; i < 12; ++i)
        for (int j = i + 1; j < 12; ++j)
            for (int k = j + 1; k < 12; ++k) {
                double dij = 0, djk = 0, dik = 0;
                for (int d = 0; d < 3; ++d) {
                    dij += (v[i][d] - v[j][d]) * (v[i][d] - v[j][d]);
                    djk += (v[j][d] - v[k][d]) * (v[j][d] - v[k][d]);
                    dik += (v[i][d] - v[k][d]) * (v[i][d] - v[k][d]);
                }
                if (dij > 5.0 || djk > 5.0 || dik > 5.0) continue;
                double e1[3], e2[3], n[3], s = 0.0;
                for (int d = 0; d < 3; ++d) {
                    e1[d] = v[j][d] - v[i][d];
                    e2[d] = v[k][d] - v[i][d];
                }
                n[0] = e1[1] * e2[2] - e1[2] * e2[1];
                n[1] = e1[2] * e2[0] - e1[0] * e2[2];
                n[2] = e1[0] * e2[1] - e1[1] * e2[0];
                for (int d = 0; d < 3; ++d) s += n[d] * (v[i][d] + v[j][d] + v[k][d]);
                fa[3 * nf] = i;
                fa[3 * nf + 1] = s > 0.0 ? j : k;
                fa[3 * nf + 2] = s > 0.0 ? k : j;
                nf++;
            }
    for (int k = 0; k < 12; ++k) {
        double len = sqrt(v[k][0] * v[k][0] + v[k][1] * v[k][1] + v[k][2] * v[k][2]);
        double s = r / len;
        for (int d = 0; d < 3; ++d) p[3 * k + d] = v[k][d] * s;
    }
    int nn = 12;
    for (int level = 0; level < m; ++level) {
        memset(cnt, 0, sizeof(int) * nn_final);
        int nf2 = 0;
        for (int f = 0; f < nf; ++f) {
            int a = fa[3 * f], b = fa[3 * f + 1], cc = fa[3 * f + 2];
            int ab = midpoint(a, b, r, p, &nn, nb, mid, cnt);
            int bc = midpoint(b, cc, r, p, &nn, nb, mid, cnt);
            int ca = midpoint(cc, a, r, p, &nn, nb, mid, cnt);
            int ch[4][3] = {{a, ab, ca}, {ab, b, bc}, {ca, bc, cc}, {ab, bc, ca}};
            for (int q = 0; q < 4; ++q)
                for (int d = 0; d < 3; ++d) fb[3 * nf2 + 3 * q + d] = ch[q][d];
            nf2 += 4;
        }
        nf = nf2;
        memcpy(fa, fb, sizeof(int) * 3 * nf);
    }
    for (int k = 0; k < nn; ++k)
        for (int d = 0; d < 3; ++d) nodes[3 * k + d] = c[d] + p[3 * k + d];
    memcpy(tri, fa, sizeof(int) * 3 * nf);
    free(p); free(fa); free(fb); free(nb); free(mid); free(cnt);
    return nn;
}
