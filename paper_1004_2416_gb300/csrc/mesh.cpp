// mesh.cpp -- host-side geometry of the IB-LBM-FEM library: the canonical
// icosahedron-subdivision sphere (Sec. II.D, Fig. subdivision) and the
// symmetric 3x3 eigen-decomposition behind the Taylor deformation (Sec. III).
//
// Canonical icosphere (the node and face order is part of the interface):
//   base node k = 4 g + j (g = 0..2, j = 0..3), s1 = (j even ? +1 : -1),
//   s2 = (j < 2 ? +1 : -1), t = golden ratio:
//     g = 0 -> (0, s1, s2 t), g = 1 -> (s1, s2 t, 0), g = 2 -> (s2 t, 0, s1),
//   each scaled by r / |v|;
//   base faces = the mutually adjacent triples i < j < k in lexicographic
//   order, stored (i, j, k) when det[v_i, v_j, v_k] > 0 (outward normal),
//   otherwise (i, k, j);
//   subdivision: faces in order, edges (a,b), (b,c), (c,a); an edge's midpoint
//   (x_a + x_b)/2 projected to radius r becomes a new node at its first
//   encounter; children (a,ab,ca), (ab,b,bc), (ca,bc,c), (ab,bc,ca);
//   the centre is added last.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <unordered_map>
#include <utility>
#include <vector>

#include "internal.h"

namespace iblbm {

namespace {

struct V3 {
    double x, y, z;
};

V3 project(const V3 &q, double r) {
    double len = std::sqrt(q.x * q.x + q.y * q.y + q.z * q.z);
    double s = r / len;
    return V3{q.x * s, q.y * s, q.z * s};
}

double triple(const V3 &a, const V3 &b, const V3 &c) {
    return a.x * (b.y * c.z - b.z * c.y) + a.y * (b.z * c.x - b.x * c.z) +
           a.z * (b.x * c.y - b.y * c.x);
}

V3 cross(const V3 &a, const V3 &b) {
    return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

}  // namespace

void icosphere(int m, double r, const double c[3], std::vector<double> &nodes,
               std::vector<int> &tri) {
    const double t = (1.0 + std::sqrt(5.0)) / 2.0;
    std::vector<V3> base(12);
    for (int k = 0; k < 12; ++k) {
        const int g = k / 4, j = k % 4;
        const double s1 = (j % 2 == 0) ? 1.0 : -1.0;
        const double s2 = (j < 2) ? 1.0 : -1.0;
        if (g == 0) base[k] = V3{0.0, s1, s2 * t};
        else if (g == 1) base[k] = V3{s1, s2 * t, 0.0};
        else base[k] = V3{s2 * t, 0.0, s1};
    }
    // adjacency of the unscaled icosahedron: edge length 2, next distance 2t
    bool adj[12][12];
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) {
            const double dx = base[i].x - base[j].x, dy = base[i].y - base[j].y,
                         dz = base[i].z - base[j].z;
            adj[i][j] = (i != j) && (dx * dx + dy * dy + dz * dz < 5.0);
        }
    std::vector<int> faces;
    for (int i = 0; i < 12; ++i)
        for (int j = i + 1; j < 12; ++j) {
            if (!adj[i][j]) continue;
            for (int k = j + 1; k < 12; ++k) {
                if (!adj[i][k] || !adj[j][k]) continue;
                const bool out = triple(base[i], base[j], base[k]) > 0.0;
                faces.push_back(i);
                faces.push_back(out ? j : k);
                faces.push_back(out ? k : j);
            }
        }
    std::vector<V3> p;
    p.reserve(10 * (size_t(1) << (2 * m)) + 2);
    for (const V3 &v : base) p.push_back(project(v, r));

    for (int level = 0; level < m; ++level) {
        std::unordered_map<uint64_t, int> mid;
        mid.reserve(faces.size());
        auto midpoint = [&](int a, int b) {
            const uint64_t key = (uint64_t)(uint32_t)std::min(a, b) << 32 | (uint32_t)std::max(a, b);
            auto it = mid.find(key);
            if (it != mid.end()) return it->second;
            const V3 q{(p[a].x + p[b].x) * 0.5, (p[a].y + p[b].y) * 0.5, (p[a].z + p[b].z) * 0.5};
            p.push_back(project(q, r));
            const int id = (int)p.size() - 1;
            mid.emplace(key, id);
            return id;
        };
        std::vector<int> next;
        next.reserve(faces.size() * 4);
        for (size_t f = 0; f < faces.size(); f += 3) {
            const int a = faces[f], b = faces[f + 1], cc = faces[f + 2];
            const int ab = midpoint(a, b);
            const int bc = midpoint(b, cc);
            const int ca = midpoint(cc, a);
            const int kids[12] = {a, ab, ca, ab, b, bc, ca, bc, cc, ab, bc, ca};
            next.insert(next.end(), kids, kids + 12);
        }
        faces.swap(next);
    }
    nodes.resize(3 * p.size());
    for (size_t n = 0; n < p.size(); ++n) {
        nodes[3 * n] = c[0] + p[n].x;
        nodes[3 * n + 1] = c[1] + p[n].y;
        nodes[3 * n + 2] = c[2] + p[n].z;
    }
    tri = faces;
}

// Eigenvalues of a symmetric 3x3 matrix from the trigonometric solution of
// its characteristic cubic (Smith, CACM 1961), each refined with an
// eigenvector from a cross product of two rows of (A - lambda I) followed by
// the Rayleigh quotient (twice), which makes the values accurate to rounding
// even where the cubic's roots are ill-conditioned.
namespace {

void mat_vec(const double A[9], const double v[3], double out[3]) {
    for (int i = 0; i < 3; ++i) out[i] = A[3 * i] * v[0] + A[3 * i + 1] * v[1] + A[3 * i + 2] * v[2];
}

bool null_vector(const double A[9], double lam, double v[3]) {
    const double r0[3] = {A[0] - lam, A[1], A[2]};
    const double r1[3] = {A[3], A[4] - lam, A[5]};
    const double r2[3] = {A[6], A[7], A[8] - lam};
    const double *rows[3] = {r0, r1, r2};
    double best = -1.0;
    for (int a = 0; a < 3; ++a) {
        const double *p = rows[a], *q = rows[(a + 1) % 3];
        double c[3] = {p[1] * q[2] - p[2] * q[1], p[2] * q[0] - p[0] * q[2], p[0] * q[1] - p[1] * q[0]};
        double n = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        if (n > best) {
            best = n;
            for (int k = 0; k < 3; ++k) v[k] = c[k];
        }
    }
    if (!(best > 0.0)) return false;
    const double inv = 1.0 / std::sqrt(best);
    for (int k = 0; k < 3; ++k) v[k] *= inv;
    return true;
}

double rayleigh(const double A[9], const double v[3]) {
    double Av[3];
    mat_vec(A, v, Av);
    return (v[0] * Av[0] + v[1] * Av[1] + v[2] * Av[2]) / (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
}

}  // namespace

void sym_eig3(const double A[9], double val[3], double vec[9]) {
    const double a11 = A[0], a22 = A[4], a33 = A[8];
    const double a12 = 0.5 * (A[1] + A[3]), a13 = 0.5 * (A[2] + A[6]), a23 = 0.5 * (A[5] + A[7]);
    const double S[9] = {a11, a12, a13, a12, a22, a23, a13, a23, a33};
    const double q = (a11 + a22 + a33) / 3.0;
    const double p1 = a12 * a12 + a13 * a13 + a23 * a23;
    const double p2 = (a11 - q) * (a11 - q) + (a22 - q) * (a22 - q) + (a33 - q) * (a33 - q) + 2.0 * p1;
    const double p = std::sqrt(p2 / 6.0);
    double lam[3];
    double V[3][3];
    if (!(p > 1e-300)) {
        for (int k = 0; k < 3; ++k) {
            val[k] = q;
            for (int i = 0; i < 3; ++i) vec[3 * i + k] = (i == k) ? 1.0 : 0.0;
        }
        return;
    }
    const double B[9] = {(a11 - q) / p, a12 / p, a13 / p, a12 / p, (a22 - q) / p, a23 / p,
                         a13 / p, a23 / p, (a33 - q) / p};
    double detB = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                  B[2] * (B[3] * B[7] - B[4] * B[6]);
    double rr = 0.5 * detB;
    rr = rr < -1.0 ? -1.0 : (rr > 1.0 ? 1.0 : rr);
    const double phi = std::acos(rr) / 3.0;
    const double two_pi_3 = 2.0943951023931954923;
    lam[2] = q + 2.0 * p * std::cos(phi);               // largest
    lam[0] = q + 2.0 * p * std::cos(phi + two_pi_3);    // smallest
    lam[1] = 3.0 * q - lam[0] - lam[2];
    // vectors of the outer eigenvalues, refined; the middle one completes
    // the orthonormal frame.
    for (int k : {0, 2}) {
        double v[3] = {0, 0, 0};
        for (int it = 0; it < 2; ++it) {
            if (!null_vector(S, lam[k], v)) break;
            lam[k] = rayleigh(S, v);
        }
        for (int i = 0; i < 3; ++i) V[i][k] = v[i];
    }
    {
        double a[3] = {V[0][2], V[1][2], V[2][2]}, b[3] = {V[0][0], V[1][0], V[2][0]};
        double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        double n = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        if (n > 0.0)
            for (int i = 0; i < 3; ++i) V[i][1] = c[i] / n;
        lam[1] = n > 0.0 ? rayleigh(S, c) : lam[1];
    }
    int order[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (lam[order[j]] < lam[order[i]]) std::swap(order[i], order[j]);
    for (int k = 0; k < 3; ++k) {
        val[k] = lam[order[k]];
        for (int i = 0; i < 3; ++i) vec[3 * i + k] = V[i][order[k]];
    }
}

}  // namespace iblbm

namespace iblbm {

// Taylor deformation of a closed membrane and its gradient with respect to
// the node positions, in double precision on the host.  Forward: face area
// vectors A n = (x2 - x1) x (x3 - x1)/2, face centroids r about a fixed origin
// o, V = 1/3 sum r.(A n), centroid offset d = sum (r.(A n)) r / (4 V), q = r - d,
// I = 1/5 sum (q.(A n)) (|q|^2 1 - q q^T), J = I / V, eigenvalues Ja <= Jb <= Jc,
// r_a^2 = 5/2 (Jb + Jc - Ja), r_c^2 = 5/2 (Ja + Jb - Jc), D = (r_a - r_c)/(r_a + r_c).
// Reverse: the same chain taken backwards, with dJ_k = v_k^T dJ v_k for the
// eigenvalues.  The origin o cancels mathematically and is held fixed.
double taylor_D_and_gradient(const double *x, int n, const int *tri, int m, double *grad) {
    double o[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) o[k] += x[3 * i + k];
    for (int k = 0; k < 3; ++k) o[k] /= n;
    std::vector<double> r(3 * (size_t)m), An(3 * (size_t)m), rn(m);
    double V = 0.0, mom[3] = {0, 0, 0};
    for (int f = 0; f < m; ++f) {
        const double *p1 = x + 3 * tri[3 * f], *p2 = x + 3 * tri[3 * f + 1], *p3 = x + 3 * tri[3 * f + 2];
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = p2[k] - p1[k];
            e2[k] = p3[k] - p1[k];
            r[3 * f + k] = (p1[k] + p2[k] + p3[k]) / 3.0 - o[k];
        }
        double *a = &An[3 * f];
        a[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
        a[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
        a[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
        rn[f] = r[3 * f] * a[0] + r[3 * f + 1] * a[1] + r[3 * f + 2] * a[2];
        V += rn[f] / 3.0;
        for (int k = 0; k < 3; ++k) mom[k] += rn[f] * r[3 * f + k];
    }
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = mom[k] / (4.0 * V);
    double I[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    std::vector<double> q(3 * (size_t)m), qn(m);
    for (int f = 0; f < m; ++f) {
        double *qq = &q[3 * f];
        for (int k = 0; k < 3; ++k) qq[k] = r[3 * f + k] - d[k];
        qn[f] = qq[0] * An[3 * f] + qq[1] * An[3 * f + 1] + qq[2] * An[3 * f + 2];
        const double q2 = qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) I[3 * a + b] += 0.2 * qn[f] * ((a == b ? q2 : 0.0) - qq[a] * qq[b]);
    }
    double J[9], val[3], vec[9];
    for (int k = 0; k < 9; ++k) J[k] = I[k] / V;
    sym_eig3(J, val, vec);
    const double ra = std::sqrt(2.5 * (val[1] + val[2] - val[0]));
    const double rc = std::sqrt(2.5 * (val[0] + val[1] - val[2]));
    const double D = (ra - rc) / (ra + rc);
    if (!grad) return D;
    // ---- reverse
    const double dra = 2.0 * rc / ((ra + rc) * (ra + rc));
    const double drc = -2.0 * ra / ((ra + rc) * (ra + rc));
    const double cra = 2.5 / (2.0 * ra), crc = 2.5 / (2.0 * rc);
    const double Jbar_k[3] = {dra * cra * -1.0 + drc * crc * 1.0,  // Ja
                              dra * cra * 1.0 + drc * crc * 1.0,   // Jb
                              dra * cra * 1.0 + drc * crc * -1.0}; // Jc
    double Jbar[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Jbar[3 * a + b] += Jbar_k[k] * vec[3 * a + k] * vec[3 * b + k];
    double Ibar[9], Vbar = 0.0;
    for (int k = 0; k < 9; ++k) {
        Ibar[k] = Jbar[k] / V;
        Vbar -= Jbar[k] * I[k] / (V * V);
    }
    const double trI = Ibar[0] + Ibar[4] + Ibar[8];
    std::vector<double> rbar(3 * (size_t)m, 0.0), Abar(3 * (size_t)m, 0.0);
    double dbar[3] = {0, 0, 0};
    for (int f = 0; f < m; ++f) {
        const double *qq = &q[3 * f];
        const double q2 = qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2];
        double Iq[3];
        for (int a = 0; a < 3; ++a) Iq[a] = Ibar[3 * a] * qq[0] + Ibar[3 * a + 1] * qq[1] + Ibar[3 * a + 2] * qq[2];
        const double qIq = qq[0] * Iq[0] + qq[1] * Iq[1] + qq[2] * Iq[2];
        const double qnbar = 0.2 * (q2 * trI - qIq);
        for (int a = 0; a < 3; ++a) {
            const double qbar = qnbar * An[3 * f + a] + 0.2 * qn[f] * (2.0 * qq[a] * trI - 2.0 * Iq[a]);
            rbar[3 * f + a] += qbar;
            dbar[a] -= qbar;
            Abar[3 * f + a] += qnbar * qq[a];
        }
    }
    double mbar[3];
    for (int k = 0; k < 3; ++k) {
        mbar[k] = dbar[k] / (4.0 * V);
        Vbar -= dbar[k] * mom[k] / (4.0 * V * V);
    }
    for (int f = 0; f < m; ++f) {
        const double *rr = &r[3 * f];
        const double rnbar = mbar[0] * rr[0] + mbar[1] * rr[1] + mbar[2] * rr[2] + Vbar / 3.0;
        for (int a = 0; a < 3; ++a) {
            rbar[3 * f + a] += rn[f] * mbar[a] + rnbar * An[3 * f + a];
            Abar[3 * f + a] += rnbar * rr[a];
        }
    }
    for (int i = 0; i < 3 * n; ++i) grad[i] = 0.0;
    for (int f = 0; f < m; ++f) {
        const int i1 = tri[3 * f], i2 = tri[3 * f + 1], i3 = tri[3 * f + 2];
        const double *p1 = x + 3 * i1, *p2 = x + 3 * i2, *p3 = x + 3 * i3;
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = p2[k] - p1[k];
            e2[k] = p3[k] - p1[k];
        }
        const double *Ab = &Abar[3 * f];
        // An = e1 x e2 / 2: e1bar = (e2 x Abar)/2, e2bar = (Abar x e1)/2
        const double e1b[3] = {0.5 * (e2[1] * Ab[2] - e2[2] * Ab[1]), 0.5 * (e2[2] * Ab[0] - e2[0] * Ab[2]),
                               0.5 * (e2[0] * Ab[1] - e2[1] * Ab[0])};
        const double e2b[3] = {0.5 * (Ab[1] * e1[2] - Ab[2] * e1[1]), 0.5 * (Ab[2] * e1[0] - Ab[0] * e1[2]),
                               0.5 * (Ab[0] * e1[1] - Ab[1] * e1[0])};
        for (int k = 0; k < 3; ++k) {
            const double rb = rbar[3 * f + k] / 3.0;
            grad[3 * i1 + k] += rb - e1b[k] - e2b[k];
            grad[3 * i2 + k] += rb + e1b[k];
            grad[3 * i3 + k] += rb + e2b[k];
        }
    }
    return D;
}


// ---- shape and mesh diagnostics (Sec. III, Sec. V) -------------------------------------

// Angular velocity of each node about the centroid in the xz plane between
// two snapshots dt apart: omega = -(phi1 - phi0)/dt, phi from +x toward +z
// (positive in the rotation sense of u_x = gdot z), the difference taken in
// (-pi, pi].  Returns the mean.
double tank_treading(int n, const double *x0, const double *x1, const double c0[3], const double c1[3],
                     double dt, double *omega) {
    double sum = 0.0;
    for (int i = 0; i < n; ++i) {
        const double dx0 = x0[3 * i] - c0[0], dz0 = x0[3 * i + 2] - c0[2];
        const double dx1 = x1[3 * i] - c1[0], dz1 = x1[3 * i + 2] - c1[2];
        // angle from the first to the second direction: atan2 of their cross
        // and dot products, already in (-pi, pi]
        const double cross = dx0 * dz1 - dz0 * dx1, dot = dx0 * dx1 + dz0 * dz1;
        const double w = -std::atan2(cross, dot) / dt;
        if (omega) omega[i] = w;
        sum += w;
    }
    return n > 0 ? sum / n : 0.0;
}

// Linear least-squares fit of Eq. (chisquare) about c by the normal equations
// (4 x 4, Cholesky), then the semiaxes 1/sqrt(lambda) of Q: the y axis is
// decoupled, the xz block is a 2 x 2 symmetric matrix solved in closed form.
// out = {zeta_x, zeta_y, zeta_z, zeta_xz, r_a, r_b, r_c, D, theta}.
int ellipsoid_fit(int n, const double *x, const double c[3], double out[9]) {
    if (n < 4) return -1;
    double M[4][4] = {}, r[4] = {};
    for (int i = 0; i < n; ++i) {
        const double px = x[3 * i] - c[0], py = x[3 * i + 1] - c[1], pz = x[3 * i + 2] - c[2];
        const double row[4] = {px * px, py * py, pz * pz, -2.0 * px * pz};
        for (int a = 0; a < 4; ++a) {
            r[a] += row[a];
            for (int b = 0; b < 4; ++b) M[a][b] += row[a] * row[b];
        }
    }
    double Lc[4][4] = {};
    for (int j = 0; j < 4; ++j) {
        double d = M[j][j];
        for (int k = 0; k < j; ++k) d -= Lc[j][k] * Lc[j][k];
        if (!(d > 0.0)) return -2;
        Lc[j][j] = std::sqrt(d);
        for (int i = j + 1; i < 4; ++i) {
            double v = M[i][j];
            for (int k = 0; k < j; ++k) v -= Lc[i][k] * Lc[j][k];
            Lc[i][j] = v / Lc[j][j];
        }
    }
    double y[4], z[4];
    for (int i = 0; i < 4; ++i) {
        double v = r[i];
        for (int k = 0; k < i; ++k) v -= Lc[i][k] * y[k];
        y[i] = v / Lc[i][i];
    }
    for (int i = 3; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < 4; ++k) v -= Lc[k][i] * z[k];
        z[i] = v / Lc[i][i];
    }
    // xz block [[zx, -zxz], [-zxz, zz]]
    const double a = z[0], b = -z[3], d = z[2];
    const double mid = 0.5 * (a + d), rad = std::sqrt(0.25 * (a - d) * (a - d) + b * b);
    const double l_small = mid - rad, l_big = mid + rad, l_y = z[1];
    if (!(l_small > 0.0) || !(l_y > 0.0)) return -3;
    double ax[3] = {1.0 / std::sqrt(l_small), 1.0 / std::sqrt(l_y), 1.0 / std::sqrt(l_big)};
    std::sort(ax, ax + 3, [](double p, double q) { return p > q; });
    // major axis in the xz plane: eigenvector of the smaller eigenvalue
    double vx, vz;
    if (std::fabs(b) > 0.0) {
        vx = b;
        vz = l_small - a;
        if (std::fabs(vx) + std::fabs(vz) == 0.0) vx = 1.0;
    } else if (a <= d) {
        vx = 1.0;
        vz = 0.0;
    } else {
        vx = 0.0;
        vz = 1.0;
    }
    if (vx < 0.0) {
        vx = -vx;
        vz = -vz;
    }
    for (int k = 0; k < 4; ++k) out[k] = z[k];
    out[4] = ax[0];
    out[5] = ax[1];
    out[6] = ax[2];
    out[7] = (ax[0] - ax[2]) / (ax[0] + ax[2]);
    out[8] = std::atan2(vz, vx);
    return 0;
}

// Relative face area deviation dA/A0 of the faces [m][3] between reference
// X0 and current x: {mean, standard deviation about the mean (1/m), max |.|}.
// Volume enclosed by the outward-oriented faces [m][3]: sum of the signed
// tetrahedra spanned with the first node.
double closed_volume(int m, const int *tri, const double *x) {
    const double *o = x + 3 * tri[0];
    double v = 0.0;
    for (int f = 0; f < m; ++f) {
        const double *a = x + 3 * tri[3 * f], *b = x + 3 * tri[3 * f + 1], *c = x + 3 * tri[3 * f + 2];
        v += triple(V3{a[0] - o[0], a[1] - o[1], a[2] - o[2]}, V3{b[0] - o[0], b[1] - o[1], b[2] - o[2]},
                    V3{c[0] - o[0], c[1] - o[1], c[2] - o[2]});
    }
    return v / 6.0;
}

void face_area_stats(int m, const int *tri, const double *X0, const double *x, double out[3]) {
    auto area = [&](const double *p, int f) {
        const double *a = p + 3 * tri[3 * f], *b = p + 3 * tri[3 * f + 1], *c = p + 3 * tri[3 * f + 2];
        const V3 u{b[0] - a[0], b[1] - a[1], b[2] - a[2]}, v{c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        const V3 w = cross(u, v);
        return 0.5 * std::sqrt(w.x * w.x + w.y * w.y + w.z * w.z);
    };
    std::vector<double> rel(m);
    double sum = 0.0, mx = 0.0;
    for (int f = 0; f < m; ++f) {
        const double a0 = area(X0, f);
        rel[f] = (area(x, f) - a0) / a0;
        sum += rel[f];
        mx = std::max(mx, std::fabs(rel[f]));
    }
    const double mean = m > 0 ? sum / m : 0.0;
    double ss = 0.0;
    for (int f = 0; f < m; ++f) ss += (rel[f] - mean) * (rel[f] - mean);
    out[0] = mean;
    out[1] = m > 0 ? std::sqrt(ss / m) : 0.0;
    out[2] = mx;
}

}  // namespace iblbm
