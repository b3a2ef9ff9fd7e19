/*
 * membrane.c -- oracle of the finite-element Skalak membrane (Sec. II.B).
 * Test infrastructure only.
 *
 * The face energy follows the paper's route literally: lengths l, l' of two
 * edges and their angle phi, the same in the reference state (l0, l0', phi0);
 * the displacement gradient entries a, b, c of Eq. (c); the invariants of
 * Eq. (lambda1); the Skalak density of Eq. (constitutivelaw); W = A0 w^S.
 * The nodal force is the definition of Eq. (forcefromenergy), F = -dW/dx,
 * obtained by forward-mode differentiation (dual numbers carrying the nine
 * partial derivatives with respect to the corner coordinates) of that same
 * energy, so that no hand-derived gradient formula enters the oracle.
 *
 * Reading: l is the edge from corner 1 to corner 3, l' the edge from corner 1
 * to corner 2 and phi the angle at corner 1 (the labels of
 * Fig. deformedface); which two edges are used does not change I1 or I2.
 *
 * Pins (tests/test_oracle_membrane.py): W = 0 and F = 0 on the reference
 * shape; rigid rotations and translations give zero force; anisotropic
 * in-plane stretch diag(l1, l2) of a rotated triangle gives the closed-form
 * invariants and energy; uniform stretch closed form; central finite
 * differences of W reproduce F; net force and net torque vanish on a
 * randomly deformed icosphere.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define ND 9
typedef struct {
    real v;
    real d[ND];
} dual;

static dual d_const(real v) {
    dual r;
    r.v = v;
    for (int k = 0; k < ND; ++k) r.d[k] = 0.0;
    return r;
}
static dual d_add(dual a, dual b) {
    dual r;
    r.v = a.v + b.v;
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
static dual d_sub(dual a, dual b) {
    dual r;
    r.v = a.v - b.v;
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
static dual d_mul(dual a, dual b) {
    dual r;
    r.v = a.v * b.v;
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
static dual d_div(dual a, dual b) {
    dual r;
    r.v = a.v / b.v;
    for (int k = 0; k < ND; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
    return r;
}
static dual d_sqrt(dual a) {
    dual r;
    r.v = r_sqrt(a.v);
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] / (2.0 * r.v);
    return r;
}
static dual d_scale(dual a, real s) {
    dual r;
    r.v = a.v * s;
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * s;
    return r;
}

/* Reference geometry of a face: l0 = |X3 - X1|, l0' = |X2 - X1|, phi0 the
 * angle at corner 1, and the reference area A0 = l0 l0' sin(phi0) / 2. */
static void reference(const real X0[9], real *l0, real *lp0,
                      real *cos0, real *sin0, real *A0) {
    real e[3], ep[3], cr[3];
    for (int a = 0; a < 3; ++a) {
        e[a] = X0[6 + a] - X0[a];
        ep[a] = X0[3 + a] - X0[a];
    }
    cr[0] = e[1] * ep[2] - e[2] * ep[1];
    cr[1] = e[2] * ep[0] - e[0] * ep[2];
    cr[2] = e[0] * ep[1] - e[1] * ep[0];
    *l0 = r_sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    *lp0 = r_sqrt(ep[0] * ep[0] + ep[1] * ep[1] + ep[2] * ep[2]);
    *cos0 = (e[0] * ep[0] + e[1] * ep[1] + e[2] * ep[2]) / (*l0 * *lp0);
    *sin0 = r_sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]) / (*l0 * *lp0);
    *A0 = 0.5 * *l0 * *lp0 * *sin0;
}

/* a, b, c of Eq. (c) and the invariants of Eq. (lambda1), on dual numbers. */
static void invariants(const real X0[9], const dual x[9], dual *I1, dual *I2,
                       real *A0) {
    real l0, lp0, cos0, sin0;
    reference(X0, &l0, &lp0, &cos0, &sin0, A0);
    dual e[3], ep[3];
    for (int a = 0; a < 3; ++a) {
        e[a] = d_sub(x[6 + a], x[a]);
        ep[a] = d_sub(x[3 + a], x[a]);
    }
    dual ee = d_add(d_add(d_mul(e[0], e[0]), d_mul(e[1], e[1])), d_mul(e[2], e[2]));
    dual pp = d_add(d_add(d_mul(ep[0], ep[0]), d_mul(ep[1], ep[1])), d_mul(ep[2], ep[2]));
    dual ep_dot = d_add(d_add(d_mul(e[0], ep[0]), d_mul(e[1], ep[1])), d_mul(e[2], ep[2]));
    dual cr0 = d_sub(d_mul(e[1], ep[2]), d_mul(e[2], ep[1]));
    dual cr1 = d_sub(d_mul(e[2], ep[0]), d_mul(e[0], ep[2]));
    dual cr2 = d_sub(d_mul(e[0], ep[1]), d_mul(e[1], ep[0]));
    dual crn = d_sqrt(d_add(d_add(d_mul(cr0, cr0), d_mul(cr1, cr1)), d_mul(cr2, cr2)));
    dual l = d_sqrt(ee);
    dual lp = d_sqrt(pp);
    dual ll = d_mul(l, lp);
    dual cosp = d_div(ep_dot, ll);
    dual sinp = d_div(crn, ll);
    /* Eq. (c) and the two lines above it */
    dual a = d_scale(l, 1.0 / l0);
    dual r = d_scale(lp, 1.0 / lp0);
    dual b = d_scale(d_sub(d_mul(r, cosp), d_scale(a, cos0)), 1.0 / sin0);
    dual c = d_scale(d_mul(r, sinp), 1.0 / sin0);
    /* Eq. (lambda1): lambda1^2 lambda2^2 = a^2 c^2,
     *                lambda1^2 + lambda2^2 = a^2 + b^2 + c^2 */
    dual a2 = d_mul(a, a), b2 = d_mul(b, b), c2 = d_mul(c, c);
    *I1 = d_sub(d_add(d_add(a2, b2), c2), d_const(2.0));
    *I2 = d_sub(d_mul(a2, c2), d_const(1.0));
}

/* Eq. (constitutivelaw) times the reference area. */
static dual face_energy(const real X0[9], const dual x[9], real ks,
                        real ka) {
    dual I1, I2;
    real A0;
    invariants(X0, x, &I1, &I2, &A0);
    dual t1 = d_sub(d_add(d_mul(I1, I1), d_scale(I1, 2.0)), d_scale(I2, 2.0));
    dual w = d_add(d_scale(t1, ks / 12.0), d_scale(d_mul(I2, I2), ka / 12.0));
    return d_scale(w, A0);
}

static void seed(const real x[9], dual xd[9]) {
    for (int k = 0; k < 9; ++k) {
        xd[k] = d_const(x[k]);
        xd[k].d[k] = 1.0;
    }
}

real orc_face_energy(const real X0[9], const real x[9], real ks,
                       real ka) {
    dual xd[9];
    for (int k = 0; k < 9; ++k) xd[k] = d_const(x[k]);
    return face_energy(X0, xd, ks, ka).v;
}

void orc_face_invariants(const real X0[9], const real x[9], real *I1,
                         real *I2) {
    dual xd[9], i1, i2;
    real A0;
    for (int k = 0; k < 9; ++k) xd[k] = d_const(x[k]);
    invariants(X0, xd, &i1, &i2, &A0);
    *I1 = i1.v;
    *I2 = i2.v;
}

/* Eq. (forcefromenergy) for one face. */
real orc_face_forces(const real X0[9], const real x[9], real ks,
                       real ka, real F[9]) {
    dual xd[9];
    seed(x, xd);
    dual W = face_energy(X0, xd, ks, ka);
    for (int k = 0; k < 9; ++k) F[k] = -W.d[k];
    return W.v;
}

/* W = sum over faces of A0_j w_j; node force = sum of the corner forces of
 * its faces, faces visited in ascending order. */
real orc_membrane_forces(int n_nodes, const real *X0, const real *x,
                           int n_tri, const int *tri, real ks, real ka,
                           real *F) {
    memset(F, 0, 3 * (size_t)n_nodes * sizeof(real));
    real W = 0.0;
    for (int f = 0; f < n_tri; ++f) {
        real X0f[9], xf[9], Ff[9];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) {
                X0f[3 * k + a] = X0[3 * tri[3 * f + k] + a];
                xf[3 * k + a] = x[3 * tri[3 * f + k] + a];
            }
        W += orc_face_forces(X0f, xf, ks, ka, Ff);
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) F[3 * tri[3 * f + k] + a] += Ff[3 * k + a];
    }
    return W;
}
