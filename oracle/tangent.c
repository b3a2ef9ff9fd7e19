/*
 * tangent.c -- forward-mode (tangent-linear) derivative of the Taylor
 * deformation of the final shape with respect to the run's parameters, by the
 * complex-step method applied to the whole oracle step.  Test infrastructure
 * only; built only with ORC_COMPLEX_STEP (real = double _Complex).
 *
 * The oracle's sub-step list of Sec. II.C (forces of Sec. II.B, spreading of
 * Eq. forcespreading, the lattice Boltzmann step of Eq. lbequation with the
 * moving walls, interpolation of Eq. velocityinterpolation, advection of Eq.
 * positionupdate) and the reductions of Sec. III are evaluated at
 *   u_wall + i h du_wall,  X0 + i h dX0,  k_s + i h dk_s  (k_alpha = C k_s),
 * starting from the Couette state of that wall speed with the capsule in its
 * reference shape.  With h far below the rounding of the real parts
 * (1e-30), Im D / h is dD along the direction to rounding: the method
 * subtracts nothing, unlike a finite difference.
 *
 * Pins (tests/test_oracle_tangent.py): the real part equals the double
 * oracle's D bit for bit; on short runs the derivative agrees with central
 * finite differences of the double oracle to their truncation error; it is
 * linear in the direction (a sum of directions gives the sum of the
 * derivatives to rounding).
 */
#include <complex.h>
#include <stdlib.h>
#include "oracle.h"

int orc_tangent_taylor_D(int nx, int ny, int nz, double tau, int delta_n,
                         double u_wall, double du_wall, int n_nodes, const double *X0,
                         const double *dX0, int n_tri, const int *tri, double ks,
                         double dks, double C, int n_steps, double h, double out[2]) {
    if (n_nodes < 4 || n_tri < 4 || n_steps < 0 || !(h > 0.0)) return -1;
    real *Xc = (real *)malloc(sizeof(real) * 3 * (size_t)n_nodes);
    if (!Xc) return -2;
    for (int k = 0; k < 3 * n_nodes; ++k) Xc[k] = X0[k] + _Complex_I * h * dX0[k];
    const real uw = u_wall + _Complex_I * h * du_wall;
    const real ksc = ks + _Complex_I * h * dks;
    orc_sim *s = orc_sim_create(nx, ny, nz, tau, delta_n, uw);
    int rc = s ? 0 : -2;
    if (!rc) rc = orc_sim_add_capsule(s, n_nodes, Xc, n_tri, tri, ksc, C * ksc) < 0 ? -1 : 0;
    if (!rc) rc = orc_sim_step(s, n_steps);
    if (!rc) {
        real *x = (real *)malloc(sizeof(real) * 3 * (size_t)n_nodes);
        real T[16];
        if (!x) {
            rc = -2;
        } else {
            orc_sim_get_nodes(s, x);
            rc = orc_taylor(n_nodes, x, n_tri, tri, T);
            if (!rc) {
                out[0] = creal(T[0]);
                out[1] = cimag(T[0]) / h;
            }
            free(x);
        }
    }
    orc_sim_destroy(s);
    free(Xc);
    return rc;
}
