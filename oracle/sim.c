/*
 * sim.c -- oracle of one complete time step of the combined IB-LBM-FEM
 * scheme, the sub-step list at the end of Sec. II.C:
 *   1. node forces F_i(t) from the positions x_i(t) by the FEM (Sec. II.B);
 *   2. spreading of F_i(t) to the force density f(X, t), Eq. (forcespreading);
 *   3. one lattice Boltzmann step with f(X, t), Eq. (lbequation);
 *   4. node velocities u_i(t+1) by interpolation of the new lattice velocity
 *      at the old positions, Eq. (velocityinterpolation);
 *   5. Euler advection x_i(t+1) = x_i(t) + u_i(t+1), Eq. (positionupdate),
 *      or, as a variant, the Adams-Bashforth rule of Sec. II.C,
 *      x_i(t+1) = x_i(t) + 3/2 u_i(t+1) - 1/2 u_i(t).
 * Test infrastructure only.
 *
 * Reading (Adams-Bashforth): the rule needs the velocity u_i(t) of the step
 * before; the first step after the start, after the nodes were set by hand or
 * after the integrator was chosen takes the Euler rule instead.
 *
 * Reading: the lattice velocity that is interpolated in sub-step 4 is
 * u(X, t+1) = (sum_i c_i f_i(X, t+1) + f(X, t)/2) / rho(X, t+1), i.e.
 * Eq. (lbmmomenta1) with the force density of the step just taken (the force
 * at t+1 is not known before the nodes move).  The same velocity is returned
 * by orc_sim_get_velocity.
 *
 * Parity status: the coupled trajectory has no closed form.  It is pinned
 * through its parts (the pins of lattice.c, ibm.c, membrane.c), by physical
 * checks (no force without deformation, mass conservation, momentum balance
 * of spreading) and by the paper's printed numbers: run to kappa t = 120 on
 * the smallest case of Tab. convergence (H = 35, 1 280 faces, 2-, 3- and
 * 4-point stencils) it gives the table's deviations from the small-deformation
 * theory of Sec. III (D/G = 25/4, theta/pi = 1/4 - 15 G/8) and volume drifts
 * in the ranges of Sec. V.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

struct orc_sim {
    int nx, ny, nz, n;
    double tau;
    real u_wall;
    size_t N;
    real *f, *f_new, *force;
    int n_caps, n_nodes, n_tri;
    int cap_node0[1024], cap_nn[1024], cap_tri0[1024], cap_nt[1024];
    real cap_ks[1024], cap_ka[1024];
    real *X0, *x, *F, *u, *u_prev;
    int *tri;
    int integrator, eq_order, have_prev;
};

orc_sim *orc_sim_create(int nx, int ny, int nz, double tau, int delta_n,
                        real u_wall) {
    if (nx < 1 || ny < 1 || nz < 1 || delta_n < 2 || delta_n > 4 || !(tau > 0.5))
        return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->nx = nx; s->ny = ny; s->nz = nz; s->n = delta_n;
    s->tau = tau; s->u_wall = u_wall;
    s->eq_order = 2;
    s->N = (size_t)nx * ny * nz;
    s->f = (real *)calloc(19 * s->N, sizeof(real));
    s->f_new = (real *)calloc(19 * s->N, sizeof(real));
    s->force = (real *)calloc(3 * s->N, sizeof(real));
    if (!s->f || !s->f_new || !s->force) {
        orc_sim_destroy(s);
        return NULL;
    }
    orc_init_couette(nx, ny, nz, u_wall, s->f);
    return s;
}

void orc_sim_destroy(orc_sim *s) {
    if (!s) return;
    free(s->f); free(s->f_new); free(s->force);
    free(s->X0); free(s->x); free(s->F); free(s->u); free(s->u_prev); free(s->tri);
    free(s);
}

int orc_sim_add_capsule(orc_sim *s, int n_nodes, const real *X0, int n_tri,
                        const int *tri, real ks, real ka) {
    if (s->n_caps >= 1024 || n_nodes < 4 || n_tri < 4) return -1;
    int nn = s->n_nodes + n_nodes, nt = s->n_tri + n_tri;
    real *X0n = (real *)realloc(s->X0, sizeof(real) * 3 * nn);
    if (X0n) s->X0 = X0n;
    real *xn = (real *)realloc(s->x, sizeof(real) * 3 * nn);
    if (xn) s->x = xn;
    real *Fn = (real *)realloc(s->F, sizeof(real) * 3 * nn);
    if (Fn) s->F = Fn;
    real *un = (real *)realloc(s->u, sizeof(real) * 3 * nn);
    if (un) s->u = un;
    real *upn = (real *)realloc(s->u_prev, sizeof(real) * 3 * nn);
    if (upn) s->u_prev = upn;
    int *tn = (int *)realloc(s->tri, sizeof(int) * 3 * nt);
    if (tn) s->tri = tn;
    if (!X0n || !xn || !Fn || !un || !upn || !tn) return -2;
    for (int t = 0; t < 3 * n_tri; ++t) {
        if (tri[t] < 0 || tri[t] >= n_nodes) return -1;
        s->tri[3 * s->n_tri + t] = tri[t];
    }
    memcpy(s->X0 + 3 * s->n_nodes, X0, sizeof(real) * 3 * n_nodes);
    memcpy(s->x + 3 * s->n_nodes, X0, sizeof(real) * 3 * n_nodes);
    memset(s->F + 3 * s->n_nodes, 0, sizeof(real) * 3 * n_nodes);
    memset(s->u + 3 * s->n_nodes, 0, sizeof(real) * 3 * n_nodes);
    int id = s->n_caps++;
    s->cap_node0[id] = s->n_nodes;
    s->cap_nn[id] = n_nodes;
    s->cap_tri0[id] = s->n_tri;
    s->cap_nt[id] = n_tri;
    s->cap_ks[id] = ks;
    s->cap_ka[id] = ka;
    s->n_nodes = nn;
    s->n_tri = nt;
    s->have_prev = 0;
    return id;
}

int orc_sim_set_integrator(orc_sim *s, int mode) {
    if (mode != 0 && mode != 1) return -1;
    s->integrator = mode;
    s->have_prev = 0;
    return 0;
}

int orc_sim_set_equilibrium(orc_sim *s, int order) {
    if (order != 1 && order != 2) return -1;
    s->eq_order = order;
    return 0;
}

int orc_sim_n_nodes(const orc_sim *s) { return s->n_nodes; }

void orc_sim_init_couette(orc_sim *s) {
    orc_init_couette(s->nx, s->ny, s->nz, s->u_wall, s->f);
    memset(s->force, 0, sizeof(real) * 3 * s->N);
}

/* Lattice velocity of Eq. (lbmmomenta1) with the last spread force. */
static void velocity_field(const orc_sim *s, real *ufield, real *rho_out) {
    const int nthreads = orc_get_threads();
    const long long N = (long long)s->N;
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
    for (long long cell = 0; cell < N; ++cell) {
        real fi[19], fc[3], rho, u[3];
        for (int i = 0; i < 19; ++i) fi[i] = s->f[i * s->N + cell];
        for (int a = 0; a < 3; ++a) fc[a] = s->force[a * s->N + cell];
        orc_moments(fi, fc, &rho, u);
        if (ufield)
            for (int a = 0; a < 3; ++a) ufield[a * s->N + cell] = u[a];
        if (rho_out) rho_out[cell] = rho;
    }
}

int orc_sim_step(orc_sim *s, int n_steps) {
    real *ufield = (real *)malloc(sizeof(real) * 3 * s->N);
    if (!ufield) return -2;
    int rc = 0;
    for (int step = 0; step < n_steps && rc == 0; ++step) {
        /* 1. FEM forces F_i(t) */
        for (int c = 0; c < s->n_caps; ++c) {
            int n0 = s->cap_node0[c];
            orc_membrane_forces(s->cap_nn[c], s->X0 + 3 * n0, s->x + 3 * n0,
                                s->cap_nt[c], s->tri + 3 * s->cap_tri0[c],
                                s->cap_ks[c], s->cap_ka[c], s->F + 3 * n0);
        }
        /* 2. spreading f(X, t) */
        rc = orc_spread(s->nx, s->ny, s->nz, s->n, s->n_nodes, s->x, s->F, s->force);
        if (rc) break;
        /* 3. lattice Boltzmann step with f(X, t) */
        rc = orc_lbm_step_eq(s->nx, s->ny, s->nz, s->tau, s->u_wall, s->f, s->force, s->f_new, s->eq_order);
        if (rc) break;
        real *tmp = s->f;
        s->f = s->f_new;
        s->f_new = tmp;
        /* 4. interpolation of u(X, t+1) at x_i(t); u_i(t) kept */
        memcpy(s->u_prev, s->u, sizeof(real) * 3 * s->n_nodes);
        velocity_field(s, ufield, NULL);
        rc = orc_interpolate(s->nx, s->ny, s->nz, s->n, s->n_nodes, s->x, ufield, s->u);
        if (rc) break;
        /* 5. advection: Euler, or Adams-Bashforth once u_i(t) exists */
        if (s->integrator == 1 && s->have_prev)
            for (int k = 0; k < 3 * s->n_nodes; ++k) s->x[k] += 1.5 * s->u[k] - 0.5 * s->u_prev[k];
        else
            for (int k = 0; k < 3 * s->n_nodes; ++k) s->x[k] += s->u[k];
        s->have_prev = 1;
    }
    free(ufield);
    return rc;
}

void orc_sim_get_f(const orc_sim *s, real *f) {
    memcpy(f, s->f, sizeof(real) * 19 * s->N);
}
void orc_sim_set_f(orc_sim *s, const real *f) {
    memcpy(s->f, f, sizeof(real) * 19 * s->N);
}
void orc_sim_get_nodes(const orc_sim *s, real *x) {
    memcpy(x, s->x, sizeof(real) * 3 * s->n_nodes);
}
void orc_sim_set_nodes(orc_sim *s, const real *x) {
    memcpy(s->x, x, sizeof(real) * 3 * s->n_nodes);
    s->have_prev = 0;
}
void orc_sim_get_force_field(const orc_sim *s, real *force) {
    memcpy(force, s->force, sizeof(real) * 3 * s->N);
}
void orc_sim_get_node_forces(const orc_sim *s, real *F) {
    memcpy(F, s->F, sizeof(real) * 3 * s->n_nodes);
}
void orc_sim_get_node_velocities(const orc_sim *s, real *u) {
    memcpy(u, s->u, sizeof(real) * 3 * s->n_nodes);
}
void orc_sim_get_density(const orc_sim *s, real *rho) { velocity_field(s, NULL, rho); }
void orc_sim_get_velocity(const orc_sim *s, real *u) { velocity_field(s, u, NULL); }
