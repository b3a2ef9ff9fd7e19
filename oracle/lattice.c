/*
 * lattice.c -- oracle of the D3Q19 BGK lattice Boltzmann step with Guo
 * forcing and moving-wall bounce-back (Sec. II.A).  Test infrastructure only.
 *
 * Pins (tests/test_oracle_lattice.py):
 *   velocity set     -- transcription of Fig. d3q19 (tests/golden/d3q19_figure.txt)
 *   weights          -- isotropy identities up to fourth order (closed form)
 *   orc_feq          -- zeroth, first and second moments (closed form)
 *   orc_guo          -- zeroth, first and second moments (closed form)
 *   orc_lbm_step     -- mass conservation, streaming of single populations,
 *                       moving-wall reflection of a single population,
 *                       stationary linear Couette profile (tau = 1) and
 *                       a linear profile at tau != 1
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include "oracle.h"

/* Threads of the whole-lattice loops (orc_set_threads; 1 = no parallel
 * region).  Each cell's update writes output elements that no other cell
 * writes (streaming is a permutation; a bounced population lands in its own
 * cell, in the direction no neighbour streams into), so results do not depend
 * on the thread count. */
static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return g_threads; }

/* Fig. d3q19: the TikZ coordinates of arrows 1..18 divided by two. */
static const int C[19][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
    {0, 0, 1},   {0, 0, -1},  {1, 0, 1},  {-1, 0, -1}, {-1, -1, 0},
    {1, 1, 0},   {-1, 0, 1},  {1, 0, -1}, {1, -1, 0},  {-1, 1, 0},
    {0, -1, 1},  {0, 1, -1},  {0, -1, -1}, {0, 1, 1}};

/* Standard D3Q19 weights: rest 1/3, axis neighbours 1/18, diagonal
 * neighbours 1/36 (the paper cites them to Qian et al. without values). */
static double weight(int i) {
    int s = abs(C[i][0]) + abs(C[i][1]) + abs(C[i][2]);
    if (s == 0) return 1.0 / 3.0;
    if (s == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static int opposite(int i) {
    for (int j = 0; j < 19; ++j)
        if (C[j][0] == -C[i][0] && C[j][1] == -C[i][1] && C[j][2] == -C[i][2])
            return j;
    return -1;
}

void orc_d3q19(int c[19][3], double w[19], int opp[19]) {
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) c[i][a] = C[i][a];
        w[i] = weight(i);
        opp[i] = opposite(i);
    }
}

/* Eq. (equilibrium). */
real orc_feq(int i, real rho, const real u[3]) {
    real cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
    real uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return weight(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* The linearised equilibrium of Sec. IV.A, f_i^eq = w_i rho (1 + 3 c_i.u):
 * the second-order terms of Eq. (equilibrium) dropped. */
real orc_feq_linear(int i, real rho, const real u[3]) {
    real cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
    return weight(i) * rho * (1.0 + 3.0 * cu);
}

/* Eq. (latticeforce) with c_s^2 = 1/3:
 * F_i = (1 - 1/(2 tau)) w_i [ (c_i - u)/c_s^2 + (c_i.u) c_i / c_s^4 ] . f */
real orc_guo(int i, double tau, const real u[3], const real f[3]) {
    const double cs2 = 1.0 / 3.0;
    real cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
    real s = 0.0;
    for (int a = 0; a < 3; ++a) {
        real term = (C[i][a] - u[a]) / cs2 + cu * C[i][a] / (cs2 * cs2);
        s += term * f[a];
    }
    return (1.0 - 1.0 / (2.0 * tau)) * weight(i) * s;
}

/* Eqs. (lbmmomenta0) and (lbmmomenta1). */
void orc_moments(const real fi[19], const real force[3], real *rho,
                 real u[3]) {
    real r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 19; ++i) {
        r += fi[i];
        for (int a = 0; a < 3; ++a) j[a] += C[i][a] * fi[i];
    }
    for (int a = 0; a < 3; ++a) {
        real fa = force ? force[a] : 0.0;
        u[a] = (j[a] + 0.5 * fa) / r;
    }
    *rho = r;
}

static int wrap(int a, int n) { return ((a % n) + n) % n; }

/* Eq. (lbequation), the sub-step 3 of the step list in Sec. II.C.
 * Collision at every cell, then each post-collision population moves to
 * x + c_i.  A population that would cross a wall plane is reflected back into
 * its own cell in the opposite direction and picks up the moving-wall term of
 * Ladd's bounce-back (cited in Sec. II.A):
 *     f_opp(i)(x, t+1) = f_i*(x, t) - 2 w_i rho0 (c_i . u_wall) / c_s^2
 * with rho0 = 1 and u_wall = (+u_wall, 0, 0) at the top plane z = nz - 1/2,
 * (-u_wall, 0, 0) at the bottom plane z = -1/2. */
int orc_lbm_step(int nx, int ny, int nz, double tau, real u_wall,
                 const real *f, const real *force, real *f_out) {
    return orc_lbm_step_eq(nx, ny, nz, tau, u_wall, f, force, f_out, 2);
}

/* The same step with the equilibrium of the given order: 2 for Eq.
 * (equilibrium), 1 for the linearised one of Sec. IV.A (the forcing term is
 * Eq. (latticeforce) in both; the paper changes only the equilibrium). */
int orc_lbm_step_eq(int nx, int ny, int nz, double tau, real u_wall,
                    const real *f, const real *force, real *f_out, int order) {
    if (nx < 1 || ny < 1 || nz < 1 || !(tau > 0.5) || (order != 1 && order != 2)) return -1;
    const size_t N = (size_t)nx * ny * nz;
    const double cs2 = 1.0 / 3.0;
    int opp[19];
    for (int i = 0; i < 19; ++i) opp[i] = opposite(i);
    const int nthreads = g_threads;
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads) if (nthreads > 1)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t cell = (size_t)x + (size_t)nx * (y + (size_t)ny * z);
                real fi[19], fc[3] = {0.0, 0.0, 0.0}, rho, u[3];
                for (int i = 0; i < 19; ++i) fi[i] = f[i * N + cell];
                if (force)
                    for (int a = 0; a < 3; ++a) fc[a] = force[a * N + cell];
                orc_moments(fi, fc, &rho, u);
                for (int i = 0; i < 19; ++i) {
                    real eq = order == 2 ? orc_feq(i, rho, u) : orc_feq_linear(i, rho, u);
                    real post = fi[i] - (fi[i] - eq) / tau + orc_guo(i, tau, u, fc);
                    int zt = z + C[i][2];
                    if (zt < 0 || zt >= nz) {
                        real uw = (zt >= nz) ? u_wall : -u_wall;
                        real cuw = C[i][0] * uw;
                        f_out[opp[i] * N + cell] =
                            post - 2.0 * weight(i) * 1.0 * cuw / cs2;
                    } else {
                        int xt = wrap(x + C[i][0], nx);
                        int yt = wrap(y + C[i][1], ny);
                        size_t t = (size_t)xt + (size_t)nx * (yt + (size_t)ny * zt);
                        f_out[i * N + t] = post;
                    }
                }
            }
    return 0;
}

/* Initial state (reading: the paper does not state one): equilibrium at
 * rho = 1 with the linear Couette profile between the moving walls,
 * shear rate 2 u_wall / H with H = nz. */
void orc_init_couette(int nx, int ny, int nz, real u_wall, real *f) {
    const size_t N = (size_t)nx * ny * nz;
    const real gamma = 2.0 * u_wall / nz;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t cell = (size_t)x + (size_t)nx * (y + (size_t)ny * z);
                real u[3] = {gamma * (z - 0.5 * (nz - 1)), 0.0, 0.0};
                for (int i = 0; i < 19; ++i) f[i * N + cell] = orc_feq(i, 1.0, u);
            }
}
