/*
 * oracle.h -- FP64 CPU oracle of the immersed-boundary lattice-Boltzmann
 * finite-element (IB-LBM-FEM) time step of Krueger, Varnik and Raabe,
 * "Efficient and accurate simulations of deformable particles immersed in a
 * fluid using a combined immersed boundary lattice Boltzmann finite element
 * method" (arXiv:1004.2416).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  The CUDA library never calls
 * it, includes it or links it, and the two share no source: no kernel, header,
 * helper, table or constant generator.
 *
 * Every routine is the paper's definition written out in plain double
 * precision (the type `real` below), in the paper's order and notation, with
 * no blocking, fusion or reordering.  Where the paper is silent or ambiguous
 * the reading taken is stated beside the code.  The whole-lattice loops may
 * run on several threads (orc_set_threads) with identical results.
 *
 * Conventions shared with the paper (Sec. II, Sec. IV):
 *   lattice units dx = dt = 1, c_s^2 = 1/3, rest density rho0 = 1;
 *   lattice cell (x, y, z), 0 <= x < nx etc., linear index x + nx*(y + ny*z);
 *   population arrays are [19][nz][ny][nx] (direction slowest);
 *   vector fields are [3][nz][ny][nx];
 *   membrane node arrays are [n][3] (x, y, z per node).
 *
 * Parity status of each function is listed in the header comment of the .c
 * file that defines it.  Return codes: 0 ok, -1 bad argument, -5 a stencil
 * cell lies outside the walls (z < 0 or z >= nz), -2 out of memory.
 */
#ifndef IBLBM_ORACLE_H
#define IBLBM_ORACLE_H

#include <math.h>

/* The arithmetic type of the method.  The oracle proper is built with
 * real = double.  Built with ORC_COMPLEX_STEP, real = double _Complex and the
 * same code evaluates the method at p + i h d: the imaginary part of any
 * result, divided by h, is its derivative along d (the complex-step method of
 * Squire and Trapp, 1998), exact to rounding because nothing is subtracted.
 * Only the helpers below depend on the choice: decisions (branches, floor,
 * the sign of |x|) take the real part, sqrt and atan2 their analytic
 * continuations. */
#ifdef ORC_COMPLEX_STEP
#include <complex.h>
#undef I /* the oracle names the inertia tensor I; the imaginary unit is _Complex_I */
typedef double _Complex real;
#define RE(x) creal(x)
static inline real r_sqrt(real x) { return csqrt(x); }
static inline real r_abs(real x) { return creal(x) < 0.0 ? -x : x; }
/* atan2 of the real parts plus its first-order change along the imaginary
 * parts: d atan2(y, x) = (x dy - y dx) / (x^2 + y^2). */
static inline real r_atan2(real y, real x) {
    const double xr = creal(x), yr = creal(y);
    return atan2(yr, xr) + _Complex_I * ((xr * cimag(y) - yr * cimag(x)) / (xr * xr + yr * yr));
}
#else
typedef double real;
#define RE(x) (x)
static inline real r_sqrt(real x) { return sqrt(x); }
static inline real r_abs(real x) { return fabs(x); }
static inline real r_atan2(real y, real x) { return atan2(y, x); }
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- lattice.c : Sec. II.A -------------------------------------------- */

/* D3Q19 velocity set in the numbering of Fig. d3q19, the standard D3Q19
 * weights (cited to Qian et al. in Sec. II.A, values not printed) and the
 * index of the opposite direction. */
void orc_d3q19(int c[19][3], double w[19], int opp[19]);

/* Eq. (equilibrium): f_i^eq = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u). */
real orc_feq(int i, real rho, const real u[3]);

/* Sec. IV.A: the linearised equilibrium w_i rho (1 + 3 c.u). */
real orc_feq_linear(int i, real rho, const real u[3]);

/* Eq. (latticeforce), Guo forcing term F_i for body force density f. */
real orc_guo(int i, double tau, const real u[3], const real f[3]);

/* Eqs. (lbmmomenta0), (lbmmomenta1): rho = sum f_i,
 * rho u = sum c_i f_i + f/2 (dt = 1). */
void orc_moments(const real fi[19], const real force[3], real *rho,
                 real u[3]);

/* One step of Eq. (lbequation) on the whole lattice: BGK collision with the
 * Guo term, streaming periodic in x and y, moving-wall bounce-back at the
 * half-way planes z = -1/2 (velocity -u_wall along x) and z = nz - 1/2
 * (velocity +u_wall).  f, f_out: [19][cells]; force: [3][cells] or NULL. */
int orc_lbm_step(int nx, int ny, int nz, double tau, real u_wall,
                 const real *f, const real *force, real *f_out);
/* The same with the equilibrium of order 2 (Eq. equilibrium) or 1 (Sec. IV.A). */
/* Threads of the whole-lattice loops (collide-and-stream and the velocity
 * field); default 1.  Results are bit-identical for every count: each output
 * element is written by one cell only, and the spreading, the membrane forces
 * and every reduction stay serial in their fixed order. */
void orc_set_threads(int n);
int orc_get_threads(void);
int orc_lbm_step_eq(int nx, int ny, int nz, double tau, real u_wall,
                    const real *f, const real *force, real *f_out, int order);

/* Equilibrium populations of the linear Couette profile
 * u_x(z) = (2 u_wall / nz) (z - (nz - 1)/2), rho = 1. */
void orc_init_couette(int nx, int ny, int nz, real u_wall, real *f);

/* ---- ibm.c : Sec. II.C -------------------------------------------------- */

/* Eqs. (2point), (3point), (4point): phi_n(r), n = 2, 3, 4. */
real orc_phi(int n, real r);

/* First lattice index of the n-point stencil around coordinate x. */
int orc_stencil_base(int n, real x);

/* Eq. (forcespreading): force_out[3][cells] = sum_i F_i delta(X - x_i).
 * force_out is overwritten (zeroed first). */
int orc_spread(int nx, int ny, int nz, int n, int n_nodes, const real *x,
               const real *F, real *force_out);

/* Eq. (velocityinterpolation): u_out[i] = sum_X u(X) delta(X - x_i),
 * u_field [3][cells]. */
int orc_interpolate(int nx, int ny, int nz, int n, int n_nodes,
                    const real *x, const real *u_field, real *u_out);

/* ---- membrane.c : Sec. II.B ---------------------------------------------- */

/* Energy A0 w^S of one face, Eqs. (constitutivelaw) and (c)-(lambda1);
 * X0, x: the three corners [3][3] in the reference and current state. */
real orc_face_energy(const real X0[9], const real x[9], real ks,
                       real ka);

/* Same energy and the corner forces F = -dW/dx (Eq. forcefromenergy). */
real orc_face_forces(const real X0[9], const real x[9], real ks,
                       real ka, real F[9]);

/* Total energy and node forces of one membrane; F [n][3] is overwritten. */
real orc_membrane_forces(int n_nodes, const real *X0, const real *x,
                           int n_tri, const int *tri, real ks, real ka,
                           real *F);

/* Invariants (I1, I2) of one face, from the a, b, c route. */
void orc_face_invariants(const real X0[9], const real x[9], real *I1,
                         real *I2);

/* ---- mesh.c : Sec. II.D --------------------------------------------------- */

/* Icosahedron subdivided m times, radius r, centre c.  nodes: room for
 * 10*4^m + 2 nodes [n][3]; tri: room for 20*4^m faces [f][3].
 * Returns the node count. */
int orc_icosphere(int m, double r, const double c[3], double *nodes, int *tri);

/* ---- taylor.c : Sec. III ------------------------------------------------- */

/* Volume, area, centroid and inertia tensor of a closed membrane, and the
 * Taylor deformation and inclination derived from them.  out[16] =
 * {D, theta, r_a, r_b, r_c, V, A, c_x, c_y, c_z,
 *  I_xx, I_yy, I_zz, I_xy, I_xz, I_yz}. */
int orc_taylor(int n_nodes, const real *x, int n_tri, const int *tri,
               real out[16]);

/* Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations: eigenvalues
 * ascending, eigenvectors in the columns of vec. */
void orc_eig3(const real A[9], real eval[3], real vec[9]);

/* ---- diag.c : shape and mesh diagnostics --------------------------------- */

/* Angular velocity omega_i = -dphi_i/dt of every node about the centroid in
 * the xz plane between two snapshots (c0, c1 the centroids); returns the mean. */
double orc_tank_treading(int n, const double *x0, const double *x1, const double c0[3],
                         const double c1[3], double dt, double *omega);
/* Eq. (chisquare) fit about c: out[9] = {zeta_x, zeta_y, zeta_z, zeta_xz,
 * r_a, r_b, r_c, D, theta}. */
int orc_ellipsoid_fit(int n, const double *x, const double c[3], double out[9]);
/* Relative face area deviation dA/A0: out = {mean, standard deviation, max |.|}. */
int orc_face_area_stats(int n_tri, const int *tri, const double *X0, const double *x, double out[3]);

/* ---- sim.c : Sec. II.C sub-step list ------------------------------------- */

typedef struct orc_sim orc_sim;

orc_sim *orc_sim_create(int nx, int ny, int nz, double tau, int delta_n,
                        real u_wall);
void orc_sim_destroy(orc_sim *s);
/* Adds a membrane; the current shape starts equal to the reference shape.
 * Returns the capsule id (>= 0) or a negative error. */
int orc_sim_add_capsule(orc_sim *s, int n_nodes, const real *X0, int n_tri,
                        const int *tri, real ks, real ka);
int orc_sim_n_nodes(const orc_sim *s);
void orc_sim_init_couette(orc_sim *s);
/* n_steps of the sub-step list: forces, spread, LBM, interpolate, advect. */
int orc_sim_step(orc_sim *s, int n_steps);
/* Variants: integrator 0 = Euler, Eq. (positionupdate); 1 = the
 * Adams-Bashforth rule of Sec. II.C.  Equilibrium order 2 = Eq. (equilibrium),
 * 1 = linearised (Sec. IV.A).  Return -1 for other values. */
int orc_sim_set_integrator(orc_sim *s, int mode);
int orc_sim_set_equilibrium(orc_sim *s, int order);
void orc_sim_get_f(const orc_sim *s, real *f);
void orc_sim_set_f(orc_sim *s, const real *f);
void orc_sim_get_nodes(const orc_sim *s, real *x);
void orc_sim_set_nodes(orc_sim *s, const real *x);
/* Last spread force density f(X, t) [3][cells]. */
void orc_sim_get_force_field(const orc_sim *s, real *force);
/* Node forces F_i(t) and interpolated velocities u_i(t+1) of the last step. */
void orc_sim_get_node_forces(const orc_sim *s, real *F);
void orc_sim_get_node_velocities(const orc_sim *s, real *u);
/* rho and u = (sum c f + f_last/2)/rho of the current populations. */
void orc_sim_get_density(const orc_sim *s, real *rho);
void orc_sim_get_velocity(const orc_sim *s, real *u);

#ifdef ORC_COMPLEX_STEP
/* ---- tangent.c (complex-step build only) ---------------------------------- */

/* The Taylor deformation D of the final shape after n_steps of the sub-step
 * list (one capsule starting in its reference shape X0, Couette start) and
 * its derivative along the direction (du_wall, dX0 [n][3], dks) in the
 * parameters (u_wall, X0, k_s) at fixed C = k_alpha / k_s: out[0] = D,
 * out[1] = dD.  h is the complex step (e.g. 1e-30). */
int orc_tangent_taylor_D(int nx, int ny, int nz, double tau, int delta_n,
                         double u_wall, double du_wall, int n_nodes, const double *X0,
                         const double *dX0, int n_tri, const int *tri, double ks,
                         double dks, double C, int n_steps, double h, double out[2]);
#endif

#ifdef __cplusplus
}
#endif
#endif
