/*
 * ibm.c -- oracle of the immersed-boundary coupling (Sec. II.C): the discrete
 * delta kernels, force spreading and velocity interpolation.  Test
 * infrastructure only.
 *
 * Pins (tests/test_oracle_ibm.py):
 *   orc_phi          -- partition of unity and vanishing first moment for
 *                       n = 2, 3, 4 at every offset; sum phi3^2 = 1/2,
 *                       sum phi4^2 = 3/8, even and odd sums of phi4 = 1/2;
 *                       continuity at the branch joins; zero outside support
 *   orc_stencil_base -- every lattice node with phi != 0 lies in the stencil
 *                       (brute force over a wide window)
 *   orc_spread       -- total force and total torque conserved (closed form
 *                       from the moment identities); adjoint of
 *                       orc_interpolate (sum F.u_i = sum_X f.u)
 *   orc_interpolate  -- exact on constant and linear fields
 *
 * Readings where the paper is silent: the stencil of coordinate x covers the
 * n lattice nodes i0 .. i0+n-1 with i0 = floor(x - n/2) + 1 (phi vanishes at the
 * edge of its support, so which of two tied nodes is taken does not change a
 * value); lattice indices wrap periodically in x and y; a stencil node below
 * z = 0 or at z >= nz is an error (-5); node coordinates are not wrapped.
 */
#include <math.h>
#include <stddef.h>
#include <string.h>
#include "oracle.h"

/* Eqs. (2point), (3point), (4point). */
real orc_phi(int n, real r) {
    real a = r_abs(r);
    if (n == 2) {
        return RE(a) <= 1.0 ? 1.0 - a : 0.0;
    }
    if (n == 3) {
        if (RE(a) <= 0.5) return (1.0 + r_sqrt(1.0 - 3.0 * r * r)) / 3.0;
        if (RE(a) <= 1.5) return (5.0 - 3.0 * a - r_sqrt(-2.0 + 6.0 * a - 3.0 * r * r)) / 6.0;
        return 0.0;
    }
    if (n == 4) {
        if (RE(a) <= 1.0) return (3.0 - 2.0 * a + r_sqrt(1.0 + 4.0 * a - 4.0 * r * r)) / 8.0;
        if (RE(a) <= 2.0) return (5.0 - 2.0 * a - r_sqrt(-7.0 + 12.0 * a - 4.0 * r * r)) / 8.0;
        return 0.0;
    }
    return 0.0;
}

int orc_stencil_base(int n, real x) { return (int)floor(RE(x) - 0.5 * n) + 1; }

static int wrap(int a, int n) { return ((a % n) + n) % n; }

/* Eq. (forcespreading), delta(r) = phi(x) phi(y) phi(z).  Nodes in order,
 * stencil nodes in (z, y, x) lexicographic order. */
int orc_spread(int nx, int ny, int nz, int n, int n_nodes, const real *x,
               const real *F, real *force_out) {
    if (n < 2 || n > 4) return -1;
    const size_t N = (size_t)nx * ny * nz;
    memset(force_out, 0, 3 * N * sizeof(real));
    for (int i = 0; i < n_nodes; ++i) {
        const real *xi = x + 3 * i;
        int b[3];
        for (int a = 0; a < 3; ++a) b[a] = orc_stencil_base(n, xi[a]);
        for (int kz = 0; kz < n; ++kz) {
            int Z = b[2] + kz;
            if (Z < 0 || Z >= nz) return -5;
            for (int ky = 0; ky < n; ++ky) {
                int Y = b[1] + ky;
                for (int kx = 0; kx < n; ++kx) {
                    int X = b[0] + kx;
                    real d = orc_phi(n, X - xi[0]) * orc_phi(n, Y - xi[1]) *
                               orc_phi(n, Z - xi[2]);
                    size_t cell = (size_t)wrap(X, nx) +
                                  (size_t)nx * (wrap(Y, ny) + (size_t)ny * Z);
                    for (int a = 0; a < 3; ++a) force_out[a * N + cell] += F[3 * i + a] * d;
                }
            }
        }
    }
    return 0;
}

/* Eq. (velocityinterpolation). */
int orc_interpolate(int nx, int ny, int nz, int n, int n_nodes,
                    const real *x, const real *u_field, real *u_out) {
    if (n < 2 || n > 4) return -1;
    const size_t N = (size_t)nx * ny * nz;
    for (int i = 0; i < n_nodes; ++i) {
        const real *xi = x + 3 * i;
        real acc[3] = {0.0, 0.0, 0.0};
        int b[3];
        for (int a = 0; a < 3; ++a) b[a] = orc_stencil_base(n, xi[a]);
        for (int kz = 0; kz < n; ++kz) {
            int Z = b[2] + kz;
            if (Z < 0 || Z >= nz) return -5;
            for (int ky = 0; ky < n; ++ky) {
                int Y = b[1] + ky;
                for (int kx = 0; kx < n; ++kx) {
                    int X = b[0] + kx;
                    real d = orc_phi(n, X - xi[0]) * orc_phi(n, Y - xi[1]) *
                               orc_phi(n, Z - xi[2]);
                    size_t cell = (size_t)wrap(X, nx) +
                                  (size_t)nx * (wrap(Y, ny) + (size_t)ny * Z);
                    for (int a = 0; a < 3; ++a) acc[a] += u_field[a * N + cell] * d;
                }
            }
        }
        for (int a = 0; a < 3; ++a) u_out[3 * i + a] = acc[a];
    }
    return 0;
}
