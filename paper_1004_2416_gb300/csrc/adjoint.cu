// adjoint.cu -- reverse-mode kernels of one IB-LBM-FEM time step.  Given the
// adjoints lam_x(t+1) of the node positions and lam_f(t+1) of the populations
// after step t, they produce lam_x(t), lam_f(t) and the step's contributions to
// the gradients of a scalar of the final state with respect to the shear
// modulus, the wall speed and the reference node positions.  The forward step
// (sub-step list of Sec. II.C) is
//   F = F(x; X0, k_s),  g = S(x) F,  f' = L(f, g; u_w),
//   U_i = sum_X u(X; f', g) delta(X - x_i),  x' = x + U,
// with u = (sum_i c_i f'_i + g/2)/rho.  The kernels below are, in the order
// they run, the transposes of: the interpolation (k_adj_interp, which also
// adds its lattice part to lam_f and lam_g), the collide-and-stream
// (k_adj_collide), the spreading (k_adj_spread) and the membrane forces
// (k_adj_membrane).  Forward quantities of step t come from a
// recomputation of the step: x(t), F(t), g(t) and the moments (j, rho) of f(t)
// and f(t+1), which are all the transposes need of the populations.
#include "device_common.cuh"
#include "ib_common.cuh"
#include "internal.h"

namespace iblbm {

// d phi_N / dr for the kernels of Eqs. (2point), (3point), (4point).
template <int N, typename T>
__device__ __forceinline__ T delta_dphi(T r) {
    const T a = fabs(r);
    const T sg = r < T(0) ? T(-1) : T(1);
    if constexpr (N == 2) {
        return a < T(1) ? -sg : T(0);
    } else if constexpr (N == 3) {
        if (a <= T(0.5)) return -r / sqrt(T(1) - T(3) * r * r);
        if (a < T(1.5))
            return sg * (T(-0.5) - (T(1) - a) / (T(2) * sqrt(fmax(T(1e-30), T(6) * a - T(3) * a * a - T(2)))));
        return T(0);
    } else {
        if (a <= T(1)) return sg * (T(-0.25) + (T(1) - T(2) * a) / (T(4) * sqrt(T(1) + T(4) * a - T(4) * a * a)));
        if (a < T(2))
            return sg * (T(-0.25) - (T(3) - T(2) * a) / (T(4) * sqrt(fmax(T(1e-30), T(12) * a - T(4) * a * a - T(7)))));
        return T(0);
    }
}

// One stencil cell of a node: weight w = delta(X - x) and its gradient with
// respect to the node position, gw = -(phi' phi phi, phi phi' phi, phi phi phi').
template <typename T>
struct SCell {
    bool ok;
    long long cell;
    T w, gw[3];
};

template <int N, typename T>
__device__ __forceinline__ SCell<T> stencil_cell(const PosView<T> &pos, const T *p, const int b[3], int k,
                                                 int nx, int ny, int nz) {
    SCell<T> c;
    c.ok = false;
    if (k >= N * N * N) return c;
    const int X = b[0] + k % N, Y = b[1] + (k / N) % N, Z = b[2] + k / (N * N);
    if (Z < 0 || Z >= nz) return c;
    T d[3];
    pos.rel(p, X, Y, Z, d);
    const T px = delta_phi<N>(d[0]), py = delta_phi<N>(d[1]), pz = delta_phi<N>(d[2]);
    const T qx = delta_dphi<N>(d[0]), qy = delta_dphi<N>(d[1]), qz = delta_dphi<N>(d[2]);
    c.ok = true;
    c.w = px * py * pz;
    c.gw[0] = -qx * py * pz;
    c.gw[1] = -px * qy * pz;
    c.gw[2] = -px * py * qz;
    c.cell = wrap_index(X, nx) + (long long)nx * (wrap_index(Y, ny) + (long long)ny * Z);
    return c;
}

template <int N, typename T>
__device__ __forceinline__ void node_stencil(const PosView<T> &pos, int node, T *p, int b[3]) {
    pos.approx(node, p);
    T pc[3];
    if constexpr (kPosLen<T> == 6) {
        pc[0] = p[0] + p[3]; pc[1] = p[1] + p[4]; pc[2] = p[2] + p[5];
    } else {
        pc[0] = p[0]; pc[1] = p[1]; pc[2] = p[2];
    }
    b[0] = stencil_first<N>(pc[0]);
    b[1] = stencil_first<N>(pc[1]);
    b[2] = stencil_first<N>(pc[2]);
}

// Moments of the stored populations of a step, kept by the recomputation so
// that the reverse sweep never reads populations: M = (j_x, j_y, j_z, rho - 1).
template <typename S, typename T>
__global__ void __launch_bounds__(256)
    k_adj_moments(const S *__restrict__ pop, typename Vec4<T>::type *__restrict__ M, long long ncell) {
    const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= ncell) return;
    T drho = T(0), j[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const T v = Store<S, T>::load(pop + i * ncell + cell);
        drho += v;
        if (q_cx(i)) j[0] += q_cx(i) > 0 ? v : -v;
        if (q_cy(i)) j[1] += q_cy(i) > 0 ? v : -v;
        if (q_cz(i)) j[2] += q_cz(i) > 0 ? v : -v;
    }
    M[cell] = typename Vec4<T>::type{j[0], j[1], j[2], drho};
}

// density and velocity (j + g/2)/rho of a cell from its stored moments
template <typename T>
__device__ __forceinline__ void cell_moments(const typename Vec4<T>::type *__restrict__ M, long long cell,
                                             T gx, T gy, T gz, T &rho, T u[3]) {
    const typename Vec4<T>::type m = M[cell];
    rho = T(1) + m.w;
    const T inv = T(1) / rho;
    u[0] = (m.x + T(0.5) * gx) * inv;
    u[1] = (m.y + T(0.5) * gy) * inv;
    u[2] = (m.z + T(0.5) * gz) * inv;
}

__device__ __forceinline__ void add_vec(float4 *f, float x, float y, float z) { add_force(f, x, y, z); }
__device__ __forceinline__ void add_vec(dvec4 *f, double x, double y, double z) { add_force(f, x, y, z); }

// ---- transpose of the interpolation U_i = sum_X u(X) delta(X - x_i) ----------------------
// lam_U = lam_x(t+1).  The node part is sum_X (lam_U_i . u(X)) grad delta, so
// lam_x(t) = lam_U + that term.  The lattice adjoint of u(X) is
// m(X) = sum_i lam_U_i delta(X - x_i); through u = (j + g/2)/rho it reaches
// the populations after the step, lam_f'(X)_j += m . (c_j - u)/rho, and the
// force density, lam_g(X) = m / (2 rho).  Both are linear in m, so every
// node adds its own share with atomics: P = lam_U w / rho, s = P . u,
// lam_f'(X)_j += P . c_j - s and mu(X) += P / 2 (the part of lam_g, which the
// collide adjoint picks up and clears).
template <int N, typename T>
__global__ void __launch_bounds__(256)
    k_adj_interp(int n_nodes, PosView<T> pos, const typename Vec4<T>::type *__restrict__ M1,
                 const typename Vec4<T>::type *__restrict__ g, const typename Vec4<T>::type *__restrict__ lamU,
                 typename Vec4<T>::type *__restrict__ mu, T *__restrict__ lam,
                 typename Vec4<T>::type *__restrict__ lamx_out, int nx, int ny, int nz, long long ncell) {
    using V4 = typename Vec4<T>::type;
    const int lane = threadIdx.x & 31;
    const int node = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (node >= n_nodes) return;
    T p[kPosLen<T>];
    int b[3];
    node_stencil<N, T>(pos, node, p, b);
    const V4 lu = lamU[node];
    T acc[3] = {T(0), T(0), T(0)};
    for (int k = lane; k < N * N * N; k += 32) {
        const SCell<T> c = stencil_cell<N, T>(pos, p, b, k, nx, ny, nz);
        if (!c.ok) continue;
        const V4 gv = g[c.cell];
        T rho, u[3];
        cell_moments<T>(M1, c.cell, gv.x, gv.y, gv.z, rho, u);
        if (c.w != T(0)) {
            const T wr = c.w / rho;
            const T P[3] = {lu.x * wr, lu.y * wr, lu.z * wr};
            const T sP = P[0] * u[0] + P[1] * u[1] + P[2] * u[2];
            add_vec(&mu[c.cell], T(0.5) * P[0], T(0.5) * P[1], T(0.5) * P[2]);
#pragma unroll
            for (int j = 0; j < 19; ++j) {
                T v = -sP;
                if (q_cx(j)) v += q_cx(j) > 0 ? P[0] : -P[0];
                if (q_cy(j)) v += q_cy(j) > 0 ? P[1] : -P[1];
                if (q_cz(j)) v += q_cz(j) > 0 ? P[2] : -P[2];
                atomicAdd(lam + j * ncell + c.cell, v);
            }
        }
        const T lu_u = lu.x * u[0] + lu.y * u[1] + lu.z * u[2];
        for (int a = 0; a < 3; ++a) acc[a] += lu_u * c.gw[a];
    }
    for (int a = 0; a < 3; ++a) acc[a] = warp_sum(acc[a]);
    if (lane == 0) lamx_out[node] = V4{lu.x + acc[0], lu.y + acc[1], lu.z + acc[2], T(0)};
}

// ---- transpose of the collide-and-stream -----------------------------------------------
// Streaming pushed f*_i(X) to X + c_i (or, across a wall, into direction
// opp(i) of X with the term -6 w_i c_ix s u_w, s = +1 at the top wall and -1 at
// the bottom one); its transpose pulls a_i = lam'(X + c_i)_i, or lam'(X)_opp(i)
// across a wall, which also gives d/du_w += a_i (-6 w_i c_ix s).  With
// rho = sum f, u = (sum c f + g/2)/rho, the BGK + Guo collision
// C_i = f_i - omega (f_i - feq_i) + Guo_i has the transpose
//   lam_j = (1 - omega) a_j + omega A_rho + K . (c_j - u)/rho,
//   A_rho = sum_i a_i dfeq_i/drho,  A_u = sum_i a_i dfeq_i/du,
//   B_u = sum_i a_i dGuo_i/du,  K = omega A_u + B_u,
// and lam_g = mu + K/(2 rho) + sum_i a_i dGuo_i/dg in force-flagged cells
// (mu: the interpolation adjoint's part).
// Every one of these sums is a linear form in the weighted moments
// S0 = sum w a, S1 = sum w a c, S2 = sum w a c c^T of the pulled adjoints
// (f_eq and the Guo term are quadratic in c), and sum a dGuo/dg equals A_u,
// so the kernel gathers the 19 adjoints once and forms the 10 moments.
// g(t) is cleared after it is read.
// I: unsigned type wide enough for the cell index (32-bit divisions when the
// lattice has fewer than 2^32 cells).
template <typename T, typename I>
__global__ void __launch_bounds__(256)
    k_adj_collide(const typename Vec4<T>::type *__restrict__ M0, typename Vec4<T>::type *__restrict__ g,
                  const uint8_t *__restrict__ flags, const T *__restrict__ lam_in, T *__restrict__ lam_out,
                  typename Vec4<T>::type *__restrict__ mu, typename Vec4<T>::type *__restrict__ lamg,
                  double *__restrict__ uw_partial, Lattice L, T omega) {
    using V4 = typename Vec4<T>::type;
    __shared__ double red[8];
    const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double uwg = 0.0;
    if (cell < L.ncell) {
        const int nx = L.nx, ny = L.ny, nz = L.nz;
        const I c = (I)cell;
        const I r = c / (I)nx;
        const int x = (int)(c - r * (I)nx);
        const I zq = r / (I)ny;
        const int y = (int)(r - zq * (I)ny), z = (int)zq;
        // offsets of the periodic neighbours in x and y and of the planes in z
        // (unsigned wrap-around: every sum lands inside the lattice)
        const I sy = (I)nx, sz = (I)nx * (I)ny;
        const I dxp = (x + 1 == nx) ? (I)1 - (I)nx : (I)1, dxm = (x == 0) ? (I)nx - (I)1 : ~(I)0;
        const I dyp = (y + 1 == ny) ? sy - sz : sy, dym = (y == 0) ? sz - sy : (I)0 - sy;
        T a[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int cx = q_cx(i), cy = q_cy(i), cz = q_cz(i);
            if ((cz > 0 && z + 1 == nz) || (cz < 0 && z == 0)) {
                a[i] = (lam_in + q_opp(i) * L.ncell)[c];
                if (cx) uwg += (double)a[i] * (-6.0 * q_w<double>(i) * cx * (cz > 0 ? 1.0 : -1.0));
            } else {
                I nb = c;
                if (cx) nb += cx > 0 ? dxp : dxm;
                if (cy) nb += cy > 0 ? dyp : dym;
                if (cz) nb += cz > 0 ? sz : (I)0 - sz;
                a[i] = (lam_in + i * L.ncell)[nb];
            }
        }
        const bool flagged = flags[((I)z * (I)L.nfy + (I)(y / L.fty)) * (I)L.nfx + (I)(x / L.ftx)] != 0;
        V4 gv{};
        if (flagged) {
            gv = g[c];
            g[c] = V4{};  // last reader of g(t): leave the buffer zero for the next recomputation
        }
        T rho, u[3];
        cell_moments<T>(M0, (long long)c, gv.x, gv.y, gv.z, rho, u);
        // weighted moments of the pulled adjoints: S0 = sum w a, S1 = sum w a c,
        // S2 = sum w a c c^T (xx, yy, zz, xy, xz, yz)
        T S0 = T(0), S1[3] = {T(0), T(0), T(0)}, S2[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int cx = q_cx(i), cy = q_cy(i), cz = q_cz(i);
            const T aw = a[i] * q_w<T>(i);
            S0 += aw;
            if (cx) { S1[0] += cx > 0 ? aw : -aw; S2[0] += aw; }
            if (cy) { S1[1] += cy > 0 ? aw : -aw; S2[1] += aw; }
            if (cz) { S1[2] += cz > 0 ? aw : -aw; S2[2] += aw; }
            if (cx && cy) S2[3] += cx * cy > 0 ? aw : -aw;
            if (cx && cz) S2[4] += cx * cz > 0 ? aw : -aw;
            if (cy && cz) S2[5] += cy * cz > 0 ? aw : -aw;
        }
        const T S2u[3] = {S2[0] * u[0] + S2[3] * u[1] + S2[4] * u[2],
                          S2[3] * u[0] + S2[1] * u[1] + S2[5] * u[2],
                          S2[4] * u[0] + S2[5] * u[1] + S2[2] * u[2]};
        const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        // A_rho = sum a dfeq/drho, A_u = sum a dfeq/du (= sum a dGuo/dg as well)
        const T Arho = S0 * (T(1) - T(1.5) * uu) + T(3) * (S1[0] * u[0] + S1[1] * u[1] + S1[2] * u[2]) +
                       T(4.5) * (u[0] * S2u[0] + u[1] * S2u[1] + u[2] * S2u[2]);
        T Au[3], K[3];
        const T guo = T(1) - T(0.5) * omega;
        for (int d = 0; d < 3; ++d) Au[d] = T(3) * S1[d] + T(9) * S2u[d] - T(3) * u[d] * S0;
        for (int d = 0; d < 3; ++d) K[d] = omega * rho * Au[d];
        if (flagged) {
            // B_u = sum a dGuo/du = -3 g S0 + 9 S2 g
            const T gg[3] = {gv.x, gv.y, gv.z};
            const T S2g[3] = {S2[0] * gg[0] + S2[3] * gg[1] + S2[4] * gg[2],
                              S2[3] * gg[0] + S2[1] * gg[1] + S2[5] * gg[2],
                              S2[4] * gg[0] + S2[5] * gg[1] + S2[2] * gg[2]};
            for (int d = 0; d < 3; ++d) K[d] += guo * (T(-3) * gg[d] * S0 + T(9) * S2g[d]);
        }
        const T inv = T(1) / rho;
        const T Ki[3] = {K[0] * inv, K[1] * inv, K[2] * inv};
        const T base = omega * Arho - (Ki[0] * u[0] + Ki[1] * u[1] + Ki[2] * u[2]);
        const T keep = T(1) - omega;
#pragma unroll
        for (int j = 0; j < 19; ++j) {
            T v = base;
            if (q_cx(j)) v += q_cx(j) > 0 ? Ki[0] : -Ki[0];
            if (q_cy(j)) v += q_cy(j) > 0 ? Ki[1] : -Ki[1];
            if (q_cz(j)) v += q_cz(j) > 0 ? Ki[2] : -Ki[2];
            (lam_out + j * L.ncell)[c] = keep * a[j] + v;
        }
        if (flagged) {
            // the interpolation's part (mu, nonzero only in stencil cells, all
            // of them flagged) is taken and cleared here
            const V4 m = mu[c];
            lamg[c] = V4{m.x + T(0.5) * Ki[0] + guo * Au[0], m.y + T(0.5) * Ki[1] + guo * Au[1],
                         m.z + T(0.5) * Ki[2] + guo * Au[2], T(0)};
            mu[c] = V4{};
        }
    }
    for (int o = 16; o > 0; o >>= 1) uwg += __shfl_xor_sync(0xffffffffu, uwg, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = uwg;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        uw_partial[blockIdx.x] += s;
    }
}

// ---- transpose of the spreading g(X) = sum_i F_i delta(X - x_i) ------------------------
// lam_F_i = sum_X lam_g(X) delta(X - x_i); lam_x_i += sum_X (lam_g . F_i) grad delta.
template <int N, typename T>
__global__ void __launch_bounds__(256)
    k_adj_spread(int n_nodes, PosView<T> pos, const typename Vec4<T>::type *__restrict__ F,
                 const typename Vec4<T>::type *__restrict__ lamg, typename Vec4<T>::type *__restrict__ lamF,
                 typename Vec4<T>::type *__restrict__ lamx, int nx, int ny, int nz) {
    using V4 = typename Vec4<T>::type;
    const int lane = threadIdx.x & 31;
    const int node = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (node >= n_nodes) return;
    T p[kPosLen<T>];
    int b[3];
    node_stencil<N, T>(pos, node, p, b);
    const V4 Fi = F[node];
    T lf[3] = {T(0), T(0), T(0)}, ax[3] = {T(0), T(0), T(0)};
    for (int k = lane; k < N * N * N; k += 32) {
        const SCell<T> c = stencil_cell<N, T>(pos, p, b, k, nx, ny, nz);
        if (!c.ok) continue;
        const V4 lg = lamg[c.cell];
        lf[0] += lg.x * c.w;
        lf[1] += lg.y * c.w;
        lf[2] += lg.z * c.w;
        const T lgF = lg.x * Fi.x + lg.y * Fi.y + lg.z * Fi.z;
        for (int a = 0; a < 3; ++a) ax[a] += lgF * c.gw[a];
    }
    for (int a = 0; a < 3; ++a) {
        lf[a] = warp_sum(lf[a]);
        ax[a] = warp_sum(ax[a]);
    }
    if (lane == 0) {
        lamF[node] = V4{lf[0], lf[1], lf[2], T(0)};
        V4 l = lamx[node];
        lamx[node] = V4{l.x + ax[0], l.y + ax[1], l.z + ax[2], T(0)};
    }
}

// ---- transpose of the membrane forces F = -dW/dx ------------------------------------------
// The Jacobian dF/dx = -Hessian(W) is symmetric, so its transpose applied to
// lam_F is the directional derivative of F along lam_F: the face gradient of
// ib.cu differentiated by hand in the direction (u', v') = (lam_b - lam_a,
// lam_c - lam_a).  The same tangent of the reference gradient dW/dX0 gives
// lam_F^T dF/dX0 = -d/de dW/dX0(x + e lam_F).  With M = dW/dG0 (G0 the
// reference Gram matrix, Ginv its inverse = [[alpha, -beta], [-beta, gamma]],
// d = g - G0):  M/A0 = c0 Ginv - w1 Ginv d Ginv,
// c0 = w/2 - k_s/6 I1 + k_s/6 I2 - k_alpha/6 I2 (I2 + 1), w1 = k_s/6 (I1 + 1),
// and dW/dU = 2 (M11 U + M12 V), dW/dV = 2 (M12 U + M22 V) for the reference
// edges U = X0_b - X0_a, V = X0_c - X0_a.  Also accumulates lam_F . F / k_s, the
// step's part of dD/dk_s at fixed k_alpha / k_s.
template <typename T>
__global__ void __launch_bounds__(256)
    k_adj_membrane(int n_nodes, PosView<T> pos, const int *__restrict__ adj_off, const int *__restrict__ adj,
                   const int4 *__restrict__ tri, const typename Vec4<T>::type *__restrict__ fconst,
                   const typename Vec4<T>::type *__restrict__ fref, const typename Vec4<T>::type *__restrict__ capmod,
                   const typename Vec4<T>::type *__restrict__ F, const typename Vec4<T>::type *__restrict__ lamF,
                   typename Vec4<T>::type *__restrict__ lamx, double *__restrict__ gX0, double *__restrict__ gks) {
    using V4 = typename Vec4<T>::type;
    const int lane = threadIdx.x & 31;
    const int node = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (node >= n_nodes) return;
    T th[3] = {T(0), T(0), T(0)}, tr[3] = {T(0), T(0), T(0)};
    T ks6_node = T(0);
    const int e0 = adj_off[node], e1 = adj_off[node + 1];
    for (int e = e0 + lane; e < e1; e += 32) {
        const int ent = adj[e];
        const int f = ent >> 2, corner = ent & 3;
        const int4 t = tri[f];
        const V4 c0 = fconst[3 * f], c1 = fconst[3 * f + 1], c2 = fconst[3 * f + 2];
        T u[3], v[3], d[3];
        pos.edge_gram(t.x, t.y, t.z, c1, c2, u, v, d);
        const V4 m = capmod[t.w];
        const T ks6 = m.x, ka6 = m.y;
        ks6_node = ks6;
        const T al = c0.x, be = c0.y, ga = c0.z, ka = c0.w, A0 = c1.x;
        const T I1 = al * d[0] - T(2) * be * d[1] + ga * d[2];
        const T I2 = I1 + ka * (d[0] * d[2] - d[1] * d[1]);
        const T g11 = c1.y + d[0], g12 = c1.z + d[1], g22 = c1.w + d[2];
        const T a2 = T(2) * A0;
        const T kI2 = ka6 * I2 * ka;
        const T s_uu = a2 * (ks6 * (I1 * al - ka * d[2]) + kI2 * g22);
        const T s_uv = -a2 * (ks6 * (I1 * be - ka * d[1]) + kI2 * g12);
        const T s_vv = a2 * (ks6 * (I1 * ga - ka * d[0]) + kI2 * g11);
        // tangent direction from the corner adjoints
        const V4 la = lamF[t.x], lb = lamF[t.y], lc = lamF[t.z];
        const T ud[3] = {lb.x - la.x, lb.y - la.y, lb.z - la.z};
        const T vd[3] = {lc.x - la.x, lc.y - la.y, lc.z - la.z};
        const T dd0 = T(2) * (u[0] * ud[0] + u[1] * ud[1] + u[2] * ud[2]);
        const T dd1 = u[0] * vd[0] + u[1] * vd[1] + u[2] * vd[2] + v[0] * ud[0] + v[1] * ud[1] + v[2] * ud[2];
        const T dd2 = T(2) * (v[0] * vd[0] + v[1] * vd[1] + v[2] * vd[2]);
        const T dI1 = al * dd0 - T(2) * be * dd1 + ga * dd2;
        const T dI2 = dI1 + ka * (dd0 * d[2] + d[0] * dd2 - T(2) * d[1] * dd1);
        const T ds_uu = a2 * (ks6 * (dI1 * al - ka * dd2) + ka6 * ka * (dI2 * g22 + I2 * dd2));
        const T ds_uv = -a2 * (ks6 * (dI1 * be - ka * dd1) + ka6 * ka * (dI2 * g12 + I2 * dd1));
        const T ds_vv = a2 * (ks6 * (dI1 * ga - ka * dd0) + ka6 * ka * (dI2 * g11 + I2 * dd0));
        T tWu[3], tWv[3];
        for (int a = 0; a < 3; ++a) {
            tWu[a] = ds_uu * u[a] + s_uu * ud[a] + ds_uv * v[a] + s_uv * vd[a];
            tWv[a] = ds_uv * u[a] + s_uv * ud[a] + ds_vv * v[a] + s_vv * vd[a];
        }
        // reference gradient tangent
        const T w1 = ks6 * (I1 + T(1)), w2 = ka6 * I2 - ks6;
        const T dw = w1 * dI1 + w2 * dI2;
        const T dc0 = dw * T(0.5) - ks6 * dI1 + ks6 * dI2 - ka6 * (T(2) * I2 + T(1)) * dI2;
        // P = Ginv d Ginv and dP = Ginv dd Ginv with Ginv = [[al, -be], [-be, ga]]
        auto sandwich = [&](T s11, T s12, T s22, T &p11, T &p12, T &p22) {
            const T q11 = al * s11 - be * s12, q12 = al * s12 - be * s22;
            const T q21 = -be * s11 + ga * s12, q22 = -be * s12 + ga * s22;
            p11 = q11 * al - q12 * be;
            p12 = -q11 * be + q12 * ga;
            p22 = -q21 * be + q22 * ga;
        };
        T P11, P12, P22, dP11, dP12, dP22;
        sandwich(d[0], d[1], d[2], P11, P12, P22);
        sandwich(dd0, dd1, dd2, dP11, dP12, dP22);
        const T dM11 = dc0 * al - ks6 * dI1 * P11 - w1 * dP11;
        const T dM12 = -dc0 * be - ks6 * dI1 * P12 - w1 * dP12;
        const T dM22 = dc0 * ga - ks6 * dI1 * P22 - w1 * dP22;
        const V4 U = fref[2 * f], V = fref[2 * f + 1];
        const T Uv[3] = {U.x, U.y, U.z}, Vv[3] = {V.x, V.y, V.z};
        T tRu[3], tRv[3];
        for (int a = 0; a < 3; ++a) {
            tRu[a] = T(2) * A0 * (dM11 * Uv[a] + dM12 * Vv[a]);
            tRv[a] = T(2) * A0 * (dM12 * Uv[a] + dM22 * Vv[a]);
        }
        for (int a = 0; a < 3; ++a) {
            if (corner == 0) {
                th[a] += tWu[a] + tWv[a];
                tr[a] -= tRu[a] + tRv[a];
            } else if (corner == 1) {
                th[a] -= tWu[a];
                tr[a] += tRu[a];
            } else {
                th[a] -= tWv[a];
                tr[a] += tRv[a];
            }
        }
    }
    for (int a = 0; a < 3; ++a) {
        th[a] = warp_sum(th[a]);
        tr[a] = warp_sum(tr[a]);
    }
    ks6_node = warp_sum(ks6_node) / T(e1 - e0);  // the same on every face of a node
    if (lane == 0) {
        V4 l = lamx[node];
        lamx[node] = V4{l.x + th[0], l.y + th[1], l.z + th[2], T(0)};
        for (int a = 0; a < 3; ++a) gX0[3 * node + a] -= (double)tr[a];
        const V4 lf = lamF[node], Fi = F[node];
        if (ks6_node != T(0))
            gks[node] += ((double)lf.x * Fi.x + (double)lf.y * Fi.y + (double)lf.z * Fi.z) / (6.0 * (double)ks6_node);
    }
}

// ---- initial Couette state: d f(0) / d u_w ------------------------------------------------
// f_i(0) = feq_i(rho = 1, u_x(z)) with u_x = (2 u_w / nz)(z - (nz - 1)/2):
// sum over cells and directions of lam_f(0)_i dfeq_i/du_x du_x/du_w.
template <typename T>
__global__ void __launch_bounds__(256)
    k_adj_init_uw(const T *__restrict__ lam, Lattice L, double u_wall, double *__restrict__ partial) {
    __shared__ double red[8];
    const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double s = 0.0;
    if (cell < L.ncell) {
        const int z = (int)(cell / ((long long)L.nx * L.ny));
        const double dux = 2.0 / L.nz * (z - 0.5 * (L.nz - 1));
        const double ux = u_wall * dux;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const double cx = q_cx(i);
            const double dfeq = q_w<double>(i) * (3.0 * cx + 9.0 * cx * ux * cx - 3.0 * ux);
            s += (double)lam[i * L.ncell + cell] * dfeq * dux;
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        partial[blockIdx.x] += t;
    }
}

// ---- launchers -------------------------------------------------------------------------------
template <typename T>
static PosView<T> adj_view(void *x, void *x_lo);
template <>
PosView<double> adj_view<double>(void *x, void *) {
    return PosView<double>{(dvec4 *)x};
}
template <>
PosView<float> adj_view<float>(void *x, void *x_lo) {
    return PosView<float>{(float4 *)x, (float4 *)x_lo};
}

static unsigned node_blocks(int n) { return (unsigned)((n + 7) / 8); }
static unsigned cell_blocks(long long n) { return (unsigned)((n + 255) / 256); }

template <int N, typename T>
static void adj_step_impl(const AdjStepArgs &A, cudaStream_t s) {
    using V4 = typename Vec4<T>::type;
    const Lattice &L = A.L;
    const MeshDev &m = A.mesh;
    const PosView<T> pos = adj_view<T>(A.x, A.x_lo);
    k_adj_interp<N, T><<<node_blocks(m.n_nodes), 256, 0, s>>>(
        m.n_nodes, pos, (const V4 *)A.M1, (const V4 *)A.g, (const V4 *)A.lamx_in, (V4 *)A.mu, (T *)A.lam_in,
        (V4 *)A.lamx_out, L.nx, L.ny, L.nz, L.ncell);
    if (L.ncell <= 0xffffffffLL)
        k_adj_collide<T, unsigned><<<cell_blocks(L.ncell), 256, 0, s>>>(
            (const V4 *)A.M0, (V4 *)A.g, A.flags, (const T *)A.lam_in, (T *)A.lam_out, (V4 *)A.mu,
            (V4 *)A.lamg, A.uw_partial, L, (T)A.omega);
    else
        k_adj_collide<T, unsigned long long><<<cell_blocks(L.ncell), 256, 0, s>>>(
            (const V4 *)A.M0, (V4 *)A.g, A.flags, (const T *)A.lam_in, (T *)A.lam_out, (V4 *)A.mu,
            (V4 *)A.lamg, A.uw_partial, L, (T)A.omega);
    k_adj_spread<N, T><<<node_blocks(m.n_nodes), 256, 0, s>>>(
        m.n_nodes, pos, (const V4 *)A.F, (const V4 *)A.lamg, (V4 *)A.lamF, (V4 *)A.lamx_out, L.nx, L.ny, L.nz);
    k_adj_membrane<T><<<node_blocks(m.n_nodes), 256, 0, s>>>(
        m.n_nodes, pos, m.adj_off, m.adj, (const int4 *)m.tri, (const V4 *)m.fconst, (const V4 *)A.fref,
        (const V4 *)m.capmod, (const V4 *)A.F, (const V4 *)A.lamF, (V4 *)A.lamx_out, A.gX0, A.gks);
}

// Storage precision only enters through the moments; the reverse sweep runs
// in double for the FP64 build and in float otherwise.
void launch_adjoint_step(int prec, int delta, const AdjStepArgs &A, cudaStream_t s) {
    if (prec == kF64) {
        if (delta == 2) adj_step_impl<2, double>(A, s);
        else if (delta == 3) adj_step_impl<3, double>(A, s);
        else adj_step_impl<4, double>(A, s);
    } else {
        if (delta == 2) adj_step_impl<2, float>(A, s);
        else if (delta == 3) adj_step_impl<3, float>(A, s);
        else adj_step_impl<4, float>(A, s);
    }
}

void launch_adjoint_moments(int prec, const Lattice &L, const void *pop, void *M, cudaStream_t s) {
    if (prec == kF64)
        k_adj_moments<double, double><<<cell_blocks(L.ncell), 256, 0, s>>>((const double *)pop, (dvec4 *)M, L.ncell);
    else if (prec == kF32)
        k_adj_moments<float, float><<<cell_blocks(L.ncell), 256, 0, s>>>((const float *)pop, (float4 *)M, L.ncell);
    else
        k_adj_moments<__half, float><<<cell_blocks(L.ncell), 256, 0, s>>>((const __half *)pop, (float4 *)M, L.ncell);
}

void launch_adjoint_init_uw(int prec, const Lattice &L, const void *lam, double u_wall, double *partial,
                            cudaStream_t s) {
    if (prec == kF64)
        k_adj_init_uw<double><<<cell_blocks(L.ncell), 256, 0, s>>>((const double *)lam, L, u_wall, partial);
    else
        k_adj_init_uw<float><<<cell_blocks(L.ncell), 256, 0, s>>>((const float *)lam, L, u_wall, partial);
}

}  // namespace iblbm
