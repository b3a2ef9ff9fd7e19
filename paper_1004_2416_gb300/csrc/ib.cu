// ib.cu -- immersed-boundary coupling and finite-element membrane forces.
//
//   k_force_spread   : node forces F_i = -dW/dx_i of the Skalak membrane
//                      (Sec. II.B, Eqs. constitutivelaw, forcefromenergy)
//                      and their spreading to the lattice (Eq. forcespreading)
//   k_interp_advect  : interpolation of the new lattice velocity at the old
//                      node positions (Eq. velocityinterpolation) and Euler
//                      advection (Eq. positionupdate)
//
// Both kernels give one warp to one membrane node.  In k_force_spread the
// lanes first take the faces around the node (one face each; a face's
// contribution to this corner is recomputed by each of its three corner
// warps, which keeps the assembly a deterministic warp reduction with no
// atomics and no per-face scratch), then the lanes take the n^3 stencil cells
// and add the spread force with one vector atomic per cell.  In
// k_interp_advect the lanes take the stencil cells, each gathers the 19
// populations of its cell (L2-resident: the stencils of all nodes cover a thin
// shell of the lattice), and a warp reduction gives the node velocity.
//
// Face energy gradient.  With the current edge vectors u = x_b - x_a,
// v = x_c - x_a, their Gram entries g11 = u.u, g12 = u.v, g22 = v.v, the
// reference Gram entries G11, G12, G22 and the reference constants
// alpha = G22/det, beta = G12/det, gamma = G11/det, kappa = 1/det
// (det = G11 G22 - G12^2; prepared on the host), the invariants of Sec. II.B
// are, with the deviations d = g - G,
//     I1 = alpha d11 - 2 beta d12 + gamma d22,
//     I2 = I1 + kappa (d11 d22 - d12^2),
// (tr(G^-1 g) - 2 and det g / det G - 1 written so that nothing of order one
// cancels), and with w1 = dw/dI1 = k_s (I1 + 1)/6, w2 = dw/dI2 =
// (k_alpha I2 - k_s)/6 and kappa G22 = alpha, kappa G12 = beta, kappa G11 = gamma
//     dW/du = s_uu u + s_uv v,   dW/dv = s_uv u + s_vv v,
//     s_uu =  2 A0 [k_s/6 (I1 alpha - kappa d22) + k_alpha/6 I2 kappa g22],
//     s_uv = -2 A0 [k_s/6 (I1 beta  - kappa d12) + k_alpha/6 I2 kappa g12],
//     s_vv =  2 A0 [k_s/6 (I1 gamma - kappa d11) + k_alpha/6 I2 kappa g11];
// the corner forces are F_b = -dW/du, F_c = -dW/dv, F_a = dW/du + dW/dv.
// In the float builds the edges and the Gram entries are formed in
// double-float arithmetic from the hi/lo node coordinates, so the deviations
// d keep their relative precision even for strains of 1e-4.
#include "device_common.cuh"
#include "ib_common.cuh"
#include "internal.h"

namespace iblbm {

template <int N, typename T>
__global__ void __launch_bounds__(256)
    k_force_spread(int n_nodes, PosView<T> pos, const int *__restrict__ adj_off,
                   const int *__restrict__ adj, const int4 *__restrict__ tri,
                   const typename Vec4<T>::type *__restrict__ fconst,
                   const typename Vec4<T>::type *__restrict__ capmod,
                   typename Vec4<T>::type *__restrict__ nodeF,
                   typename Vec4<T>::type *__restrict__ force, uint8_t *__restrict__ flags,
                   RunDesc single, const RunDesc *__restrict__ runs,
                   const int *__restrict__ node_run, int *status) {
    using V4 = typename Vec4<T>::type;
    const int lane = threadIdx.x & 31;
    const int node = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (node >= n_nodes) return;
    const RunDesc R = runs ? runs[node_run[node]] : single;

    T fx = T(0), fy = T(0), fz = T(0);
    const int e0 = adj_off[node], e1 = adj_off[node + 1];
    for (int e = e0 + lane; e < e1; e += 32) {
        const int ent = adj[e];
        const int f = ent >> 2, corner = ent & 3;
        const int4 t = tri[f];
        const V4 c0 = fconst[3 * f];      // alpha, beta, gamma, kappa
        const V4 c1 = fconst[3 * f + 1];  // A0, G11, G12, G22 (hi parts in float builds)
        const V4 c2 = fconst[3 * f + 2];  // lo parts of G11, G12, G22 (float builds)
        T u[3], v[3], d[3];
        pos.edge_gram(t.x, t.y, t.z, c1, c2, u, v, d);
        const V4 m = capmod[t.w];  // k_s/6, k_alpha/6
        const T I1 = c0.x * d[0] - T(2) * c0.y * d[1] + c0.z * d[2];
        const T I2 = I1 + c0.w * (d[0] * d[2] - d[1] * d[1]);
        const T a2 = T(2) * c1.x;
        const T kI2 = m.y * I2 * c0.w;  // k_alpha/6 I2 kappa
        const T s_uu = a2 * (m.x * (I1 * c0.x - c0.w * d[2]) + kI2 * (c1.w + d[2]));
        const T s_uv = -a2 * (m.x * (I1 * c0.y - c0.w * d[1]) + kI2 * (c1.z + d[1]));
        const T s_vv = a2 * (m.x * (I1 * c0.z - c0.w * d[0]) + kI2 * (c1.y + d[0]));
        T ku, kv;
        if (corner == 0) {
            ku = s_uu + s_uv;
            kv = s_uv + s_vv;
        } else if (corner == 1) {
            ku = -s_uu;
            kv = -s_uv;
        } else {
            ku = -s_uv;
            kv = -s_vv;
        }
        fx += ku * u[0] + kv * v[0];
        fy += ku * u[1] + kv * v[1];
        fz += ku * u[2] + kv * v[2];
    }
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    fz = warp_sum(fz);
    if (lane == 0) nodeF[node] = V4{fx, fy, fz, T(0)};

    T p[kPosLen<T>];
    pos.approx(node, p);
    T pc[3];
    if constexpr (kPosLen<T> == 6) {
        pc[0] = p[0] + p[3]; pc[1] = p[1] + p[4]; pc[2] = p[2] + p[5];
    } else {
        pc[0] = p[0]; pc[1] = p[1]; pc[2] = p[2];
    }
    const int bx = stencil_first<N>(pc[0]), by = stencil_first<N>(pc[1]), bz = stencil_first<N>(pc[2]);
    constexpr int NC = N * N * N;
    for (int k = lane; k < NC; k += 32) {
        const int kx = k % N, ky = (k / N) % N, kz = k / (N * N);
        const int X = bx + kx, Y = by + ky, Z = bz + kz;
        if (Z < 0 || Z >= R.nz) {
            set_status(status, kStatusStencil);
            continue;
        }
        T d[3];
        pos.rel(p, X, Y, Z, d);
        const T w = delta_phi<N>(d[0]) * delta_phi<N>(d[1]) * delta_phi<N>(d[2]);
        if (w == T(0)) continue;
        const int xw = wrap_index(X, R.nx), yw = wrap_index(Y, R.ny);
        const long long cell = xw + (long long)R.nx * (yw + (long long)R.ny * Z);
        add_force(&force[R.cell_off + cell], w * fx, w * fy, w * fz);
        flags[R.tile_off + ((long long)Z * R.nty + yw / R.ty) * R.ntx + xw / R.tx] = 1;
    }
}

template <int N, typename S, typename T>
__global__ void __launch_bounds__(256)
    k_interp_advect(int n_nodes, PosView<T> pos, const S *__restrict__ pop,
                    const typename Vec4<T>::type *__restrict__ force,
                    typename Vec4<T>::type *__restrict__ nodeU, RunDesc single,
                    const RunDesc *__restrict__ runs, const int *__restrict__ node_run) {
    using V4 = typename Vec4<T>::type;
    const int lane = threadIdx.x & 31;
    const int node = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (node >= n_nodes) return;
    const RunDesc R = runs ? runs[node_run[node]] : single;
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const long long ncell = R.ncell;
    pop += 19 * R.cell_off;
    force += R.cell_off;
    T p[kPosLen<T>];
    pos.approx(node, p);
    T pc[3];
    if constexpr (kPosLen<T> == 6) {
        pc[0] = p[0] + p[3]; pc[1] = p[1] + p[4]; pc[2] = p[2] + p[5];
    } else {
        pc[0] = p[0]; pc[1] = p[1]; pc[2] = p[2];
    }
    const int bx = stencil_first<N>(pc[0]), by = stencil_first<N>(pc[1]), bz = stencil_first<N>(pc[2]);
    // Each lane owns up to ITER stencil cells; all their population loads are
    // issued before any is used.
    constexpr int NC = N * N * N;
    constexpr int ITER = (NC + 31) / 32;
    T w[ITER];
    long long cell[ITER];
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int k = lane + 32 * it;
        const int kx = k % N, ky = (k / N) % N, kz = k / (N * N);
        const int X = bx + kx, Y = by + ky, Z = bz + kz;
        w[it] = T(0);
        cell[it] = 0;
        if (k < NC && Z >= 0 && Z < nz) {  // a stencil beyond a wall is reported by the spreading
            T d[3];
            pos.rel(p, X, Y, Z, d);
            w[it] = delta_phi<N>(d[0]) * delta_phi<N>(d[1]) * delta_phi<N>(d[2]);
            cell[it] = wrap_index(X, nx) + (long long)nx * (wrap_index(Y, ny) + (long long)ny * Z);
        }
    }
    T g[ITER][19];
#pragma unroll
    for (int it = 0; it < ITER; ++it)
#pragma unroll
        for (int i = 0; i < 19; ++i)
            g[it][i] = (w[it] != T(0)) ? Store<S, T>::load(pop + i * ncell + cell[it]) : T(0);
    T ax = T(0), ay = T(0), az = T(0);
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        if (w[it] == T(0)) continue;
        T drho = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            drho += g[it][i];
            if (q_cx(i)) jx += q_cx(i) > 0 ? g[it][i] : -g[it][i];
            if (q_cy(i)) jy += q_cy(i) > 0 ? g[it][i] : -g[it][i];
            if (q_cz(i)) jz += q_cz(i) > 0 ? g[it][i] : -g[it][i];
        }
        const V4 f = force[cell[it]];
        const T inv_rho = T(1) / (T(1) + drho);
        ax += w[it] * ((jx + T(0.5) * f.x) * inv_rho);
        ay += w[it] * ((jy + T(0.5) * f.y) * inv_rho);
        az += w[it] * ((jz + T(0.5) * f.z) * inv_rho);
    }
    ax = warp_sum(ax);
    ay = warp_sum(ay);
    az = warp_sum(az);
    if (lane == 0) {
        nodeU[node] = V4{ax, ay, az, T(0)};
        pos.advance(node, ax, ay, az);
    }
}

// ---- node array conversions ---------------------------------------------------
template <typename T>
__global__ void k_nodes_to_f64(PosView<T> pos, const typename Vec4<T>::type *F,
                               const typename Vec4<T>::type *U, int which, int first, int count,
                               double *out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    int n = first + k;
    double r[3];
    if (which == 0) {
        T p[kPosLen<T>];
        pos.approx(n, p);
        if constexpr (kPosLen<T> == 6) {
            for (int a = 0; a < 3; ++a) r[a] = (double)p[a] + (double)p[3 + a];
        } else {
            for (int a = 0; a < 3; ++a) r[a] = (double)p[a];
        }
    } else {
        auto v = (which == 1) ? F[n] : U[n];
        r[0] = (double)v.x; r[1] = (double)v.y; r[2] = (double)v.z;
    }
    out[3 * k] = r[0];
    out[3 * k + 1] = r[1];
    out[3 * k + 2] = r[2];
}

__global__ void k_f64_to_nodes_d(dvec4 *x, int first, int count, const double *in) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    x[first + k] = dvec4{in[3 * k], in[3 * k + 1], in[3 * k + 2], 0.0};
}

__global__ void k_f64_to_nodes_f(float4 *hi, float4 *lo, int first, int count, const double *in) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    float h[3], l[3];
    for (int a = 0; a < 3; ++a) {
        double v = in[3 * k + a];
        h[a] = (float)v;
        l[a] = (float)(v - (double)h[a]);
    }
    hi[first + k] = make_float4(h[0], h[1], h[2], 0.0f);
    lo[first + k] = make_float4(l[0], l[1], l[2], 0.0f);
}

// ---- launchers ------------------------------------------------------------------
template <typename T>
static PosView<T> view(const MeshDev &m);
template <>
PosView<double> view<double>(const MeshDev &m) {
    return PosView<double>{(dvec4 *)m.x};
}
template <>
PosView<float> view<float>(const MeshDev &m) {
    return PosView<float>{(float4 *)m.x, (float4 *)m.x_lo};
}

// Two warps (nodes) per block: a few thousand node warps then spread evenly
// over the 152 SMs (whole 8-warp blocks left some SMs with half as many
// warps again as others, and those set the kernel's time).
constexpr int kNodesPerBlock = 2;

// The single lattice as a run descriptor (its force flags are the lattice's).
static RunDesc single_run(const Lattice &L) {
    RunDesc R{};
    R.nx = L.nx;
    R.ny = L.ny;
    R.nz = L.nz;
    R.tx = L.ftx;
    R.ty = L.fty;
    R.ntx = L.nfx;
    R.nty = L.nfy;
    R.ncell = L.ncell;
    return R;
}

template <int N, typename T>
static void force_spread_impl(const Lattice &L, const MeshDev &m, void *force, uint8_t *flags,
                              int *status, const RunDesc *runs, const int *node_run,
                              cudaStream_t s) {
    using V4 = typename Vec4<T>::type;
    unsigned nb = (unsigned)((m.n_nodes + kNodesPerBlock - 1) / kNodesPerBlock);
    k_force_spread<N, T><<<nb, 32 * kNodesPerBlock, 0, s>>>(
        m.n_nodes, view<T>(m), m.adj_off, m.adj, (const int4 *)m.tri, (const V4 *)m.fconst,
        (const V4 *)m.capmod, (V4 *)m.F, (V4 *)force, flags, single_run(L), runs, node_run,
        status);
}

template <int N, typename S, typename T>
static void interp_impl(const Lattice &L, const MeshDev &m, const void *pop, const void *force,
                        const RunDesc *runs, const int *node_run, cudaStream_t s) {
    using V4 = typename Vec4<T>::type;
    unsigned nb = (unsigned)((m.n_nodes + kNodesPerBlock - 1) / kNodesPerBlock);
    k_interp_advect<N, S, T><<<nb, 32 * kNodesPerBlock, 0, s>>>(
        m.n_nodes, view<T>(m), (const S *)pop, (const V4 *)force, (V4 *)m.u, single_run(L), runs,
        node_run);
}

void launch_force_spread(int prec, int delta, const Lattice &L, const MeshDev &m, void *force,
                         uint8_t *flags, int *status, const RunDesc *runs, const int *node_run,
                         cudaStream_t s) {
    if (m.n_nodes == 0) return;
    if (prec == kF64) {
        if (delta == 2) force_spread_impl<2, double>(L, m, force, flags, status, runs, node_run, s);
        else if (delta == 3) force_spread_impl<3, double>(L, m, force, flags, status, runs, node_run, s);
        else force_spread_impl<4, double>(L, m, force, flags, status, runs, node_run, s);
    } else {
        if (delta == 2) force_spread_impl<2, float>(L, m, force, flags, status, runs, node_run, s);
        else if (delta == 3) force_spread_impl<3, float>(L, m, force, flags, status, runs, node_run, s);
        else force_spread_impl<4, float>(L, m, force, flags, status, runs, node_run, s);
    }
}

void launch_interp_advect(int prec, int delta, const Lattice &L, const MeshDev &m, const void *pop,
                          const void *force, const RunDesc *runs, const int *node_run,
                          cudaStream_t s) {
    if (m.n_nodes == 0) return;
    if (prec == kF64) {
        if (delta == 2) interp_impl<2, double, double>(L, m, pop, force, runs, node_run, s);
        else if (delta == 3) interp_impl<3, double, double>(L, m, pop, force, runs, node_run, s);
        else interp_impl<4, double, double>(L, m, pop, force, runs, node_run, s);
    } else if (prec == kF32) {
        if (delta == 2) interp_impl<2, float, float>(L, m, pop, force, runs, node_run, s);
        else if (delta == 3) interp_impl<3, float, float>(L, m, pop, force, runs, node_run, s);
        else interp_impl<4, float, float>(L, m, pop, force, runs, node_run, s);
    } else {
        if (delta == 2) interp_impl<2, __half, float>(L, m, pop, force, runs, node_run, s);
        else if (delta == 3) interp_impl<3, __half, float>(L, m, pop, force, runs, node_run, s);
        else interp_impl<4, __half, float>(L, m, pop, force, runs, node_run, s);
    }
}

void launch_nodes_to_f64(int prec, const MeshDev &m, int which, int first, int count, double *out,
                         cudaStream_t s) {
    if (count <= 0) return;
    unsigned nb = (unsigned)((count + 255) / 256);
    if (prec == kF64)
        k_nodes_to_f64<double><<<nb, 256, 0, s>>>(view<double>(m), (const dvec4 *)m.F,
                                                  (const dvec4 *)m.u, which, first, count, out);
    else
        k_nodes_to_f64<float><<<nb, 256, 0, s>>>(view<float>(m), (const float4 *)m.F,
                                                 (const float4 *)m.u, which, first, count, out);
}

void launch_f64_to_nodes(int prec, const MeshDev &m, int first, int count, const double *in,
                         cudaStream_t s) {
    if (count <= 0) return;
    unsigned nb = (unsigned)((count + 255) / 256);
    if (prec == kF64)
        k_f64_to_nodes_d<<<nb, 256, 0, s>>>((dvec4 *)m.x, first, count, in);
    else
        k_f64_to_nodes_f<<<nb, 256, 0, s>>>((float4 *)m.x, (float4 *)m.x_lo, first, count, in);
}

}  // namespace iblbm
