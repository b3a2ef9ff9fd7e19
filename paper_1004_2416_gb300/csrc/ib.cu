// ib.cu -- immersed-boundary coupling and finite-element membrane forces.
//
//   k_force_spread   : node forces F_i = -dW/dx_i of the Skalak membrane
//                      (Sec. II.B, Eqs. constitutivelaw, forcefromenergy)
//                      and their spreading to the lattice (Eq. forcespreading)
//   k_interp_advect  : interpolation of the new lattice velocity at the old
//                      node positions (Eq. velocityinterpolation) and Euler
//                      advection (Eq. positionupdate)
//
// k_force_spread gives one warp to one or four membrane nodes.  A group of
// lanes first takes the faces around its node (one face each; a face's
// contribution to this corner is recomputed by each of its three corner
// groups, which keeps the assembly a deterministic group reduction with no
// atomics and no per-face scratch), then the group's lanes take pieces of the
// node's stencil (whole rows of n cells along x with four nodes per warp;
// one or two cells with one) and add the spread force with one vector atomic
// per cell.  k_interp_advect gives a group of lanes to a node in the same
// way: the lanes take stencil pieces, read the velocity of each cell (formed
// once per cell of the flagged tiles by k_flag_velocity, L2-resident, or
// formed from the populations on the spot) and a group reduction gives the
// node velocity.  The delta function is separable: its x factors are formed
// once per lane when the pieces are whole rows, its y and z factors once per
// piece.
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
#include <algorithm>
#include <type_traits>

#include "device_common.cuh"
#include "ib_common.cuh"
#include "internal.h"

namespace iblbm {

// The 3N separable delta factors of a node's N^3 stencil, formed once by the
// G lanes of the node's group and exchanged by shuffles: factor k is
// delta_phi<N> along axis k / N at stencil offset k % N, from the same
// difference (cell coordinate - node position) as a factor formed cell by
// cell, so the same value; lane gl forms factors gl and, where 3N > G,
// gl + G.  share() is called by every lane of the warp together.
template <int N, typename T, int G>
struct GroupFactors {
    static constexpr int NF = 3 * N;
    static_assert(NF <= 2 * G, "two factors per lane at most");
    T fa, fb;
    template <typename P>
    __device__ __forceinline__ GroupFactors(const P &pos, const T *p, int bx, int by, int bz, int gl) {
        auto factor = [&](int k) {
            const int ax = k / N, j = k % N;
            T d[3];
            pos.rel(p, bx + j, by + j, bz + j, d);
            return delta_phi<N>(ax == 0 ? d[0] : (ax == 1 ? d[1] : d[2]));
        };
        fa = factor(gl < NF ? gl : 0);
        fb = T(0);
        if constexpr (NF > G) {
            if (gl + G < NF) fb = factor(gl + G);
        }
    }
    __device__ __forceinline__ T share(int k) const {
        T v = __shfl_sync(0xffffffffu, fa, k < G ? k : 0, G);
        if constexpr (NF > G) {
            const T b = __shfl_sync(0xffffffffu, fb, k >= G ? k - G : 0, G);
            if (k >= G) v = b;
        }
        return v;
    }
};

// One warp takes NPW nodes (1 or 4).  Face phase: a group of 32 / NPW lanes
// per node, one adjacent face per lane (a loop for higher valences), a
// fixed-order butterfly reduction within the group that leaves the node force
// in every lane of the group.  Stencil phase: the group's lanes take the
// node's n^2 stencil rows.  Four nodes per warp waste fewer lanes on the faces
// (a node has five or six) when there are enough nodes to fill the GPU; one
// node per warp keeps more warps in flight otherwise.
// FIX: add into the 64-bit fixed-point accumulator `fix` (three per cell)
// instead of the float force density (deterministic spreading).
template <int N, typename T, int NPW, bool SLAB = false, bool FIX = false>
__global__ void __launch_bounds__(256)
    k_force_spread(int n_nodes, PosView<T> pos, const int *__restrict__ adj_off,
                   const int4 *__restrict__ adj4, const int *__restrict__ node_cap,
                   const typename Vec4<T>::type *__restrict__ fconst,
                   const typename Vec4<T>::type *__restrict__ capmod,
                   typename Vec4<T>::type *__restrict__ nodeF,
                   typename Vec4<T>::type *__restrict__ force, uint8_t *__restrict__ flags,
                   RunDesc single, const RunDesc *__restrict__ runs,
                   const int *__restrict__ node_run, int *status, unsigned long long *__restrict__ fix) {
    using V4 = typename Vec4<T>::type;
    prior_grid_wait();  // the node positions come from the previous interpolation
    allow_dependents();
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    constexpr int kFsNodes = NPW, kFsGroup = 32 / NPW;
    const long long node0 = warp * kFsNodes;
    if (node0 >= n_nodes) return;
    const int grp = lane / kFsGroup, gl = lane % kFsGroup;
    const int node = (int)(node0 + grp);
    const bool valid = node < n_nodes;

    T fx = T(0), fy = T(0), fz = T(0);
    const int e0 = valid ? adj_off[node] : 0, e1 = valid ? adj_off[node + 1] : 0;
    const V4 m = capmod[valid ? node_cap[node] : 0];  // k_s/6, k_alpha/6 of the node's capsule
    for (int e = e0 + gl; e < e1; e += kFsGroup) {
        // (face * 4 + corner, a, b, c): the positions can be loaded next
        const int4 q = adj4[e];
        if (!(IBLBM_OK(q.y, 1, n_nodes) && IBLBM_OK(q.z, 1, n_nodes) && IBLBM_OK(q.w, 1, n_nodes))) continue;
        const int f = q.x >> 2, corner = q.x & 3;
        const V4 c0 = fconst[3 * f];      // alpha, beta, gamma, kappa
        const V4 c1 = fconst[3 * f + 1];  // A0, G11, G12, G22 (hi parts in float builds)
        const V4 c2 = fconst[3 * f + 2];  // lo parts of G11, G12, G22 (float builds)
        T u[3], v[3], d[3];
        pos.edge_gram(q.y, q.z, q.w, c1, c2, u, v, d);
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
#pragma unroll
    for (int o = kFsGroup / 2; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    if (valid && gl == 0) nodeF[node] = V4{fx, fy, fz, T(0)};

    // Stencil phase: lane gl of the node's group takes the stencil pieces
    // gl, gl + 32 / NPW, ... of its node (CX cells along x of one row
    // (ky, kz)); a piece's wrapped row base is formed once, its delta
    // weights come from the node's 3N separable factors, formed once across
    // the group and shared by shuffles (GroupFactors), so every lane stays
    // until they are formed; a group past the last node forms those of the
    // last node and leaves before writing.  Force flag tiles are powers of two.
    // pieces: whole rows with four nodes per warp; with one node per warp
    // pieces that spread the n^3 cells over most of the 32 lanes
    constexpr int CX = NPW == 1 ? (N == 4 ? 2 : 1) : N, SPR = N / CX, NS = N * N * SPR;
    constexpr int G = kFsGroup, RPL = (NS + G - 1) / G;  // pieces per lane, at most
    const int nd = valid ? node : n_nodes - 1;
    T p[kPosLen<T>];
    pos.approx(nd, p);
    T pc[3];
    if constexpr (kPosLen<T> == 6) {
        pc[0] = p[0] + p[3]; pc[1] = p[1] + p[4]; pc[2] = p[2] + p[5];
    } else {
        pc[0] = p[0]; pc[1] = p[1]; pc[2] = p[2];
    }
    const int bx = stencil_first<N>(pc[0]), by = stencil_first<N>(pc[1]), bz = stencil_first<N>(pc[2]);
    const RunDesc R = runs ? runs[node_run[nd]] : single;
    const int sx = __ffs(R.tx) - 1, sy = __ffs(R.ty) - 1;
    const int xw0 = wrap_index(bx, SLAB ? R.gnx : R.nx), yw0 = wrap_index(by, R.ny);
    // the x, y and z factors of the lane's pieces
    T WX[RPL][CX], WY[RPL], WZ[RPL];
    {
        const GroupFactors<N, T, G> gf(pos, p, bx, by, bz, gl);
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int sl = (gl + G * j) % NS;  // pieces past the last are not used
            const int r = sl / SPR, kx0 = (sl % SPR) * CX;
            WY[j] = gf.share(N + r % N);
            WZ[j] = gf.share(2 * N + r / N);
#pragma unroll
            for (int c = 0; c < CX; ++c) WX[j][c] = gf.share(kx0 + c);
        }
    }
    if (!valid) return;
    V4 *fr = force + R.cell_off;
    uint8_t *flr = flags + R.tile_off;
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int sl = gl + G * j;
        if (sl >= NS) break;
        const int r = sl / SPR, kx0 = (sl % SPR) * CX;
        const int Z = bz + r / N;
        if (Z < 0 || Z >= R.nz) {
            set_status(status, kStatusStencil);
            continue;
        }
        const T wy = WY[j], wz = WZ[j];
        const int yw = wrap_next<N>(yw0, r % N, R.ny);
        const long long rc = (long long)R.nx * (yw + (long long)R.ny * Z);
        const long long rt = ((long long)Z * R.nty + (yw >> sy)) * R.ntx;
        int last = -1;
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            const T w = WX[j][c] * wy * wz;
            if (w == T(0)) continue;
            const int xa = xw0 + kx0 + c;
            int xw;
            if constexpr (SLAB) {  // the slab's own columns only
                xw = (xa < R.gnx ? xa : xa - R.gnx) - R.x0;
                if (xw < 0 || xw >= R.nx) continue;
            } else {
                xw = xa < R.nx ? xa : wrap_index(xa, R.nx);
            }
            if (IBLBM_OK(rc + xw, 1, R.ncell)) {
                if constexpr (FIX)
                    add_force_fix(fix + 3 * (R.cell_off + rc + xw), w * fx, w * fy, w * fz, status);
                else
                    add_force(&fr[rc + xw], w * fx, w * fy, w * fz);
            }
            const int xt = xw >> sx;
            if (xt != last) {
                if (IBLBM_OK(rt + xt, 1, (long long)R.ntx * R.nty * R.nz)) flr[rt + xt] = 1;
                last = xt;
            }
        }
    }
}

// u = (sum_i c_i f_i + g/2) / rho of one cell from its 19 stored deviations g
// (Eq. velocityinterpolation's u(X, t+1) with the half-force correction).
template <typename T>
__device__ __forceinline__ typename Vec4<T>::type velocity_from(const T g[19], const typename Vec4<T>::type &f) {
    T drho = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        drho += g[i];
        if (q_cx(i)) jx += q_cx(i) > 0 ? g[i] : -g[i];
        if (q_cy(i)) jy += q_cy(i) > 0 ? g[i] : -g[i];
        if (q_cz(i)) jz += q_cz(i) > 0 ? g[i] : -g[i];
    }
    const T inv_rho = T(1) / (T(1) + drho);
    return typename Vec4<T>::type{(jx + T(0.5) * f.x) * inv_rho, (jy + T(0.5) * f.y) * inv_rho,
                                  (jz + T(0.5) * f.z) * inv_rho, T(0)};
}

// Velocity u = (sum_i c_i f_i + g/2) / rho of every cell in a force-flagged
// tile (Eq. velocityinterpolation's u(X, t+1)), once per cell: every stencil
// cell of the interpolation lies in a tile the spreading flagged, and each cell
// serves a dozen or so nodes.  One warp per tile (its lanes walk the tile's
// cells); for a batch the tiles come from the work list of (run, tile) pairs.
template <typename S, typename T>
__global__ void __launch_bounds__(256)
    k_flag_velocity(const S *__restrict__ pop, const typename Vec4<T>::type *__restrict__ force,
                    const uint8_t *__restrict__ flags, typename Vec4<T>::type *__restrict__ uvel,
                    RunDesc single, long long n_tiles, const RunDesc *__restrict__ runs,
                    const int2 *__restrict__ items) {
    using V4 = typename Vec4<T>::type;
    prior_grid_wait();
    allow_dependents();
    const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (w >= n_tiles) return;
    int tile;
    RunDesc R;
    if (runs) {
        const int2 it = items[w];
        R = runs[it.x];
        tile = it.y;
    } else {
        R = single;
        tile = (int)w;
    }
    if (!flags[R.tile_off + tile]) return;
    const int lane = threadIdx.x & 31;
    const int per_z = R.ntx * R.nty;
    const int z = tile / per_z, rem = tile - z * per_z;
    const int tyi = rem / R.ntx, txi = rem - tyi * R.ntx;
    pop += 19 * R.cell_off;
    force += R.cell_off;
    uvel += R.cell_off;
    for (int c = lane; c < R.tx * R.ty; c += 32) {
        const int x = txi * R.tx + c % R.tx, y = tyi * R.ty + c / R.tx;
        if (x >= R.nx || y >= R.ny) continue;
        const long long cell = x + (long long)R.nx * (y + (long long)R.ny * z);
        T g[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) g[i] = Store<S, T>::load(pop + i * R.ncell + cell);
        uvel[cell] = velocity_from<T>(g, force[cell]);
    }
}

// Four stored deviations of consecutive cells in float (16-byte, or 8-byte
// binary16, vector load); the values equal Store<S, float>::load's.
template <typename S>
__device__ __forceinline__ void load_quad(const S *p, float v[4]);
template <>
__device__ __forceinline__ void load_quad<float>(const float *p, float v[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void load_quad<__half>(const __half *p, float v[4]) {
    const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
    v[0] = a.x * kHalfInvScale; v[1] = a.y * kHalfInvScale;
    v[2] = b.x * kHalfInvScale; v[3] = b.y * kHalfInvScale;
}

// k_flag_velocity for a lattice flagged per ftx-cell segment of an x-row
// (ftx a multiple of 4 dividing nx, so flag index = cell / ftx): one thread
// takes four consecutive cells of a segment with vector loads (the same
// arithmetic per cell).  A block covers 256 consecutive quads and first
// packs its flagged ones onto its first threads (a ballot per warp and the
// warps' counts in shared memory), so that a flagged quad does not hold a
// warp of mostly idle lanes: in a dense suspension about one quad in eight
// is flagged, in short runs along x.
template <typename S>
__global__ void __launch_bounds__(256, sizeof(S) == 2 ? 4 : 3)
    k_flag_velocity_x4(const S *__restrict__ pop, const float4 *__restrict__ force,
                       const uint8_t *__restrict__ flags, float4 *__restrict__ uvel, long long ncell,
                       int ftx) {
    __shared__ int warp_count[8];
    __shared__ unsigned char packed[256];  // the block's flagged quads, in order
    prior_grid_wait();
    allow_dependents();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long q0 = 256 * (long long)blockIdx.x;  // first quad of the block
    const long long own = 4 * (q0 + tid);
    const bool flagged = own < ncell && flags[own / ftx];
    const unsigned ballot = __ballot_sync(0xffffffffu, flagged);
    if (lane == 0) warp_count[warp] = __popc(ballot);
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        before += w < warp ? warp_count[w] : 0;
        total += warp_count[w];
    }
    if (flagged) packed[before + __popc(ballot & ((1u << lane) - 1u))] = (unsigned char)tid;
    __syncthreads();
    if (tid >= total) return;
    const long long cell0 = 4 * (q0 + packed[tid]);
    // velocity_from's sums, in its order, as the loads arrive
    float drho[4] = {0.f, 0.f, 0.f, 0.f}, jx[4] = {0.f, 0.f, 0.f, 0.f};
    float jy[4] = {0.f, 0.f, 0.f, 0.f}, jz[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        float v[4];
        load_quad<S>(pop + i * ncell + cell0, v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            drho[k] += v[k];
            if (q_cx(i)) jx[k] += q_cx(i) > 0 ? v[k] : -v[k];
            if (q_cy(i)) jy[k] += q_cy(i) > 0 ? v[k] : -v[k];
            if (q_cz(i)) jz[k] += q_cz(i) > 0 ? v[k] : -v[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 f = force[cell0 + k];
        const float inv_rho = 1.f / (1.f + drho[k]);
        uvel[cell0 + k] = make_float4((jx[k] + 0.5f * f.x) * inv_rho, (jy[k] + 0.5f * f.y) * inv_rho,
                                      (jz[k] + 0.5f * f.z) * inv_rho, 0.f);
    }
}

// Interpolation and advection, NPW = 1 or 4 nodes per warp (four for dense
// suspensions), a group of 32 / NPW lanes per node.  Lane gl of a group takes
// the stencil pieces gl, gl + 32 / NPW, ... of its node (piece = CX
// consecutive cells along x of one stencil row (ky, kz); y and z weights once per piece, x weights once
// per lane when the pieces are whole rows) and the group sums in a fixed
// order.  PRE: read the cell velocities of k_flag_velocity; otherwise the lane
// gathers the 19 populations and the force of each cell and forms u itself
// with the same arithmetic, so for the same NPW both forms give the same
// bits (the launcher takes NPW = 4 only with PRE).  The loads
// depend only on the cell index and are issued before the weights are used
// (cells of zero weight are read and not used).  Groups past the last node
// repeat its work and write nothing.
template <int N, typename S, typename T, bool PRE, int NPW, bool SLAB = false>
__global__ void __launch_bounds__(256)
    k_interp_advect(int n_nodes, PosView<T> pos, const typename Vec4<T>::type *__restrict__ uvel,
                    const S *__restrict__ pop, const typename Vec4<T>::type *__restrict__ force,
                    typename Vec4<T>::type *__restrict__ nodeU, RunDesc single,
                    const RunDesc *__restrict__ runs, const int *__restrict__ node_run, PosView<T> snap,
                    int ab2) {
    using V4 = typename Vec4<T>::type;
    constexpr int G = 32 / NPW;
    // cells per piece (whole rows with four nodes per warp; single cells with
    // one, so that one load instruction of the warp covers whole x-rows of the
    // stencil), pieces per row
    constexpr int CX = NPW == 1 ? 1 : N, SPR = N / CX;
    constexpr int NS = N * N * SPR;                              // pieces per node
    constexpr int RPL = (NS + G - 1) / G;                        // pieces per lane, at most
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (warp * NPW >= n_nodes) return;  // the whole warp
    const long long gnode = warp * NPW + lane / G;
    const int gl = lane % G;
    const bool valid = gnode < n_nodes;
    const int node = valid ? (int)gnode : n_nodes - 1;
    const RunDesc R = runs ? runs[node_run[node]] : single;
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    T p[kPosLen<T>];
    pos.approx(node, p);
    T pc[3];
    if constexpr (kPosLen<T> == 6) {
        pc[0] = p[0] + p[3]; pc[1] = p[1] + p[4]; pc[2] = p[2] + p[5];
    } else {
        pc[0] = p[0]; pc[1] = p[1]; pc[2] = p[2];
    }
    const int bx = stencil_first<N>(pc[0]), by = stencil_first<N>(pc[1]), bz = stencil_first<N>(pc[2]);
    const int xw0 = wrap_index(bx, SLAB ? R.gnx : nx), yw0 = wrap_index(by, ny);
    // this lane's pieces; a stencil beyond a wall is reported by the spreading
    bool in[RPL];
    long long rc[RPL];
    int Z[RPL], KX[RPL], XW[RPL][CX];
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int sl = gl + G * j, r = sl / SPR;
        KX[j] = (sl % SPR) * CX;
        Z[j] = bz + r / N;
        in[j] = sl < NS && Z[j] >= 0 && Z[j] < nz;
        rc[j] = in[j] ? (long long)nx * (wrap_next<N>(yw0, r % N, ny) + (long long)ny * Z[j]) : 0;
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            const int xa = xw0 + KX[j] + c;
            if constexpr (SLAB) {  // the slab's own columns; -1 elsewhere
                const int xl = (xa < R.gnx ? xa : xa - R.gnx) - R.x0;
                XW[j][c] = (xl >= 0 && xl < nx) ? xl : -1;
            } else {
                XW[j][c] = xa < nx ? xa : wrap_index(xa, nx);
            }
        }
    }
    // the x, y and z delta factors of the lane's pieces, from the node's 3N
    // factors formed once across the group and shared (every lane of the
    // warp takes part: a group past the last node works on the last node)
    T WX[RPL][CX], WY[RPL], WZ[RPL];
    {
        const GroupFactors<N, T, G> gf(pos, p, bx, by, bz, gl);
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int sl = (gl + G * j) % NS;  // pieces past the last are not used
            const int r = sl / SPR, kx0 = (sl % SPR) * CX;
            WY[j] = gf.share(N + r % N);
            WZ[j] = gf.share(2 * N + r / N);
#pragma unroll
            for (int c = 0; c < CX; ++c) WX[j][c] = gf.share(kx0 + c);
        }
    }
    // positions, stencil indices and x factors need nothing of the collide
    // or velocity kernel before this one; the velocities do
    prior_grid_wait();
    allow_dependents();
    T ax = T(0), ay = T(0), az = T(0);
    if constexpr (PRE) {
        const V4 *ur = uvel + R.cell_off;
        V4 u[RPL][CX];
#pragma unroll
        for (int j = 0; j < RPL; ++j)
#pragma unroll
            for (int c = 0; c < CX; ++c)
                u[j][c] = in[j] && IBLBM_OK(rc[j] + XW[j][c], 1, R.ncell) ? ur[rc[j] + XW[j][c]] : V4{};
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            if (!in[j]) continue;
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                const T w = WX[j][c] * WY[j] * WZ[j];
                if (w == T(0)) continue;
                ax += w * u[j][c].x;
                ay += w * u[j][c].y;
                az += w * u[j][c].z;
            }
        }
    } else {
        const S *pr = pop + 19 * R.cell_off;
        const V4 *fr = force + R.cell_off;
        constexpr bool ALL = RPL * CX <= 4;  // every load of the lane in flight at once
        T g[ALL ? RPL : 1][CX][19];
        V4 f[ALL ? RPL : 1][CX];
        auto load = [&](int j, int slot) {
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                const bool own = in[j] && (!SLAB || XW[j][c] >= 0) && IBLBM_OK(rc[j] + XW[j][c], 1, R.ncell);
#pragma unroll
                for (int i = 0; i < 19; ++i)
                    g[slot][c][i] = own ? Store<S, T>::load(pr + i * R.ncell + rc[j] + XW[j][c]) : T(0);
                f[slot][c] = own ? fr[rc[j] + XW[j][c]] : V4{};
            }
        };
        if constexpr (ALL) {
#pragma unroll
            for (int j = 0; j < RPL; ++j) load(j, j);
        }
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            if (!in[j]) continue;
            const int slot = ALL ? j : 0;
            if constexpr (!ALL) load(j, 0);
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                if (SLAB && XW[j][c] < 0) continue;
                const T w = WX[j][c] * WY[j] * WZ[j];
                if (w == T(0)) continue;
                const V4 u = velocity_from<T>(g[slot][c], f[slot][c]);
                ax += w * u.x;
                ay += w * u.y;
                az += w * u.z;
            }
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    if constexpr (SLAB) {  // the slab's partial sum; the nodes move once all slabs are summed
        if (valid && gl == 0) nodeU[node] = V4{ax, ay, az, T(0)};
        return;
    }
    if (valid && gl == 0) {
        if (ab2) {  // Sec. II.C: x += 3/2 u_i(t+1) - 1/2 u_i(t)
            const V4 uo = nodeU[node];
            pos.advance(node, T(1.5) * ax - T(0.5) * uo.x, T(1.5) * ay - T(0.5) * uo.y,
                        T(1.5) * az - T(0.5) * uo.z, snap);
        } else {  // Eq. (positionupdate)
            pos.advance(node, ax, ay, az, snap);
        }
        nodeU[node] = V4{ax, ay, az, T(0)};
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
                              cudaStream_t s, bool ov, unsigned long long *fix) {
    using V4 = typename Vec4<T>::type;
    // four nodes per warp once one-node warps would exceed 32 per SM
    const bool four = m.n_nodes >= 152 * 32;
    const long long warps = four ? (m.n_nodes + 3) / 4 : m.n_nodes;
    const int wpb = warps >= 152 * 16 ? 4 : 2;
    const unsigned nb = (unsigned)((warps + wpb - 1) / wpb);
    auto kern = fix ? (four ? k_force_spread<N, T, 4, false, true> : k_force_spread<N, T, 1, false, true>)
                    : (four ? k_force_spread<N, T, 4> : k_force_spread<N, T, 1>);
    launch_maybe_overlapped(kern, dim3(nb), dim3(32 * wpb), s, ov,
        m.n_nodes, view<T>(m), m.adj_off, (const int4 *)m.adj4, m.node_cap, (const V4 *)m.fconst,
        (const V4 *)m.capmod, (V4 *)m.F, (V4 *)force, flags, single_run(L), runs, node_run,
        status, fix);
}

// The fixed-point sums of the cells of the flagged tiles to the force
// density (one thread per cell), zeroing the accumulators for the next step.
template <typename T>
__global__ void __launch_bounds__(256)
    k_fix_to_force(RunDesc R, unsigned long long *__restrict__ fix, typename Vec4<T>::type *__restrict__ force,
                   const uint8_t *__restrict__ flags) {
    using V4 = typename Vec4<T>::type;
    prior_grid_wait();  // the sums come from the spreading
    allow_dependents();
    const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= R.ncell) return;
    const int x = (int)(cell % R.nx);
    const long long rest = cell / R.nx;
    const int y = (int)(rest % R.ny), z = (int)(rest / R.ny);
    if (!flags[((long long)z * R.nty + y / R.ty) * R.ntx + x / R.tx]) return;
    unsigned long long *q = fix + 3 * cell;
    const T inv = T(1) / T(1ll << kFixBits<T>);
    force[cell] = V4{(T)(long long)q[0] * inv, (T)(long long)q[1] * inv, (T)(long long)q[2] * inv, T(0)};
    q[0] = 0ull;
    q[1] = 0ull;
    q[2] = 0ull;
}

template <int N, typename S, typename T>
static void interp_impl(const Lattice &L, const MeshDev &m, const void *uvel, const void *pop,
                        const void *force, const RunDesc *runs, const int *node_run, cudaStream_t s,
                        void *snap_x, void *snap_lo, int ab2, bool ov) {
    using V4 = typename Vec4<T>::type;
    MeshDev sm{};
    sm.x = snap_x;
    sm.x_lo = snap_lo;
    const PosView<T> snap = view<T>(sm);
    // four nodes per warp when reading the cell velocities and one-node warps
    // would exceed 32 per SM; gathering the populations keeps one node per
    // warp (all 19 loads of its cells in flight at once)
    const bool four = uvel && m.n_nodes >= 152 * 32;
    const long long warps = four ? (m.n_nodes + 3) / 4 : m.n_nodes;
    const int wpb = four && warps >= 152 * 16 ? 4 : kNodesPerBlock;
    const unsigned nb = (unsigned)((warps + wpb - 1) / wpb);
    auto kern = uvel ? (four ? k_interp_advect<N, S, T, true, 4> : k_interp_advect<N, S, T, true, 1>)
                     : k_interp_advect<N, S, T, false, 1>;
    launch_maybe_overlapped(kern, dim3(nb), dim3(32 * wpb), s, ov, m.n_nodes, view<T>(m), (const V4 *)uvel,
                            (const S *)pop, (const V4 *)force, (V4 *)m.u, single_run(L), runs, node_run, snap,
                            ab2);
}

template <typename S, typename T>
static void flag_velocity_impl(const Lattice &L, const void *pop, const void *force, const uint8_t *flags,
                               void *uvel, const RunDesc *runs, const int2 *items, long long n_items,
                               cudaStream_t s, bool ov) {
    using V4 = typename Vec4<T>::type;
    if constexpr (!std::is_same<S, double>::value) {
        if (!runs && L.lanes_row && L.fty == 1 && L.ftx % 4 == 0 && L.nx % L.ftx == 0) {
            const long long quads = L.ncell / 4;
            if (quads <= 0) return;
            launch_maybe_overlapped(k_flag_velocity_x4<S>, dim3((unsigned)((quads + 255) / 256)), dim3(256), s, ov,
                                    (const S *)pop, (const float4 *)force, flags, (float4 *)uvel, L.ncell,
                                    L.ftx);
            return;
        }
    }
    const long long n = runs ? n_items : L.ntiles;
    if (n <= 0) return;
    launch_maybe_overlapped(k_flag_velocity<S, T>, dim3((unsigned)((n + 7) / 8)), dim3(256), s, ov,
                            (const S *)pop, (const V4 *)force, flags, (V4 *)uvel, single_run(L), n, runs, items);
}

void launch_force_spread(int prec, int delta, const Lattice &L, const MeshDev &m, void *force,
                         uint8_t *flags, int *status, const RunDesc *runs, const int *node_run,
                         cudaStream_t s, bool overlap, unsigned long long *fix) {
    if (m.n_nodes == 0) return;
    if (prec == kF64) {
        if (delta == 2) force_spread_impl<2, double>(L, m, force, flags, status, runs, node_run, s, overlap, fix);
        else if (delta == 3) force_spread_impl<3, double>(L, m, force, flags, status, runs, node_run, s, overlap, fix);
        else force_spread_impl<4, double>(L, m, force, flags, status, runs, node_run, s, overlap, fix);
    } else {
        if (delta == 2) force_spread_impl<2, float>(L, m, force, flags, status, runs, node_run, s, overlap, fix);
        else if (delta == 3) force_spread_impl<3, float>(L, m, force, flags, status, runs, node_run, s, overlap, fix);
        else force_spread_impl<4, float>(L, m, force, flags, status, runs, node_run, s, overlap, fix);
    }
}

void launch_fix_to_force(int prec, const Lattice &L, unsigned long long *fix, void *force, const uint8_t *flags,
                         cudaStream_t s, bool overlap) {
    const unsigned nb = (unsigned)((L.ncell + 255) / 256);
    if (prec == kF64)
        launch_maybe_overlapped(k_fix_to_force<double>, dim3(nb), dim3(256), s, overlap, single_run(L), fix,
                                (dvec4 *)force, flags);
    else
        launch_maybe_overlapped(k_fix_to_force<float>, dim3(nb), dim3(256), s, overlap, single_run(L), fix,
                                (float4 *)force, flags);
}

void launch_flag_velocity(int prec, const Lattice &L, const void *pop, const void *force, const uint8_t *flags,
                          void *uvel, const RunDesc *runs, const int2 *items, long long n_items,
                          cudaStream_t s, bool overlap) {
    if (prec == kF64) flag_velocity_impl<double, double>(L, pop, force, flags, uvel, runs, items, n_items, s, overlap);
    else if (prec == kF32) flag_velocity_impl<float, float>(L, pop, force, flags, uvel, runs, items, n_items, s, overlap);
    else flag_velocity_impl<__half, float>(L, pop, force, flags, uvel, runs, items, n_items, s, overlap);
}

void launch_interp_advect(int prec, int delta, const Lattice &L, const MeshDev &m, const void *uvel,
                          const void *pop, const void *force, const RunDesc *runs, const int *node_run,
                          cudaStream_t s, void *snap_x, void *snap_lo, int ab2, bool overlap) {
    if (m.n_nodes == 0) return;
    if (prec == kF64) {
        if (delta == 2) interp_impl<2, double, double>(L, m, uvel, pop, force, runs, node_run, s, snap_x, snap_lo, ab2, overlap);
        else if (delta == 3) interp_impl<3, double, double>(L, m, uvel, pop, force, runs, node_run, s, snap_x, snap_lo, ab2, overlap);
        else interp_impl<4, double, double>(L, m, uvel, pop, force, runs, node_run, s, snap_x, snap_lo, ab2, overlap);
    } else if (prec == kF32) {
        if (delta == 2) interp_impl<2, float, float>(L, m, uvel, pop, force, runs, node_run, s, snap_x, snap_lo, ab2, overlap);
        else if (delta == 3) interp_impl<3, float, float>(L, m, uvel, pop, force, runs, node_run, s, snap_x, snap_lo, ab2, overlap);
        else interp_impl<4, float, float>(L, m, uvel, pop, force, runs, node_run, s, snap_x, snap_lo, ab2, overlap);
    } else {
        if (delta == 2) interp_impl<2, __half, float>(L, m, uvel, pop, force, runs, node_run, s, snap_x, snap_lo, ab2, overlap);
        else if (delta == 3) interp_impl<3, __half, float>(L, m, uvel, pop, force, runs, node_run, s, snap_x, snap_lo, ab2, overlap);
        else interp_impl<4, __half, float>(L, m, uvel, pop, force, runs, node_run, s, snap_x, snap_lo, ab2, overlap);
    }
}

// ---- x-slabs ---------------------------------------------------------------------
static RunDesc slab_run(const Lattice &L) {
    RunDesc R = single_run(L);
    R.x0 = L.x0;
    R.gnx = L.gnx;
    return R;
}

template <int N, typename T>
static void force_spread_slab_impl(const Lattice &L, const MeshDev &m, void *force, uint8_t *flags, int *status,
                                   cudaStream_t s) {
    using V4 = typename Vec4<T>::type;
    const unsigned nb = (unsigned)((m.n_nodes + kNodesPerBlock - 1) / kNodesPerBlock);
    k_force_spread<N, T, 1, true><<<nb, 32 * kNodesPerBlock, 0, s>>>(
        m.n_nodes, view<T>(m), m.adj_off, (const int4 *)m.adj4, m.node_cap, (const V4 *)m.fconst,
        (const V4 *)m.capmod, (V4 *)m.F, (V4 *)force, flags, slab_run(L), nullptr, nullptr, status, nullptr);
}

template <int N, typename S, typename T>
static void interp_partial_slab_impl(const Lattice &L, const MeshDev &m, const void *pop, const void *force,
                                     void *part, cudaStream_t s) {
    using V4 = typename Vec4<T>::type;
    const unsigned nb = (unsigned)((m.n_nodes + kNodesPerBlock - 1) / kNodesPerBlock);
    MeshDev none{};
    k_interp_advect<N, S, T, false, 1, true><<<nb, 32 * kNodesPerBlock, 0, s>>>(
        m.n_nodes, view<T>(m), nullptr, (const S *)pop, (const V4 *)force, (V4 *)part, slab_run(L), nullptr,
        nullptr, view<T>(none), 0);
}

// u = sum of the slabs' partials in slab order; x += u (Eq. positionupdate).
template <typename T>
__global__ void k_slab_advect(int n_nodes, PosView<T> pos, typename Vec4<T>::type *__restrict__ nodeU,
                              const typename Vec4<T>::type *const *__restrict__ parts, int n_parts) {
    using V4 = typename Vec4<T>::type;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_nodes) return;
    T ux = T(0), uy = T(0), uz = T(0);
    for (int p = 0; p < n_parts; ++p) {
        const V4 q = parts[p][i];
        ux += q.x;
        uy += q.y;
        uz += q.z;
    }
    PosView<T> none{};
    pos.advance(i, ux, uy, uz, none);
    nodeU[i] = V4{ux, uy, uz, T(0)};
}

void launch_force_spread_slab(int prec, int delta, const Lattice &L, const MeshDev &m, void *force,
                              uint8_t *flags, int *status, cudaStream_t s) {
    if (m.n_nodes == 0) return;
    if (prec == kF64) {
        if (delta == 2) force_spread_slab_impl<2, double>(L, m, force, flags, status, s);
        else if (delta == 3) force_spread_slab_impl<3, double>(L, m, force, flags, status, s);
        else force_spread_slab_impl<4, double>(L, m, force, flags, status, s);
    } else {
        if (delta == 2) force_spread_slab_impl<2, float>(L, m, force, flags, status, s);
        else if (delta == 3) force_spread_slab_impl<3, float>(L, m, force, flags, status, s);
        else force_spread_slab_impl<4, float>(L, m, force, flags, status, s);
    }
}

void launch_interp_partial_slab(int prec, int delta, const Lattice &L, const MeshDev &m, const void *pop,
                                const void *force, void *part, cudaStream_t s) {
    if (m.n_nodes == 0) return;
    if (prec == kF64) {
        if (delta == 2) interp_partial_slab_impl<2, double, double>(L, m, pop, force, part, s);
        else if (delta == 3) interp_partial_slab_impl<3, double, double>(L, m, pop, force, part, s);
        else interp_partial_slab_impl<4, double, double>(L, m, pop, force, part, s);
    } else if (prec == kF32) {
        if (delta == 2) interp_partial_slab_impl<2, float, float>(L, m, pop, force, part, s);
        else if (delta == 3) interp_partial_slab_impl<3, float, float>(L, m, pop, force, part, s);
        else interp_partial_slab_impl<4, float, float>(L, m, pop, force, part, s);
    } else {
        if (delta == 2) interp_partial_slab_impl<2, __half, float>(L, m, pop, force, part, s);
        else if (delta == 3) interp_partial_slab_impl<3, __half, float>(L, m, pop, force, part, s);
        else interp_partial_slab_impl<4, __half, float>(L, m, pop, force, part, s);
    }
}

void launch_slab_advect(int prec, const MeshDev &m, const void *const *parts, int n_parts, cudaStream_t s) {
    if (m.n_nodes == 0) return;
    const unsigned nb = (unsigned)((m.n_nodes + 127) / 128);
    if (prec == kF64)
        k_slab_advect<double><<<nb, 128, 0, s>>>(m.n_nodes, view<double>(m), (dvec4 *)m.u,
                                                 (const dvec4 *const *)parts, n_parts);
    else
        k_slab_advect<float><<<nb, 128, 0, s>>>(m.n_nodes, view<float>(m), (float4 *)m.u,
                                                (const float4 *const *)parts, n_parts);
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

// Copy of the node positions (and their low parts) into a snapshot, in one
// launch: 16-byte words, those of x first.
__global__ void k_copy_words(const uint4 *__restrict__ a, uint4 *__restrict__ a_out, long long na,
                             const uint4 *__restrict__ b, uint4 *__restrict__ b_out, long long nb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < na + nb;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < na) a_out[i] = a[i];
        else b_out[i - na] = b[i - na];
    }
}

void launch_snapshot_nodes(int prec, const MeshDev &m, int count, void *x_out, void *lo_out, cudaStream_t s) {
    if (count <= 0) return;
    const long long na = (long long)count * (prec == kF64 ? 2 : 1);  // dvec4: two words per node
    const long long nb = (prec == kF64 || !m.x_lo) ? 0 : (long long)count;
    const long long n = na + nb;
    const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 4 * 152);
    k_copy_words<<<blocks, 256, 0, s>>>((const uint4 *)m.x, (uint4 *)x_out, na, (const uint4 *)m.x_lo,
                                        (uint4 *)lo_out, nb);
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

IBLBM_BOUNDS_ACCESSOR(bounds_faults_ib)

}  // namespace iblbm
