// lbm.cu -- D3Q19 BGK collide-and-stream with Guo forcing and moving-wall
// bounce-back (Sec. II.A, Eqs. lbequation, equilibrium, latticeforce,
// lbmmomenta0/1), plus the lattice initialisation and read-back kernels.
//
// Data layout: populations are stored as deviations g_i = f_i - w_i from the
// rest equilibrium, structure of arrays [19][nz][ny][nx] (x fastest), in the
// storage type S (double, float or scaled half); arithmetic in T (double or
// float).  Two population buffers: the step reads f(t) from one and pushes
// f(t+1) into the other.  The force density is an array of 4-vectors per
// cell; only tiles flagged by the spreading kernel hold non-zero force, so
// the collide kernel reads it only there and zeroes the previous step's
// tiles as it passes.
#include "device_common.cuh"
#include "internal.h"

namespace iblbm {

// One thread per cell, one 32 x 8 x 1 tile per block.  Reads 19 coalesced
// values of f(t) at its own cell, collides, and pushes each post-collision
// value to the neighbour cell x + c_i (periodic in x and y).  A value that
// would cross a wall plane is reflected into the opposite direction of the
// same cell with Ladd's moving-wall term -2 w_i (c_i . u_w) / c_s^2.
template <typename S, typename T>
__global__ void __launch_bounds__(kTileX *kTileY)
    k_collide_stream(const S *__restrict__ src, S *__restrict__ dst,
                     const typename Vec4<T>::type *__restrict__ fcur,
                     const uint8_t *__restrict__ flag_cur,
                     typename Vec4<T>::type *__restrict__ fold, uint8_t *__restrict__ flag_old,
                     int nx, int ny, int nz, int ntx, int nty, long long ncell, T omega,
                     T u_wall, int *status) {
    using V4 = typename Vec4<T>::type;
    const int x = blockIdx.x * kTileX + threadIdx.x;
    const int y = blockIdx.y * kTileY + threadIdx.y;
    const int z = blockIdx.z;
    const long long tile = ((long long)z * nty + blockIdx.y) * ntx + blockIdx.x;
    const bool inside = (x < nx) && (y < ny);
    const long long cell = x + (long long)nx * (y + (long long)ny * z);

    // Block-uniform flags.  The previous step's force tiles are cleared here:
    // nothing reads them after the interpolation of the previous step.
    const bool has_old = flag_old[tile] != 0;
    const bool has_cur = flag_cur[tile] != 0;
    if (has_old) {
        if (inside) fold[cell] = V4{};
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) flag_old[tile] = 0;
    }
    if (!inside) return;

    T g[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) g[i] = Store<S, T>::load(src + i * ncell + cell);

    T drho = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        drho += g[i];
        if (q_cx(i)) jx += q_cx(i) > 0 ? g[i] : -g[i];
        if (q_cy(i)) jy += q_cy(i) > 0 ? g[i] : -g[i];
        if (q_cz(i)) jz += q_cz(i) > 0 ? g[i] : -g[i];
    }
    T fx = T(0), fy = T(0), fz = T(0);
    if (has_cur) {
        V4 f = fcur[cell];
        fx = f.x;
        fy = f.y;
        fz = f.z;
    }
    const T rho = T(1) + drho;
    if (!(rho > T(0.5) && rho < T(2))) set_status(status, kStatusUnstable);
    const T inv_rho = T(1) / rho;
    const T ux = (jx + T(0.5) * fx) * inv_rho;
    const T uy = (jy + T(0.5) * fy) * inv_rho;
    const T uz = (jz + T(0.5) * fz) * inv_rho;
    const T uu15 = T(1.5) * (ux * ux + uy * uy + uz * uz);
    const T guo = T(1) - T(0.5) * omega;
    const T uf = ux * fx + uy * fy + uz * fz;

    const int xp = (x + 1 == nx) ? 0 : x + 1;
    const int xm = (x == 0) ? nx - 1 : x - 1;
    const int yp = (y + 1 == ny) ? 0 : y + 1;
    const int ym = (y == 0) ? ny - 1 : y - 1;

#pragma unroll
    for (int i = 0; i < 19; ++i) {
        constexpr T zero = T(0);
        const int cx = q_cx(i), cy = q_cy(i), cz = q_cz(i);
        const T w = q_w<T>(i);
        T cu = zero;
        if (cx) cu += cx > 0 ? ux : -ux;
        if (cy) cu += cy > 0 ? uy : -uy;
        if (cz) cu += cz > 0 ? uz : -uz;
        // Eq. (equilibrium) minus the rest weight
        const T geq = w * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - uu15));
        T post = g[i] - omega * (g[i] - geq);
        if (has_cur) {
            // Eq. (latticeforce) with c_s^2 = 1/3
            T cf = zero;
            if (cx) cf += cx > 0 ? fx : -fx;
            if (cy) cf += cy > 0 ? fy : -fy;
            if (cz) cf += cz > 0 ? fz : -fz;
            post += guo * w * (T(3) * (cf - uf) + T(9) * cu * cf);
        }
        const int zt = z + cz;
        if ((cz > 0 && zt == nz) || (cz < 0 && z == 0)) {
            const T uw = (cz > 0) ? u_wall : -u_wall;
            const T wall = (cx == 0) ? zero : T(6) * w * (cx > 0 ? uw : -uw);
            Store<S, T>::store(dst + q_opp(i) * ncell + cell, post - wall);
        } else {
            const int xt = cx > 0 ? xp : (cx < 0 ? xm : x);
            const int yt = cy > 0 ? yp : (cy < 0 ? ym : y);
            const long long t = xt + (long long)nx * (yt + (long long)ny * zt);
            Store<S, T>::store(dst + i * ncell + t, post);
        }
    }
}

template <typename S, typename T>
__global__ void k_init_fluid(S *pop, int nx, int ny, int nz, long long ncell, int mode,
                             double u_wall) {
    long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= ncell) return;
    int z = (int)(cell / ((long long)nx * ny));
    double ux = 0.0;
    if (mode == 1) ux = 2.0 * u_wall / nz * (z - 0.5 * (nz - 1));
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        double cu = q_cx(i) * ux;
        double geq = q_w<double>(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * ux * ux);
        Store<S, T>::store(pop + i * ncell + cell, (T)geq);
    }
}

template <typename S, typename T>
__global__ void k_moments(const S *pop, const typename Vec4<T>::type *force, long long ncell,
                          double *rho_out, double *u_out) {
    long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= ncell) return;
    double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        double g = (double)Store<S, T>::load(pop + i * ncell + cell);
        drho += g;
        j[0] += q_cx(i) * g;
        j[1] += q_cy(i) * g;
        j[2] += q_cz(i) * g;
    }
    auto f = force[cell];
    double rho = 1.0 + drho;
    if (rho_out) rho_out[cell] = rho;
    if (u_out) {
        u_out[cell] = (j[0] + 0.5 * (double)f.x) / rho;
        u_out[ncell + cell] = (j[1] + 0.5 * (double)f.y) / rho;
        u_out[2 * ncell + cell] = (j[2] + 0.5 * (double)f.z) / rho;
    }
}

template <typename S, typename T>
__global__ void k_pop_to_f64(const S *pop, long long ncell, double *out) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= 19 * ncell) return;
    int i = (int)(k / ncell);
    out[k] = (double)Store<S, T>::load(pop + k) + q_w<double>(i);
}

template <typename S, typename T>
__global__ void k_f64_to_pop(const double *in, long long ncell, S *pop) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= 19 * ncell) return;
    int i = (int)(k / ncell);
    Store<S, T>::store(pop + k, (T)(in[k] - q_w<double>(i)));
}

template <typename T>
__global__ void k_force_to_f64(const typename Vec4<T>::type *force, long long ncell, double *out) {
    long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= ncell) return;
    auto f = force[cell];
    out[cell] = (double)f.x;
    out[ncell + cell] = (double)f.y;
    out[2 * ncell + cell] = (double)f.z;
}

static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <typename S, typename T>
static void collide_impl(const Lattice &L, const CollideArgs &a, cudaStream_t s) {
    using V4 = typename Vec4<T>::type;
    dim3 grid(L.ntx, L.nty, L.nz), block(kTileX, kTileY);
    k_collide_stream<S, T><<<grid, block, 0, s>>>(
        (const S *)a.src, (S *)a.dst, (const V4 *)a.fcur, a.flag_cur, (V4 *)a.fold, a.flag_old,
        L.nx, L.ny, L.nz, L.ntx, L.nty, L.ncell, (T)(1.0 / a.tau), (T)a.u_wall, a.status);
}

void launch_collide_stream(int prec, const Lattice &L, const CollideArgs &a, cudaStream_t s) {
    if (prec == kF64) collide_impl<double, double>(L, a, s);
    else if (prec == kF32) collide_impl<float, float>(L, a, s);
    else collide_impl<__half, float>(L, a, s);
}

void launch_init_fluid(int prec, const Lattice &L, void *pop, int mode, double u_wall,
                       cudaStream_t s) {
    unsigned nb = blocks_for(L.ncell, 256);
    if (prec == kF64) k_init_fluid<double, double><<<nb, 256, 0, s>>>((double *)pop, L.nx, L.ny, L.nz, L.ncell, mode, u_wall);
    else if (prec == kF32) k_init_fluid<float, float><<<nb, 256, 0, s>>>((float *)pop, L.nx, L.ny, L.nz, L.ncell, mode, u_wall);
    else k_init_fluid<__half, float><<<nb, 256, 0, s>>>((__half *)pop, L.nx, L.ny, L.nz, L.ncell, mode, u_wall);
}

void launch_moments(int prec, const Lattice &L, const void *pop, const void *force, double *rho,
                    double *u, cudaStream_t s) {
    unsigned nb = blocks_for(L.ncell, 256);
    if (prec == kF64) k_moments<double, double><<<nb, 256, 0, s>>>((const double *)pop, (const dvec4 *)force, L.ncell, rho, u);
    else if (prec == kF32) k_moments<float, float><<<nb, 256, 0, s>>>((const float *)pop, (const float4 *)force, L.ncell, rho, u);
    else k_moments<__half, float><<<nb, 256, 0, s>>>((const __half *)pop, (const float4 *)force, L.ncell, rho, u);
}

void launch_pop_to_f64(int prec, const Lattice &L, const void *pop, double *out, cudaStream_t s) {
    unsigned nb = blocks_for(19 * L.ncell, 256);
    if (prec == kF64) k_pop_to_f64<double, double><<<nb, 256, 0, s>>>((const double *)pop, L.ncell, out);
    else if (prec == kF32) k_pop_to_f64<float, float><<<nb, 256, 0, s>>>((const float *)pop, L.ncell, out);
    else k_pop_to_f64<__half, float><<<nb, 256, 0, s>>>((const __half *)pop, L.ncell, out);
}

void launch_f64_to_pop(int prec, const Lattice &L, const double *in, void *pop, cudaStream_t s) {
    unsigned nb = blocks_for(19 * L.ncell, 256);
    if (prec == kF64) k_f64_to_pop<double, double><<<nb, 256, 0, s>>>(in, L.ncell, (double *)pop);
    else if (prec == kF32) k_f64_to_pop<float, float><<<nb, 256, 0, s>>>(in, L.ncell, (float *)pop);
    else k_f64_to_pop<__half, float><<<nb, 256, 0, s>>>(in, L.ncell, (__half *)pop);
}

void launch_force_to_f64(int prec, const Lattice &L, const void *force, double *out, cudaStream_t s) {
    unsigned nb = blocks_for(L.ncell, 256);
    if (prec == kF64) k_force_to_f64<double><<<nb, 256, 0, s>>>((const dvec4 *)force, L.ncell, out);
    else k_force_to_f64<float><<<nb, 256, 0, s>>>((const float4 *)force, L.ncell, out);
}

}  // namespace iblbm
