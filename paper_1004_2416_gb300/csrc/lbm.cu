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
#include <algorithm>
#include <type_traits>

#include "device_common.cuh"
#include "internal.h"

namespace iblbm {

// Collide-and-stream of one cell (x, y, z) of an nx x ny x nz lattice whose
// populations start at src / dst and force density at fcur.  Reads the 19
// values of f(t) at the cell, collides, and pushes each post-collision value to
// the neighbour cell x + c_i (periodic in x and y).  A value that would cross
// a wall plane is reflected into the opposite direction of the same cell with
// Ladd's moving-wall term -2 w_i (c_i . u_w) / c_s^2.
// LIN: the linearised equilibrium w_i rho (1 + 3 c_i.u) of Sec. IV.A instead
// of Eq. (equilibrium); the forcing term is Eq. (latticeforce) either way.
template <typename S, typename T, bool LIN = false>
__device__ __forceinline__ void collide_cell(const S *__restrict__ src, S *__restrict__ dst,
                                             const typename Vec4<T>::type *__restrict__ fcur,
                                             bool has_cur, int x, int y, int z, int nx, int ny,
                                             int nz, long long ncell, T omega, T u_wall,
                                             int *status,
                                             typename Vec4<T>::type *__restrict__ moments = nullptr) {
    using V4 = typename Vec4<T>::type;
    const long long cell = x + (long long)nx * (y + (long long)ny * z);
    if (!IBLBM_OK(cell, 1, ncell)) return;
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
    if (moments) moments[cell] = V4{jx, jy, jz, drho};
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
    // A = drho - 3/2 rho u.u: the part of the equilibrium (minus the weight)
    // common to all directions (drho alone for the linearised form)
    const T A = LIN ? drho : drho - T(1.5) * rho * (ux * ux + uy * uy + uz * uz);
    const T ufm = T(-3) * (ux * fx + uy * fy + uz * fz);
    const T keep = T(1) - omega, guo = T(1) - T(0.5) * omega;

    // push offsets of the neighbour cells (periodic in x and y)
    const long long sz = (long long)nx * ny;
    const long long dyp = (y + 1 == ny) ? -(long long)(ny - 1) * nx : (long long)nx;
    const long long dym = (y == 0) ? (long long)(ny - 1) * nx : -(long long)nx;
    const int dxp = (x + 1 == nx) ? 1 - nx : 1, dxm = (x == 0) ? nx - 1 : -1;
    auto emit = [&](const int i, const T post) {
        const int cx = q_cx(i), cy = q_cy(i), cz = q_cz(i);
        if ((cz > 0 && z + 1 == nz) || (cz < 0 && z == 0)) {
            const T uw = (cz > 0) ? u_wall : -u_wall;
            const T wall = (cx == 0) ? T(0) : T(6) * q_w<T>(i) * (cx > 0 ? uw : -uw);
            Store<S, T>::store(dst + q_opp(i) * ncell + cell, post - wall);
        } else {
            const long long t = cell + (cx > 0 ? dxp : (cx < 0 ? dxm : 0)) +
                                (cy > 0 ? dyp : (cy < 0 ? dym : 0)) + cz * sz;
            if (IBLBM_OK(t, 1, ncell)) Store<S, T>::store(dst + i * ncell + t, post);
        }
    };
    // rest direction: equilibrium w0 A, force term w0 (1 - omega/2)(-3 u.f)
    {
        const T w = q_w<T>(0);
        T post = keep * g[0] + omega * w * A;
        if (has_cur) post += guo * w * ufm;
        emit(0, post);
    }
    // opposite pairs (c, -c), c with its first nonzero component positive:
    // with r = rho c.u the equilibrium (minus the weight) is
    // w (A + 9/2 r c.u +- 3 r) (Eq. equilibrium; the linearised form drops the
    // quadratic term) and the force term (Eq. latticeforce, c_s^2 = 1/3)
    // (1 - omega/2) w (9 (c.u)(c.f) - 3 u.f +- 3 c.f)
#pragma unroll
    for (int j = 1; j < 19; j += 2) {
        const int ip = (q_cx(j) > 0 || (q_cx(j) == 0 && (q_cy(j) > 0 || (q_cy(j) == 0 && q_cz(j) > 0))))
                           ? j : q_opp(j);
        const int im = q_opp(ip);
        const int cx = q_cx(ip), cy = q_cy(ip), cz = q_cz(ip);
        const T w = q_w<T>(ip);
        T cu = cx ? ux : (cy ? uy : uz);
        if (cx && cy) cu = cy > 0 ? cu + uy : cu - uy;
        if ((cx || cy) && cz) cu = cz > 0 ? cu + uz : cu - uz;
        const T r = rho * cu;
        const T e = LIN ? A : A + T(4.5) * r * cu;
        T postp = keep * g[ip] + omega * w * (e + T(3) * r);
        T postm = keep * g[im] + omega * w * (e - T(3) * r);
        if (has_cur) {
            T cf = cx ? fx : (cy ? fy : fz);
            if (cx && cy) cf = cy > 0 ? cf + fy : cf - fy;
            if ((cx || cy) && cz) cf = cz > 0 ? cf + fz : cf - fz;
            const T base = T(9) * cu * cf + ufm;
            postp += guo * w * (base + T(3) * cf);
            postm += guo * w * (base - T(3) * cf);
        }
        emit(ip, postp);
        emit(im, postm);
    }
}

// One thread per cell, one 32 x 8 x 1 tile per block.
template <typename S, typename T, bool LIN>
__global__ void __launch_bounds__(kTileX *kTileY)
    k_collide_stream(const S *__restrict__ src, S *__restrict__ dst,
                     const typename Vec4<T>::type *__restrict__ fcur,
                     const uint8_t *__restrict__ flag_cur,
                     typename Vec4<T>::type *__restrict__ fold, uint8_t *__restrict__ flag_old,
                     int nx, int ny, int nz, int ntx, int nty, long long ncell, T omega,
                     T u_wall, int *status, typename Vec4<T>::type *__restrict__ moments) {
    using V4 = typename Vec4<T>::type;
    prior_grid_wait();
    allow_dependents();
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
    collide_cell<S, T, LIN>(src, dst, fcur, has_cur, x, y, z, nx, ny, nz, ncell, omega, u_wall, status, moments);
}

// Batched, persistent collide-and-stream over many independent lattices
// (runs).  The work list holds (run, tile) pairs of every run; each block
// walks it with a grid stride.  A run's tiles have its own shape tx x ty
// (tx * ty = 256 threads), picked per box size by the autotuner; the force
// flags of a run use the same tiles.
template <typename S, typename T, bool LIN>
__global__ void __launch_bounds__(256)
    k_collide_batch(const S *__restrict__ src, S *__restrict__ dst,
                    const typename Vec4<T>::type *__restrict__ fcur,
                    const uint8_t *__restrict__ flag_cur,
                    typename Vec4<T>::type *__restrict__ fold, uint8_t *__restrict__ flag_old,
                    const RunDesc *__restrict__ runs, const int2 *__restrict__ items, int n_items,
                    int *status) {
    using V4 = typename Vec4<T>::type;
    prior_grid_wait();
    allow_dependents();
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int2 w = items[it];
        const RunDesc R = runs[w.x];
        const int per_z = R.ntx * R.nty;
        const int z = w.y / per_z, rem = w.y - z * per_z;
        const int tyi = rem / R.ntx, txi = rem - tyi * R.ntx;
        const int x = txi * R.tx + ((int)threadIdx.x & (R.tx - 1));  // tile sides are powers of two
        const int y = tyi * R.ty + ((int)threadIdx.x >> (__ffs(R.tx) - 1));
        const bool inside = x < R.nx && y < R.ny;
        const long long tile = R.tile_off + w.y;
        const bool has_old = flag_old[tile] != 0;
        const bool has_cur = flag_cur[tile] != 0;
        if (has_old) {
            if (inside) fold[R.cell_off + x + (long long)R.nx * (y + (long long)R.ny * z)] = V4{};
            __syncthreads();
            if (threadIdx.x == 0) flag_old[tile] = 0;
        }
        if (inside)
            collide_cell<S, T, LIN>(src + 19 * R.cell_off, dst + 19 * R.cell_off, fcur + R.cell_off,
                               has_cur, x, y, z, R.nx, R.ny, R.nz, R.ncell, (T)R.omega,
                               (T)R.u_wall, status);
    }
}

// Vector loads and stores of 4 consecutive cells of one direction.  The
// *_raw forms move the stored values without the binary16 scale (kScale
// storage units per unit of g; a power of two, so scaling is exact).
template <typename S>
struct Quad;
template <>
struct Quad<float> {
    static constexpr float kScale = 1.f;
    static __device__ __forceinline__ void load_raw(const float *p, float2 &a, float2 &b) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        a = make_float2(q.x, q.y);
        b = make_float2(q.z, q.w);
    }
    static __device__ __forceinline__ void store_raw(float *p, float a, float b, float c, float d) {
        *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
    }
    static __device__ __forceinline__ void load(const float *p, float v[4]) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    static __device__ __forceinline__ void store(float *p, float a, float b, float c, float d) {
        *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
    }
};
template <>
struct Quad<__half> {
    static constexpr float kScale = kHalfScale;
    static __device__ __forceinline__ void load_raw(const __half *p, float2 &a, float2 &b) {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
        a = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
        b = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
    }
    static __device__ __forceinline__ void store_raw(__half *p, float a, float b, float c, float d) {
        const __half2 lo = __floats2half2_rn(a, b);
        const __half2 hi = __floats2half2_rn(c, d);
        uint2 q;
        q.x = *reinterpret_cast<const unsigned *>(&lo);
        q.y = *reinterpret_cast<const unsigned *>(&hi);
        *reinterpret_cast<uint2 *>(p) = q;
    }
    static __device__ __forceinline__ void load(const __half *p, float v[4]) {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
        v[0] = a.x * kHalfInvScale; v[1] = a.y * kHalfInvScale;
        v[2] = b.x * kHalfInvScale; v[3] = b.y * kHalfInvScale;
    }
    static __device__ __forceinline__ void store(__half *p, float a, float b, float c, float d) {
        const __half2 lo = __floats2half2_rn(a * kHalfScale, b * kHalfScale);
        const __half2 hi = __floats2half2_rn(c * kHalfScale, d * kHalfScale);
        uint2 q;
        q.x = *reinterpret_cast<const unsigned *>(&lo);
        q.y = *reinterpret_cast<const unsigned *>(&hi);
        *reinterpret_cast<uint2 *>(p) = q;
    }
};

// The same quad loads from shared memory (a staged tile), in storage units.
template <typename S>
struct QuadSmem;
template <>
struct QuadSmem<float> {
    static __device__ __forceinline__ void load(const float *p, float2 &a, float2 &b) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        a = make_float2(q.x, q.y);
        b = make_float2(q.z, q.w);
    }
};
template <>
struct QuadSmem<__half> {
    static __device__ __forceinline__ void load(const __half *p, float2 &a, float2 &b) {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        a = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
        b = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
    }
};

// Vectorised collide-and-stream for nx = 4 * LR, LR a power of two <= 256:
// each thread owns 4 consecutive cells of one x-row and LR lanes cover the
// row.  With LR <= 32 a warp covers 32 / LR rows; with LR > 32 a row spans
// LR / 32 warps.  A block has 8 warps, or holds one row (X4Shape).  All 19
// loads and the stores are 16-byte (float) or 8-byte (half) vectors.
// Streaming along x shifts a thread's 4
// post-collision values by one cell; the value that crosses into the
// neighbouring thread's quad comes by a warp shuffle (within the row's lane
// segment when LR <= 32, which also closes the periodic wrap in x).  When a
// row spans several warps every lane still stores its quad as one vector;
// the edge lane that got the wrong crossing value (the shuffle wraps within
// its own warp) rewrites that one cell after a block barrier with the value
// the neighbouring warp's edge lane left in shared memory.  One force flag
// per thread's quad.
// Paired FP32 arithmetic (two cells per instruction).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Scalar store of a value already in storage units.
template <typename S>
struct StoreRaw;
template <>
struct StoreRaw<float> {
    static __device__ __forceinline__ void store(float *p, float v) { *p = v; }
};
template <>
struct StoreRaw<__half> {
    static __device__ __forceinline__ void store(__half *p, float v) { *p = __float2half_rn(v); }
};

template <int LR>
__device__ __forceinline__ float from_left(float v, int lane) {
    constexpr int W = LR <= 32 ? LR : 32;
    const int lx = lane & (W - 1);
    return __shfl_sync(0xffffffffu, v, (lx + W - 1) & (W - 1), W);
}
template <int LR>
__device__ __forceinline__ float from_right(float v, int lane) {
    constexpr int W = LR <= 32 ? LR : 32;
    const int lx = lane & (W - 1);
    return __shfl_sync(0xffffffffu, v, (lx + 1) & (W - 1), W);
}

// Slot of a direction with c_x != 0 (1, 2 and 7..14) among the ten such
// directions.
__host__ __device__ constexpr int edge_slot(int i) { return i <= 2 ? i - 1 : i - 5; }

// rows of a block of NWB warps
template <int LR, int NWB = 8>
__host__ __device__ constexpr int rows_per_block() {
    return LR <= 32 ? NWB * (32 / LR) : NWB / (LR / 32);
}

// The 19 direction arrays of a population buffer as the vectorised kernel
// addresses them: DirPtrs passes the 19 base pointers as kernel parameters (an
// address is a base pointer from the parameter bank plus the cell offset),
// DirStride one base pointer and the direction stride.
template <typename P>
struct DirPtrs {
    P *p[19];
    __device__ __forceinline__ P *operator()(int i, int) const { return p[i]; }
};
template <typename P>
struct DirStride {
    P *base;
    __device__ __forceinline__ P *operator()(int i, int ncell) const { return base + (size_t)i * ncell; }
};
template <typename D, typename P>
D make_dirs(P *base, int ncell) {
    D d{};
    if constexpr (std::is_same<D, DirStride<P>>::value) {
        d.base = base;
    } else {
        for (int i = 0; i < 19; ++i) d.p[i] = base + (size_t)i * ncell;
    }
    return d;
}

// Launch shape of k_collide_stream_x4: blocks of eight warps, two per SM
// (128 registers).  Binary16 rows that span several warps take one row per
// block, so that the barrier before the warp-edge rewrite holds only the
// warps of that row, and, for two or four warps per row, about 20 warps per
// SM in 96 registers, the populations kept as loaded and converted where
// used (QuadRawHalf).  Measured on the 256 x 128 x 128 FP16 lattice
// (two warps per row): 70.6 us per collide with eight-warp blocks, 67.6 with
// four-warp blocks, 66.6 with one-row blocks at 20 warps per SM.
template <typename S, int LR>
struct X4Shape {
    static constexpr bool kRowBlocks = sizeof(S) == 2 && LR > 32;
    static constexpr int kWarps = kRowBlocks ? LR / 32 : 8;
    static constexpr bool kRaw = kRowBlocks && LR <= 128;
    static constexpr int kMinBlocks = kRaw ? 20 / kWarps : 2;
    // binary16: the direction base pointers as parameters (256 x 128 x 128
    // lattice: 66.5 -> 63.9 us per collide); float storage keeps one base and
    // the stride (on the 128^3 lattice the table took 9 % of the kernel's
    // instructions away but none of its time, which the HBM sets)
    using Src = std::conditional_t<sizeof(S) == 2, DirPtrs<const S>, DirStride<const S>>;
    using Dst = std::conditional_t<sizeof(S) == 2, DirPtrs<S>, DirStride<S>>;
};

// The 19 populations of a thread's quad as collide_quad reads them: pair h
// (cells (0,1) or (2,3)) of direction i, in storage units, once for the
// moments and once for the collision of its direction.  QuadRegs holds them
// as floats; QuadRawHalf holds the binary16 words as loaded (38 registers
// instead of 76) and converts at each use, through an opaque conversion that
// the compiler can neither merge with the first nor hoist, so that the
// quad's 76 floats are never live at once.  Both give the same values.
struct QuadRegs {
    const float2 (&g)[19][2];
    __device__ __forceinline__ float2 moment(int i, int h) const { return g[i][h]; }
    __device__ __forceinline__ float2 use(int i, int h) const { return g[i][h]; }
};
struct QuadRawHalf {
    const uint2 (&w)[19];
    __device__ __forceinline__ float2 moment(int i, int h) const {
        const unsigned v = h ? w[i].y : w[i].x;
        return __half22float2(*reinterpret_cast<const __half2 *>(&v));
    }
    __device__ __forceinline__ float2 use(int i, int h) const {
        float a, b;
        asm volatile("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
                     : "=f"(a), "=f"(b)
                     : "r"(h ? w[i].y : w[i].x));
        return make_float2(a, b);
    }
};

// Collision and streaming of one thread's quad (4 consecutive cells of a row)
// from its 19 populations g (pairs (0,1) and (2,3), storage units), shared by
// the kernel that loads them from global memory and the one that loads them
// from a tile staged in shared memory.  Every lane of the block calls it (the
// inactive ones too: they join the shuffles and, for rows spanning several
// warps, the block barrier of the warp-edge rewrite; `edge` holds one row of
// ten values per warp).
template <typename S, int LR, bool WM, bool LIN, typename Src, typename Dst>
__device__ __forceinline__ void collide_quad(const Src &g, const Dst &dst,
                                             const float4 *__restrict__ fcur, bool has_cur, bool active, int row,
                                             int y, int z, int x0, int cell0, int lane, int warp, int ny, int nz,
                                             int ncell, float omega, float u_wall, int *status,
                                             float4 *__restrict__ moments, float (*edge)[10]) {
    constexpr int NX = 4 * LR;
    constexpr float SC = Quad<S>::kScale, ISC = 1.f / Quad<S>::kScale;
    // per cell: moments, velocity with the half force, and the pair vectors
    // of the per-direction arithmetic.  A = D + kScale rho (-3/2 u.u) is the
    // part of the equilibrium (minus the weight) common to all directions
    // (D alone for the linearised form); Ufm = -3 u.f.
    float2 Ux[2], Uy[2], Uz[2], Rs[2], A[2], Fx[2], Fy[2], Fz[2], Ufm[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float2 d = make_float2(0.f, 0.f), jx = d, jy = d, jz = d;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float2 gi = g.moment(i, h);
            d = add2(d, gi);
            if (q_cx(i)) jx = q_cx(i) > 0 ? add2(jx, gi) : sub2(jx, gi);
            if (q_cy(i)) jy = q_cy(i) > 0 ? add2(jy, gi) : sub2(jy, gi);
            if (q_cz(i)) jz = q_cz(i) > 0 ? add2(jz, gi) : sub2(jz, gi);
        }
        float fv[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        if (has_cur && IBLBM_OK(cell0, 4, ncell)) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float4 f = fcur[cell0 + 2 * h + e];
                fv[e][0] = f.x; fv[e][1] = f.y; fv[e][2] = f.z;
            }
        }
        float ux[2], uy[2], uz[2], rs[2], ac[2], ufm[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float dr = e ? d.y : d.x;
            const float de = dr * ISC, jxe = (e ? jx.y : jx.x) * ISC;
            const float jye = (e ? jy.y : jy.x) * ISC, jze = (e ? jz.y : jz.x) * ISC;
            if constexpr (WM) {
                if (active && IBLBM_OK(cell0 + 2 * h + e, 1, ncell))
                    moments[cell0 + 2 * h + e] = make_float4(jxe, jye, jze, de);
            }
            const float rho = 1.f + de;
            if (active && !(rho > 0.5f && rho < 2.f)) set_status(status, kStatusUnstable);
            const float inv = 1.f / rho;
            ux[e] = (jxe + 0.5f * fv[e][0]) * inv;
            uy[e] = (jye + 0.5f * fv[e][1]) * inv;
            uz[e] = (jze + 0.5f * fv[e][2]) * inv;
            rs[e] = SC * rho;
            ac[e] = LIN ? dr : dr + rs[e] * (-1.5f * (ux[e] * ux[e] + uy[e] * uy[e] + uz[e] * uz[e]));
            ufm[e] = -3.f * (ux[e] * fv[e][0] + uy[e] * fv[e][1] + uz[e] * fv[e][2]);
        }
        Ux[h] = make_float2(ux[0], ux[1]);
        Uy[h] = make_float2(uy[0], uy[1]);
        Uz[h] = make_float2(uz[0], uz[1]);
        Rs[h] = make_float2(rs[0], rs[1]);
        A[h] = make_float2(ac[0], ac[1]);
        Fx[h] = make_float2(fv[0][0], fv[1][0]);
        Fy[h] = make_float2(fv[0][1], fv[1][1]);
        Fz[h] = make_float2(fv[0][2], fv[1][2]);
        Ufm[h] = make_float2(ufm[0], ufm[1]);
    }
    const float guo_s = SC * (1.f - 0.5f * omega);
    const float2 keep2 = make_float2(1.f - omega, 1.f - omega);
    const bool top = z + 1 == nz, bottom = z == 0;
    // destination row offsets: this row, the periodic neighbour rows in y, the planes in z
    const int row0 = NX * row, plane = NX * ny;
    const int dyp = (y + 1 == ny) ? NX * (1 - ny) : NX, dym = (y == 0) ? NX * (ny - 1) : -NX;

    // x shift, wall bounce-back and store of the post-collision values p of
    // direction i
    auto emit = [&](const int i, const float p[4]) {
        const int cx = q_cx(i), cy = q_cy(i), cz = q_cz(i);
        // x shift of the quad (before any branch: every lane takes part)
        float o0 = p[0], o1 = p[1], o2 = p[2], o3 = p[3];
        if (cx > 0) {
            const float in = from_left<LR>(p[3], lane);
            o0 = in; o1 = p[0]; o2 = p[1]; o3 = p[2];
        } else if (cx < 0) {
            const float in = from_right<LR>(p[0], lane);
            o0 = p[1]; o1 = p[2]; o2 = p[3]; o3 = in;
        }
        if (!active) return;
        if (cz > 0 ? top : (cz < 0 ? bottom : false)) {
            // bounce-back into the opposite direction of the same cells, with
            // the moving-wall term in storage units
            const float uw = (cz > 0) ? u_wall : -u_wall;
            const float wall = (cx == 0) ? 0.f : SC * 6.f * q_w<float>(i) * (cx > 0 ? uw : -uw);
            if (IBLBM_OK(cell0, 4, ncell))
                Quad<S>::store_raw(dst(q_opp(i), ncell) + cell0, p[0] - wall, p[1] - wall,
                                   p[2] - wall, p[3] - wall);
        } else {
            S *rowp = dst(i, ncell) + (row0 + (cy > 0 ? dyp : (cy < 0 ? dym : 0)) + cz * plane);
            if (IBLBM_OK((long long)(row0 + (cy > 0 ? dyp : (cy < 0 ? dym : 0)) + cz * plane) + x0, 4, ncell))
                Quad<S>::store_raw(rowp + x0, o0, o1, o2, o3);
            if constexpr (LR > 32) {
                // the value that crosses into the neighbouring warp
                if (cx > 0 && lane == 31) edge[warp][edge_slot(i)] = p[3];
                if (cx < 0 && lane == 0) edge[warp][edge_slot(i)] = p[0];
            }
        }
    };

    // rest direction: c = 0, equilibrium w0 A, force term w0 (1 - omega/2) (-3 u.f)
    {
        const float w = q_w<float>(0);
        const float2 omw = make_float2(omega * w, omega * w), gw = make_float2(guo_s * w, guo_s * w);
        float p[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 post = fma2(omw, A[h], mul2(keep2, g.use(0, h)));
            if (has_cur) post = fma2(gw, Ufm[h], post);
            p[2 * h] = post.x;
            p[2 * h + 1] = post.y;
        }
        emit(0, p);
    }
    // direction pairs (c, -c), c with its first nonzero component positive:
    // with r = kScale rho c.u the equilibrium (minus the weight) is
    // w (A + 9/2 r c.u +- 3 r) (Eq. equilibrium; the linearised form drops the
    // quadratic term) and the force term (Eq. latticeforce)
    // (1 - omega/2) w (9 (c.u)(c.f) - 3 u.f +- 3 c.f)
#pragma unroll
    for (int j = 1; j < 19; j += 2) {
        const int ip = (q_cx(j) > 0 || (q_cx(j) == 0 && (q_cy(j) > 0 || (q_cy(j) == 0 && q_cz(j) > 0))))
                           ? j : q_opp(j);
        const int im = q_opp(ip);
        const int cx = q_cx(ip), cy = q_cy(ip), cz = q_cz(ip);
        const float w = q_w<float>(ip);
        const float2 omw = make_float2(omega * w, omega * w), gw = make_float2(guo_s * w, guo_s * w);
        float pp[4], pm[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            // c.u from the first nonzero component (positive) on
            float2 cu = cx ? Ux[h] : (cy ? Uy[h] : Uz[h]);
            if (cx && cy) cu = cy > 0 ? add2(cu, Uy[h]) : sub2(cu, Uy[h]);
            if ((cx || cy) && cz) cu = cz > 0 ? add2(cu, Uz[h]) : sub2(cu, Uz[h]);
            const float2 r = mul2(Rs[h], cu);
            const float2 e = LIN ? A[h] : fma2(mul2(r, make_float2(4.5f, 4.5f)), cu, A[h]);
            const float2 gp = fma2(r, make_float2(3.f, 3.f), e);
            const float2 gm = fma2(r, make_float2(-3.f, -3.f), e);
            float2 postp = fma2(omw, gp, mul2(keep2, g.use(ip, h)));
            float2 postm = fma2(omw, gm, mul2(keep2, g.use(im, h)));
            if (has_cur) {
                float2 cf = cx ? Fx[h] : (cy ? Fy[h] : Fz[h]);
                if (cx && cy) cf = cy > 0 ? add2(cf, Fy[h]) : sub2(cf, Fy[h]);
                if ((cx || cy) && cz) cf = cz > 0 ? add2(cf, Fz[h]) : sub2(cf, Fz[h]);
                const float2 base = fma2(mul2(cu, cf), make_float2(9.f, 9.f), Ufm[h]);
                postp = fma2(gw, fma2(cf, make_float2(3.f, 3.f), base), postp);
                postm = fma2(gw, fma2(cf, make_float2(-3.f, -3.f), base), postm);
            }
            pp[2 * h] = postp.x;
            pp[2 * h + 1] = postp.y;
            pm[2 * h] = postm.x;
            pm[2 * h + 1] = postm.y;
        }
        emit(ip, pp);
        emit(im, pm);
    }
    if constexpr (LR > 32) {
        // lane 0 (c_x > 0) and lane 31 (c_x < 0) stored a value from their own
        // warp's other edge; rewrite that cell with the neighbouring warp's
        __syncthreads();
        if (active && (lane == 0 || lane == 31)) {
            constexpr int WPR = LR / 32;
            const int wr = warp % WPR, wb = warp - wr;
            const int from = wb + (lane == 0 ? (wr + WPR - 1) % WPR : (wr + 1) % WPR);
#pragma unroll
            for (int i = 1; i < 19; ++i) {
                const int cx = q_cx(i), cy = q_cy(i), cz = q_cz(i);
                if (cx == 0 || (cz > 0 ? top : (cz < 0 ? bottom : false))) continue;
                if ((cx > 0) != (lane == 0)) continue;
                S *rowp = dst(i, ncell) + (row0 + (cy > 0 ? dyp : (cy < 0 ? dym : 0)) + cz * plane);
                if (IBLBM_OK((long long)(row0 + (cy > 0 ? dyp : (cy < 0 ? dym : 0)) + cz * plane) + x0 +
                                 (cx > 0 ? 0 : 3), 1, ncell))
                    StoreRaw<S>::store(rowp + x0 + (cx > 0 ? 0 : 3), edge[from][edge_slot(i)]);
            }
        }
    }
}

// WM: also write the moments of f(t), float4 (j, rho - 1) per cell.
// LIN: the linearised equilibrium (as collide_cell).
template <typename S, int LR, bool WM, bool LIN = false>
__global__ void __launch_bounds__(32 * X4Shape<S, LR>::kWarps, X4Shape<S, LR>::kMinBlocks)
    k_collide_stream_x4(const typename X4Shape<S, LR>::Src src, const typename X4Shape<S, LR>::Dst dst,
                        const float4 *__restrict__ fcur, const uint8_t *__restrict__ flag_cur,
                        float4 *__restrict__ fold, uint8_t *__restrict__ flag_old, int ny, int nz,
                        int ncell, float omega, float u_wall, int *status, float4 *__restrict__ moments) {
    constexpr int NX = 4 * LR;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nrows = ny * nz;
    int row_raw, lx;
    if constexpr (LR <= 32) {
        row_raw = blockIdx.x * rows_per_block<LR, X4Shape<S, LR>::kWarps>() + warp * (32 / LR) + lane / LR;
        lx = lane & (LR - 1);
    } else {
        constexpr int WPR = LR / 32;
        row_raw = blockIdx.x * rows_per_block<LR, X4Shape<S, LR>::kWarps>() + warp / WPR;
        lx = (warp % WPR) * 32 + lane;
    }
    const bool active = row_raw < nrows;
    const int row = active ? row_raw : nrows - 1;  // inactive lanes still join the exchanges
    const int y = row % ny, z = row / ny;
    const int x0 = 4 * lx;
    const int cell0 = x0 + NX * row;
    __shared__ float edge[8][10];  // rows spanning several warps: crossing values by warp and direction

    // the force flags and density come from the spreading kernel before this
    // one (reading the populations before waiting for it puts the flags'
    // round trip after the loads: slower)
    prior_grid_wait();
    allow_dependents();

    // one force flag per quad: this thread's own
    constexpr int FTX = 4;  // one force flag per quad (Lattice::ftx)
    const int fidx = row * (NX / FTX) + x0 / FTX;
    const bool flag_ok = IBLBM_OK(fidx, 1, (long long)nrows * (NX / FTX));
    const bool has_old = flag_ok && flag_old[fidx] != 0;
    const bool has_cur = flag_ok && flag_cur[fidx] != 0;
    if (has_old && active && IBLBM_OK(cell0, 4, ncell)) {
#pragma unroll
        for (int k = 0; k < 4; ++k) fold[cell0 + k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (has_old && active) flag_old[fidx] = 0;

    // Arithmetic on cell pairs (0,1) and (2,3) with the paired FP32
    // instructions of sm_100+, in storage units: G = kScale g, so binary16
    // values are used as loaded (exact power-of-two scale folded into the
    // per-cell quantities).
    const bool quad_ok = IBLBM_OK(cell0, 4, ncell);  // constant true in the normal build
    if constexpr (X4Shape<S, LR>::kRaw) {
        uint2 raw[19];
#pragma unroll
        for (int i = 0; i < 19; ++i)
            raw[i] = quad_ok ? __ldg(reinterpret_cast<const uint2 *>(src(i, ncell) + cell0))
                             : make_uint2(0u, 0u);
        collide_quad<S, LR, WM, LIN>(QuadRawHalf{raw}, dst, fcur, has_cur, active, row, y, z, x0, cell0, lane,
                                     warp, ny, nz, ncell, omega, u_wall, status, moments, edge);
    } else {
        float2 g[19][2];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            if (quad_ok) {
                Quad<S>::load_raw(src(i, ncell) + cell0, g[i][0], g[i][1]);
            } else {
                g[i][0] = make_float2(0.f, 0.f);
                g[i][1] = g[i][0];
            }
        }
        collide_quad<S, LR, WM, LIN>(QuadRegs{g}, dst, fcur, has_cur, active, row, y, z, x0, cell0, lane, warp,
                                     ny, nz, ncell, omega, u_wall, status, moments, edge);
    }
}

// ---- the same on tiles staged in shared memory by the bulk-copy engine ---------------
// Persistent variant of k_collide_stream_x4: each block walks tiles of TR =
// THREADS * 4 / nx consecutive rows.  For every tile one thread issues 19
// bulk copies (one per direction, the tile's rows being contiguous in each
// direction's array) into one of two shared-memory buffers; the copies of the
// next tile run while the block computes the current one, so the warps never
// wait on global loads and their issue slots go to the arithmetic and the
// stores.  A wait that runs past wait_ns nanoseconds records kStatusTimeout,
// waits (bounded) for the copies still in flight and leaves the block.
template <typename S, int LR, bool LIN, int THREADS>
__global__ void __launch_bounds__(THREADS, 2)
    k_collide_stream_tma(const S *__restrict__ src, S *__restrict__ dst, const float4 *__restrict__ fcur,
                         const uint8_t *__restrict__ flag_cur, float4 *__restrict__ fold,
                         uint8_t *__restrict__ flag_old, int ny, int nz, int ncell, float omega, float u_wall,
                         int *status, int n_tiles, unsigned long long wait_ns) {
    constexpr int NX = 4 * LR;
    constexpr int TR = THREADS * 4 / NX;  // rows per tile
    constexpr int TILE = TR * NX;         // cells per tile
    constexpr int NW = THREADS / 32;
    static_assert(TR >= 1 && TR * NX == THREADS * 4, "a tile is a whole number of rows");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S *stage = reinterpret_cast<S *>(smem_raw);  // [2][19][TILE]
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float edge[NW][10];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int lr, lx;  // row within the tile, lane within the row
    if constexpr (LR <= 32) {
        lr = warp * (32 / LR) + lane / LR;
        lx = lane & (LR - 1);
    } else {
        constexpr int WPR = LR / 32;
        lr = warp / WPR;
        lx = (warp % WPR) * 32 + lane;
    }
    const int nrows = ny * nz;
    const int x0 = 4 * lx;

    prior_grid_wait();
    allow_dependents();
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        fence_async_smem();
    }
    __syncthreads();
    // thread 0: copies of tile t into buffer b
    auto issue = [&](int t, int b) {
        const int r0 = t * TR;
        const int nr = min(TR, nrows - r0);
        const unsigned bytes = (unsigned)(nr * NX * (int)sizeof(S));
        mbar_expect_bytes(&bar[b], 19u * bytes);
#pragma unroll 1
        for (int i = 0; i < 19; ++i)
            if (IBLBM_OK((long long)r0 * NX, (long long)nr * NX, ncell))  // else the wait gives up, reported
                bulk_copy_to_smem(stage + ((size_t)b * 19 + i) * TILE, src + (size_t)i * ncell + (size_t)r0 * NX,
                                  bytes, &bar[b]);
    };
    int pending[2] = {0, 0};  // thread 0: copies issued and not yet waited for, per buffer
    if (threadIdx.x == 0) {
        if ((int)blockIdx.x < n_tiles) { issue(blockIdx.x, 0); pending[0] = 1; }
        if ((int)(blockIdx.x + gridDim.x) < n_tiles) { issue(blockIdx.x + gridDim.x, 1); pending[1] = 1; }
    }
    constexpr int FTX = 4;  // one force flag per quad (Lattice::ftx)
    int k = 0;
    bool gave_up = false;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++k) {
        const int b = k & 1;
        const unsigned parity = (unsigned)((k >> 1) & 1);
        const bool ok = mbar_wait_bounded(&bar[b], parity, wait_ns);
        if (__syncthreads_or(!ok)) {
            gave_up = true;
            break;
        }
        if (threadIdx.x == 0) pending[b] = 0;
        const int row_raw = t * TR + lr;
        const bool active = row_raw < nrows;
        const int row = active ? row_raw : nrows - 1;  // inactive lanes still join the exchanges
        const int y = row % ny, z = row / ny;
        const int cell0 = x0 + NX * row;
        const int fidx = row * (NX / FTX) + x0 / FTX;
        const bool flag_ok = IBLBM_OK(fidx, 1, (long long)nrows * (NX / FTX));
        const bool has_old = flag_ok && flag_old[fidx] != 0;
        const bool has_cur = flag_ok && flag_cur[fidx] != 0;
        if (has_old && active && IBLBM_OK(cell0, 4, ncell)) {
#pragma unroll
            for (int q = 0; q < 4; ++q) fold[cell0 + q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (has_old && active) flag_old[fidx] = 0;
        // this thread's quad from the staged tile (an inactive lane reads row 0 of the tile)
        const S *tile = stage + (size_t)b * 19 * TILE + (active ? lr : 0) * NX + x0;
        float2 g[19][2];
#pragma unroll
        for (int i = 0; i < 19; ++i) QuadSmem<S>::load(tile + (size_t)i * TILE, g[i][0], g[i][1]);
        collide_quad<S, LR, false, LIN>(QuadRegs{g}, DirStride<S>{dst}, fcur, has_cur, active, row, y, z,
                                        x0, cell0, lane, warp, ny, nz, ncell, omega, u_wall, status, nullptr, edge);
        __syncthreads();  // buffer b is read: it may be refilled
        if (threadIdx.x == 0 && t + 2 * (int)gridDim.x < n_tiles) {
            fence_async_smem();
            issue(t + 2 * gridDim.x, b);
            pending[b] = 1;
        }
    }
    if (gave_up && threadIdx.x == 0) {
        set_status(status, kStatusTimeout);
        // no copy may still write into the block's shared memory when it leaves
        for (int b = 0; b < 2; ++b) {
            const int kb = (k & 1) == b ? k : k + 1;  // next use of buffer b
            if (pending[b]) mbar_wait_bounded(&bar[b], (unsigned)((kb >> 1) & 1), 2000000000ull);
        }
    }
}

// ---- two cells per thread (rows of even length, float arithmetic) ------------------
// Cells (x, x + 1), x even, of a row of even length: one 8-byte (float) or
// 4-byte (binary16) load per direction, arithmetic on the pair with the
// packed FP32 instructions, the directions with c_x = 0 and the wall
// bounce-back stored as pairs, the shifted directions cell by cell.  The
// arithmetic is collide_cell's (opposite pairs), in physical units.
template <typename S>
struct Pair;
template <>
struct Pair<float> {
    static __device__ __forceinline__ float2 load(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
    static __device__ __forceinline__ void store(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
    static __device__ __forceinline__ void store1(float *p, float v) { *p = v; }
};
template <>
struct Pair<__half> {
    static __device__ __forceinline__ float2 load(const __half *p) {
        const float2 f = __half22float2(__ldg(reinterpret_cast<const __half2 *>(p)));
        return make_float2(f.x * kHalfInvScale, f.y * kHalfInvScale);
    }
    static __device__ __forceinline__ void store(__half *p, float2 v) {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.x * kHalfScale, v.y * kHalfScale);
    }
    static __device__ __forceinline__ void store1(__half *p, float v) { *p = __float2half_rn(v * kHalfScale); }
};

template <typename S, bool LIN>
__device__ __forceinline__ void collide_pair(const S *__restrict__ src, S *__restrict__ dst,
                                             const float4 *__restrict__ fcur, bool has_cur, int x, int y,
                                             int z, int nx, int ny, int nz, long long ncell, float omega,
                                             float u_wall, int *status) {
    const long long cell = x + (long long)nx * (y + (long long)ny * z);
    if (!IBLBM_OK(cell, 2, ncell)) return;
    float2 g[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) g[i] = Pair<S>::load(src + i * ncell + cell);
    float2 d = make_float2(0.f, 0.f), jx = d, jy = d, jz = d;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        d = add2(d, g[i]);
        if (q_cx(i)) jx = q_cx(i) > 0 ? add2(jx, g[i]) : sub2(jx, g[i]);
        if (q_cy(i)) jy = q_cy(i) > 0 ? add2(jy, g[i]) : sub2(jy, g[i]);
        if (q_cz(i)) jz = q_cz(i) > 0 ? add2(jz, g[i]) : sub2(jz, g[i]);
    }
    float fv[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    if (has_cur) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float4 f = fcur[cell + e];
            fv[e][0] = f.x; fv[e][1] = f.y; fv[e][2] = f.z;
        }
    }
    float ux[2], uy[2], uz[2], rh[2], ac[2], ufm[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float de = e ? d.y : d.x;
        const float rho = 1.f + de;
        if (!(rho > 0.5f && rho < 2.f)) set_status(status, kStatusUnstable);
        const float inv = 1.f / rho;
        ux[e] = ((e ? jx.y : jx.x) + 0.5f * fv[e][0]) * inv;
        uy[e] = ((e ? jy.y : jy.x) + 0.5f * fv[e][1]) * inv;
        uz[e] = ((e ? jz.y : jz.x) + 0.5f * fv[e][2]) * inv;
        rh[e] = rho;
        ac[e] = LIN ? de : de - 1.5f * rho * (ux[e] * ux[e] + uy[e] * uy[e] + uz[e] * uz[e]);
        ufm[e] = -3.f * (ux[e] * fv[e][0] + uy[e] * fv[e][1] + uz[e] * fv[e][2]);
    }
    const float2 Ux = make_float2(ux[0], ux[1]), Uy = make_float2(uy[0], uy[1]), Uz = make_float2(uz[0], uz[1]);
    const float2 R = make_float2(rh[0], rh[1]), A = make_float2(ac[0], ac[1]), Ufm = make_float2(ufm[0], ufm[1]);
    const float2 Fx = make_float2(fv[0][0], fv[1][0]), Fy = make_float2(fv[0][1], fv[1][1]);
    const float2 Fz = make_float2(fv[0][2], fv[1][2]);
    const float guo = 1.f - 0.5f * omega;
    const float2 keep2 = make_float2(1.f - omega, 1.f - omega);

    // push offsets (periodic in x and y): cell x never wraps to the right and
    // cell x + 1 never to the left
    const long long sz = (long long)nx * ny;
    const long long dyp = (y + 1 == ny) ? -(long long)(ny - 1) * nx : (long long)nx;
    const long long dym = (y == 0) ? (long long)(ny - 1) * nx : -(long long)nx;
    const int dxm0 = (x == 0) ? nx - 1 : -1, dxp1 = (x + 2 == nx) ? 1 - nx : 1;
    auto emit = [&](const int i, const float2 post) {
        const int cx = q_cx(i), cy = q_cy(i), cz = q_cz(i);
        if ((cz > 0 && z + 1 == nz) || (cz < 0 && z == 0)) {
            const float uw = (cz > 0) ? u_wall : -u_wall;
            const float wall = (cx == 0) ? 0.f : 6.f * q_w<float>(i) * (cx > 0 ? uw : -uw);
            Pair<S>::store(dst + q_opp(i) * ncell + cell, make_float2(post.x - wall, post.y - wall));
        } else {
            const long long o = cell + (cy > 0 ? dyp : (cy < 0 ? dym : 0)) + cz * sz;
            S *b = dst + i * ncell + o;
            if (cx == 0) {
                if (IBLBM_OK(o, 2, ncell)) Pair<S>::store(b, post);
            } else if (cx > 0) {
                if (IBLBM_OK(o + 1, 1, ncell)) Pair<S>::store1(b + 1, post.x);
                if (IBLBM_OK(o + 1 + dxp1, 1, ncell)) Pair<S>::store1(b + 1 + dxp1, post.y);
            } else {
                if (IBLBM_OK(o + dxm0, 1, ncell)) Pair<S>::store1(b + dxm0, post.x);
                if (IBLBM_OK(o, 1, ncell)) Pair<S>::store1(b, post.y);
            }
        }
    };
    {
        const float w = q_w<float>(0);
        float2 post = fma2(make_float2(omega * w, omega * w), A, mul2(keep2, g[0]));
        if (has_cur) post = fma2(make_float2(guo * w, guo * w), Ufm, post);
        emit(0, post);
    }
#pragma unroll
    for (int j = 1; j < 19; j += 2) {
        const int ip = (q_cx(j) > 0 || (q_cx(j) == 0 && (q_cy(j) > 0 || (q_cy(j) == 0 && q_cz(j) > 0))))
                           ? j : q_opp(j);
        const int im = q_opp(ip);
        const int cx = q_cx(ip), cy = q_cy(ip), cz = q_cz(ip);
        const float w = q_w<float>(ip);
        const float2 omw = make_float2(omega * w, omega * w), gw = make_float2(guo * w, guo * w);
        float2 cu = cx ? Ux : (cy ? Uy : Uz);
        if (cx && cy) cu = cy > 0 ? add2(cu, Uy) : sub2(cu, Uy);
        if ((cx || cy) && cz) cu = cz > 0 ? add2(cu, Uz) : sub2(cu, Uz);
        const float2 r = mul2(R, cu);
        const float2 e = LIN ? A : fma2(mul2(r, make_float2(4.5f, 4.5f)), cu, A);
        float2 postp = fma2(omw, fma2(r, make_float2(3.f, 3.f), e), mul2(keep2, g[ip]));
        float2 postm = fma2(omw, fma2(r, make_float2(-3.f, -3.f), e), mul2(keep2, g[im]));
        if (has_cur) {
            float2 cf = cx ? Fx : (cy ? Fy : Fz);
            if (cx && cy) cf = cy > 0 ? add2(cf, Fy) : sub2(cf, Fy);
            if ((cx || cy) && cz) cf = cz > 0 ? add2(cf, Fz) : sub2(cf, Fz);
            const float2 base = fma2(mul2(cu, cf), make_float2(9.f, 9.f), Ufm);
            postp = fma2(gw, fma2(cf, make_float2(3.f, 3.f), base), postp);
            postm = fma2(gw, fma2(cf, make_float2(-3.f, -3.f), base), postm);
        }
        emit(ip, postp);
        emit(im, postm);
    }
}

// k_collide_stream for rows of even length: a 32 x 8 x 1 tile per block of
// 16 x 8 threads, two cells per thread.
template <typename S, bool LIN>
__global__ void __launch_bounds__(kTileX / 2 * kTileY)
    k_collide_pair(const S *__restrict__ src, S *__restrict__ dst, const float4 *__restrict__ fcur,
                   const uint8_t *__restrict__ flag_cur, float4 *__restrict__ fold, uint8_t *__restrict__ flag_old,
                   int nx, int ny, int nz, int ntx, int nty, long long ncell, float omega, float u_wall,
                   int *status) {
    prior_grid_wait();
    allow_dependents();
    const int x = blockIdx.x * kTileX + 2 * (int)threadIdx.x;
    const int y = blockIdx.y * kTileY + (int)threadIdx.y;
    const int z = blockIdx.z;
    const long long tile = ((long long)z * nty + blockIdx.y) * ntx + blockIdx.x;
    const bool inside = (x < nx) && (y < ny);  // nx even: x + 1 < nx as well
    const long long cell = x + (long long)nx * (y + (long long)ny * z);
    const bool has_old = flag_old[tile] != 0;
    const bool has_cur = flag_cur[tile] != 0;
    if (has_old) {
        if (inside) {
            fold[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
            fold[cell + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) flag_old[tile] = 0;
    }
    if (!inside) return;
    collide_pair<S, LIN>(src, dst, fcur, has_cur, x, y, z, nx, ny, nz, ncell, omega, u_wall, status);
}

// k_collide_batch for runs whose rows all have even length: 128 threads per
// (run, tile) item, two cells per thread.
template <typename S, bool LIN>
__global__ void __launch_bounds__(128)
    k_collide_pair_batch(const S *__restrict__ src, S *__restrict__ dst, const float4 *__restrict__ fcur,
                         const uint8_t *__restrict__ flag_cur, float4 *__restrict__ fold,
                         uint8_t *__restrict__ flag_old, const RunDesc *__restrict__ runs,
                         const int2 *__restrict__ items, int n_items, int *status) {
    prior_grid_wait();
    allow_dependents();
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int2 w = items[it];
        const RunDesc R = runs[w.x];
        const int per_z = R.ntx * R.nty;
        const int z = w.y / per_z, rem = w.y - z * per_z;
        const int tyi = rem / R.ntx, txi = rem - tyi * R.ntx;
        const int hx = R.tx >> 1;  // pairs per tile row (tile sides are powers of two)
        const int x = txi * R.tx + 2 * ((int)threadIdx.x & (hx - 1));
        const int y = tyi * R.ty + ((int)threadIdx.x >> (__ffs(hx) - 1));
        const bool inside = x < R.nx && y < R.ny;
        const long long tile = R.tile_off + w.y;
        const bool has_old = flag_old[tile] != 0;
        const bool has_cur = flag_cur[tile] != 0;
        if (has_old) {
            if (inside) {
                const long long c = R.cell_off + x + (long long)R.nx * (y + (long long)R.ny * z);
                fold[c] = make_float4(0.f, 0.f, 0.f, 0.f);
                fold[c + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();
            if (threadIdx.x == 0) flag_old[tile] = 0;
        }
        if (inside)
            collide_pair<S, LIN>(src + 19 * R.cell_off, dst + 19 * R.cell_off, fcur + R.cell_off, has_cur, x, y,
                                 z, R.nx, R.ny, R.nz, R.ncell, (float)R.omega, (float)R.u_wall, status);
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

// Sets *bad when any of the n uploaded values is not finite.
__global__ void k_flag_nonfinite(const double *in, long long n, int *bad) {
    bool any = false;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        any |= !isfinite(in[k]);
    if (__syncthreads_or(any) && threadIdx.x == 0) *bad = 1;
}

// Converts uploaded FP64 populations to the storage format, unless the check
// before it found a non-finite value (the lattice then stays as it was).
template <typename S, typename T>
__global__ void k_f64_to_pop(const double *in, long long ncell, S *pop, const int *bad) {
    if (*bad) return;
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

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || n < 1) {
            cudaGetLastError();
            n = 152;
        }
    }
    return n;
}

// Threads per block of the staged kernel: a tile of THREADS * 4 cells is
// 19 * 1024 * 2 = 38 912 bytes per buffer in half storage (256 threads) and
// 19 * 512 * 4 = 38 912 bytes in float storage (128 threads); two buffers per
// block and two blocks per SM, so that one block computes while the other's
// copies arrive.
template <typename S>
constexpr int staged_threads() { return sizeof(S) == 2 ? 256 : 128; }

bool collide_staging_supported(int prec, const Lattice &L) {
    if (prec == kF64 || !L.lanes_row) return false;
    const int nx = 4 * L.lanes_row;
    const int threads = prec == kF32 ? staged_threads<float>() : staged_threads<__half>();
    return (nx * (prec == kF32 ? 4 : 2)) % 16 == 0 && nx <= 4 * threads;
}


template <typename S, int LR, bool LIN>
static void collide_staged(const Lattice &L, const CollideArgs &a, cudaStream_t s, bool ov) {
    constexpr int T = staged_threads<S>();
    constexpr int NX = 4 * LR;
    constexpr int TR = T * 4 / NX;
    const size_t smem = 2 * 19 * (size_t)T * 4 * sizeof(S);
    auto kern = k_collide_stream_tma<S, LR, LIN, T>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int nrows = L.ny * L.nz;
    const int n_tiles = (nrows + TR - 1) / TR;
    const int grid = std::min(n_tiles, 2 * sm_count());
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t c = {};
    c.gridDim = dim3(grid);
    c.blockDim = dim3(T);
    c.dynamicSmemBytes = smem;
    c.stream = s;
    c.attrs = at;
    c.numAttrs = ov ? 1 : 0;
    cudaLaunchKernelEx(&c, kern, (const S *)a.src, (S *)a.dst, (const float4 *)a.fcur, a.flag_cur,
                       (float4 *)a.fold, a.flag_old, L.ny, L.nz, (int)L.ncell, (float)(1.0 / a.tau),
                       (float)a.u_wall, a.status, n_tiles, a.wait_ns);
}

template <typename S, int LR>
static void collide_x4(const Lattice &L, const CollideArgs &a, cudaStream_t s, bool ov) {
    using Sh = X4Shape<S, LR>;
    constexpr int rpb = rows_per_block<LR, Sh::kWarps>();
    constexpr unsigned threads = 32 * Sh::kWarps;
    const auto sp = make_dirs<typename Sh::Src>((const S *)a.src, (int)L.ncell);
    const auto dp = make_dirs<typename Sh::Dst>((S *)a.dst, (int)L.ncell);
    const int nrows = L.ny * L.nz;
    if constexpr ((4 * LR * sizeof(S)) % 16 == 0 && LR <= staged_threads<S>()) {
        if (a.staged && !a.moments) {
            if (a.eq_order == 1) collide_staged<S, LR, true>(L, a, s, ov);
            else collide_staged<S, LR, false>(L, a, s, ov);
            return;
        }
    }
    const unsigned nb = (unsigned)((nrows + rpb - 1) / rpb);
    // the moments are kept only by the adjoint's recomputation, which runs
    // with the full equilibrium
    if (a.moments)
        launch_maybe_overlapped(k_collide_stream_x4<S, LR, true>, dim3(nb), dim3(threads), s, ov,
            sp, dp, (const float4 *)a.fcur, a.flag_cur, (float4 *)a.fold,
            a.flag_old, L.ny, L.nz, (int)L.ncell, (float)(1.0 / a.tau), (float)a.u_wall, a.status,
            (float4 *)a.moments);
    else if (a.eq_order == 1)
        launch_maybe_overlapped(k_collide_stream_x4<S, LR, false, true>, dim3(nb), dim3(threads), s, ov,
            sp, dp, (const float4 *)a.fcur, a.flag_cur, (float4 *)a.fold,
            a.flag_old, L.ny, L.nz, (int)L.ncell, (float)(1.0 / a.tau), (float)a.u_wall, a.status,
            nullptr);
    else
        launch_maybe_overlapped(k_collide_stream_x4<S, LR, false>, dim3(nb), dim3(threads), s, ov,
            sp, dp, (const float4 *)a.fcur, a.flag_cur, (float4 *)a.fold,
            a.flag_old, L.ny, L.nz, (int)L.ncell, (float)(1.0 / a.tau), (float)a.u_wall, a.status,
            nullptr);
}

template <typename S>
static bool collide_vec(const Lattice &L, const CollideArgs &a, cudaStream_t s, bool ov) {
    switch (L.lanes_row) {
        case 1: collide_x4<S, 1>(L, a, s, ov); return true;
        case 2: collide_x4<S, 2>(L, a, s, ov); return true;
        case 4: collide_x4<S, 4>(L, a, s, ov); return true;
        case 8: collide_x4<S, 8>(L, a, s, ov); return true;
        case 16: collide_x4<S, 16>(L, a, s, ov); return true;
        case 32: collide_x4<S, 32>(L, a, s, ov); return true;
        case 64: collide_x4<S, 64>(L, a, s, ov); return true;
        case 128: collide_x4<S, 128>(L, a, s, ov); return true;
        case 256: collide_x4<S, 256>(L, a, s, ov); return true;
        default: return false;
    }
}

template <typename S, typename T>
static void collide_impl(const Lattice &L, const CollideArgs &a, cudaStream_t s, bool ov) {
    using V4 = typename Vec4<T>::type;
    dim3 grid(L.ntx, L.nty, L.nz), block(kTileX, kTileY);
    if constexpr (!std::is_same<T, double>::value) {
        if (L.nx % 2 == 0 && !a.moments) {  // the adjoint's recomputation keeps the one-cell kernel
            auto kern = a.eq_order == 1 ? k_collide_pair<S, true> : k_collide_pair<S, false>;
            launch_maybe_overlapped(kern, grid, dim3(kTileX / 2, kTileY), s, ov, (const S *)a.src, (S *)a.dst,
                                    (const float4 *)a.fcur, a.flag_cur, (float4 *)a.fold, a.flag_old, L.nx, L.ny,
                                    L.nz, L.ntx, L.nty, L.ncell, (float)(1.0 / a.tau), (float)a.u_wall, a.status);
            return;
        }
    }
    auto kern = a.eq_order == 1 ? k_collide_stream<S, T, true> : k_collide_stream<S, T, false>;
    launch_maybe_overlapped(kern, grid, block, s, ov,
        (const S *)a.src, (S *)a.dst, (const V4 *)a.fcur, a.flag_cur, (V4 *)a.fold, a.flag_old,
        L.nx, L.ny, L.nz, L.ntx, L.nty, L.ncell, (T)(1.0 / a.tau), (T)a.u_wall, a.status,
        (V4 *)a.moments);
}

void launch_collide_stream(int prec, const Lattice &L, const CollideArgs &a, cudaStream_t s, bool overlap) {
    if (prec == kF64) collide_impl<double, double>(L, a, s, overlap);
    else if (prec == kF32) {
        if (!collide_vec<float>(L, a, s, overlap)) collide_impl<float, float>(L, a, s, overlap);
    } else {
        if (!collide_vec<__half>(L, a, s, overlap)) collide_impl<__half, float>(L, a, s, overlap);
    }
}

template <typename S, typename T>
static void collide_batch_impl(const BatchArgs &b, const CollideArgs &a, cudaStream_t s, bool ov) {
    using V4 = typename Vec4<T>::type;
    if constexpr (!std::is_same<T, double>::value) {
        if (b.pairs) {
            auto kern = a.eq_order == 1 ? k_collide_pair_batch<S, true> : k_collide_pair_batch<S, false>;
            launch_maybe_overlapped(kern, dim3(b.grid), dim3(128), s, ov, (const S *)a.src, (S *)a.dst,
                                    (const float4 *)a.fcur, a.flag_cur, (float4 *)a.fold, a.flag_old, b.runs, b.items,
                                    b.n_items, a.status);
            return;
        }
    }
    auto kern = a.eq_order == 1 ? k_collide_batch<S, T, true> : k_collide_batch<S, T, false>;
    launch_maybe_overlapped(kern, dim3(b.grid), dim3(256), s, ov,
        (const S *)a.src, (S *)a.dst, (const V4 *)a.fcur, a.flag_cur, (V4 *)a.fold, a.flag_old,
        b.runs, b.items, b.n_items, a.status);
}

void launch_collide_batch(int prec, const BatchArgs &b, const CollideArgs &a, cudaStream_t s, bool overlap) {
    if (b.n_items == 0) return;
    if (prec == kF64) collide_batch_impl<double, double>(b, a, s, overlap);
    else if (prec == kF32) collide_batch_impl<float, float>(b, a, s, overlap);
    else collide_batch_impl<__half, float>(b, a, s, overlap);
}

// ---- x-slab boundary planes -------------------------------------------------------------
// A slab streams with its own periodic wrap in x, so after its collide the
// populations with c_x = +1 that crossed its right edge sit in its column
// x = 0, and those with c_x = -1 that crossed its left edge in its column
// x = nx - 1.  Packing these ten columns and writing each slab's from its
// neighbour's (left neighbour for c_x = +1, right for c_x = -1) turns the
// wraps into the global periodic streaming of Eq. (lbequation).  Entries of a
// column that the moving-wall bounce-back filled (the rows whose stream
// source lies beyond a wall) are the cell's own and are kept.
__host__ __device__ constexpr int plane_dir(int k) {
    // c_x = +1: 1, 7, 10, 12, 13; c_x = -1: 2, 8, 9, 11, 14 (Fig. d3q19)
    constexpr int t[10] = {1, 7, 10, 12, 13, 2, 8, 9, 11, 14};
    return t[k];
}

template <typename E>
__global__ void k_plane_pack(const E *__restrict__ pop, int nx, int ny, int nz, long long ncell,
                             E *__restrict__ out) {
    const long long per = (long long)ny * nz;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= 10 * per) return;
    const int k = (int)(idx / per);
    const long long yz = idx % per;
    const int xcol = k < 5 ? 0 : nx - 1;
    out[idx] = pop[plane_dir(k) * ncell + yz * nx + xcol];
}

template <typename E>
__global__ void k_plane_unpack(E *__restrict__ pop, int nx, int ny, int nz, long long ncell,
                               const E *__restrict__ left, const E *__restrict__ right) {
    const long long per = (long long)ny * nz;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= 10 * per) return;
    const int k = (int)(idx / per);
    const long long yz = idx % per;
    const int z = (int)(yz / ny);
    const int i = plane_dir(k), cz = q_cz(i);
    if (z - cz < 0 || z - cz >= nz) return;  // filled by the wall's bounce-back
    const int xcol = k < 5 ? 0 : nx - 1;
    pop[i * ncell + yz * nx + xcol] = (k < 5 ? left : right)[idx];
}

void launch_plane_pack(int prec, const Lattice &L, const void *pop, void *out, cudaStream_t s) {
    const long long n = 10LL * L.ny * L.nz;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (prec == kF64) k_plane_pack<unsigned long long><<<nb, 256, 0, s>>>((const unsigned long long *)pop, L.nx, L.ny, L.nz, L.ncell, (unsigned long long *)out);
    else if (prec == kF32) k_plane_pack<unsigned><<<nb, 256, 0, s>>>((const unsigned *)pop, L.nx, L.ny, L.nz, L.ncell, (unsigned *)out);
    else k_plane_pack<unsigned short><<<nb, 256, 0, s>>>((const unsigned short *)pop, L.nx, L.ny, L.nz, L.ncell, (unsigned short *)out);
}

void launch_plane_unpack(int prec, const Lattice &L, void *pop, const void *left, const void *right,
                         cudaStream_t s) {
    const long long n = 10LL * L.ny * L.nz;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (prec == kF64) k_plane_unpack<unsigned long long><<<nb, 256, 0, s>>>((unsigned long long *)pop, L.nx, L.ny, L.nz, L.ncell, (const unsigned long long *)left, (const unsigned long long *)right);
    else if (prec == kF32) k_plane_unpack<unsigned><<<nb, 256, 0, s>>>((unsigned *)pop, L.nx, L.ny, L.nz, L.ncell, (const unsigned *)left, (const unsigned *)right);
    else k_plane_unpack<unsigned short><<<nb, 256, 0, s>>>((unsigned short *)pop, L.nx, L.ny, L.nz, L.ncell, (const unsigned short *)left, (const unsigned short *)right);
}

// ---- checkpoint section checksum ------------------------------------------------------
// Sum modulo 2^64 of mix(w_k + k * 0x9e3779b97f4a7c15) over the 64-bit words
// w_k of a byte range (the last word zero-padded), mix being the SplitMix64
// finaliser (a bijection).  Addition modulo 2^64 does not depend on order, so
// the device's atomic sum and the host loop of capi.cpp give the same value,
// and a change of any single byte changes exactly one term.
__device__ __forceinline__ unsigned long long ck_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_checksum(const unsigned char *__restrict__ p, unsigned long long n_bytes,
                           unsigned long long *__restrict__ out) {
    const unsigned long long n_words = (n_bytes + 7) / 8;
    unsigned long long acc = 0;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n_words;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long w = 0;
        if (8 * k + 8 <= n_bytes) {
            w = ((const unsigned long long *)p)[k];  // sections start 256-byte aligned
        } else {
            for (unsigned long long b = 8 * k; b < n_bytes; ++b) w |= (unsigned long long)p[b] << (8 * (b - 8 * k));
        }
        acc += ck_mix(w + k * 0x9e3779b97f4a7c15ull);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

void launch_checksum(const void *p, size_t n_bytes, unsigned long long *out, cudaStream_t s) {
    const size_t words = (n_bytes + 7) / 8;
    const unsigned blocks = (unsigned)std::min<size_t>((words + 255) / 256, 152 * 8);
    if (blocks) k_checksum<<<blocks, 256, 0, s>>>((const unsigned char *)p, n_bytes, out);
}

const char *collide_kernel_name(int prec, const Lattice &L, bool staged) {
    static const char *const tma_f32[9] = {
        "k_collide_stream_tma<float,1>",  "k_collide_stream_tma<float,2>",  "k_collide_stream_tma<float,4>",
        "k_collide_stream_tma<float,8>",  "k_collide_stream_tma<float,16>", "k_collide_stream_tma<float,32>",
        "k_collide_stream_tma<float,64>", "k_collide_stream_tma<float,128>", "k_collide_stream_tma<float,256>"};
    static const char *const tma_f16[9] = {
        "k_collide_stream_tma<__half,1>",  "k_collide_stream_tma<__half,2>",  "k_collide_stream_tma<__half,4>",
        "k_collide_stream_tma<__half,8>",  "k_collide_stream_tma<__half,16>", "k_collide_stream_tma<__half,32>",
        "k_collide_stream_tma<__half,64>", "k_collide_stream_tma<__half,128>", "k_collide_stream_tma<__half,256>"};
    if (staged && collide_staging_supported(prec, L)) {
        int k = 0;
        while ((1 << k) < L.lanes_row) ++k;
        return prec == kF32 ? tma_f32[k] : tma_f16[k];
    }
    return collide_kernel_name(prec, L);
}

const char *collide_kernel_name(int prec, const Lattice &L) {
    static const char *const x4_f32[9] = {
        "k_collide_stream_x4<float,1>",  "k_collide_stream_x4<float,2>",  "k_collide_stream_x4<float,4>",
        "k_collide_stream_x4<float,8>",  "k_collide_stream_x4<float,16>", "k_collide_stream_x4<float,32>",
        "k_collide_stream_x4<float,64>", "k_collide_stream_x4<float,128>", "k_collide_stream_x4<float,256>"};
    static const char *const x4_f16[9] = {
        "k_collide_stream_x4<__half,1>",  "k_collide_stream_x4<__half,2>",  "k_collide_stream_x4<__half,4>",
        "k_collide_stream_x4<__half,8>",  "k_collide_stream_x4<__half,16>", "k_collide_stream_x4<__half,32>",
        "k_collide_stream_x4<__half,64>", "k_collide_stream_x4<__half,128>", "k_collide_stream_x4<__half,256>"};
    if (prec == kF64) return "k_collide_stream<double,double>";
    if (L.lanes_row) {
        int k = 0;
        while ((1 << k) < L.lanes_row) ++k;
        return prec == kF32 ? x4_f32[k] : x4_f16[k];
    }
    if (L.nx % 2 == 0) return prec == kF32 ? "k_collide_pair<float>" : "k_collide_pair<__half>";
    return prec == kF32 ? "k_collide_stream<float,float>" : "k_collide_stream<__half,float>";
}

const char *collide_batch_kernel_name(int prec, bool pairs) {
    if (prec == kF64) return "k_collide_batch<double,double>";
    if (pairs) return prec == kF32 ? "k_collide_pair_batch<float>" : "k_collide_pair_batch<__half>";
    return prec == kF32 ? "k_collide_batch<float,float>" : "k_collide_batch<__half,float>";
}

int collide_batch_blocks_per_sm(int prec, bool pairs) {
    int n = 0;
    cudaError_t e;
    if (pairs && prec == kF32)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_collide_pair_batch<float, false>, 128, 0);
    else if (pairs && prec == kF16)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_collide_pair_batch<__half, false>, 128, 0);
    else if (prec == kF64)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_collide_batch<double, double, false>, 256, 0);
    else if (prec == kF32)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_collide_batch<float, float, false>, 256, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_collide_batch<__half, float, false>, 256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
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

void launch_f64_to_pop(int prec, const Lattice &L, const double *in, void *pop, int *bad, cudaStream_t s) {
    const long long n = 19 * L.ncell;
    unsigned nc = (unsigned)std::min<long long>(blocks_for(n, 256), 8LL * sm_count());
    k_flag_nonfinite<<<nc, 256, 0, s>>>(in, n, bad);
    unsigned nb = blocks_for(n, 256);
    if (prec == kF64) k_f64_to_pop<double, double><<<nb, 256, 0, s>>>(in, L.ncell, (double *)pop, bad);
    else if (prec == kF32) k_f64_to_pop<float, float><<<nb, 256, 0, s>>>(in, L.ncell, (float *)pop, bad);
    else k_f64_to_pop<__half, float><<<nb, 256, 0, s>>>(in, L.ncell, (__half *)pop, bad);
}

void launch_force_to_f64(int prec, const Lattice &L, const void *force, double *out, cudaStream_t s) {
    unsigned nb = blocks_for(L.ncell, 256);
    if (prec == kF64) k_force_to_f64<double><<<nb, 256, 0, s>>>((const dvec4 *)force, L.ncell, out);
    else k_force_to_f64<float><<<nb, 256, 0, s>>>((const float4 *)force, L.ncell, out);
}

IBLBM_BOUNDS_ACCESSOR(bounds_faults_lbm)

}  // namespace iblbm
