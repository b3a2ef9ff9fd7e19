// ib_common.cuh -- node-position views and warp helpers shared by the
// immersed-boundary kernels (ib.cu) and their adjoints (adjoint.cu).
#pragma once

#include "device_common.cuh"

namespace iblbm {

template <typename T>
struct PosView;

// FP64 build: positions as double 4-vectors.
template <>
struct PosView<double> {
    dvec4 *x;
    __device__ __forceinline__ void edges(int a, int b, int c, double u[3], double v[3]) const {
        dvec4 pa = x[a], pb = x[b], pc = x[c];
        u[0] = pb.x - pa.x; u[1] = pb.y - pa.y; u[2] = pb.z - pa.z;
        v[0] = pc.x - pa.x; v[1] = pc.y - pa.y; v[2] = pc.z - pa.z;
    }
    // edges u, v and the Gram deviations d = g - G0 (G0 in c1.y, c1.z, c1.w)
    __device__ __forceinline__ void edge_gram(int a, int b, int c, const dvec4 &c1, const dvec4 &c2,
                                              double u[3], double v[3], double d[3]) const {
        edges(a, b, c, u, v);
        d[0] = (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) - c1.y;
        d[1] = (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) - c1.z;
        d[2] = (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) - c1.w;
    }
    __device__ __forceinline__ void approx(int n, double p[3]) const {
        dvec4 q = x[n];
        p[0] = q.x; p[1] = q.y; p[2] = q.z;
    }
    // lattice node minus node position
    __device__ __forceinline__ void rel(const double p[3], int X, int Y, int Z, double d[3]) const {
        d[0] = X - p[0]; d[1] = Y - p[1]; d[2] = Z - p[2];
    }
    // x_n += (dx, dy, dz); the new position also goes to `copy` if it has storage
    __device__ __forceinline__ void advance(int n, double dx, double dy, double dz,
                                            const PosView<double> &copy) const {
        dvec4 q = x[n];
        q.x += dx; q.y += dy; q.z += dz;
        x[n] = q;
        if (copy.x) copy.x[n] = q;
    }
};

// Float builds: positions as hi + lo float pairs.
template <>
struct PosView<float> {
    float4 *hi;
    float4 *lo;
    __device__ __forceinline__ void edges(int a, int b, int c, float u[3], float v[3]) const {
        float4 ha = hi[a], hb = hi[b], hc = hi[c];
        float4 la = lo[a], lb = lo[b], lc = lo[c];
        u[0] = (hb.x - ha.x) + (lb.x - la.x);
        u[1] = (hb.y - ha.y) + (lb.y - la.y);
        u[2] = (hb.z - ha.z) + (lb.z - la.z);
        v[0] = (hc.x - ha.x) + (lc.x - la.x);
        v[1] = (hc.y - ha.y) + (lc.y - la.y);
        v[2] = (hc.z - ha.z) + (lc.z - la.z);
    }
    // Edges as double-float pairs, Gram entries in double-float, deviations
    // from the reference Gram entries (hi in c1.y..w, lo in c2.x..z) in float.
    __device__ __forceinline__ void edge_gram(int a, int b, int c, const float4 &c1, const float4 &c2,
                                              float u[3], float v[3], float d[3]) const {
        float4 ha = hi[a], hb = hi[b], hc = hi[c];
        float4 la = lo[a], lb = lo[b], lc = lo[c];
        DF U[3], V[3];
        U[0] = df_two_sum(hb.x - ha.x, lb.x - la.x);
        U[1] = df_two_sum(hb.y - ha.y, lb.y - la.y);
        U[2] = df_two_sum(hb.z - ha.z, lb.z - la.z);
        V[0] = df_two_sum(hc.x - ha.x, lc.x - la.x);
        V[1] = df_two_sum(hc.y - ha.y, lc.y - la.y);
        V[2] = df_two_sum(hc.z - ha.z, lc.z - la.z);
        DF g11 = df_add(df_add(df_mul(U[0], U[0]), df_mul(U[1], U[1])), df_mul(U[2], U[2]));
        DF g12 = df_add(df_add(df_mul(U[0], V[0]), df_mul(U[1], V[1])), df_mul(U[2], V[2]));
        DF g22 = df_add(df_add(df_mul(V[0], V[0]), df_mul(V[1], V[1])), df_mul(V[2], V[2]));
        d[0] = (g11.h - c1.y) + (g11.l - c2.x);
        d[1] = (g12.h - c1.z) + (g12.l - c2.y);
        d[2] = (g22.h - c1.w) + (g22.l - c2.z);
        for (int k = 0; k < 3; ++k) {
            u[k] = U[k].h;
            v[k] = V[k].h;
        }
    }
    // p holds hi in [0..2] and lo in [3..5]
    __device__ __forceinline__ void approx(int n, float p[6]) const {
        float4 h = hi[n], l = lo[n];
        p[0] = h.x; p[1] = h.y; p[2] = h.z;
        p[3] = l.x; p[4] = l.y; p[5] = l.z;
    }
    __device__ __forceinline__ void rel(const float p[6], int X, int Y, int Z, float d[3]) const {
        d[0] = ((float)X - p[0]) - p[3];
        d[1] = ((float)Y - p[1]) - p[4];
        d[2] = ((float)Z - p[2]) - p[5];
    }
    __device__ __forceinline__ void advance(int n, float dx, float dy, float dz, const PosView<float> &copy) const {
        float4 h = hi[n], l = lo[n];
        two_sum_add(h.x, l.x, dx);
        two_sum_add(h.y, l.y, dy);
        two_sum_add(h.z, l.z, dz);
        hi[n] = h;
        lo[n] = l;
        if (copy.hi) {
            copy.hi[n] = h;
            copy.lo[n] = l;
        }
    }
};

template <typename T>
constexpr int kPosLen = 3;
template <>
constexpr int kPosLen<float> = 6;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic spreading: the force density accumulates in 64-bit fixed
// point (integer additions are associative, so the sum does not depend on
// the order of the atomics), kFixBits fractional bits: 2^-40 (about 1e-12)
// in the float builds, 2^-52 in the FP64 build; a contribution of magnitude
// 2^22 (float) or 2^10 (FP64) or more is refused with kStatusForceRange.
template <typename T>
constexpr int kFixBits = 40;
template <>
constexpr int kFixBits<double> = 52;
__device__ __forceinline__ void add_force_fix(unsigned long long *f, float x, float y, float z, int *status) {
    constexpr float S = 1099511627776.0f;  // 2^40
    const float v[3] = {x * S, y * S, z * S};
    if (!(fabsf(v[0]) < 4.6e18f && fabsf(v[1]) < 4.6e18f && fabsf(v[2]) < 4.6e18f)) {
        set_status(status, kStatusForceRange);
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) atomicAdd(f + k, (unsigned long long)__float2ll_rn(v[k]));
}
__device__ __forceinline__ void add_force_fix(unsigned long long *f, double x, double y, double z, int *status) {
    constexpr double S = 4503599627370496.0;  // 2^52
    const double v[3] = {x * S, y * S, z * S};
    if (!(fabs(v[0]) < 4.6e18 && fabs(v[1]) < 4.6e18 && fabs(v[2]) < 4.6e18)) {
        set_status(status, kStatusForceRange);
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) atomicAdd(f + k, (unsigned long long)__double2ll_rn(v[k]));
}

__device__ __forceinline__ void add_force(float4 *f, float x, float y, float z) {
    atomicAdd(f, make_float4(x, y, z, 0.0f));
}
__device__ __forceinline__ void add_force(dvec4 *f, double x, double y, double z) {
    atomicAdd(&f->x, x);
    atomicAdd(&f->y, y);
    atomicAdd(&f->z, z);
}

}  // namespace iblbm
