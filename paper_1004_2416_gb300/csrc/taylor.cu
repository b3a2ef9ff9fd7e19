// taylor.cu -- double-precision capsule reductions behind the Taylor
// deformation of Sec. III: volume, surface area, centroid and the inertia
// tensor I_ab = 1/5 sum_faces A_i (r_i^2 delta_ab r_g - r_ia r_ib r_ig) n_ig
// about the centroid.
//
// The faces of a capsule are split over several blocks (FP64 arithmetic is
// scarce per SM, so a capsule is spread over many SMs).  Three launches, each
// a fixed-order reduction, so results are bitwise reproducible:
//   1. per block: V = 1/3 sum r.(A n), A = sum |A n|, m = sum (r.(A n)) r with
//      r the face centroid minus the capsule's origin (its reference centre);
//   2. per block: the block first totals the stage-1 partials of its capsule,
//      forms the centroid c = origin + m / (4 V), then sums the inertia terms
//      of its faces about c;
//   3. per capsule: totals of both stages -> {V, A, c, I} in the output.
// Per-block partials live in a scratch array [blocks][16] (stage 1 in
// entries 0..4, stage 2 in entries 8..13).
#include "device_common.cuh"
#include "internal.h"

namespace iblbm {

template <typename T>
struct NodeRead;
template <>
struct NodeRead<double> {
    const dvec4 *x;
    __device__ __forceinline__ void get(int n, double p[3]) const {
        dvec4 q = x[n];
        p[0] = q.x; p[1] = q.y; p[2] = q.z;
    }
};
template <>
struct NodeRead<float> {
    const float4 *hi;
    const float4 *lo;
    __device__ __forceinline__ void get(int n, double p[3]) const {
        float4 h = hi[n], l = lo[n];
        p[0] = (double)h.x + (double)l.x;
        p[1] = (double)h.y + (double)l.y;
        p[2] = (double)h.z + (double)l.z;
    }
};

constexpr int kTB = kTaylorFacesPerBlock;  // threads per block, one face each

// Fixed-order block sum of K doubles per thread; result valid in thread 0.
template <int K>
__device__ __forceinline__ void block_sum(double v[K], double (*sh)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int w = 0; w < kTB / 32; ++w) s += sh[w][k];
            v[k] = s;
        }
    }
}

template <typename R>
__device__ __forceinline__ void face_geom(R nodes, const int4 t, double cen[3], double An[3]) {
    double a[3], b[3], c[3];
    nodes.get(t.x, a);
    nodes.get(t.y, b);
    nodes.get(t.z, c);
    double e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = b[k] - a[k];
        e2[k] = c[k] - a[k];
        cen[k] = (a[k] + b[k] + c[k]) * (1.0 / 3.0);
    }
    An[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
    An[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
    An[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
}

template <typename R>
__global__ void __launch_bounds__(kTB) k_taylor_stage1(R nodes, const int4 *__restrict__ tri, TaylorPlan p) {
    __shared__ double sh[kTB / 32][5];
    const int b = blockIdx.x;
    const int cap = p.blk_cap[b];
    double v[5] = {0, 0, 0, 0, 0};
    if ((int)threadIdx.x < p.blk_nface[b]) {
        const int4 t = tri[p.blk_face0[b] + threadIdx.x];
        double cen[3], An[3];
        face_geom(nodes, t, cen, An);
        double r[3];
        for (int k = 0; k < 3; ++k) r[k] = cen[k] - p.origin[3 * cap + k];
        const double rn = r[0] * An[0] + r[1] * An[1] + r[2] * An[2];
        v[0] = rn * (1.0 / 3.0);
        v[1] = sqrt(An[0] * An[0] + An[1] * An[1] + An[2] * An[2]);
        v[2] = rn * r[0];
        v[3] = rn * r[1];
        v[4] = rn * r[2];
    }
    block_sum<5>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 5; ++k) p.partial[16 * b + k] = v[k];
}

// Totals of K partial entries (from entry `first`) over the blocks of one
// capsule, by one full warp: lane l sums blocks l, l+32, ... in order, then a
// fixed butterfly; every lane returns the same totals.
template <int K>
__device__ __forceinline__ void capsule_totals(const TaylorPlan &p, int cap, int first, double tot[K]) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < K; ++k) tot[k] = 0.0;
    for (int b = p.cap_blk0[cap] + lane; b < p.cap_blk0[cap + 1]; b += 32)
        for (int k = 0; k < K; ++k) tot[k] += p.partial[16 * b + first + k];
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) tot[k] += __shfl_xor_sync(0xffffffffu, tot[k], o);
}

template <typename R>
__global__ void __launch_bounds__(kTB) k_taylor_stage2(R nodes, const int4 *__restrict__ tri, TaylorPlan p) {
    __shared__ double sh[kTB / 32][6];
    __shared__ double cen_sh[3];
    const int b = blockIdx.x;
    const int cap = p.blk_cap[b];
    if (threadIdx.x < 32) {
        double tot[5];
        capsule_totals<5>(p, cap, 0, tot);
        if (threadIdx.x == 0)
            for (int k = 0; k < 3; ++k) cen_sh[k] = p.origin[3 * cap + k] + tot[2 + k] / (4.0 * tot[0]);
    }
    __syncthreads();
    double v[6] = {0, 0, 0, 0, 0, 0};
    if ((int)threadIdx.x < p.blk_nface[b]) {
        const int4 t = tri[p.blk_face0[b] + threadIdx.x];
        double cen[3], An[3];
        face_geom(nodes, t, cen, An);
        double r[3];
        for (int k = 0; k < 3; ++k) r[k] = cen[k] - cen_sh[k];
        const double rn = (r[0] * An[0] + r[1] * An[1] + r[2] * An[2]) * 0.2;
        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        v[0] = (r2 - r[0] * r[0]) * rn;
        v[1] = (r2 - r[1] * r[1]) * rn;
        v[2] = (r2 - r[2] * r[2]) * rn;
        v[3] = -r[0] * r[1] * rn;
        v[4] = -r[0] * r[2] * rn;
        v[5] = -r[1] * r[2] * rn;
    }
    block_sum<6>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) p.partial[16 * b + 8 + k] = v[k];
}

// One block of 32 warps; warp w takes capsules w, w + 32, ...  In recording
// mode the block writes the next ring slot and then advances the counter.
__global__ void __launch_bounds__(1024) k_taylor_stage3(TaylorPlan p, int record) {
    double *base = p.out;
    unsigned long long count = 0;
    if (record) {
        count = *p.ring_count;
        base = p.ring + (size_t)(count % (unsigned long long)p.ring_len) * p.n_caps * 12;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int cap = warp; cap < p.n_caps; cap += blockDim.x >> 5) {
        double tot[5], I[6];
        capsule_totals<5>(p, cap, 0, tot);
        capsule_totals<6>(p, cap, 8, I);
        if (lane == 0) {
            double *o = base + 12 * cap;
            o[0] = tot[0];
            o[1] = tot[1];
            for (int k = 0; k < 3; ++k) o[2 + k] = p.origin[3 * cap + k] + tot[2 + k] / (4.0 * tot[0]);
            for (int k = 0; k < 6; ++k) o[5 + k] = I[k];
            o[11] = 0.0;
        }
    }
    __syncthreads();
    if (record && threadIdx.x == 0) *p.ring_count = count + 1;
}

template <typename R>
static void taylor_impl(R nodes, const MeshDev &m, const TaylorPlan &p, bool record, cudaStream_t s) {
    k_taylor_stage1<R><<<p.total_blocks, kTB, 0, s>>>(nodes, (const int4 *)m.tri, p);
    k_taylor_stage2<R><<<p.total_blocks, kTB, 0, s>>>(nodes, (const int4 *)m.tri, p);
    k_taylor_stage3<<<1, 1024, 0, s>>>(p, record ? 1 : 0);
}

void launch_taylor(int prec, const MeshDev &m, const TaylorPlan &p, bool record, cudaStream_t s) {
    if (p.n_caps == 0 || (record && !p.ring)) return;
    if (prec == kF64)
        taylor_impl(NodeRead<double>{(const dvec4 *)m.x}, m, p, record, s);
    else
        taylor_impl(NodeRead<float>{(const float4 *)m.x, (const float4 *)m.x_lo}, m, p, record, s);
}

}  // namespace iblbm
