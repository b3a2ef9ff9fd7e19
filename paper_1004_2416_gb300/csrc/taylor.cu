// taylor.cu -- double-precision capsule reductions behind the Taylor
// deformation of Sec. III: volume, surface area, centroid and the inertia
// tensor I_ab = 1/5 sum_faces A_i (r_i^2 delta_ab r_g - r_ia r_ib r_ig) n_ig
// about the centroid.
//
// One launch per reduction: one thread-block cluster per capsule (and per
// position snapshot, grid y, so that consecutive records share a launch)
// makes two passes over the capsule's faces, each ending in a fixed-order sum
// over the cluster (block sums exchanged through distributed shared memory),
// so results are bitwise reproducible:
//   1. V = 1/3 sum r.(A n), A = sum |A n|, m = sum (r.(A n)) r with r the face
//      centroid minus the capsule's origin (its reference centre), and the
//      centroid c = origin + m / (4 V);
//   2. the inertia terms of the faces about c.
// In the float builds the per-face terms are formed in float from the
// positions relative to the origin, each thread adds its few faces (about
// four) in float, and the sums over threads, blocks and the cluster are
// carried in double.
//
// The allocation-free entry point at the end keeps a three-launch form whose
// per-block partial sums live in a fixed device array.
#include <cooperative_groups.h>
#include <type_traits>
#include <mutex>
#include <string>

#include "device_common.cuh"
#include "iblbm.h"
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
    // the same view moved to snapshot k of a ring of snapshots of `stride` nodes
    __device__ __forceinline__ NodeRead at(long long k, long long stride) const {
        return NodeRead{x + k * stride};
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
    __device__ __forceinline__ NodeRead at(long long k, long long stride) const {
        return NodeRead{hi + k * stride, lo + k * stride};
    }
};

// A launch reduces n_snap position snapshots at once (grid y): snapshot k
// lives in slot (first + k) of a ring of `slots` snapshots of n_nodes each
// (one snapshot, slot 0, for the current positions).
struct SnapSet {
    int first, slots, n_snap;
    long long stride;
    __device__ __forceinline__ long long slot(int k) const { return (first + k) % slots; }
};

constexpr int kTB = kTaylorThreads;  // threads per block

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

// Terms of one face for the two stages.  FP64 build: double throughout.
// Float builds: node coordinates relative to the capsule origin are formed
// from the hi/lo pairs and the face terms are evaluated in float (relative
// error ~1e-7, well inside the float build's tolerance); only the sums over
// faces and blocks are carried in double.
template <typename R>
struct FaceMath;

template <>
struct FaceMath<NodeRead<double>> {
    static __device__ __forceinline__ void stage1(const NodeRead<double> &nodes, int4 t,
                                                  const double o[3], double v[5]) {
        double cen[3], An[3];
        face_geom(nodes, t, cen, An);
        double r[3];
        for (int k = 0; k < 3; ++k) r[k] = cen[k] - o[k];
        const double rn = r[0] * An[0] + r[1] * An[1] + r[2] * An[2];
        v[0] = rn * (1.0 / 3.0);
        v[1] = sqrt(An[0] * An[0] + An[1] * An[1] + An[2] * An[2]);
        v[2] = rn * r[0];
        v[3] = rn * r[1];
        v[4] = rn * r[2];
    }
    static __device__ __forceinline__ void stage2(const NodeRead<double> &nodes, int4 t,
                                                  const double o[3], const double c[3], double v[6]) {
        double cen[3], An[3];
        face_geom(nodes, t, cen, An);
        double r[3];
        for (int k = 0; k < 3; ++k) r[k] = cen[k] - c[k];
        const double rn = (r[0] * An[0] + r[1] * An[1] + r[2] * An[2]) * 0.2;
        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        v[0] = (r2 - r[0] * r[0]) * rn;
        v[1] = (r2 - r[1] * r[1]) * rn;
        v[2] = (r2 - r[2] * r[2]) * rn;
        v[3] = -r[0] * r[1] * rn;
        v[4] = -r[0] * r[2] * rn;
        v[5] = -r[1] * r[2] * rn;
    }
};

template <>
struct FaceMath<NodeRead<float>> {
    // node n relative to the origin, whose hi/lo split is (oh, ol)
    static __device__ __forceinline__ void rel(const NodeRead<float> &nodes, int n, const float oh[3],
                                               const float ol[3], float r[3]) {
        const float4 h = nodes.hi[n], l = nodes.lo[n];
        r[0] = (h.x - oh[0]) + (l.x - ol[0]);
        r[1] = (h.y - oh[1]) + (l.y - ol[1]);
        r[2] = (h.z - oh[2]) + (l.z - ol[2]);
    }
    // the capsule origin as a float pair (hi, lo): formed once per thread,
    // not per face (double arithmetic is scarce on this GPU)
    static __device__ __forceinline__ void split(const double o[3], float oh[3], float ol[3]) {
        for (int k = 0; k < 3; ++k) {
            oh[k] = (float)o[k];
            ol[k] = (float)(o[k] - (double)oh[k]);
        }
    }
    static __device__ __forceinline__ void geom(const NodeRead<float> &nodes, int4 t, const float oh[3],
                                                const float ol[3], float cen[3], float An[3]) {
        float a[3], b[3], c[3];
        rel(nodes, t.x, oh, ol, a);
        rel(nodes, t.y, oh, ol, b);
        rel(nodes, t.z, oh, ol, c);
        float e1[3], e2[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = b[k] - a[k];
            e2[k] = c[k] - a[k];
            cen[k] = (a[k] + b[k] + c[k]) * (1.0f / 3.0f);
        }
        An[0] = 0.5f * (e1[1] * e2[2] - e1[2] * e2[1]);
        An[1] = 0.5f * (e1[2] * e2[0] - e1[0] * e2[2]);
        An[2] = 0.5f * (e1[0] * e2[1] - e1[1] * e2[0]);
    }
    // the terms in float (a thread adds its few faces in float and the sums
    // over threads and blocks are carried in double), from the face centroid
    // relative to the origin r and the area vector An
    static __device__ __forceinline__ void terms1(const float r[3], const float An[3], float v[5]) {
        const float rn = r[0] * An[0] + r[1] * An[1] + r[2] * An[2];
        v[0] = rn * (1.0f / 3.0f);
        v[1] = sqrtf(An[0] * An[0] + An[1] * An[1] + An[2] * An[2]);
        v[2] = rn * r[0];
        v[3] = rn * r[1];
        v[4] = rn * r[2];
    }
    // co = capsule centroid - origin in float, formed once per thread
    static __device__ __forceinline__ void terms2(const float cen[3], const float An[3], const float co[3],
                                                  float v[6]) {
        float r[3];
        for (int k = 0; k < 3; ++k) r[k] = cen[k] - co[k];
        const float rn = (r[0] * An[0] + r[1] * An[1] + r[2] * An[2]) * 0.2f;
        const float r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        v[0] = (r2 - r[0] * r[0]) * rn;
        v[1] = (r2 - r[1] * r[1]) * rn;
        v[2] = (r2 - r[2] * r[2]) * rn;
        v[3] = -r[0] * r[1] * rn;
        v[4] = -r[0] * r[2] * rn;
        v[5] = -r[1] * r[2] * rn;
    }
};

// Fixed-order sum over the block (blockDim.x a multiple of 32, at most 1024)
// of K doubles per thread: a butterfly within each warp, then the warps' sums
// in warp order by thread 0, which alone holds the result.  `sh` may be reused
// right after a call (it begins with a barrier).
template <int K>
__device__ __forceinline__ void block_sum_any(double v[K], double (*sh)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int k = 0; k < K; ++k) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += sh[w][k];
            v[k] = t;
        }
    }
}

// One thread-block cluster of CS blocks per capsule and snapshot (grid x:
// capsules times CS, grid y: snapshots); FP64 arithmetic is scarce per SM on
// this GPU, so a large capsule spreads its faces over the CS SMs of the
// cluster, whose blocks exchange partial sums through distributed shared
// memory within the one launch.  Block `rank` takes the faces
// f0 + rank * blockDim.x + threadIdx.x + k * CS * blockDim.x in order.
// Pass 1 gives each block's V, A and first-moment sums; after a cluster
// barrier every block adds the CS partials in rank order (the same bits in
// every block) and forms the centroid c = origin + m / (4 V); pass 2 sums the
// inertia terms about c, and block 0 adds those partials in rank order.  In
// recording mode snapshot k goes to ring record count + k and the last
// cluster to finish advances the record counter by the number of snapshots.
// Bounds-checked build: the nodes of face f lie among the n_nodes of a snapshot.
#ifdef IBLBM_BOUNDS_CHECK
#define IBLBM_FACE_OK(f)                                                                     \
    (IBLBM_OK(tri[f].x, 1, ss.stride) && IBLBM_OK(tri[f].y, 1, ss.stride) && IBLBM_OK(tri[f].z, 1, ss.stride))
#else
#define IBLBM_FACE_OK(f) (true)
#endif

template <typename R>
__global__ void __launch_bounds__(kTaylorClusterThreads) k_taylor_cluster(R nodes0, const int4 *__restrict__ tri,
                                                                          TaylorPlan p, SnapSet ss, int record) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ double sh[kTaylorClusterThreads / 32][6];
    __shared__ double part1[6], part2[6];  // this block's sums of pass 1 and 2 (read by the cluster)
    __shared__ double cen_sh[5];           // V, A, centroid
    const int CS = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const R nodes = nodes0.at(ss.slot(blockIdx.y), ss.stride);
    const int cap = blockIdx.x / CS;
    const int f0 = p.cap_face0[cap], f1 = p.cap_face0[cap + 1];
    const double o[3] = {p.origin[3 * cap], p.origin[3 * cap + 1], p.origin[3 * cap + 2]};
    const int stride = CS * blockDim.x;
    double v[6] = {0, 0, 0, 0, 0, 0};
    float oh[3], ol[3];  // float builds: the origin as a float pair
    if constexpr (std::is_same<R, NodeRead<float>>::value) FaceMath<R>::split(o, oh, ol);
    if constexpr (std::is_same<R, NodeRead<float>>::value) {
        float vf[5] = {0, 0, 0, 0, 0};
#pragma unroll 4
        for (int f = f0 + rank * blockDim.x + threadIdx.x; f < f1; f += stride) {
            if (!IBLBM_FACE_OK(f)) continue;
            float r[3], An[3], w[5];
            FaceMath<R>::geom(nodes, tri[f], oh, ol, r, An);
            FaceMath<R>::terms1(r, An, w);
            for (int k = 0; k < 5; ++k) vf[k] += w[k];
        }
        for (int k = 0; k < 5; ++k) v[k] = (double)vf[k];
    } else {
#pragma unroll 4
        for (int f = f0 + rank * blockDim.x + threadIdx.x; f < f1; f += stride) {
            double w[5];
            if (!IBLBM_FACE_OK(f)) continue;
            FaceMath<R>::stage1(nodes, tri[f], o, w);
            for (int k = 0; k < 5; ++k) v[k] += w[k];
        }
    }
    block_sum_any<6>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 5; ++k) part1[k] = v[k];
    cluster.sync();
    if (threadIdx.x == 0) {
        double t[5] = {0, 0, 0, 0, 0};
        for (int r = 0; r < CS; ++r) {
            const double *q = cluster.map_shared_rank(part1, r);
            for (int k = 0; k < 5; ++k) t[k] += q[k];
        }
        cen_sh[0] = t[0];
        cen_sh[1] = t[1];
        for (int k = 0; k < 3; ++k) cen_sh[2 + k] = o[k] + t[2 + k] / (4.0 * t[0]);
    }
    __syncthreads();
    const double c[3] = {cen_sh[2], cen_sh[3], cen_sh[4]};
    double I[6] = {0, 0, 0, 0, 0, 0};
    if constexpr (std::is_same<R, NodeRead<float>>::value) {
        float If[6] = {0, 0, 0, 0, 0, 0};
        float co[3];
        for (int k = 0; k < 3; ++k) co[k] = (float)(c[k] - o[k]);
#pragma unroll 4
        for (int f = f0 + rank * blockDim.x + threadIdx.x; f < f1; f += stride) {
            if (!IBLBM_FACE_OK(f)) continue;
            float cen[3], An[3], w[6];
            FaceMath<R>::geom(nodes, tri[f], oh, ol, cen, An);
            FaceMath<R>::terms2(cen, An, co, w);
            for (int k = 0; k < 6; ++k) If[k] += w[k];
        }
        for (int k = 0; k < 6; ++k) I[k] = (double)If[k];
    } else {
#pragma unroll 4
        for (int f = f0 + rank * blockDim.x + threadIdx.x; f < f1; f += stride) {
            double w[6];
            if (!IBLBM_FACE_OK(f)) continue;
            FaceMath<R>::stage2(nodes, tri[f], o, c, w);
            for (int k = 0; k < 6; ++k) I[k] += w[k];
        }
    }
    block_sum_any<6>(I, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) part2[k] = I[k];
    cluster.sync();
    if (rank == 0 && threadIdx.x == 0) {
        double t[6] = {0, 0, 0, 0, 0, 0};
        for (int r = 0; r < CS; ++r) {
            const double *q = cluster.map_shared_rank(part2, r);
            for (int k = 0; k < 6; ++k) t[k] += q[k];
        }
        // every cluster reads the record counter before its ticket, so before
        // the last one advances it
        const unsigned long long count = record ? *p.ring_count : 0ull;
        double *out = record ? p.ring + (size_t)((count + blockIdx.y) % (unsigned long long)p.ring_len) * p.n_caps * 12
                             : p.out;
        double *r = out + 12 * cap;
        for (int k = 0; k < 5; ++k) r[k] = cen_sh[k];
        for (int k = 0; k < 6; ++k) r[5 + k] = t[k];
        r[11] = 0.0;
        if (record) {
            __threadfence();
            if (atomicAdd(p.ticket, 1u) == (gridDim.x / CS) * gridDim.y - 1) {
                *p.ticket = 0u;
                *p.ring_count = count + gridDim.y;
            }
        }
    }
    cluster.sync();  // the other blocks' shared memory stays until block 0 has read it
}

template <typename R>
static void taylor_impl(R nodes, const MeshDev &m, const TaylorPlan &p, bool record, SnapSet ss,
                        cudaStream_t s) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = p.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t c = {};
    c.gridDim = dim3(p.n_caps * p.cluster, ss.n_snap);
    c.blockDim = dim3(kTaylorClusterThreads);
    c.dynamicSmemBytes = 0;
    c.stream = s;
    c.attrs = at;
    c.numAttrs = 1;
    cudaLaunchKernelEx(&c, k_taylor_cluster<R>, nodes, (const int4 *)m.tri, p, ss, record ? 1 : 0);
}

int taylor_max_cluster() {
    static int best = 0;
    if (best) return best;
    // 16 blocks per cluster where the GPU allows it (non-portable size), else 8
    int b = 8;
    if (cudaFuncSetAttribute(k_taylor_cluster<NodeRead<float>>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_taylor_cluster<NodeRead<double>>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess) {
        cudaLaunchConfig_t c = {};
        c.gridDim = dim3(16);
        c.blockDim = dim3(kTaylorClusterThreads);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        c.attrs = at;
        c.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_taylor_cluster<NodeRead<float>>, &c) == cudaSuccess && n > 0) b = 16;
    }
    cudaGetLastError();
    best = b;
    return best;
}

void launch_taylor(int prec, const MeshDev &m, const TaylorPlan &p, bool record, cudaStream_t s) {
    launch_taylor_snapshots(prec, m, p, record, m.x, m.x_lo, 0, 1, 1, s);
}

void launch_taylor_snapshots(int prec, const MeshDev &m, const TaylorPlan &p, bool record, const void *snap_x,
                             const void *snap_lo, int first, int slots, int n_snap, cudaStream_t s) {
    if (p.n_caps == 0 || n_snap < 1 || (record && !p.ring)) return;
    const SnapSet ss{first, slots, n_snap, (long long)m.n_nodes};
    if (prec == kF64)
        taylor_impl(NodeRead<double>{(const dvec4 *)snap_x}, m, p, record, ss, s);
    else
        taylor_impl(NodeRead<float>{(const float4 *)snap_x, (const float4 *)snap_lo}, m, p, record, ss, s);
}


// ---- allocation-free variant ---------------------------------------------------------
// Some callers cannot allocate device memory when they need these reductions:
// code whose whole device budget is handed to another allocator (a framework's
// caching allocator or a fixed arena), plug-ins called back from such a
// framework, or a tight loop in which an allocation would synchronise the
// device.  For them the per-block
// partial sums of the three stages live in this fixed array, which every GPU
// that loads the library holds until the process exits.
constexpr int kNoAllocMaxBlocks = 1024;  // 1024 blocks x 128 faces = 131072 faces
static __device__ __align__(256) double g_noalloc_partial[kNoAllocMaxBlocks * 16];

struct PlainRead {
    const double *x;  // [n][3]
    __device__ __forceinline__ void get(int n, double p[3]) const {
        p[0] = x[3 * n];
        p[1] = x[3 * n + 1];
        p[2] = x[3 * n + 2];
    }
};

__device__ __forceinline__ bool face_ok(const int *tri, int f, int n_nodes, int4 &t) {
    t = make_int4(tri[3 * f], tri[3 * f + 1], tri[3 * f + 2], 0);
    return t.x >= 0 && t.x < n_nodes && t.y >= 0 && t.y < n_nodes && t.z >= 0 && t.z < n_nodes;
}

// Totals of K partial entries (from `first`) over nb blocks, by one warp.
template <int K>
__device__ __forceinline__ void plain_totals(const double *partial, int nb, int first, double tot[K]) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < K; ++k) tot[k] = 0.0;
    for (int b = lane; b < nb; b += 32)
        for (int k = 0; k < K; ++k) tot[k] += partial[16 * b + first + k];
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) tot[k] += __shfl_xor_sync(0xffffffffu, tot[k], o);
}

__global__ void __launch_bounds__(kTB) k_noalloc_stage1(const double *__restrict__ x, int n_nodes,
                                                        const int *__restrict__ tri, int n_tri,
                                                        double ox, double oy, double oz,
                                                        double *__restrict__ partial) {
    __shared__ double sh[kTB / 32][6];
    const int f = blockIdx.x * kTB + threadIdx.x;
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (f < n_tri) {
        int4 t;
        if (face_ok(tri, f, n_nodes, t)) {
            double cen[3], An[3];
            face_geom(PlainRead{x}, t, cen, An);
            const double r[3] = {cen[0] - ox, cen[1] - oy, cen[2] - oz};
            const double rn = r[0] * An[0] + r[1] * An[1] + r[2] * An[2];
            v[0] = rn * (1.0 / 3.0);
            v[1] = sqrt(An[0] * An[0] + An[1] * An[1] + An[2] * An[2]);
            v[2] = rn * r[0];
            v[3] = rn * r[1];
            v[4] = rn * r[2];
        } else {
            v[5] = 1.0;  // face skipped: a node index outside [0, n_nodes)
        }
    }
    block_sum<6>(v, sh);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 5; ++k) partial[16 * blockIdx.x + k] = v[k];
        partial[16 * blockIdx.x + 15] = v[5];
    }
}

__global__ void __launch_bounds__(kTB) k_noalloc_stage2(const double *__restrict__ x, int n_nodes,
                                                        const int *__restrict__ tri, int n_tri,
                                                        double ox, double oy, double oz,
                                                        double *__restrict__ partial) {
    __shared__ double sh[kTB / 32][6];
    __shared__ double cen_sh[3];
    if (threadIdx.x < 32) {
        double tot[5];
        plain_totals<5>(partial, gridDim.x, 0, tot);
        if (threadIdx.x == 0) {
            cen_sh[0] = ox + tot[2] / (4.0 * tot[0]);
            cen_sh[1] = oy + tot[3] / (4.0 * tot[0]);
            cen_sh[2] = oz + tot[4] / (4.0 * tot[0]);
        }
    }
    __syncthreads();
    const int f = blockIdx.x * kTB + threadIdx.x;
    double v[6] = {0, 0, 0, 0, 0, 0};
    int4 t;
    if (f < n_tri && face_ok(tri, f, n_nodes, t)) {
        double cen[3], An[3];
        face_geom(PlainRead{x}, t, cen, An);
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
        for (int k = 0; k < 6; ++k) partial[16 * blockIdx.x + 8 + k] = v[k];
}

__global__ void k_noalloc_stage3(const double *__restrict__ partial, int nb, double ox, double oy,
                                 double oz, double *__restrict__ out) {
    double tot[5], I[6], bad[1];
    plain_totals<5>(partial, nb, 0, tot);
    plain_totals<6>(partial, nb, 8, I);
    plain_totals<1>(partial, nb, 15, bad);
    if (threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
        out[2] = ox + tot[2] / (4.0 * tot[0]);
        out[3] = oy + tot[3] / (4.0 * tot[0]);
        out[4] = oz + tot[4] / (4.0 * tot[0]);
        for (int k = 0; k < 6; ++k) out[5 + k] = I[k];
        out[11] = bad[0];
    }
}

IBLBM_BOUNDS_ACCESSOR(bounds_faults_taylor)

}  // namespace iblbm

namespace {
// Device address of g_noalloc_partial, looked up once per device and kept for
// the life of the process (a device reset would invalidate it; the header
// says so).
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[256] = {nullptr};
}  // namespace

extern "C" int iblbm_taylor_sums_noalloc(const double *nodes, int n_nodes, const int32_t *tri,
                                         int n_tri, const double origin[3], double *out,
                                         void *stream) {
    using namespace iblbm;
    if (!nodes || !tri || !origin || !out || n_nodes < 4 || n_tri < 4) {
        set_thread_error("iblbm_taylor_sums_noalloc: null pointer, or fewer than 4 nodes or faces");
        return IBLBM_ERR_ARG;
    }
    if (n_tri > kNoAllocMaxBlocks * kTB) {
        set_thread_error("iblbm_taylor_sums_noalloc: more than 131072 faces (the size of its fixed scratch)");
        return IBLBM_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        set_thread_error("iblbm_taylor_sums_noalloc: no usable current CUDA device");
        return IBLBM_ERR_CUDA;
    }
    double *partial = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            // First call on this device (with it current): look up the device
            // address of the fixed scratch array.
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
            if (e != cudaSuccess) {
                cudaGetLastError();
                set_thread_error(std::string("iblbm_taylor_sums_noalloc: cudaGetSymbolAddress failed: ") +
                                 cudaGetErrorString(e));
                return IBLBM_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = (double *)p;
        }
        partial = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (n_tri + kTB - 1) / kTB;
    cudaGetLastError();
    k_noalloc_stage1<<<nb, kTB, 0, s>>>(nodes, n_nodes, tri, n_tri, origin[0], origin[1], origin[2], partial);
    k_noalloc_stage2<<<nb, kTB, 0, s>>>(nodes, n_nodes, tri, n_tri, origin[0], origin[1], origin[2], partial);
    k_noalloc_stage3<<<1, 32, 0, s>>>(partial, nb, origin[0], origin[1], origin[2], out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_thread_error(std::string("iblbm_taylor_sums_noalloc: launch failed: ") + cudaGetErrorString(e));
        return IBLBM_ERR_CUDA;
    }
    return IBLBM_OK;
}

namespace iblbm {

}  // namespace iblbm
