// device_common.cuh -- device-side building blocks shared by the kernels of
// the IB-LBM-FEM library: the D3Q19 velocity set, the discrete delta
// functions, storage conversions and double-float node coordinates.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace iblbm {

// Kernel-side error bits (OR-ed into the device status word).
enum : int {
    kStatusUnstable = 1,  // density out of (0.5, 2) or NaN
    kStatusStencil = 2,   // an IBM stencil cell beyond a wall
    kStatusTimeout = 4,   // a bounded wait for staged data gave up
    kStatusForceRange = 8,  // a force contribution beyond the deterministic spreading's fixed-point range
};

// D3Q19 velocity set numbered as in Fig. d3q19 of the paper (the arrow i
// points to twice (cx, cy, cz) in the figure's coordinates).
#define IBLBM_D3Q19_CX {0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, -1, 1, 1, -1, 0, 0, 0, 0}
#define IBLBM_D3Q19_CY {0, 0, 0, 1, -1, 0, 0, 0, 0, -1, 1, 0, 0, -1, 1, -1, 1, -1, 1}
#define IBLBM_D3Q19_CZ {0, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1}
// index of -c_i
#define IBLBM_D3Q19_OPP {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17}

__host__ __device__ constexpr int q_cx(int i) {
    constexpr int t[19] = IBLBM_D3Q19_CX;
    return t[i];
}
__host__ __device__ constexpr int q_cy(int i) {
    constexpr int t[19] = IBLBM_D3Q19_CY;
    return t[i];
}
__host__ __device__ constexpr int q_cz(int i) {
    constexpr int t[19] = IBLBM_D3Q19_CZ;
    return t[i];
}
__host__ __device__ constexpr int q_opp(int i) {
    constexpr int t[19] = IBLBM_D3Q19_OPP;
    return t[i];
}
// Weight by speed class: |c|^2 = 0 -> 1/3, 1 -> 1/18, 2 -> 1/36.
template <typename T>
__host__ __device__ constexpr T q_w(int i) {
    return (i == 0) ? T(1) / T(3) : (i <= 6 ? T(1) / T(18) : T(1) / T(36));
}

// Scale applied to the half-precision population deviations so that their
// typical magnitude (1e-6 .. 1e-1) stays in the normal range of binary16.
constexpr float kHalfScale = 4096.0f;
constexpr float kHalfInvScale = 1.0f / 4096.0f;

template <typename S, typename T>
struct Store;
template <>
struct Store<double, double> {
    static __device__ __forceinline__ double load(const double *p) { return __ldg(p); }
    static __device__ __forceinline__ void store(double *p, double v) { *p = v; }
};
template <>
struct Store<float, float> {
    static __device__ __forceinline__ float load(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ void store(float *p, float v) { *p = v; }
};
template <>
struct Store<__half, float> {
    static __device__ __forceinline__ float load(const __half *p) {
        return __half2float(__ldg(p)) * kHalfInvScale;
    }
    static __device__ __forceinline__ void store(__half *p, float v) {
        *p = __float2half_rn(v * kHalfScale);
    }
};

struct __align__(32) dvec4 {
    double x, y, z, w;
};

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = dvec4;
};

// ---- discrete delta functions, Eqs. (2point), (3point), (4point) ----------
template <int N, typename T>
__device__ __forceinline__ T delta_phi(T r) {
    T a = fabs(r);
    if constexpr (N == 2) {
        return a < T(1) ? T(1) - a : T(0);
    } else if constexpr (N == 3) {
        if (a <= T(0.5)) return (T(1) + sqrt(T(1) - T(3) * a * a)) * (T(1) / T(3));
        if (a < T(1.5)) return (T(5) - T(3) * a - sqrt(fmax(T(0), T(6) * a - T(3) * a * a - T(2)))) * (T(1) / T(6));
        return T(0);
    } else {
        if (a <= T(1)) return (T(3) - T(2) * a + sqrt(T(1) + T(4) * a - T(4) * a * a)) * T(0.125);
        if (a < T(2)) return (T(5) - T(2) * a - sqrt(fmax(T(0), T(12) * a - T(4) * a * a - T(7)))) * T(0.125);
        return T(0);
    }
}

// First lattice index of the N-point stencil around coordinate x: the N
// nodes i0 .. i0+N-1 with i0 = floor(x - N/2) + 1 contain every node where the
// kernel is non-zero.
template <int N, typename T>
__device__ __forceinline__ int stencil_first(T x) {
    return static_cast<int>(floor(x - T(0.5) * N)) + 1;
}

// ---- node coordinates -----------------------------------------------------
// FP64 build: plain doubles.  Float builds: an unevaluated sum hi + lo of two
// floats, advanced with an error-free two-sum, so that the ~1e-3 per-step
// displacement of a node at coordinate ~100 keeps ~48 bits over 1e4+ steps.
struct Coord2f {
    float hi, lo;
};

__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float d) {
    float s = hi + d;
    float bb = s - hi;
    float err = (hi - (s - bb)) + (d - bb);
    float l = lo + err;
    float t = s + l;
    lo = l - (t - s);
    hi = t;
}

// Double-float (unevaluated sum h + l of two floats) helpers.
struct DF {
    float h, l;
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    return DF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = a + b;
    return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = df_two_sum(a.h, b.h);
    return df_fast_two_sum(s.h, s.l + (a.l + b.l));
}

__device__ __forceinline__ int wrap_index(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}
// wrap_index(w0 + k, n) for w0 already in [0, n) and 0 <= k < N: one
// subtraction when n >= N (no division), else the general form.
template <int N>
__device__ __forceinline__ int wrap_next(int w0, int k, int n) {
    const int a = w0 + k;
    if (a < n) return a;
    return n >= N ? a - n : wrap_index(a, n);
}

__device__ __forceinline__ void set_status(int *status, int bit) { atomicOr(status, bit); }

// ---- bounds-checked build (-DIBLBM_BOUNDS_CHECK, lib/libiblbm_checked.so) ----
// IBLBM_OK(i, k, n): whether the k elements i .. i + k - 1 lie in [0, n).  The
// kernels guard their computed accesses with it: in the checked build a
// failed check is counted in this translation unit's fault counter and the
// access is skipped (loads read 0), so the kernel never leaves its buffers;
// in the normal build it is the constant true and its arguments are not
// evaluated.  bounds_faults_*() read (and clear) the counter from the host.
#ifdef IBLBM_BOUNDS_CHECK
static __device__ unsigned long long g_bounds_faults;
__device__ __forceinline__ bool bounds_ok(long long i, long long k, long long n) {
    if (i < 0 || i + k > n) {
        atomicAdd(&g_bounds_faults, 1ull);
        return false;
    }
    return true;
}
#define IBLBM_OK(i, k, n) (::iblbm::bounds_ok((long long)(i), (long long)(k), (long long)(n)))
#define IBLBM_BOUNDS_ACCESSOR(name)                                                        \
    unsigned long long name() {                                                            \
        unsigned long long v = 0, z = 0;                                                   \
        if (cudaMemcpyFromSymbol(&v, g_bounds_faults, sizeof(v)) != cudaSuccess) {         \
            cudaGetLastError();                                                            \
            return ~0ull;                                                                  \
        }                                                                                  \
        cudaMemcpyToSymbol(g_bounds_faults, &z, sizeof(z));                                \
        return v;                                                                          \
    }
#else
#define IBLBM_OK(i, k, n) (true)
#define IBLBM_BOUNDS_ACCESSOR(name) \
    unsigned long long name() { return 0ull; }
#endif

// Programmatic dependent launch (sm_90 and later).  A time-step kernel may be
// launched while its predecessor in the stream still runs.  It calls
// prior_grid_wait() before it touches anything that the predecessor writes,
// or writes anything that the predecessor reads, and then allow_dependents(),
// which lets the next kernel launch.  Waiting first makes the chain
// transitive: when a kernel starts, the kernel two places before it has
// completed, so what it does before the wait may read data of that kernel or
// older ones.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void prior_grid_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---- staging of tiles in shared memory by the bulk-copy (TMA) engine ----------------
// An mbarrier in shared memory counts the bytes of the bulk copies issued
// against it; a thread that waits on its phase parity sees the copied data.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Makes mbarrier initialisations visible to the other threads and to the
// bulk-copy engine (followed by a block barrier).
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Orders this thread's generic-proxy shared-memory accesses (an mbarrier
// init, reads of a buffer about to be refilled) before later bulk copies.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_bytes(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to this block's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_copy_to_smem(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Waits for phase `parity` of `bar`, giving up after limit_ns nanoseconds
// (0: gives up at once, without polling, so that the failure path can be
// exercised deterministically).  Returns whether the phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, unsigned long long limit_ns) {
    if (limit_ns == 0) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

}  // namespace iblbm
