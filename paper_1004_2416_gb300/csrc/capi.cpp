// capi.cpp -- the C ABI of include/iblbm.h: simulation object, device memory,
// membrane tables, the time-step sequence (captured in CUDA graphs) and the
// read-back paths.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "iblbm.h"
#include "internal.h"

using namespace iblbm;

namespace {

struct Capsule {
    int node0, n_nodes, face0, n_faces;
    int run;  // lattice (run) of a batch; 0 for a single lattice
    double ks, ka;
    double origin[3];  // reference centre (mean of the reference nodes)
};

// Tile shapes the batched collide kernel can use (tx * ty = 256 threads).
constexpr int kTileShapes[6][2] = {{32, 8}, {16, 16}, {8, 32}, {64, 4}, {128, 2}, {256, 1}};

constexpr int kGraphSteps = 32;  // steps per captured graph (even)
constexpr int kMaxStepGraphs = 16;  // captured step sequences kept per object

thread_local std::string g_create_error;

// A named range on the host timeline of a profiler (NVTX; a few nanoseconds
// when no tool is attached): the API calls below and, inside a step, each
// kernel group as it is enqueued or captured.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

}  // namespace

void iblbm::set_thread_error(const std::string &msg) { g_create_error = msg; }

struct iblbm_sim {
    Lattice L{};
    int prec = 1;
    int delta = 3;
    double tau = 1.0;
    double u_wall = 0.0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // Side stream for the Taylor records.  The interpolation of a recorded
    // step also writes the new positions into the next slot of a ring of
    // 2 kTaylorBatch snapshots (two halves); when a half is full (or at a
    // flush) one launch on the side stream reduces its snapshots, concurrently
    // with the next steps, and is joined before the half is written again.
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
    // Kernel timing in captured steps: the timing events are recorded on a
    // branch of the graph (this stream, forked from the main stream after each
    // kernel group and joined at the end of the graph), so the main chain of
    // kernels keeps its kernel-to-kernel edges.
    cudaStream_t tstream = nullptr;
    cudaEvent_t ev_tfork = nullptr;
    bool side_pending[2] = {false, false};
    void *snap_x = nullptr, *snap_lo = nullptr;  // [2 kTaylorBatch][n_nodes] in the layout of mesh.x / x_lo
    int rec_half = 0, rec_fill = 0;  // half being filled and its snapshots so far
    int rec_batch = 1;               // snapshots per half (<= kTaylorBatch)
    const char *launch_fail = nullptr;  // first kernel group whose launch failed
    iblbm_allocator alloc{};
    bool has_alloc = false;
    size_t pop_bytes = 0;   // one population buffer
    size_t vec_bytes = 0;   // one force buffer
    size_t flag_bytes = 0;  // one flag buffer
    void *pop[2] = {nullptr, nullptr};
    int cur = 0;  // pop[cur] holds f(t); force[cur] the last spread force
    void *force[2] = {nullptr, nullptr};
    uint8_t *flags[2] = {nullptr, nullptr};
    void *uvel = nullptr;  // velocity of the cells of the flagged tiles (Vec4 per cell)
    int interp_mode = -1;  // -1 automatic, 0 gather at the stencil cells, 1 cell velocities first
    int staging = -1;      // collide populations staged by bulk copies: -1 automatic, 0 off, 1 on
    unsigned long long wait_ns = 1000000000ull;  // longest device wait for staged data
    int overlap = -1;      // step kernels overlapping their predecessor: -1 automatic, 0 off, 1 on
    // deterministic spreading: the force density summed in 64-bit fixed point
    // ([ncell][3], zero between steps), then converted (iblbm_set_deterministic_spreading)
    unsigned long long *d_fix = nullptr;
    // Method variants: node advection 0 = Euler (Eq. positionupdate), 1 =
    // Adams-Bashforth (Sec. II.C), which needs the node velocities of the step
    // before (ab2_ready); equilibrium order 2 = Eq. (equilibrium), 1 = the
    // linearised form of Sec. IV.A.
    int integrator = 0;
    bool ab2_ready = false;
    int eq_order = 2;
    int *d_status = nullptr;

    std::vector<Capsule> caps;
    std::vector<double> X0;  // reference nodes [n][3]
    // current positions of the nodes of a mesh whose rebuild failed (its device
    // tables are gone; the next ensure_mesh starts from these)
    std::vector<double> x_pending;
    std::vector<int> tri;    // faces [f][3], global node indices
    bool mesh_dirty = false;
    int dev_nodes = 0;  // nodes present in the device arrays
    MeshDev mesh{};
    std::vector<void *> mesh_allocs;
    TaylorPlan plan{};
    std::vector<void *> plan_allocs;

    double *d_scratch = nullptr;
    unsigned long long *d_cksum = nullptr;  // checkpoint section checksums
    // iblbm_read_async: the positions are copied into a snapshot on the main
    // stream; their conversion to doubles, the capsule reductions and the
    // copies to the host run from it on the read-back stream, so the steps
    // enqueued after a read-back do not wait for it.  Two sets of buffers,
    // alternating; a set is written again once the read-back stream is done
    // with it (ev_rdone).
    cudaStream_t rstream = nullptr;
    cudaEvent_t ev_rsnap[2] = {nullptr, nullptr}, ev_rdone[2] = {nullptr, nullptr};
    bool rb_used[2] = {false, false};
    int rb_next = 0;
    void *rb_x[2] = {nullptr, nullptr}, *rb_lo[2] = {nullptr, nullptr};  // layout of mesh.x / x_lo
    double *rb_nodes[2] = {nullptr, nullptr}, *rb_sums[2] = {nullptr, nullptr};
    int rb_nodes_cap = 0, rb_caps_cap = 0;  // nodes and capsules the buffers hold
    size_t scratch_bytes = 0;

    // Taylor recording: after every `rec_every`-th step (0 = off) the device
    // reductions of all capsules go into a ring of `rec_ring` records.
    int rec_every = 0;
    int rec_ring = 0;
    double *d_ring = nullptr;
    unsigned long long *d_ring_count = nullptr;
    std::vector<int64_t> rec_steps;  // step number of every record enqueued

    // Batch of independent runs (iblbm_batch_create): run table, work list of
    // (run, tile) pairs for the persistent collide kernel, per-node run index.
    bool batch = false;
    std::vector<RunDesc> runs;
    std::vector<long long> run_tile_cap;  // flags reserved per run (largest tile count)
    RunDesc *d_runs = nullptr;
    int2 *d_items = nullptr;
    int n_items = 0;
    int batch_grid = 0;
    bool batch_pairs = false;  // the batch collide takes two cells per thread
    int *d_node_run = nullptr;

    // Adjoint: checkpoints of the forward run and the buffers of the reverse sweep.
    struct Adjoint {
        bool ready = false;
        int K = 0;
        int64_t n = 0, t_start = 0;
        bool couette_start = false;
        std::vector<void *> ck_pop, ck_x;
        // Two sets of recomputation buffers: the segment before the one being
        // swept backwards is recomputed into the other set on a second stream.
        struct Trace {
            void *pop[2] = {nullptr, nullptr};  // recomputation populations (ping-pong)
            std::vector<void *> M, g, flags, x, F;  // kept forward quantities of a segment
        } tr[2];
        cudaStream_t rstream = nullptr;  // recomputation stream
        cudaEvent_t ev_start = nullptr, ev_rec[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr};
        void *lam[2] = {nullptr, nullptr}, *lamx[2] = {nullptr, nullptr};
        void *mu = nullptr, *lamg = nullptr, *lamF = nullptr, *fref = nullptr;
        uint8_t *zero_flags = nullptr;
        double *uw_partial = nullptr, *gX0 = nullptr, *gks = nullptr;
        void *save_x = nullptr, *save_F = nullptr, *save_u = nullptr;
        bool g_dirty = true;             // tr_g may hold a force density (zeroed before use)
        std::vector<void *> allocs;      // reverse-sweep buffers, kept while K is unchanged
        std::vector<void *> ck_allocs;   // checkpoints of the last forward run
        // captured recomputations (kind 0) keyed by (segment length, set) and
        // reverse sweeps (kind 1) by (length, set, parity of the adjoint double
        // buffers at the start); valid for graph_mesh / graph_uw
        std::vector<std::pair<std::array<int, 4>, cudaGraphExec_t>> graphs;
        MeshDev graph_mesh{};
        double graph_uw = 0.0;
    } adj;
    int init_mode = 0;

    // Captured step sequences: any run of steps from a phase of the recording
    // period replays one of these graphs (at most kMaxStepGraphs, least
    // recently used dropped first).
    struct StepGraph {
        int len = 0;            // steps in the graph
        int cur = 0;            // buffer parity at its start (pop[cur] holds f(t))
        int first_rec = -1;     // step of its first Taylor record (-1: none)
        cudaGraphExec_t exec = nullptr;
        int64_t kernels = 0;    // kernels per replay
        uint64_t used = 0;      // replay stamp (least recently used is dropped)
        std::vector<cudaEvent_t> ev;  // kernel timing: 4 per step (see kernel_timing)
        bool timed = false;     // replayed since the last read of its events
    };
    std::vector<StepGraph> sgraphs;
    uint64_t graph_clock = 0;
    bool kernel_timing = false;  // graphs carry event nodes around the kernel groups
    int64_t launches = 0;               // kernels launched for time steps
    int graph_len = 0;
    // x-slab group (iblbm_create_slabs): the slabs, each a lattice object of
    // its own holding the global columns L.x0 .. L.x0 + L.nx - 1, with the
    // membranes replicated on every slab; the group object itself holds no
    // lattice buffers.
    std::vector<iblbm_sim *> slabs;
    void *slab_planes = nullptr;       // packed boundary columns, one block per slab
    size_t slab_plane_bytes = 0;       // one slab's block
    void *slab_parts = nullptr;        // node-velocity partials, one Vec4 array per slab
    void **slab_part_ptrs = nullptr;   // device array of the partials' addresses
    int slab_parts_nodes = -1;
    size_t slab_parts_bytes = 0;       // held by slab_parts (per-process slab phases)
    int64_t steps = 0;
    std::string err;
};

namespace {

void adj_free(iblbm_sim *s);
bool is_group(const iblbm_sim *s);
int group_unsupported(iblbm_sim *s);
int group_step(iblbm_sim *s, int64_t n_steps);
int group_field(iblbm_sim *s, int what, double *host, bool set);

int fail(iblbm_sim *s, int code, const std::string &msg) {
    if (s) s->err = msg;
    return code;
}

int cuda_fail(iblbm_sim *s, cudaError_t e, const char *what) {
    return fail(s, IBLBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, #call);     \
    } while (0)

void *dev_alloc(iblbm_sim *s, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (s->has_alloc) {
        p = s->alloc.alloc(bytes, (void *)s->stream, s->alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dev_free(iblbm_sim *s, void *p) {
    if (!p) return;
    if (s->has_alloc) s->alloc.free(p, (void *)s->stream, s->alloc.ctx);
    else cudaFree(p);
}

void free_step_graph(iblbm_sim::StepGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : g.ev) cudaEventDestroy(e);
    g.exec = nullptr;
    g.ev.clear();
}

void drop_graphs(iblbm_sim *s) {
    for (auto &g : s->sgraphs) free_step_graph(g);
    s->sgraphs.clear();
}

int ensure_scratch(iblbm_sim *s, size_t bytes) {
    if (s->scratch_bytes >= bytes) return IBLBM_OK;
    // whole MiB, so that requests a few words apart (a field read back, then
    // the same field uploaded with its status word) share one allocation
    bytes = (bytes + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
    dev_free(s, s->d_scratch);
    s->d_scratch = (double *)dev_alloc(s, bytes);
    s->scratch_bytes = s->d_scratch ? bytes : 0;
    if (!s->d_scratch) return fail(s, IBLBM_ERR_OOM, "scratch allocation failed");
    return IBLBM_OK;
}

size_t real_bytes(const iblbm_sim *s) { return s->prec == kF64 ? 8 : 4; }

void free_ring(iblbm_sim *s);
void join_side(iblbm_sim *s);
void reduce_snapshots(iblbm_sim *s);

// iblbm_read_async's buffers: released once the read-back stream is done
// with them.
void free_readback(iblbm_sim *s) {
    if (s->rstream) cudaStreamSynchronize(s->rstream);
    for (int b = 0; b < 2; ++b) {
        dev_free(s, s->rb_x[b]);
        dev_free(s, s->rb_lo[b]);
        dev_free(s, s->rb_nodes[b]);
        dev_free(s, s->rb_sums[b]);
        s->rb_x[b] = s->rb_lo[b] = nullptr;
        s->rb_nodes[b] = s->rb_sums[b] = nullptr;
        s->rb_used[b] = false;
    }
    s->rb_nodes_cap = s->rb_caps_cap = 0;
}

// Both sets of read-back buffers for n nodes and nc capsules; on a refused
// block none is kept.
int ensure_readback(iblbm_sim *s, int n, int nc) {
    if (s->rb_nodes_cap >= n && s->rb_caps_cap >= nc && s->rb_x[0]) return IBLBM_OK;
    free_readback(s);
    const size_t v4 = 4 * real_bytes(s) * (size_t)n;
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
        s->rb_x[b] = dev_alloc(s, v4);
        s->rb_lo[b] = s->prec == kF64 ? nullptr : dev_alloc(s, (size_t)16 * n);
        s->rb_nodes[b] = (double *)dev_alloc(s, sizeof(double) * 3 * (size_t)n);
        s->rb_sums[b] = (double *)dev_alloc(s, sizeof(double) * 12 * (size_t)(nc > 0 ? nc : 1));
        ok = s->rb_x[b] && (s->prec == kF64 || s->rb_lo[b]) && s->rb_nodes[b] && s->rb_sums[b];
    }
    if (!ok) {
        free_readback(s);
        return fail(s, IBLBM_ERR_OOM, "read-back buffer allocation failed");
    }
    s->rb_nodes_cap = n;
    s->rb_caps_cap = nc;
    return IBLBM_OK;
}

// (Re)builds the device membrane tables after capsules were added.  Current
// node positions of existing capsules are kept.
int ensure_mesh(iblbm_sim *s) {
    if (!s->mesh_dirty) return IBLBM_OK;
    join_side(s);  // nothing may still read the tables that are rebuilt below
    CK(cudaStreamSynchronize(s->stream));
    if (s->rstream) CK(cudaStreamSynchronize(s->rstream));  // nor a read-back
    const int nn = (int)(s->X0.size() / 3), nf = (int)(s->tri.size() / 3), nc = (int)s->caps.size();
    std::vector<double> xcur(s->X0);
    if (s->dev_nodes > 0) {
        int rc = ensure_scratch(s, sizeof(double) * 3 * s->dev_nodes);
        if (rc) return rc;
        launch_nodes_to_f64(s->prec, s->mesh, 0, 0, s->dev_nodes, s->d_scratch, s->stream);
        CK(cudaMemcpyAsync(xcur.data(), s->d_scratch, sizeof(double) * 3 * s->dev_nodes,
                           cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        s->x_pending.assign(xcur.begin(), xcur.begin() + 3 * (size_t)s->dev_nodes);
    } else {
        std::copy(s->x_pending.begin(), s->x_pending.begin() + std::min(s->x_pending.size(), xcur.size()),
                  xcur.begin());
    }
    // from here on the old tables are gone: a failure below leaves no device
    // pointer to them, and a later call rebuilds from x_pending
    drop_graphs(s);
    free_ring(s);
    for (void *p : s->mesh_allocs) dev_free(s, p);
    s->mesh_allocs.clear();
    for (void *p : s->plan_allocs) dev_free(s, p);
    s->plan_allocs.clear();
    s->mesh = MeshDev{};
    s->plan = TaylorPlan{};
    s->dev_nodes = 0;

    const size_t rb = real_bytes(s);
    const size_t v4 = 4 * rb;
    auto A = [&](size_t bytes) {
        void *p = dev_alloc(s, bytes);
        if (p) s->mesh_allocs.push_back(p);
        return p;
    };
    MeshDev m{};
    m.n_nodes = nn;
    m.n_faces = nf;
    m.n_caps = nc;
    m.x = A(v4 * nn);
    m.x_lo = s->prec == kF64 ? nullptr : A(v4 * nn);
    s->snap_x = A(2 * kTaylorBatch * v4 * nn);
    s->snap_lo = s->prec == kF64 ? nullptr : A(2 * kTaylorBatch * v4 * nn);
    if (!s->snap_x || (s->prec != kF64 && !s->snap_lo))
        return fail(s, IBLBM_ERR_OOM, "membrane table allocation failed");
    s->rec_half = 0;
    s->rec_fill = 0;
    // batches pay where the launches cost more than the reductions (few faces);
    // a large suspension reduces each record at once
    s->rec_batch = nf <= 32768 ? kTaylorBatch : 1;
    m.F = A(v4 * nn);
    m.u = A(v4 * nn);
    void *adj_off = A(sizeof(int) * (nn + 1));
    void *adj = A(sizeof(int) * 3 * nf);
    void *adj4 = A(sizeof(int) * 12 * nf);
    void *node_cap = A(sizeof(int) * nn);
    void *tri4 = A(sizeof(int) * 4 * nf);
    void *fconst = A(3 * v4 * nf);
    void *capmod = A(v4 * nc);
    void *node_run = s->batch ? A(sizeof(int) * nn) : nullptr;
    if (!m.x || (s->prec != kF64 && !m.x_lo) || !m.F || !m.u || !adj_off || !adj || !adj4 || !node_cap || !tri4 ||
        !fconst || !capmod || (s->batch && !node_run))
        return fail(s, IBLBM_ERR_OOM, "membrane table allocation failed");
    if (s->batch) {
        std::vector<int> nr(nn, 0);
        for (const Capsule &cp : s->caps)
            for (int n = cp.node0; n < cp.node0 + cp.n_nodes; ++n) nr[n] = cp.run;
        CK(cudaMemcpyAsync(node_run, nr.data(), sizeof(int) * nn, cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    s->d_node_run = (int *)node_run;

    // node -> (face, corner) lists in ascending face order
    std::vector<int> off(nn + 1, 0), ent(3 * (size_t)nf);
    for (int f = 0; f < nf; ++f)
        for (int k = 0; k < 3; ++k) off[s->tri[3 * f + k] + 1]++;
    for (int n = 0; n < nn; ++n) {
        if (off[n + 1] > 32) return fail(s, IBLBM_ERR_ARG, "a node belongs to more than 32 faces");
        off[n + 1] += off[n];
    }
    {
        std::vector<int> fill(off.begin(), off.end() - 1);
        for (int f = 0; f < nf; ++f)
            for (int k = 0; k < 3; ++k) ent[fill[s->tri[3 * f + k]]++] = 4 * f + k;
    }
    // the same entries with their face's nodes, so that one load gives the
    // force kernel everything it needs before the positions
    std::vector<int> ent4(12 * (size_t)nf), ncap(nn, 0);
    for (size_t e = 0; e < ent.size(); ++e) {
        const int f = ent[e] >> 2;
        ent4[4 * e] = ent[e];
        for (int k = 0; k < 3; ++k) ent4[4 * e + 1 + k] = s->tri[3 * f + k];
    }
    for (int c = 0; c < nc; ++c)
        for (int n = s->caps[c].node0; n < s->caps[c].node0 + s->caps[c].n_nodes; ++n) ncap[n] = c;
    std::vector<int> t4(4 * (size_t)nf);
    std::vector<double> fc(12 * (size_t)nf, 0.0), cm(4 * (size_t)nc, 0.0);
    const bool split = s->prec != kF64;  // float builds: G as float hi + lo
    for (int c = 0; c < nc; ++c) {
        const Capsule &cp = s->caps[c];
        cm[4 * c] = cp.ks / 6.0;
        cm[4 * c + 1] = cp.ka / 6.0;
        for (int f = cp.face0; f < cp.face0 + cp.n_faces; ++f) t4[4 * f + 3] = c;
    }
    for (int f = 0; f < nf; ++f) {
        const int a = s->tri[3 * f], b = s->tri[3 * f + 1], c = s->tri[3 * f + 2];
        t4[4 * f] = a;
        t4[4 * f + 1] = b;
        t4[4 * f + 2] = c;
        double U[3], V[3];
        for (int k = 0; k < 3; ++k) {
            U[k] = s->X0[3 * b + k] - s->X0[3 * a + k];
            V[k] = s->X0[3 * c + k] - s->X0[3 * a + k];
        }
        const double G11 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
        const double G12 = U[0] * V[0] + U[1] * V[1] + U[2] * V[2];
        const double G22 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
        const double det = G11 * G22 - G12 * G12;
        if (!(det > 0.0)) return fail(s, IBLBM_ERR_ARG, "degenerate reference face");
        double *q = fc.data() + 12 * (size_t)f;
        q[0] = G22 / det;  // alpha
        q[1] = G12 / det;  // beta
        q[2] = G11 / det;  // gamma
        q[3] = 1.0 / det;  // kappa
        q[4] = 0.5 * std::sqrt(det);  // A0
        const double G[3] = {G11, G12, G22};
        for (int k = 0; k < 3; ++k) {
            const double hi = split ? (double)(float)G[k] : G[k];
            q[5 + k] = hi;
            q[8 + k] = split ? (double)(float)(G[k] - hi) : 0.0;
        }
    }
    auto up_real = [&](void *dst, const std::vector<double> &v) -> cudaError_t {
        if (s->prec == kF64)
            return cudaMemcpyAsync(dst, v.data(), v.size() * 8, cudaMemcpyHostToDevice, s->stream);
        std::vector<float> f(v.begin(), v.end());
        cudaError_t e = cudaMemcpyAsync(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        return e;
    };
    CK(cudaMemcpyAsync(adj_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(adj, ent.data(), sizeof(int) * ent.size(), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(adj4, ent4.data(), sizeof(int) * ent4.size(), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(node_cap, ncap.data(), sizeof(int) * ncap.size(), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(tri4, t4.data(), sizeof(int) * t4.size(), cudaMemcpyHostToDevice, s->stream));
    CK(up_real(fconst, fc));
    CK(up_real(capmod, cm));
    CK(cudaMemsetAsync(m.F, 0, v4 * nn, s->stream));
    CK(cudaMemsetAsync(m.u, 0, v4 * nn, s->stream));
    m.adj_off = (const int *)adj_off;
    m.adj = (const int *)adj;
    m.adj4 = (const int *)adj4;
    m.node_cap = (const int *)node_cap;
    m.tri = (const int *)tri4;
    m.fconst = fconst;
    m.capmod = capmod;
    s->mesh = m;
    // positions
    {
        int rc = ensure_scratch(s, sizeof(double) * 3 * std::max(nn, 1));
        if (rc) return rc;
        CK(cudaMemcpyAsync(s->d_scratch, xcur.data(), sizeof(double) * 3 * nn, cudaMemcpyHostToDevice,
                           s->stream));
        launch_f64_to_nodes(s->prec, s->mesh, 0, nn, s->d_scratch, s->stream);
        CK(cudaGetLastError());
    }
    // Taylor plan: one block per capsule
    {
        std::vector<int> cf0(nc + 1, 0);
        std::vector<double> org(3 * (size_t)nc);
        int maxf = 1;
        for (int c = 0; c < nc; ++c) {
            const Capsule &cp = s->caps[c];
            cf0[c] = cp.face0;
            maxf = std::max(maxf, cp.n_faces);
            for (int k = 0; k < 3; ++k) org[3 * c + k] = cp.origin[k];
        }
        cf0[nc] = nf;
        auto P = [&](size_t bytes) {
            void *p = dev_alloc(s, bytes);
            if (p) s->plan_allocs.push_back(p);
            return p;
        };
        TaylorPlan p{};
        p.n_caps = nc;
        p.cluster = taylor_cluster_size(maxf, taylor_max_cluster(), nc);
        p.cap_face0 = (const int *)P(sizeof(int) * (nc + 1));
        p.origin = (const double *)P(sizeof(double) * 3 * nc);
        p.out = (double *)P(sizeof(double) * 12 * nc);
        p.ticket = (unsigned *)P(sizeof(unsigned));
        if (!p.cap_face0 || !p.origin || !p.out || !p.ticket)
            return fail(s, IBLBM_ERR_OOM, "Taylor plan allocation failed");
        CK(cudaMemsetAsync(p.ticket, 0, sizeof(unsigned), s->stream));
        CK(cudaMemcpyAsync((void *)p.cap_face0, cf0.data(), sizeof(int) * (nc + 1), cudaMemcpyHostToDevice,
                           s->stream));
        CK(cudaMemcpyAsync((void *)p.origin, org.data(), sizeof(double) * 3 * nc, cudaMemcpyHostToDevice, s->stream));
        s->plan = p;
    }
    CK(cudaStreamSynchronize(s->stream));
    s->dev_nodes = nn;
    s->x_pending.clear();
    s->mesh_dirty = false;
    s->ab2_ready = false;
    return IBLBM_OK;
}

int graph_len_for(const iblbm_sim *s) {
    const int e = s->rec_every;
    if (e <= 0) return kGraphSteps;
    int g = e * ((kGraphSteps + e - 1) / e);
    if (g % 2) g *= 2;  // keep the buffer parity of a replay unchanged
    return g;
}

bool record_after(const iblbm_sim *s, int64_t step_index) {
    return s->rec_every > 0 && s->d_ring && (step_index + 1) % s->rec_every == 0;
}

int ensure_ring(iblbm_sim *s) {
    if (s->rec_every <= 0 || s->d_ring || s->caps.empty()) return IBLBM_OK;
    s->d_ring = (double *)dev_alloc(s, sizeof(double) * 12 * s->caps.size() * (size_t)s->rec_ring);
    s->d_ring_count = (unsigned long long *)dev_alloc(s, sizeof(unsigned long long));
    if (!s->d_ring || !s->d_ring_count) {
        dev_free(s, s->d_ring);
        dev_free(s, s->d_ring_count);
        s->d_ring = nullptr;
        s->d_ring_count = nullptr;
        return fail(s, IBLBM_ERR_OOM, "record ring allocation failed");
    }
    CK(cudaMemsetAsync(s->d_ring_count, 0, sizeof(unsigned long long), s->stream));
    s->rec_steps.clear();
    s->plan.ring = s->d_ring;
    s->plan.ring_len = s->rec_ring;
    s->plan.ring_count = s->d_ring_count;
    return IBLBM_OK;
}

void free_ring(iblbm_sim *s) {
    dev_free(s, s->d_ring);
    dev_free(s, s->d_ring_count);
    s->d_ring = nullptr;
    s->d_ring_count = nullptr;
    s->plan.ring = nullptr;
    s->plan.ring_count = nullptr;
    s->rec_steps.clear();
}

// Whether the interpolation reads velocities formed once per cell of the
// flagged tiles: automatic when the stencils touch (counting repeats) more than
// a quarter of the cells, i.e. in dense suspensions.
// Programmatic dependent launch of the step kernels: automatically where the
// membrane kernels take four nodes per warp (a dense suspension, whose
// interpolation has a long position-only prologue); measured slower or no
// faster for one capsule.
bool launch_overlap(const iblbm_sim *s) {
    if (s->overlap >= 0) return s->overlap == 1;
    return s->mesh.n_nodes >= 152 * 32;
}

// Whether the single-lattice collide stages its populations in shared memory
// by bulk copies: only on request (mode 1).  Measured on the 256x128x128
// FP16 and 128^3 FP32 lattices the staged kernel is slower than direct loads
// (86.7 vs 72.1 us and 54.0 vs 46.6 us per launch): with every warp of a block
// computing the same tile and meeting at its barriers, the issue slots idle
// that the direct kernel's independent blocks fill.
bool collide_staged(const iblbm_sim *s) {
    if (s->batch || !collide_staging_supported(s->prec, s->L)) return false;
    return s->staging == 1;
}

bool cell_velocity_first(const iblbm_sim *s) {
    if (s->interp_mode >= 0) return s->interp_mode == 1;
    const double touches = (double)s->mesh.n_nodes * s->delta * s->delta * s->delta;
    const double cells = s->batch ? (double)(s->vec_bytes / (4 * real_bytes(s))) : (double)s->L.ncell;
    return touches > 0.25 * cells;
}

// One time step (sub-step list of Sec. II.C) enqueued on the stream, with an
// optional record of the capsule reductions (sub-step 6) at its end.  With
// `ev` non-null, events are recorded around each kernel group:
// ev[0] | spread | ev[1] | collide | ev[2] | cell velocities, interpolate | ev[3] | reductions | ev[4],
// the reductions then running on the main stream (profile mode).  With
// `graph_ev` non-null instead (a step captured for kernel timing), the four
// events ev[0..3] become event nodes of the graph and the record keeps its
// place on the side stream.
void enqueue_step(iblbm_sim *s, bool record = false, cudaEvent_t *ev = nullptr, cudaEvent_t *graph_ev = nullptr) {
    const int c = s->cur, n = 1 - s->cur;
    const bool det = s->d_fix != nullptr && !s->batch;
    auto mark = [s](const char *what) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess && !s->launch_fail) s->launch_fail = what;
    };
    auto gmark = [s, graph_ev](int k) {
        if (!graph_ev) return;
        cudaEventRecord(s->ev_tfork, s->stream);
        cudaStreamWaitEvent(s->tstream, s->ev_tfork, 0);
        cudaEventRecordWithFlags(graph_ev[k], s->tstream, cudaEventRecordExternal);
    };
    const bool ov = launch_overlap(s);
    if (ev) cudaEventRecord(ev[0], s->stream);
    gmark(0);
    nvtxRangePushA("membrane force + spreading");
    launch_force_spread(s->prec, s->delta, s->L, s->mesh, s->force[n], s->flags[n], s->d_status,
                        s->batch ? s->d_runs : nullptr, s->d_node_run, s->stream, ov, det ? s->d_fix : nullptr);
    if (det && s->mesh.n_nodes > 0)
        launch_fix_to_force(s->prec, s->L, s->d_fix, s->force[n], s->flags[n], s->stream, ov);
    mark("membrane force + spreading");
    nvtxRangePop();
    if (ev) cudaEventRecord(ev[1], s->stream);
    gmark(1);
    nvtxRangePushA("collide-stream");
    CollideArgs a;
    a.src = s->pop[c];
    a.dst = s->pop[n];
    a.fcur = s->force[n];
    a.flag_cur = s->flags[n];
    a.fold = s->force[c];
    a.flag_old = s->flags[c];
    a.tau = s->tau;
    a.u_wall = s->u_wall;
    a.status = s->d_status;
    a.eq_order = s->eq_order;
    a.staged = collide_staged(s);
    a.wait_ns = s->wait_ns;
    if (s->batch) {
        BatchArgs b{s->d_runs, s->d_items, s->n_items, s->batch_grid, s->batch_pairs};
        launch_collide_batch(s->prec, b, a, s->stream, ov);
    } else {
        launch_collide_stream(s->prec, s->L, a, s->stream, ov);
    }
    mark("collide-stream");
    nvtxRangePop();
    if (ev) cudaEventRecord(ev[2], s->stream);
    gmark(2);
    nvtxRangePushA("interpolation + advection");
    const bool pre = cell_velocity_first(s);
    if (pre) {
        launch_flag_velocity(s->prec, s->L, s->pop[n], s->force[n], s->flags[n], s->uvel,
                             s->batch ? s->d_runs : nullptr, s->d_items, s->n_items, s->stream, ov);
        mark("velocity of the flagged cells");
    }
    const bool side_rec = record && !ev;  // timed runs keep the record on the main stream
    const int h = s->rec_half;
    if (side_rec && s->rec_fill == 0 && s->side_pending[h]) {  // the half's last batch still reads it
        cudaStreamWaitEvent(s->stream, s->ev_join[h], 0);
        s->side_pending[h] = false;
        mark("join of the Taylor record");
    }
    const size_t slot = (size_t)h * s->rec_batch + s->rec_fill;
    const size_t v4 = 4 * real_bytes(s) * (size_t)s->mesh.n_nodes;
    void *sx = side_rec ? (char *)s->snap_x + slot * v4 : nullptr;
    void *sl = side_rec && s->snap_lo ? (char *)s->snap_lo + slot * (size_t)16 * s->mesh.n_nodes : nullptr;
    launch_interp_advect(s->prec, s->delta, s->L, s->mesh, pre ? s->uvel : nullptr, s->pop[n], s->force[n],
                         s->batch ? s->d_runs : nullptr, s->d_node_run, s->stream, sx, sl,
                         s->integrator == 1 && s->ab2_ready ? 1 : 0, ov);
    s->ab2_ready = true;  // m.u now holds u_i(t+1)
    mark("interpolation + advection");
    nvtxRangePop();
    if (ev) cudaEventRecord(ev[3], s->stream);
    gmark(3);
    if (record) {
        if (ev) {
            launch_taylor(s->prec, s->mesh, s->plan, true, s->stream);
        } else if (++s->rec_fill == s->rec_batch) {
            reduce_snapshots(s);
        }
        mark("Taylor record");
    }
    if (ev) cudaEventRecord(ev[4], s->stream);
    s->launches += 3 + (det && s->mesh.n_nodes > 0 ? 1 : 0) + (pre ? 1 : 0) + (record && ev ? 1 : 0);
    s->cur = n;
}

// Reduces the snapshots of the half being filled on the side stream (one
// launch) and moves on to the other half.
void reduce_snapshots(iblbm_sim *s) {
    const int h = s->rec_half;
    if (s->rec_fill > 0) {
        cudaEventRecord(s->ev_fork, s->stream);
        cudaStreamWaitEvent(s->side, s->ev_fork, 0);
        launch_taylor_snapshots(s->prec, s->mesh, s->plan, true, s->snap_x, s->snap_lo, h * s->rec_batch,
                                2 * s->rec_batch, s->rec_fill, s->side);
        s->launches += 1;
        cudaEventRecord(s->ev_join[h], s->side);
        s->side_pending[h] = true;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess && !s->launch_fail) s->launch_fail = "Taylor record";
    }
    s->rec_half = 1 - h;
    s->rec_fill = 0;
}

// Reduces any snapshots not yet reduced and makes the main stream wait for
// the outstanding Taylor records.
void join_side(iblbm_sim *s) {
    if (s->rec_fill > 0) reduce_snapshots(s);
    for (int b = 0; b < 2; ++b)
        if (s->side_pending[b]) {
            cudaStreamWaitEvent(s->stream, s->ev_join[b], 0);
            s->side_pending[b] = false;
        }
}

int check_sim(const iblbm_sim *s) { return s ? IBLBM_OK : IBLBM_ERR_ARG; }

int status_from_bits(int bits) {
    if (bits & 9) return IBLBM_ERR_UNSTABLE;
    if (bits & 2) return IBLBM_ERR_STENCIL;
    if (bits & 4) return IBLBM_ERR_TIMEOUT;
    return IBLBM_OK;
}

const char *status_message(int rc) {
    switch (rc) {
        case IBLBM_ERR_UNSTABLE: return "density left (0.5, 2) or became non-finite";
        case IBLBM_ERR_STENCIL: return "an IBM stencil cell lies beyond a wall (z < 0 or z >= nz)";
        default: return "a device wait for staged populations gave up (results of that step are incomplete)";
    }
}

int sync_status(iblbm_sim *s) {
    CK(cudaSetDevice(s->device));
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    if (s->rstream) CK(cudaStreamSynchronize(s->rstream));  // iblbm_read_async's copies
    int bits = 0;
    CK(cudaMemcpy(&bits, s->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (bits) {
        CK(cudaMemset(s->d_status, 0, sizeof(int)));
        int rc = status_from_bits(bits);
        if (!(bits & 1) && (bits & 8))
            return fail(s, rc, "a spread force contribution left the fixed-point range of the deterministic spreading");
        return fail(s, rc, status_message(rc));
    }
    return IBLBM_OK;
}

int capsule_range(iblbm_sim *s, int id, int *first, int *count) {
    if (id == -1) {
        *first = 0;
        *count = (int)(s->X0.size() / 3);
        return IBLBM_OK;
    }
    if (id < 0 || id >= (int)s->caps.size()) return fail(s, IBLBM_ERR_ARG, "no such capsule");
    *first = s->caps[id].node0;
    *count = s->caps[id].n_nodes;
    return IBLBM_OK;
}

int add_capsule(iblbm_sim *s, int run, const double *xyz, int n_nodes, const int *tri, int n_tri,
                int *id) {
    if (n_nodes < 4 || n_tri < 4 || !xyz || !tri) return fail(s, IBLBM_ERR_ARG, "bad mesh arguments");
    if (run < 0 || run >= (s->batch ? (int)s->runs.size() : 1)) return fail(s, IBLBM_ERR_ARG, "no such run");
    for (int k = 0; k < 3 * n_tri; ++k)
        if (tri[k] < 0 || tri[k] >= n_nodes) return fail(s, IBLBM_ERR_ARG, "face index out of range");
    for (int k = 0; k < 3 * n_nodes; ++k)
        if (!std::isfinite(xyz[k])) return fail(s, IBLBM_ERR_ARG, "non-finite node coordinate");
    Capsule c{};
    c.node0 = (int)(s->X0.size() / 3);
    c.n_nodes = n_nodes;
    c.face0 = (int)(s->tri.size() / 3);
    c.n_faces = n_tri;
    c.run = run;
    c.ks = 0.0;
    c.ka = 0.0;
    for (int k = 0; k < 3; ++k) {
        double m = 0.0;
        for (int n = 0; n < n_nodes; ++n) m += xyz[3 * n + k];
        c.origin[k] = m / n_nodes;
    }
    s->X0.insert(s->X0.end(), xyz, xyz + 3 * (size_t)n_nodes);
    for (int k = 0; k < 3 * n_tri; ++k) s->tri.push_back(tri[k] + c.node0);
    s->caps.push_back(c);
    s->mesh_dirty = true;
    if (id) *id = (int)s->caps.size() - 1;
    return IBLBM_OK;
}

}  // namespace

extern "C" {

const char *iblbm_status_string(int status) {
    switch (status) {
        case IBLBM_OK: return "IBLBM_OK";
        case IBLBM_ERR_ARG: return "IBLBM_ERR_ARG";
        case IBLBM_ERR_OOM: return "IBLBM_ERR_OOM";
        case IBLBM_ERR_CUDA: return "IBLBM_ERR_CUDA";
        case IBLBM_ERR_UNSTABLE: return "IBLBM_ERR_UNSTABLE";
        case IBLBM_ERR_STENCIL: return "IBLBM_ERR_STENCIL";
        case IBLBM_ERR_TIMEOUT: return "IBLBM_ERR_TIMEOUT";
        case IBLBM_ERR_STATE: return "IBLBM_ERR_STATE";
        default: return "IBLBM_ERR_UNKNOWN";
    }
}

const char *iblbm_last_error(const iblbm_sim *s) {
    return s ? s->err.c_str() : g_create_error.c_str();
}

}  // extern "C"

namespace {

// Streams, events and the state buffers for `cells` lattice cells and
// `tiles` force flags; zeroes forces, flags and the status word.
int setup_object(iblbm_sim *s, void *stream, const iblbm_allocator *alloc, long long cells,
                 long long tiles) {
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "no CUDA device";
        return IBLBM_ERR_CUDA;
    }
    if (alloc) {
        s->alloc = *alloc;
        s->has_alloc = true;
    }
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            g_create_error = "cudaStreamCreate failed";
            return IBLBM_ERR_CUDA;
        }
        s->own_stream = true;
    }
    // The Taylor record runs beside the next step's spreading and collide; at
    // the highest priority its few blocks start at once instead of queueing
    // behind the collide's, so the interpolation that joins it does not wait.
    int least_prio = 0, greatest_prio = 0;
    cudaDeviceGetStreamPriorityRange(&least_prio, &greatest_prio);
    if (cudaStreamCreateWithPriority(&s->side, cudaStreamNonBlocking, greatest_prio) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_join[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_join[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->tstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_tfork, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s->rstream, cudaStreamNonBlocking, least_prio) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_rsnap[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_rsnap[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_rdone[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_rdone[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "stream or event creation failed";
        return IBLBM_ERR_CUDA;
    }
    const size_t el = s->prec == kF64 ? 8 : (s->prec == kF32 ? 4 : 2);
    s->pop_bytes = 19 * el * (size_t)cells;
    s->vec_bytes = 4 * real_bytes(s) * (size_t)cells;
    s->flag_bytes = (size_t)tiles;
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) {
        s->pop[k] = dev_alloc(s, s->pop_bytes);
        s->force[k] = dev_alloc(s, s->vec_bytes);
        s->flags[k] = (uint8_t *)dev_alloc(s, s->flag_bytes);
        ok = s->pop[k] && s->force[k] && s->flags[k];
    }
    s->d_status = (int *)dev_alloc(s, sizeof(int));
    s->uvel = dev_alloc(s, s->vec_bytes);
    if (!ok || !s->d_status || !s->uvel) {
        g_create_error = "device allocation failed";
        return IBLBM_ERR_OOM;
    }
    for (int k = 0; k < 2; ++k) {
        cudaMemsetAsync(s->force[k], 0, s->vec_bytes, s->stream);
        cudaMemsetAsync(s->flags[k], 0, s->flag_bytes, s->stream);
    }
    cudaMemsetAsync(s->d_status, 0, sizeof(int), s->stream);
    return IBLBM_OK;
}

int finish_create(iblbm_sim *s, iblbm_sim **out) {
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_create_error = std::string("initialisation failed: ") + cudaGetErrorString(e);
        iblbm_destroy(s);
        return IBLBM_ERR_CUDA;
    }
    *out = s;
    return IBLBM_OK;
}

// Lattice of one run and the byte offsets of its populations and forces.
Lattice run_lattice(const iblbm_sim *s, int run, size_t *pop_off, size_t *vec_off) {
    if (!s->batch) {
        *pop_off = 0;
        *vec_off = 0;
        return s->L;
    }
    const RunDesc &R = s->runs[run];
    const size_t el = s->prec == kF64 ? 8 : (s->prec == kF32 ? 4 : 2);
    *pop_off = 19 * el * (size_t)R.cell_off;
    *vec_off = 4 * real_bytes(s) * (size_t)R.cell_off;
    return make_lattice(R.nx, R.ny, R.nz, false);
}

// (Re)builds the work list of the batched collide kernel and uploads the run
// table; flag regions of the runs are fixed (reserved for the largest tile
// count of any tile shape).
int upload_batch_tables(iblbm_sim *s) {
    std::vector<int2> items;
    long long off = 0;
    for (size_t r = 0; r < s->runs.size(); ++r) {
        RunDesc &R = s->runs[r];
        R.ntx = (R.nx + R.tx - 1) / R.tx;
        R.nty = (R.ny + R.ty - 1) / R.ty;
        R.tile_off = off;
        off += s->run_tile_cap[r];
        const int nt = R.ntx * R.nty * R.nz;
        for (int t = 0; t < nt; ++t) items.push_back(make_int2((int)r, t));
    }
    dev_free(s, s->d_runs);
    dev_free(s, s->d_items);
    s->d_runs = (RunDesc *)dev_alloc(s, sizeof(RunDesc) * s->runs.size());
    s->d_items = (int2 *)dev_alloc(s, sizeof(int2) * items.size());
    if (!s->d_runs || !s->d_items) {
        // no tables at all rather than half of them: the steps refuse to run
        dev_free(s, s->d_runs);
        dev_free(s, s->d_items);
        s->d_runs = nullptr;
        s->d_items = nullptr;
        s->n_items = 0;
        return fail(s, IBLBM_ERR_OOM, "run table allocation failed");
    }
    CK(cudaMemcpyAsync(s->d_runs, s->runs.data(), sizeof(RunDesc) * s->runs.size(),
                       cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->n_items = (int)items.size();
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    s->batch_pairs = s->prec != kF64;
    for (const RunDesc &R : s->runs) s->batch_pairs = s->batch_pairs && R.nx % 2 == 0;
    const long long want = (long long)sms * collide_batch_blocks_per_sm(s->prec, s->batch_pairs);
    s->batch_grid = (int)std::max(1LL, std::min<long long>(want, s->n_items));
    drop_graphs(s);
    return IBLBM_OK;
}

}  // namespace

extern "C" {

int iblbm_create(iblbm_sim **out, int nx, int ny, int nz, double tau, int precision,
                 int delta_points, void *stream, const iblbm_allocator *alloc) {
    if (!out) return IBLBM_ERR_ARG;
    *out = nullptr;
    g_create_error.clear();
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > 2147483647LL) {
        g_create_error = "lattice dimensions out of range";
        return IBLBM_ERR_ARG;
    }
    if (!(tau > 0.5) || !std::isfinite(tau)) {
        g_create_error = "tau must exceed 1/2";
        return IBLBM_ERR_ARG;
    }
    if (precision < 0 || precision > 2 || delta_points < 2 || delta_points > 4) {
        g_create_error = "precision must be 0..2 and delta_points 2..4";
        return IBLBM_ERR_ARG;
    }
    if (alloc && (!alloc->alloc || !alloc->free)) {
        g_create_error = "allocator needs both alloc and free";
        return IBLBM_ERR_ARG;
    }
    iblbm_sim *s = new (std::nothrow) iblbm_sim();
    if (!s) return IBLBM_ERR_OOM;
    s->L = make_lattice(nx, ny, nz, precision != kF64);
    s->prec = precision;
    s->delta = delta_points;
    s->tau = tau;
    int rc = setup_object(s, stream, alloc, s->L.ncell, s->L.ntiles);
    if (rc) {
        iblbm_destroy(s);
        return rc;
    }
    launch_init_fluid(s->prec, s->L, s->pop[0], 0, 0.0, s->stream);
    return finish_create(s, out);
}

int iblbm_batch_create(iblbm_sim **out, const iblbm_run_spec *specs, int n_runs, int precision,
                       int delta_points, void *stream, const iblbm_allocator *alloc) {
    if (!out) return IBLBM_ERR_ARG;
    *out = nullptr;
    g_create_error.clear();
    if (!specs || n_runs < 1 || n_runs > (1 << 20)) {
        g_create_error = "need 1 <= n_runs <= 2^20 run specifications";
        return IBLBM_ERR_ARG;
    }
    if (precision < 0 || precision > 2 || delta_points < 2 || delta_points > 4) {
        g_create_error = "precision must be 0..2 and delta_points 2..4";
        return IBLBM_ERR_ARG;
    }
    if (alloc && (!alloc->alloc || !alloc->free)) {
        g_create_error = "allocator needs both alloc and free";
        return IBLBM_ERR_ARG;
    }
    long long cells = 0, tiles = 0;
    for (int r = 0; r < n_runs; ++r) {
        const iblbm_run_spec &q = specs[r];
        if (q.nx < 1 || q.ny < 1 || q.nz < 1 || !(q.tau > 0.5) || !std::isfinite(q.tau) ||
            !std::isfinite(q.u_wall) || std::fabs(q.u_wall) > 0.3) {
            g_create_error = "run " + std::to_string(r) + ": bad size, tau or wall speed";
            return IBLBM_ERR_ARG;
        }
        cells += (long long)q.nx * q.ny * q.nz;
    }
    if (cells > 2147483647LL) {
        g_create_error = "more than 2^31 - 1 cells in the batch";
        return IBLBM_ERR_ARG;
    }
    iblbm_sim *s = new (std::nothrow) iblbm_sim();
    if (!s) return IBLBM_ERR_OOM;
    s->batch = true;
    s->prec = precision;
    s->delta = delta_points;
    s->tau = specs[0].tau;
    s->u_wall = specs[0].u_wall;
    long long off = 0;
    for (int r = 0; r < n_runs; ++r) {
        const iblbm_run_spec &q = specs[r];
        RunDesc R{};
        R.nx = q.nx;
        R.ny = q.ny;
        R.nz = q.nz;
        R.tx = 32;
        R.ty = 8;
        R.cell_off = off;
        R.ncell = (long long)q.nx * q.ny * q.nz;
        R.omega = 1.0 / q.tau;
        R.u_wall = q.u_wall;
        off += R.ncell;
        long long cap = 0;
        for (const auto &sh : kTileShapes)
            cap = std::max(cap, (long long)((q.nx + sh[0] - 1) / sh[0]) * ((q.ny + sh[1] - 1) / sh[1]) * q.nz);
        s->run_tile_cap.push_back(cap);
        tiles += cap;
        s->runs.push_back(R);
    }
    s->L = make_lattice(specs[0].nx, specs[0].ny, specs[0].nz, false);
    int rc = setup_object(s, stream, alloc, cells, tiles);
    if (!rc) rc = upload_batch_tables(s);
    if (rc) {
        if (!s->err.empty()) g_create_error = s->err;
        iblbm_destroy(s);
        return rc;
    }
    for (int r = 0; r < n_runs; ++r) {
        size_t po, vo;
        const Lattice Lr = run_lattice(s, r, &po, &vo);
        launch_init_fluid(s->prec, Lr, (char *)s->pop[0] + po, 0, 0.0, s->stream);
    }
    return finish_create(s, out);
}

int iblbm_destroy(iblbm_sim *s) {
    if (is_group(s)) {
        cudaStreamSynchronize(s->stream);
        for (iblbm_sim *p : s->slabs) iblbm_destroy(p);
        dev_free(s, s->slab_planes);
        dev_free(s, s->slab_parts);
        dev_free(s, s->slab_part_ptrs);
        if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
        delete s;
        return IBLBM_OK;
    }
    if (!s) return IBLBM_OK;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->side) cudaStreamSynchronize(s->side);
    if (s->rstream) cudaStreamSynchronize(s->rstream);
    drop_graphs(s);
    for (int k = 0; k < 2; ++k) {
        dev_free(s, s->pop[k]);
        dev_free(s, s->force[k]);
        dev_free(s, s->flags[k]);
    }
    dev_free(s, s->d_status);
    dev_free(s, s->d_fix);
    dev_free(s, s->uvel);
    free_readback(s);
    dev_free(s, s->d_scratch);
    dev_free(s, s->d_cksum);
    dev_free(s, s->slab_planes);
    dev_free(s, s->slab_parts);
    dev_free(s, s->slab_part_ptrs);
    dev_free(s, s->d_runs);
    dev_free(s, s->d_items);
    adj_free(s);
    free_ring(s);
    for (void *p : s->mesh_allocs) dev_free(s, p);
    for (void *p : s->plan_allocs) dev_free(s, p);
    if (s->side) {
        cudaStreamSynchronize(s->side);
        cudaStreamDestroy(s->side);
    }
    if (s->tstream) {
        cudaStreamSynchronize(s->tstream);
        cudaStreamDestroy(s->tstream);
    }
    if (s->rstream) cudaStreamDestroy(s->rstream);
    for (int k = 0; k < 2; ++k) {
        if (s->ev_rsnap[k]) cudaEventDestroy(s->ev_rsnap[k]);
        if (s->ev_rdone[k]) cudaEventDestroy(s->ev_rdone[k]);
    }
    if (s->ev_tfork) cudaEventDestroy(s->ev_tfork);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    for (cudaEvent_t e : s->ev_join)
        if (e) cudaEventDestroy(e);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return IBLBM_OK;
}

int iblbm_get_info(const iblbm_sim *s, iblbm_info *out) {
    if (!s || !out) return IBLBM_ERR_ARG;
    if (is_group(s)) {
        int rc = iblbm_get_info(s->slabs[0], out);
        out->nx = s->L.nx;
        out->step = s->steps;
        int64_t launches = 0;
        for (const iblbm_sim *p : s->slabs) launches += p->launches;
        out->kernel_launches = launches;
        return rc;
    }
    out->nx = s->L.nx;
    out->ny = s->L.ny;
    out->nz = s->L.nz;
    out->precision = s->prec;
    out->delta_points = s->delta;
    out->n_capsules = (int)s->caps.size();
    out->n_nodes = (int)(s->X0.size() / 3);
    out->n_faces = (int)(s->tri.size() / 3);
    out->step = s->steps;
    out->n_runs = s->batch ? (int)s->runs.size() : 1;
    out->tau = s->tau;
    out->u_wall = s->u_wall;
    out->kernel_launches = s->launches;
    return IBLBM_OK;
}

int iblbm_set_shear_walls(iblbm_sim *s, double u_wall) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) {
        for (iblbm_sim *p : s->slabs) {
            int rc = iblbm_set_shear_walls(p, u_wall);
            if (rc) return fail(s, rc, p->err);
        }
        s->u_wall = u_wall;
        return IBLBM_OK;
    }
    if (!std::isfinite(u_wall) || std::fabs(u_wall) > 0.3)
        return fail(s, IBLBM_ERR_ARG, "wall speed must be finite and |u_wall| <= 0.3");
    s->u_wall = u_wall;
    drop_graphs(s);
    if (s->batch) {  // every run of a batch
        for (RunDesc &R : s->runs) R.u_wall = u_wall;
        CK(cudaSetDevice(s->device));
        join_side(s);
        CK(cudaStreamSynchronize(s->stream));
        return upload_batch_tables(s);
    }
    return IBLBM_OK;
}

int iblbm_add_capsule_icosphere(iblbm_sim *s, double cx, double cy, double cz, double radius,
                                int subdivisions, int *capsule_id) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) {  // the membranes are replicated on every slab
        for (iblbm_sim *p : s->slabs) {
            int rc = iblbm_add_capsule_icosphere(p, cx, cy, cz, radius, subdivisions, capsule_id);
            if (rc) return fail(s, rc, p->err);
        }
        return IBLBM_OK;
    }
    if (subdivisions < 0 || subdivisions > 7 || !(radius > 0.0) || !std::isfinite(radius))
        return fail(s, IBLBM_ERR_ARG, "subdivisions must be 0..7 and radius positive");
    std::vector<double> nodes;
    std::vector<int> tri;
    const double c[3] = {cx, cy, cz};
    icosphere(subdivisions, radius, c, nodes, tri);
    return add_capsule(s, 0, nodes.data(), (int)(nodes.size() / 3), tri.data(), (int)(tri.size() / 3),
                       capsule_id);
}

int iblbm_icosphere(int subdivisions, double radius, const double center[3], double *nodes_out,
                    int32_t *tri_out) {
    if (subdivisions < 0 || subdivisions > 7 || !(radius > 0.0) || !std::isfinite(radius) || !center)
        return IBLBM_ERR_ARG;
    std::vector<double> nodes;
    std::vector<int> tri;
    icosphere(subdivisions, radius, center, nodes, tri);
    if (nodes_out) std::memcpy(nodes_out, nodes.data(), sizeof(double) * nodes.size());
    if (tri_out)
        for (size_t k = 0; k < tri.size(); ++k) tri_out[k] = tri[k];
    return IBLBM_OK;
}

int iblbm_taylor_gradient(const double *nodes, int n_nodes, const int32_t *tri, int n_tri,
                          double *D_out, double *dD_dx) {
    if (!nodes || !tri || !D_out || n_nodes < 4 || n_tri < 4) return IBLBM_ERR_ARG;
    for (int k = 0; k < 3 * n_tri; ++k)
        if (tri[k] < 0 || tri[k] >= n_nodes) return IBLBM_ERR_ARG;
    *D_out = taylor_D_and_gradient(nodes, n_nodes, (const int *)tri, n_tri, dD_dx);
    return std::isfinite(*D_out) ? IBLBM_OK : IBLBM_ERR_ARG;
}

int iblbm_add_capsule_mesh(iblbm_sim *s, const double *ref_xyz, int n_nodes, const int32_t *tri,
                           int n_tri, int *capsule_id) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) {
        for (iblbm_sim *p : s->slabs) {
            int rc = iblbm_add_capsule_mesh(p, ref_xyz, n_nodes, tri, n_tri, capsule_id);
            if (rc) return fail(s, rc, p->err);
        }
        return IBLBM_OK;
    }
    return add_capsule(s, 0, ref_xyz, n_nodes, (const int *)tri, n_tri, capsule_id);
}

int iblbm_set_skalak(iblbm_sim *s, int capsule_id, double k_s, double C) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) {
        for (iblbm_sim *p : s->slabs) {
            int rc = iblbm_set_skalak(p, capsule_id, k_s, C);
            if (rc) return fail(s, rc, p->err);
        }
        return IBLBM_OK;
    }
    if (!(k_s >= 0.0) || !(C >= 0.0) || !std::isfinite(k_s) || !std::isfinite(C))
        return fail(s, IBLBM_ERR_ARG, "moduli must be finite and non-negative");
    if (capsule_id < -1 || capsule_id >= (int)s->caps.size())
        return fail(s, IBLBM_ERR_ARG, "no such capsule");
    for (int c = 0; c < (int)s->caps.size(); ++c)
        if (capsule_id == -1 || capsule_id == c) {
            s->caps[c].ks = k_s;
            s->caps[c].ka = C * k_s;
        }
    if (s->mesh_dirty) return IBLBM_OK;  // uploaded with the tables
    CK(cudaSetDevice(s->device));
    const int nc = (int)s->caps.size();
    if (s->prec == kF64) {
        std::vector<double> cm(4 * (size_t)nc, 0.0);
        for (int c = 0; c < nc; ++c) {
            cm[4 * c] = s->caps[c].ks / 6.0;
            cm[4 * c + 1] = s->caps[c].ka / 6.0;
        }
        CK(cudaMemcpyAsync((void *)s->mesh.capmod, cm.data(), cm.size() * 8, cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    } else {
        std::vector<float> cm(4 * (size_t)nc, 0.0f);
        for (int c = 0; c < nc; ++c) {
            cm[4 * c] = (float)(s->caps[c].ks / 6.0);
            cm[4 * c + 1] = (float)(s->caps[c].ka / 6.0);
        }
        CK(cudaMemcpyAsync((void *)s->mesh.capmod, cm.data(), cm.size() * 4, cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    return IBLBM_OK;
}

int iblbm_init_fluid(iblbm_sim *s, int mode) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) {
        for (iblbm_sim *p : s->slabs) {
            int rc = iblbm_init_fluid(p, mode);
            if (rc) return fail(s, rc, p->err);
        }
        s->steps = 0;
        return IBLBM_OK;
    }
    if (mode != 0 && mode != 1) return fail(s, IBLBM_ERR_ARG, "mode must be 0 or 1");
    CK(cudaSetDevice(s->device));
    join_side(s);
    s->cur = 0;
    const int nr = s->batch ? (int)s->runs.size() : 1;
    for (int r = 0; r < nr; ++r) {
        size_t po, vo;
        const Lattice Lr = run_lattice(s, r, &po, &vo);
        const double uw = s->batch ? s->runs[r].u_wall : s->u_wall;
        launch_init_fluid(s->prec, Lr, (char *)s->pop[0] + po, mode, uw, s->stream);
    }
    for (int k = 0; k < 2; ++k) {
        CK(cudaMemsetAsync(s->force[k], 0, s->vec_bytes, s->stream));
        CK(cudaMemsetAsync(s->flags[k], 0, s->flag_bytes, s->stream));
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    s->steps = 0;
    s->init_mode = mode;
    if (s->d_ring) {
        CK(cudaMemset(s->d_ring_count, 0, sizeof(unsigned long long)));
        s->rec_steps.clear();
    }
    return IBLBM_OK;
}

}  // extern "C"

namespace {

// Step (0-based, within a captured sequence) of the first Taylor record of a
// sequence that starts `phase` steps into the recording period, or -1 when
// none of its `len` steps records.
int first_record(const iblbm_sim *s, int phase, int len) {
    if (s->rec_every <= 0 || !s->d_ring) return -1;
    const int k0 = (s->rec_every - 1 - phase % s->rec_every) % s->rec_every;
    return k0 < len ? k0 : -1;
}

// The captured sequence of `len` steps from buffer parity `cur` whose first
// record is at step first_rec, captured now if not cached.  Capturing runs
// nothing: the host state it touches (buffer parity, the Adams-Bashforth
// history flag, the snapshot ring) is put back, and only records still
// pending from earlier steps are reduced and joined first.
int step_graph(iblbm_sim *s, int len, int cur, int first_rec, iblbm_sim::StepGraph **out) {
    for (auto &g : s->sgraphs)
        if (g.len == len && g.cur == cur && g.first_rec == first_rec) {
            *out = &g;
            return IBLBM_OK;
        }
    if ((int)s->sgraphs.size() >= kMaxStepGraphs) {
        auto lru = std::min_element(s->sgraphs.begin(), s->sgraphs.end(),
                                    [](const iblbm_sim::StepGraph &a, const iblbm_sim::StepGraph &b) {
                                        return a.used < b.used;
                                    });
        CK(cudaStreamSynchronize(s->stream));  // its last replay may still run
        free_step_graph(*lru);
        s->sgraphs.erase(lru);
    }
    iblbm_sim::StepGraph g;
    g.len = len;
    g.cur = cur;
    g.first_rec = first_rec;
    if (s->kernel_timing) {
        g.ev.assign(4 * (size_t)len, nullptr);
        for (auto &e : g.ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) {
                free_step_graph(g);
                return cuda_fail(s, r, "timing event creation");
            }
        }
    }
    const int cur0 = s->cur;
    const bool ab2_0 = s->ab2_ready;
    join_side(s);  // the sequence starts with no record pending, at the first half
    s->rec_half = 0;
    s->rec_fill = 0;
    const int64_t launches0 = s->launches;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        free_step_graph(g);
        return cuda_fail(s, e, "graph capture");
    }
    s->cur = cur;
    s->ab2_ready = true;  // only captured with the history in place (or Euler)
    for (int k = 0; k < len; ++k) {
        const bool rec = first_rec >= 0 && k >= first_rec && (k - first_rec) % s->rec_every == 0;
        enqueue_step(s, rec, nullptr, g.ev.empty() ? nullptr : g.ev.data() + 4 * (size_t)k);
    }
    join_side(s);  // the sequence joins its own records before it ends
    if (!g.ev.empty()) {  // and its timing branch
        cudaEventRecord(s->ev_tfork, s->tstream);
        cudaStreamWaitEvent(s->stream, s->ev_tfork, 0);
    }
    e = cudaStreamEndCapture(s->stream, &graph);
    s->cur = cur0;
    s->ab2_ready = ab2_0;
    s->rec_half = 0;
    s->rec_fill = 0;
    g.kernels = s->launches - launches0;  // counted when replayed
    s->launches = launches0;
    if (e == cudaSuccess && s->launch_fail) e = cudaErrorLaunchFailure;
    if (e == cudaSuccess)
        // kernel nodes keep the priority of the stream they were captured on
        e = cudaGraphInstantiate(&g.exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    // the device copy of the graph is made now, not at its first launch (a
    // prepared call's first replay then costs what the others do)
    if (e == cudaSuccess) {
        e = cudaGraphUpload(g.exec, s->stream);
        if (e != cudaSuccess) cudaGraphExecDestroy(g.exec);
    }
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g.exec = nullptr;
        free_step_graph(g);
        if (s->launch_fail)
            return fail(s, IBLBM_ERR_CUDA, std::string("kernel launch failed in capture: ") + s->launch_fail);
        return cuda_fail(s, e, "graph capture");
    }
    s->sgraphs.push_back(std::move(g));
    *out = &s->sgraphs.back();
    return IBLBM_OK;
}

// Splits n steps from the current state into the pieces iblbm_step takes:
// a direct step while the Adams-Bashforth history is missing, then captured
// sequences -- up to the next start of the recording period, whole graphs of
// graph_len_for() steps, and the remainder.  With `run` false the sequences
// are only captured (iblbm_prepare_steps).
int run_steps(iblbm_sim *s, int64_t n_steps, bool run) {
    const int G = graph_len_for(s);
    if (G != s->graph_len) {
        drop_graphs(s);
        s->graph_len = G;
    }
    const int period = s->rec_every > 0 ? s->rec_every : 1;
    int cur = s->cur;
    int64_t steps = s->steps;
    bool ab2 = s->ab2_ready;
    int64_t left = n_steps;
    while (left > 0) {
        if (s->integrator == 1 && !ab2) {
            // the first Adams-Bashforth step takes Euler's rule, launched directly
            if (run) {
                const bool rec = record_after(s, s->steps);
                enqueue_step(s, rec);
                if (rec) s->rec_steps.push_back(s->steps + 1);
                s->steps++;
                if (s->launch_fail) break;
            }
            cur = 1 - cur;
            steps++;
            ab2 = true;
            left--;
            continue;
        }
        const int phase = (int)(steps % period);
        const int len = (int)std::min<int64_t>(left, phase ? period - phase : G);
        iblbm_sim::StepGraph *g = nullptr;
        int rc = step_graph(s, len, cur, first_record(s, phase, len), &g);
        if (rc) return rc;
        if (run) {
            join_side(s);
            CK(cudaGraphLaunch(g->exec, s->stream));
            g->used = ++s->graph_clock;
            g->timed = !g->ev.empty();
            s->launches += g->kernels;
            for (int k = 0; k < len; ++k)
                if (record_after(s, s->steps + k)) s->rec_steps.push_back(s->steps + k + 1);
            s->steps += len;
            s->cur = len % 2 ? 1 - s->cur : s->cur;
            s->ab2_ready = true;
        }
        cur = len % 2 ? 1 - cur : cur;
        steps += len;
        left -= len;
    }
    if (s->launch_fail)
        return fail(s, IBLBM_ERR_CUDA, std::string("kernel launch failed: ") + s->launch_fail);
    CK(cudaGetLastError());
    return IBLBM_OK;
}

// A batch whose run tables could not be (re)allocated has none: no step may run.
int batch_tables_ok(iblbm_sim *s) {
    if (s->batch && (!s->d_runs || !s->d_items))
        return fail(s, IBLBM_ERR_OOM, "the batch's run tables are missing (an allocation failed)");
    return IBLBM_OK;
}

int step_prologue(iblbm_sim *s, int64_t n_steps) {
    if (n_steps < 0) return fail(s, IBLBM_ERR_ARG, "negative step count");
    CK(cudaSetDevice(s->device));
    cudaGetLastError();  // an error left by some earlier, unrelated call is not ours
    int rc = batch_tables_ok(s);
    if (rc) return rc;
    rc = ensure_mesh(s);
    if (rc) return rc;
    rc = ensure_ring(s);
    if (rc) return rc;
    s->launch_fail = nullptr;
    return IBLBM_OK;
}

}  // namespace

extern "C" {

int iblbm_step(iblbm_sim *s, int64_t n_steps) {
    Range range("iblbm_step");
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) {
        if (n_steps < 0) return fail(s, IBLBM_ERR_ARG, "negative step count");
        return group_step(s, n_steps);
    }
    int rc = step_prologue(s, n_steps);
    return rc ? rc : run_steps(s, n_steps, true);
}

int iblbm_prepare_steps(iblbm_sim *s, int64_t n_steps) {
    Range range("iblbm_prepare_steps");
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    int rc = step_prologue(s, n_steps);
    return rc ? rc : run_steps(s, n_steps, false);
}

int iblbm_set_kernel_timing(iblbm_sim *s, int on) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    if (on != 0 && on != 1) return fail(s, IBLBM_ERR_ARG, "on must be 0 or 1");
    CK(cudaSetDevice(s->device));
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    drop_graphs(s);
    s->kernel_timing = on == 1;
    return IBLBM_OK;
}

int iblbm_get_kernel_times(iblbm_sim *s, double ms_out[3], int64_t *n_steps) {
    if (!s || !ms_out) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    int rc = sync_status(s);
    if (rc) return rc;
    double acc[3] = {0, 0, 0};
    int64_t n = 0;
    for (auto &g : s->sgraphs) {
        if (!g.timed) continue;
        for (int k = 0; k < g.len; ++k)
            for (int j = 0; j < 3; ++j) {
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, g.ev[4 * (size_t)k + j], g.ev[4 * (size_t)k + j + 1]));
                acc[j] += ms;
            }
        n += g.len;
        g.timed = false;
    }
    for (int j = 0; j < 3; ++j) ms_out[j] = n ? acc[j] / n : 0.0;
    if (n_steps) *n_steps = n;
    return IBLBM_OK;
}

const char *iblbm_collide_kernel(const iblbm_sim *s) {
    if (!s) return "";
    if (is_group(s)) return iblbm_collide_kernel(s->slabs[0]);
    if (s->batch) return collide_batch_kernel_name(s->prec, s->batch_pairs);
    return collide_kernel_name(s->prec, s->L, collide_staged(s));
}

int iblbm_set_collide_staging(iblbm_sim *s, int mode) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    if (mode < -1 || mode > 1) return fail(s, IBLBM_ERR_ARG, "mode must be -1, 0 or 1");
    if (mode == 1 && (s->batch || !collide_staging_supported(s->prec, s->L)))
        return fail(s, IBLBM_ERR_STATE,
                    "staged collide needs a single float or half lattice with nx/4 a power of two <= 256 and "
                    "nx times the element size a multiple of 16 bytes");
    CK(cudaSetDevice(s->device));
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    drop_graphs(s);
    s->staging = mode;
    return IBLBM_OK;
}

int iblbm_set_device_wait_limit(iblbm_sim *s, int64_t ns) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    if (ns < 0) return fail(s, IBLBM_ERR_ARG, "the limit must be >= 0 ns");
    CK(cudaSetDevice(s->device));
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    drop_graphs(s);
    s->wait_ns = (unsigned long long)ns;
    return IBLBM_OK;
}

}  // extern "C"

namespace {

void adj_drop_graphs(iblbm_sim *s) {
    for (auto &g : s->adj.graphs) cudaGraphExecDestroy(g.second);
    s->adj.graphs.clear();
}

void adj_free(iblbm_sim *s) {
    iblbm_sim::Adjoint &A = s->adj;
    if (A.rstream) cudaStreamSynchronize(A.rstream);
    adj_drop_graphs(s);
    for (void *p : A.allocs) dev_free(s, p);
    for (void *p : A.ck_allocs) dev_free(s, p);
    if (A.rstream) cudaStreamDestroy(A.rstream);
    for (cudaEvent_t e : {A.ev_start, A.ev_rec[0], A.ev_rec[1], A.ev_rev[0], A.ev_rev[1]})
        if (e) cudaEventDestroy(e);
    s->adj = iblbm_sim::Adjoint{};
}

void adj_free_checkpoints(iblbm_sim *s) {
    for (void *p : s->adj.ck_allocs) dev_free(s, p);
    s->adj.ck_allocs.clear();
    s->adj.ck_pop.clear();
    s->adj.ck_x.clear();
}

void *ck_alloc(iblbm_sim *s, size_t bytes) {
    void *p = dev_alloc(s, bytes);
    if (p) s->adj.ck_allocs.push_back(p);
    return p;
}

bool same_mesh(const MeshDev &a, const MeshDev &b) {
    return a.n_nodes == b.n_nodes && a.n_faces == b.n_faces && a.n_caps == b.n_caps && a.x == b.x &&
           a.x_lo == b.x_lo && a.F == b.F && a.u == b.u && a.adj_off == b.adj_off && a.adj == b.adj &&
           a.tri == b.tri && a.fconst == b.fconst && a.capmod == b.capmod;
}

void *adj_alloc(iblbm_sim *s, size_t bytes) {
    void *p = dev_alloc(s, bytes);
    if (p) s->adj.allocs.push_back(p);
    return p;
}

size_t pos_bytes(const iblbm_sim *s) { return (size_t)s->mesh.n_nodes * 32; }  // dvec4 or hi+lo float4
size_t nodevec_bytes(const iblbm_sim *s) { return (size_t)s->mesh.n_nodes * 4 * real_bytes(s); }

cudaError_t copy_pos_out(iblbm_sim *s, void *dst, cudaStream_t st = nullptr) {
    if (!st) st = s->stream;
    const size_t n = (size_t)s->mesh.n_nodes;
    if (s->prec == kF64) return cudaMemcpyAsync(dst, s->mesh.x, n * 32, cudaMemcpyDeviceToDevice, st);
    cudaError_t e = cudaMemcpyAsync(dst, s->mesh.x, n * 16, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((char *)dst + n * 16, s->mesh.x_lo, n * 16, cudaMemcpyDeviceToDevice, st);
    return e;
}

cudaError_t copy_pos_in(iblbm_sim *s, const void *src, cudaStream_t st = nullptr) {
    if (!st) st = s->stream;
    const size_t n = (size_t)s->mesh.n_nodes;
    if (s->prec == kF64) return cudaMemcpyAsync(s->mesh.x, src, n * 32, cudaMemcpyDeviceToDevice, st);
    cudaError_t e = cudaMemcpyAsync(s->mesh.x, src, n * 16, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->mesh.x_lo, (const char *)src + n * 16, n * 16, cudaMemcpyDeviceToDevice, st);
    return e;
}

}  // namespace

extern "C" {

int iblbm_adjoint_forward(iblbm_sim *s, int64_t n_steps, int checkpoint_every) {
    Range range("iblbm_adjoint_forward");
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    if (s->batch) return fail(s, IBLBM_ERR_STATE, "the adjoint works on a single lattice");
    if (s->caps.size() != 1) return fail(s, IBLBM_ERR_STATE, "the adjoint needs exactly one capsule");
    if (s->integrator != 0 || s->eq_order != 2)
        return fail(s, IBLBM_ERR_STATE, "the adjoint covers Euler advection and the full equilibrium only");
    if (n_steps < 1 || checkpoint_every < 1 || checkpoint_every > n_steps)
        return fail(s, IBLBM_ERR_ARG, "need n_steps >= 1 and 1 <= checkpoint_every <= n_steps");
    CK(cudaSetDevice(s->device));
    int rc = ensure_mesh(s);
    if (rc) return rc;
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    // the reverse-sweep buffers depend on K and on the mesh size only
    if (s->adj.K != checkpoint_every || !same_mesh(s->adj.graph_mesh, s->mesh)) adj_free(s);
    else adj_free_checkpoints(s);
    iblbm_sim::Adjoint &A = s->adj;
    A.ready = false;
    A.K = checkpoint_every;
    A.n = n_steps;
    A.t_start = s->steps;
    A.couette_start = (s->steps == 0 && s->init_mode == 1);
    const int64_t nck = (n_steps + A.K - 1) / A.K;
    for (int64_t c = 0; c < nck; ++c) {
        void *p = ck_alloc(s, s->pop_bytes), *x = ck_alloc(s, pos_bytes(s));
        if (!p || !x) {
            adj_free(s);
            return fail(s, IBLBM_ERR_OOM, "checkpoint allocation failed");
        }
        A.ck_pop.push_back(p);
        A.ck_x.push_back(x);
    }
    for (int64_t c = 0; c < nck; ++c) {
        CK(cudaMemcpyAsync(A.ck_pop[c], s->pop[s->cur], s->pop_bytes, cudaMemcpyDeviceToDevice, s->stream));
        CK(copy_pos_out(s, A.ck_x[c]));
        rc = iblbm_step(s, std::min<int64_t>(A.K, n_steps - c * A.K));
        if (rc) return rc;
    }
    rc = sync_status(s);
    if (rc) return rc;
    A.ready = true;
    return IBLBM_OK;
}

int iblbm_adjoint_backward(iblbm_sim *s, int capsule_id, double *D_out, double *dD_dks, double *dD_duw,
                           double *dD_dX0, double *dD_dx0) {
    Range range("iblbm_adjoint_backward");
    if (!s || !D_out) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    iblbm_sim::Adjoint &A = s->adj;
    if (!A.ready || s->steps != A.t_start + A.n || s->mesh_dirty)
        return fail(s, IBLBM_ERR_STATE, "run iblbm_adjoint_forward first, with no step since");
    if (capsule_id != 0) return fail(s, IBLBM_ERR_ARG, "no such capsule");
    CK(cudaSetDevice(s->device));
    int rc = sync_status(s);
    if (rc) return rc;
    const MeshDev &m = s->mesh;
    const int n = m.n_nodes, nf = m.n_faces;
    const size_t vb = 4 * real_bytes(s);
    const int K = A.K;
    // reverse-sweep buffers (kept for repeated backward passes)
    if (A.tr[0].M.empty()) {
        bool ok = true;
        for (auto &T : A.tr) {
            T.pop[0] = adj_alloc(s, s->pop_bytes);
            T.pop[1] = adj_alloc(s, s->pop_bytes);
            ok = ok && T.pop[0] && T.pop[1];
            for (int k = 0; k <= K && ok; ++k) {
                void *p = adj_alloc(s, 4 * real_bytes(s) * (size_t)s->L.ncell);
                ok = p != nullptr;
                T.M.push_back(p);
            }
            for (int k = 0; k < K && ok; ++k) {
                T.g.push_back(adj_alloc(s, s->vec_bytes));
                T.flags.push_back(adj_alloc(s, s->flag_bytes));
                T.x.push_back(adj_alloc(s, pos_bytes(s)));
                T.F.push_back(adj_alloc(s, nodevec_bytes(s)));
                ok = T.g.back() && T.flags.back() && T.x.back() && T.F.back();
            }
        }
        const size_t lb = 19 * real_bytes(s) * (size_t)s->L.ncell;
        for (int k = 0; k < 2 && ok; ++k) {
            A.lam[k] = adj_alloc(s, lb);
            A.lamx[k] = adj_alloc(s, nodevec_bytes(s));
            ok = A.lam[k] && A.lamx[k];
        }
        A.mu = adj_alloc(s, s->vec_bytes);
        A.lamg = adj_alloc(s, s->vec_bytes);
        A.lamF = adj_alloc(s, nodevec_bytes(s));
        A.fref = adj_alloc(s, 2 * vb * nf);
        A.zero_flags = (uint8_t *)adj_alloc(s, s->flag_bytes);
        A.uw_partial = (double *)adj_alloc(s, sizeof(double) * (size_t)((s->L.ncell + 255) / 256));
        A.gX0 = (double *)adj_alloc(s, sizeof(double) * 3 * n);
        A.gks = (double *)adj_alloc(s, sizeof(double) * n);
        // the final state is restored from these afterwards
        A.save_x = adj_alloc(s, pos_bytes(s));
        A.save_F = adj_alloc(s, nodevec_bytes(s));
        A.save_u = adj_alloc(s, nodevec_bytes(s));
        ok = ok && A.mu && A.lamg && A.lamF && A.fref && A.zero_flags && A.uw_partial && A.gX0 && A.gks &&
             A.save_x && A.save_F && A.save_u;
        if (!ok) {
            adj_free(s);
            return fail(s, IBLBM_ERR_OOM, "adjoint buffer allocation failed");
        }
        CK(cudaStreamCreateWithFlags(&A.rstream, cudaStreamNonBlocking));
        for (cudaEvent_t *e : {&A.ev_start, &A.ev_rec[0], &A.ev_rec[1], &A.ev_rev[0], &A.ev_rev[1]})
            CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        CK(cudaMemset(A.zero_flags, 0, s->flag_bytes));
        A.graph_mesh = m;
    }
    {
        // reference edges of every face
        std::vector<double> fr(8 * (size_t)nf, 0.0);
        for (int f = 0; f < nf; ++f) {
            const int a = s->tri[3 * f], b = s->tri[3 * f + 1], c = s->tri[3 * f + 2];
            for (int k = 0; k < 3; ++k) {
                fr[8 * f + k] = s->X0[3 * b + k] - s->X0[3 * a + k];
                fr[8 * f + 4 + k] = s->X0[3 * c + k] - s->X0[3 * a + k];
            }
        }
        if (s->prec == kF64) {
            CK(cudaMemcpy(A.fref, fr.data(), fr.size() * 8, cudaMemcpyHostToDevice));
        } else {
            std::vector<float> ff(fr.begin(), fr.end());
            CK(cudaMemcpy(A.fref, ff.data(), ff.size() * 4, cudaMemcpyHostToDevice));
        }
    }
    void *const save_x = A.save_x, *const save_F = A.save_F, *const save_u = A.save_u;
    CK(copy_pos_out(s, save_x));
    CK(cudaMemcpyAsync(save_F, m.F, nodevec_bytes(s), cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(save_u, m.u, nodevec_bytes(s), cudaMemcpyDeviceToDevice, s->stream));
    // seed: D of the final shape and dD/dx (host, FP64)
    std::vector<double> xT(3 * (size_t)n), seed(3 * (size_t)n);
    rc = ensure_scratch(s, sizeof(double) * 3 * n);
    if (rc) return rc;
    launch_nodes_to_f64(s->prec, m, 0, 0, n, s->d_scratch, s->stream);
    CK(cudaMemcpyAsync(xT.data(), s->d_scratch, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    *D_out = taylor_D_and_gradient(xT.data(), n, s->tri.data(), nf, seed.data());
    if (s->prec == kF64) {
        std::vector<double> sv(4 * (size_t)n, 0.0);
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) sv[4 * i + k] = seed[3 * i + k];
        CK(cudaMemcpy(A.lamx[0], sv.data(), sv.size() * 8, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> sv(4 * (size_t)n, 0.0f);
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) sv[4 * i + k] = (float)seed[3 * i + k];
        CK(cudaMemcpy(A.lamx[0], sv.data(), sv.size() * 4, cudaMemcpyHostToDevice));
    }
    const size_t lb = 19 * real_bytes(s) * (size_t)s->L.ncell;
    const int nblk = (int)((s->L.ncell + 255) / 256);
    CK(cudaMemsetAsync(A.lam[0], 0, lb, s->stream));
    CK(cudaMemsetAsync(A.mu, 0, s->vec_bytes, s->stream));
    CK(cudaMemsetAsync(A.lamg, 0, s->vec_bytes, s->stream));
    CK(cudaMemsetAsync(A.uw_partial, 0, sizeof(double) * nblk, s->stream));
    CK(cudaMemsetAsync(A.gX0, 0, sizeof(double) * 3 * n, s->stream));
    CK(cudaMemsetAsync(A.gks, 0, sizeof(double) * n, s->stream));
    if (A.g_dirty)
        for (auto &T : A.tr)
            for (void *p : T.g) CK(cudaMemsetAsync(p, 0, s->vec_bytes, s->stream));
    A.g_dirty = true;  // until the sweep has completed
    if (A.graph_uw != s->u_wall) {
        adj_drop_graphs(s);
        A.graph_uw = s->u_wall;
    }
    const int64_t nck = (int64_t)A.ck_pop.size();
    // Recomputation of one segment into trace set b on the recomputation
    // stream: every forward quantity of its steps is kept.  The force
    // densities T.g[k] are all zero here: zeroed at allocation, and the reverse
    // step of step k clears the cells it has read.  The collide keeps the
    // moments of f(k) (M[k]); those of the segment's last state come from a
    // moments pass.  Only this stream moves the mesh positions.
    auto recompute = [&](int len, int b, cudaStream_t st) {
        const iblbm_sim::Adjoint::Trace &T = A.tr[b];
        for (int k = 0; k < len; ++k) {
            copy_pos_out(s, T.x[k], st);
            cudaMemsetAsync(T.flags[k], 0, s->flag_bytes, st);
            MeshDev mk = m;
            mk.F = T.F[k];  // node forces of step k, kept for the reverse step
            launch_force_spread(s->prec, s->delta, s->L, mk, T.g[k], (uint8_t *)T.flags[k], s->d_status,
                                nullptr, nullptr, st);
            CollideArgs a{};
            a.src = T.pop[k & 1];
            a.dst = T.pop[(k + 1) & 1];
            a.fcur = T.g[k];
            a.flag_cur = (const uint8_t *)T.flags[k];
            a.fold = T.g[k];  // never written: flag_old is all zero
            a.flag_old = A.zero_flags;
            a.tau = s->tau;
            a.u_wall = s->u_wall;
            a.status = s->d_status;
            a.moments = T.M[k];
            launch_collide_stream(s->prec, s->L, a, st);
            launch_interp_advect(s->prec, s->delta, s->L, m, nullptr, T.pop[(k + 1) & 1], T.g[k], nullptr,
                                 nullptr, st);
        }
        launch_adjoint_moments(s->prec, s->L, T.pop[len & 1], T.M[len], st);
    };
    // reverse sweep over a segment kept in set b, on the main stream
    auto reverse = [&](int len, int b, int cur0) {
        const iblbm_sim::Adjoint::Trace &T = A.tr[b];
        int c = cur0;
        for (int k = len - 1; k >= 0; --k) {
            AdjStepArgs q{};
            q.L = s->L;
            q.mesh = m;
            q.x = T.x[k];
            q.x_lo = s->prec == kF64 ? nullptr : (char *)T.x[k] + (size_t)n * 16;
            q.M0 = T.M[k];
            q.M1 = T.M[k + 1];
            q.g = T.g[k];
            q.flags = (const uint8_t *)T.flags[k];
            q.F = T.F[k];
            q.fref = A.fref;
            q.lamx_in = A.lamx[c];
            q.lamx_out = A.lamx[1 - c];
            q.lam_in = A.lam[c];
            q.lam_out = A.lam[1 - c];
            q.mu = A.mu;
            q.lamg = A.lamg;
            q.lamF = A.lamF;
            q.uw_partial = A.uw_partial;
            q.gX0 = A.gX0;
            q.gks = A.gks;
            q.omega = 1.0 / s->tau;
            launch_adjoint_step(s->prec, s->delta, q, s->stream);
            c = 1 - c;
        }
    };
    // launch of a captured graph of either kind (captured on first use)
    auto run_graph = [&](int kind, int len, int b, int cur0, cudaStream_t st) -> int {
        const std::array<int, 4> key{kind, len, b, cur0};
        cudaGraphExec_t ge = nullptr;
        for (auto &g : A.graphs)
            if (g.first == key) ge = g.second;
        if (!ge) {
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            if (kind == 0) recompute(len, b, st);
            else reverse(len, b, cur0);
            cudaError_t e = cudaStreamEndCapture(st, &graph);
            if (e != cudaSuccess) return cuda_fail(s, e, "capture of the adjoint segment");
            e = cudaGraphInstantiate(&ge, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(s, e, "instantiation of the adjoint segment");
            A.graphs.push_back({key, ge});
        }
        CK(cudaGraphLaunch(ge, st));
        return IBLBM_OK;
    };
    auto seg_len = [&](int64_t seg) { return (int)std::min<int64_t>(K, A.n - seg * K); };
    // recomputation of segment seg into set b: its checkpoint, then the graph
    auto enqueue_recompute = [&](int64_t seg, int b) -> int {
        cudaStream_t st = A.rstream;
        CK(cudaMemcpyAsync(A.tr[b].pop[0], A.ck_pop[seg], s->pop_bytes, cudaMemcpyDeviceToDevice, st));
        CK(copy_pos_in(s, A.ck_x[seg], st));
        int r = run_graph(0, seg_len(seg), b, 0, st);
        if (r) return r;
        CK(cudaEventRecord(A.ev_rec[b], st));
        return IBLBM_OK;
    };
    // everything enqueued so far (saved final state, zeroed buffers) comes first
    CK(cudaEventRecord(A.ev_start, s->stream));
    CK(cudaStreamWaitEvent(A.rstream, A.ev_start, 0));
    int cur = 0;
    rc = enqueue_recompute(nck - 1, 0);
    if (rc) return rc;
    for (int64_t seg = nck - 1; seg >= 0; --seg) {
        const int b = (int)((nck - 1 - seg) & 1);
        if (seg > 0) {
            // the other set is free once the sweep of segment seg + 1 is done
            if (seg + 1 < nck) CK(cudaStreamWaitEvent(A.rstream, A.ev_rev[1 - b], 0));
            rc = enqueue_recompute(seg - 1, 1 - b);
            if (rc) return rc;
        }
        CK(cudaStreamWaitEvent(s->stream, A.ev_rec[b], 0));
        const int len = seg_len(seg);
        rc = run_graph(1, len, b, cur, s->stream);
        if (rc) return rc;
        CK(cudaEventRecord(A.ev_rev[b], s->stream));
        if (len % 2) cur = 1 - cur;
    }
    if (A.couette_start) launch_adjoint_init_uw(s->prec, s->L, A.lam[cur], s->u_wall, A.uw_partial, s->stream);
    CK(cudaGetLastError());
    // gradients to the host
    std::vector<double> uwp(nblk), gk(n), g0(3 * (size_t)n);
    CK(cudaMemcpyAsync(uwp.data(), A.uw_partial, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(gk.data(), A.gks, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(g0.data(), A.gX0, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s->stream));
    std::vector<double> lx(4 * (size_t)n);
    if (s->prec == kF64) {
        CK(cudaMemcpyAsync(lx.data(), A.lamx[cur], sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    } else {
        std::vector<float> lf(4 * (size_t)n);
        CK(cudaMemcpyAsync(lf.data(), A.lamx[cur], sizeof(float) * 4 * n, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        for (size_t k = 0; k < lf.size(); ++k) lx[k] = lf[k];
    }
    double duw = 0.0, dks = 0.0;
    for (double v : uwp) duw += v;
    for (double v : gk) dks += v;
    if (dD_dks) *dD_dks = dks;
    if (dD_duw) *dD_duw = duw;
    if (dD_dX0) std::memcpy(dD_dX0, g0.data(), sizeof(double) * 3 * n);
    if (dD_dx0)
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) dD_dx0[3 * i + k] = lx[4 * i + k];
    // restore the final state of the forward run
    CK(copy_pos_in(s, save_x));
    CK(cudaMemcpyAsync(m.F, save_F, nodevec_bytes(s), cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(m.u, save_u, nodevec_bytes(s), cudaMemcpyDeviceToDevice, s->stream));
    rc = sync_status(s);
    if (rc == IBLBM_OK) A.g_dirty = false;
    return rc;
}

int iblbm_set_taylor_recording(iblbm_sim *s, int every, int ring) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    if (every < 0 || (every > 0 && (ring < 1 || ring > (1 << 24))))
        return fail(s, IBLBM_ERR_ARG, "every must be >= 0 and ring in 1..2^24");
    CK(cudaSetDevice(s->device));
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    free_ring(s);
    drop_graphs(s);
    s->rec_every = every;
    s->rec_ring = every > 0 ? ring : 0;
    return IBLBM_OK;
}

static void taylor_from_sums(const double r[12], double out[16]);

int iblbm_get_taylor_records(iblbm_sim *s, int capsule_id, int max_records, double *out,
                             int64_t *steps_out, int *n_out) {
    if (!s || !n_out || max_records < 0) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    if (capsule_id < 0 || capsule_id >= (int)s->caps.size()) return fail(s, IBLBM_ERR_ARG, "no such capsule");
    int rc = sync_status(s);
    if (rc) return rc;
    *n_out = 0;
    if (!s->d_ring) return IBLBM_OK;
    unsigned long long count = 0;
    CK(cudaMemcpy(&count, s->d_ring_count, sizeof(count), cudaMemcpyDeviceToHost));
    const long long avail = std::min<long long>((long long)count, s->rec_ring);
    const long long n = std::min<long long>(avail, max_records);
    const int nc = (int)s->caps.size();
    for (long long k = 0; k < n; ++k) {
        const unsigned long long idx = count - n + k;  // oldest first
        const size_t slot = (size_t)(idx % (unsigned long long)s->rec_ring);
        double r[12];
        CK(cudaMemcpy(r, s->d_ring + (slot * nc + capsule_id) * 12, sizeof(r), cudaMemcpyDeviceToHost));
        if (out) taylor_from_sums(r, out + 16 * k);
        if (steps_out) steps_out[k] = idx < s->rec_steps.size() ? s->rec_steps[idx] : -1;
    }
    *n_out = (int)n;
    return IBLBM_OK;
}

int iblbm_profile_kernels(iblbm_sim *s, int n_steps, double ms_out[4]) {
    Range range("iblbm_profile_kernels");
    if (!s || !ms_out || n_steps < 1 || n_steps > 100000) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    CK(cudaSetDevice(s->device));
    int rc = batch_tables_ok(s);
    if (rc) return rc;
    rc = ensure_mesh(s);
    if (rc) return rc;
    rc = ensure_ring(s);
    if (rc) return rc;
    join_side(s);
    std::vector<cudaEvent_t> ev(5 * (size_t)n_steps, nullptr);
    for (auto &e : ev) CK(cudaEventCreate(&e));
    for (int k = 0; k < n_steps; ++k) {
        const bool rec = record_after(s, s->steps);
        enqueue_step(s, rec, ev.data() + 5 * (size_t)k);
        if (rec) s->rec_steps.push_back(s->steps + 1);
        s->steps++;
    }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    double acc[4] = {0, 0, 0, 0};
    for (int k = 0; k < n_steps && e == cudaSuccess; ++k)
        for (int j = 0; j < 4; ++j) {
            float ms = 0.0f;
            e = cudaEventElapsedTime(&ms, ev[5 * k + j], ev[5 * k + j + 1]);
            acc[j] += ms;
        }
    for (auto &x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) return cuda_fail(s, e, "kernel timing");
    for (int j = 0; j < 4; ++j) ms_out[j] = acc[j] / n_steps;
    return IBLBM_OK;
}

int iblbm_sync(iblbm_sim *s) {
    Range range("iblbm_sync");
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) {
        int first = IBLBM_OK;
        for (iblbm_sim *p : s->slabs) {
            int rc = sync_status(p);
            if (rc && !first) first = fail(s, rc, p->err);
        }
        return first;
    }
    return sync_status(s);
}

int iblbm_tank_treading(const double *x_then, const double *x_now, int n_nodes, const double c_then[3],
                        const double c_now[3], double dt, double *omega_nodes, double *omega_mean) {
    if (!x_then || !x_now || !c_then || !c_now || n_nodes < 1 || !(dt != 0.0) || !std::isfinite(dt)) {
        set_thread_error("need node arrays, centroids, n_nodes >= 1 and a finite dt != 0");
        return IBLBM_ERR_ARG;
    }
    const double m = tank_treading(n_nodes, x_then, x_now, c_then, c_now, dt, omega_nodes);
    if (omega_mean) *omega_mean = m;
    return IBLBM_OK;
}

int iblbm_ellipsoid_fit(const double *nodes, int n_nodes, const double center[3], double out[9]) {
    if (!nodes || !center || !out || n_nodes < 4) {
        set_thread_error("need nodes, center, out and n_nodes >= 4");
        return IBLBM_ERR_ARG;
    }
    if (ellipsoid_fit(n_nodes, nodes, center, out)) {
        set_thread_error("the node cloud does not determine an ellipsoid (singular or not positive)");
        return IBLBM_ERR_ARG;
    }
    return IBLBM_OK;
}

int iblbm_mesh_quality(iblbm_sim *s, int capsule_id, double out[4]) {
    if (!s || !out) return IBLBM_ERR_ARG;
    if (is_group(s)) return iblbm_mesh_quality(s->slabs[0], capsule_id, out);
    if (capsule_id < 0 || capsule_id >= (int)s->caps.size()) return fail(s, IBLBM_ERR_ARG, "no such capsule");
    const Capsule &c = s->caps[capsule_id];
    std::vector<double> x(3 * (size_t)c.n_nodes);
    int rc = iblbm_get_nodes(s, capsule_id, x.data());
    if (rc) return rc;
    std::vector<int> tri(3 * (size_t)c.n_faces);
    for (size_t k = 0; k < tri.size(); ++k) tri[k] = s->tri[3 * (size_t)c.face0 + k] - c.node0;
    const double *X0 = &s->X0[3 * (size_t)c.node0];
    face_area_stats(c.n_faces, tri.data(), X0, x.data(), out);
    const double v0 = closed_volume(c.n_faces, tri.data(), X0);
    out[3] = closed_volume(c.n_faces, tri.data(), x.data()) / v0 - 1.0;
    return IBLBM_OK;
}

int iblbm_set_integrator(iblbm_sim *s, int mode) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) {
        if (mode != 0) return fail(s, IBLBM_ERR_STATE, "a slab group advects by Euler's rule only");
        return IBLBM_OK;
    }
    if (mode != 0 && mode != 1) return fail(s, IBLBM_ERR_ARG, "integrator must be 0 (Euler) or 1 (Adams-Bashforth)");
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    drop_graphs(s);
    s->integrator = mode;
    s->ab2_ready = false;
    s->adj.ready = false;
    return IBLBM_OK;
}

int iblbm_set_equilibrium(iblbm_sim *s, int order) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) {
        for (iblbm_sim *p : s->slabs) {
            int rc = iblbm_set_equilibrium(p, order);
            if (rc) return fail(s, rc, p->err);
        }
        return IBLBM_OK;
    }
    if (order != 1 && order != 2) return fail(s, IBLBM_ERR_ARG, "equilibrium order must be 1 or 2");
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    drop_graphs(s);
    s->eq_order = order;
    s->adj.ready = false;
    return IBLBM_OK;
}

int iblbm_set_interp_mode(iblbm_sim *s, int mode) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    if (mode < -1 || mode > 1) return fail(s, IBLBM_ERR_ARG, "mode must be -1, 0 or 1");
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    drop_graphs(s);
    s->interp_mode = mode;
    return IBLBM_OK;
}

int iblbm_bounds_checked(void) {
#ifdef IBLBM_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

int iblbm_bounds_faults(iblbm_sim *s, unsigned long long *count) {
    if (!s || !count) return IBLBM_ERR_ARG;
    CK(cudaSetDevice(s->device));
    CK(cudaDeviceSynchronize());
    const unsigned long long a = bounds_faults_lbm(), b = bounds_faults_ib(), c = bounds_faults_taylor();
    if (a == ~0ull || b == ~0ull || c == ~0ull) return fail(s, IBLBM_ERR_CUDA, "fault counter not readable");
    *count = a + b + c;
    return IBLBM_OK;
}

int iblbm_set_deterministic_spreading(iblbm_sim *s, int on) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s) || s->batch || s->L.gnx != s->L.nx || s->L.x0 != 0)
        return fail(s, IBLBM_ERR_STATE, "deterministic spreading is for a single whole lattice");
    if (on != 0 && on != 1) return fail(s, IBLBM_ERR_ARG, "on must be 0 or 1");
    CK(cudaSetDevice(s->device));
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    drop_graphs(s);
    if (on && !s->d_fix) {
        const size_t bytes = sizeof(unsigned long long) * 3 * (size_t)s->L.ncell;
        s->d_fix = (unsigned long long *)dev_alloc(s, bytes);
        if (!s->d_fix) return fail(s, IBLBM_ERR_OOM, "fixed-point accumulator allocation failed");
        CK(cudaMemsetAsync(s->d_fix, 0, bytes, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    } else if (!on && s->d_fix) {
        dev_free(s, s->d_fix);
        s->d_fix = nullptr;
    }
    return IBLBM_OK;
}

int iblbm_set_launch_overlap(iblbm_sim *s, int mode) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    if (mode < -1 || mode > 1) return fail(s, IBLBM_ERR_ARG, "mode must be -1, 0 or 1");
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    drop_graphs(s);
    s->overlap = mode;
    return IBLBM_OK;
}

}  // extern "C"

namespace {

int check_run(iblbm_sim *s, int run) {
    if (run < 0 || run >= (s->batch ? (int)s->runs.size() : 1)) return fail(s, IBLBM_ERR_ARG, "no such run");
    return IBLBM_OK;
}

// what: 0 velocity [3][cells], 1 density [cells], 2 populations [19][cells],
// 3 force density [3][cells]
int lattice_get(iblbm_sim *s, int run, int what, double *host_out) {
    if (!s || !host_out) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    int rc = check_run(s, run);
    if (rc) return rc;
    rc = sync_status(s);
    if (rc) return rc;
    size_t po, vo;
    const Lattice Lr = run_lattice(s, run, &po, &vo);
    const size_t per = (what == 1) ? 1 : (what == 2 ? 19 : 3);
    const size_t n = per * (size_t)Lr.ncell;
    rc = ensure_scratch(s, sizeof(double) * n);
    if (rc) return rc;
    const void *pop = (const char *)s->pop[s->cur] + po;
    const void *force = (const char *)s->force[s->cur] + vo;
    if (what == 0) launch_moments(s->prec, Lr, pop, force, nullptr, s->d_scratch, s->stream);
    else if (what == 1) launch_moments(s->prec, Lr, pop, force, s->d_scratch, nullptr, s->stream);
    else if (what == 2) launch_pop_to_f64(s->prec, Lr, pop, s->d_scratch, s->stream);
    else launch_force_to_f64(s->prec, Lr, force, s->d_scratch, s->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(host_out, s->d_scratch, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return IBLBM_OK;
}

int lattice_set_populations(iblbm_sim *s, int run, const double *host_in) {
    if (!s || !host_in) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    int rc = check_run(s, run);
    if (rc) return rc;
    rc = sync_status(s);
    if (rc) return rc;
    size_t po, vo;
    const Lattice Lr = run_lattice(s, run, &po, &vo);
    const size_t n = 19 * (size_t)Lr.ncell;
    // the finiteness check runs on the device, on the uploaded copy: a word
    // after the n values records a non-finite one and the conversion then
    // leaves the lattice untouched
    rc = ensure_scratch(s, sizeof(double) * (n + 1));
    if (rc) return rc;
    int *bad = (int *)(s->d_scratch + n);
    CK(cudaMemsetAsync(bad, 0, sizeof(int), s->stream));
    CK(cudaMemcpyAsync(s->d_scratch, host_in, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
    launch_f64_to_pop(s->prec, Lr, s->d_scratch, (char *)s->pop[s->cur] + po, bad, s->stream);
    CK(cudaGetLastError());
    int bad_host = 0;
    CK(cudaMemcpyAsync(&bad_host, bad, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (bad_host) return fail(s, IBLBM_ERR_ARG, "non-finite population");
    return IBLBM_OK;
}

int whole_lattice_only(iblbm_sim *s) {
    if (s && s->batch && s->runs.size() > 1)
        return fail(s, IBLBM_ERR_STATE, "a batch of several runs: use the per-run getter");
    return IBLBM_OK;
}

}  // namespace

extern "C" {

int iblbm_get_velocity(iblbm_sim *s, double *out) {
    if (is_group(s)) return out ? group_field(s, 0, out, false) : IBLBM_ERR_ARG;
    int rc = whole_lattice_only(s);
    return rc ? rc : lattice_get(s, 0, 0, out);
}
int iblbm_get_density(iblbm_sim *s, double *out) {
    if (is_group(s)) return out ? group_field(s, 1, out, false) : IBLBM_ERR_ARG;
    int rc = whole_lattice_only(s);
    return rc ? rc : lattice_get(s, 0, 1, out);
}
int iblbm_get_populations(iblbm_sim *s, double *out) {
    if (is_group(s)) return out ? group_field(s, 2, out, false) : IBLBM_ERR_ARG;
    int rc = whole_lattice_only(s);
    return rc ? rc : lattice_get(s, 0, 2, out);
}
int iblbm_get_force_field(iblbm_sim *s, double *out) {
    if (is_group(s)) return out ? group_field(s, 3, out, false) : IBLBM_ERR_ARG;
    int rc = whole_lattice_only(s);
    return rc ? rc : lattice_get(s, 0, 3, out);
}
int iblbm_set_populations(iblbm_sim *s, const double *in) {
    if (is_group(s)) return in ? group_field(s, 2, const_cast<double *>(in), true) : IBLBM_ERR_ARG;
    int rc = whole_lattice_only(s);
    return rc ? rc : lattice_set_populations(s, 0, in);
}
int iblbm_get_run_velocity(iblbm_sim *s, int run, double *out) { return lattice_get(s, run, 0, out); }
int iblbm_get_run_populations(iblbm_sim *s, int run, double *out) { return lattice_get(s, run, 2, out); }
int iblbm_set_run_populations(iblbm_sim *s, int run, const double *in) {
    return lattice_set_populations(s, run, in);
}

int iblbm_add_capsule_icosphere_in_run(iblbm_sim *s, int run, double cx, double cy, double cz,
                                       double radius, int subdivisions, int *capsule_id) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    if (subdivisions < 0 || subdivisions > 7 || !(radius > 0.0) || !std::isfinite(radius))
        return fail(s, IBLBM_ERR_ARG, "subdivisions must be 0..7 and radius positive");
    std::vector<double> nodes;
    std::vector<int> tri;
    const double c[3] = {cx, cy, cz};
    icosphere(subdivisions, radius, c, nodes, tri);
    return add_capsule(s, run, nodes.data(), (int)(nodes.size() / 3), tri.data(), (int)(tri.size() / 3),
                       capsule_id);
}

int iblbm_get_run_tile(const iblbm_sim *s, int run, int *tx, int *ty) {
    if (!s || !tx || !ty) return IBLBM_ERR_ARG;
    if (!s->batch) {
        *tx = s->L.ftx;
        *ty = s->L.fty;
        return run == 0 ? IBLBM_OK : IBLBM_ERR_ARG;
    }
    if (run < 0 || run >= (int)s->runs.size()) return IBLBM_ERR_ARG;
    *tx = s->runs[run].tx;
    *ty = s->runs[run].ty;
    return IBLBM_OK;
}

int iblbm_autotune_tiles(iblbm_sim *s, int repeats) {
    if (!s || repeats < 1 || repeats > 1000) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    if (!s->batch) return IBLBM_OK;  // a single lattice has fixed kernels
    if (s->steps != 0) return fail(s, IBLBM_ERR_STATE, "tile autotuning must precede the first step");
    CK(cudaSetDevice(s->device));
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    // distinct box sizes
    std::vector<std::array<int, 3>> sizes;
    for (const RunDesc &R : s->runs) {
        std::array<int, 3> k = {R.nx, R.ny, R.nz};
        if (std::find(sizes.begin(), sizes.end(), k) == sizes.end()) sizes.push_back(k);
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const std::vector<RunDesc> saved = s->runs;
    std::vector<int> best_shape(sizes.size(), 0);
    for (size_t z = 0; z < sizes.size(); ++z) {
        float best = 1e30f;
        for (int c = 0; c < 6; ++c) {
            // only the runs of this size, all with candidate shape c
            s->runs = saved;
            std::vector<int> keep;
            for (size_t r = 0; r < s->runs.size(); ++r) {
                RunDesc &R = s->runs[r];
                R.tx = kTileShapes[c][0];
                R.ty = kTileShapes[c][1];
                if (R.nx == sizes[z][0] && R.ny == sizes[z][1] && R.nz == sizes[z][2]) keep.push_back((int)r);
            }
            int rc = upload_batch_tables(s);
            if (rc) break;
            std::vector<int2> items;
            for (int r : keep) {
                const RunDesc &R = s->runs[r];
                const int nt = R.ntx * R.nty * R.nz;
                for (int t = 0; t < nt; ++t) items.push_back(make_int2(r, t));
            }
            CK(cudaMemcpy(s->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
            BatchArgs b{s->d_runs, s->d_items, (int)items.size(),
                        std::min(s->batch_grid, (int)items.size()), s->batch_pairs};
            CollideArgs a{};
            a.src = s->pop[s->cur];
            a.dst = s->pop[1 - s->cur];  // overwritten by the next step
            a.fcur = s->force[1 - s->cur];
            a.flag_cur = s->flags[1 - s->cur];  // all zero before the first step
            a.fold = s->force[s->cur];
            a.flag_old = s->flags[s->cur];
            a.status = s->d_status;
            launch_collide_batch(s->prec, b, a, s->stream);  // warm-up
            CK(cudaEventRecord(e0, s->stream));
            for (int k = 0; k < repeats; ++k) launch_collide_batch(s->prec, b, a, s->stream);
            CK(cudaEventRecord(e1, s->stream));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                best_shape[z] = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->runs = saved;
    for (RunDesc &R : s->runs)
        for (size_t z = 0; z < sizes.size(); ++z)
            if (R.nx == sizes[z][0] && R.ny == sizes[z][1] && R.nz == sizes[z][2]) {
                R.tx = kTileShapes[best_shape[z]][0];
                R.ty = kTileShapes[best_shape[z]][1];
            }
    return upload_batch_tables(s);
}

static int node_get(iblbm_sim *s, int id, int which, double *host_out) {
    if (!s || !host_out) return IBLBM_ERR_ARG;
    if (is_group(s)) return node_get(s->slabs[0], id, which, host_out);
    int rc = sync_status(s);
    if (rc) return rc;
    int first, count;
    rc = capsule_range(s, id, &first, &count);
    if (rc) return rc;
    rc = ensure_mesh(s);
    if (rc) return rc;
    if (count == 0) return IBLBM_OK;
    rc = ensure_scratch(s, sizeof(double) * 3 * count);
    if (rc) return rc;
    launch_nodes_to_f64(s->prec, s->mesh, which, first, count, s->d_scratch, s->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(host_out, s->d_scratch, sizeof(double) * 3 * count, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return IBLBM_OK;
}

int iblbm_get_nodes(iblbm_sim *s, int id, double *out) { return node_get(s, id, 0, out); }
int iblbm_get_node_forces(iblbm_sim *s, int id, double *out) { return node_get(s, id, 1, out); }
int iblbm_get_node_velocities(iblbm_sim *s, int id, double *out) { return node_get(s, id, 2, out); }

int iblbm_set_nodes(iblbm_sim *s, int id, const double *host_in) {
    if (!s || !host_in) return IBLBM_ERR_ARG;
    if (is_group(s)) {
        for (iblbm_sim *p : s->slabs) {
            int rc = iblbm_set_nodes(p, id, host_in);
            if (rc) return fail(s, rc, p->err);
        }
        return IBLBM_OK;
    }
    int rc = sync_status(s);
    if (rc) return rc;
    int first, count;
    rc = capsule_range(s, id, &first, &count);
    if (rc) return rc;
    for (int k = 0; k < 3 * count; ++k)
        if (!std::isfinite(host_in[k])) return fail(s, IBLBM_ERR_ARG, "non-finite node coordinate");
    rc = ensure_mesh(s);
    if (rc) return rc;
    if (count == 0) return IBLBM_OK;
    rc = ensure_scratch(s, sizeof(double) * 3 * count);
    if (rc) return rc;
    CK(cudaMemcpyAsync(s->d_scratch, host_in, sizeof(double) * 3 * count, cudaMemcpyHostToDevice, s->stream));
    launch_f64_to_nodes(s->prec, s->mesh, first, count, s->d_scratch, s->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    s->ab2_ready = false;  // the velocity history no longer matches the positions
    return IBLBM_OK;
}

int iblbm_get_mesh(iblbm_sim *s, int id, int *n_nodes, int *n_tri, int32_t *tri_out) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) return iblbm_get_mesh(s->slabs[0], id, n_nodes, n_tri, tri_out);
    if (id < 0 || id >= (int)s->caps.size()) return fail(s, IBLBM_ERR_ARG, "no such capsule");
    const Capsule &c = s->caps[id];
    if (n_nodes) *n_nodes = c.n_nodes;
    if (n_tri) *n_tri = c.n_faces;
    if (tri_out)
        for (int k = 0; k < 3 * c.n_faces; ++k) tri_out[k] = s->tri[3 * c.face0 + k] - c.node0;
    return IBLBM_OK;
}

int iblbm_get_taylor(iblbm_sim *s, int id, double out[16]) {
    if (!s || !out) return IBLBM_ERR_ARG;
    if (is_group(s)) return iblbm_get_taylor(s->slabs[0], id, out);
    if (id < 0 || id >= (int)s->caps.size()) return fail(s, IBLBM_ERR_ARG, "no such capsule");
    int rc = sync_status(s);
    if (rc) return rc;
    rc = ensure_mesh(s);
    if (rc) return rc;
    launch_taylor(s->prec, s->mesh, s->plan, false, s->stream);
    CK(cudaGetLastError());
    double r[12];
    CK(cudaMemcpyAsync(r, s->plan.out + 12 * id, sizeof(r), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    taylor_from_sums(r, out);
    return IBLBM_OK;
}

int iblbm_read_async(iblbm_sim *s, double *host_nodes, double *host_sums) {
    Range range("iblbm_read_async");
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    CK(cudaSetDevice(s->device));
    int rc = ensure_mesh(s);
    if (rc) return rc;
    const int n = s->mesh.n_nodes, nc = (int)s->caps.size();
    const bool want_nodes = host_nodes && n > 0, want_sums = host_sums && nc > 0;
    if (!want_nodes && !want_sums) return IBLBM_OK;
    rc = ensure_readback(s, n, nc);
    if (rc) return rc;
    const int b = s->rb_next;
    s->rb_next = 1 - b;
    // the snapshot: set b once the read-back stream is done with its last use
    if (s->rb_used[b]) CK(cudaStreamWaitEvent(s->stream, s->ev_rdone[b], 0));
    if (n >= 152 * 32) {
        // many nodes: one copy kernel (200 capsules of 642 nodes: a step with
        // its read-back 8 % faster than with two copy-engine copies)
        launch_snapshot_nodes(s->prec, s->mesh, n, s->rb_x[b], s->rb_lo[b], s->stream);
        CK(cudaGetLastError());
    } else {
        // few: the copy engine (one capsule of 2 562 nodes: steadier and up to
        // 6 % faster than the kernel)
        CK(cudaMemcpyAsync(s->rb_x[b], s->mesh.x, 4 * real_bytes(s) * (size_t)n, cudaMemcpyDeviceToDevice,
                           s->stream));
        if (s->mesh.x_lo)
            CK(cudaMemcpyAsync(s->rb_lo[b], s->mesh.x_lo, (size_t)16 * n, cudaMemcpyDeviceToDevice, s->stream));
    }
    CK(cudaEventRecord(s->ev_rsnap[b], s->stream));
    CK(cudaStreamWaitEvent(s->rstream, s->ev_rsnap[b], 0));
    MeshDev m = s->mesh;  // the same tables, positions from the snapshot
    m.x = s->rb_x[b];
    m.x_lo = s->rb_lo[b];
    if (want_nodes) {
        launch_nodes_to_f64(s->prec, m, 0, 0, n, s->rb_nodes[b], s->rstream);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(host_nodes, s->rb_nodes[b], sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost,
                           s->rstream));
    }
    if (want_sums) {
        TaylorPlan p = s->plan;  // an immediate reduction into this set's output
        p.out = s->rb_sums[b];
        launch_taylor(s->prec, m, p, false, s->rstream);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(host_sums, s->rb_sums[b], sizeof(double) * 12 * (size_t)nc, cudaMemcpyDeviceToHost,
                           s->rstream));
    }
    CK(cudaEventRecord(s->ev_rdone[b], s->rstream));
    s->rb_used[b] = true;
    return IBLBM_OK;
}

int iblbm_taylor_from_sums(const double sums[12], double out[16]) {
    if (!sums || !out) return IBLBM_ERR_ARG;
    taylor_from_sums(sums, out);
    return IBLBM_OK;
}

// ---- adjoint in one call ---------------------------------------------------------

int iblbm_adjoint_taylor(iblbm_sim *s, int capsule_id, int64_t n_steps, int checkpoint_every, double *dD_dks,
                         double *dD_dCa, double *dD_dX0, double *D) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    if (capsule_id != 0 || s->caps.size() != 1) return fail(s, IBLBM_ERR_ARG, "no such capsule");
    int rc = iblbm_adjoint_forward(s, n_steps, checkpoint_every);
    if (rc) return rc;
    const Capsule &c = s->caps[0];
    const int n = c.n_nodes;
    std::vector<double> gX0(3 * (size_t)n), gx0(3 * (size_t)n);
    double d = 0.0, dks = 0.0, duw = 0.0;
    rc = iblbm_adjoint_backward(s, 0, &d, &dks, &duw, gX0.data(), gx0.data());
    if (rc) return rc;
    // nominal radius: mean distance of the reference nodes from their mean
    double r = 0.0;
    for (int i = 0; i < n; ++i) {
        const double *X = &s->X0[3 * (size_t)(c.node0 + i)];
        const double dx = X[0] - c.origin[0], dy = X[1] - c.origin[1], dz = X[2] - c.origin[2];
        r += std::sqrt(dx * dx + dy * dy + dz * dz);
    }
    r /= n;
    const double eta = (s->tau - 0.5) / 3.0;
    // G = (2 u_wall / nz) eta r / k_s  =>  dD/dG = dD/du_wall * nz k_s / (2 eta r)
    if (dD_dCa) *dD_dCa = duw * s->L.nz * c.ks / (2.0 * eta * r);
    if (dD_dks) *dD_dks = dks;
    if (dD_dX0)
        for (size_t k = 0; k < gX0.size(); ++k) dD_dX0[k] = gX0[k] + gx0[k];
    if (D) *D = d;
    return IBLBM_OK;
}

// ---- checkpoint and restart -------------------------------------------------------

}  // extern "C"

namespace {

struct CkptHeader {
    char magic[8];
    int32_t version, precision, delta, n_runs;
    int32_t nx, ny, nz, init_mode;
    int32_t n_nodes, n_faces, n_caps, flags;  // flags bit 0: Adams-Bashforth history present
    int64_t steps;
    uint64_t pop_bytes, vec_bytes, flag_bytes, x_bytes, xlo_bytes, node_bytes;
    uint64_t sum[7];  // checksum of each section (see launch_checksum)
};
static_assert(sizeof(CkptHeader) <= 256, "checkpoint header must fit its 256-byte slot");

constexpr char kCkptMagic[8] = {'I', 'B', 'L', 'B', 'M', 'C', 'K', '1'};

size_t ck_align(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr int32_t kCkptVersion = 2;

// Host twin of launch_checksum (lbm.cu): the same sum modulo 2^64 of the
// SplitMix64 finaliser of each 64-bit word plus its index times
// 0x9e3779b97f4a7c15, the last word zero-padded.  The words are read
// little-endian byte by byte (both hosts are little-endian, as is the GPU).
uint64_t ck_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

uint64_t checksum_host(const unsigned char *p, size_t n) {
    uint64_t acc = 0;
    const size_t words = (n + 7) / 8;
    for (size_t k = 0; k < words; ++k) {
        uint64_t w = 0;
        for (size_t b = 8 * k; b < n && b < 8 * k + 8; ++b) w |= (uint64_t)p[b] << (8 * (b - 8 * k));
        acc += ck_mix(w + (uint64_t)k * 0x9e3779b97f4a7c15ull);
    }
    return acc;
}

// Checksums of n device ranges, into sums[] (host), on the object's stream.
int checksums_device(iblbm_sim *s, const void *const *p, const size_t *n, int count, uint64_t *sums) {
    if (!s->d_cksum) {
        s->d_cksum = (unsigned long long *)dev_alloc(s, sizeof(unsigned long long) * 8);
        if (!s->d_cksum) return fail(s, IBLBM_ERR_OOM, "checksum buffer allocation failed");
    }
    CK(cudaMemsetAsync(s->d_cksum, 0, sizeof(unsigned long long) * 8, s->stream));
    for (int k = 0; k < count; ++k)
        if (n[k]) launch_checksum(p[k], n[k], s->d_cksum + k, s->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(sums, s->d_cksum, sizeof(uint64_t) * count, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return IBLBM_OK;
}

// Section offsets: header, populations, force density, flags, x, x_lo, F, u.
struct CkptLayout {
    size_t off[8];
    size_t total;
};

CkptLayout ckpt_layout(const CkptHeader &h) {
    const size_t sz[7] = {h.pop_bytes, h.vec_bytes, h.flag_bytes, h.x_bytes, h.xlo_bytes, h.node_bytes,
                          h.node_bytes};
    CkptLayout L;
    L.off[0] = 0;
    size_t o = 256;
    for (int k = 0; k < 7; ++k) {
        L.off[k + 1] = o;
        o += ck_align(sz[k]);
    }
    L.total = o;
    return L;
}

CkptHeader ckpt_header(const iblbm_sim *s) {
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = kCkptVersion;
    h.precision = s->prec;
    h.delta = s->delta;
    h.n_runs = s->batch ? (int32_t)s->runs.size() : 1;
    h.nx = s->L.nx;
    h.ny = s->L.ny;
    h.nz = s->L.nz;
    h.init_mode = s->init_mode;
    h.n_nodes = s->mesh.n_nodes;
    h.n_faces = s->mesh.n_faces;
    h.n_caps = (int32_t)s->caps.size();
    h.flags = s->ab2_ready ? 1 : 0;
    h.steps = s->steps;
    h.pop_bytes = s->pop_bytes;
    h.vec_bytes = s->vec_bytes;
    h.flag_bytes = s->flag_bytes;
    const size_t rb = s->prec == kF64 ? 8 : 4;
    h.x_bytes = (size_t)s->mesh.n_nodes * 4 * rb;
    h.xlo_bytes = s->prec == kF64 ? 0 : (size_t)s->mesh.n_nodes * 16;
    h.node_bytes = (size_t)s->mesh.n_nodes * 4 * rb;
    return h;
}

// buf must be device memory (on_device) or host memory (not on_device)
int check_side(iblbm_sim *s, const void *buf, int on_device) {
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, buf);
    if (e != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    const bool dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    if (on_device && !dev) return fail(s, IBLBM_ERR_ARG, "on_device = 1 but the buffer is not device memory");
    if (!on_device && at.type == cudaMemoryTypeDevice)
        return fail(s, IBLBM_ERR_ARG, "on_device = 0 but the buffer is device memory");
    return IBLBM_OK;
}

}  // namespace

extern "C" {

int iblbm_checkpoint_size(iblbm_sim *s, size_t *bytes) {
    if (!s || !bytes) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    CK(cudaSetDevice(s->device));
    int rc = ensure_mesh(s);
    if (rc) return rc;
    *bytes = ckpt_layout(ckpt_header(s)).total;
    return IBLBM_OK;
}

int iblbm_checkpoint_save(iblbm_sim *s, void *buf, int on_device) {
    Range range("iblbm_checkpoint_save");
    if (!s || !buf) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    int rc = sync_status(s);
    if (rc) return rc;
    rc = ensure_mesh(s);
    if (rc) return rc;
    rc = check_side(s, buf, on_device);
    if (rc) return rc;
    const CkptHeader h = ckpt_header(s);
    const CkptLayout L = ckpt_layout(h);
    char *b = (char *)buf;
    const void *src[7] = {s->pop[s->cur], s->force[s->cur], s->flags[s->cur], s->mesh.x, s->mesh.x_lo,
                          s->mesh.F, s->mesh.u};
    const size_t sz[7] = {h.pop_bytes, h.vec_bytes, h.flag_bytes, h.x_bytes, h.xlo_bytes, h.node_bytes,
                          h.node_bytes};
    CkptHeader hs = h;
    rc = checksums_device(s, src, sz, 7, hs.sum);
    if (rc) return rc;
    // padding bytes (after the header and each section) are written as zeros
    auto zero = [&](size_t off, size_t n) -> cudaError_t {
        if (!n) return cudaSuccess;
        if (on_device) return cudaMemsetAsync(b + off, 0, n, s->stream);
        std::memset(b + off, 0, n);
        return cudaSuccess;
    };
    CK(cudaMemcpyAsync(b, &hs, sizeof(hs), cudaMemcpyDefault, s->stream));
    CK(zero(sizeof(hs), 256 - sizeof(hs)));
    for (int k = 0; k < 7; ++k) {
        if (sz[k]) CK(cudaMemcpyAsync(b + L.off[k + 1], src[k], sz[k], cudaMemcpyDefault, s->stream));
        const size_t end = k < 6 ? L.off[k + 2] : L.total;
        CK(zero(L.off[k + 1] + sz[k], end - L.off[k + 1] - sz[k]));
    }
    CK(cudaStreamSynchronize(s->stream));
    return IBLBM_OK;
}

int iblbm_checkpoint_restore(iblbm_sim *s, const void *buf, size_t buf_bytes, int on_device) {
    Range range("iblbm_checkpoint_restore");
    if (!s || !buf) return IBLBM_ERR_ARG;
    if (is_group(s)) return group_unsupported(s);
    int rc = sync_status(s);
    if (rc) return rc;
    rc = ensure_mesh(s);
    if (rc) return rc;
    rc = check_side(s, buf, on_device);
    if (rc) return rc;
    if (buf_bytes < 256) return fail(s, IBLBM_ERR_ARG, "checkpoint buffer shorter than its header");
    CkptHeader h;
    CK(cudaMemcpy(&h, buf, sizeof(h), cudaMemcpyDefault));
    const CkptHeader mine = ckpt_header(s);
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != kCkptVersion)
        return fail(s, IBLBM_ERR_ARG, "not a checkpoint of this library (magic or version)");
    if (h.precision != mine.precision || h.delta != mine.delta || h.n_runs != mine.n_runs || h.nx != mine.nx ||
        h.ny != mine.ny || h.nz != mine.nz || h.n_nodes != mine.n_nodes || h.n_faces != mine.n_faces ||
        h.n_caps != mine.n_caps || h.pop_bytes != mine.pop_bytes || h.vec_bytes != mine.vec_bytes ||
        h.flag_bytes != mine.flag_bytes || h.x_bytes != mine.x_bytes || h.xlo_bytes != mine.xlo_bytes ||
        h.node_bytes != mine.node_bytes)
        return fail(s, IBLBM_ERR_ARG, "checkpoint of a different configuration");
    if (h.steps < 0 || (h.init_mode != 0 && h.init_mode != 1))
        return fail(s, IBLBM_ERR_ARG, "corrupt checkpoint header");
    const CkptLayout L = ckpt_layout(h);
    if (buf_bytes < L.total)
        return fail(s, IBLBM_ERR_ARG, "checkpoint buffer of " + std::to_string(buf_bytes) + " bytes, " +
                                          std::to_string(L.total) + " needed");
    const char *b = (const char *)buf;
    void *dst[7] = {s->pop[s->cur], s->force[s->cur], s->flags[s->cur], s->mesh.x, s->mesh.x_lo,
                    s->mesh.F, s->mesh.u};
    const size_t sz[7] = {h.pop_bytes, h.vec_bytes, h.flag_bytes, h.x_bytes, h.xlo_bytes, h.node_bytes,
                          h.node_bytes};
    // every section is checked before anything is written
    uint64_t sums[7];
    if (on_device) {
        const void *p[7];
        for (int k = 0; k < 7; ++k) p[k] = b + L.off[k + 1];
        rc = checksums_device(s, p, sz, 7, sums);
        if (rc) return rc;
    } else {
        for (int k = 0; k < 7; ++k) sums[k] = checksum_host((const unsigned char *)b + L.off[k + 1], sz[k]);
    }
    static const char *const kSection[7] = {"populations", "force density", "force flags", "node positions",
                                            "node position low parts", "node forces", "node velocities"};
    for (int k = 0; k < 7; ++k)
        if (sums[k] != h.sum[k])
            return fail(s, IBLBM_ERR_ARG, std::string("checkpoint checksum mismatch in the ") + kSection[k] +
                                              " section (corrupt or truncated data)");
    for (int k = 0; k < 7; ++k)
        if (sz[k]) CK(cudaMemcpyAsync(dst[k], b + L.off[k + 1], sz[k], cudaMemcpyDefault, s->stream));
    // the other force buffer is all zero between steps
    CK(cudaMemsetAsync(s->force[1 - s->cur], 0, s->vec_bytes, s->stream));
    CK(cudaMemsetAsync(s->flags[1 - s->cur], 0, s->flag_bytes, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->steps = h.steps;
    s->init_mode = h.init_mode;
    s->ab2_ready = (h.flags & 1) != 0;
    s->adj.ready = false;
    return IBLBM_OK;
}

}  // extern "C"

// {V, A, c, I} of the device reductions -> the 16 outputs of iblbm_get_taylor.
static void taylor_from_sums(const double r[12], double out[16]) {
    const double V = r[0];
    const double I[9] = {r[5], r[8], r[9], r[8], r[6], r[10], r[9], r[10], r[7]};
    double J[9], val[3], vec[9];
    for (int k = 0; k < 9; ++k) J[k] = I[k] / V;
    sym_eig3(J, val, vec);
    const double ra = std::sqrt(std::max(0.0, 2.5 * (val[1] + val[2] - val[0])));
    const double rb = std::sqrt(std::max(0.0, 2.5 * (val[0] + val[2] - val[1])));
    const double rc = std::sqrt(std::max(0.0, 2.5 * (val[0] + val[1] - val[2])));
    double vx = vec[0], vz = vec[6];
    if (vx < 0.0) {
        vx = -vx;
        vz = -vz;
    }
    out[0] = (ra - rc) / (ra + rc);
    out[1] = std::atan2(vz, vx);
    out[2] = ra;
    out[3] = rb;
    out[4] = rc;
    out[5] = V;
    out[6] = r[1];
    out[7] = r[2];
    out[8] = r[3];
    out[9] = r[4];
    for (int k = 0; k < 6; ++k) out[10 + k] = r[5 + k];
}

// ---- x-slab decomposition -------------------------------------------------------------
//
// A group of P slab objects covers one periodic lattice of nx columns: slab p
// holds the global columns x0_p .. x0_p + w_p - 1.  Per time step (the
// sub-step list of Sec. II.C), on the group's stream:
//   1. every slab: membrane forces of the replicated membranes and spreading
//      into its own cells (Eq. forcespreading), then collide and stream with
//      its own periodic wrap in x (Eq. lbequation);
//   2. the ten boundary columns of every slab are packed, and every slab takes
//      its c_x = +1 column x = 0 from its left neighbour and its c_x = -1 column
//      x = w_p - 1 from its right one: the wraps become the global streaming;
//   3. every slab interpolates the new lattice velocity over its own cells
//      (Eq. velocityinterpolation, a partial sum per node);
//   4. every slab adds the P partials in slab order and advances its copy of
//      the nodes (Eq. positionupdate), so all copies stay identical.
// The exchange is 10 ny nz populations per slab boundary plus 3 numbers per
// node, the data the slabs of several GPUs would send each other.
namespace {

bool is_group(const iblbm_sim *s) { return s && !s->slabs.empty(); }

int group_unsupported(iblbm_sim *s) {
    return fail(s, IBLBM_ERR_STATE, "not available on a slab group (x-slab decomposition)");
}

int group_each(iblbm_sim *s, int (*fn)(iblbm_sim *, void *), void *arg) {
    for (iblbm_sim *p : s->slabs) {
        int rc = fn(p, arg);
        if (rc) return fail(s, rc, std::string("slab: ") + p->err);
    }
    return IBLBM_OK;
}

int group_ensure_buffers(iblbm_sim *s) {
    iblbm_sim *p0 = s->slabs[0];
    const int P = (int)s->slabs.size();
    if (!s->slab_planes) {
        const size_t el = s->prec == kF64 ? 8 : (s->prec == kF32 ? 4 : 2);
        s->slab_plane_bytes = (10 * el * (size_t)s->L.ny * s->L.nz + 255) & ~(size_t)255;
        s->slab_planes = dev_alloc(s, s->slab_plane_bytes * P);
        if (!s->slab_planes) return fail(s, IBLBM_ERR_OOM, "slab exchange buffer allocation failed");
    }
    const int nn = p0->mesh.n_nodes;
    if (s->slab_parts_nodes != nn) {
        dev_free(s, s->slab_parts);
        dev_free(s, s->slab_part_ptrs);
        const size_t v4 = (4 * real_bytes(p0) * (size_t)std::max(nn, 1) + 255) & ~(size_t)255;
        s->slab_parts = dev_alloc(s, v4 * P);
        s->slab_part_ptrs = (void **)dev_alloc(s, sizeof(void *) * P);
        if (!s->slab_parts || !s->slab_part_ptrs) return fail(s, IBLBM_ERR_OOM, "slab partials allocation failed");
        std::vector<void *> ptrs(P);
        for (int k = 0; k < P; ++k) ptrs[k] = (char *)s->slab_parts + k * v4;
        CK(cudaMemcpyAsync(s->slab_part_ptrs, ptrs.data(), sizeof(void *) * P, cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        s->slab_parts_nodes = nn;
    }
    return IBLBM_OK;
}

int group_step(iblbm_sim *s, int64_t n_steps) {
    const int P = (int)s->slabs.size();
    for (iblbm_sim *p : s->slabs) {
        CK(cudaSetDevice(p->device));
        int rc = ensure_mesh(p);
        if (rc) return fail(s, rc, std::string("slab: ") + p->err);
    }
    int rc = group_ensure_buffers(s);
    if (rc) return rc;
    iblbm_sim *p0 = s->slabs[0];
    const size_t v4 = (4 * real_bytes(p0) * (size_t)std::max(p0->mesh.n_nodes, 1) + 255) & ~(size_t)255;
    cudaGetLastError();
    for (int64_t t = 0; t < n_steps; ++t) {
        for (iblbm_sim *p : s->slabs) {
            const int c = p->cur, n = 1 - p->cur;
            launch_force_spread_slab(p->prec, p->delta, p->L, p->mesh, p->force[n], p->flags[n], p->d_status,
                                     p->stream);
            CollideArgs a;
            a.src = p->pop[c];
            a.dst = p->pop[n];
            a.fcur = p->force[n];
            a.flag_cur = p->flags[n];
            a.fold = p->force[c];
            a.flag_old = p->flags[c];
            a.tau = p->tau;
            a.u_wall = p->u_wall;
            a.status = p->d_status;
            a.eq_order = p->eq_order;
            launch_collide_stream(p->prec, p->L, a, p->stream, false);
        }
        for (int k = 0; k < P; ++k) {
            iblbm_sim *p = s->slabs[k];
            launch_plane_pack(p->prec, p->L, p->pop[1 - p->cur], (char *)s->slab_planes + k * s->slab_plane_bytes,
                              p->stream);
        }
        for (int k = 0; k < P; ++k) {
            iblbm_sim *p = s->slabs[k];
            const char *base = (const char *)s->slab_planes;
            launch_plane_unpack(p->prec, p->L, p->pop[1 - p->cur], base + ((k + P - 1) % P) * s->slab_plane_bytes,
                                base + ((k + 1) % P) * s->slab_plane_bytes, p->stream);
        }
        for (int k = 0; k < P; ++k) {
            iblbm_sim *p = s->slabs[k];
            const int n = 1 - p->cur;
            launch_interp_partial_slab(p->prec, p->delta, p->L, p->mesh, p->pop[n], p->force[n],
                                       (char *)s->slab_parts + k * v4, p->stream);
        }
        for (iblbm_sim *p : s->slabs) {
            launch_slab_advect(p->prec, p->mesh, (const void *const *)s->slab_part_ptrs, P, p->stream);
            p->cur = 1 - p->cur;
            p->steps++;
            p->ab2_ready = true;
            p->launches += 5;
        }
        s->steps++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(s, e, "slab step launch");
    }
    return IBLBM_OK;
}

// A global field [comp][nz][ny][nx] from (get) or to (set) the slabs' own
// [comp][nz][ny][w] fields.
int group_field(iblbm_sim *s, int what, double *host, bool set) {
    const int nx = s->L.nx, ny = s->L.ny, nz = s->L.nz;
    const int comps = what == 1 ? 1 : (what == 2 ? 19 : 3);
    const size_t rows = (size_t)comps * nz * ny;
    for (iblbm_sim *p : s->slabs) {
        const int w = p->L.nx, x0 = p->L.x0;
        std::vector<double> part(rows * w);
        if (set)
            for (size_t r = 0; r < rows; ++r) std::memcpy(&part[r * w], host + r * nx + x0, sizeof(double) * w);
        const int rc = set ? lattice_set_populations(p, 0, part.data()) : lattice_get(p, 0, what, part.data());
        if (rc) return fail(s, rc, std::string("slab: ") + p->err);
        if (!set)
            for (size_t r = 0; r < rows; ++r) std::memcpy(host + r * nx + x0, &part[r * w], sizeof(double) * w);
    }
    return IBLBM_OK;
}

}  // namespace

extern "C" {

int iblbm_create_slabs(iblbm_sim **out, int nx, int ny, int nz, double tau, int precision, int delta_points,
                       int n_slabs, void *stream, const iblbm_allocator *alloc) {
    if (!out) return IBLBM_ERR_ARG;
    *out = nullptr;
    g_create_error.clear();
    if (n_slabs < 1 || n_slabs > 64 || nx < 4 * n_slabs) {
        g_create_error = "need 1 <= n_slabs <= 64 and at least 4 columns per slab";
        return IBLBM_ERR_ARG;
    }
    if (ny < 1 || nz < 1 || (long long)nx * ny * nz > 2147483647LL || !(tau > 0.5) || !std::isfinite(tau) ||
        precision < 0 || precision > 2 || delta_points < 2 || delta_points > 4 ||
        (alloc && (!alloc->alloc || !alloc->free))) {
        g_create_error = "lattice, tau, precision, stencil or allocator out of range (as iblbm_create)";
        return IBLBM_ERR_ARG;
    }
    int rc = IBLBM_OK;
    iblbm_sim *s = new (std::nothrow) iblbm_sim();
    if (!s) return IBLBM_ERR_OOM;
    s->L = make_lattice(nx, ny, nz, precision != kF64);
    s->prec = precision;
    s->delta = delta_points;
    s->tau = tau;
    cudaGetDevice(&s->device);
    if (alloc) {
        s->alloc = *alloc;
        s->has_alloc = true;
    }
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        g_create_error = "cudaStreamCreate failed";
        return IBLBM_ERR_CUDA;
    } else {
        s->own_stream = true;
    }
    int x0 = 0;
    for (int k = 0; k < n_slabs; ++k) {
        const int w = nx / n_slabs + (k < nx % n_slabs ? 1 : 0);
        iblbm_sim *p = nullptr;
        rc = iblbm_create(&p, w, ny, nz, tau, precision, delta_points, (void *)s->stream, alloc);
        if (rc) {
            iblbm_destroy(s);
            return rc;
        }
        p->L.x0 = x0;
        p->L.gnx = nx;
        s->slabs.push_back(p);
        x0 += w;
    }
    *out = s;
    return IBLBM_OK;
}

int iblbm_get_slab(const iblbm_sim *s, int slab, int *x0, int *width) {
    if (!s || !is_group(s) || slab < 0 || slab >= (int)s->slabs.size()) return IBLBM_ERR_ARG;
    if (x0) *x0 = s->slabs[slab]->L.x0;
    if (width) *width = s->slabs[slab]->L.nx;
    return IBLBM_OK;
}

}  // extern "C"

// ---- x-slab phases for drivers that hold one slab per process ------------------------------
// The group step above, split into the calls a process holding one slab of a
// lattice makes between its exchanges with the other processes (over the
// host, NCCL or peer copies): begin (forces, spreading, collide-and-stream),
// the boundary columns out and the neighbours' in, the partial node
// velocities out, and the end of the step with every slab's partials.
namespace {

int slab_phase_check(iblbm_sim *s) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s) || s->batch) return fail(s, IBLBM_ERR_STATE, "slab phases take a single lattice object");
    return IBLBM_OK;
}

size_t slab_column_bytes(const iblbm_sim *s) {
    const size_t el = s->prec == kF64 ? 8 : (s->prec == kF32 ? 4 : 2);
    return 10 * el * (size_t)s->L.ny * s->L.nz;
}

size_t slab_part_bytes(const iblbm_sim *s) { return 4 * real_bytes(s) * (size_t)s->mesh.n_nodes; }

int slab_buffers(iblbm_sim *s, size_t parts_bytes) {
    if (!s->slab_planes) {
        s->slab_plane_bytes = (slab_column_bytes(s) + 255) & ~(size_t)255;
        s->slab_planes = dev_alloc(s, 3 * s->slab_plane_bytes);  // own, left, right
        if (!s->slab_planes) return fail(s, IBLBM_ERR_OOM, "slab column buffer allocation failed");
    }
    const size_t pb = std::max<size_t>(parts_bytes, 16);
    if (s->slab_parts_bytes < pb) {
        CK(cudaStreamSynchronize(s->stream));  // a pending step may still read the old buffer
        dev_free(s, s->slab_parts);
        s->slab_parts = dev_alloc(s, pb);
        s->slab_parts_bytes = s->slab_parts ? pb : 0;
        if (!s->slab_parts) return fail(s, IBLBM_ERR_OOM, "slab partials allocation failed");
    }
    if (!s->slab_part_ptrs) {
        s->slab_part_ptrs = (void **)dev_alloc(s, sizeof(void *) * 64);
        if (!s->slab_part_ptrs) return fail(s, IBLBM_ERR_OOM, "slab pointer table allocation failed");
    }
    return IBLBM_OK;
}

}  // namespace

extern "C" {

int iblbm_slab_configure(iblbm_sim *s, int x0, int nx_global) {
    if (!s) return IBLBM_ERR_ARG;
    if (is_group(s) || s->batch) return fail(s, IBLBM_ERR_STATE, "a slab is a single lattice object");
    if (s->d_fix) return fail(s, IBLBM_ERR_STATE, "slab phases spread with float atomics only");
    if (x0 < 0 || nx_global < s->L.nx || x0 + s->L.nx > nx_global || s->L.nx < 4)
        return fail(s, IBLBM_ERR_ARG, "need 0 <= x0, x0 + nx <= nx_global and nx >= 4");
    CK(cudaSetDevice(s->device));
    join_side(s);
    CK(cudaStreamSynchronize(s->stream));
    drop_graphs(s);
    s->L.x0 = x0;
    s->L.gnx = nx_global;
    return IBLBM_OK;
}

int iblbm_slab_step_begin(iblbm_sim *s) {
    int rc = slab_phase_check(s);
    if (rc) return rc;
    if (s->rec_every > 0 || s->integrator != 0)
        return fail(s, IBLBM_ERR_STATE, "slab phases take Euler advection and no Taylor recording");
    CK(cudaSetDevice(s->device));
    rc = ensure_mesh(s);
    if (rc) return rc;
    const int c = s->cur, n = 1 - s->cur;
    launch_force_spread_slab(s->prec, s->delta, s->L, s->mesh, s->force[n], s->flags[n], s->d_status, s->stream);
    CollideArgs a;
    a.src = s->pop[c];
    a.dst = s->pop[n];
    a.fcur = s->force[n];
    a.flag_cur = s->flags[n];
    a.fold = s->force[c];
    a.flag_old = s->flags[c];
    a.tau = s->tau;
    a.u_wall = s->u_wall;
    a.status = s->d_status;
    a.eq_order = s->eq_order;
    launch_collide_stream(s->prec, s->L, a, s->stream, false);
    CK(cudaGetLastError());
    return IBLBM_OK;
}

int iblbm_slab_columns_size(iblbm_sim *s, size_t *bytes) {
    if (!s || !bytes) return IBLBM_ERR_ARG;
    *bytes = slab_column_bytes(s);
    return IBLBM_OK;
}

int iblbm_slab_get_columns(iblbm_sim *s, void *out, int on_device) {
    int rc = slab_phase_check(s);
    if (rc) return rc;
    if (!out) return IBLBM_ERR_ARG;
    rc = slab_buffers(s, 0);
    if (rc) return rc;
    launch_plane_pack(s->prec, s->L, s->pop[1 - s->cur], s->slab_planes, s->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, s->slab_planes, slab_column_bytes(s),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return IBLBM_OK;
}

int iblbm_slab_set_columns(iblbm_sim *s, const void *left, const void *right, int on_device) {
    int rc = slab_phase_check(s);
    if (rc) return rc;
    if (!left || !right) return IBLBM_ERR_ARG;
    rc = slab_buffers(s, 0);
    if (rc) return rc;
    const size_t b = slab_column_bytes(s);
    char *l = (char *)s->slab_planes + s->slab_plane_bytes, *r = l + s->slab_plane_bytes;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(l, left, b, k, s->stream));
    CK(cudaMemcpyAsync(r, right, b, k, s->stream));
    launch_plane_unpack(s->prec, s->L, s->pop[1 - s->cur], l, r, s->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    return IBLBM_OK;
}

int iblbm_slab_partials_size(iblbm_sim *s, size_t *bytes) {
    if (!s || !bytes) return IBLBM_ERR_ARG;
    int rc = ensure_mesh(s);
    if (rc) return rc;
    *bytes = slab_part_bytes(s);
    return IBLBM_OK;
}

int iblbm_slab_get_partials(iblbm_sim *s, void *out, int on_device) {
    int rc = slab_phase_check(s);
    if (rc) return rc;
    if (!out) return IBLBM_ERR_ARG;
    const size_t pb = slab_part_bytes(s);
    rc = slab_buffers(s, pb);
    if (rc) return rc;
    const int n = 1 - s->cur;
    launch_interp_partial_slab(s->prec, s->delta, s->L, s->mesh, s->pop[n], s->force[n], s->slab_parts, s->stream);
    CK(cudaGetLastError());
    if (pb)
        CK(cudaMemcpyAsync(out, s->slab_parts, pb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return IBLBM_OK;
}

int iblbm_slab_step_end(iblbm_sim *s, const void *parts, int n_parts, int on_device) {
    int rc = slab_phase_check(s);
    if (rc) return rc;
    if (!parts || n_parts < 1 || n_parts > 64) return fail(s, IBLBM_ERR_ARG, "need 1..64 partial arrays");
    const size_t pb = slab_part_bytes(s);
    rc = slab_buffers(s, pb * (n_parts + 1));
    if (rc) return rc;
    // the partials after this slab's own, then their addresses
    char *base = (char *)s->slab_parts + pb;
    CK(cudaMemcpyAsync(base, parts, pb * n_parts, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       s->stream));
    std::vector<void *> ptrs(n_parts);
    for (int k = 0; k < n_parts; ++k) ptrs[k] = base + k * pb;
    CK(cudaMemcpyAsync(s->slab_part_ptrs, ptrs.data(), sizeof(void *) * n_parts, cudaMemcpyHostToDevice,
                       s->stream));
    launch_slab_advect(s->prec, s->mesh, (const void *const *)s->slab_part_ptrs, n_parts, s->stream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // the pointer table is host memory's copy
    if (e != cudaSuccess) return cuda_fail(s, e, "slab advection");
    s->cur = 1 - s->cur;
    s->steps++;
    s->ab2_ready = true;
    s->launches += 5;
    return IBLBM_OK;
}

}  // extern "C"
