// internal.h -- interfaces between the host runtime (capi.cpp, mesh.cpp) and
// the CUDA kernels (lbm.cu, ib.cu, taylor.cu) of the IB-LBM-FEM library.
// Plain C++ (no CUDA syntax) so that host files compile with g++.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace iblbm {

// Lattice geometry.  The scalar collide-stream kernel works on tiles of
// kTileX x kTileY x 1 cells; the vectorised one on whole x-rows (4 cells per
// thread, nx/4 lanes per row, nx/4 a power of two <= 256).  The sparse
// force-density flags have the granularity of the kernel in use:
// ftx x fty x 1 cells per flag (32 x 8 tiles, or the 4-cell quad of one
// thread of the vectorised kernel, so that its collide reads the force, and
// the velocity pass of a dense suspension forms u, only where stencils touch).
constexpr int kTileX = 32;
constexpr int kTileY = 8;

struct Lattice {
    int nx, ny, nz;
    // x-slab of a larger periodic lattice: this lattice holds the global
    // columns x0 .. x0 + nx - 1 of gnx (x0 = 0, gnx = nx for a whole lattice)
    int x0 = 0, gnx = 0;
    int ntx, nty;   // scalar-kernel tiles along x and y
    int lanes_row;  // vectorised kernel: nx / 4 lanes per row; 0 = scalar kernel
    int ftx, fty;   // cells per force flag along x and y
    int nfx, nfy;   // flags along x and y
    long long ncell;
    long long ntiles;  // number of force flags
};

inline bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// vec: allow the vectorised kernel (float and half storage).
inline Lattice make_lattice(int nx, int ny, int nz, bool vec) {
    Lattice L;
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.ntx = (nx + kTileX - 1) / kTileX;
    L.nty = (ny + kTileY - 1) / kTileY;
    L.lanes_row = (vec && nx % 4 == 0 && is_pow2(nx / 4) && nx / 4 <= 256) ? nx / 4 : 0;
    L.ftx = L.lanes_row ? 4 : kTileX;  // vector kernel: one flag per thread's 4-cell quad
    L.fty = L.lanes_row ? 1 : kTileY;
    L.nfx = (nx + L.ftx - 1) / L.ftx;
    L.nfy = (ny + L.fty - 1) / L.fty;
    L.ncell = (long long)nx * ny * nz;
    L.ntiles = (long long)L.nfx * L.nfy * nz;
    L.x0 = 0;
    L.gnx = nx;
    return L;
}

enum Prec { kF64 = 0, kF32 = 1, kF16 = 2 };

// One lattice of a batch of independent runs (a single simulation is a batch
// of one run for the IB kernels).  The runs' cells, force vectors and
// populations are concatenated: populations of run r start at 19 * cell_off
// ([19][ncell] within the run), its force vectors at cell_off, its force flags
// at tile_off.  Tiles (= force flag tiles) are tx x ty x 1 cells.
struct RunDesc {
    int nx, ny, nz;
    int tx, ty;    // tile shape
    int ntx, nty;  // tiles along x and y
    int x0, gnx;   // x-slab: global origin and global width (0, nx otherwise)
    int pad;
    long long cell_off, tile_off, ncell;
    double omega, u_wall;
};

struct BatchArgs {
    const RunDesc *runs;   // device [n_runs]
    const int2 *items;     // device [n_items]: (run, tile within the run)
    int n_items;
    int grid;              // persistent grid size
    bool pairs = false;    // every run's rows have even length: two cells per thread (float builds)
};

// Device views of the membrane data, all capsules concatenated.
struct MeshDev {
    int n_nodes;
    int n_faces;
    int n_caps;
    // node coordinates: FP64 build double4[n]; float builds hi/lo float4[n]
    void *x;      // double4* or float4* (hi)
    void *x_lo;   // float4* (lo) or nullptr
    void *F;      // node forces, double4* / float4*
    void *u;      // node velocities, double4* / float4*
    const int *adj_off;   // [n_nodes + 1]
    const int *adj;       // [adj_off[n]] entries face*4 + corner
    const int *adj4;      // int4 [adj_off[n]]: face*4 + corner, and the face's nodes a, b, c
    const int *node_cap;  // [n_nodes] capsule of each node
    const int *tri;       // int4 [n_faces]: a, b, c, capsule
    const void *fconst;   // Vec4 [n_faces][3]: (alpha, beta, gamma, kappa),
                          // (A0, G11, G12, G22), (G11, G12, G22 low parts, 0)
    const void *capmod;   // Vec4 [n_caps]: k_s/6, k_alpha/6, 0, 0
};

// ---- lbm.cu -------------------------------------------------------------------
struct CollideArgs {
    const void *src;   // populations f(t) (deviations), storage type
    void *dst;         // populations f(t+1)
    const void *fcur;  // Vec4 force density of this step
    const uint8_t *flag_cur;
    void *fold;        // Vec4 force density of the previous step (cleared here)
    uint8_t *flag_old;
    double tau;
    double u_wall;
    int *status;
    // optional: moments (j_x, j_y, j_z, rho - 1) of f(t) per cell, Vec4 (the
    // adjoint's recomputation keeps them); null in a plain step
    void *moments = nullptr;
    int eq_order = 2;  // 2: Eq. (equilibrium); 1: the linearised form of Sec. IV.A
    // vectorised kernel: stage the populations in shared memory by bulk copies
    // (where collide_staging_supported), giving up a wait after wait_ns
    bool staged = false;
    unsigned long long wait_ns = 1000000000ull;
};
// Whether the vectorised lattice can take the staged (bulk-copy) collide:
// float or half storage, rows of nx = 4 * lanes_row cells with nx * element
// size a multiple of 16 bytes.
bool collide_staging_supported(int prec, const Lattice &L);
// Launchers of the time-step kernels take `overlap`: launch with programmatic
// stream serialization, so that the kernel may start while the previous kernel
// of the stream still runs (the kernels wait for it where they must; see
// prior_grid_wait).  Only the plain time step sets it.
template <typename... P, typename... A>
inline void launch_maybe_overlapped(void (*kernel)(P...), dim3 grid, dim3 block, cudaStream_t s, bool overlap,
                                    A... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t c = {};
    c.gridDim = grid;
    c.blockDim = block;
    c.dynamicSmemBytes = 0;
    c.stream = s;
    c.attrs = at;
    c.numAttrs = overlap ? 1 : 0;
    cudaLaunchKernelEx(&c, kernel, args...);
}
void launch_collide_stream(int prec, const Lattice &L, const CollideArgs &a, cudaStream_t s, bool overlap = false);
// batched persistent variant: CollideArgs pointers are the concatenated buffers
void launch_collide_batch(int prec, const BatchArgs &b, const CollideArgs &a, cudaStream_t s,
                          bool overlap = false);
int collide_batch_blocks_per_sm(int prec, bool pairs);
// x-slabs: the ten boundary columns of a slab's populations (c_x = +1 at
// x = 0, c_x = -1 at x = nx - 1, each [nz][ny]) to and from a packed buffer
// of 10 * ny * nz elements; unpack takes the c_x = +1 columns from `left`
// (the left neighbour's packed buffer) and the c_x = -1 ones from `right`,
// skipping the rows the wall bounce-back filled.
void launch_plane_pack(int prec, const Lattice &L, const void *pop, void *out, cudaStream_t s);
void launch_plane_unpack(int prec, const Lattice &L, void *pop, const void *left, const void *right,
                         cudaStream_t s);
// Checksum of a device byte range (added into *out, which the caller zeroes):
// the sum modulo 2^64 of the SplitMix64 finaliser of each 64-bit word plus
// its index times 0x9e3779b97f4a7c15 (last word zero-padded).
void launch_checksum(const void *p, size_t n_bytes, unsigned long long *out, cudaStream_t s);
// Name of the collide-and-stream kernel a plain step launches (static string).
const char *collide_kernel_name(int prec, const Lattice &L);
const char *collide_kernel_name(int prec, const Lattice &L, bool staged);
const char *collide_batch_kernel_name(int prec, bool pairs);
// mode 0: rest; mode 1: linear Couette equilibrium
void launch_init_fluid(int prec, const Lattice &L, void *pop, int mode, double u_wall, cudaStream_t s);
// rho [ncell] and u [3][ncell] in double from populations + half the force
void launch_moments(int prec, const Lattice &L, const void *pop, const void *force, double *rho,
                    double *u, cudaStream_t s);
void launch_pop_to_f64(int prec, const Lattice &L, const void *pop, double *out, cudaStream_t s);
// Checks the n = 19 ncell uploaded values on the device (*bad = 1 on a
// non-finite one; *bad must be 0 before) and converts them unless one was.
void launch_f64_to_pop(int prec, const Lattice &L, const double *in, void *pop, int *bad, cudaStream_t s);
void launch_force_to_f64(int prec, const Lattice &L, const void *force, double *out, cudaStream_t s);

// ---- ib.cu ----------------------------------------------------------------------
// runs / node_run: device run table and per-node run index of a batch, or
// null for a single lattice described by L.
// fix (may be null): deterministic spreading, the sums in 64-bit fixed
// point in fix [ncell][3] (zero on entry), turned into the force density of
// the flagged tiles by launch_fix_to_force, which zeroes them again.
void launch_force_spread(int prec, int delta, const Lattice &L, const MeshDev &m, void *force,
                         uint8_t *flags, int *status, const RunDesc *runs, const int *node_run,
                         cudaStream_t s, bool overlap = false, unsigned long long *fix = nullptr);
void launch_fix_to_force(int prec, const Lattice &L, unsigned long long *fix, void *force, const uint8_t *flags,
                         cudaStream_t s, bool overlap = false);
// velocity (Vec4) of every cell of the force-flagged tiles from the
// populations after the step and the step's force density; items / n_items:
// the batch work list of (run, tile) pairs, or null for a single lattice
void launch_flag_velocity(int prec, const Lattice &L, const void *pop, const void *force, const uint8_t *flags,
                          void *uvel, const RunDesc *runs, const int2 *items, long long n_items,
                          cudaStream_t s, bool overlap = false);
// interpolation at the nodes and Euler advection: of the cell velocities uvel
// when not null, else of velocities formed at each stencil cell from the
// populations pop and the force density force (the same arithmetic)
// snap_x / snap_lo (may be null): a second copy of the advanced positions,
// in the layout of m.x / m.x_lo.  ab2: advance by the Adams-Bashforth rule
// with the previous node velocities in m.u instead of Euler's.
void launch_interp_advect(int prec, int delta, const Lattice &L, const MeshDev &m, const void *uvel,
                          const void *pop, const void *force, const RunDesc *runs, const int *node_run,
                          cudaStream_t s, void *snap_x = nullptr, void *snap_lo = nullptr, int ab2 = 0,
                          bool overlap = false);
// x-slab of a lattice (L.gnx > L.nx): the spreading and the interpolation
// take only the slab's own cells of every node's stencil (x indices wrap
// with the global width); the interpolation writes the partial node
// velocities to m.u without moving the nodes, and launch_slab_advect adds the
// partials of all slabs, in slab order, and advances the nodes (Euler).
void launch_force_spread_slab(int prec, int delta, const Lattice &L, const MeshDev &m, void *force,
                              uint8_t *flags, int *status, cudaStream_t s);
void launch_interp_partial_slab(int prec, int delta, const Lattice &L, const MeshDev &m, const void *pop,
                                const void *force, void *part, cudaStream_t s);
// parts: device array of n_parts pointers to the slabs' partial velocities
// (Vec4 per node); the sum goes to m.u and the nodes move by it
void launch_slab_advect(int prec, const MeshDev &m, const void *const *parts, int n_parts, cudaStream_t s);
// node data <-> host doubles [n][3]
void launch_nodes_to_f64(int prec, const MeshDev &m, int which, int first, int count, double *out,
                         cudaStream_t s);
void launch_f64_to_nodes(int prec, const MeshDev &m, int first, int count, const double *in,
                         cudaStream_t s);
// m.x (and m.x_lo in the float builds) of `count` nodes copied to x_out (lo_out).
void launch_snapshot_nodes(int prec, const MeshDev &m, int count, void *x_out, void *lo_out, cudaStream_t s);

// ---- adjoint.cu ---------------------------------------------------------------------
// Buffers of one reverse step (step t of a single lattice).
struct AdjStepArgs {
    Lattice L;
    MeshDev mesh;
    void *x, *x_lo;         // stored node positions x(t) (hi/lo for float builds)
    const void *M0;         // moments of f(t): Vec4 per cell (j_x, j_y, j_z, rho - 1)
    const void *M1;         // moments of f(t+1)
    void *g;                // force density g(t); cleared by the reverse step
    const uint8_t *flags;   // force flags of step t
    const void *F;          // node forces F(t)
    const void *fref;       // reference edges U, V per face, Vec4 [2][n_faces]
    void *lamx_in;          // node adjoint after the step (Vec4 per node)
    void *lamx_out;         // node adjoint before the step
    void *lam_in;           // population adjoint after the step, T [19][ncell] (also corrected in place)
    void *lam_out;          // population adjoint before the step
    void *mu, *lamg;        // lattice work fields, Vec4 per cell
    void *lamF;             // node-force adjoint, Vec4 per node
    double *uw_partial;     // per collide-adjoint block: d/du_wall (accumulated)
    double *gX0;            // [n][3] d/dX0 (accumulated)
    double *gks;            // [n] d/dk_s (accumulated)
    double omega;
};
void launch_adjoint_step(int prec, int delta, const AdjStepArgs &A, cudaStream_t s);
// moments (j, rho - 1) of a population set, Vec4 per cell, for the reverse sweep
void launch_adjoint_moments(int prec, const Lattice &L, const void *pop, void *M, cudaStream_t s);
// sum over cells of lam_f(0) . d f(0)/d u_wall for the linear-Couette start
void launch_adjoint_init_uw(int prec, const Lattice &L, const void *lam, double u_wall, double *partial,
                            cudaStream_t s);

// ---- taylor.cu ----------------------------------------------------------------------
// Per-capsule FP64 sums: out[c*12 + k] = {V, A, cx, cy, cz, Ixx, Iyy, Izz, Ixy, Ixz, Iyz, 0}
struct TaylorPlan {
    int n_caps;
    int cluster;            // blocks per capsule (one thread-block cluster), 1..16
    const int *cap_face0;   // [n_caps + 1] first face of each capsule
    const double *origin;   // [n_caps][3]
    double *out;            // [n_caps][12] results of an immediate reduction
    double *ring;           // [ring_len][n_caps][12] recorded results (or null)
    int ring_len;
    unsigned long long *ring_count;  // records written so far
    unsigned *ticket;       // blocks of a recording launch done (returns to 0)
};
// Blocks of kTaylorClusterThreads threads per capsule: about four faces per
// thread, at most max_cluster (taylor_max_cluster()), and no more than keep
// all capsules' blocks within one per SM of 152: a suspension has blocks
// enough, and the record runs beside the steps, whose kernels lose the SMs
// it holds.  (Two faces per thread in blocks of 256 measured slower: 30 vs
// 27.5 us for eight records of one 5120-face capsule, 72 vs 46 us for one
// record of 200 1280-face capsules; for those 200 capsules one block each
// instead of three: step 176.0 -> 167.7 us with a record every step.)
constexpr int kTaylorClusterThreads = 128;
inline int taylor_cluster_size(int max_faces_per_capsule, int max_cluster, int n_caps) {
    int c = (max_faces_per_capsule + 4 * kTaylorClusterThreads - 1) / (4 * kTaylorClusterThreads);
    const int fill = n_caps > 0 ? 152 / n_caps : 152;
    if (c > fill) c = fill;
    return c < 1 ? 1 : (c > max_cluster ? max_cluster : c);
}
// Largest cluster the reduction kernel may use on this GPU (16 where allowed, else 8).
int taylor_max_cluster();
// Threads per block of the allocation-free reduction (one face per thread).
constexpr int kTaylorThreads = 128;
// record = false: results to p.out; record = true: to the next ring slot.
void launch_taylor(int prec, const MeshDev &m, const TaylorPlan &p, bool record, cudaStream_t s);
// The same for n_snap (<= kTaylorBatch) position snapshots in one launch:
// snapshot k in slot (first + k) % slots of a ring of snapshots laid out like
// m.x / m.x_lo ([slots][n_nodes]); recorded to n_snap consecutive ring records.
constexpr int kTaylorBatch = 8;
void launch_taylor_snapshots(int prec, const MeshDev &m, const TaylorPlan &p, bool record, const void *snap_x,
                             const void *snap_lo, int first, int slots, int n_snap, cudaStream_t s);

// Bounds-checked build: index faults counted by the kernels of each
// translation unit since the last call (0 in the normal build).
unsigned long long bounds_faults_lbm();
unsigned long long bounds_faults_ib();
unsigned long long bounds_faults_taylor();

// Message returned by iblbm_last_error(NULL) in the calling thread (capi.cpp).
void set_thread_error(const std::string &msg);

// ---- mesh.cpp (host) -------------------------------------------------------------------
// Canonical icosphere: nodes [n][3], faces [f][3]
void icosphere(int m, double r, const double c[3], std::vector<double> &nodes,
               std::vector<int> &tri);
// Host eigen-decomposition of a symmetric 3x3 matrix: ascending values,
// eigenvectors in columns of vec (row-major 3x3).
void sym_eig3(const double A[9], double val[3], double vec[9]);
// Taylor deformation D of a closed membrane and, if grad is not null, dD/dx
// [n][3] (host, FP64).
double taylor_D_and_gradient(const double *x, int n, const int *tri, int m, double *grad);
// Diagnostics (host): node angular velocities about the centroid in the xz
// plane (returns the mean); the fit of Eq. (chisquare); face area deviations.
double tank_treading(int n, const double *x0, const double *x1, const double c0[3], const double c1[3],
                     double dt, double *omega);
int ellipsoid_fit(int n, const double *x, const double c[3], double out[9]);
void face_area_stats(int m, const int *tri, const double *X0, const double *x, double out[3]);
double closed_volume(int m, const int *tri, const double *x);

}  // namespace iblbm
