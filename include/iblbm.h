/*
 * iblbm.h -- C ABI of the GB300 (sm_103a) implementation of the combined
 * immersed-boundary lattice-Boltzmann finite-element (IB-LBM-FEM) time step of
 * Krueger, Varnik and Raabe (arXiv:1004.2416), used to simulate deformable
 * capsules in simple shear flow.
 *
 * One simulation object holds a D3Q19 lattice of nx*ny*nz fluid cells
 * (periodic in x and y, bounded by half-way bounce-back walls at
 * z = -1/2 and z = nz - 1/2 that move along x with -u_wall and +u_wall) and
 * any number of closed triangulated membranes (capsules).  All state lives in
 * the memory of the CUDA device that was current when the object was created.
 *
 * General conventions
 *   - Every call returns an iblbm_status (0 = success).  On failure
 *     iblbm_last_error() gives a message.  No call traps, aborts or throws.
 *   - Calls are asynchronous on the stream given to iblbm_create() except the
 *     getters, setters and iblbm_sync(), which synchronise that stream.
 *     Errors raised inside kernels (a stencil crossing a wall, a non-finite or
 *     runaway density) are recorded in a device status word and returned by
 *     the next synchronising call.
 *   - Lattice cell (x, y, z) has linear index x + nx*(y + ny*z).  Scalar
 *     fields are [nz][ny][nx], vector fields [3][nz][ny][nx], population
 *     fields [19][nz][ny][nx], all double precision on the host side.
 *   - Membrane node arrays are [n][3] doubles (x, y, z per node), node
 *     coordinates are unwrapped (not reduced modulo the periodic box).
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3, rest density 1.
 *   - The library owns all device memory it allocates; the caller owns every
 *     host buffer passed in.  Host buffers are only accessed during the call.
 *   - Objects are not thread-safe: one thread at a time per object.
 */
#ifndef IBLBM_H
#define IBLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct iblbm_sim iblbm_sim;

typedef enum {
    IBLBM_OK = 0,
    IBLBM_ERR_ARG = -1,      /* invalid argument or size */
    IBLBM_ERR_OOM = -2,      /* device or host allocation failed */
    IBLBM_ERR_CUDA = -3,     /* a CUDA runtime call failed */
    IBLBM_ERR_UNSTABLE = -4, /* density left (0.5, 2) or became NaN */
    IBLBM_ERR_STENCIL = -5,  /* an IBM stencil cell lies beyond a wall */
    IBLBM_ERR_TIMEOUT = -6,  /* a bounded device wait for staged data gave up */
    IBLBM_ERR_STATE = -7     /* call not valid in the current state */
} iblbm_status;

/* Storage precision of the populations.
 *   IBLBM_FP64: populations, arithmetic and node positions in double.
 *   IBLBM_FP32: populations stored as float deviations from the rest
 *               equilibrium f_i - w_i, float arithmetic, node positions as
 *               unevaluated float pairs (hi + lo).
 *   IBLBM_FP16: as IBLBM_FP32 but the deviations stored as scaled halves. */
typedef enum { IBLBM_FP64 = 0, IBLBM_FP32 = 1, IBLBM_FP16 = 2 } iblbm_precision;

/* Optional device allocator (for instance a caching allocator of the
 * caller's framework).  alloc returns device memory of at least `bytes`
 * bytes usable on `stream`, or NULL; free releases it. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, void *stream, void *ctx);
    void *ctx;
} iblbm_allocator;

typedef struct {
    int nx, ny, nz;
    int precision;     /* iblbm_precision */
    int delta_points;  /* 2, 3 or 4 */
    int n_capsules;
    int n_nodes;       /* all capsules */
    int n_faces;       /* all capsules */
    int64_t step;      /* completed time steps */
    double tau;
    double u_wall;
    int n_runs;        /* lattices of a batch (1 for a single lattice) */
    int64_t kernel_launches; /* kernels the library has launched for time steps
                                (membrane, collide, interpolation and record
                                kernels; a graph replay counts its kernels) */
} iblbm_info;

/* One independent lattice of a batch (see iblbm_batch_create). */
typedef struct {
    int nx, ny, nz;
    double tau;
    double u_wall;  /* walls at z = -1/2 and nz - 1/2 move with -u_wall, +u_wall */
} iblbm_run_spec;

/* ---- life cycle ---------------------------------------------------------- */

/* Creates a lattice of nx*ny*nz cells with BGK relaxation time tau
 * (Eq. lbequation, Sec. II.A; tau > 1/2), the given population precision and
 * the n-point discrete delta function of Eqs. (2point)-(4point) (Sec. II.C,
 * delta_points = 2, 3 or 4).  stream: a cudaStream_t (NULL = legacy default
 * stream); alloc: NULL for cudaMalloc.  The fluid starts at rest at
 * density 1 with resting walls.  Limits: 1 <= nx, ny, nz and
 * nx*ny*nz <= 2^31 - 1.  *out is NULL on failure. */
int iblbm_create(iblbm_sim **out, int nx, int ny, int nz, double tau,
                 int precision, int delta_points, void *stream,
                 const iblbm_allocator *alloc);

/* Creates a batch of n_runs independent lattices (runs) of uneven sizes, each
 * with its own relaxation time and wall speed, advanced together: every time
 * step is one launch per sub-step for all runs, the collide-and-stream being a
 * persistent kernel that walks a work list of (run, tile) pairs.  Capsules
 * are added to a run with iblbm_add_capsule_icosphere_in_run; capsule ids are
 * global over the batch.  Fluid getters of the whole lattice apply only to a
 * batch of one run; use the iblbm_get_run_* functions otherwise.  Limits: as
 * iblbm_create for each run, 1 <= n_runs <= 2^20, all cells <= 2^31 - 1. */
int iblbm_batch_create(iblbm_sim **out, const iblbm_run_spec *runs, int n_runs,
                       int precision, int delta_points, void *stream,
                       const iblbm_allocator *alloc);

/* x-slab decomposition of one lattice (the natural split along the flow
 * direction x; it keeps the walls local).  Creates a group of n_slabs lattice
 * objects, slab k holding nx/n_slabs (+1 for the first nx mod n_slabs) global
 * columns starting at x0_k, all on the current device and the given stream,
 * driven as one lattice of nx*ny*nz cells.  Per time step every slab spreads
 * the forces of the membranes (which every slab holds, replicated) into its
 * own cells and collides and streams with its own periodic wrap in x; then
 * each slab takes the ten boundary columns of the populations with c_x = +1
 * (at x = 0) from its left neighbour and those with c_x = -1 (at x = w - 1)
 * from its right one, which turns the wraps into the global streaming of
 * Eq. (lbequation) (entries the moving-wall bounce-back filled are kept); each
 * slab interpolates the new velocity over its own cells (a partial sum per
 * node, Eq. velocityinterpolation) and every slab advances its copy of the
 * nodes by the sum of the partials taken in slab order (Eq. positionupdate),
 * so the copies stay identical.  Per step and slab boundary the slabs
 * exchange 10 ny nz populations, plus 3 numbers per node.  The group takes
 * the calls of a single lattice for configuration (walls, capsules, moduli,
 * fluid start, equilibrium order, Euler advection), stepping, iblbm_sync, the
 * whole-lattice field getters and setter (assembled from the slabs), node
 * getters and setter, meshes, Taylor deformation and mesh quality; the other
 * calls return IBLBM_ERR_STATE.  Limits: 1 <= n_slabs <= 64, at least four
 * columns per slab, otherwise as iblbm_create.  iblbm_get_slab gives the
 * first global column and the width of slab k. */
int iblbm_create_slabs(iblbm_sim **out, int nx, int ny, int nz, double tau,
                       int precision, int delta_points, int n_slabs,
                       void *stream, const iblbm_allocator *alloc);
int iblbm_get_slab(const iblbm_sim *sim, int slab, int *x0, int *width);

/* The x-slab step of a group, in the calls a process holding one slab of a
 * lattice makes between its exchanges with the other processes (over the
 * host, NCCL or peer copies), for a single lattice object of w columns:
 *   iblbm_slab_configure  makes it the global columns x0 .. x0 + w - 1 of a
 *                         periodic lattice of nx_global columns (its IB
 *                         kernels then take only these columns of each
 *                         stencil, wrapping with nx_global); before stepping;
 *   iblbm_slab_step_begin forces, spreading into the slab, collide-and-stream
 *                         with the slab's own wrap (asynchronous);
 *   iblbm_slab_get_columns / iblbm_slab_set_columns
 *                         the ten boundary columns (iblbm_slab_columns_size
 *                         bytes: the five c_x = +1 populations at x = 0, then
 *                         the five c_x = -1 at x = w - 1, each [nz][ny], in the
 *                         storage format) out, and in from the left and right
 *                         neighbours' outputs;
 *   iblbm_slab_get_partials
 *                         this slab's partial node velocities
 *                         (iblbm_slab_partials_size bytes, a 4-vector of the
 *                         storage's float type per node);
 *   iblbm_slab_step_end   the partials of all n_parts slabs, consecutive, in
 *                         slab order: their sum moves the nodes (Euler) and the
 *                         step completes.
 * Buffers are host memory (on_device = 0) or device memory of the object's
 * device (on_device = 1), owned by the caller.  A group of processes that
 * calls these in this order with the right neighbours computes what
 * iblbm_create_slabs computes, bit for bit.  Euler advection and no Taylor
 * recording (IBLBM_ERR_STATE otherwise); the column and partial calls
 * synchronise. */
int iblbm_slab_configure(iblbm_sim *sim, int x0, int nx_global);
int iblbm_slab_step_begin(iblbm_sim *sim);
int iblbm_slab_columns_size(iblbm_sim *sim, size_t *bytes);
int iblbm_slab_get_columns(iblbm_sim *sim, void *out, int on_device);
int iblbm_slab_set_columns(iblbm_sim *sim, const void *left, const void *right,
                           int on_device);
int iblbm_slab_partials_size(iblbm_sim *sim, size_t *bytes);
int iblbm_slab_get_partials(iblbm_sim *sim, void *out, int on_device);
int iblbm_slab_step_end(iblbm_sim *sim, const void *parts, int n_parts,
                        int on_device);

/* Frees all device and host memory of the object (NULL is accepted). */
int iblbm_destroy(iblbm_sim *sim);

/* Message of the last failure on this object ("" if none).  With sim ==
 * NULL, the message of the last failed call in this thread that takes no
 * simulation object (iblbm_create, iblbm_taylor_sums_noalloc). */
const char *iblbm_last_error(const iblbm_sim *sim);

/* Static name of a status code. */
const char *iblbm_status_string(int status);

int iblbm_get_info(const iblbm_sim *sim, iblbm_info *out);

/* ---- configuration ------------------------------------------------------- */

/* Simple shear by moving walls (Sec. II.A, after Eq. lbmmomenta1): the wall
 * at z = nz - 1/2 moves with +u_wall along x, the wall at z = -1/2 with
 * -u_wall, so the shear rate is 2 u_wall / nz.  Uses Ladd's moving-wall
 * bounce-back with the rest density 1. */
int iblbm_set_shear_walls(iblbm_sim *sim, double u_wall);

/* Adds a spherical capsule meshed by icosahedron subdivision (Sec. II.D,
 * Fig. subdivision): 20*4^m faces and 10*4^m + 2 nodes, 0 <= m <= 7, on a
 * sphere of the given radius around (cx, cy, cz).  The node and face order is
 * the library's canonical order (documented with the design).  The reference
 * shape is the initial shape, with k_s = k_alpha = 0 until iblbm_set_skalak.
 * *capsule_id receives the new id (0, 1, ...). */
int iblbm_add_capsule_icosphere(iblbm_sim *sim, double cx, double cy,
                                double cz, double radius, int subdivisions,
                                int *capsule_id);

/* Adds a capsule from a closed triangle mesh: ref_xyz [n_nodes][3] is both
 * the reference and the initial shape, tri [n_tri][3] node indices
 * (0-based, counter-clockwise seen from outside).  A node may belong to at
 * most 32 faces. */
int iblbm_add_capsule_mesh(iblbm_sim *sim, const double *ref_xyz, int n_nodes,
                           const int32_t *tri, int n_tri, int *capsule_id);

/* As iblbm_add_capsule_icosphere, into run `run` of a batch (run 0 for a
 * single lattice); coordinates are those of the run's own lattice. */
int iblbm_add_capsule_icosphere_in_run(iblbm_sim *sim, int run, double cx,
                                       double cy, double cz, double radius,
                                       int subdivisions, int *capsule_id);

/* Batch only: times the persistent collide-and-stream kernel on the runs of
 * each distinct box size with each tile shape (32x8, 16x16, 8x32, 64x4,
 * 128x2, 256x1 cells per 256-thread block), `repeats` launches per shape,
 * and keeps the fastest shape per size.  Must precede the first step (it
 * overwrites the second population buffer only).  A single lattice has fixed
 * kernels and returns at once. */
int iblbm_autotune_tiles(iblbm_sim *sim, int repeats);

/* Tile shape (cells along x and y per block) used for a run. */
int iblbm_get_run_tile(const iblbm_sim *sim, int run, int *tx, int *ty);

/* Skalak law, Eq. (constitutivelaw) (Sec. II.B): shear modulus k_s and
 * area-dilation modulus k_alpha = C k_s.  capsule_id = -1 sets every capsule.
 * The reduced shear rate of Sec. III is G = shear_rate * eta * r / k_s with
 * eta = (tau - 1/2)/3. */
int iblbm_set_skalak(iblbm_sim *sim, int capsule_id, double k_s, double C);

/* Initial fluid state.  mode 0: rest (f_i = w_i).  mode 1: equilibrium of the
 * linear Couette profile u_x(z) = (2 u_wall / nz)(z - (nz - 1)/2) at density
 * 1 (the state reached by simple shear between the walls).  Also clears the
 * force density and the step counter. */
int iblbm_init_fluid(iblbm_sim *sim, int mode);

/* ---- time stepping --------------------------------------------------------- */

/* Advances n_steps >= 0 time steps, each the sub-step list at the end of
 * Sec. II.C: membrane forces from the current node positions (Sec. II.B,
 * Eq. forcefromenergy), spreading (Eq. forcespreading), one collide-and-stream
 * step with Guo forcing (Eqs. lbequation, equilibrium, latticeforce,
 * lbmmomenta0/1), interpolation of the new lattice velocity at the old node
 * positions (Eq. velocityinterpolation) and Euler advection
 * (Eq. positionupdate).  The lattice velocity that is interpolated is
 * (sum_i c_i f_i(t+1) + f(t)/2) / rho(t+1).  The steps replay captured CUDA
 * graphs: n is split into a piece up to the next start of the Taylor
 * recording period, whole graphs of 32 steps (or of a multiple of the
 * recording period) and the remainder, each a graph captured on first use
 * and cached (up to 16 per object, least recently used dropped).  Only the
 * first step after choosing the Adams-Bashforth rule is launched kernel by
 * kernel.  Asynchronous. */
int iblbm_step(iblbm_sim *sim, int64_t n_steps);

/* Captures and instantiates, without running anything, the graphs that
 * iblbm_step(sim, n_steps) would replay from the current state, so that the
 * following iblbm_step call only launches them (capture and instantiation
 * cost host time, about 10 us per kernel).  Reduces and joins Taylor records
 * still pending from earlier steps.  Asynchronous. */
int iblbm_prepare_steps(iblbm_sim *sim, int64_t n_steps);

/* Kernel timing inside the captured step graphs: with on = 1 every graph
 * captured from now on carries CUDA event nodes around each step's kernel
 * groups (membrane forces + spreading | collide-and-stream | cell velocities +
 * interpolation + advection); the Taylor records stay on their side stream,
 * so the steps run as they do without timing.  Drops the cached graphs.
 * iblbm_get_kernel_times then returns the mean device time per step in
 * milliseconds of the three groups, ms_out[3], over the steps of the last
 * replay of every graph replayed since the previous call, and their number
 * in *n_steps (may be NULL); zeros when none.  Synchronising.
 * IBLBM_ERR_ARG for on outside {0, 1}. */
int iblbm_set_kernel_timing(iblbm_sim *sim, int on);
int iblbm_get_kernel_times(iblbm_sim *sim, double ms_out[3], int64_t *n_steps);

/* Static name of the collide-and-stream kernel the steps of this object
 * launch (template arguments included), "" for NULL. */
const char *iblbm_collide_kernel(const iblbm_sim *sim);

/* How the collide-and-stream kernel of a single float or half lattice whose
 * rows take the vectorised kernel (nx/4 a power of two <= 256, nx times the
 * element size a multiple of 16 bytes, nx <= 512 for float, <= 1024 for
 * half) reads its populations (Eq. lbequation
 * in both): mode 0, every thread loads its 19 populations from global
 * memory; mode 1, a persistent kernel has the bulk-copy engine stage tiles of
 * whole rows of all 19 populations in shared memory, the next tile arriving
 * while the block computes the current one; -1 (default) is mode 0, which
 * measured faster on GB300 for float and half storage.  The results are the
 * same bit for bit.  IBLBM_ERR_ARG for another
 * mode, IBLBM_ERR_STATE for mode 1 on a lattice that cannot take it.
 * Synchronising. */
int iblbm_set_collide_staging(iblbm_sim *sim, int mode);

/* Longest time in nanoseconds a kernel waits for data it has staged before it
 * gives up (default 1e9): the kernel then records IBLBM_ERR_TIMEOUT, waits
 * (again bounded) for its copies in flight and returns, leaving that step's
 * populations incomplete; the next synchronising call returns the error.
 * 0 gives up at the first wait, without polling (to exercise the path).
 * Only the staged collide waits.  IBLBM_ERR_ARG for a negative limit.
 * Synchronising. */
int iblbm_set_device_wait_limit(iblbm_sim *sim, int64_t ns);

/* Sub-step 6 of the step list of Sec. II.C, kept on the device: after every
 * `every`-th step (counted from iblbm_init_fluid; every = 0 switches it off)
 * the double-precision reductions behind iblbm_get_taylor (volume, area,
 * centroid, inertia tensor of every capsule) are recorded into a device ring
 * of `ring` records (1 <= ring <= 2^24), inside the same captured step
 * sequence, without host synchronisation.  Resets earlier records. */
int iblbm_set_taylor_recording(iblbm_sim *sim, int every, int ring);

/* The most recent min(max_records, available) records of one capsule, oldest
 * first: out [n][16] as in iblbm_get_taylor (may be NULL), steps_out [n] the
 * step count after which each was taken (may be NULL), *n_records = n.
 * Synchronising. */
int iblbm_get_taylor_records(iblbm_sim *sim, int capsule_id, int max_records,
                             double *out, int64_t *steps_out, int *n_records);

/* Method variants the paper describes beside the main scheme.
 * iblbm_set_integrator: node advection by Eq. (positionupdate) (mode 0, the
 * default) or by the Adams-Bashforth rule of Sec. II.C,
 * x_i(t+1) = x_i(t) + 3/2 u_i(t+1) - 1/2 u_i(t) (mode 1); the first step after
 * the choice, after capsules are added or nodes are set takes the Euler rule
 * (no u_i(t) yet).  iblbm_set_equilibrium: order 2 (default) for Eq.
 * (equilibrium), order 1 for the linearised equilibrium
 * w_i rho (1 + 3 c_i.u) of Sec. IV.A (the forcing term is Eq. (latticeforce)
 * in both).  The adjoint covers mode 0 and order 2 only (IBLBM_ERR_STATE
 * otherwise).  IBLBM_ERR_ARG for other values.  Synchronising. */
int iblbm_set_integrator(iblbm_sim *sim, int mode);
int iblbm_set_equilibrium(iblbm_sim *sim, int order);

/* How the interpolation (Eq. velocityinterpolation) gets u(X, t+1): mode 0,
 * every node's lanes form u from the 19 populations and the force at each
 * stencil cell; mode 1, a pass first forms u once for every cell of the tiles
 * the spreading flagged and the nodes read it; -1 (default) chooses mode 1
 * when the nodes' stencils touch more than a quarter of the cells (dense
 * suspensions).  Both give the same numbers bit for bit below 152 x 32
 * nodes; above, mode 1 reduces four nodes per warp and the two agree to the
 * rounding of the summation order.  IBLBM_ERR_ARG for another mode.
 * Synchronising. */
int iblbm_set_interp_mode(iblbm_sim *sim, int mode);

/* Bounds-checked build (no counterpart in the paper: a development aid).
 * The library built with -DIBLBM_BOUNDS_CHECK (lib/libiblbm_checked.so; the
 * binding loads it when IBLBM_LIBRARY=checked) range-checks the computed
 * indices of the time-step kernels (streaming neighbours, stencil cells,
 * force tiles, mesh node and face references): an index out of range is
 * counted and replaced by 0, so the access stays inside its buffer and the
 * kernel never faults.  iblbm_bounds_checked returns 1 in that build, 0 in
 * the normal one; iblbm_bounds_faults gives the number of such faults since
 * its last call (always 0 in the normal build).  Synchronises the device. */
int iblbm_bounds_checked(void);
int iblbm_bounds_faults(iblbm_sim *sim, unsigned long long *count);

/* Deterministic spreading (on = 1; off = 0, the default): the force density
 * of Eq. (forcespreading) is summed in 64-bit fixed point, whose integer
 * additions give the same bits in any order, then converted to the storage
 * type for the collide.  With it every time step is bit-reproducible (float
 * atomics otherwise add in an order that varies between runs), so a restart
 * from a checkpoint continues the same trajectory bit for bit with membranes
 * too.  Resolution 2^-40 (float and half storage) or 2^-52 (FP64 build) per
 * contribution; a contribution of magnitude 2^22 (float) or 2^10 (FP64) or
 * more is not added and the next synchronising call returns
 * IBLBM_ERR_UNSTABLE.  Costs three 64-bit integer atomics per stencil cell
 * instead of one vector atomic, a conversion pass over the force tiles and
 * 24 bytes per cell of device memory.  A single whole lattice only
 * (IBLBM_ERR_STATE for a batch, a slab group or a lattice configured as a
 * slab, and iblbm_slab_configure refuses a lattice that has it on);
 * IBLBM_ERR_ARG for another value.  Synchronising. */
int iblbm_set_deterministic_spreading(iblbm_sim *sim, int on);

/* Whether the kernels of a time step are launched with programmatic
 * dependent launch: each kernel may start while the one before it in the
 * step finishes, does what needs nothing of that kernel (the interpolation
 * reads the node positions and forms its stencil indices and weights) and
 * then waits for it.  mode 1 on, 0 off (one kernel after the other), -1
 * (default) on where the membrane kernels take four nodes per warp (more than
 * 152 x 32 nodes: dense suspensions, where it measured faster; for a single
 * capsule it measured no faster or slower).  The results are the same up to
 * the order of the spreading's atomic additions.  IBLBM_ERR_ARG for another
 * mode.  Synchronising. */
int iblbm_set_launch_overlap(iblbm_sim *sim, int mode);

/* Runs n_steps (1..100000) further time steps without graph capture, with
 * CUDA events on the object's stream around each kernel group, and returns
 * the mean device time per step in milliseconds of: ms_out[0] membrane
 * forces + spreading, [1] collide-and-stream, [2] interpolation + advection,
 * [3] Taylor recording (0 when off).  Advances the simulation like
 * iblbm_step.  Synchronising. */
int iblbm_profile_kernels(iblbm_sim *sim, int n_steps, double ms_out[4]);

/* ---- adjoint (gradient of the final Taylor deformation) ----------------------
 *
 * Reverse-mode differentiation of n time steps, for a single lattice with
 * exactly one capsule.  iblbm_adjoint_forward advances n_steps like
 * iblbm_step, keeping a checkpoint of the populations and node positions every
 * `checkpoint_every` steps (at the start of each segment).
 * iblbm_adjoint_backward then gives the Taylor deformation D of the final
 * shape (Sec. III) and its derivatives: with respect to the shear modulus k_s
 * at fixed C = k_alpha / k_s, to the wall speed u_wall (including, when the
 * run started from iblbm_init_fluid(1) at step 0, the dependence of the
 * initial Couette state on u_wall), to the reference node positions X0
 * (dD_dX0, [n][3]) and to the node positions at the start of the run
 * (dD_dx0, [n][3]); when the capsule started in its reference shape, the
 * derivative with respect to that shape is dD_dX0 + dD_dx0.  Each segment is
 * recomputed from its checkpoint, keeping every forward quantity of its
 * steps, and swept backwards through the transposes of the interpolation,
 * collide-and-stream, spreading and membrane-force kernels; dD/dx of the final
 * shape seeds the sweep.  The simulation is left in its final state.  Any
 * output pointer but D may be NULL.  Synchronising. */
int iblbm_adjoint_forward(iblbm_sim *sim, int64_t n_steps, int checkpoint_every);
int iblbm_adjoint_backward(iblbm_sim *sim, int capsule_id, double *D,
                           double *dD_dks, double *dD_duw, double *dD_dX0,
                           double *dD_dx0);

/* Both halves in one call, for a capsule that starts in its reference shape:
 * advances n_steps with checkpoints every checkpoint_every steps and returns
 * dD/dk_s (fixed C and u_wall), dD/dCa and dD/dX0 [n][3] (the reference shape,
 * which is also the initial shape), and D if not NULL.  Ca is the reduced
 * shear rate G = gdot eta r / k_s of Sec. III, varied through the wall speed
 * at fixed k_s: gdot = 2 u_wall / nz, eta = (tau - 1/2) / 3, and r the mean
 * distance of the reference nodes from their mean (the icosphere radius).
 * Errors as the two calls above.  Synchronising. */
int iblbm_adjoint_taylor(iblbm_sim *sim, int capsule_id, int64_t n_steps,
                         int checkpoint_every, double *dD_dks, double *dD_dCa,
                         double *dD_dX0, double *D);

/* ---- checkpoint and restart ---------------------------------------------------
 *
 * A checkpoint holds the dynamic state after a completed step: the
 * populations f(t), the force density of the last spreading with its tile
 * flags, the node positions (with their low parts in float builds), the last
 * node forces and velocities, the step count and the fluid start mode.  The
 * configuration (lattice, precision, stencil, meshes, moduli, walls, tau) is
 * not stored: a checkpoint restores only into an object created and filled
 * with the same configuration, which restore checks (sizes, precision, node
 * and face counts) before writing anything.
 * iblbm_checkpoint_size gives the byte size of a checkpoint.
 * iblbm_checkpoint_save writes it to buf: device memory (on_device = 1) or
 * host memory (on_device = 0, pageable or pinned), owned by the caller, at
 * least that size; iblbm_checkpoint_restore reads it back from a buffer of
 * buf_bytes bytes.  Layout: a 256-byte header (magic "IBLBMCK1", version 2,
 * sizes, and a 64-bit checksum of each section: the sum modulo 2^64 of the
 * SplitMix64 finaliser applied to each little-endian 64-bit word plus its
 * index times 0x9e3779b97f4a7c15, the last word zero-padded), then the
 * sections above, each at a 256-byte aligned offset, in the library's storage
 * formats.  Restore checks the header, the buffer length and every section's
 * checksum before it writes anything.  Errors: IBLBM_ERR_ARG for NULL
 * pointers, a buffer on the wrong side, a bad header, a configuration
 * mismatch, a buffer shorter than the checkpoint or a checksum mismatch;
 * IBLBM_ERR_CUDA for a failed copy.  Both calls synchronise; a pending
 * adjoint forward run is discarded by a restore. */
int iblbm_checkpoint_size(iblbm_sim *sim, size_t *bytes);
int iblbm_checkpoint_save(iblbm_sim *sim, void *buf, int on_device);
int iblbm_checkpoint_restore(iblbm_sim *sim, const void *buf, size_t buf_bytes,
                             int on_device);

/* Waits for the stream and returns the first device error recorded since the
 * last call that returned it (then clears it). */
int iblbm_sync(iblbm_sim *sim);

/* Host-only utility, needs no device: the canonical icosphere used by
 * iblbm_add_capsule_icosphere (Sec. II.D) -- node coordinates nodes_out
 * [10*4^m + 2][3] and faces tri_out [20*4^m][3] (either may be NULL). */
int iblbm_icosphere(int subdivisions, double radius, const double center[3],
                    double *nodes_out, int32_t *tri_out);

/* Host-only utility: the Taylor deformation D of Sec. III of one closed
 * membrane (nodes [n][3], faces [m][3]) and, if dD_dx is not NULL, its
 * gradient with respect to the node positions [n][3], in double precision by
 * a reverse pass through the inertia-tensor and eigenvalue computation. */
int iblbm_taylor_gradient(const double *nodes, int n_nodes, const int32_t *tri,
                          int n_tri, double *D_out, double *dD_dx);

/* Host-only diagnostics of a capsule shape (Sec. III), no device needed.
 * iblbm_tank_treading: the angular velocity omega_i = -dphi_i/dt of each node
 * between two snapshots [n][3] taken dt apart, phi_i its angle about the
 * capsule centroid (c_then, c_now) projected on the xz plane, measured from +x
 * toward +z (so the rotation of simple shear u_x = gdot z is positive; a stiff
 * sphere turns at gdot/2), the angle difference taken in (-pi, pi];
 * omega_nodes [n] and *omega_mean (the mean) may be NULL.
 * iblbm_ellipsoid_fit: the linear least-squares fit of Eq. (chisquare) to the
 * nodes [n][3] relative to center, out[9] = {zeta_x, zeta_y, zeta_z, zeta_xz,
 * r_a, r_b, r_c (semiaxes 1/sqrt of the eigenvalues of Q, descending),
 * D = (r_a - r_c)/(r_a + r_c), theta (major axis in the xz plane, from +x
 * toward +z, x component >= 0)}; IBLBM_ERR_ARG when the fit is singular or Q
 * is not positive definite.  Errors: IBLBM_ERR_ARG for NULL pointers or
 * sizes; the message is in iblbm_last_error(NULL). */
int iblbm_tank_treading(const double *x_then, const double *x_now, int n_nodes,
                        const double c_then[3], const double c_now[3], double dt,
                        double *omega_nodes, double *omega_mean);
int iblbm_ellipsoid_fit(const double *nodes, int n_nodes, const double center[3],
                        double out[9]);

/* Mesh degradation of a capsule (Sec. V, Fig. degrade) from its current nodes:
 * out[4] = {mean, standard deviation (about the mean, over faces) and largest
 * magnitude of the relative face area deviation dA/A0 against the reference
 * faces, relative volume drift V/V0 - 1 (signed tetrahedra)}.  Synchronising. */
int iblbm_mesh_quality(iblbm_sim *sim, int capsule_id, double out[4]);

/* ---- read-back and state access (synchronising) ------------------------------ */

/* Lattice velocity u = (sum_i c_i f_i + f/2)/rho of the current populations
 * with the force density of the last step (Eq. lbmmomenta1), [3][nz][ny][nx]. */
int iblbm_get_velocity(iblbm_sim *sim, double *host_out);

/* Density rho = sum_i f_i (Eq. lbmmomenta0), [nz][ny][nx]. */
int iblbm_get_density(iblbm_sim *sim, double *host_out);

/* Full populations f_i (not deviations), [19][nz][ny][nx], velocity i as in
 * Fig. d3q19.  The setter uploads host_in (pinned memory copies fastest),
 * checks it on the device and returns IBLBM_ERR_ARG, leaving the lattice as
 * it was, if any value is not finite. */
int iblbm_get_populations(iblbm_sim *sim, double *host_out);
int iblbm_set_populations(iblbm_sim *sim, const double *host_in);

/* Force density f(X, t) spread in the last step (Eq. forcespreading),
 * [3][nz][ny][nx]; zero before the first step. */
int iblbm_get_force_field(iblbm_sim *sim, double *host_out);

/* Per-run variants of the velocity and population access of a batch
 * ([3][nz][ny][nx] and [19][nz][ny][nx] of that run). */
int iblbm_get_run_velocity(iblbm_sim *sim, int run, double *host_out);
int iblbm_get_run_populations(iblbm_sim *sim, int run, double *host_out);
int iblbm_set_run_populations(iblbm_sim *sim, int run, const double *host_in);

/* Node positions [n][3] of one capsule (capsule_id >= 0) or of all capsules
 * in id order (capsule_id = -1). */
int iblbm_get_nodes(iblbm_sim *sim, int capsule_id, double *host_out);
int iblbm_set_nodes(iblbm_sim *sim, int capsule_id, const double *host_in);

/* Node forces F_i(t) of the last step (Eq. forcefromenergy) and node
 * velocities u_i(t+1) of the last step (Eq. velocityinterpolation), [n][3]. */
int iblbm_get_node_forces(iblbm_sim *sim, int capsule_id, double *host_out);
int iblbm_get_node_velocities(iblbm_sim *sim, int capsule_id, double *host_out);

/* Node and face counts of one capsule and its faces [n_tri][3]
 * (tri_out may be NULL). */
int iblbm_get_mesh(iblbm_sim *sim, int capsule_id, int *n_nodes, int *n_tri,
                   int32_t *tri_out);

/* Shape of one capsule (Sec. III): out[16] = {D, theta, r_a, r_b, r_c, V, A,
 * c_x, c_y, c_z, I_xx, I_yy, I_zz, I_xy, I_xz, I_yz}.  V, A, centroid c and
 * the inertia tensor I of the paper's face sum about c are reduced in double
 * precision on the device; I/V is diagonalised on the host; r_a >= r_b >= r_c
 * are the semi-axes of the ellipsoid with the same tensor,
 * D = (r_a - r_c)/(r_a + r_c) the Taylor deformation, theta the angle of the
 * major axis in the xz plane, from +x toward +z. */
int iblbm_get_taylor(iblbm_sim *sim, int capsule_id, double out[16]);

/* ---- asynchronous read-back -------------------------------------------------------
 *
 * Copies the node positions into a snapshot on the object's stream, after
 * the work already enqueued, and returns without synchronising; the rest runs
 * from the snapshot on a read-back stream of the object, so that the steps
 * enqueued after this call do not wait for it:
 *   host_nodes  (may be NULL) the positions of all nodes, [n_nodes][3]
 *               doubles, capsules in order (as iblbm_get_nodes(sim, -1, ..));
 *   host_sums   (may be NULL) the device reductions of every capsule,
 *               [n_capsules][12] doubles {V, A, c_x, c_y, c_z, I_xx, I_yy,
 *               I_zz, I_xy, I_xz, I_yz, 0} (as behind iblbm_get_taylor;
 *               iblbm_taylor_from_sums turns one into the 16 shape values).
 * The host buffers belong to the caller and are written by the read-back
 * stream: read them after the next iblbm_sync (which waits for that stream
 * too), and leave them alone until then.  Page-locked buffers (cudaHostAlloc,
 * cudaHostRegister, torch pin_memory) let the copies run while the host
 * enqueues further steps; pageable buffers make the copies synchronous.  The
 * snapshots and device conversions use two sets of buffers of the object,
 * taken in turn, so later read-backs may be enqueued at once (a set is
 * reused after the read-back stream is done with it).  Device errors come
 * back from the next iblbm_sync.  IBLBM_ERR_ARG for a null object,
 * IBLBM_ERR_OOM when the buffers cannot be allocated (none is kept). */
int iblbm_read_async(iblbm_sim *sim, double *host_nodes, double *host_sums);

/* The 16 shape values of iblbm_get_taylor from one capsule's 12 reduced sums
 * (host arithmetic only; no object needed).  IBLBM_ERR_ARG for null
 * pointers. */
int iblbm_taylor_from_sums(const double sums[12], double out[16]);

/* ---- allocation-free capsule reductions ------------------------------------------
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory at the moment they need the reductions
 * behind the Taylor deformation: code whose device memory is entirely handed
 * to another allocator (a framework's caching allocator or a fixed arena),
 * plug-ins called back from such a framework, or tight loops where an
 * allocation would synchronise the device.  It computes what iblbm_get_taylor
 * reduces on the device for one closed membrane, on buffers the caller owns,
 * and allocates nothing.
 *
 *   nodes   device pointer, [n_nodes][3] doubles (n_nodes >= 4)
 *   tri     device pointer, [n_tri][3] int32 node indices, counter-clockwise
 *           seen from outside (4 <= n_tri <= 131072)
 *   origin  host pointer, 3 doubles: a point near the membrane; face terms
 *           are taken relative to it (results do not depend on it beyond
 *           rounding)
 *   out     device pointer, 12 doubles: {V, A, c_x, c_y, c_z, I_xx, I_yy,
 *           I_zz, I_xy, I_xz, I_yz, skipped} -- volume, area, centroid and the
 *           inertia tensor about the centroid, as in iblbm_get_taylor; skipped
 *           counts faces ignored because a node index lay outside
 *           [0, n_nodes) (0 for valid input)
 *   stream  cudaStream_t (NULL = legacy default stream); the call is
 *           asynchronous on it and reads and writes the buffers only there.
 *
 * Scratch: the per-block partial sums live in one fixed device array of
 * 1024 x 16 doubles (128 KiB) that every GPU which loads the library holds
 * until the process exits; n_tri beyond 131072 is rejected with
 * IBLBM_ERR_ARG.  Every call on a device shares that array and it keeps the
 * last call's contents; nothing in it needs to start at zero, because each
 * call overwrites every entry it reads.  Calls that overlap on the GPU (for
 * instance on two streams at once) race on the array and give wrong results.
 * The first call on each device, made with that device current, looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it for the life of
 * the process; make that first call before any stream capture.  A device
 * reset (cudaDeviceReset) or the destruction of the device's primary context
 * invalidates the kept address: do not call this entry point afterwards in the
 * same process.  Errors: IBLBM_ERR_ARG for null pointers or sizes out of
 * range, IBLBM_ERR_CUDA if the lookup or a launch fails; the message is in
 * iblbm_last_error(NULL).  Calls no cudaMalloc, cudaFree or other allocating
 * routine. */
int iblbm_taylor_sums_noalloc(const double *nodes, int n_nodes,
                              const int32_t *tri, int n_tri,
                              const double origin[3], double *out,
                              void *stream);

#ifdef __cplusplus
}
#endif
#endif
