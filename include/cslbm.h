/*
 * cslbm.h -- C ABI of the GB300 curved-space lattice Boltzmann library
 * (the method of Flouris et al., "Fluid structure interaction with curved
 * space lattice Boltzmann", arXiv 1803.07822).
 *
 * One channel (a regular D3Q19 lattice carrying a metric field) lives in a
 * context.  Every device buffer belongs to the caller: the library asks how
 * many bytes it needs (cslbm_workspace_bytes), the caller allocates them (e.g.
 * as a torch tensor) and hands them to cslbm_create.  The library never calls
 * cudaMalloc or cudaFree.  The context itself is a small host object.
 *
 * Conventions shared by every entry point
 *   - lattice n = (n0, n1, n2); node = x + n0*(y + n1*z) (axis 0 fastest);
 *     N = n0*n1*n2.  Lattice units: dx = dt = 1.
 *   - fields are structure-of-arrays: component c of node v at [c*N + v].
 *   - g6 [6][N] FP64: g_00, g_01, g_02, g_11, g_12, g_22 (the metric g_ij).
 *   - dg18 [18][N] FP64: d_k g_ij at row k*6 + ij, ij in the order of g6.
 *   - J9 [9][N] FP64: the chart's Jacobian J^a_i = d h^a / d x^i at row a*3+i.
 *   - a face (axis a, side s) holds the nodes with x_a = 0 (s = 0) or
 *     x_a = n_a - 1 (s = 1); its nodes are ordered by the two other axes,
 *     lower axis fastest.
 *   - `on_device` != 0: pointers are device memory on the context's device;
 *     0: pointers are host memory (pinned memory is fastest); the library
 *     copies through a staging area inside the workspace.
 *   - All work is enqueued on the context's stream.  Entry points that return
 *     a host value (mass, wall force, host-buffer readout) synchronise that
 *     stream before returning.
 *   - Errors: every entry point returns a cslbm_status; the message of the
 *     last failure on the calling thread is returned by cslbm_last_error().
 *     A failing call leaves the context usable unless it returns CSLBM_ECUDA.
 */
#ifndef CSLBM_H
#define CSLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CSLBM_OK = 0,
    CSLBM_EINVAL = 1,    /* bad argument (sizes, axes, null pointers, tau <= 1/2) */
    CSLBM_ECUDA = 2,     /* a CUDA call failed; the message names it */
    CSLBM_ENOMEM = 3,    /* workspace smaller than cslbm_workspace_bytes */
    CSLBM_EUNSTABLE = 4, /* non-finite density or velocity found by cslbm_check */
    CSLBM_ETIMEOUT = 5,  /* a bounded device wait of the fused step pass expired */
    CSLBM_ESTATE = 6     /* call out of order (e.g. step before init) */
} cslbm_status;

/* Storage of the distributions.  All variants store f - w_lambda (weight
 * shifted); FP32/FP16/BF16 compute in FP32, FP64 computes in FP64. */
typedef enum { CSLBM_FP32 = 0, CSLBM_FP16S = 1, CSLBM_BF16S = 2, CSLBM_FP64 = 3 } cslbm_storage;

/* Face rules (Sec. V.A: no-slip by a fixed velocity on the boundary node,
 * open boundaries by extrapolation from the inner neighbours).  A node on
 * several non-periodic faces follows WALL over INFLOW over OUTFLOW, ties by
 * axis then low side first. */
typedef enum { CSLBM_PERIODIC = 0, CSLBM_WALL = 1, CSLBM_INFLOW = 2, CSLBM_OUTFLOW = 3 } cslbm_bc;

typedef struct {
    int n[3];           /* nodes per axis; >= 3 on non-periodic axes */
    int bc_lo[3];       /* cslbm_bc of the low face of each axis */
    int bc_hi[3];       /* ... of the high face; periodic on both or neither */
    double tau;         /* BGK relaxation time (Eq. CE-LB), > 1/2 */
    double theta;       /* normalised temperature (App. B); <= 0 selects c_s^2 = 1/3 */
    double fext[3];     /* body-force density, contravariant, constant (Eq. forcing-B) */
    int storage;        /* cslbm_storage */
    int transform_flags;/* bit 0: transform a_(2) itself instead of the momentum flux Pi */
    int step_kernel;    /* cslbm_step_kernel: which step pass runs (same results up to rounding) */
} cslbm_params;

/* Step pass.  The row-staged pass copies whole lattice rows to shared memory
 * with the bulk-copy engine; it applies to FP32/FP16/BF16 storage with
 * n[0] <= 256, n[0] a multiple of 4, n[0] * bytes per stored population a
 * multiple of 16 and at least 256 nodes.  Its fused form also forms the
 * momentum field in the same (cooperative) launch; it needs axis 2 to be
 * non-periodic.  AUTO takes the fused row pass, else the row pass, else the
 * flat gather pass; ROWS the row pass (momentum field in a kernel of its
 * own), else the flat pass; FLAT always the flat pass.  All give the same
 * results up to rounding. */
typedef enum { CSLBM_STEP_AUTO = 0, CSLBM_STEP_FLAT = 1, CSLBM_STEP_ROWS = 2 } cslbm_step_kernel;

typedef struct cslbm_ctx cslbm_ctx;

/* Bytes of device workspace a context with these parameters needs (about
 * 520 per node in FP32).  EINVAL for invalid parameters: an axis with no
 * node, an axis periodic on one face only, a non-periodic axis of fewer than
 * 3 nodes, tau <= 1/2, an unknown storage or step kernel, more than 65,535
 * planes (n[2]), or 25 n0 n1 n2 >= 2^32 (the kernels' 32-bit field offsets:
 * at most 171,798,691 nodes per context). */
cslbm_status cslbm_workspace_bytes(const cslbm_params* p, size_t* bytes);

/* Create a context on the current CUDA device.  `workspace` is caller-owned
 * device memory of at least cslbm_workspace_bytes (256-byte aligned), kept
 * alive until cslbm_destroy; `stream` is a cudaStream_t (NULL = legacy
 * default stream).  The metric starts flat (g = delta, J = I). */
cslbm_status cslbm_create(const cslbm_params* p, void* workspace, size_t bytes, void* stream,
                          cslbm_ctx** out);

/* Release the host context; never touches the caller's device memory. */
cslbm_status cslbm_destroy(cslbm_ctx* ctx);

/* Metric update kernel (App. A): from g_ij and d_k g_ij compute, per node and
 * in FP64, the inverse metric g^ij, sqrt(g) = sqrt(det g_ij) and
 *   Gamma^i_jk = 1/2 g^il (d_j g_kl + d_k g_jl - d_l g_jk),
 * stored in the compute precision.  No transformation of f: use before
 * cslbm_init_equilibrium or for a static metric.  EINVAL if det g <= 0
 * anywhere (checked on the device, reported after a sync). */
cslbm_status cslbm_set_metric(cslbm_ctx* ctx, const double* g6, const double* dg18, int on_device);

/* Set the chart Jacobian J9 used for Cartesian readout, wall forces and the
 * next chart change.  No transformation of f.  The library keeps the Jacobian
 * at the precision of its arithmetic: FP64 for FP64 storage, else rounded to
 * FP32 (the precision D phi is formed in); the same holds for the Jnew9 of
 * every chart change. */
cslbm_status cslbm_set_jacobian(cslbm_ctx* ctx, const double* J9, int on_device);

/* Chart change (Sec. IV.B): the metric update of cslbm_set_metric for the new
 * chart, then the distributions and the forcing history are transformed node
 * by node with D phi = Jnew^-1 Jold (Jold = the current Jacobian): a_(0) kept,
 * a_(1) -> D phi a_(1), Pi -> D phi Pi D phi^T (or a_(2) itself, see
 * transform_flags), recomposed to second order with the new sqrt(g).  The
 * history's A, B, C transform as scalar, vector and rank-2 tensor.  Jnew
 * becomes the current Jacobian.  ESTATE before cslbm_init_equilibrium.  A
 * metric with det g <= 0 somewhere is flagged on the device and reported as
 * EINVAL by the next cslbm_check (the call itself does not synchronise). */
cslbm_status cslbm_update_metric(cslbm_ctx* ctx, const double* g6, const double* dg18,
                                 const double* Jnew9, int on_device);

/* The chart change of Sec. IV.B (cslbm_update_metric) with the metric
 * derivatives dg18 [18][N] and the new Jacobian Jnew9 [9][N] in FP32, the
 * metric g6 [6][N] still in FP64 (its inversion is FP64).  For FP32, FP16 and BF16 storage the library rounds
 * dg and J to FP32 before any use (Gamma and D phi are formed in FP32), so
 * the state this call leaves is bit for bit the one cslbm_update_metric
 * leaves with the same values in FP64; it lets a caller that uploads the
 * chart every few steps move 156 instead of 264 bytes per node.  Every array
 * is device memory owned by the caller and read before the call's work on
 * the context's stream ends.  EINVAL for FP64 storage, a null or host
 * pointer; ESTATE before cslbm_init_equilibrium; det g <= 0 as for
 * cslbm_update_metric (reported by the next cslbm_check). */
cslbm_status cslbm_update_metric_mixed(cslbm_ctx* ctx, const double* g6, const float* dg18, const float* Jnew9);

/* Initial state f = f^eq(rho, u; g) (App. B) with the boundary rule on the
 * boundary nodes, and forcing history F(x,-dt) := F(x,0).  rho [N] and
 * u3 [3][N] (contravariant) are FP64; NULL selects rho = 1 / u = 0. */
cslbm_status cslbm_init_equilibrium(cslbm_ctx* ctx, const double* rho, const double* u3,
                                    int on_device);

/* Velocity imposed on the nodes of a WALL or INFLOW face (Sec. IV.A velocity
 * coupling): u3 [3][face nodes] FP64, contravariant.  NULL sets zero.
 * EINVAL for a periodic or outflow face. */
cslbm_status cslbm_set_boundary_velocity(cslbm_ctx* ctx, int axis, int side, const double* u3,
                                         int on_device);

/* Advance nsteps of the curved-space LB equation (Eq. CE-LB) split into
 * collision (Eq. collision) and streaming (Eq. streaming), with the Hermite
 * equilibrium (App. B), the forcing of Eqs. forcing2 / forcing-A/B/C with the
 * trapezoidal history, the isotropic lattice gradient of App. D and the
 * boundary rule.  Asynchronous.  ESTATE before cslbm_init_equilibrium, EINVAL
 * for nsteps < 0. */
cslbm_status cslbm_step(cslbm_ctx* ctx, int nsteps);

/* Density and velocity (Eqs. fields1/2): rho [N], u3 [3][N], FP64;
 * contravariant u^i, or Cartesian v^a = J^a_i u^i when cartesian != 0.
 * ESTATE before cslbm_init_equilibrium.  Synchronises for host outputs. */
cslbm_status cslbm_get_moments(cslbm_ctx* ctx, double* rho, double* u3, int cartesian,
                               int on_device);

/* Total mass sum_x sqrt(g) rho (volume element of App. A), FP64. Syncs.
 * ESTATE before cslbm_init_equilibrium. */
cslbm_status cslbm_total_mass(cslbm_ctx* ctx, double* out);

/* Force of the fluid on the face (axis, side), Cartesian, FP64 (Sec. IV.A
 * force coupling):  F^a = s sum_nodes J^a_i T^{i axis} sqrt(g), s = -1 for
 * the low face and +1 for the high face, T of Eq. fields3. Syncs.  ESTATE
 * before cslbm_init_equilibrium, EINVAL for a bad face. */
cslbm_status cslbm_wall_force(cslbm_ctx* ctx, int axis, int side, double out3[3]);

/* Non-finite or supersonic (|u|^2 g > 0.3^2 in lattice units) state?
 * Returns CSLBM_EUNSTABLE if so, CSLBM_OK otherwise.  Also reports, first,
 * a pending det g <= 0 flag of cslbm_update_metric (EINVAL) and a bounded
 * wait of the row-staged or fused step pass that ran out (ETIMEOUT; the
 * pass's counters are reset).  ESTATE before cslbm_init_equilibrium. Syncs. */
cslbm_status cslbm_check(cslbm_ctx* ctx);

/* Test hook of the bounded waits (no counterpart in the paper).  The fused
 * step pass synchronises its CTAs through per-iteration publication counts,
 * and every wait in it gives up after half a second, setting the error flag
 * that cslbm_check reports as CSLBM_ETIMEOUT.  This call makes the next
 * fused launch of ctx (one cslbm_step LBM step; later launches are
 * unaffected) give up after wait_ns nanoseconds instead, and makes its CTA 0
 * leave momentum iteration `iteration` uncounted, so that every step tile
 * waiting on that iteration times out.  The state that step leaves is not a
 * valid LBM state (tiles stepped without their rho u rows); restore one with
 * cslbm_load_state after cslbm_check.  EINVAL when the fused pass does not
 * apply to ctx (see cslbm_params.step_kernel), for iteration < 0, or for
 * wait_ns outside (0, 5e8]. */
cslbm_status cslbm_test_withhold_publication(cslbm_ctx* ctx, int iteration, long long wait_ns);

/* Checkpoint: the bytes of the evolving state (distributions + forcing
 * history), copied to/from `buf` (device or host per on_device).  EINVAL for a
 * buffer smaller than cslbm_state_bytes; saving needs a state (ESTATE), and
 * loading one gives the context a state. */
cslbm_status cslbm_state_bytes(const cslbm_ctx* ctx, size_t* bytes);
cslbm_status cslbm_save_state(cslbm_ctx* ctx, void* buf, size_t bytes, int on_device);
cslbm_status cslbm_load_state(cslbm_ctx* ctx, const void* buf, size_t bytes, int on_device);

/* Profiling.  While enabled, each LBM step enqueued by cslbm_step is
 * bracketed by CUDA events on the context's stream and every kernel launch
 * of the library is counted.  Enabling resets the counters. */
cslbm_status cslbm_profile_enable(cslbm_ctx* ctx, int enable);

/* Sum of the event-timed durations of the profiled LBM steps (ms), their
 * number, and the kernel launches counted since profiling was enabled.
 * Synchronises the stream. */
cslbm_status cslbm_profile_read(cslbm_ctx* ctx, double* step_ms, long long* nsteps, long long* launches);

/* Total mass as cslbm_total_mass, for callers that may not allocate device
 * memory and must leave the context's reduction scratch alone: code in a
 * real-time loop or a host callback that must not enter the CUDA allocator,
 * or a plugin whose host framework owns every allocation.  The paper has no
 * counterpart; this is a property of the library, not of the method.
 * Allocates nothing: the per-block partial sums live in a file-scope device
 * array of 2^18 doubles (2 MiB, held by every GPU that loads the library
 * until the process exits), so lattices of more than 67,108,864 nodes are
 * rejected with CSLBM_EINVAL.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with the context's device
 * current, which must be the current device; make that first call before any
 * stream capture.  The partials are added in a fixed order, so repeated calls
 * on the same state give the same bits.  Every call shares the array and it
 * keeps the last call's contents: calls that overlap on the GPU race.  Syncs
 * the context's stream. */
cslbm_status cslbm_total_mass_static(cslbm_ctx* ctx, double* out);

/* ---------------------------------------------------------------------------
 * Adjoint: gradients of a wall force with respect to the geometry (FP32 or
 * FP64 storage; periodic faces and walls at rest; static metric; state
 * initialised at rest with cslbm_init_equilibrium(ctx, NULL, NULL, ...)).
 * The caller keeps the forward states (checkpoints) and walks back in time:
 *   attach -> (forward: init, steps, the final state in the context)
 *   seed_wall_force -> for t = T-1 .. 0 { load state(t); step_backward }
 *   -> init_backward -> metric_grad.
 * All device pointers; asynchronous on the context's stream.
 * ------------------------------------------------------------------------- */

/* Device workspace bytes of the adjoint fields of a context (EINVAL for
 * FP16/BF16 storage or inflow/outflow faces). */
cslbm_status cslbm_adjoint_workspace_bytes(const cslbm_ctx* ctx, size_t* bytes);

/* Attach a caller-owned, 256-byte aligned workspace for the adjoint fields
 * (zeroed). */
cslbm_status cslbm_adjoint_attach(cslbm_ctx* ctx, void* workspace, size_t bytes);

/* Objective e3 . F, F the force of the fluid on the wall (axis, side) as
 * cslbm_wall_force computes it from the context's current state (the state
 * after the last forward step; Sec. III, momentum exchange on the wall
 * nodes): sets the adjoint of the state to dJ/dstate and the geometry and
 * Jacobian adjoints to dJ/dgeometry, dJ/dJ. */
cslbm_status cslbm_adjoint_seed_wall_force(cslbm_ctx* ctx, int axis, int side, const double e3[3]);

/* The adjoint of one LBM step (Sec. II, Eqs. collision and streaming, with
 * the forcing of Eqs. forcing-A/B/C and the lattice gradient of App. D): the
 * context's state must be the state before the step; the adjoint state moves
 * from after the step to before it and the step's geometry derivatives are
 * added. */
cslbm_status cslbm_step_backward(cslbm_ctx* ctx);

/* The adjoint of the rest initialisation (f = f^eq(rho = 1, u = 0), the
 * history F(-1) := F(0)): adds its geometry derivatives. */
cslbm_status cslbm_adjoint_init_backward(cslbm_ctx* ctx);

/* The accumulated geometry adjoint through the metric kernel (App. A: g^-1,
 * sqrt(g), Christoffel symbols from g and dg): FP64 gradients of the
 * objective with respect to g6 [6][N] and dg18 [18][N] (the inputs of
 * cslbm_set_metric, passed again), and with respect to the Jacobian J9
 * [9][N] (grad_J9 may be null). */
cslbm_status cslbm_adjoint_metric_grad(cslbm_ctx* ctx, const double* g6, const double* dg18, double* grad_g6,
                                       double* grad_dg18, double* grad_J9);

/* ---------------------------------------------------------------------------
 * Chart change with interpolation (Sec. IV.B, transition maps): the new node
 * x~ takes the old state's moments at x = psi(x~) = h^-1(h~(x~)), generally
 * off the old grid, by trilinear interpolation of the fields a_(0), a_(1),
 * Pi (or a_(2)) of f and of the forcing history and of the old Jacobian;
 * then D phi = J~(x~)^-1 J(x), the tensor transformation and the
 * recomposition with the new sqrt(g) as in cslbm_update_metric.  A periodic
 * axis wraps x, a non-periodic one clamps it to [0, n - 1].
 * ------------------------------------------------------------------------- */

/* Scratch bytes of cslbm_update_metric_interp: 20 values per node at the
 * compute precision (FP64 for FP64 storage, FP32 otherwise). */
cslbm_status cslbm_transform_interp_scratch_bytes(const cslbm_ctx* ctx, size_t* bytes);

/* cslbm_update_metric with interpolation.  g6 [6][N], dg18 [18][N], Jnew9
 * [9][N] as in cslbm_update_metric; psi3 [3][N] the old lattice coordinates
 * (x, y, z) of the point of every new node.  Every array, scratch included,
 * is device memory (EINVAL otherwise); ENOMEM for a short scratch; ESTATE
 * before init_equilibrium.  Asynchronous, like cslbm_update_metric. */
cslbm_status cslbm_update_metric_interp(cslbm_ctx* ctx, const double* g6, const double* dg18, const double* Jnew9,
                                        const double* psi3, void* scratch, size_t scratch_bytes);

/* ---------------------------------------------------------------------------
 * Isotropic lattice derivatives (App. D, improved lattice derivatives): with
 * the D3Q19 weights w and velocities c,
 *   G_i f = (1/c_s^2) sum_l w_l c_l^i f(x + c_l)          (order 2)
 *   L f   = (2/c_s^2) sum_l w_l (f(x + c_l) - f(x))       (the Laplacian)
 *   d_i f = G_i[f - (c_s^2/2) L f]                       (order 4)
 * Beyond a non-periodic face a field is continued by the polynomial of degree
 * `order` through the order + 1 nodes nearest the face, axis by axis.  FP64,
 * on the context's stream.  Every pointer is device memory (EINVAL
 * otherwise); an axis with a non-periodic face needs order + 1 nodes and
 * every axis 2 (EINVAL).
 * ------------------------------------------------------------------------- */

/* Scratch bytes of cslbm_lattice_gradient for ncomp fields: F = f - (c_s^2/2)
 * L f (order 4) or the continued f (order 2) on the lattice padded by one
 * site at non-periodic faces, ncomp x padded nodes doubles. */
cslbm_status cslbm_lattice_gradient_scratch_bytes(const cslbm_ctx* ctx, int ncomp, int order, size_t* bytes);

/* grad[(k ncomp + c) N + v] = d_k f_c at node v for the fields f [ncomp][N]
 * (layout of the context's lattice), order 2 or 4.  For ncomp = 6 and f = g6
 * the output is dg18 in the layout cslbm_set_metric takes.  Asynchronous;
 * ENOMEM for a short scratch (caller-owned, device memory). */
cslbm_status cslbm_lattice_gradient(cslbm_ctx* ctx, const double* f, int ncomp, int order, double* grad,
                                    void* scratch, size_t scratch_bytes);

/* Scratch bytes of cslbm_set_metric_lattice / cslbm_update_metric_lattice:
 * 18 N doubles of dg plus the gradient's own scratch for 6 fields. */
cslbm_status cslbm_metric_lattice_scratch_bytes(const cslbm_ctx* ctx, int order, size_t* bytes);

/* cslbm_set_metric / cslbm_update_metric with dg computed from g6 on the
 * lattice (order 2 or 4) instead of supplied: the geometry from the metric
 * alone (App. D: metric, Christoffel symbols precomputed at fourth order).
 * g6 (and Jnew9) are device memory. */
cslbm_status cslbm_set_metric_lattice(cslbm_ctx* ctx, const double* g6, int order, void* scratch,
                                      size_t scratch_bytes);
cslbm_status cslbm_update_metric_lattice(cslbm_ctx* ctx, const double* g6, const double* Jnew9, int order,
                                         void* scratch, size_t scratch_bytes);

/* ---------------------------------------------------------------------------
 * Batched form: nb independent channels (each its own cslbm_params, FP32
 * storage, any sizes) advanced together.  Each channel is an ordinary
 * context, reachable with cslbm_batch_context, on which every call above
 * works (geometry, boundary velocities, initialisation, moments, mass, wall
 * force, state); its own cslbm_step takes the flat gather pass.
 * ------------------------------------------------------------------------- */
typedef struct cslbm_batch cslbm_batch;

/* Device workspace bytes of a batch of nb channels with parameters p[0..nb). */
cslbm_status cslbm_batch_workspace_bytes(int nb, const cslbm_params* p, size_t* bytes);

/* Create the batch in a caller-owned, 256-byte aligned device workspace; the
 * channels' contexts use `stream`, the batch steps run on a stream of its own
 * ordered after and before `stream` with events.  EINVAL for a channel that
 * is not FP32 or for invalid parameters, ENOMEM for a short workspace. */
cslbm_status cslbm_batch_create(int nb, const cslbm_params* p, void* workspace, size_t bytes, void* stream,
                                cslbm_batch** out);
cslbm_status cslbm_batch_context(cslbm_batch* b, int i, cslbm_ctx** out);

/* nsteps time steps of every channel (Sec. II, Eqs. collision and streaming,
 * per channel): ONE persistent launch per step over all channels, whose CTAs
 * (all resident: a cooperative launch) take runs of nodes from a device-side
 * queue for the momentum field, meet at a grid barrier, then take the step's
 * runs from a second queue; two steps are replayed at a time from a CUDA
 * graph.  Asynchronous; ESTATE when a channel has no state. */
cslbm_status cslbm_batch_step(cslbm_batch* b, int nsteps);

/* Autotuner of the batch step's tile shape: times every candidate -- nodes
 * per block (128, 256, 512) x nodes per work item (1, 4, 16 blocks) x blocks
 * per SM (the resident maximum and half of it) -- on this batch, reps
 * repetitions of one step from the current state each (the state does not
 * advance), keeps the fastest and returns it in shape3 = {nodes per block,
 * nodes per work item, blocks per SM} and its time per step in *ms (either
 * may be null).  Synchronises. */
cslbm_status cslbm_batch_tune(cslbm_batch* b, int reps, int* shape3, float* ms);

/* Set the batch step's tile shape {nodes per block, nodes per work item,
 * blocks per SM} by hand; EINVAL unless nodes per block is 128, 256 or 512,
 * nodes per work item a power of two in 128..8192 that it divides, and
 * blocks per SM between 1 and the number that can be resident. */
cslbm_status cslbm_batch_set_shape(cslbm_batch* b, const int* shape3);

/* The last tuning's candidates: *count of them; the first `max` shapes (3 ints
 * each, as cslbm_batch_tune returns them) and times per step (ms) copied out. */
cslbm_status cslbm_batch_tune_results(const cslbm_batch* b, int max, int* shapes, float* ms, int* count);

/* CSLBM_ETIMEOUT (once, then the flag is cleared) when the grid barrier of a
 * batch step ran out of its bounded wait (half a second), CSLBM_OK
 * otherwise.  Synchronises the batch's stream. */
cslbm_status cslbm_batch_check(cslbm_batch* b);

/* Kernels launched by cslbm_batch_step so far (graph replays included). */
cslbm_status cslbm_batch_launches(const cslbm_batch* b, long long* launches);
cslbm_status cslbm_batch_destroy(cslbm_batch* b);

/* ---------------------------------------------------------------------------
 * Two dimensions (D2Q9): the same method on the nine-velocity square lattice
 * (the paper's 2-D flag simulations).  Node v = x + n0 y; FP64 inputs
 * g3 [3][N] = g00, g01, g11, dg6 [6][N] = d_k g_ij at (k * 3 + ij), J4 [4][N]
 * = J^a_i at (a * 2 + i); face velocity of face (axis, side) [2][n of the
 * other axis], contravariant.  Storage and arithmetic FP32 or FP64.  Same
 * ownership and error conventions as above; on_device = 0 means host arrays
 * (staged through the workspace, synchronising).
 * ------------------------------------------------------------------------- */
typedef struct {
    int n[2];             /* nodes along axes 0 and 1 */
    int bc_lo[2], bc_hi[2];
    double tau, theta;    /* theta <= 0: 1/3 */
    double fext[2];       /* body force density, contravariant */
    int storage;          /* CSLBM_FP32 or CSLBM_FP64 */
} cslbm2d_params;
typedef struct cslbm2d_ctx cslbm2d_ctx;

/* Device workspace bytes (EINVAL for invalid parameters or FP16/BF16
 * storage); create in a caller-owned, 256-byte aligned workspace (ENOMEM when
 * short), destroy (never frees caller memory). */
cslbm_status cslbm2d_workspace_bytes(const cslbm2d_params* p, size_t* bytes);
cslbm_status cslbm2d_create(const cslbm2d_params* p, void* workspace, size_t bytes, void* stream, cslbm2d_ctx** out);
cslbm_status cslbm2d_destroy(cslbm2d_ctx* ctx);
/* geometry (App. A in 2-D: g^ij, sqrt(g), Gamma) from g and dg; EINVAL when g
 * is not positive definite somewhere (synchronises) */
cslbm_status cslbm2d_set_metric(cslbm2d_ctx* ctx, const double* g3, const double* dg6, int on_device);
/* the chart's Jacobian J4 [4][N] for Cartesian readout and wall forces
 * (Sec. IV.A, vector transformation between the lattice and Cartesian space) */
cslbm_status cslbm2d_set_jacobian(cslbm2d_ctx* ctx, const double* J4, int on_device);
/* chart change: new geometry and the node-wise transformation of f and of
 * the forcing history (Sec. IV.B) */
cslbm_status cslbm2d_update_metric(cslbm2d_ctx* ctx, const double* g3, const double* dg6, const double* Jnew4,
                                   int on_device);
/* velocity imposed on a wall or inflow face (Sec. V, boundary nodes on the
 * wall), u2 [2][n of the other axis], contravariant; EINVAL on a periodic face */
cslbm_status cslbm2d_set_boundary_velocity(cslbm2d_ctx* ctx, int axis, int side, const double* u2, int on_device);
/* f = f^eq(rho, u; g) (App. B, equilibrium coefficients), F(-dt) := F(0);
 * rho [N] and u2 [2][N] (contravariant) may be null for 1 and 0; ESTATE
 * before the metric is set */
cslbm_status cslbm2d_init_equilibrium(cslbm2d_ctx* ctx, const double* rho, const double* u2, int on_device);
/* nsteps LBM steps (Sec. II, Eqs. collision and streaming, with the forcing
 * of Eqs. forcing-A/B/C), two kernels each, asynchronous; ESTATE before
 * init_equilibrium */
cslbm_status cslbm2d_step(cslbm2d_ctx* ctx, int nsteps);
/* rho [N], u2 [2][N] (Sec. II, Eqs. fields: contravariant, or Cartesian
 * v = J u) of the state with the boundary rule applied; synchronises */
cslbm_status cslbm2d_get_moments(cslbm2d_ctx* ctx, double* rho, double* u2, int cartesian, int on_device);
/* FP64 sum of sqrt(g) rho (the mass of Sec. V.B); synchronises */
cslbm_status cslbm2d_total_mass(cslbm2d_ctx* ctx, double* out);
/* force of the fluid on face (axis, side), s sum J T^{i axis} sqrt(g) per unit
 * depth (Sec. IV.A, momentum exchange on the nodes), FP64; synchronises */
cslbm_status cslbm2d_wall_force(cslbm2d_ctx* ctx, int axis, int side, double out2[2]);

/* Message of the last failure on this thread ("" if none). */
const char* cslbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CSLBM_H */
