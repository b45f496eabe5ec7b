/*
 * dg.h -- C ABI of the GB300 (sm_103a) discontinuous Galerkin Euler library.
 *
 * The library evaluates the collocated Gauss-Legendre DG right-hand side of
 * the 3D compressible Euler equations on periodic Cartesian hexahedral meshes
 * and advances it with the five-stage low-storage Runge-Kutta scheme, after
 * Kirby & Mavriplis, "GPU-Accelerated Discontinuous Galerkin Methods: 30x
 * Speedup on 345 Billion Unknowns" (arXiv 2006.15698):
 *   governing equations and flux ........................ Sec. II.A, Eq. 1-2
 *   ideal-gas closure, gamma ............................. Sec. II.A, Eq. 3
 *   weak form integrated by parts ........................ Sec. II.B, Eq. 4-5
 *   Lax-Friedrichs interface flux ........................ Sec. II.B
 *   nodal Lagrange basis on N = p+1 Gauss-Legendre points  Sec. II.B, Eq. 6-7
 *   low-storage explicit RK time integration ............. Sec. II.B, Sec. IV, Sec. VI.A
 *
 * Conventions shared by every call
 * --------------------------------
 * State arrays.  A state holds the conservative variables
 * (rho, rho u, rho v, rho w, rho E) at every node of every element, as
 *     Q[field][element][k][j][i]     (C order, i fastest)
 * with element index e = ex + nx*(ey + ny*ez) and node (i,j,k) at the
 * Gauss-Legendre points xi_i, xi_j, xi_k of the reference cube [-1,1]^3, i.e.
 * at x = x0 + (ex + (xi_i + 1)/2) hx, hx = Lx/nx (likewise y, z).  The scalar
 * type is double for DG_FP64 meshes and float for DG_FP32 meshes;
 * dg_mesh_sizes gives the byte size.  State arrays are DEVICE memory owned by
 * the caller (for instance torch tensors), starting on a 16-byte boundary
 * (cudaMalloc and torch allocations do; a misaligned state is DG_ERR_ARG);
 * the library never allocates, frees or retains them, and reads/writes them
 * only inside the calls.
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).  Every call except dg_mesh_create/destroy/sizes,
 * dg_status_string and dg_last_error is asynchronous on that stream: it
 * validates its arguments on the host, enqueues kernels and returns.  Calls
 * on one mesh handle share the handle's workspace, so they must be ordered
 * (one stream, or explicit events); concurrent calls on one handle race.
 *
 * Errors.  Arguments are checked on the host before anything is enqueued
 * (DG_ERR_ARG, DG_ERR_UNSUPPORTED).  A CUDA launch or allocation failure is
 * DG_ERR_CUDA / DG_ERR_OOM.  Kernels never trap: a non-positive or non-finite
 * density or pressure seen by dg_cfl_dt sets a sticky device flag that
 * dg_last_error reports (DG_ERR_NONFINITE) and the time step it writes is NaN.
 *
 * Device.  A mesh handle belongs to the device that was current when it was
 * created; calls must be made with that device current.
 */
#ifndef DG_GB300_H
#define DG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DG_OK = 0,
    DG_ERR_ARG = 1,         /* a NULL pointer, non-positive size, bad enum value */
    DG_ERR_UNSUPPORTED = 2, /* p outside [0, DG_MAX_P] */
    DG_ERR_OOM = 3,         /* device allocation of the handle's workspace failed */
    DG_ERR_CUDA = 4,        /* a CUDA call or kernel launch failed */
    DG_ERR_NONFINITE = 5,   /* a kernel met rho <= 0, p <= 0 or a NaN (device flag) */
    DG_ERR_BOUNDS = 6,      /* reserved: an index check in a checking build failed */
    DG_ERR_TIMEOUT = 7,     /* reserved: a bounded wait ran out */
    DG_ERR_TOO_LARGE = 8    /* the problem does not fit the fixed static scratch of
                               dg_rhs_static (DG_STATIC_SCRATCH_BYTES) */
} dg_status;

typedef enum {
    DG_FP64 = 0, /* double state, double arithmetic */
    DG_FP32 = 1  /* float state and volume/surface arithmetic; the time step's
                    maximum and dt, the integrals and the norms in double (each
                    node's wave speed is evaluated in float, as the state) */
} dg_precision;

typedef enum {
    DG_INIT_UNIFORM = 0, /* params {rho, u, v, w, p} */
    DG_INIT_VORTEX = 1,  /* params {beta, xc, yc, u_inf, v_inf, w_inf, t} */
    DG_INIT_TGV = 2      /* params {rho0, V0, Mach} */
} dg_init_kind;

#define DG_MAX_P 6
#define DG_NORMS_LEN 7

typedef struct dg_mesh dg_mesh;

/* Create a handle for a periodic box [x0, x0+Lx] x [y0, y0+Ly] x [z0, z0+Lz]
 * split into nx*ny*nz equal hexahedral elements of polynomial degree p
 * (N = p+1 Gauss-Legendre nodes per direction, Sec. II.B, Eq. 7), ratio of
 * specific heats gamma (Eq. 3).  The handle computes the 1D operators of the
 * collocated basis on the host (nodes, weights, weak derivative, face
 * interpolation and lift vectors) and allocates its device workspace on the
 * current device: for DG_FP64 the interface-flux buffer (3 faces x N^2
 * points x 5 fields per element), for DG_FP32 a second state array (the
 * fused single-pass stage writes its output there while neighbours still
 * read the input), plus the reduction partials and the error flag.  Sizes: 1 <= nx, ny, nz; nx*ny*nz*N^3 < 2^40; 0 <= p <= 6;
 * L > 0; gamma > 1.  On success *out owns the handle (free with
 * dg_mesh_destroy).  Errors: DG_ERR_ARG, DG_ERR_UNSUPPORTED, DG_ERR_OOM,
 * DG_ERR_CUDA; *out is set to NULL on error. */
dg_status dg_mesh_create(int nx, int ny, int nz, int p,
                         double x0, double y0, double z0,
                         double Lx, double Ly, double Lz,
                         double gamma, dg_precision precision, dg_mesh **out);

/* Free the handle and its device workspace (synchronises the device first).
 * NULL is ignored. */
void dg_mesh_destroy(dg_mesh *mesh);

/* Sizes of the mesh: n_dof = elements * N^3 nodes, n_unknowns = 5 * n_dof
 * (Sec. V-VI count both), state_bytes = bytes of one state array,
 * workspace_bytes = device bytes the handle holds.  Any output may be NULL. */
dg_status dg_mesh_sizes(const dg_mesh *mesh, int64_t *n_dof, int64_t *n_unknowns,
                        size_t *state_bytes, size_t *workspace_bytes);

/* Fill the device state Q with an initial condition evaluated at the nodes
 * (kinds and parameters above; the vortex is the isentropic vortex carried by
 * (u_inf, v_inf, w_inf) to time t, columnar along z, with minimum-image
 * distances on the periodic box; TGV is the Taylor-Green vortex with
 * p0 = rho0 V0^2 / (gamma Mach^2)).  params is a HOST array of nparams
 * doubles.  Errors: DG_ERR_ARG (unknown kind, too few params, NULL). */
dg_status dg_state_init(const dg_mesh *mesh, dg_init_kind kind, const double *params,
                        int nparams, void *Q, void *stream);

/* Semi-discrete right-hand side dQ/dt = M^{-1} R(Q) of Eq. 5 with collocated
 * quadrature: the volume term (sum-factorised weak derivative of the Euler
 * fluxes, Eq. 2), minus the lifted local Lax-Friedrichs interface fluxes of
 * the six faces, divided by the diagonal mass matrix.  Q and R are device
 * states of this mesh; R must not overlap Q.  Uses the handle's interface-
 * flux buffer. */
dg_status dg_rhs(const dg_mesh *mesh, const void *Q, void *R, void *stream);

/* Stable time step for the current state (the paper states no rule; this
 * library uses dt = cfl * min(hx, hy, hz) / ((2p+1) * Lambda) with
 * Lambda = max over nodes of sum_d (|u_d| + c), c = sqrt(gamma p / rho);
 * DG_FP64: every operation correctly rounded in a fixed order, so dt is
 * reproducible bit for bit; DG_FP32: node speeds in float, the maximum and
 * dt in double).  Writes dt to the DEVICE double *dt_dev,
 * with no host synchronisation.  A node with rho <= 0, p <= 0 or NaN makes
 * dt NaN and sets the DG_ERR_NONFINITE flag.  Errors: DG_ERR_ARG (cfl <= 0). */
dg_status dg_cfl_dt(const dg_mesh *mesh, const void *Q, double cfl, double *dt_dev,
                    void *stream);

/* One step of the five-stage fourth-order 2N-storage Runge-Kutta scheme
 * (Carpenter & Kennedy 1994; Sec. VI.A "LSERK45") with the time step read
 * from the DEVICE double *dt_dev:  for s = 1..5:
 *     dQ <- A_s dQ + dt * dQ/dt(Q),   Q <- Q + B_s dQ      (A_1 = 0)
 * Q is updated in place; dQ is a device state-sized register whose incoming
 * contents are ignored (it holds the last stage's increment on return).
 * Each stage evaluates the right-hand side of the whole mesh at the
 * stage-start state.  Uses the handle's interface-flux buffer. */
dg_status dg_rk_step(const dg_mesh *mesh, void *Q, void *dQ, const double *dt_dev,
                     void *stream);

/* One stage of dg_rk_step's scheme (stage = 0..4, A_1 = 0):
 *     dQ <- A_s dQ + dt * dQ/dt(Qin),   Qout <- Qin + B_s dQ
 * with the right-hand side of the whole mesh at Qin.  Five calls with
 * stages 0..4 are one LSERK45 step (for DG_FP64 with Qin == Qout they equal
 * dg_rk_step bit for bit; for DG_FP32 Qout must be another state buffer,
 * because neighbouring elements still read Qin while the stage writes, and
 * the stages alternate between two states).  The stage-by-stage form is what
 * a z slab (below) needs: its halo traces change between stages.  Errors:
 * DG_ERR_ARG (NULL, stage out of range, dQ equal to Qin or Qout, Qin == Qout
 * for DG_FP32, unaligned states), DG_ERR_UNSUPPORTED (a DG_FP32 slab whose
 * degree runs the tile stage kernel). */
dg_status dg_rk_stage(const dg_mesh *mesh, const void *Qin, void *Qout, void *dQ,
                      const double *dt_dev, int stage, void *stream);

/* z slabs: one periodic mesh partitioned across GPUs (Sec. III and Sec. IV:
 * the paper splits its mesh over MPI ranks, each GPU holding a partition, and
 * neighbouring partitions exchange element face data every stage).
 *
 * A slab is a dg_mesh of nz layers of a taller box that is periodic in x and
 * y (create it with the slab's own z0 and Lz = nz * hz, hz the element size
 * of the whole box).  dg_mesh_set_zhalo makes its z boundary an interface to
 * other slabs instead of the periodic wrap: the -z neighbour of layer 0 and
 * the +z neighbour of layer nz-1 are then known only through their face
 * traces, read from two caller-owned DEVICE buffers of the state's scalar
 * type, each 5 * nx*ny * N^2 values in the layout H[field][ey*nx + ex][j*N + i]
 * (face point (i, j) of the element column (ex, ey)):
 *     halo_lo  the +z-end traces of the layer below layer 0
 *     halo_hi  the -z-end traces of the layer above layer nz-1.
 * The handle keeps the pointers (not the contents): every later dg_rhs and
 * dg_rk_stage reads the buffers as they are when its kernels run.  Passing
 * two NULLs restores the periodic wrap.  For DG_FP64 the first call
 * allocates the handle's buffer for the -z interface fluxes of layer 0
 * (5 * nx*ny * N^2 doubles).  dg_rk_step and dg_advance return
 * DG_ERR_UNSUPPORTED while halos are set (their stages would need new halos
 * in between); dg_cfl_dt and dg_norms are local and unchanged.
 *
 * dg_zhalo_traces writes what the slab's neighbours need, in the same
 * layout: send_lo = layer 0's traces at its -z end (the halo_hi of the slab
 * below), send_hi = layer nz-1's traces at its +z end (the halo_lo of the
 * slab above).  The traces are computed with the same arithmetic as the
 * stage kernels' own, so a mesh split into slabs whose halos are filled from
 * their neighbours' dg_zhalo_traces before every stage evolves bit for bit
 * as the undivided mesh (time steps: the minimum of the slabs' dg_cfl_dt,
 * which equals the undivided mesh's; integrals: the sums of the slabs').
 *
 * Errors: DG_ERR_ARG (NULL mesh or state, one halo NULL and the other not,
 * send_lo == send_hi), DG_ERR_UNSUPPORTED (a DG_FP32 mesh whose degree runs
 * the tile stage kernel), DG_ERR_OOM. */
dg_status dg_mesh_set_zhalo(dg_mesh *mesh, const void *halo_lo, const void *halo_hi);
dg_status dg_zhalo_traces(const dg_mesh *mesh, const void *Q, void *send_lo, void *send_hi,
                          void *stream);

/* Quadrature integrals of the state with the collocated rule (weight
 * J w_i w_j w_k per node, J = hx hy hz / 8), accumulated in double in a fixed
 * order (the result is bitwise reproducible for a given mesh):
 *   out[0..4] = integral of each conserved field,
 *   out[5]    = integral of the kinetic energy |rho u|^2 / (2 rho),
 *   out[6]    = ||Q - Qref|| / ||Qref|| (L2 over the five fields), 0 if Qref is NULL.
 * out is a DEVICE array of DG_NORMS_LEN doubles, written asynchronously. */
dg_status dg_norms(const dg_mesh *mesh, const void *Q, const void *Qref, double *out,
                   void *stream);

/* nsteps steps of the loop "time step, LSERK45 step, integrals" in one call
 * (an addition of this library, not in the paper).  For k = 0 .. nsteps-1:
 *     dts[k]                     = the dg_cfl_dt time step of the current Q,
 *     Q                          <- dg_rk_step(Q, dQ, &dts[k]),
 *     integ[k*DG_NORMS_LEN ...]  = dg_norms(Q, NULL) of the new Q (if integ).
 * Q, dts and integ are those of the separate calls, bit for bit.  The
 * integrals of a step and the maximum wave speed for the next step's time
 * step come from one read of the new state.  DG_FP32: the steps alternate
 * between Q and the handle's second state (a step's fifth stage writes only
 * the new state, into the buffer the step did not start from; the next
 * step's first stage does not read dQ), so no copy of the state is made per
 * step; after an odd nsteps the result is copied into Q once.  On return dQ
 * holds the RK register of the last step's fourth stage (DG_FP32; DG_FP64:
 * as dg_rk_step leaves it): callers treat it as scratch.
 * dts and integ (nullable) are DEVICE arrays of nsteps and
 * nsteps * DG_NORMS_LEN doubles; Q and dQ as for dg_rk_step.  A non-positive
 * density or pressure met by any time-step evaluation sets the
 * DG_ERR_NONFINITE flag as dg_cfl_dt does.  Errors: DG_ERR_ARG (NULL, Q == dQ,
 * unaligned states, cfl <= 0, nsteps < 1). */
dg_status dg_advance(const dg_mesh *mesh, void *Q, void *dQ, double cfl, int nsteps,
                     double *dts, double *integ, void *stream);

/* dg_advance on a state that lives in HOST memory (an addition of this
 * library): Q_host (the state, layout as above, read and overwritten) is
 * copied into the device state Q, dg_advance runs nsteps steps on the device
 * (Q, dQ: caller-owned device buffers as for dg_advance), and the new state,
 * the nsteps time steps and (if integ_host is not NULL) the nsteps *
 * DG_NORMS_LEN integrals are copied back into Q_host, dts_host and
 * integ_host.  The call returns once `stream` has finished all of it
 * (synchronises).  Host buffers should be page-locked (cudaHostAlloc, a
 * pinned torch tensor): pageable memory works but is staged by the driver.
 * DG_FP64 with a page-locked Q_host: the state moves in 8 ranges of whole z
 * layers on a stream and events the mesh creates on the first such call: in,
 * with the first time-step reduction and the first stage's face kernel
 * following each range as it lands; back, each range of the new state while
 * the last stage computes the next ranges and the integrals (the same
 * kernels and floats as dg_advance).  The time steps and integrals pass through a device buffer
 * the mesh keeps for the largest nsteps so far (the first call, or a larger nsteps,
 * allocates it: not for code that cannot allocate).  Errors: those of
 * dg_advance (checked before any copy), DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_advance_host(dg_mesh *mesh, void *Q_host, void *Q, void *dQ, double cfl, int nsteps,
                          double *dts_host, double *integ_host, void *stream);

/* Per-kernel timing, the library's counterpart of the per-kernel breakdown
 * the paper reports (Sec. VI.B, Table II: Volume, Surface, Update-Project).
 * Between dg_profile_begin and dg_profile_end every kernel launch made for
 * this mesh is bracketed by two CUDA events recorded on its launching stream.
 * dg_profile_end synchronises on the last event, and writes, per kernel kind
 * (array index), the summed device time in milliseconds and the number of
 * launches:
 *   DG_KERNEL_FACE   interface traces + Lax-Friedrichs fluxes (DG_FP64)
 *   DG_KERNEL_VOLUME volume flux derivative + lift + (RK update or rhs write)
 *                    (DG_FP64)
 *   DG_KERNEL_CFL    time-step reduction (two launches counted as one)
 *   DG_KERNEL_NORMS  integrals (two launches counted as one)
 *   DG_KERNEL_INIT   initial state
 *   DG_KERNEL_STAGE  fused single-pass stage: faces, volume, lift and update
 *                    or rhs write in one kernel (DG_FP32)
 *   DG_KERNEL_COPY   device copy of the second state back to Q after the
 *                    five ping-pong stages of a DG_FP32 step
 *   DG_KERNEL_EPILOGUE dg_advance's pass at the end of a step: integrals and
 *                    next time step (and the DG_FP32 fifth-stage update),
 *                    with their one-block final reductions
 * ms and launches are HOST arrays of DG_PROFILE_KINDS entries.  Recording
 * costs one event pair per launch; begin discards earlier records. */
#define DG_PROFILE_KINDS 8
enum { DG_KERNEL_FACE = 0, DG_KERNEL_VOLUME = 1, DG_KERNEL_CFL = 2, DG_KERNEL_NORMS = 3,
       DG_KERNEL_INIT = 4, DG_KERNEL_STAGE = 5, DG_KERNEL_COPY = 6, DG_KERNEL_EPILOGUE = 7 };
dg_status dg_profile_begin(dg_mesh *mesh);
dg_status dg_profile_end(dg_mesh *mesh, double *ms, int64_t *launches);

/* Tile shapes of the DG_FP32 fused stage (an implementation choice, not in
 * the paper).  The fused stage works on tiles of TX x TY elements of one z
 * layer; each polynomial degree has a few tile variants, and a process-wide
 * table selects one per degree (default variant 0).  The table is read at
 * every DG_FP32 mesh launch and when a batch is created; it is meant to be
 * filled once from an autotuner's results before work starts (not changed
 * while kernels of the process are being enqueued from other threads).
 *   dg_tile_variant_count  number of variants for degree p (0 if p unsupported)
 *   dg_tile_shape          (TX, TY) of a variant
 *   dg_set_tile_variant    select a variant (DG_ERR_ARG if out of range)
 *   dg_get_tile_variant    selected variant (-1 if p unsupported) */
int dg_tile_variant_count(int p);
dg_status dg_tile_shape(int p, int variant, int *tx, int *ty);
dg_status dg_set_tile_variant(int p, int variant);
int dg_get_tile_variant(int p);

/* Stage kernel of the DG_FP32 single-mesh path (an implementation choice,
 * not in the paper), per degree in a process-wide table like the tile table
 * above (same threading rule; a batch's shared instances always run the line
 * kernel, its own-launch instances follow this table):
 *   DG_STAGE_TILE    one CTA per tile of one z layer (the tile variant above);
 *                    the neighbour's face-normal lines read through L2
 *   DG_STAGE_COLUMN  one CTA per column of elements, walking up a chunk of z
 *                    layers with the next layers prefetched into shared
 *                    memory (cp.async); every z interface computed once
 *   DG_STAGE_LINES   the same column walk with one thread per z node line:
 *                    z fluxes, z traces and z interface fluxes stay in
 *                    registers; the same floats as DG_STAGE_COLUMN
 * All give the same right-hand side up to float rounding order.
 *   dg_set_stage_kernel  DG_ERR_UNSUPPORTED for p outside [0, DG_MAX_P],
 *                        DG_ERR_ARG for an unknown kind
 *   dg_get_stage_kernel  the kind (-1 if p unsupported); default DG_STAGE_LINES */
enum { DG_STAGE_TILE = 0, DG_STAGE_COLUMN = 1, DG_STAGE_LINES = 2 };
dg_status dg_set_stage_kernel(int p, int kind);
int dg_get_stage_kernel(int p);

/* Batches: many independent DG_FP32 meshes advanced together (the paper
 * solves one mesh; batching uneven independent problems is an addition).
 * Each instance is a periodic box like a dg_mesh (same meaning of nx..gamma)
 * with caller-owned float device states Q (the solution) and dQ (the RK
 * register), in the layout above.  dg_batch_create computes every instance's
 * operators, allocates one second state per instance (the stage's ping-pong
 * buffer) unless the caller gives one, and the per-instance time steps.
 * dg_batch_step advances every instance by nsteps LSERK45 steps, each with
 * its own CFL time step (same rule as dg_cfl_dt): per step one launch
 * computes all the shared instances' time steps, then, per RK stage, one
 * launch per polynomial degree runs the single-mesh line stage kernel's body
 * (DG_STAGE_LINES) over work items (instance, column of elements, chunk of
 * at most 8 z layers) of every shared instance of that degree.  Instances of
 * at least dg_get_batch_direct_nodes() nodes (default 2^13) are not shared:
 * each runs the single-mesh stage kernel of its degree (dg_set_stage_kernel)
 * in launches of its own, on up to four streams the batch owns, forked from
 * `stream` after the time steps and joined back to it at the end of every
 * step, so that they overlap one another and the shared launches.  Either
 * way an instance's result is that of the same mesh stepped alone with the
 * same stage kernel (the line kernel for shared instances), bit for bit.
 * The stages alternate between Q and the batch's second states,
 * so an even number of steps ends in Q by itself; after an odd number the
 * second states are copied back (one device memcpy per instance).  With
 * use_graph != 0 the launches of two steps (and of one step) are recorded
 * once into CUDA graphs on `stream` (a created stream, not the legacy
 * default) and replayed; a changed cfl records new graphs.  Calls on one
 * batch must be ordered.
 * dg_batch_sizes returns the total DOF and the number of shared stage work
 * items; dg_batch_dt copies the time steps of the last step to a HOST array
 * of n doubles (synchronises); dg_batch_norms writes instance idx's
 * integrals as dg_norms does; dg_batch_state_init fills instance idx's Q like
 * dg_state_init; dg_batch_last_error reads and clears the batch's
 * non-finite flag.  Errors as for dg_mesh_create and dg_rk_step.
 * dg_set_batch_direct_nodes sets that size threshold for batches created
 * afterwards (process-wide, like the tuning tables; 0: every instance runs its
 * own launches; INT64_MAX: all are shared); DG_ERR_ARG for a negative
 * value. */
typedef struct {
    int nx, ny, nz, p;
    double x0, y0, z0, Lx, Ly, Lz, gamma;
    void *Q;  /* float device state of the instance (caller-owned) */
    void *dQ; /* float device RK register, state-sized (caller-owned) */
    void *Qt; /* optional float device second state, state-sized (caller-owned);
                 NULL: the batch allocates one and frees it with the batch */
} dg_instance;
typedef struct dg_batch dg_batch;
dg_status dg_batch_create(int n, const dg_instance *instances, dg_batch **out);
void dg_batch_destroy(dg_batch *batch);
/* Replace a batch's instance list by a new one (any n, sizes and degrees:
 * requests joining and leaving a serving loop), as if the batch had been
 * created for it, keeping its device arrays and streams where they are large
 * enough (no allocation, free or device-wide synchronisation when they are;
 * second states the batch allocated for the old list are freed).  Recorded
 * graphs are dropped and recorded again at the next graph step.  The batch
 * must be idle: every step enqueued on it has completed (the new
 * descriptors are copied over the old ones).  Errors as dg_batch_create; on
 * an error the batch holds no instances until a successful update. */
dg_status dg_batch_update(dg_batch *batch, int n, const dg_instance *instances);
dg_status dg_set_batch_direct_nodes(int64_t nodes);
int64_t dg_get_batch_direct_nodes(void);
dg_status dg_batch_sizes(const dg_batch *batch, int64_t *n_dof, int64_t *n_items);
dg_status dg_batch_state_init(const dg_batch *batch, int idx, dg_init_kind kind,
                              const double *params, int nparams, void *stream);
dg_status dg_batch_step(dg_batch *batch, double cfl, int nsteps, int use_graph, void *stream);
dg_status dg_batch_dt(const dg_batch *batch, double *dt_host);
dg_status dg_batch_norms(const dg_batch *batch, int idx, const void *Qref, double *out,
                         void *stream);
dg_status dg_batch_last_error(const dg_batch *batch);

/* Allocation-free right-hand side (the paper has no counterpart).
 *
 * Some callers cannot let a library allocate device memory: code that runs
 * under a fixed device-memory budget, or inside a host framework whose own
 * allocator already holds the free memory and forbids allocations by
 * plugins.  Such callers cannot create a dg_mesh, because dg_mesh_create
 * allocates the handle's workspace.  This entry point evaluates the same
 * dQ/dt as dg_rhs for the mesh its arguments describe (the arguments mean what
 * they mean for dg_mesh_create) without allocating or freeing anything: the
 * 1D operators are computed on the host on every call.  Q and R are
 * caller-owned device states in the layout above, double for DG_FP64 and
 * float for DG_FP32, each exactly 5 * nx*ny*nz*(p+1)^3 scalars (the library
 * cannot check their size: a smaller buffer is read or written out of
 * bounds); R must not overlap Q.
 *
 * DG_FP64 needs scratch for the interface fluxes: it lives in one static
 * device array of DG_STATIC_SCRATCH_BYTES (16 MiB) that every GPU which
 * loads this library holds until the process exits.
 *   Size limit: 15 * nx*ny*nz*(p+1)^2 doubles; a mesh that needs more is
 *   rejected with DG_ERR_TOO_LARGE before anything is enqueued (p = 4 fits
 *   up to 5,592 elements, 16^3 = 4,096 does).
 *   Set-up: the first DG_FP64 call on each device looks up the device
 *   address of the static array (cudaGetSymbolAddress, with that device
 *   current) and keeps it for the life of the process; make that first call
 *   before any stream capture.  A device reset (cudaDeviceReset) between
 *   calls is not supported: the kept address would no longer be valid.
 *   Sharing: every DG_FP64 call uses the same array, which keeps whatever
 *   the last call left in it (each call writes the part it reads before
 *   reading it, so nothing needs clearing).  Calls whose GPU work can
 *   overlap -- issued on different streams, or from several host threads --
 *   race on the array; the caller must order them.
 * DG_FP32 needs no scratch (its single-pass kernel keeps the interface
 * fluxes in shared memory): no size limit beyond dg_mesh_create's, no set-up
 * and no sharing between calls.
 *
 * Errors: DG_ERR_ARG / DG_ERR_UNSUPPORTED for the argument checks of
 * dg_mesh_create and dg_rhs, DG_ERR_TOO_LARGE as above, DG_ERR_CUDA if the
 * set-up or a launch fails. */
#define DG_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
dg_status dg_rhs_static(int nx, int ny, int nz, int p,
                        double x0, double y0, double z0,
                        double Lx, double Ly, double Lz,
                        double gamma, dg_precision precision,
                        const void *Q, void *R, void *stream);

/* Measured multiply-add throughput of the current GPU's CUDA cores in
 * flop/s (an FMA counts 2) at the given precision: independent FMA chains
 * on every resident thread of the device, one untimed and one timed launch
 * (about 20 ms; synchronises the device).  The roofline denominator of the
 * double-state kernels, whose time goes to the FP64 pipe (the paper reports
 * its kernels against the V100's peak flop rate, Sec. VI.B, Table II).  ms
 * (nullable) receives the timed launch's duration.  Allocates and frees a
 * few bytes of device memory.  Errors: DG_ERR_ARG, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_fma_throughput(dg_precision precision, double *flop_per_s, double *ms);

/* Measured FP64 tensor-core (DMMA) throughput of the current GPU in flop/s:
 * independent accumulators through mma.sync m8n8k4 f64 (512 flop per warp
 * instruction) on every resident warp; with mix = 1 the odd warps run FP64
 * FMA chains of the same flop count instead, which shows whether the two
 * kinds of FP64 work share one pipe.  Answers whether the sum-factorised
 * contractions (N x N matrices, N <= 7) could move to tensor cores.  Same
 * conventions as dg_fma_throughput. */
dg_status dg_dmma_throughput(int mix, double *flop_per_s, double *ms);

/* Self-check of the double form's sound-speed square root (a refined
 * reciprocal-square-root approximation, not the correctly rounded sqrt):
 * for n positive doubles a (DEVICE), writes the kernels' root to fast[] and
 * CUDA's correctly rounded __dsqrt_rn to ieee[] (both DEVICE, n doubles),
 * asynchronously on stream.  Lets a test bound the difference in ulp. */
dg_status dg_selfcheck_sqrt(const double *a, double *fast, double *ieee, int64_t n, void *stream);

/* Static text for a status code. */
const char *dg_status_string(dg_status status);

/* Read and clear the handle's sticky device error flag (synchronises the
 * device).  DG_OK if no kernel raised it since the last read. */
dg_status dg_last_error(const dg_mesh *mesh);

#ifdef __cplusplus
}
#endif

#endif /* DG_GB300_H */
