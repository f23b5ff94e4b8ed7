/*
 * sllbm.h -- C ABI of the GB300 semi-Lagrangian lattice Boltzmann step library
 * (libsllbm.so).  Implements the per-time-step fused update of the compressible
 * 3D SLLBM of arXiv:2012.05537 (Wilde, Kraemer, Reith, Foysi) with the 45-velocity
 * degree-9 cubature set: semi-Lagrangian streaming by cell-oriented Lagrange
 * interpolation on Gauss-Lobatto-Chebyshev support points (Sec. II.A, Eq.
 * interpolation), moments (Eq. moments), fourth-order Hermite equilibrium (Eq.
 * discreteEquilibrium, App. A, App. B), the second energy population g, pressure-
 * dependent relaxation time with Sutherland viscosity (Sec. II.A, Sec. III.C), BGK
 * collision (Eq. LBM) and the optional quasi-equilibrium Prandtl term (App. D).
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  Units      lattice units with c_s^2 = T_ref = 1; the Hermite tensors use xi/c_s.
 *  Mesh       periodic, uniform hexahedral cells, cells[d] per direction on
 *             [0, L[d]); order-p Gauss-Lobatto-Chebyshev support points, p in {2,3,4};
 *             N[d] = cells[d]*p unique nodes per direction (a cell's right-face nodes
 *             are the next cell's left-face nodes).  Node (x,y,z) has index
 *             n = (z*N[1] + y)*N[0] + x (x fastest); along a direction the node
 *             c*p + a (a in [0,p)) sits at c*h + (1 - cos(pi a/p)) h/2, h = L/cells.
 *  Velocities the 45 abscissae in the order returned by sllbm_velset_table():
 *             origin; icosahedron |xi|=sqrt(3); dodecahedron |xi|=3; icosahedron
 *             |xi|=sqrt(15).
 *  Populations a state buffer holds the 2*45 populations of every node in the storage
 *             type (SLLBM_F64: double, SLLBM_F32: float, SLLBM_F16DEV: IEEE half,
 *             SLLBM_BF16DEV: bfloat16; the 16-bit types hold deviations, see
 *             sllbm_storage) in the order
 *             buf[i][z][y][x][h]: velocity slowest, then the node, then h = 0 for f and
 *             h = 1 for g, so f_i and g_i of a node sit side by side.  The FP64
 *             interface of sllbm_set_populations / sllbm_get_populations uses the order
 *             pop[h][i][z][y][x] instead.  The stored state is the post-collision
 *             population; sllbm_step() streams it (pull, departure point x - dt*xi_i)
 *             and collides the result, ping-ponging two buffers.
 *  Streams    every call that touches the GPU is enqueued on the CUDA stream given
 *             to sllbm_create() and is asynchronous unless stated otherwise.
 *  Errors     every int-returning call returns SLLBM_OK (0) or a negative SLLBM_E*
 *             code; no call aborts the process.  After SLLBM_ECUDA the CUDA error is
 *             kept in the context (sllbm_last_cuda_error).
 *  Ownership  the context owns its small tables (and, if no buffers were given, its
 *             population buffers).  Buffers given to sllbm_set_buffers() stay owned by
 *             the caller and must outlive the context's use of them.
 */
#ifndef SLLBM_H
#define SLLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SLLBM_OK 0
#define SLLBM_EINVAL (-1)     /* bad argument (size, order, null pointer, ...) */
#define SLLBM_ENOMEM (-2)     /* device or host allocation failed */
#define SLLBM_ECUDA (-3)      /* a CUDA runtime call failed; see sllbm_last_cuda_error */
#define SLLBM_ENONFINITE (-4) /* non-finite or non-positive rho/T seen by the step check */
#define SLLBM_ETIMEOUT (-5)   /* a bounded device-side wait gave up */
#define SLLBM_ENOTREADY (-6)  /* population buffers not set or not initialised */
#define SLLBM_EABORTED (-7)   /* a launch ended early on a host abort request (sllbm_request_abort) */
#define SLLBM_EIO (-8)        /* a checkpoint file could not be opened, written or read */

typedef struct sllbm_ctx sllbm_ctx; /* opaque */

/* Periodic uniform hexahedral mesh (Sec. III.C uses the triply periodic [0,2 pi]^3). */
typedef struct {
    int cells[3];  /* cells per direction, >= 1 */
    double L[3];   /* domain lengths */
} sllbm_mesh;

typedef enum { SLLBM_D3Q45 = 0 } sllbm_velset;

typedef enum {
    SLLBM_F64 = 0,     /* double populations, FP64 arithmetic */
    SLLBM_F32 = 1,     /* float populations, FP32 arithmetic */
    SLLBM_F16DEV = 2,  /* IEEE half deviations, FP32 arithmetic (see below) */
    SLLBM_BF16DEV = 3  /* bfloat16 deviations, FP32 arithmetic (see below) */
} sllbm_storage;
/* Mixed-precision storage: SLLBM_F16DEV and SLLBM_BF16DEV store, per node and velocity,
 * d_i = f_i/w_i - rho0 and d_gi = g_i/w_i - (2 C_v - 3) T0 rho0 (rho0, T0 of the context's
 * parameters) in 16 bits.  The step interpolates the deviations in FP32 (the Lagrange
 * weights of each pass sum to one), forms rho - rho0, rho u and 2 rho (T - T0) C_v from
 * deviation sums with the exact quadrature identities sum w_i = 1, sum w_i xi_i = 0,
 * sum w_i |xi_i|^2 = 3 (no cancellation against the reference state), collides in FP32 and
 * stores deviations again.  Both step kernels run these types. */

/* Physical and run parameters.  Taylor-Green scaling (Sec. III.C): U0 = Ma*sqrt(gamma*T0),
 * mu_inf = rho0*U0*1/Re (reference length 1), unless mu_inf_override > 0. */
typedef struct {
    double Ma;              /* Mach number of the Taylor-Green initial field */
    double Re;              /* Reynolds number, Re = U0 L / nu_inf with L = 1 */
    double Pr;              /* Prandtl number used by the App. D term */
    double gamma;           /* heat capacity ratio; C_v = 1/(gamma-1) */
    double T0;              /* uniform initial temperature of the TGV field */
    double rho0;            /* reference density of the TGV field */
    double dt_or_courant;   /* time step dt, or Courant number if dt_is_courant */
    int dt_is_courant;      /* 1: dt = C * min_d(L[d]/N[d]) / max_i|xi_i| (C = Courant number) */
    int pr_correction;      /* 1: apply the quasi-equilibrium Prandtl term (App. D) */
    sllbm_storage storage;  /* population storage / arithmetic type */
    int nonfinite_check;    /* 1: the step kernel flags non-finite rho or T (in the collision:
                               a stream-only context does not check) */
    double tgv_C;           /* density numerator C of the TGV field; < 0 selects gamma*Ma^2 */
    double mu_inf_override; /* > 0: use this mu_inf instead of rho0*U0/Re */
    int collide;            /* 1: stream and collide (normal); 0: stream only */
    int kernel;             /* step kernel: 0 automatic, 1 generic tile kernel, 2 TMA-fed
                               persistent kernel (FP32 and the 16-bit deviation storages, the
                               Prandtl term with FP32 storage; needs
                               N[0] a multiple of 2 (FP32) or 4 (16-bit), cells divisible by its
                               tile of 4x4x2 (p = 2), 2x3x1 (p = 3: y may end in a partial
                               tile) or 2x2x1 cells (p = 4), collide on, not both the
                               Prandtl term and compensated sums; else SLLBM_EINVAL).
                               Automatic: the TMA-fed kernel where it can run and the mesh
                               (a slab: its interior) has at least 0.5 M (p = 2), 3 M
                               (p = 3) or 1.5 M (p = 4) nodes, except with the Prandtl term,
                               at p = 3 with 16-bit storage outside slab contexts, and with
                               compensated moment sums at p = 3, or at p = 4 with 16-bit
                               storage outside slab contexts (the faster kernel in each
                               case, as measured) */
} sllbm_params;

/* Read-only description of a created context. */
typedef struct {
    int N[3];          /* nodes per direction */
    int p;             /* polynomial order */
    int64_t nodes;     /* N[0]*N[1]*N[2] */
    int Q;             /* 45 */
    double dt;         /* time step */
    double U0;         /* TGV velocity amplitude */
    double mu_inf;     /* reference dynamic viscosity */
    double max_xi;     /* largest |xi_i| */
    size_t pop_bytes;  /* bytes of one population buffer (2*Q*nodes*sizeof(storage)) */
    int storage;       /* sllbm_storage */
    int max_cell_shift;/* largest |departure cell shift| over velocities and directions */
    int step_kernel;   /* kernel sllbm_step launches: 1 generic tile kernel, 2 TMA-fed kernel */
    int step_variant;  /* see sllbm_set_step_variant */
} sllbm_info_t;

/* Fills p_out with the defaults used for the paper's Re = 1600 Taylor-Green runs
 * (Sec. III.C): Ma 0.5, Re 1600, Pr 0.7, gamma 1.4, T0 = rho0 = 1, Courant 1,
 * Prandtl term off, FP32 storage, collide on. */
void sllbm_default_params(sllbm_params *p_out);

/* Creates a context: validates mesh/order/params, builds the velocity set, the GLC
 * support points and the per-velocity separable interpolation tables (departure cell
 * shift and p+1 Lagrange weights per velocity, direction and local node index; the
 * uniform-mesh reduction of the matrices Psi_i, Sec. IV.B), and records the stream
 * (cudaStream_t passed as void*, NULL = legacy default stream).  Allocates nothing
 * large on the device.  Errors: SLLBM_EINVAL (cells < 1, p not in {2,3,4}, dt <= 0,
 * a departure shift beyond 100 cells, unknown storage), SLLBM_ENOMEM, SLLBM_ECUDA. */
int sllbm_create(const sllbm_mesh *mesh, int p, sllbm_velset vs, const sllbm_params *prm,
                 void *cuda_stream, sllbm_ctx **out);

/* Domain decomposition along z (one process or context per part of a mesh too large for
 * one device).  The pull streaming of Sec. II.A reads, for a node, only the (p+1)^3
 * support points of the cell its departure point falls in, at most max_cell_shift cells
 * away, so a slab of consecutive z-cells advances exactly like the whole periodic mesh
 * once the cells next to it hold the neighbouring slabs' current state.
 *
 * sllbm_create_slab creates a context for the interior cells [z_begin, z_begin + z_cells)
 * of the periodic mesh `mesh` (same arguments and errors as sllbm_create otherwise).
 * Its state holds ghost = max_cell_shift + 1 cells of halo below and above the interior:
 * N[2] = (z_cells + 2 ghost) p planes in the usual layout, with the z-cells numbered on
 * the whole mesh (cell z_begin - ghost first, periodic), so sllbm_init_tgv and
 * sllbm_init_fields set the slab's part of the whole-mesh fields, and sllbm_step updates
 * the interior planes only (the generic tile kernel, or the TMA-fed kernel where the
 * interior cells are whole tiles of it: its source boxes then reach into the ghost planes
 * and never wrap along z).  Before every step the caller refreshes
 * the halos: sllbm_halo_pack(side 0) copies lowest interior planes of the current state to
 * a device buffer for the slab below, sllbm_halo_pack(side 1) highest ones for the slab
 * above; sllbm_halo_unpack(side 0 / 1) writes a buffer received from the slab below / above
 * into the ghost planes below / above.  Only the planes a velocity's source boxes reach
 * are moved: with kmin and kmin + span the smallest and largest departure cell shift of
 * velocity i along z, the ghost region below holds -kmin cells of it (kmin < 0) and the
 * one above (kmin + span) cells plus the shared face plane (kmin + span >= 0); its other
 * ghost planes are never read.  A packed buffer holds, velocity after velocity, those
 * planes in the order [plane][y][x][h]: sllbm_slab_halo_bytes(side) bytes for what
 * sllbm_halo_pack(side) writes and the neighbour's sllbm_halo_unpack(1 - side) reads
 * (halo_bytes of sllbm_slab_info is the larger of the two sides); device memory owned by
 * the caller; both calls are one asynchronous kernel launch on cuda_stream (a cudaStream_t
 * as void*; NULL: the context's stream).
 *
 * To overlap the exchange with the step, split it: sllbm_step_begin launches the tiles
 * whose source cells are all interior (they read no ghost cell; nothing is swapped yet),
 * sllbm_step_end the remaining tiles next to the ghost cells, and then swaps the state as
 * sllbm_step does (and, with the non-finite check on, synchronises and reports it as
 * sllbm_step does).  Between the two the caller packs, exchanges and unpacks the halos of
 * the current state on another stream (packing reads, and unpacking writes, nothing the
 * interior tiles touch) and makes the context's stream wait for the unpacks before
 * sllbm_step_end.  The result equals sllbm_step's bit for bit.
 * Errors: SLLBM_EINVAL for z_begin outside the mesh, z_cells < 1 or above the mesh, a
 * slab thinner than its ghost width (its halo would come from two neighbours), a TMA-fed
 * kernel request the interior cells cannot tile, and for slab contexts that are a part of a
 * mesh (not all of it) in sllbm_diag*, the
 * reverse-mode calls and batches; sllbm_halo_*, sllbm_slab_info and
 * sllbm_step_begin/_end on a context that is not a slab, side not 0 or 1, a NULL buffer or
 * a context without state: SLLBM_EINVAL (sllbm_step_begin/_end before initialisation:
 * SLLBM_ENOTREADY); a failed copy or launch: SLLBM_ECUDA. */
int sllbm_create_slab(const sllbm_mesh *mesh, int p, sllbm_velset vs, const sllbm_params *prm,
                      int z_begin, int z_cells, void *cuda_stream, sllbm_ctx **out);
int sllbm_slab_info(const sllbm_ctx *ctx, int *ghost_cells, size_t *halo_bytes);
int sllbm_slab_halo_bytes(const sllbm_ctx *ctx, int side, size_t *bytes);
int sllbm_halo_pack(sllbm_ctx *ctx, int side, void *halo, void *cuda_stream);
int sllbm_halo_unpack(sllbm_ctx *ctx, int side, const void *halo, void *cuda_stream);
/* For a slab that spans the whole mesh along z (z_begin = 0, z_cells = mesh cells): the
 * periodic halo refresh in place, one kernel launch on cuda_stream (NULL: the context's
 * stream) that copies, per velocity, the interior planes each ghost region needs from the
 * opposite end of the interior (what packing, exchanging and unpacking with itself would
 * do).  sllbm_step (and every call that steps: sllbm_run_host, sllbm_run_host_many,
 * sllbm_autotune) and sllbm_step_begin make this refresh themselves before each step of
 * such a slab, so it advances the periodic mesh exactly as an ordinary context does, bit
 * for bit, with no exchange by the caller; the TMA-fed kernel then never loads source boxes
 * that wrap around along z (about 20 % faster on the 128^3-node mesh).  SLLBM_EINVAL for
 * other contexts. */
int sllbm_halo_periodic(sllbm_ctx *ctx, void *cuda_stream);
int sllbm_step_begin(sllbm_ctx *ctx);
int sllbm_step_end(sllbm_ctx *ctx);

/* Frees everything the context owns (not caller buffers). NULL is accepted. */
void sllbm_destroy(sllbm_ctx *ctx);

/* Copies the context description into *info. */
int sllbm_get_info(const sllbm_ctx *ctx, sllbm_info_t *info);

/* Velocity set (Sec. II.B): xi[45*3] (row-major, x,y,z) and w[45], host pointers. */
int sllbm_velset_table(const sllbm_ctx *ctx, double *xi, double *w);

/* Gives the context two device buffers of pop_bytes each (caller-owned, e.g. torch
 * tensors); popA becomes the current state.  bytes < pop_bytes -> SLLBM_EINVAL.
 * If never called, sllbm_init_* allocates two buffers owned by the context. */
int sllbm_set_buffers(sllbm_ctx *ctx, void *popA, void *popB, size_t bytes);

/* Device pointer to the buffer holding the current state (NULL before init). */
void *sllbm_current_buffer(const sllbm_ctx *ctx);

/* Taylor-Green initialisation (Sec. III.C, constant-temperature initial condition):
 * f_i = f_i^eq(rho, u, T0), g_i = (2C_v - D) T0 f_i^eq at every node, computed in FP64. */
int sllbm_init_tgv(sllbm_ctx *ctx);

/* Equilibrium initialisation from given FP64 fields rho[nodes], u[3][nodes], T[nodes]
 * (host pointers if on_device == 0, device pointers otherwise). */
int sllbm_init_fields(sllbm_ctx *ctx, const double *rho, const double *u, const double *T,
                      int on_device);

/* Sets the current state from FP64 populations pop[2][45][nodes] (host or device),
 * rounding to the storage type. */
int sllbm_set_populations(sllbm_ctx *ctx, const double *pop, int on_device);

/* Copies the current state to FP64 pop[2][45][nodes] (host or device).  Synchronous
 * when on_device == 0. */
int sllbm_get_populations(sllbm_ctx *ctx, double *pop, int on_device);

/* Advances n >= 0 time steps: each step is one launch of the fused kernel (pull
 * streaming of all 90 populations, moments, equilibrium, BGK [+ Prandtl term]),
 * alternating the two buffers.  Asynchronous.  With nonfinite_check on, the
 * check flags are read back (synchronising) after the last step: SLLBM_ETIMEOUT if a
 * bounded device wait gave up, SLLBM_ENONFINITE if any node had non-finite or
 * non-positive rho or T. */
int sllbm_step(sllbm_ctx *ctx, int n);

/* Synchronises the stream and reports device-side trouble since the last call: returns
 * SLLBM_ETIMEOUT (and clears it) if a bounded wait inside a step kernel gave up,
 * SLLBM_EABORTED (and clears it) if a launch stopped on an abort request, else SLLBM_OK.
 * Kernels never spin without a limit; after such an error the state is garbage. */
int sllbm_status(sllbm_ctx *ctx);

/* Density, velocity and temperature of the current state, Eq. (moments), FP64:
 * rho[nodes], u[3][nodes], T[nodes]; host pointers (synchronous) if on_device == 0. */
int sllbm_moments(sllbm_ctx *ctx, double *rho, double *u, double *T, int on_device);

/* Sec. III.C diagnostics of the current state, volume-averaged, FP64, host outputs:
 * Ek = <rho|u|^2/2>/(rho0 U0^2), eps_s = <mu/mu_inf |curl u|^2>/(rho0 Re U0^2),
 * eps_c = (4/3)<mu/mu_inf (div u)^2>/(rho0 Re U0^2), with per-cell Clenshaw-Curtis
 * quadrature on the support points and cell-local Lagrange derivatives.
 * Synchronous.  Uses a context-owned device scratch buffer (allocated on first use).
 * A slab context must span the whole mesh (its interior is the mesh; the support points
 * wrap around within it, so the ghost planes are not read): SLLBM_EINVAL for a part of a
 * mesh. */
int sllbm_diag(sllbm_ctx *ctx, double *Ek, double *eps_s, double *eps_c);

/* sllbm_diag without any device allocation (the paper has no counterpart: this is a
 * library-interface matter).  For callers that cannot let the library allocate: their
 * device memory is owned by another allocator or a fixed budget, or their loop must not
 * pay for cudaMalloc/cudaFree (cudaFree synchronises the device).  The scratch is a
 * static device array inside the library holding one partial triple per cell: meshes
 * with more than 65536 cells get SLLBM_EINVAL.  Results equal sllbm_diag's up to the
 * order of the FP64 sums.  sllbm_create looks up the array's device address on the
 * context's device (cudaGetSymbolAddress), so this call does no set-up of its own.  Calls
 * share the array, so calls that overlap on the GPU (other streams or contexts) race.
 * The current device must be the context's (SLLBM_EINVAL otherwise).  Synchronous; host
 * outputs. */
int sllbm_diag_noalloc(sllbm_ctx *ctx, double *Ek, double *eps_s, double *eps_c);

/* End-to-end call with HOST buffers: copies pop_in (pop_bytes, storage type, host
 * memory; pinned for full speed) to the device, advances n steps, copies the result
 * to pop_out (host) and synchronises the stream. */
int sllbm_run_host(sllbm_ctx *ctx, const void *pop_in, void *pop_out, int n);

/* Pipelined end-to-end runs of `count` independent states: state k is copied from HOST
 * pop_in[k] (pop_bytes, storage type; pinned host memory for full speed), advanced n steps
 * and copied back to HOST pop_out[k].  Three device slots (six buffers of pop_bytes,
 * allocated on the first call, separate from the context's buffers) and two copy streams
 * let the device-to-host copy of one state, the host-to-device copy of the next and the
 * steps in between overlap.  The context's own state and buffers are left as they were.
 * Synchronous.  Errors: SLLBM_EINVAL (NULL pointers, count < 1, n < 0), SLLBM_ENOMEM (the
 * slots), SLLBM_ECUDA. */
int sllbm_run_host_many(sllbm_ctx *ctx, const void *const *pop_in, void *const *pop_out, int count, int n);

/* Waits for all work the context enqueued. */
int sllbm_sync(sllbm_ctx *ctx);

/* Copies a state (storage type and order, pop_bytes bytes, device pointer) into the
 * current buffer and marks the context initialised.  Asynchronous.  Errors: SLLBM_EINVAL
 * (NULL), SLLBM_ENOMEM (the context had to allocate its buffers), SLLBM_ECUDA. */
int sllbm_load_state(sllbm_ctx *ctx, const void *state);

/* Sets mu_inf, the viscosity scale of the Sutherland law, which fixes the relaxation time
 * tau = mu_inf (mu/mu_inf)(T) / (rho T dt) + 1/2 (Sec. II.A, Sec. III.C) for the following
 * steps.  SLLBM_EINVAL unless mu_inf > 0. */
int sllbm_set_mu_inf(sllbm_ctx *ctx, double mu_inf);

/* ---- kernel choice, autotuning, batched launch ------------------------------------------
 * A step can run on several kernels with identical results up to FP rounding order: the
 * TMA-fed persistent kernel (FP32 or 16-bit deviations; whole tiles in x and z) and the generic tile
 * kernel with its default tile or, for FP32 storage without the Prandtl term, one of two
 * smaller tiles (more CTAs on small meshes).  Variants: 0 TMA-fed kernel; 1 generic,
 * default tile (FP32: p = 2 4x4x2 cells, p = 3 2x2x2, p = 4 2x2x1); 2 and 3 generic,
 * alternative tiles (p = 2: 4x2x2 and 2x2x1 cells; p = 3: 2x2x1 and 1x1x1; p = 4: 2x1x1 and
 * 1x1x1). */

/* Selects the step kernel of the following steps.  SLLBM_EINVAL if the variant cannot run
 * this context. */
int sllbm_set_step_variant(sllbm_ctx *ctx, int variant);

/* Autotuner: times `steps` steps (CUDA events, after one warm-up step) of every variant
 * that can run this context, starting each from the current state, keeps the fastest and
 * restores the current state (a temporary device copy of one state is allocated).
 * Synchronous.  Outputs (either may be NULL): the chosen variant and its time per step in
 * milliseconds.  Errors: SLLBM_EINVAL (steps < 1), SLLBM_ENOTREADY (not initialised),
 * SLLBM_ENOMEM (the temporary copy), SLLBM_ECUDA; on an error the variant is unchanged. */
int sllbm_autotune(sllbm_ctx *ctx, int steps, int *variant, double *ms_per_step);

/* Batched launch of many contexts (instances of uneven size, order and parameters) as one
 * CUDA graph.  sllbm_batch_create captures two steps of every context, with the contexts
 * spread over `streams` worker streams (longest-processing-time-first on the per-step cost
 * estimate: the autotuned times if every context was autotuned, else the node counts) so
 * that small instances run concurrently; the graph forks from and joins to cuda_stream,
 * which must be a created
 * stream (not the legacy default stream, NULL: SLLBM_EINVAL).  Each context must be
 * initialised, on the current device, with nonfinite_check off, and must not take part in
 * another batch.  The contexts keep ownership of their buffers and stay usable on their
 * own; a batch is invalid (SLLBM_EINVAL from sllbm_batch_step) once one of them was stepped
 * an odd number of times outside it.  Synchronous.  Errors: SLLBM_EINVAL (the conditions
 * above, n < 1, streams < 1, a context given twice), SLLBM_ENOMEM, SLLBM_ECUDA (stream
 * capture or graph instantiation failed; the contexts are left as they were). */
typedef struct sllbm_batch sllbm_batch;
int sllbm_batch_create(sllbm_ctx *const *ctxs, int n, int streams, void *cuda_stream, sllbm_batch **out);

/* Advances every context of the batch by nsteps (even, >= 0) steps: nsteps/2 graph
 * launches on the batch's stream, ordered after work already queued on the contexts'
 * streams and before work queued on them later.  Asynchronous.  Errors: SLLBM_EINVAL (odd or
 * negative nsteps, or a context stepped an odd number of times outside the batch),
 * SLLBM_ECUDA. */
int sllbm_batch_step(sllbm_batch *b, int nsteps);

/* The same, as ONE persistent kernel launch per polynomial order and step: every context
 * of order p is a job of a work list of (context, tile) items that persistent CTAs (grid =
 * SMs x resident CTAs) walk, each tile with the generic kernel's tile body and the context's
 * own arguments and tables (copied to shared memory when a CTA moves to another context);
 * the launches of the (up to three) orders run on separate worker streams and two steps
 * are captured into one graph.  With tune_steps > 0 an autotuner picks the tile shape per
 * order (the default tile, one size smaller, one cell): it times tune_steps (rounded up to
 * even) replays of the captured graph, from the current states, keeps another shape for
 * an order only if that makes the graph at least 2 % faster (one order at a time), and
 * restores the states.  FP32 storage
 * without the Prandtl term or compensated moment sums only (SLLBM_EINVAL otherwise); other
 * conditions as sllbm_batch_create.  Synchronous. */
int sllbm_batch_create_persistent(sllbm_ctx *const *ctxs, int n, void *cuda_stream, int tune_steps,
                                  sllbm_batch **out);

/* Tile shape chosen per order in a persistent batch (0 default, 1 one size smaller, 2 one
 * cell; -1 for an order the batch does not contain); any output may be NULL. */
int sllbm_batch_shapes(const sllbm_batch *b, int *shape_p2, int *shape_p3, int *shape_p4);

/* Host-only planning helper used by sllbm_batch_create: assigns n jobs with the given
 * costs to `streams` streams, longest first, each to the least-loaded stream (ties: lowest
 * index); writes assign[n].  SLLBM_EINVAL for n < 1, streams < 1 or a negative cost. */
int sllbm_batch_plan(const double *cost, int n, int streams, int *assign);

void sllbm_batch_destroy(sllbm_batch *b);

/* ---- reverse mode ---------------------------------------------------------------------
 * The paper has no adjoint.  These calls are the transposes of the derivatives of the
 * forward operators above, from which gradients of a scalar of the final state through n
 * steps are assembled (checkpointing is the caller's).  They need SLLBM_F32 or SLLBM_F64
 * storage and the Prandtl term off (SLLBM_EINVAL otherwise).  Adjoint populations have the
 * order of a state buffer, buf[i][z][y][x][h], and the adjoint type (sllbm_set_adjoint_type;
 * by default the storage type); every pointer is a device
 * pointer; calls are asynchronous on the context's stream.  On the first call the context
 * allocates two state-sized scratch buffers (freed by sllbm_destroy; SLLBM_ENOMEM if that
 * fails). */

/* Type of the adjoint populations of the following reverse-mode calls: the storage type
 * (the default), or SLLBM_F64 for an SLLBM_F32 context, which keeps the adjoint in FP64
 * next to the FP32 forward states (the streamed states h stay FP32; the collision VJP and
 * the transposed streaming run in FP64).  SLLBM_EINVAL for other combinations. */
int sllbm_set_adjoint_type(sllbm_ctx *ctx, int storage);

/* dst = S src (transpose == 0) or dst = S^T src: the semi-Lagrangian streaming of all 90
 * populations alone (Eq. interpolation, pull), or its transpose, as three 1D passes, on
 * state-sized arrays of the storage type.  src and dst may be the same buffer.  For
 * SLLBM_F32 and SLLBM_F64 storage (SLLBM_EINVAL otherwise). */
int sllbm_stream_apply(sllbm_ctx *ctx, const void *src, void *dst, int transpose);

/* One step backward.  For the step F (pull streaming S, then the BGK collision C of
 * Eq. LBM at every node) taken from the state state_prev, and lam_next the adjoint of the
 * state it produced: lam_prev = (dF/dstate)^T lam_next = S^T (dC/dh)^T lam_next at
 * h = S state_prev, and *dmu += lam_next . dF/dmu_inf (*dmu: one FP64 device scalar,
 * accumulated).  lam_prev must not alias state_prev or lam_next. */
int sllbm_adjoint_step(sllbm_ctx *ctx, const void *state_prev, const void *lam_next, void *lam_prev,
                       double *dmu);

/* lam = dEk/dstate at state, with Ek as sllbm_diag defines and normalises it (the g
 * entries are zero). */
int sllbm_ek_adjoint(sllbm_ctx *ctx, const void *state, void *lam);

/* lam = dJ/dstate at state for J = wk Ek + ws eps_s + wc eps_c, the Sec. III.C diagnostics
 * as sllbm_diag defines and normalises them (the dissipation's gradient takes wk = 0,
 * ws = wc = 1).  FP64 arithmetic: the node fields rho, u, T; per quadrature point of every
 * cell the derivatives of its integrand with respect to the nine velocity-gradient entries
 * (cell-local Lagrange derivatives) and to T (Sutherland law); per node the sum over the
 * points whose integrand involves it, mapped to f and g through the moments.  Uses the
 * reverse-mode scratch buffers (allocated on first use); lam in the adjoint type. */
int sllbm_diag_adjoint(sllbm_ctx *ctx, const void *state, void *lam, double wk, double ws, double wc);

/* Transpose of sllbm_init_fields (equilibrium populations of the FP64 fields rho[nodes],
 * u[3][nodes], T[nodes]): grad_rho[n], grad_u[3][nodes], grad_T[n] = derivatives of
 * sum(lam * init(rho, u, T)) with respect to rho, u, T at node n, FP64 device arrays,
 * any of the three may be NULL. */
int sllbm_init_fields_adjoint(sllbm_ctx *ctx, const double *rho, const double *u, const double *T,
                              const void *lam, double *grad_rho, double *grad_u, double *grad_T);

/* ---- run control, fault injection, checkpoints ------------------------------------------
 * The paper describes none of these; they are the library's operational interface. */

/* Limit of each bounded device-side wait of the TMA-fed persistent kernel, in seconds
 * (default 2 s; 0 <= seconds <= 60, else SLLBM_EINVAL), for the following steps.  A wait
 * that runs past it makes the launch leave early (the state it wrote is then incomplete)
 * and sets the error that sllbm_status (or sllbm_step with nonfinite_check on) reports as
 * SLLBM_ETIMEOUT; the context stays usable.  The kernel's final wait for its own copies in
 * flight keeps the 2 s limit whatever is set here. */
int sllbm_set_wait_limit(sllbm_ctx *ctx, double seconds);

/* Sets (on != 0) or clears the context's abort request, a device word that the TMA-fed
 * persistent kernel reads at every tile boundary: a launch that sees it set stops issuing
 * work, lets its copies in flight land and returns, and sllbm_status then reports
 * SLLBM_EABORTED (the state is incomplete).  The word is written on a side stream, so a
 * request also reaches launches already queued or running on the context's stream; it
 * stays set until cleared.  The generic and batched kernels run a fixed amount of work
 * without waits and do not read it.  Synchronous with respect to the write only. */
int sllbm_request_abort(sllbm_ctx *ctx, int on);

/* Test hook, process-wide, host side: the next `after` device allocations made by the
 * library succeed and the one after them fails as if the device were out of memory (the
 * calling entry point returns SLLBM_ENOMEM or SLLBM_ECUDA as documented); the hook then
 * disarms itself.  after = -1 disarms it.  Makes no CUDA call. */
int sllbm_debug_fail_allocs(int after);

/* Compensated moment sums (on != 0) for the following steps of a context with FP32
 * arithmetic (SLLBM_F32 and the 16-bit deviation storages): rho, rho u and the energy sum
 * of Eq. (moments), and the temperature's 2 rho E - rho |u|^2, are accumulated with
 * error-free two-sum / two-product steps, so that each carries about one FP32 rounding
 * instead of one per term.  Both step kernels run it: the TMA-fed kernel (without the
 * Prandtl term) and the generic tile kernel's default tile (its alternative tiles sum
 * plainly, so the flag returns the context to the default tile); the automatic kernel
 * choice is made again.  FP64 storage ignores it.  SLLBM_EINVAL if the context's
 * parameters force the TMA-fed kernel and carry the Prandtl term. */
int sllbm_set_compensated(sllbm_ctx *ctx, int on);

/* Steps taken since the state was last set (initialisation, sllbm_set_populations,
 * sllbm_load_state) or loaded from a checkpoint (the checkpoint's count). */
int64_t sllbm_step_count(const sllbm_ctx *ctx);

/* Checkpoint file: a 128-byte header then the current state buffer as stored (pop_bytes,
 * storage type and order of a state buffer).  Header, host byte order: char magic[8] =
 * "SLLBMCK1"; uint32 version = 1; int32 storage, p, velset, cells[3], pr_correction;
 * double L[3], dt, mu_inf, rho0, T0; int64 steps; uint64 payload_bytes; 16 reserved
 * bytes.  sllbm_checkpoint_info reads one without a context or GPU. */
typedef struct {
    int storage, p, velset;
    int cells[3];
    int pr_correction;
    double L[3];
    double dt, mu_inf, rho0, T0;
    int64_t steps;
    uint64_t payload_bytes;
} sllbm_checkpoint_t;

/* Writes the context's current state and its description to `path` (synchronous).
 * Errors: SLLBM_EINVAL (NULL, slab context), SLLBM_ENOTREADY, SLLBM_ENOMEM (host copy),
 * SLLBM_ECUDA, SLLBM_EIO. */
int sllbm_save(sllbm_ctx *ctx, const char *path);

/* Loads a checkpoint into the context's current buffer (allocating the buffers if none
 * were set), restores mu_inf and the step count, and marks the context initialised
 * (synchronous).  The file must describe the same storage, order, cells, domain lengths,
 * time step and reference state rho0, T0 as the context, else SLLBM_EINVAL (as for a bad
 * magic, version or size, or a truncated payload); SLLBM_EIO if it cannot be opened. */
int sllbm_load(sllbm_ctx *ctx, const char *path);

/* Host-only, needs no context or GPU: reads and checks a checkpoint's header and that its
 * payload is complete.  SLLBM_EIO (cannot open), SLLBM_EINVAL (not a valid checkpoint). */
int sllbm_checkpoint_info(const char *path, sllbm_checkpoint_t *out);

/* ALU-peak microbenchmark (no counterpart in the paper; it supplies the measured ALU
 * roofline of the step): times one launch of independent dependent FMA chains over every
 * SM of the current device on the given stream (after one warm-up launch) and returns the
 * rate in flop/s (an FMA counts 2).  kind: 0 FP32 fma.rn.f32, 1 packed FP32x2
 * fma.rn.f32x2 (2 FMAs per instruction), 2 FP64 fma.rn.f64.  `iters` scales the work
 * (each thread executes 128 iters FMA instructions).  *seconds (may be NULL) receives the
 * timed launch's duration.  Synchronous; allocates nothing.  SLLBM_EINVAL for an unknown
 * kind or iters < 1, SLLBM_ECUDA. */
int sllbm_fma_peak(int kind, int iters, void *cuda_stream, double *flops_per_s, double *seconds);

/* Last CUDA error code seen by the context (cudaError_t as int, 0 if none). */
int sllbm_last_cuda_error(const sllbm_ctx *ctx);

/* Number of kernel launches the context has issued so far (all kernels). */
int64_t sllbm_launch_count(const sllbm_ctx *ctx);

/* Host-only, needs no context or GPU: the 45 abscissae xi[45*3] and weights w[45] of the
 * degree-9 cubature set (Sec. II.B, Fig. 2) in the canonical order described above. */
int sllbm_velset_d3q45(double *xi, double *w);

/* Host-only, needs no context or GPU: the precomputed streaming table of one direction
 * `dir` (0,1,2) for order p, cell size h and time step dt -- the uniform-mesh form of the
 * departure search and of the interpolation matrices Psi_i (Sec. II.A, Sec. IV.B).  For
 * velocity i and local node a in [0,p) the departure point of node c*p + a lies in cell
 * c + shift[i*p + a] at the reference coordinate whose Lagrange weights on the cell's
 * GLC points are weights[(i*p + a)*(p+1) + j], j = 0..p.  Arrays are caller-owned with
 * 45*p and 45*p*(p+1) entries.  SLLBM_EINVAL for p not in {2,3,4}, h <= 0 or dt < 0. */
int sllbm_stream_table(int p, double h, double dt, int dir, int *shift, double *weights);

/* Static description of an error code. */
const char *sllbm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* SLLBM_H */
