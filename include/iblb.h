/*
 * iblb.h -- C-ABI of the GB300 immersed boundary - lattice Boltzmann (IBLB)
 * wetting library (libiblb.so).
 *
 * The library advances droplet simulations of the IBLB wetting method of
 * Bellantoni et al., "On the hydrodynamic behaviour of the immersed boundary -
 * lattice Boltzmann method for wetting problems", Sec. 2:
 *   - lattice Boltzmann equation, BGK relaxation, exact streaming (Eq. 1-2),
 *     second-order equilibrium (Eq. 3), Guo forcing (Eq. 4), moments with the
 *     half-force correction (Eq. 5-6), on D2Q9 or D3Q19;
 *   - halfway bounce-back at two flat solid walls normal to the last axis
 *     (y in 2D, z in 3D), periodic along the other axes;
 *   - a closed Lagrangian interface (ring in 2D, triangle mesh in 3D) carrying
 *     surface tension plus the wetting potential Pi(d) (Eq. 9-11), spread to
 *     the lattice and coupled back by velocity interpolation (Eq. 7-8) with
 *     the Peskin 4-point delta, and advected by forward Euler.
 *
 * Conventions (all calls):
 *   - Lattice units: dx = dt = 1.  Cell (x, y, z) has index x + nx*(y + ny*z);
 *     nz = 1 in 2D.  The first and last layer along the wall axis are solid
 *     (when walls != 0); the lower wall plane is at coordinate 0.5 and the
 *     wall distance of a node is d = q_wall_axis - 0.5.
 *   - Host arrays are FP64 unless stated otherwise; the caller owns them.
 *     Populations are exchanged as f_i (not deviations), layout [Q][cells];
 *     velocities as [dim][cells]; node positions as [N][dim].
 *   - All device state is owned by the library.  Work is enqueued on the CUDA
 *     stream given at creation; calls that return host data synchronise it.
 *   - Every call returns an iblb_status; iblb_last_error() gives the text of
 *     the last failure on a handle.  Faults detected on the device (a node at
 *     or below the wall plane, a non-finite density) are latched in a device
 *     flag and reported by the next synchronising call; they never trap.
 *   - A handle is not thread-safe: use one handle per host thread / stream.
 */
#ifndef IBLB_H
#define IBLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IBLB_OK = 0,
    IBLB_EINVAL = 1,          /* bad argument or configuration */
    IBLB_ENOMEM = 2,          /* device allocation failed / budget exceeded */
    IBLB_ECUDA = 3,           /* a CUDA runtime call failed */
    IBLB_ENODE_IN_WALL = 4,   /* an interface node reached d <= 0 */
    IBLB_ENONFINITE = 5,      /* a density became NaN / Inf */
    IBLB_ETIMEOUT = 6,        /* a bounded device wait gave up */
    IBLB_EAGAIN = 7,          /* batch: no room for this request right now */
    IBLB_ECLASSIFY = 8        /* a lattice column crosses the interface more than
                                 16 times (inside / outside test) */
} iblb_status;

typedef enum { IBLB_D2Q9 = 9, IBLB_D3Q19 = 19 } iblb_lattice;

/* Population storage.  All forms hold deviations f_i - w_i from the rest
 * state; arithmetic is FP64 for IBLB_FP64 and FP32 otherwise.  IBLB_FP16_DEV
 * stores (f_i - w_i) * 2^fp16_scale_exp in binary16, rounded stochastically,
 * and is limited to lattices of fewer than 2^32 cells (IBLB_EINVAL above). */
typedef enum { IBLB_FP64 = 0, IBLB_FP32_DEV = 1, IBLB_FP16_DEV = 2 } iblb_storage;

typedef struct {
    int lattice;            /* IBLB_D2Q9 or IBLB_D3Q19 */
    int nx, ny, nz;         /* lattice extent (nz = 1 for D2Q9) */
    int walls;              /* 1: solid first/last layer along the wall axis;
                               0: periodic along every axis */
    int wetting;            /* 1: apply Pi(d) (Eq. 10) to the interface nodes */
    double tau;             /* BGK relaxation time, > 0.5 */
    double sigma;           /* surface tension */
    double xi;              /* regularisation length of Pi */
    double theta_eq_deg;    /* equilibrium contact angle; sets A by Eq. 11 */
    int pi_n, pi_m;         /* exponents of Pi, n > m > 1 */
    double body_force[3];   /* uniform force density on every fluid cell */
    int storage;            /* iblb_storage */
    int fp16_scale_exp;     /* binary16 scale exponent (0 selects 16) */
    double tau_out;         /* relaxation time outside the interface (Sec. 2:
                               viscosity ratio lambda = (tau - 1/2) /
                               (tau_out - 1/2)); 0 = tau.  Inside / outside is
                               found each step by ray tracing along the wall
                               axis through every lattice column. */
    double wall_u_lo[3];    /* velocity of the lower / upper wall (moving-wall */
    double wall_u_hi[3];    /* bounce-back, 2 w_i (c_i . u_w) / c_s^2 with
                               rho_w = 1; used for the drop in shear, Sec. 4).
                               Tangential components only (the wall-axis
                               component, and z in 2D, must be 0), |u| <= 0.3;
                               needs walls = 1.  All zero = resting walls. */
    int deterministic_spread; /* 1: spread the nodal forces (Eq. 8) as an
                               ordered gather (each cell sums the nodes whose
                               stencils cover it in a fixed order) instead of
                               a scatter with atomic additions, so that runs
                               are bitwise reproducible; 0: atomics (faster;
                               FP64 sums then vary in their last bits). */
    double shear_modulus;   /* elastic interface (the elasticity outlook of
                               Sec. 5; Sec. 2 forms the interface force from a
                               finite-element strain energy): shear modulus G_s
                               of Skalak's law W = G_s/4 [I1^2 + 2 I1 - 2 I2 +
                               C I2^2] per unit reference area on linear
                               triangles (2D rings: plane strain), whose
                               reference shape is the interface as set by
                               iblb_set_interface; added to the surface
                               tension.  0 = no elasticity (a clean drop). */
    double skalak_c;        /* Skalak's area-dilation parameter C (> -1/2; the
                               area modulus is G_s (1 + 2C)) */
} iblb_config;

typedef struct {
    double mass;          /* sum of rho over fluid cells (FP64) */
    double volume;        /* enclosed area (2D) / volume (3D) of the interface */
    double height;        /* max - min node coordinate along the wall axis */
    double theta_deg;     /* apparent contact angle of the circle/sphere fit */
    double r_cl;          /* contact-line half-width (2D) / radius (3D) */
    double film;          /* mean wall distance of the nodes under the drop */
    double d_min;         /* minimum node wall distance */
    double centre[3];     /* fitted circle / sphere centre */
    double radius;        /* fitted radius */
} iblb_obs;

typedef struct iblb_sim* iblb_handle;

/* Create a simulation at rest (rho = 1, u = 0, f_i = w_i) on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The configuration is
 * the paper's statement of the problem, Sec. 2: the lattice and velocity
 * stencil with the populations f_i of Eq. 1, the relaxation time tau of
 * Eq. 2 (and tau_out, tau(x, t) for the viscosity ratio lambda), the
 * surface tension sigma of Eq. 9, and n, m, xi and theta_eq of Eq. 10-11,
 * from which A is computed by Eq. 11.  Allocates the device state: two
 * population buffers, the moments, the force density and the band flags;
 * the library owns it.  cfg is read only.  *out receives the handle (NULL
 * on failure).  Returns IBLB_EINVAL for a bad config (reason in
 * iblb_last_error(NULL)), IBLB_ENOMEM if the device cannot hold it,
 * IBLB_ECUDA if a CUDA call fails. */
iblb_status iblb_create(const iblb_config* cfg, void* cuda_stream, iblb_handle* out);

/* Free the device state of a handle (synchronises its stream first).  A NULL
 * handle is ignored.  A library service; the paper has no counterpart. */
void        iblb_destroy(iblb_handle h);

/* Text of the last failure on a handle (NULL: of the last failed
 * iblb_create on this thread); owned by the library, valid until the next
 * call on the handle.  A library service; the paper has no counterpart. */
const char* iblb_last_error(iblb_handle h);
const char* iblb_status_string(iblb_status s);

/* Set the interface (Sec. 2: N Lagrangian nodes q_j on a triangular mesh
 * whose number of triangles stays fixed; the 2D analogue is a closed ring).
 * xyz [n_nodes][dim] host FP64.  2D: the nodes form a closed ring in
 * counter-clockwise order and `tri` must be NULL.  3D: tri [n_faces][3]
 * host int32, outward-oriented.  n_nodes = 0 removes the interface.  Both
 * arrays are copied (the caller keeps them).  IBLB_EINVAL on a bad array or
 * index, IBLB_ENODE_IN_WALL if a node lies at or below the wall plane with
 * wetting on; synchronises. */
iblb_status iblb_set_interface(iblb_handle h, const double* xyz, int n_nodes,
                               const int* tri, int n_faces);

/* Advance n_steps time steps (asynchronous on the stream).  Each step is
 * one update of Sec. 2 with every term at time t: nodal forces at q(t)
 * (surface tension and the wetting force phi_Pi,j of Eq. 9-11) -> spread
 * F(t) (Eq. 8) -> the lattice Boltzmann equation (Eq. 1) with BGK
 * relaxation (Eq. 2-3), the Guo source (Eq. 4) and the moments with the
 * half-force correction (Eq. 5-6), fused as one pull-streaming kernel ->
 * interpolate u(t) at q(t) (Eq. 7) -> the forward Euler update of the nodes.
 * The last step of a call also stores rho and u of every cell for
 * iblb_read_fields.  IBLB_EINVAL for n_steps < 0; device faults are reported
 * by the next synchronising call. */
iblb_status iblb_step(iblb_handle h, int n_steps);

/* Synchronise the stream and report any latched device fault (a library
 * service; the paper has no counterpart). */
iblb_status iblb_clear_faults(iblb_handle h);  /* clear the latched device
                                                  faults (synchronises); the
                                                  state that produced them is
                                                  left as it is */
iblb_status iblb_sync(iblb_handle h);

/* Read back the state after the last step: rho [cells] and u [dim][cells]
 * of the last moment evaluation (Eq. 5-6, with the force of that step; zero
 * on solid cells) and the node positions q_j after the last Euler update,
 * xyz [N][dim].  Caller-owned host buffers, FP64; any pointer may be NULL.
 * Synchronises; returns a latched device fault as its status. */
iblb_status iblb_read_fields(iblb_handle h, double* rho, double* u, double* xyz);

/* Replace / read the populations f_i of Eq. 1, host FP64 [Q][cells]
 * (caller-owned; converted from / to the storage form).  Synchronise. */
iblb_status iblb_set_populations(iblb_handle h, const double* f);
iblb_status iblb_get_populations(iblb_handle h, double* f);

/* FP64 observables of the current state: mass (the sum of rho, Eq. 5, over
 * the fluid cells), enclosed area / volume of the interface, the height h
 * as the distance between the highest and lowest nodes along the wall axis
 * (as the paper extracts h(t), Sec. 3), and the apparent contact angle,
 * contact-line position and film thickness epsilon (Sec. 2) from a
 * least-squares circle / sphere fit through the nodes above 3 xi, cut at the
 * lowest node (the paper measures only h; the estimator is this library's).
 * out is caller-owned.  Synchronises. */
iblb_status iblb_observables(iblb_handle h, iblb_obs* out);

/* ---- single-stage entry points (each runs one kernel of the step) ---- */

/* Set every population to the equilibrium (Sec. 2, Eq. 3) of the given
 * fields: rho [cells] (NULL: 1 everywhere), u [dim][cells]; host buffers
 * owned by the caller and only read, layout [component][z][y][x], FP64.
 * E.g. a fully developed shear flow (Sec. 4).  Solid layers are set too (they
 * are never read).  IBLB_EINVAL on a NULL handle or u; IBLB_ECUDA if a copy
 * or the kernel fails.  Synchronises. */
iblb_status iblb_set_equilibrium(iblb_handle h, const double* rho, const double* u);

/* Deformation of the current interface in the shear plane (x and the wall
 * axis), Sec. 4, Eq. 15: out[5] = {D = (r1 - r3)/(r1 + r3), r1, r3,
 * inclination of the r1 axis to x (degrees), enclosed area / volume}.  r1, r3
 * are the semi-axes of the ellipse (ellipsoid) with the same central second
 * moments as the enclosed region.  Needs a CCW ring of >= 3 nodes / an
 * outward mesh of >= 4 faces (IBLB_EINVAL otherwise).  Synchronises. */
iblb_status iblb_deformation(iblb_handle h, double* out);

/* Inside / outside classification of every cell by the current interface
 * (Sec. 2: the ray tracing behind tau(x, t)): mask [cells], caller-owned host
 * buffer, layout [z][y][x], 1 = inside.  Rays run along the wall axis; a
 * cell is inside when an odd number of crossings lies below its centre.
 * Works whether or not tau_out is set.  IBLB_ECLASSIFY when a column is
 * crossed more than 16 times; IBLB_EINVAL on NULL arguments.  Synchronises. */
iblb_status iblb_inside_mask(iblb_handle h, unsigned char* mask);

/* Nodal forces phi [N][dim], normals [N][dim] and 1-ring measures chi [N]
 * at the current interface (any pointer may be NULL). Synchronises. */
iblb_status iblb_nodal_forces(iblb_handle h, double* phi, double* normal, double* chi);

/* Spread the current nodal forces plus the body force: F [dim][cells].
 * Leaves the device force buffer cleared.  Synchronises. */
iblb_status iblb_force_field(iblb_handle h, double* F);

/* Interpolate a given velocity field u [dim][cells] to the current nodes:
 * qdot [N][dim].  Does not move the nodes.  Synchronises. */
iblb_status iblb_interpolate(iblb_handle h, const double* u, double* qdot);

/* ---- measurement ---- */

/* Kernel ids for iblb_step_profiled. */
enum {
    IBLB_K_FORCES = 0,
    IBLB_K_SPREAD = 1,
    IBLB_K_STREAM_COLLIDE = 2,
    IBLB_K_INTERP_ADVECT = 3,
    IBLB_K_BAND_CELLS = 4,  /* overlapped step: the second pass over the band cells */
    IBLB_K_COUNT = 5
};

/* Run n_steps outside any CUDA graph with a CUDA event pair around every
 * kernel launch; kernel_ms[IBLB_K_COUNT] receives the summed device time of
 * each kernel (ms).  When iblb_step would overlap (iblb_tuning.step_overlap),
 * the profiled steps run the same kernels one after the other on one
 * stream: IBLB_K_STREAM_COLLIDE is then the bulk pass (every cell, body
 * force only) and IBLB_K_BAND_CELLS the band pass; otherwise the band
 * bucket is 0.  Synchronises. */
iblb_status iblb_step_profiled(iblb_handle h, int n_steps, double* kernel_ms);

/* Launch shape of the stream-collide kernel (results do not depend on it).
 *   variant 0: the plain kernel, one cell per thread, block_x threads per
 *              block along x (64, 128 or 256), evict-first stores of the new
 *              populations when streaming_stores != 0;
 *   variant 2: two x-adjacent cells per thread with 8 / 4-byte population
 *              loads and stores and packed FP32x2 arithmetic (FP32 and
 *              binary16 storage, even nx), block_x threads per block;
 *   variant 3: two y-adjacent cells per thread (rows y, y + 1 of a layer)
 *              with scalar loads and stores and packed FP32x2 arithmetic
 *              (D3Q19, FP32 and binary16 storage), block_x threads per block;
 *   variant 1: the pipelined kernel: persistent CTAs in which a producer warp
 *              stages the source rows in shared memory with bulk asynchronous
 *              copies and consumer_warps warps collide from there;
 *              ctas_per_sm = 2 with 8 consumer warps, or 1 with 16 or 24.
 *              Usable when nx is a multiple of 32 up to 1024 (tiles of
 *              rows_per_tile whole rows) or a multiple of 256 (row
 *              segments); otherwise the plain kernel runs. */
typedef struct {
    int variant;
    int block_x;
    int streaming_stores;
    int rows_per_tile;
    int ctas_per_sm;
    int consumer_warps;
    long long wait_limit_cycles;  /* pipelined kernel: clock cycles a wait on
                                     its pipeline may take before the kernel
                                     gives up, latches IBLB_ETIMEOUT and stops
                                     (the populations of that step are then
                                     incomplete); 0 = about 2 s.  Copies in
                                     flight are always waited for (bounded by
                                     about 2 s) before the kernel exits. */
    int ib_grouped;               /* 3D interfaces: 0 (default) spreads and
                                     interpolates with one thread per node
                                     and one global addition (read) per
                                     stencil point; 1 by spatial groups of
                                     nodes (the nodes of one 8 x 8 x 8 tile
                                     of the lattice; a group sums its
                                     stencils in, or reads them from, a box
                                     of the lattice in shared memory).
                                     Results differ only by the order of the
                                     additions.  Not changed by
                                     iblb_autotune. */
    int step_overlap;             /* iblb_step with an interface: 0 (default)
                                     overlaps on 3D lattices of at least 2^20
                                     cells, 1 always, 2 never.  Overlapped, a
                                     step runs the stream-collide of every
                                     cell with the body force only on one
                                     stream while the nodal forces are
                                     computed and spread on another, then
                                     updates the cells of the flagged band
                                     segments again, from the same sources,
                                     with their force density (the same
                                     arithmetic as one pass).  Not used with
                                     a viscosity ratio, nor by
                                     iblb_step_profiled.  Not changed by
                                     iblb_autotune. */
} iblb_tuning;

/* Set / read the launch shape.  iblb_set_tuning synchronises. */
iblb_status iblb_set_tuning(iblb_handle h, const iblb_tuning* t);
iblb_status iblb_get_tuning(iblb_handle h, iblb_tuning* t);

/* Autotuner: time every applicable launch shape (plain kernel with 64, 128
 * and 256-thread blocks; x-pair and row-pair kernels likewise; pipelined
 * kernel with 1, 2 or 4 rows per tile and 8, 16 or 24 consumer warps) over
 * `trials` launches each, after 4 * trials untimed warm-up launches, in two
 * passes (the faster pass of each shape counts), and keep the fastest.  The
 * trial launches read the current populations and write only the second
 * (scratch) population buffer, so the simulation state is left unchanged.
 * `chosen` (may be NULL) receives the kept shape.  Synchronises. */
iblb_status iblb_autotune(iblb_handle h, int trials, iblb_tuning* chosen);

/* The stream-collide variant in use (0 plain, 1 pipelined, 2 x pairs,
 * 3 row pairs). */
int iblb_stream_collide_variant(iblb_handle h);

/* Algorithmic HBM bytes of one stream-collide launch: populations read once
 * and written once per fluid cell. */
double iblb_stream_bytes_per_step(iblb_handle h);
long long iblb_fluid_cells(iblb_handle h);

/* ---- batched engine and serving admission ----
 *
 * These calls are services of this library: the paper runs one simulation
 * at a time, and each slot computes exactly the step of iblb_step (Sec. 2,
 * Eq. 1-11 and forward Euler).  A batch advances many independent droplet simulations ("slots") of one
 * lattice type and one storage form with shared launches: every phase of a
 * time step is one launch over all active slots (the stream-collide phase a
 * persistent kernel walking a (slot, tile) work list).  Slot state lives in
 * one device arena of hbm_budget_bytes allocated at creation; a request is
 * admitted when its footprint fits (first fit), else IBLB_EAGAIN.  Slots
 * must have walls, no body force, and the batch's lattice and storage; the
 * walls may move tangentially (wall_u_lo / wall_u_hi, Ladd's moving-wall
 * bounce-back as in iblb_step), and a slot may have a viscosity ratio
 * (tau_out: its inside / outside classification is rebuilt every step, as
 * in iblb_step).  While some active slot has moving walls or a viscosity
 * ratio the stream-collide launch is the instantiation that carries those
 * terms.
 * Each slot's tile shape (32-cell row segments per stream-collide work item) is
 * chosen at admission by timing the candidates on that slot (cached per
 * lattice width).  Calls on one batch are not thread-safe. */
typedef struct iblb_batch_s* iblb_batch;

typedef struct {
    int slots_used, slots_active, slots_done;
    size_t arena_bytes, free_bytes;
    long long kernel_launches;
} iblb_batch_info;

/* Device bytes one slot of this configuration and interface takes. */
size_t iblb_batch_footprint(const iblb_config* cfg, int n_nodes, int n_faces);

/* Create a batch for slots of one lattice (IBLB_D2Q9 / IBLB_D3Q19) and one
 * storage form, with a device arena of hbm_budget_bytes (rounded down to
 * 256 B) and up to max_slots slots, working on cuda_stream.  The library
 * owns the arena.  IBLB_EINVAL for bad arguments, IBLB_ENOMEM if the arena
 * cannot be allocated. */
iblb_status iblb_batch_create(int lattice, int storage, size_t hbm_budget_bytes, int max_slots,
                              void* cuda_stream, iblb_batch* out);
void        iblb_batch_destroy(iblb_batch b);
const char* iblb_batch_last_error(iblb_batch b);

/* Admit a simulation at rest with the given configuration (as iblb_create:
 * the problem statement of Sec. 2) and interface (as iblb_set_interface)
 * for n_steps steps; *slot_out receives its slot.  cfg, xyz and tri are
 * copied.  IBLB_EAGAIN: no free slot or no room in the arena now (retry
 * after releases); IBLB_EINVAL: a configuration the batch cannot take (see
 * above) or a bad interface.  Synchronises. */
iblb_status iblb_batch_admit(iblb_batch b, const iblb_config* cfg, const double* xyz, int n_nodes,
                             const int* tri, int n_faces, long long n_steps, int* slot_out);

/* Advance every active slot by up to max_steps steps of Sec. 2 (as
 * iblb_step; asynchronous).  A slot stops at its own last step and becomes
 * done; *n_completed (may be NULL) counts the slots that completed during
 * this call. */
iblb_status iblb_batch_run(iblb_batch b, int max_steps, int* n_completed);

/* As iblb_batch_run, for measurement: the steps run one launch at a time
 * (no CUDA graph) with a CUDA event pair around each phase.
 * kernel_ms[IBLB_K_COUNT] receives the summed device time of each phase (ms;
 * indices as for iblb_step_profiled); *stream_collide_bytes (may be NULL)
 * the summed algorithmic bytes of the stream-collide launches (populations
 * read once and written once per fluid cell of every active slot).  Results
 * are those of iblb_batch_run.  IBLB_EINVAL on a NULL batch or kernel_ms.
 * Synchronises after every step. */
iblb_status iblb_batch_run_profiled(iblb_batch b, int max_steps, int* n_completed,
                                    double* kernel_ms, double* stream_collide_bytes);
iblb_status iblb_batch_sync(iblb_batch b);

/* Slots that are done and not yet released (up to cap of them in the
 * caller's done_slots; *n_done is their total number).  Host bookkeeping
 * only: it does not wait for the device (iblb_batch_sync does). */
iblb_status iblb_batch_poll(iblb_batch b, int* done_slots, int cap, int* n_done);

/* Steps done by a slot, and its latched device faults as a status. */
iblb_status iblb_batch_slot_status(iblb_batch b, int slot, long long* steps_done);

/* FP64 observables / fields of a slot (as iblb_observables / iblb_read_fields;
 * the fields are those of the slot's last step).  Synchronise. */
iblb_status iblb_batch_observables(iblb_batch b, int slot, iblb_obs* out);
iblb_status iblb_batch_read_fields(iblb_batch b, int slot, double* rho, double* u, double* xyz);

/* Free a slot and its arena memory. */
iblb_status iblb_batch_release(iblb_batch b, int slot);
iblb_status iblb_batch_stats(iblb_batch b, iblb_batch_info* info);

/* Steps until the next active slot completes (-1 if none is active); host
 * bookkeeping, no synchronisation.  Lets a serving loop advance a batch
 * exactly to its next completion. */
long long iblb_batch_steps_to_next_completion(iblb_batch b);

/* The 32-cell row segments per stream-collide work item chosen by the tile
 * autotuner for a slot. */
int iblb_batch_slot_tile(iblb_batch b, int slot);

/* ---- mass reduction without device allocation ----
 *
 * The paper has no counterpart: this is a service of the library.
 *
 * iblb_mass_static computes the same FP64 mass as iblb_observables (sum of
 * rho over the fluid cells) for a population array the caller owns, without
 * allocating device memory.  It is meant for callers that cannot call
 * cudaMalloc when they need the number: a process that reserves all of its
 * GPU memory up front (for example a serving loop running from a fixed
 * pool), code that runs while another component owns the device allocator,
 * or an embedding that forbids device allocations after initialisation.
 *
 *   f_dev     device pointer to the populations in this library's storage
 *             form: deviations f_i - w_i, layout [Q][nx*ny*nz] (x fastest),
 *             double (IBLB_FP64), float (IBLB_FP32_DEV) or binary16 scaled
 *             by 2^fp16_scale_exp (IBLB_FP16_DEV; 0 selects 16)
 *   mass_dev  device pointer to one double that receives the mass
 *   walls     1: the first and last layer along the wall axis are solid and
 *             excluded, as in iblb_config
 *   cuda_stream  stream the two kernels are enqueued on (asynchronous)
 *
 * Scratch: per-block partial sums live in one file-scope device array of
 * IBLB_STATIC_PARTIALS doubles (512 KiB), which every GPU that loads the
 * library holds until the process exits.  One partial covers 16384 cells, so
 * lattices above IBLB_STATIC_PARTIALS * 16384 cells are rejected with
 * IBLB_EINVAL before anything is launched.  Each call overwrites the
 * partials it uses (the array keeps the last call's values; nothing needs
 * to start at zero), and all calls share the array: calls that overlap on
 * the GPU (on different streams, or from different threads) race and give
 * wrong results.  The first call on a device does the set-up: with that
 * device current it resolves the array's device address (which also makes
 * the CUDA runtime load this library's device code on that device, if it
 * has not yet done so) and keeps the address for later calls.  So make that
 * first call during start-up: before any stream capture, and before the
 * caller reserves the device memory it will run from.  The kept address
 * belongs to the device's primary context of this process: after a
 * cudaDeviceReset the array and its address are gone, and this entry point
 * must not be called again in that process.  Later calls make no cudaMalloc,
 * cudaFree or other allocating call.  Returns IBLB_EINVAL for bad
 * arguments, IBLB_ECUDA if a CUDA call fails. */
#define IBLB_STATIC_PARTIALS 65536
iblb_status iblb_mass_static(const void* f_dev, int lattice, int storage, int nx, int ny, int nz,
                             int walls, int fp16_scale_exp, double* mass_dev, void* cuda_stream);

/* Number of kernels this library has launched since load (counting every
 * launch, including those inside CUDA graphs). */
long long iblb_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif
