/*
 * cdugks.h -- C ABI of the GB300 (sm_103a) implementation of one time step of
 * the Coupled Discrete Unified Gas Kinetic Scheme (CDUGKS) of Zamora,
 * Slaughter & Abel, arXiv:2208.09132.
 *
 * The state of a problem instance is the pair of reduced distributions g
 * (velocity distribution, eq. g) and b (total-energy distribution, eq. b) on
 * every (spatial cell, discrete velocity) point, plus the conserved variables
 * W = (rho, rho u, rho E) of every cell, which the scheme tracks explicitly
 * (Sec. 2: "The rule is made explicit by updating the conserved variables W").
 * One call of cdugks_step advances all of it by the update of Sec. 2.1
 * ("The Algorithm"): the quarter-step shift of eq. phibarplus, van Leer
 * limited upwind reconstruction (eq. VanLeer) along the characteristics
 * (eq. relation), the face moments of eqs. rhobar-rhoEbar, the face
 * equilibrium (eqs. geq, beq) and inversion of eq. phibar, the microflux of
 * eq. flux, the conserved-variable update of eqs. rhoupdate-rhoEupdate and the
 * distribution update of eq. phiupdate.  External acceleration is zero.
 *
 * Conventions
 *   - Every call returns int: CDUGKS_OK (0) or a negative CDUGKS_ERR_*.
 *     No exception crosses the ABI.  cdugks_strerror() names a code;
 *     cdugks_last_error() gives the message of the last failure on this thread.
 *   - Device memory is owned by the caller: cdugks_workspace_bytes() says how
 *     much, cdugks_bind() hands it over (256-byte aligned base).  The library
 *     allocates no device memory of its own and never frees caller memory.
 *   - All device work is enqueued on the stream given to cdugks_bind().
 *     cdugks_step() is asynchronous; cdugks_moments(), cdugks_conserved(),
 *     cdugks_distributions(), cdugks_get_state() and cdugks_sync_status()
 *     synchronise that stream.
 *   - Host pointers are borrowed for the duration of the call only.
 *   - Cell order is x fastest, then y, then z.  Velocity order is the tensor
 *     product of the 1D grids with the first component fastest.
 *   - A handle is not thread safe; distinct handles are independent.
 */
#ifndef CDUGKS_H
#define CDUGKS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CDUGKS_API __attribute__((visibility("default")))
#else
#define CDUGKS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define CDUGKS_OK 0
#define CDUGKS_ERR_INVALID (-1)     /* bad argument or problem description */
#define CDUGKS_ERR_OOM (-2)         /* bound workspace too small */
#define CDUGKS_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define CDUGKS_ERR_NONFINITE (-4)   /* a conserved variable became NaN/Inf */
#define CDUGKS_ERR_TIMEOUT (-5)     /* a bounded device wait gave up: the launch that
                                       reported it stopped early, so its results are
                                       incomplete; a wait that runs out for a real
                                       reason (not the test hook) may leave tensor
                                       copies in flight, so treat every later result
                                       in that CUDA context as untrusted and destroy
                                       the handle rather than re-initialise it */
#define CDUGKS_ERR_UNBOUND (-6)     /* no workspace bound / state not initialised */
#define CDUGKS_ERR_NEGATIVE (-7)    /* density or temperature became <= 0 */

/* -------------------------------------------------------- problem setup */
#define CDUGKS_BC_PERIODIC 0        /* wrap-around */
#define CDUGKS_BC_SPECULAR 1        /* mirror wall: normal velocity reversed */
#define CDUGKS_BC_DIRICHLET 2       /* ghosts hold the equilibrium of the initial edge state */

#define CDUGKS_RULE_TRAPEZOID 0     /* composite trapezoid weights */
#define CDUGKS_RULE_BOOLE 1         /* composite Boole (4th-order Newton-Cotes), n = 4m+1 */

#define CDUGKS_FP64 0               /* g, b stored and computed in double */
#define CDUGKS_FP32 1               /* g, b stored in float and the per-point arithmetic
                                       in float; W, rho, u, T (T from E - u^2/2) in
                                       double.  The velocity-space sums of a velocity
                                       group are summed per chunk of 4 velocities in
                                       float and the chunk sums folded into float
                                       Kahan pairs (compensated summation); the
                                       groups' partial sums are added in double, in
                                       a fixed order. */

/* Spatial grid: dim = D in {1,2,3}; n[a] cells on [lo[a], hi[a]] along axis
 * a < D (entries a >= D ignored); bc[a][0] / bc[a][1] the low / high side.
 * Periodic must be set on both sides of an axis or on neither; specular
 * needs n[a] >= 2 and a velocity range symmetric about 0 on that axis. */
typedef struct {
    int dim;
    int n[3];
    double lo[3], hi[3];
    int bc[3][2];
} cdugks_grid;

/* Velocity grid (Sec. 2, discrete velocity method): n[a] >= 2 nodes on
 * [lo[a], hi[a]] including both ends, tensor product over a < dim. */
typedef struct {
    int n[3];
    double lo[3], hi[3];
    int rule;
} cdugks_vgrid;

/* Physics (Sec. 2): K internal degrees of freedom (gamma = (K+5)/(K+3));
 * gas constant R (0.5 in the paper); viscosity mu = mu_ref (T/T_ref)^omega
 * (eq. visc); Prandtl number Pr = tau_g / tau_b; dt > 0 fixes the time step,
 * dt <= 0 takes the CFL rule of Sec. 4, dt = cfl dx_min / (2 |xi|_max). */
typedef struct {
    double K, R;
    double mu_ref, T_ref, omega;
    double Pr;
    double cfl, dt;
    int precision;                  /* CDUGKS_FP64 or CDUGKS_FP32 */
} cdugks_phys;

typedef struct cdugks cdugks_t;     /* opaque handle; host metadata only */

/* Validate the description and create a handle (no device work).
 * Errors: INVALID.  *out is NULL on failure. */
CDUGKS_API int cdugks_create(const cdugks_grid *grid, const cdugks_vgrid *vgrid, const cdugks_phys *phys,
                  cdugks_t **out);

/* Device bytes the caller must provide to cdugks_bind (phase-space state in
 * two buffers, conserved variables, face-moment partial sums, velocity tables,
 * status word). */
CDUGKS_API int cdugks_workspace_bytes(const cdugks_t *h, size_t *bytes);

/* Hand over caller-owned device memory (>= cdugks_workspace_bytes, 256-byte
 * aligned) and the cudaStream_t (as void*; NULL = legacy default stream) all
 * later device work is ordered on.  Uploads the velocity tables.
 * Errors: INVALID (null/misaligned), OOM (too small), CUDA. */
CDUGKS_API int cdugks_bind(cdugks_t *h, void *device_ptr, size_t bytes, void *cuda_stream);

/* Maxwell-Boltzmann initialisation (Sec. 3.4: all problems start from
 * eqs. geq/beq for the given moments).  rho_u_T: host array [Nc][2+D] of
 * cell-centre density, velocity components and temperature.  W^0 is
 * (rho, rho u, rho (u^2/2 + c_v T)) with c_v = (3+K)R/2.  Synchronous.
 * Errors: INVALID (non-positive rho/T), UNBOUND, CUDA. */
CDUGKS_API int cdugks_init(cdugks_t *h, const double *rho_u_T);

/* Enqueue nsteps time steps of Sec. 2.1 on the bound stream (asynchronous).
 * With a captured graph (cdugks_capture) whole multiples of its step count
 * are replayed from it, the rest launched one by one; results are the same.
 * Errors: UNBOUND, INVALID (nsteps < 0), CUDA (launch failure). */
CDUGKS_API int cdugks_step(cdugks_t *h, int nsteps);

/* Capture steps_per_graph time steps in CUDA graphs (one per parity of the
 * ping-pong state buffer the replay starts from) so that later cdugks_step
 * calls replay them: one launch per steps_per_graph steps instead of 4 + D,
 * which matters for small problems whose steps last microseconds.  0 drops
 * the graphs.  Needs a non-default stream; changing the tile shape or the
 * velocity groups, or binding again, drops the graphs.  Capturing enqueues
 * no work.  Errors: UNBOUND, INVALID (steps_per_graph outside [0, 4096] or
 * the default stream), CUDA. */
CDUGKS_API int cdugks_capture(cdugks_t *h, int steps_per_graph);

/* Advance nsteps steps exactly as cdugks_step does, timing each phase with
 * CUDA events on the bound stream: ms_out[0..3] = mean milliseconds per step
 * of sweep A (face moments), the face constants, sweep B (fluxes and
 * distribution update) and the W update.  Synchronises once at the end.
 * Errors: UNBOUND, INVALID (nsteps outside [1, 1e5] or null ms_out), CUDA. */
CDUGKS_API int cdugks_profile_step(cdugks_t *h, int nsteps, double *ms_out);

/* Synchronise the stream and report the device status word: OK, or
 * NONFINITE / NEGATIVE if any step since the last check produced a
 * non-finite conserved variable or rho <= 0 or T <= 0, or TIMEOUT if a
 * kernel's bounded wait for its tensor copies gave up (the kernel then stops
 * and that step's result is incomplete).  Clears the word. */
CDUGKS_API int cdugks_sync_status(cdugks_t *h);

/* Macroscopic fields from the tracked W: host out[Nc][2+D] = rho, u[D], T.
 * Synchronous (device-to-host copy of Nc*(2+D) doubles). */
CDUGKS_API int cdugks_moments(cdugks_t *h, double *out);

/* Pressure tensor and heat flux of every cell from its distributions at the
 * current time level (a diagnostic; the step does not use them).  With rho,
 * rho u, rho E the moments of g and b (Sec. 2):
 *     P_ab = sum_i w_i (xi - u)_a (xi - u)_b g_i,
 *     q_a  = sum_i w_i xi_a b_i - u_a rho E - sum_b P_ab u_b
 * (the total-energy flux less convection and pressure work).  Host
 * out[Nc][D*D + D]: P row-major, then q; sums in FP64 on the device.
 * Synchronous.  Errors: UNBOUND, INVALID (null out), CUDA. */
CDUGKS_API int cdugks_stress_heat_flux(cdugks_t *h, double *out);

/* The tracked conserved variables W: host out[Nc][2+D]. Synchronous. */
CDUGKS_API int cdugks_conserved(cdugks_t *h, double *out);

/* The distributions g, b at the current time level, host [Nc][Nv] each, as
 * double (converted from the storage precision).  Uses the idle state buffer
 * on the device as scratch.  Synchronous. */
CDUGKS_API int cdugks_distributions(cdugks_t *h, double *g, double *b);

/* The distributions of n selected cells (indices in [0, Nc)), host
 * [n][Nv] each as double, at the current time level.  Uses the idle state
 * buffer on the device as scratch; copies only the selected cells back.
 * Synchronous. */
CDUGKS_API int cdugks_cell_distributions(cdugks_t *h, const long long *cells, int n, double *g, double *b);

/* Checkpoint: opaque host image of the device state (distributions in their
 * storage form, W, step count).  cdugks_set_state restores it bitwise, so a
 * restarted run reproduces an uninterrupted one exactly. */
CDUGKS_API int cdugks_state_bytes(const cdugks_t *h, size_t *bytes);
CDUGKS_API int cdugks_get_state(cdugks_t *h, void *host, size_t bytes);
CDUGKS_API int cdugks_set_state(cdugks_t *h, const void *host, size_t bytes);

/* Introspection. */
typedef struct {
    int dim;
    long long ncells;               /* Nc */
    int nvel;                       /* Nv (unpadded) */
    int nvel_padded;                /* Nv rounded up to the 32-velocity tile */
    double dt;                      /* time step in use */
    long long steps;                /* steps taken since cdugks_init */
    int precision;
    int velocity_groups;            /* velocity-space split of the sweeps */
    double state_bytes;             /* bytes of one copy of (g, b) on the device */
    int tile_id;                    /* tile shape of the sweeps (cdugks_set_tile) */
    int tile[3];                    /* its cells per axis */
} cdugks_info_t;
CDUGKS_API int cdugks_info(const cdugks_t *h, cdugks_info_t *info);

/* Tuning: split velocity space into groups of tiles for the two sweeps
 * (0 = automatic).  Results are independent of the split up to the order of
 * the final sums over groups (a fixed order, so runs are reproducible). */
CDUGKS_API int cdugks_set_velocity_groups(cdugks_t *h, int groups);

/* Tuning: the spatial tile shape of the sweeps, one of cdugks_tile_count()
 * instantiated shapes per (precision, dim) (0 = default).  Results do not
 * depend on the shape. */
CDUGKS_API int cdugks_tile_count(int precision, int dim);
CDUGKS_API int cdugks_set_tile(cdugks_t *h, int tile_id);
/* out[0..2]: cells per axis of a tile shape; out[3] its sweep mode.  Bits
 * 0-1 say where the sweeps take phibar+ and the van Leer slopes from:
 *   0  they form both on their halo boxes;
 *   1  phibar+ of every point is formed once per step in its own pass (one
 *      more state-size buffer in the workspace);
 *   2  phibar+ and the slopes of every point are formed once per step in a
 *      stencil pass (one more state-size buffer and D more for the slopes;
 *      periodic and specular boundaries only).
 * Bit 2 (value 4, face store): sweep A keeps the reconstructed phibar of
 * every face and velocity (about D more state-size buffers) and sweep B only
 * forms the fluxes from them instead of reconstructing again.
 * Bit 3 (value 8): the shape implements the face-gradient reconstruction
 * (cdugks_set_reconstruction); the others the upwind-cell one.
 * Bit 4 (value 16): the shape implements the Shakhov collision model
 * (cdugks_set_collision); the others the two-time model.
 * Bit 5 (value 32): the shape implements the external acceleration
 * (cdugks_set_acceleration); the others none.
 * Every mode but 0 must be selected before cdugks_bind; modes with bits 0-1
 * nonzero are not batched (modes 0 and 4 are).  A face-store shape of the
 * two-time model steps a handle created with Pr = 1 (no b-source, Sec. 2)
 * with sweeps compiled without the b-source terms; the mode reported here
 * does not change. */
CDUGKS_API int cdugks_tile_shape(int precision, int dim, int tile_id, int *out);

/* The reconstruction of phibar at a face (Sec. 2.1).
 *   CDUGKS_RECON_UPWIND_CELL (default): phibar+ of the upwind cell carried
 *     along the characteristic with that cell's limited slope vector,
 *     phibar(x_f, t + h) = phibar+_up + (x_f - h xi - x_up) . sigma_up.
 *   CDUGKS_RECON_FACE_GRADIENT: the paper's variant, in which the slopes are
 *     themselves reconstructed at the face from their own limited gradients:
 *     sigma_f = sigma_up + (x_f - x_up) . grad sigma_up and
 *     phibar(x_f, t + h) = phibar+_up + (x_f - x_up) . sigma_up - h xi . sigma_f.
 *     Three halo cells; D = 1 or 2; 3 cells next to a specular wall; not
 *     in cdugks_step_noalloc.  The two agree to second order.
 * Select before cdugks_bind; it picks the default shape of that
 * reconstruction, and cdugks_set_tile then accepts only shapes that
 * implement it (tile_shape out[3] bit 3).
 * Errors: INVALID (unknown value, bound handle, no such shape, short wall). */
#define CDUGKS_RECON_UPWIND_CELL 0
#define CDUGKS_RECON_FACE_GRADIENT 1
CDUGKS_API int cdugks_set_reconstruction(cdugks_t *h, int recon);

/* Collision model (call before cdugks_bind; default TEDDF).
 *   CDUGKS_COLLISION_TEDDF    the paper's model (Sec. 2): tau_g = mu/p,
 *                             tau_b = tau_g/Pr and the b-source
 *                             Z/tau_bg (g - g_eq).
 *   CDUGKS_COLLISION_SHAKHOV  the Shakhov S-model, the other route to Pr != 1
 *                             that Sec. 1 names: one relaxation time
 *                             tau = mu/p for g and b, no b-source, and
 *                             equilibria with the heat-flux correction
 *                               g_S = g_M (1 + cq (c^2/RT - D - 2)),
 *                               b_S = b_M + cq g_M ((|xi|^2/2)(c^2/RT - D - 2)
 *                                     + (3 - D + K)(c^2 - D RT)/2),
 *                             cq = (1 - Pr) c.q / ((K + 5) p RT), c = xi - u:
 *                             Shakhov's model for all 3 + K degrees of
 *                             freedom, integrated over those the velocity
 *                             grid does not resolve.  The heat flux q of a
 *                             face comes from the reconstructed values
 *                             (divided by 1 + h Pr/(2 tau)), that of a cell
 *                             at t_{n+1} from the explicit part of the update
 *                             (divided by 1 + dt Pr/(2 tau)); both relative
 *                             to the place's conserved variables.  The
 *                             initial Maxwellian state has q = 0.
 * Selecting a model selects the first tile shape that implements it (and
 * the selected reconstruction); the Shakhov shapes are face-store shapes.
 * Not available in batches or cdugks_step_noalloc.  Errors: INVALID (unknown
 * model, already bound, no shape for this dimension and reconstruction, or a
 * Dirichlet boundary with a stored-slope Shakhov shape). */
#define CDUGKS_COLLISION_TEDDF 0
#define CDUGKS_COLLISION_SHAKHOV 1
CDUGKS_API int cdugks_set_collision(cdugks_t *h, int model);

/* Uniform external acceleration a (host double[3], components beyond dim 0;
 * NULL or all zero turns it off; call before cdugks_bind).  It switches on
 * the force terms of eqs. gsource/bsource: S_g = -a.grad_xi g and
 * a.xi g - a.grad_xi b in S_b, the velocity gradients by central differences
 * on the velocity grid (the distribution taken as 0 beyond its ends).  The
 * sources enter phibar+ with h/2 (eq. phibarplus) and phi* with dt at t_n
 * (the rectangle rule of Sec. 2); W gains dt (0, rho^n a, (rho u)^n . a); the
 * face W gains (h/2) rho a and then (h/2) (rho u) . a (eqs. rhoubar,
 * rhoEbar); the inverse of eq. phibar at a face takes the force gradients of
 * phibar there and a.xi g with the face g.  A specular wall face leaves out
 * the normal component of the force (the wall takes it), so walls pass no
 * mass.  Ghost cells take phibar+ by their rule (copy, mirror image,
 * Dirichlet equilibrium).  Selects the first tile shape that implements it
 * (prepared face-store shapes, mode bit 5); the upwind-cell reconstruction
 * and the two-time collision model only; not batched, not in
 * cdugks_step_noalloc.  Errors: INVALID (non-finite, nonzero beyond dim,
 * already bound, no shape). */
CDUGKS_API int cdugks_set_acceleration(cdugks_t *h, const double *a);

/* Testing hook for the failure path of the bounded device waits (on = 1;
 * 0 restores normal operation).  While on, sweep A issues none of its tensor
 * copies and its wait gives up after 2^10 tries instead of 2^22: a step on a
 * tile shape that stages with tensor copies (the fused shapes of 1D/2D
 * problems large enough for interior tiles) stops its sweep and the next
 * cdugks_sync_status reports CDUGKS_ERR_TIMEOUT.  Nothing faults or hangs;
 * that step's results are incomplete (cdugks_init or cdugks_set_state
 * restores a valid state) and the handle stays usable.  Drops captured
 * graphs. */
CDUGKS_API int cdugks_test_wait_timeout(cdugks_t *h, int on);

/* ---------------------------------------------------------------- batches
 * Many independent instances stepped together: every kernel of a time step
 * is one launch over a device work list of all members' (tile, velocity
 * group) items, so uneven instances fill the GPU together.  Members must be
 * bound and initialised, of one precision and dim; each keeps its own
 * workspace.  The batch needs a small caller-owned workspace for its tables
 * and runs on its own stream; do not touch the members on other streams
 * between cdugks_batch_bind and cdugks_batch_sync.  Members may use different
 * tile shapes (up to 8) and physics: every fused shape (two-time or Shakhov
 * collision model, either reconstruction) and the acceleration shapes batch;
 * the prepared and stored shapes without acceleration do not.  Results of a
 * member are the same as stepping it alone with the same tile shape and
 * groups. */
typedef struct cdugks_batch cdugks_batch_t;
CDUGKS_API int cdugks_batch_create(cdugks_t *const *members, int n, cdugks_batch_t **out);
CDUGKS_API int cdugks_batch_workspace_bytes(const cdugks_batch_t *b, size_t *bytes);
CDUGKS_API int cdugks_batch_bind(cdugks_batch_t *b, void *device_ptr, size_t bytes, void *cuda_stream);
/* Capture steps_per_graph batched steps in a CUDA graph (0 drops it); later
 * cdugks_batch_step calls replay it for whole multiples.  Needs a non-default
 * stream.  The buffer parity of each member lives on the device, so replays
 * are valid for any number of steps. */
CDUGKS_API int cdugks_batch_capture(cdugks_batch_t *b, int steps_per_graph);
/* Enqueue nsteps steps of every member (asynchronous). */
CDUGKS_API int cdugks_batch_step(cdugks_batch_t *b, int nsteps);
/* Synchronise the batch stream and report the first member status error. */
CDUGKS_API int cdugks_batch_sync(cdugks_batch_t *b);
/* Change the membership between steps (continuous batching): admit a bound,
 * initialised handle of the batch's precision and dim, or retire a member
 * (which keeps its state and may be read or stepped alone afterwards).  Both
 * first finish the work in flight on the batch stream, then drop the binding
 * and any captured graph: query cdugks_batch_workspace_bytes and call
 * cdugks_batch_bind again before the next step.  A batch keeps at least one
 * member; an admitted handle's own stream is synchronised too.
 * Errors: INVALID (null, duplicate, not a member, last member, unbatchable
 * shape, precision or dim mismatch), UNBOUND (member not ready), CUDA. */
CDUGKS_API int cdugks_batch_admit(cdugks_batch_t *b, cdugks_t *member);
CDUGKS_API int cdugks_batch_retire(cdugks_batch_t *b, cdugks_t *member);
CDUGKS_API void cdugks_batch_destroy(cdugks_batch_t *b);
/* Persistent batched step (on = 1; 0 returns to one launch per kernel).  Every
 * phase of every member -- sweep A, face constants, sweep B, W update, the
 * steps of Sec. 2.1 -- for all the steps of one cdugks_batch_step call (or of
 * one captured graph) runs in ONE launch: CTAs take work items from a device
 * list in dependency order and wait, per member, for the items an item needs
 * (bounded waits; a wait that gives up stops the launch and the next
 * cdugks_batch_sync reports CDUGKS_ERR_TIMEOUT).  All members must share one
 * tile shape that has this step (fused face-store shapes: 1D 64/128/256 and
 * 2D 32 x 8 in FP32, 1D 64 in FP64).  max_members / max_items reserve room in
 * the batch workspace (at least the current sizes; items are the batch's work
 * items per step): while later cdugks_batch_admit / cdugks_batch_retire calls
 * of members of that shape fit, they rewrite the device tables in place and
 * keep the binding and any captured graph; otherwise they unbind as usual and
 * the plan reserves room for the new sizes (bind again).
 * Results equal the per-kernel launches bit for bit.  Unbinds the batch (query
 * the workspace size and bind again).  Errors: INVALID (several shapes, a shape
 * without it, more than 1024 members). */
CDUGKS_API int cdugks_batch_set_persistent(cdugks_batch_t *b, int on, int max_members, long long max_items);
/* 1 if the batch is bound (after admit / retire: whether to bind again). */
CDUGKS_API int cdugks_batch_bound(const cdugks_batch_t *b);
/* Persistent batches only: one launch in which member i (in the order of
 * creation and admission, retired members removed) advances steps[i] >= 0
 * steps (n = the number of members); the items of a member past its count are
 * skipped.  Asynchronous on the batch stream (the counts are copied before the
 * call returns).  Errors: UNBOUND, INVALID (not persistent, wrong n, negative
 * count), CUDA. */
CDUGKS_API int cdugks_batch_step_members(cdugks_batch_t *b, const int *steps, int n);
/* Testing hook for the persistent step's bounded waits (on = 1; 0 restores):
 * the first face item waits for one item more than exists and every wait gives
 * up after 2^12 polls, so a step stops early and cdugks_batch_sync reports
 * CDUGKS_ERR_TIMEOUT; nothing faults or hangs.  Drops a captured graph. */
CDUGKS_API int cdugks_batch_test_wait_timeout(cdugks_batch_t *b, int on);

CDUGKS_API void cdugks_destroy(cdugks_t *h);
CDUGKS_API const char *cdugks_strerror(int code);
CDUGKS_API const char *cdugks_last_error(void);

/* Allocation-free time step (the paper has no counterpart: this is a
 * convenience of this library).  For callers that cannot allocate device
 * memory themselves -- code inside a framework whose memory pool owns the GPU
 * and only lends out existing buffers, or a latency-critical loop where a
 * device allocation could synchronise the device or fail -- this advances the
 * state by exactly one step without cdugks_bind and without any allocation.
 *   h        a handle from cdugks_create (binding it is not required)
 *   phi_in   device state at t_n in the layout of the distribution block of
 *            cdugks_get_state: [Nvp/4][Nc][g|b][4] values of the handle's
 *            precision (32-byte aligned)
 *   phi_out  device buffer of the same size for t_{n+1} (not phi_in)
 *   W        device conserved variables [2+D][Nc] doubles, updated in place
 *   stream   cudaStream_t as void* (NULL = legacy default stream)
 * Asynchronous.  No device status word is reported: after synchronising the
 * stream the caller must check W itself (every entry finite, rho > 0 and
 * rho E > |rho u|^2 / (2 rho) in every cell) before trusting the state.  Every other
 * piece of device scratch lives in one fixed 32 MiB array in this library
 * (held by every GPU that loads it until the process exits): problems whose
 * cell/face tables and face-moment sums exceed it are rejected with
 * CDUGKS_ERR_INVALID and a message giving the size needed.  Periodic and
 * specular boundaries only.  All calls share that array, and it keeps what
 * the last call left in it: calls whose work may overlap on one GPU (for
 * instance calls on two streams) race on it, so serialise them.  The first
 * call on each device
 * looks up the array's device address; make that first call before any
 * stream capture.  Errors: INVALID, CUDA. */
CDUGKS_API int cdugks_step_noalloc(cdugks_t *h, const void *phi_in, void *phi_out, double *W, void *cuda_stream);

/* Hard-sphere convention for a Knudsen number (an input convention, not part
 * of the scheme): mu_ref = (5/16) Kn L rho_ref sqrt(2 pi R T_ref). */
CDUGKS_API double cdugks_mu_from_kn(double kn, double rho_ref, double T_ref, double R, double length);

#ifdef __cplusplus
}
#endif
#endif
