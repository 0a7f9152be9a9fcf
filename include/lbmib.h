/*
 * lbmib.h - C ABI of the GB300 LBM-IB library.
 *
 * The library advances one time step of the combined lattice Boltzmann / immersed
 * boundary method of Coclite et al., "Kinematic and Dynamic Forcing Strategies for
 * Predicting the Transport of Inertial Capsules via a combined Lattice Boltzmann -
 * Immersed Boundary Method" (arXiv:1903.03356):
 *   - D2Q9 BGK lattice update with a body-force term (Section 2.1-2.2, Eq. 1-7),
 *   - moving-least-squares interpolation and spreading between the lattice and the
 *     membrane vertices (Section 2.2, Eq. 8-9; Section 2.3 step 3; Section 2.4 step iii),
 *   - membrane stretch, bending and area forces (Section 2.2.1, Eq. 10-14),
 *   - hydrodynamic tractions from normal probes (Section 2.2.2, Eq. 15-16),
 *   - the Kinematic scheme (Section 2.4, steps i-viii, Eq. 25) or the Dynamic scheme
 *     (Section 2.3.2, steps 1-8, Eq. 21-24).
 *
 * Conventions shared by every call
 *   Units dx = dt = 1, rho_0 = 1, c_s^2 = 1/3, nu = (tau - 1/2)/3. Lattice node (i, j)
 *   sits at (x, y) = (i, j); fields are row-major ny x nx (index j * nx + i). x is
 *   periodic. With walls, half-way bounce-back walls sit at y = -1/2 and y = ny - 1/2
 *   and move along x with the given velocities. Capsule rings are counter-clockwise;
 *   coordinate arrays interleave x and y (2n doubles).
 *
 *   Memory: the library never allocates device memory. The caller allocates one
 *   device arena of lbmib_arena_bytes() bytes (at least 256-byte aligned) and keeps it
 *   alive until lbmib_destroy(). Host pointers passed to any call belong to the caller
 *   and are only read or written during the call. The context itself is host memory
 *   owned by the library.
 *
 *   Ordering: all device work is issued on the CUDA stream given to lbmib_create (NULL
 *   means the legacy default stream). lbmib_step only enqueues work; read calls
 *   synchronise that stream.
 *
 *   Errors: every call returns an lbmib_status; lbmib_last_error() gives a message.
 *   Device-side conditions (a support leaving the channel, an unstable velocity) are
 *   recorded in a sticky status word and reported by the next synchronising call.
 */
#ifndef LBMIB_H
#define LBMIB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbmib_ctx lbmib_ctx;

typedef enum {
    LBMIB_OK = 0,
    LBMIB_ERR_ARG = 1,      /* invalid argument (sizes, ids, NULL where not allowed)  */
    LBMIB_ERR_OOM = 2,      /* arena too small or capacity exceeded                   */
    LBMIB_ERR_CUDA = 3,     /* a CUDA call failed; the message names it               */
    LBMIB_ERR_UNSTABLE = 4, /* |u| > 0.3 or a NaN in the lattice (sticky)             */
    LBMIB_ERR_SUPPORT = 5,  /* an MLS support or probe left the channel (sticky)      */
    LBMIB_ERR_TIMEOUT = 6,  /* a bounded device wait gave up (sticky)                 */
    LBMIB_ERR_STATE = 7     /* call not valid in the current state                    */
} lbmib_status;

/* Storage of the lattice populations. Populations are stored shifted by their rest
 * weights (f_i - w_i). FP64 computes in double; FP32 and FP16 compute the collision in
 * float (FP16 storage keeps the shifted value times a power-of-two scale). Membrane
 * vertices, their velocities and forces are double in every mode. */
typedef enum { LBMIB_FP64 = 0, LBMIB_FP32 = 1, LBMIB_FP16 = 2 } lbmib_storage;

/* Coupling scheme of a step: Kinematic IB (Section 2.4) or Dynamic IB (Section 2.3). */
typedef enum { LBMIB_KINEMATIC = 0, LBMIB_DYNAMIC = 1 } lbmib_scheme;

typedef struct {
    int nx, ny;             /* lattice size, each >= 3                                */
    int walls;              /* 0: periodic in y; 1: moving bounce-back walls in y      */
    double tau;             /* BGK relaxation time (Eq. 1), > 0.5                      */
    double u_bottom;        /* x-velocity of the wall at y = -1/2                     */
    double u_top;           /* x-velocity of the wall at y = ny - 1/2                 */
    double gx, gy;          /* uniform body-force density (added to f_ib, Eq. 5)      */
    lbmib_storage storage;
    int max_capsules;       /* capacity for capsules                                  */
    int max_nodes;          /* capacity for membrane vertices over all capsules       */
} lbmib_config;

/* Device arena size (bytes) for a configuration; 0 if the configuration is invalid. */
size_t lbmib_arena_bytes(const lbmib_config* cfg);

/* Create a context over the caller's device arena. cuda_stream is a cudaStream_t (or
 * NULL). The fluid starts at rest (rho = 1, u = 0). *out receives the context. */
lbmib_status lbmib_create(const lbmib_config* cfg, void* d_arena, size_t arena_bytes,
                          void* cuda_stream, lbmib_ctx** out);

/* Release the context's host memory and CUDA graphs (the arena stays the caller's). */
void lbmib_destroy(lbmib_ctx* ctx);

/* Message of the last failing call on this context (never NULL). */
const char* lbmib_last_error(const lbmib_ctx* ctx);

/* Set the fluid to the Eq. 2 equilibrium of the given host fields (ny*nx doubles each;
 * NULL means rho = 1 or u = 0). Clears the immersed-boundary force field. */
lbmib_status lbmib_init_fields(lbmib_ctx* ctx, const double* rho, const double* ux,
                               const double* uy);

/* Add a capsule: xy (2n doubles, host) is its stress-free shape and initial position
 * (Section 2.2.1: reference lengths, angles and area are taken from it). k_s, k_b, k_a
 * are the stretch (Eq. 10), bending (Eq. 12) and area (Eq. 14) constants; node_mass is
 * the per-vertex mass m_v (Eq. 21). n must be in [3, 1024]. *id_out gets its id. */
lbmib_status lbmib_add_capsule(lbmib_ctx* ctx, const double* xy, int n, double k_s,
                               double k_b, double k_a, double node_mass, int* id_out);

/* Add a rigid particle (Section 2.3.1): xy (2n doubles, host, counter-clockwise) is its
 * ring of markers, fixed in the body frame about the ring's area centroid c; mass and
 * inertia (moment of inertia about c) are > 0; it starts at rest. It moves only with
 * the Dynamic scheme: its markers' desired velocity is the rigid-body velocity
 * u + omega x (X - c) (steps 1-3); after the fluid update the load of the outer probes,
 * F = sum_l (tau+ . n+ - p+ n+) l_l (Eq. 17) and M = sum_l r_l x that (Eq. 18, r_l from c
 * to the element centroid), plus the Eq. 27 repulsion on its markers when on, drives
 * u and omega by Eq. 19-20, and c and the angle by the same second-order backward
 * formula. lbmib_step with the Kinematic scheme then fails with LBMIB_ERR_STATE, and
 * lbmib_adjoint does not cover it. Shares the capsule capacity and ids with
 * lbmib_add_capsule; its vertex data read through lbmib_read_capsule (velocities: the
 * rigid-body motion; internal forces zero; external forces half of each element's
 * outer traction at each end). *id_out gets its id. */
lbmib_status lbmib_add_rigid(lbmib_ctx* ctx, const double* xy, int n, double mass, double inertia,
                             int* id_out);

/* Body state of rigid particle id (9 doubles, host): c_x, c_y, rotation angle, u_x, u_y,
 * omega, and the last load F_x, F_y, M. Synchronises. LBMIB_ERR_ARG if id is not a rigid
 * particle. */
lbmib_status lbmib_read_rigid(lbmib_ctx* ctx, int id, double* out);

/* Move capsule id to positions xy (2n doubles, host) without changing its stress-free
 * shape; its time history restarts (the next step is a start-up step). */
lbmib_status lbmib_set_capsule_positions(lbmib_ctx* ctx, int id, const double* xy);

/* Advance nsteps time steps with the given scheme (enqueued, asynchronous).
 * Kinematic (Section 2.4, steps i-viii): spread the internal forces at X^n, update the
 * lattice, interpolate u (Eq. 7 with half of the spread force) at X^n, advance by Eq. 25.
 * Dynamic (Section 2.3.2, steps 1-8): interpolate U at X^n from the populations before
 * any IB force (rho u = sum f e + g/2), spread c_l (u_v - U) with c_l the vertex's share of
 * the arc length, update the lattice, take the probe tractions (Eq. 15-16) on the updated
 * populations (again before any IB force) and the internal forces at X^n, and advance by
 * Eq. 23 with U as the tentative velocity and Eq. 24.
 * A capsule's first step after being added starts its history: Kinematic uses forward
 * Euler, Dynamic sets u_v = U and X^{-1} = X^0 - u_v. */
lbmib_status lbmib_step(lbmib_ctx* ctx, long long nsteps, lbmib_scheme scheme);

/* Wait for the stream and report any sticky device status. */
lbmib_status lbmib_sync(lbmib_ctx* ctx);

/* Open channel (Section 2.1: known-velocity boundaries of Zou and He; Section 3.2:
 * parabolic inlet and constant outlet pressure). From the next step on, x is no longer
 * periodic: column x = 0 is an inlet whose nodes get the velocity (u_in[y], 0) and column
 * x = nx - 1 an outlet whose nodes get density rho_out (pressure rho_out / 3) and zero
 * y-velocity. The three populations entering through each column are rebuilt from the
 * others (mass and normal momentum fix the density or the normal velocity; the
 * non-equilibrium part bounces back along the normal; the diagonals share the tangential
 * one; with a body force g the known momentum is rho u - g/2). The whole column is
 * closed, wall rows included. u_in: ny host doubles, |u| < 0.3, copied during the call;
 * rho_out in (0.5, 2). u_in = NULL makes x periodic again. MLS supports of vertices and
 * probes must then stay within columns 1 .. nx - 2 (LBMIB_ERR_SUPPORT otherwise); the
 * repulsion takes x distances without the periodic image. Not covered by lbmib_adjoint
 * (LBMIB_ERR_STATE); not part of the saved state (set it again after lbmib_load_state).
 * Synchronises the context stream. */
lbmib_status lbmib_set_inflow(lbmib_ctx* ctx, const double* u_in, double rho_out);

/* Capsule-capsule repulsion (Section 3.4, Eq. 27): from the next step on, every vertex
 * of a capsule feels coeff * sqrt(dx / d^5) along its inward normal (the negated,
 * normalised sum of the outward normals of its two elements) from every vertex of every
 * other capsule at distance d < cutoff (minimum image along periodic axes); dx = 1.
 * coeff = 0 selects the printed 1e-4 / (8 sqrt 2); cutoff = 0 turns the repulsion off
 * (the default). The force joins the spread force (Kinematic) or the total vertex force
 * of Eq. 23 (Dynamic). Neighbours are found through a grid of cells of at least 1.5 x
 * the largest reference capsule extent + cutoff; a capsule that outgrows its cell, or
 * more than 16 capsules hashed to one grid bucket, raise LBMIB_ERR_STATE at the next
 * synchronising call. Errors: LBMIB_ERR_ARG (cutoff outside [0, 16], coeff < 0). */
lbmib_status lbmib_set_repulsion(lbmib_ctx* ctx, double cutoff, double coeff);

/* Fluid fields at the current time into host arrays (ny*nx doubles each, any may be
 * NULL): rho (Eq. 6) and u (Eq. 7) with half of the body force plus the last spread
 * immersed-boundary force. Synchronises. */
lbmib_status lbmib_read_fields(lbmib_ctx* ctx, double* rho, double* ux, double* uy);

/* Pre-collision populations f_i at the current time (unshifted), host array of
 * 9*ny*nx doubles ordered [i][j][x]. Synchronises. */
lbmib_status lbmib_read_populations(lbmib_ctx* ctx, double* f);

/* Last spread immersed-boundary force field f_ib (without the uniform body force),
 * host arrays of ny*nx doubles (either may be NULL). Synchronises. */
lbmib_status lbmib_read_force_field(lbmib_ctx* ctx, double* fx, double* fy);

/* Capsule state into host arrays of 2n doubles (any may be NULL): positions X^n,
 * node velocities (Kinematic: last interpolated velocity; Dynamic: u_v of Eq. 24),
 * the last internal forces F^int (Eq. 22) and external forces F^ext (Eq. 15-16). */
lbmib_status lbmib_read_capsule(lbmib_ctx* ctx, int id, double* xy, double* vel,
                                double* fint, double* fext);

/* Observables of capsule id (Section 3.1-3.2): out = {area, perimeter, Taylor D,
 * centroid x, centroid y, swelling ratio Sw, inclination of the major axis,
 * relative perimeter change delta_p}. D comes from the eigenvalues of the area
 * second-moment tensor. Synchronises. */
lbmib_status lbmib_observables(lbmib_ctx* ctx, int id, double out[8]);

/* Observables of every capsule: out (8 * capsule count doubles, host) in the order of
 * lbmib_observables, capsule by capsule. Synchronises. */
lbmib_status lbmib_observables_all(lbmib_ctx* ctx, double* out);

/* MLS interpolation (Eq. 8) of the current fluid at n host points xy (2n doubles):
 * out (8n doubles, host) = {ux, uy, rho, p, dux/dx, dux/dy, duy/dx, duy/dy} per point.
 * n <= max_nodes. Synchronises. */
lbmib_status lbmib_interpolate(lbmib_ctx* ctx, const double* xy, int n, double* out);

/* Same as lbmib_interpolate, for callers that cannot allocate device memory at the time
 * of the call: callbacks on real-time loops that must not trigger the implicit
 * synchronisation of an allocation, hosts whose device memory belongs to another
 * framework's allocator (which would see a cudaMalloc as memory it does not account
 * for), or processes held to a fixed device-memory budget. The paper has no
 * counterpart; this is a library convenience. The call allocates nothing: the device staging of the points and results
 * lives in a static array of the library, sized for 16384 points (1.25 MiB held on every
 * device that loads the library until the process exits). n > 16384 is rejected with
 * LBMIB_ERR_ARG. The first call on a device resolves the array's device address (with
 * the context's device made current for that moment); make that first call before any
 * stream capture. Every call on a device shares the one array and its contents persist
 * between calls, so calls whose device work overlaps (several streams, or several
 * host threads) race: serialise them. Synchronises. */
lbmib_status lbmib_interpolate_noalloc(lbmib_ctx* ctx, const double* xy, int n, double* out);

/* Checkpoint: lbmib_state_bytes() gives the size of a snapshot of the populations,
 * the force fields and all capsule state; lbmib_save_state() writes it into a host
 * buffer of that size and lbmib_load_state() restores it into a context created with
 * the same configuration. Both synchronise. */
size_t lbmib_state_bytes(const lbmib_ctx* ctx);
lbmib_status lbmib_save_state(lbmib_ctx* ctx, void* host_buf, size_t bytes);
lbmib_status lbmib_load_state(lbmib_ctx* ctx, const void* host_buf, size_t bytes);

/* Device addresses of the context's fields, for zero-copy views (the one call that gives
 * out device pointers; they point into the caller's arena). field:
 *   LBMIB_FIELD_POPULATIONS  the latest post-collision populations in the storage type,
 *                            stored shifted (f_i - w_i; FP16 times the storage scale),
 *                            laid out [9][ny][pitch] with pitch >= nx elements per row;
 *                            the pre-collision populations of the next step are their
 *                            pull f_i(x) = f*_i(x - e_i) (reflected at walls).
 *   LBMIB_FIELD_FORCE        the immersed-boundary force density of the last spread,
 *                            double [2][ny][nx] (x plane, then y); pitch = nx.
 * The two population and force buffers alternate from step to step: an address is valid
 * until the next lbmib_step. Synchronises the context stream. */
enum { LBMIB_FIELD_POPULATIONS = 0, LBMIB_FIELD_FORCE = 1 };
lbmib_status lbmib_field_ptr(lbmib_ctx* ctx, int field, void** ptr, int* pitch);

/* Options (lbmib_set_option):
 *   LBMIB_OPT_GRAPHS        1 (default): replay steps from captured CUDA graphs;
 *                           0: launch kernels directly.
 *   LBMIB_OPT_TIMING        1: record CUDA events around every lattice-update launch
 *                           (forces direct launches); read with lbmib_kernel_time.
 *   LBMIB_OPT_GRAPH_STEPS   steps per captured graph (default 64; each graph opens with
 *                           its own force and spread and closes with its own update).
 *   LBMIB_OPT_FP16_SCALE    log2 of the FP16 storage scale (default 10).
 *   LBMIB_OPT_LATTICE_VARIANT launch shape of the lattice-update kernel: bits 0-11 the
 *                           block size (128 or 256), bit 18 a 64-register cap (eight
 *                           128-thread or four 256-thread blocks resident per SM), bit 19 (FP16
 *                           storage) the kernel that moves 8 nodes per thread as packed
 *                           16-byte vectors. Default: 128 threads, with the cap for
 *                           FP32/FP16 storage and bit 19 for FP16. Results do not
 *                           depend on it; only speed does.
 *   LBMIB_OPT_OVERLAP       1: the immersed-boundary kernels run on a second stream of
 *                           the library, overlapping the lattice update of the same
 *                           step (force and spread) and of the next step (node
 *                           update); 0: every kernel on the context stream; -1
 *                           (default): on while there are fewer than two capsules per
 *                           multiprocessor. Results do not depend on it.
 *   LBMIB_OPT_ARCS          CTAs per capsule in the immersed-boundary kernels, 1..8:
 *                           each takes an even share of the ring's vertices, and the
 *                           kernels that need the enclosed area run a capsule's CTAs
 *                           as one thread-block cluster. 0 (default): one CTA per
 *                           capsule while the capsules number at least the
 *                           multiprocessors, otherwise min(8, multiprocessors /
 *                           capsules, vertices / 16). Results do not depend on it
 *                           beyond the order of the area sum.
 *   LBMIB_OPT_FUSE_IB       1 (default): within one lbmib_step call, the node update
 *                           of a step and the force and spread of the next run as one
 *                           kernel when every capsule has one CTA and the context
 *                           holds no rigid particles: the Dynamic scheme (both read
 *                           the same lattice state; Section 2.3.2 steps 7-8 and 1-3),
 *                           and the Kinematic one without repulsion (the advance,
 *                           then the membrane forces at the new positions and their
 *                           spread; Section 2.4); 0: separate kernels. The state
 *                           between calls and the results do not depend on it.
 *   LBMIB_OPT_IB_FP64       1: with FP32 or FP16 storage the immersed-boundary kernels
 *                           gather in storage precision and do the MLS solve, the
 *                           membrane and traction forces and the node update in FP64
 *                           (slower: GB300's FP64 rate); 0 (default): they compute in
 *                           FP32 around FP64 positions, stored velocities and enclosed areas.
 *                           No effect with FP64 storage.                             */
enum {
    LBMIB_OPT_GRAPHS = 1,
    LBMIB_OPT_TIMING = 2,
    LBMIB_OPT_GRAPH_STEPS = 3,
    LBMIB_OPT_FP16_SCALE = 4,
    LBMIB_OPT_LATTICE_VARIANT = 5,
    LBMIB_OPT_OVERLAP = 6,
    LBMIB_OPT_ARCS = 7,
    LBMIB_OPT_FUSE_IB = 8,
    LBMIB_OPT_IB_FP64 = 9
};
lbmib_status lbmib_set_option(lbmib_ctx* ctx, int option, long long value);

/* Timing of the lattice-update kernel (collide-stream, Eq. 4) since the last reset,
 * measured with CUDA events on the context stream while LBMIB_OPT_TIMING is on:
 * total milliseconds and launch count. reset != 0 clears the record. Synchronises. */
lbmib_status lbmib_kernel_time(lbmib_ctx* ctx, double* total_ms, long long* launches,
                               int reset);

/* Timing of the forced-node patch and of the immersed-boundary node update (with the
 * next step's force and spread when fused) since the last reset, from CUDA events
 * recorded while LBMIB_OPT_TIMING is on, in the steps whose kernels all ran on the
 * context stream (no overlap, closed channel): total milliseconds of each and the
 * number of steps timed; `listed` is the length of the last spread's touched-node list
 * (a node covered by several capsules' tiles counts once per tile). Any pointer may be
 * null. reset != 0 clears the record. Synchronises. */
lbmib_status lbmib_ib_kernel_time(lbmib_ctx* ctx, double* patch_ms, double* ib_ms, long long* steps,
                                  long long* listed, int reset);

/* Number of kernels this context has launched (graph replays count their kernels). */
long long lbmib_launch_count(const lbmib_ctx* ctx);

/* Bytes the lattice-update kernel must move per lattice update: 18 populations of the
 * storage type (9 read, 9 written). */
double lbmib_bytes_per_update(const lbmib_ctx* ctx);

/* ---------------------------------------------------------------------------------
 * Adjoint: gradients of a capsule objective J(X^T) after nsteps steps of either scheme
 * (Kinematic, Section 2.4; Dynamic, Section 2.3.2) from the current state, with respect
 * to k_s and k_b of every capsule and the uniform body force (gx, gy). The initial state
 * (populations, last spread force, capsule positions and history) is held fixed.
 * Computed by a reverse sweep over the exact discrete step (collision, streaming, MLS
 * interpolation and spreading, membrane forces, and for the Dynamic scheme the
 * c_l-weighted forcing, the probe tractions of Eq. 15-16 and the Eq. 23-24 update); MLS
 * supports are differentiated as they stand (a vertex crossing a half-integer line
 * switches support, which the derivative ignores).
 * --------------------------------------------------------------------------------- */
enum {
    LBMIB_OBJ_TAYLOR_D = 0,     /* Taylor deformation D of the capsule (Section 3.1)   */
    LBMIB_OBJ_CENTROID_Y = 1,   /* centroid y (lateral position in a channel)          */
    LBMIB_OBJ_CENTROID_X = 2    /* centroid x                                          */
};

/* Device workspace (bytes) for lbmib_adjoint over nsteps steps with a checkpoint every
 * ckpt_every steps: ceil(nsteps / ckpt_every) + 1 state checkpoints (none when
 * ckpt_every >= nsteps), a tape of min(ckpt_every, nsteps) + 1 population buffers and
 * the adjoint fields. 0 on invalid arguments. */
size_t lbmib_adjoint_workspace_bytes(const lbmib_ctx* ctx, long long nsteps, int ckpt_every);

/* Run nsteps steps of `scheme` from the current state (the context ends nsteps steps
 * later, as after lbmib_step) and return J at the end (*J, may be NULL) and its gradient
 * grad[2 * ncapsules + 2] = {dJ/dk_s of each capsule, dJ/dk_b of each capsule,
 * dJ/dgx, dJ/dgy}. objective: LBMIB_OBJ_*; capsule: whose ring J measures. d_work:
 * device workspace of lbmib_adjoint_workspace_bytes (256-byte aligned). Segments of
 * ckpt_every steps are recomputed from their checkpoints during the reverse sweep.
 * Synchronises. Errors: LBMIB_ERR_ARG (arguments, unknown scheme), LBMIB_ERR_OOM
 * (workspace too small), sticky device conditions of the run. */
lbmib_status lbmib_adjoint(lbmib_ctx* ctx, long long nsteps, lbmib_scheme scheme,
                           int ckpt_every, int objective, int capsule, void* d_work,
                           size_t work_bytes, double* J, double* grad);

/* ---------------------------------------------------------------------------------
 * Batched persistent launch: many independent cases, each its own small lattice with at
 * most one capsule, advanced together by the Kinematic scheme (Section 2.4, steps
 * i-viii, Eq. 25) in one kernel launch per lbmib_batch_step call. Every case follows
 * exactly the single-context step of LBMIB_KINEMATIC; cases never interact.
 *
 * A case's capsule must stay inside a shared-memory tile sized from its initial ring
 * (largest bounding-box side + 8 nodes, squared, times 1.5); a capsule that outgrows it,
 * or whose tile would wrap onto itself on a periodic lattice, stops moving and raises
 * LBMIB_ERR_SUPPORT at the next synchronising call.
 * --------------------------------------------------------------------------------- */
typedef struct lbmib_batch lbmib_batch;

typedef struct {
    int nx, ny;             /* lattice size, each >= 3, nx * ny < 2^31               */
    int walls;              /* as lbmib_config                                        */
    double tau;             /* > 0.5                                                  */
    double u_bottom, u_top; /* wall x-velocities (ignored without walls)              */
    double gx, gy;          /* uniform body-force density                             */
    const double* rho;      /* initial fields, host, nx*ny row-major; NULL = rest     */
    const double* ux;       /*   (rho 1, u 0); read during lbmib_batch_create only    */
    const double* uy;
    const double* xy;       /* capsule ring, 2n interleaved, counter-clockwise; it is */
    int n;                  /*   also the stress-free shape. n = 0: no capsule,       */
    double k_s, k_b, k_a;   /*   else 3 <= n <= 1024. Constants of Eq. 10, 12, 14.    */
    double node_mass;       /* > 0 when n > 0 (unused by the Kinematic scheme)        */
} lbmib_case;

/* Device arena size (bytes) for a batch; 0 if a case or the storage is invalid. */
size_t lbmib_batch_arena_bytes(const lbmib_case* cases, int ncases, lbmib_storage storage);

/* Create a batch over caller-owned device memory (as lbmib_create): copies the case
 * table and initial state (populations at equilibrium with the given fields, Section
 * 2.1). autotune_steps > 0 times each candidate launch shape (256, 512 or 1024 threads
 * per CTA, from one CTA per SM up to as many as fit) for that many steps, keeps the
 * fastest and restarts every case from its initial state; 0 uses 512 threads with as
 * many CTAs as fit. Synchronises.
 * Errors: LBMIB_ERR_ARG (a case invalid, a ring clockwise, arena misaligned),
 * LBMIB_ERR_OOM (arena too small), LBMIB_ERR_CUDA. */
lbmib_status lbmib_batch_create(const lbmib_case* cases, int ncases, lbmib_storage storage,
                                void* d_arena, size_t arena_bytes, void* cuda_stream,
                                int autotune_steps, lbmib_batch** out);
void lbmib_batch_destroy(lbmib_batch* batch);
const char* lbmib_batch_last_error(const lbmib_batch* batch);

/* Advance every case by nsteps (0 <= nsteps < 2^30) with one persistent launch
 * (replayed from a CUDA graph captured for this nsteps). Enqueues only. */
lbmib_status lbmib_batch_step(lbmib_batch* batch, long long nsteps);

/* Wait for the batch stream; report sticky device conditions (LBMIB_ERR_UNSTABLE,
 * LBMIB_ERR_SUPPORT). */
lbmib_status lbmib_batch_sync(lbmib_batch* batch);

/* Populations of case c (unshifted f_i, host double [9][ny][nx]). Synchronises. */
lbmib_status lbmib_batch_read_populations(lbmib_batch* batch, int c, double* f);

/* Vertex positions and last interpolated velocities of case c (2n each, NULL to skip;
 * nothing is written when the case has no capsule). Synchronises. */
lbmib_status lbmib_batch_read_capsule(lbmib_batch* batch, int c, double* xy, double* vel);

/* Observables of every case's capsule (host double [ncases][8], layout of
 * lbmib_observables_all; rows of cases without a capsule are zero). Synchronises. */
lbmib_status lbmib_batch_observables(lbmib_batch* batch, double* out);

/* Launch shape in use: threads per CTA, resident CTAs, tile cells per CTA. */
lbmib_status lbmib_batch_config(const lbmib_batch* batch, int* threads, int* grid,
                                int* tile_cells);

#ifdef __cplusplus
}
#endif

#endif /* LBMIB_H */
