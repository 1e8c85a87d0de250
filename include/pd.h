/*
 * pd.h - C ABI of the GB300 PeriDEM hot-path library (libpd.so).
 *
 * One explicit velocity-Verlet step of bond-based peridynamics (PMB bonds with
 * critical-stretch breaking) inside every grain, short-range nodal contact
 * between grains and fragments, and rigid planar walls, after the paper's
 * Sec. 2-5 (equation of motion, Eq. motion; bond force, Eq. pmb and
 * Eq. peri-damage; contact, Eq. repulsive-force and the self-contact law; wall
 * contact, Sec. 4.1; time integration, Sec. 5.2).  Plus the bulk-stress MLP
 * surrogate (pd_mlp_*), which the paper motivates (RVE use, Sec. 1 and 6.4) but
 * does not specify.
 *
 * Conventions for every call:
 *  - Units are SI.  Node arrays are row-major n x 3 float64 (x0 y0 z0 x1 ...).
 *  - Node indices are the caller's order everywhere; the library's internal
 *    (grain-major, Morton) order never leaks through the ABI.
 *  - Input arrays are host pointers, read during the call and not retained:
 *    the caller keeps ownership.  Outputs go to caller-allocated host buffers.
 *  - Every call returns a pd_status; pd_last_error() gives the message.
 *  - Device memory is obtained through pd_options.alloc/free when given
 *    (e.g. a framework's caching allocator), else cudaMalloc/cudaFree.  The
 *    context owns it until pd_destroy.
 *  - Work runs on pd_options.stream (a cudaStream_t; NULL = the legacy default
 *    stream).  Calls that return data synchronise that stream.
 *  - A context is not thread-safe.  Errors raised on the device (non-finite
 *    state, wall penetration) are latched; the context then refuses pd_step
 *    until pd_set_state is called.
 */
#ifndef PD_H
#define PD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pd_ctx pd_ctx;
typedef struct pd_mlp pd_mlp;

typedef enum {
    PD_OK = 0,
    PD_EINVAL = -1,      /* bad argument: null pointer, size, value out of range */
    PD_ENOMEM = -2,      /* the allocator returned NULL */
    PD_ECUDA = -3,       /* a CUDA runtime call failed (message has the CUDA error) */
    PD_ESTATE = -4,      /* call out of order (e.g. pd_step before pd_build_bonds) */
    PD_ECAPACITY = -5,   /* a fixed capacity was exceeded and could not be regrown */
    PD_ENONFINITE = -6,  /* a force, displacement or velocity became NaN/inf */
    PD_ETIMEOUT = -7,    /* a bounded device wait gave up */
    PD_EWALL = -8        /* a node went a whole contact radius behind a wall */
} pd_status;

/* Arithmetic of the bond loop. */
enum { PD_MIXED = 0,  /* FP32 bond arithmetic; xi and eta from double-float pairs
                         (48-bit significands), FP64 state and accumulation */
       PD_FP64 = 1 }; /* every operation in FP64 */

/* Material (one per context).  Bond-based PD fixes nu = 1/4 in 3-D (Sec. 3.1.1),
 * so K = 2E/3.  constants = 0: c = 18K/(pi delta^4), s0 = sqrt(5 G0/(9 K delta));
 * constants = 1: the paper's table row (c = 12E/(pi delta^4 (1-nu)),
 * s0 = sqrt(5 pi G0/(12 E delta))).  K_n = contact_factor * 18K/(pi delta^5)
 * (Sec. 3.2).  break_mode = 0 breaks a bond when s > s0 (definition of the bond
 * memory gamma); 1 when |s| > s0 (the sentence before the table).
 * beta_d: normal contact damping (Sec. 3.3, Eq. damping-force), N s/m^7, 0 =
 * none.  Every contact pair adds beta_d ((v_j - v_i) . e) e V_j to the force
 * density of i (e = unit vector from p_i to p_j), and every node within R_c of
 * a wall adds beta_d ((v_wall - v_i) . n) n |S| (the wall substitution of
 * Sec. 4.1, |S| the cap volume), which the wall reaction includes.  The
 * velocity is the half-step velocity of velocity Verlet (pd_forces: the
 * current velocity).  Reading: the printed law pushes approaching points
 * together and normalises v; the dissipative linear law is used. */
typedef struct {
    double E;               /* Young's modulus, Pa (> 0) */
    double rho;             /* density, kg/m^3 (> 0) */
    double G0;              /* critical energy release rate, J/m^2 (> 0; inf = unbreakable) */
    double contact_radius;  /* R_c, m (> 0) */
    double contact_factor;  /* f_c in K_n (>= 0; 0 disables contact stiffness) */
    int constants;          /* 0 or 1, see above */
    int break_mode;         /* 0 or 1, see above */
    double beta_d;          /* normal contact damping coefficient (>= 0), see above */
    int micromodulus;       /* 0 = constant (default); 1 = conic c (delta - |xi|) (table of
                               Sec. 3.1.1): c = 90 K / (pi delta^5), s0 = sqrt(2 G0 / (3 K delta));
                               with constants = 1 the printed row, c = 60 E / (pi delta^5 (1 - nu)),
                               s0 = sqrt(7 pi G0 / (12 E delta)).  The bond force, the self-contact
                               law and pd_stable_dt use c(|xi|); pd_stable_dt_noalloc takes a
                               constant micromodulus only. */
    double mu;              /* stick-slip friction coefficient (>= 0; 0 = frictionless), Sec. 3.3
                               (Eq. regularized-friction).  A contact pair adds
                               -min(rho |v_t| / (dt (V_i + V_j)), mu f_r) V_j v_t / |v_t| to the force
                               density of i, v_t the part of v_i - v_j across the contact normal and
                               f_r the pair's repulsion per volume squared; a node within R_c of a
                               wall adds -min(rho |v_t| / dt, mu K_n (R_c - zbar) |S|) v_t / |v_t|,
                               v_t the part of v_i - v_wall along the wall, which the wall reaction
                               includes.  Readings: the force opposes the slip; the printed stick
                               branch rho |v_t| / dt is divided by V_i + V_j (a rigid wall: by |S|),
                               which conserves momentum and stops an isolated pair's sliding in one
                               step.  Velocities as for beta_d.  dt is that of the latest pd_step
                               (pd_step with nsteps = 0 sets it; 0 before any: the Coulomb limit,
                               slip at any speed); when it changes, pd_step first evaluates the
                               acceleration again with the new dt. */
    int wall_overlap;       /* 0 = the single-wall terms are summed (default); 1 = inclusion-
                               exclusion of Sec. 4.1.1: for every pair of walls with orthogonal
                               normals that a node touches, minus the repulsion of the region of
                               its R_c ball beyond both, K_n (R_c - |c - p|) |S| away from that
                               region's centroid c; plus the same for every mutually orthogonal
                               triple.  Damping and friction stay single-wall sums; the wall
                               reactions take each term's component along their own normal.
                               Readings: the regions' volumes and centroids are computed (the paper
                               gives the principle only), the triple term's stray V_x is dropped,
                               and walls that are not orthogonal keep the plain sum.  A material
                               with mu > 0 or wall_overlap = 1 runs without shared-memory tiles. */
} pd_material;

typedef struct {
    int device;                          /* CUDA device ordinal */
    void *stream;                        /* cudaStream_t, NULL = legacy default stream */
    void *(*alloc)(size_t bytes, void *alloc_ctx);  /* NULL: cudaMalloc */
    void (*free)(void *ptr, void *alloc_ctx);
    void *alloc_ctx;
    int precision;                       /* PD_MIXED or PD_FP64 */
    int contact;                         /* 1: nodal contact on, 0: off */
    int contact_every;                   /* steps between contact-list rebuilds; 0 = automatic */
    double skin;                         /* Verlet skin of the contact list, m; 0 = 0.5 R_c */
    int lanes_per_node;                  /* lanes sharing one node's bonds: 4, 8, 16, 32; 0 = autotune */
    int graph_chunk;                     /* steps per captured CUDA graph; 0 = 64 */
    int tiles;                           /* mixed path: shared-memory tiles 1 = on, -1 = off,
                                            0 = chosen by the autotuner (on when lanes are fixed) */
    int64_t cand_capacity;               /* initial capacity of the contact-candidate list
                                            (entries); 0 = max(1024, 8 n).  A rebuild that
                                            overflows it rolls its segment back and grows it. */
    int pairs;                           /* mixed path: each bond evaluated once, from its
                                            lower-index end, in two passes (Eq. pmb is pairwise
                                            antisymmetric): 1 = on, -1 = off, 0 = chosen by the
                                            autotuner; pairs = 1 with tiles = 1 is PD_EINVAL */
    int persistent;                      /* pd_step runs the steps between two contact-list
                                            rebuilds in one cooperative launch (a grid-wide
                                            barrier between steps; same results bit for bit):
                                            1 = on, -1 = off, 0 = chosen by the library.  Applies
                                            to the per-slot global-gather kernels; ignored while
                                            profiling. */
    int barrier_absent;                  /* test aid, 0 in use: the grid-wide barrier of the
                                            multi-step kernel waits for this many more blocks
                                            than it launches, so that its bounded wait (1 s)
                                            runs out: pd_step then returns PD_ETIMEOUT, the
                                            state of the segment's start is restored, and the
                                            error is latched until pd_set_state. */
} pd_options;

/* A rigid plane (Sec. 4.1).  normal points into the domain (unit length). */
typedef struct {
    double normal[3];
    double point[3];     /* a point of the plane at the current time */
    double velocity[3];  /* rigid translation velocity, m/s */
} pd_wall;

/* Bond-removal filter (Sec. 5.3), applied once in pd_build_bonds.
 * kind 1, notch (Sec. 5.3.1): a[0..3] = plane (a, b, c, d); the bond x1 -> x2 is
 *   removed if the plane parameter t = -(a x1 + b y1 + c z1 + d)/(a dx + b dy + c dz)
 *   satisfies 0 < t < 1 and the crossing point lies in the box a[4..6]..a[7..9]
 *   (the notch face; the paper's plane is unbounded).  x1 is the endpoint with
 *   the smaller caller index, so both directions decide alike.
 * kind 2, inner sphere (Sec. 5.3.2): a[0..2] centre, a[3] radius; the bond is
 *   removed if either end lies strictly inside. */
typedef struct {
    int kind;
    double a[12];
} pd_bond_filter;

/* Fills *opt with defaults: device 0, default stream, cudaMalloc, PD_MIXED,
 * contact on, automatic rebuild period and skin, autotuned lanes and tiles,
 * chunk 64. */
void pd_default_options(pd_options *opt);

/* Creates a context for n nodes (Sec. 2.1: nodes x with volumes, grouped in
 * grains P_i).  x: n*3 reference positions; vol: n volumes (> 0); grain: n grain
 * ids (>= 0); v0: n*3 initial velocities or NULL for rest.  u starts at 0, t at 0.
 * Sorts the nodes grain-major and in Morton order inside each grain (internal).
 * Errors: PD_EINVAL (n < 1, n > 2^31-1, null arrays, bad material/options),
 * PD_ENOMEM, PD_ECUDA.  On error *out is NULL. */
pd_status pd_create(int64_t n, const double *x, const double *vol, const int32_t *grain,
                    const double *v0, const pd_material *mat, const pd_options *opt,
                    pd_ctx **out);

/* Builds the bond family (Sec. 3.1): ordered pairs (i, j), i != j, of the same
 * grain with |x_j - x_i| < horizon (strict; Eq. pmb), squared distance
 * evaluated in FP64 as ((dx*dx + dy*dy) + dz*dz) without FMA, minus the
 * filters.  Sets the micromodulus and critical stretch for this horizon, marks
 * every bond intact, and evaluates the forces at the current state (which may
 * already break bonds).  May be called again to rebuild from scratch.
 * Errors: PD_EINVAL (horizon <= 0, nfilt < 0, bad filter kind),
 * PD_ECAPACITY (more than 2^31-1 bonds), PD_ENOMEM, PD_ECUDA. */
pd_status pd_build_bonds(pd_ctx *ctx, double horizon, int nfilt, const pd_bond_filter *filt);

/* Replaces the wall set (0 <= nw <= 6).  Wall forces sum the single-wall cap
 * terms (Sec. 4.1); with pd_material.wall_overlap = 1 the inclusion-exclusion
 * of Sec. 4.1.1 over orthogonal walls that a node touches is applied on top. */
pd_status pd_set_walls(pd_ctx *ctx, int nw, const pd_wall *walls);

/* Current wall points (nw*3), after the walls moved with their velocity. */
pd_status pd_get_walls(pd_ctx *ctx, double *points);

/* Body force density b (N/m^3), added to every node (Eq. intra_particle). */
pd_status pd_set_body_force(pd_ctx *ctx, const double b[3]);

/* Critical time step of the explicit scheme on the current bonds (the paper
 * states dt came from a stability analysis, Sec. 5.2; the bound used is
 * Silling-Askari's dt = min_i sqrt(2 rho / sum_j V_j c / |xi_ij|)).
 * Errors: PD_ESTATE before pd_build_bonds. */
pd_status pd_stable_dt(pd_ctx *ctx, double *dt_crit);

/* Advances nsteps velocity-Verlet steps of size dt (Sec. 5.2):
 *   v += dt/2 a; u += dt v; walls move; a = (F(u) + b)/rho; v += dt/2 a,
 * where F is the bond force with breaking (Eq. peri-damage), contact and wall
 * force.  Captured and replayed as CUDA graphs.  Blocks until done.  The
 * steps run in segments of 2 graph chunks (up to 128 steps; a chunk is the
 * largest multiple of the rebuild period within graph_chunk); a segment
 * whose contact list went stale or overflowed is rolled back to its own start
 * and rerun with a shorter rebuild period or larger lists.  The contact list is
 * rebuilt often enough for the fastest node (or wall) to gain 50% in speed
 * (150% while speeds are growing).  A call of one step rebuilds it only when the
 * list on the device no longer holds for the current state (not built since the
 * bonds were, or the displacement bound since the last rebuild past half the
 * skin; a state applied by pd_set_state* is evaluated on a list rebuilt from it);
 * the forces do not depend on which rebuild made the list, so the trajectory is
 * the same either way.  With friction (mu > 0) the call first
 * records dt as the friction's time step and, if it changed, evaluates the
 * acceleration at the current state again with it; nsteps = 0 does only that.
 * Errors: PD_ESTATE (no bonds yet, or a latched device error), PD_EINVAL
 * (dt <= 0, nsteps < 0), PD_ENONFINITE / PD_EWALL (state restored to the start
 * of the segment in which it happened, so t tells how far the call got, and
 * latched), PD_ECAPACITY, PD_ECUDA. */
pd_status pd_step(pd_ctx *ctx, double dt, int64_t nsteps);

/* Damage phi_i = 1 - intact_i / initial_i, 0 for nodes without bonds (Sec. 3.1.1;
 * the paper's wording describes the complement).  phi: n doubles, caller order. */
pd_status pd_damage(pd_ctx *ctx, double *phi);

/* Wall reactions and bulk stress from the last force evaluation.
 * wall_force (nullable): nw*3, force exerted by the nodes on each wall.
 * area (nullable when nw == 0): nw face areas used to turn reactions into
 * tractions.  sigma: Voigt (xx, yy, zz, yz, xz, xy); per wall the column
 * sigma e_k = -(R_l / A_l)(m_l . e_k) with m_l = -normal the aggregate's outward
 * normal, averaged over walls facing the same axis and symmetrised; compression
 * is negative (reading of "bulk strength" in Sec. 6.4/6.5). */
pd_status pd_bulk_stress(pd_ctx *ctx, const double *area, double sigma[6], double *wall_force);

/* The same stress from the wall forces averaged over time: every step adds
 * dt * R_l (the reaction of its force evaluation) to an impulse J_l; this call
 * returns sigma of the mean forces J_l / T, the mean forces themselves
 * (wall_force, nullable, nw*3) and T, the time covered (span, nullable), then
 * zeroes J and T.  pd_create, pd_set_walls and pd_set_state also zero them.
 * The paper reports wall forces over time (Sec. 6.4); the average over a
 * window is the macroscopic stress of a representative volume without the
 * contact chatter of single steps.  All zeros while T = 0. */
pd_status pd_bulk_stress_mean(pd_ctx *ctx, const double *area, double sigma[6], double *wall_force,
                              double *span);

/* Fragments (particles that split off; the paper identifies them, Sec. 1, but
 * gives no algorithm): the connected components of the graph of nodes and
 * intact bonds at the current state.  label (n, nullable, caller order): the
 * smallest caller index in the node's fragment; *nfrag: number of fragments.
 * Errors: PD_ESTATE before pd_build_bonds, PD_ENOMEM, PD_ECUDA. */
pd_status pd_fragments(pd_ctx *ctx, int32_t *label, int64_t *nfrag);

/* Per-fragment statistics at the current state, fragments in increasing label
 * order: node count (size), summed nodal volume, and damage read as the broken
 * fraction of the fragment's initial bond slots (1 - intact / initial, 0 without
 * bonds).  nfrag must equal pd_fragments' count for this state (PD_EINVAL
 * otherwise); each output (nfrag entries) is nullable.  A fragment's volume is
 * summed in a fixed order (its nodes by caller index, strided over one warp,
 * then a fixed butterfly), so repeated calls on one state agree bit for bit. */
pd_status pd_fragment_stats(pd_ctx *ctx, int64_t nfrag, int64_t *size, double *volume, double *damage);

/* Number of directed bonds B (each undirected bond counted twice). */
pd_status pd_num_bonds(pd_ctx *ctx, int64_t *B);

/* Canonical bond list: rowptr (n+1) and col (B), rows in caller order, columns
 * ascending caller indices. */
pd_status pd_bonds(pd_ctx *ctx, int64_t *rowptr, int32_t *col);

/* Contact pairs at the current state (Sec. 3.2 and self-contact): ordered
 * pairs (i, j), i != j, with |p_j - p_i| < R_c (FP64, no FMA), excluding same-
 * grain pairs whose bond is intact; sorted by (i, j), caller indices.
 * ij == NULL: *npairs receives the count.  Otherwise *npairs is the capacity in
 * pairs on entry and the count on return (PD_ECAPACITY if too small). */
pd_status pd_contacts(pd_ctx *ctx, int64_t *npairs, int32_t *ij);

/* Force density F (n*3, caller order) at the current state without stepping:
 * applies breaking exactly as a step does.  Damping and friction see the
 * current velocity; friction the time step of the latest pd_step. */
pd_status pd_forces(pd_ctx *ctx, double *F);

/* State for checkpoints and parity: u, v (n*3), broken (B bytes, 1 = broken, in
 * pd_bonds order), t.  Any output may be NULL.  On the mixed path u and v are
 * held as double-float pairs kept on the FP64 grid (hi + lo is a double after
 * every update and every pd_set_state), so the doubles returned are the state
 * exactly, not a rounding of it. */
pd_status pd_get_state(pd_ctx *ctx, double *u, double *v, uint8_t *broken, double *t);

/* Sets the state (any input may be NULL to keep it), clears a latched device
 * error and re-evaluates the forces (which may break bonds).  u and v are
 * checked on the device before anything is applied: a non-finite value in
 * either returns PD_EINVAL and leaves the whole state unchanged.  Each value is
 * held as the pair hi = RN(x), lo = x - hi rounded towards zero (hi + lo is x,
 * or x with its last bits cut, within 2^-47 |x| + 2^-149 of it; the FP64 path
 * holds x).  Every given part is compared on
 * the device with the current state first; when applying it would change
 * nothing (a state that pd_get_state returned, sent back unchanged, on any
 * path) it is not applied again, and, when the material has no
 * velocity-dependent forces (beta_d = 0, mu = 0), the force evaluation is
 * skipped too.  Since the live pairs lie on the FP64 grid, setting a state read
 * out at step k gives the state the run held at step k, whether the context is
 * that run's or a fresh one with the same options, walls and time: the run goes
 * on bit for bit as the uninterrupted one (a checkpoint restart is exact; with damping or friction the stored
 * acceleration saw the last step's half-step velocity, the re-evaluation sees
 * the current one, so there the restarted run is the one an uninterrupted run
 * with a pd_set_state at step k gives).  The wall impulses of
 * pd_bulk_stress_mean are zeroed in any case.  Errors: PD_EINVAL (non-finite u
 * or v), PD_ESTATE (bond memory before pd_build_bonds), PD_ECUDA, and those of
 * the force evaluation. */
pd_status pd_set_state(pd_ctx *ctx, const double *u, const double *v, const uint8_t *broken,
                       const double *t);

/* pd_get_state and pd_set_state with the bond memory packed: broken_bits holds
 * ceil(B/32) words, bit (c % 32) of word (c / 32) set when slot c of the
 * pd_bonds order is broken (bits past B are 0 on output and ignored on input).
 * The same state in an eighth of the bytes, for checkpoints and host round
 * trips; otherwise identical (NULL keeps, errors, re-evaluation). */
pd_status pd_get_state_packed(pd_ctx *ctx, double *u, double *v, uint32_t *broken_bits, double *t);
pd_status pd_set_state_packed(pd_ctx *ctx, const double *u, const double *v, const uint32_t *broken_bits,
                              const double *t);

/* Autotuning record of the bond loop: lanes per node chosen, the kernel chosen
 * (0 = every directed slot gathers its neighbour from global memory, 1 =
 * shared-memory tiles, 2 = each bond once in two passes) and the measured time
 * (ms) of one force evaluation per candidate: ms[0..3] kernel 0 with 4, 8, 16, 32
 * lanes, ms[4..7] kernel 1, ms[8..11] kernel 2 (0 = not run).  The kernel is the
 * one with the fastest evaluation; its lane count the smallest within 3% of that
 * time (a full step's per-node work favours fewer lanes).  Any pointer may be
 * NULL. */
pd_status pd_tuning(pd_ctx *ctx, int *lanes, int *kernel, double ms[12]);

/* Profiling switch.  When on, pd_step launches its kernels one by one (no CUDA
 * graph) with CUDA events around every fused force/update launch, so that
 * pd_last_step_stats can report that kernel's own device time.  Off by default. */
pd_status pd_set_profiling(pd_ctx *ctx, int on);

/* Timing of the last pd_step: ms_force = summed device milliseconds of the
 * fused force/update launches (only when profiling is on, else 0); ms_total =
 * device milliseconds of the call's segments (event-timed on the context's
 * stream; attempts that were rolled back are not counted); launches = kernels
 * launched by those segments. */
pd_status pd_last_step_stats(pd_ctx *ctx, double *ms_force, double *ms_total, int64_t *launches);

/* Counters since pd_create (each pointer nullable): steps taken, contact-list
 * rebuilds of those steps, and segments rolled back and rerun because the list
 * went stale or overflowed (see pd_step). */
pd_status pd_step_counters(pd_ctx *ctx, int64_t *steps, int64_t *rebuilds, int64_t *rollbacks);

/* pd_set_state / pd_set_state_packed calls since pd_create (each pointer
 * nullable): applied (the forces were evaluated again) and unchanged (the state
 * equalled the current one and the evaluation was skipped). */
pd_status pd_state_counters(pd_ctx *ctx, int64_t *applied, int64_t *unchanged);

const char *pd_last_error(const pd_ctx *ctx);
void pd_destroy(pd_ctx *ctx);

/* Allocation-free critical time step.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory when they need the
 * step, e.g. code running while a memory pool is frozen, a runtime that owns
 * every device allocation itself, or a host callback where cudaMalloc is not
 * allowed.  Same bound as pd_stable_dt, dt = min_i sqrt(2 rho / sum_j V_j c /
 * |x_j - x_i|) over rows with at least one bond, computed from the caller's
 * DEVICE arrays: x (n*3 FP64, row-major), vol (n), rowptr (n+1, int64), col
 * (rowptr[n] int32 node indices); c is the micromodulus and rho the density.
 * Writes the step to the caller's device double *dt_out (INFINITY when no row
 * has a bond) on `stream` (cudaStream_t, NULL = legacy stream); does not
 * synchronise.
 * It allocates nothing: its scratch (per-block partial minima) is a file-scope
 * device array of 65,536 doubles (512 KiB) that every GPU loading this library
 * holds until the process exits.  Hence n <= 16,777,216; larger n gives
 * PD_EINVAL.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  The address is kept with the process-unique ID of the
 * context it was looked up in: after cudaDeviceReset (or any other teardown of
 * the context) the next call finds a new context ID and looks the address up
 * again, so that call, too, belongs outside a capture.  All calls on a device
 * share the array, so calls that overlap on the GPU (other streams, other
 * threads) race; each call writes every partial it reads, so nothing needs
 * clearing between calls.
 * Errors: PD_EINVAL (null pointer, n < 1, n too large, c or rho <= 0),
 * PD_ECUDA (no current device, symbol lookup or launch failed; taken from the
 * calls' own return codes).  A runtime error that an earlier call left pending
 * is neither reported by this call nor cleared by it; an error this call raises
 * is cleared when none was pending. */
pd_status pd_stable_dt_noalloc(int64_t n, const double *x, const double *vol, const int64_t *rowptr,
                               const int32_t *col, double c, double rho, void *stream, double *dt_out);

/* ---------------------------------------------------------------------------
 * Bulk-stress surrogate: an MLP dims[0] -> ... -> dims[nlayers] with exact GELU
 * between layers, BF16 weights and activations, FP32 accumulation, FP32 master
 * weights, MSE loss and Adam (beta 0.9/0.999, eps 1e-8).  Not in the paper.
 * Parameter vector layout: for each layer, W (out x in, row-major) then b (out).
 * ------------------------------------------------------------------------- */

/* dims: nlayers+1 widths, each a multiple of 1 and <= 1024; seed draws the
 * initial weights (uniform +-1/sqrt(fan_in), SplitMix64); device/stream as in
 * pd_options (stream NULL = default). */
pd_status pd_mlp_create(const int *dims, int nlayers, uint64_t seed, int device, void *stream,
                        pd_mlp **out);
/* Y (batch x dims[nlayers], FP32) = MLP(X); X (batch x dims[0], FP32) is
 * rounded to BF16 (nearest-even). Host pointers. */
pd_status pd_mlp_forward(pd_mlp *m, const float *X, int64_t batch, float *Y);
/* Same with device pointers (no copies, no synchronisation; a tensor-core
 * wait that gave up is reported by the next pd_mlp_forward). */
pd_status pd_mlp_forward_device(pd_mlp *m, const float *X, int64_t batch, float *Y);
/* Forward kernels: 0 (default) = the fused tcgen05 kernel (TMA-fed weights,
 * TMEM accumulators, activations kept in shared memory across layers) when
 * every layer is at most 256 wide on an sm_100+ GPU, else mma.sync GEMMs;
 * 1 = mma.sync GEMMs only; 2 = the tcgen05 kernel only (a forward that it
 * cannot run returns PD_EINVAL).  The same switch selects the training kernels:
 * 0 and 2 train on tcgen05 (the fused forward also stores the pre-activations
 * and the transposed layer inputs; weight and data gradients are TMA-fed
 * tcgen05 GEMMs, hidden widths multiples of 32), 1 on the mma.sync GEMMs.
 * PD_EINVAL for any other value. */
pd_status pd_mlp_set_forward_path(pd_mlp *m, int path);
/* One Adam step on the MSE loss of (X, T); *loss receives the loss before the
 * update (nullable).  Host pointers. */
pd_status pd_mlp_train_step(pd_mlp *m, const float *X, const float *T, int64_t batch, float lr,
                            float *loss);
/* Same with device pointers; loss is a device float (nullable). */
pd_status pd_mlp_train_step_device(pd_mlp *m, const float *X, const float *T, int64_t batch,
                                   float lr, float *loss);
/* Gradient of the MSE loss (FP32, parameter layout) without updating. */
pd_status pd_mlp_grad(pd_mlp *m, const float *X, const float *T, int64_t batch, float *grad,
                      float *loss);
pd_status pd_mlp_num_params(pd_mlp *m, int64_t *count);
pd_status pd_mlp_get_params(pd_mlp *m, float *w);
/* Sets the FP32 master weights and resets Adam's moments and step count. */
pd_status pd_mlp_set_params(pd_mlp *m, const float *w);
const char *pd_mlp_last_error(const pd_mlp *m);
void pd_mlp_destroy(pd_mlp *m);

#ifdef __cplusplus
}
#endif
#endif /* PD_H */
