/*
 * rb.h -- C ABI of librb, the GB300 (sm_103a) tree gravity + tree collision
 * library for collisional N-body simulations after REBOUND (Rein & Liu 2012).
 *
 * Every step is the drift-kick-drift (DKD) scheme of Sect. 3: drift dt/2,
 * boundaries (Sect. 2.3), octree at the mid-step positions (Sect. 4.2),
 * Barnes-Hut self-gravity (Eq. 1, Sect. 4.2), kick dt, drift dt/2,
 * boundaries, then collision detection -- the tree search (Sect. 5.2, Eq. 3)
 * or the plane sweep (Sect. 5.3) -- and the resolution of the collisions
 * found (Sect. 5, Eq. 2).  All of it runs in the
 * library's CUDA kernels on one GPU; nothing falls back to the CPU.
 *
 * Conventions shared by every call:
 *  - Return value: RB_OK (0) or a negative RB_ERR_* code.  No call throws or
 *    aborts across the ABI; rb_last_error() describes the last failure.
 *  - Host pointers ("host") are read or written before the call returns and
 *    stay owned by the caller.  Device memory is owned by the library and
 *    allocated with cudaMallocAsync on the simulation's stream.
 *  - Particle ids: 0..n-1 in the order given to rb_set_particles for that
 *    box; they are stable while particles move, and removed particles (open
 *    boundaries) leave gaps.  Per-particle outputs are in ascending id order.
 *  - Units are the caller's; G fixes them.  Positions are relative to the box
 *    centre: a box spans [-L_a/2, L_a/2) along axis a; its tree's root cube
 *    has side L_x and contains it (L_y, L_z <= L_x, e.g. an elongated
 *    shearing box of radial size L_x).
 */
#ifndef RB_H
#define RB_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    RB_OK = 0,
    RB_ERR_ARG = -1,       /* invalid argument or configuration */
    RB_ERR_CAPACITY = -2,  /* a fixed-size device buffer overflowed twice in a row */
    RB_ERR_TIMEOUT = -3,   /* a bounded device wait gave up */
    RB_ERR_NONFINITE = -4, /* a position became NaN or infinite */
    RB_ERR_CUDA = -5,      /* a CUDA runtime call failed */
    RB_ERR_STATE = -6      /* call out of order (e.g. no particles yet) */
};

/* Boundary conditions of Sect. 2.3. */
enum { RB_BC_OPEN = 0, RB_BC_PERIODIC = 1, RB_BC_SHEAR = 2 };
/* Integrators: leap-frog (Sect. 3.1), symplectic epicycle integrator (Sect. 3.3). */
enum { RB_INT_LEAPFROG = 0, RB_INT_SEI = 1 };
/* Precision of the gravity walk.  Positions, velocities, moments and the
 * kick/drift are FP64 in every mode. */
enum { RB_WALK_FP64 = 0, RB_WALK_FP32 = 1, RB_WALK_FP32_LEARNED = 2 };
/* Collision detectors: none; the tree search of Sect. 5.2 (particles that
 * overlap at the end of the step, Eq. 3 pruning); the plane sweep along x of
 * Sect. 5.3 (straight-line trajectories over the drift around the detection
 * time, tau in [-dt/2, dt/2], that come closer than R_a + R_b). */
enum { RB_COLL_NONE = 0, RB_COLL_TREE = 1, RB_COLL_SWEEP = 2 };
/* Laws of the normal coefficient of restitution (Sect. 5 allows a constant
 * or a velocity-dependent one): cfg.eps_restitution, or the power law
 * eps(v_n) = min(1, (|v_n| / v_c)^(-p)) of the normal approach speed. */
enum { RB_EPS_CONSTANT = 0, RB_EPS_POWER = 1 };
/* Order in which the walks and the collision search take their targets, 32
 * per warp (a launch shape: results per target do not depend on it, except
 * for the FP32 summation order of the walk): the Morton order of the tree;
 * a 2D Hilbert order of (x, y) on a 1024 x 1024 grid of the root cube (thin
 * sheets: a warp's targets then span a compact patch of the sheet); a 3D
 * Hilbert order on a 128^3 grid.  The box comes first in every order. */
enum { RB_TILE_MORTON = 0, RB_TILE_HILBERT_XY = 1, RB_TILE_HILBERT_XYZ = 2 };

typedef struct rb_config {
    double G;               /* gravitational constant of Eq. 1 */
    double omega;           /* epicyclic frequency Omega (SEI, shear offsets) */
    double omega_z;         /* vertical frequency Omega_z; <= 0 means = omega (Sect. 3.3) */
    double box[3];          /* box side per axis (periodic lengths; open boxes remove particles
                               outside them); box[1], box[2] <= box[0], the root cube's side */
    double theta;           /* critical opening angle (Sect. 4.2), > 0 */
    double eps_restitution; /* normal coefficient of restitution (Eq. 2), in [0, 1] */
    double softening;       /* gravitational softening b of Eq. 1, >= 0 */
    double dt;              /* time step (Sect. 3), > 0 */
    double t0;              /* time at step 0 (sets the shear offset) */
    int nghost[3];          /* ghost boxes per direction (Sect. 2.3); z needs z_periodic */
    int boundary;           /* RB_BC_* */
    int z_periodic;         /* 1: z periodic (RB_BC_PERIODIC/SHEAR); 0: open in z */
    int integrator;         /* RB_INT_* */
    int walk;               /* RB_WALK_* */
    int quadrupole;         /* 1: monopole + quadrupole cells (Sect. 4.2); 0: monopole */
    int gravity;            /* 1: tree self-gravity; 0: none */
    int collisions;         /* RB_COLL_*: detector whose pairs are resolved (Eq. 2) */
    int reserved[5];        /* must be zero */
} rb_config;

typedef struct rb_stats_t {
    int64_t steps;            /* steps taken since rb_set_particles / rb_set_time */
    int64_t n_live;           /* particles in all boxes */
    int64_t cells;            /* tree cells (branching nodes) in the last gravity tree */
    int64_t pairs_found;      /* collision pairs found in the last step */
    int64_t pairs_resolved;   /* pairs that were approaching and were resolved */
    int64_t cell_interactions;/* accepted cells in the last gravity walk (all particles, images) */
    int64_t leaf_interactions;/* exact particle terms in the last gravity walk */
    int64_t mac_tests;        /* opening-angle tests in the last gravity walk */
    int64_t fp64_rechecks;    /* FP32 opening tests decided again in FP64 (guard band) */
    int64_t pair_capacity;    /* current pair buffer capacity */
    int64_t kernels_per_step; /* kernel launches in one captured step graph */
    int64_t walk_block;       /* threads per block of the gravity walk */
    int64_t search_block;     /* threads per block of the collision search */
    double  t;                /* simulation time */
    double  ms_last_step;     /* device time of the last step (events), ms */
    /* device time of each stage of the last step when profiling is on (ms):
     * 0 drift+keys, 1 sort+gather, 2 tree, 3 moments, 4 gravity walk,
     * 5 kick+drift+keys, 6 sort+gather, 7 tree, 8 collision records,
     * 9 collision search, 10 pair sort, 11 resolution */
    double  ms_stage[12];
    int64_t corrections;      /* learned walk: band cells corrected by the network in the last walk */
    int64_t warp_iterations;  /* FP32 walk: warp iterations of the last walk (union walk: entries
                                 processed, 32 targets each; group walk: frontier rounds, list
                                 entries and mixed-subtree iterations) */
    int64_t walk_group;       /* FP32 walk shape: 0 union walk, 4 group walk (4-lane subgroups
                                 for the mixed subtrees) */
    int64_t tile_order;       /* order in which walks and search take their targets (RB_TILE_*) */
    int64_t search_visits;    /* tree search: entries (cells and leaves) tested by the targets of
                                 the last collision search, all images; counted only at
                                 rb_set_profiling level 2 (else 0; 0 for the plane sweep) */
    int64_t search_iterations;/* tree search: warp iterations of that search (32 targets each) */
} rb_stats_t;

typedef struct rb_sim rb_sim; /* opaque, owned by the library */

/* Create a simulation of `nbox` independent boxes (1, or B for an ensemble
 * advanced together) that share `cfg`; box sizes default to cfg->box.
 * cuda_stream: a cudaStream_t (NULL: the library creates its own).  The
 * stream must outlive the simulation.  *out receives the handle.
 * Errors: RB_ERR_ARG (theta <= 0, dt <= 0, eps outside [0,1], a box side
 * <= 0 or box[1] or box[2] above box[0], nghost < 0 or > 7, SEI without
 * omega, an unknown detector, reserved != 0), RB_ERR_CUDA. */
int rb_create(const rb_config* cfg, int nbox, void* cuda_stream, rb_sim** out);

/* Set the side lengths of box `box` (host array of 3; L[1], L[2] <= L[0]).
 * Meant before rb_set_particles; called later, it keeps the current
 * particles of every box (ids renumbered over the live ones if an open
 * boundary removed some) and restarts the step counter. */
int rb_set_box(rb_sim* sim, int box, const double L[3]);

/* Copy n particles (host arrays: positions, velocities, masses, radii) into
 * box `box`, replacing what it held; ids become 0..n-1 in this order and
 * the step counter restarts at 0 (time cfg->t0 or the last rb_set_time).
 * The other boxes keep their current particles (ids renumbered over the
 * live ones if an open face removed some, as rb_set_box does).
 * Errors: RB_ERR_ARG (n < 0, box out of range, a particle outside the root
 * box, r < 0, m < 0, total particles above 2^24), RB_ERR_NONFINITE. */
int rb_set_particles(rb_sim* sim, int box, int64_t n, const double* x, const double* y,
                     const double* z, const double* vx, const double* vy, const double* vz,
                     const double* m, const double* r);

/* Advance every box by nsteps DKD steps (Sect. 3) on the simulation's
 * stream, replaying a captured CUDA graph per step; returns once the steps
 * are done and the device error word was checked.  A pair-buffer overflow is
 * repaired inside the step (buffer grown, the search re-run before any
 * velocity changes); RB_ERR_CAPACITY only if that fails.  Other errors:
 * RB_ERR_NONFINITE (a position became non-finite or left the box by more
 * than 4096 box lengths in one drift half), RB_ERR_STATE (a malformed tree
 * met by a walk; the learned walk without weights), RB_ERR_TIMEOUT (a
 * bounded device wait gave up: the resolution queue's or a radix pass's
 * look-back), RB_ERR_CUDA. */
int rb_step(rb_sim* sim, int64_t nsteps);

/* Copy the live particles of box `box`, in ascending id order, into host
 * arrays of capacity cap (any output pointer may be NULL).  *n_out receives
 * the live count (also when it exceeds cap; then RB_ERR_ARG). */
int rb_get_particles(rb_sim* sim, int box, int64_t cap, int64_t* n_out, double* x, double* y,
                     double* z, double* vx, double* vy, double* vz, double* m, double* r,
                     int64_t* id);

/* Energy and momentum of box `box` (Sect. 6.2) at the current time:
 * E = sum m v^2 / 2 + W (+ sum m (Omega_z^2 z^2 / 2 - 3/2 Omega^2 x^2) for
 * SEI), W = (1/2) sum m_i phi_i with phi from an FP64 tree walk at theta over
 * the ghost images (0 when gravity is off); P = sum m v (host array of 3). */
int rb_energy(rb_sim* sim, int box, double* E, double P[3]);
/* The terms rb_energy adds up (Sect. 6.2), for checking each on its own:
 * terms (host array of 6) = K = sum m |v|^2 / 2, U = the SEI tidal and
 * vertical term (0 for leap-frog), W = (1/2) sum m_i phi_i, P_x, P_y, P_z.
 * Errors: as rb_energy. */
int rb_energy_terms(rb_sim* sim, int box, double terms[6]);

/* Test and measurement hooks. */

/* Build the gravity tree on the current positions and evaluate the walk
 * without moving anything; results are read with rb_get_accelerations,
 * rb_get_counts and rb_get_tree.  The time used for the ghost offsets is
 * the current time. */
int rb_compute_gravity(rb_sim* sim);
/* Accelerations of the last gravity walk (kick or rb_compute_gravity), host
 * arrays in id order. */
int rb_get_accelerations(rb_sim* sim, int box, int64_t cap, double* ax, double* ay, double* az);
/* Per-particle counts of the last gravity walk: accepted cells, exact
 * particle terms, opening-angle tests (host arrays in id order). */
int rb_get_counts(rb_sim* sim, int box, int64_t cap, int64_t* ncell, int64_t* nleaf,
                  int64_t* nmac);
/* Branching cells of the last gravity tree of box `box`: depth, the ids of
 * their particles (concatenated, `count` each) and FP64 moments
 * (M; centre of mass xyz; Q as xx, yy, zz, xy, xz, yz).  *ncell receives the
 * number of cells; arrays may be NULL.  member_cap bounds member_ids. */
int rb_get_tree(rb_sim* sim, int box, int64_t cap, int64_t* ncell, int32_t* depth,
                int64_t* count, double* M, double* com, double* Q, int64_t member_cap,
                int64_t* member_ids);
/* Run the configured detector (tree search, Sect. 5.2, or plane sweep,
 * Sect. 5.3, with the current velocities) on the current positions without
 * resolving; read the pairs with rb_get_pairs. */
int rb_detect_collisions(rb_sim* sim);
/* Collision pairs of the last search of box `box` in resolution order: ids
 * a < b and the ghost image code of b as seen from a,
 * code = (gx+7) | (gy+7) << 4 | (gz+7) << 8 (host arrays). */
int rb_get_pairs(rb_sim* sim, int box, int64_t cap, int64_t* n, int64_t* id_a, int64_t* id_b,
                 int32_t* code);
/* Test hook: set the collision pair buffer to `cap` pairs (>= 1).  A search
 * that finds more pairs than fit resolves nothing; the step then grows the
 * buffer and searches again before any velocity changes, so results do not
 * depend on cap. */
int rb_set_pair_capacity(rb_sim* sim, int64_t cap);
/* Test hook: with `on` nonzero the first pair of every sorted collision queue
 * waits for one predecessor too many, so it never becomes ready; the
 * resolution's threads wait for its queue slot at most half a second and the
 * step returns RB_ERR_TIMEOUT with the device context intact (velocities then
 * hold a partial resolution).  0 restores normal resolution. */
int rb_debug_hold_pair(rb_sim* sim, int on);
/* Set / read the simulation time (restarts the step counter at t). */
int rb_set_time(rb_sim* sim, double t);
int rb_get_time(rb_sim* sim, double* t);
/* Counters of the last step (host struct). */
int rb_stats(rb_sim* sim, rb_stats_t* out);
/* on = 1: record CUDA events between the stages of every step (event nodes
 * inside the step graph) so rb_stats reports per-stage device times.
 * on = 2: also run the tree collision search in its counting variant, so
 * rb_stats reports search_visits and search_iterations (that variant is
 * about 9% slower; at 0 and 1 both counters read 0).  on = 0 turns both off.
 * Errors: RB_ERR_ARG (on outside 0..2). */
int rb_set_profiling(rb_sim* sim, int on);
/* Time the gravity walk and the tree collision search on the current
 * positions at 64, 128 and 256 threads per block, for the plain FP32 walk at
 * each warp shape (walk_group 0 and 4), and under each tile order (with the
 * cost of the sort that builds it); best of 3 after a warm-up each, and keep
 * the fastest combination; results are cached per (particle-count bucket,
 * theta, walk mode, batched) for the process, and use_cache = 1 takes a
 * cached choice without timing.  Positions and velocities are not changed. */
int rb_autotune(rb_sim* sim, int use_cache);
/* Set the launch shapes directly: walk_block and search_block 64, 128 or 256
 * threads per block; walk_group (plain FP32 walk) 0 for the union walk, in
 * which each warp walks the union of its 32 targets' walks, or 4 for the
 * group walk, in which cells that all 32 targets of a warp provably accept
 * or open are decided once (Sect. 4.2 opening test against the bounding box
 * of the targets; accepted cells go to an interaction list staged in shared
 * memory) and the remaining subtrees are walked by subgroups of 4 lanes;
 * tile_order one of RB_TILE_*.  Each target's accepted cells do not depend
 * on them (each target runs its own walk).  Errors: RB_ERR_ARG for any
 * other value. */
int rb_set_launch_shape(rb_sim* sim, int walk_block, int search_block, int walk_group, int tile_order);
/* Test particles (Sect. 4: particles that feel gravity without exerting it):
 * in every box, particles with id >= n_active keep their mass for collisions
 * and kinetic energy but are not sources of Eq. 1.  n_active < 0 (the
 * default): every particle is a source.  Errors: RB_ERR_ARG (null sim). */
int rb_set_n_active(rb_sim* sim, int64_t n_active);
/* Restitution law of Eq. 2: RB_EPS_CONSTANT (cfg.eps_restitution) or
 * RB_EPS_POWER with v_c > 0 and p >= 0 (RB_ERR_ARG otherwise). */
int rb_set_restitution(rb_sim* sim, int law, double v_c, double p);
/* Destroy the simulation and free its device memory. */
void rb_destroy(rb_sim* sim);

/* Learned far-field correction.  Not in the paper: a network
 * 12 -> 64 -> 64 -> 64 -> 3 (GELU, tanh form) predicts, for a target point p
 * and an accepted cell (Sect. 4.2), the residual between the cell's exact
 * force (Eq. 1 over its particles) and its multipole force, in units of
 * G M / R^2 (R = |p - com|).  Inputs: r_hat (3), w/R, log10 N_c,
 * (com - centre)/w (3), and with Qh = Q/(M w^2): r_hat.Qh.r_hat, |Qh r_hat|,
 * tr(Qh^2), det(Qh).  Weights: 9347 floats, W1 (12x64), b1, W2 (64x64), b2,
 * W3 (64x64), b3, W4 (64x3), b4, each W row-major input x output; the
 * kernels run them as BF16 on tensor cores with FP32 accumulation. */
#define RB_MLP_PARAMS 9347
/* Load the weights (host array) and the fallback angle theta_fb in
 * (0, cfg.theta]: with walk = RB_WALK_FP32_LEARNED the walk runs at
 * cfg.theta and adds the predicted residual of every accepted cell with
 * w/R > theta_fb.  The network runs inside the walk on each warp's queued
 * band cells (inputs computed in FP32 from the walk records), so there is
 * no per-particle limit on corrected cells; rb_stats reports how many there
 * were.  Errors: RB_ERR_ARG (count or angle), RB_ERR_NONFINITE. */
int rb_load_mlp(rb_sim* sim, const float* w, int64_t nw, double theta_fallback);
/* Training samples from the current positions of every box: a tree walk at
 * theta_hi records the accepted cells with w/R > theta_lo, each kept with
 * probability prob (a counter-based hash of the request and seed); for each
 * the 12 inputs (X, host, cap x 12) and the residual (Y, cap x 3) are
 * computed in FP64.  meta (cap x 5, may be NULL): target id, image code,
 * cell depth, lowest particle id in the cell, particles in the cell.
 * *n_out = samples written (min(found, cap)). */
int rb_mlp_samples(rb_sim* sim, double theta_hi, double theta_lo, double prob, uint64_t seed,
                   int64_t cap, int64_t* n_out, float* X, float* Y, int64_t* meta);
/* Train on n samples (host X n x 12, Y n x 3) with Adam (lr, beta 0.9 /
 * 0.999, eps 1e-8) on the mean squared error, minibatches of `batch` rows
 * in an order shuffled per epoch from `seed`.  Inputs and outputs are
 * standardised per column for training: w_init (host, 9347) is the start in
 * standardised units; w_out (host, 9347) is the result with the scales
 * folded back into W1, b1, W4, b4 (raw units, ready for rb_load_mlp);
 * loss_hist (host, epochs; may be NULL) is each epoch's mean loss, the
 * standardised loss times the mean output variance.  No simulation needed;
 * NULL stream: the call makes its own. */
int rb_mlp_train(const float* X, const float* Y, int64_t n, int epochs, int batch, double lr,
                 uint64_t seed, const float* w_init, float* w_out, float* loss_hist,
                 void* cuda_stream);
/* Gradient (host, 9347) and mean squared error of the whole set (n rows)
 * under weights w, as the training kernels compute them (BF16 operands,
 * FP32 accumulation). */
int rb_mlp_grad(const float* w, const float* X, const float* Y, int64_t n, float* grad, float* loss,
                void* cuda_stream);
/* Debug form of rb_mlp_grad: the same gradient and loss with every operand,
 * activation and sum in FP32 (no BF16 rounding; products summed in index
 * order, rows in row order, so the result is deterministic), for checking
 * the backward pass element by element against an FP64 reference.
 * 1 <= n <= 4096 (it keeps one gradient per row); RB_ERR_ARG otherwise. */
int rb_mlp_grad_fp32(const float* w, const float* X, const float* Y, int64_t n, float* grad,
                     float* loss, void* cuda_stream);

/* Energy and momentum sums without any device allocation.  The paper has no
 * counterpart: this entry point serves callers that cannot call cudaMalloc,
 * for instance a process whose device memory belongs to another runtime's
 * pool or budget, or a latency-bound loop that must avoid the implicit
 * device synchronisation of an allocation.
 * Inputs (device pointers, n particles each, caller-owned): m, x, z, vx, vy,
 * vz, and phi (may be NULL: W = 0; x and z may be NULL unless integrator is
 * RB_INT_SEI).  Output: out, a caller-owned device array of 7 doubles, filled
 * with sum m|v|^2/2, the SEI tidal and vertical term
 * sum m (omega_z^2 z^2 / 2 - 3/2 omega^2 x^2) (0 for leap-frog; omega_z <= 0
 * means omega_z = omega, as in rb_create), sum m phi / 2, the three momentum
 * components and n, the same terms rb_energy adds up.  Runs asynchronously on
 * cuda_stream (NULL: the legacy default stream), which must belong to the
 * current device; the arrays must be on that device too.
 * Scratch: a fixed 448 KiB array of per-block partial sums in the library's
 * own device memory, present on every GPU that loads the library until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress), so make the first call on each device
 * before any stream capture.  Every call overwrites the partial sums it
 * reads; calls that overlap on the GPU share the array and race.
 * Errors: RB_ERR_ARG for n < 0 or n > 16,777,216 (the partial-sum array holds
 * one slot per 2048 particles), a missing array or a stream of another device,
 * with a message in rb_last_error(NULL); RB_ERR_CUDA if the address lookup or
 * a launch fails (a launch error left by earlier work on the calling thread is
 * cleared before the launches).
 * It calls no cudaMalloc, cudaFree or allocating library routine. */
int rb_energy_sums_noalloc(int64_t n, const double* m, const double* x, const double* z,
                           const double* vx, const double* vy, const double* vz,
                           const double* phi, int integrator, double omega, double omega_z,
                           double* out, void* cuda_stream);
/* The sort that puts particles in Morton order before every tree build (it
 * replaces the tree reconstruction of Sect. 4.2), the collision queue in
 * canonical pair order (Sect. 5) and the pair ends of the resolution, run on
 * host arrays: a stable LSD radix sort of (key, value) pairs by key bits
 * [0, key_bits), 8-bit digits.  keys / vals: host arrays of n entries, sorted
 * in place (vals may be NULL).  cap >= n sizes the device buffers while the
 * count n is read on the device, as the step's sorts of pairs run; cap < 2^30.
 * key_bits in [1, 64].  cuda_stream: the stream to run on (NULL: the default
 * stream); the call returns when the result is on the host.  It allocates and
 * frees its own device buffers.  Errors: RB_ERR_ARG (bad sizes or key_bits, a
 * missing array), RB_ERR_CUDA, RB_ERR_TIMEOUT (a bounded wait between blocks
 * of a pass gave up), with a message in rb_last_error(NULL). */
int rb_sort_pairs_u64(int64_t n, int64_t cap, int key_bits, uint64_t* keys, uint32_t* vals,
                      void* cuda_stream);
/* Description of the last error of `sim`, or with sim NULL of the last
 * failed rb_create, rb_energy_sums_noalloc or rb_sort_pairs_u64 on the
 * calling thread (that
 * message is kept per host thread, so threads that fail at the same time do
 * not overwrite each other's).  Storage owned by the library, valid until the
 * next failing call of the same simulation or thread. */
const char* rb_last_error(const rb_sim* sim);

#ifdef __cplusplus
}
#endif
#endif
