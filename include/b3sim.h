/*
 * b3sim.h -- C ABI of the B300 population simulator.
 *
 * What it computes.  The paper (Sec. 4 "Initial Benchmarking", "Simulation
 * Parameters"; Sec. 5) times a physics engine that advances many independent
 * *variants* of a robot scene for a fixed number of steps, on the CPU and on
 * the GPU, and (Sec. 6) splits the variants between the two.  This library is
 * that engine for one GPU: every variant is an articulated modular robot (a
 * core cube plus hinge-jointed cubic bricks or balls, or a single free box or
 * ball) on a ground plane, and one call advances the whole population by n
 * steps.
 * Each step, per variant, in this order:
 *   1. CPG controller: s <- s + dt W s (W antisymmetric from the per-hinge
 *      weights), hinge torque tau = clamp(kp (theta_max clamp(x,-1,1) - theta)
 *      - kd theta_dot, -tau_max, tau_max);
 *   2. forward kinematics down the body tree;
 *   3. bias forces c(q, v) by recursive Newton-Euler, gravity as base
 *      acceleration;
 *   4. joint-space inertia M(q) by the composite-rigid-body algorithm plus a
 *      hinge armature;
 *   5. Cholesky M = L L^T and v_free = v + dt M^-1 (tau - c);
 *   6. contacts: box/plane vertices, a sphere's lowest point; box/box
 *      separating-axis test with face clipping or an edge-edge point,
 *      sphere/box and sphere/sphere at one point; at most contact_cap
 *      contacts (the deepest, in list order);
 *   7. soft projected Gauss-Seidel over the contact impulses (ERP/CFM soft
 *      constraints, penetration recovery speed capped at max_correct_vel,
 *      disk friction cone, pgs_iters sweeps, list order);
 *   8. semi-implicit Euler: root position, quaternion exponential map,
 *      hinge angles.
 * Fitness is the core's xy displacement since the start of the run.
 *
 * Generalized coordinates of a variant with nb bodies (nh = nb - 1 hinges):
 *   q = (p_root[3], quat_root[4] (w,x,y,z), theta[nh])     nq = nb + 6
 *   v = (v_root[3] world frame, omega_root[3] body frame, theta_dot[nh])
 *                                                          nv = nb + 5
 *   cpg = (x_1, y_1, x_2, y_2, ...)                        2 nh entries
 * Host state arrays use fixed row strides SIM_QW, SIM_VW, SIM_SW floats per
 * variant; unused tail entries are ignored on input and zero on output.
 *
 * Execution.  Variants of up to SIM_WARP_MAX_BODIES bodies are stepped one
 * warp each (lane = body / dof / contact row / body pair), variants that are
 * one free body one thread each, and larger variants (long chains, nv > 31)
 * one block of two warps each: the tree passes, the Cholesky rows, contact
 * generation and the contact rows are split over the block's 64 threads
 * with block barriers at the phase boundaries, and the triangular solves and
 * the Gauss-Seidel sweep run on one warp (each lane holding up to three
 * dofs), as they are sequential in their pivots and contacts.  All three
 * take the same steps in the same order.
 *
 * Ownership.  All device memory is owned by the context.  Every host
 * pointer is owned by the caller and only read (or written) during the
 * call.  Nothing crosses the ABI as an exception; every entry point returns
 * a sim_status, and sim_last_error() explains the last failure.
 * Threading: one context per host thread; a context is not re-entrant.
 * Stream: work is enqueued on the context's stream (sim_config.stream, a
 * cudaStream_t cast to uint64_t, or 0 for a stream the context creates).
 */
#ifndef B3SIM_H
#define B3SIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sim_ctx sim_ctx_t;   /* opaque context                       */

#define SIM_MAX_BODIES 64   /* core + up to 63 hinged bodies              */
#define SIM_WARP_MAX_BODIES 26  /* up to here (nv <= 31) a variant is stepped
                               by one warp; larger ones (up to 64 bodies,
                               nv <= 69: long chains) by a block of two
                               warps, see "Execution" above             */
#define SIM_QW 72           /* host row stride of q  (nq <= 70)            */
#define SIM_VW 72           /* host row stride of v  (nv <= 69)            */
#define SIM_SW 128          /* host row stride of the CPG state (<= 126)   */
#define SIM_MAX_CONTACT_CAP 64
#define SIM_MAX_CANDIDATES 256       /* contact candidates per step ...      */
#define SIM_MAX_CANDIDATES_CHAIN 512 /* ... and for variants of more than
                                        SIM_WARP_MAX_BODIES bodies (8 vertices
                                        of 64 boxes)                         */

typedef enum {
    SIM_OK = 0,
    SIM_EINVAL = -1,   /* bad argument: null pointer, size or range       */
    SIM_ECUDA = -2,    /* a CUDA call failed                              */
    SIM_ENOMEM = -3,   /* device or host allocation failed                */
    SIM_ESTATE = -4    /* call out of order (e.g. step before population) */
} sim_status;

/* per-variant status bits, returned by sim_read_state */
#define SIM_ST_NONFINITE 1u        /* state became non-finite: frozen      */
#define SIM_ST_OVERFLOW 2u         /* more contacts than contact_cap       */
#define SIM_ST_CHOL 4u             /* non-positive Cholesky pivot: frozen  */
#define SIM_ST_CANDIDATES 8u       /* more than SIM_MAX_CANDIDATES (or
                                      SIM_MAX_CANDIDATES_CHAIN) contact
                                      candidates; the extra were dropped    */

typedef struct {
    double dt;                /* step [s]                                    */
    float gravity[3];         /* [m/s^2], z up                               */
    int32_t pgs_iters;        /* Gauss-Seidel sweeps per step (>= 1)         */
    float soft_tau;           /* contact time constant [s]                   */
    float soft_zeta;          /* contact damping ratio                       */
    float mu;                 /* friction coefficient                        */
    int32_t contact_cap;      /* 1..SIM_MAX_CONTACT_CAP                      */
    float kp, kd, tau_max;    /* PD servo gains and torque limit             */
    float theta_max;          /* CPG amplitude [rad]                         */
    float armature;           /* rotor inertia added on hinge diagonals      */
    int32_t ground;           /* 1: body/plane contacts                      */
    int32_t box_box;          /* 1: body/body contacts inside a robot        */
    int32_t actuate;          /* 1: CPG + PD torques                         */
    float max_correct_vel;    /* cap of the penetration recovery speed [m/s] */
    int32_t device;           /* CUDA device ordinal                         */
    uint64_t stream;          /* cudaStream_t or 0                           */
    int32_t steps_per_launch; /* persistent chunk; 0: library default (5000) */
    int32_t warps_per_block;  /* 1, 2, 4 or 8; 0: sim_autotune's choice,
                                 1 until it runs                             */
    float min_cfm;            /* floor of a contact row's softness R [1/kg]:
                                 R = max(kappa A, min_cfm); bounds the
                                 impulse of rows the dofs can barely move    */
    int32_t phase_lock;       /* 1: the warps of a block pass the step's phase
                                 boundaries together (block barriers: fewer
                                 distinct phases per SM at a time, but every
                                 phase waits for the block's slowest robot);
                                 0: off (default)                           */
    int32_t warps_per_sm;     /* resident warps per SM the step kernel's
                                 registers are sized for: 16 (128 registers a
                                 thread) or 12 (168: each warp faster, fewer
                                 robots at once; not with 8 warps per
                                 block); 0: autotuned (default 16)          */
} sim_config;

/* Model of one variant.  Arrays have n_bodies entries (per body) unless
 * stated; body 0 is the core (free root), parent[b] < b for b >= 1. */
typedef struct {
    int32_t n_bodies;             /* 1..SIM_MAX_BODIES                        */
    const int8_t* parent;         /* parent body, -1 for body 0               */
    const int8_t* hinge_axis;     /* hinge axis index 0..2 in the body frame  */
    const uint64_t* exclude;      /* bit j: body never collides with body j   */
    const float* joint_frame;     /* 12 per body: R (3x3 row-major), p (3):
                                     body frame at zero angle in its parent  */
    const float* half_size;       /* 3 per body: box half extents [m]; a
                                     sphere has all three equal its radius   */
    const float* box_center;      /* 3 per body: box or sphere centre in the
                                     body frame [m]                          */
    const float* mass;            /* [kg]; inertia is that of the solid shape */
    const float* cpg_w_internal;  /* per body: oscillator weight of hinge b   */
    const float* cpg_w_couple;    /* per body: coupling of hinge b to the
                                     hinge of its parent (0 if parent = 0)   */
    const int8_t* geom;           /* per body: SIM_GEOM_BOX or SIM_GEOM_SPHERE;
                                     NULL: every body is a box               */
} sim_variant_desc;

/* body geometries: a box meets the plane at its vertices and other bodies by
 * the separating-axis test; a sphere meets the plane, a box or a sphere at
 * one point (the deepest, midway between the two surfaces) */
#define SIM_GEOM_BOX 0
#define SIM_GEOM_SPHERE 1

typedef struct {
    double contacts;          /* sum over variants and steps of contacts     */
    double narrow_pairs;      /* box/box pairs through the narrow phase      */
    double broad_pairs;       /* box/box pairs through the broad phase       */
    double variant_steps;     /* variants x steps advanced                   */
    double sm_cycles;         /* sum over variants of SM clock cycles spent
                                 in the step loop (per-warp clock64)         */
} sim_counters;

/* Create a context on cfg->device.  Copies cfg.  *out is NULL on failure. */
int sim_create(const sim_config* cfg, sim_ctx_t** out);

/* Free the context and all its device memory.  NULL is accepted. */
int sim_destroy(sim_ctx_t* ctx);

/* Replace the population with n variants (n >= 1).  Copies every array.
 * The state is reset to q = v = 0, cpg = 0 and must be set with
 * sim_set_state before stepping.  Internally variants are reordered by size;
 * every other call uses the caller's order. */
int sim_set_population(sim_ctx_t* ctx, const sim_variant_desc* v, int32_t n);

/* Set state of variants [first, first+count) from host rows (strides SIM_QW,
 * SIM_VW, SIM_SW).  cpg may be NULL (kept).  Clears their status bits and
 * records the current core xy as the fitness origin.  Synchronous. */
int sim_set_state(sim_ctx_t* ctx, int32_t first, int32_t count, const float* q,
                  const float* v, const float* cpg);

/* Device-buffer variants of sim_set_state, sim_read_state and sim_fitness,
 * for callers whose data already lives on the GPU (e.g. torch tensors via
 * their data pointers): same row layouts and rules, but every buffer is
 * caller-owned device (or managed) memory of cfg->device, nothing is copied
 * through the host and nothing synchronises.  The work is queued on the
 * context stream (sim_stream): inputs must be ready before it runs (written
 * on that stream, or ordered by an event the caller makes it wait on) and
 * stay unchanged, and outputs valid, until the stream has passed the call.
 * A buffer that is not device memory of that device is rejected with
 * SIM_EINVAL.  Outputs that are NULL are skipped. */
int sim_set_state_dev(sim_ctx_t* ctx, int32_t first, int32_t count, const float* q, const float* v,
                      const float* cpg);
int sim_read_state_dev(sim_ctx_t* ctx, int32_t first, int32_t count, float* q, float* v, float* cpg,
                       uint32_t* status);
int sim_fitness_dev(sim_ctx_t* ctx, float* out, int32_t n);

/* The context's stream (a cudaStream_t) into *stream. */
int sim_stream(const sim_ctx_t* ctx, uint64_t* stream);

/* Advance every variant n_steps (>= 0) steps.  Asynchronous on the context
 * stream (a captured CUDA graph per distinct n_steps); launch errors are
 * returned, execution errors surface at the next synchronising call. */
int sim_step_n(sim_ctx_t* ctx, int32_t n_steps);

/* Copy state of variants [first, first+count) to host rows; any output
 * pointer may be NULL.  status gets the per-variant SIM_ST_* bits.
 * Synchronises the context stream. */
int sim_read_state(sim_ctx_t* ctx, int32_t first, int32_t count, float* q, float* v,
                   float* cpg, uint32_t* status);

/* Core xy displacement of variants [0, n) since their last sim_set_state.
 * Synchronises the context stream. */
int sim_fitness(sim_ctx_t* ctx, float* out, int32_t n);

/* Time the candidate launch shapes on probe_steps steps of the current
 * population (state is saved and restored) and keep the fastest. */
int sim_autotune(sim_ctx_t* ctx, int32_t probe_steps);

/* The launch shape sim_step_n uses now (after sim_autotune, the chosen one):
 * warps per block, phase lock, steps per persistent launch and the resident
 * warps per SM the kernel's registers are sized for.  Any output may be
 * NULL. */
int sim_launch_shape(const sim_ctx_t* ctx, int32_t* warps_per_block, int32_t* phase_lock,
                     int32_t* steps_per_launch,
                     int32_t* warps_per_sm);

/* Work counters accumulated since sim_set_population (synchronises). */
int sim_counters_read(sim_ctx_t* ctx, sim_counters* out);

/* Contact list of the last step of variant i (caller's order): up to
 * max_contacts rows of 8 floats (point relative to the core origin (3),
 * normal from body b to body a (3), depth, body a) and the body b of each
 * row (-1: ground) in b_out.  *n_out gets the count.  Synchronises. */
int sim_debug_contacts(sim_ctx_t* ctx, int32_t i, int32_t max_contacts, float* rows,
                       int32_t* b_out, int32_t* n_out);

/* Solver detail of the last step of variant i (caller's order): v_free
 * (SIM_VW floats, the velocity before contacts) and the contact impulses
 * (3 floats per contact: normal, tangent 1, tangent 2; room for
 * 3 * SIM_MAX_CONTACT_CAP floats).  *n_out gets the contact count.
 * cycles_per_step (may be NULL, else 11 floats) gets the SM clock cycles per
 * step that the variant's warp spent in its last launch: [0] the whole step,
 * [1..10] its phases (CPG + FK, inertias + RNEA + CRBA, Cholesky + v_free,
 * ground contacts, box/box contacts, contact cap, contact rows, Gauss-Seidel,
 * integration, unused).  Synchronises. */
int sim_debug_solver(sim_ctx_t* ctx, int32_t i, float* vfree, float* lambda, int32_t* n_out,
                     float* cycles_per_step);

/* Cost of each variant [0, n) (caller's order) in the last launch: the SM
 * clock cycles per step its warp took, sharing its SM with the other warps
 * (0 before the first launch and for frozen variants).  For schedulers such
 * as the hybrid CPU + GPU allocation.  Synchronises. */
int sim_robot_cost(sim_ctx_t* ctx, float* out, int32_t n);

/* Host evaluation of the step kernel's FP64 sine / cosine routine (the one
 * that the hinge angles go through on the device, compiled here for the
 * host): s[i], c[i] for x[i], i < n.  Inspection and testing only; no device
 * work, no context needed.  SIM_EINVAL for NULL arrays or n < 0. */
int sim_debug_sincos(const double* x, int32_t n, double* s, double* c);

/* ---- Stepping without any allocation --------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory when they step: hosts whose device memory is
 * owned by another allocator or fixed up front (game engines, embedded
 * controllers, plugins inside a larger GPU application, where a cudaMalloc
 * would bypass the host's accounting or fail against its budget), and
 * real-time loops that must not block in the driver (cudaMalloc and cudaFree
 * may synchronise the device).
 *
 * sim_step_n_noalloc advances n variants that the CALLER keeps in device
 * memory it already owns.  It calls no cudaMalloc, cudaFree or allocating
 * library routine.  Its per-variant scratch (contact candidates, narrow-phase
 * staging rows, contact Jacobian rows, Gauss-Seidel constants and a Delassus
 * matrix of up to 32 contacts, about 95 KB per variant) is a fixed array
 * inside this library: SIM_NOALLOC_MAX_VARIANTS variants, about 6 MB, held by
 * every device that loads the library until the process exits.  Larger n
 * is rejected with SIM_EINVAL.
 *   - cfg->device is made current; cfg->stream (0: the legacy default
 *     stream) receives the work, asynchronously.
 *   - The first call on a device looks up the scratch's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture
 *     on that device.
 *   - All calls share the one scratch array, which keeps the last call's
 *     contents; calls whose work overlaps on the GPU (other streams, other
 *     host threads) race on it and must be serialised by the caller.
 *   - Variants have at most SIM_WARP_MAX_BODIES bodies (the layout below has
 *     32 body slots); longer chains need a context (sim_set_population).
 *   - Every variant is stepped by the general warp-per-robot step kernel of
 *     sim_step_n, in the order given (no size sorting).  Variants that are a
 *     single free body take that general kernel here too, not the
 *     one-thread-per-body kernel sim_step_n uses for them, so their results
 *     differ from sim_step_n's by FP32 rounding (about 1e-5 m over 200 steps
 *     of a tumbling cube).
 *   - Failures are reported per host thread: sim_last_error(NULL) returns the
 *     message of the calling thread's last failed call.
 * Device layout expected in *pop (all device pointers, caller-owned):
 *   model_f  n x SIM_MODEL_NF x 32 floats, [variant][field][body slot]:
 *            joint frame R (9, row-major), joint frame p (3), half size (3),
 *            box centre (3), mass, principal inertia about the centre
 *            (3: box m(hy^2+hz^2)/3, m(hx^2+hz^2)/3, m(hx^2+hy^2)/3; sphere
 *            2 m r^2 / 5 each), CPG weight, CPG coupling, bounding radius
 *            (box |half size|, sphere r), geometry (0.0 box, 1.0 sphere);
 *            slots >= n_bodies hold R = identity and zeros.
 *   model_i  n x SIM_MODEL_NI x 32 int32: parent (-1 for body 0 and unused
 *            slots), hinge axis, path mask (bit j for every body on the path
 *            from body 0 to this body, both ends included), child mask, depth
 *            (body 0: 0).
 *   meta     n x 4 int32: n_bodies, maximum depth, pair count, offset of the
 *            variant's pairs in `pairs`; the buffer must be 16-byte aligned
 *            (each row is read as one vector), else SIM_EINVAL.
 *   pairs    uint16 (a << 8) | b for every body pair a < b that may collide
 *            (b's parent is not a, and neither excludes the other).
 *   q, v, cpg, status  state rows with strides 32, 32, 64 floats and one
 *            uint32 status word per variant (as in sim_read_state).
 * Returns SIM_OK, SIM_EINVAL (bad argument; sim_last_error(NULL) says which)
 * or SIM_ECUDA. */
#define SIM_NOALLOC_MAX_VARIANTS 64
#define SIM_MODEL_NF 26
#define SIM_MODEL_NI 5

typedef struct {
    int32_t n;                /* variants, 1..SIM_NOALLOC_MAX_VARIANTS        */
    const float* model_f;
    const int32_t* model_i;
    const int32_t* meta;
    const uint16_t* pairs;
    float* q;
    float* v;
    float* cpg;
    uint32_t* status;
} sim_device_population;

int sim_step_n_noalloc(const sim_config* cfg, const sim_device_population* pop, int32_t n_steps);

/* ---- FP32 peak of the device (measurement; no counterpart in the paper) ----
 * The step kernel runs on the FP32 FMA pipe (no dense contraction in the
 * step), so its roofline denominator is what that pipe delivers: this call
 * launches `launches` back-to-back kernels of independent FFMA chains (every
 * resident thread of every SM, 8 chains a thread, 64 warps per SM) on a
 * private stream of `device` and returns their FLOP count (an FMA is 2) and
 * device time in milliseconds (CUDA events around all launches), plus the SM
 * count.  About 40 ms per launch.  Synchronises; returns SIM_OK, SIM_EINVAL
 * (launches < 1 or NULL outputs; sim_last_error(NULL) says which) or
 * SIM_ECUDA. */
int sim_fp32_peak(int32_t device, int32_t launches, double* flops, float* ms, int32_t* sm_count);

/* Human-readable description of the last failure on this context ("" if
 * none).  ctx may be NULL for a failure in sim_create or
 * sim_step_n_noalloc: that message is kept per host thread. */
const char* sim_last_error(const sim_ctx_t* ctx);

#ifdef __cplusplus
}
#endif

#endif
